// Host-side plumbing of the C ABI: error strings, status words, validation.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "ps_internal.cuh"

namespace ps {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

ps_status fail(ps_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

ps_status check_cuda(cudaError_t err, const char* what) {
  if (err == cudaSuccess) return PS_OK;
  return fail(PS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(err));
}

ps_status check_launch(const char* what) {
  return check_cuda(cudaGetLastError(), what);
}

ps_status validate_grid(const ps_grid* g) {
  if (!g) return fail(PS_ERR_INVALID_ARG, "grid is NULL");
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < 3 || g->n[d] > 2048)
      return fail(PS_ERR_INVALID_ARG, "grid n[%d]=%d outside [3, 2048]", d, g->n[d]);
    if (!(g->L[d] > 0.0) || !std::isfinite(g->L[d]))
      return fail(PS_ERR_INVALID_ARG, "grid L[%d] must be finite and > 0", d);
  }
  return PS_OK;
}

size_t dtype_size(ps_dtype t) {
  switch (t) {
    case PS_F32: return 4;
    case PS_F64: return 8;
    case PS_BF16: return 2;
    case PS_F16: return 2;
    case PS_F32X4: return 16;
    case PS_BF16X4: return 8;
    case PS_F16X4: return 8;
  }
  return 0;
}

int64_t coef_pitch(int nx, ps_dtype t) {
  const int64_t v = 16 / (int64_t)dtype_size(t);
  return ((int64_t)nx + 3 + v - 1) / v * v;
}

GridArgs make_grid_args(const ps_grid* g, int coef_t) {
  GridArgs a;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g->n[d];
    a.m[d] = g->n[d] + 3;
    a.inv_h[d] = (double)g->n[d] / g->L[d];
    a.inv_hf[d] = (float)a.inv_h[d];
  }
  a.rx = coef_t < 0 ? 0 : (int)coef_pitch(g->n[0], (ps_dtype)coef_t);
  return a;
}

ps_status make_brick_args(const ps_grid* g, const int32_t brick[3], BrickArgs* out) {
  if (!brick) return fail(PS_ERR_INVALID_ARG, "brick is NULL");
  int64_t nbins = 1;
  for (int d = 0; d < 3; ++d) {
    if (brick[d] < 1 || brick[d] > 64)
      return fail(PS_ERR_INVALID_ARG, "brick[%d]=%d outside [1, 64]", d, brick[d]);
    out->B[d] = brick[d];
    out->nb[d] = (g->n[d] + brick[d] - 1) / brick[d];
    nbins *= out->nb[d];
  }
  if (nbins >= (int64_t)1 << 31) return fail(PS_ERR_INVALID_ARG, "too many bins");
  out->nbins = nbins;
  return PS_OK;
}

Tuning& tuning() {
  static Tuning t;
  return t;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 1;
  return n;
}

}  // namespace ps

using namespace ps;

extern "C" const char* ps_last_error(void) { return g_err; }

extern "C" ps_status ps_tune_set(const char* key, int64_t value) {
  if (!key) return fail(PS_ERR_INVALID_ARG, "key is NULL");
  if (!strcmp(key, "brick_kernel")) {
    if (value != -1 && value != 0 && value != 2 && value != 5)
      return fail(PS_ERR_INVALID_ARG, "brick_kernel is -1 (auto), 0, 2 or 5");
    tuning().brick_kernel = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "brick_min_stage")) {
    if (value < 0 || value > (1 << 20)) return fail(PS_ERR_INVALID_ARG, "brick_min_stage in [0, 2^20]");
    tuning().brick_min_stage = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "solve_xw")) {
    if (value != 0 && value != 8 && value != 16 && value != 32)
      return fail(PS_ERR_INVALID_ARG, "solve_xw is 0, 8, 16 or 32");
    tuning().solve_xw = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "solve_stream")) {
    if (value < 0 || value > 1) return fail(PS_ERR_INVALID_ARG, "solve_stream is 0 or 1");
    tuning().solve_stream = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "solve_zt")) {
    if (value != 0 && value != 16 && value != 32 && value != 64 && value != 128 && value != 256)
      return fail(PS_ERR_INVALID_ARG, "solve_zt is 0, 16, 32, 64, 128 or 256");
    tuning().solve_zt = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "solve_stages")) {
    if (value != 0 && (value < 2 || value > 4))
      return fail(PS_ERR_INVALID_ARG, "solve_stages is 0, 2, 3 or 4");
    tuning().solve_stages = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "node_tma")) {
    if (value < 0 || value > 1) return fail(PS_ERR_INVALID_ARG, "node_tma is 0 or 1");
    tuning().node_tma = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "batch_run_below")) {
    if (value < 0 || value > (1 << 20)) return fail(PS_ERR_INVALID_ARG, "batch_run_below in [0, 2^20]");
    tuning().batch_run_below = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "batch_persistent")) {
    if (value < 0 || value > 1) return fail(PS_ERR_INVALID_ARG, "batch_persistent is 0 or 1");
    tuning().batch_persistent = (int)value;
    return PS_OK;
  }
  if (!strcmp(key, "wait_probe")) {
    if (value < 0 || value > (1 << 30)) return fail(PS_ERR_INVALID_ARG, "wait_probe in [0, 2^30]");
    tuning().wait_probe = (int)value;
    return PS_OK;
  }
  return fail(PS_ERR_INVALID_ARG, "unknown tuning key '%s'", key);
}

extern "C" int64_t ps_tune_get(const char* key) {
  if (!key) return -1;
  if (!strcmp(key, "brick_kernel")) return tuning().brick_kernel;
  if (!strcmp(key, "brick_min_stage")) return tuning().brick_min_stage;
  if (!strcmp(key, "node_tma")) return tuning().node_tma;
  if (!strcmp(key, "solve_xw")) return tuning().solve_xw;
  if (!strcmp(key, "solve_stream")) return tuning().solve_stream;
  if (!strcmp(key, "solve_zt")) return tuning().solve_zt;
  if (!strcmp(key, "solve_stages")) return tuning().solve_stages;
  if (!strcmp(key, "wait_probe")) return tuning().wait_probe;
  if (!strcmp(key, "batch_persistent")) return tuning().batch_persistent;
  if (!strcmp(key, "batch_run_below")) return tuning().batch_run_below;
  return -1;
}

extern "C" const char* ps_version(void) { return "ps 0.1 (sm_103a)"; }

extern "C" int64_t ps_coef_row_pitch(int nx, ps_dtype coef_t) {
  if (nx < 1 || dtype_size(coef_t) == 0) return 0;
  return coef_pitch(nx, coef_t);
}

extern "C" ps_status ps_status_clear(int32_t* status, void* stream) {
  if (!status) return fail(PS_ERR_INVALID_ARG, "status is NULL");
  return check_cuda(cudaMemsetAsync(status, 0, 4 * sizeof(int32_t), as_stream(stream)),
                    "ps_status_clear");
}

extern "C" ps_status ps_status_read(const int32_t* status, int32_t* host_out,
                                    void* stream) {
  if (!status || !host_out) return fail(PS_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  ps_status rc = check_cuda(cudaMemcpyAsync(host_out, status, 4 * sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, st),
                            "ps_status_read copy");
  if (rc) return rc;
  rc = check_cuda(cudaStreamSynchronize(st), "ps_status_read sync");
  if (rc) return rc;
  if (host_out[0] != PS_DEV_OK)
    return fail(PS_ERR_DEVICE_STATUS, "device status %d at index %lld (%d events)",
                host_out[0],
                (long long)(((uint64_t)(uint32_t)host_out[2] << 32) | (uint32_t)host_out[1]),
                host_out[3]);
  return PS_OK;
}
