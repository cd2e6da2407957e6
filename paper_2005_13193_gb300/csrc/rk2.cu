// Second-order Runge-Kutta particle advance (Sec. 2.1; Sec. 4.3), read as
// Heun's predictor-corrector, with the per-step re-binning that stands in for
// the paper's particle migration between sub-domains (Sec. 4.3).  As the
// paper finds the few particles that leave a sub-domain while it updates
// positions, the step kernel can count every particle's new bin while it
// stores the new position (rebin 2 and 3), so that the next step's sort
// starts at the scan: the sort then reads the positions once instead of twice.
#include <cmath>

#include "ps_internal.cuh"

namespace ps {
ps_status rk2_launch_direct(const ps_grid* grid, ps_dtype coef_t, const void* c0,
                            const float* s0, const void* c1, const float* s1, int64_t np,
                            double* pos, float* vel_out, double dt, int32_t* status,
                            cudaStream_t st);
ps_status rk2_launch_staged(const ps_grid* grid, const int32_t brick[3], int E,
                            ps_dtype coef_t, const void* c0, const float* s0,
                            const void* c1, const float* s1, int64_t np,
                            const double* pos_in, double* pos_out, const int32_t* offs,
                            float* vel_out, const int64_t* ids_in, int64_t* ids_out,
                            double dt, int32_t* status, int32_t* next_counts,
                            int32_t* next_bin, cudaStream_t st);
}  // namespace ps

using namespace ps;

// Halo extension beyond the brick's own stencils.  0: the halo is exactly
// the union of the stencils of the brick's cells; predictors that leave it
// (a few percent of particles per step at Courant numbers below one) read
// their stencil from global memory instead.
static constexpr int kRk2HaloExtension = 0;

// Workspace of the binned step: bin counters, scan scratch, per-particle
// rank and bin, bin bounds, sorted positions and ids.  counts and bin_of
// carry the counting of the positions a step wrote to the next sort.
struct Rk2Ws {
  int32_t* counts;
  int32_t* scan_tmp;
  int32_t* rank;
  int32_t* offs;
  int32_t* bin_of;
  double* pos_s;
  int64_t* ids_s;
};

static ps_status carve_rk2_ws(const BrickArgs& ba, int64_t np, void* ws, size_t ws_bytes,
                              Rk2Ws* w) {
  const size_t need = bin_ws_bytes(ba, np, true, true, true, true);
  if (!ws || ws_bytes < need - 256 || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(PS_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need - 256);
  Carver c(ws);
  w->counts = c.take<int32_t>(ba.nbins + 1);
  w->scan_tmp = c.take<int32_t>(scan_tmp_elems(ba.nbins) + 1);
  w->rank = c.take<int32_t>(np);
  w->offs = c.take<int32_t>(ba.nbins + 1);
  w->bin_of = c.take<int32_t>(np);
  w->pos_s = c.take<double>(3 * np);
  w->ids_s = c.take<int64_t>(np);
  return PS_OK;
}

static ps_status clear_counts(const BrickArgs& ba, const Rk2Ws& w, cudaStream_t st) {
  return check_cuda(cudaMemsetAsync(w.counts, 0, sizeof(int32_t) * (ba.nbins + 1), st),
                    "next-step counts memset");
}

extern "C" size_t ps_rk2_workspace_size(const ps_grid* grid, const int32_t brick[3],
                                        int64_t np) {
  if (!brick) return 0;
  BrickArgs ba;
  if (validate_grid(grid) || make_brick_args(grid, brick, &ba) || np < 0) return 0;
  return bin_ws_bytes(ba, np, true, true, true, true);
}

extern "C" ps_status ps_rk2_step(const ps_grid* grid, ps_dtype coef_t, const void* coef_n,
                                 const void* coef_np1, const float* scale_n,
                                 const float* scale_np1, int64_t np, double* pos,
                                 int64_t* ids, float* vel_out, double dt,
                                 const int32_t brick[3], int rebin, int32_t* bin_offsets,
                                 void* ws, size_t ws_bytes, int32_t* status, void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  if (coef_t != PS_F32 && coef_t != PS_F64 && coef_t != PS_BF16 && coef_t != PS_F16 &&
      coef_t != PS_F32X4 && coef_t != PS_BF16X4 && coef_t != PS_F16X4)
    return fail(PS_ERR_INVALID_ARG, "bad coefficient dtype");
  if (!coef_n) return fail(PS_ERR_INVALID_ARG, "coef_n is NULL");
  const bool quant = coef_t == PS_BF16 || coef_t == PS_F16 || coef_t == PS_BF16X4 ||
                     coef_t == PS_F16X4;
  if (quant && (!scale_n || (coef_np1 && !scale_np1)))
    return fail(PS_ERR_INVALID_ARG, "scales required for BF16/F16 coefficients");
  if (np < 0 || np >= ((int64_t)1 << 31)) return fail(PS_ERR_INVALID_ARG, "np out of range");
  if (rebin < 0 || rebin > 3) return fail(PS_ERR_INVALID_ARG, "rebin is 0, 1, 2 or 3");
  if (!std::isfinite(dt)) return fail(PS_ERR_INVALID_ARG, "dt must be finite");
  if (np > 0 && !pos) return fail(PS_ERR_INVALID_ARG, "pos is NULL");
  cudaStream_t st = as_stream(stream);
  const void* c1 = coef_np1 ? coef_np1 : coef_n;
  const float* s1 = coef_np1 ? scale_np1 : scale_n;

  if (!brick || coef_t == PS_F64) {
    if (brick && rebin)
      return fail(PS_ERR_UNSUPPORTED, "binned RK2 needs F32/BF16/F16 coefficients");
    if (np == 0) return PS_OK;
    return rk2_launch_direct(grid, coef_t, coef_n, scale_n, c1, s1, np, pos, vel_out, dt,
                             status, st);
  }
  BrickArgs ba;
  if ((rc = make_brick_args(grid, brick, &ba))) return rc;
  GridArgs ga = make_grid_args(grid);
  Rk2Ws w{};
  if (rebin == 0) {
    if (!bin_offsets) return fail(PS_ERR_INVALID_ARG, "rebin=0 needs bin_offsets");
    // with a workspace the step also counts the positions it writes, for a
    // following ps_rk2_sort(counted = 1) or ps_rk2_step(rebin = 3)
    if (ws) {
      if ((rc = carve_rk2_ws(ba, np, ws, ws_bytes, &w))) return rc;
      if ((rc = clear_counts(ba, w, st))) return rc;
    }
    if (np == 0) return PS_OK;
    return rk2_launch_staged(grid, brick, kRk2HaloExtension, coef_t, coef_n, scale_n,
                             coef_np1, scale_np1, np, pos, pos, bin_offsets, vel_out, nullptr,
                             nullptr, dt, status, w.counts, w.bin_of, st);
  }
  if ((rc = carve_rk2_ws(ba, np, ws, ws_bytes, &w))) return rc;
  int32_t* offs = bin_offsets ? bin_offsets : w.offs;
  // rebin 3: the counting was done by the previous step's kernel
  rc = bin_run(ga, ba, np, pos, w.bin_of, offs, nullptr, w.pos_s, ids, ids ? w.ids_s : nullptr,
               w.counts, w.rank, w.scan_tmp, status, st, rebin == 3);
  if (rc) return rc;
  // rebin 2 and 3: this step's kernel counts the positions it writes for the
  // next step's sort (bin per particle, bin counters)
  const bool carry = rebin >= 2;
  if (carry && (rc = clear_counts(ba, w, st))) return rc;
  if (np == 0) return PS_OK;
  return rk2_launch_staged(grid, brick, kRk2HaloExtension, coef_t, coef_n, scale_n, coef_np1,
                           scale_np1, np, w.pos_s, pos, offs, vel_out, ids ? w.ids_s : nullptr,
                           ids, dt, status, carry ? w.counts : nullptr,
                           carry ? w.bin_of : nullptr, st);
}

extern "C" ps_status ps_rk2_sort(const ps_grid* grid, const int32_t brick[3], int64_t np,
                                 const double* pos, const int64_t* ids, int counted,
                                 double* pos_sorted, int64_t* ids_sorted,
                                 int32_t* bin_offsets, void* ws, size_t ws_bytes,
                                 int32_t* status, void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  BrickArgs ba;
  if ((rc = make_brick_args(grid, brick, &ba))) return rc;
  if (np < 0 || np >= ((int64_t)1 << 31)) return fail(PS_ERR_INVALID_ARG, "np out of range");
  if (counted != 0 && counted != 1) return fail(PS_ERR_INVALID_ARG, "counted is 0 or 1");
  if (!bin_offsets || (np > 0 && (!pos || !pos_sorted)))
    return fail(PS_ERR_INVALID_ARG, "pos, pos_sorted and bin_offsets are required");
  if ((ids == nullptr) != (ids_sorted == nullptr))
    return fail(PS_ERR_INVALID_ARG, "ids and ids_sorted go together");
  if (np > 0 && pos == pos_sorted) return fail(PS_ERR_INVALID_ARG, "pos_sorted must not be pos");
  Rk2Ws w{};
  if ((rc = carve_rk2_ws(ba, np, ws, ws_bytes, &w))) return rc;
  return bin_run(make_grid_args(grid), ba, np, pos, w.bin_of, bin_offsets, nullptr, pos_sorted,
                 ids, ids_sorted, w.counts, w.rank, w.scan_tmp, status, as_stream(stream),
                 counted == 1);
}
