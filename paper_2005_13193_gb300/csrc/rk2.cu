// Second-order Runge-Kutta particle advance (Sec. 2.1; Sec. 4.3), read as
// Heun's predictor-corrector, with the per-step re-binning that stands in for
// the paper's particle migration between sub-domains (Sec. 4.3).
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
                            double dt, int32_t* status, cudaStream_t st);
}  // namespace ps

using namespace ps;

// Halo extension beyond the brick's own stencils.  0: the halo is exactly
// the union of the stencils of the brick's cells; predictors that leave it
// (a few percent of particles per step at Courant numbers below one) read
// their stencil from global memory instead.
static constexpr int kRk2HaloExtension = 0;

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
  if (!rebin) {
    if (!bin_offsets) return fail(PS_ERR_INVALID_ARG, "rebin=0 needs bin_offsets");
    if (np == 0) return PS_OK;
    return rk2_launch_staged(grid, brick, kRk2HaloExtension, coef_t, coef_n, scale_n,
                             coef_np1, scale_np1, np, pos, pos, bin_offsets, vel_out, nullptr,
                             nullptr, dt, status, st);
  }
  const size_t need = bin_ws_bytes(ba, np, true, true, true, true);
  if (!ws || ws_bytes < need - 256 || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(PS_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need - 256);
  Carver c(ws);
  int32_t* counts = c.take<int32_t>(ba.nbins + 1);
  int32_t* scan_tmp = c.take<int32_t>(scan_tmp_elems(ba.nbins) + 1);
  int32_t* rank = c.take<int32_t>(np);
  int32_t* offs_ws = c.take<int32_t>(ba.nbins + 1);
  int32_t* bin_of = c.take<int32_t>(np);
  double* pos_s = c.take<double>(3 * np);
  int64_t* ids_s = c.take<int64_t>(np);
  int32_t* offs = bin_offsets ? bin_offsets : offs_ws;
  rc = bin_run(ga, ba, np, pos, bin_of, offs, nullptr, pos_s, ids, ids ? ids_s : nullptr,
               counts, rank, scan_tmp, status, st);
  if (rc) return rc;
  if (np == 0) return PS_OK;
  return rk2_launch_staged(grid, brick, kRk2HaloExtension, coef_t, coef_n, scale_n, coef_np1,
                           scale_np1, np, pos_s, pos, offs, vel_out, ids ? ids_s : nullptr,
                           ids, dt, status, st);
}
