// Operations 2 and 3 of Sec. 2.2 (basis functions and the 64-term sum of
// Eq. (spline)), their adjoint, and the second-order Runge-Kutta particle
// advance of Sec. 2.1 / Sec. 4.3.
//
// Two gather strategies:
//  * direct: a quad of lanes per particle, lane q owning stencil column
//    x = a_x + q; every (j,k) row is one 16-byte segment per quad.  Works for
//    any particle order (the "unsorted" path).
//  * staged: particles stored in brick order (Sec. 3's dynamic mapping read as
//    a bin sort); one CTA per brick copies the brick's coefficient halo once
//    into shared memory as float4 (u, v, w, 0), and 8 lanes per particle read
//    it with conflict-free 128-bit loads.  This is the GPU form
//    of the paper's "fetch only the coefficients a particle needs": the halo
//    is the union of the stencils of the brick's particles.
//
// FP64 work per particle is one multiply per axis (done by three lanes in
// parallel); floor and fraction come from the bits of the product, the RK2
// predictor position is located in FP32 relative to the stage-1 cell, and the
// position update is one FMA per axis.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "bin_device.cuh"
#include "staged.cuh"

namespace ps {
namespace {

// The first three lanes of each group of G lanes locate one axis each; the
// cell indices and fractions are broadcast to the whole group.  xd returns
// the FP64 coordinate of the lane's own axis (lanes 0..2 of the group).
template <int G, typename A>
__device__ __forceinline__ bool locate_group(const GridArgs& g, const double* pos, int64_t np,
                                             int64_t p, int lane, int cell[3], A t[3],
                                             double& xd) {
  const int sub = lane & (G - 1), base = lane & ~(G - 1);
  int cd = 0;
  A td = A(0);
  xd = 0.0;
  if (sub < 3) {
    xd = pos[sub * np + p];
    bool okd;
    if constexpr (std::is_same<A, double>::value)
      okd = locate_f64(xd, g.inv_h[sub], g.n[sub], cd, td);
    else
      okd = locate(xd, g.inv_h[sub], g.n[sub], cd, td);
    if (!okd) cd = -1;
  }
  bool ok = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    cell[d] = __shfl_sync(FULL, cd, base + d);
    t[d] = __shfl_sync(FULL, td, base + d);
    ok &= cell[d] >= 0;
    cell[d] = max(cell[d], 0);
  }
  return ok;
}

template <typename A, bool GRAD>
struct Basis {
  int a[3];
  A b[3][4];
  A db[3][4];
  __device__ __forceinline__ void set(const int cell[3], const A t[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      a[d] = cell[d];
      bspline<A>(t[d], b[d]);
      if (GRAD) dbspline<A>(t[d], db[d]);
    }
  }
};

// Predictor position of a Heun step located in FP32 relative to the stage-1
// cell: t* = t + u dt n/L, cell* = cell + floor(t*) (mod n).
__device__ __forceinline__ void advance_cell(int n, int cell, float t, float du, int& c2,
                                             float& t2) {
  float tt = t + du;
  float fl = floorf(tt);
  if (!(fabsf(fl) < 1.0e9f)) fl = 0.f;  // non-finite velocity: keep the cell
  tt -= fl;
  int c = cell + (int)fl;
  if (c < 0 || c >= n) {
    c %= n;
    if (c < 0) c += n;
  }
  c2 = c;
  t2 = fminf(fmaxf(tt, 0.f), 1.f);
}

// Direct gather by a quad: lane q accumulates its column over the 16 rows.
template <typename Tc, int NC, bool GRAD, typename A>
__device__ __forceinline__ void quad_rows(const GridArgs& g, const Tc* __restrict__ coef,
                                          const float* __restrict__ scale,
                                          const Basis<A, GRAD>& B, int q, A acc[NC],
                                          A accy[NC], A accz[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = accy[c] = accz[c] = A(0);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const A w = B.b[1][j] * B.b[2][k];
      A wy = A(0), wz = A(0);
      if (GRAD) {
        wy = B.db[1][j] * B.b[2][k];
        wz = B.b[1][j] * B.db[2][k];
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const A v = load_coef<Tc>(coef, scale, g, c, B.a[2] + k, B.a[1] + j, B.a[0] + q);
        acc[c] += w * v;
        if (GRAD) {
          accy[c] += wy * v;
          accz[c] += wz * v;
        }
      }
    }
}

// MODE 0: vel; 1: vel + grad; 2: g_pos = sum_c g_vel[c] grad[c][.]
template <typename Tc, int NC, int MODE>
__global__ void __launch_bounds__(256) interp_direct(GridArgs g, const Tc* __restrict__ coef,
                                                     const float* __restrict__ scale,
                                                     int64_t np,
                                                     const double* __restrict__ pos,
                                                     const int64_t* __restrict__ perm,
                                                     float* __restrict__ vel,
                                                     float* __restrict__ grad,
                                                     const float* __restrict__ gvel,
                                                     double* __restrict__ gpos,
                                                     int32_t* status) {
  using A = typename AccOf<Tc>::type;
  constexpr bool GRAD = MODE >= 1;
  const int lane = threadIdx.x & 31, q = lane & 3;
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const bool valid = s < np;
  const int64_t p = valid ? (perm ? perm[s] : s) : 0;
  int cell[3];
  A t[3];
  double xd;
  const bool ok = locate_group<4, A>(g, pos, valid ? np : 0, p, lane, cell, t, xd) || !valid;
  Basis<A, GRAD> B;
  B.set(cell, t);
  A acc[NC], accy[NC], accz[NC];
  quad_rows<Tc, NC, GRAD, A>(g, coef, scale, B, q, acc, accy, accz);
  const A bq = pick4(B.b[0], q);
  A u[NC], gx[NC], gy[NC], gz[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    u[c] = group_sum<4>(bq * acc[c]);
    if (GRAD) {
      const A dbq = pick4(B.db[0], q);
      gx[c] = group_sum<4>(dbq * acc[c]) * (A)g.inv_h[0];
      gy[c] = group_sum<4>(bq * accy[c]) * (A)g.inv_h[1];
      gz[c] = group_sum<4>(bq * accz[c]) * (A)g.inv_h[2];
    }
  }
  if (!valid || q != 0) return;
  if (!ok) flag_status(status, PS_DEV_NONFINITE_POS, p);
  const float nanf_ = __int_as_float(0x7fc00000);
  if (MODE <= 1) {
#pragma unroll
    for (int c = 0; c < NC; ++c) vel[(int64_t)c * np + p] = ok ? (float)u[c] : nanf_;
    if (MODE == 1 && grad) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        grad[((int64_t)c * 3 + 0) * np + p] = ok ? (float)gx[c] : nanf_;
        grad[((int64_t)c * 3 + 1) * np + p] = ok ? (float)gy[c] : nanf_;
        grad[((int64_t)c * 3 + 2) * np + p] = ok ? (float)gz[c] : nanf_;
      }
    }
  } else {
    A sx = A(0), sy = A(0), sz = A(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const A w = (A)gvel[(int64_t)c * np + p];
      sx += w * gx[c];
      sy += w * gy[c];
      sz += w * gz[c];
    }
    const double nand = __longlong_as_double(0x7ff8000000000000ll);
    gpos[p] = ok ? (double)sx : nand;
    gpos[np + p] = ok ? (double)sy : nand;
    gpos[2 * np + p] = ok ? (double)sz : nand;
  }
}

// Scatter-add of g_vel * basis weights onto the periodic nodes: the adjoint
// of the 64-term sum followed by the adjoint of the periodic padding (fold).
template <int NC>
__global__ void __launch_bounds__(256) scatter_field(GridArgs g, int64_t np,
                                                    const double* __restrict__ pos,
                                                    const float* __restrict__ gvel,
                                                    float* __restrict__ gfield,
                                                    int32_t* status) {
  const int lane = threadIdx.x & 31, q = lane & 3;
  const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const bool valid = p0 < np;
  const int64_t p = valid ? p0 : 0;
  int cell[3];
  float t[3];
  double xd;
  const bool ok = locate_group<4, float>(g, pos, valid ? np : 0, p, lane, cell, t, xd);
  if (!valid) return;  // no shuffles below
  if (!ok) {
    if (q == 0) flag_status(status, PS_DEV_NONFINITE_POS, p);
    return;
  }
  Basis<float, false> B;
  B.set(cell, t);
  float gc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) gc[c] = gvel[(int64_t)c * np + p] * pick4(B.b[0], q);
  const int64_t vol = (int64_t)g.n[0] * g.n[1] * g.n[2];
  const int nodex = padded_to_node(B.a[0] + q, g.n[0]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int nodez = padded_to_node(B.a[2] + k, g.n[2]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nodey = padded_to_node(B.a[1] + j, g.n[1]);
      const float w = B.b[1][j] * B.b[2][k];
      const int64_t off = ((int64_t)nodez * g.n[1] + nodey) * g.n[0] + nodex;
#pragma unroll
      for (int c = 0; c < NC; ++c) atomicAdd(gfield + c * vol + off, w * gc[c]);
    }
  }
}

// Second derivatives of Eq. (spline) by a quad of lanes per particle (lane q
// owns stencil column a_x + q): six sums per component over the 16 (j, k)
// rows with the y and z factors of each derivative, the x factor applied per
// lane before the quad reduction.  hess [ncomp][6][np]: xx, yy, zz, xy, xz, yz.
template <typename Tc, int NC>
__global__ void __launch_bounds__(256) interp_hessian_direct(GridArgs g,
                                                             const Tc* __restrict__ coef,
                                                             const float* __restrict__ scale,
                                                             int64_t np,
                                                             const double* __restrict__ pos,
                                                             float* __restrict__ hess,
                                                             int32_t* status) {
  using A = typename AccOf<Tc>::type;
  const int lane = threadIdx.x & 31, q = lane & 3;
  const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const bool valid = p0 < np;
  const int64_t p = valid ? p0 : 0;
  int cell[3];
  A t[3];
  double xd;
  const bool ok = locate_group<4, A>(g, pos, valid ? np : 0, p, lane, cell, t, xd) || !valid;
  A b[3][4], db[3][4], d2[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    bspline<A>(t[d], b[d]);
    dbspline<A>(t[d], db[d]);
    ddbspline<A>(t[d], d2[d]);
  }
  A s0[NC], sy[NC], sz[NC], syy[NC], szz[NC], syz[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) s0[c] = sy[c] = sz[c] = syy[c] = szz[c] = syz[c] = A(0);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const A v = load_coef<Tc>(coef, scale, g, c, cell[2] + k, cell[1] + j, cell[0] + q);
        s0[c] += b[1][j] * b[2][k] * v;
        sy[c] += db[1][j] * b[2][k] * v;
        sz[c] += b[1][j] * db[2][k] * v;
        syy[c] += d2[1][j] * b[2][k] * v;
        szz[c] += b[1][j] * d2[2][k] * v;
        syz[c] += db[1][j] * db[2][k] * v;
      }
    }
  const A bq = pick4(b[0], q), dbq = pick4(db[0], q), d2q = pick4(d2[0], q);
  const A hx = (A)g.inv_h[0], hy = (A)g.inv_h[1], hz = (A)g.inv_h[2];
  A h[NC][6];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    h[c][0] = group_sum<4>(d2q * s0[c]) * (hx * hx);
    h[c][1] = group_sum<4>(bq * syy[c]) * (hy * hy);
    h[c][2] = group_sum<4>(bq * szz[c]) * (hz * hz);
    h[c][3] = group_sum<4>(dbq * sy[c]) * (hx * hy);
    h[c][4] = group_sum<4>(dbq * sz[c]) * (hx * hz);
    h[c][5] = group_sum<4>(bq * syz[c]) * (hy * hz);
  }
  if (!valid || q != 0) return;
  if (!ok) flag_status(status, PS_DEV_NONFINITE_POS, p);
  const float nanf_ = __int_as_float(0x7fc00000);
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int e = 0; e < 6; ++e) hess[((int64_t)c * 6 + e) * np + p] = ok ? (float)h[c][e] : nanf_;
}

// Lagrangian acceleration a = du/dt + (u . grad) u by a quad per particle:
// u and its gradient from c0, u from c1 (if given) for the time difference.
template <typename Tc>
__global__ void __launch_bounds__(256) lagrangian_accel_direct(
    GridArgs g, const Tc* __restrict__ c0, const float* __restrict__ s0,
    const Tc* __restrict__ c1, const float* __restrict__ s1, double inv_dt, int64_t np,
    const double* __restrict__ pos, float* __restrict__ acc, float* __restrict__ vel,
    int32_t* status) {
  using A = typename AccOf<Tc>::type;
  const int lane = threadIdx.x & 31, q = lane & 3;
  const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const bool valid = p0 < np;
  const int64_t p = valid ? p0 : 0;
  int cell[3];
  A t[3];
  double xd;
  const bool ok = locate_group<4, A>(g, pos, valid ? np : 0, p, lane, cell, t, xd) || !valid;
  Basis<A, true> B;
  B.set(cell, t);
  A a0[3], ay[3], az[3];
  quad_rows<Tc, 3, true, A>(g, c0, s0, B, q, a0, ay, az);
  const A bq = pick4(B.b[0], q), dbq = pick4(B.db[0], q);
  A u[3], gx[3], gy[3], gz[3], u1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u[c] = group_sum<4>(bq * a0[c]);
    gx[c] = group_sum<4>(dbq * a0[c]) * (A)g.inv_h[0];
    gy[c] = group_sum<4>(bq * ay[c]) * (A)g.inv_h[1];
    gz[c] = group_sum<4>(bq * az[c]) * (A)g.inv_h[2];
    u1[c] = u[c];
  }
  if (c1) {
    Basis<A, false> B1;
    B1.set(cell, t);
    quad_rows<Tc, 3, false, A>(g, c1, s1, B1, q, a0, ay, az);
#pragma unroll
    for (int c = 0; c < 3; ++c) u1[c] = group_sum<4>(bq * a0[c]);
  }
  if (!valid || q != 0) return;
  if (!ok) flag_status(status, PS_DEV_NONFINITE_POS, p);
  const float nanf_ = __int_as_float(0x7fc00000);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const A a = gx[c] * u[0] + gy[c] * u[1] + gz[c] * u[2] + (u1[c] - u[c]) * (A)inv_dt;
    acc[(int64_t)c * np + p] = ok ? (float)a : nanf_;
    if (vel) vel[(int64_t)c * np + p] = ok ? (float)u[c] : nanf_;
  }
}

// Fused Heun step with direct gathers (any particle order).
template <typename Tc>
__global__ void __launch_bounds__(256) rk2_direct(GridArgs g, const Tc* __restrict__ c0,
                                                  const float* __restrict__ s0,
                                                  const Tc* __restrict__ c1,
                                                  const float* __restrict__ s1, int64_t np,
                                                  double* pos, float* __restrict__ vel_out,
                                                  double dt, float3 dtih, int32_t* status) {
  using A = typename AccOf<Tc>::type;
  const int lane = threadIdx.x & 31, q = lane & 3;
  const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const bool valid = p0 < np;
  const int64_t p = valid ? p0 : 0;
  int cell[3];
  A t[3];
  double xd;
  bool ok = locate_group<4, A>(g, pos, valid ? np : 0, p, lane, cell, t, xd);
  Basis<A, false> B;
  B.set(cell, t);
  A acc[3], ay[3], az[3];
  quad_rows<Tc, 3, false, A>(g, c0, s0, B, q, acc, ay, az);
  A bq = pick4(B.b[0], q);
  A u1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) u1[c] = group_sum<4>(bq * acc[c]);
  const float dti[3] = {dtih.x, dtih.y, dtih.z};
  int c2[3];
  A t2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if constexpr (std::is_same<A, double>::value) {
      // FP64 coefficients: locate the predictor exactly as x + dt u1
      double xs = __shfl_sync(FULL, xd, (lane & ~3) + d) + dt * u1[d];
      double tt;
      ok &= locate_f64(xs, g.inv_h[d], g.n[d], c2[d], tt);
      t2[d] = tt;
    } else {
      float tt;
      advance_cell(g.n[d], cell[d], t[d], ok ? (float)u1[d] * dti[d] : 0.f, c2[d], tt);
      t2[d] = tt;
    }
  }
  B.set(c2, t2);
  quad_rows<Tc, 3, false, A>(g, c1, s1, B, q, acc, ay, az);
  bq = pick4(B.b[0], q);
  A u2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) u2[c] = group_sum<4>(bq * acc[c]);
  if (!valid) return;
  if (!ok && q == 0) flag_status(status, PS_DEV_NONFINITE_POS, p);
  if (q < 3) {
    const double nand = __longlong_as_double(0x7ff8000000000000ll);
    const double w = (double)(sel3(u1, q) + sel3(u2, q));
    pos[(int64_t)q * np + p] = ok ? fma(dt * 0.5, w, xd) : nand;
    if (vel_out)
      vel_out[(int64_t)q * np + p] = ok ? (float)sel3(u1, q) : __int_as_float(0x7fc00000);
  }
}

// Particle records in shared memory, one entry per particle of the current
// round (kRecords), stored field-major so that neither the per-axis writers
// nor the 8-lane readers conflict on banks:
//   b[d][i]    float4  b_0..3(t_d) of particle i along axis d
//   u[i]       float4  (u, v, w, ok) result of the last gather
//   db[d][i]   float4  b'_0..3(t_d)   (gradient mode only)
//   loc[d][i]  int     brick-local stencil start along d, -1 = outside halo
//   cell[d][i] int     global cell along d, -1 = position not finite
//   nbc[d][i]  int     brick of the new position along d (Heun step only)
// 80 particles per round: a brick of the mid density (64 particles on
// average, Poisson) rarely needs a second, mostly empty round, and the 240
// (particle, axis) tasks still fit two per thread.
constexpr int kRecords = 80;   // particles per round
constexpr int kThreads = 128;  // threads per brick CTA

struct Recs {
  float4* f;  // b[3], u, then db[3] in gradient mode
  int* ip;    // lw, cell[3], then nbc[3] in the Heun step
  __device__ __forceinline__ float4* b(int d) const { return f + d * kRecords; }
  __device__ __forceinline__ float4* u() const { return f + 3 * kRecords; }
  __device__ __forceinline__ float4* db(int d) const { return f + (4 + d) * kRecords; }
  // byte d of lw[i]: brick-local stencil start along d, -1 outside the halo,
  // -2 position not finite
  __device__ __forceinline__ int* lw() const { return ip; }
  __device__ __forceinline__ int* cell(int d) const { return ip + (1 + d) * kRecords; }
  __device__ __forceinline__ int* nbc(int d) const { return ip + (4 + d) * kRecords; }
};
__host__ __device__ constexpr size_t rec_bytes(bool grad) {
  return (size_t)kRecords * (grad ? 7 * sizeof(float4) + 4 * sizeof(int)
                                  : 4 * sizeof(float4) + 7 * sizeof(int));
}

template <bool GRAD>
__device__ __forceinline__ Recs carve_recs(void* base) {
  Recs r;
  r.f = static_cast<float4*>(base);
  r.ip = reinterpret_cast<int*>(r.f + (GRAD ? 7 : 4) * kRecords);
  return r;
}

// One (particle, axis) task of phases A / A': basis along the axis and the
// brick-local index of the stencil start.  The z basis is stored in the order
// (b0, b2, b1, b3) so that a gather lane reads its pair (b_kh, b_kh+2) at once.
template <bool GRAD>
__device__ __forceinline__ void write_axis(const Recs& R, int i, int d, int cell, float t,
                                           bool ok, int P0, int S) {
  float b[4];
  bspline<float>(t, b);
  R.b(d)[i] = d == 2 ? make_float4(b[0], b[2], b[1], b[3]) : make_float4(b[0], b[1], b[2], b[3]);
  if (GRAD) {
    float db[4];
    dbspline<float>(t, db);
    R.db(d)[i] =
        d == 2 ? make_float4(db[0], db[2], db[1], db[3]) : make_float4(db[0], db[1], db[2], db[3]);
  }
  const int l = cell - P0;
  const int code = !ok ? -2 : ((unsigned)l <= (unsigned)(S - 4) ? l : -1);
  reinterpret_cast<signed char*>(R.lw())[4 * i + d] = (signed char)code;
  R.cell(d)[i] = cell;
}

__device__ __forceinline__ float f4get(const float4 v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// Phase B: 8 lanes per particle.  Lane (q, kh) covers stencil column
// x = a_x + q and the z rows k = kh, kh + 2, all four y rows; the partial
// sums meet in a 3-level butterfly.  Shared-memory reads of one particle
// (one 8-lane phase of a 128-bit load) are conflict-free because rows k and
// k+2 are PS = 4 (mod 8) float4 apart.  Returns ok (all axes finite).
template <typename Tc, int NC, bool GRAD>
__device__ __forceinline__ bool gather8(const float4* __restrict__ halo, int PS, int Sx,
                                        const Recs& R, int i, const GridArgs& g,
                                        const Tc* __restrict__ coef,
                                        const float* __restrict__ scale, int q, int kh,
                                        float out[NC], float dx[NC], float dy[NC],
                                        float dz[NC], bool staged_ok = true) {
  const float bxq = reinterpret_cast<const float*>(R.b(0))[4 * i + q];
  const float4 by = R.b(1)[i];
  const float2 bzp = reinterpret_cast<const float2*>(R.b(2))[2 * i + kh];
  const float bz[2] = {bzp.x, bzp.y};
  const int w = R.lw()[i];
  const bool ok = (__vcmpeq4(w, 0xfefefefe) & 0x00ffffff) == 0;
  const bool inh = staged_ok && (w & 0x00808080) == 0;
  float4 dby = make_float4(0.f, 0.f, 0.f, 0.f);
  float dbz[2] = {0.f, 0.f};
  if (GRAD) {
    dby = R.db(1)[i];
    const float2 d2 = reinterpret_cast<const float2*>(R.db(2))[2 * i + kh];
    dbz[0] = d2.x;
    dbz[1] = d2.y;
  }
  float acc[NC], accy[NC], accz[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = accy[c] = accz[c] = 0.f;
  if (inh) {
    const int lx = (signed char)(w & 0xff), ly = (signed char)((w >> 8) & 0xff),
              lz = (signed char)((w >> 16) & 0xff);
    const float4* hp = halo + (lz + kh) * PS + ly * Sx + lx + q;
    if constexpr (NC == 3 && !GRAD) {
      // u and v as one packed pair (two FP32 FMAs per instruction, each
      // rounded as fmaf), w alone
      float2 auv = make_float2(0.f, 0.f);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 v = hp[2 * kk * PS + j * Sx];
          const float w = f4get(by, j) * bz[kk];
          auv = __ffma2_rn(make_float2(w, w), make_float2(v.x, v.y), auv);
          acc[2] = fmaf(w, v.z, acc[2]);
        }
      }
      acc[0] = auv.x;
      acc[1] = auv.y;
    } else {
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 v = hp[2 * kk * PS + j * Sx];
          const float vv[3] = {v.x, v.y, v.z};
          const float w = f4get(by, j) * bz[kk];
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = fmaf(w, vv[c], acc[c]);
          if (GRAD) {
            const float wy = f4get(dby, j) * bz[kk], wz = f4get(by, j) * dbz[kk];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              accy[c] = fmaf(wy, vv[c], accy[c]);
              accz[c] = fmaf(wz, vv[c], accz[c]);
            }
          }
        }
      }
    }
  } else {
    const int ax = max(R.cell(0)[i], 0), ay = max(R.cell(1)[i], 0), az = max(R.cell(2)[i], 0);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float w = f4get(by, j) * bz[kk];
        // a node's components by one load, the values load_coef would give
        float nv[3] = {0.f, 0.f, 0.f};
        if constexpr (IsNode4<Tc>::value && NC == 3) {
          const int64_t row = (int64_t)(az + kh + 2 * kk) * g.m[1] + ay + j;
          if constexpr (IsNode16<Tc>::value) {
            const Tc n = coef[row * g.rx + ax + q];
#pragma unroll
            for (int c = 0; c < 3; ++c) nv[c] = node16_value(n.v[c]) * __ldg(scale + row * 4 + c);
          } else {
            const float4 n = __ldg(reinterpret_cast<const float4*>(coef) + row * g.rx + ax + q);
            nv[0] = n.x;
            nv[1] = n.y;
            nv[2] = n.z;
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float v = (IsNode4<Tc>::value && NC == 3)
                              ? nv[c]
                              : (float)load_coef<Tc>(coef, scale, g, c, az + kh + 2 * kk, ay + j,
                                                     ax + q);
          acc[c] = fmaf(w, v, acc[c]);
          if (GRAD) {
            accy[c] = fmaf(f4get(dby, j) * bz[kk], v, accy[c]);
            accz[c] = fmaf(f4get(by, j) * dbz[kk], v, accz[c]);
          }
        }
      }
    }
  }
  if constexpr (NC == 3) {
    // the butterfly over the group with u and v packed (each sum rounded as
    // the scalar one)
    const float2 uv = group_sum2<8>(__fmul2_rn(make_float2(bxq, bxq), make_float2(acc[0], acc[1])));
    out[0] = uv.x;
    out[1] = uv.y;
    out[2] = group_sum<8>(bxq * acc[2]);
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = group_sum<8>(bxq * acc[c]);
  }
  if (GRAD) {
    const float dbxq = reinterpret_cast<const float*>(R.db(0))[4 * i + q];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      dx[c] = group_sum<8>(dbxq * acc[c]) * g.inv_hf[0];
      dy[c] = group_sum<8>(bxq * accy[c]) * g.inv_hf[1];
      dz[c] = group_sum<8>(bxq * accz[c]) * g.inv_hf[2];
    }
  }
  return ok;
}

// Particles [beg, end) of one brick whose halo is in shared memory, in rounds
// of kRecords:
//   A  one thread per (particle, axis): locate (exact FP64 index arithmetic),
//      basis along the axis, brick-local index;
//   B  8 lanes per particle: gather and sum (writes the result or u1);
//   A' (Heun) one thread per (particle, axis): predictor cell in FP32;
//   B' second gather (u2);
//   C  one thread per (particle, axis): FP64 position update and stores.
template <typename Tc, int NC, int MODE, int KS = 0>
__device__ __forceinline__ void process_brick(const StagedArgs& a, int beg, int end,
                                              const int P0[3], const float4* halo,
                                              const Recs& R,
                                              unsigned long long* mbar = nullptr,
                                              const unsigned char* raw16 = nullptr,
                                              unsigned parity = 0,
                                              unsigned long long* probe = nullptr) {
  constexpr bool GRAD = MODE == 1;
  bool copied = true;  // the halo's tensor copy completed (or there is none)
  const GridArgs& g = a.g;
  const Tc* coef = static_cast<const Tc*>(a.coef);
  const int tid = threadIdx.x, lane = tid & 31;
  const int q = lane & 3, kh = (lane >> 2) & 1, sub = lane & 7;
  const int warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t np = a.np;
  const float nanf_ = __int_as_float(0x7fc00000);
  constexpr int TPT = (3 * kRecords + kThreads - 1) / kThreads;  // tasks per thread
  const HaloGeo<KS> hg(a);

  for (int cb = beg; cb < end; cb += kRecords) {
    const int m = min(kRecords, end - cb);
    // phase A: tasks (particle i, axis d), task = d * m + i
    int ti[TPT], td[TPT], tcell[TPT];
    float tt[TPT];
    double tx[TPT];
    int64_t tp[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int task = tid + k * kThreads;
      td[k] = task < m ? 0 : (task < 2 * m ? 1 : (task < 3 * m ? 2 : -1));
      ti[k] = task - max(td[k], 0) * m;
      tcell[k] = 0;
      tt[k] = 0.f;
      tx[k] = 0.0;
      tp[k] = 0;
      if (td[k] >= 0) {
        const int i = ti[k], d = td[k];
        tp[k] = a.perm ? a.perm[cb + i] : (int64_t)(cb + i);
        tx[k] = a.pos_in[d * np + tp[k]];
        const bool ok = locate(tx[k], g.inv_h[d], g.n[d], tcell[k], tt[k]);
        write_axis<GRAD>(R, i, d, tcell[k], tt[k], ok, sel3(P0, d),
                         d == 0 ? hg.Sx : (d == 1 ? hg.Sy : hg.Sz));
      }
    }
    __syncthreads();
    // the barrier above also ordered the mbarrier's initialisation before
    // these waits; a copy that does not complete in time is reported and the
    // brick's particles read global memory (one decision for the whole
    // block: the 16-bit widening below is shared)
    if (mbar && cb == beg) {
      bool done = tma_wait(mbar, parity);
      if (done && probe) done = tma_wait(probe, 0, a.wait_probe);
      copied = __syncthreads_and(done);
      if (!copied && threadIdx.x == 0) flag_status(a.status, PS_DEV_TIMEOUT, beg);
    }
    // (16-bit node copies come only with the 8^3 halo of 12-node rows)
    if constexpr (IsNode16<Tc>::value && KS == 12) {
      if (raw16 && cb == beg) {
        // the copied 16-bit nodes and their rows' scales -> float4 halo in
        // the same buffer, slice by slice; the copy's rows are SX nodes long,
        // the halo's rows too (dense planes)
        const Tc* nodes = reinterpret_cast<const Tc*>(raw16);
        const float4* scl = reinterpret_cast<const float4*>(
            raw16 + (node16_scale_offset(hg.Sz, hg.PS, hg.Sy) -
                     node16_raw_offset(hg.Sz, hg.PS, hg.Sy, hg.SX)));
        float4* h = const_cast<float4*>(halo);
        constexpr int npts = HaloGeo<KS>::Sz * HaloGeo<KS>::Sy * HaloGeo<KS>::SX;
        constexpr int per = (npts + kNode16Slices - 1) / kNode16Slices;
        constexpr int kPer = (per + kThreads - 1) / kThreads;  // nodes per thread per slice
#pragma unroll 1
        for (int sl = 0; sl < kNode16Slices; ++sl) {
          const int lo = sl * per, hi = min(npts, lo + per);
          float4 v[kPer];
#pragma unroll
          for (int k = 0; k < kPer; ++k) {
            const int it = lo + threadIdx.x + k * kThreads;
            if (it < hi) {
              const Tc n = nodes[it];
              const float4 sc = scl[it / hg.SX];
              v[k] = make_float4(node16_value(n.v[0]) * sc.x, node16_value(n.v[1]) * sc.y,
                                 node16_value(n.v[2]) * sc.z, 0.f);
            }
          }
          __syncthreads();
#pragma unroll
          for (int k = 0; k < kPer; ++k) {
            const int it = lo + threadIdx.x + k * kThreads;
            if (it < hi) h[it] = v[k];
          }
        }
        __syncthreads();
      }
    }
    // phase B: gathers, 8 lanes per particle; the loop is uniform per warp
    // (the butterfly uses full-warp shuffles), idle groups redo record b4
    for (int b4 = warp * 4; b4 < m; b4 += nwarps * 4) {
      const int i = b4 + (lane >> 3);
      const bool vi = i < m;
      float u[NC], dx[NC], dy[NC], dz[NC];
      const bool oki = gather8<Tc, NC, GRAD>(halo, hg.PS, hg.SX, R, vi ? i : b4, g, coef, a.scale,
                                             q, kh, u, dx, dy, dz, copied);
      if (!vi) continue;
      if constexpr (MODE <= 1) {
        const int64_t pi = a.perm ? a.perm[cb + i] : (int64_t)(cb + i);
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (sub == c) a.vel[(int64_t)c * np + pi] = oki ? u[c] : nanf_;
        if (GRAD && a.grad) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (sub == 3) a.grad[((int64_t)c * 3 + 0) * np + pi] = oki ? dx[c] : nanf_;
            if (sub == 4) a.grad[((int64_t)c * 3 + 1) * np + pi] = oki ? dy[c] : nanf_;
            if (sub == 5) a.grad[((int64_t)c * 3 + 2) * np + pi] = oki ? dz[c] : nanf_;
          }
        }
        if (sub == 7 && !oki) flag_status(a.status, PS_DEV_NONFINITE_POS, pi);
      } else {
        if (sub == 0) R.u()[i] = make_float4(u[0], u[1], u[2], __int_as_float(oki ? 1 : 0));
      }
    }
    __syncthreads();
    if constexpr (MODE == 2) {
    // phase A': predictor located in FP32 relative to the stage-1 cell
    float tu1[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      tu1[k] = 0.f;
      if (td[k] >= 0) {
        const int i = ti[k], d = td[k];
        const float4 r = R.u()[i];
        const bool ok = __float_as_int(r.w) != 0;
        tu1[k] = f4get(r, d);
        float t2 = tt[k] + (ok ? tu1[k] * a.dtih[d] : 0.f);
        float fl = floorf(t2);
        if (!(fabsf(fl) < 1.0e9f)) fl = 0.f;
        t2 = fminf(fmaxf(t2 - fl, 0.f), 1.f);
        int c = tcell[k] + (int)fl;
        if (c < 0 || c >= g.n[d]) {
          c %= g.n[d];
          if (c < 0) c += g.n[d];
        }
        write_axis<false>(R, i, d, c, t2, ok, sel3(P0, d), d == 0 ? hg.Sx : (d == 1 ? hg.Sy : hg.Sz));
        if (a.coef2 && ok)  // second field: its coefficients are not staged
          reinterpret_cast<signed char*>(R.lw())[4 * i + d] = (signed char)-1;
        // the predictor's fraction waits in nbc for phase C (the same task
        // reads it there before it writes the slot)
        if (a.next_counts) R.nbc(d)[i] = __float_as_int(t2);
      }
    }
    __syncthreads();
    // phase B': second gathers
    const Tc* cf2 = a.coef2 ? static_cast<const Tc*>(a.coef2) : coef;
    const float* sc2 = a.coef2 ? a.scale2 : a.scale;
    for (int b4 = warp * 4; b4 < m; b4 += nwarps * 4) {
      const int i = b4 + (lane >> 3);
      const bool vi = i < m;
      float u[NC], dx[NC], dy[NC], dz[NC];
      const bool oki = gather8<Tc, NC, false>(halo, hg.PS, hg.SX, R, vi ? i : b4, g, cf2, sc2, q,
                                              kh, u, dx, dy, dz, copied);
      if (vi && sub == 0) R.u()[i] = make_float4(u[0], u[1], u[2], __int_as_float(oki ? 1 : 0));
    }
    __syncthreads();
    // phase C: FP64 position update, one thread per (particle, axis); with
    // next_counts the new brick coordinate along the axis goes to nbc
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      if (td[k] >= 0) {
        const int i = ti[k], d = td[k];
        const float4 r = R.u()[i];
        const bool ok = __float_as_int(r.w) != 0;
        const int64_t pp = tp[k];
        const double xn = ok ? fma(a.dt * 0.5, (double)(tu1[k] + f4get(r, d)), tx[k])
                             : __longlong_as_double(0x7ff8000000000000ll);
        a.pos_out[d * np + pp] = xn;
        if (a.vel) a.vel[d * np + pp] = ok ? tu1[k] : nanf_;
        if (d == 0) {
          if (a.ids_out) a.ids_out[pp] = a.ids_in[pp];
          if (!ok) flag_status(a.status, PS_DEV_NONFINITE_POS, pp);
        }
        if (a.next_counts) {
          // The new cell: the predictor's cell plus the floor of its fraction
          // plus the corrector's displacement dt (u2 - u1) / 2 in cells, in
          // FP32 (x^{n+1} = x* + dt (u2 - u1) / 2).  That floor is the exact
          // one wherever the sum lies 2^-10 or more from a cell face and
          // |x n/L| < 2^30: the FP32 and FP64 roundings on both routes stay
          // below 1e-6 cell.  Elsewhere (and for positions that are not
          // finite) the FP64 location decides.
          const float w = __int_as_float(R.nbc(d)[i]) +
                          0.5f * a.dtih[d] * (f4get(r, d) - tu1[k]);
          const float fl = floorf(w), fr = w - fl;
          int c;
          if (ok && fr >= 0x1p-10f && fr <= 1.f - 0x1p-10f && fabsf(fl) <= 2.f &&
              (__double2hiint(tx[k]) & 0x7fffffff) < a.xguard_hi[d]) {
            const int nd = g.n[d];
            c = R.cell(d)[i] + (int)fl;  // in [-2, n + 1], n >= 3
            c = c < 0 ? c + nd : (c >= nd ? c - nd : c);
          } else {
            float tn;
            if (!locate(xn, g.inv_h[d], g.n[d], c, tn)) c = -1;
          }
          R.nbc(d)[i] = c < 0 ? -1 : (a.bshift[d] >= 0 ? c >> a.bshift[d] : c / a.b.B[d]);
        }
      }
    }
    __syncthreads();
    // phase D: the next step's counting, one thread per particle in the last
    // warps, which hold fewer (particle, axis) tasks in phases A and C than
    // the first ones (nothing below reads these records before the next
    // round's phase C, several barriers on)
    constexpr int kCountWarps = (kRecords + 31) / 32;
    if (a.next_counts && warp >= nwarps - kCountWarps) {
      const int i = tid - (nwarps - kCountWarps) * 32;
      const bool vi = i < m;
      const int64_t pp = vi ? (a.perm ? a.perm[cb + i] : (int64_t)(cb + i)) : 0;
      int key = vi ? bin_of_coords(a.b, R.nbc(0)[i], R.nbc(1)[i], R.nbc(2)[i]) : 0;
      if (a.next_runs > 0 && key >= 0) key = (int)((int64_t)key * a.next_runs / a.b.nbins);
      count_into_bin(a.next_counts, a.next_bin, a.status, vi, pp, key, a.next_key_base);
    }
    }  // MODE == 2
  }
  // a copy still in flight must land before the block's memory is released
  if (!copied) tma_wait(mbar, parity);
}

// Phased form of one brick: stage the halo (unless the brick holds fewer than
// min_stage particles, whose stencils are then read from global memory), then
// the location / gather / update phases of process_brick.
template <typename Tc, int NC, int MODE, bool TMA = false>
__device__ __forceinline__ void brick_phased(const StagedArgs& a, int bin, float4* smem,
                                             const StagedArgs* maps = nullptr) {
  const int beg = a.offs[bin], end = a.offs[bin + 1];
  if (beg >= end) return;
  const int nbx = a.b.nb[0], nby = a.b.nb[1];
  const int bzi = bin / (nbx * nby);
  const int rem = bin - bzi * nbx * nby;
  const int byi = rem / nbx, bxi = rem - byi * nbx;
  const int P0[3] = {bxi * a.b.B[0] - a.E, byi * a.b.B[1] - a.E, bzi * a.b.B[2] - a.E};
  const Tc* coef = static_cast<const Tc*>(a.coef);
  float4* halo = smem;
  const Recs R = carve_recs<MODE == 1>(smem + a.S[2] * a.PS);
  if (end - beg < a.min_stage || a.chunked) {
    // an origin far from every cell sends every stencil to global memory
    const int far[3] = {-(1 << 29), -(1 << 29), -(1 << 29)};
    process_brick<Tc, NC, MODE>(a, beg, end, far, halo, R);
    return;
  }
  if constexpr (TMA && IsNode4<Tc>::value) {
    // `maps` (with the tensor maps) is the kernel argument block or lies in
    // global memory; the destinations must be 128-byte aligned
    if (a.tma && maps && is_cube11_rows12(a) && (smem_u32(halo) & 127) == 0) {
      __shared__ __align__(8) unsigned long long mbar, probe_bar;
      using G = HaloGeo<12>;
      // test knob: a barrier that nothing completes, waited on after the copy
      unsigned long long* probe = a.wait_probe > 0 ? &probe_bar : nullptr;
      if (probe && threadIdx.x == 0) tma_init_barrier(probe);
      if constexpr (IsNode16<Tc>::value) {
        unsigned char* base = reinterpret_cast<unsigned char*>(halo);
        unsigned char* raw = base + node16_raw_offset(G::Sz, G::PS, G::Sy, G::SX);
        unsigned char* sraw = base + node16_scale_offset(G::Sz, G::PS, G::Sy);
        if (threadIdx.x == 0)
          tma_issue_node16(&maps->tmap, &maps->tmap2, raw, sraw, &mbar, P0,
                           (unsigned)(G::Sz * G::Sy * (G::SX * 8 + 16)));
        process_brick<Tc, NC, MODE, 12>(a, beg, end, P0, halo, R, &mbar,
                                        raw, 0, probe);
      } else {
        if (threadIdx.x == 0)
          tma_issue_halo(&maps->tmap, halo, &mbar, P0,
                         (unsigned)(sizeof(float4) * G::PS * G::Sz));
        process_brick<Tc, NC, MODE, 12>(a, beg, end, P0, halo, R, &mbar,
                                        nullptr, 0, probe);
      }
      return;
    }
  }
  // no barrier here: phase A of the first round does not read the halo, and
  // the barrier that follows it also publishes the staged halo
  if (a.vec && is_cube11(a)) {
    stage_halo_vec<Tc, NC, 11>(a, coef, P0, halo, false);
    process_brick<Tc, NC, MODE, 11>(a, beg, end, P0, halo, R);
    return;
  }
  if (a.vec && is_cube11_rows12(a)) {
    stage_halo_vec<Tc, NC, 12>(a, coef, P0, halo, false);
    process_brick<Tc, NC, MODE, 12>(a, beg, end, P0, halo, R);
    return;
  }
  if (a.vec)
    stage_halo_vec<Tc, NC>(a, coef, P0, halo, false);
  else
    stage_halo<Tc, NC>(a, coef, P0, halo, false);
  process_brick<Tc, NC, MODE>(a, beg, end, P0, halo, R);
}

// MODE 0: vel; 1: vel + grad; 2: fused Heun step.  One CTA per brick.  The
// argument block is a grid constant so that its tensor map can be named by
// the tensor copy.
template <typename Tc, int NC, int MODE>
__global__ void __launch_bounds__(kThreads, sizeof(Tc) == 2 ? 6 : 7)
    interp_staged(const __grid_constant__ StagedArgs a) {
  extern __shared__ __align__(128) float4 smem_a128[];
  brick_phased<Tc, NC, MODE, true>(a, blockIdx.x, smem_a128, &a);
}

// Global brick b of a many-field batch: the field is the last f with
// bin_base[f] <= b; its arguments are copied to shared memory (sa), its tensor
// map stays in the global table.  Empty bins return at once.  Every thread of
// the block calls.
template <typename Tc, int NC, int MODE>
__device__ __forceinline__ void batch_brick(const StagedArgs* __restrict__ tab,
                                            const int* __restrict__ bin_base, int nfields,
                                            int b, float4* smem, StagedArgs& sa) {
  // field 0's offsets are the global offsets: empty bins leave at once
  const int32_t* goffs = tab[0].offs;
  if (goffs[b] >= goffs[b + 1]) return;
  int lo = 0, hi = nfields;  // bin_base[lo] <= b < bin_base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (bin_base[mid] <= b) lo = mid;
    else hi = mid;
  }
  constexpr int kWords = (int)(sizeof(StagedArgs) / sizeof(int4));
  static_assert(sizeof(StagedArgs) % sizeof(int4) == 0, "argument block copied in 16 bytes");
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    reinterpret_cast<int4*>(&sa)[i] = reinterpret_cast<const int4*>(tab + lo)[i];
  // the field's tensor map stays in the global table (a tensor copy cannot
  // name one in shared memory); order its upload before the copy proxy
  if (threadIdx.x == 0 && IsNode4<Tc>::value && tab[lo].tma) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<unsigned long long>(&tab[lo].tmap))
                 : "memory");
    if (IsNode16<Tc>::value)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                       reinterpret_cast<unsigned long long>(&tab[lo].tmap2))
                   : "memory");
  }
  __syncthreads();
  brick_phased<Tc, NC, MODE, true>(sa, b - bin_base[lo], smem, tab + lo);
}

// Many fields in one launch: block b handles global brick b.
template <typename Tc, int NC, int MODE>
__global__ void __launch_bounds__(kThreads, 5)
    interp_staged_batch(const StagedArgs* __restrict__ tab, const int* __restrict__ bin_base,
                        int nfields) {
  extern __shared__ __align__(128) float4 smem_b128[];
  __shared__ StagedArgs sa;
  batch_brick<Tc, NC, MODE>(tab, bin_base, nfields, blockIdx.x, smem_b128, sa);
}

constexpr int kParamFields = 48;  // 48 x 640 bytes of arguments: within the 32 KB of parameters
struct BatchParams {
  StagedArgs a[kParamFields];
  int bin_base[kParamFields + 1];
  int nfields;
};
static_assert(sizeof(BatchParams) <= 32764, "kernel parameters are limited to 32764 bytes");

// A batch of at most kParamFields fields passes its argument table as one
// kernel parameter: the brick body then reads each field's arguments from the
// constant bank, as the single-field kernel does (72 registers, 7 blocks per
// SM), instead of from a shared-memory copy (96 registers, 5 blocks); the
// tensor maps are named in parameter space like the single-field kernel's.
template <typename Tc, int NC, int MODE>
__global__ void __launch_bounds__(kThreads, sizeof(Tc) == 2 ? 6 : 7)
    interp_staged_batch_p(const __grid_constant__ BatchParams tab) {
  extern __shared__ __align__(128) float4 smem_bp128[];
  const int b = blockIdx.x;
  // field 0's offsets are the global offsets: empty bins leave at once
  const int32_t* goffs = tab.a[0].offs;
  if (goffs[b] >= goffs[b + 1]) return;
  int lo = 0, hi = tab.nfields;  // bin_base[lo] <= b < bin_base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tab.bin_base[mid] <= b) lo = mid;
    else hi = mid;
  }
  brick_phased<Tc, NC, MODE, true>(tab.a[lo], b - tab.bin_base[lo], smem_bp128, &tab.a[lo]);
}

// ----------------------------------------------------- persistent batch ----
// All Heun steps of a many-field batch in one cooperative launch: per step
// the three scan phases, the scatter into bin order, then the bricks of all
// fields, which count the bins of the positions they write for the next
// step (the first step counts from the positions, scatters by rank and
// clears the counters; later ones scatter from the counts, which end at
// zero); the phases are separated by grid-wide barriers.  Each barrier is an arrival
// counter and a generation word; a wait gives up after about 2^31 clocks,
// sets the block-stop word and PS_DEV_TIMEOUT, and every block leaves at its
// next barrier.  sync[3] is a word nothing sets: with wait_probe > 0 (a test
// knob) every block waits on it after the first barrier, for that many
// clocks, so that the give-up path runs.  sync[4] is the brick pass's claim
// counter: blocks take kClaim consecutive global bins at a time.
struct BatchRun {
  const StagedArgs* tab;   // per-field brick-kernel arguments
  const int* bin_base;     // nfields + 1
  const BinField* bintab;  // per-field binning table
  int nfields;
  int nsteps;
  int64_t total_bins, np;
  double* pos;             // the caller's positions (bin order after a step)
  int64_t* ids;
  double* pos_s;           // copies in bin order (workspace)
  int64_t* ids_s;
  int32_t* bin_of;
  int32_t* rank;
  int32_t* counts;         // total_bins + 1, zero at launch
  int32_t* offsets;        // total_bins + 1
  int32_t* scan_tmp;
  int32_t* status;
  unsigned* sync;          // arrivals, generation, stop, never set, claims; zero at launch
  int wait_probe;
};

__device__ __forceinline__ bool grid_barrier(const BatchRun& r, int& nbar) {
  __shared__ int go;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vs = r.sync;
    bool ok = vs[2] == 0;
    if (ok) {
      const unsigned gen = vs[1];
      __threadfence();
      if (atomicAdd(&r.sync[0], 1u) + 1u == gridDim.x) {
        atomicExch(&r.sync[0], 0u);
        __threadfence();
        atomicAdd(&r.sync[1], 1u);
      } else {
        const long long t0 = clock64();
        while (vs[1] == gen) {
          if (vs[2]) {
            ok = false;
            break;
          }
          if (clock64() - t0 > (1ll << 31)) {
            if (atomicExch(&r.sync[2], 1u) == 0u) flag_status(r.status, PS_DEV_TIMEOUT, nbar);
            ok = false;
            break;
          }
          __nanosleep(100);
        }
      }
      __threadfence();
      if (ok && r.wait_probe > 0 && nbar == 0) {
        const long long t0 = clock64();
        while (vs[3] == 0 && clock64() - t0 <= r.wait_probe) __nanosleep(100);
        if (vs[3] == 0) {
          if (atomicExch(&r.sync[2], 1u) == 0u) flag_status(r.status, PS_DEV_TIMEOUT, nbar);
          ok = false;
        }
      }
    }
    go = ok ? 1 : 0;
  }
  __syncthreads();
  ++nbar;
  return go != 0;
}

constexpr int kClaim = 4;  // global bins per claim of the persistent brick pass

template <typename Tc>
__global__ void __launch_bounds__(kThreads, 5) batch_persistent(const __grid_constant__ BatchRun r) {
  extern __shared__ __align__(128) float4 smem_bp[];
  __shared__ StagedArgs sa;
  __shared__ int32_t scan_sh[kThreads / 32];
  __shared__ int64_t claim;
  int nbar = 0;
  const int lane = threadIdx.x & 31;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const int64_t ntiles = (r.total_bins + kScanTile - 1) / kScanTile;
  for (int step = 0; step < r.nsteps; ++step) {
    // the first step counts from the positions; later ones scan the counts
    // the previous step's bricks took
    if (step == 0) {
      batch_count_range(r.bintab, r.nfields, r.np, r.pos, r.bin_of, r.rank, r.counts, r.status,
                        gt - lane, gs);
      if (!grid_barrier(r, nbar)) return;
    }
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
      scan_tile_sum<kThreads>(r.counts, r.total_bins, t, r.scan_tmp, scan_sh);
    if (!grid_barrier(r, nbar)) return;
    if (blockIdx.x == 0) scan_tile_offsets_block<kThreads>(r.scan_tmp, ntiles, scan_sh);
    if (!grid_barrier(r, nbar)) return;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
      scan_tile<kThreads>(r.counts, r.total_bins, r.scan_tmp, r.offsets, -1, t, ntiles,
                          scan_sh);
    if (!grid_barrier(r, nbar)) return;
    if (step == 0) {
      scatter_range(r.np, r.pos, r.bin_of, r.rank, r.offsets, nullptr, r.pos_s, r.ids,
                    r.ids ? r.ids_s : nullptr, gt, gs);
      for (int64_t i = gt; i <= r.total_bins; i += gs) r.counts[i] = 0;
    } else {  // the counters end at zero, ready for this step's counting
      scatter_counted_range(r.np, r.pos, r.bin_of, r.counts, r.offsets, nullptr, r.pos_s,
                            r.ids, r.ids ? r.ids_s : nullptr, r.total_bins, r.status, gt >> 5,
                            gs >> 5);
    }
    if (gt == 0) atomicExch(&r.sync[4], 0u);
    if (!grid_barrier(r, nbar)) return;
    // bricks claimed kClaim at a time (their costs vary with their particles)
    while (true) {
      if (threadIdx.x == 0) claim = (int64_t)atomicAdd(&r.sync[4], 1u) * kClaim;
      __syncthreads();
      const int64_t b0 = claim;
      __syncthreads();
      if (b0 >= r.total_bins) break;
      for (int64_t b = b0; b < b0 + kClaim && b < r.total_bins; ++b) {
        batch_brick<Tc, 3, 2>(r.tab, r.bin_base, r.nfields, (int)b, smem_bp, sa);
        __syncthreads();  // sa and the shared memory are refilled by the next brick
      }
    }
    if (!grid_barrier(r, nbar)) return;
  }
}

// ------------------------------------------------- thread per particle ----
// One thread carries a particle through every step: exact location, the 12
// basis values, its 64 stencil points read from the staged halo (128-bit
// loads; lanes of a warp hit random banks, the price of needing no records,
// shuffles or further barriers), the Heun predictor and the FP64 update.

template <int NC, bool GRAD>
struct Sum1 {
  float u[NC], gx[NC], gy[NC], gz[NC];
};

// 64-term sum of Eq. (spline) by one thread; `row(k, j)` returns the four
// x-consecutive points of stencil row (j, k) as float4 (u, v, w, -).
template <int NC, bool GRAD, typename RowFn>
__device__ __forceinline__ void sum64(const float bx[4], const float by[4], const float bz[4],
                                      const float dbx[4], const float dby[4], const float dbz[4],
                                      RowFn row, Sum1<NC, GRAD>& r) {
#pragma unroll
  for (int c = 0; c < NC; ++c) r.u[c] = r.gx[c] = r.gy[c] = r.gz[c] = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float4 v[4];
      row(k, j, v);
      const float w = by[j] * bz[k];
      float wy = 0.f, wz = 0.f;
      if (GRAD) {
        wy = dby[j] * bz[k];
        wz = by[j] * dbz[k];
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float v0 = c == 0 ? v[0].x : (c == 1 ? v[0].y : v[0].z);
        const float v1 = c == 0 ? v[1].x : (c == 1 ? v[1].y : v[1].z);
        const float v2 = c == 0 ? v[2].x : (c == 1 ? v[2].y : v[2].z);
        const float v3 = c == 0 ? v[3].x : (c == 1 ? v[3].y : v[3].z);
        float sx = bx[0] * v0;
        sx = fmaf(bx[1], v1, sx);
        sx = fmaf(bx[2], v2, sx);
        sx = fmaf(bx[3], v3, sx);
        r.u[c] = fmaf(w, sx, r.u[c]);
        if (GRAD) {
          float dx = dbx[0] * v0;
          dx = fmaf(dbx[1], v1, dx);
          dx = fmaf(dbx[2], v2, dx);
          dx = fmaf(dbx[3], v3, dx);
          r.gx[c] = fmaf(w, dx, r.gx[c]);
          r.gy[c] = fmaf(wy, sx, r.gy[c]);
          r.gz[c] = fmaf(wz, sx, r.gz[c]);
        }
      }
    }
}

template <typename Tc, int NC, bool GRAD>
__device__ __forceinline__ void gather1(const StagedArgs& a, const Tc* __restrict__ coef,
                                        const float* __restrict__ scale,
                                        const float4* __restrict__ halo, const int P0[3],
                                        const int cell[3], const float t[3],
                                        Sum1<NC, GRAD>& r) {
  const GridArgs& g = a.g;
  float bx[4], by[4], bz[4], dbx[4], dby[4], dbz[4];
  bspline<float>(t[0], bx);
  bspline<float>(t[1], by);
  bspline<float>(t[2], bz);
  if (GRAD) {
    dbspline<float>(t[0], dbx);
    dbspline<float>(t[1], dby);
    dbspline<float>(t[2], dbz);
  }
  const int lx = cell[0] - P0[0], ly = cell[1] - P0[1], lz = cell[2] - P0[2];
  const bool inh = (unsigned)lx <= (unsigned)(a.S[0] - 4) &&
                   (unsigned)ly <= (unsigned)(a.S[1] - 4) &&
                   (unsigned)lz <= (unsigned)(a.S[2] - 4);
  if (inh) {
    const float4* base = halo + lz * a.PS + ly * a.SX + lx;
    const int PS = a.PS, Sx = a.SX;
    sum64<NC, GRAD>(bx, by, bz, dbx, dby, dbz,
                    [&](int k, int j, float4 v[4]) {
                      const float4* rp = base + k * PS + j * Sx;
                      v[0] = rp[0];
                      v[1] = rp[1];
                      v[2] = rp[2];
                      v[3] = rp[3];
                    },
                    r);
  } else {
    sum64<NC, GRAD>(bx, by, bz, dbx, dby, dbz,
                    [&](int k, int j, float4 v[4]) {
#pragma unroll
                      for (int i = 0; i < 4; ++i) {
                        float vv[3] = {0.f, 0.f, 0.f};
#pragma unroll
                        for (int c = 0; c < NC; ++c)
                          vv[c] = load_coef<Tc>(coef, scale, g, c, cell[2] + k, cell[1] + j,
                                                cell[0] + i);
                        v[i] = make_float4(vv[0], vv[1], vv[2], 0.f);
                      }
                    },
                    r);
  }
  if (GRAD) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      r.gx[c] *= g.inv_hf[0];
      r.gy[c] *= g.inv_hf[1];
      r.gz[c] *= g.inv_hf[2];
    }
  }
}

template <typename Tc, int NC, int MODE>
__global__ void __launch_bounds__(64) interp_thread(StagedArgs a) {
  extern __shared__ float4 smem[];
  constexpr bool GRAD = MODE == 1;
  const int bin = blockIdx.x;
  const int beg = a.offs[bin], end = a.offs[bin + 1];
  if (beg >= end) return;
  const int nbx = a.b.nb[0], nby = a.b.nb[1];
  const int bzi = bin / (nbx * nby);
  const int rem = bin - bzi * nbx * nby;
  const int byi = rem / nbx, bxi = rem - byi * nbx;
  const int P0[3] = {bxi * a.b.B[0] - a.E, byi * a.b.B[1] - a.E, bzi * a.b.B[2] - a.E};
  const Tc* coef = static_cast<const Tc*>(a.coef);
  float4* halo = smem;
  if (a.vec)
    stage_halo_vec<Tc, NC>(a, coef, P0, halo);
  else
    stage_halo<Tc, NC>(a, coef, P0, halo);
  const GridArgs& g = a.g;
  const int64_t np = a.np;
  const float nanf_ = __int_as_float(0x7fc00000);
  for (int s = beg + threadIdx.x; s < end; s += blockDim.x) {
    const int64_t p = a.perm ? a.perm[s] : (int64_t)s;
    double x[3];
    int cell[3];
    float t[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      x[d] = a.pos_in[d * np + p];
      ok &= locate(x[d], g.inv_h[d], g.n[d], cell[d], t[d]);
    }
    Sum1<NC, GRAD> r;
    gather1<Tc, NC, GRAD>(a, coef, a.scale, halo, P0, cell, t, r);
    if constexpr (MODE <= 1) {
#pragma unroll
      for (int c = 0; c < NC; ++c) a.vel[(int64_t)c * np + p] = ok ? r.u[c] : nanf_;
      if (GRAD && a.grad) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          a.grad[((int64_t)c * 3 + 0) * np + p] = ok ? r.gx[c] : nanf_;
          a.grad[((int64_t)c * 3 + 1) * np + p] = ok ? r.gy[c] : nanf_;
          a.grad[((int64_t)c * 3 + 2) * np + p] = ok ? r.gz[c] : nanf_;
        }
      }
      if (!ok) flag_status(a.status, PS_DEV_NONFINITE_POS, p);
    } else {
      const float u1[3] = {r.u[0], r.u[1], r.u[2]};
      int c2[3];
      float t2[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float tt = t[d] + (ok ? u1[d] * a.dtih[d] : 0.f);
        float fl = floorf(tt);
        if (!(fabsf(fl) < 1.0e9f)) fl = 0.f;
        t2[d] = fminf(fmaxf(tt - fl, 0.f), 1.f);
        int c = cell[d] + (int)fl;
        if (c < 0 || c >= g.n[d]) {
          c %= g.n[d];
          if (c < 0) c += g.n[d];
        }
        c2[d] = c;
      }
      Sum1<NC, false> r2;
      if (a.coef2) {
        // second field: its coefficients are not staged
        int far[3] = {P0[0] - 1000000, 0, 0};
        gather1<Tc, NC, false>(a, static_cast<const Tc*>(a.coef2), a.scale2, halo, far, c2, t2,
                               r2);
      } else {
        gather1<Tc, NC, false>(a, coef, a.scale, halo, P0, c2, t2, r2);
      }
      const double half_dt = a.dt * 0.5;
      int bc[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double xn = ok ? fma(half_dt, (double)(u1[d] + r2.u[d]), x[d])
                             : __longlong_as_double(0x7ff8000000000000ll);
        a.pos_out[d * np + p] = xn;
        if (a.vel) a.vel[d * np + p] = ok ? u1[d] : nanf_;
        bc[d] = a.next_counts ? brick_coord(g, a.b, xn, d) : 0;
      }
      if (a.ids_out) a.ids_out[p] = a.ids_in[p];
      if (!ok) flag_status(a.status, PS_DEV_NONFINITE_POS, p);
      if (a.next_counts) {
        // the next step's counting, one atomic per particle (this loop's
        // lanes leave it at different trips)
        int key = bin_of_coords(a.b, bc[0], bc[1], bc[2]);
        if (key < 0) {
          flag_status(a.status, PS_DEV_NONFINITE_POS, p);
          key = 0;
        }
        a.next_bin[p] = key;
        atomicAdd(&a.next_counts[key], 1);
      }
    }
  }
}

// ------------------------------------------------------------------ host ----

template <typename F>
ps_status with_coef_type(ps_dtype t, F&& f) {
  switch (t) {
    case PS_F32: return f(float{});
    case PS_F64: return f(double{});
    case PS_BF16: return f(__nv_bfloat16{});
    case PS_F16: return f(__half{});
    case PS_F32X4: return f(float4{});
    case PS_BF16X4: return f(bf16x4{});
    case PS_F16X4: return f(f16x4{});
  }
  return fail(PS_ERR_INVALID_ARG, "bad coefficient dtype %d", (int)t);
}

ps_status check_coef(ps_dtype coef_t, const void* coef, const float* scale) {
  if (coef_t != PS_F32 && coef_t != PS_F64 && coef_t != PS_BF16 && coef_t != PS_F16 &&
      coef_t != PS_F32X4 && coef_t != PS_BF16X4 && coef_t != PS_F16X4)
    return fail(PS_ERR_INVALID_ARG, "bad coefficient dtype %d", (int)coef_t);
  if (!coef) return fail(PS_ERR_INVALID_ARG, "coef is NULL");
  if ((coef_t == PS_BF16 || coef_t == PS_F16 || coef_t == PS_BF16X4 || coef_t == PS_F16X4) &&
      !scale)
    return fail(PS_ERR_INVALID_ARG, "scale required for BF16/F16 coefficients");
  return PS_OK;
}

unsigned quad_blocks(int64_t np) { return (unsigned)((np * 4 + 255) / 256); }

int plane_stride(int sx, int sy) {
  int ps = sx * sy;
  while ((ps & 7) != 4) ++ps;
  return ps;
}

ps_status fill_staged(const ps_grid* grid, ps_dtype coef_t, const int32_t brick[3], int E,
                      bool grad, StagedArgs* a, size_t* smem) {
  ps_status rc = make_brick_args(grid, brick, &a->b);
  if (rc) return rc;
  a->g = make_grid_args(grid, coef_t);
  a->E = E;
  for (int d = 0; d < 3; ++d) {
    a->S[d] = a->b.B[d] + 3 + 2 * E;
    const int B = a->b.B[d];
    a->bshift[d] = (B & (B - 1)) ? -1 : __builtin_ctz((unsigned)B);
    const double xg = 1073741824.0 / a->g.inv_h[d];  // 2^30 cells
    int64_t bits;
    memcpy(&bits, &xg, sizeof(bits));
    a->xguard_hi[d] = (int)(bits >> 32);
  }
  if (a->S[0] > 32) return fail(PS_ERR_UNSUPPORTED, "brick x extent above 29 cells");
  a->SX = a->S[0];
  a->PS = plane_stride(a->SX, a->S[1]);
  // vector staging needs E = 0, bricks tiling the grid, 16-byte-aligned halo
  // rows and the last row vector inside the row pitch
  const int V = coef_t == PS_F32 ? 4 : (coef_t == PS_BF16 || coef_t == PS_F16 ? 8 : 0);
  bool vec = E == 0 && V > 0 && a->b.B[0] % V == 0;
  for (int d = 0; d < 3; ++d) vec = vec && grid->n[d] % a->b.B[d] == 0;
  const int qx = (a->S[0] + V - 1) / (V > 0 ? V : 1);
  vec = vec && qx <= 4 && (a->b.nb[0] - 1) * a->b.B[0] + qx * V <= a->g.rx;
  if (coef_t == PS_F32X4 || coef_t == PS_BF16X4 || coef_t == PS_F16X4) {
    // node rows: any x offset is a whole node; the halo stays inside
    // the padded array when the bricks tile the grid
    vec = E == 0;
    for (int d = 0; d < 3; ++d) vec = vec && grid->n[d] % a->b.B[d] == 0;
    // rows padded so that a plane is 4 (mod 8) nodes long: the layout a
    // tensor copy of the halo box produces, conflict-free for the gathers
    for (int sx = a->S[0]; vec && sx < a->S[0] + 8; ++sx)
      if ((sx * a->S[1]) % 8 == 4) {
        a->SX = sx;
        a->PS = sx * a->S[1];
        break;
      }
  }
  a->vec = vec ? 1 : 0;
  a->tma = 0;
  a->min_stage = tuning().brick_min_stage;
  a->wait_probe = tuning().wait_probe;
  // (tensor copies of 16-bit nodes land inside the float4 halo's buffer)
  *smem = (size_t)a->S[2] * a->PS * sizeof(float4) + rec_bytes(grad);
  if (*smem > 227 * 1024) return fail(PS_ERR_UNSUPPORTED, "brick halo exceeds shared memory");
  return PS_OK;
}

}  // namespace

// Tensor map of the node halo box (4 floats x SX nodes x S[1] rows x S[2]
// planes) over the PS_F32X4 array; the driver's encoder is looked up once.
bool encode_node_halo_map(StagedArgs* a, ps_dtype coef_t) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static bool looked = false;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!looked) {
      looked = true;
      cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
      void* fn = nullptr;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                           &q) == cudaSuccess &&
          q == cudaDriverEntryPointSuccess)
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
      else
        cudaGetLastError();
    }
  }
  if (!encode) return false;
  const GridArgs& g = a->g;
  const cuuint32_t unit[4] = {1, 1, 1, 1};
  const cuuint64_t m1 = (cuuint64_t)g.m[1], m2 = (cuuint64_t)g.m[2], rx = (cuuint64_t)g.rx;
  if (coef_t == PS_F32X4) {
    const cuuint64_t dims[4] = {4, rx, m1, m2};
    const cuuint64_t strides[3] = {16, rx * 16, rx * m1 * 16};
    const cuuint32_t box[4] = {4, (cuuint32_t)a->SX, (cuuint32_t)a->S[1], (cuuint32_t)a->S[2]};
    return encode(&a->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(a->coef),
                  dims, strides, box, unit, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  // 16-bit nodes: pairs of nodes (16 bytes) are the inner unit; rx is even
  const cuuint64_t dims[4] = {8, rx / 2, m1, m2};
  const cuuint64_t strides[3] = {16, rx * 8, rx * m1 * 8};
  const cuuint32_t box[4] = {8, (cuuint32_t)a->SX / 2, (cuuint32_t)a->S[1],
                             (cuuint32_t)a->S[2]};
  const CUtensorMapDataType t =
      coef_t == PS_BF16X4 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  if (encode(&a->tmap, t, 4, const_cast<void*>(a->coef), dims, strides, box, unit,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  // the rows' scales (s_u, s_v, s_w, 1): [m2][m1][4] floats
  const cuuint64_t sdims[3] = {4, m1, m2};
  const cuuint64_t sstrides[2] = {16, m1 * 16};
  const cuuint32_t sbox[3] = {4, (cuuint32_t)a->S[1], (cuuint32_t)a->S[2]};
  return encode(&a->tmap2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(a->scale),
                sdims, sstrides, sbox, unit, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// Use a tensor copy for the halo when the coefficients are nodes, the halo
// rows fit the copy layout and the array is 16-byte aligned.
void attach_tma(StagedArgs* a, ps_dtype coef_t) {
  a->tma = 0;
  const bool n16 = coef_t == PS_BF16X4 || coef_t == PS_F16X4;
  if ((coef_t != PS_F32X4 && !n16) || !a->vec || !tuning().node_tma) return;
  if ((a->SX * a->S[1]) % 8 != 4 || a->SX > 256 || a->S[1] > 256 || a->S[2] > 256) return;
  if (!a->coef || (reinterpret_cast<uintptr_t>(a->coef) & 15)) return;
  if (n16 && ((a->SX & 1) || (a->b.B[0] & 1) || (a->g.rx & 1) || !a->scale ||
              (reinterpret_cast<uintptr_t>(a->scale) & 15)))
    return;
  a->tma = encode_node_halo_map(a, coef_t) ? 1 : 0;
}

template <typename Tc> struct DtypeOf { static constexpr int v = -1; };
template <> struct DtypeOf<float> { static constexpr int v = PS_F32; };
template <> struct DtypeOf<float4> { static constexpr int v = PS_F32X4; };
template <> struct DtypeOf<__nv_bfloat16> { static constexpr int v = PS_BF16; };
template <> struct DtypeOf<__half> { static constexpr int v = PS_F16; };
template <> struct DtypeOf<bf16x4> { static constexpr int v = PS_BF16X4; };
template <> struct DtypeOf<f16x4> { static constexpr int v = PS_F16X4; };

template <typename Tc, int NC, int MODE>
ps_status launch_staged(const StagedArgs& a, size_t smem, cudaStream_t st) {
  // brick_kernel -1 (default): the measured-faster form per case, the quad
  // kernel for the gradient tensor and for 16-bit coefficients (planar ones
  // too, so that both storages of the same values give the same bits), the
  // phased kernel otherwise
  int k = tuning().brick_kernel;
  if (k < 0) k = (MODE == 1 || IsQuant<Tc>::value) ? 5 : 0;
  if constexpr (NC == 3 && DtypeOf<Tc>::v >= 0) {
    if (k == 5) {
      bool done = false;
      ps_status rc = launch_quad(a, (ps_dtype)DtypeOf<Tc>::v, MODE, st, &done);
      if (rc || done) return rc;
    }
  }
  if (k == 2) {
    auto tk = interp_thread<Tc, NC, MODE>;
    const size_t hs = (size_t)a.S[2] * a.PS * sizeof(float4);
    if (hs > 48 * 1024) {
      ps_status rc = check_cuda(
          cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs),
          "thread-kernel smem attribute");
      if (rc) return rc;
    }
    tk<<<(unsigned)a.b.nbins, 64, hs, st>>>(a);
    return check_launch("interp_thread");
  }
  auto kern = interp_staged<Tc, NC, MODE>;
  if (smem > 48 * 1024) {
    ps_status rc = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "staged smem attribute");
    if (rc) return rc;
  }
  if (a.b.nbins > 0x7fffffff) return fail(PS_ERR_UNSUPPORTED, "too many bins");
  kern<<<(unsigned)a.b.nbins, kThreads, smem, st>>>(a);
  return check_launch("interp_staged");
}

float3 dt_over_h(const GridArgs& g, double dt) {
  return make_float3((float)(dt * g.inv_h[0]), (float)(dt * g.inv_h[1]),
                     (float)(dt * g.inv_h[2]));
}

}  // namespace

// ---------------------------------------------------------------- batch ----
// Helpers of the many-field form (batch.cu); StagedArgs stays private to this
// file and travels as opaque bytes.

size_t staged_args_size() { return sizeof(StagedArgs); }

// Arguments of one field's fused Heun step inside a batch: positions are the
// concatenated [3][np_total] arrays, offs points at the field's first bin.
ps_status staged_fill_rk2(const ps_grid* grid, ps_dtype coef_t, const int32_t brick[3],
                          const void* coef, const float* scale, int64_t np_total,
                          const double* pos_in, double* pos_out, const int32_t* offs,
                          float* vel, const int64_t* ids_in, int64_t* ids_out, double dt,
                          int32_t* status, int chunked, int32_t* next_counts, int32_t* next_bin,
                          int next_key_base, int next_runs, void* out, size_t* smem) {
  if (coef_t == PS_F64) return fail(PS_ERR_UNSUPPORTED, "batched RK2 needs F32/BF16/F16");
  StagedArgs a{};
  ps_status rc = fill_staged(grid, coef_t, brick, 0, false, &a, smem);
  if (rc) return rc;
  a.coef = coef;
  a.scale = scale;
  attach_tma(&a, coef_t);
  a.np = np_total;
  a.pos_in = pos_in;
  a.pos_out = pos_out;
  a.offs = offs;
  a.vel = vel;
  a.ids_in = ids_in;
  a.ids_out = ids_out;
  a.dt = dt;
  const float3 d = dt_over_h(a.g, dt);
  a.dtih[0] = d.x;
  a.dtih[1] = d.y;
  a.dtih[2] = d.z;
  a.status = status;
  a.chunked = chunked;
  a.next_counts = next_counts;
  a.next_bin = next_bin;
  a.next_key_base = next_key_base;
  a.next_runs = next_runs;
  memcpy(out, &a, sizeof(a));
  return PS_OK;
}

// Launch the batched fused Heun step over total_bins bricks of nfields
// fields.  Set prepare = true once before any stream capture (it only sets the
// shared-memory limit of the kernel).
ps_status staged_batch_launch(ps_dtype coef_t, const void* d_tab, const int* d_bin_base,
                              const void* h_tab, const int* h_bin_base, int nfields,
                              int64_t total_bins, size_t smem, bool prepare, cudaStream_t st) {
  return with_coef_type(coef_t, [&](auto tag) -> ps_status {
    using Tc = decltype(tag);
    if constexpr (std::is_same<Tc, double>::value) {
      return fail(PS_ERR_UNSUPPORTED, "batched RK2 needs F32/BF16/F16");
    } else {
      auto kern = interp_staged_batch<Tc, 3, 2>;
      auto kern_p = interp_staged_batch_p<Tc, 3, 2>;
      if (prepare) {
        ps_status rc = PS_OK;
        if (smem > 48 * 1024) {
          rc = check_cuda(
              cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
              "batch smem attribute");
          if (!rc)
            rc = check_cuda(cudaFuncSetAttribute(
                                kern_p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                            "batch smem attribute");
        }
        return rc;
      }
      if (total_bins <= 0) return PS_OK;
      if (h_tab && h_bin_base && nfields <= kParamFields) {
        // the table by value (a graph captures it with the launch)
        BatchParams tab;
        memcpy(tab.a, h_tab, (size_t)nfields * sizeof(StagedArgs));
        memcpy(tab.bin_base, h_bin_base, (size_t)(nfields + 1) * sizeof(int));
        tab.nfields = nfields;
        kern_p<<<(unsigned)total_bins, kThreads, smem, st>>>(tab);
        return check_launch("interp_staged_batch_p");
      }
      kern<<<(unsigned)total_bins, kThreads, smem, st>>>(
          static_cast<const StagedArgs*>(d_tab), d_bin_base, nfields);
      return check_launch("interp_staged_batch");
    }
  });
}

// All nsteps Heun steps of a batch in one cooperative launch (batch_persistent):
// a grid of every block the device holds at once.  counts and sync must be
// zero at launch (the caller clears them on the same stream).
ps_status staged_batch_persistent(ps_dtype coef_t, const void* d_tab, const int* d_bin_base,
                                  const BinField* d_bintab, int nfields, int64_t total_bins,
                                  int64_t np, int nsteps, double* pos, int64_t* ids,
                                  double* pos_s, int64_t* ids_s, int32_t* bin_of, int32_t* rank,
                                  int32_t* counts, int32_t* offsets, int32_t* scan_tmp,
                                  int32_t* status, unsigned* sync, size_t smem,
                                  cudaStream_t st) {
  return with_coef_type(coef_t, [&](auto tag) -> ps_status {
    using Tc = decltype(tag);
    if constexpr (std::is_same<Tc, double>::value) {
      return fail(PS_ERR_UNSUPPORTED, "batched RK2 needs F32/BF16/F16");
    } else {
      auto kern = batch_persistent<Tc>;
      if (smem > 48 * 1024) {
        ps_status rc = check_cuda(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "persistent batch smem attribute");
        if (rc) return rc;
      }
      int per_sm = 0;
      ps_status rc = check_cuda(
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem),
          "persistent batch occupancy");
      if (rc) return rc;
      if (per_sm < 1) return fail(PS_ERR_UNSUPPORTED, "persistent batch kernel does not fit an SM");
      BatchRun r;
      r.tab = static_cast<const StagedArgs*>(d_tab);
      r.bin_base = d_bin_base;
      r.bintab = d_bintab;
      r.nfields = nfields;
      r.nsteps = nsteps;
      r.total_bins = total_bins;
      r.np = np;
      r.pos = pos;
      r.ids = ids;
      r.pos_s = pos_s;
      r.ids_s = ids_s;
      r.bin_of = bin_of;
      r.rank = rank;
      r.counts = counts;
      r.offsets = offsets;
      r.scan_tmp = scan_tmp;
      r.status = status;
      r.sync = sync;
      r.wait_probe = tuning().wait_probe;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(per_sm * sm_count()));
      cfg.blockDim = dim3(kThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return check_cuda(cudaLaunchKernelEx(&cfg, kern, r), "persistent batch launch");
    }
  });
}

// RK2 kernels used by ps_rk2_step (rk2.cu).
ps_status rk2_launch_direct(const ps_grid* grid, ps_dtype coef_t, const void* c0,
                            const float* s0, const void* c1, const float* s1, int64_t np,
                            double* pos, float* vel_out, double dt, int32_t* status,
                            cudaStream_t st) {
  GridArgs g = make_grid_args(grid, coef_t);
  const float3 dtih = dt_over_h(g, dt);
  return with_coef_type(coef_t, [&](auto tag) -> ps_status {
    using Tc = decltype(tag);
    rk2_direct<Tc><<<quad_blocks(np), 256, 0, st>>>(g, static_cast<const Tc*>(c0), s0,
                                                    static_cast<const Tc*>(c1), s1, np, pos,
                                                    vel_out, dt, dtih, status);
    return check_launch("rk2_direct");
  });
}

ps_status rk2_launch_staged(const ps_grid* grid, const int32_t brick[3], int E,
                            ps_dtype coef_t, const void* c0, const float* s0,
                            const void* c1, const float* s1, int64_t np,
                            const double* pos_in, double* pos_out, const int32_t* offs,
                            float* vel_out, const int64_t* ids_in, int64_t* ids_out,
                            double dt, int32_t* status, int32_t* next_counts,
                            int32_t* next_bin, cudaStream_t st) {
  if (coef_t == PS_F64)
    return fail(PS_ERR_UNSUPPORTED, "staged RK2 needs F32/BF16/F16 coefficients");
  StagedArgs a{};
  size_t smem;
  ps_status rc = fill_staged(grid, coef_t, brick, E, false, &a, &smem);
  if (rc) return rc;
  a.coef = c0;
  a.scale = s0;
  a.coef2 = c1;
  a.scale2 = s1;
  attach_tma(&a, coef_t);
  a.np = np;
  a.pos_in = pos_in;
  a.pos_out = pos_out;
  a.offs = offs;
  a.vel = vel_out;
  a.ids_in = ids_in;
  a.ids_out = ids_out;
  a.dt = dt;
  const float3 d = dt_over_h(a.g, dt);
  a.dtih[0] = d.x;
  a.dtih[1] = d.y;
  a.dtih[2] = d.z;
  a.status = status;
  a.next_counts = next_counts;
  a.next_bin = next_bin;
  return with_coef_type(coef_t, [&](auto tag) -> ps_status {
    using Tc = decltype(tag);
    if constexpr (std::is_same<Tc, double>::value) return PS_ERR_UNSUPPORTED;
    else return launch_staged<Tc, 3, 2>(a, smem, st);
  });
}

}  // namespace ps

using namespace ps;

extern "C" ps_status ps_interp(const ps_grid* grid, int ncomp, ps_dtype coef_t,
                               const void* coef, const float* scale, int64_t np,
                               const double* pos, const int64_t* perm,
                               const int32_t* bin_offsets, const int32_t brick[3],
                               float* vel, float* grad, int32_t* status, void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  if (ncomp != 1 && ncomp != 3) return fail(PS_ERR_INVALID_ARG, "ncomp must be 1 or 3");
  if ((coef_t == PS_F32X4 || coef_t == PS_BF16X4 || coef_t == PS_F16X4) && ncomp != 3)
    return fail(PS_ERR_INVALID_ARG, "node coefficients need ncomp == 3");
  if ((rc = check_coef(coef_t, coef, scale))) return rc;
  if (np < 0) return fail(PS_ERR_INVALID_ARG, "np < 0");
  if (np == 0) return PS_OK;
  if (!pos || !vel) return fail(PS_ERR_INVALID_ARG, "pos and vel are required");
  if (perm && !bin_offsets) return fail(PS_ERR_INVALID_ARG, "perm needs bin_offsets");
  if (bin_offsets && !brick) return fail(PS_ERR_INVALID_ARG, "bin_offsets needs brick");
  cudaStream_t st = as_stream(stream);
  GridArgs g = make_grid_args(grid, coef_t);
  const bool staged = bin_offsets && coef_t != PS_F64;
  if (!staged) {
    return with_coef_type(coef_t, [&](auto tag) -> ps_status {
      using Tc = decltype(tag);
      const Tc* c = static_cast<const Tc*>(coef);
      if (ncomp == 3) {
        if (grad)
          interp_direct<Tc, 3, 1><<<quad_blocks(np), 256, 0, st>>>(
              g, c, scale, np, pos, perm, vel, grad, nullptr, nullptr, status);
        else
          interp_direct<Tc, 3, 0><<<quad_blocks(np), 256, 0, st>>>(
              g, c, scale, np, pos, perm, vel, nullptr, nullptr, nullptr, status);
      } else {
        if (grad)
          interp_direct<Tc, 1, 1><<<quad_blocks(np), 256, 0, st>>>(
              g, c, scale, np, pos, perm, vel, grad, nullptr, nullptr, status);
        else
          interp_direct<Tc, 1, 0><<<quad_blocks(np), 256, 0, st>>>(
              g, c, scale, np, pos, perm, vel, nullptr, nullptr, nullptr, status);
      }
      return check_launch("interp_direct");
    });
  }
  StagedArgs a{};
  size_t smem;
  if ((rc = fill_staged(grid, coef_t, brick, 0, grad != nullptr, &a, &smem))) return rc;
  a.coef = coef;
  a.scale = scale;
  attach_tma(&a, coef_t);
  a.np = np;
  a.pos_in = pos;
  a.perm = perm;
  a.offs = bin_offsets;
  a.vel = vel;
  a.grad = grad;
  a.status = status;
  return with_coef_type(coef_t, [&](auto tag) -> ps_status {
    using Tc = decltype(tag);
    if constexpr (std::is_same<Tc, double>::value) {
      return PS_ERR_UNSUPPORTED;
    } else {
      if (ncomp == 3)
        return grad ? launch_staged<Tc, 3, 1>(a, smem, st) : launch_staged<Tc, 3, 0>(a, smem, st);
      return grad ? launch_staged<Tc, 1, 1>(a, smem, st) : launch_staged<Tc, 1, 0>(a, smem, st);
    }
  });
}

extern "C" ps_status ps_interp_backward(const ps_grid* grid, int ncomp, ps_dtype coef_t,
                                        const void* coef, const float* scale, int64_t np,
                                        const double* pos, const float* g_vel,
                                        double* g_pos, float* g_field, void* ws,
                                        size_t ws_bytes, int32_t* status, void* stream) {
  (void)ws;
  (void)ws_bytes;
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  if (ncomp != 1 && ncomp != 3) return fail(PS_ERR_INVALID_ARG, "ncomp must be 1 or 3");
  if ((coef_t == PS_F32X4 || coef_t == PS_BF16X4 || coef_t == PS_F16X4) && ncomp != 3)
    return fail(PS_ERR_INVALID_ARG, "node coefficients need ncomp == 3");
  if (np < 0) return fail(PS_ERR_INVALID_ARG, "np < 0");
  if (np > 0 && (!pos || !g_vel)) return fail(PS_ERR_INVALID_ARG, "pos and g_vel required");
  cudaStream_t st = as_stream(stream);
  GridArgs g = make_grid_args(grid, coef_t);
  if (g_pos && np > 0) {
    if ((rc = check_coef(coef_t, coef, scale))) return rc;
    rc = with_coef_type(coef_t, [&](auto tag) -> ps_status {
      using Tc = decltype(tag);
      const Tc* c = static_cast<const Tc*>(coef);
      if (ncomp == 3)
        interp_direct<Tc, 3, 2><<<quad_blocks(np), 256, 0, st>>>(
            g, c, scale, np, pos, nullptr, nullptr, nullptr, g_vel, g_pos, status);
      else
        interp_direct<Tc, 1, 2><<<quad_blocks(np), 256, 0, st>>>(
            g, c, scale, np, pos, nullptr, nullptr, nullptr, g_vel, g_pos, status);
      return check_launch("interp_backward_pos");
    });
    if (rc) return rc;
  }
  if (g_field) {
    const int64_t vol = grid_volume(grid);
    rc = check_cuda(cudaMemsetAsync(g_field, 0, sizeof(float) * vol * ncomp, st),
                    "g_field memset");
    if (rc) return rc;
    if (np > 0) {
      if (ncomp == 3)
        scatter_field<3><<<quad_blocks(np), 256, 0, st>>>(g, np, pos, g_vel, g_field, status);
      else
        scatter_field<1><<<quad_blocks(np), 256, 0, st>>>(g, np, pos, g_vel, g_field, status);
      if ((rc = check_launch("scatter_field"))) return rc;
    }
    rc = solve_unpadded_inplace_f32(grid, ncomp, g_field, st);
    if (rc) return rc;
  }
  return PS_OK;
}

// Brick-staged form of the second derivatives (mode 3) or the Lagrangian
// acceleration (mode 4) by the quad kernel; *done false where it does not
// apply (the caller then gathers directly).
static ps_status staged_extra(const ps_grid* grid, ps_dtype coef_t, const void* coef,
                              const float* scale, const void* coef2, const float* scale2,
                              double inv_dt, int64_t np, const double* pos,
                              const int64_t* perm, const int32_t* bin_offsets,
                              const int32_t brick[3], float* out, float* vel, int32_t* status,
                              int mode, cudaStream_t st, bool* done) {
  *done = false;
  StagedArgs a{};
  size_t smem;
  ps_status rc = fill_staged(grid, coef_t, brick, 0, false, &a, &smem);
  if (rc) return rc;
  a.coef = coef;
  a.scale = scale;
  a.coef2 = coef2;
  a.scale2 = scale2;
  attach_tma(&a, coef_t);
  a.np = np;
  a.pos_in = pos;
  a.perm = perm;
  a.offs = bin_offsets;
  a.grad = out;
  a.vel = vel;
  a.dt = inv_dt;
  a.status = status;
  return launch_quad(a, coef_t, mode, st, done);
}

extern "C" ps_status ps_interp_hessian(const ps_grid* grid, int ncomp, ps_dtype coef_t,
                                       const void* coef, const float* scale, int64_t np,
                                       const double* pos, const int64_t* perm,
                                       const int32_t* bin_offsets, const int32_t brick[3],
                                       float* hess, int32_t* status, void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  if (ncomp != 1 && ncomp != 3) return fail(PS_ERR_INVALID_ARG, "ncomp must be 1 or 3");
  if ((coef_t == PS_F32X4 || coef_t == PS_BF16X4 || coef_t == PS_F16X4) && ncomp != 3)
    return fail(PS_ERR_INVALID_ARG, "node coefficients need ncomp == 3");
  if ((rc = check_coef(coef_t, coef, scale))) return rc;
  if (np < 0) return fail(PS_ERR_INVALID_ARG, "np < 0");
  if (np == 0) return PS_OK;
  if (!pos || !hess) return fail(PS_ERR_INVALID_ARG, "pos and hess are required");
  if (perm && !bin_offsets) return fail(PS_ERR_INVALID_ARG, "perm needs bin_offsets");
  if (bin_offsets && !brick) return fail(PS_ERR_INVALID_ARG, "bin_offsets needs brick");
  cudaStream_t st = as_stream(stream);
  if (bin_offsets && ncomp == 3 && coef_t != PS_F64) {
    bool done = false;
    rc = staged_extra(grid, coef_t, coef, scale, nullptr, nullptr, 0.0, np, pos, perm,
                      bin_offsets, brick, hess, nullptr, status, 3, st, &done);
    if (rc || done) return rc;
  }
  GridArgs g = make_grid_args(grid, coef_t);
  return with_coef_type(coef_t, [&](auto tag) -> ps_status {
    using Tc = decltype(tag);
    const Tc* c = static_cast<const Tc*>(coef);
    if (ncomp == 3)
      interp_hessian_direct<Tc, 3><<<quad_blocks(np), 256, 0, st>>>(g, c, scale, np, pos, hess,
                                                                     status);
    else
      interp_hessian_direct<Tc, 1><<<quad_blocks(np), 256, 0, st>>>(g, c, scale, np, pos, hess,
                                                                     status);
    return check_launch("interp_hessian_direct");
  });
}

extern "C" ps_status ps_lagrangian_accel(const ps_grid* grid, ps_dtype coef_t,
                                         const void* coef_n, const float* scale_n,
                                         const void* coef_np1, const float* scale_np1,
                                         double dt_field, int64_t np, const double* pos,
                                         const int64_t* perm, const int32_t* bin_offsets,
                                         const int32_t brick[3], float* acc, float* vel,
                                         int32_t* status, void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  if ((rc = check_coef(coef_t, coef_n, scale_n))) return rc;
  if (coef_np1 && (rc = check_coef(coef_t, coef_np1, scale_np1))) return rc;
  if (coef_np1 && !(dt_field > 0.0 && std::isfinite(dt_field)))
    return fail(PS_ERR_INVALID_ARG, "dt_field must be finite and > 0");
  if (np < 0) return fail(PS_ERR_INVALID_ARG, "np < 0");
  if (np == 0) return PS_OK;
  if (!pos || !acc) return fail(PS_ERR_INVALID_ARG, "pos and acc are required");
  if (perm && !bin_offsets) return fail(PS_ERR_INVALID_ARG, "perm needs bin_offsets");
  if (bin_offsets && !brick) return fail(PS_ERR_INVALID_ARG, "bin_offsets needs brick");
  cudaStream_t st = as_stream(stream);
  const double inv_dt = coef_np1 ? 1.0 / dt_field : 0.0;
  if (bin_offsets && coef_t != PS_F64) {
    bool done = false;
    rc = staged_extra(grid, coef_t, coef_n, scale_n, coef_np1, scale_np1, inv_dt, np, pos, perm,
                      bin_offsets, brick, acc, vel, status, 4, st, &done);
    if (rc || done) return rc;
  }
  GridArgs g = make_grid_args(grid, coef_t);
  return with_coef_type(coef_t, [&](auto tag) -> ps_status {
    using Tc = decltype(tag);
    lagrangian_accel_direct<Tc><<<quad_blocks(np), 256, 0, st>>>(
        g, static_cast<const Tc*>(coef_n), scale_n, static_cast<const Tc*>(coef_np1), scale_np1,
        inv_dt, np, pos, acc, vel, status);
    return check_launch("lagrangian_accel_direct");
  });
}
