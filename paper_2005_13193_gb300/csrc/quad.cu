// Brick-staged interpolation (Sec. 2.2, Operations 2 and 3) and the fused
// second-order Runge-Kutta particle advance (Sec. 2.1, Sec. 4.3) with a quad
// of lanes per particle ("brick_kernel" 5).
//
// One thread block per brick of cells.  The brick's coefficient halo (the
// union of the stencils of its cells, (B+3)^3 nodes) is brought into shared
// memory as float4 (u, v, w, 0) per node by one tensor copy (node
// coefficients) or by plain loads (planar coefficients); rows of SX nodes and
// planes of PS nodes with PS = 2 or 6 (mod 8).
//
//  A  one thread per particle: exact FP64 location of all three axes, the
//     fractions, the brick-local stencil start; the record is appended to one
//     of two lists by the parity of the stencil's first 16-byte bank group.
//  B  a quad of lanes per particle, lane k owning stencil z-row k (16 nodes
//     held in registers): the 16-term (y, x) sum in the lane, the z sum over
//     the quad.  The four lanes of a quad read four distinct bank groups of
//     one parity (k PS = 0, 2, 4, 6 mod 8); the two quads of an 8-lane load
//     phase take particles from opposite lists, so their groups do not meet.
//     Heun step: the predictor is located in FP32 from the stage-1 cell; when
//     it stays in that cell (most particles at Courant numbers well below one)
//     the second sum reuses the stencil held in registers, otherwise the quad
//     reloads it.  The FP64 update, the velocity and the next step's bin
//     count follow in the same quad; no block barrier after phase A.
//
// Particles whose stencil is not inside the staged halo (stale bins, a
// predictor that left the brick, bricks below the staging threshold, a halo
// copy that did not complete in time) read their nodes from global memory,
// so results never depend on the bins being fresh.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "staged.cuh"

namespace ps {
namespace {

constexpr int kQT = 128;  // threads per block = particles per round

// Halo geometry.  CT > 0: the compile-time 8^3 brick (11 nodes per axis) with
// rows of CT nodes (14 for float4 nodes: planes of 154 = 2 mod 8 nodes; 12 for
// 16-bit nodes: planes of 132 = 4 mod 16 nodes); CT = 0 reads the launch
// arguments.
template <int CT> struct QGeo {
  static constexpr int Sx = 11, Sy = 11, Sz = 11, SX = CT, PS = CT * 11;
  __device__ __forceinline__ explicit QGeo(const StagedArgs&) {}
};
template <> struct QGeo<0> {
  int Sx, Sy, Sz, SX, PS;
  __device__ __forceinline__ explicit QGeo(const StagedArgs& a)
      : Sx(a.S[0]), Sy(a.S[1]), Sz(a.S[2]), SX(a.SX), PS(a.PS) {}
};

// Per-round particle records, filled by phase A, read by the quads:
//   rt[s]  (t_x, t_y, t_z, w)  fractions; w = local stencil start (bytes 0-2)
//                              and bit 24 = stencil inside the staged halo
//   rc[s]  (cell_x, cell_y, cell_z, r | nonfinite << 30), r = round index
//   x[d * kQT + r]             FP64 coordinate (Heun step)
// Slots of the even-parity list grow from 0, those of the odd one from
// kQT - 1 down.
__host__ __device__ constexpr size_t qrec_bytes() {
  return (size_t)kQT * (sizeof(float4) + sizeof(int4) + 3 * sizeof(double));
}

// Halo region of a brick in float4 units: float4 nodes, or 16-bit nodes
// followed (at a 128-byte boundary) by the rows' float4 scales.
template <typename Tc>
__host__ __device__ constexpr int halo_f4(int Sz, int Sy, int PS) {
  return IsNode16<Tc>::value ? (((Sz * PS * 8 + 127) & ~127) + Sz * Sy * 16 + 15) / 16
                             : Sz * PS;
}
template <typename Tc>
__host__ __device__ constexpr int scale_off_bytes(int Sz, int PS) {
  return (Sz * PS * 8 + 127) & ~127;
}

// Slot of position s in the interleaved order even, odd, even, odd, ...
// (then the rest of the longer list).
__device__ __forceinline__ int quad_slot(int s, int ne, int no) {
  const int nm = min(ne, no);
  if (s < 2 * nm) return (s & 1) ? kQT - 1 - (s >> 1) : (s >> 1);
  const int r = nm + (s - 2 * nm);
  return ne >= no ? r : kQT - 1 - r;
}

// The 16 nodes (j, i) of z-row k of a stencil: from the staged halo when
// `inh` (local start l), else from global memory (padded start = cell).  A
// 16-bit node halo holds the raw nodes (8 bytes each) and, in `scl`, the
// (s_u, s_v, s_w, 1) scale of every halo row; each value is widened and
// multiplied by its row's power-of-two scale (exact) as it is read.
template <typename Tc, int CT>
__device__ __forceinline__ void quad_fetch(float v[16][3], bool inh, const int l[3],
                                           const int cell[3], int k, const float4* halo,
                                           const float4* scl, const QGeo<CT>& geo,
                                           const GridArgs& g, const Tc* __restrict__ coef,
                                           const float* __restrict__ scale) {
  if constexpr (IsNode16<Tc>::value) {
    if (inh) {
      const Tc* hp = reinterpret_cast<const Tc*>(halo) + (l[2] + k) * geo.PS + l[1] * geo.SX + l[0];
      const float4* sp = scl + (l[2] + k) * geo.Sy + l[1];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 sc = sp[j];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const Tc n = hp[j * geo.SX + i];
          v[4 * j + i][0] = __fmul_rn(node16_value(n.v[0]), sc.x);
          v[4 * j + i][1] = __fmul_rn(node16_value(n.v[1]), sc.y);
          v[4 * j + i][2] = __fmul_rn(node16_value(n.v[2]), sc.z);
        }
      }
      return;
    }
  }
  if (inh) {
    const float4* hp = halo + (l[2] + k) * geo.PS + l[1] * geo.SX + l[0];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 q = hp[j * geo.SX + i];
        v[4 * j + i][0] = q.x;
        v[4 * j + i][1] = q.y;
        v[4 * j + i][2] = q.z;
      }
  } else {
    const int Pz = cell[2] + k;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if constexpr (IsNode4<Tc>::value && !IsNode16<Tc>::value) {
          const int64_t node = ((int64_t)Pz * g.m[1] + cell[1] + j) * g.rx + cell[0] + i;
          const float4 q = __ldg(reinterpret_cast<const float4*>(coef) + node);
          v[4 * j + i][0] = q.x;
          v[4 * j + i][1] = q.y;
          v[4 * j + i][2] = q.z;
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c)
            v[4 * j + i][c] =
                (float)load_coef<Tc>(coef, scale, g, c, Pz, cell[1] + j, cell[0] + i);
        }
      }
  }
}

// Uniform cubic B-spline weights (Sec. 2.2, Operation 2) and their
// derivatives with every rounding explicit, so that each instantiation of the
// kernels below evaluates them identically.
__device__ __forceinline__ void qbasis(float t, float b[4]) {
  const float s = __fsub_rn(1.f, t);
  const float t2 = __fmul_rn(t, t), t3 = __fmul_rn(t2, t);
  const float sixth = 1.f / 6.f;
  b[0] = __fmul_rn(__fmul_rn(__fmul_rn(s, s), s), sixth);
  b[1] = __fmul_rn(__fmaf_rn(3.f, t3, __fmaf_rn(-6.f, t2, 4.f)), sixth);
  b[2] = __fmul_rn(__fmaf_rn(-3.f, t3, __fmaf_rn(3.f, t2, __fmaf_rn(3.f, t, 1.f))), sixth);
  b[3] = __fmul_rn(t3, sixth);
}
__device__ __forceinline__ void qdbasis(float t, float d[4]) {
  const float s = __fsub_rn(1.f, t);
  const float tt = __fmul_rn(t, t);
  d[0] = __fmul_rn(__fmul_rn(s, s), -0.5f);
  d[1] = __fmul_rn(__fmaf_rn(3.f, tt, __fmul_rn(-4.f, t)), 0.5f);
  d[2] = __fmul_rn(__fmaf_rn(-3.f, tt, __fmaf_rn(2.f, t, 1.f)), 0.5f);
  d[3] = __fmul_rn(tt, 0.5f);
}

// d2 b / dt2 of the same basis (piecewise linear: the spline is twice
// continuously differentiable, Sec. 2.2).
__device__ __forceinline__ void qddbasis(float t, float d[4]) {
  d[0] = __fsub_rn(1.f, t);
  d[1] = __fmaf_rn(3.f, t, -2.f);
  d[2] = __fmaf_rn(-3.f, t, 1.f);
  d[3] = t;
}

// The six second derivatives (in cells^-2) of the three components at
// (t_x, t_y, t_z): out[e][c], e = xx, yy, zz, xy, xz, yz; every lane of the
// quad returns them (the same bits).
__device__ __forceinline__ void quad_sum_hess(const float v[16][3], const float t[3], int k,
                                              float out[6][3]) {
  float bx[4], by[4], dbx[4], dby[4], ddbx[4], ddby[4], z4[4];
  qbasis(t[0], bx);
  qbasis(t[1], by);
  qdbasis(t[0], dbx);
  qdbasis(t[1], dby);
  qddbasis(t[0], ddbx);
  qddbasis(t[1], ddby);
  qbasis(t[2], z4);
  const float bz = pick4(z4, k);
  qdbasis(t[2], z4);
  const float dbz = pick4(z4, k);
  qddbasis(t[2], z4);
  const float ddbz = pick4(z4, k);
  // y sums of the x sums: A = by s0, Bx = by s1, By = dby s0, Cxx = by s2,
  // Cyy = ddby s0, Cxy = dby s1 (s0, s1, s2: x sums with b, b', b'')
  float A[3] = {0.f, 0.f, 0.f}, Bx[3] = {0.f, 0.f, 0.f}, By[3] = {0.f, 0.f, 0.f};
  float Cxx[3] = {0.f, 0.f, 0.f}, Cyy[3] = {0.f, 0.f, 0.f}, Cxy[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s0 = __fmul_rn(bx[0], v[4 * j][c]), s1 = __fmul_rn(dbx[0], v[4 * j][c]),
            s2 = __fmul_rn(ddbx[0], v[4 * j][c]);
#pragma unroll
      for (int i = 1; i < 4; ++i) {
        s0 = __fmaf_rn(bx[i], v[4 * j + i][c], s0);
        s1 = __fmaf_rn(dbx[i], v[4 * j + i][c], s1);
        s2 = __fmaf_rn(ddbx[i], v[4 * j + i][c], s2);
      }
      A[c] = __fmaf_rn(by[j], s0, A[c]);
      Bx[c] = __fmaf_rn(by[j], s1, Bx[c]);
      By[c] = __fmaf_rn(dby[j], s0, By[c]);
      Cxx[c] = __fmaf_rn(by[j], s2, Cxx[c]);
      Cyy[c] = __fmaf_rn(ddby[j], s0, Cyy[c]);
      Cxy[c] = __fmaf_rn(dby[j], s1, Cxy[c]);
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    out[0][c] = __fmul_rn(bz, Cxx[c]);
    out[1][c] = __fmul_rn(bz, Cyy[c]);
    out[2][c] = __fmul_rn(ddbz, A[c]);
    out[3][c] = __fmul_rn(bz, Cxy[c]);
    out[4][c] = __fmul_rn(dbz, Bx[c]);
    out[5][c] = __fmul_rn(dbz, By[c]);
  }
#pragma unroll
  for (int e = 0; e < 6; ++e)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      out[e][c] = __fadd_rn(out[e][c], __shfl_xor_sync(FULL, out[e][c], 1));
      out[e][c] = __fadd_rn(out[e][c], __shfl_xor_sync(FULL, out[e][c], 2));
    }
}

// Sum of the quad's stencil with the basis at (t_x, t_y, t_z): every lane
// returns the three components, with the same bits in all four lanes (the
// products and the butterfly's sums are rounded explicitly).  GRAD also
// returns the three derivatives (in cells) per component: out[4][3] = value,
// d/dx, d/dy, d/dz.
template <bool GRAD>
__device__ __forceinline__ void quad_sum(const float v[16][3], const float t[3], int k,
                                         float out[4][3]) {
  float bx[4], by[4], bz4[4];
  qbasis(t[0], bx);
  qbasis(t[1], by);
  qbasis(t[2], bz4);
  const float bz = pick4(bz4, k);
  float dbx[4], dby[4], dbz = 0.f;
  if (GRAD) {
    float d4[4];
    qdbasis(t[0], dbx);
    qdbasis(t[1], dby);
    qdbasis(t[2], d4);
    dbz = pick4(d4, k);
  }
  float A[3] = {0.f, 0.f, 0.f}, Bx[3] = {0.f, 0.f, 0.f}, By[3] = {0.f, 0.f, 0.f};
  // u and v as packed pairs (two FP32 operations per instruction, each
  // rounded as its scalar form), w alone
  float2 A2 = make_float2(0.f, 0.f), Bx2 = A2, By2 = A2;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 vr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) vr[i] = make_float2(v[4 * j + i][0], v[4 * j + i][1]);
    float2 sx2 = __fmul2_rn(make_float2(bx[0], bx[0]), vr[0]);
#pragma unroll
    for (int i = 1; i < 4; ++i) sx2 = __ffma2_rn(make_float2(bx[i], bx[i]), vr[i], sx2);
    A2 = __ffma2_rn(make_float2(by[j], by[j]), sx2, A2);
    float sx = __fmul_rn(bx[0], v[4 * j][2]);
    sx = __fmaf_rn(bx[1], v[4 * j + 1][2], sx);
    sx = __fmaf_rn(bx[2], v[4 * j + 2][2], sx);
    sx = __fmaf_rn(bx[3], v[4 * j + 3][2], sx);
    A[2] = __fmaf_rn(by[j], sx, A[2]);
    if (GRAD) {
      float2 dx2 = __fmul2_rn(make_float2(dbx[0], dbx[0]), vr[0]);
#pragma unroll
      for (int i = 1; i < 4; ++i) dx2 = __ffma2_rn(make_float2(dbx[i], dbx[i]), vr[i], dx2);
      Bx2 = __ffma2_rn(make_float2(by[j], by[j]), dx2, Bx2);
      By2 = __ffma2_rn(make_float2(dby[j], dby[j]), sx2, By2);
      float dx = __fmul_rn(dbx[0], v[4 * j][2]);
      dx = __fmaf_rn(dbx[1], v[4 * j + 1][2], dx);
      dx = __fmaf_rn(dbx[2], v[4 * j + 2][2], dx);
      dx = __fmaf_rn(dbx[3], v[4 * j + 3][2], dx);
      Bx[2] = __fmaf_rn(by[j], dx, Bx[2]);
      By[2] = __fmaf_rn(dby[j], sx, By[2]);
    }
  }
  A[0] = A2.x;
  A[1] = A2.y;
  Bx[0] = Bx2.x;
  Bx[1] = Bx2.y;
  By[0] = By2.x;
  By[1] = By2.y;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    out[0][c] = __fmul_rn(bz, A[c]);
    if (GRAD) {
      out[1][c] = __fmul_rn(bz, Bx[c]);
      out[2][c] = __fmul_rn(bz, By[c]);
      out[3][c] = __fmul_rn(dbz, A[c]);
    }
  }
  // z sum over the quad (xor butterfly: every lane ends with the same bits)
#pragma unroll
  for (int r = 0; r < (GRAD ? 4 : 1); ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      out[r][c] = __fadd_rn(out[r][c], __shfl_xor_sync(FULL, out[r][c], 1));
      out[r][c] = __fadd_rn(out[r][c], __shfl_xor_sync(FULL, out[r][c], 2));
    }
}

// A round of up to kQT particles of one brick as the quads see it.
struct QStage {
  const float4* halo;
  const float4* scl; // row scales of a 16-bit node halo
  const float4* rt;  // records by slot
  const int4* rc;
  const double* x;   // FP64 coordinates [3][kQT] by round index
  int P0[3];
  int cb, m, bin, ne, no;
  bool staged;       // the halo holds the brick's nodes
};

// Phase A for the particle of round index r (thread r; `v` = it exists):
// exact location of the three axes from the FP64 coordinates x, the record
// appended to the even or the odd list by the parity of its stencil's first
// bank group.  cnt[0], cnt[1]: the two lists' sizes (shared counters).  All
// 32 lanes of the warp call.
template <int CT>
__device__ __forceinline__ void quad_locate(const StagedArgs& a, const QGeo<CT>& geo,
                                            const int P0[3], bool staged, int r, bool v,
                                            const double x[3], float4* rt, int4* rc,
                                            int* cnt) {
  const GridArgs& g = a.g;
  const int lane = threadIdx.x & 31;
  int cell[3] = {0, 0, 0};
  float t[3] = {0.f, 0.f, 0.f};
  bool ok = v;
  if (v) {
#pragma unroll
    for (int d = 0; d < 3; ++d) ok &= locate(x[d], g.inv_h[d], g.n[d], cell[d], t[d]);
  }
  const int S3[3] = {geo.Sx, geo.Sy, geo.Sz};
  int l[3];
  bool inh = staged && ok;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    l[d] = cell[d] - P0[d];
    inh = inh && (unsigned)l[d] <= (unsigned)(S3[d] - 4);
  }
  const bool odd = inh && ((l[0] + geo.SX * l[1]) & 1);
  const unsigned bo = __ballot_sync(FULL, v && odd), be = __ballot_sync(FULL, v && !odd);
  int base_e = 0, base_o = 0;
  if (lane == 0) {
    if (be) base_e = atomicAdd(&cnt[0], __popc(be));
    if (bo) base_o = atomicAdd(&cnt[1], __popc(bo));
  }
  base_e = __shfl_sync(FULL, base_e, 0);
  base_o = __shfl_sync(FULL, base_o, 0);
  const unsigned lt = (1u << lane) - 1u;
  const int slot = odd ? kQT - 1 - (base_o + __popc(bo & lt)) : base_e + __popc(be & lt);
  if (v) {
    const int w = inh ? (l[0] | (l[1] << 8) | (l[2] << 16) | (1 << 24)) : 0;
    rt[slot] = make_float4(t[0], t[1], t[2], __int_as_float(w));
    rc[slot] = make_int4(cell[0], cell[1], cell[2], r | (ok ? 0 : 1 << 30));
  }
}

// Phase B for chunk ch (eight particles) of a round, by one warp: quad
// (lane >> 2) takes position 8 ch + (lane >> 2) of the interleaved lists.
// MODE 0: velocities; 1: velocities and the gradient tensor; 2: fused Heun
// step; 3: second derivatives; 4: Lagrangian acceleration.  `stays` counts
// (per warp) the particles whose next bin is st.bin.
template <typename Tc, int MODE, int CT>
__device__ __forceinline__ void quad_chunk(const StagedArgs& a, const QGeo<CT>& geo,
                                           const QStage& st, int ch, int& stays,
                                           int phase = 0) {
  const GridArgs& g = a.g;
  const Tc* coef = static_cast<const Tc*>(a.coef);
  const int lane = threadIdx.x & 31, k = lane & 3;
  const int64_t np = a.np;
  const float nanf_ = __int_as_float(0x7fc00000);
  const int S3[3] = {geo.Sx, geo.Sy, geo.Sz};
  const int s = 8 * ch + (lane >> 2);
  const bool valid = s < st.m;
  const int slot = quad_slot(valid ? s : 8 * ch, st.ne, st.no);
  const float4 rt = st.rt[slot];
  const int4 rc = st.rc[slot];
  const bool ok = (rc.w & (1 << 30)) == 0;
  const int r = rc.w & 0xffff;
  const int wl = __float_as_int(rt.w);
  const bool inh = st.staged && ((wl >> 24) & 1);
  int l[3] = {wl & 0xff, (wl >> 8) & 0xff, (wl >> 16) & 0xff};
  int cell[3] = {rc.x, rc.y, rc.z};
  const float t[3] = {rt.x, rt.y, rt.z};
  const int64_t p = a.perm ? a.perm[st.cb + r] : (int64_t)(st.cb + r);
  float v[16][3];
  if constexpr (MODE == 4) {
    if (phase == 2) {
      // the later field's stencil, from its halo staged in the same buffer;
      // the convective term and u were left in the round's x records
      quad_fetch<Tc, CT>(v, inh, l, cell, k, st.halo, st.scl, geo, g,
                         static_cast<const Tc*>(a.coef2), a.scale2);
      float w[4][3];
      quad_sum<false>(v, t, k, w);
      if (valid) {
        if (k < 3) {
          const float* part = reinterpret_cast<const float*>(st.x) + 6 * slot;
          const float acc = __fmaf_rn(__fsub_rn(sel3(w[0], k), part[3 + k]), (float)a.dt,
                                      part[k]);
          a.grad[(int64_t)k * np + p] = ok ? acc : nanf_;
        }
      }
      return;
    }
  }
  quad_fetch<Tc, CT>(v, inh, l, cell, k, st.halo, st.scl, geo, g, coef, a.scale);
  if constexpr (MODE == 3) {
    // second derivatives -> hess [3][6][np] (a.grad), scaled by n_a/L_a n_b/L_b
    float h[6][3];
    quad_sum_hess(v, t, k, h);
    if (valid) {
      if (k < 3) {
        const float hx = g.inv_hf[0], hy = g.inv_hf[1], hz = g.inv_hf[2];
        const float sc[6] = {__fmul_rn(hx, hx), __fmul_rn(hy, hy), __fmul_rn(hz, hz),
                             __fmul_rn(hx, hy), __fmul_rn(hx, hz), __fmul_rn(hy, hz)};
#pragma unroll
        for (int e = 0; e < 6; ++e)
          a.grad[((int64_t)k * 6 + e) * np + p] = ok ? __fmul_rn(sel3(h[e], k), sc[e]) : nanf_;
      } else if (!ok) {
        flag_status(a.status, PS_DEV_NONFINITE_POS, p);
      }
    }
    return;
  }
  float u1[4][3];
  quad_sum<MODE == 1 || MODE == 4>(v, t, k, u1);
  if constexpr (MODE == 4) {
    // Lagrangian acceleration a = (u . grad) u + du/dt -> a.grad [3][np]: u
    // and its gradient from coef; with a later field (coef2) du/dt =
    // (u(coef2) - u) / dt_field (a.dt = 1 / dt_field), gathered in a second
    // phase (the convective term and u wait in the round's x records)
    if (valid) {
      if (k < 3) {
        const float gx = __fmul_rn(sel3(u1[1], k), g.inv_hf[0]);
        const float gy = __fmul_rn(sel3(u1[2], k), g.inv_hf[1]);
        const float gz = __fmul_rn(sel3(u1[3], k), g.inv_hf[2]);
        float conv = __fmul_rn(gx, u1[0][0]);
        conv = __fmaf_rn(gy, u1[0][1], conv);
        conv = __fmaf_rn(gz, u1[0][2], conv);
        if (a.coef2) {
          float* part = reinterpret_cast<float*>(const_cast<double*>(st.x)) + 6 * slot;
          part[k] = conv;
          part[3 + k] = sel3(u1[0], k);
        } else {
          a.grad[(int64_t)k * np + p] = ok ? conv : nanf_;
        }
        if (a.vel) a.vel[(int64_t)k * np + p] = ok ? sel3(u1[0], k) : nanf_;
      } else if (!ok) {
        flag_status(a.status, PS_DEV_NONFINITE_POS, p);
      }
    }
    return;
  }
  if constexpr (MODE <= 1) {
    if (valid) {
      if (k < 3) a.vel[(int64_t)k * np + p] = ok ? sel3(u1[0], k) : nanf_;
      if (MODE == 1 && a.grad && k < 3) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
          a.grad[((int64_t)k * 3 + d) * np + p] =
              ok ? __fmul_rn(sel3(u1[1 + d], k), g.inv_hf[d]) : nanf_;
      }
      if (k == 3 && !ok) flag_status(a.status, PS_DEV_NONFINITE_POS, p);
    }
  } else {
    // predictor x* = x + dt u1, located in FP32 from the stage-1 cell
    float t2[3];
    int c2[3], l2[3];
    bool moved = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float tt = __fmaf_rn(ok ? u1[0][d] : 0.f, a.dtih[d], t[d]);
      float f = floorf(tt);
      if (!(fabsf(f) < 1.0e9f)) f = 0.f;  // non-finite velocity: keep the cell
      t2[d] = fminf(fmaxf(__fsub_rn(tt, f), 0.f), 1.f);
      const int fl = (int)f;
      moved |= fl != 0;
      int c = cell[d] + fl;
      if (c < 0 || c >= g.n[d]) {
        c %= g.n[d];
        if (c < 0) c += g.n[d];
      }
      c2[d] = c;
      l2[d] = c - st.P0[d];
    }
    if (moved || a.coef2) {
      // the second field's coefficients are not staged
      bool inh2 = st.staged && !a.coef2;
#pragma unroll
      for (int d = 0; d < 3; ++d) inh2 = inh2 && (unsigned)l2[d] <= (unsigned)(S3[d] - 4);
      quad_fetch<Tc, CT>(v, inh2, l2, c2, k, st.halo, st.scl, geo, g,
                         a.coef2 ? static_cast<const Tc*>(a.coef2) : coef,
                         a.coef2 ? a.scale2 : a.scale);
    }
    float u2[4][3];
    quad_sum<false>(v, t2, k, u2);
    // lane k < 3 owns axis k from here on
    const int d = k < 3 ? k : 0;
    const float u1d = sel3(u1[0], d), u2d = sel3(u2[0], d);
    const double xd = st.x[d * kQT + r];
    const double xn = ok ? fma(a.dt * 0.5, (double)__fadd_rn(u1d, u2d), xd)
                         : __longlong_as_double(0x7ff8000000000000ll);
    if (valid) {
      if (k < 3) {
        a.pos_out[d * np + p] = xn;
        if (a.vel) a.vel[d * np + p] = ok ? u1d : nanf_;
      } else {
        if (a.ids_out) a.ids_out[p] = a.ids_in[p];
        if (!ok) flag_status(a.status, PS_DEV_NONFINITE_POS, p);
      }
    }
    if (a.next_counts) {
      // The new cell along axis k: the predictor's cell plus the floor of
      // its fraction plus the corrector's displacement dt (u2 - u1) / 2 in
      // cells, in FP32 (x^{n+1} = x* + dt (u2 - u1) / 2); that floor is the
      // exact one wherever the sum lies 2^-10 or more from a cell face and
      // |x n/L| < 2^30 (the roundings on both routes stay below 1e-6 cell).
      // Elsewhere, and for positions that are not finite, the FP64 location
      // decides.
      int bc = -1;
      if (k < 3) {
        const float w = sel3(t2, d) + 0.5f * a.dtih[d] * (u2d - u1d);
        const float f = floorf(w), fr = w - f;
        int c;
        if (ok && fr >= 0x1p-10f && fr <= 1.f - 0x1p-10f && fabsf(f) <= 2.f &&
            (__double2hiint(xd) & 0x7fffffff) < a.xguard_hi[d]) {
          const int nd = g.n[d];
          c = sel3(c2, d) + (int)f;  // in [-2, n + 1], n >= 3
          c = c < 0 ? c + nd : (c >= nd ? c - nd : c);
        } else {
          float tn;
          if (!locate(xn, g.inv_h[d], g.n[d], c, tn)) c = -1;
        }
        bc = c < 0 ? -1 : (a.bshift[d] >= 0 ? c >> a.bshift[d] : c / a.b.B[d]);
      }
      const int qb = lane & ~3;
      int key = bin_of_coords(a.b, __shfl_sync(FULL, bc, qb), __shfl_sync(FULL, bc, qb + 1),
                              __shfl_sync(FULL, bc, qb + 2));
      // The bin goes to next_bin[p]; the counters take the totals only (the
      // scatter takes the ranks).  Particles that stay in this brick are
      // counted per warp and added once per round; the others add one each.
      // A rejected position is counted in bin 0 and reported, as the
      // counting pass of the sort does.
      const bool mine = valid && k == 0;
      if (mine && key < 0) {
        flag_status(a.status, PS_DEV_NONFINITE_POS, p);
        key = 0;
      }
      if (mine) a.next_bin[p] = key;
      const bool stay = mine && key == st.bin;
      stays += __popc(__ballot_sync(FULL, stay));
      if (mine && !stay) atomicAdd(&a.next_counts[key], 1);
    }
  }
}

// ---------------------------------------------------- one block per brick --
// The brick's halo of a.coef by plain loads, in the layout the gathers read
// (float4 nodes, or raw 16-bit nodes with their rows' scales).  No barrier.
template <typename Tc, int CT>
__device__ __forceinline__ void quad_stage_loads(const StagedArgs& a, const QGeo<CT>& geo,
                                                 const QStage& st, float4* halo) {
  const Tc* coef = static_cast<const Tc*>(a.coef);
  const int tid = threadIdx.x;
  if constexpr (IsNode16<Tc>::value) {
    const GridArgs& g = a.g;
    const int nrow = geo.Sy * geo.Sz;
    Tc* h16 = reinterpret_cast<Tc*>(halo);
    for (int it = tid; it < nrow * geo.Sx; it += blockDim.x) {
      const int r = it / geo.Sx, x = it - r * geo.Sx;
      const int lz = r / geo.Sy, ly = r - lz * geo.Sy;
      const int64_t row = (int64_t)wrap_row(st.P0[2] + lz, g.n[2]) * g.m[1] +
                          wrap_row(st.P0[1] + ly, g.n[1]);
      h16[lz * geo.PS + ly * geo.SX + x] = coef[row * g.rx + wrap_row(st.P0[0] + x, g.n[0])];
    }
    float4* sc = const_cast<float4*>(st.scl);
    for (int r = tid; r < nrow; r += blockDim.x) {
      const int lz = r / geo.Sy, ly = r - lz * geo.Sy;
      const int64_t row = (int64_t)wrap_row(st.P0[2] + lz, g.n[2]) * g.m[1] +
                          wrap_row(st.P0[1] + ly, g.n[1]);
      sc[r] = __ldg(reinterpret_cast<const float4*>(a.scale) + row);
    }
  } else if (a.vec) {
    stage_halo_vec<Tc, 3>(a, coef, st.P0, halo, false);
  } else {
    stage_halo<Tc, 3>(a, coef, st.P0, halo, false);
  }
}

// The brick's halo by a tensor copy (node coefficients) or plain loads; its
// particles in rounds of kQT: phase A by all threads, a block barrier, phase
// B by the warps in turn.
template <typename Tc, int MODE, int CT>
__device__ __forceinline__ void quad_brick(const StagedArgs& a, float4* smem) {
  const int bin = blockIdx.x;
  const int beg = a.offs[bin], end = a.offs[bin + 1];
  if (beg >= end) return;
  const QGeo<CT> geo(a);
  const int nbx = a.b.nb[0], nby = a.b.nb[1];
  const int bzi = bin / (nbx * nby);
  const int rem = bin - bzi * nbx * nby;
  const int byi = rem / nbx, bxi = rem - byi * nbx;
  const Tc* coef = static_cast<const Tc*>(a.coef);
  QStage st;
  st.P0[0] = bxi * a.b.B[0];
  st.P0[1] = byi * a.b.B[1];
  st.P0[2] = bzi * a.b.B[2];
  float4* halo = smem;
  float4* rt = smem + halo_f4<Tc>(geo.Sz, geo.Sy, geo.PS);
  int4* rc = reinterpret_cast<int4*>(rt + kQT);
  double* xs = reinterpret_cast<double*>(rc + kQT);
  st.halo = halo;
  st.scl = reinterpret_cast<const float4*>(reinterpret_cast<const unsigned char*>(halo) +
                                           scale_off_bytes<Tc>(geo.Sz, geo.PS));
  st.rt = rt;
  st.rc = rc;
  st.x = xs;
  st.bin = bin;
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ int cnt[2][2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t np = a.np;

  const bool staged = end - beg >= a.min_stage && !a.chunked;
  bool tma = false;
  if constexpr (IsNode4<Tc>::value)
    tma = staged && a.tma && (smem_u32(halo) & 127) == 0;
  if (tid == 0) {
    cnt[0][0] = cnt[0][1] = cnt[1][0] = cnt[1][1] = 0;
    if (tma) {
      if (a.wait_probe > 0) tma_init_barrier(&mbar[1]);
      if constexpr (IsNode16<Tc>::value) {
        // raw 16-bit nodes (node pairs as the copy's 16-byte unit) and the
        // rows' scales, both on one barrier
        tma_issue_node16(&a.tmap, &a.tmap2, halo, const_cast<float4*>(st.scl), &mbar[0], st.P0,
                         (unsigned)(geo.Sz * geo.Sy * (geo.SX * 8 + 16)));
      } else {
        tma_init_barrier(&mbar[0]);
        tma_copy_halo(&a.tmap, halo, &mbar[0], st.P0,
                      (unsigned)(sizeof(float4) * geo.SX * geo.Sy * geo.Sz));
      }
    }
  }
  if (staged && !tma) quad_stage_loads<Tc, CT>(a, geo, st, halo);
  __syncthreads();  // counters, barrier initialisation, staged halo

  bool copied = staged;  // the tensor copy of the halo completed (or there is none)
  bool halo_ok = staged; // the halo buffer holds the nodes the next gathers read
  int stays = 0;
  int round = 0;
  for (int cb = beg; cb < end; cb += kQT, ++round) {
    const int mr = min(kQT, end - cb);
    {
      const bool v = tid < mr;
      double x[3] = {0.0, 0.0, 0.0};
      if (v) {
        const int64_t p = a.perm ? a.perm[cb + tid] : (int64_t)(cb + tid);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          x[d] = a.pos_in[d * np + p];
          if (MODE == 2) xs[d * kQT + tid] = x[d];
        }
      }
      quad_locate<CT>(a, geo, st.P0, staged, tid, v, x, rt, rc, cnt[round & 1]);
    }
    __syncthreads();
    if (round == 0 && tma) {
      // the barrier above also ordered the mbarrier's initialisation before
      // these waits; a copy that does not complete in time is reported and
      // the brick's particles read global memory
      bool done = tma_wait(&mbar[0], 0);
      if (done && a.wait_probe > 0) done = tma_wait(&mbar[1], 0, a.wait_probe);
      if (!done) {
        copied = false;
        halo_ok = false;
        if (lane == 0) flag_status(a.status, PS_DEV_TIMEOUT, beg);
      }
    }
    st.ne = cnt[round & 1][0];
    st.no = cnt[round & 1][1];
    st.cb = cb;
    st.m = mr;
    st.staged = halo_ok;
    if (tid == 0 && cb + kQT < end) {
      // the next round's counters (last read in the previous round)
      cnt[(round + 1) & 1][0] = 0;
      cnt[(round + 1) & 1][1] = 0;
    }
    for (int ch = warp; 8 * ch < mr; ch += nwarps) quad_chunk<Tc, MODE, CT>(a, geo, st, ch, stays);
    if constexpr (MODE == 4) {
      if (a.coef2) {
        // the later field's halo replaces this one (plain loads), then the
        // second gathers; a tensor copy that had not landed must first (its
        // bounded wait again), else the second field is read from global
        // memory (one decision for the block: the staging is shared)
        __syncthreads();
        bool can = staged;
        if (tma && !copied) {
          copied = tma_wait(&mbar[0], 0);
          can = can && copied;
        }
        can = __syncthreads_and(can);
        bool by_copy = false;
        if constexpr (IsNode4<Tc>::value && !IsNode16<Tc>::value) {
          // tmap2 holds the later field's node map (tma == 2): one more
          // tensor copy into the same buffer, the barrier's next phase
          if (can && tma && a.tma == 2 && round == 0) {
            by_copy = true;
            if (tid == 0) {
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              tma_copy_halo(&a.tmap2, halo, &mbar[0], st.P0,
                            (unsigned)(sizeof(float4) * geo.SX * geo.Sy * geo.Sz));
            }
            const bool done2 = tma_wait(&mbar[0], 1);
            can = __syncthreads_and(done2);
            if (!done2) {
              copied = tma_wait(&mbar[0], 1);  // must land before the block ends
              if (lane == 0) flag_status(a.status, PS_DEV_TIMEOUT, beg);
            }
          }
        }
        if (can && !by_copy) {
          StagedArgs a2 = a;
          a2.coef = a.coef2;
          a2.scale = a.scale2;
          quad_stage_loads<Tc, CT>(a2, geo, st, halo);
        }
        st.staged = can;
        __syncthreads();
        for (int ch = warp; 8 * ch < mr; ch += nwarps)
          quad_chunk<Tc, MODE, CT>(a, geo, st, ch, stays, 2);
        if (cb + kQT < end) {
          // the next round's first phase reads the first field's halo again
          __syncthreads();
          if (can) quad_stage_loads<Tc, CT>(a, geo, st, halo);
          halo_ok = can;
        }
      }
    }
    if (cb + kQT < end) __syncthreads();  // the records are refilled
  }
  if (MODE == 2 && a.next_counts && lane == 0 && stays) atomicAdd(&a.next_counts[bin], stays);
  // a copy still in flight must land before the block's memory is released
  if (tma && !copied) tma_wait(&mbar[0], 0);
}

// CT: the halo geometry of the 8^3 brick fixed at compile time.
template <typename Tc, int MODE, int CT>
__global__ void __launch_bounds__(kQT, 5) quad_kernel(const __grid_constant__ StagedArgs a) {
  extern __shared__ __align__(128) float4 smem_q[];
  quad_brick<Tc, MODE, CT>(a, smem_q);
}

// Row length SX >= S[0] with SX * S[1] = 2 or 6 (mod 8); 0 if none exists
// (S[1] a multiple of 4).
int quad_row(int sx, int sy) {
  for (int r = sx; r < sx + 8; ++r)
    if (((r * sy) & 3) == 2) return r;
  return 0;
}
// 16-bit nodes: an even row length (node pairs are the tensor copy's unit),
// preferably with SX * S[1] = 4 (mod 16), so that the four z-rows of a quad
// read four bank pairs 4 nodes apart.
int quad_row16(int sx, int sy) {
  const int r0 = sx + (sx & 1);
  for (int r = r0; r < r0 + 16; r += 2)
    if (((r * sy) & 15) == 4) return r;
  return r0;
}
template <typename Tc> struct NodeDtype { static constexpr int v = -1; };
template <> struct NodeDtype<float4> { static constexpr int v = PS_F32X4; };
template <> struct NodeDtype<bf16x4> { static constexpr int v = PS_BF16X4; };
template <> struct NodeDtype<f16x4> { static constexpr int v = PS_F16X4; };

template <typename Tc, int MODE>
ps_status launch_quad_t(const StagedArgs& a0, cudaStream_t st, bool* done) {
  StagedArgs a = a0;
  constexpr bool n16 = IsNode16<Tc>::value;
  const int SX = n16 ? quad_row16(a.S[0], a.S[1]) : quad_row(a.S[0], a.S[1]);
  if (SX == 0 || a.E != 0) return PS_OK;  // not handled here
  a.SX = SX;
  a.PS = SX * a.S[1];
  a.wait_probe = tuning().wait_probe;
  a.tma = 0;
  if constexpr (NodeDtype<Tc>::v >= 0)
    if (a0.tma && SX <= 256) a.tma = encode_node_halo_map(&a, (ps_dtype)NodeDtype<Tc>::v) ? 1 : 0;
  if constexpr (MODE == 4 && std::is_same<Tc, float4>::value) {
    // the later field's node map in tmap2 (tma = 2)
    if (a.tma == 1 && a.coef2) {
      StagedArgs t = a;
      t.coef = a.coef2;
      if (encode_node_halo_map(&t, PS_F32X4)) {
        a.tmap2 = t.tmap;
        a.tma = 2;
      }
    }
  }
  const size_t smem = (size_t)halo_f4<Tc>(a.S[2], a.S[1], a.PS) * sizeof(float4) + qrec_bytes();
  if (smem > 227 * 1024) return PS_OK;
  if (a.b.nbins > 0x7fffffff) return fail(PS_ERR_UNSUPPORTED, "too many bins");
  const bool cube = a.S[0] == 11 && a.S[1] == 11 && a.S[2] == 11;
  auto kern = quad_kernel<Tc, MODE, 0>;
  if constexpr (n16) {
    if (cube && a.SX == 12) kern = quad_kernel<Tc, MODE, 12>;
  } else {
    if (cube && a.SX == 14) kern = quad_kernel<Tc, MODE, 14>;
  }
  if (smem > 48 * 1024) {
    ps_status rc = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "quad smem attribute");
    if (rc) return rc;
  }
  *done = true;
  kern<<<(unsigned)a.b.nbins, kQT, smem, st>>>(a);
  return check_launch("quad_kernel");
}

}  // namespace

// Brick kernel 5 for three components: F32 node coefficients or planar
// F32/BF16/F16.  *done stays false where this form does not apply (E != 0, no
// row length with the bank property, 16-bit nodes, a halo above the shared
// memory), and the caller takes another form.
ps_status launch_quad(const StagedArgs& a, ps_dtype coef_t, int mode, cudaStream_t st,
                      bool* done) {
  *done = false;
  auto go = [&](auto tag) -> ps_status {
    using Tc = decltype(tag);
    switch (mode) {
      case 0: return launch_quad_t<Tc, 0>(a, st, done);
      case 1: return launch_quad_t<Tc, 1>(a, st, done);
      case 2: return launch_quad_t<Tc, 2>(a, st, done);
      case 3: return launch_quad_t<Tc, 3>(a, st, done);
      default: return launch_quad_t<Tc, 4>(a, st, done);
    }
  };
  switch (coef_t) {
    case PS_F32X4: return go(float4{});
    case PS_F32: return go(float{});
    case PS_BF16: return go(__nv_bfloat16{});
    case PS_F16: return go(__half{});
    case PS_BF16X4: return go(bf16x4{});
    case PS_F16X4: return go(f16x4{});
    default: return PS_OK;
  }
}

}  // namespace ps
