// Shared pieces of the brick-staged kernels (interp.cu, quad.cu): the launch
// argument block, the halo geometry, the tensor-copy and mbarrier helpers and
// the plain-load halo staging.  Internal to libps.
#pragma once

#include <type_traits>

#include <cuda.h>

#include "ps_internal.cuh"

namespace ps {

struct StagedArgs {
  GridArgs g;
  BrickArgs b;
  int E;        // extra halo cells on each side
  int S[3];     // staged extent per axis: B + 3 + 2E
  int SX;       // row stride in float4 units (= S[0])
  int PS;       // plane stride in float4 units: >= SX*S[1], = 4 (mod 8)
  int vec;      // 1: halo rows are whole 16-byte vectors inside the array
  int min_stage;  // bricks with fewer particles gather from global memory
  int tma;        // 1: the node halo is one tensor copy described by tmap
  int chunked;    // 1: bins are runs of particles (sparse field): no halo
  int wait_probe; // > 0: test knob, a wait on a barrier nothing completes
                  // (this many clocks) follows the halo's own wait
  const void* coef;
  const float* scale;
  const void* coef2;  // second-stage field of an RK2 step; NULL = same as coef
  const float* scale2;
  int64_t np;
  const double* pos_in;
  double* pos_out;
  const int64_t* perm;
  const int32_t* offs;
  float* vel;
  float* grad;
  const int64_t* ids_in;
  int64_t* ids_out;
  double dt;
  float dtih[3];  // dt * n/L per axis
  int32_t* status;
  // counting pass of the next step's bin sort (NULL = off): each particle's
  // new bin at its slot in pos_out, bin counters (zeroed beforehand)
  int32_t* next_counts;
  int32_t* next_bin;
  int32_t next_key_base;  // added to the key stored in next_bin (batched bins)
  int32_t next_runs;      // > 0: bins are runs, run = brick * next_runs / nbins
  int bshift[3];  // log2 of the brick extent, -1 if not a power of two
  // high word of the double 2^30 L/n per axis: |x| has a smaller high word
  // (sign cleared) only if |x n/L| < 2^30, read without an FP64 operation
  int xguard_hi[3];
  CUtensorMap tmap;   // node halo box (valid when tma == 1)
  CUtensorMap tmap2;  // 16-bit nodes: the box of the halo rows' scales
};

// Tensor map of the node halo box (4 floats x a.SX nodes x S[1] rows x S[2]
// planes) over a node coefficient array (interp.cu).
bool encode_node_halo_map(StagedArgs* a, ps_dtype coef_t);

// The quad-per-particle brick kernel (quad.cu) for three components; mode 0
// velocities, 1 with the gradient tensor, 2 fused Heun step, 3 second
// derivatives (into a.grad), 4 Lagrangian acceleration (into a.grad; a.dt
// holds 1 / dt_field).  Leaves *done false where it does not apply.
ps_status launch_quad(const StagedArgs& a, ps_dtype coef_t, int mode, cudaStream_t st,
                      bool* done);

#ifdef __CUDACC__
namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T pick4(const T b[4], int q) {
  return q == 0 ? b[0] : (q == 1 ? b[1] : (q == 2 ? b[2] : b[3]));
}
template <typename T>
__device__ __forceinline__ T sel3(const T v[3], int i) {
  return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int d = 1; d < G; d <<= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}
// The same butterfly on a packed pair: two shuffles and one packed add per
// level, each component rounded as group_sum's.
template <int G>
__device__ __forceinline__ float2 group_sum2(float2 v) {
#pragma unroll
  for (int d = 1; d < G; d <<= 1)
    v = __fadd2_rn(v, make_float2(__shfl_xor_sync(FULL, v.x, d), __shfl_xor_sync(FULL, v.y, d)));
  return v;
}

template <typename Tc>
__device__ __forceinline__ typename AccOf<Tc>::type load_coef(const Tc* coef,
                                                              const float* scale,
                                                              const GridArgs& g, int c,
                                                              int Pz, int Py, int Px) {
  if constexpr (IsNode16<Tc>::value) {
    // component c of a 16-bit node, times its line's scale
    const int64_t row = (int64_t)Pz * g.m[1] + Py;
    return node16_value(coef[row * g.rx + Px].v[c]) * __ldg(scale + row * 4 + c);
  } else if constexpr (IsNode4<Tc>::value) {
    // component c of node (Pz, Py, Px); the node's other components share
    // the 16-byte segment
    const int64_t node = ((int64_t)Pz * g.m[1] + Py) * g.rx + Px;
    return __ldg(reinterpret_cast<const float*>(coef + node) + c);
  } else {
    const int64_t m1 = g.m[1], m2 = g.m[2];
    const int64_t row = ((int64_t)c * m2 + Pz) * m1 + Py;
    typename AccOf<Tc>::type v = CoefLoad<Tc>::ld(coef + row * g.rx + Px);
    if (IsQuant<Tc>::value) v *= __ldg(scale + row);
    return v;
  }
}

// ------------------------------------------------------------- staged ----



// Halo geometry (extents, row and plane strides in float4 units).  KS > 0
// fixes at compile time the cubic halo of KS points per axis of the 8^3
// brick (KS = 11, plane stride 124 = 4 mod 8), so that every index in the
// staging and the gathers folds into immediates; KS = 0 reads the launch
// arguments.
template <int KS> struct HaloGeo {
  int Sx, Sy, Sz, SX, PS;
  __device__ __forceinline__ explicit HaloGeo(const StagedArgs& a)
      : Sx(a.S[0]), Sy(a.S[1]), Sz(a.S[2]), SX(a.SX), PS(a.PS) {}
};
template <> struct HaloGeo<11> {
  static constexpr int Sx = 11, Sy = 11, Sz = 11, SX = 11, PS = 124;
  __device__ __forceinline__ explicit HaloGeo(const StagedArgs&) {}
};
// The same halo with 12-point rows: the layout of a tensor copy of a node
// halo, whose plane of 12 x 11 points is 132 = 4 (mod 8) float4 long.
template <> struct HaloGeo<12> {
  static constexpr int Sx = 11, Sy = 11, Sz = 11, SX = 12, PS = 132;
  __device__ __forceinline__ explicit HaloGeo(const StagedArgs&) {}
};
__device__ __forceinline__ bool is_cube11(const StagedArgs& a) {
  return a.S[0] == 11 && a.S[1] == 11 && a.S[2] == 11 && a.SX == 11 && a.PS == 124;
}
__device__ __forceinline__ bool is_cube11_rows12(const StagedArgs& a) {
  return a.S[0] == 11 && a.S[1] == 11 && a.S[2] == 11 && a.SX == 12 && a.PS == 132;
}

// ------------------------------------------------- tensor-copy staging ----
// One thread arms an mbarrier with the byte count of the box and issues the
// tensor copy of the brick's node halo; the copy completes the barrier's
// phase, after which every thread that waited on it sees the data.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tma_init_barrier(unsigned long long* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Arms the barrier's current phase with the box's byte count and issues the
// copy (the barrier was initialised before).
__device__ __forceinline__ void tma_copy_halo(const CUtensorMap* map, float4* dst,
                                              unsigned long long* mbar, const int P0[3],
                                              unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(0), "r"(P0[0]), "r"(P0[1]), "r"(P0[2]),
      "r"(smem_u32(mbar))
      : "memory");
}
__device__ __forceinline__ void tma_issue_halo(const CUtensorMap* map, float4* dst,
                                               unsigned long long* mbar, const int P0[3],
                                               unsigned bytes) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(0), "r"(P0[0]), "r"(P0[1]), "r"(P0[2]),
      "r"(smem_u32(mbar))
      : "memory");
}
// 16-bit node halos: the tensor copies put the raw nodes and their rows'
// scales into the float4 halo's own buffer, near its end (both 128-byte
// aligned), and the block widens them in place in kNode16Slices slices of
// nodes: each slice is read into registers, a barrier, then written as
// float4.  The float4 writes of a slice reach raw bytes of its own or of
// earlier slices only, and the scales only in the last slice (checked below
// for the compile-time 8^3 halo).  Offsets in bytes from the halo's start.
constexpr int kNode16Slices = 4;
__host__ __device__ constexpr int align_down128(int v) { return v & ~127; }
__host__ __device__ constexpr int node16_scale_offset(int Sz, int PS, int Sy) {
  return align_down128(Sz * PS * 16 - Sz * Sy * 16);
}
__host__ __device__ constexpr int node16_raw_offset(int Sz, int PS, int Sy, int SX) {
  return align_down128(node16_scale_offset(Sz, PS, Sy) - Sz * Sy * SX * 8);
}
// slice s (s < kNode16Slices - 1) writes float4 nodes below (s + 1) * per;
// the raw nodes of slice s + 1 start at raw + 8 (s + 1) per
__host__ __device__ constexpr bool node16_in_place_ok(int Sz, int PS, int Sy, int SX) {
  const int npts = Sz * Sy * SX, per = (npts + kNode16Slices - 1) / kNode16Slices;
  bool ok = Sz * PS >= npts && node16_raw_offset(Sz, PS, Sy, SX) >= 0;
  for (int s = 0; s + 1 < kNode16Slices; ++s) {
    const int end_write = 16 * (s + 1) * per;
    ok = ok && end_write <= node16_raw_offset(Sz, PS, Sy, SX) + 8 * (s + 1) * per &&
         end_write <= node16_scale_offset(Sz, PS, Sy);
  }
  return ok;
}
static_assert(node16_in_place_ok(11, 132, 11, 12), "16-bit node halo cannot widen in place");

__device__ __forceinline__ void tma_issue_node16(const CUtensorMap* nodes,
                                                 const CUtensorMap* scales, void* raw,
                                                 void* sraw, unsigned long long* mbar,
                                                 const int P0[3], unsigned bytes) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
  // node pairs are the 16-byte inner unit: x coordinate P0[0] / 2
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(raw)),
      "l"(reinterpret_cast<unsigned long long>(nodes)), "r"(0), "r"(P0[0] >> 1), "r"(P0[1]),
      "r"(P0[2]), "r"(smem_u32(mbar))
      : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(sraw)),
      "l"(reinterpret_cast<unsigned long long>(scales)), "r"(0), "r"(P0[1]), "r"(P0[2]),
      "r"(smem_u32(mbar))
      : "memory");
}

// Waits for the barrier's phase of the given parity, giving up after `limit`
// clocks (default 2^31, about a second); returns whether the phase completed.
__device__ __forceinline__ bool tma_wait(unsigned long long* mbar, unsigned parity = 0,
                                         long long limit = 1ll << 31) {
  const unsigned a = smem_u32(mbar);
  // the suspend-time hint (ns) lets the thread sleep until the phase
  // completes instead of polling; each try returns within the hint
  const unsigned hint = limit < (1ll << 24) ? 1000u : 1000000u;
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(hint)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// Padded index (any integer) -> interior padded index of the same node.
__device__ __forceinline__ int wrap_row(int P, int n) {
  while (P < 1) P += n;
  while (P > n) P -= n;
  return P;
}

// Copy the brick halo (S[0] x S[1] x S[2] padded points) into shared memory
// as float4 (u, v, w, 0) per point.  16 (or 32) lanes walk x within a row,
// the block covers 16 (or 8) rows at a time; each thread loads four rows
// before storing them so that the loads overlap.
template <typename Tc, int NC>
__device__ __forceinline__ void stage_halo(const StagedArgs& a, const Tc* __restrict__ coef,
                                           const int P0[3], float4* halo, bool sync = true) {
  const GridArgs& g = a.g;
  const int Sx = a.S[0], Sy = a.S[1], Sz = a.S[2];
  const bool narrow = Sx <= 16;
  const int tx = narrow ? (threadIdx.x & 15) : (threadIdx.x & 31);
  const int ty = narrow ? (threadIdx.x >> 4) : (threadIdx.x >> 5);
  const int RS = narrow ? (int)(blockDim.x >> 4) : (int)(blockDim.x >> 5);  // rows per step
  const bool xact = tx < Sx;
  const int Px = wrap_row(P0[0] + tx, g.n[0]);
  const int64_t m0 = g.rx, m1 = g.m[1], m2 = g.m[2];
  const int64_t cs = m0 * m1 * m2;
  const int nrows = Sy * Sz;
  int ly = ty % Sy, lz = ty / Sy;
  for (int r = ty; r < nrows; r += 4 * RS) {
    float v[4][NC];
    int dst[4];
    bool act[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      act[u] = xact && (r + u * RS) < nrows;
      const int Py = wrap_row(P0[1] + ly, g.n[1]);
      const int Pz = wrap_row(P0[2] + lz, g.n[2]);
      const int64_t row = (int64_t)Pz * m1 + Py;
      dst[u] = lz * a.PS + ly * a.SX + tx;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float x = 0.f;
        if (act[u]) {
          if constexpr (IsNode16<Tc>::value) {
            x = node16_value(coef[row * m0 + Px].v[c]) * __ldg(a.scale + row * 4 + c);
          } else if constexpr (IsNode4<Tc>::value) {
            x = __ldg(reinterpret_cast<const float*>(coef + row * m0 + Px) + c);
          } else {
            x = (float)CoefLoad<Tc>::ld(coef + c * cs + row * m0 + Px);
            if (IsQuant<Tc>::value) x *= __ldg(a.scale + c * m2 * m1 + row);
          }
        }
        v[u][c] = x;
      }
      ly += RS;
      while (ly >= Sy) {
        ly -= Sy;
        ++lz;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (act[u])
        halo[dst[u]] = make_float4(v[u][0], NC > 1 ? v[u][NC > 1 ? 1 : 0] : 0.f,
                                   NC > 2 ? v[u][NC > 2 ? 2 : 0] : 0.f, 0.f);
  }
  if (sync) __syncthreads();
}

// Vector staging.  With E = 0 and bricks that tile the grid, the halo of
// brick b spans padded indices [b B, b B + B + 2] on every axis, inside the
// padded array; when B is a multiple of the vector width V (16 bytes) every
// halo row starts on a 16-byte boundary (the row pitch is a multiple of 16
// bytes), so each row is read with ceil(S_x / V) 16-byte loads per component
// and transposed in registers into the float4-per-point layout.
template <typename Tc> struct Vec16;
template <> struct Vec16<float> {
  static constexpr int V = 4;
  static __device__ __forceinline__ void load(const float* p, float s, float out[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = v.x * s; out[1] = v.y * s; out[2] = v.z * s; out[3] = v.w * s;
  }
};
template <typename H> struct Vec16Half {
  static constexpr int V = 8;
  static __device__ __forceinline__ void load(const H* p, float s, float out[8]) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const unsigned short lo = (unsigned short)(w[i] & 0xffffu), hi = (unsigned short)(w[i] >> 16);
      out[2 * i] = CoefLoadBits<H>::f(lo) * s;
      out[2 * i + 1] = CoefLoadBits<H>::f(hi) * s;
    }
  }
};
template <> struct Vec16<__nv_bfloat16> : Vec16Half<__nv_bfloat16> {};
template <> struct Vec16<__half> : Vec16Half<__half> {};

template <typename Tc, int NC, int KS>
__device__ __forceinline__ void stage_halo_vec_planar(const StagedArgs& a,
                                                      const Tc* __restrict__ coef,
                                                      const int P0[3], float4* halo, bool sync);

// Node coefficients: one 16-byte load and store per halo point, consecutive
// threads along the rows.
template <typename Tc, int KS>
__device__ __forceinline__ void stage_nodes(const StagedArgs& a, const Tc* __restrict__ coef,
                                            const int P0[3], float4* halo) {
  const HaloGeo<KS> hg(a);
  const int64_t rx = a.g.rx, m1 = a.g.m[1];
  const Tc* b0 = coef + ((int64_t)P0[2] * m1 + P0[1]) * rx + P0[0];
  const int nrow = hg.Sy * hg.Sz, npts = nrow * hg.Sx;
  for (int it = threadIdx.x; it < npts; it += blockDim.x) {
    const int r = it / hg.Sx, x = it - r * hg.Sx;
    const int lz = r / hg.Sy, ly = r - lz * hg.Sy;
    const int64_t roff = (int64_t)lz * m1 + ly;
    if constexpr (IsNode16<Tc>::value) {
      const Tc n = b0[roff * rx + x];
      const float4 sc = __ldg(reinterpret_cast<const float4*>(a.scale) +
                              ((int64_t)P0[2] * m1 + P0[1]) + roff);
      halo[lz * hg.PS + ly * hg.SX + x] =
          make_float4(node16_value(n.v[0]) * sc.x, node16_value(n.v[1]) * sc.y,
                      node16_value(n.v[2]) * sc.z, 0.f);
    } else {
      halo[lz * hg.PS + ly * hg.SX + x] = __ldg(b0 + roff * rx + x);
    }
  }
}

template <typename Tc, int NC, int KS = 0>
__device__ __forceinline__ void stage_halo_vec(const StagedArgs& a, const Tc* __restrict__ coef,
                                               const int P0[3], float4* halo, bool sync = true) {
  if constexpr (IsNode4<Tc>::value) {
    stage_nodes<Tc, KS>(a, coef, P0, halo);
    if (sync) __syncthreads();
  } else {
    stage_halo_vec_planar<Tc, NC, KS>(a, coef, P0, halo, sync);
  }
}

template <typename Tc, int NC, int KS>
__device__ __forceinline__ void stage_halo_vec_planar(const StagedArgs& a,
                                                      const Tc* __restrict__ coef,
                                                      const int P0[3], float4* halo, bool sync) {
  constexpr int V = Vec16<Tc>::V;
  constexpr int U = 8 / V;               // rows in flight per thread
  const GridArgs& g = a.g;
  const HaloGeo<KS> hg(a);
  const int Sx = hg.Sx, Sy = hg.Sy, Sz = hg.Sz;
  const int qx = (Sx + V - 1) / V;       // vectors per halo row (<= 4)
  const int qd = threadIdx.x & 3, rs = threadIdx.x >> 2;
  const int RS = blockDim.x >> 2;        // rows per block step
  const int64_t rx = g.rx, m1 = g.m[1], m2 = g.m[2];
  const int64_t cs = rx * m1 * m2;
  const int nrows = Sy * Sz;
  if (V == 4 && qx == 3 && (Sx & 1)) {
    // Items in groups of 24 = 8 rows x 3 vectors, ordered so that the eight
    // lanes of each 128-bit store phase write (rows r..r+3, vectors 0-1) or
    // (rows r..r+7, vector 2): with an odd row stride these hit eight distinct
    // 16-byte bank groups.
    const Tc* b0 = coef + ((int64_t)P0[2] * m1 + P0[1]) * rx + P0[0];
    const int nitems = (nrows + 7) / 8 * 24;
    for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
      const int grp = it / 24, l = it - grp * 24;
      const int rr = l < 16 ? (l >> 1) : l - 16;
      const int q = l < 16 ? (l & 1) : 2;
      const int r = grp * 8 + rr;
      if (r >= nrows) continue;
      const int lz = r / Sy, ly = r - lz * Sy;
      const int64_t roff = ((int64_t)lz * m1 + ly) * rx + q * 4;
      float v[NC][4];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float sc = 1.f;
        if (IsQuant<Tc>::value)
          sc = __ldg(a.scale + ((int64_t)c * m2 + P0[2] + lz) * m1 + P0[1] + ly);
        Vec16<Tc>::load(b0 + c * cs + roff, sc, v[c]);
      }
      const int h0 = lz * hg.PS + ly * hg.SX + q * 4;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (q * 4 + i < Sx)
          halo[h0 + i] = make_float4(v[0][i], NC > 1 ? v[NC > 1 ? 1 : 0][i] : 0.f,
                                     NC > 2 ? v[NC > 2 ? 2 : 0][i] : 0.f, 0.f);
    }
    if (sync) __syncthreads();
    return;
  }
  const Tc* base = coef + ((int64_t)P0[2] * m1 + P0[1]) * rx + P0[0] + qd * V;
  for (int r0 = rs; r0 < nrows; r0 += U * RS) {
    float v[U][NC][V];
    int h0[U];
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u * RS;
      act[u] = qd < qx && r < nrows;
      const int lz = r / Sy, ly = r - lz * Sy;
      h0[u] = lz * hg.PS + ly * hg.SX + qd * V;
      const int64_t roff = ((int64_t)lz * m1 + ly) * rx;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (act[u]) {
          float s = 1.f;
          if (IsQuant<Tc>::value)
            s = __ldg(a.scale + ((int64_t)c * m2 + P0[2] + lz) * m1 + P0[1] + ly);
          Vec16<Tc>::load(base + c * cs + roff, s, v[u][c]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (act[u])
#pragma unroll
        for (int i = 0; i < V; ++i)
          if (qd * V + i < Sx)
            halo[h0[u] + i] = make_float4(v[u][0][i], NC > 1 ? v[u][NC > 1 ? 1 : 0][i] : 0.f,
                                          NC > 2 ? v[u][NC > 2 ? 2 : 0][i] : 0.f, 0.f);
  }
  if (sync) __syncthreads();
}


}  // namespace
#endif  // __CUDACC__

}  // namespace ps
