// Operation 1 of Sec. 2.2: periodic cubic-spline coefficients.
//
// Every grid line of N nodes solves (1/6) c[j-1] + (4/6) c[j] + (1/6) c[j+1]
// = g[j] (indices mod N).  With S the cyclic shift, A = (4 + S + S^-1)/6
// factors as A = -(1/(6 z)) (1 - z S)(1 - z S^-1), z = sqrt(3) - 2 (the root
// of z^2 + 4 z + 1 = 0 inside the unit circle).  Hence
//     c = -6 z * (1 - z S)^-1 (1 - z S^-1)^-1 g,
// a causal first-order recursion y[j] = g[j] + z y[j-1] followed by an
// anti-causal one w[j] = y[j] + z w[j+1], both periodic, and a gain -6 z.
// This is the exact inverse that the paper's Thomas + periodic-correction
// solve computes; only the rounding order differs.
//
// Each pencil is split into chunks held in registers by different threads.
// A chunk first runs its recursion from a zero state; the true state entering
// chunk m is then sum_j (prod of z^len over the chunks in between) * (chunk
// end value), taken cyclically over the preceding chunks and divided by
// 1 - z^N when the sum wraps the whole pencil.  The products fall below
// 1e-12 (FP32) or 1e-24 (FP64) after a chunk or two, where the sum stops, so
// every pencil is read once and written once.
//
// FP32 coefficients of FP32 fields on rows of 128, 256 or 512 values take two
// streamed passes (x and y of every plane, then z; see below).  Otherwise
// three passes: y, then z (strided: threads along x read coalesced rows),
// then x (one warp per row, staged through shared memory), which writes the
// padded N+3 layout with periodic ghosts and, for BF16/FP16, a power-of-two
// scale per x-line.
#include <mutex>
#include <type_traits>

#include "ps_internal.cuh"

namespace ps {
namespace {

// [c][z][y][x] view with unit x stride.
struct View {
  int64_t off, sc, sz, sy;
};

template <typename T> struct Thr;
template <> struct Thr<float> { static constexpr float v = 1e-12f; };
template <> struct Thr<double> { static constexpr double v = 1e-24; };

template <typename To> __device__ __forceinline__ To cvt_out(float v);
template <> __device__ __forceinline__ float cvt_out<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half cvt_out<__half>(float v) {
  return __float2half_rn(v);
}
template <typename To> __device__ __forceinline__ To cvt_out_d(double v) { return (To)v; }

// Strided-axis pass.  blockDim = (XW, M): XW consecutive x, M chunks of the
// pencil.  grid = (ceil(nx/XW), n_other, ncomp).  src and dst may alias
// exactly (in place): each thread reads all its elements before any write and
// owns them.
// z^k for k = 0..64 (the recursions' pole), in both precisions; filled once
// per device from the host's FP64 value of z.
__constant__ float c_zpow_f[65];
__constant__ double c_zpow_d[65];
template <typename T> __device__ __forceinline__ T zpow(int k);
template <> __device__ __forceinline__ float zpow<float>(int k) { return c_zpow_f[k]; }
template <> __device__ __forceinline__ double zpow<double>(int k) { return c_zpow_d[k]; }

// One chunk of a pencil held in registers, len <= LMAX values: the causal
// recursion from a zero state (returns its end state), the causal fix-up
// v_i += c z^(i+1), the anti-causal recursion (returns its start state) and
// its fix-up v_i += c z^(len-i).  Full chunks (len == LMAX) run without
// predicates and take the powers of z from the constant table.
template <typename T, int LMAX>
__device__ __forceinline__ T chunk_causal(T v[LMAX], int len, T z) {
  T y = T(0);
  if (len == LMAX) {
#pragma unroll
    for (int i = 0; i < LMAX; ++i) v[i] = y = v[i] + z * y;
  } else {
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i < len) v[i] = y = v[i] + z * y;
  }
  return y;
}
template <typename T, int LMAX>
__device__ __forceinline__ void chunk_causal_fix(T v[LMAX], int len, T c) {
#pragma unroll
  for (int i = 0; i < LMAX; ++i)
    if (len == LMAX || i < len) v[i] += c * zpow<T>(i + 1);
}
template <typename T, int LMAX>
__device__ __forceinline__ T chunk_anticausal(T v[LMAX], int len, T z) {
  T w = T(0);
  if (len == LMAX) {
#pragma unroll
    for (int i = LMAX - 1; i >= 0; --i) v[i] = w = v[i] + z * w;
  } else {
#pragma unroll
    for (int i = LMAX - 1; i >= 0; --i)
      if (i < len) v[i] = w = v[i] + z * w;
  }
  return w;
}
template <typename T, int LMAX>
__device__ __forceinline__ void chunk_anticausal_fix(T v[LMAX], int len, T c, T z) {
  if (len == LMAX) {
#pragma unroll
    for (int i = 0; i < LMAX; ++i) v[i] += c * zpow<T>(LMAX - i);
  } else {
    T pw = z * c;
#pragma unroll
    for (int i = LMAX - 1; i >= 0; --i)
      if (i < len) {
        v[i] += pw;
        pw *= z;
      }
  }
}
// z^len of a chunk.
template <typename T>
__device__ __forceinline__ T chunk_zlen(int len) {
  return len <= 64 ? zpow<T>(len) : T(0);
}

template <typename Tin, typename T, int LMAX>
__global__ void __launch_bounds__(1024) solve_strided(
    const Tin* src, int64_t s_off, int64_t s_sc, int64_t s_so, int64_t s_si,
    T* dst, int64_t d_off, int64_t d_sc, int64_t d_so, int64_t d_si, int nx,
    int n, T z, T gain) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int XW = blockDim.x, M = blockDim.y;
  T* sa = reinterpret_cast<T*>(smem_raw);
  T* se = sa + XW * M;
  const int tx = threadIdx.x, m = threadIdx.y;
  const int x = blockIdx.x * XW + tx;
  const int64_t o = blockIdx.y, c = blockIdx.z;
  const int L = (n + M - 1) / M;
  const int s0 = m * L;
  int len = n - s0;
  len = len < 0 ? 0 : (len > L ? L : len);
  if (x >= nx) len = 0;
  const Tin* sp = src + s_off + c * s_sc + o * s_so + x + (int64_t)s0 * s_si;
  T* dp = dst + d_off + c * d_sc + o * d_so + x + (int64_t)s0 * d_si;
  const T thr = Thr<T>::v;

  // offsets inside a chunk fit in 32 bits (LMAX * stride < 2^31 for n <= 2048)
  const int si = (int)s_si, di = (int)d_si;
  T v[LMAX];
  if (len == LMAX) {
#pragma unroll
    for (int i = 0; i < LMAX; ++i) v[i] = (T)sp[i * si];
  } else {
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i < len) v[i] = (T)sp[i * si];
  }

  // causal sweep from a zero state; chunk carries by a geometric sum
  const T y = chunk_causal<T, LMAX>(v, len, z);
  const int me = m * XW + tx;
  sa[me] = chunk_zlen<T>(len);
  se[me] = y;
  __syncthreads();
  T carry = T(0), fac = T(1);
  int j = 1;
  for (; j <= M; ++j) {
    int idx = m - j;
    if (idx < 0) idx += M;
    const int k = idx * XW + tx;
    carry += fac * se[k];
    fac *= sa[k];
    if (fabs(fac) < thr) break;
  }
  if (j > M) carry = carry / (T(1) - fac);
  chunk_causal_fix<T, LMAX>(v, len, carry);
  __syncthreads();

  // anti-causal sweep from a zero state
  se[me] = chunk_anticausal<T, LMAX>(v, len, z);
  __syncthreads();
  carry = T(0);
  fac = T(1);
  for (j = 1; j <= M; ++j) {
    int idx = m + j;
    if (idx >= M) idx -= M;
    const int k = idx * XW + tx;
    carry += fac * se[k];
    fac *= sa[k];
    if (fabs(fac) < thr) break;
  }
  if (j > M) carry = carry / (T(1) - fac);
  chunk_anticausal_fix<T, LMAX>(v, len, carry, z);
  if (len == LMAX) {
#pragma unroll
    for (int i = 0; i < LMAX; ++i) dp[i * di] = gain * v[i];
  } else {
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i < len) dp[i * di] = gain * v[i];
  }
}

__device__ __forceinline__ float pow2_at_least(float mx) {
  if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
  int e;
  float f = frexpf(mx, &e);  // mx = f * 2^e, f in [0.5, 1)
  return f == 0.5f ? ldexpf(1.f, e - 1) : ldexpf(1.f, e);
}

// e + floor(e / L) for e < 32 (L + 1): (e + 1/2) / L is at least 1/(2L) away
// from an integer, far more than the FP32 rounding of the product, so the
// truncation is exact (checked exhaustively for L <= 128).
__device__ __forceinline__ int skew(int e, float inv_L) {
  return e + (int)(((float)e + 0.5f) * inv_L);
}
// The same index when every lane's chunk is full (L == LMAX, known at
// compile time): e + e / L, a shift for the power-of-two chunk lengths.
template <int LMAX>
__device__ __forceinline__ int skew_l(int e, int L, float inv_L) {
  return L == LMAX ? e + e / LMAX : skew(e, inv_L);
}

// x pass: one warp per x-line.  The line is staged in shared memory with a
// skew (element e at e + e/L) so that lane l reads its chunk [l L, l L + L)
// without bank conflicts; chunk carries move between lanes by shuffles.
// padded = 0: dst is an unpadded view.  padded = 1: dst is the padded
// coefficient array; every line is written to all its periodic images.
// The recursions of one periodic line held by a warp, lane l holding its
// chunk v[0..len) (the line's values [l L, l L + len)): causal and
// anti-causal, each with its chunk carries by shuffles; before the gain.
template <typename T, int LMAX>
__device__ __forceinline__ void line_recur(T (&v)[LMAX], int len, int lane, T z) {
  const unsigned FULL = 0xffffffffu;
  const T thr = Thr<T>::v;
  const T y = chunk_causal<T, LMAX>(v, len, z);
  const T a = chunk_zlen<T>(len);
  T carry = T(0), fac = T(1);
  bool wrapped = true;
  for (int j = 1; j <= 32; ++j) {
    const int sl = (lane - j) & 31;
    const T ej = __shfl_sync(FULL, y, sl);
    const T aj = __shfl_sync(FULL, a, sl);
    carry += fac * ej;
    fac *= aj;
    if (__all_sync(FULL, fabs(fac) < thr)) {
      wrapped = false;
      break;
    }
  }
  if (wrapped) carry = carry / (T(1) - fac);
  chunk_causal_fix<T, LMAX>(v, len, carry);

  const T w = chunk_anticausal<T, LMAX>(v, len, z);
  carry = T(0);
  fac = T(1);
  wrapped = true;
  for (int j = 1; j <= 32; ++j) {
    const int sl = (lane + j) & 31;
    const T fj = __shfl_sync(FULL, w, sl);
    const T aj = __shfl_sync(FULL, a, sl);
    carry += fac * fj;
    fac *= aj;
    if (__all_sync(FULL, fabs(fac) < thr)) {
      wrapped = false;
      break;
    }
  }
  if (wrapped) carry = carry / (T(1) - fac);
  chunk_anticausal_fix<T, LMAX>(v, len, carry, z);
}

// One periodic line of nx values held by a warp in its skewed shared buffer
// (element e at e + e/L): the recursions, times the gain.  With QUANT the
// values are divided by the line's power-of-two scale, which is returned.
template <typename T, int LMAX, bool QUANT>
__device__ __forceinline__ float line_solve(T* buf, int nx, int L, int lane, T z, T gain) {
  const unsigned FULL = 0xffffffffu;
  const int s0 = lane * L;
  int len = nx - s0;
  len = len < 0 ? 0 : (len > L ? L : len);
  T* mine = buf + lane * (L + 1);
  T v[LMAX];
  if (len == LMAX) {
#pragma unroll
    for (int i = 0; i < LMAX; ++i) v[i] = mine[i];
  } else {
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i < len) v[i] = mine[i];
  }
  line_recur<T, LMAX>(v, len, lane, z);

  float sc = 1.f;
  if (QUANT) {
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i < len) mx = fmaxf(mx, fabsf((float)(gain * v[i])));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, d));
    sc = pow2_at_least(mx);
  }
  const T inv_sc = (T)(1.f / sc);  // exact: sc is a power of two
  if (len == LMAX) {
#pragma unroll
    for (int i = 0; i < LMAX; ++i) mine[i] = gain * v[i] * inv_sc;
  } else {
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i < len) mine[i] = gain * v[i] * inv_sc;
  }
  __syncwarp();
  return sc;
}

template <typename T, typename Tout, int LMAX, bool QUANT>
__global__ void __launch_bounds__(256) solve_x(const T* src, View sv, Tout* dst, View dv,
                                               float* scale, int nx, int ny, int nz,
                                               int ncomp, int L, int padded, T z,
                                               T gain) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  T* buf = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 32 * (L + 1);
  // rows = ncomp * nz * ny <= 3 * 2048^2: 32-bit index arithmetic
  const int nrows = ncomp * nz * ny;
  const int row = (int)blockIdx.x * nwarps + warp;
  if (row >= nrows) return;  // whole warp; no block-level barrier below
  const int yy = row % ny;
  const int r2 = row / ny;
  const int zz = r2 % nz;
  const int c = r2 / nz;

  const float inv_L = 1.f / (float)L;
  const T* sp = src + sv.off + c * sv.sc + zz * sv.sz + yy * sv.sy;
  for (int e = lane; e < nx; e += 32) buf[skew_l<LMAX>(e, L, inv_L)] = sp[e];
  __syncwarp();
  const float sc = line_solve<T, LMAX, QUANT>(buf, nx, L, lane, z, gain);

  if (!padded) {
    Tout* orow = dst + dv.off + c * dv.sc + zz * dv.sz + yy * dv.sy;
    for (int e = lane; e < nx; e += 32) orow[e] = (Tout)buf[skew_l<LMAX>(e, L, inv_L)];
    return;
  }
  int pys[2], pzs[2];
  int npy = 1, npz = 1;
  pys[0] = yy + 1;
  if (yy == ny - 1) pys[npy++] = 0;
  else if (yy == 0) pys[npy++] = ny + 1;
  else if (yy == 1) pys[npy++] = ny + 2;
  pzs[0] = zz + 1;
  if (zz == nz - 1) pzs[npz++] = 0;
  else if (zz == 0) pzs[npz++] = nz + 1;
  else if (zz == 1) pzs[npz++] = nz + 2;
  for (int iz = 0; iz < npz; ++iz)
    for (int iy = 0; iy < npy; ++iy) {
      const int Pz = pzs[iz], Py = pys[iy];
      Tout* orow = dst + dv.off + c * dv.sc + Pz * dv.sz + Py * dv.sy;
      // the row pitch dv.sy >= nx + 3; the tail of the row is zeroed
      for (int P = lane; P < dv.sy; P += 32) {
        const int e = skew_l<LMAX>(padded_to_node(P, nx), L, inv_L);
        const T val = P < nx + 3 ? buf[e] : T(0);
        if constexpr (sizeof(T) == 8)
          orow[P] = cvt_out_d<Tout>((double)val);
        else
          orow[P] = cvt_out<Tout>((float)val);
      }
      if (QUANT && lane == 0) scale[((int64_t)c * (nz + 3) + Pz) * (ny + 3) + Py] = sc;
    }
}

// x pass writing node coefficients: a block of three warps takes one (z, y)
// line; warp c solves component c in its skewed buffer, then the block writes
// the padded row (rx nodes, the tail zero) and its periodic images as nodes
// (u, v, w, 0): float4, or 16-bit values divided by the power-of-two scale of
// their component's line, the scales stored as (s_u, s_v, s_w, 1) per row.
template <typename NodeT> struct NodeOut;
template <> struct NodeOut<float4> {
  static __device__ __forceinline__ float4 make(float a, float b, float c) {
    return make_float4(a, b, c, 0.f);
  }
};
template <typename H> struct NodeOut<Node16<H>> {
  static __device__ __forceinline__ Node16<H> make(float a, float b, float c) {
    Node16<H> n;
    n.v[0] = cvt_out<H>(a);
    n.v[1] = cvt_out<H>(b);
    n.v[2] = cvt_out<H>(c);
    n.v[3] = cvt_out<H>(0.f);
    return n;
  }
};

template <typename T, int LMAX, typename NodeT>
__global__ void __launch_bounds__(96) solve_x_node4(const T* src, View sv, NodeT* dst,
                                                    float* scale4, int64_t rx, int nx, int ny,
                                                    int nz, int L, T z, T gain) {
  constexpr bool Q = IsNode16<NodeT>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float line_scale[3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* buf = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 32 * (L + 1);
  const int yy = blockIdx.x, zz = blockIdx.y;  // one (z, y) row per block
  const float inv_L = 1.f / (float)L;
  const T* sp = src + sv.off + warp * sv.sc + zz * sv.sz + yy * sv.sy;
  for (int e = lane; e < nx; e += 32) buf[skew_l<LMAX>(e, L, inv_L)] = sp[e];
  __syncwarp();
  const float sc = line_solve<T, LMAX, Q>(buf, nx, L, lane, z, gain);
  if (lane == 0) line_scale[warp] = sc;
  __syncthreads();
  const T* b0 = reinterpret_cast<const T*>(smem_raw);
  const T* b1 = b0 + 32 * (L + 1);
  const T* b2 = b1 + 32 * (L + 1);
  int pys[2], pzs[2];
  int npy = 1, npz = 1;
  pys[0] = yy + 1;
  if (yy == ny - 1) pys[npy++] = 0;
  else if (yy == 0) pys[npy++] = ny + 1;
  else if (yy == 1) pys[npy++] = ny + 2;
  pzs[0] = zz + 1;
  if (zz == nz - 1) pzs[npz++] = 0;
  else if (zz == 0) pzs[npz++] = nz + 1;
  else if (zz == 1) pzs[npz++] = nz + 2;
  for (int iz = 0; iz < npz; ++iz)
    for (int iy = 0; iy < npy; ++iy) {
      const int64_t r = (int64_t)pzs[iz] * (ny + 3) + pys[iy];
      NodeT* orow = dst + r * rx;
      for (int P = threadIdx.x; P < rx; P += blockDim.x) {
        float a = 0.f, b = 0.f, c = 0.f;
        if (P < nx + 3) {
          const int e = skew_l<LMAX>(padded_to_node(P, nx), L, inv_L);
          a = (float)b0[e];
          b = (float)b1[e];
          c = (float)b2[e];
        }
        orow[P] = NodeOut<NodeT>::make(a, b, c);
      }
      if (Q && threadIdx.x < 4)
        scale4[r * 4 + threadIdx.x] = threadIdx.x < 3 ? line_scale[threadIdx.x] : 1.f;
    }
}

// ------------------------------------------------------------- wide lines ----
// x lines longer than a warp takes at 16 values a lane (nx > 512, FP32): W
// warps hold one line, 32 W lanes with chunks of L <= 16 values, the line in
// one skewed buffer (element e at e + e / L).  The chunk carries go through
// shared memory (cy, ca: one value per lane) with block barriers instead of
// shuffles; with QUANT the line's maximum is taken across its W warps
// (red[W]).  Every thread of the block calls it; returns the line's scale.
template <bool QUANT>
__device__ float line_solve_wide(float* buf, int nx, int L, int vl, int nvl, float z, float gain,
                                 float* cy, float* ca, float* red) {
  constexpr int LMAX = 16;
  const float thr = Thr<float>::v;
  int len = nx - vl * L;
  len = len < 0 ? 0 : (len > L ? L : len);
  float* mine = buf + vl * (L + 1);
  float v[LMAX];
  if (len == LMAX) {
#pragma unroll
    for (int i = 0; i < LMAX; ++i) v[i] = mine[i];
  } else {
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i < len) v[i] = mine[i];
  }
  const float y = chunk_causal<float, LMAX>(v, len, z);
  const float a = chunk_zlen<float>(len);
  cy[vl] = y;
  ca[vl] = a;
  __syncthreads();
  float carry = 0.f, fac = 1.f;
  bool wrapped = true;
  for (int j = 1; j <= nvl; ++j) {
    int sl = vl - j;
    if (sl < 0) sl += nvl;
    carry += fac * cy[sl];
    fac *= ca[sl];
    if (fabsf(fac) < thr) {
      wrapped = false;
      break;
    }
  }
  if (wrapped) carry = carry / (1.f - fac);
  chunk_causal_fix<float, LMAX>(v, len, carry);
  const float w = chunk_anticausal<float, LMAX>(v, len, z);
  __syncthreads();  // every lane has read the causal end states
  cy[vl] = w;
  __syncthreads();
  carry = 0.f;
  fac = 1.f;
  wrapped = true;
  for (int j = 1; j <= nvl; ++j) {
    int sl = vl + j;
    if (sl >= nvl) sl -= nvl;
    carry += fac * cy[sl];
    fac *= ca[sl];
    if (fabsf(fac) < thr) {
      wrapped = false;
      break;
    }
  }
  if (wrapped) carry = carry / (1.f - fac);
  chunk_anticausal_fix<float, LMAX>(v, len, carry, z);
  float sc = 1.f;
  if (QUANT) {
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i < len) mx = fmaxf(mx, fabsf(gain * v[i]));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
    if ((vl & 31) == 0) red[vl >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int k = 0; k < nvl / 32; ++k) mx = fmaxf(mx, red[k]);
    sc = pow2_at_least(mx);
  }
  const float inv_sc = 1.f / sc;  // exact: sc is a power of two
#pragma unroll
  for (int i = 0; i < LMAX; ++i)
    if (i < len) mine[i] = gain * v[i] * inv_sc;
  return sc;
}

// The planar x pass on wide lines: one (c, z, y) line per block of 32 W
// threads; writes as solve_x.  (e + 1/2) / L stays 1/(2L) from an integer,
// far above the FP32 rounding of the product for lines of 2^20 values, so
// skew() is exact here too.
template <typename Tout, bool QUANT>
__global__ void __launch_bounds__(512) solve_x_wide(const float* src, View sv, Tout* dst,
                                                    View dv, float* scale, int nx, int ny, int nz,
                                                    int L, int padded, float z, float gain) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x, nvl = blockDim.x;
  float* buf = reinterpret_cast<float*>(smem_raw);  // nvl (L + 1)
  float* cy = buf + nvl * (L + 1);
  float* ca = cy + nvl;
  float* red = ca + nvl;
  const int row = blockIdx.x;  // c * nz * ny + z * ny + y
  const int yy = row % ny, r2 = row / ny, zz = r2 % nz, c = r2 / nz;
  const float inv_L = 1.f / (float)L;
  const float* sp = src + sv.off + c * sv.sc + zz * sv.sz + yy * sv.sy;
  for (int e = t; e < nx; e += nvl) buf[skew(e, inv_L)] = sp[e];
  __syncthreads();
  const float sc = line_solve_wide<QUANT>(buf, nx, L, t, nvl, z, gain, cy, ca, red);
  __syncthreads();
  if (!padded) {
    Tout* orow = dst + dv.off + c * dv.sc + zz * dv.sz + yy * dv.sy;
    for (int e = t; e < nx; e += nvl) orow[e] = (Tout)buf[skew(e, inv_L)];
    return;
  }
  int Py[2], Pz[2];
  int npy = 1, npz = 1;
  Py[0] = yy + 1;
  if (yy == ny - 1) Py[npy++] = 0;
  else if (yy == 0) Py[npy++] = ny + 1;
  else if (yy == 1) Py[npy++] = ny + 2;
  Pz[0] = zz + 1;
  if (zz == nz - 1) Pz[npz++] = 0;
  else if (zz == 0) Pz[npz++] = nz + 1;
  else if (zz == 1) Pz[npz++] = nz + 2;
  for (int iz = 0; iz < npz; ++iz)
    for (int iy = 0; iy < npy; ++iy) {
      Tout* orow = dst + dv.off + c * dv.sc + Pz[iz] * dv.sz + Py[iy] * dv.sy;
      for (int P = t; P < dv.sy; P += nvl) {
        const float val = P < nx + 3 ? buf[skew(padded_to_node(P, nx), inv_L)] : 0.f;
        orow[P] = cvt_out<Tout>(val);
      }
      if (QUANT && t == 0) scale[((int64_t)c * (nz + 3) + Pz[iz]) * (ny + 3) + Py[iy]] = sc;
    }
}

// The node x pass on wide lines: one (z, y) row per block, W warps per
// component (96 W threads); writes as solve_x_node4.
template <typename NodeT>
__global__ void __launch_bounds__(768) solve_x_node4_wide(const float* src, View sv, NodeT* dst,
                                                          float* scale4, int64_t rx, int nx,
                                                          int ny, int nz, int L, float z,
                                                          float gain) {
  constexpr bool Q = IsNode16<NodeT>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float line_scale[3];
  const int nvl = blockDim.x / 3, comp = threadIdx.x / nvl, vl = threadIdx.x - comp * nvl;
  const int LB = nvl * (L + 1);
  float* base = reinterpret_cast<float*>(smem_raw);
  float* buf = base + comp * LB;                       // 3 lines
  float* cy = base + 3 * LB + comp * 2 * nvl;          // 3 x (cy, ca)
  float* ca = cy + nvl;
  float* red = base + 3 * LB + 6 * nvl + comp * (nvl / 32);
  const int yy = blockIdx.x, zz = blockIdx.y;
  const float inv_L = 1.f / (float)L;
  const float* sp = src + sv.off + comp * sv.sc + zz * sv.sz + yy * sv.sy;
  for (int e = vl; e < nx; e += nvl) buf[skew(e, inv_L)] = sp[e];
  __syncthreads();
  const float sc = line_solve_wide<Q>(buf, nx, L, vl, nvl, z, gain, cy, ca, red);
  if (vl == 0) line_scale[comp] = sc;
  __syncthreads();
  const float* b0 = base;
  const float* b1 = b0 + LB;
  const float* b2 = b1 + LB;
  int Py[2], Pz[2];
  int npy = 1, npz = 1;
  Py[0] = yy + 1;
  if (yy == ny - 1) Py[npy++] = 0;
  else if (yy == 0) Py[npy++] = ny + 1;
  else if (yy == 1) Py[npy++] = ny + 2;
  Pz[0] = zz + 1;
  if (zz == nz - 1) Pz[npz++] = 0;
  else if (zz == 0) Pz[npz++] = nz + 1;
  else if (zz == 1) Pz[npz++] = nz + 2;
  for (int iz = 0; iz < npz; ++iz)
    for (int iy = 0; iy < npy; ++iy) {
      const int64_t r = (int64_t)Pz[iz] * (ny + 3) + Py[iy];
      NodeT* orow = dst + r * rx;
      for (int P = threadIdx.x; P < rx; P += blockDim.x) {
        float a = 0.f, b = 0.f, c = 0.f;
        if (P < nx + 3) {
          const int e = skew(padded_to_node(P, nx), inv_L);
          a = b0[e];
          b = b1[e];
          c = b2[e];
        }
        orow[P] = NodeOut<NodeT>::make(a, b, c);
      }
      if (Q && threadIdx.x < 4)
        scale4[r * 4 + threadIdx.x] = threadIdx.x < 3 ? line_scale[threadIdx.x] : 1.f;
    }
}

// Wide-line geometry: W warps of chunks L (even, <= 16) for nx > 512.
struct WideGeo {
  int W, L;
};
WideGeo wide_geo(int nx) {
  WideGeo g;
  g.W = (nx + 511) / 512;
  const int L = (nx + 32 * g.W - 1) / (32 * g.W);
  g.L = L + (L & 1);
  return g;
}

// ------------------------------------------------------- two-pass solve ----
// The x and y solves of every (c, z) plane in one pass, the z solve in a
// second pass that writes the padded layout (planar, or (u, v, w, 0)
// nodes): the array is read twice and written twice instead of three times
// (the periodic images, a few faces, are copied after).
// A thread streams one pencil along the pass's axis in chunks of kSB lines:
//  * the causal recursion runs in order, from the state that a zero-start
//    sweep over the pencil's last kSB lines (chunk 0, read first) leaves;
//  * the anti-causal values of chunk q start from the value at chunk q+1's
//    first line of an anti-causal sweep entering chunk q+1's end at zero,
//    sum_i z^i y_i over chunk q+1's causal values y; in chunk q+1's raw
//    values g and the causal state s entering it that is
//    s A_len + sum_j g_j W_len[j], formed as the chunk arrives;
//  * the last chunk enters from the pencil's first line (that value, taken
//    from chunk 1) and hands its exact start on to the chunk before it.
// Each truncation drops terms below |z|^kSB = 7.2e-10 of the values beyond
// it (a geometric tail, at most 1e-9 relative): far below FP32 rounding, as
// the carry threshold of the chunked passes above.
// Chunks arrive through a ring of S shared-memory stages filled by 16-byte
// cp.async copies, S - 1 chunks ahead of the one in use (the wait is
// cp.async.wait_group's: no spinning); a thread keeps the causal values of
// the chunk before in registers.
constexpr int kSB = 16;

// W_len[j] = sum_{i=j}^{len-1} z^(2i-j), A_len = sum_{i<len} z^(2i+1) for
// len = 1..kSB (FP64 sums of the powers of z on the host).
__constant__ float c_sb_w[kSB + 1][kSB];
__constant__ float c_sb_a[kSB + 1];

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Chunk q of a streamed pencil of n >= 2 kSB lines: q = 0 is the warm-up
// (the last kSB lines), q >= 1 the lines [(q - 1) kSB, min(q kSB, n)).
__device__ __forceinline__ int sb_start(int q, int n) { return q == 0 ? n - kSB : (q - 1) * kSB; }
__device__ __forceinline__ int sb_len(int q, int n) {
  const int r = n - (q - 1) * kSB;
  return q == 0 ? kSB : (r < kSB ? r : kSB);
}

// The value entering the end of the chunk before this one: this chunk's raw
// values g (len of them), the causal state s entering it, a0 the value
// entering its own end.  Explicitly rounded operations keep every instance
// bit-identical.
__device__ __forceinline__ float sb_lookahead(const float (&g)[kSB], int len, float s, float a0) {
  float a;
  if (len == kSB) {  // every chunk but a pencil's last: weights by constant index
    a = __fmul_rn(s, c_sb_a[kSB]);
#pragma unroll
    for (int j = 0; j < kSB; ++j) a = __fmaf_rn(g[j], c_sb_w[kSB][j], a);
    return __fmaf_rn(zpow<float>(kSB), a0, a);
  }
  a = __fmul_rn(s, c_sb_a[len]);
#pragma unroll
  for (int j = 0; j < kSB; ++j)
    if (j < len) a = __fmaf_rn(g[j], c_sb_w[len][j], a);
  return __fmaf_rn(zpow<float>(len), a0, a);
}
// The causal recursion over a chunk, in place, from state s (updated).
__device__ __forceinline__ void sb_causal(float (&g)[kSB], int len, float z, float& s) {
  float y = s;
  if (len == kSB) {
#pragma unroll
    for (int j = 0; j < kSB; ++j) g[j] = y = __fmaf_rn(z, y, g[j]);
  } else {
#pragma unroll
    for (int j = 0; j < kSB; ++j)
      if (j < len) g[j] = y = __fmaf_rn(z, y, g[j]);
  }
  s = y;
}

// One pencil per thread, n >= 2 kSB lines, every thread of the block in
// step: copy(q) issues the block's copies of chunk q into stage q % S,
// read(q, g) takes this thread's raw values of chunk q from its stage,
// emit(q, y, len, w) runs the anti-causal recursion over chunk q's causal
// values from w and writes them, after(q, len) follows every emit (it may
// hold a block barrier).
template <int S, typename Copy, typename Read, typename Emit, typename After>
__device__ __forceinline__ void sb_stream(int n, float z, Copy copy, Read read, Emit emit,
                                          After after) {
  const int nq = (n + kSB - 1) / kSB;
#pragma unroll
  for (int q = 0; q < S - 1; ++q) {
    if (q <= nq) copy(q);
    cp_async_commit();
  }
  int next = S - 1;
  auto fetch = [&](int q, float (&g)[kSB]) {
    cp_async_wait<S - 2>();
    __syncthreads();  // chunk q is in; every thread has read chunk q - 1
    if (next <= nq) copy(next);  // into chunk q - 1's stage
    cp_async_commit();
    ++next;
    read(q, g);
  };
  float A[kSB], B[kSB];
  float s = 0.f;
  fetch(0, A);
  sb_causal(A, kSB, z, s);  // the warm-up leaves the state entering line 0
  fetch(1, B);
  const float s_wrap = sb_lookahead(B, kSB, s, 0.f);  // the value at line 0
  sb_causal(B, kSB, z, s);
  int q = 2;
  auto step = [&](float (&g)[kSB], float (&yp)[kSB]) {
    const int len = sb_len(q, n);
    fetch(q, g);
    const float a = sb_lookahead(g, len, s, q == nq ? s_wrap : 0.f);
    emit(q - 1, yp, kSB, a);
    after(q - 1, kSB);
    sb_causal(g, len, z, s);
    if (q == nq) {
      emit(q, g, len, s_wrap);
      after(q, len);
    }
    ++q;
  };
  for (;;) {
    step(A, B);
    if (q > nq) break;
    step(B, A);
    if (q > nq) break;
  }
  cp_async_wait<0>();
}

// Pass 1: one block per (c, z) plane of an unpadded array, nx = 32 LMAX
// (LMAX = 4, 8 or 16), one thread per x column, streaming y.  A stage holds
// kSB rows with x at x + 4 floor(x / 32): the 16-byte copies stay aligned, a
// lane's chunk of LMAX values is read and written as 16-byte accesses on
// distinct banks, and a warp's column reads fall on distinct banks.  Each
// chunk's rows are solved along x in place (a warp per row), then every
// thread takes its column through the y recursions and stores its outputs,
// coalesced across the warp.
template <int LMAX, int S>
__global__ void __launch_bounds__(32 * LMAX, 1024 / (32 * LMAX)) solve_xy_stream(
    const float* src, View sv, float* dst, View dv, int ny, int nz, float z, float gain) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NX = 32 * LMAX, T = NX, RP = NX + NX / 8;  // padded row
  constexpr int PR = NX / 4;                                // 16-byte pieces per row
  float* stage = reinterpret_cast<float*>(smem_raw);       // [S][kSB][RP]
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int c = blockIdx.x / nz, zz = blockIdx.x - c * nz;
  const float* sp = src + sv.off + c * sv.sc + zz * sv.sz;
  float* dp = dst + dv.off + c * dv.sc + zz * dv.sz + t;
  const int xcol = t + 4 * (t >> 5);                        // this thread's column
  const int xchunk = lane * LMAX + 4 * ((lane * LMAX) >> 5);  // this lane's chunk

  auto copy = [&](int q) {
    const int len = sb_len(q, ny);
    const float* g = sp + sb_start(q, ny) * sv.sy;
    float* st = stage + (q % S) * kSB * RP;
    const int m = t % PR;
#pragma unroll
    for (int j = t / PR; j < kSB; j += T / PR)
      if (j < len) cp_async16(st + j * RP + 4 * m + 4 * (m >> 3), g + j * sv.sy + 4 * m);
  };
  auto read = [&](int q, float (&g)[kSB]) {
    const int len = sb_len(q, ny);
    float* st = stage + (q % S) * kSB * RP;
    // the chunk's rows along x, in place
    for (int j = warp; j < len; j += T / 32) {
      float* row = st + j * RP + xchunk;
      float v[LMAX];
#pragma unroll
      for (int e = 0; e < LMAX; e += 4) {  // a chunk never straddles 32 values
        const float4 f = *reinterpret_cast<const float4*>(row + e);
        v[e] = f.x;
        v[e + 1] = f.y;
        v[e + 2] = f.z;
        v[e + 3] = f.w;
      }
      line_recur<float, LMAX>(v, LMAX, lane, z);
#pragma unroll
      for (int e = 0; e < LMAX; e += 4)
        *reinterpret_cast<float4*>(row + e) =
            make_float4(__fmul_rn(gain, v[e]), __fmul_rn(gain, v[e + 1]),
                        __fmul_rn(gain, v[e + 2]), __fmul_rn(gain, v[e + 3]));
    }
    __syncthreads();
    const float* col = st + xcol;
    if (len == kSB) {
#pragma unroll
      for (int j = 0; j < kSB; ++j) g[j] = col[j * RP];
    } else {
#pragma unroll
      for (int j = 0; j < kSB; ++j) g[j] = j < len ? col[j * RP] : 0.f;
    }
  };
  auto emit = [&](int qo, float (&y)[kSB], int len, float w) {
    float* o = dp + sb_start(qo, ny) * dv.sy;
    if (len == kSB) {
#pragma unroll
      for (int i = kSB - 1; i >= 0; --i) {
        w = __fmaf_rn(z, w, y[i]);
        o[i * dv.sy] = __fmul_rn(gain, w);
      }
    } else {
#pragma unroll
      for (int i = kSB - 1; i >= 0; --i)
        if (i < len) {
          w = __fmaf_rn(z, w, y[i]);
          o[i * dv.sy] = __fmul_rn(gain, w);
        }
    }
  };
  sb_stream<S>(ny, z, copy, read, emit, [](int, int) {});
}

// Output addressing of a line stream: element (c, line, other, x) at off +
// c sc + line sz + other sy + x sx floats (planar: sx = 1; nodes: c is the
// float in the node, sx = 4; into a padded layout, off points at its
// interior).
struct OutView {
  int64_t off, sc, sz, sy, sx;
};

// Lines along one axis of an unpadded array (nx a multiple of 4, rows
// 16-byte aligned): the source's line stride sv.sz, blockIdx.y the other
// axis at stride sv.sy; ZT columns of x per block, one thread per (column,
// component), streaming the nl lines.  It may write in place (a thread
// reads all of its pencil's lines before it writes them).  LPC = 1: one
// component, from blockIdx.z.  LPC = 4: nodes, four consecutive threads per
// column hold u, v, w and the zero fourth value (it reads u's values and
// stores zeros), so a warp stores eight whole nodes (128 bytes) per line.  A
// stage holds kSB lines of the block's columns per component (component
// blocks padded by 8 floats: the three components of a column fall on
// distinct banks).
template <int LPC, int ZT, int S>
__global__ void __launch_bounds__(ZT * LPC, 1024 / (ZT * LPC)) solve_line_stream(
    const float* src, View sv, float* dst, OutView ov, int nx, int nl, float z, float gain) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NCB = LPC == 1 ? 1 : 3;               // components per block
  constexpr int CS = kSB * ZT + (LPC == 1 ? 0 : 8);   // one component's lines
  constexpr int T = ZT * LPC, PL = ZT / 4;            // 16-byte pieces per line
  float* stage = reinterpret_cast<float*>(smem_raw);  // [S][NCB][CS]
  const int t = threadIdx.x;
  const int col = t / LPC, x0 = blockIdx.x * ZT, x = x0 + col;
  const int k = LPC == 1 ? 0 : t % LPC, c0 = LPC == 1 ? (int)blockIdx.z : 0;
  const bool pad = LPC == 4 && k == 3;
  const float* sp = src + sv.off + c0 * sv.sc + blockIdx.y * sv.sy + x0;
  const int sz = (int)ov.sz;  // < 2^31 elements per plane
  float* op = dst + ov.off + (c0 + k) * ov.sc + blockIdx.y * ov.sy + x * ov.sx;
  const float og = pad ? 0.f : gain;
  const bool xin = 4 * (t % PL) < nx - x0;

  // piece p = t + T u of a chunk: line (p / PL) % kSB of component
  // p / (PL kSB), 16 bytes at 4 (p % PL)
  auto copy = [&](int q) {
    const int len = sb_len(q, nl), r0 = sb_start(q, nl);
    float* st = stage + (q % S) * NCB * CS;
    if (!xin) return;
#pragma unroll
    for (int p = t; p < NCB * kSB * PL; p += T) {
      const int m = p % PL, j = (p / PL) % kSB, kk = p / (PL * kSB);
      if (j < len)
        cp_async16(st + kk * CS + j * ZT + 4 * m, sp + kk * sv.sc + (r0 + j) * sv.sz + 4 * m);
    }
  };
  auto read = [&](int q, float (&g)[kSB]) {
    const int len = sb_len(q, nl);
    const float* st = stage + (q % S) * NCB * CS + (pad ? 0 : k) * CS + col;
    if (len == kSB) {
#pragma unroll
      for (int j = 0; j < kSB; ++j) g[j] = st[j * ZT];
    } else {
#pragma unroll
      for (int j = 0; j < kSB; ++j) g[j] = j < len ? st[j * ZT] : 0.f;
    }
  };
  auto emit = [&](int qo, float (&y)[kSB], int len, float w) {
    if (x >= nx) return;
    float* rp = op + (int64_t)sb_start(qo, nl) * sz;
    if (len == kSB) {
#pragma unroll
      for (int i = kSB - 1; i >= 0; --i) {
        w = __fmaf_rn(z, w, y[i]);
        rp[i * sz] = pad ? 0.f : __fmul_rn(og, w);
      }
    } else {
#pragma unroll
      for (int i = kSB - 1; i >= 0; --i)
        if (i < len) {
          w = __fmaf_rn(z, w, y[i]);
          rp[i * sz] = pad ? 0.f : __fmul_rn(og, w);
        }
    }
  };
  sb_stream<S>(nl, z, copy, read, emit, [](int, int) {});
}

// The periodic images of a padded array whose interior is written: along
// each axis P = 0, n + 1, n + 2 holds the value at P = n, 1, 2 (node
// padded_to_node(P) + 1), and the row tail [nx + 3, rx) is zero.  E is
// float (planar, component blockIdx.y, stride cs) or float4 (nodes).
// fill_x_images: one thread per interior row, its three x images and tail.
template <typename E>
__global__ void fill_x_images(E* a, int64_t cs, int64_t rx, int nx, int ny, int nz) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= (int64_t)nz * ny) return;
  const int Pz = 1 + (int)(r / ny), Py = 1 + (int)(r % ny);
  E* row = a + blockIdx.y * cs + ((int64_t)Pz * (ny + 3) + Py) * rx;
  const E e0 = row[nx], e1 = row[1], e2 = row[2];
  row[0] = e0;
  row[nx + 1] = e1;
  row[nx + 2] = e2;
  for (int64_t P = nx + 3; P < rx; ++P) row[P] = E{};
}
// fill_yz_images: one block per row with Pz or Py in {0, n + 1, n + 2},
// copied whole from its interior row (every P mapped to the interior too,
// so it reads nothing fill_x_images writes).
template <typename E>
__global__ void fill_yz_images(E* a, int64_t cs, int64_t rx, int nx, int ny, int nz) {
  const int b = blockIdx.x, my = ny + 3;
  int Pz, Py;
  if (b < 3 * my) {
    const int gi = b / my;
    Pz = gi == 0 ? 0 : nz + gi;
    Py = b % my;
  } else {
    const int b2 = b - 3 * my, gi = b2 % 3;
    Pz = 1 + b2 / 3;
    Py = gi == 0 ? 0 : ny + gi;
  }
  const int sz_ = padded_to_node(Pz, nz) + 1, sy_ = padded_to_node(Py, ny) + 1;
  E* base = a + blockIdx.y * cs;
  E* row = base + ((int64_t)Pz * my + Py) * rx;
  const E* srow = base + ((int64_t)sz_ * my + sy_) * rx;
  for (int64_t P = threadIdx.x; P < rx; P += blockDim.x)
    row[P] = P < nx + 3 ? srow[padded_to_node((int)P, nx) + 1] : E{};
}

// ------------------------------------------------------------------ host ----

struct StridedCfg {
  int XW, M, lmax;
};

template <typename T>
StridedCfg strided_cfg(int n) {
  StridedCfg c;
  if (sizeof(T) == 8) {
    c.lmax = 16;
    c.M = (n + 15) / 16;
    c.XW = c.M <= 32 ? 16 : 8;
  } else if (n <= 512) {
    // 16-wide blocks: two or more blocks per SM overlap one another's
    // barriers and loads (measured 9% faster than 32-wide at 512^3)
    c.lmax = 16;
    c.M = (n + 15) / 16;
    c.XW = tuning().solve_xw > 0 ? tuning().solve_xw : 16;
  } else if (n <= 1024) {
    c.lmax = 32;
    c.M = (n + 31) / 32;
    c.XW = tuning().solve_xw > 0 ? tuning().solve_xw : 16;
  } else {
    c.lmax = 32;
    c.M = (n + 31) / 32;
    c.XW = 16;
  }
  return c;
}

template <typename Tin, typename T>
ps_status launch_strided(const Tin* src, View sv, int64_t s_so, int64_t s_si, T* dst,
                         View dv, int64_t d_so, int64_t d_si, int nx, int n,
                         int n_other, int ncomp, T z, T gain, cudaStream_t st) {
  StridedCfg cfg = strided_cfg<T>(n);
  if ((s_si > 0 ? s_si : -s_si) * cfg.lmax >= ((int64_t)1 << 31) ||
      (d_si > 0 ? d_si : -d_si) * cfg.lmax >= ((int64_t)1 << 31))
    return fail(PS_ERR_UNSUPPORTED, "line stride too large for one chunk");
  dim3 block(cfg.XW, cfg.M);
  dim3 grid((nx + cfg.XW - 1) / cfg.XW, n_other, ncomp);
  size_t smem = 2 * sizeof(T) * cfg.XW * cfg.M;
  if (cfg.lmax == 16)
    solve_strided<Tin, T, 16><<<grid, block, smem, st>>>(src, sv.off, sv.sc, s_so, s_si,
                                                         dst, dv.off, dv.sc, d_so, d_si,
                                                         nx, n, z, gain);
  else
    solve_strided<Tin, T, 32><<<grid, block, smem, st>>>(src, sv.off, sv.sc, s_so, s_si,
                                                         dst, dv.off, dv.sc, d_so, d_si,
                                                         nx, n, z, gain);
  return check_launch("solve_strided");
}

int x_chunk(int nx) {
  int L = (nx + 31) / 32;
  return L + (L & 1);  // even: odd row stride L+1 keeps lanes on distinct banks
}

template <typename T, typename Tout, bool QUANT, int LMAX>
ps_status launch_x_l(const T* src, View sv, Tout* dst, View dv, float* scale, int nx,
                     int ny, int nz, int ncomp, int L, int padded, T z, T gain,
                     cudaStream_t st) {
  const int warps = sizeof(T) == 8 && L > 16 ? 4 : 8;
  size_t smem = (size_t)warps * 32 * (L + 1) * sizeof(T);
  auto kern = solve_x<T, Tout, LMAX, QUANT>;
  if (smem > 48 * 1024) {
    ps_status rc = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "solve_x smem attribute");
    if (rc) return rc;
  }
  int64_t rows = (int64_t)ncomp * nz * ny;
  int64_t blocks = (rows + warps - 1) / warps;
  kern<<<(unsigned)blocks, warps * 32, smem, st>>>(src, sv, dst, dv, scale, nx, ny, nz,
                                                   ncomp, L, padded, z, gain);
  return check_launch("solve_x");
}

template <typename T, typename Tout, bool QUANT>
ps_status launch_x(const T* src, View sv, Tout* dst, View dv, float* scale, int nx,
                   int ny, int nz, int ncomp, int padded, T z, T gain, cudaStream_t st) {
  const int L = x_chunk(nx);
  if constexpr (sizeof(T) == 4) {
    if (L > 16) {  // wide lines: W warps per line
      const WideGeo wg = wide_geo(nx);
      const int nvl = 32 * wg.W;
      const size_t smem = ((size_t)nvl * (wg.L + 1) + 2 * nvl + wg.W) * sizeof(float);
      auto kern = solve_x_wide<Tout, QUANT>;
      if (smem > 48 * 1024) {
        ps_status rc = check_cuda(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "solve_x_wide smem attribute");
        if (rc) return rc;
      }
      const int64_t rows = (int64_t)ncomp * nz * ny;
      kern<<<(unsigned)rows, nvl, smem, st>>>(src, sv, dst, dv, scale, nx, ny, nz, wg.L, padded,
                                              z, gain);
      return check_launch("solve_x_wide");
    }
  }
  if (L <= 2)
    return launch_x_l<T, Tout, QUANT, 2>(src, sv, dst, dv, scale, nx, ny, nz, ncomp, L,
                                          padded, z, gain, st);
  if (L <= 4)
    return launch_x_l<T, Tout, QUANT, 4>(src, sv, dst, dv, scale, nx, ny, nz, ncomp, L,
                                          padded, z, gain, st);
  if (L <= 8)
    return launch_x_l<T, Tout, QUANT, 8>(src, sv, dst, dv, scale, nx, ny, nz, ncomp, L,
                                          padded, z, gain, st);
  if (L <= 16)
    return launch_x_l<T, Tout, QUANT, 16>(src, sv, dst, dv, scale, nx, ny, nz, ncomp, L,
                                           padded, z, gain, st);
  if constexpr (sizeof(T) == 8) {
    if (L <= 32)
      return launch_x_l<T, Tout, QUANT, 32>(src, sv, dst, dv, scale, nx, ny, nz, ncomp, L,
                                             padded, z, gain, st);
  }
  return fail(PS_ERR_UNSUPPORTED, "FP64 solve supports n <= 1024");
}

template <int LMAX, typename NodeT>
ps_status launch_x_node4_l(const float* src, View sv, NodeT* dst, float* scale4, int64_t rx,
                           int nx, int ny, int nz, int L, float z, float gain, cudaStream_t st) {
  const size_t smem = (size_t)3 * 32 * (L + 1) * sizeof(float);
  auto kern = solve_x_node4<float, LMAX, NodeT>;
  if (smem > 48 * 1024) {
    ps_status rc = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "solve_x_node4 smem attribute");
    if (rc) return rc;
  }
  kern<<<dim3((unsigned)ny, (unsigned)nz), 96, smem, st>>>(src, sv, dst, scale4, rx, nx, ny,
                                                             nz, L, z, gain);
  return check_launch("solve_x_node4");
}

template <typename NodeT>
ps_status launch_x_node4(const float* src, View sv, NodeT* dst, float* scale4, int64_t rx,
                         int nx, int ny, int nz, float z, float gain, cudaStream_t st) {
  const int L = x_chunk(nx);
  if (L <= 2) return launch_x_node4_l<2>(src, sv, dst, scale4, rx, nx, ny, nz, L, z, gain, st);
  if (L <= 4) return launch_x_node4_l<4>(src, sv, dst, scale4, rx, nx, ny, nz, L, z, gain, st);
  if (L <= 8) return launch_x_node4_l<8>(src, sv, dst, scale4, rx, nx, ny, nz, L, z, gain, st);
  if (L <= 16)
    return launch_x_node4_l<16>(src, sv, dst, scale4, rx, nx, ny, nz, L, z, gain, st);
  // wide lines: W warps per component
  const WideGeo wg = wide_geo(nx);
  const int nvl = 32 * wg.W;
  const size_t smem = ((size_t)3 * nvl * (wg.L + 1) + 6 * nvl + 3 * wg.W) * sizeof(float);
  auto kern = solve_x_node4_wide<NodeT>;
  if (smem > 48 * 1024) {
    ps_status rc = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "solve_x_node4_wide smem attribute");
    if (rc) return rc;
  }
  kern<<<dim3((unsigned)ny, (unsigned)nz), 3 * nvl, smem, st>>>(src, sv, dst, scale4, rx, nx, ny,
                                                                  nz, wg.L, z, gain);
  return check_launch("solve_x_node4_wide");
}

// Two-pass solve: applies to FP32 fields and FP32 coefficients (planar or
// nodes) when a row is 128, 256 or 512 values (a warp's chunks of 4, 8 or
// 16) and every streamed pencil holds two chunks (tune "solve_stream" 0
// keeps the three passes).  It needs the unpadded FP32 intermediate in the
// workspace.
bool stream_grid(const ps_grid* g) {
  const int nx = g->n[0];
  return (nx == 128 || nx == 256 || nx == 512) && g->n[1] >= 2 * kSB && g->n[2] >= 2 * kSB;
}
bool stream_solve_ok(const ps_grid* g) {
  return tuning().solve_stream && stream_grid(g);
}

template <int LMAX, int S>
ps_status launch_xy_stream_s(const float* src, View sv, float* dst, View dv, int ny, int nz,
                             int ncomp, float z, float gain, cudaStream_t st) {
  constexpr int NX = 32 * LMAX;
  const size_t smem = (size_t)S * kSB * (NX + NX / 8) * sizeof(float);
  auto kern = solve_xy_stream<LMAX, S>;
  if (smem > 48 * 1024) {
    ps_status rc = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "solve_xy_stream smem attribute");
    if (rc) return rc;
  }
  kern<<<(unsigned)(ncomp * nz), NX, smem, st>>>(src, sv, dst, dv, ny, nz, z, gain);
  return check_launch("solve_xy_stream");
}

template <int LMAX>
ps_status launch_xy_stream_l(const float* src, View sv, float* dst, View dv, int ny, int nz,
                             int ncomp, float z, float gain, cudaStream_t st) {
  const int S = tuning().solve_stages > 0 ? tuning().solve_stages : 3;
  if (S == 2) return launch_xy_stream_s<LMAX, 2>(src, sv, dst, dv, ny, nz, ncomp, z, gain, st);
  if (S == 4) return launch_xy_stream_s<LMAX, 4>(src, sv, dst, dv, ny, nz, ncomp, z, gain, st);
  return launch_xy_stream_s<LMAX, 3>(src, sv, dst, dv, ny, nz, ncomp, z, gain, st);
}

// nx = 128, 256 or 512 (stream_grid)
ps_status launch_xy_stream(const float* src, View sv, float* dst, View dv, int nx, int ny,
                           int nz, int ncomp, float z, float gain, cudaStream_t st) {
  if (nx == 128) return launch_xy_stream_l<4>(src, sv, dst, dv, ny, nz, ncomp, z, gain, st);
  if (nx == 256) return launch_xy_stream_l<8>(src, sv, dst, dv, ny, nz, ncomp, z, gain, st);
  return launch_xy_stream_l<16>(src, sv, dst, dv, ny, nz, ncomp, z, gain, st);
}

template <int LPC, int ZT>
ps_status launch_line_stream_t(const float* src, View sv, float* dst, OutView ov, int nx,
                               int nother, int nl, int cblocks, float z, float gain,
                               cudaStream_t st) {
  constexpr int S = 4;
  const size_t smem = (size_t)S * (LPC == 1 ? 1 : 3) * (kSB * ZT + (LPC == 1 ? 0 : 8)) * 4;
  auto kern = solve_line_stream<LPC, ZT, S>;
  if (smem > 48 * 1024) {
    ps_status rc = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "solve_line_stream smem attribute");
    if (rc) return rc;
  }
  dim3 grid((unsigned)((nx + ZT - 1) / ZT), (unsigned)nother, (unsigned)cblocks);
  kern<<<grid, ZT * LPC, smem, st>>>(src, sv, dst, ov, nx, nl, z, gain);
  return check_launch("solve_line_stream");
}

// nother lines of nl values (the other axis at blockIdx.y); cblocks:
// components (LPC = 1) or 1 (nodes, LPC = 4).
template <int LPC>
ps_status launch_line_stream(const float* src, View sv, float* dst, OutView ov, int nx,
                             int nother, int nl, int cblocks, float z, float gain,
                             cudaStream_t st) {
  // measured at 512^3: one component 256 columns per block, nodes 64 (256 threads)
  const int zt = tuning().solve_zt > 0 ? tuning().solve_zt : (LPC == 1 ? 256 : 64);
#define PS_LS(L, Z) \
  return launch_line_stream_t<L, Z>(src, sv, dst, ov, nx, nother, nl, cblocks, z, gain, st)
  if (LPC == 1) {
    if (zt <= 32) PS_LS(1, 32);
    if (zt <= 64) PS_LS(1, 64);
    if (zt <= 128) PS_LS(1, 128);
    PS_LS(1, 256);
  }
  if (zt <= 16) PS_LS(4, 16);
  if (zt <= 32) PS_LS(4, 32);
  PS_LS(4, 64);
#undef PS_LS
}

// The periodic images and row tails of a padded array whose interior is
// written; ncomp arrays cs elements apart.
template <typename E>
ps_status launch_fill_images(E* a, int64_t cs, int64_t rx, int nx, int ny, int nz, int ncomp,
                             cudaStream_t st) {
  const int64_t rows = (int64_t)nz * ny;
  fill_x_images<E><<<dim3((unsigned)((rows + 255) / 256), (unsigned)ncomp), 256, 0, st>>>(
      a, cs, rx, nx, ny, nz);
  ps_status rc = check_launch("fill_x_images");
  if (rc) return rc;
  fill_yz_images<E><<<dim3((unsigned)(3 * (ny + 3) + 3 * nz), (unsigned)ncomp), 128, 0, st>>>(
      a, cs, rx, nx, ny, nz);
  return check_launch("fill_yz_images");
}

// Fill the constant tables of z^k once per device (the host's FP64 z).
ps_status upload_zpow(double zd) {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  ps_status rc = check_cuda(cudaGetDevice(&dev), "get device");
  if (rc) return rc;
  if (dev < 0 || dev >= 64) return fail(PS_ERR_UNSUPPORTED, "device index %d", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return PS_OK;
  double pd[65];
  float pf[65];
  pd[0] = 1.0;
  for (int k = 1; k <= 64; ++k) pd[k] = pd[k - 1] * zd;
  for (int k = 0; k <= 64; ++k) pf[k] = (float)pd[k];
  if ((rc = check_cuda(cudaMemcpyToSymbol(c_zpow_d, pd, sizeof(pd)), "z powers (FP64)"))) return rc;
  if ((rc = check_cuda(cudaMemcpyToSymbol(c_zpow_f, pf, sizeof(pf)), "z powers (FP32)"))) return rc;
  // the streamed passes' look-ahead weights (index 0 unused)
  float w[kSB + 1][kSB] = {}, a[kSB + 1] = {};
  for (int len = 1; len <= kSB; ++len) {
    double sa = 0.0;
    for (int i = 0; i < len; ++i) sa += pd[2 * i + 1];
    a[len] = (float)sa;
    for (int j = 0; j < len; ++j) {
      double sw = 0.0;
      for (int i = j; i < len; ++i) sw += pd[2 * i - j];
      w[len][j] = (float)sw;
    }
  }
  if ((rc = check_cuda(cudaMemcpyToSymbol(c_sb_w, w, sizeof(w)), "look-ahead weights"))) return rc;
  if ((rc = check_cuda(cudaMemcpyToSymbol(c_sb_a, a, sizeof(a)), "look-ahead state weights")))
    return rc;
  done[dev] = true;
  return PS_OK;
}

View unpadded_view(const ps_grid* g) {
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  return View{0, nx * ny * nz, nx * ny, nx};
}
// Padded coefficient array with row pitch `rx` elements.
View padded_view(const ps_grid* g, int64_t rx) {
  const int64_t my = g->n[1] + 3, mz = g->n[2] + 3;
  return View{0, rx * my * mz, rx * my, rx};
}
View interior_view(const ps_grid* g, int64_t rx) {
  View v = padded_view(g, rx);
  v.off = v.sz + v.sy + 1;
  return v;
}

// FP32 field -> padded planar FP32 coefficients: the x-y pass into the
// unpadded workspace, the z pass into the padded layout's interior, then its
// periodic images.
ps_status run_solve_stream_planar(const ps_grid* g, int ncomp, const float* field, float* inter,
                                  float* coef, int64_t rx, cudaStream_t st) {
  const double zd = sqrt(3.0) - 2.0;
  if (ps_status zrc = upload_zpow(zd)) return zrc;
  const float z = (float)zd, gain = (float)(-6.0 * zd);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  View fv = unpadded_view(g), pv = padded_view(g, rx);
  ps_status rc = launch_xy_stream(field, fv, inter, fv, nx, ny, nz, ncomp, z, gain, st);
  if (rc) return rc;
  OutView ov{pv.off + pv.sz + pv.sy + 1, pv.sc, pv.sz, pv.sy, 1};  // the interior
  rc = launch_line_stream<1>(inter, fv, coef, ov, nx, ny, nz, ncomp, z, gain, st);
  if (rc) return rc;
  return launch_fill_images<float>(coef, pv.sc, rx, nx, ny, nz, ncomp, st);
}

// FP32 field -> FP32 nodes: the x-y pass into the unpadded workspace, the z
// pass over the three components writing (u, v, w, 0) nodes, then the
// periodic images.
ps_status run_solve_stream_node4(const ps_grid* g, const float* field, float* inter,
                                 float4* out, int64_t rx, cudaStream_t st) {
  const double zd = sqrt(3.0) - 2.0;
  if (ps_status zrc = upload_zpow(zd)) return zrc;
  const float z = (float)zd, gain = (float)(-6.0 * zd);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  View fv = unpadded_view(g);
  ps_status rc = launch_xy_stream(field, fv, inter, fv, nx, ny, nz, 3, z, gain, st);
  if (rc) return rc;
  const int64_t my = ny + 3;
  OutView ov{(my * rx + rx + 1) * 4, 1, my * rx * 4, rx * 4, 4};  // the interior
  rc = launch_line_stream<4>(inter, fv, reinterpret_cast<float*>(out), ov, nx, ny, nz, 1, z,
                             gain, st);
  if (rc) return rc;
  return launch_fill_images<float4>(out, 0, rx, nx, ny, nz, 1, st);
}

// The y and z passes of the three-pass solve as line streams (FP32, an
// unpadded intermediate with 16-byte rows, ny and nz >= 32): y from the
// field into the intermediate (or in place), then z in place.
bool stream3_grid(const ps_grid* g) {
  return g->n[0] % 4 == 0 && g->n[1] >= 2 * kSB && g->n[2] >= 2 * kSB;
}
ps_status run_yz_streams(const ps_grid* g, int ncomp, const float* field, float* inter,
                         float z, float gain, cudaStream_t st) {
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int64_t cs = nx * ny * nz;
  const View yv{0, cs, nx, nx * ny};  // lines along y, the other axis z
  const OutView yo{0, cs, nx, nx * ny, 1};
  ps_status rc = launch_line_stream<1>(field, yv, inter, yo, (int)nx, (int)nz, (int)ny, ncomp,
                                       z, gain, st);
  if (rc) return rc;
  const View zv{0, cs, nx * ny, nx};  // lines along z, the other axis y
  const OutView zo{0, cs, nx * ny, nx, 1};
  return launch_line_stream<1>(inter, zv, inter, zo, (int)nx, (int)ny, (int)nz, ncomp, z, gain,
                               st);
}

// y pass (src -> dst), z pass (in place on dst), x pass (dst -> out).  With
// FP32 throughout, an unpadded intermediate and the grid stream3_grid takes,
// the y and z passes are line streams.
template <typename Tin, typename T, typename Tout, bool QUANT>
ps_status run_solve(const ps_grid* g, int ncomp, const Tin* field, View fv, T* inter,
                    View iv, Tout* out, View ov, float* scale, int padded,
                    cudaStream_t st) {
  const double zd = sqrt(3.0) - 2.0;
  if (ps_status zrc = upload_zpow(zd)) return zrc;
  const T z = (T)zd, gain = (T)(-6.0 * zd);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  ps_status rc = PS_OK;
  bool streamed = false;
  if constexpr (std::is_same<Tin, float>::value && std::is_same<T, float>::value) {
    const bool unpadded = iv.off == 0 && iv.sy == nx && iv.sz == (int64_t)nx * ny;
    const bool aligned = ((reinterpret_cast<uintptr_t>(field) | reinterpret_cast<uintptr_t>(inter)) &
                          15) == 0;
    if (tuning().solve_stream && stream3_grid(g) && unpadded && aligned) {
      rc = run_yz_streams(g, ncomp, field, inter, z, gain, st);
      streamed = true;
    }
  }
  if (!streamed) {
    rc = launch_strided<Tin, T>(field, fv, fv.sz, fv.sy, inter, iv, iv.sz, iv.sy, nx, ny, nz,
                                ncomp, z, gain, st);
    if (rc) return rc;
    rc = launch_strided<T, T>(inter, iv, iv.sy, iv.sz, inter, iv, iv.sy, iv.sz, nx, nz, ny,
                              ncomp, z, gain, st);
  }
  if (rc) return rc;
  return launch_x<T, Tout, QUANT>(inter, iv, out, ov, scale, nx, ny, nz, ncomp, padded, z,
                                  gain, st);
}

// y and z passes into the unpadded FP32 workspace, then the node x pass.
template <typename Tin, typename NodeT>
ps_status run_solve_node4(const ps_grid* g, const Tin* field, View fv, float* inter,
                          NodeT* out, float* scale4, int64_t rx, cudaStream_t st) {
  const double zd = sqrt(3.0) - 2.0;
  if (ps_status zrc = upload_zpow(zd)) return zrc;
  const float z = (float)zd, gain = (float)(-6.0 * zd);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  ps_status rc = PS_OK;
  bool streamed = false;
  if constexpr (std::is_same<Tin, float>::value) {
    if (tuning().solve_stream && stream3_grid(g) &&
        ((reinterpret_cast<uintptr_t>(field) | reinterpret_cast<uintptr_t>(inter)) & 15) == 0) {
      rc = run_yz_streams(g, 3, field, inter, z, gain, st);
      streamed = true;
    }
  }
  if (!streamed) {
    rc = launch_strided<Tin, float>(field, fv, fv.sz, fv.sy, inter, fv, fv.sz, fv.sy, nx, ny, nz,
                                    3, z, gain, st);
    if (rc) return rc;
    rc = launch_strided<float, float>(inter, fv, fv.sy, fv.sz, inter, fv, fv.sy, fv.sz, nx, nz,
                                      ny, 3, z, gain, st);
  }
  if (rc) return rc;
  return launch_x_node4(inter, fv, out, scale4, rx, nx, ny, nz, z, gain, st);
}

}  // namespace

ps_status solve_unpadded_inplace_f32(const ps_grid* g, int ncomp, float* a,
                                     cudaStream_t st) {
  View v = unpadded_view(g);
  return run_solve<float, float, float, false>(g, ncomp, a, v, a, v, a, v, nullptr, 0, st);
}

}  // namespace ps

using namespace ps;

extern "C" size_t ps_spline_coeffs_workspace_size(const ps_grid* grid, int ncomp,
                                                  ps_dtype coef_t) {
  if (!grid || ncomp < 1) return 0;
  if (coef_t == PS_BF16 || coef_t == PS_F16 || coef_t == PS_F32X4 || coef_t == PS_BF16X4 ||
      coef_t == PS_F16X4 ||
      (coef_t == PS_F32 && validate_grid(grid) == PS_OK && (stream_grid(grid) || stream3_grid(grid))))
    return align_up((size_t)ncomp * (size_t)grid_volume(grid) * sizeof(float), 256) + 256;
  return 0;
}

extern "C" ps_status ps_spline_coeffs(const ps_grid* grid, int ncomp, ps_dtype field_t,
                                      const void* field, ps_dtype coef_t, void* coef,
                                      float* scale, void* ws, size_t ws_bytes,
                                      void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  if (ncomp < 1 || ncomp > 16) return fail(PS_ERR_INVALID_ARG, "ncomp=%d outside [1,16]", ncomp);
  if (!field || !coef) return fail(PS_ERR_INVALID_ARG, "field and coef must be non-NULL");
  if (field_t != PS_F32 && field_t != PS_F64)
    return fail(PS_ERR_INVALID_ARG, "field dtype must be F32 or F64");
  const bool node = coef_t == PS_F32X4 || coef_t == PS_BF16X4 || coef_t == PS_F16X4;
  const bool quant = coef_t == PS_BF16 || coef_t == PS_F16 || coef_t == PS_BF16X4 ||
                     coef_t == PS_F16X4;
  if (coef_t != PS_F32 && coef_t != PS_F64 && !node && !quant)
    return fail(PS_ERR_INVALID_ARG, "bad coef dtype");
  if (node && ncomp != 3)
    return fail(PS_ERR_INVALID_ARG, "node coefficients need ncomp == 3");
  if (quant && !scale) return fail(PS_ERR_INVALID_ARG, "scale required for BF16/F16");
  if (coef_t == PS_F64)
    for (int d = 0; d < 3; ++d)
      if (grid->n[d] > 1024) return fail(PS_ERR_UNSUPPORTED, "FP64 coefficients need n <= 1024");
  cudaStream_t st = as_stream(stream);
  const int64_t rx = coef_pitch(grid->n[0], coef_t);
  const View fv = unpadded_view(grid), pv = padded_view(grid, rx), iv = interior_view(grid, rx);
  const float* ff = static_cast<const float*>(field);
  const double* fd = static_cast<const double*>(field);

  const bool aligned16 = (reinterpret_cast<uintptr_t>(field) & 15) == 0;
  if (coef_t == PS_F32) {
    float* c = static_cast<float*>(coef);
    // the two-pass solve when the workspace holds its intermediate, else
    // the three passes in place
    const size_t inter_bytes = (size_t)ncomp * (size_t)grid_volume(grid) * sizeof(float);
    const bool have_ws = ws && ws_bytes >= inter_bytes && (reinterpret_cast<uintptr_t>(ws) & 255) == 0;
    if (field_t == PS_F32 && stream_solve_ok(grid) && aligned16 && have_ws)
      return run_solve_stream_planar(grid, ncomp, ff, static_cast<float*>(ws), c, rx, st);
    if (field_t == PS_F32 && tuning().solve_stream && stream3_grid(grid) && aligned16 && have_ws)
      return run_solve<float, float, float, false>(grid, ncomp, ff, fv, static_cast<float*>(ws),
                                                   fv, c, pv, nullptr, 1, st);
    return field_t == PS_F32
               ? run_solve<float, float, float, false>(grid, ncomp, ff, fv, c, iv, c, pv,
                                                       nullptr, 1, st)
               : run_solve<double, float, float, false>(grid, ncomp, fd, fv, c, iv, c, pv,
                                                        nullptr, 1, st);
  }
  if (coef_t == PS_F64) {
    double* c = static_cast<double*>(coef);
    return field_t == PS_F32
               ? run_solve<float, double, double, false>(grid, ncomp, ff, fv, c, iv, c, pv,
                                                         nullptr, 1, st)
               : run_solve<double, double, double, false>(grid, ncomp, fd, fv, c, iv, c,
                                                          pv, nullptr, 1, st);
  }
  // quantised or node output: FP32 intermediate in the workspace
  size_t need = ps_spline_coeffs_workspace_size(grid, ncomp, coef_t);
  if (!ws || ws_bytes < need - 256 || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(PS_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need - 256);
  float* inter = static_cast<float*>(ws);
  if (coef_t == PS_F32X4) {
    float4* c = static_cast<float4*>(coef);
    if (field_t == PS_F32 && stream_solve_ok(grid) && aligned16)
      return run_solve_stream_node4(grid, ff, inter, c, rx, st);
    return field_t == PS_F32 ? run_solve_node4<float>(grid, ff, fv, inter, c, nullptr, rx, st)
                             : run_solve_node4<double>(grid, fd, fv, inter, c, nullptr, rx, st);
  }
  if (coef_t == PS_BF16X4) {
    bf16x4* c = static_cast<bf16x4*>(coef);
    return field_t == PS_F32 ? run_solve_node4<float>(grid, ff, fv, inter, c, scale, rx, st)
                             : run_solve_node4<double>(grid, fd, fv, inter, c, scale, rx, st);
  }
  if (coef_t == PS_F16X4) {
    f16x4* c = static_cast<f16x4*>(coef);
    return field_t == PS_F32 ? run_solve_node4<float>(grid, ff, fv, inter, c, scale, rx, st)
                             : run_solve_node4<double>(grid, fd, fv, inter, c, scale, rx, st);
  }
  if (coef_t == PS_BF16) {
    __nv_bfloat16* c = static_cast<__nv_bfloat16*>(coef);
    return field_t == PS_F32
               ? run_solve<float, float, __nv_bfloat16, true>(grid, ncomp, ff, fv, inter,
                                                              fv, c, pv, scale, 1, st)
               : run_solve<double, float, __nv_bfloat16, true>(grid, ncomp, fd, fv, inter,
                                                               fv, c, pv, scale, 1, st);
  }
  __half* c = static_cast<__half*>(coef);
  return field_t == PS_F32
             ? run_solve<float, float, __half, true>(grid, ncomp, ff, fv, inter, fv, c, pv,
                                                     scale, 1, st)
             : run_solve<double, float, __half, true>(grid, ncomp, fd, fv, inter, fv, c, pv,
                                                      scale, 1, st);
}
