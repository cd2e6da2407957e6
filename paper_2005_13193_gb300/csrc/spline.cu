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
// Passes: y, then z (strided: threads along x read coalesced rows), then x
// (one warp per row, staged through shared memory), which writes the padded
// N+3 layout with periodic ghosts and, for BF16/FP16, a power-of-two scale per
// x-line.
#include <mutex>

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
// One periodic line of nx values held by a warp in its skewed shared buffer
// (element e at e + e/L): the causal and anti-causal recursions with their
// chunk carries, times the gain.  With QUANT the values are divided by the
// line's power-of-two scale, which is returned.
template <typename T, int LMAX, bool QUANT>
__device__ __forceinline__ float line_solve(T* buf, int nx, int L, int lane, T z, T gain) {
  const unsigned FULL = 0xffffffffu;
  const T thr = Thr<T>::v;
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
  if (L <= 32)
    return launch_x_l<T, Tout, QUANT, 32>(src, sv, dst, dv, scale, nx, ny, nz, ncomp, L,
                                           padded, z, gain, st);
  if constexpr (sizeof(T) == 4)
    return launch_x_l<T, Tout, QUANT, 64>(src, sv, dst, dv, scale, nx, ny, nz, ncomp, L,
                                           padded, z, gain, st);
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
  if (L <= 32)
    return launch_x_node4_l<32>(src, sv, dst, scale4, rx, nx, ny, nz, L, z, gain, st);
  return launch_x_node4_l<64>(src, sv, dst, scale4, rx, nx, ny, nz, L, z, gain, st);
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

// y pass (src -> dst), z pass (in place on dst), x pass (dst -> out).
template <typename Tin, typename T, typename Tout, bool QUANT>
ps_status run_solve(const ps_grid* g, int ncomp, const Tin* field, View fv, T* inter,
                    View iv, Tout* out, View ov, float* scale, int padded,
                    cudaStream_t st) {
  const double zd = sqrt(3.0) - 2.0;
  if (ps_status zrc = upload_zpow(zd)) return zrc;
  const T z = (T)zd, gain = (T)(-6.0 * zd);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  ps_status rc = launch_strided<Tin, T>(field, fv, fv.sz, fv.sy, inter, iv, iv.sz, iv.sy,
                                        nx, ny, nz, ncomp, z, gain, st);
  if (rc) return rc;
  rc = launch_strided<T, T>(inter, iv, iv.sy, iv.sz, inter, iv, iv.sy, iv.sz, nx, nz, ny,
                            ncomp, z, gain, st);
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
  ps_status rc = launch_strided<Tin, float>(field, fv, fv.sz, fv.sy, inter, fv, fv.sz, fv.sy,
                                            nx, ny, nz, 3, z, gain, st);
  if (rc) return rc;
  rc = launch_strided<float, float>(inter, fv, fv.sy, fv.sz, inter, fv, fv.sy, fv.sz, nx, nz, ny,
                                    3, z, gain, st);
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
      coef_t == PS_F16X4)
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

  if (coef_t == PS_F32) {
    float* c = static_cast<float*>(coef);
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
