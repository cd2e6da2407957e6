// Internal helpers shared by the CUDA translation units of libps.
// Nothing here is part of the public C ABI (include/ps.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ps.h"

namespace ps {

// ---------------------------------------------------------------- host ----

void set_error(const char* fmt, ...);
ps_status fail(ps_status code, const char* fmt, ...);
ps_status check_cuda(cudaError_t err, const char* what);
// cudaGetLastError after a launch
ps_status check_launch(const char* what);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Carves 256-byte-aligned pieces out of a caller workspace.
struct Carver {
  char* base;
  size_t used = 0;
  explicit Carver(void* p) : base(static_cast<char*>(p)) {}
  template <typename T>
  T* take(size_t count) {
    used = align_up(used, 256);
    T* out = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += count * sizeof(T);
    return out;
  }
};

ps_status validate_grid(const ps_grid* g);
inline int64_t grid_volume(const ps_grid* g) {
  return (int64_t)g->n[0] * g->n[1] * g->n[2];
}
inline int64_t padded_volume(const ps_grid* g) {
  return (int64_t)(g->n[0] + 3) * (g->n[1] + 3) * (g->n[2] + 3);
}
size_t dtype_size(ps_dtype t);

// Per-launch geometry passed by value to kernels.
struct GridArgs {
  int n[3];        // nodes per axis
  int m[3];        // padded extents n+3
  int rx;          // coefficient row pitch in elements (>= n[0]+3, 16-byte rows)
  double inv_h[3]; // n/L, computed on the host in FP64
  float inv_hf[3]; // the same, rounded to FP32 (derivative scaling)
};
// rx is left 0 unless a coefficient dtype is given.
GridArgs make_grid_args(const ps_grid* g, int coef_t = -1);
// Row pitch (elements) of a padded coefficient array: nx+3 rounded up to a
// multiple of 16 bytes.
int64_t coef_pitch(int nx, ps_dtype t);

struct BrickArgs {
  int B[3];   // brick edge in cells per axis
  int nb[3];  // bricks per axis
  int64_t nbins;
};
ps_status make_brick_args(const ps_grid* g, const int32_t brick[3], BrickArgs* out);

// Launch-shape choices an autotuner may change (ps_tune_set).
struct Tuning {
  int brick_kernel = -1;      // -1 auto, 0 phased, 2 thread per particle, 5 quad
  int brick_min_stage = 8;    // per-brick kernel: fewer particles skip the halo
  int node_tma = 1;           // PS_F32X4 halos by tensor copy
  int solve_xw = 0;           // x extent of a strided-pass block (0: default)
  int solve_stream = 1;       // FP32 solves in two streamed passes (y-x, then z)
  int solve_zt = 0;           // columns per block of the streamed z pass (0: default)
  int solve_stages = 0;       // shared-memory stages of the streamed y-x pass (0: 3)
  int wait_probe = 0;         // test knob: clocks of a wait that cannot complete
  int batch_run_below = 16;   // batched fields with fewer particles per brick on
                              // average are binned in runs, not bricks
  int batch_persistent = 1;   // batched steps: one cooperative launch (1) or a launch
                              // per phase and step (0)
};
Tuning& tuning();
int sm_count();

// ------------------------------------------------------- cross-file API ----

// Periodic solves in place on an unpadded F32 array [ncomp][nz][ny][nx]
// (the transposed solve of the backward pass; the matrix is symmetric).
ps_status solve_unpadded_inplace_f32(const ps_grid* g, int ncomp, float* a,
                                     cudaStream_t st);

// Binning pieces (bin.cu).
size_t bin_ws_bytes(const BrickArgs& b, int64_t np, bool need_offsets,
                    bool need_bin_of, bool need_pos_sorted, bool need_ids);
ps_status bin_run(const GridArgs& ga, const BrickArgs& ba, int64_t np,
                  const double* pos, int32_t* bin_of, int32_t* bin_offsets,
                  int64_t* perm, double* pos_sorted, const int64_t* ids,
                  int64_t* ids_sorted, int32_t* counts, int32_t* rank,
                  int32_t* scan_tmp, int32_t* status, cudaStream_t st, bool counted);
size_t scan_tmp_elems(int64_t nbins);

// Many-field binning (batch.cu): one entry per field.
struct BinField {
  GridArgs g;
  BrickArgs b;
  int64_t pbase;     // first particle of the field in the concatenated arrays
  int32_t bin_base;  // first global bin of the field
  int32_t chunk;     // > 0: bins are runs of about `chunk` particles, not bricks
  int32_t nruns;     // runs of a field with chunk > 0
};
// Scan of counts the step kernels took, then the counted scatter (the counts
// end at zero).
ps_status bin_rescan_counted(int64_t total_bins, int64_t np, const double* pos,
                             const int32_t* bin_of, int32_t* bin_offsets, double* pos_sorted,
                             const int64_t* ids, int64_t* ids_sorted, int32_t* counts,
                             int32_t* scan_tmp, int32_t* status, cudaStream_t st);
ps_status bin_run_batch(const BinField* d_tab, int nfields, int64_t total_bins, int64_t np,
                        const double* pos, int32_t* bin_of, int32_t* bin_offsets,
                        double* pos_sorted, const int64_t* ids, int64_t* ids_sorted,
                        int32_t* counts, int32_t* rank, int32_t* scan_tmp, int32_t* status,
                        cudaStream_t st);

// Many-field brick kernel (interp.cu).
size_t staged_args_size();
ps_status staged_fill_rk2(const ps_grid* grid, ps_dtype coef_t, const int32_t brick[3],
                          const void* coef, const float* scale, int64_t np_total,
                          const double* pos_in, double* pos_out, const int32_t* offs,
                          float* vel, const int64_t* ids_in, int64_t* ids_out, double dt,
                          int32_t* status, int chunked, int32_t* next_counts, int32_t* next_bin,
                          int next_key_base, int next_runs, void* out, size_t* smem);
// Particles per bin of a field binned in runs of particles instead of bricks.
constexpr int kBatchChunk = 128;
// h_tab, h_bin_base: host copies of the same tables; with at most 48 fields
// they go by value as a kernel parameter (else pass NULL).
ps_status staged_batch_launch(ps_dtype coef_t, const void* d_tab, const int* d_bin_base,
                              const void* h_tab, const int* h_bin_base, int nfields,
                              int64_t total_bins, size_t smem, bool prepare, cudaStream_t st);
// All nsteps Heun steps of a batch in one cooperative launch (counts and sync,
// four words, zero at launch).
ps_status staged_batch_persistent(ps_dtype coef_t, const void* d_tab, const int* d_bin_base,
                                  const BinField* d_bintab, int nfields, int64_t total_bins,
                                  int64_t np, int nsteps, double* pos, int64_t* ids,
                                  double* pos_s, int64_t* ids_s, int32_t* bin_of, int32_t* rank,
                                  int32_t* counts, int32_t* offsets, int32_t* scan_tmp,
                                  int32_t* status, unsigned* sync, size_t smem,
                                  cudaStream_t st);

// -------------------------------------------------------------- device ----

#ifdef __CUDACC__

// Record a device-side anomaly: first code and index win, count accumulates.
__device__ __forceinline__ void flag_status(int32_t* st, int code, int64_t idx) {
  if (!st) return;
  if (atomicCAS(&st[0], 0, code) == 0) {
    st[1] = (int32_t)(uint32_t)(idx & 0xffffffffll);
    st[2] = (int32_t)(idx >> 32);
  }
  atomicAdd(&st[3], 1);
}

// Operation 2, index part (Sec. 2.2).  s = x * (n/L) is one rounded FP64
// multiply; a = floor(s) and the fraction t = s - a are then read exactly
// from the bits of s with integer arithmetic (FP64 issue slots are scarce on
// this GPU), and cell = a mod n.  t is returned rounded toward zero to 24
// bits (within one FP32 ulp of s - a); the cell index is exact.
// Returns false for a non-finite position or |s| >= 2^50.
__device__ __forceinline__ bool locate(double x, double inv_h, int n, int& cell, float& t) {
  const double s = __dmul_rn(x, inv_h);
  const long long bits = __double_as_longlong(s);
  const int bexp = (int)((bits >> 52) & 0x7ff);
  cell = 0;
  t = 0.f;
  if (bexp >= 1023 + 50) return false;  // |s| >= 2^50, Inf or NaN
  const bool neg = bits < 0;
  const unsigned long long M = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
  long long a;
  unsigned int hi;  // top 24 fraction bits of |s|
  bool frac_zero;
  if (bexp < 1023) {  // |s| < 1
    if (bexp == 0 && M == 0) return true;  // +-0
    const unsigned long long MM = bexp == 0 ? M : (M | (1ull << 52));
    const int sh = 1075 - (bexp == 0 ? 1 : bexp);  // > 52 fraction bits
    hi = sh - 24 >= 64 ? 0u : (unsigned int)(MM >> (sh - 24));
    frac_zero = false;
    a = neg ? -1 : 0;
  } else {
    const int sh = 1075 - bexp;  // 3..52 fraction bits
    const unsigned long long MM = M | (1ull << 52);
    const unsigned long long ip = MM >> sh;
    const unsigned long long fr = MM & ((1ull << sh) - 1);
    hi = sh > 24 ? (unsigned int)(fr >> (sh - 24)) : (unsigned int)(fr << (24 - sh));
    frac_zero = fr == 0;
    a = neg ? (frac_zero ? -(long long)ip : -(long long)ip - 1) : (long long)ip;
  }
  const float two_m24 = __int_as_float(0x33800000);  // 2^-24
  t = neg ? (frac_zero ? 0.f : (float)((1u << 24) - hi) * two_m24) : (float)hi * two_m24;
  long long m = a;
  if (m < 0 || m >= n) {
    m %= n;
    if (m < 0) m += n;
  }
  cell = (int)m;
  return true;
}

// Brick coordinate along axis d of a position (cell / B), -1 for a position
// that locate rejects.  The counting pass of the bin sort and the kernels that
// count for the next step's sort both derive bins from these two functions,
// so a particle lands in the same bin whichever of them counts it.
__device__ __forceinline__ int brick_coord(const GridArgs& g, const BrickArgs& b, double x,
                                           int d) {
  int c;
  float t;
  return locate(x, g.inv_h[d], g.n[d], c, t) ? c / b.B[d] : -1;
}

// Bin of brick (bx, by, bz), x fastest; -1 if a coordinate is -1.
__device__ __forceinline__ int bin_of_coords(const BrickArgs& b, int bx, int by, int bz) {
  return (bx | by | bz) < 0 ? -1 : (bz * b.nb[1] + by) * b.nb[0] + bx;
}

// Counting step of the bin sort for the particles a warp holds: lane l has
// particle p (valid) whose bin is key (-1: position rejected; it is counted
// in bin 0 and reported, as the counting pass does).  The bin goes to
// bin_of[p]; lanes with equal keys add to the bin's counter with one atomic
// whose result is not waited for (the scatter takes the ranks later).  All
// 32 lanes must call.
__device__ __forceinline__ void count_into_bin(int32_t* counts, int32_t* bin_of,
                                               int32_t* status, bool valid, int64_t p,
                                               int key, int key_base = 0) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (valid && key < 0) {
    flag_status(status, PS_DEV_NONFINITE_POS, p);
    key = 0;
  }
  const int k = valid ? key : -1 - lane;  // unique per lane when invalid
  const unsigned peers = __match_any_sync(FULL, k);
  if (valid && lane == __ffs(peers) - 1) atomicAdd(&counts[k], __popc(peers));
  if (valid) bin_of[p] = key_base + k;
}

// FP64 variant for FP64 coefficients: t = s - floor(s) in FP64.
__device__ __forceinline__ bool locate_f64(double x, double inv_h, int n, int& cell,
                                           double& t) {
  const double s = __dmul_rn(x, inv_h);
  cell = 0;
  t = 0.0;
  if (!(fabs(s) < 1125899906842624.0)) return false;  // 2^50
  const double a = floor(s);
  t = __dsub_rn(s, a);
  long long m = ((long long)a) % n;
  if (m < 0) m += n;
  cell = (int)m;
  return true;
}

// Uniform cubic B-spline on nodes a-1, a, a+1, a+2 at local coordinate t.
template <typename T>
__device__ __forceinline__ void bspline(T t, T b[4]) {
  const T s = T(1) - t;
  const T t2 = t * t, t3 = t2 * t;
  const T sixth = T(1) / T(6);
  b[0] = s * s * s * sixth;
  b[1] = (T(3) * t3 - T(6) * t2 + T(4)) * sixth;
  b[2] = (T(-3) * t3 + T(3) * t2 + T(3) * t + T(1)) * sixth;
  b[3] = t3 * sixth;
}

template <typename T>
__device__ __forceinline__ void dbspline(T t, T d[4]) {
  const T s = T(1) - t;
  const T half = T(1) / T(2);
  d[0] = -s * s * half;
  d[1] = (T(3) * t * t - T(4) * t) * half;
  d[2] = (T(-3) * t * t + T(2) * t + T(1)) * half;
  d[3] = t * t * half;
}

// d2 b / dt2: piecewise linear (the spline is twice continuously
// differentiable, Sec. 2.2).
template <typename T>
__device__ __forceinline__ void ddbspline(T t, T d[4]) {
  d[0] = T(1) - t;
  d[1] = T(3) * t - T(2);
  d[2] = T(1) - T(3) * t;
  d[3] = t;
}

// Coefficient element -> arithmetic type.
template <typename Tc> struct CoefLoad;
template <> struct CoefLoad<float> {
  static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
};
template <> struct CoefLoad<double> {
  static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
};
template <> struct CoefLoad<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
};
template <> struct CoefLoad<__half> {
  static __device__ __forceinline__ float ld(const __half* p) {
    return __half2float(__ldg(p));
  }
};

// Raw 16-bit pattern -> float.
template <typename H> struct CoefLoadBits;
template <> struct CoefLoadBits<__nv_bfloat16> {
  static __device__ __forceinline__ float f(unsigned short b) {
    return __uint_as_float((unsigned)b << 16);
  }
};
template <> struct CoefLoadBits<__half> {
  static __device__ __forceinline__ float f(unsigned short b) {
    return __half2float(__ushort_as_half(b));
  }
};

template <typename Tc> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };
template <typename Tc> struct IsQuant { static constexpr bool value = false; };
// float4 coefficients: one 16-byte node (u, v, w, 0) per grid point (PS_F32X4).
template <typename Tc> struct IsNode4 { static constexpr bool value = false; };
template <> struct IsNode4<float4> { static constexpr bool value = true; };
// 16-bit nodes (PS_BF16X4, PS_F16X4): four values in 8 bytes, scaled per
// component and x-line.
template <typename H> struct alignas(8) Node16 {
  H v[4];
};
using bf16x4 = Node16<__nv_bfloat16>;
using f16x4 = Node16<__half>;
template <> struct IsNode4<bf16x4> { static constexpr bool value = true; };
template <> struct IsNode4<f16x4> { static constexpr bool value = true; };
template <> struct IsQuant<bf16x4> { static constexpr bool value = true; };
template <> struct IsQuant<f16x4> { static constexpr bool value = true; };
template <typename Tc> struct IsNode16 { static constexpr bool value = false; };
template <> struct IsNode16<bf16x4> { static constexpr bool value = true; };
template <> struct IsNode16<f16x4> { static constexpr bool value = true; };
__device__ __forceinline__ float node16_value(__nv_bfloat16 h) { return __bfloat162float(h); }
__device__ __forceinline__ float node16_value(__half h) { return __half2float(h); }
template <> struct IsQuant<__nv_bfloat16> { static constexpr bool value = true; };
template <> struct IsQuant<__half> { static constexpr bool value = true; };

// Padded index (possibly outside [0, n+2]) -> interior padded index holding
// the same periodic node: node (P-1) mod n lives at P' = node + 1.
__device__ __forceinline__ int wrap_interior(int P, int n) {
  int m = (P - 1) % n;
  if (m < 0) m += n;
  return m + 1;
}

// Padded index in [0, n+2] -> periodic node (P-1) mod n.
__device__ __forceinline__ int padded_to_node(int P, int n) {
  int m = P - 1;
  if (m < 0) m += n;
  else if (m >= n) m -= n;
  return m;
}

#endif  // __CUDACC__

}  // namespace ps
