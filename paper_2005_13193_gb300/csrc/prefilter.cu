// Spline coefficients through the periodic inverse cut to |d| <= K: the
// spline prefilter written as a convolution.  The system of Sec. 2.2 (1/6,
// 4/6, 1/6 on every periodic line of N nodes) has the circulant inverse
//   G_N(d) = sqrt(3) (r^|d| + r^(N-|d|)) / (1 - r^N),  r = sqrt(3) - 2,
// whose entries fall off as |r|^|d| = 0.268^|d|; keeping |d| <= K gives
//   c_j = sum_{d=-K..K} G_N(d) g_{(j+d) mod N}
// along each axis.  Unlike the chunked recursions of spline.cu, every output
// depends only on its 2K + 1 neighbours, so no carries pass between threads
// (at 2K + 1 multiply-adds per value and axis instead of about four).  With
// K = 15 the neglected entries sum to 3.4e-9 per axis, below FP32 rounding.
//
// Passes: z, then y (one thread per x column and run of kRun outputs along
// the axis, lanes along x), then x (one warp per row), which also writes the
// N+3 padded layout of ps_spline_coeffs(PS_F32) from a node row staged in
// shared memory.
#include <cmath>

#include "ps_internal.cuh"

namespace ps {
namespace {

constexpr int kKMax = 15;                  // largest K
constexpr int kRun = 16;                   // outputs per thread, strided passes
constexpr int kWin = kRun + 2 * kKMax;     // inputs per thread, strided passes
constexpr int kRunX = 8;                   // outputs per thread, x pass
constexpr int kWinX = kRunX + 2 * kKMax;   // inputs per thread, x pass

struct Taps {
  float g[kKMax + 1];  // g[d] = G_N(d) for d <= K, 0 beyond
};

// Filter along an axis of stride s_axis and length n.  Block (256, 1, 1):
// x = blockIdx.x * 256 + threadIdx.x; outputs j0 .. j0 + kRun - 1 along the
// axis with j0 = blockIdx.y * kRun; the line's start is
// (blockIdx.z / inner) * outer_stride + (blockIdx.z % inner) * inner_stride.
__global__ void __launch_bounds__(256) fir_strided(const float* __restrict__ src,
                                                   float* __restrict__ dst, int nx, int n,
                                                   int64_t s_axis, int inner,
                                                   int64_t outer_stride, int64_t inner_stride,
                                                   Taps t) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int j0 = blockIdx.y * kRun;
  const int64_t base = (int64_t)(blockIdx.z / inner) * outer_stride +
                       (int64_t)(blockIdx.z % inner) * inner_stride + x;
  int m = (j0 - kKMax) % n;
  if (m < 0) m += n;
  float w[kWin];
#pragma unroll
  for (int i = 0; i < kWin; ++i) {
    w[i] = src[base + (int64_t)m * s_axis];
    if (++m == n) m = 0;
  }
#pragma unroll
  for (int o = 0; o < kRun; ++o) {
    if (j0 + o < n) {
      float acc = t.g[0] * w[o + kKMax];
#pragma unroll
      for (int d = 1; d <= kKMax; ++d)
        acc = fmaf(t.g[d], w[o + kKMax - d] + w[o + kKMax + d], acc);
      dst[base + (int64_t)(j0 + o) * s_axis] = acc;
    }
  }
}

__device__ __forceinline__ int pad_node(int P, int n) {
  int m = P - 1;
  if (m < 0) m += n;
  else if (m >= n) m -= n;
  return m;
}

// x pass and padding: one warp per padded row (Py, Pz, component), kRowsX
// rows per block.  The warp stages its node row in its own slice of shared
// memory at index e + e / 8, so that the lanes' windows (kRunX apart) fall on
// distinct banks; each lane then writes runs of kRunX consecutive padded
// values (zeros beyond nx + 3) as two 16-byte stores, 32 runs per trip.
constexpr int kRowsX = 4;
__global__ void __launch_bounds__(32 * kRowsX) fir_x_pad(const float* __restrict__ src,
                                                         float* __restrict__ dst, int nx,
                                                         int ny, int nz, int64_t rx, Taps t) {
  extern __shared__ float rows[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Py = blockIdx.x * kRowsX + warp, Pz = blockIdx.y, c = blockIdx.z;
  if (Py >= ny + 3) return;  // whole warp; no block-level barrier below
  float* row = rows + warp * (nx + nx / 8 + 1);
  const int y = pad_node(Py, ny), z = pad_node(Pz, nz);
  const float* sp = src + (((int64_t)c * nz + z) * ny + y) * nx;
  for (int e = lane; e < nx; e += 32) row[e + (e >> 3)] = sp[e];
  __syncwarp();
  float* orow = dst + (((int64_t)c * (nz + 3) + Pz) * (ny + 3) + Py) * rx;
  for (int P0 = lane * kRunX; P0 < rx; P0 += 32 * kRunX) {
    // node of padded index P is P - 1 (mod nx): the window starts at node
    // P0 - 1 - kKMax
    int m = (P0 - 1 - kKMax) % nx;
    if (m < 0) m += nx;
    float w[kWinX];
#pragma unroll
    for (int i = 0; i < kWinX; ++i) {
      w[i] = row[m + (m >> 3)];
      if (++m == nx) m = 0;
    }
    float out[kRunX];
#pragma unroll
    for (int o = 0; o < kRunX; ++o) {
      float acc = t.g[0] * w[o + kKMax];
#pragma unroll
      for (int d = 1; d <= kKMax; ++d)
        acc = fmaf(t.g[d], w[o + kKMax - d] + w[o + kKMax + d], acc);
      out[o] = P0 + o < nx + 3 ? acc : 0.f;
    }
    // rx is a multiple of 4 and P0 of 8: whole 16-byte vectors inside the row
    reinterpret_cast<float4*>(orow + P0)[0] = make_float4(out[0], out[1], out[2], out[3]);
    if (P0 + 4 < rx)
      reinterpret_cast<float4*>(orow + P0)[1] = make_float4(out[4], out[5], out[6], out[7]);
  }
}

Taps make_taps(int n, int K) {
  Taps t{};
  const double r = std::sqrt(3.0) - 2.0;
  const double rn = std::pow(r, (double)n);
  for (int d = 0; d <= K; ++d)
    t.g[d] = (float)(std::sqrt(3.0) * (std::pow(r, (double)d) + std::pow(r, (double)(n - d))) /
                     (1.0 - rn));
  return t;
}

size_t volume(const ps_grid* g, int ncomp) {
  return (size_t)ncomp * g->n[0] * g->n[1] * g->n[2];
}

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" size_t ps_spline_truncated_workspace_size(const ps_grid* grid, int ncomp) {
  if (validate_grid(grid) || ncomp < 1) return 0;
  return 2 * align_up(volume(grid, ncomp) * sizeof(float), 256) + 256;
}

extern "C" ps_status ps_spline_coeffs_truncated(const ps_grid* grid, int ncomp,
                                                const float* field, int K, float* coef,
                                                void* ws, size_t ws_bytes, void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  if (ncomp < 1 || ncomp > 3) return fail(PS_ERR_INVALID_ARG, "ncomp must be 1..3");
  if (K < 1 || K > kKMax) return fail(PS_ERR_INVALID_ARG, "K must be 1..%d", kKMax);
  for (int d = 0; d < 3; ++d)
    if (2 * K + 1 > grid->n[d])
      return fail(PS_ERR_INVALID_ARG, "2K+1 = %d exceeds n[%d] = %d", 2 * K + 1, d, grid->n[d]);
  if (!field || !coef) return fail(PS_ERR_INVALID_ARG, "field and coef are required");
  if (reinterpret_cast<uintptr_t>(coef) & 15)
    return fail(PS_ERR_INVALID_ARG, "coef must be 16-byte aligned");
  const size_t need = ps_spline_truncated_workspace_size(grid, ncomp);
  if (!ws || ws_bytes < need - 256 || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(PS_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need - 256);
  const int nx = grid->n[0], ny = grid->n[1], nz = grid->n[2];
  Carver cv(ws);
  float* a = cv.take<float>(volume(grid, ncomp));
  float* b = cv.take<float>(volume(grid, ncomp));
  cudaStream_t st = as_stream(stream);
  const unsigned gx = (unsigned)((nx + 255) / 256);
  // z: lines of (component, y); y: lines of (component, z)
  fir_strided<<<dim3(gx, (unsigned)((nz + kRun - 1) / kRun), (unsigned)(ncomp * ny)), 256, 0,
                st>>>(field, a, nx, nz, (int64_t)nx * ny, ny, (int64_t)nx * ny * nz,
                      (int64_t)nx, make_taps(nz, K));
  if ((rc = check_launch("fir_strided z"))) return rc;
  fir_strided<<<dim3(gx, (unsigned)((ny + kRun - 1) / kRun), (unsigned)(ncomp * nz)), 256, 0,
                st>>>(a, b, nx, ny, (int64_t)nx, 1, (int64_t)nx * ny, 0, make_taps(ny, K));
  if ((rc = check_launch("fir_strided y"))) return rc;
  const int64_t rx = coef_pitch(nx, PS_F32);
  const size_t smem = (size_t)kRowsX * (nx + nx / 8 + 1) * sizeof(float);
  fir_x_pad<<<dim3((unsigned)((ny + 3 + kRowsX - 1) / kRowsX), (unsigned)(nz + 3),
                   (unsigned)ncomp),
              32 * kRowsX, smem, st>>>(b, coef, nx, ny, nz, rx, make_taps(nx, K));
  return check_launch("fir_x_pad");
}
