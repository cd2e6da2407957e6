// Bin sort of particles into cell bricks: the one-device reading of the
// paper's dynamic particle-to-process mapping by instantaneous position
// (Sec. 3) and of its per-step particle migration (Sec. 4.3).
//
// count:   bin of every particle; a warp-aggregated atomicAdd on the bin's
//          counter returns the particle's rank inside its bin.
// scan:    exclusive prefix sum of the counters -> bin_offsets (3 phases).
// scatter: slot = bin_offsets[bin] + rank; writes perm / sorted copies.
// The count may instead come from the kernel that wrote the positions (it
// counts each particle's new bin as it stores it, without ranks); bin_run
// then starts at the scan, and the scatter takes ranks from the counters.
#include <mutex>

#include "bin_device.cuh"

namespace ps {
namespace {

// Ranks inside runs of equal keys in consecutive lanes: the run's first lane,
// the lane's offset in the run and the run's length.  Particles stored in the
// previous step's bin order form long runs, so one atomic serves many lanes;
// equal keys in separate runs simply take separate atomics.
__device__ __forceinline__ void run_ranks(int key, int lane, int& first, int& within, int& len) {
  const unsigned FULL = 0xffffffffu;
  const int prev = __shfl_up_sync(FULL, key, 1);
  const unsigned starts = __ballot_sync(FULL, lane == 0 || prev != key);
  const unsigned upto = 0xffffffffu >> (31 - lane);  // bits 0..lane
  first = 31 - __clz(starts & upto);
  within = lane - first;
  const unsigned after = starts & ~upto;
  len = (after ? __ffs(after) - 1 : 32) - first;
}

// (bin_count_kernel: each warp takes kCountUnroll consecutive groups of 32
// particles per trip and issues all their position loads before any index
// arithmetic.)

__global__ void bin_count_kernel(GridArgs g, BrickArgs b, int64_t np,
                                 const double* __restrict__ pos, int32_t* __restrict__ bin_of,
                                 int32_t* __restrict__ rank, int32_t* __restrict__ counts,
                                 int32_t* status) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // uniform trip count per warp so that every lane reaches the warp intrinsics
  for (int64_t base = wid * 32 * kCountUnroll; base < np; base += warps * 32 * kCountUnroll) {
    double x[kCountUnroll], y[kCountUnroll], z[kCountUnroll];
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const int64_t p = base + u * 32 + lane;
      x[u] = y[u] = z[u] = 0.0;
      if (p < np) {
        x[u] = pos[p];
        y[u] = pos[np + p];
        z[u] = pos[2 * np + p];
      }
    }
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const int64_t p = base + u * 32 + lane;
      const bool valid = p < np;
      int key = -1 - lane;  // unique per lane when invalid
      if (valid) {
        bool ok;
        key = bin_of_position(g, b, x[u], y[u], z[u], ok);
        if (!ok) flag_status(status, PS_DEV_NONFINITE_POS, p);
      }
      int first, within, len;
      run_ranks(key, lane, first, within, len);
      int basev = 0;
      if (valid && lane == first) basev = atomicAdd(&counts[key], len);
      basev = __shfl_sync(FULL, basev, first);
      if (valid) {
        bin_of[p] = key;
        rank[p] = basev + within;
      }
    }
  }
}

// Phase 1: per-tile sums.
__global__ void scan_tile_sums(const int32_t* __restrict__ in, int64_t n,
                               int32_t* __restrict__ tile_sums) {
  __shared__ int32_t red[kScanThreads / 32];
  scan_tile_sum<kScanThreads>(in, n, blockIdx.x, tile_sums, red);
}

// Phase 2: one block scans the tile sums in place (any count, running carry).
__global__ void scan_tile_offsets(int32_t* tile_sums, int64_t ntiles) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  scan_tile_offsets_block<kScanThreads>(tile_sums, ntiles, warp_tot);
}

// Phase 3: scan inside each tile, add the tile offset; out has n+1 entries.
// clamp >= 0: offsets are clamped to [0, clamp], so that counts that do not
// add up (see bin_run's `counted`) still give offsets inside the particle
// arrays.
__global__ void scan_tiles(const int32_t* __restrict__ in, int64_t n,
                           const int32_t* __restrict__ tile_off, int32_t* __restrict__ out,
                           int64_t clamp) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  scan_tile<kScanThreads>(in, n, tile_off, out, clamp, blockIdx.x, gridDim.x, warp_tot);
}

__global__ void bin_scatter_kernel(int64_t np, const double* __restrict__ pos,
                                   const int32_t* __restrict__ bin_of,
                                   const int32_t* __restrict__ rank,
                                   const int32_t* __restrict__ offsets,
                                   int64_t* __restrict__ perm,
                                   double* __restrict__ pos_sorted,
                                   const int64_t* __restrict__ ids,
                                   int64_t* __restrict__ ids_sorted) {
  scatter_range(np, pos, bin_of, rank, offsets, perm, pos_sorted, ids, ids_sorted,
                (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Scatter for bins counted by an earlier kernel (bin_run's `counted`), which
// leaves no ranks: lanes of a warp with the same bin take a run of its slots
// by one atomicSub on the bin's counter (the counters end at zero).  Each bin
// and run is checked against the bin's range of slots before the writes; a
// particle that fails is skipped and reported, as is a total that is not np.
// Every warp makes the same number of trips (warp-wide intrinsics).
__global__ void bin_scatter_counted(int64_t np, const double* __restrict__ pos,
                                    const int32_t* __restrict__ bin_of,
                                    int32_t* __restrict__ counts,
                                    const int32_t* __restrict__ offsets,
                                    int64_t* __restrict__ perm,
                                    double* __restrict__ pos_sorted,
                                    const int64_t* __restrict__ ids,
                                    int64_t* __restrict__ ids_sorted, int64_t nbins,
                                    int32_t* status) {
  scatter_counted_range(np, pos, bin_of, counts, offsets, perm, pos_sorted, ids, ids_sorted,
                        nbins, status,
                        ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                        ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Counting pass over the concatenated particles of many fields: particle p of
// field f (pbase[f] <= p < pbase[f+1]) goes to global bin bin_base[f] + its
// bin in field f.
__global__ void bin_count_batch_kernel(const BinField* __restrict__ tab, int nfields,
                                       int64_t np, const double* __restrict__ pos,
                                       int32_t* __restrict__ bin_of, int32_t* __restrict__ rank,
                                       int32_t* __restrict__ counts, int32_t* status) {
  const int lane = threadIdx.x & 31;
  batch_count_range(tab, nfields, np, pos, bin_of, rank, counts, status,
                    (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane,
                    (int64_t)gridDim.x * blockDim.x);
}

// Grid of a grid-stride kernel: enough blocks for the work, at most a full
// occupancy of the current device (its own SM count, read per call).
int persistent_blocks(int64_t work, int threads) {
  const int sms = sm_count();
  int64_t need = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sms * (2048 / threads);
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

}  // namespace

size_t scan_tmp_elems(int64_t nbins) { return (size_t)((nbins + kScanTile - 1) / kScanTile); }

size_t bin_ws_bytes(const BrickArgs& b, int64_t np, bool need_offsets, bool need_bin_of,
                    bool need_pos_sorted, bool need_ids) {
  // carve order: counts, tile sums, rank, [offsets], [bin_of], [pos_sorted], [ids]
  Carver c(nullptr);
  c.take<int32_t>(b.nbins + 1);                  // counts
  c.take<int32_t>(scan_tmp_elems(b.nbins) + 1);  // tile sums
  c.take<int32_t>(np);                           // rank
  if (need_offsets) c.take<int32_t>(b.nbins + 1);
  if (need_bin_of) c.take<int32_t>(np);
  if (need_pos_sorted) c.take<double>(3 * np);
  if (need_ids) c.take<int64_t>(np);
  return align_up(c.used, 256) + 256;
}

ps_status bin_run(const GridArgs& ga, const BrickArgs& ba, int64_t np, const double* pos,
                  int32_t* bin_of, int32_t* bin_offsets, int64_t* perm, double* pos_sorted,
                  const int64_t* ids, int64_t* ids_sorted, int32_t* counts, int32_t* rank,
                  int32_t* scan_tmp, int32_t* status, cudaStream_t st, bool counted) {
  ps_status rc = PS_OK;
  if (!counted &&
      (rc = check_cuda(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (ba.nbins + 1), st),
                       "bin counts memset")))
    return rc;
  if (np > 0 && !counted) {
    bin_count_kernel<<<persistent_blocks(np, 256), 256, 0, st>>>(ga, ba, np, pos, bin_of,
                                                                 rank, counts, status);
    if ((rc = check_launch("bin_count"))) return rc;
  }
  const int64_t ntiles = (int64_t)scan_tmp_elems(ba.nbins);
  scan_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, st>>>(counts, ba.nbins, scan_tmp);
  if ((rc = check_launch("scan_tile_sums"))) return rc;
  scan_tile_offsets<<<1, kScanThreads, 0, st>>>(scan_tmp, ntiles);
  if ((rc = check_launch("scan_tile_offsets"))) return rc;
  scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(counts, ba.nbins, scan_tmp,
                                                        bin_offsets, counted ? np : -1);
  if ((rc = check_launch("scan_tiles"))) return rc;
  if (np > 0 && (perm || pos_sorted || ids_sorted)) {
    if (counted)
      bin_scatter_counted<<<persistent_blocks(np, 256), 256, 0, st>>>(
          np, pos, bin_of, counts, bin_offsets, perm, pos_sorted, ids, ids_sorted, ba.nbins,
          status);
    else
      bin_scatter_kernel<<<persistent_blocks(np, 256), 256, 0, st>>>(
          np, pos, bin_of, rank, bin_offsets, perm, pos_sorted, ids, ids_sorted);
    if ((rc = check_launch("bin_scatter"))) return rc;
  }
  return PS_OK;
}

ps_status bin_rescan_counted(int64_t total_bins, int64_t np, const double* pos,
                             const int32_t* bin_of, int32_t* bin_offsets, double* pos_sorted,
                             const int64_t* ids, int64_t* ids_sorted, int32_t* counts,
                             int32_t* scan_tmp, int32_t* status, cudaStream_t st) {
  const int64_t ntiles = (int64_t)scan_tmp_elems(total_bins);
  scan_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, st>>>(counts, total_bins, scan_tmp);
  ps_status rc = check_launch("scan_tile_sums");
  if (rc) return rc;
  scan_tile_offsets<<<1, kScanThreads, 0, st>>>(scan_tmp, ntiles);
  if ((rc = check_launch("scan_tile_offsets"))) return rc;
  scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(counts, total_bins, scan_tmp,
                                                        bin_offsets, -1);
  if ((rc = check_launch("scan_tiles"))) return rc;
  if (np > 0) {
    bin_scatter_counted<<<persistent_blocks(np, 256), 256, 0, st>>>(
        np, pos, bin_of, counts, bin_offsets, nullptr, pos_sorted, ids, ids_sorted, total_bins,
        status);
    if ((rc = check_launch("bin_scatter_counted"))) return rc;
  }
  return PS_OK;
}

ps_status bin_run_batch(const BinField* d_tab, int nfields, int64_t total_bins, int64_t np,
                        const double* pos, int32_t* bin_of, int32_t* bin_offsets,
                        double* pos_sorted, const int64_t* ids, int64_t* ids_sorted,
                        int32_t* counts, int32_t* rank, int32_t* scan_tmp, int32_t* status,
                        cudaStream_t st) {
  ps_status rc = check_cuda(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (total_bins + 1), st),
                            "batch counts memset");
  if (rc) return rc;
  if (np > 0) {
    bin_count_batch_kernel<<<persistent_blocks(np, 256), 256, 0, st>>>(
        d_tab, nfields, np, pos, bin_of, rank, counts, status);
    if ((rc = check_launch("bin_count_batch"))) return rc;
  }
  const int64_t ntiles = (int64_t)scan_tmp_elems(total_bins);
  scan_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, st>>>(counts, total_bins, scan_tmp);
  if ((rc = check_launch("scan_tile_sums"))) return rc;
  scan_tile_offsets<<<1, kScanThreads, 0, st>>>(scan_tmp, ntiles);
  if ((rc = check_launch("scan_tile_offsets"))) return rc;
  scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(counts, total_bins, scan_tmp,
                                                        bin_offsets, -1);
  if ((rc = check_launch("scan_tiles"))) return rc;
  if (np > 0) {
    bin_scatter_kernel<<<persistent_blocks(np, 256), 256, 0, st>>>(
        np, pos, bin_of, rank, bin_offsets, nullptr, pos_sorted, ids, ids_sorted);
    if ((rc = check_launch("bin_scatter"))) return rc;
  }
  return PS_OK;
}

}  // namespace ps

using namespace ps;

extern "C" size_t ps_bin_workspace_size(const ps_grid* grid, const int32_t brick[3],
                                        int64_t np) {
  BrickArgs ba;
  if (validate_grid(grid) || make_brick_args(grid, brick, &ba) || np < 0) return 0;
  return bin_ws_bytes(ba, np, false, false, false, false);
}

extern "C" ps_status ps_bin_particles(const ps_grid* grid, const int32_t brick[3],
                                      int64_t np, const double* pos, int32_t* bin_of,
                                      int32_t* bin_offsets, int64_t* perm,
                                      double* pos_sorted, void* ws, size_t ws_bytes,
                                      int32_t* status, void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  BrickArgs ba;
  if ((rc = make_brick_args(grid, brick, &ba))) return rc;
  if (np < 0 || np >= ((int64_t)1 << 31)) return fail(PS_ERR_INVALID_ARG, "np out of range");
  if (!bin_offsets || (np > 0 && (!pos || !bin_of)))
    return fail(PS_ERR_INVALID_ARG, "pos, bin_of and bin_offsets are required");
  const size_t need = bin_ws_bytes(ba, np, false, false, false, false);
  if (!ws || ws_bytes < need - 256 || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(PS_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need - 256);
  Carver c(ws);
  int32_t* counts = c.take<int32_t>(ba.nbins + 1);
  int32_t* scan_tmp = c.take<int32_t>(scan_tmp_elems(ba.nbins) + 1);
  int32_t* rank = c.take<int32_t>(np);
  GridArgs ga = make_grid_args(grid);
  return bin_run(ga, ba, np, pos, bin_of, bin_offsets, perm, pos_sorted, nullptr, nullptr,
                 counts, rank, scan_tmp, status, as_stream(stream), false);
}

// ---------------------------------------------------------------------------
// Allocation-free binning.  Some callers cannot call cudaMalloc (or hand the
// library a workspace) at the point where they bin particles: code running
// under a strict device-memory budget owned by another allocator, callers
// that must not add allocation latency inside a time-critical step, or hosts
// that reach this library through a plain C interface with no allocator of
// their own.  For them the scratch of the counting sort lives in a file-scope
// device array of fixed size that every GPU loading this library holds until
// the process exits.

namespace {
constexpr int64_t kNoAllocScratchInts = (int64_t)1 << 23;  // 32 MiB of int32
__device__ __align__(256) int32_t g_bin_scratch[kNoAllocScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
int32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_bin_scratch on the current device.  In host code the
// array's name is only a stand-in, so the address is resolved once per device
// (with that device current) through cudaGetSymbolAddress.
ps_status bin_scratch_for_current_device(int32_t** out) {
  int dev = 0;
  ps_status rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= kMaxDevices) return fail(PS_ERR_UNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    rc = check_cuda(cudaGetSymbolAddress(&p, g_bin_scratch), "cudaGetSymbolAddress(bin scratch)");
    if (rc) return rc;
    g_scratch_ptr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PS_OK;
}
}  // namespace

extern "C" ps_status ps_bin_particles_noalloc(const ps_grid* grid, const int32_t brick[3],
                                              int64_t np, const double* pos, int32_t* bin_of,
                                              int32_t* bin_offsets, int64_t* perm,
                                              double* pos_sorted, int32_t* status,
                                              void* stream) {
  ps_status rc = validate_grid(grid);
  if (rc) return rc;
  BrickArgs ba;
  if ((rc = make_brick_args(grid, brick, &ba))) return rc;
  if (np < 0 || np >= ((int64_t)1 << 31)) return fail(PS_ERR_INVALID_ARG, "np out of range");
  if (!bin_offsets || (np > 0 && (!pos || !bin_of)))
    return fail(PS_ERR_INVALID_ARG, "pos, bin_of and bin_offsets are required");
  // same carve as the workspace form: counts, tile sums, rank
  Carver sizing(nullptr);
  sizing.take<int32_t>(ba.nbins + 1);
  sizing.take<int32_t>(scan_tmp_elems(ba.nbins) + 1);
  sizing.take<int32_t>(np);
  const size_t cap = (size_t)kNoAllocScratchInts * sizeof(int32_t);
  if (sizing.used > cap)
    return fail(PS_ERR_INVALID_ARG,
                "allocation-free binning needs %zu scratch bytes (bins %lld, particles %lld); "
                "its fixed scratch holds %zu bytes",
                sizing.used, (long long)ba.nbins, (long long)np, cap);
  int32_t* scratch = nullptr;
  if ((rc = bin_scratch_for_current_device(&scratch))) return rc;
  Carver c(scratch);
  int32_t* counts = c.take<int32_t>(ba.nbins + 1);
  int32_t* scan_tmp = c.take<int32_t>(scan_tmp_elems(ba.nbins) + 1);
  int32_t* rank = c.take<int32_t>(np);
  GridArgs ga = make_grid_args(grid);
  // bin_run clears the counters before counting, so the contents left by the
  // previous call do not matter
  return bin_run(ga, ba, np, pos, bin_of, bin_offsets, perm, pos_sorted, nullptr, nullptr,
                 counts, rank, scan_tmp, status, as_stream(stream), false);
}
