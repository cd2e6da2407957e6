// Device pieces of the bin sort shared by the sort kernels (bin.cu) and the
// persistent many-field kernel (interp.cu): the bin of a position, the
// counting pass over many fields, the three phases of the exclusive scan of
// the bin counters (tiles of kScanTile counters, blocks of any multiple of 32
// threads), and the scatter into bin order.  Internal to libps.
#pragma once

#include "ps_internal.cuh"

namespace ps {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int bin_of_position(const GridArgs& g, const BrickArgs& b,
                                               double x, double y, double z, bool& ok) {
  const int key = bin_of_coords(b, brick_coord(g, b, x, 0), brick_coord(g, b, y, 1),
                                brick_coord(g, b, z, 2));
  ok = key >= 0;
  return ok ? key : 0;
}

// Counting pass over the concatenated particles of many fields: particle p of
// field f (pbase[f] <= p < pbase[f+1]) goes to global bin bin_base[f] + its
// bin in field f; a warp-aggregated atomic on the bin's counter gives its
// rank.  The calling warp covers kBatchUnroll groups of 32 particles from
// warp_start (their position loads issued before any index arithmetic), then
// steps by kBatchUnroll * stride; every lane of the warp calls.
constexpr int kBatchUnroll = 4;
__device__ __forceinline__ void batch_count_range(const BinField* __restrict__ tab,
                                                  int nfields, int64_t np,
                                                  const double* __restrict__ pos,
                                                  int32_t* __restrict__ bin_of,
                                                  int32_t* __restrict__ rank,
                                                  int32_t* __restrict__ counts, int32_t* status,
                                                  int64_t warp_start, int64_t stride) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (int64_t base = warp_start; base < np; base += stride * kBatchUnroll) {
    double x[kBatchUnroll], y[kBatchUnroll], z[kBatchUnroll];
#pragma unroll
    for (int u = 0; u < kBatchUnroll; ++u) {
      const int64_t p = base + u * stride + lane;
      x[u] = y[u] = z[u] = 0.0;
      if (p < np) {
        x[u] = pos[p];
        y[u] = pos[np + p];
        z[u] = pos[2 * np + p];
      }
    }
#pragma unroll
    for (int u = 0; u < kBatchUnroll; ++u) {
      const int64_t gb = base + u * stride;  // warp-uniform
      if (gb >= np) break;
      const int64_t p = gb + lane;
      const bool valid = p < np;
      int key = -1 - lane;
      if (valid) {
        int lo = 0, hi = nfields;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (tab[mid].pbase <= p) lo = mid;
          else hi = mid;
        }
        bool ok;
        const int b = bin_of_position(tab[lo].g, tab[lo].b, x[u], y[u], z[u], ok);
        if (!ok) flag_status(status, PS_DEV_NONFINITE_POS, p);
        // a sparse field: runs, each an equal span of the bricks' order
        key = tab[lo].bin_base +
              (tab[lo].chunk > 0 ? (int)((int64_t)b * tab[lo].nruns / tab[lo].b.nbins) : b);
      }
      const unsigned peers = __match_any_sync(FULL, key);
      const int leader = __ffs(peers) - 1;
      const int within = __popc(peers & ((1u << lane) - 1));
      int basev = 0;
      if (valid && lane == leader) basev = atomicAdd(&counts[key], __popc(peers));
      basev = __shfl_sync(peers, basev, leader);
      if (valid) {
        bin_of[p] = key;
        rank[p] = basev + within;
      }
    }
  }
}

// Block-wide exclusive scan of one value per thread (T threads, warp_tot:
// T/32 shared ints); returns the block total.  Every thread calls.
template <int T>
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t& excl, int32_t* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int32_t woff = 0, total = 0;
  for (int w = 0; w < T / 32; ++w) {
    const int32_t t = warp_tot[w];
    if (w < warp) woff += t;
    total += t;
  }
  __syncthreads();
  excl = woff + incl - v;
  return total;
}

// Phase 1: the sum of tile `tile` (kScanTile counters) by one block of T
// threads; red: T/32 shared ints.
template <int T>
__device__ __forceinline__ void scan_tile_sum(const int32_t* __restrict__ in, int64_t n,
                                              int64_t tile, int32_t* __restrict__ tile_sums,
                                              int32_t* red) {
  constexpr int I = kScanTile / T;
  const int64_t tile0 = tile * kScanTile;
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    const int64_t idx = tile0 + (int64_t)i * T + threadIdx.x;
    if (idx < n) s += in[idx];
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < T / 32; ++w) t += red[w];
    tile_sums[tile] = t;
  }
  __syncthreads();
}

// Phase 2: one block scans the tile sums in place (any count, running carry).
template <int T>
__device__ __forceinline__ void scan_tile_offsets_block(int32_t* tile_sums, int64_t ntiles,
                                                        int32_t* warp_tot) {
  int32_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += T) {
    const int64_t idx = base + threadIdx.x;
    const int32_t v = idx < ntiles ? tile_sums[idx] : 0;
    int32_t excl;
    const int32_t tot = block_excl_scan<T>(v, excl, warp_tot);
    if (idx < ntiles) tile_sums[idx] = carry + excl;
    carry += tot;
  }
}

// Phase 3: scan inside tile `tile`, add the tile offset; out has n+1 entries
// (the last tile writes out[n]).  clamp >= 0: offsets clamped to [0, clamp].
template <int T>
__device__ __forceinline__ void scan_tile(const int32_t* __restrict__ in, int64_t n,
                                          const int32_t* __restrict__ tile_off,
                                          int32_t* __restrict__ out, int64_t clamp,
                                          int64_t tile, int64_t ntiles, int32_t* warp_tot) {
  constexpr int I = kScanTile / T;
  const int64_t tile0 = tile * kScanTile;
  // each thread takes I consecutive elements
  int32_t v[I];
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    const int64_t idx = tile0 + (int64_t)threadIdx.x * I + i;
    v[i] = idx < n ? in[idx] : 0;
    s += v[i];
  }
  int32_t excl;
  const int32_t tot = block_excl_scan<T>(s, excl, warp_tot);
  int32_t run = tile_off[tile] + excl;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    const int64_t idx = tile0 + (int64_t)threadIdx.x * I + i;
    if (idx < n) out[idx] = clamp < 0 ? run : (int32_t)min(max((int64_t)run, (int64_t)0), clamp);
    run += v[i];
  }
  if (tile == ntiles - 1 && threadIdx.x == 0) {
    const int32_t last = tile_off[tile] + tot;
    out[n] = clamp < 0 ? last : (int32_t)min(max((int64_t)last, (int64_t)0), clamp);
  }
}

// Each thread takes kCountUnroll particles per trip, the dependent loads (bin,
// offset, then the payload) of several in flight together.
constexpr int kCountUnroll = 4;

// Scatter into bin order from counts the step kernels took (the counted
// re-binning): bins in bin_of, bounds in offsets; each run of equal bins in a
// warp takes its slots with one atomicSub on the bin's counter, so the
// counters end at zero.  Slots outside a bin's range are not written and are
// reported (PS_DEV_BAD_BINS).  Warp wid of `warps` covers groups of
// kCountUnroll x 32 particles; every lane of the warp calls.
__device__ __forceinline__ void scatter_counted_range(int64_t np, const double* __restrict__ pos,
                                    const int32_t* __restrict__ bin_of,
                                    int32_t* __restrict__ counts,
                                    const int32_t* __restrict__ offsets,
                                    int64_t* __restrict__ perm,
                                    double* __restrict__ pos_sorted,
                                    const int64_t* __restrict__ ids,
                                    int64_t* __restrict__ ids_sorted, int64_t nbins,
                                    int32_t* status, int64_t wid, int64_t warps) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (wid == 0 && lane == 0 && offsets[nbins] != np)
    flag_status(status, PS_DEV_BAD_BINS, offsets[nbins]);
  for (int64_t base = wid * 32 * kCountUnroll; base < np; base += warps * 32 * kCountUnroll) {
    int key[kCountUnroll];
    double x[kCountUnroll], y[kCountUnroll], z[kCountUnroll];
    int64_t id[kCountUnroll];
    // bins and payloads of all groups first
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const int64_t p = base + u * 32 + lane;
      key[u] = -1 - lane;  // unique per lane when invalid
      x[u] = y[u] = z[u] = 0.0;
      id[u] = 0;
      if (p < np) {
        const int bn = bin_of[p];
        if ((uint64_t)(int64_t)bn < (uint64_t)nbins) key[u] = bn;
        else flag_status(status, PS_DEV_BAD_BINS, p);
        if (pos_sorted) {
          x[u] = pos[p];
          y[u] = pos[np + p];
          z[u] = pos[2 * np + p];
        }
        if (ids_sorted) id[u] = ids[p];
      }
    }
    // one atomic per run of equal bins, all groups' atomics in flight together
    unsigned peers[kCountUnroll];
    int old[kCountUnroll];
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      peers[u] = __match_any_sync(FULL, key[u]);
      old[u] = 0;
      if (key[u] >= 0 && lane == __ffs(peers[u]) - 1)
        old[u] = atomicSub(&counts[key[u]], __popc(peers[u]));
    }
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const int leader = __ffs(peers[u]) - 1;
      const int top = __shfl_sync(FULL, old[u], leader);
      if (key[u] < 0) continue;
      const int64_t p = base + u * 32 + lane;
      const int len = __popc(peers[u]);
      const int r = top - len + __popc(peers[u] & ((1u << lane) - 1u));
      const int64_t lo = offsets[key[u]], hi = offsets[key[u] + 1];
      if (top - len < 0 || (int64_t)top > hi - lo) {
        flag_status(status, PS_DEV_BAD_BINS, p);
        continue;
      }
      const int64_t slot = lo + r;
      if (perm) perm[slot] = p;
      if (pos_sorted) {
        pos_sorted[slot] = x[u];
        pos_sorted[np + slot] = y[u];
        pos_sorted[2 * np + slot] = z[u];
      }
      if (ids_sorted) ids_sorted[slot] = id[u];
    }
  }
}


// Scatter into bin order: slot = offsets[bin_of[p]] + rank[p]; the calling
// thread starts at particle `first` and steps by `stride`.
__device__ __forceinline__ void scatter_range(int64_t np, const double* __restrict__ pos,
                                              const int32_t* __restrict__ bin_of,
                                              const int32_t* __restrict__ rank,
                                              const int32_t* __restrict__ offsets,
                                              int64_t* __restrict__ perm,
                                              double* __restrict__ pos_sorted,
                                              const int64_t* __restrict__ ids,
                                              int64_t* __restrict__ ids_sorted, int64_t first,
                                              int64_t stride) {
  for (int64_t p0 = first; p0 < np; p0 += stride * kCountUnroll) {
    int64_t slot[kCountUnroll];
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const int64_t p = p0 + u * stride;
      slot[u] = p < np ? (int64_t)offsets[bin_of[p]] + rank[p] : -1;
    }
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const int64_t p = p0 + u * stride;
      if (slot[u] < 0) continue;
      if (perm) perm[slot[u]] = p;
      if (pos_sorted) {
        pos_sorted[slot[u]] = pos[p];
        pos_sorted[np + slot[u]] = pos[np + p];
        pos_sorted[2 * np + slot[u]] = pos[2 * np + p];
      }
      if (ids_sorted) ids_sorted[slot[u]] = ids[p];
    }
  }
}

}  // namespace
}  // namespace ps
