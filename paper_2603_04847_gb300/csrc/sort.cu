// Per-tile duplication and depth ordering of projected splats.
//
//   depth sort  stable LSD radix sort of the B*N records r = b*N + j by the
//               float bits of their camera depth (invisible records last);
//               ties keep record order, i.e. index order within a view
//   scan        exclusive prefix sum of tiles-touched in depth order
//   duplicate   one (global tile, r) instance per covered tile, emitted in
//               depth order
//   tile sort   stable LSD radix sort of the instances by tile id, over the
//               bits the largest tile id uses only
//   ranges      [start, end) per global tile
//
// Sorting 8-byte records by depth once and then 8-byte instances by tile
// moves far fewer bytes than sorting 12-byte instances by a 47-bit
// (tile, depth) key, and gives the same order: (tile, depth, j).
//
// The instance count stays on the device: every kernel after the scan reads
// it, and all grids are sized from host-known bounds (records, capacity, SM
// count), so the whole stage can be captured in a CUDA graph.  Each radix
// pass is the classic three-kernel form (per-block digit histogram,
// per-digit scan over blocks, stable scatter); no block waits on another.
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048 items per tile

__device__ inline uint32_t block_exclusive_scan_u32(uint32_t v, uint32_t* total, uint32_t* sm) {
  // sm: >= 32 words.  Returns exclusive prefix of v over the block.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (warp == 0) {
    uint32_t w = lane < nw ? sm[lane] : 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < nw) sm[lane] = w;
  }
  __syncthreads();
  const uint32_t warp_prefix = warp > 0 ? sm[warp - 1] : 0u;
  if (total) *total = sm[nw - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

// Depth sort keys: float bits of the depth (positive, so the bits order like
// the values) for visible records, all ones for invisible ones.
__global__ void __launch_bounds__(256) depth_keys_kernel(gs_projected proj, uint32_t M,
                                                         uint32_t* __restrict__ keys,
                                                         uint32_t* __restrict__ vals) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < M; r += gridDim.x * blockDim.x) {
    const bool vis = proj.n_tiles[r] != 0;
    keys[r] = vis ? __float_as_uint(reinterpret_cast<const float4*>(proj.splat)[3 * (size_t)r].w)
                  : 0xffffffffu;
    vals[r] = r;
  }
}

// Sum of n_tiles[order[k]] per scan tile (64-bit to detect overflow).
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                                   const uint32_t* __restrict__ order,
                                                                   size_t M,
                                                                   unsigned long long* tile_sums) {
  __shared__ unsigned long long red[kScanThreads / 32];
  const size_t base = (size_t)blockIdx.x * kScanTile;
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const size_t k = base + (size_t)i * kScanThreads + threadIdx.x;
    if (k < M) s += in[order[k]];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    tile_sums[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile sums in one block; writes the instance count
// and raises GS_FLAG_CAPACITY when it exceeds the capacity.
__global__ void __launch_bounds__(1024) scan_tiles_kernel(unsigned long long* tile_sums, int n_tiles,
                                                          size_t capacity, uint32_t* n_instances,
                                                          int32_t* status) {
  __shared__ unsigned long long sm[32];
  const int per = (n_tiles + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per;
  const int hi = min(lo + per, n_tiles);
  unsigned long long s = 0;
  for (int k = lo; k < hi; ++k) s += tile_sums[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    unsigned long long w = lane < nw ? sm[lane] : 0ull;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < nw) sm[lane] = w;
  }
  __syncthreads();
  unsigned long long run = (warp > 0 ? sm[warp - 1] : 0ull) + x - s;
  for (int k = lo; k < hi; ++k) {
    const unsigned long long v = tile_sums[k];
    tile_sums[k] = run;
    run += v;
  }
  if (threadIdx.x == blockDim.x - 1) {
    // the full count (saturated to 32 bits) tells the host how much capacity
    // it needs; every consumer uses min(count, capacity)
    const unsigned long long total = run;
    if (total > (unsigned long long)capacity) set_flag(status, GS_FLAG_CAPACITY);
    *n_instances = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t* __restrict__ in,
                                                                  const uint32_t* __restrict__ order,
                                                                  size_t M,
                                                                  const unsigned long long* tile_offs,
                                                                  uint32_t* __restrict__ out) {
  __shared__ uint32_t sm[32];
  const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const size_t k = base + i;
    v[i] = k < M ? in[order[k]] : 0u;
    s += v[i];
  }
  const uint32_t ex = block_exclusive_scan_u32(s, nullptr, sm);
  // offsets beyond 2^32 cannot be valid instances (capacity < 2^32): clamp
  unsigned long long run = tile_offs[blockIdx.x] + ex;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const size_t k = base + i;
    if (k < M) out[k] = run > 0xffffffffull ? 0xffffffffu : (uint32_t)run;
    run += v[i];
  }
}

struct SlotTiles {
  int tiles_x;
  int tile_offset;
};

// Instances in depth order: position k of the depth-sorted records emits
// its tiles at offs[k] onwards.
__global__ void __launch_bounds__(256) duplicate_kernel(gs_projected proj, const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ offs, int N, gs_cameras cams,
                                                        gs_batch batch, uint32_t* __restrict__ tiles,
                                                        uint32_t* __restrict__ vals, size_t capacity,
                                                        int32_t* status) {
  __shared__ SlotTiles st[GS_MAX_BATCH];
  for (int b = threadIdx.x; b < batch.B; b += blockDim.x) {
    const int v = slot_view(cams, batch, b);
    st[b].tiles_x = (cams.wh[2 * v] + batch.tile - 1) / batch.tile;
    st[b].tile_offset = batch.tile_offset[b];
  }
  __syncthreads();
  const size_t M = (size_t)batch.B * N;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < M;
       k += (size_t)gridDim.x * blockDim.x) {
    const uint32_t r = order[k];
    const uint32_t n = proj.n_tiles[r];
    if (n == 0) continue;
    const int b = (int)(r / (uint32_t)N);
    const ushort4 rc = reinterpret_cast<const ushort4*>(proj.rect)[r];
    size_t o = offs[k];
    if (o + n > capacity) set_flag(status, GS_FLAG_CAPACITY);
    const int tx_n = st[b].tiles_x, t0 = st[b].tile_offset;
    for (int ty = rc.y; ty <= rc.w; ++ty)
      for (int tx = rc.x; tx <= rc.z; ++tx) {
        if (o < capacity) {
          tiles[o] = (uint32_t)(t0 + ty * tx_n + tx);
          vals[o] = r;
        }
        ++o;
      }
  }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits.
// The item count is either host-known (n_dev == nullptr) or read on the
// device, clamped to the buffer capacity.
//
// Each block owns a contiguous chunk of the items (a multiple of the 4096-item
// tile).  Pass = histogram per block, scan per digit over blocks, scatter.
// The scatter works tile by tile: every warp ranks its own 256 contiguous
// items (8 rounds of 32) against a warp-private running count per digit;
// one block step turns the per-warp counts into offsets within the tile;
// items are staged digit-sorted in shared memory and then written out in
// that order, so consecutive threads write consecutive addresses of a
// digit's run (full sectors, not one scattered word per item).  Equal
// digits keep their input order: tiles, warps, rounds and lanes are all
// taken in input order.

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kWarpItems = 256;                       // 8 rounds of 32 per warp
constexpr int kTileItems = kSortWarps * kWarpItems;   // 4096

__device__ inline uint32_t radix_count(const uint32_t* n_dev, uint32_t n_host, size_t capacity) {
  return n_dev ? (uint32_t)min((size_t)*n_dev, capacity) : n_host;
}

__device__ inline void chunk_of(uint32_t n, int nb, int blk, uint32_t& lo, uint32_t& hi) {
  uint32_t chunk = (n + nb - 1) / nb;
  chunk = (chunk + kTileItems - 1) / kTileItems * kTileItems;
  lo = min((uint32_t)blk * chunk, n);
  hi = min(lo + chunk, n);
}

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                                  const uint32_t* n_dev, uint32_t n_host,
                                                                  size_t capacity, int shift,
                                                                  uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kSortWarps][256];
  for (int i = threadIdx.x; i < kSortWarps * 256; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint32_t n = radix_count(n_dev, n_host, capacity);
  uint32_t lo, hi;
  chunk_of(n, gridDim.x, blockIdx.x, lo, hi);
  const int warp = threadIdx.x >> 5;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&h[warp][(keys[i] >> shift) & 0xffu], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) t += h[w][d];
    hist[(size_t)d * gridDim.x + blockIdx.x] = t;
  }
}

// Block d: exclusive scan over the row of digit d (block order), in place,
// in one blocked pass; digit total to totals[d].
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t* hist, int row_len, uint32_t* totals) {
  __shared__ uint32_t sm[32];
  uint32_t* row = hist + (size_t)blockIdx.x * row_len;
  const int per = (row_len + blockDim.x - 1) / blockDim.x;
  const int lo = min((int)threadIdx.x * per, row_len), hi = min(lo + per, row_len);
  uint32_t s = 0;
  for (int k = lo; k < hi; ++k) s += row[k];
  uint32_t tot;
  uint32_t run = block_exclusive_scan_u32(s, &tot, sm);
  for (int k = lo; k < hi; ++k) {
    const uint32_t v = row[k];
    row[k] = run;
    run += v;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* n_dev, uint32_t n_host, size_t capacity, int shift,
    const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals) {
  __shared__ uint32_t s_base[256];     // global start of this block's next items of each digit
  __shared__ uint32_t s_tot[256];      // items of each digit in the current tile
  __shared__ uint32_t s_dstart[256];   // exclusive scan of s_tot
  __shared__ uint16_t s_wrun[kSortWarps][256];
  __shared__ uint32_t s_keys[kTileItems];
  __shared__ uint32_t s_vals[kTileItems];
  __shared__ uint32_t sm[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    const uint32_t t = tid < 256 ? totals[tid] : 0u;
    const uint32_t ex = block_exclusive_scan_u32(t, nullptr, sm);
    if (tid < 256) s_base[tid] = ex + hist[(size_t)tid * gridDim.x + blockIdx.x];
  }
  const uint32_t n = radix_count(n_dev, n_host, capacity);
  uint32_t lo, hi;
  chunk_of(n, gridDim.x, blockIdx.x, lo, hi);
  const unsigned lt_mask = (1u << lane) - 1u;
  for (uint32_t tile = lo; tile < hi; tile += kTileItems) {
    const uint32_t tile_n = min((uint32_t)kTileItems, hi - tile);
    for (int d = lane; d < 256; d += 32) s_wrun[warp][d] = 0;
    __syncwarp();
    // 1. warp-local stable ranking of the warp's 8 rounds of 32 items
    uint32_t k[8], v[8], r[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const uint32_t li = (uint32_t)(warp * kWarpItems + s * 32 + lane);
      const bool valid = li < tile_n;
      k[s] = valid ? kin[tile + li] : 0u;
      v[s] = valid ? vin[tile + li] : 0u;
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const uint32_t li = (uint32_t)(warp * kWarpItems + s * 32 + lane);
      const bool valid = li < tile_n;
      const uint32_t d = valid ? (k[s] >> shift) & 0xffu : 256u + (uint32_t)lane;  // unique sentinel
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      r[s] = valid ? (uint32_t)s_wrun[warp][d] + __popc(peers & lt_mask) : 0u;
      __syncwarp();
      if (valid && (peers & lt_mask) == 0) s_wrun[warp][d] += (uint16_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // 2. per digit: offsets of the warps within the tile, tile totals
    if (tid < 256) {
      uint32_t acc = 0;
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = s_wrun[w][tid];
        s_wrun[w][tid] = (uint16_t)acc;
        acc += c;
      }
      s_tot[tid] = acc;
    }
    __syncthreads();
    {
      const uint32_t t = tid < 256 ? s_tot[tid] : 0u;
      const uint32_t ex = block_exclusive_scan_u32(t, nullptr, sm);
      if (tid < 256) s_dstart[tid] = ex;
    }
    __syncthreads();
    // 3. stage digit-sorted in shared memory
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const uint32_t li = (uint32_t)(warp * kWarpItems + s * 32 + lane);
      if (li < tile_n) {
        const uint32_t d = (k[s] >> shift) & 0xffu;
        const uint32_t p = s_dstart[d] + s_wrun[warp][d] + r[s];
        s_keys[p] = k[s];
        s_vals[p] = v[s];
      }
    }
    __syncthreads();
    // 4. write runs: consecutive threads, consecutive positions of a digit
    for (uint32_t p = tid; p < tile_n; p += kSortThreads) {
      const uint32_t key = s_keys[p];
      const uint32_t d = (key >> shift) & 0xffu;
      const uint32_t pos = s_base[d] + (p - s_dstart[d]);
      kout[pos] = key;
      vout[pos] = s_vals[p];
    }
    __syncthreads();
    if (tid < 256) s_base[tid] += s_tot[tid];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) tile_ranges_kernel(const uint32_t* __restrict__ tiles,
                                                          const uint32_t* n_dev, size_t capacity,
                                                          uint32_t* __restrict__ ranges) {
  const uint32_t n = (uint32_t)min((size_t)*n_dev, capacity);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = tiles[i];
    if (i == 0) {
      ranges[2 * t] = 0;
    } else {
      const uint32_t p = tiles[i - 1];
      if (p != t) {
        ranges[2 * p + 1] = i;
        ranges[2 * t] = i;
      }
    }
    if (i == n - 1) ranges[2 * t + 1] = n;
  }
}

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct SortWs {
  uint32_t* dkeys[2];   // depth keys, double-buffered [M]
  uint32_t* dvals[2];   // record ids [M]
  uint32_t* offs;       // instance offset per depth-sorted record [M]
  unsigned long long* tile_sums;
  uint32_t* tiles_alt;  // [capacity]
  uint32_t* vals_alt;   // [capacity]
  uint32_t* hist;
  uint32_t* totals;
  size_t bytes;
};

SortWs sort_ws_layout(void* base, size_t M, size_t capacity, int nb) {
  SortWs w;
  char* p = (char*)base;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* q = p + o;
    o += align_up(bytes);
    return q;
  };
  for (int i = 0; i < 2; ++i) w.dkeys[i] = (uint32_t*)take(M * 4);
  for (int i = 0; i < 2; ++i) w.dvals[i] = (uint32_t*)take(M * 4);
  w.offs = (uint32_t*)take(M * 4);
  w.tile_sums = (unsigned long long*)take(((M + kScanTile - 1) / kScanTile) * 8 + 8);
  w.tiles_alt = (uint32_t*)take(capacity * 4);
  w.vals_alt = (uint32_t*)take(capacity * 4);
  w.hist = (uint32_t*)take((size_t)256 * nb * 4);
  w.totals = (uint32_t*)take(256 * 4);
  w.bytes = o;
  return w;
}

int radix_blocks() { return tuning().sort_blocks_per_sm * device_sm_count(); }

// Stable LSD passes over bits [0, bits) of (kA, vA); kA/vA point at the
// sorted result afterwards.
void radix_sort_u32(uint32_t*& kA, uint32_t*& vA, uint32_t*& kB, uint32_t*& vB, const uint32_t* n_dev,
                    uint32_t n_host, size_t capacity, int bits, SortWs& w, int nb, cudaStream_t st) {
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<nb, kSortThreads, 0, st>>>(kA, n_dev, n_host, capacity, shift, w.hist);
    radix_scan_kernel<<<256, 1024, 0, st>>>(w.hist, nb, w.totals);
    radix_scatter_kernel<<<nb, kSortThreads, 0, st>>>(kA, vA, kB, vB, n_dev, n_host, capacity, shift, w.hist,
                                                       w.totals);
    std::swap(kA, kB);
    std::swap(vA, vB);
  }
}

}  // namespace

int sort_tile_bits(int n_tiles_total) {
  int tb = 0;
  while ((1ll << tb) < (long long)n_tiles_total) ++tb;
  return tb;
}

size_t sort_workspace_bytes(int N, const gs_batch& batch, size_t capacity) {
  return sort_ws_layout(nullptr, (size_t)batch.B * N, capacity, radix_blocks()).bytes;
}

cudaError_t launch_sort_tiles(int N, const gs_cameras& cams, const gs_batch& batch,
                              const gs_projected& proj, uint32_t* tiles, uint32_t* vals,
                              size_t capacity, uint32_t* ranges, uint32_t* n_instances, void* ws,
                              int32_t* status, cudaStream_t st) {
  const size_t M = (size_t)batch.B * N;
  const int nb = radix_blocks();
  SortWs w = sort_ws_layout(ws, M, capacity, nb);
  cudaError_t e;
  e = cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)batch.n_tiles, st);
  if (e != cudaSuccess) return e;
  const int n_scan_tiles = (int)((M + kScanTile - 1) / kScanTile);
  if (n_scan_tiles == 0) return cudaMemsetAsync(n_instances, 0, 4, st);

  // 1. stable depth sort of the records (32-bit keys, host-known count)
  const int grid = (int)std::min<size_t>((M + 255) / 256, (size_t)nb * 8);
  depth_keys_kernel<<<grid, 256, 0, st>>>(proj, (uint32_t)M, w.dkeys[0], w.dvals[0]);
  uint32_t *dkA = w.dkeys[0], *dvA = w.dvals[0], *dkB = w.dkeys[1], *dvB = w.dvals[1];
  radix_sort_u32(dkA, dvA, dkB, dvB, nullptr, (uint32_t)M, M, 32, w, nb, st);
  const uint32_t* order = dvA;

  // 2. instance offsets in depth order
  scan_reduce_kernel<<<n_scan_tiles, kScanThreads, 0, st>>>(proj.n_tiles, order, M, w.tile_sums);
  scan_tiles_kernel<<<1, 1024, 0, st>>>(w.tile_sums, n_scan_tiles, capacity, n_instances, status);
  scan_apply_kernel<<<n_scan_tiles, kScanThreads, 0, st>>>(proj.n_tiles, order, M, w.tile_sums, w.offs);

  // 3. duplicate into whichever buffer leaves the tile-sorted result in
  //    tiles/vals, then 4. stable sort by tile id
  const int tbits = sort_tile_bits(batch.n_tiles);
  const int passes = (tbits + 7) / 8;
  uint32_t* kA = (passes & 1) ? w.tiles_alt : tiles;
  uint32_t* vA = (passes & 1) ? w.vals_alt : vals;
  uint32_t* kB = (passes & 1) ? tiles : w.tiles_alt;
  uint32_t* vB = (passes & 1) ? vals : w.vals_alt;
  duplicate_kernel<<<grid, 256, 0, st>>>(proj, order, w.offs, N, cams, batch, kA, vA, capacity, status);
  radix_sort_u32(kA, vA, kB, vB, n_instances, 0, capacity, tbits, w, nb, st);

  // 5. ranges
  tile_ranges_kernel<<<nb * 4, 256, 0, st>>>(tiles, n_instances, capacity, ranges);
  return cudaGetLastError();
}

int sort_kernel_count(const gs_batch& batch) {
  const int passes = (sort_tile_bits(batch.n_tiles) + 7) / 8;
  // depth keys 1, depth sort 4 x 3, scan 3, duplicate 1, tile sort 3 / pass, ranges 1
  return 1 + 4 * 3 + 3 + 1 + 3 * passes + 1;
}

}  // namespace gs
