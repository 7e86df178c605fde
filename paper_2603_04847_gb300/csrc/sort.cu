// Per-tile duplication and depth ordering of projected splats.
//
//   depth sort  stable LSD radix sort of the B*N records r = b*N + j by the
//               float bits of their camera depth (keys written by the
//               projection; invisible records last); ties keep record
//               order, i.e. index order within a view.  The keys are taken
//               relative to the smallest visible one, so three 8-bit passes
//               suffice when the visible depths span < 2^24 float codes
//               (a factor of ~8 in depth); a fourth runs otherwise
//   scan        exclusive prefix sum of tiles-touched in depth order
//   expand      one (global tile, r) instance per covered tile, emitted in
//               depth order; each block owns one contiguous output range
//   tile sort   stable LSD radix sort of the instances by tile id, over the
//               bits the largest tile id uses only (8-bit digits, or 9-bit
//               ones where that saves a pass: 17 bits as 9 + 8, 18 as 9 + 9)
//   ranges      [start, end) per global tile
//
// Sorting 8-byte records by depth once and then 8-byte instances by tile
// moves far fewer bytes than sorting 12-byte instances by a 47-bit
// (tile, depth) key, and gives the same order: (tile, depth, j).
//
// Each radix pass is ONE kernel (the single-sweep form with decoupled
// look-back): the digit counts of every pass are known before the first
// pass (one histogram of the depth keys; the tile-id histogram is counted
// while the instances are emitted), so a block only needs, per digit, the
// number of smaller-indexed items carrying that digit, which it gets from
// the counts its predecessor blocks publish.  Blocks take their 4096-item
// tile from an atomic counter, so every block a tile waits on is already
// running; each wait is bounded and raises GS_FLAG_SORT_STALL when the
// bound runs out instead of hanging.  A pass that gave up still writes only
// inside its output (its offsets are partial sums of the true ones), and it
// sets a stall word in the workspace: every later kernel of the stage reads
// that word first and does nothing, so the instance count stays 0, the
// ranges stay zeroed and the renders see empty tiles -- no kernel ever reads
// the unsorted data.
//
// The instance count stays on the device: every kernel after the scan reads
// it, and all grids are sized from host-known bounds (records, capacity, SM
// count), so the whole stage can be captured in a CUDA graph.
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048 records per scan block
constexpr int kExpandStage = 4096;                    // instances staged per expand window

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRounds = 8;                            // rounds of 32 items per warp
constexpr int kWarpItems = 32 * kRounds;              // 256
constexpr int kTileItems = kSortWarps * kWarpItems;   // 4096 items per radix tile
constexpr int kMaxDigits = 4;                         // 32-bit keys, 8-bit digits
constexpr int kMaxTileBins = 512;                     // tile-id digits of up to 9 bits
// digit histograms: depth [kMaxDigits][256], then tile ids [kMaxDigits][512]
constexpr int kHistWords = kMaxDigits * 256 + kMaxDigits * kMaxTileBins;

// Look-back words: state in the top two bits, count in the low 62.
constexpr unsigned long long kLbAggregate = 1ull << 62;  // this tile's own count
constexpr unsigned long long kLbInclusive = 2ull << 62;  // count over tiles 0..t
constexpr unsigned long long kLbCount = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 20;   // polls of one unpublished word (default)
constexpr int kLbWindow = 4;          // predecessors read per look-back step

__device__ inline void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ inline unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

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

// Zeroes, per call: the digit histograms, the tile counters, the look-back
// words of the depth passes, the ranges and the instance count.
struct SortZero {
  uint32_t* ghist;                 // [kHistWords]
  uint32_t* counters;              // [2 * kMaxDigits]
  unsigned long long* lb_depth;    // [kMaxDigits * depth tiles * 256]
  size_t lb_depth_words;
  uint32_t* ranges;                // [2 * n_tiles]
  size_t ranges_words;
  uint32_t* n_instances;
  uint32_t* stall;                 // [1] set by a pass whose wait ran out
  uint32_t* range;                 // [3] min, max of the visible depth keys, invisible count
};

__global__ void __launch_bounds__(256) sort_zero_kernel(SortZero z) {
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
  for (size_t i = i0; i < kHistWords; i += step) z.ghist[i] = 0;
  for (size_t i = i0; i < 2 * kMaxDigits; i += step) z.counters[i] = 0;
  for (size_t i = i0; i < z.lb_depth_words; i += step) z.lb_depth[i] = 0;
  for (size_t i = i0; i < z.ranges_words; i += step) z.ranges[i] = 0;
  if (i0 == 0) {
    *z.n_instances = 0;
    *z.stall = 0;
    z.range[0] = 0xffffffffu;
    z.range[1] = 0u;
    z.range[2] = 0u;
  }
}

// The depth keys are sorted as key - min over the visible keys (invisible
// records, key 0xffffffff, as a key above every visible one): when the
// visible keys span fewer than 2^24 - 1 codes -- float bits of depths within
// a factor of ~8 of each other, as in any one scene -- three 8-bit passes
// order them and the fourth is skipped.
__device__ inline uint32_t invisible_key(const uint32_t* range) {
  return (range[1] >= range[0] && range[1] - range[0] < 0xffffffu) ? 0x00ffffffu : 0xffffffffu;
}

__device__ inline uint32_t remap_depth(uint32_t key, uint32_t kmin, uint32_t inv) {
  return key == 0xffffffffu ? inv : key - kmin;
}

// range[0] = min, range[1] = max over the visible keys, range[2] += the
// number of invisible ones.
__global__ void __launch_bounds__(256) depth_range_kernel(const uint32_t* __restrict__ keys, uint32_t n,
                                                          uint32_t* range) {
  uint32_t lo = 0xffffffffu, hi = 0u, ninv = 0u;
  const uint32_t nv = n / 4;
  const uint4* k4 = reinterpret_cast<const uint4*>(keys);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    const uint4 q = k4[i];
    const uint32_t v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (v[e] == 0xffffffffu) {
        ++ninv;
      } else {
        lo = min(lo, v[e]);
        hi = max(hi, v[e]);
      }
    }
  }
  for (uint32_t i = 4 * nv + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t v = keys[i];
    if (v == 0xffffffffu) {
      ++ninv;
    } else {
      lo = min(lo, v);
      hi = max(hi, v);
    }
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  ninv = __reduce_add_sync(0xffffffffu, ninv);
  if ((threadIdx.x & 31) == 0) {
    if (lo != 0xffffffffu) atomicMin(&range[0], lo);
    if (hi != 0u) atomicMax(&range[1], hi);
    if (ninv) atomicAdd(&range[2], ninv);
  }
}

// Counts of each 8-bit digit of the remapped depth keys of keys[0, n), for
// digits 0..n_digits-1: ghist[d * 256 + v] += number of keys whose digit d
// is v.  keys 16-byte aligned.  A thread whose four keys share a digit value adds them at once
// (the high digits of nearby depths mostly agree).
__global__ void __launch_bounds__(256) digit_hist_kernel(const uint32_t* __restrict__ keys, uint32_t n,
                                                         int n_digits, uint32_t* __restrict__ ghist,
                                                         const uint32_t* range) {
  __shared__ uint32_t h[kMaxDigits][256];
  for (int i = threadIdx.x; i < kMaxDigits * 256; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint32_t kmin = range[0], inv = invisible_key(range);
  const uint32_t nv = n / 4;
  const uint4* k4 = reinterpret_cast<const uint4*>(keys);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    uint4 q = k4[i];
    q.x = remap_depth(q.x, kmin, inv);
    q.y = remap_depth(q.y, kmin, inv);
    q.z = remap_depth(q.z, kmin, inv);
    q.w = remap_depth(q.w, kmin, inv);
    for (int d = 0; d < n_digits; ++d) {
      const int s = 8 * d;
      const uint32_t a = (q.x >> s) & 0xffu, b = (q.y >> s) & 0xffu;
      const uint32_t c = (q.z >> s) & 0xffu, e = (q.w >> s) & 0xffu;
      if (a == b && b == c && c == e) {
        atomicAdd(&h[d][a], 4u);
      } else {
        atomicAdd(&h[d][a], 1u);
        atomicAdd(&h[d][b], 1u);
        atomicAdd(&h[d][c], 1u);
        atomicAdd(&h[d][e], 1u);
      }
    }
  }
  for (uint32_t i = 4 * nv + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t key = remap_depth(keys[i], kmin, inv);
    for (int d = 0; d < n_digits; ++d) atomicAdd(&h[d][(key >> (8 * d)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_digits * 256; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&ghist[i], c);
  }
}

// One stable radix pass over the RB-bit digit at `shift` (RB = 8, or 9
// where two 9-bit passes cover a key that needs three of 8 bits).
//   kin/vin    input keys / values; vin == nullptr means value = index
//   kout/vout  output; kout may be nullptr (keys not needed afterwards)
//   ghist      [2^RB] counts of this digit over all n items
//   gather     if gather_src: gather_dst[pos] = gather_src[value] as well
//              (8-byte elements)
// Per tile: every warp ranks its 256 contiguous items (8 rounds of 32)
// against a warp-private running count per digit (peers found with one
// ballot per digit bit, which measured faster than a warp match); one block step turns the per-warp counts into
// offsets within the tile and the tile's digit counts, which are published
// for the successors; items are staged digit-sorted in shared memory; the
// look-back adds up the counts of the preceding tiles per digit; the staged
// items are written out in order, so consecutive threads write consecutive
// addresses of a digit's run.  Equal digits keep their input
// order: tiles, warps, rounds and lanes are all taken in input order.
template <int RB>
__global__ void __launch_bounds__(kSortThreads, 3) onesweep_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* n_dev, uint32_t n_host, size_t capacity, int shift,
    const uint32_t* __restrict__ ghist, unsigned long long* lookback, uint32_t* tile_counter,
    const uint2* __restrict__ gather_src, uint2* __restrict__ gather_dst, uint32_t gather_n, int32_t* status,
    uint32_t* stall, int spin_limit, int fake_stall, int role, const uint32_t* range) {
  constexpr int kBins = 1 << RB;
  constexpr uint32_t kMask = kBins - 1;
  static_assert(kBins <= kSortThreads, "one thread per digit value");
  __shared__ uint32_t s_base[kBins];    // output position of this tile's first item of each digit
  __shared__ uint32_t s_tot[kBins];     // items of each digit in this tile
  __shared__ uint32_t s_dstart[kBins];  // exclusive scan of s_tot
  __shared__ uint16_t s_wrun[kSortWarps][kBins];
  __shared__ uint32_t s_keys[kTileItems];
  __shared__ uint32_t s_vals[kTileItems];
  __shared__ uint32_t sm[32];
  __shared__ uint32_t s_tile, s_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // depth passes: role 1 (first) remaps the raw keys; role 2 (third) is the
  // last one when the remapped keys fit 24 bits and then gathers; role 3
  // (fourth) runs only when they do not
  const bool four = role >= 1 && invisible_key(range) == 0xffffffffu;
  if (role == 3 && !four) return;  // grid-uniform
  const bool last_pass = (role == 2 && !four) || role == 3;
  if (role == 2 && !four) kout = nullptr;
  if (role >= 2 && !last_pass) gather_src = nullptr;
  if (tid == 0) {
    // an earlier pass gave up: its output is not sorted, do nothing (read
    // by one thread: another block of this pass may set it meanwhile)
    s_stop = *(volatile uint32_t*)stall;
    if (!s_stop) s_tile = atomicAdd(tile_counter, 1u);
  }
  for (int d = lane; d < kBins; d += 32) s_wrun[warp][d] = 0;
  __syncthreads();
  if (s_stop) return;  // block-uniform
  const uint32_t t = s_tile;
  const uint32_t n = n_dev ? (uint32_t)min((size_t)*n_dev, capacity) : n_host;
  if ((size_t)t * kTileItems >= n) return;  // block-uniform
  const uint32_t tile0 = t * kTileItems;
  const uint32_t tile_n = min((uint32_t)kTileItems, n - tile0);

  // 1. load the keys and rank within the warp
  // ranks within the warp's digit run are < 256 (at most 7 earlier rounds
  // of 32 plus 31 lanes): four to a register
  static_assert(kRounds <= 8, "a rank must fit in 8 bits");
  uint32_t k[kRounds], rp[(kRounds + 3) / 4];
#pragma unroll
  for (int s = 0; s < kRounds; ++s) {
    const uint32_t li = (uint32_t)(warp * kWarpItems + s * 32 + lane);
    k[s] = li < tile_n ? kin[tile0 + li] : 0u;
  }
  if (role == 1) {
    const uint32_t kmin = range[0], inv = invisible_key(range);
#pragma unroll
    for (int s = 0; s < kRounds; ++s) k[s] = remap_depth(k[s], kmin, inv);
  }
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int s = 0; s < kRounds; ++s) {
    const uint32_t li = (uint32_t)(warp * kWarpItems + s * 32 + lane);
    const bool valid = li < tile_n;
    const uint32_t d = (k[s] >> shift) & kMask;
    unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const unsigned m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
      peers &= ((d >> b) & 1u) ? m : ~m;
    }
    const uint32_t rank = valid ? (uint32_t)s_wrun[warp][d] + __popc(peers & lt_mask) : 0u;
    rp[s >> 2] = (s & 3) ? (rp[s >> 2] | (rank << (8 * (s & 3)))) : rank;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) s_wrun[warp][d] += (uint16_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();


  // 2. per digit: offsets of the warps within the tile, the tile's count,
  //    published at once so that successors need not wait for step 5
  if (tid < kBins) {
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = s_wrun[w][tid];
      s_wrun[w][tid] = (uint16_t)acc;
      acc += c;
    }
    s_tot[tid] = acc;
    st_relaxed_u64(&lookback[(size_t)t * kBins + tid], (t == 0 ? kLbInclusive : kLbAggregate) | acc);
  }
  __syncthreads();

  // 3. digit starts within the tile and over all items
  const uint32_t ex_local = block_exclusive_scan_u32(tid < kBins ? s_tot[tid] : 0u, nullptr, sm);
  if (tid < kBins) s_dstart[tid] = ex_local;
  const uint32_t ex_global = block_exclusive_scan_u32(tid < kBins ? ghist[tid] : 0u, nullptr, sm);

  // 4. stage digit-sorted in shared memory (before the look-back, which
  //    then finds more predecessors done)
#pragma unroll
  for (int s = 0; s < kRounds; ++s) {
    const uint32_t li = (uint32_t)(warp * kWarpItems + s * 32 + lane);
    if (li < tile_n) {
      const uint32_t d = (k[s] >> shift) & kMask;
      const uint32_t p = s_dstart[d] + s_wrun[warp][d] + ((rp[s >> 2] >> (8 * (s & 3))) & 0xffu);
      s_keys[p] = k[s];
      s_vals[p] = vin ? vin[tile0 + li] : tile0 + li;
    }
  }

  // 5. look-back: items of digit d in tiles 0..t-1.  The words of kLbWindow
  //    predecessors are read at once and summed back to the nearest
  //    inclusive one; an unpublished word is polled again (bounded).
  if (tid < kBins) {
    unsigned long long before = 0;
    long long j = (long long)t - 1;
    int polls = 0;
    while (j >= 0) {
      unsigned long long w[kLbWindow];
#pragma unroll
      for (int q = 0; q < kLbWindow; ++q)
        w[q] = j - q >= 0 ? ld_relaxed_u64(&lookback[(size_t)(j - q) * kBins + tid]) : kLbInclusive;
      if (fake_stall) {  // test hook: the predecessors never publish
#pragma unroll
        for (int q = 0; q < kLbWindow; ++q) w[q] = 0;
      }
      int adv = 0;
      bool found = false, blocked = false;
#pragma unroll
      for (int q = 0; q < kLbWindow; ++q) {
        if (!found && !blocked) {
          const unsigned long long state = w[q] >> 62;
          if (state == 0) {
            blocked = true;
          } else {
            before += w[q] & kLbCount;
            ++adv;
            found = state != 1;
          }
        }
      }
      if (found) break;
      j -= adv;
      if (adv == 0) {
        if (++polls > spin_limit) {
          set_flag(status, GS_FLAG_SORT_STALL);
          atomicExch(stall, 1u);
          break;
        }
        __nanosleep(128);
      }
    }
    if (t > 0) st_relaxed_u64(&lookback[(size_t)t * kBins + tid], kLbInclusive | (before + s_tot[tid]));
    s_base[tid] = ex_global + (uint32_t)before;
  }
  __syncthreads();

  // 6. write runs: consecutive threads, consecutive positions of a digit
#pragma unroll 2
  for (int i = 0; i < kRounds; ++i) {
    const uint32_t p = (uint32_t)(tid + i * kSortThreads);
    if (p < tile_n) {
      const uint32_t key = s_keys[p];
      const uint32_t d = (key >> shift) & kMask;
      const uint32_t pos = s_base[d] + (p - s_dstart[d]);
      const uint32_t val = s_vals[p];
      if (kout) kout[pos] = key;
      vout[pos] = val;
      if (gather_src && val < gather_n) gather_dst[pos] = gather_src[val];
    }
  }
}

// Tiles touched by the record at depth position k: the area of its tile
// rectangle for the visible records (the first n_visible in depth order),
// none for the others (whose rectangles were not written).
__device__ inline uint32_t rect_area(ushort4 r) {
  return (uint32_t)(r.z - r.x + 1) * (uint32_t)(r.w - r.y + 1);
}

__device__ inline size_t visible_records(size_t M, const uint32_t* range) {
  return M - range[2];  // the invisible records sort last
}

// Sum of tiles touched per scan block (64-bit to detect overflow).
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const ushort4* __restrict__ rectd, size_t M,
                                                                   const uint32_t* __restrict__ range,
                                                                   unsigned long long* block_sums,
                                                                   const uint32_t* stall) {
  __shared__ unsigned long long red[kScanThreads / 32];
  const size_t base = (size_t)blockIdx.x * kScanTile;
  // the depth order is not valid after a stalled pass: no instances
  const size_t n_vis = *(volatile const uint32_t*)stall ? 0 : visible_records(M, range);
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const size_t k = base + (size_t)i * kScanThreads + threadIdx.x;
    if (k < n_vis) s += rect_area(rectd[k]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    block_sums[blockIdx.x] = t;
  }
}

// Exclusive scan of the block sums in one block; writes the instance count
// and raises GS_FLAG_CAPACITY when it exceeds the capacity.
__global__ void __launch_bounds__(1024) scan_blocks_kernel(unsigned long long* block_sums, int n_blocks,
                                                           size_t capacity, uint32_t* n_instances,
                                                           int32_t* status) {
  __shared__ unsigned long long sm[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < n_blocks; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const unsigned long long v = i < n_blocks ? block_sums[i] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ull;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      sm[lane] = w;
    }
    __syncthreads();
    const unsigned long long excl = carry + (warp > 0 ? sm[warp - 1] : 0ull) + x - v;
    if (i < n_blocks) block_sums[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long total = carry;
    *n_instances = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    if (total > capacity) set_flag(status, GS_FLAG_CAPACITY);
  }
}

struct SlotTiles {
  int tiles_x;
  int tile_offset;
};

// Emits the instances of 2048 depth-sorted records.  Their instances are
// one contiguous output range (from the scan); each thread's 8 records are
// contiguous within it.  Instance j of a record is its j-th covered tile in
// row-major order.  The instances are staged in shared memory per window and
// written out coalesced.  Also counts the tile-id digits for the tile sort
// and zeroes a share of the tile sort's look-back words.
__global__ void __launch_bounds__(kScanThreads) expand_kernel(
    const ushort4* __restrict__ rectd, const uint32_t* __restrict__ order3, const uint32_t* __restrict__ order4,
    size_t M, const uint32_t* __restrict__ range,
    const unsigned long long* __restrict__ block_offs, gs_projected proj, int N, gs_cameras cams,
    gs_batch batch, uint32_t* __restrict__ tiles, uint32_t* __restrict__ vals, size_t capacity,
    const uint32_t* n_instances, int n_digits, int tile_rb, uint32_t* __restrict__ ghist,
    unsigned long long* __restrict__ lb_tile, size_t lb_tile_stride, const uint32_t* stall) {
  __shared__ uint32_t s_t[kExpandStage];
  __shared__ uint32_t s_v[kExpandStage];
  __shared__ SlotTiles st[GS_MAX_BATCH];
  __shared__ uint32_t h[kMaxDigits][kMaxTileBins];
  __shared__ uint32_t sm[32];
  const int tid = threadIdx.x;
  const int tbins = 1 << tile_rb;
  const uint32_t tmask = (uint32_t)tbins - 1u;
  for (int b = tid; b < batch.B; b += blockDim.x) {
    const int v = slot_view(cams, batch, b);
    st[b].tiles_x = (cams.wh[2 * v] + batch.tile - 1) / batch.tile;
    st[b].tile_offset = batch.tile_offset[b];
  }
  for (int i = tid; i < kMaxDigits * kMaxTileBins; i += blockDim.x) (&h[0][0])[i] = 0;

  // zero the look-back words of the tile sort's tiles that will be used
  {
    const size_t n_used = min((size_t)*n_instances, capacity);
    const size_t words = ((n_used + kTileItems - 1) / kTileItems) * (size_t)tbins;
    for (int p = 0; p < n_digits; ++p)
      for (size_t i = (size_t)blockIdx.x * blockDim.x + tid; i < words; i += (size_t)gridDim.x * blockDim.x)
        lb_tile[p * lb_tile_stride + i] = 0;
  }

  const size_t base = (size_t)blockIdx.x * kScanTile;
  const size_t n_vis = *(volatile const uint32_t*)stall ? 0 : visible_records(M, range);
  // the depth order is where the last depth pass left it (three passes or four)
  const uint32_t* __restrict__ order = invisible_key(range) == 0xffffffffu ? order4 : order3;
  uint32_t c[kScanItems], rr[kScanItems];
  ushort4 rc[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const size_t k = base + (size_t)tid * kScanItems + i;
    const bool vis = k < n_vis;
    rc[i] = vis ? rectd[k] : make_ushort4(0, 0, 0, 0);
    rr[i] = vis ? order[k] : 0u;
    c[i] = vis ? rect_area(rc[i]) : 0u;
    s += c[i];
  }
  uint32_t slot[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) slot[i] = c[i] ? rr[i] / (uint32_t)N : 0u;
  uint32_t total;
  const uint32_t my0 = block_exclusive_scan_u32(s, &total, sm);  // this thread's first output

  // The thread's records are contiguous in depth order, so their instances
  // are the contiguous outputs [my0, my0 + s) of the block.  Per window of
  // kExpandStage outputs, every thread writes its records' instances into
  // shared memory (walking each rectangle row-major from the window's
  // start), then the block copies the window out coalesced and counts the
  // tile-id digits.
  const unsigned long long g0 = block_offs[blockIdx.x];
  const uint32_t n_out = g0 >= capacity ? 0u : (uint32_t)min((unsigned long long)total, capacity - g0);
  for (uint32_t w0 = 0; w0 < n_out; w0 += kExpandStage) {
    const uint32_t w1 = min(w0 + (uint32_t)kExpandStage, n_out);
    uint32_t q = my0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const uint32_t lo = max(q, w0), hi = min(q + c[i], w1);
      if (lo < hi) {
        const ushort4 r4 = rc[i];
        const SlotTiles sl = st[slot[i]];
        const uint32_t w = (uint32_t)(r4.z - r4.x + 1);
        const uint32_t j = lo - q;
        const uint32_t jy = j / w;
        uint32_t jx = j - jy * w;
        uint32_t row = (uint32_t)(sl.tile_offset + (int)(r4.y + jy) * sl.tiles_x + (int)r4.x);
        for (uint32_t p = lo; p < hi; ++p) {
          s_t[p - w0] = row + jx;
          s_v[p - w0] = rr[i];
          if (++jx == w) {
            jx = 0;
            row += (uint32_t)sl.tiles_x;
          }
        }
      }
      q += c[i];
    }
    __syncthreads();
    for (uint32_t p = tid; p < w1 - w0; p += kScanThreads) {
      const uint32_t tile = s_t[p];
      tiles[g0 + w0 + p] = tile;
      vals[g0 + w0 + p] = s_v[p];
      for (int d = 0; d < n_digits; ++d) atomicAdd(&h[d][(tile >> (tile_rb * d)) & tmask], 1u);
    }
    __syncthreads();
  }
  for (int i = tid; i < n_digits * tbins; i += blockDim.x) {
    const int d = i / tbins, v = i - d * tbins;
    const uint32_t cnt = h[d][v];
    if (cnt) atomicAdd(&ghist[d * tbins + v], cnt);
  }
}

// ranges[2t], ranges[2t+1] = first and one-past-last position of tile t in
// the sorted tiles[0, n); four items per thread (tiles 16-byte aligned).
__global__ void __launch_bounds__(256) tile_ranges_kernel(const uint32_t* __restrict__ tiles,
                                                          const uint32_t* n_dev, size_t capacity,
                                                          uint32_t* __restrict__ ranges,
                                                          const uint32_t* stall) {
  if (*(volatile const uint32_t*)stall) return;  // the lists are not sorted: leave every tile empty
  const uint32_t n = (uint32_t)min((size_t)*n_dev, capacity);
  const uint32_t nq = (uint32_t)(((size_t)n + 3) / 4);
  for (uint32_t qi = blockIdx.x * blockDim.x + threadIdx.x; qi < nq; qi += gridDim.x * blockDim.x) {
    const uint32_t i0 = 4 * qi;
    uint32_t t[4];
    if ((size_t)i0 + 4 <= n) {
      const uint4 q = reinterpret_cast<const uint4*>(tiles)[qi];
      t[0] = q.x, t[1] = q.y, t[2] = q.z, t[3] = q.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) t[e] = i0 + e < n ? tiles[i0 + e] : 0u;
    }
    uint32_t prev = i0 > 0 ? tiles[i0 - 1] : 0u;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t i = i0 + e;
      if (i < n) {
        if (i == 0) {
          ranges[2 * t[e]] = 0;
        } else if (prev != t[e]) {
          ranges[2 * prev + 1] = i;
          ranges[2 * t[e]] = i;
        }
        if (i == n - 1) ranges[2 * t[e] + 1] = n;
        prev = t[e];
      }
    }
  }
}

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t radix_tiles(size_t items) { return (items + kTileItems - 1) / kTileItems; }

struct SortWs {
  uint32_t* dkeys[2];   // depth keys, double-buffered [M]
  uint32_t* dvals[2];   // record ids [M]
  ushort4* rectd;       // tile rectangles, in depth order [M]
  unsigned long long* block_sums;
  uint32_t* tiles_alt;  // [capacity]
  uint32_t* vals_alt;   // [capacity]
  uint32_t* ghist;      // [kHistWords]: depth digits [4][256], tile digits [4][512]
  uint32_t* counters;   // [2][kMaxDigits] tile counters per pass
  unsigned long long* lb_depth;  // [kMaxDigits][depth tiles][256]
  unsigned long long* lb_tile;   // [tile passes][instance tiles][2^tile_rb]
  uint32_t* stall;               // [1] a pass gave up waiting (zeroed per call)
  uint32_t* range;               // [3] depth-key min, max, invisible count
  size_t bytes;
};

SortWs sort_ws_layout(void* base, size_t M, size_t capacity, int tile_passes, int tile_rb) {
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
  w.rectd = (ushort4*)take(M * 8);
  w.block_sums = (unsigned long long*)take(((M + kScanTile - 1) / kScanTile) * 8 + 8);
  w.tiles_alt = (uint32_t*)take(capacity * 4);
  w.vals_alt = (uint32_t*)take(capacity * 4);
  w.ghist = (uint32_t*)take(kHistWords * 4);
  w.counters = (uint32_t*)take(2 * kMaxDigits * 4);
  w.lb_depth = (unsigned long long*)take(kMaxDigits * radix_tiles(M) * 256 * 8);
  w.lb_tile = (unsigned long long*)take((size_t)tile_passes * radix_tiles(capacity) * ((size_t)1 << tile_rb) * 8);
  w.stall = (uint32_t*)take(4);
  w.range = (uint32_t*)take(12);
  w.bytes = o;
  return w;
}

// Grid of a grid-stride kernel: enough blocks for the items, at most
// sort_blocks_per_sm x 2048 threads per SM.
int grid_stride_blocks(size_t items, int threads) {
  const size_t want = (items + threads - 1) / threads;
  const size_t cap = (size_t)tuning().sort_blocks_per_sm * device_sm_count() * (2048 / threads);
  return (int)std::max<size_t>(1, std::min(want, cap));
}

}  // namespace

int sort_tile_bits(int n_tiles_total) {
  int tb = 0;
  while ((1ll << tb) < (long long)n_tiles_total) ++tb;
  return tb;
}

namespace {
// Tile-id passes: 8-bit digits, or 9-bit ones where they need fewer passes
// (17 or 18 bits: two instead of three).
struct TilePlan {
  int passes, rb;
};
TilePlan tile_plan(int n_tiles) {
  const int tbits = sort_tile_bits(n_tiles);
  const int p8 = (tbits + 7) / 8, p9 = (tbits + 8) / 9;
  return p9 < p8 ? TilePlan{p9, 9} : TilePlan{p8, 8};
}
}  // namespace

size_t sort_workspace_bytes(int N, const gs_batch& batch, size_t capacity) {
  const TilePlan tp = tile_plan(batch.n_tiles);
  return sort_ws_layout(nullptr, (size_t)batch.B * N, capacity, tp.passes, tp.rb).bytes;
}

cudaError_t launch_sort_tiles(int N, const gs_cameras& cams, const gs_batch& batch,
                              const gs_projected& proj, uint32_t* tiles, uint32_t* vals,
                              size_t capacity, uint32_t* ranges, uint32_t* n_instances, void* ws,
                              int32_t* status, cudaStream_t st) {
  const size_t M = (size_t)batch.B * N;
  const TilePlan tp = tile_plan(batch.n_tiles);
  const int passes = tp.passes;
  SortWs w = sort_ws_layout(ws, M, capacity, passes, tp.rb);
  uint32_t* ghist_depth = w.ghist;
  uint32_t* ghist_tile = w.ghist + kMaxDigits * 256;

  SortZero z{w.ghist, w.counters, w.lb_depth, kMaxDigits * radix_tiles(M) * 256, ranges,
             2 * (size_t)batch.n_tiles, n_instances, w.stall, w.range};
  // the wait bound of the look-back; a negative setting is the test hook in
  // which predecessors never publish (every wait runs out after |value| polls)
  const int spin_cfg = tuning().sort_spin_limit;
  const int spin_limit = spin_cfg == 0 ? kSpinLimit : (spin_cfg > 0 ? spin_cfg : -spin_cfg);
  const int fake_stall = spin_cfg < 0 ? 1 : 0;
  sort_zero_kernel<<<grid_stride_blocks(std::max(z.lb_depth_words, z.ranges_words), 256), 256, 0, st>>>(z);
  const int n_scan_blocks = (int)((M + kScanTile - 1) / kScanTile);
  if (n_scan_blocks == 0) return cudaGetLastError();

  // 1. stable depth sort of the records: keys from the projection (as key -
  //    min over the visible ones), values = record ids; the last pass (the
  //    third when the keys fit 24 bits, else the fourth) writes no keys but
  //    gathers the tile rectangles into depth order
  depth_range_kernel<<<grid_stride_blocks(M / 4 + 1, 256), 256, 0, st>>>(proj.depth_key, (uint32_t)M, w.range);
  digit_hist_kernel<<<grid_stride_blocks(M / 4 + 1, 256), 256, 0, st>>>(proj.depth_key, (uint32_t)M, kMaxDigits,
                                                                         ghist_depth, w.range);
  const int depth_grid = (int)radix_tiles(M);
  const size_t lbd_stride = radix_tiles(M) * 256;
  const uint32_t* kin = proj.depth_key;
  const uint32_t* vin = nullptr;
  for (int pass = 0; pass < kMaxDigits; ++pass) {
    const bool may_be_last = pass >= kMaxDigits - 2;
    uint32_t* ko = pass == kMaxDigits - 1 ? nullptr : w.dkeys[pass & 1];
    uint32_t* vo = w.dvals[pass & 1];
    const int role = pass == 0 ? 1 : (pass == kMaxDigits - 2 ? 2 : (pass == kMaxDigits - 1 ? 3 : 0));
    onesweep_kernel<8><<<depth_grid, kSortThreads, 0, st>>>(
        kin, vin, ko, vo, nullptr, (uint32_t)M, M, 8 * pass, ghist_depth + 256 * pass,
        w.lb_depth + lbd_stride * pass, w.counters + pass,
        may_be_last ? reinterpret_cast<const uint2*>(proj.rect) : nullptr,
        may_be_last ? reinterpret_cast<uint2*>(w.rectd) : nullptr, (uint32_t)M, status, w.stall, spin_limit,
        fake_stall, role, w.range);
    kin = ko;
    vin = vo;
  }

  // 2. instance offsets in depth order, 3. expand into whichever buffer
  //    leaves the tile-sorted result in tiles/vals, 4. stable tile sort
  scan_reduce_kernel<<<n_scan_blocks, kScanThreads, 0, st>>>(w.rectd, M, w.range, w.block_sums, w.stall);
  scan_blocks_kernel<<<1, 1024, 0, st>>>(w.block_sums, n_scan_blocks, capacity, n_instances, status);
  uint32_t* kA = (passes & 1) ? w.tiles_alt : tiles;
  uint32_t* vA = (passes & 1) ? w.vals_alt : vals;
  uint32_t* kB = (passes & 1) ? tiles : w.tiles_alt;
  uint32_t* vB = (passes & 1) ? vals : w.vals_alt;
  const size_t tbins = (size_t)1 << tp.rb;
  const size_t lbt_stride = radix_tiles(capacity) * tbins;
  expand_kernel<<<n_scan_blocks, kScanThreads, 0, st>>>(w.rectd, w.dvals[0], w.dvals[1], M, w.range, w.block_sums, proj, N, cams, batch, kA, vA,
                                                         capacity, n_instances, passes, tp.rb, ghist_tile, w.lb_tile,
                                                         lbt_stride, w.stall);
  const int tile_grid = (int)radix_tiles(capacity);
  const int tbits = sort_tile_bits(batch.n_tiles);
  for (int pass = 0; pass < passes; ++pass) {
    // a last pass with 8 bits or fewer left (17-bit tile ids in 9 + 8) ranks
    // 8: the digit's ninth bit is zero for every item, its counts sit in the
    // first 256 bins of the pass's histogram and its look-back words in the
    // first half of the pass's (zeroed) region
    const int bits = std::min(tp.rb, tbits - tp.rb * pass);
    auto* kern = bits > 8 ? onesweep_kernel<9> : onesweep_kernel<8>;
    kern<<<tile_grid, kSortThreads, 0, st>>>(kA, vA, kB, vB, n_instances, 0, capacity, tp.rb * pass,
                                             ghist_tile + tbins * pass, w.lb_tile + lbt_stride * pass,
                                             w.counters + kMaxDigits + pass, nullptr, nullptr, 0u, status, w.stall,
                                             spin_limit, fake_stall, 0, nullptr);
    std::swap(kA, kB);
    std::swap(vA, vB);
  }

  // 5. ranges
  tile_ranges_kernel<<<grid_stride_blocks(capacity / 4 + 1, 256), 256, 0, st>>>(tiles, n_instances, capacity,
                                                                                 ranges, w.stall);
  return cudaGetLastError();
}

int sort_kernel_count(const gs_batch& batch) {
  const int passes = tile_plan(batch.n_tiles).passes;
  // zero 1, depth range 1, depth histogram 1, depth passes 4 (the fourth
  // returns at once when three suffice), scan 2, expand 1, tile passes,
  // ranges 1
  return 1 + 1 + 1 + kMaxDigits + 2 + 1 + passes + 1;
}

}  // namespace gs
