// Photometric loss of Eq. 5 (Algorithm 1, "L_photo") with its SSIM term, and
// its gradient with respect to the rendered image.
//
// SSIM is the index of Wang et al. (2004) as 3DGS trains with it (the paper
// fixes only its weight): per colour channel, a separable 11x11 Gaussian
// window (sigma 1.5, 1-D taps normalised to sum 1), C1 = 0.01^2,
// C2 = 0.03^2, zero padding outside the view.  For one view of n = 3 W H
// values, L = l1_w mean|x - y| + ssim_w (1 - mean S) with
//   S = (2 mx my + C1)(2 cxy + C2) / ((mx^2 + my^2 + C1)(vx + vy + C2)),
//   mx = w*x, vx = w*(x^2) - mx^2, cxy = w*(x y) - mx my   (w* = window sum).
// With g = -ssim_w / n and the per-pixel factors
//   M1 = g (dS/dmx - 2 mx dS/dvx - my dS/dcxy),  M2 = g dS/dvx,  M3 = g dS/dcxy
// (dS/dmx taken with vx, cxy fixed), the gradient is
//   dL/dx = w*M1 + 2 x (w*M2) + y (w*M3) + l1_w sign(x - y) / n,
// the window sum being its own adjoint (symmetric taps, zero padding).
//
// Two kernels, one 256-thread block per 32x32 pixel block (a 32-pixel tile
// of the batch, or four 16-pixel tiles): the forward stages x and y of one
// channel with a 5-pixel halo in shared memory; the horizontal pass gives
// each thread four consecutive outputs of a staged row (14 inputs read once
// for 4 x 5 window sums), the vertical pass four consecutive outputs of a
// column (14 rows of the five horizontal sums); it writes M1..M3 (planar,
// channel-major) and the block's loss.  The backward stages M1..M3 the same
// way and writes v_image.  Shared-memory rows are padded so that both
// passes are free of bank conflicts.
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kR = 5;              // window radius
constexpr int kTaps = 2 * kR + 1;  // 11
constexpr int kBE = 32;            // pixel block edge
constexpr int kSE = kBE + 2 * kR;  // staged edge: 42
constexpr int kThreads = 256;
constexpr int kRun = 4;            // consecutive outputs per thread in each pass
constexpr int kRunH5 = 2;          // the forward's horizontal pass (five sums): two
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

// The 1-D window taps, identical in both kernels.
__device__ inline void window_taps(float* w) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kTaps; ++k) {
    const float d = (float)(k - kR);
    w[k] = expf(-d * d / (2.f * 1.5f * 1.5f));
    s += w[k];
  }
  const float is = 1.f / s;
#pragma unroll
  for (int k = 0; k < kTaps; ++k) w[k] *= is;
}

struct PixBlock {
  int W, H;      // the slot's view size
  int u0, v0;    // first pixel of the 32x32 block
  int64_t px;    // the slot's first pixel in the batch layout
  float inv_n;   // 1 / (3 W H)
  int valid;     // 0: this tile anchors no block (16-pixel tiles: odd x or y)
};

// The 32x32 block anchored at global tile gt (tile edge batch.tile, 16 or
// 32): the slot by binary search over tile_offset.  A 16-pixel tile anchors
// a block when both of its tile coordinates are even.  One thread's work.
__device__ inline void find_pixel_block(const gs_batch& batch, const gs_cameras& cams, int gt, PixBlock* out) {
  int lo = 0, hi = batch.B - 1;
  while (lo < hi) {  // last slot with tile_offset[slot] <= gt
    const int mid = (lo + hi + 1) >> 1;
    if (batch.tile_offset[mid] <= gt) lo = mid;
    else hi = mid - 1;
  }
  const int v = slot_view(cams, batch, lo);
  PixBlock b;
  b.W = cams.wh[2 * v];
  b.H = cams.wh[2 * v + 1];
  const int T = batch.tile;
  const int tiles_x = (b.W + T - 1) / T;
  const int l = gt - batch.tile_offset[lo];
  const int tx = l % tiles_x, ty = l / tiles_x;
  b.valid = ((T == kBE) || ((tx % 2) == 0 && (ty % 2) == 0)) && slot_consistent(batch, lo, b.W, b.H);
  b.u0 = tx * T;
  b.v0 = ty * T;
  b.px = batch.px_offset[lo];
  b.inv_n = 1.f / (3.f * (float)b.W * (float)b.H);
  *out = b;
}

// Stages channel c of NA per-pixel arrays around block b into s[0..NA)
// (zero outside the view).  Array k is interleaved [.., 3] when
// planar_stride == 0, else planar a[c * planar_stride + p].  Every load of
// the thread is issued before its first shared-memory store, so a block
// waits one memory latency per staging, not one per loop trip.
template <int NA>
__device__ inline void stage(const float* const* a, int c, int64_t planar_stride, const PixBlock& b,
                             float (*const* s)[kSE + 1]) {
  constexpr int kIt = (kSE * kSE + kThreads - 1) / kThreads;
  // the slot's channel-c base of each array; offsets within a view are
  // 32-bit (a view holds far fewer than 2^31 values)
  const float* base[NA];
  const int step = planar_stride ? 1 : 3;
#pragma unroll
  for (int k = 0; k < NA; ++k) base[k] = a[k] + (planar_stride ? c * planar_stride + b.px : 3 * b.px + c);
  float val[NA][kIt];
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int i = threadIdx.x + it * kThreads;
    const int r = i / kSE, q = i - r * kSE;
    const int u = b.u0 - kR + q, v = b.v0 - kR + r;
    const bool in = i < kSE * kSE && u >= 0 && u < b.W && v >= 0 && v < b.H;
    const int off = (v * b.W + u) * step;
#pragma unroll
    for (int k = 0; k < NA; ++k) val[k][it] = in ? base[k][off] : 0.f;
  }
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int i = threadIdx.x + it * kThreads;
    if (i < kSE * kSE) {
      const int r = i / kSE, q = i - r * kSE;
#pragma unroll
      for (int k = 0; k < NA; ++k) s[k][r][q] = val[k][it];
    }
  }
}

__device__ inline float block_sum(float v, float* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
  return t;  // valid in thread 0
}

// The tiles of the batch that anchor a 32x32 block (all of them for 32-pixel
// tiles, those with both tile coordinates even for 16-pixel ones), compacted
// into list[0 .. *count) in no particular order (each block writes its own
// pixels; only the loss's summation order depends on it).
__global__ void __launch_bounds__(256) photo_blocks_kernel(gs_batch batch, gs_cameras cams, uint32_t* count,
                                                           uint32_t* list) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = false;
  if (gt < batch.n_tiles && gt < batch.tile_offset[batch.B]) {
    PixBlock b;
    find_pixel_block(batch, cams, gt, &b);
    valid = b.valid;
  }
  const unsigned ballot = __ballot_sync(0xffffffffu, valid);
  if (ballot == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(ballot) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(ballot));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (valid) list[base + __popc(ballot & ((1u << lane) - 1u))] = (uint32_t)gt;
}

// Horizontal window sums of NQ staged arrays: hs[q][r][q0 + o] for the
// kRun outputs of each task (staged row r, first output q0); each input is
// read once per task.  f(j) returns the NQ values of staged column q0 + j.
template <int NQ, int RUN, typename F>
__device__ inline void horizontal_pass(const float* w, float (*hs)[kSE][kBE + 1], F f) {
  constexpr int kGroups = kBE / RUN;
  for (int t = threadIdx.x; t < kSE * kGroups; t += kThreads) {
    const int r = t / kGroups, q0 = (t % kGroups) * RUN;
    float a[RUN][NQ];
#pragma unroll
    for (int o = 0; o < RUN; ++o)
#pragma unroll
      for (int q = 0; q < NQ; ++q) a[o][q] = 0.f;
#pragma unroll
    for (int j = 0; j < RUN + 2 * kR; ++j) {
      float val[NQ];
      f(r, q0 + j, val);
#pragma unroll
      for (int o = 0; o < RUN; ++o) {
        const int k = j - o;
        if (k >= 0 && k < kTaps) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) a[o][q] = fmaf(w[k], val[q], a[o][q]);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < RUN; ++o)
#pragma unroll
      for (int q = 0; q < NQ; ++q) hs[q][r][q0 + o] = a[o][q];
  }
}

// Vertical window sums of the NQ horizontal sums for the RUN outputs of
// column col from row row0: m[o][q].
template <int NQ, int RUN>
__device__ inline void vertical_pass(const float* w, float (*hs)[kSE][kBE + 1], int col, int row0,
                                     float (*m)[NQ]) {
#pragma unroll
  for (int o = 0; o < RUN; ++o)
#pragma unroll
    for (int q = 0; q < NQ; ++q) m[o][q] = 0.f;
#pragma unroll
  for (int j = 0; j < RUN + 2 * kR; ++j) {
    float val[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) val[q] = hs[q][row0 + j][col];
#pragma unroll
    for (int o = 0; o < RUN; ++o) {
      const int k = j - o;
      if (k >= 0 && k < kTaps) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) m[o][q] = fmaf(w[k], val[q], m[o][q]);
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads, 3) photo_fwd_kernel(gs_batch batch, gs_cameras cams,
                                                             const uint32_t* __restrict__ count,
                                                             const uint32_t* __restrict__ list,
                                                             const float* __restrict__ image,
                                                             const float* __restrict__ target, float l1_w,
                                                             float ssim_w, double* loss, float* __restrict__ m1,
                                                             float* __restrict__ m2, float* __restrict__ m3) {
  __shared__ float sx[kSE][kSE + 1], sy[kSE][kSE + 1];
  __shared__ float hs[5][kSE][kBE + 1];  // horizontal sums of x, y, x^2, y^2, x y
  __shared__ PixBlock blk;
  __shared__ float red[kThreads / 32];
  if (blockIdx.x >= *count) return;  // the grid is sized for every tile
  if (threadIdx.x == 0) find_pixel_block(batch, cams, (int)list[blockIdx.x], &blk);
  float w[kTaps];
  window_taps(w);
  __syncthreads();
  const PixBlock b = blk;
  float acc = 0.f;
  if (b.valid && b.u0 < b.W && b.v0 < b.H) {  // block-uniform
    const int64_t P = batch.n_pixels;
    const int col = threadIdx.x % kBE, row0 = (threadIdx.x / kBE) * kRun;
    for (int c = 0; c < 3; ++c) {
      {
        const float* src[2] = {image, target};
        float (*dst[2])[kSE + 1] = {sx, sy};
        stage<2>(src, c, 0, b, dst);
      }
      __syncthreads();
      horizontal_pass<5, kRunH5>(w, hs, [&](int r, int q, float* val) {
        const float xv = sx[r][q], yv = sy[r][q];
        val[0] = xv;
        val[1] = yv;
        val[2] = xv * xv;
        val[3] = yv * yv;
        val[4] = xv * yv;
      });
      __syncthreads();
      float m[kRun][5];
      vertical_pass<5, kRun>(w, hs, col, row0, m);
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        const int u = b.u0 + col, v = b.v0 + row0 + o;
        if (u < b.W && v < b.H) {
          const float mx = m[o][0], my = m[o][1];
          const float vx = m[o][2] - mx * mx, vy = m[o][3] - my * my, cxy = m[o][4] - mx * my;
          const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
          const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
          const float D = 1.f / (B1 * B2);
          const float S = A1 * A2 * D;
          const float dS_dmx = 2.f * my * A2 * D - 2.f * mx * S / B1;
          const float dS_dvx = -S / B2;
          const float dS_dcxy = 2.f * A1 * D;
          const float g = -ssim_w * b.inv_n;
          const int64_t p = b.px + (int64_t)v * b.W + u;
          m1[c * P + p] = g * (dS_dmx - 2.f * mx * dS_dvx - my * dS_dcxy);
          m2[c * P + p] = g * dS_dvx;
          m3[c * P + p] = g * dS_dcxy;
          const float d = sx[row0 + o + kR][col + kR] - sy[row0 + o + kR][col + kR];
          acc += b.inv_n * (ssim_w * (1.f - S) + l1_w * fabsf(d));
        }
      }
      __syncthreads();  // the staged arrays are rewritten for the next channel
    }
  }
  const float t = block_sum(acc, red);
  if (threadIdx.x == 0 && loss != nullptr && t != 0.f) atomicAdd(loss, (double)t);
}

__global__ void __launch_bounds__(kThreads, 3) photo_bwd_kernel(gs_batch batch, gs_cameras cams,
                                                             const uint32_t* __restrict__ count,
                                                             const uint32_t* __restrict__ list,
                                                             const float* __restrict__ image,
                                                             const float* __restrict__ target, float l1_w,
                                                             const float* __restrict__ m1,
                                                             const float* __restrict__ m2,
                                                             const float* __restrict__ m3,
                                                             float* __restrict__ v_image) {
  __shared__ float s1[kSE][kSE + 1], s2[kSE][kSE + 1], s3[kSE][kSE + 1];
  __shared__ float hs[3][kSE][kBE + 1];
  __shared__ PixBlock blk;
  if (blockIdx.x >= *count) return;  // the grid is sized for every tile
  if (threadIdx.x == 0) find_pixel_block(batch, cams, (int)list[blockIdx.x], &blk);
  float w[kTaps];
  window_taps(w);
  __syncthreads();
  const PixBlock b = blk;
  if (!(b.valid && b.u0 < b.W && b.v0 < b.H)) return;  // block-uniform
  const int64_t P = batch.n_pixels;
  const int col = threadIdx.x % kBE, row0 = (threadIdx.x / kBE) * kRun;
  for (int c = 0; c < 3; ++c) {
    // this thread's four pixels of the channel, read along with the staging
    float xv[kRun], yv[kRun];
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
      const int u = b.u0 + col, v = b.v0 + row0 + o;
      const int64_t p = b.px + (int64_t)v * b.W + u;
      const bool in = u < b.W && v < b.H;
      xv[o] = in ? image[3 * p + c] : 0.f;
      yv[o] = in ? target[3 * p + c] : 0.f;
    }
    {
      const float* src[3] = {m1, m2, m3};
      float (*dst[3])[kSE + 1] = {s1, s2, s3};
      stage<3>(src, c, P, b, dst);
    }
    __syncthreads();
    horizontal_pass<3, kRun>(w, hs, [&](int r, int q, float* val) {
      val[0] = s1[r][q];
      val[1] = s2[r][q];
      val[2] = s3[r][q];
    });
    __syncthreads();
    float f[kRun][3];
    vertical_pass<3, kRun>(w, hs, col, row0, f);
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
      const int u = b.u0 + col, v = b.v0 + row0 + o;
      if (u < b.W && v < b.H) {
        const int64_t p = b.px + (int64_t)v * b.W + u;
        const float d = xv[o] - yv[o];
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        v_image[3 * p + c] = f[o][0] + 2.f * xv[o] * f[o][1] + yv[o] * f[o][2] + l1_w * b.inv_n * sgn;
      }
    }
    __syncthreads();
  }
}

}  // namespace

size_t photo_loss_ws_bytes(int64_t n_pixels, int32_t n_tiles) {
  return (size_t)n_pixels * 9 * sizeof(float) + ((size_t)n_tiles + 1) * sizeof(uint32_t);
}

cudaError_t launch_photo_loss(const gs_batch& batch, const gs_cameras& cams, const float* image,
                              const float* target, float l1_weight, float ssim_weight, double* loss,
                              float* v_image, float* ws, cudaStream_t st) {
  if (batch.n_tiles == 0 || batch.n_pixels == 0) return cudaSuccess;
  const int64_t P = batch.n_pixels;
  float* m1 = ws;
  float* m2 = ws + 3 * P;
  float* m3 = ws + 6 * P;
  uint32_t* count = reinterpret_cast<uint32_t*>(ws + 9 * P);
  uint32_t* list = count + 1;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  photo_blocks_kernel<<<(batch.n_tiles + 255) / 256, 256, 0, st>>>(batch, cams, count, list);
  photo_fwd_kernel<<<batch.n_tiles, kThreads, 0, st>>>(batch, cams, count, list, image, target, l1_weight,
                                                       ssim_weight, loss, m1, m2, m3);
  photo_bwd_kernel<<<batch.n_tiles, kThreads, 0, st>>>(batch, cams, count, list, image, target, l1_weight, m1, m2,
                                                       m3, v_image);
  return cudaGetLastError();
}

}  // namespace gs
