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
// Two kernels, one 256-thread block per 16x16 pixel block (a tile of the
// batch holds one or four of them): the forward stages x and y of one
// channel with a 5-pixel halo in shared memory, runs the window as a
// horizontal pass over the 26 staged rows and a vertical pass per pixel,
// and writes M1..M3 (planar, channel-major) and the block's loss; the
// backward stages M1..M3 the same way and writes v_image.  Both are bound
// by FP32 issue (~55 FMAs per window quantity per pixel and channel).
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kR = 5;              // window radius
constexpr int kTaps = 2 * kR + 1;  // 11
constexpr int kBE = 16;            // pixel block edge
constexpr int kSE = kBE + 2 * kR;  // staged edge: 26
constexpr int kThreads = kBE * kBE;
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
  int u0, v0;    // first pixel of the 16x16 block
  int64_t px;    // the slot's first pixel in the batch layout
  float inv_n;   // 1 / (3 W H)
};

// 16x16 block `sub` of global tile gt (tile edge batch.tile): the slot by
// binary search over tile_offset.  Thread 0 only.
__device__ inline void find_pixel_block(const gs_batch& batch, const gs_cameras& cams, int gt, int sub,
                                        PixBlock* out) {
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
  const int per = T / kBE;
  b.u0 = (l % tiles_x) * T + (sub % per) * kBE;
  b.v0 = (l / tiles_x) * T + (sub / per) * kBE;
  b.px = batch.px_offset[lo];
  b.inv_n = 1.f / (3.f * (float)b.W * (float)b.H);
  *out = b;
}

// Stages channel c of the per-pixel array a (interleaved [.., 3] when
// planar_stride == 0, else planar a[c * planar_stride + p]) around block b
// into s (zero outside the view).
__device__ inline void stage(const float* __restrict__ a, int c, int64_t planar_stride, const PixBlock& b,
                             float (*s)[kSE + 1]) {
  for (int i = threadIdx.x; i < kSE * kSE; i += kThreads) {
    const int r = i / kSE, q = i - r * kSE;
    const int u = b.u0 - kR + q, v = b.v0 - kR + r;
    float val = 0.f;
    if (u >= 0 && u < b.W && v >= 0 && v < b.H) {
      const int64_t p = b.px + (int64_t)v * b.W + u;
      val = planar_stride ? a[c * planar_stride + p] : a[3 * p + c];
    }
    s[r][q] = val;
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

__global__ void __launch_bounds__(kThreads) photo_fwd_kernel(gs_batch batch, gs_cameras cams,
                                                             const float* __restrict__ image,
                                                             const float* __restrict__ target, float l1_w,
                                                             float ssim_w, double* loss, float* __restrict__ m1,
                                                             float* __restrict__ m2, float* __restrict__ m3) {
  __shared__ float sx[kSE][kSE + 1], sy[kSE][kSE + 1];
  __shared__ float hs[5][kSE][kBE];  // horizontal sums of x, y, x^2, y^2, x y
  __shared__ PixBlock blk;
  __shared__ float red[kThreads / 32];
  float w[kTaps];
  window_taps(w);
  const int tx = threadIdx.x % kBE, ty = threadIdx.x / kBE;
  const int64_t P = batch.n_pixels;
  const int subs = (batch.tile / kBE) * (batch.tile / kBE);
  float acc = 0.f;
  for (int sub = 0; sub < subs; ++sub) {
    if (threadIdx.x == 0) find_pixel_block(batch, cams, blockIdx.x, sub, &blk);
    __syncthreads();
    const PixBlock b = blk;
    __syncthreads();  // blk is rewritten by the next sub-block
    if (b.u0 >= b.W || b.v0 >= b.H) continue;  // block-uniform
    const int u = b.u0 + tx, v = b.v0 + ty;
    const bool inside = u < b.W && v < b.H;
    const int64_t p = b.px + (int64_t)v * b.W + u;
    for (int c = 0; c < 3; ++c) {
      stage(image, c, 0, b, sx);
      stage(target, c, 0, b, sy);
      __syncthreads();
      for (int i = threadIdx.x; i < kSE * kBE; i += kThreads) {
        const int r = i / kBE, q = i - r * kBE;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) {
          const float xv = sx[r][q + k], yv = sy[r][q + k];
          a0 = fmaf(w[k], xv, a0);
          a1 = fmaf(w[k], yv, a1);
          a2 = fmaf(w[k], xv * xv, a2);
          a3 = fmaf(w[k], yv * yv, a3);
          a4 = fmaf(w[k], xv * yv, a4);
        }
        hs[0][r][q] = a0;
        hs[1][r][q] = a1;
        hs[2][r][q] = a2;
        hs[3][r][q] = a3;
        hs[4][r][q] = a4;
      }
      __syncthreads();
      float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
      for (int k = 0; k < kTaps; ++k) {
        mx = fmaf(w[k], hs[0][ty + k][tx], mx);
        my = fmaf(w[k], hs[1][ty + k][tx], my);
        exx = fmaf(w[k], hs[2][ty + k][tx], exx);
        eyy = fmaf(w[k], hs[3][ty + k][tx], eyy);
        exy = fmaf(w[k], hs[4][ty + k][tx], exy);
      }
      if (inside) {
        const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
        const float D = 1.f / (B1 * B2);
        const float S = A1 * A2 * D;
        const float dS_dmx = 2.f * my * A2 * D - 2.f * mx * S / B1;
        const float dS_dvx = -S / B2;
        const float dS_dcxy = 2.f * A1 * D;
        const float g = -ssim_w * b.inv_n;
        m1[c * P + p] = g * (dS_dmx - 2.f * mx * dS_dvx - my * dS_dcxy);
        m2[c * P + p] = g * dS_dvx;
        m3[c * P + p] = g * dS_dcxy;
        const float d = sx[ty + kR][tx + kR] - sy[ty + kR][tx + kR];
        acc += b.inv_n * (ssim_w * (1.f - S) + l1_w * fabsf(d));
      }
      __syncthreads();  // the staged arrays are rewritten for the next channel
    }
  }
  const float t = block_sum(acc, red);
  if (threadIdx.x == 0 && loss != nullptr && t != 0.f) atomicAdd(loss, (double)t);
}

__global__ void __launch_bounds__(kThreads) photo_bwd_kernel(gs_batch batch, gs_cameras cams,
                                                             const float* __restrict__ image,
                                                             const float* __restrict__ target, float l1_w,
                                                             const float* __restrict__ m1,
                                                             const float* __restrict__ m2,
                                                             const float* __restrict__ m3,
                                                             float* __restrict__ v_image) {
  __shared__ float s1[kSE][kSE + 1], s2[kSE][kSE + 1], s3[kSE][kSE + 1];
  __shared__ float hs[3][kSE][kBE];
  __shared__ PixBlock blk;
  float w[kTaps];
  window_taps(w);
  const int tx = threadIdx.x % kBE, ty = threadIdx.x / kBE;
  const int64_t P = batch.n_pixels;
  const int subs = (batch.tile / kBE) * (batch.tile / kBE);
  for (int sub = 0; sub < subs; ++sub) {
    if (threadIdx.x == 0) find_pixel_block(batch, cams, blockIdx.x, sub, &blk);
    __syncthreads();
    const PixBlock b = blk;
    __syncthreads();
    if (b.u0 >= b.W || b.v0 >= b.H) continue;  // block-uniform
    const int u = b.u0 + tx, v = b.v0 + ty;
    const bool inside = u < b.W && v < b.H;
    const int64_t p = b.px + (int64_t)v * b.W + u;
    for (int c = 0; c < 3; ++c) {
      stage(m1, c, P, b, s1);
      stage(m2, c, P, b, s2);
      stage(m3, c, P, b, s3);
      __syncthreads();
      for (int i = threadIdx.x; i < kSE * kBE; i += kThreads) {
        const int r = i / kBE, q = i - r * kBE;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) {
          a0 = fmaf(w[k], s1[r][q + k], a0);
          a1 = fmaf(w[k], s2[r][q + k], a1);
          a2 = fmaf(w[k], s3[r][q + k], a2);
        }
        hs[0][r][q] = a0;
        hs[1][r][q] = a1;
        hs[2][r][q] = a2;
      }
      __syncthreads();
      float f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
      for (int k = 0; k < kTaps; ++k) {
        f1 = fmaf(w[k], hs[0][ty + k][tx], f1);
        f2 = fmaf(w[k], hs[1][ty + k][tx], f2);
        f3 = fmaf(w[k], hs[2][ty + k][tx], f3);
      }
      if (inside) {
        const float xv = image[3 * p + c], yv = target[3 * p + c];
        const float d = xv - yv;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        v_image[3 * p + c] = f1 + 2.f * xv * f2 + yv * f3 + l1_w * b.inv_n * sgn;
      }
      __syncthreads();
    }
  }
}

}  // namespace

size_t photo_loss_ws_bytes(int64_t n_pixels) { return (size_t)n_pixels * 9 * sizeof(float); }

cudaError_t launch_photo_loss(const gs_batch& batch, const gs_cameras& cams, const float* image,
                              const float* target, float l1_weight, float ssim_weight, double* loss,
                              float* v_image, float* ws, cudaStream_t st) {
  if (batch.n_tiles == 0 || batch.n_pixels == 0) return cudaSuccess;
  const int64_t P = batch.n_pixels;
  float* m1 = ws;
  float* m2 = ws + 3 * P;
  float* m3 = ws + 6 * P;
  photo_fwd_kernel<<<batch.n_tiles, kThreads, 0, st>>>(batch, cams, image, target, l1_weight, ssim_weight, loss,
                                                       m1, m2, m3);
  photo_bwd_kernel<<<batch.n_tiles, kThreads, 0, st>>>(batch, cams, image, target, l1_weight, m1, m2, m3,
                                                       v_image);
  return cudaGetLastError();
}

}  // namespace gs
