// Front-to-back alpha compositing over per-tile depth-ordered lists
// (Algorithm 1 "Rasterize"), and its backward pass with the L1 term of Eq. 5
// fused in.
//
// One thread block per 16x16 tile of any view in the batch, one pixel per
// thread; each warp owns an 8x4 block of the tile.  Splat records (48 B) are
// staged in shared memory 256 at a time with one cooperative load per
// thread, which also computes an 8-bit mask of the warps whose pixels the
// splat's alpha >= 1/255 support can reach (a conservative bounding box);
// a warp skips every staged splat whose bit it lacks with one uniform
// branch, before any per-pixel arithmetic.  A pixel stops before the splat
// that would drop its transmittance below 1e-4; the block leaves when all
// its pixels are done.
//
// The backward recomputes compositing back to front from T_final (only
// T_final and n_contrib are stored per pixel).  All 256 pixels of a block
// walk the same splat in lockstep, so its nine screen-space gradients are
// reduced in registers: a transposing warp reduction (9 shuffles for 8
// values + 5 for the ninth) followed by shared-memory adds from 9 lanes per
// warp, and one vector atomic per splat per tile into global memory.
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kTile = 16;
constexpr int kThreads = kTile * kTile;

struct TileInfo {
  int slot;
  int W, H;
  int tx, ty;
  long long px_offset;
  float inv_norm;  // 1 / (3 W H) for the per-view L1 mean
};

__device__ inline void find_tile(const gs_batch& batch, const gs_cameras& cams, int gt, TileInfo* ti) {
  if (threadIdx.x == 0) {
    int lo = 0, hi = batch.B - 1;
    while (lo < hi) {  // last slot with tile_offset[slot] <= gt
      const int mid = (lo + hi + 1) >> 1;
      if (batch.tile_offset[mid] <= gt) lo = mid;
      else hi = mid - 1;
    }
    const int v = slot_view(cams, batch, lo);
    TileInfo t;
    t.slot = lo;
    t.W = cams.wh[2 * v];
    t.H = cams.wh[2 * v + 1];
    const int tiles_x = (t.W + kTile - 1) / kTile;
    const int l = gt - batch.tile_offset[lo];
    t.tx = l % tiles_x;
    t.ty = l / tiles_x;
    t.px_offset = batch.px_offset[lo];
    t.inv_norm = 1.f / (3.f * (float)t.W * (float)t.H);
    *ti = t;
  }
}

// Pixel of thread `tid` in its 16x16 tile: warp w covers the 8x4 block at
// ((w & 1) * 8, (w >> 1) * 4), lane l the pixel (l & 7, l >> 3) in it.
__device__ inline void tile_pixel(int tid, int& lx, int& ly) {
  const int w = tid >> 5, l = tid & 31;
  lx = (w & 1) * 8 + (l & 7);
  ly = (w >> 1) * 4 + (l >> 3);
}

// Bit w set iff the bounding box of the splat's support {q <= q_max} can
// reach a pixel centre of warp w's 8x4 block in the tile at pixel (x0, y0).
// The box is widened by 2 % + 0.01 in q and 0.01 px: the FP32 evaluation of q
// for strongly anisotropic conics carries relative errors of that order, so
// no pixel that the exact alpha test would accept is ever skipped.
__device__ inline uint32_t warp_mask(const float4 xyo, const float4 con, float x0, float y0) {
  const float detc = con.x * con.z - con.y * con.y;
  const float qc = (con.w + 1e-3f) * 1.02f + 0.01f;
  const float rx = sqrtf(qc * con.z / detc) + 0.01f;
  const float ry = sqrtf(qc * con.x / detc) + 0.01f;
  uint32_t m = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const float bx0 = x0 + (float)((w & 1) * 8) + 0.5f, by0 = y0 + (float)((w >> 1) * 4) + 0.5f;
    const bool hit = (xyo.x + rx >= bx0) && (xyo.x - rx <= bx0 + 7.f) && (xyo.y + ry >= by0) &&
                     (xyo.y - ry <= by0 + 3.f);
    m |= hit ? (1u << w) : 0u;
  }
  return m;
}

// alpha of a staged splat at pixel centre (px, py); returns false when the
// splat cannot contribute (alpha < 1/255).  Shared by forward and backward
// so both take identical decisions.
__device__ inline bool splat_alpha(const float4 xyo, const float4 con, float px, float py,
                                   float& dx, float& dy, float& G, float& alpha) {
  dx = px - xyo.x;
  dy = py - xyo.y;
  const float q = con.x * dx * dx + 2.f * con.y * dx * dy + con.z * dy * dy;
  // q_max = 2 ln(255 o): beyond it (with margin far above FP32 error)
  // alpha is certainly below 1/255
  if (q > con.w + 1e-3f) return false;
  G = __expf(-0.5f * q);
  alpha = fminf(kAlphaMax, xyo.z * G);
  return alpha >= kAlphaMin;
}

__global__ void __launch_bounds__(kThreads) render_fwd_kernel(
    gs_batch batch, gs_cameras cams, const float4* __restrict__ splat, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, const float* __restrict__ bg, float* __restrict__ image,
    float* __restrict__ T_final, uint32_t* __restrict__ n_contrib) {
  __shared__ TileInfo ti;
  __shared__ float4 s_xyo[kThreads];
  __shared__ float4 s_con[kThreads];
  __shared__ float4 s_col[kThreads];
  __shared__ uint32_t s_mask[kThreads];
  const int gt = blockIdx.x;
  find_tile(batch, cams, gt, &ti);
  __syncthreads();
  int lx, ly;
  tile_pixel(threadIdx.x, lx, ly);
  const uint32_t wbit = 1u << (threadIdx.x >> 5);
  const int u = ti.tx * kTile + lx, v = ti.ty * kTile + ly;
  const bool inside = u < ti.W && v < ti.H;
  const float px = (float)u + 0.5f, py = (float)v + 0.5f;
  const float x0 = (float)(ti.tx * kTile), y0 = (float)(ti.ty * kTile);
  const uint32_t start = ranges[2 * gt], end = ranges[2 * gt + 1];
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0;
  bool done = !inside;
  for (uint32_t base = start; base < end; base += kThreads) {
    if (__syncthreads_count(done) == kThreads) break;
    const uint32_t idx = base + threadIdx.x;
    if (idx < end) {
      const uint32_t r = vals[idx];
      const float4 xyo = splat[3 * (size_t)r];
      const float4 con = splat[3 * (size_t)r + 1];
      s_xyo[threadIdx.x] = xyo;
      s_con[threadIdx.x] = con;
      s_col[threadIdx.x] = splat[3 * (size_t)r + 2];
      s_mask[threadIdx.x] = warp_mask(xyo, con, x0, y0);
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kThreads, end - base);
    for (int k = 0; k < cnt && !done; ++k) {
      if (!(s_mask[k] & wbit)) continue;  // uniform across the warp
      float dx, dy, G, alpha;
      if (!splat_alpha(s_xyo[k], s_con[k], px, py, dx, dy, G, alpha)) continue;
      const float Tn = T * (1.f - alpha);
      if (Tn < kTMin) {
        done = true;
        break;
      }
      const float4 c = s_col[k];
      const float w = alpha * T;
      C0 += c.x * w;
      C1 += c.y * w;
      C2 += c.z * w;
      T = Tn;
      last = base - start + (uint32_t)k + 1u;
    }
  }
  if (inside) {
    const size_t p = (size_t)ti.px_offset + (size_t)v * ti.W + u;
    image[3 * p + 0] = C0 + T * bg[0];
    image[3 * p + 1] = C1 + T * bg[1];
    image[3 * p + 2] = C2 + T * bg[2];
    T_final[p] = T;
    n_contrib[p] = last;
  }
}

// Sum of v[0..7] over the warp, transposed: afterwards lane L holds the sum
// of element ((L >> 2) & 7).  9 shuffles instead of 40.
__device__ inline float warp_sum8_transposed(const float* v, int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  float a[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = h16 ? v[i] : v[i + 4];
    const float keep = h16 ? v[i + 4] : v[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float b[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h8 ? a[i] : a[i + 2];
    const float keep = h8 ? a[i + 2] : a[i];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float c = (h4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h4 ? b[0] : b[1], 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

__global__ void __launch_bounds__(kThreads) render_bwd_kernel(
    gs_batch batch, gs_cameras cams, const float4* __restrict__ splat, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, const float* __restrict__ bg, const float* __restrict__ image,
    const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
    const float* __restrict__ v_image, const float* __restrict__ target, float l1_weight, double* loss,
    float* __restrict__ v2d) {
  __shared__ TileInfo ti;
  __shared__ float4 s_xyo[kThreads];
  __shared__ float4 s_con[kThreads];
  __shared__ float4 s_col[kThreads];
  __shared__ uint32_t s_rec[kThreads];
  __shared__ uint32_t s_mask[kThreads];
  __shared__ float s_g[kThreads][9];
  __shared__ uint32_t s_max;
  __shared__ float s_loss[kThreads / 32];
  const int gt = blockIdx.x;
  if (threadIdx.x == 0) s_max = 0;
  find_tile(batch, cams, gt, &ti);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  int lx, ly;
  tile_pixel(threadIdx.x, lx, ly);
  const uint32_t wbit = 1u << (threadIdx.x >> 5);
  const int u = ti.tx * kTile + lx, v = ti.ty * kTile + ly;
  const bool inside = u < ti.W && v < ti.H;
  const float px = (float)u + 0.5f, py = (float)v + 0.5f;
  const float x0 = (float)(ti.tx * kTile), y0 = (float)(ti.ty * kTile);
  const uint32_t start = ranges[2 * gt];
  float T = 1.f, S0 = 0.f, S1 = 0.f, S2 = 0.f, vC0 = 0.f, vC1 = 0.f, vC2 = 0.f;
  uint32_t nc = 0;
  float lsum = 0.f;
  if (inside) {
    const size_t p = (size_t)ti.px_offset + (size_t)v * ti.W + u;
    T = T_final[p];
    nc = n_contrib[p];
    S0 = T * bg[0];
    S1 = T * bg[1];
    S2 = T * bg[2];
    if (v_image) {
      vC0 = v_image[3 * p];
      vC1 = v_image[3 * p + 1];
      vC2 = v_image[3 * p + 2];
    } else {
      const float s = l1_weight * ti.inv_norm;
      const float d0 = image[3 * p] - target[3 * p];
      const float d1 = image[3 * p + 1] - target[3 * p + 1];
      const float d2 = image[3 * p + 2] - target[3 * p + 2];
      vC0 = d0 > 0.f ? s : (d0 < 0.f ? -s : 0.f);
      vC1 = d1 > 0.f ? s : (d1 < 0.f ? -s : 0.f);
      vC2 = d2 > 0.f ? s : (d2 < 0.f ? -s : 0.f);
      lsum = s * (fabsf(d0) + fabsf(d1) + fabsf(d2));
    }
    if (vC0 == 0.f && vC1 == 0.f && vC2 == 0.f) nc = 0;
    atomicMax(&s_max, nc);
  }
  if (loss != nullptr && v_image == nullptr) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0) s_loss[threadIdx.x >> 5] = lsum;
  }
  __syncthreads();
  if (loss != nullptr && v_image == nullptr && threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += (double)s_loss[w];
    if (t != 0.0) atomicAdd(loss, t);
  }
  const uint32_t n_end = s_max;  // positions [0, n_end) of the tile list
  const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, nc);
  for (int bend = (int)n_end; bend > 0; bend -= kThreads) {
    const int bstart = max(0, bend - kThreads);
    const int cnt = bend - bstart;
    if (threadIdx.x < cnt) {
      const uint32_t r = vals[start + bstart + threadIdx.x];
      const float4 xyo = splat[3 * (size_t)r];
      const float4 con = splat[3 * (size_t)r + 1];
      s_rec[threadIdx.x] = r;
      s_xyo[threadIdx.x] = xyo;
      s_con[threadIdx.x] = con;
      s_col[threadIdx.x] = splat[3 * (size_t)r + 2];
      s_mask[threadIdx.x] = warp_mask(xyo, con, x0, y0);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) s_g[threadIdx.x][i] = 0.f;
    __syncthreads();
    for (int k = cnt - 1; k >= 0; --k) {
      const uint32_t pos = (uint32_t)(bstart + k);
      // uniform across the warp: past all its pixels' last contributor, or
      // the splat cannot reach its 8x4 block
      if (pos >= warp_nc || !(s_mask[k] & wbit)) continue;
      float g[9];
      bool contrib = false;
      if (pos < nc) {
        float dx, dy, G, alpha;
        const float4 xyo = s_xyo[k];
        const float4 con = s_con[k];
        if (splat_alpha(xyo, con, px, py, dx, dy, G, alpha)) {
          contrib = true;
          const float4 c = s_col[k];
          const float ra = __fdividef(1.f, 1.f - alpha);  // 1 - alpha >= 0.01
          const float Tk = T * ra;
          const float w = alpha * Tk;
          g[6] = w * vC0;
          g[7] = w * vC1;
          g[8] = w * vC2;
          const float va = vC0 * (c.x * Tk - S0 * ra) + vC1 * (c.y * Tk - S1 * ra) +
                           vC2 * (c.z * Tk - S2 * ra);
          S0 += c.x * w;
          S1 += c.y * w;
          S2 += c.z * w;
          T = Tk;
          if (xyo.z * G < kAlphaMax) {
            const float vq = -0.5f * alpha * va;
            g[5] = va * G;
            g[0] = -2.f * vq * (con.x * dx + con.y * dy);
            g[1] = -2.f * vq * (con.y * dx + con.z * dy);
            g[2] = vq * dx * dx;
            g[3] = 2.f * vq * dx * dy;
            g[4] = vq * dy * dy;
          } else {
#pragma unroll
            for (int i = 0; i < 6; ++i) g[i] = 0.f;
          }
        }
      }
      if (!contrib) {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = 0.f;
      }
      if (__ballot_sync(0xffffffffu, contrib)) {
        // order: 0 mx, 1 my, 2 a, 3 b, 4 c, 5 opacity, 6 r, 7 g | 8 b
        const float s8 = warp_sum8_transposed(g, lane);
        float s9 = g[8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s9 += __shfl_xor_sync(0xffffffffu, s9, off);
        if ((lane & 3) == 0) atomicAdd(&s_g[k][(lane >> 2) & 7], s8);
        if (lane == 1) atomicAdd(&s_g[k][8], s9);
      }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      const float* sg = s_g[threadIdx.x];
      const float4 a = make_float4(sg[0], sg[1], sg[2], sg[3]);
      const float4 b = make_float4(sg[4], sg[5], sg[6], sg[7]);
      const bool nz = a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f || b.x != 0.f ||
                      b.y != 0.f || b.z != 0.f || b.w != 0.f || sg[8] != 0.f;
      if (nz) {
        float4* dst = reinterpret_cast<float4*>(v2d) + 3 * (size_t)s_rec[threadIdx.x];
        atomicAdd(dst, a);
        atomicAdd(dst + 1, b);
        atomicAdd(reinterpret_cast<float*>(dst + 2), sg[8]);
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_render_fwd(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                              const uint32_t* vals, const uint32_t* ranges, const float* bg,
                              float* image, float* T_final, uint32_t* n_contrib, cudaStream_t st) {
  if (batch.n_tiles == 0) return cudaSuccess;
  render_fwd_kernel<<<batch.n_tiles, kThreads, 0, st>>>(
      batch, cams, reinterpret_cast<const float4*>(proj.splat), vals, ranges, bg, image, T_final,
      n_contrib);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                              const uint32_t* vals, const uint32_t* ranges, const float* bg,
                              const float* image, const float* T_final, const uint32_t* n_contrib,
                              const float* v_image, const float* target, float l1_weight,
                              double* loss, float* v2d, cudaStream_t st) {
  if (batch.n_tiles == 0) return cudaSuccess;
  render_bwd_kernel<<<batch.n_tiles, kThreads, 0, st>>>(
      batch, cams, reinterpret_cast<const float4*>(proj.splat), vals, ranges, bg, image, T_final,
      n_contrib, v_image, target, l1_weight, loss, v2d);
  return cudaGetLastError();
}

}  // namespace gs
