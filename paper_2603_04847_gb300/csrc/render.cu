// Front-to-back alpha compositing over per-tile depth-ordered lists
// (Algorithm 1 "Rasterize"), and its backward pass with the L1 term of Eq. 5
// fused in.
//
// One thread block per tile of any view in the batch (16x16 tiles: 128
// threads; 32x32 tiles: 512 threads; the batch's tile size is chosen by the
// autotuner).  Each warp owns an 8x8 block of the tile and each thread two
// pixels of it,
// (x, y) and (x + 4, y): the per-splat shared-memory loads, the cull test
// and the loop overhead are paid once per two pixels, and in the backward
// one warp reduction covers 64 pixels.
//
// Splat records are staged in shared memory kBatch at a time (64, 128 or 256,
// chosen for the forward and the backward separately by the autotuner
// through gs_set_tuning).  Staging turns each record into the exponent form
// alpha_raw = 2^e with
//   e = A dx^2 + B dx dy + C dy^2 + log2(opacity),
//   A = -a/(2 ln 2), B = -b/ln 2, C = -c/(2 ln 2)  (conic a, b, c),
// so that the alpha >= 1/255 test is one compare and one exp2 per pixel, and
// computes a 4-bit mask of the warps whose 8x8 block the splat's support can
// reach (a conservative bounding box).  Each warp then compacts the staged
// splats with its bit into a list (ballots) and walks only those.  Forward
// and backward evaluate alpha with the same function on the same staged
// values, so they take identical decisions.
//
// The backward recomputes compositing back to front from T_final (only
// T_final and n_contrib are stored per pixel).  All lanes of a warp walk the
// same splat in lockstep, so its nine per-splat sums (colour gradients and
// the moments of the conic/mean/opacity gradients) are reduced in registers
// — a transposing warp reduction (9 shuffles for 8 values + 5 for the
// ninth) — then stored by 9 lanes into the warp's own shared-memory slots
// (kBatch <= 128; with 256 the warps share one slot set through shared
// atomics), summed over the warps per splat, and written with one vector
// atomic per splat per tile.
#include "gs_internal.h"

namespace gs {

namespace {

// Tile shapes: kTile x kTile pixels per block, two pixels per thread, an
// 8x8 pixel block per warp.
template <int kTile>
struct Shape {
  static constexpr int kThreads = kTile * kTile / 2;
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kWarpsX = kTile / 8;
  static_assert(kWarps <= 32, "one mask bit per warp");
};
constexpr float kLn2 = 0.69314718055994531f;
constexpr float kHalfLog2e = 0.72134752044448170f;  // 1 / (2 ln 2)

struct TileInfo {
  int slot;
  int W, H;
  int tx, ty;
  long long px_offset;
  float inv_norm;  // 1 / (3 W H) for the per-view L1 mean
};

template <int kTile>
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

// Pixels of thread `tid` in its tile: warp w covers the 8x8 block at
// ((w % kWarpsX) * 8, (w / kWarpsX) * 8); lane l the pixels (l & 3, l >> 2)
// and ((l & 3) + 4, l >> 2) in it — one row, so that the row-dependent part
// of the exponent is computed once for both.
template <int kTile>
__device__ inline void tile_pixels(int tid, int& lx, int& ly) {
  constexpr int kWX = Shape<kTile>::kWarpsX;
  const int w = tid >> 5, l = tid & 31;
  lx = (w % kWX) * 8 + (l & 3);
  ly = (w / kWX) * 8 + (l >> 2);
}

// Bit w set iff the splat's support {q <= q_max} can reach a pixel centre
// of warp w's 8x8 block in the tile at pixel (x0, y0).  The test is exact
// for the ellipse against the block's rectangle of pixel centres: the
// minimum of q over the rectangle is 0 when the mean lies inside it, else
// it is reached on the edge line facing the mean in x or the one in y, where
// the line minimum of q = c (dy + (b/c) dx)^2 + (det/c) dx^2 (resp. with x, y
// and a, c exchanged) is taken at the clamped stationary point.  Both forms
// are sums of non-negative terms, so FP32 evaluation loses nothing to
// cancellation.  q_max is widened by 2 % + 0.01 and the rectangle by 0.01 px:
// the FP32 evaluation of alpha for strongly anisotropic conics carries
// relative errors of that order, so no pixel whose alpha can pass the test
// is ever skipped.
template <int kTile>
__device__ inline uint32_t warp_mask(const float4 xyo, const float4 con, float x0, float y0) {
  constexpr int kWX = Shape<kTile>::kWarpsX;
  const float a = con.x, b = con.y, c = con.z;
  const float det = a * c - b * b;
  const float qc = (con.w + 1e-3f) * 1.02f + 0.01f;
  const float ia = __frcp_rn(a), ic = __frcp_rn(c);
  const float ba = b * ia, bc = b * ic, da = det * ia, dc = det * ic;
  uint32_t m = 0;
#pragma unroll
  for (int w = 0; w < Shape<kTile>::kWarps; ++w) {
    const float bx0 = x0 + (float)((w % kWX) * 8) + 0.49f, by0 = y0 + (float)((w / kWX) * 8) + 0.49f;
    const float bx1 = bx0 + 7.02f, by1 = by0 + 7.02f;
    // on the vertical line through the rectangle's x nearest the mean
    const float dx = fminf(fmaxf(xyo.x, bx0), bx1) - xyo.x;
    const float ev = fminf(fmaxf(xyo.y - bc * dx, by0), by1) - xyo.y + bc * dx;
    const float qv = c * ev * ev + dc * dx * dx;
    // on the horizontal line through the rectangle's y nearest the mean
    const float dy = fminf(fmaxf(xyo.y, by0), by1) - xyo.y;
    const float eh = fminf(fmaxf(xyo.x - ba * dy, bx0), bx1) - xyo.x + ba * dy;
    const float qh = a * eh * eh + da * dy * dy;
    m |= (fminf(qv, qh) <= qc) ? (1u << w) : 0u;
  }
  return m;
}

__device__ inline float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ inline float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Stages record r into slot `s` of the shared arrays.
template <int kTile>
__device__ inline void stage_splat(int s, uint32_t r, const float4* __restrict__ splat, float x0, float y0,
                                   float2* s_m, float4* s_q, float4* s_c, uint32_t* s_mask) {
  const float4 xyo = splat[3 * (size_t)r];
  const float4 con = splat[3 * (size_t)r + 1];
  const float4 col = splat[3 * (size_t)r + 2];
  s_m[s] = make_float2(xyo.x, xyo.y);
  s_q[s] = make_float4(-kHalfLog2e * con.x, -2.f * kHalfLog2e * con.y, -kHalfLog2e * con.z, lg2_approx(xyo.z));
  s_c[s] = make_float4(col.x, col.y, col.z, 1.f / xyo.z);
  s_mask[s] = warp_mask<kTile>(xyo, con, x0, y0);
}

// Exponent e = A dx^2 + B dx dy + C dy^2 + log2 o of alpha_raw = 2^e at
// offset (dx, dy), from the row terms Bdy = B dy and sy = C dy^2 + log2 o
// (row_terms).  Written with explicit roundings so that every kernel
// computes the same value from the same staged inputs.
__device__ inline void row_terms(const float4 q, float dy, float& Bdy, float& sy) {
  Bdy = __fmul_rn(q.y, dy);
  sy = __fmaf_rn(__fmul_rn(q.z, dy), dy, q.w);
}

__device__ inline float splat_exponent(const float4 q, float dx, float Bdy, float sy) {
  return __fmaf_rn(__fmaf_rn(q.x, dx, Bdy), dx, sy);
}

// Positions s < min(cnt, limit) of the staged batch whose mask has this
// warp's bit, in increasing order, into list; returns how many.  Warp-wide.
template <int kBatch>
__device__ inline int warp_list(const uint32_t* s_mask, uint32_t wbit, int cnt, int limit, uint8_t* list,
                                int lane) {
  const int lim = min(cnt, limit);
  int n = 0;
#pragma unroll
  for (int c = 0; c < kBatch; c += 32) {
    const int s = c + lane;
    const bool hit = s < lim && (s_mask[s] & wbit);
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    if (hit) list[n + __popc(b & ((1u << lane) - 1u))] = (uint8_t)s;
    n += __popc(b);
  }
  __syncwarp();
  return n;
}

// 10 blocks of 16x16 per SM (48 registers, no spills) measured 3 % faster
// than the 8 that 64 registers allow
template <int kTile, int kBatch, bool kCountAdded>
__global__ void __launch_bounds__(Shape<kTile>::kThreads, (kTile == 16 ? 10 : 2)) render_fwd_kernel(
    gs_batch batch, gs_cameras cams, const float4* __restrict__ splat, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, const float* __restrict__ bg, float* __restrict__ image,
    float* __restrict__ T_final, uint32_t* __restrict__ n_contrib, uint32_t* __restrict__ n_added) {
  constexpr int kThreads = Shape<kTile>::kThreads;
  __shared__ TileInfo ti;
  __shared__ float2 s_m[kBatch];
  __shared__ float4 s_q[kBatch];
  __shared__ float4 s_c[kBatch];
  __shared__ uint32_t s_mask[kBatch];
  __shared__ uint8_t s_list[kThreads / 32][kBatch];
  const int gt = blockIdx.x;
  find_tile<kTile>(batch, cams, gt, &ti);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lx, ly;
  tile_pixels<kTile>(threadIdx.x, lx, ly);
  const uint32_t wbit = 1u << warp;
  const int u0 = ti.tx * kTile + lx, u1 = u0 + 4, v = ti.ty * kTile + ly;
  const bool in0 = u0 < ti.W && v < ti.H, in1 = u1 < ti.W && v < ti.H;
  const float px0 = (float)u0 + 0.5f, px1 = (float)u1 + 0.5f, py = (float)v + 0.5f;
  const float x0 = (float)(ti.tx * kTile), y0 = (float)(ti.ty * kTile);
  const uint32_t start = ranges[2 * gt], end = ranges[2 * gt + 1];
  float T0 = 1.f, T1 = 1.f;
  float C00 = 0.f, C01 = 0.f, C02 = 0.f, C10 = 0.f, C11 = 0.f, C12 = 0.f;
  uint32_t last0 = 0, last1 = 0, add0 = 0, add1 = 0;
  bool done0 = !in0, done1 = !in1;
  // a finished pixel gets an unreachable threshold, so the per-splat test
  // is one compare (alpha = min(0.99, alpha_raw) >= 1/255 iff
  // alpha_raw >= 1/255)
  float thr0 = done0 ? 2.f : kAlphaMin, thr1 = done1 ? 2.f : kAlphaMin;
  for (uint32_t base = start; base < end; base += kBatch) {
    if (__syncthreads_count(done0 && done1) == kThreads) break;
    for (int s = threadIdx.x; s < kBatch; s += kThreads) {
      const uint32_t idx = base + s;
      if (idx < end) stage_splat<kTile>(s, vals[idx], splat, x0, y0, s_m, s_q, s_c, s_mask);
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kBatch, end - base);
    const int n_mine = warp_list<kBatch>(s_mask, wbit, cnt, kBatch, s_list[warp], lane);
    if (done0 && done1) continue;
    for (int i = 0; i < n_mine; ++i) {
      const int k = s_list[warp][i];
      const float2 m = s_m[k];
      const float4 q = s_q[k];
      float Bdy, sy;
      row_terms(q, py - m.y, Bdy, sy);
      const float r0 = ex2_approx(splat_exponent(q, px0 - m.x, Bdy, sy));
      const float r1 = ex2_approx(splat_exponent(q, px1 - m.x, Bdy, sy));
      const bool c0 = r0 >= thr0;
      const bool c1 = r1 >= thr1;
      if (!(c0 || c1)) continue;
      const float4 c = s_c[k];
      const uint32_t pos1 = base - start + (uint32_t)k + 1u;
      if (c0) {
        const float a0 = fminf(kAlphaMax, r0);
        const float Tn = T0 * (1.f - a0);
        if (Tn < kTMin) {
          done0 = true;
          thr0 = 2.f;
        } else {
          const float w = a0 * T0;
          C00 += c.x * w;
          C01 += c.y * w;
          C02 += c.z * w;
          T0 = Tn;
          last0 = pos1;
          if constexpr (kCountAdded) ++add0;
        }
      }
      if (c1) {
        const float a1 = fminf(kAlphaMax, r1);
        const float Tn = T1 * (1.f - a1);
        if (Tn < kTMin) {
          done1 = true;
          thr1 = 2.f;
        } else {
          const float w = a1 * T1;
          C10 += c.x * w;
          C11 += c.y * w;
          C12 += c.z * w;
          T1 = Tn;
          last1 = pos1;
          if constexpr (kCountAdded) ++add1;
        }
      }
      if (done0 && done1) break;
    }
  }
  if (in0) {
    const size_t p = (size_t)ti.px_offset + (size_t)v * ti.W + u0;
    image[3 * p + 0] = C00 + T0 * bg[0];
    image[3 * p + 1] = C01 + T0 * bg[1];
    image[3 * p + 2] = C02 + T0 * bg[2];
    T_final[p] = T0;
    n_contrib[p] = last0;
    if constexpr (kCountAdded) n_added[p] = add0;
  }
  if (in1) {
    const size_t p = (size_t)ti.px_offset + (size_t)v * ti.W + u1;
    image[3 * p + 0] = C10 + T1 * bg[0];
    image[3 * p + 1] = C11 + T1 * bg[1];
    image[3 * p + 2] = C12 + T1 * bg[2];
    T_final[p] = T1;
    n_contrib[p] = last1;
    if constexpr (kCountAdded) n_added[p] = add1;
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

// Per-pixel backward state.
// The colour composited behind the current splat, S, enters the gradient
// only through v . S (v = dL/dC is fixed per pixel), so that dot product is
// carried instead of S.
struct PixBwd {
  float T, vS, v0, v1, v2;
  uint32_t nc;
};

// Backward of one accepted splat at one pixel (alpha_raw = 2^e, alpha its
// clamp); adds this pixel's terms into g.  With u = alpha dL/dalpha (so
// dL/dq = -u/2 for q = a dx^2 + 2 b dx dy + c dy^2, d = pixel - mean) the
// conic, mean and opacity gradients are linear in the moments
//   g0 = sum u dx, g1 = sum u dy, g2 = sum u dx^2, g3 = sum u dx dy,
//   g4 = sum u dy^2, g5 = sum dL/dalpha alpha_raw
// (pixels where alpha is clamped at 0.99 contribute none), which are
// accumulated instead and mapped to gradients once per splat
// (moments_to_grad); g6..8 are the colour gradients.
__device__ inline void bwd_pixel(PixBwd& P, const float4 c, float dx, float dy, float araw, float alpha,
                                 float* g) {
  const float ra = __fdividef(1.f, 1.f - alpha);  // 1 - alpha >= 0.01
  const float Tk = P.T * ra;                      // transmittance before this splat
  const float w = alpha * Tk;
  g[6] += w * P.v0;
  g[7] += w * P.v1;
  g[8] += w * P.v2;
  const float vc = P.v0 * c.x + P.v1 * c.y + P.v2 * c.z;
  const float va = vc * Tk - P.vS * ra;  // dL/dalpha = v . (c T_k - S / (1 - alpha))
  P.vS += vc * w;
  P.T = Tk;
  if (araw < kAlphaMax) {
    const float u = alpha * va;
    const float udx = u * dx, udy = u * dy;
    g[0] += udx;
    g[1] += udy;
    g[2] += udx * dx;
    g[3] += udx * dy;
    g[4] += udy * dy;
    g[5] += va * araw;
  }
}

// Screen-space gradient record of a splat from its summed moments (see
// bwd_pixel), with the staged exponent form q = (A, B, C, log2 o), A =
// -a/(2 ln 2), B = -b/ln 2, C = -c/(2 ln 2), and inv_o = 1/o:
//   dL/dmean = -dL/dd = sum u (a dx + b dy, b dx + c dy)
//            = -ln 2 (2A M0 + B M1, B M0 + 2C M1)
//   dL/da = -M2/2, dL/db = -M3, dL/dc = -M4/2, dL/do = M5 / o.
__device__ inline void moments_to_grad(const float* M, float4 q, float inv_o, float4& ga, float4& gb) {
  ga = make_float4(-kLn2 * (2.f * q.x * M[0] + q.y * M[1]), -kLn2 * (q.y * M[0] + 2.f * q.z * M[1]), -0.5f * M[2],
                   -M[3]);
  gb = make_float4(-0.5f * M[4], M[5] * inv_o, M[6], M[7]);
}

__device__ inline void load_pixel(PixBwd& P, bool inside, size_t p, const TileInfo& ti, const float* bg,
                                  const float* __restrict__ image, const float* __restrict__ T_final,
                                  const uint32_t* __restrict__ n_contrib, const float* __restrict__ v_image,
                                  const float* __restrict__ target, float l1_weight, float& lsum) {
  P.T = 1.f;
  P.vS = 0.f;
  P.v0 = P.v1 = P.v2 = 0.f;
  P.nc = 0;
  if (!inside) return;
  P.T = T_final[p];
  P.nc = n_contrib[p];
  if (v_image) {
    P.v0 = v_image[3 * p];
    P.v1 = v_image[3 * p + 1];
    P.v2 = v_image[3 * p + 2];
  } else {
    const float s = l1_weight * ti.inv_norm;
    const float d0 = image[3 * p] - target[3 * p];
    const float d1 = image[3 * p + 1] - target[3 * p + 1];
    const float d2 = image[3 * p + 2] - target[3 * p + 2];
    P.v0 = d0 > 0.f ? s : (d0 < 0.f ? -s : 0.f);
    P.v1 = d1 > 0.f ? s : (d1 < 0.f ? -s : 0.f);
    P.v2 = d2 > 0.f ? s : (d2 < 0.f ? -s : 0.f);
    lsum += s * (fabsf(d0) + fabsf(d1) + fabsf(d2));
  }
  P.vS = P.T * (P.v0 * bg[0] + P.v1 * bg[1] + P.v2 * bg[2]);
  if (P.v0 == 0.f && P.v1 == 0.f && P.v2 == 0.f) P.nc = 0;
}

// 9 blocks of 16x16 per SM (56 registers, no spills) measured ~2 % faster
// than the 8 that 64 registers allow
template <int kTile, int kBatch>
__global__ void __launch_bounds__(Shape<kTile>::kThreads, (kTile == 16 ? 9 : 2)) render_bwd_kernel(
    gs_batch batch, gs_cameras cams, const float4* __restrict__ splat, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, const float* __restrict__ bg, const float* __restrict__ image,
    const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
    const float* __restrict__ v_image, const float* __restrict__ target, float l1_weight, double* loss,
    float* __restrict__ v2d) {
  constexpr int kThreads = Shape<kTile>::kThreads;
  __shared__ TileInfo ti;
  __shared__ float2 s_m[kBatch];
  __shared__ float4 s_q[kBatch];
  __shared__ float4 s_c[kBatch];
  __shared__ uint32_t s_mask[kBatch];
  __shared__ uint8_t s_list[kThreads / 32][kBatch];
  __shared__ uint32_t s_rec[kBatch];
  // per-warp gradient slots where they fit in shared memory, else one set
  // shared by the warps through shared atomics
  constexpr int kW = Shape<kTile>::kWarps;
  constexpr int kSlots = kBatch * (48 + 37 * kW) <= 45000 ? kW : 1;
  __shared__ float s_g[kSlots][kBatch][9];
  __shared__ uint32_t s_max;
  __shared__ float s_loss[kThreads / 32];
  const int gt = blockIdx.x;
  if (threadIdx.x == 0) s_max = 0;
  find_tile<kTile>(batch, cams, gt, &ti);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  int lx, ly;
  tile_pixels<kTile>(threadIdx.x, lx, ly);
  const uint32_t wbit = 1u << (threadIdx.x >> 5);
  const int u0 = ti.tx * kTile + lx, u1 = u0 + 4, v = ti.ty * kTile + ly;
  const bool in0 = u0 < ti.W && v < ti.H, in1 = u1 < ti.W && v < ti.H;
  const float px0 = (float)u0 + 0.5f, px1 = (float)u1 + 0.5f, py = (float)v + 0.5f;
  const float x0 = (float)(ti.tx * kTile), y0 = (float)(ti.ty * kTile);
  const uint32_t start = ranges[2 * gt];
  float lsum = 0.f;
  PixBwd P0, P1;
  load_pixel(P0, in0, (size_t)ti.px_offset + (size_t)v * ti.W + u0, ti, bg, image, T_final, n_contrib, v_image,
             target, l1_weight, lsum);
  load_pixel(P1, in1, (size_t)ti.px_offset + (size_t)v * ti.W + u1, ti, bg, image, T_final, n_contrib, v_image,
             target, l1_weight, lsum);
  const uint32_t nc_max = max(P0.nc, P1.nc);
  if (nc_max) atomicMax(&s_max, nc_max);
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
  const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, nc_max);
  for (int bend = (int)n_end; bend > 0; bend -= kBatch) {
    const int bstart = max(0, bend - kBatch);
    const int cnt = bend - bstart;
    for (int s = threadIdx.x; s < kBatch; s += kThreads) {
      if (s < cnt) {
        const uint32_t r = vals[start + bstart + s];
        s_rec[s] = r;
        stage_splat<kTile>(s, r, splat, x0, y0, s_m, s_q, s_c, s_mask);
      }
#pragma unroll
      for (int w = 0; w < kSlots; ++w)
#pragma unroll
        for (int i = 0; i < 9; ++i) s_g[w][s][i] = 0.f;
    }
    __syncthreads();
    // this warp's splats: before all its pixels' last contributor and able
    // to reach its 8x8 block; walked back to front
    const int n_mine =
        warp_list<kBatch>(s_mask, wbit, cnt, (int)warp_nc - bstart, s_list[threadIdx.x >> 5], lane);
    for (int i = n_mine - 1; i >= 0; --i) {
      const int k = s_list[threadIdx.x >> 5][i];
      const uint32_t pos = (uint32_t)(bstart + k);
      const float2 m = s_m[k];
      const float4 q = s_q[k];
      const float dy = py - m.y;
      float Bdy, sy;
      row_terms(q, dy, Bdy, sy);
      float g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = 0.f;
      bool contrib = false;
      if (pos < P0.nc) {
        const float dx = px0 - m.x;
        const float araw = ex2_approx(splat_exponent(q, dx, Bdy, sy));
        const float alpha = fminf(kAlphaMax, araw);
        if (alpha >= kAlphaMin) {
          contrib = true;
          bwd_pixel(P0, s_c[k], dx, dy, araw, alpha, g);
        }
      }
      if (pos < P1.nc) {
        const float dx = px1 - m.x;
        const float araw = ex2_approx(splat_exponent(q, dx, Bdy, sy));
        const float alpha = fminf(kAlphaMax, araw);
        if (alpha >= kAlphaMin) {
          contrib = true;
          bwd_pixel(P1, s_c[k], dx, dy, araw, alpha, g);
        }
      }
      if (__ballot_sync(0xffffffffu, contrib)) {
        const float s8 = warp_sum8_transposed(g, lane);
        float s9 = g[8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s9 += __shfl_xor_sync(0xffffffffu, s9, off);
        if constexpr (kSlots > 1) {
          float* dst = s_g[threadIdx.x >> 5][k];
          if ((lane & 3) == 0) dst[(lane >> 2) & 7] = s8;
          if (lane == 1) dst[8] = s9;
        } else {
          if ((lane & 3) == 0) atomicAdd(&s_g[0][k][(lane >> 2) & 7], s8);
          if (lane == 1) atomicAdd(&s_g[0][k][8], s9);
        }
      }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < cnt; s += kThreads) {
      float sg[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int w = 0; w < kSlots; ++w) acc += s_g[w][s][i];
        sg[i] = acc;
      }
      const bool nz = sg[0] != 0.f || sg[1] != 0.f || sg[2] != 0.f || sg[3] != 0.f || sg[4] != 0.f ||
                      sg[5] != 0.f || sg[6] != 0.f || sg[7] != 0.f || sg[8] != 0.f;
      if (nz) {
        float4 a, b;
        moments_to_grad(sg, s_q[s], s_c[s].w, a, b);
        float4* dst = reinterpret_cast<float4*>(v2d) + 3 * (size_t)s_rec[s];
        atomicAdd(dst, a);
        atomicAdd(dst + 1, b);
        atomicAdd(reinterpret_cast<float*>(dst + 2), sg[8]);
      }
    }
    __syncthreads();
  }
}

}  // namespace

namespace {

template <int kTile, int kBatch>
void render_fwd_launch(const gs_batch& batch, const gs_cameras& cams, const float4* sp, const uint32_t* vals,
                       const uint32_t* ranges, const float* bg, float* image, float* T_final,
                       uint32_t* n_contrib, uint32_t* n_added, cudaStream_t st) {
  // the per-pixel count of composited splats is a diagnostic: the kernel
  // without it saves two instructions per composited splat
  if (n_added)
    render_fwd_kernel<kTile, kBatch, true><<<batch.n_tiles, Shape<kTile>::kThreads, 0, st>>>(
        batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added);
  else
    render_fwd_kernel<kTile, kBatch, false><<<batch.n_tiles, Shape<kTile>::kThreads, 0, st>>>(
        batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added);
}

template <int kTile>
void render_fwd_tile(int rb, const gs_batch& batch, const gs_cameras& cams, const float4* sp,
                     const uint32_t* vals, const uint32_t* ranges, const float* bg, float* image, float* T_final,
                     uint32_t* n_contrib, uint32_t* n_added, cudaStream_t st) {
  if (rb == 64)
    render_fwd_launch<kTile, 64>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
  else if (rb == 128)
    render_fwd_launch<kTile, 128>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
  else
    render_fwd_launch<kTile, 256>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
}

template <int kTile, int kBatch>
void render_bwd_launch(const gs_batch& batch, const gs_cameras& cams, const float4* sp, const uint32_t* vals,
                       const uint32_t* ranges, const float* bg, const float* image, const float* T_final,
                       const uint32_t* n_contrib, const float* v_image, const float* target, float l1_weight,
                       double* loss, float* v2d, cudaStream_t st) {
  render_bwd_kernel<kTile, kBatch><<<batch.n_tiles, Shape<kTile>::kThreads, 0, st>>>(
      batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, v_image, target, l1_weight, loss, v2d);
}

template <int kTile>
void render_bwd_tile(int rb, const gs_batch& batch, const gs_cameras& cams, const float4* sp,
                     const uint32_t* vals, const uint32_t* ranges, const float* bg, const float* image,
                     const float* T_final, const uint32_t* n_contrib, const float* v_image, const float* target,
                     float l1_weight, double* loss, float* v2d, cudaStream_t st) {
  if (rb == 64)
    render_bwd_launch<kTile, 64>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, v_image, target,
                                 l1_weight, loss, v2d, st);
  else if (rb == 128)
    render_bwd_launch<kTile, 128>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, v_image, target,
                                  l1_weight, loss, v2d, st);
  else
    render_bwd_launch<kTile, 256>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, v_image, target,
                                  l1_weight, loss, v2d, st);
}

}  // namespace

cudaError_t launch_render_fwd(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                              const uint32_t* vals, const uint32_t* ranges, const float* bg,
                              float* image, float* T_final, uint32_t* n_contrib, uint32_t* n_added,
                              cudaStream_t st) {
  if (batch.n_tiles == 0) return cudaSuccess;
  const float4* sp = reinterpret_cast<const float4*>(proj.splat);
  const int rb = tuning().render_fwd_batch;
  if (batch.tile == 32)
    render_fwd_tile<32>(rb, batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
  else
    render_fwd_tile<16>(rb, batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                              const uint32_t* vals, const uint32_t* ranges, const float* bg,
                              const float* image, const float* T_final, const uint32_t* n_contrib,
                              const float* v_image, const float* target, float l1_weight,
                              double* loss, float* v2d, cudaStream_t st) {
  if (batch.n_tiles == 0) return cudaSuccess;
  const float4* sp = reinterpret_cast<const float4*>(proj.splat);
  const int rb = tuning().render_bwd_batch;
  if (batch.tile == 32)
    render_bwd_tile<32>(rb, batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, v_image, target,
                        l1_weight, loss, v2d, st);
  else
    render_bwd_tile<16>(rb, batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, v_image, target,
                        l1_weight, loss, v2d, st);
  return cudaGetLastError();
}

}  // namespace gs
