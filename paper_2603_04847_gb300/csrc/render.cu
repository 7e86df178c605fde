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
//
// The kernels are templates on the scalar type: the FP32 instantiation is
// the product path; the FP64 one (double records, exact exp2/log2 in place
// of the approximate units, 64 splats staged per round) exists to check the
// path against finite differences in double precision.
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

template <typename T>
struct RC;
template <>
struct RC<float> {
  static constexpr float ln2 = 0.69314718055994531f;
  static constexpr float half_log2e = 0.72134752044448170f;  // 1 / (2 ln 2)
};
template <>
struct RC<double> {
  static constexpr double ln2 = 0.69314718055994531;
  static constexpr double half_log2e = 0.72134752044448170;
};

// Vector types of the staged records.
template <typename T>
struct V2;
template <typename T>
struct V4;
template <>
struct V2<float> {
  using type = float2;
};
template <>
struct V4<float> {
  using type = float4;
};
struct alignas(16) dbl4 {
  double x, y, z, w;
};
template <>
struct V2<double> {
  using type = double2;
};
template <>
struct V4<double> {
  using type = dbl4;
};
template <typename T>
using v2_t = typename V2<T>::type;
template <typename T>
using v4_t = typename V4<T>::type;

__device__ inline float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ inline double2 mk2(double a, double b) { return make_double2(a, b); }
__device__ inline float4 mk4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ inline dbl4 mk4(double a, double b, double c, double d) { return dbl4{a, b, c, d}; }

// The approximate FP32 units of the product path; exact in FP64.
__device__ inline float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ inline double ex2a(double x) { return exp2(x); }
__device__ inline float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ inline double lg2a(double x) { return log2(x); }
__device__ inline float rcp_rn(float x) { return __frcp_rn(x); }
__device__ inline double rcp_rn(double x) { return 1.0 / x; }
__device__ inline float recip_fast(float x) { return __fdividef(1.f, x); }
__device__ inline double recip_fast(double x) { return 1.0 / x; }
__device__ inline float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ inline double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ inline float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ inline double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
struct TileInfo {
  int slot;
  int ok;          // the slot's offsets hold its view (else nothing to do)
  int W, H;
  int tx, ty;
  long long px_offset;
  T inv_norm;      // 1 / (3 W H) for the per-view L1 mean
};

// The cameras' image sizes (all the compositing needs of them).
struct Sizes {
  int n_cams;
  const int32_t* wh;
};

template <int kTile, typename T>
__device__ inline void find_tile(const gs_batch& batch, const Sizes& cams, int gt, TileInfo<T>* ti) {
  if (threadIdx.x == 0) {
    int lo = 0, hi = batch.B - 1;
    while (lo < hi) {  // last slot with tile_offset[slot] <= gt
      const int mid = (lo + hi + 1) >> 1;
      if (batch.tile_offset[mid] <= gt) lo = mid;
      else hi = mid - 1;
    }
    const int v = slot_view_n(cams.n_cams, batch, lo);
    TileInfo<T> t;
    t.slot = lo;
    t.W = cams.wh[2 * v];
    t.H = cams.wh[2 * v + 1];
    const int tiles_x = (t.W + kTile - 1) / kTile;
    const int l = gt - batch.tile_offset[lo];
    t.tx = l % tiles_x;
    t.ty = l / tiles_x;
    t.px_offset = batch.px_offset[lo];
    t.inv_norm = T(1) / (T(3) * (T)t.W * (T)t.H);
    t.ok = slot_consistent(batch, lo, t.W, t.H);
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
template <int kTile, typename T>
__device__ inline uint32_t warp_mask(T mx, T my, T a, T b, T c, T qmax, T x0, T y0) {
  constexpr int kWX = Shape<kTile>::kWarpsX;
  const T det = a * c - b * b;
  const T qc = (qmax + T(1e-3f)) * T(1.02f) + T(0.01f);
  const T ia = rcp_rn(a), ic = rcp_rn(c);
  const T ba = b * ia, bc = b * ic, da = det * ia, dc = det * ic;
  uint32_t m = 0;
#pragma unroll
  for (int w = 0; w < Shape<kTile>::kWarps; ++w) {
    const T bx0 = x0 + (T)((w % kWX) * 8) + T(0.49f), by0 = y0 + (T)((w / kWX) * 8) + T(0.49f);
    const T bx1 = bx0 + T(7.02f), by1 = by0 + T(7.02f);
    // on the vertical line through the rectangle's x nearest the mean
    const T dx = gmin(gmax(mx, bx0), bx1) - mx;
    const T ev = gmin(gmax(my - bc * dx, by0), by1) - my + bc * dx;
    const T qv = c * ev * ev + dc * dx * dx;
    // on the horizontal line through the rectangle's y nearest the mean
    const T dy = gmin(gmax(my, by0), by1) - my;
    const T eh = gmin(gmax(mx - ba * dy, bx0), bx1) - mx + ba * dy;
    const T qh = a * eh * eh + da * dy * dy;
    m |= (gmin(qv, qh) <= qc) ? (1u << w) : 0u;
  }
  return m;
}

// The 12 scalars of record r.
__device__ inline void load_record(const float* splat, uint32_t r, float (&v)[12]) {
  const float4* p = reinterpret_cast<const float4*>(splat) + 3 * (size_t)r;
  const float4 a = p[0], b = p[1], c = p[2];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
}
__device__ inline void load_record(const double* splat, uint32_t r, double (&v)[12]) {
  const double2* p = reinterpret_cast<const double2*>(splat) + 6 * (size_t)r;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double2 q = p[i];
    v[2 * i] = q.x;
    v[2 * i + 1] = q.y;
  }
}

// Stages record r into slot `s` of the shared arrays.
template <int kTile, typename T>
__device__ inline void stage_splat(int s, uint32_t r, const T* __restrict__ splat, T x0, T y0, v2_t<T>* s_m,
                                   v4_t<T>* s_q, v4_t<T>* s_c, uint32_t* s_mask) {
  T v[12];
  load_record(splat, r, v);
  const T k = RC<T>::half_log2e;
  s_m[s] = mk2(v[0], v[1]);
  s_q[s] = mk4(-k * v[4], T(-2) * k * v[5], -k * v[6], lg2a(v[2]));
  s_c[s] = mk4(v[8], v[9], v[10], T(1) / v[2]);
  s_mask[s] = warp_mask<kTile>(v[0], v[1], v[4], v[5], v[6], v[7], x0, y0);
}

// Exponent e = A dx^2 + B dx dy + C dy^2 + log2 o of alpha_raw = 2^e at
// offset (dx, dy), from the row terms Bdy = B dy and sy = C dy^2 + log2 o
// (row_terms).  Written with explicit roundings so that every kernel
// computes the same value from the same staged inputs.
template <typename Q, typename T>
__device__ inline void row_terms(const Q q, T dy, T& Bdy, T& sy) {
  Bdy = mul_rn(q.y, dy);
  sy = fma_rn(mul_rn(q.z, dy), dy, q.w);
}

template <typename Q, typename T>
__device__ inline T splat_exponent(const Q q, T dx, T Bdy, T sy) {
  return fma_rn(fma_rn(q.x, dx, Bdy), dx, sy);
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

// Blocks per SM: 10 of 16x16 for the FP32 forward (48 registers, no
// spills) measured 3 % faster than the 8 that 64 registers allow; 9 for the
// FP32 backward (56 registers, ~2 % faster than 8).  The FP64 checking
// path takes what it needs.
template <typename T, int kTile>
constexpr int fwd_min_blocks() {
  return sizeof(T) == 4 ? (kTile == 16 ? 10 : 2) : 1;
}
template <typename T, int kTile>
constexpr int bwd_min_blocks() {
  return sizeof(T) == 4 ? (kTile == 16 ? 9 : 2) : 1;
}

template <typename T, int kTile, int kBatch, bool kCountAdded>
__global__ void __launch_bounds__(Shape<kTile>::kThreads, (fwd_min_blocks<T, kTile>())) render_fwd_kernel(
    gs_batch batch, Sizes cams, const T* __restrict__ splat, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, const T* __restrict__ bg, T* __restrict__ image,
    T* __restrict__ T_final, uint32_t* __restrict__ n_contrib, uint32_t* __restrict__ n_added) {
  constexpr int kThreads = Shape<kTile>::kThreads;
  __shared__ TileInfo<T> ti;
  __shared__ v2_t<T> s_m[kBatch];
  __shared__ v4_t<T> s_q[kBatch];
  __shared__ v4_t<T> s_c[kBatch];
  __shared__ uint32_t s_mask[kBatch];
  __shared__ uint8_t s_list[kThreads / 32][kBatch];
  const int gt = blockIdx.x;
  // the grid covers the batch's tile capacity; tiles past the views' own
  // end (a batch laid out on the device) have nothing to do
  if (gt >= batch.tile_offset[batch.B]) return;
  find_tile<kTile>(batch, cams, gt, &ti);
  __syncthreads();
  if (!ti.ok) return;  // block-uniform
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lx, ly;
  tile_pixels<kTile>(threadIdx.x, lx, ly);
  const uint32_t wbit = 1u << warp;
  const int u0 = ti.tx * kTile + lx, u1 = u0 + 4, v = ti.ty * kTile + ly;
  const bool in0 = u0 < ti.W && v < ti.H, in1 = u1 < ti.W && v < ti.H;
  const T px0 = (T)u0 + T(0.5), px1 = (T)u1 + T(0.5), py = (T)v + T(0.5);
  const T x0 = (T)(ti.tx * kTile), y0 = (T)(ti.ty * kTile);
  const uint32_t start = ranges[2 * gt], end = ranges[2 * gt + 1];
  const T amin = Consts<T>::alpha_min, amax = Consts<T>::alpha_max, tmin = Consts<T>::t_min;
  T T0 = T(1), T1 = T(1);
  T C00 = T(0), C01 = T(0), C02 = T(0), C10 = T(0), C11 = T(0), C12 = T(0);
  uint32_t last0 = 0, last1 = 0, add0 = 0, add1 = 0;
  bool done0 = !in0, done1 = !in1;
  // a finished pixel gets an unreachable threshold, so the per-splat test
  // is one compare (alpha = min(0.99, alpha_raw) >= 1/255 iff
  // alpha_raw >= 1/255)
  T thr0 = done0 ? T(2) : amin, thr1 = done1 ? T(2) : amin;
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
      const v2_t<T> m = s_m[k];
      const v4_t<T> q = s_q[k];
      T Bdy, sy;
      row_terms(q, py - m.y, Bdy, sy);
      const T r0 = ex2a(splat_exponent(q, px0 - m.x, Bdy, sy));
      const T r1 = ex2a(splat_exponent(q, px1 - m.x, Bdy, sy));
      const bool c0 = r0 >= thr0;
      const bool c1 = r1 >= thr1;
      if (!(c0 || c1)) continue;
      const v4_t<T> c = s_c[k];
      const uint32_t pos1 = base - start + (uint32_t)k + 1u;
      if (c0) {
        const T a0 = gmin(amax, r0);
        const T Tn = T0 * (T(1) - a0);
        if (Tn < tmin) {
          done0 = true;
          thr0 = T(2);
        } else {
          const T w = a0 * T0;
          C00 += c.x * w;
          C01 += c.y * w;
          C02 += c.z * w;
          T0 = Tn;
          last0 = pos1;
          if constexpr (kCountAdded) ++add0;
        }
      }
      if (c1) {
        const T a1 = gmin(amax, r1);
        const T Tn = T1 * (T(1) - a1);
        if (Tn < tmin) {
          done1 = true;
          thr1 = T(2);
        } else {
          const T w = a1 * T1;
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
template <typename T>
__device__ inline T warp_sum8_transposed(const T* v, int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  T a[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T send = h16 ? v[i] : v[i + 4];
    const T keep = h16 ? v[i + 4] : v[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  T b[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const T send = h8 ? a[i] : a[i + 2];
    const T keep = h8 ? a[i + 2] : a[i];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  T c = (h4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h4 ? b[0] : b[1], 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

// Per-pixel backward state.
// The colour composited behind the current splat, S, enters the gradient
// only through v . S (v = dL/dC is fixed per pixel), so that dot product is
// carried instead of S.
template <typename T>
struct PixBwd {
  T T_, vS, v0, v1, v2;
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
template <typename T, typename C4>
__device__ inline void bwd_pixel(PixBwd<T>& P, const C4 c, T dx, T dy, T araw, T alpha, T* g) {
  const T ra = recip_fast(T(1) - alpha);  // 1 - alpha >= 0.01
  const T Tk = P.T_ * ra;                 // transmittance before this splat
  const T w = alpha * Tk;
  g[6] += w * P.v0;
  g[7] += w * P.v1;
  g[8] += w * P.v2;
  const T vc = P.v0 * c.x + P.v1 * c.y + P.v2 * c.z;
  const T va = vc * Tk - P.vS * ra;  // dL/dalpha = v . (c T_k - S / (1 - alpha))
  P.vS += vc * w;
  P.T_ = Tk;
  if (araw < Consts<T>::alpha_max) {
    const T u = alpha * va;
    const T udx = u * dx, udy = u * dy;
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
//   dL/da = -M2/2, dL/db = -M3, dL/dc = -M4/2, dL/do = M5 / o;
// written into the record (mean2d x, y, conic a, b, c, opacity, colour).
template <typename T, typename Q4>
__device__ inline void moments_to_grad(const T* M, Q4 q, T inv_o, T* r) {
  const T l2 = RC<T>::ln2;
  r[0] = -l2 * (T(2) * q.x * M[0] + q.y * M[1]);
  r[1] = -l2 * (q.y * M[0] + T(2) * q.z * M[1]);
  r[2] = T(-0.5) * M[2];
  r[3] = -M[3];
  r[4] = T(-0.5) * M[4];
  r[5] = M[5] * inv_o;
  r[6] = M[6];
  r[7] = M[7];
  r[8] = M[8];
}

// record r of v2d += g[0..8] (one vector atomic per 4 floats in FP32).
__device__ inline void add_record(float* v2d, uint32_t r, const float* g) {
  float4* dst = reinterpret_cast<float4*>(v2d) + 3 * (size_t)r;
  atomicAdd(dst, make_float4(g[0], g[1], g[2], g[3]));
  atomicAdd(dst + 1, make_float4(g[4], g[5], g[6], g[7]));
  atomicAdd(reinterpret_cast<float*>(dst + 2), g[8]);
}
__device__ inline void add_record(double* v2d, uint32_t r, const double* g) {
  double* dst = v2d + 12 * (size_t)r;
#pragma unroll
  for (int i = 0; i < 9; ++i) atomicAdd(dst + i, g[i]);
}

// Outputs of the deterministic backward: every (record, tile) instance
// gets a slot of its own, so no two tiles add into the same memory and the
// per-record sums are formed afterwards in a fixed order (det_reduce_kernel).
// Record r's slots are base[r] .. base[r] + n_tiles[r] - 1 (base is the
// exclusive scan of n_tiles in record order); the tile (tx, ty) of its
// rectangle (x0, y0, x1, y1) has slot base[r] + (ty - y0) (x1 - x0 + 1) +
// (tx - x0).  Slots at or past cap (the instance buffers overflowed, which
// the sort has flagged) are neither written nor read.
struct DetOut {
  const uint32_t* base;
  const ushort4* rect;
  float4* p8;          // [cap][2]: the moments 0..7 of the slot
  float* p1;           // [cap]: moment 8
  size_t cap;
  double* tile_loss;   // [tiles]: each tile's L1 sum (fused L1 only)
};

__device__ inline uint32_t det_slot(const DetOut& det, uint32_t r, int tx, int ty) {
  const ushort4 rc = det.rect[r];
  return det.base[r] + (uint32_t)(ty - (int)rc.y) * (uint32_t)(rc.z - rc.x + 1) + (uint32_t)(tx - (int)rc.x);
}

__device__ inline void det_store(const DetOut& det, uint32_t slot, const float* g) {
  if (slot >= det.cap) return;
  det.p8[2 * (size_t)slot] = make_float4(g[0], g[1], g[2], g[3]);
  det.p8[2 * (size_t)slot + 1] = make_float4(g[4], g[5], g[6], g[7]);
  det.p1[slot] = g[8];
}

template <typename T>
__device__ inline void load_pixel(PixBwd<T>& P, bool inside, size_t p, const TileInfo<T>& ti, const T* bg,
                                  const T* __restrict__ image, const T* __restrict__ T_final,
                                  const uint32_t* __restrict__ n_contrib, const T* __restrict__ v_image,
                                  const T* __restrict__ target, T l1_weight, T& lsum) {
  P.T_ = T(1);
  P.vS = T(0);
  P.v0 = P.v1 = P.v2 = T(0);
  P.nc = 0;
  if (!inside) return;
  P.T_ = T_final[p];
  P.nc = n_contrib[p];
  if (v_image) {
    P.v0 = v_image[3 * p];
    P.v1 = v_image[3 * p + 1];
    P.v2 = v_image[3 * p + 2];
  } else {
    const T s = l1_weight * ti.inv_norm;
    const T d0 = image[3 * p] - target[3 * p];
    const T d1 = image[3 * p + 1] - target[3 * p + 1];
    const T d2 = image[3 * p + 2] - target[3 * p + 2];
    P.v0 = d0 > T(0) ? s : (d0 < T(0) ? -s : T(0));
    P.v1 = d1 > T(0) ? s : (d1 < T(0) ? -s : T(0));
    P.v2 = d2 > T(0) ? s : (d2 < T(0) ? -s : T(0));
    lsum += s * (fabs(d0) + fabs(d1) + fabs(d2));
  }
  P.vS = P.T_ * (P.v0 * bg[0] + P.v1 * bg[1] + P.v2 * bg[2]);
  if (P.v0 == T(0) && P.v1 == T(0) && P.v2 == T(0)) P.nc = 0;
}

// kDet (FP32 only): each (record, tile) sum goes to its own slot of `det`
// instead of being added into the record, and every instance of the tile's
// list gets its slot written (zeros where nothing was composited).
template <typename T, int kTile, int kBatch, bool kDet>
__global__ void __launch_bounds__(Shape<kTile>::kThreads, (bwd_min_blocks<T, kTile>())) render_bwd_kernel(
    gs_batch batch, Sizes cams, const T* __restrict__ splat, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, const T* __restrict__ bg, const T* __restrict__ image,
    const T* __restrict__ T_final, const uint32_t* __restrict__ n_contrib, const T* __restrict__ v_image,
    const T* __restrict__ target, T l1_weight, double* loss, T* __restrict__ v2d, DetOut det) {
  static_assert(!kDet || sizeof(T) == 4, "the deterministic backward is FP32");
  constexpr int kThreads = Shape<kTile>::kThreads;
  __shared__ TileInfo<T> ti;
  // staged splats, two buffers: a batch is staged while the previous one's
  // sums are written out
  __shared__ v2_t<T> s_m[2][kBatch];
  __shared__ v4_t<T> s_q[2][kBatch];
  __shared__ v4_t<T> s_c[2][kBatch];
  __shared__ uint32_t s_mask[2][kBatch];
  __shared__ uint8_t s_list[kThreads / 32][kBatch];
  __shared__ uint32_t s_rec[2][kBatch];
  __shared__ uint32_t s_slot[2][kDet ? kBatch : 1];
  // per-warp gradient slots where they fit in shared memory, else one set
  // shared by the warps through shared atomics
  constexpr int kW = Shape<kTile>::kWarps;
  constexpr int kSlots =
      kBatch * (2 * ((int)(10 * sizeof(T)) + 12) + kW + (int)(9 * sizeof(T)) * kW) <= 45000 ? kW : 1;
  __shared__ T s_g[kSlots][kBatch][9];
  __shared__ uint32_t s_max;
  __shared__ T s_loss[kThreads / 32];
  const int gt = blockIdx.x;
  if (gt >= batch.tile_offset[batch.B]) return;  // past the views' tiles
  if (threadIdx.x == 0) s_max = 0;
  find_tile<kTile>(batch, cams, gt, &ti);
  __syncthreads();
  if (!ti.ok) {  // block-uniform; such a slot has no instances
    if constexpr (kDet)
      if (threadIdx.x == 0 && det.tile_loss) det.tile_loss[gt] = 0.0;
    return;
  }
  const int lane = threadIdx.x & 31;
  int lx, ly;
  tile_pixels<kTile>(threadIdx.x, lx, ly);
  const uint32_t wbit = 1u << (threadIdx.x >> 5);
  const int u0 = ti.tx * kTile + lx, u1 = u0 + 4, v = ti.ty * kTile + ly;
  const bool in0 = u0 < ti.W && v < ti.H, in1 = u1 < ti.W && v < ti.H;
  const T px0 = (T)u0 + T(0.5), px1 = (T)u1 + T(0.5), py = (T)v + T(0.5);
  const T x0 = (T)(ti.tx * kTile), y0 = (T)(ti.ty * kTile);
  const uint32_t start = ranges[2 * gt];
  T lsum = T(0);
  PixBwd<T> P0, P1;
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
    if constexpr (kDet) {
      if (det.tile_loss) det.tile_loss[gt] = t;
    } else {
      if (t != 0.0) atomicAdd(loss, t);
    }
  }
  const uint32_t n_end = s_max;  // positions [0, n_end) of the tile list
  const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, nc_max);
  const T amin = Consts<T>::alpha_min, amax = Consts<T>::alpha_max;
  // Batches back to front.  The first phase of a round writes out the
  // previous batch's sums (zeroing their slots) and stages this batch into
  // the other buffer, on different threads where the block has enough of
  // them; the second composites.  Two barriers a round.
#pragma unroll 1
  for (int i = threadIdx.x; i < kSlots * kBatch * 9; i += kThreads) (&s_g[0][0][0])[i] = T(0);
  int prev_cnt = 0, buf = 0;
  for (int bend = (int)n_end;; bend -= kBatch) {
    const int bstart = max(0, bend - kBatch);
    const int cnt = bend > 0 ? bend - bstart : 0;
    for (int u = threadIdx.x; u < 2 * kBatch; u += kThreads) {
      if (u < kBatch) {
        const int s = u, pb = buf ^ 1;
        if (s < prev_cnt) {
          T sg[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            T acc = T(0);
#pragma unroll
            for (int w = 0; w < kSlots; ++w) {
              acc += s_g[w][s][i];
              s_g[w][s][i] = T(0);
            }
            sg[i] = acc;
          }
          const bool nz = sg[0] != T(0) || sg[1] != T(0) || sg[2] != T(0) || sg[3] != T(0) || sg[4] != T(0) ||
                          sg[5] != T(0) || sg[6] != T(0) || sg[7] != T(0) || sg[8] != T(0);
          T rec[9];
          if constexpr (kDet) {
            if (nz) moments_to_grad(sg, s_q[pb][s], s_c[pb][s].w, rec);
            else
#pragma unroll
              for (int i = 0; i < 9; ++i) rec[i] = T(0);
            det_store(det, s_slot[pb][s], rec);
          } else if (nz) {
            moments_to_grad(sg, s_q[pb][s], s_c[pb][s].w, rec);
            add_record(v2d, s_rec[pb][s], rec);
          }
        }
      } else {
        const int s = u - kBatch;
        if (s < cnt) {
          const uint32_t r = vals[start + bstart + s];
          s_rec[buf][s] = r;
          stage_splat<kTile>(s, r, splat, x0, y0, s_m[buf], s_q[buf], s_c[buf], s_mask[buf]);
          if constexpr (kDet) s_slot[buf][s] = det_slot(det, r, ti.tx, ti.ty);
        }
      }
    }
    if (cnt == 0) break;  // block-uniform
    __syncthreads();
    // this warp's splats: before all its pixels' last contributor and able
    // to reach its 8x8 block; walked back to front
    const int n_mine =
        warp_list<kBatch>(s_mask[buf], wbit, cnt, (int)warp_nc - bstart, s_list[threadIdx.x >> 5], lane);
    for (int i = n_mine - 1; i >= 0; --i) {
      const int k = s_list[threadIdx.x >> 5][i];
      const uint32_t pos = (uint32_t)(bstart + k);
      const v2_t<T> m = s_m[buf][k];
      const v4_t<T> q = s_q[buf][k];
      const T dy = py - m.y;
      T Bdy, sy;
      row_terms(q, dy, Bdy, sy);
      T g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = T(0);
      bool contrib = false;
      if (pos < P0.nc) {
        const T dx = px0 - m.x;
        const T araw = ex2a(splat_exponent(q, dx, Bdy, sy));
        const T alpha = gmin(amax, araw);
        if (alpha >= amin) {
          contrib = true;
          bwd_pixel(P0, s_c[buf][k], dx, dy, araw, alpha, g);
        }
      }
      if (pos < P1.nc) {
        const T dx = px1 - m.x;
        const T araw = ex2a(splat_exponent(q, dx, Bdy, sy));
        const T alpha = gmin(amax, araw);
        if (alpha >= amin) {
          contrib = true;
          bwd_pixel(P1, s_c[buf][k], dx, dy, araw, alpha, g);
        }
      }
      if (__ballot_sync(0xffffffffu, contrib)) {
        const T s8 = warp_sum8_transposed(g, lane);
        T s9 = g[8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s9 += __shfl_xor_sync(0xffffffffu, s9, off);
        if constexpr (kSlots > 1) {
          T* dst = s_g[threadIdx.x >> 5][k];
          if ((lane & 3) == 0) dst[(lane >> 2) & 7] = s8;
          if (lane == 1) dst[8] = s9;
        } else {
          if ((lane & 3) == 0) atomicAdd(&s_g[0][k][(lane >> 2) & 7], s8);
          if (lane == 1) atomicAdd(&s_g[0][k][8], s9);
        }
      }
    }
    __syncthreads();
    prev_cnt = cnt;
    buf ^= 1;
  }
  if constexpr (kDet) {
    // instances behind every pixel's last contributor: zero slots
    const uint32_t n_list = ranges[2 * gt + 1] - start;
    const float zero[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (uint32_t pos = n_end + threadIdx.x; pos < n_list; pos += kThreads)
      det_store(det, det_slot(det, vals[start + pos], ti.tx, ti.ty), zero);
  }
}

}  // namespace

namespace {

template <typename T, int kTile, int kBatch>
void render_fwd_launch(const gs_batch& batch, const Sizes& cams, const T* sp, const uint32_t* vals,
                       const uint32_t* ranges, const T* bg, T* image, T* T_final, uint32_t* n_contrib,
                       uint32_t* n_added, cudaStream_t st) {
  // the per-pixel count of composited splats is a diagnostic: the kernel
  // without it saves two instructions per composited splat
  if (n_added)
    render_fwd_kernel<T, kTile, kBatch, true><<<batch.n_tiles, Shape<kTile>::kThreads, 0, st>>>(
        batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added);
  else
    render_fwd_kernel<T, kTile, kBatch, false><<<batch.n_tiles, Shape<kTile>::kThreads, 0, st>>>(
        batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added);
}

template <int kTile>
void render_fwd_tile(int rb, const gs_batch& batch, const Sizes& cams, const float* sp, const uint32_t* vals,
                     const uint32_t* ranges, const float* bg, float* image, float* T_final, uint32_t* n_contrib,
                     uint32_t* n_added, cudaStream_t st) {
  if (rb == 64)
    render_fwd_launch<float, kTile, 64>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
  else if (rb == 128)
    render_fwd_launch<float, kTile, 128>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
  else
    render_fwd_launch<float, kTile, 256>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
}

template <typename T, int kTile, int kBatch, bool kDet = false>
void render_bwd_launch(const gs_batch& batch, const Sizes& cams, const T* sp, const uint32_t* vals,
                       const uint32_t* ranges, const T* bg, const T* image, const T* T_final,
                       const uint32_t* n_contrib, const T* v_image, const T* target, T l1_weight, double* loss,
                       T* v2d, cudaStream_t st, const DetOut& det = DetOut{}) {
  render_bwd_kernel<T, kTile, kBatch, kDet><<<batch.n_tiles, Shape<kTile>::kThreads, 0, st>>>(
      batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib, v_image, target, l1_weight, loss, v2d, det);
}

template <int kTile, bool kDet = false>
void render_bwd_tile(int rb, const gs_batch& batch, const Sizes& cams, const float* sp, const uint32_t* vals,
                     const uint32_t* ranges, const float* bg, const float* image, const float* T_final,
                     const uint32_t* n_contrib, const float* v_image, const float* target, float l1_weight,
                     double* loss, float* v2d, cudaStream_t st, const DetOut& det = DetOut{}) {
  if (rb == 64)
    render_bwd_launch<float, kTile, 64, kDet>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib,
                                              v_image, target, l1_weight, loss, v2d, st, det);
  else if (rb == 128)
    render_bwd_launch<float, kTile, 128, kDet>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib,
                                               v_image, target, l1_weight, loss, v2d, st, det);
  else
    render_bwd_launch<float, kTile, 256, kDet>(batch, cams, sp, vals, ranges, bg, image, T_final, n_contrib,
                                               v_image, target, l1_weight, loss, v2d, st, det);
}

// ---- the deterministic backward's fixed-order reductions -----------------

constexpr int kDetThreads = 1024;
constexpr int kDetItems = 4;
constexpr int kDetTile = kDetThreads * kDetItems;

// Block-wide inclusive scan of one u64 per thread (kDetThreads threads).
__device__ inline unsigned long long det_block_scan(unsigned long long x, unsigned long long* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = sm[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    sm[lane] = w;
  }
  __syncthreads();
  const unsigned long long r = x + (warp > 0 ? sm[warp - 1] : 0ull);
  __syncthreads();
  return r;
}

// Sum of n_tiles over each kDetTile records.
__global__ void __launch_bounds__(kDetThreads) det_scan_reduce_kernel(const uint32_t* __restrict__ n_tiles, size_t M,
                                                                      unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long sm[32];
  const size_t r0 = (size_t)blockIdx.x * kDetTile + (size_t)threadIdx.x * kDetItems;
  unsigned long long x = 0;
#pragma unroll
  for (int i = 0; i < kDetItems; ++i)
    if (r0 + i < M) x += n_tiles[r0 + i];
  x = det_block_scan(x, sm);
  if (threadIdx.x == kDetThreads - 1) bsum[blockIdx.x] = x;
}

// Exclusive scan of the block sums, in place, in one block.
__global__ void __launch_bounds__(kDetThreads) det_scan_top_kernel(unsigned long long* bsum, int n_blocks) {
  __shared__ unsigned long long sm[32];
  __shared__ unsigned long long s_last;
  unsigned long long carry = 0;
  for (int b0 = 0; b0 < n_blocks; b0 += kDetThreads) {
    const int i = b0 + threadIdx.x;
    const unsigned long long x = i < n_blocks ? bsum[i] : 0ull;
    const unsigned long long inc = det_block_scan(x, sm);
    if (i < n_blocks) bsum[i] = carry + inc - x;
    if (threadIdx.x == kDetThreads - 1) s_last = inc;
    __syncthreads();
    carry += s_last;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[n_blocks] = carry;  // all instances of the records
}

// base[r] = sum of n_tiles over the records before r (0xffffffff past 32
// bits: such records have no slot).
__global__ void __launch_bounds__(kDetThreads) det_scan_down_kernel(const uint32_t* __restrict__ n_tiles, size_t M,
                                                                    const unsigned long long* __restrict__ bsum,
                                                                    uint32_t* __restrict__ base) {
  __shared__ unsigned long long sm[32];
  const size_t r0 = (size_t)blockIdx.x * kDetTile + (size_t)threadIdx.x * kDetItems;
  uint32_t v[kDetItems];
  unsigned long long x = 0;
#pragma unroll
  for (int i = 0; i < kDetItems; ++i) {
    v[i] = r0 + i < M ? n_tiles[r0 + i] : 0u;
    x += v[i];
  }
  unsigned long long e = det_block_scan(x, sm) - x + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kDetItems; ++i) {
    if (r0 + i < M) base[r0 + i] = e > 0xffffffffull ? 0xffffffffu : (uint32_t)e;
    e += v[i];
  }
}

// v2d[r] = sum over record r's slots in slot order; culled records get
// zeros, and so does every record when the tile lists do not hold all the
// records' instances (the sort overflowed its capacity or stopped: it has
// flagged that, and some slots were never written).
__global__ void __launch_bounds__(256) det_reduce_kernel(const uint32_t* __restrict__ n_tiles,
                                                         const uint32_t* __restrict__ base,
                                                         const unsigned long long* __restrict__ total,
                                                         const uint32_t* __restrict__ n_instances,
                                                         const float4* __restrict__ p8,
                                                         const float* __restrict__ p1, size_t cap, size_t M,
                                                         float* __restrict__ v2d) {
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  const bool complete = *total <= cap && *total == (unsigned long long)*n_instances;
  const uint32_t n = complete ? n_tiles[r] : 0u;
  const size_t b = base[r];
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), c = a;
  float d = 0.f;
  for (uint32_t k = 0; k < n; ++k) {
    const size_t sl = b + k;
    if (sl >= cap) break;
    const float4 x = p8[2 * sl], y = p8[2 * sl + 1];
    a.x += x.x; a.y += x.y; a.z += x.z; a.w += x.w;
    c.x += y.x; c.y += y.y; c.z += y.z; c.w += y.w;
    d += p1[sl];
  }
  float4* dst = reinterpret_cast<float4*>(v2d) + 3 * r;
  dst[0] = a;
  dst[1] = c;
  dst[2] = make_float4(d, 0.f, 0.f, 0.f);
}

// loss += the tiles' L1 sums, in a fixed order.
__global__ void __launch_bounds__(kDetThreads) det_loss_kernel(const double* __restrict__ tile_loss,
                                                               const gs_batch batch, double* loss) {
  __shared__ double sm[kDetThreads];
  const int n = batch.tile_offset[batch.B];
  double x = 0.0;
  for (int i = threadIdx.x; i < n; i += kDetThreads) x += tile_loss[i];
  sm[threadIdx.x] = x;
  __syncthreads();
  for (int w = kDetThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && sm[0] != 0.0) atomicAdd(loss, sm[0]);
}

}  // namespace

cudaError_t launch_render_fwd(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                              const uint32_t* vals, const uint32_t* ranges, const float* bg,
                              float* image, float* T_final, uint32_t* n_contrib, uint32_t* n_added,
                              cudaStream_t st) {
  if (batch.n_tiles == 0) return cudaSuccess;
  const Sizes sz{cams.n_cams, cams.wh};
  const int rb = tuning().render_fwd_batch;
  if (batch.tile == 32)
    render_fwd_tile<32>(rb, batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
  else
    render_fwd_tile<16>(rb, batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, n_added, st);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                              const uint32_t* vals, const uint32_t* ranges, const float* bg,
                              const float* image, const float* T_final, const uint32_t* n_contrib,
                              const float* v_image, const float* target, float l1_weight,
                              double* loss, float* v2d, cudaStream_t st) {
  if (batch.n_tiles == 0) return cudaSuccess;
  const Sizes sz{cams.n_cams, cams.wh};
  const int rb = tuning().render_bwd_batch;
  if (batch.tile == 32)
    render_bwd_tile<32>(rb, batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, v_image, target,
                        l1_weight, loss, v2d, st);
  else
    render_bwd_tile<16>(rb, batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, v_image, target,
                        l1_weight, loss, v2d, st);
  return cudaGetLastError();
}

namespace {
struct DetLayout {
  size_t base, bsum, p8, p1, tile_loss, bytes;
};
inline size_t det_align(size_t x) { return (x + 255) & ~(size_t)255; }
DetLayout det_layout(size_t M, int n_tiles, size_t cap) {
  DetLayout L;
  const size_t nblk = (M + kDetTile - 1) / kDetTile;
  L.base = 0;
  L.bsum = det_align(L.base + M * sizeof(uint32_t));
  L.p8 = det_align(L.bsum + (nblk + 1) * sizeof(unsigned long long));
  L.p1 = det_align(L.p8 + cap * 2 * sizeof(float4));
  L.tile_loss = det_align(L.p1 + cap * sizeof(float));
  L.bytes = det_align(L.tile_loss + (size_t)n_tiles * sizeof(double));
  return L;
}
}  // namespace

size_t render_bwd_det_bytes(size_t M, int n_tiles, size_t capacity) {
  return det_layout(M, n_tiles, capacity).bytes;
}

cudaError_t launch_render_bwd_det(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                                  size_t M, const uint32_t* vals, const uint32_t* ranges,
                                  const uint32_t* n_instances, const float* bg, const float* image,
                                  const float* T_final, const uint32_t* n_contrib, const float* v_image,
                                  const float* target, float l1_weight, double* loss, float* v2d, void* det_ws,
                                  size_t capacity, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  const DetLayout L = det_layout(M, batch.n_tiles, capacity);
  char* w = static_cast<char*>(det_ws);
  uint32_t* base = reinterpret_cast<uint32_t*>(w + L.base);
  unsigned long long* bsum = reinterpret_cast<unsigned long long*>(w + L.bsum);
  DetOut det;
  det.base = base;
  det.rect = reinterpret_cast<const ushort4*>(proj.rect);
  det.p8 = reinterpret_cast<float4*>(w + L.p8);
  det.p1 = reinterpret_cast<float*>(w + L.p1);
  det.cap = capacity;
  const bool fused_loss = loss != nullptr && v_image == nullptr;
  det.tile_loss = fused_loss ? reinterpret_cast<double*>(w + L.tile_loss) : nullptr;
  const int nblk = (int)((M + kDetTile - 1) / kDetTile);
  det_scan_reduce_kernel<<<nblk, kDetThreads, 0, st>>>(proj.n_tiles, M, bsum);
  det_scan_top_kernel<<<1, kDetThreads, 0, st>>>(bsum, nblk);
  det_scan_down_kernel<<<nblk, kDetThreads, 0, st>>>(proj.n_tiles, M, bsum, base);
  if (batch.n_tiles > 0) {
    const Sizes sz{cams.n_cams, cams.wh};
    const int rb = tuning().render_bwd_batch;
    if (batch.tile == 32)
      render_bwd_tile<32, true>(rb, batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, v_image,
                                target, l1_weight, loss, v2d, st, det);
    else
      render_bwd_tile<16, true>(rb, batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, v_image,
                                target, l1_weight, loss, v2d, st, det);
  }
  det_reduce_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(proj.n_tiles, base, bsum + nblk, n_instances,
                                                                 det.p8, det.p1, capacity, M, v2d);
  if (fused_loss && batch.n_tiles > 0) det_loss_kernel<<<1, kDetThreads, 0, st>>>(det.tile_loss, batch, loss);
  return cudaGetLastError();
}

cudaError_t launch_render_fwd_f64(const gs_batch& batch, const gs_cameras_f64& cams, const gs_projected_f64& proj,
                                  const uint32_t* vals, const uint32_t* ranges, const double* bg, double* image,
                                  double* T_final, uint32_t* n_contrib, uint32_t* n_added, cudaStream_t st) {
  if (batch.n_tiles == 0) return cudaSuccess;
  const Sizes sz{cams.n_cams, cams.wh};
  if (batch.tile == 32)
    render_fwd_launch<double, 32, 64>(batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, n_added,
                                      st);
  else
    render_fwd_launch<double, 16, 64>(batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, n_added,
                                      st);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd_f64(const gs_batch& batch, const gs_cameras_f64& cams, const gs_projected_f64& proj,
                                  const uint32_t* vals, const uint32_t* ranges, const double* bg,
                                  const double* image, const double* T_final, const uint32_t* n_contrib,
                                  const double* v_image, const double* target, double l1_weight, double* loss,
                                  double* v2d, cudaStream_t st) {
  if (batch.n_tiles == 0) return cudaSuccess;
  const Sizes sz{cams.n_cams, cams.wh};
  if (batch.tile == 32)
    render_bwd_launch<double, 32, 64>(batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, v_image,
                                      target, l1_weight, loss, v2d, st);
  else
    render_bwd_launch<double, 16, 64>(batch, sz, proj.splat, vals, ranges, bg, image, T_final, n_contrib, v_image,
                                      target, l1_weight, loss, v2d, st);
  return cudaGetLastError();
}

}  // namespace gs
