// EWA projection of Gaussians into a batch of views, forward and backward
// (the rasterizer the paper uses, Sec. 3.3 "Implementation"; the mean is
// projected with pi of Sec. 3.2).
//
// One thread owns one Gaussian and loops over the batch's views, so its
// parameters are read from HBM once per step and the view-independent work
// (activations, rotation, scaled axes) is done once.  Records are written
// structure-of-arrays by record index r = b * N + j, coalesced across the
// warp.  The backward recomputes the forward from the parameters (nothing
// but the screen-space gradients is read back) and keeps the parameter
// gradients of all views in registers; the per-view pose tangent is
// reduced warp (FP32 shuffles) -> block (FP32, fixed order) -> per-block
// double partial, and a second kernel sums the partials in a fixed order.
#include "gs_internal.h"

namespace gs {

namespace {

struct GaussGeo {
  float mu[3];
  float s[3];
  float qn[4];
  float qinv;     // 1 / |q|
  float R[9];     // rotation of the unit quaternion
  float M[9];     // R diag(s)
  float o;        // opacity
  float ol;
  bool ok;
};

// The raw parameters of one Gaussian, loaded apart from the arithmetic on
// them so that a kernel can issue these loads together with its others.
struct GeoRaw {
  float mu[3], ls[3];
  float4 q;
  float ol;
};

__device__ inline GeoRaw load_geo_raw(const gs_gaussians& g, int j) {
  GeoRaw r;
  const float* m = g.mean + 3 * (size_t)j;
  const float* ls = g.log_scale + 3 * (size_t)j;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.mu[i] = m[i];
    r.ls[i] = ls[i];
  }
  r.q = reinterpret_cast<const float4*>(g.quat)[j];
  r.ol = g.opacity_logit[j];
  return r;
}

__device__ inline GaussGeo make_geo(const GeoRaw& r) {
  GaussGeo G;
  const float4 q = r.q;
  G.ol = r.ol;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    G.mu[i] = r.mu[i];
    const float l = r.ls[i];
    ok = ok && finitef(G.mu[i]) && finitef(l);
    G.s[i] = expf(l);
  }
  ok = ok && finitef(q.x) && finitef(q.y) && finitef(q.z) && finitef(q.w) && finitef(G.ol);
  const float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  ok = ok && n2 > 0.f;
  const float inv = rsqrtf(n2);
  G.qinv = inv;
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  G.qn[0] = w; G.qn[1] = x; G.qn[2] = y; G.qn[3] = z;
  G.R[0] = 1.f - 2.f * (y * y + z * z);
  G.R[1] = 2.f * (x * y - w * z);
  G.R[2] = 2.f * (x * z + w * y);
  G.R[3] = 2.f * (x * y + w * z);
  G.R[4] = 1.f - 2.f * (x * x + z * z);
  G.R[5] = 2.f * (y * z - w * x);
  G.R[6] = 2.f * (x * z - w * y);
  G.R[7] = 2.f * (y * z + w * x);
  G.R[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) G.M[3 * r + c] = G.R[3 * r + c] * G.s[c];
  G.o = 1.f / (1.f + expf(-G.ol));
  G.ok = ok;
  return G;
}

// View-dependent part of the projection, shared by forward and backward so
// that both see identical FP32 values.
struct ViewGeo {
  float xc[3];
  float Mc[9];      // R_cam M
  float Sc[6];      // camera-frame covariance xx xy xz yy yz zz
  float tx, ty;     // clamped x/z, y/z
  bool clx, cly;
  float j00, j02, j11, j12;
  float S2[3];      // 2-D covariance xx xy yy (dilated)
  float det;
  float conic[3];
  float m2[2];
  float dir[3];
  float dnorm;
  bool visible;     // passes near/far and det > 0 (not yet opacity/rect)
};

__device__ inline void view_geo(const GaussGeo& G, const SlotCam& c, float near_p, float far_p,
                                ViewGeo& V) {
  const float* W = c.R;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    V.xc[r] = W[3 * r] * G.mu[0] + W[3 * r + 1] * G.mu[1] + W[3 * r + 2] * G.mu[2] + c.t[r];
  const float z = V.xc[2];
  V.visible = (z >= near_p) && (z <= far_p);
  if (!V.visible) return;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      V.Mc[3 * r + k] = W[3 * r] * G.M[k] + W[3 * r + 1] * G.M[3 + k] + W[3 * r + 2] * G.M[6 + k];
  const float* A = V.Mc;
  V.Sc[0] = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
  V.Sc[1] = A[0] * A[3] + A[1] * A[4] + A[2] * A[5];
  V.Sc[2] = A[0] * A[6] + A[1] * A[7] + A[2] * A[8];
  V.Sc[3] = A[3] * A[3] + A[4] * A[4] + A[5] * A[5];
  V.Sc[4] = A[3] * A[6] + A[4] * A[7] + A[5] * A[8];
  V.Sc[5] = A[6] * A[6] + A[7] * A[7] + A[8] * A[8];
  const float iz = 1.f / z;
  const float ux = V.xc[0] * iz, uy = V.xc[1] * iz;
  V.tx = fminf(fmaxf(ux, -c.limx), c.limx);
  V.ty = fminf(fmaxf(uy, -c.limy), c.limy);
  V.clx = (ux < -c.limx) || (ux > c.limx);
  V.cly = (uy < -c.limy) || (uy > c.limy);
  V.j00 = c.fx * iz;
  V.j11 = c.fy * iz;
  V.j02 = -c.fx * V.tx * iz;
  V.j12 = -c.fy * V.ty * iz;
  const float* S = V.Sc;
  V.S2[0] = V.j00 * V.j00 * S[0] + 2.f * V.j00 * V.j02 * S[2] + V.j02 * V.j02 * S[5] + kDilation;
  V.S2[1] = V.j00 * V.j11 * S[1] + V.j00 * V.j12 * S[2] + V.j02 * V.j11 * S[4] + V.j02 * V.j12 * S[5];
  V.S2[2] = V.j11 * V.j11 * S[3] + 2.f * V.j11 * V.j12 * S[4] + V.j12 * V.j12 * S[5] + kDilation;
  V.det = V.S2[0] * V.S2[2] - V.S2[1] * V.S2[1];
  V.visible = V.det > 0.f;
  if (!V.visible) return;
  const float idet = 1.f / V.det;
  V.conic[0] = V.S2[2] * idet;
  V.conic[1] = -V.S2[1] * idet;
  V.conic[2] = V.S2[0] * idet;
  V.m2[0] = c.fx * ux + c.cx;
  V.m2[1] = c.fy * uy + c.cy;
  float d0 = G.mu[0] - c.campos[0], d1 = G.mu[1] - c.campos[1], d2 = G.mu[2] - c.campos[2];
  V.dnorm = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  const float idn = 1.f / V.dnorm;
  V.dir[0] = d0 * idn;
  V.dir[1] = d1 * idn;
  V.dir[2] = d2 * idn;
}

constexpr int kProjThreads = 128;

// SH coefficients of the block's Gaussians [j0, j0 + n_local), contiguous in
// global memory, loaded with coalesced reads into shared memory transposed
// (coefficient-major, one padded column per thread) so that each thread then
// reads its own 3K values without bank conflicts.
// A full block whose slice is 16-byte aligned issues all its vector loads
// before the first shared-memory store, so it waits one memory latency
// rather than one per loop trip.
template <int KK>
__device__ inline void load_sh_block(const float* __restrict__ sh, int j0, int n_local,
                                     float (*s_sh)[kProjThreads + 1]) {
  const float* src = sh + (size_t)j0 * KK;
  if (n_local == kProjThreads && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    constexpr int kVec = KK * kProjThreads / 4;
    constexpr int kIt = (kVec + kProjThreads - 1) / kProjThreads;
    const float4* src4 = reinterpret_cast<const float4*>(src);
    float4 v[kIt];
#pragma unroll
    for (int u = 0; u < kIt; ++u) {
      const int q = u * kProjThreads + threadIdx.x;
      if (q < kVec) v[u] = src4[q];
    }
#pragma unroll
    for (int u = 0; u < kIt; ++u) {
      const int q = u * kProjThreads + threadIdx.x;
      if (q < kVec) {
        const float c[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int f = 4 * q + e;
          const int jl = f / KK;
          s_sh[f - jl * KK][jl] = c[e];
        }
      }
    }
    return;
  }
  const int total = n_local * KK;
  for (int f = threadIdx.x; f < total; f += kProjThreads) {
    const int jl = f / KK;
    s_sh[f - jl * KK][jl] = src[f];
  }
}

// dst[f] += column-major shared sums for the block's contiguous slice of
// [n_local, KK] gradients; the full-block, aligned case reads all of its
// slice before the first store (one memory latency per block).
template <int KK>
__device__ inline void add_sh_block(float* __restrict__ dst, int n_local, float (*s_v)[kProjThreads + 1]) {
  if (n_local == kProjThreads && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
    constexpr int kVec = KK * kProjThreads / 4;
    constexpr int kIt = (kVec + kProjThreads - 1) / kProjThreads;
    float4* dst4 = reinterpret_cast<float4*>(dst);
    float4 v[kIt];
#pragma unroll
    for (int u = 0; u < kIt; ++u) {
      const int q = u * kProjThreads + threadIdx.x;
      if (q < kVec) v[u] = dst4[q];
    }
#pragma unroll
    for (int u = 0; u < kIt; ++u) {
      const int q = u * kProjThreads + threadIdx.x;
      if (q < kVec) {
        float c[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int f = 4 * q + e;
          const int jl = f / KK;
          c[e] += s_v[f - jl * KK][jl];
        }
        dst4[q] = make_float4(c[0], c[1], c[2], c[3]);
      }
    }
    return;
  }
  const int total = n_local * KK;
  for (int f = threadIdx.x; f < total; f += kProjThreads) {
    const int jl = f / KK;
    const float gv = s_v[f - jl * KK][jl];
    if (gv != 0.f) dst[f] += gv;
  }
}

template <int DEG>
__global__ void __launch_bounds__(kProjThreads) project_fwd_kernel(gs_gaussians g, gs_cameras cams,
                                                                   gs_batch batch, gs_projected out,
                                                                   int32_t* status) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ SlotCam sc[GS_MAX_BATCH];
  __shared__ float s_sh[K * 3][kProjThreads + 1];
  load_slot_cams(cams, batch, sc);
  const int N = g.n;
  const int j0 = blockIdx.x * kProjThreads;
  load_sh_block<K * 3>(g.sh, j0, min(kProjThreads, N - j0), s_sh);
  __syncthreads();
  const int j = j0 + threadIdx.x;
  if (j >= N) return;
  const GaussGeo G = make_geo(load_geo_raw(g, j));
  float shv[K * 3];
#pragma unroll
  for (int i = 0; i < K * 3; ++i) shv[i] = s_sh[i][threadIdx.x];
  bool ok = G.ok;
#pragma unroll
  for (int i = 0; i < K * 3; ++i) ok = ok && finitef(shv[i]);
  if (!ok) set_flag(status, GS_FLAG_NONFINITE);
  const bool opaque_enough = G.o >= kAlphaMin;
  const float Qcut = 2.f * logf(255.f * G.o);
  const int T = batch.tile;
  for (int b = 0; b < batch.B; ++b) {
    const size_t rec = (size_t)b * N + j;
    const SlotCam& c = sc[b];
    uint32_t ntiles = 0;
    uint32_t dkey = 0xffffffffu;
    if (ok && opaque_enough) {
      ViewGeo V;
      view_geo(G, c, cams.near_plane, cams.far_plane, V);
      if (V.visible) {
        const float rx = sqrtf(Qcut * V.S2[0]);
        const float ry = sqrtf(Qcut * V.S2[2]);
        float x0 = ceilf(V.m2[0] - rx - 0.5f) - 1.f;
        float y0 = ceilf(V.m2[1] - ry - 0.5f) - 1.f;
        float x1 = floorf(V.m2[0] + rx - 0.5f) + 1.f;
        float y1 = floorf(V.m2[1] + ry - 0.5f) + 1.f;
        x0 = fmaxf(x0, 0.f);
        y0 = fmaxf(y0, 0.f);
        x1 = fminf(x1, (float)(c.W - 1));
        y1 = fminf(y1, (float)(c.H - 1));
        if (x0 <= x1 && y0 <= y1) {
          const int tx0 = (int)x0 / T, ty0 = (int)y0 / T;
          const int tx1 = (int)x1 / T, ty1 = (int)y1 / T;
          ntiles = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
          dkey = __float_as_uint(V.xc[2]);
          float Y[K];
          sh_basis(DEG, V.dir[0], V.dir[1], V.dir[2], Y);
          float col[3];
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            float v = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) v += shv[3 * k + ch] * Y[k];
            col[ch] = fmaxf(v, 0.f);
          }
          float4* sp = reinterpret_cast<float4*>(out.splat) + 3 * rec;
          sp[0] = make_float4(V.m2[0], V.m2[1], G.o, V.xc[2]);
          sp[1] = make_float4(V.conic[0], V.conic[1], V.conic[2], Qcut);
          sp[2] = make_float4(col[0], col[1], col[2], 0.f);
          reinterpret_cast<ushort4*>(out.rect)[rec] =
              make_ushort4((unsigned short)tx0, (unsigned short)ty0, (unsigned short)tx1,
                           (unsigned short)ty1);
        }
      }
    }
    out.n_tiles[rec] = ntiles;
    out.depth_key[rec] = dkey;
  }
}

// Screen-space gradient record layout (12 floats per record):
// 0 mean2d x, 1 mean2d y, 2 conic a, 3 conic b, 4 conic c, 5 opacity,
// 6..8 colour, 9..11 unused.
template <int DEG>
constexpr size_t project_bwd_smem() {
  return sizeof(float) * 2 * (DEG + 1) * (DEG + 1) * 3 * (kProjThreads + 1);
}

template <int DEG>
__global__ void __launch_bounds__(kProjThreads, 3) project_bwd_kernel(gs_gaussians g, gs_cameras cams,
                                                                      gs_batch batch, gs_projected proj,
                                                                      const float* __restrict__ v2d,
                                                                      gs_gaussian_grads dg,
                                                                      double* __restrict__ partial) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ SlotCam sc[GS_MAX_BATCH];
  // per warp and view: the warp's six pose-tangent sums (FP32: the FP64
  // pipe is a small fraction of the FP32 rate; one conversion per block)
  __shared__ float s_tan[kProjThreads / 32][GS_MAX_BATCH * 6];
  // dynamic: coefficients and their gradient accumulators, one padded
  // column per thread
  extern __shared__ float s_dyn[];
  float (*s_sh)[kProjThreads + 1] = reinterpret_cast<float (*)[kProjThreads + 1]>(s_dyn);
  float (*s_vsh)[kProjThreads + 1] = reinterpret_cast<float (*)[kProjThreads + 1]>(s_dyn + K * 3 * (kProjThreads + 1));
  for (int i = threadIdx.x; i < (kProjThreads / 32) * GS_MAX_BATCH * 6; i += blockDim.x) (&s_tan[0][0])[i] = 0.f;
  const int N = g.n;
  const int j0 = blockIdx.x * kProjThreads;
  const int n_local = min(kProjThreads, N - j0);
  const int j = j0 + threadIdx.x;
  const bool active = j < N;
  // the parameters and the first view's record are loaded together with
  // the SH block, before the barrier
  GeoRaw raw;
  const float4* vrec = reinterpret_cast<const float4*>(v2d);
  float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb4 = na;
  float ncol = 0.f;
  if (active) {
    raw = load_geo_raw(g, j);
    na = vrec[3 * (size_t)j];
    nb4 = vrec[3 * (size_t)j + 1];
    ncol = vrec[3 * (size_t)j + 2].x;
  }
  load_slot_cams(cams, batch, sc);
  load_sh_block<K * 3>(g.sh, j0, n_local, s_sh);
#pragma unroll
  for (int i = 0; i < K * 3; ++i) s_vsh[i][threadIdx.x] = 0.f;
  __syncthreads();
  GaussGeo G;
  if (active) G = make_geo(raw);
  float vmu[3] = {0.f, 0.f, 0.f};
  float GM[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) GM[i] = 0.f;
  float vol = 0.f;
  bool any = false;

  // Screen-space gradients of invisible records are zero (the compositing
  // backward zeroes all records first), so every view's record can be read
  // unconditionally; the next view's is loaded while this one is processed.
  for (int b = 0; b < batch.B; ++b) {
    float tan[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float4 va = na, vb = nb4;
    const float vcol_b = ncol;
    if (active && b + 1 < batch.B) {
      const size_t nrec = (size_t)(b + 1) * N + j;
      na = vrec[3 * nrec];
      nb4 = vrec[3 * nrec + 1];
      ncol = vrec[3 * nrec + 2].x;
    }
    const bool live = active && ((va.x != 0.f) || (va.y != 0.f) || (va.z != 0.f) || (va.w != 0.f) ||
                                 (vb.x != 0.f) || (vb.y != 0.f) || (vb.z != 0.f) || (vb.w != 0.f) ||
                                 (vcol_b != 0.f));
    if (live) {
      any = true;
      const SlotCam& c = sc[b];
      ViewGeo V;
      view_geo(G, c, cams.near_plane, cams.far_plane, V);
      const float v_mx = va.x, v_my = va.y, v_a = va.z, v_b = va.w;
      const float v_c = vb.x, v_o = vb.y;
      float vcol[3] = {vb.z, vb.w, vcol_b};
      // --- colour: SH and view direction --------------------------------
      float Y[K];
      sh_basis(DEG, V.dir[0], V.dir[1], V.dir[2], Y);
      float wk[K];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float raw = 0.5f;
#pragma unroll
        for (int k = 0; k < K; ++k) raw += s_sh[3 * k + ch][threadIdx.x] * Y[k];
        if (raw < 0.f) vcol[ch] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float s0 = s_sh[3 * k][threadIdx.x], s1 = s_sh[3 * k + 1][threadIdx.x],
                    s2 = s_sh[3 * k + 2][threadIdx.x];
        wk[k] = s0 * vcol[0] + s1 * vcol[1] + s2 * vcol[2];
        s_vsh[3 * k][threadIdx.x] += Y[k] * vcol[0];
        s_vsh[3 * k + 1][threadIdx.x] += Y[k] * vcol[1];
        s_vsh[3 * k + 2][threadIdx.x] += Y[k] * vcol[2];
      }
      float vdir[3] = {0.f, 0.f, 0.f};
      sh_basis_grad_dot(DEG, V.dir[0], V.dir[1], V.dir[2], wk, vdir);
      const float dd = vdir[0] * V.dir[0] + vdir[1] * V.dir[1] + vdir[2] * V.dir[2];
      const float idn = 1.f / V.dnorm;
      float vdv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        vdv[i] = (vdir[i] - dd * V.dir[i]) * idn;
        vmu[i] += vdv[i];
      }
      // v_campos = -vdv; its pose effect: g_rho += -R v_campos = R vdv
      // --- opacity -------------------------------------------------------
      vol += v_o;
      // --- conic -> 2-D covariance: G_S2 = -Q G_Q Q -----------------------
      const float a = V.conic[0], bq = V.conic[1], cq = V.conic[2];
      const float hb = 0.5f * v_b;
      const float X00 = v_a * a + hb * bq, X01 = v_a * bq + hb * cq;
      const float X10 = hb * a + v_c * bq, X11 = hb * bq + v_c * cq;
      const float gxx = -(a * X00 + bq * X10);
      const float gxy = -(a * X01 + bq * X11);
      const float gyy = -(bq * X01 + cq * X11);
      // --- S2 = J Sc J^T: H = G_S2 J, G_Sc = J^T H, G_J = 2 H Sc ----------
      const float H00 = gxx * V.j00, H01 = gxy * V.j11, H02 = gxx * V.j02 + gxy * V.j12;
      const float H10 = gxy * V.j00, H11 = gyy * V.j11, H12 = gxy * V.j02 + gyy * V.j12;
      float GSc[9];
      GSc[0] = V.j00 * H00; GSc[1] = V.j00 * H01; GSc[2] = V.j00 * H02;
      GSc[3] = V.j11 * H10; GSc[4] = V.j11 * H11; GSc[5] = V.j11 * H12;
      GSc[6] = V.j02 * H00 + V.j12 * H10;
      GSc[7] = V.j02 * H01 + V.j12 * H11;
      GSc[8] = V.j02 * H02 + V.j12 * H12;
      // symmetrise (exact symmetry is lost only to rounding)
      {
        const float s01 = 0.5f * (GSc[1] + GSc[3]);
        const float s02 = 0.5f * (GSc[2] + GSc[6]);
        const float s12 = 0.5f * (GSc[5] + GSc[7]);
        GSc[1] = GSc[3] = s01;
        GSc[2] = GSc[6] = s02;
        GSc[5] = GSc[7] = s12;
      }
      const float* S = V.Sc;
      // full symmetric Sc
      const float Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
      // G_J entries used: (0,0), (0,2), (1,1), (1,2)
      const float GJ00 = 2.f * (H00 * Sf[0] + H01 * Sf[3] + H02 * Sf[6]);
      const float GJ02 = 2.f * (H00 * Sf[2] + H01 * Sf[5] + H02 * Sf[8]);
      const float GJ11 = 2.f * (H10 * Sf[1] + H11 * Sf[4] + H12 * Sf[7]);
      const float GJ12 = 2.f * (H10 * Sf[2] + H11 * Sf[5] + H12 * Sf[8]);
      // --- Sc = Mc Mc^T, Mc = W M:  G_Mc = 2 G_Sc Mc; G_M += W^T G_Mc ---
      float GMc[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          GMc[3 * r + k] = 2.f * (GSc[3 * r] * V.Mc[k] + GSc[3 * r + 1] * V.Mc[3 + k] +
                                  GSc[3 * r + 2] * V.Mc[6 + k]);
      const float* W = c.R;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          GM[3 * r + k] += W[r] * GMc[k] + W[3 + r] * GMc[3 + k] + W[6 + r] * GMc[6 + k];
      // pose, rotation through the covariance: g_phi += 2 vee(G_Sc Sc)
      {
        float B[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int k = 0; k < 3; ++k)
            B[3 * r + k] = GSc[3 * r] * Sf[k] + GSc[3 * r + 1] * Sf[3 + k] + GSc[3 * r + 2] * Sf[6 + k];
        tan[3] += 2.f * (B[7] - B[5]);
        tan[4] += 2.f * (B[2] - B[6]);
        tan[5] += 2.f * (B[3] - B[1]);
      }
      // --- J(x_c) and mean2d -> v_xc ------------------------------------
      const float z = V.xc[2];
      const float iz = 1.f / z, iz2 = iz * iz;
      float vxc[3];
      const float dJ02dx = V.clx ? 0.f : -c.fx * iz2;
      const float dJ12dy = V.cly ? 0.f : -c.fy * iz2;
      const float dJ02dz = c.fx * V.tx * iz2 + (V.clx ? 0.f : c.fx * V.xc[0] * iz2 * iz);
      const float dJ12dz = c.fy * V.ty * iz2 + (V.cly ? 0.f : c.fy * V.xc[1] * iz2 * iz);
      vxc[0] = GJ02 * dJ02dx + v_mx * c.fx * iz;
      vxc[1] = GJ12 * dJ12dy + v_my * c.fy * iz;
      vxc[2] = -GJ00 * c.fx * iz2 - GJ11 * c.fy * iz2 + GJ02 * dJ02dz + GJ12 * dJ12dz -
               (v_mx * c.fx * V.xc[0] + v_my * c.fy * V.xc[1]) * iz2;
      // --- x_c = W mu + t ------------------------------------------------
#pragma unroll
      for (int i = 0; i < 3; ++i) vmu[i] += W[i] * vxc[0] + W[3 + i] * vxc[1] + W[6 + i] * vxc[2];
      // pose: g_rho = v_xc + W vdv; g_phi += x_c x v_xc
      tan[0] = vxc[0] + W[0] * vdv[0] + W[1] * vdv[1] + W[2] * vdv[2];
      tan[1] = vxc[1] + W[3] * vdv[0] + W[4] * vdv[1] + W[5] * vdv[2];
      tan[2] = vxc[2] + W[6] * vdv[0] + W[7] * vdv[1] + W[8] * vdv[2];
      tan[3] += V.xc[1] * vxc[2] - V.xc[2] * vxc[1];
      tan[4] += V.xc[2] * vxc[0] - V.xc[0] * vxc[2];
      tan[5] += V.xc[0] * vxc[1] - V.xc[1] * vxc[0];
    }
    // warp reduce the 6 tangent values into the warp's own slots
    const unsigned any_live = __ballot_sync(0xffffffffu, live);
    if (any_live) {
      const int lane = threadIdx.x & 31;
      float mine = 0.f;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        float v = tan[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == i) mine = v;
      }
      if (lane < 6) s_tan[threadIdx.x >> 5][6 * b + lane] = mine;
    }
  }

  if (active && any) {
    // the accumulators are read before any of them is written, so the
    // thread waits one memory latency for all of them
    float* gls = dg.log_scale + 3 * (size_t)j;
    float4* gq = reinterpret_cast<float4*>(dg.quat) + j;
    float* gm = dg.mean + 3 * (size_t)j;
    float acc_ls[3], acc_mu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc_ls[k] = gls[k];
      acc_mu[k] = gm[k];
    }
    float4 cur = *gq;
    float acc_o = dg.opacity_logit[j];
    // --- M = R diag(s): G_R = G_M diag(s), dL/ds_c = sum_r G_M[r][c] R[r][c]
    float GR[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) GR[3 * r + k] = GM[3 * r + k] * G.s[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float gs = GM[k] * G.R[k] + GM[3 + k] * G.R[3 + k] + GM[6 + k] * G.R[6 + k];
      gls[k] = acc_ls[k] + gs * G.s[k];
    }
    const float w = G.qn[0], x = G.qn[1], y = G.qn[2], zq = G.qn[3];
    float vq[4];
    vq[0] = -2.f * zq * GR[1] + 2.f * y * GR[2] + 2.f * zq * GR[3] - 2.f * x * GR[5] -
            2.f * y * GR[6] + 2.f * x * GR[7];
    vq[1] = 2.f * y * GR[1] + 2.f * zq * GR[2] + 2.f * y * GR[3] - 4.f * x * GR[4] -
            2.f * w * GR[5] + 2.f * zq * GR[6] + 2.f * w * GR[7] - 4.f * x * GR[8];
    vq[2] = -4.f * y * GR[0] + 2.f * x * GR[1] + 2.f * w * GR[2] + 2.f * x * GR[3] +
            2.f * zq * GR[5] - 2.f * w * GR[6] + 2.f * zq * GR[7] - 4.f * y * GR[8];
    vq[3] = -4.f * zq * GR[0] - 2.f * w * GR[1] + 2.f * x * GR[2] + 2.f * w * GR[3] -
            4.f * zq * GR[4] + 2.f * y * GR[5] + 2.f * x * GR[6] + 2.f * y * GR[7];
    const float dq = vq[0] * w + vq[1] * x + vq[2] * y + vq[3] * zq;
    cur.x += (vq[0] - dq * w) * G.qinv;
    cur.y += (vq[1] - dq * x) * G.qinv;
    cur.z += (vq[2] - dq * y) * G.qinv;
    cur.w += (vq[3] - dq * zq) * G.qinv;
    *gq = cur;
#pragma unroll
    for (int i = 0; i < 3; ++i) gm[i] = acc_mu[i] + vmu[i];
    dg.opacity_logit[j] = acc_o + vol * G.o * (1.f - G.o);
  }
  // SH gradients: through shared memory, then one coalesced read-modify-write
  // of the block's contiguous slice of dg.sh
  __syncthreads();
  add_sh_block<K * 3>(dg.sh + (size_t)j0 * K * 3, n_local, s_vsh);
  __syncthreads();
  for (int i = threadIdx.x; i < batch.B * 6; i += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kProjThreads / 32; ++w) t += s_tan[w][i];
    partial[(size_t)blockIdx.x * batch.B * 6 + i] = (double)t;
  }
}

}  // namespace

cudaError_t launch_project_fwd(const gs_gaussians& g, const gs_cameras& cams,
                               const gs_batch& batch, const gs_projected& out, int32_t* status,
                               cudaStream_t st) {
  const int threads = kProjThreads;
  const int blocks = (g.n + threads - 1) / threads;
  if (blocks == 0) return cudaSuccess;
  switch (g.sh_degree) {
    case 0: project_fwd_kernel<0><<<blocks, threads, 0, st>>>(g, cams, batch, out, status); break;
    case 1: project_fwd_kernel<1><<<blocks, threads, 0, st>>>(g, cams, batch, out, status); break;
    case 2: project_fwd_kernel<2><<<blocks, threads, 0, st>>>(g, cams, batch, out, status); break;
    default: project_fwd_kernel<3><<<blocks, threads, 0, st>>>(g, cams, batch, out, status); break;
  }
  return cudaGetLastError();
}

int project_bwd_blocks(int n) { return (n + kProjThreads - 1) / kProjThreads; }

template <int DEG>
cudaError_t launch_project_bwd_deg(const gs_gaussians& g, const gs_cameras& cams, const gs_batch& batch,
                                   const gs_projected& proj, const float* v2d, const gs_gaussian_grads& dg,
                                   double* partial, int blocks, cudaStream_t st) {
  constexpr size_t smem = project_bwd_smem<DEG>();
  // the opt-in for more than 48 KB of shared memory, once per device
  static bool configured[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    e = cudaFuncSetAttribute(project_bwd_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  project_bwd_kernel<DEG><<<blocks, kProjThreads, smem, st>>>(g, cams, batch, proj, v2d, dg, partial);
  return cudaGetLastError();
}

cudaError_t launch_project_bwd(const gs_gaussians& g, const gs_cameras& cams,
                               const gs_batch& batch, const gs_projected& proj, const float* v2d,
                               const gs_gaussian_grads& dg, double* partial,
                               double* g_pose_tangent, cudaStream_t st) {
  const int blocks = project_bwd_blocks(g.n);
  if (blocks == 0) return cudaSuccess;
  cudaError_t e;
  switch (g.sh_degree) {
    case 0: e = launch_project_bwd_deg<0>(g, cams, batch, proj, v2d, dg, partial, blocks, st); break;
    case 1: e = launch_project_bwd_deg<1>(g, cams, batch, proj, v2d, dg, partial, blocks, st); break;
    case 2: e = launch_project_bwd_deg<2>(g, cams, batch, proj, v2d, dg, partial, blocks, st); break;
    default: e = launch_project_bwd_deg<3>(g, cams, batch, proj, v2d, dg, partial, blocks, st); break;
  }
  if (e != cudaSuccess) return e;
  return launch_pose_partials_finalize(partial, blocks, batch, cams.n_cams, g_pose_tangent, st);
}

}  // namespace gs
