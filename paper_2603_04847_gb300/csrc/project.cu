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

template <typename T>
struct GaussGeo {
  T mu[3];
  T s[3];
  T qn[4];
  T qinv;     // 1 / |q|
  T R[9];     // rotation of the unit quaternion
  T M[9];     // R diag(s)
  T o;        // opacity
  T ol;
  bool ok;
};

template <typename T>
struct Quat4 {
  T x, y, z, w;
};

// The raw parameters of one Gaussian, loaded apart from the arithmetic on
// them so that a kernel can issue these loads together with its others.
template <typename T>
struct GeoRaw {
  T mu[3], ls[3];
  Quat4<T> q;
  T ol;
};

__device__ inline Quat4<float> load_quat(const float* q, int j) {
  const float4 v = reinterpret_cast<const float4*>(q)[j];
  return Quat4<float>{v.x, v.y, v.z, v.w};
}
__device__ inline Quat4<double> load_quat(const double* q, int j) {
  const double2 a = reinterpret_cast<const double2*>(q)[2 * (size_t)j];
  const double2 b = reinterpret_cast<const double2*>(q)[2 * (size_t)j + 1];
  return Quat4<double>{a.x, a.y, b.x, b.y};
}

__device__ inline void store_quat(float* p, const Quat4<float>& q) {
  *reinterpret_cast<float4*>(p) = make_float4(q.x, q.y, q.z, q.w);
}
__device__ inline void store_quat(double* p, const Quat4<double>& q) {
  reinterpret_cast<double2*>(p)[0] = make_double2(q.x, q.y);
  reinterpret_cast<double2*>(p)[1] = make_double2(q.z, q.w);
}

template <typename T>
__device__ inline GeoRaw<T> load_geo_raw(const GaussT<T>& g, int j) {
  GeoRaw<T> r;
  const T* m = g.mean + 3 * (size_t)j;
  const T* ls = g.log_scale + 3 * (size_t)j;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.mu[i] = m[i];
    r.ls[i] = ls[i];
  }
  r.q = load_quat(g.quat, j);
  r.ol = g.opacity_logit[j];
  return r;
}

template <typename T>
__device__ inline GaussGeo<T> make_geo(const GeoRaw<T>& r) {
  GaussGeo<T> G;
  const Quat4<T> q = r.q;
  G.ol = r.ol;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    G.mu[i] = r.mu[i];
    const T l = r.ls[i];
    ok = ok && finitef(G.mu[i]) && finitef(l);
    G.s[i] = gexp(l);
  }
  ok = ok && finitef(q.x) && finitef(q.y) && finitef(q.z) && finitef(q.w) && finitef(G.ol);
  const T n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  ok = ok && n2 > T(0);
  const T inv = grsqrt(n2);
  G.qinv = inv;
  const T w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  G.qn[0] = w; G.qn[1] = x; G.qn[2] = y; G.qn[3] = z;
  G.R[0] = T(1) - T(2) * (y * y + z * z);
  G.R[1] = T(2) * (x * y - w * z);
  G.R[2] = T(2) * (x * z + w * y);
  G.R[3] = T(2) * (x * y + w * z);
  G.R[4] = T(1) - T(2) * (x * x + z * z);
  G.R[5] = T(2) * (y * z - w * x);
  G.R[6] = T(2) * (x * z - w * y);
  G.R[7] = T(2) * (y * z + w * x);
  G.R[8] = T(1) - T(2) * (x * x + y * y);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) G.M[3 * r + c] = G.R[3 * r + c] * G.s[c];
  G.o = T(1) / (T(1) + gexp(-G.ol));
  G.ok = ok;
  return G;
}

// View-dependent part of the projection, shared by forward and backward so
// that both see identical values.
template <typename T>
struct ViewGeo {
  T xc[3];
  T Mc[9];      // R_cam M
  T Sc[6];      // camera-frame covariance xx xy xz yy yz zz
  T tx, ty;     // clamped x/z, y/z
  bool clx, cly;
  T j00, j02, j11, j12;
  T S2[3];      // 2-D covariance xx xy yy (dilated)
  T det;
  T idet;       // 1 / det
  T conic[3];
  T m2[2];
  T dir[3];
  T dnorm;
  bool visible;     // passes near/far and det > 0 (not yet opacity/rect)
};

template <typename T>
__device__ inline void view_geo(const GaussGeo<T>& G, const SlotCamT<T>& c, T near_p, T far_p, ViewGeo<T>& V) {
  const T* W = c.R;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    V.xc[r] = W[3 * r] * G.mu[0] + W[3 * r + 1] * G.mu[1] + W[3 * r + 2] * G.mu[2] + c.t[r];
  const T z = V.xc[2];
  V.visible = (z >= near_p) && (z <= far_p);
  if (!V.visible) return;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      V.Mc[3 * r + k] = W[3 * r] * G.M[k] + W[3 * r + 1] * G.M[3 + k] + W[3 * r + 2] * G.M[6 + k];
  const T* A = V.Mc;
  V.Sc[0] = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
  V.Sc[1] = A[0] * A[3] + A[1] * A[4] + A[2] * A[5];
  V.Sc[2] = A[0] * A[6] + A[1] * A[7] + A[2] * A[8];
  V.Sc[3] = A[3] * A[3] + A[4] * A[4] + A[5] * A[5];
  V.Sc[4] = A[3] * A[6] + A[4] * A[7] + A[5] * A[8];
  V.Sc[5] = A[6] * A[6] + A[7] * A[7] + A[8] * A[8];
  const T iz = T(1) / z;
  const T ux = V.xc[0] * iz, uy = V.xc[1] * iz;
  V.tx = gmin(gmax(ux, -c.limx), c.limx);
  V.ty = gmin(gmax(uy, -c.limy), c.limy);
  V.clx = (ux < -c.limx) || (ux > c.limx);
  V.cly = (uy < -c.limy) || (uy > c.limy);
  V.j00 = c.fx * iz;
  V.j11 = c.fy * iz;
  V.j02 = -c.fx * V.tx * iz;
  V.j12 = -c.fy * V.ty * iz;
  const T* S = V.Sc;
  const T dil = Consts<T>::dilation;
  V.S2[0] = V.j00 * V.j00 * S[0] + T(2) * V.j00 * V.j02 * S[2] + V.j02 * V.j02 * S[5] + dil;
  V.S2[1] = V.j00 * V.j11 * S[1] + V.j00 * V.j12 * S[2] + V.j02 * V.j11 * S[4] + V.j02 * V.j12 * S[5];
  V.S2[2] = V.j11 * V.j11 * S[3] + T(2) * V.j11 * V.j12 * S[4] + V.j12 * V.j12 * S[5] + dil;
  V.det = V.S2[0] * V.S2[2] - V.S2[1] * V.S2[1];
  V.visible = V.det > T(0);
  if (!V.visible) return;
  const T idet = T(1) / V.det;
  V.idet = idet;
  V.conic[0] = V.S2[2] * idet;
  V.conic[1] = -V.S2[1] * idet;
  V.conic[2] = V.S2[0] * idet;
  V.m2[0] = c.fx * ux + c.cx;
  V.m2[1] = c.fy * uy + c.cy;
  T d0 = G.mu[0] - c.campos[0], d1 = G.mu[1] - c.campos[1], d2 = G.mu[2] - c.campos[2];
  V.dnorm = gsqrt(d0 * d0 + d1 * d1 + d2 * d2);
  const T idn = T(1) / V.dnorm;
  V.dir[0] = d0 * idn;
  V.dir[1] = d1 * idn;
  V.dir[2] = d2 * idn;
}

constexpr int kProjThreads = 128;

// SH coefficients of the block's Gaussians [j0, j0 + n_local), contiguous in
// global memory, loaded with coalesced reads into shared memory transposed
// (coefficient-major, one padded column per thread) so that each thread then
// reads its own 3K values without bank conflicts.
// A full FP32 block whose slice is 16-byte aligned issues all its vector
// loads before the first shared-memory store, so it waits one memory
// latency rather than one per loop trip.
template <typename T, int KK>
__device__ inline void load_sh_block(const T* __restrict__ sh, int j0, int n_local, T (*s_sh)[kProjThreads + 1]) {
  const T* src = sh + (size_t)j0 * KK;
  if constexpr (sizeof(T) == 4) {
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
  }
  const int total = n_local * KK;
  for (int f = threadIdx.x; f < total; f += kProjThreads) {
    const int jl = f / KK;
    s_sh[f - jl * KK][jl] = src[f];
  }
}

// dst[f] += column-major shared sums for the block's contiguous slice of
// [n_local, KK] gradients; the full-block, aligned FP32 case reads all of
// its slice before the first store (one memory latency per block).
template <typename T, int KK>
__device__ inline void add_sh_block(T* __restrict__ dst, int n_local, T (*s_v)[kProjThreads + 1]) {
  if constexpr (sizeof(T) == 4) {
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
  }
  const int total = n_local * KK;
  for (int f = threadIdx.x; f < total; f += kProjThreads) {
    const int jl = f / KK;
    const T gv = s_v[f - jl * KK][jl];
    if (gv != T(0)) dst[f] += gv;
  }
}

// The three 4-vectors of a splat record (12 scalars).
__device__ inline void store_splat(float* sp, size_t rec, const float (&v)[12]) {
  float4* p = reinterpret_cast<float4*>(sp) + 3 * rec;
  p[0] = make_float4(v[0], v[1], v[2], v[3]);
  p[1] = make_float4(v[4], v[5], v[6], v[7]);
  p[2] = make_float4(v[8], v[9], v[10], v[11]);
}
__device__ inline void store_splat(double* sp, size_t rec, const double (&v)[12]) {
  double2* p = reinterpret_cast<double2*>(sp) + 6 * rec;
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

// The first nine scalars of a screen-space gradient record (12 per record).
__device__ inline void load_rec9(const float* v2d, size_t rec, float (&o)[9]) {
  const float4* p = reinterpret_cast<const float4*>(v2d) + 3 * rec;
  const float4 a = p[0], b = p[1];
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  o[8] = p[2].x;
}
// Zeroes record rec (all 12 scalars) after it has been read.
__device__ inline void clear_rec(float* v2d, size_t rec) {
  float4* p = reinterpret_cast<float4*>(v2d) + 3 * rec;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  p[0] = z;
  p[1] = z;
  p[2] = z;
}
__device__ inline void clear_rec(double* v2d, size_t rec) {
  double2* p = reinterpret_cast<double2*>(v2d) + 6 * rec;
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = make_double2(0.0, 0.0);
}
__device__ inline void load_rec9(const double* v2d, size_t rec, double (&o)[9]) {
  const double2* p = reinterpret_cast<const double2*>(v2d) + 6 * rec;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 v = p[i];
    o[2 * i] = v.x;
    o[2 * i + 1] = v.y;
  }
  o[8] = p[4].x;
}

// FP32: 5 blocks of 128 per SM (96 registers; the SH3 form spills 16 bytes):
// 1.49 -> 1.47 ms on the 16-view, 5M-Gaussian step, where 6 blocks spill 88
// bytes and lose
template <typename T, int DEG>
__global__ void __launch_bounds__(kProjThreads, sizeof(T) == 4 ? 5 : 1)
    project_fwd_kernel(GaussT<T> g, CamsT<T> cams, gs_batch batch, ProjT<T> out, int32_t* status) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ SlotCamT<T> sc[GS_MAX_BATCH];
  __shared__ T s_sh[K * 3][kProjThreads + 1];
  load_slot_cams(cams, batch, sc);
  const int N = g.n;
  const int j0 = blockIdx.x * kProjThreads;
  load_sh_block<T, K * 3>(g.sh, j0, min(kProjThreads, N - j0), s_sh);
  __syncthreads();
  const int j = j0 + threadIdx.x;
  if (j >= N) return;
  const GaussGeo<T> G = make_geo(load_geo_raw(g, j));
  T shv[K * 3];
#pragma unroll
  for (int i = 0; i < K * 3; ++i) shv[i] = s_sh[i][threadIdx.x];
  bool ok = G.ok;
#pragma unroll
  for (int i = 0; i < K * 3; ++i) ok = ok && finitef(shv[i]);
  if (!ok) set_flag(status, GS_FLAG_NONFINITE);
  const bool opaque_enough = G.o >= Consts<T>::alpha_min;
  const T Qcut = T(2) * glog(T(255) * G.o);
  const int TL = batch.tile;
  for (int b = 0; b < batch.B; ++b) {
    const size_t rec = (size_t)b * N + j;
    const SlotCamT<T>& c = sc[b];
    uint32_t ntiles = 0;
    uint32_t dkey = 0xffffffffu;
    if (ok && opaque_enough && c.active) {
      ViewGeo<T> V;
      view_geo(G, c, cams.near_plane, cams.far_plane, V);
      if (V.visible) {
        const T rx = gsqrt(Qcut * V.S2[0]);
        const T ry = gsqrt(Qcut * V.S2[2]);
        // the pixels whose centre lies in the support's bounding box, with
        // 1/64 px of margin (~100 times the float rounding of the bounds)
        const T mg = T(1) / T(64);
        T x0 = gceil(V.m2[0] - rx - T(0.5) - mg);
        T y0 = gceil(V.m2[1] - ry - T(0.5) - mg);
        T x1 = gfloor(V.m2[0] + rx - T(0.5) + mg);
        T y1 = gfloor(V.m2[1] + ry - T(0.5) + mg);
        x0 = gmax(x0, T(0));
        y0 = gmax(y0, T(0));
        x1 = gmin(x1, (T)(c.W - 1));
        y1 = gmin(y1, (T)(c.H - 1));
        if (x0 <= x1 && y0 <= y1) {
          const int tx0 = (int)x0 / TL, ty0 = (int)y0 / TL;
          const int tx1 = (int)x1 / TL, ty1 = (int)y1 / TL;
          ntiles = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
          // positive floats order like their bits; the FP64 path keys on
          // the float rounding of its depth (ties keep index order)
          dkey = __float_as_uint((float)V.xc[2]);
          T Y[K];
          sh_basis<T>(DEG, V.dir[0], V.dir[1], V.dir[2], Y);
          T col[3];
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            T v = T(0.5);
#pragma unroll
            for (int k = 0; k < K; ++k) v += shv[3 * k + ch] * Y[k];
            col[ch] = gmax(v, T(0));
          }
          const T rv[12] = {V.m2[0], V.m2[1], G.o, V.xc[2], V.conic[0], V.conic[1], V.conic[2], Qcut,
                            col[0], col[1], col[2], T(0)};
          store_splat(out.splat, rec, rv);
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
template <typename T, int DEG>
constexpr size_t project_bwd_smem() {
  return sizeof(T) * 2 * (DEG + 1) * (DEG + 1) * 3 * (kProjThreads + 1);
}

// 3 blocks of 128 per SM for FP32 (168 registers); the FP64 instantiation
// is a checking path and takes what it needs
// Blocks per SM the FP32 projection backward is compiled for (its register
// budget): 3 (163 registers, no spills).  At 4 the SH3 kernel spills 88
// bytes and measured 4.01 against 3.33 ms on the 16-view, 5M-Gaussian step.
constexpr int kProjBwdMinBlocks = 3;

template <typename T, int DEG>
__global__ void __launch_bounds__(kProjThreads, sizeof(T) == 4 ? kProjBwdMinBlocks : 1) project_bwd_kernel(
    GaussT<T> g, CamsT<T> cams, gs_batch batch, ProjT<T> proj, T* __restrict__ v2d, GradsT<T> dg,
    double* __restrict__ partial, bool clear) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ SlotCamT<T> sc[GS_MAX_BATCH];
  // per warp and view: the warp's six pose-tangent sums (FP32 in the FP32
  // path: the FP64 pipe is a small fraction of the FP32 rate; one
  // conversion per block)
  __shared__ T s_tan[kProjThreads / 32][GS_MAX_BATCH * 6];
  // dynamic: coefficients and their gradient accumulators, one padded
  // column per thread
  extern __shared__ __align__(16) unsigned char s_dyn_raw[];
  T* s_dyn = reinterpret_cast<T*>(s_dyn_raw);
  T (*s_sh)[kProjThreads + 1] = reinterpret_cast<T (*)[kProjThreads + 1]>(s_dyn);
  T (*s_vsh)[kProjThreads + 1] = reinterpret_cast<T (*)[kProjThreads + 1]>(s_dyn + K * 3 * (kProjThreads + 1));
  for (int i = threadIdx.x; i < (kProjThreads / 32) * GS_MAX_BATCH * 6; i += blockDim.x) (&s_tan[0][0])[i] = T(0);
  const int N = g.n;
  const int j0 = blockIdx.x * kProjThreads;
  const int n_local = min(kProjThreads, N - j0);
  const int j = j0 + threadIdx.x;
  const bool active = j < N;
  // the parameters and the first view's record are loaded together with
  // the SH block, before the barrier
  GeoRaw<T> raw;
  T nrec[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) nrec[i] = T(0);
  if (active) {
    raw = load_geo_raw(g, j);
    load_rec9(v2d, (size_t)j, nrec);
  }
  load_slot_cams(cams, batch, sc);
  load_sh_block<T, K * 3>(g.sh, j0, n_local, s_sh);
#pragma unroll
  for (int i = 0; i < K * 3; ++i) s_vsh[i][threadIdx.x] = T(0);
  __syncthreads();
  GaussGeo<T> G;
  if (active) G = make_geo(raw);
  T vmu[3] = {T(0), T(0), T(0)};
  T GM[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) GM[i] = T(0);
  // dL/d log-scale, summed over the views in the eigenframe of each view's
  // 2-D covariance (see below)
  T gls_eig[3] = {T(0), T(0), T(0)};
  T vol = T(0);
  bool any = false;

  // Screen-space gradients of invisible records are zero (the compositing
  // backward zeroes all records first), so every view's record can be read
  // unconditionally; the next view's is loaded while this one is processed.
  for (int b = 0; b < batch.B; ++b) {
    T tan[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T cur[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) cur[i] = nrec[i];
    if (active && b + 1 < batch.B) load_rec9(v2d, (size_t)(b + 1) * N + j, nrec);
    // record b has been read (its load was issued a view earlier), so the
    // store does not wait on it; a store right behind the load of the same
    // address would hold up the prefetch
    if (clear && active) clear_rec(v2d, (size_t)b * N + j);
    bool nz = false;
#pragma unroll
    for (int i = 0; i < 9; ++i) nz = nz || (cur[i] != T(0));
    const bool live = active && nz;
    if (live) {
      any = true;
      const SlotCamT<T>& c = sc[b];
      T vcol[3] = {cur[6], cur[7], cur[8]};
      // --- colour: SH and view direction, before the projection's
      // geometry, so that their registers are free again by then -------
      struct {
        T dir[3], dnorm;
      } V;
      {
        const T d0 = G.mu[0] - c.campos[0], d1 = G.mu[1] - c.campos[1], d2 = G.mu[2] - c.campos[2];
        V.dnorm = gsqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const T idn0 = T(1) / V.dnorm;
        V.dir[0] = d0 * idn0;
        V.dir[1] = d1 * idn0;
        V.dir[2] = d2 * idn0;
      }
      T Y[K];
      sh_basis<T>(DEG, V.dir[0], V.dir[1], V.dir[2], Y);
      T wk[K];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        T raw = T(0.5);
#pragma unroll
        for (int k = 0; k < K; ++k) raw += s_sh[3 * k + ch][threadIdx.x] * Y[k];
        if (raw < T(0)) vcol[ch] = T(0);
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T s0 = s_sh[3 * k][threadIdx.x], s1 = s_sh[3 * k + 1][threadIdx.x],
                s2 = s_sh[3 * k + 2][threadIdx.x];
        wk[k] = s0 * vcol[0] + s1 * vcol[1] + s2 * vcol[2];
        s_vsh[3 * k][threadIdx.x] += Y[k] * vcol[0];
        s_vsh[3 * k + 1][threadIdx.x] += Y[k] * vcol[1];
        s_vsh[3 * k + 2][threadIdx.x] += Y[k] * vcol[2];
      }
      T vdir[3] = {T(0), T(0), T(0)};
      sh_basis_grad_dot<T>(DEG, V.dir[0], V.dir[1], V.dir[2], wk, vdir);
      const T dd = vdir[0] * V.dir[0] + vdir[1] * V.dir[1] + vdir[2] * V.dir[2];
      const T idn = T(1) / V.dnorm;
      T vdv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        vdv[i] = (vdir[i] - dd * V.dir[i]) * idn;
        vmu[i] += vdv[i];
      }
      // v_campos = -vdv; its pose effect: g_rho += -R v_campos = R vdv
      // --- the projection's geometry --------------------------------------
      ViewGeo<T> VG;
      view_geo(G, c, cams.near_plane, cams.far_plane, VG);
      const ViewGeo<T>& V2 = VG;
      const T v_mx = cur[0], v_my = cur[1], v_a = cur[2], v_b = cur[3];
      const T v_c = cur[4], v_o = cur[5];
      // --- opacity -------------------------------------------------------
      vol += v_o;
      // --- conic -> 2-D covariance: G_S2 = -Q G_Q Q -----------------------
      const T a = V2.conic[0], bq = V2.conic[1], cq = V2.conic[2];
      const T hb = T(0.5) * v_b;
      const T X00 = v_a * a + hb * bq, X01 = v_a * bq + hb * cq;
      const T X10 = hb * a + v_c * bq, X11 = hb * bq + v_c * cq;
      const T gxx = -(a * X00 + bq * X10);
      const T gxy = -(a * X01 + bq * X11);
      const T gyy = -(bq * X01 + cq * X11);
      // --- log-scale gradient in the eigenframe of S2 ----------------------
      // d L / d log s_c = 2 B_c^T G_S2 B_c with B_c = J Mc e_c (the 2-D image
      // of scaled axis c).  Written in x, y, G_S2 = -Q G_Q Q is dominated by
      // its short-axis component, and the long-axis one -- which carries
      // the long axis' scale gradient -- drowns in its FP32 rounding for
      // elongated splats.  In the eigenframe (lambda_1 >= lambda_2, unit
      // e_1, e_2) each component is formed on its own:
      //   G'_ij = e_i^T G_Q e_j,  G_S2'_ij = -G'_ij / (lambda_i lambda_j),
      //   d L / d log s_c = 2 sum_ij G_S2'_ij (e_i . B_c)(e_j . B_c),
      // with lambda_1 a sum of non-negative terms, 1 / lambda_2 =
      // lambda_1 / det and e_1 from the branch without cancellation.
      {
        const T xx = V2.S2[0], xy = V2.S2[1], yy = V2.S2[2];
        const T h = T(0.5) * (xx - yy);
        const T rr = gsqrt(h * h + xy * xy);
        const T l1 = T(0.5) * (xx + yy) + rr;
        const T il1 = T(1) / l1, il2 = l1 * V2.idet;   // 1/lambda_2 = lambda_1 / det
        T e1x = h >= T(0) ? h + rr : xy, e1y = h >= T(0) ? xy : rr - h;
        const T n2 = e1x * e1x + e1y * e1y;
        if (n2 > T(0)) {
          const T inv = grsqrt(n2);
          e1x *= inv;
          e1y *= inv;
        } else {  // isotropic: any frame
          e1x = T(1);
          e1y = T(0);
        }
        const T e2x = -e1y, e2y = e1x;
        const T G11 = v_a * e1x * e1x + v_b * e1x * e1y + v_c * e1y * e1y;
        const T G22 = v_a * e2x * e2x + v_b * e2x * e2y + v_c * e2y * e2y;
        const T G12 = v_a * e1x * e2x + hb * (e1x * e2y + e1y * e2x) + v_c * e1y * e2y;
        const T S11 = -G11 * il1 * il1, S22 = -G22 * il2 * il2, S12 = -G12 * il1 * il2;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T Bx = V2.j00 * V2.Mc[k] + V2.j02 * V2.Mc[6 + k];
          const T By = V2.j11 * V2.Mc[3 + k] + V2.j12 * V2.Mc[6 + k];
          const T b1 = e1x * Bx + e1y * By, b2 = e2x * Bx + e2y * By;
          gls_eig[k] += T(2) * (S11 * b1 * b1 + T(2) * S12 * b1 * b2 + S22 * b2 * b2);
        }
      }
      // --- S2 = J Sc J^T: H = G_S2 J, G_Sc = J^T H, G_J = 2 H Sc ----------
      const T H00 = gxx * V2.j00, H01 = gxy * V2.j11, H02 = gxx * V2.j02 + gxy * V2.j12;
      const T H10 = gxy * V2.j00, H11 = gyy * V2.j11, H12 = gxy * V2.j02 + gyy * V2.j12;
      T GSc[9];
      GSc[0] = V2.j00 * H00; GSc[1] = V2.j00 * H01; GSc[2] = V2.j00 * H02;
      GSc[3] = V2.j11 * H10; GSc[4] = V2.j11 * H11; GSc[5] = V2.j11 * H12;
      GSc[6] = V2.j02 * H00 + V2.j12 * H10;
      GSc[7] = V2.j02 * H01 + V2.j12 * H11;
      GSc[8] = V2.j02 * H02 + V2.j12 * H12;
      // symmetrise (exact symmetry is lost only to rounding)
      {
        const T s01 = T(0.5) * (GSc[1] + GSc[3]);
        const T s02 = T(0.5) * (GSc[2] + GSc[6]);
        const T s12 = T(0.5) * (GSc[5] + GSc[7]);
        GSc[1] = GSc[3] = s01;
        GSc[2] = GSc[6] = s02;
        GSc[5] = GSc[7] = s12;
      }
      const T* S = V2.Sc;
      // full symmetric Sc
      const T Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
      // G_J entries used: (0,0), (0,2), (1,1), (1,2)
      const T GJ00 = T(2) * (H00 * Sf[0] + H01 * Sf[3] + H02 * Sf[6]);
      const T GJ02 = T(2) * (H00 * Sf[2] + H01 * Sf[5] + H02 * Sf[8]);
      const T GJ11 = T(2) * (H10 * Sf[1] + H11 * Sf[4] + H12 * Sf[7]);
      const T GJ12 = T(2) * (H10 * Sf[2] + H11 * Sf[5] + H12 * Sf[8]);
      // --- Sc = Mc Mc^T, Mc = W M:  G_Mc = 2 G_Sc Mc; G_M += W^T G_Mc ---
      T GMc[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          GMc[3 * r + k] = T(2) * (GSc[3 * r] * V2.Mc[k] + GSc[3 * r + 1] * V2.Mc[3 + k] +
                                  GSc[3 * r + 2] * V2.Mc[6 + k]);
      const T* W = c.R;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          GM[3 * r + k] += W[r] * GMc[k] + W[3 + r] * GMc[3 + k] + W[6 + r] * GMc[6 + k];
      // pose, rotation through the covariance: g_phi += 2 vee(G_Sc Sc)
      {
        T B[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int k = 0; k < 3; ++k)
            B[3 * r + k] = GSc[3 * r] * Sf[k] + GSc[3 * r + 1] * Sf[3 + k] + GSc[3 * r + 2] * Sf[6 + k];
        tan[3] += T(2) * (B[7] - B[5]);
        tan[4] += T(2) * (B[2] - B[6]);
        tan[5] += T(2) * (B[3] - B[1]);
      }
      // --- J(x_c) and mean2d -> v_xc ------------------------------------
      const T z = V2.xc[2];
      const T iz = T(1) / z, iz2 = iz * iz;
      T vxc[3];
      const T dJ02dx = V2.clx ? T(0) : -c.fx * iz2;
      const T dJ12dy = V2.cly ? T(0) : -c.fy * iz2;
      const T dJ02dz = c.fx * V2.tx * iz2 + (V2.clx ? T(0) : c.fx * V2.xc[0] * iz2 * iz);
      const T dJ12dz = c.fy * V2.ty * iz2 + (V2.cly ? T(0) : c.fy * V2.xc[1] * iz2 * iz);
      vxc[0] = GJ02 * dJ02dx + v_mx * c.fx * iz;
      vxc[1] = GJ12 * dJ12dy + v_my * c.fy * iz;
      vxc[2] = -GJ00 * c.fx * iz2 - GJ11 * c.fy * iz2 + GJ02 * dJ02dz + GJ12 * dJ12dz -
               (v_mx * c.fx * V2.xc[0] + v_my * c.fy * V2.xc[1]) * iz2;
      // --- x_c = W mu + t ------------------------------------------------
#pragma unroll
      for (int i = 0; i < 3; ++i) vmu[i] += W[i] * vxc[0] + W[3 + i] * vxc[1] + W[6 + i] * vxc[2];
      // pose: g_rho = v_xc + W vdv; g_phi += x_c x v_xc
      tan[0] = vxc[0] + W[0] * vdv[0] + W[1] * vdv[1] + W[2] * vdv[2];
      tan[1] = vxc[1] + W[3] * vdv[0] + W[4] * vdv[1] + W[5] * vdv[2];
      tan[2] = vxc[2] + W[6] * vdv[0] + W[7] * vdv[1] + W[8] * vdv[2];
      tan[3] += V2.xc[1] * vxc[2] - V2.xc[2] * vxc[1];
      tan[4] += V2.xc[2] * vxc[0] - V2.xc[0] * vxc[2];
      tan[5] += V2.xc[0] * vxc[1] - V2.xc[1] * vxc[0];
    }
    // warp reduce the 6 tangent values into the warp's own slots
    const unsigned any_live = __ballot_sync(0xffffffffu, live);
    if (any_live) {
      const int lane = threadIdx.x & 31;
      T mine = T(0);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        T v = tan[i];
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
    T* gls = dg.log_scale + 3 * (size_t)j;
    T* gqp = dg.quat + 4 * (size_t)j;
    T* gm = dg.mean + 3 * (size_t)j;
    T acc_ls[3], acc_mu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc_ls[k] = gls[k];
      acc_mu[k] = gm[k];
    }
    Quat4<T> cq = load_quat(dg.quat, j);
    T acc_o = dg.opacity_logit[j];
    // --- M = R diag(s): G_R = G_M diag(s); the scale gradient was summed in
    // each view's eigenframe
    T GR[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) GR[3 * r + k] = GM[3 * r + k] * G.s[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) gls[k] = acc_ls[k] + gls_eig[k];
    const T w = G.qn[0], x = G.qn[1], y = G.qn[2], zq = G.qn[3];
    T vq[4];
    vq[0] = -T(2) * zq * GR[1] + T(2) * y * GR[2] + T(2) * zq * GR[3] - T(2) * x * GR[5] -
            T(2) * y * GR[6] + T(2) * x * GR[7];
    vq[1] = T(2) * y * GR[1] + T(2) * zq * GR[2] + T(2) * y * GR[3] - T(4) * x * GR[4] -
            2.f * w * GR[5] + T(2) * zq * GR[6] + T(2) * w * GR[7] - T(4) * x * GR[8];
    vq[2] = -T(4) * y * GR[0] + T(2) * x * GR[1] + T(2) * w * GR[2] + T(2) * x * GR[3] +
            2.f * zq * GR[5] - T(2) * w * GR[6] + T(2) * zq * GR[7] - T(4) * y * GR[8];
    vq[3] = -T(4) * zq * GR[0] - T(2) * w * GR[1] + T(2) * x * GR[2] + T(2) * w * GR[3] -
            4.f * zq * GR[4] + T(2) * y * GR[5] + T(2) * x * GR[6] + T(2) * y * GR[7];
    const T dq = vq[0] * w + vq[1] * x + vq[2] * y + vq[3] * zq;
    cq.x += (vq[0] - dq * w) * G.qinv;
    cq.y += (vq[1] - dq * x) * G.qinv;
    cq.z += (vq[2] - dq * y) * G.qinv;
    cq.w += (vq[3] - dq * zq) * G.qinv;
    store_quat(gqp, cq);
#pragma unroll
    for (int i = 0; i < 3; ++i) gm[i] = acc_mu[i] + vmu[i];
    dg.opacity_logit[j] = acc_o + vol * G.o * (T(1) - G.o);
  }
  // SH gradients: through shared memory, then one coalesced read-modify-write
  // of the block's contiguous slice of dg.sh
  __syncthreads();
  add_sh_block<T, K * 3>(dg.sh + (size_t)j0 * K * 3, n_local, s_vsh);
  __syncthreads();
  for (int i = threadIdx.x; i < batch.B * 6; i += blockDim.x) {
    T t = T(0);
#pragma unroll
    for (int w = 0; w < kProjThreads / 32; ++w) t += s_tan[w][i];
    partial[(size_t)blockIdx.x * batch.B * 6 + i] = (double)t;
  }
}

}  // namespace

namespace {

template <typename T>
cudaError_t project_fwd_t(const GaussT<T>& g, const CamsT<T>& cams, const gs_batch& batch, const ProjT<T>& out,
                          int32_t* status, cudaStream_t st) {
  const int threads = kProjThreads;
  const int blocks = (g.n + threads - 1) / threads;
  if (blocks == 0) return cudaSuccess;
  switch (g.sh_degree) {
    case 0: project_fwd_kernel<T, 0><<<blocks, threads, 0, st>>>(g, cams, batch, out, status); break;
    case 1: project_fwd_kernel<T, 1><<<blocks, threads, 0, st>>>(g, cams, batch, out, status); break;
    case 2: project_fwd_kernel<T, 2><<<blocks, threads, 0, st>>>(g, cams, batch, out, status); break;
    default: project_fwd_kernel<T, 3><<<blocks, threads, 0, st>>>(g, cams, batch, out, status); break;
  }
  return cudaGetLastError();
}

template <typename T, int DEG>
cudaError_t project_bwd_deg(const GaussT<T>& g, const CamsT<T>& cams, const gs_batch& batch, const ProjT<T>& proj,
                            T* v2d, const GradsT<T>& dg, double* partial, int blocks, bool clear, cudaStream_t st) {
  constexpr size_t smem = project_bwd_smem<T, DEG>();
  // the opt-in for more than 48 KB of shared memory, once per device
  static bool configured[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    e = cudaFuncSetAttribute(project_bwd_kernel<T, DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  project_bwd_kernel<T, DEG><<<blocks, kProjThreads, smem, st>>>(g, cams, batch, proj, v2d, dg, partial, clear);
  return cudaGetLastError();
}

template <typename T>
cudaError_t project_bwd_t(const GaussT<T>& g, const CamsT<T>& cams, const gs_batch& batch, const ProjT<T>& proj,
                          T* v2d, const GradsT<T>& dg, double* partial, double* g_pose_tangent, bool clear,
                          cudaStream_t st) {
  const int blocks = project_bwd_blocks(g.n);
  if (blocks == 0) return cudaSuccess;
  cudaError_t e;
  switch (g.sh_degree) {
    case 0: e = project_bwd_deg<T, 0>(g, cams, batch, proj, v2d, dg, partial, blocks, clear, st); break;
    case 1: e = project_bwd_deg<T, 1>(g, cams, batch, proj, v2d, dg, partial, blocks, clear, st); break;
    case 2: e = project_bwd_deg<T, 2>(g, cams, batch, proj, v2d, dg, partial, blocks, clear, st); break;
    default: e = project_bwd_deg<T, 3>(g, cams, batch, proj, v2d, dg, partial, blocks, clear, st); break;
  }
  if (e != cudaSuccess) return e;
  return launch_pose_partials_finalize(partial, blocks, batch, cams.n_cams, g_pose_tangent, st);
}

}  // namespace

int project_bwd_blocks(int n) { return (n + kProjThreads - 1) / kProjThreads; }

cudaError_t launch_project_fwd(const gs_gaussians& g, const gs_cameras& cams, const gs_batch& batch,
                               const gs_projected& out, int32_t* status, cudaStream_t st) {
  return project_fwd_t<float>(view_of(g), view_of(cams), batch, view_of(out), status, st);
}

cudaError_t launch_project_fwd_f64(const gs_gaussians_f64& g, const gs_cameras_f64& cams, const gs_batch& batch,
                                   const gs_projected_f64& out, int32_t* status, cudaStream_t st) {
  return project_fwd_t<double>(view_of(g), view_of(cams), batch, view_of(out), status, st);
}

cudaError_t launch_project_bwd(const gs_gaussians& g, const gs_cameras& cams, const gs_batch& batch,
                               const gs_projected& proj, float* v2d, const gs_gaussian_grads& dg,
                               double* partial, double* g_pose_tangent, bool clear_records, cudaStream_t st) {
  return project_bwd_t<float>(view_of(g), view_of(cams), batch, view_of(proj), v2d, view_of(dg), partial,
                              g_pose_tangent, clear_records, st);
}

cudaError_t launch_project_bwd_f64(const gs_gaussians_f64& g, const gs_cameras_f64& cams, const gs_batch& batch,
                                   const gs_projected_f64& proj, const double* v2d, const gs_gaussian_grads_f64& dg,
                                   double* partial, double* g_pose_tangent, cudaStream_t st) {
  return project_bwd_t<double>(view_of(g), view_of(cams), batch, view_of(proj), const_cast<double*>(v2d),
                               view_of(dg), partial, g_pose_tangent, false, st);
}

}  // namespace gs
