// Pose composition and optimiser steps:
//  - pose_se3_update: T_i = Exp(xi_i) T_i^(0) (Algorithm 1, "Apply pose
//    adjustment"), the SE(3) gradient map g_xi = Jl(xi)^T g_tangent with the
//    closed-form left Jacobian of SE(3) (Barfoot, State Estimation for
//    Robotics), and an Adam step on xi (Sec. 3.3: Adam, lr 1e-5).  One
//    thread per camera; FP32 except for the series coefficients (a
//    double instantiation serves the FP64 path).
//  - Adam on parameter arrays (Algorithm 1, "Update Gaussians" / "Update
//    track points"), elementwise and HBM-bound.
//  - the fixed-order sum of per-block pose partials used by the projection
//    backward and the track term.
#include "gs_internal.h"

namespace gs {

namespace {

template <typename T>
__device__ inline void skew(const T* w, T* S) {
  S[0] = T(0);  S[1] = -w[2]; S[2] = w[1];
  S[3] = w[2];  S[4] = T(0);  S[5] = -w[0];
  S[6] = -w[1]; S[7] = w[0];  S[8] = T(0);
}

template <typename T>
__device__ inline void mm3(const T* A, const T* B, T* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

// Scalar coefficients of Exp and of the SE(3) left Jacobian for angle th:
// A = sin th / th, B = (1 - cos th) / th^2, C = (th - sin th) / th^3 and the
// Q-block coefficients c2 = (th^2 + 2 cos th - 2) / (2 th^4),
// c3 = (2 th - 3 sin th + th cos th) / (2 th^5) (c1 = C).  They cancel badly
// in single precision, so they alone are formed in double (one sincos);
// Taylor series near 0.
template <typename T>
struct Se3Coef {
  T A, B, C, c2, c3;
};

template <typename T>
__device__ inline Se3Coef<T> se3_coef(double th) {
  Se3Coef<T> k;
  const double t2 = th * th;
  if (th < 1e-3) {
    k.A = (T)(1.0 - t2 / 6.0 + t2 * t2 / 120.0);
    k.B = (T)(0.5 - t2 / 24.0 + t2 * t2 / 720.0);
    k.C = (T)(1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0);
    k.c2 = (T)(1.0 / 24.0 - t2 / 720.0 + t2 * t2 / 40320.0);
    k.c3 = (T)(1.0 / 120.0 - t2 / 2520.0);
  } else {
    double s, c;
    sincos(th, &s, &c);
    k.A = (T)(s / th);
    k.B = (T)((1.0 - c) / t2);
    k.C = (T)((th - s) / (t2 * th));
    k.c2 = (T)((t2 + 2.0 * c - 2.0) / (2.0 * t2 * t2));
    k.c3 = (T)((2.0 * th - 3.0 * s + th * c) / (2.0 * t2 * t2 * th));
  }
  return k;
}

__device__ inline float gexp2(float x) { return exp2f(x); }
__device__ inline double gexp2(double x) { return exp2(x); }
__device__ inline float glog2(float x) { return log2f(x); }
__device__ inline double glog2(double x) { return log2(x); }

template <typename T>
__global__ void pose_update_kernel(int V, const T* __restrict__ T0, T* __restrict__ xi,
                                   const double* __restrict__ g_tangent, T* __restrict__ g_xi,
                                   T* __restrict__ m, T* __restrict__ v, int use_adam,
                                   T lr, T beta1, T beta2, T eps,
                                   const int32_t* __restrict__ step, T* __restrict__ Rt_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  T x[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) x[c] = xi[6 * i + c];
  const T* rho = x;
  const T* phi = x + 3;
  const double th = sqrt((double)phi[0] * phi[0] + (double)phi[1] * phi[1] + (double)phi[2] * phi[2]);
  Se3Coef<T> k = se3_coef<T>(th);
  T P[9], Rh[9], P2[9];
  skew(phi, P);
  skew(rho, Rh);
  mm3(P, P, P2);
  T Jl[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) Jl[e] = ((e % 4) == 0 ? T(1) : T(0)) + k.B * P[e] + k.C * P2[e];
  T PR[9], RP[9], PRP[9], PPR[9], RPP[9], PRPP[9], PPRP[9], Q[9];
  mm3(P, Rh, PR);
  mm3(Rh, P, RP);
  mm3(PR, P, PRP);
  mm3(P, PR, PPR);
  mm3(RP, P, RPP);
  mm3(PRP, P, PRPP);
  mm3(P, PRP, PPRP);
#pragma unroll
  for (int e = 0; e < 9; ++e)
    Q[e] = T(0.5) * Rh[e] + k.C * (PR[e] + RP[e] + PRP[e]) + k.c2 * (PPR[e] + RPP[e] - T(3) * PRP[e]) +
           k.c3 * (PRPP[e] + PPRP[e]);
  // g_xi = Jl^T g with Jl = [[Jl, Q], [0, Jl]]
  const double* gd = g_tangent + 6 * i;
  T g[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) g[c] = (T)gd[c];
  T gx[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gx[c] = Jl[c] * g[0] + Jl[3 + c] * g[1] + Jl[6 + c] * g[2];
    gx[3 + c] = Q[c] * g[0] + Q[3 + c] * g[1] + Q[6 + c] * g[2] + Jl[c] * g[3] + Jl[3 + c] * g[4] +
                Jl[6 + c] * g[5];
  }
  if (g_xi)
#pragma unroll
    for (int c = 0; c < 6; ++c) g_xi[6 * i + c] = gx[c];
  if (use_adam) {
    const T t = (T)*step;
    const T bc1 = T(1) - gexp2(t * glog2(beta1));
    const T bc2 = T(1) - gexp2(t * glog2(beta2));
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const T mm = beta1 * m[6 * i + c] + (T(1) - beta1) * gx[c];
      const T vv = beta2 * v[6 * i + c] + (T(1) - beta2) * gx[c] * gx[c];
      m[6 * i + c] = mm;
      v[6 * i + c] = vv;
      x[c] -= lr * (mm / bc1) / (gsqrt(vv / bc2) + eps);
      xi[6 * i + c] = x[c];
    }
    const double th2 = sqrt((double)x[3] * x[3] + (double)x[4] * x[4] + (double)x[5] * x[5]);
    k = se3_coef<T>(th2);
    skew(x + 3, P);
    mm3(P, P, P2);
  }
  // Rt_out = Exp(xi) T0
  T ER[9], EV[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const T I = (e % 4) == 0 ? T(1) : T(0);
    ER[e] = I + k.A * P[e] + k.B * P2[e];
    EV[e] = I + k.B * P[e] + k.C * P2[e];
  }
  T Et[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) Et[r] = EV[3 * r] * x[0] + EV[3 * r + 1] * x[1] + EV[3 * r + 2] * x[2];
  const T* Tp = T0 + 12 * i;
  T R0[9], t0[3];
#pragma unroll
  for (int e = 0; e < 9; ++e) R0[e] = Tp[e];
#pragma unroll
  for (int e = 0; e < 3; ++e) t0[e] = Tp[9 + e];
  T R[9];
  mm3(ER, R0, R);
  T* out = Rt_out + 12 * i;
#pragma unroll
  for (int e = 0; e < 9; ++e) out[e] = R[e];
#pragma unroll
  for (int r = 0; r < 3; ++r) out[9 + r] = ER[3 * r] * t0[0] + ER[3 * r + 1] * t0[1] + ER[3 * r + 2] * t0[2] + Et[r];
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float beta1, float beta2,
                            float eps, const int32_t* __restrict__ step) {
  const int t = *step;
  const float bc1 = 1.f - powf(beta1, (float)t);
  const float bc2 = 1.f - powf(beta2, (float)t);
  const float a = lr / bc1;
  const float rb2 = 1.f / bc2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= a * mi / (sqrtf(vi * rb2) + eps);
  }
}

// Several Adam groups in one launch: the index space is cut into chunks of
// kAdamChunk elements, chunk c belonging to the group whose chunk range holds
// it; 16-byte aligned groups use 128-bit loads and stores.
constexpr int kAdamChunk = 4096;
constexpr int kAdamMaxGroups = 8;

struct AdamGroups {
  gs_adam_group g[kAdamMaxGroups];
  int chunk_start[kAdamMaxGroups + 1];
  int n;
};

__device__ inline void adam_elem(float& p, float g, float& m, float& v, float a, float beta1, float beta2,
                                 float rb2, float eps) {
  m = beta1 * m + (1.f - beta1) * g;
  v = beta2 * v + (1.f - beta2) * g * g;
  p -= a * m / (sqrtf(v * rb2) + eps);
}

__global__ void __launch_bounds__(256) adam_groups_kernel(AdamGroups G, float beta1, float beta2, float eps,
                                                          const int32_t* __restrict__ step) {
  const int t = *step;
  const float bc1 = 1.f - powf(beta1, (float)t);
  const float rb2 = 1.f / (1.f - powf(beta2, (float)t));
  const int n_chunks = G.chunk_start[G.n];
  for (int c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    int gi = 0;
    while (c >= G.chunk_start[gi + 1]) ++gi;
    const gs_adam_group A = G.g[gi];
    const int64_t lo = (int64_t)(c - G.chunk_start[gi]) * kAdamChunk;
    const int64_t hi = min(lo + (int64_t)kAdamChunk, A.n);
    const float a = A.lr / bc1;
    const bool vec = (((uintptr_t)A.p | (uintptr_t)A.g | (uintptr_t)A.m | (uintptr_t)A.v) & 15) == 0;
    if (vec) {
      const int64_t hi4 = lo + ((hi - lo) & ~(int64_t)3);
      // two float4 of each stream per thread in flight: all eight loads
      // are issued before the first store (the streams may not alias one
      // another, which the compiler cannot know)
      const int64_t step4 = 4 * (int64_t)blockDim.x;
      for (int64_t i = lo + 4 * threadIdx.x; i < hi4; i += 2 * step4) {
        const int64_t j = i + step4;
        const bool two = j < hi4;
        float4 p0 = *reinterpret_cast<float4*>(A.p + i), p1;
        const float4 g0 = *reinterpret_cast<const float4*>(A.g + i);
        float4 m0 = *reinterpret_cast<float4*>(A.m + i), m1;
        float4 v0 = *reinterpret_cast<float4*>(A.v + i), v1;
        float4 g1;
        if (two) {
          p1 = *reinterpret_cast<float4*>(A.p + j);
          g1 = *reinterpret_cast<const float4*>(A.g + j);
          m1 = *reinterpret_cast<float4*>(A.m + j);
          v1 = *reinterpret_cast<float4*>(A.v + j);
        }
        adam_elem(p0.x, g0.x, m0.x, v0.x, a, beta1, beta2, rb2, eps);
        adam_elem(p0.y, g0.y, m0.y, v0.y, a, beta1, beta2, rb2, eps);
        adam_elem(p0.z, g0.z, m0.z, v0.z, a, beta1, beta2, rb2, eps);
        adam_elem(p0.w, g0.w, m0.w, v0.w, a, beta1, beta2, rb2, eps);
        *reinterpret_cast<float4*>(A.p + i) = p0;
        *reinterpret_cast<float4*>(A.m + i) = m0;
        *reinterpret_cast<float4*>(A.v + i) = v0;
        if (two) {
          adam_elem(p1.x, g1.x, m1.x, v1.x, a, beta1, beta2, rb2, eps);
          adam_elem(p1.y, g1.y, m1.y, v1.y, a, beta1, beta2, rb2, eps);
          adam_elem(p1.z, g1.z, m1.z, v1.z, a, beta1, beta2, rb2, eps);
          adam_elem(p1.w, g1.w, m1.w, v1.w, a, beta1, beta2, rb2, eps);
          *reinterpret_cast<float4*>(A.p + j) = p1;
          *reinterpret_cast<float4*>(A.m + j) = m1;
          *reinterpret_cast<float4*>(A.v + j) = v1;
        }
      }
      for (int64_t i = hi4 + threadIdx.x; i < hi; i += blockDim.x)
        adam_elem(A.p[i], A.g[i], A.m[i], A.v[i], a, beta1, beta2, rb2, eps);
    } else {
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        adam_elem(A.p[i], A.g[i], A.m[i], A.v[i], a, beta1, beta2, rb2, eps);
    }
  }
}

__global__ void step_advance_kernel(int32_t* step) { *step += 1; }

// blockIdx.y = slot; the slot's pixels are copied with a grid-stride loop
// over its floats.
__global__ void __launch_bounds__(256) gather_view_pixels_kernel(const float* __restrict__ src,
                                                                 const int64_t* __restrict__ src_px_offset,
                                                                 gs_cameras cams, gs_batch batch, int channels,
                                                                 float* __restrict__ dst) {
  const int b = blockIdx.y;
  const int v = slot_view(cams, batch, b);
  const int64_t n_dst = (batch.px_offset[b + 1] - batch.px_offset[b]) * channels;
  const int64_t n_src = (src_px_offset[v + 1] - src_px_offset[v]) * channels;
  const int64_t n = n_dst < n_src ? n_dst : n_src;
  const float* s = src + src_px_offset[v] * channels;
  float* d = dst + batch.px_offset[b] * channels;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

// Per-slot pixel and tile offsets of a batch from its view ids and the
// cameras' sizes (one thread: B <= GS_MAX_BATCH slots).  The batch's
// n_pixels / n_tiles are the capacity of its buffers: the first slot that
// would pass either, and every slot after it, gets no pixels and no tiles
// (GS_FLAG_CAPACITY), so no kernel can index past the buffers.
__global__ void batch_layout_kernel(gs_cameras cams, gs_batch batch, int64_t* __restrict__ px_offset,
                                    int32_t* __restrict__ tile_offset, int32_t* status) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const long long T = batch.tile;
  long long px = 0, tl = 0;
  bool full = false;
  px_offset[0] = 0;
  tile_offset[0] = 0;
  for (int b = 0; b < batch.B; ++b) {
    const int v = slot_view(cams, batch, b);
    const long long W = max(cams.wh[2 * v], 0), H = max(cams.wh[2 * v + 1], 0);
    const long long np = W * H, nt = ((W + T - 1) / T) * ((H + T - 1) / T);
    if (!full && px + np <= batch.n_pixels && tl + nt <= (long long)batch.n_tiles) {
      px += np;
      tl += nt;
    } else if (!full) {
      full = true;
      set_flag(status, GS_FLAG_CAPACITY);
    }
    px_offset[b + 1] = px;
    tile_offset[b + 1] = (int32_t)tl;
  }
}

// g_pose_tangent[v] += the partials of every slot rendering camera v, in a
// fixed order.  A camera may fill several slots of a batch: the block of its
// first slot sums them all (slot order, then block order) and the blocks of
// its other slots do nothing, so no two blocks write one camera's entries.
constexpr int kFinThreads = 1024;
__global__ void __launch_bounds__(kFinThreads)
    pose_partial_finalize_kernel(const double* __restrict__ partial, int n_blocks, gs_batch batch, int n_cams,
                                 double* g_pose_tangent) {
  const int b = blockIdx.x / 6, i = blockIdx.x % 6;
  const int v = batch.views[b];
  for (int b2 = 0; b2 < b; ++b2)
    if (batch.views[b2] == v) return;  // block-uniform: an earlier slot owns camera v
  __shared__ double red[kFinThreads];
  // four interleaved running sums per thread (rows k, k + T, k + 2T, k + 3T
  // of each group of 4T), then pairwise: a fixed order with short
  // dependent chains (FP64 adds are slow to retire on this part)
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b2 = b; b2 < batch.B; ++b2) {
    if (batch.views[b2] != v) continue;
    for (int k0 = 0; k0 < n_blocks; k0 += 4 * kFinThreads) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q * kFinThreads + (int)threadIdx.x;
        if (k < n_blocks) acc[q] += partial[(size_t)k * batch.B * 6 + 6 * b2 + i];
      }
    }
  }
  const double s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0 && (unsigned)v < (unsigned)n_cams) g_pose_tangent[6 * v + i] += red[0];
}

}  // namespace

cudaError_t launch_pose_partials_finalize(const double* partial, int n_blocks, const gs_batch& batch,
                                          int n_cams, double* g_pose_tangent, cudaStream_t st) {
  pose_partial_finalize_kernel<<<batch.B * 6, kFinThreads, 0, st>>>(partial, n_blocks, batch, n_cams,
                                                                    g_pose_tangent);
  return cudaGetLastError();
}

namespace {
template <typename T>
cudaError_t pose_update_t(int V, const T* T0, T* xi, const double* g_tangent, T* g_xi, T* m, T* v,
                          const gs_adam* hp, T* Rt_out, cudaStream_t st) {
  if (V == 0) return cudaSuccess;
  const int threads = 128;
  pose_update_kernel<T><<<(V + threads - 1) / threads, threads, 0, st>>>(
      V, T0, xi, g_tangent, g_xi, m, v, hp ? 1 : 0, hp ? (T)hp->lr : T(0), hp ? (T)hp->beta1 : T(0),
      hp ? (T)hp->beta2 : T(0), hp ? (T)hp->eps : T(0), hp ? hp->step : nullptr, Rt_out);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_pose_update(int V, const float* T0, float* xi, const double* g_tangent, float* g_xi,
                               float* m, float* v, const gs_adam* hp, float* Rt_out, cudaStream_t st) {
  return pose_update_t<float>(V, T0, xi, g_tangent, g_xi, m, v, hp, Rt_out, st);
}

cudaError_t launch_pose_update_f64(int V, const double* T0, double* xi, const double* g_tangent, double* g_xi,
                                   double* m, double* v, const gs_adam* hp, double* Rt_out, cudaStream_t st) {
  return pose_update_t<double>(V, T0, xi, g_tangent, g_xi, m, v, hp, Rt_out, st);
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, const gs_adam& hp,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t want = (n + threads - 1) / threads;
  const int blocks = (int)std::min<int64_t>(want, (int64_t)device_sm_count() * 8);
  adam_kernel<<<blocks, threads, 0, st>>>(p, g, m, v, n, hp.lr, hp.beta1, hp.beta2, hp.eps, hp.step);
  return cudaGetLastError();
}

cudaError_t launch_adam_groups(const gs_adam_group* groups, int n_groups, const gs_adam& hp, cudaStream_t st) {
  AdamGroups G;
  G.n = n_groups;
  G.chunk_start[0] = 0;
  for (int i = 0; i < n_groups; ++i) {
    G.g[i] = groups[i];
    G.chunk_start[i + 1] = G.chunk_start[i] + (int)((groups[i].n + kAdamChunk - 1) / kAdamChunk);
  }
  for (int i = n_groups; i < kAdamMaxGroups; ++i) G.chunk_start[i + 1] = G.chunk_start[n_groups];
  const int n_chunks = G.chunk_start[n_groups];
  if (n_chunks == 0) return cudaSuccess;
  const int blocks = std::min(n_chunks, device_sm_count() * 8);
  adam_groups_kernel<<<blocks, 256, 0, st>>>(G, hp.beta1, hp.beta2, hp.eps, hp.step);
  return cudaGetLastError();
}

cudaError_t launch_gather_view_pixels(const float* src, const int64_t* src_px_offset, const gs_cameras& cams,
                                      const gs_batch& batch, int channels, float* dst, cudaStream_t st) {
  if (batch.n_pixels == 0) return cudaSuccess;
  const int gx = std::max(1, std::min(4 * device_sm_count() / std::max(batch.B, 1) + 1, 1024));
  gather_view_pixels_kernel<<<dim3(gx, batch.B), 256, 0, st>>>(src, src_px_offset, cams, batch, channels, dst);
  return cudaGetLastError();
}

cudaError_t launch_batch_layout(const gs_cameras& cams, const gs_batch& batch, int64_t* px_offset,
                                int32_t* tile_offset, int32_t* status, cudaStream_t st) {
  batch_layout_kernel<<<1, 32, 0, st>>>(cams, batch, px_offset, tile_offset, status);
  return cudaGetLastError();
}

cudaError_t launch_step_advance(int32_t* step, cudaStream_t st) {
  step_advance_kernel<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

}  // namespace gs
