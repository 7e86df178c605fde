// Normal-equation blocks of one Levenberg-Marquardt iteration of the SfM
// bundle adjustment of Eq. 4 (Sec. 3.2, "Bundle Adjustment").
//
// One thread per observation o = (camera i, point k, pixel x) computes the
// residual r = pi_i(X_k) - x, the Huber weight w = rho'(|r|^2) and the
// Jacobians Jp = dr/d(rho, phi) of the left perturbation T <- Exp(d) T and
// JX = dr/dX_k.  With x_c = R X + t and P = d pi / d x_c:
//   dx_c/drho = I,  dx_c/dphi = -[x_c]_x,  dx_c/dX = R,
//   Jp = [P, -P [x_c]_x],  JX = P R.
// It writes Wo = w Jp^T JX, and adds w JX^T JX, w JX^T r to its point and
// w Jp^T Jp, w Jp^T r to its camera.  Observations are normally sorted by
// camera (view-CSR), so a warp whose valid lanes share one camera sums the
// camera's 42 values with shuffles and adds them once; otherwise each lane
// adds its own.  Double precision throughout: the sums feed a linear solve.
#include <algorithm>
#include <vector>

#include "gs_internal.h"

namespace gs {

namespace {

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// kBlocks false: the objective alone (a trial step's), nothing else written.
template <bool kBlocks>
__global__ void __launch_bounds__(256) ba_assemble_kernel(
    const float* __restrict__ X, int n_points, gs_cameras cams, const int32_t* __restrict__ obs_point,
    const int32_t* __restrict__ obs_cam, const float2* __restrict__ obs_xy, int64_t M, double delta,
    double* __restrict__ U, double* __restrict__ Vp, double* __restrict__ gc, double* __restrict__ gp,
    double* __restrict__ Wo, double* objective) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int cam = -1, pt = -1;
  bool valid = false;
  double jp[2][6], jx[2][3], r0 = 0.0, r1 = 0.0, w = 0.0, rho = 0.0;
#pragma unroll
  for (int a = 0; a < 6; ++a) jp[0][a] = jp[1][a] = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) jx[0][a] = jx[1][a] = 0.0;
  if (o < M) {
    const int i = obs_cam[o], k = obs_point[o];
    if ((unsigned)i < (unsigned)cams.n_cams && (unsigned)k < (unsigned)n_points) {
      const float* T = cams.Rt + 12 * (size_t)i;
      double R[9], t[3];
#pragma unroll
      for (int a = 0; a < 9; ++a) R[a] = T[a];
#pragma unroll
      for (int a = 0; a < 3; ++a) t[a] = T[9 + a];
      const double Xk[3] = {X[3 * (size_t)k], X[3 * (size_t)k + 1], X[3 * (size_t)k + 2]};
      double xc[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) xc[a] = R[3 * a] * Xk[0] + R[3 * a + 1] * Xk[1] + R[3 * a + 2] * Xk[2] + t[a];
      if (xc[2] > (double)cams.near_plane) {
        valid = true;
        cam = i;
        pt = k;
        const double fx = cams.K[4 * i], fy = cams.K[4 * i + 1], cx = cams.K[4 * i + 2], cy = cams.K[4 * i + 3];
        const double x = xc[0], y = xc[1], z = xc[2], iz = 1.0 / z;
        const float2 ob = obs_xy[o];
        r0 = fx * x * iz + cx - (double)ob.x;
        r1 = fy * y * iz + cy - (double)ob.y;
        const double s = r0 * r0 + r1 * r1, d2 = delta * delta;
        const double rs = sqrt(s);
        w = s <= d2 ? 1.0 : delta / rs;
        rho = s <= d2 ? s : 2.0 * delta * rs - d2;
        const double P00 = fx * iz, P02 = -fx * x * iz * iz, P11 = fy * iz, P12 = -fy * y * iz * iz;
        jp[0][0] = P00;
        jp[0][2] = P02;
        jp[1][1] = P11;
        jp[1][2] = P12;
        jp[0][3] = P02 * y;
        jp[0][4] = P00 * z - P02 * x;
        jp[0][5] = -P00 * y;
        jp[1][3] = P12 * y - P11 * z;
        jp[1][4] = -P12 * x;
        jp[1][5] = P11 * x;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          jx[0][c] = P00 * R[c] + P02 * R[6 + c];
          jx[1][c] = P11 * R[3 + c] + P12 * R[6 + c];
        }
      }
    }
    if constexpr (kBlocks) {
      double* wo = Wo + 18 * o;
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) wo[3 * a + c] = w * (jp[0][a] * jx[0][c] + jp[1][a] * jx[1][c]);
    }
  }
  if (kBlocks && valid) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        atomicAdd(&Vp[9 * (size_t)pt + 3 * a + c], w * (jx[0][a] * jx[0][c] + jx[1][a] * jx[1][c]));
      atomicAdd(&gp[3 * (size_t)pt + a], w * (jx[0][a] * r0 + jx[1][a] * r1));
    }
  }
  const unsigned vm = __ballot_sync(0xffffffffu, valid);
  if (vm != 0u) {  // warp-uniform
    const int cref = __shfl_sync(0xffffffffu, cam, __ffs(vm) - 1);
    if (!kBlocks) {
      // objective only
    } else if (__all_sync(0xffffffffu, !valid || cam == cref)) {
#pragma unroll
      for (int a = 0; a < 6; ++a) {
#pragma unroll
        for (int b = 0; b < 6; ++b) {
          const double v = warp_sum_d(w * (jp[0][a] * jp[0][b] + jp[1][a] * jp[1][b]));
          if (lane == 0) atomicAdd(&U[36 * (size_t)cref + 6 * a + b], v);
        }
        const double g = warp_sum_d(w * (jp[0][a] * r0 + jp[1][a] * r1));
        if (lane == 0) atomicAdd(&gc[6 * (size_t)cref + a], g);
      }
    } else if (valid) {
#pragma unroll
      for (int a = 0; a < 6; ++a) {
#pragma unroll
        for (int b = 0; b < 6; ++b)
          atomicAdd(&U[36 * (size_t)cam + 6 * a + b], w * (jp[0][a] * jp[0][b] + jp[1][a] * jp[1][b]));
        atomicAdd(&gc[6 * (size_t)cam + a], w * (jp[0][a] * r0 + jp[1][a] * r1));
      }
    }
    if (objective != nullptr) {
      const double tot = warp_sum_d(rho);
      if (lane == 0) atomicAdd(objective, tot);
    }
  }
}

}  // namespace

cudaError_t launch_ba_assemble(const float* X, int n_points, const gs_cameras& cams, const int32_t* obs_point,
                               const int32_t* obs_cam, const float* obs_xy, int64_t n_obs, float delta, double* U,
                               double* Vp, double* gc, double* gp, double* Wo, double* objective,
                               cudaStream_t st) {
  if (n_obs == 0) return cudaSuccess;
  const int64_t blocks = (n_obs + 255) / 256;
  if (U == nullptr)
    ba_assemble_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(X, n_points, cams, obs_point, obs_cam,
                                                                reinterpret_cast<const float2*>(obs_xy), n_obs,
                                                                (double)delta, U, Vp, gc, gp, Wo, objective);
  else
    ba_assemble_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(X, n_points, cams, obs_point, obs_cam,
                                                               reinterpret_cast<const float2*>(obs_xy), n_obs,
                                                               (double)delta, U, Vp, gc, gp, Wo, objective);
  return cudaGetLastError();
}

// The trial parameters of a step: T_i' = Exp(dc_i) T_i (left perturbation,
// translation first; computed in double, stored as float) and
// X_k' = X_k + dp_k.  Exp of d = (rho, phi): R = I + a [phi]x + b [phi]x^2,
// t = (I + b [phi]x + c [phi]x^2) rho with a = sin(th)/th,
// b = (1 - cos(th))/th^2, c = (th - sin(th))/th^3 (th = |phi|; their
// first-order limits below th = 1e-8).
namespace {

__global__ void __launch_bounds__(128) ba_apply_kernel(int V, int P, const float* __restrict__ Rt,
                                                       const float* __restrict__ X, const double* __restrict__ dc,
                                                       const double* __restrict__ dp, float* __restrict__ Rt_out,
                                                       float* __restrict__ X_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < V) {
    const double* d = dc + 6 * (size_t)t;
    const double p0 = d[3], p1 = d[4], p2 = d[5];
    const double th = sqrt(p0 * p0 + p1 * p1 + p2 * p2);
    double a, b, c;
    if (th < 1e-8) {
      a = 1.0;
      b = 0.5;
      c = 1.0 / 6.0;
    } else {
      const double s = sin(th), co = cos(th);
      a = s / th;
      b = (1.0 - co) / (th * th);
      c = (th - s) / (th * th * th);
    }
    const double Wx[9] = {0.0, -p2, p1, p2, 0.0, -p0, -p1, p0, 0.0};
    double W2[9];
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) W2[3 * r + q] = Wx[3 * r] * Wx[q] + Wx[3 * r + 1] * Wx[3 + q] + Wx[3 * r + 2] * Wx[6 + q];
    double E[9], J[9];
    for (int e = 0; e < 9; ++e) {
      const double I = (e % 4) == 0 ? 1.0 : 0.0;
      E[e] = I + a * Wx[e] + b * W2[e];
      J[e] = I + b * Wx[e] + c * W2[e];
    }
    const float* T = Rt + 12 * (size_t)t;
    double R[9], tv[3];
    for (int e = 0; e < 9; ++e) R[e] = T[e];
    for (int e = 0; e < 3; ++e) tv[e] = T[9 + e];
    float* O = Rt_out + 12 * (size_t)t;
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q)
        O[3 * r + q] = (float)(E[3 * r] * R[q] + E[3 * r + 1] * R[3 + q] + E[3 * r + 2] * R[6 + q]);
      const double jr = J[3 * r] * d[0] + J[3 * r + 1] * d[1] + J[3 * r + 2] * d[2];
      O[9 + r] = (float)(E[3 * r] * tv[0] + E[3 * r + 1] * tv[1] + E[3 * r + 2] * tv[2] + jr);
    }
  }
  if (t < P) {
    for (int e = 0; e < 3; ++e) X_out[3 * (size_t)t + e] = (float)((double)X[3 * (size_t)t + e] + dp[3 * (size_t)t + e]);
  }
}

}  // namespace

cudaError_t launch_ba_apply(int V, int P, const float* Rt, const float* X, const double* dc, const double* dp,
                            float* Rt_out, float* X_out, cudaStream_t st) {
  const int n = V > P ? V : P;
  if (n == 0) return cudaSuccess;
  ba_apply_kernel<<<(n + 127) / 128, 128, 0, st>>>(V, P, Rt, X, dc, dp, Rt_out, X_out);
  return cudaGetLastError();
}

// Elimination of the points (Schur complement) from the damped system of
// one LM iteration:
//   S = U_d - sum_k W_ik V_k^-1 W_jk^T,   rhs = -gc + sum_k W_ik V_k^-1 gp_k,
// U_d = U + lambda diag(U), V_d likewise; a camera or point block with no
// observation (all zero) becomes the identity with a zero right-hand side.
// The observations of a point come as a CSR list (point_obs_offset,
// point_obs).  The sum over pairs of observations of a point equals the
// product of the per-camera sums of W (the expression is bilinear), so
// repeated (camera, point) pairs need no merging.
namespace {

__device__ inline bool block_empty(const double* A, int n) {
  for (int a = 0; a < n; ++a)
    if (A[a] != 0.0) return false;
  return true;
}

__global__ void __launch_bounds__(64) ba_camera_init_kernel(int V, const double* __restrict__ U,
                                                            const double* __restrict__ gc, double lambda_h,
                                                            const double* __restrict__ lambda_d,
                                                            double* __restrict__ S, double* __restrict__ rhs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  const double lambda = lambda_d ? *lambda_d : lambda_h;
  const double* Ui = U + 36 * (size_t)i;
  const bool empty = block_empty(Ui, 36);
  const size_t n = 6 * (size_t)V;
  for (int a = 0; a < 6; ++a) {
    for (int b = 0; b < 6; ++b) {
      double v = empty ? (a == b ? 1.0 : 0.0) : Ui[6 * a + b];
      if (a == b) v += lambda * v;
      S[(6 * (size_t)i + a) * n + 6 * (size_t)i + b] = v;
    }
    rhs[6 * (size_t)i + a] = empty ? 0.0 : -gc[6 * (size_t)i + a];
  }
}

// The damped point block's inverse (adjugate over determinant; the block is
// symmetric positive definite after damping) and the point's right-hand side.
__device__ inline void point_block(const double* __restrict__ Vp, const double* __restrict__ gp, int k,
                                   double lambda, double* Vi, double* g) {
  const double* A = Vp + 9 * (size_t)k;
  const bool empty = block_empty(A, 9);
  double M[9];
  for (int a = 0; a < 9; ++a) M[a] = empty ? ((a % 4) == 0 ? 1.0 : 0.0) : A[a];
  M[0] += lambda * M[0];
  M[4] += lambda * M[4];
  M[8] += lambda * M[8];
  const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
  const double c10 = M[2] * M[7] - M[1] * M[8], c11 = M[0] * M[8] - M[2] * M[6], c12 = M[1] * M[6] - M[0] * M[7];
  const double c20 = M[1] * M[5] - M[2] * M[4], c21 = M[2] * M[3] - M[0] * M[5], c22 = M[0] * M[4] - M[1] * M[3];
  const double id = 1.0 / (M[0] * c00 + M[1] * c01 + M[2] * c02);
  Vi[0] = c00 * id; Vi[1] = c10 * id; Vi[2] = c20 * id;
  Vi[3] = c01 * id; Vi[4] = c11 * id; Vi[5] = c21 * id;
  Vi[6] = c02 * id; Vi[7] = c12 * id; Vi[8] = c22 * id;
  for (int a = 0; a < 3; ++a) g[a] = empty ? 0.0 : gp[3 * (size_t)k + a];
}

// The damped point blocks' inverses, one thread per point.
__global__ void __launch_bounds__(128) ba_point_vinv_kernel(int P, const double* __restrict__ Vp,
                                                            const double* __restrict__ gp, double lambda_h,
                                                            const double* __restrict__ lambda_d,
                                                            double* __restrict__ Vinv) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const double lambda = lambda_d ? *lambda_d : lambda_h;
  double Vi[9], g[3];
  point_block(Vp, gp, k, lambda, Vi, g);
  for (int a = 0; a < 9; ++a) Vinv[9 * (size_t)k + a] = Vi[a];
}

__device__ inline void point_schur_entry(int V, int P, int64_t M, int64_t p, const double* __restrict__ gp,
                                         const double* __restrict__ Vp, const double* __restrict__ Wo,
                                         const int32_t* __restrict__ obs_cam, const int64_t* __restrict__ off,
                                         const int32_t* __restrict__ point_obs, const double* __restrict__ Vinv,
                                         double* __restrict__ S, double* __restrict__ rhs) {
  // the point whose list holds p: the last k with off[k] <= p
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  const int k = lo;
  const int64_t oa = point_obs[p];
  if (oa < 0 || oa >= M) return;
  const int ca = obs_cam[oa];
  if ((unsigned)ca >= (unsigned)V) return;
  const bool empty = block_empty(Vp + 9 * (size_t)k, 9);
  double Vi[9], g[3];
  for (int e = 0; e < 9; ++e) Vi[e] = Vinv[9 * (size_t)k + e];
  for (int e = 0; e < 3; ++e) g[e] = empty ? 0.0 : gp[3 * (size_t)k + e];
  const size_t n = 6 * (size_t)V;
  const double* Wa = Wo + 18 * oa;
  double Y[18];  // W_a V^-1, 6x3
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 3; ++c)
      Y[3 * r + c] = Wa[3 * r] * Vi[c] + Wa[3 * r + 1] * Vi[3 + c] + Wa[3 * r + 2] * Vi[6 + c];
  for (int r = 0; r < 6; ++r)
    atomicAdd(&rhs[6 * (size_t)ca + r], Y[3 * r] * g[0] + Y[3 * r + 1] * g[1] + Y[3 * r + 2] * g[2]);
  for (int64_t q = off[k]; q < off[k + 1]; ++q) {
    const int64_t ob = point_obs[q];
    if (ob < 0 || ob >= M) continue;
    const int cb = obs_cam[ob];
    if ((unsigned)cb >= (unsigned)V || cb > ca) continue;
    const double* Wb = Wo + 18 * ob;
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) {
        if (cb == ca && c > r) continue;
        atomicAdd(&S[(6 * (size_t)ca + r) * n + 6 * (size_t)cb + c],
                  -(Y[3 * r] * Wb[3 * c] + Y[3 * r + 1] * Wb[3 * c + 1] + Y[3 * r + 2] * Wb[3 * c + 2]));
      }
  }
}

// One thread per entry p of the points' observation lists (observation a
// of point k): its share of rhs, and of S for every observation b of the
// same point whose camera is not after a's.  S is symmetric and the camera
// solve reads its lower triangle only, so the blocks above the diagonal are
// left out (and, within a diagonal block, the entries above its diagonal).
__global__ void __launch_bounds__(128) ba_point_schur_kernel(
    int V, int P, int64_t M, const double* __restrict__ gp, const double* __restrict__ Vp,
    const double* __restrict__ Wo, const int32_t* __restrict__ obs_cam, const int64_t* __restrict__ off,
    const int32_t* __restrict__ point_obs, const double* __restrict__ Vinv, double* __restrict__ S,
    double* __restrict__ rhs) {
  const int64_t total = off[P];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x)
    point_schur_entry(V, P, M, p, gp, Vp, Wo, obs_cam, off, point_obs, Vinv, S, rhs);
}


// --- the elimination by camera pairs ---------------------------------------
// The same sums as ba_point_schur_kernel without atomics.  A host-built plan
// lists, per camera pair (ca, cb), cb <= ca, every incidence (k, a, b): an
// ordered pair of observations a, b of point k with cameras ca, cb.  Per
// LM iteration:
//   obs_y     Y_a = W_a V_k^-1 (6x3) and Y_a g_k (6) per observation;
//   chunk     a warp per chunk of at most kPairChunk incidences of one pair:
//             sum Y_a W_b^T (6x6) and, where a = b, sum Y_a g_k, summed per
//             lane, then over the lanes in a fixed order, into 42 partials;
//   finalize  per pair and entry, the chunks' partials in chunk order,
//             subtracted from S (rhs: added, diagonal pairs only).
// Each entry of S is then formed in one fixed order: the result does not
// depend on scheduling.
constexpr int kPairValues = 42;  // 36 entries of the 6x6 block, 6 of the rhs
constexpr int kObsY = 24;        // per observation: Y (18), Y g (6)

__global__ void __launch_bounds__(128) ba_obs_y_kernel(int V, int P, int64_t M, const double* __restrict__ gp,
                                                       const double* __restrict__ Vp, const double* __restrict__ Wo,
                                                       const int32_t* __restrict__ obs_cam,
                                                       const int64_t* __restrict__ off,
                                                       const int32_t* __restrict__ point_obs,
                                                       const double* __restrict__ Vinv, double* __restrict__ Y) {
  const int64_t total = off[P];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= p) lo = mid;
      else hi = mid - 1;
    }
    const int k = lo;
    const int64_t a = point_obs[p];
    if (a < 0 || a >= M || (unsigned)obs_cam[a] >= (unsigned)V) continue;
    const bool empty = block_empty(Vp + 9 * (size_t)k, 9);
    double Vi[9], g[3];
    for (int e = 0; e < 9; ++e) Vi[e] = Vinv[9 * (size_t)k + e];
    for (int e = 0; e < 3; ++e) g[e] = empty ? 0.0 : gp[3 * (size_t)k + e];
    const double* Wa = Wo + 18 * a;
    double* y = Y + kObsY * a;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      double yr[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        yr[c] = Wa[3 * r] * Vi[c] + Wa[3 * r + 1] * Vi[3 + c] + Wa[3 * r + 2] * Vi[6 + c];
        y[3 * r + c] = yr[c];
      }
      y[18 + r] = yr[0] * g[0] + yr[1] * g[1] + yr[2] * g[2];
    }
  }
}

constexpr int kPairWarps = 4;
__global__ void __launch_bounds__(32 * kPairWarps) ba_pair_chunk_kernel(
    int n_chunks, const int32_t* __restrict__ inc, const int64_t* __restrict__ chunk_start,
    const int32_t* __restrict__ obs_cam, const double* __restrict__ Y, const double* __restrict__ Wo,
    double* __restrict__ partial) {
  __shared__ double sh[kPairWarps][kPairValues][33];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int chunk = blockIdx.x * kPairWarps + warp;
  if (chunk >= n_chunks) return;  // warp-uniform; no block-wide barrier below
  // a chunk's incidences share one camera pair: on the diagonal only the
  // block's lower triangle is needed (the finalize reads no more)
  const int64_t i0 = chunk_start[chunk];
  const bool diag = obs_cam[inc[3 * i0 + 1]] == obs_cam[inc[3 * i0 + 2]];
  double acc[kPairValues];
#pragma unroll
  for (int e = 0; e < kPairValues; ++e) acc[e] = 0.0;
  for (int64_t i = i0 + lane; i < chunk_start[chunk + 1]; i += 32) {
    const int a = inc[3 * i + 1], b = inc[3 * i + 2];
    const double* ya = Y + kObsY * (size_t)a;
    const double* wb = Wo + 18 * (size_t)b;
    double yv[18], wv[18];
#pragma unroll
    for (int e = 0; e < 18; ++e) {
      yv[e] = ya[e];
      wv[e] = wb[e];
    }
    if (diag) {
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c)
          acc[6 * r + c] += yv[3 * r] * wv[3 * c] + yv[3 * r + 1] * wv[3 * c + 1] + yv[3 * r + 2] * wv[3 * c + 2];
    } else {
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c)
          acc[6 * r + c] += yv[3 * r] * wv[3 * c] + yv[3 * r + 1] * wv[3 * c + 1] + yv[3 * r + 2] * wv[3 * c + 2];
    }
    if (a == b) {
#pragma unroll
      for (int r = 0; r < 6; ++r) acc[36 + r] += ya[18 + r];
    }
  }
#pragma unroll
  for (int e = 0; e < kPairValues; ++e) sh[warp][e][lane] = acc[e];
  __syncwarp();
  // over the lanes: four interleaved running sums (lanes l, l + 8, l + 16,
  // l + 24), then pairwise -- a fixed order with a short dependent chain
  for (int e = lane; e < kPairValues; e += 32) {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int l = 0; l < 8; ++l)
#pragma unroll
      for (int j = 0; j < 4; ++j) t[j] += sh[warp][e][l + 8 * j];
    partial[(size_t)chunk * kPairValues + e] = (t[0] + t[1]) + (t[2] + t[3]);
  }
}

__global__ void __launch_bounds__(128) ba_pair_finalize_kernel(int V, int n_pairs, const int32_t* __restrict__ pair_cams,
                                                               const int32_t* __restrict__ pair_chunks,
                                                               const double* __restrict__ partial,
                                                               double* __restrict__ S, double* __restrict__ rhs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_pairs * kPairValues) return;
  const int p = (int)(t / kPairValues), e = (int)(t % kPairValues);
  const int ca = pair_cams[2 * p], cb = pair_cams[2 * p + 1];
  if ((unsigned)ca >= (unsigned)V || (unsigned)cb >= (unsigned)V || cb > ca) return;
  double sum = 0.0;
  for (int j = pair_chunks[p]; j < pair_chunks[p + 1]; ++j) sum += partial[(size_t)j * kPairValues + e];
  const size_t n = 6 * (size_t)V;
  if (e < 36) {
    const int r = e / 6, c = e % 6;
    if (ca == cb && c > r) return;  // the diagonal block's lower triangle
    S[(6 * (size_t)ca + r) * n + 6 * (size_t)cb + c] -= sum;
  } else if (ca == cb) {
    rhs[6 * (size_t)ca + (e - 36)] += sum;
  }
}

__global__ void __launch_bounds__(128) ba_back_substitute_kernel(
    int V, int P, int64_t M, const double* __restrict__ Vinv, const double* __restrict__ Vp,
    const double* __restrict__ gp, const double* __restrict__ Wo, const int32_t* __restrict__ obs_cam,
    const int64_t* __restrict__ off, const int32_t* __restrict__ point_obs, const double* __restrict__ dc,
    double* __restrict__ dp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const bool empty = block_empty(Vp + 9 * (size_t)k, 9);
  double b[3];
  for (int a = 0; a < 3; ++a) b[a] = empty ? 0.0 : -gp[3 * (size_t)k + a];
  for (int64_t p = off[k]; p < off[k + 1]; ++p) {
    const int64_t o = point_obs[p];
    if (o < 0 || o >= M) continue;
    const int c = obs_cam[o];
    if ((unsigned)c >= (unsigned)V) continue;
    const double* W = Wo + 18 * o;
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < 6; ++r) b[a] -= W[3 * r + a] * dc[6 * (size_t)c + r];
  }
  const double* Vi = Vinv + 9 * (size_t)k;
  for (int a = 0; a < 3; ++a) dp[3 * (size_t)k + a] = Vi[3 * a] * b[0] + Vi[3 * a + 1] * b[1] + Vi[3 * a + 2] * b[2];
}

// The reduced camera system with camera 0 held fixed, S' dc' = rhs' (S' =
// S without camera 0's six rows and columns, n = 6 (V - 1) unknowns), by a
// tiled right-looking Cholesky factorization S' = L L^T in place over the
// lower triangle of S', then two triangular solves.  Tiles are kChT x kChT
// (the last row and column of tiles ragged).  For each tile column k:
//   diag   factors tile (k, k) in shared memory (one block);
//   panel  L_ik = A_ik L_kk^-T for the tiles below it (one block per tile);
//   update A_ij -= L_ik L_jk^T for k < j <= i (four blocks per tile),
// so the O(n^3 / 6) flops of the updates are spread over the SMs.  A pivot
// that is not positive (S' not positive definite) sets a marker in S[0]
// (camera 0's rows are not part of S' and free to use as scratch) that the
// later kernels read: they then do nothing, and the solve writes dc = 0
// and raises GS_FLAG_NOT_SPD.  S[1 .. n] receive the reciprocals of L's
// diagonal, which the solve uses.
constexpr int kChT = 32;

__device__ inline bool chol_failed(const double* S) { return *(volatile const double*)S != 0.0; }

__global__ void ba_chol_init_kernel(double* S) { S[0] = 0.0; }

// Tile (k, k) in shared memory, one barrier per column.  FP64 issues at
// ~2 lanes per clock per SM, one pipe per SM quarter, so a warp's FP64
// instruction occupies its quarter's pipe for many cycles and the pivots'
// serial chain must not queue behind the trailing update:
//   warp 0     lane r - 1 owns the diagonal entry (r, r): in step c it
//              subtracts l_rc^2, and lane c (owner of (c + 1, c + 1), which
//              has then had its last update) forms the next pivot's
//              reciprocal square root at once;
//   warps 1-3  the strict lower trailing triangle of step c, spread evenly
//              over their 96 threads through a shared table of the
//              triangle's (row, column) offsets.
// Column c is scaled when the tile is written back.
constexpr int kDiagThreads = 128;
constexpr int kDiagUpd = kDiagThreads - 32;

// 1 / sqrt(d) for a pivot d > 0: an FP32 estimate (relative error ~2^-22)
// refined by one step of Halley's iteration for the reciprocal square
// root, y <- y (1 + e/2 + 3e^2/8) with e = 1 - d y^2, which cubes the
// relative error (to the FP64 rounding level, ~1 ulp).  Five dependent FP64
// operations instead of a square root and a division: the pivot is on the
// factorization's serial path.  Outside the range where the FP32 estimate
// is normal, the plain form.
__device__ inline double pivot_rsqrt(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  const double y = (double)rsqrtf((float)d);
  const double e = fma(-d * y, y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}

__global__ void __launch_bounds__(kDiagThreads) ba_chol_diag_kernel(int n, size_t ld, double* __restrict__ S,
                                                                     int k) {
  __shared__ double a[kChT][kChT + 1];
  __shared__ double s_piv[kChT], s_inv[kChT];
  __shared__ uint8_t s_tri[kChT * (kChT - 1) / 2][2];  // (i, j), j < i, row by row
  __shared__ int s_bad;
  if (chol_failed(S)) return;
  double* A = S + 6 * ld + 6;
  const int r0 = k * kChT, m = min(kChT, n - r0);
  const int t = threadIdx.x;
  for (int e = t; e < kChT * kChT; e += kDiagThreads) {
    const int r = e / kChT, c = e % kChT;
    a[r][c] = (r < m && c <= r) ? A[(size_t)(r0 + r) * ld + r0 + c] : 0.0;
  }
  if (t < kChT) {  // row i of the triangle table: entries i (i - 1) / 2 + j, j < i
    for (int j = 0; j < t; ++j) {
      s_tri[t * (t - 1) / 2 + j][0] = (uint8_t)t;
      s_tri[t * (t - 1) / 2 + j][1] = (uint8_t)j;
    }
  }
  if (t == 0) s_bad = 0;
  __syncthreads();
  if (t == 0) {
    const double d = a[0][0];
    if (d > 0.0 && isfinite(d)) {
      s_piv[0] = d;
      s_inv[0] = pivot_rsqrt(d);
    } else {
      s_bad = 1;
    }
  }
  __syncthreads();
  for (int c = 0; c < m; ++c) {
    if (s_bad) break;  // block-uniform
    const double inv = s_inv[c];
    if (t < 32) {
      const int r = t + 1;  // diagonal entry (r, r)
      if (r > c && r < m) {
        const double l = a[r][c] * inv;
        a[r][r] -= l * l;
        if (r == c + 1) {  // its last update: the next pivot
          const double d = a[r][r];
          if (d > 0.0 && isfinite(d)) {
            s_piv[r] = d;
            s_inv[r] = pivot_rsqrt(d);
          } else {
            s_bad = 1;
          }
        }
      }
    } else {
      // trailing strict lower triangle: rows c + 1 + i, columns c + 1 + j, j < i
      const int w = m - c - 1, cnt = w * (w - 1) / 2;
      for (int e = t - 32; e < cnt; e += kDiagUpd) {
        const int r = c + 1 + s_tri[e][0], q = c + 1 + s_tri[e][1];
        a[r][q] -= (a[r][c] * inv) * (a[q][c] * inv);
      }
    }
    __syncthreads();
  }
  if (s_bad) {
    if (t == 0) S[0] = 1.0;
    return;
  }
  for (int e = t; e < m * m; e += kDiagThreads) {
    const int r = e / m, c = e % m;
    if (c <= r) A[(size_t)(r0 + r) * ld + r0 + c] = (r == c ? s_piv[c] : a[r][c]) * s_inv[c];  // sqrt(d) = d / sqrt(d)
  }
  if (t < m) S[1 + r0 + t] = s_inv[t];  // the reciprocal of L's diagonal, for the solve
}

// Tile (k + 1 + blockIdx.x, k): X L_kk^T = A_ik.  Four threads per row, each
// owning every fourth column of it in registers (forward substitution,
// right-looking on the unscaled unknowns: once v_c is final, the owners of
// the later columns subtract v_c M_jc at once, M = L_kk with column c
// scaled by 1 / L_cc, so a step of the serial path is one shuffle and one
// FMA; each unknown is scaled by its 1 / L_cc at the end).  The reciprocal
// pivots come from the diagonal kernel (S[1 ..]).  A panel lies below a
// full diagonal tile: only the last tile column is ragged, and it has none.
__global__ void __launch_bounds__(4 * kChT) ba_chol_panel_kernel(int n, size_t ld, double* __restrict__ S, int k) {
  __shared__ double M[kChT][kChT + 1];
  __shared__ double inv[kChT];
  if (chol_failed(S)) return;
  double* A = S + 6 * ld + 6;
  const int c0 = k * kChT;
  const int r0 = (k + 1 + (int)blockIdx.x) * kChT, mi = min(kChT, n - r0);
  if ((int)threadIdx.x < kChT) inv[threadIdx.x] = S[1 + c0 + threadIdx.x];
  __syncthreads();
  for (int e = threadIdx.x; e < kChT * kChT; e += blockDim.x) {
    const int r = e / kChT, c = e % kChT;
    M[r][c] = c < r ? A[(size_t)(c0 + r) * ld + c0 + c] * inv[c] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x / 4, p = threadIdx.x % 4;  // row r, columns p, p + 4, ...
  const int lane = threadIdx.x % 32;
  constexpr int kOwn = kChT / 4;
  double x[kOwn];
#pragma unroll
  for (int i = 0; i < kOwn; ++i) x[i] = r < mi ? A[(size_t)(r0 + r) * ld + c0 + p + 4 * i] : 0.0;
#pragma unroll
  for (int c = 0; c < kChT; ++c) {
    const double vc = __shfl_sync(0xffffffffu, x[c >> 2], (lane & ~3) | (c & 3));
#pragma unroll
    for (int i = 0; i < kOwn; ++i)
      if (p + 4 * i > c) x[i] = fma(-vc, M[p + 4 * i][c], x[i]);
  }
  if (r < mi) {
#pragma unroll
    for (int i = 0; i < kOwn; ++i) A[(size_t)(r0 + r) * ld + c0 + p + 4 * i] = x[i] * inv[p + 4 * i];
  }
}

// Rows [8 z, 8 z + 8) of tile (i, j) = (k + 1 + blockIdx.y, k + 1 +
// blockIdx.x), j <= i: A_ij -= L_ik L_jk^T, a thread per entry (four
// blocks per tile spread the FP64 work over more SMs).
constexpr int kUpdRows = 8;
__global__ void __launch_bounds__(kUpdRows * kChT) ba_chol_update_kernel(int n, size_t ld, double* __restrict__ S,
                                                                          int k) {
  __shared__ double Li[kUpdRows][kChT + 1];
  __shared__ double Lj[kChT][kChT + 1];
  if (blockIdx.x > blockIdx.y) return;  // upper triangle of tiles
  if (chol_failed(S)) return;
  double* A = S + 6 * ld + 6;
  const int c0 = k * kChT;  // a full tile column (see the panel)
  const int i0 = (k + 1 + (int)blockIdx.y) * kChT + kUpdRows * (int)blockIdx.z;
  const int mi = max(0, min(kUpdRows, n - i0));
  const int j0 = (k + 1 + (int)blockIdx.x) * kChT, mj = min(kChT, n - j0);
  const bool diag_tile = blockIdx.x == blockIdx.y;
  if (mi == 0) return;  // block-uniform: rows past the ragged last tile
  const int tx = threadIdx.x % kChT, ty = threadIdx.x / kChT;
  Li[ty][tx] = ty < mi ? A[(size_t)(i0 + ty) * ld + c0 + tx] : 0.0;
  for (int r = ty; r < kChT; r += kUpdRows) Lj[r][tx] = r < mj ? A[(size_t)(j0 + r) * ld + c0 + tx] : 0.0;
  __syncthreads();
  const int r = ty, c = tx;  // row i0 + r, column j0 + c
  const int rt = kUpdRows * (int)blockIdx.z + r;  // the row within its tile
  if (r >= mi || c >= mj || (diag_tile && c > rt)) return;  // diagonal tile: lower triangle only
  double v = 0.0;
#pragma unroll
  for (int q = 0; q < kChT; ++q) v += Li[r][q] * Lj[c][q];
  A[(size_t)(i0 + r) * ld + j0 + c] -= v;
}

// L y = b, then L^T x = y, tile by tile in one block; dc = (0, x).  Per
// tile: warp r sums row r's products with the other tiles' solved unknowns,
// then warp 0 solves the tile's triangle with a lane per row (the solved
// unknown of each column broadcast by a shuffle).  The unknowns stay in
// shared memory.
__global__ void __launch_bounds__(1024) ba_chol_solve_kernel(int V, double* __restrict__ S,
                                                             const double* __restrict__ rhs,
                                                             double* __restrict__ dc, int32_t* status) {
  __shared__ double Ld[kChT][kChT + 1];
  __shared__ double inv[kChT];
  __shared__ double part[kChT];
  extern __shared__ double y[];  // [n]: y, then x in place
  const int n = 6 * (V - 1);
  const size_t ld = 6 * (size_t)V;
  const double* A = S + 6 * ld + 6;
  const double* b = rhs + 6;
  for (int a = threadIdx.x; a < 6; a += blockDim.x) dc[a] = 0.0;
  if (chol_failed(S)) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dc[6 + i] = 0.0;
    if (threadIdx.x == 0 && status) atomicOr(status, GS_FLAG_NOT_SPD);
    return;
  }
  const int T = (n + kChT - 1) / kChT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // 32 warps
  for (int pass = 0; pass < 2; ++pass) {  // 0: L y = b; 1: L^T x = y
    for (int tt = 0; tt < T; ++tt) {
      const int t = pass == 0 ? tt : T - 1 - tt;
      const int r0 = t * kChT, m = min(kChT, n - r0);
      // the tile's triangle scaled so that each substitution step is one
      // FMA: column c by 1 / L_cc (forward), row c by 1 / L_cc (backward)
      for (int e = threadIdx.x; e < kChT * kChT; e += blockDim.x) {
        const int r = e / kChT, c = e % kChT;
        Ld[r][c] = (r < m && c <= r) ? A[(size_t)(r0 + r) * ld + r0 + c] * S[1 + r0 + (pass == 0 ? c : r)] : 0.0;
      }
      if ((int)threadIdx.x < m) inv[threadIdx.x] = S[1 + r0 + threadIdx.x];
      if (warp < m) {
        const int r = warp;
        double v = 0.0;
        if (pass == 0) {
          for (int q = lane; q < r0; q += 32) v += A[(size_t)(r0 + r) * ld + q] * y[q];
        } else {
          for (int q = r0 + m + lane; q < n; q += 32) v += A[(size_t)q * ld + r0 + r] * y[q];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) part[r] = (pass == 0 ? b[r0 + r] : y[r0 + r]) - v;
      }
      __syncthreads();
      if (warp == 0) {
        // right-looking substitution on the unscaled unknowns: lane c's
        // value is final once step c comes, then only the FMA of the later
        // (earlier) lanes depends on it; each lane scales its own at the end
        double v = lane < m ? part[lane] : 0.0;
        if (pass == 0) {
          for (int c = 0; c < m; ++c) {
            const double vc = __shfl_sync(0xffffffffu, v, c);
            if (lane > c && lane < m) v = fma(-Ld[lane][c], vc, v);
          }
        } else {
          for (int c = m - 1; c >= 0; --c) {
            const double vc = __shfl_sync(0xffffffffu, v, c);
            if (lane < c) v = fma(-Ld[c][lane], vc, v);
          }
        }
        if (lane < m) y[r0 + lane] = v * inv[lane];
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) dc[6 + i] = y[i];
}

}  // namespace

cudaError_t launch_ba_schur(int V, int P, int64_t M, const double* U, const double* Vp, const double* gc,
                            const double* gp, const double* Wo, const int32_t* obs_cam, const int64_t* point_obs_offset,
                            const int32_t* point_obs, double lambda, const double* lambda_dev, double* S,
                            double* rhs, double* Vinv,
                            cudaStream_t st) {
  if (V == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(double) * 36 * (size_t)V * (size_t)V, st);
  if (e != cudaSuccess) return e;
  ba_camera_init_kernel<<<(V + 63) / 64, 64, 0, st>>>(V, U, gc, lambda, lambda_dev, S, rhs);
  if (P > 0) {
    ba_point_vinv_kernel<<<(P + 127) / 128, 128, 0, st>>>(P, Vp, gp, lambda, lambda_dev, Vinv);
    // a thread per list entry (grid-stride: the host sizes the grid from
    // the observation count, the kernel reads the lists' true length)
    if (M > 0)
      ba_point_schur_kernel<<<(unsigned)std::min<int64_t>((M + 127) / 128, 65535), 128, 0, st>>>(V, P, M, gp, Vp, Wo, obs_cam,
                                                                          point_obs_offset, point_obs, Vinv, S, rhs);
  }
  return cudaGetLastError();
}

// Host side of the elimination by camera pairs: the incidences (k, a, b)
// of every point's ordered observation pairs with cam(b) <= cam(a) (entries
// outside [0, M) or with a camera outside [0, V) skipped), grouped by
// camera pair in order of (ca, cb), within a pair in order of k, then a's and
// b's positions in the point's list; each pair's list cut into chunks of at
// most `chunk`.  With null outputs only the sizes are returned.
int64_t ba_pair_plan(int V, int P, int64_t M, const int32_t* obs_cam, const int64_t* off, const int32_t* point_obs,
                     int chunk, int32_t* n_pairs_out, int32_t* n_chunks_out, int32_t* inc, int32_t* pair_cams,
                     int32_t* pair_chunks, int64_t* chunk_start) {
  struct Inc {
    int64_t pair;
    int32_t k, a, b;
  };
  std::vector<Inc> all;
  std::vector<int32_t> valid;
  for (int k = 0; k < P; ++k) {
    valid.clear();
    for (int64_t q = off[k]; q < off[k + 1]; ++q) {
      const int64_t o = point_obs[q];
      if (o < 0 || o >= M || (unsigned)obs_cam[o] >= (unsigned)V) continue;
      valid.push_back((int32_t)o);
    }
    for (const int32_t a : valid)
      for (const int32_t b : valid) {
        const int ca = obs_cam[a], cb = obs_cam[b];
        if (cb <= ca) all.push_back({(int64_t)ca * V + cb, k, a, b});
      }
  }
  std::stable_sort(all.begin(), all.end(), [](const Inc& x, const Inc& y) { return x.pair < y.pair; });
  int32_t n_pairs = 0, n_chunks = 0;
  for (size_t i = 0; i < all.size();) {
    size_t j = i;
    while (j < all.size() && all[j].pair == all[i].pair) ++j;
    const int64_t cnt = (int64_t)(j - i);
    if (pair_cams) {
      pair_cams[2 * n_pairs] = (int32_t)(all[i].pair / V);
      pair_cams[2 * n_pairs + 1] = (int32_t)(all[i].pair % V);
      pair_chunks[n_pairs] = n_chunks;
      for (int64_t c = 0; c < cnt; c += chunk) chunk_start[n_chunks + c / chunk] = (int64_t)i + c;
    }
    n_chunks += (int32_t)((cnt + chunk - 1) / chunk);
    ++n_pairs;
    i = j;
  }
  if (pair_cams) {
    pair_chunks[n_pairs] = n_chunks;
    chunk_start[n_chunks] = (int64_t)all.size();
    for (size_t i = 0; i < all.size(); ++i) {
      inc[3 * i] = all[i].k;
      inc[3 * i + 1] = all[i].a;
      inc[3 * i + 2] = all[i].b;
    }
  }
  *n_pairs_out = n_pairs;
  *n_chunks_out = n_chunks;
  return (int64_t)all.size();
}

size_t ba_schur_pairs_workspace_bytes(int64_t M, int n_chunks) {
  return sizeof(double) * ((size_t)kObsY * (size_t)std::max<int64_t>(M, 1) + (size_t)kPairValues * (size_t)n_chunks);
}

cudaError_t launch_ba_schur_pairs(int V, int P, int64_t M, const double* U, const double* Vp, const double* gc,
                                  const double* gp, const double* Wo, const int32_t* obs_cam,
                                  const int64_t* point_obs_offset, const int32_t* point_obs, const int32_t* inc,
                                  const int32_t* pair_cams, int n_pairs, const int32_t* pair_chunks,
                                  const int64_t* chunk_start, int n_chunks, double lambda, const double* lambda_dev,
                                  double* S, double* rhs, double* Vinv, void* ws, cudaStream_t st) {
  if (V == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(double) * 36 * (size_t)V * (size_t)V, st);
  if (e != cudaSuccess) return e;
  ba_camera_init_kernel<<<(V + 63) / 64, 64, 0, st>>>(V, U, gc, lambda, lambda_dev, S, rhs);
  if (P == 0 || M == 0) return cudaGetLastError();
  double* Y = (double*)ws;
  double* partial = Y + (size_t)kObsY * (size_t)M;
  ba_point_vinv_kernel<<<(P + 127) / 128, 128, 0, st>>>(P, Vp, gp, lambda, lambda_dev, Vinv);
  ba_obs_y_kernel<<<(unsigned)std::min<int64_t>((M + 127) / 128, 65535), 128, 0, st>>>(
      V, P, M, gp, Vp, Wo, obs_cam, point_obs_offset, point_obs, Vinv, Y);
  if (n_chunks > 0) {
    ba_pair_chunk_kernel<<<(n_chunks + kPairWarps - 1) / kPairWarps, 32 * kPairWarps, 0, st>>>(
        n_chunks, inc, chunk_start, obs_cam, Y, Wo, partial);
    const int64_t nt = (int64_t)n_pairs * kPairValues;
    ba_pair_finalize_kernel<<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(V, n_pairs, pair_cams, pair_chunks, partial,
                                                                         S, rhs);
  }
  return cudaGetLastError();
}

cudaError_t launch_ba_solve_cameras(int V, double* S, const double* rhs, double* dc, int32_t* status,
                                   cudaStream_t st) {
  if (V <= 0) return cudaSuccess;
  const int n = 6 * (V - 1);
  const size_t ld = 6 * (size_t)V;
  const int T = (n + kChT - 1) / kChT;
  ba_chol_init_kernel<<<1, 1, 0, st>>>(S);
  for (int k = 0; k < T; ++k) {
    ba_chol_diag_kernel<<<1, kDiagThreads, 0, st>>>(n, ld, S, k);
    if (k + 1 < T) {
      ba_chol_panel_kernel<<<T - k - 1, 4 * kChT, 0, st>>>(n, ld, S, k);
      ba_chol_update_kernel<<<dim3(T - k - 1, T - k - 1, kChT / kUpdRows), kUpdRows * kChT, 0, st>>>(n, ld, S, k);
    }
  }
  const size_t ysm = (size_t)n * sizeof(double);
  if (ysm > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(ba_chol_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)ysm);
    if (e != cudaSuccess) return e;
  }
  ba_chol_solve_kernel<<<1, 1024, ysm, st>>>(V, S, rhs, dc, status);
  return cudaGetLastError();
}

namespace {
// Accept or reject the trial parameters of one LM iteration (Marquardt):
// both kernels read the objectives before the second one writes them.
__global__ void ba_lm_copy_kernel(int V, int P, const double* __restrict__ obj, float* __restrict__ Rt,
                                  float* __restrict__ X, const float* __restrict__ Rt_trial,
                                  const float* __restrict__ X_trial) {
  if (!(obj[1] < obj[0])) return;  // grid-uniform
  const size_t nR = 12 * (size_t)V, n = nR + 3 * (size_t)P;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    if (e < nR) Rt[e] = Rt_trial[e];
    else X[e - nR] = X_trial[e - nR];
  }
}

__global__ void ba_lm_decide_kernel(double* obj, double* lambda, int32_t* n_accepted, double* history,
                                    int32_t history_len, int32_t* n_iter) {
  const bool accept = obj[1] < obj[0];
  if (accept) {
    obj[0] = obj[1];
    *lambda /= 10.0;
    if (n_accepted) ++*n_accepted;
  } else {
    *lambda *= 10.0;
  }
  if (n_iter) {
    const int it = *n_iter;
    if (history && it < history_len) history[it] = obj[0];
    *n_iter = it + 1;
  }
}
}  // namespace

cudaError_t launch_ba_lm_accept(int V, int P, double* obj, double* lambda, float* Rt, float* X, const float* Rt_trial,
                                const float* X_trial, int32_t* n_accepted, double* history, int32_t history_len,
                                int32_t* n_iter, cudaStream_t st) {
  const size_t n = 12 * (size_t)V + 3 * (size_t)P;
  if (n > 0)
    ba_lm_copy_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(V, P, obj, Rt, X, Rt_trial,
                                                                                         X_trial);
  ba_lm_decide_kernel<<<1, 1, 0, st>>>(obj, lambda, n_accepted, history, history_len, n_iter);
  return cudaGetLastError();
}

cudaError_t launch_ba_back_substitute(int V, int P, int64_t M, const double* Vinv, const double* Vp, const double* gp,
                                      const double* Wo, const int32_t* obs_cam, const int64_t* point_obs_offset,
                                      const int32_t* point_obs, const double* dc, double* dp, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  ba_back_substitute_kernel<<<(P + 127) / 128, 128, 0, st>>>(V, P, M, Vinv, Vp, gp, Wo, obs_cam, point_obs_offset,
                                                              point_obs, dc, dp);
  return cudaGetLastError();
}

}  // namespace gs
