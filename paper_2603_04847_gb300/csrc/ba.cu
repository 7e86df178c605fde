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
#include "gs_internal.h"

namespace gs {

namespace {

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

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
    double* wo = Wo + 18 * o;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) wo[3 * a + c] = w * (jp[0][a] * jx[0][c] + jp[1][a] * jx[1][c]);
  }
  if (valid) {
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
    if (__all_sync(0xffffffffu, !valid || cam == cref)) {
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
  ba_assemble_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, n_points, cams, obs_point, obs_cam,
                                                       reinterpret_cast<const float2*>(obs_xy), n_obs,
                                                       (double)delta, U, Vp, gc, gp, Wo, objective);
  return cudaGetLastError();
}

}  // namespace gs
