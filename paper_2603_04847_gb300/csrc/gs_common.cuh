// Device-side building blocks shared by the libgs kernels (sm_103a).
//
// Everything here is device code written for this library (FP32, and the
// FP64 instantiation of the same kernels); the FP64 test oracle shares none
// of it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

// Compositing constants of the rasterizer that the paper uses (Sec. 3.3,
// "Implementation"): the published 3DGS choices.
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kDilation = 0.3f;
constexpr float kGuard = 1.3f;

// The same constants for either scalar type (the FP64 instantiation of the
// kernels, used to check them against finite differences).
template <typename T>
struct Consts;
template <>
struct Consts<float> {
  static constexpr float alpha_min = kAlphaMin, alpha_max = kAlphaMax, t_min = kTMin;
  static constexpr float dilation = kDilation, guard = kGuard;
};
template <>
struct Consts<double> {
  static constexpr double alpha_min = 1.0 / 255.0, alpha_max = 0.99, t_min = 1e-4;
  static constexpr double dilation = 0.3, guard = 1.3;
};

// Device views of the ABI structs for scalar type T (float: gs_cameras,
// gs_gaussians, ...; double: their _f64 counterparts).
template <typename T>
struct CamsT {
  int32_t n_cams;
  const int32_t* wh;
  const T* K;
  const T* Rt;
  T near_plane, far_plane;
};
template <typename T>
struct GaussT {
  int32_t n, sh_degree;
  const T* mean;
  const T* log_scale;
  const T* quat;
  const T* opacity_logit;
  const T* sh;
};
template <typename T>
struct GradsT {
  T* mean;
  T* log_scale;
  T* quat;
  T* opacity_logit;
  T* sh;
};
template <typename T>
struct ProjT {
  T* splat;  // [B*N, 12]
  uint16_t* rect;
  uint32_t* n_tiles;
  uint32_t* depth_key;
};

inline CamsT<float> view_of(const gs_cameras& c) {
  return CamsT<float>{c.n_cams, c.wh, c.K, c.Rt, c.near_plane, c.far_plane};
}
inline GaussT<float> view_of(const gs_gaussians& g) {
  return GaussT<float>{g.n, g.sh_degree, g.mean, g.log_scale, g.quat, g.opacity_logit, g.sh};
}
inline GradsT<float> view_of(const gs_gaussian_grads& g) {
  return GradsT<float>{g.mean, g.log_scale, g.quat, g.opacity_logit, g.sh};
}
inline ProjT<float> view_of(const gs_projected& p) { return ProjT<float>{p.splat, p.rect, p.n_tiles, p.depth_key}; }
inline CamsT<double> view_of(const gs_cameras_f64& c) {
  return CamsT<double>{c.n_cams, c.wh, c.K, c.Rt, c.near_plane, c.far_plane};
}
inline GaussT<double> view_of(const gs_gaussians_f64& g) {
  return GaussT<double>{g.n, g.sh_degree, g.mean, g.log_scale, g.quat, g.opacity_logit, g.sh};
}
inline GradsT<double> view_of(const gs_gaussian_grads_f64& g) {
  return GradsT<double>{g.mean, g.log_scale, g.quat, g.opacity_logit, g.sh};
}
inline ProjT<double> view_of(const gs_projected_f64& p) { return ProjT<double>{p.splat, p.rect, p.n_tiles, p.depth_key}; }

// Scalar math of either type.
__device__ inline float gexp(float x) { return expf(x); }
__device__ inline double gexp(double x) { return exp(x); }
__device__ inline float glog(float x) { return logf(x); }
__device__ inline double glog(double x) { return log(x); }
__device__ inline float gsqrt(float x) { return sqrtf(x); }
__device__ inline double gsqrt(double x) { return sqrt(x); }
__device__ inline float grsqrt(float x) { return rsqrtf(x); }
__device__ inline double grsqrt(double x) { return 1.0 / sqrt(x); }
__device__ inline float gmin(float a, float b) { return fminf(a, b); }
__device__ inline double gmin(double a, double b) { return fmin(a, b); }
__device__ inline float gmax(float a, float b) { return fmaxf(a, b); }
__device__ inline double gmax(double a, double b) { return fmax(a, b); }
__device__ inline float gceil(float a) { return ceilf(a); }
__device__ inline double gceil(double a) { return ceil(a); }
__device__ inline float gfloor(float a) { return floorf(a); }
__device__ inline double gfloor(double a) { return floor(a); }

// True when slot b's share of the batch's offsets is exactly the size of
// its view (W H pixels, tiles_x tiles_y tiles).  A slot that fails this
// (emptied by gs_batch_layout, or offsets left from other views) is skipped
// by every kernel, so no kernel can index past the slot's share.
__device__ inline bool slot_consistent(const gs_batch& batch, int b, int W, int H) {
  const long long T = batch.tile;
  const long long nt = ((W + T - 1) / T) * ((H + T - 1) / T);
  return (long long)batch.tile_offset[b + 1] - batch.tile_offset[b] == nt &&
         batch.px_offset[b + 1] - batch.px_offset[b] == (long long)W * H;
}

// Per-slot camera data staged in shared memory by every batched kernel.
template <typename T>
struct SlotCamT {
  T R[9];
  T t[3];
  T fx, fy, cx, cy;
  T campos[3];      // camera centre -R^T t
  T limx, limy;     // guard band on x/z, y/z
  int W, H;
  int tiles_x, tiles_y;
  int view;
  int tile_offset;
  long long px_offset;
  int active;       // the slot's offsets hold exactly its view (0: emptied
                    // by gs_batch_layout, or offsets not laid out for it)
};
using SlotCam = SlotCamT<float>;

// Camera index of slot b; an out-of-range id (a caller error the host
// cannot see) is mapped to camera 0 instead of reading out of bounds.
__device__ inline int slot_view_n(int n_cams, const gs_batch& batch, int b) {
  const int v = batch.views[b];
  return ((unsigned)v < (unsigned)n_cams) ? v : 0;
}
__device__ inline int slot_view(const gs_cameras& cams, const gs_batch& batch, int b) {
  return slot_view_n(cams.n_cams, batch, b);
}

// Loads the B slot cameras of a batch into `sc` (shared); call from all
// threads of the block, followed by __syncthreads().
template <typename T>
__device__ inline void load_slot_cams(const CamsT<T>& cams, const gs_batch& batch, SlotCamT<T>* sc) {
  for (int b = threadIdx.x; b < batch.B; b += blockDim.x) {
    const int v = slot_view_n(cams.n_cams, batch, b);
    SlotCamT<T> c;
    const T* Rt = cams.Rt + 12 * v;
#pragma unroll
    for (int i = 0; i < 9; ++i) c.R[i] = Rt[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) c.t[i] = Rt[9 + i];
    c.fx = cams.K[4 * v + 0];
    c.fy = cams.K[4 * v + 1];
    c.cx = cams.K[4 * v + 2];
    c.cy = cams.K[4 * v + 3];
    c.W = cams.wh[2 * v];
    c.H = cams.wh[2 * v + 1];
    for (int i = 0; i < 3; ++i)
      c.campos[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
    c.limx = Consts<T>::guard * T(0.5) * (T)c.W / c.fx;
    c.limy = Consts<T>::guard * T(0.5) * (T)c.H / c.fy;
    c.tiles_x = (c.W + batch.tile - 1) / batch.tile;
    c.tiles_y = (c.H + batch.tile - 1) / batch.tile;
    c.view = v;
    c.tile_offset = batch.tile_offset[b];
    c.px_offset = batch.px_offset[b];
    c.active = c.W > 0 && c.H > 0 && slot_consistent(batch, b, c.W, c.H);
    sc[b] = c;
  }
}

__device__ inline void set_flag(int32_t* status, int32_t flag) {
  if (status) atomicOr(status, flag);
}

// Real spherical harmonics up to degree 3 in the coefficient order and sign
// convention of the original 3DGS renderer.  Normalisation constants are the
// textbook values sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) (times sqrt 2 for m != 0).
template <typename T>
struct ShC;
template <>
struct ShC<float> {
  static constexpr float k00 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
  static constexpr float k1 = 0.4886025119029199f;     // sqrt(3/(4 pi))
  static constexpr float k2a = 1.0925484305920792f;    // sqrt(15/pi)/2
  static constexpr float k2b = 0.31539156525252005f;   // sqrt(5/pi)/4
  static constexpr float k2c = 0.5462742152960396f;    // sqrt(15/pi)/4
  static constexpr float k3a = 0.5900435899266435f;    // sqrt(35/(2 pi))/4
  static constexpr float k3b = 2.890611442640554f;     // sqrt(105/pi)/2
  static constexpr float k3c = 0.4570457994644658f;    // sqrt(21/(2 pi))/4
  static constexpr float k3d = 0.3731763325901154f;    // sqrt(7/pi)/4
  static constexpr float k3e = 1.445305721320277f;     // sqrt(105/pi)/4
};
template <>
struct ShC<double> {
  static constexpr double k00 = 0.28209479177387814, k1 = 0.4886025119029199, k2a = 1.0925484305920792,
                          k2b = 0.31539156525252005, k2c = 0.5462742152960396, k3a = 0.5900435899266435,
                          k3b = 2.890611442640554, k3c = 0.4570457994644658, k3d = 0.3731763325901154,
                          k3e = 1.445305721320277;
};

// Y[0..K) for unit direction (x, y, z).
template <typename T>
__device__ inline void sh_basis(int deg, T x, T y, T z, T* Y) {
  using C = ShC<T>;
  Y[0] = C::k00;
  if (deg < 1) return;
  Y[1] = -C::k1 * y;
  Y[2] = C::k1 * z;
  Y[3] = -C::k1 * x;
  if (deg < 2) return;
  const T xx = x * x, yy = y * y, zz = z * z;
  Y[4] = C::k2a * x * y;
  Y[5] = -C::k2a * y * z;
  Y[6] = C::k2b * (T(2) * zz - xx - yy);
  Y[7] = -C::k2a * x * z;
  Y[8] = C::k2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -C::k3a * y * (T(3) * xx - yy);
  Y[10] = C::k3b * x * y * z;
  Y[11] = -C::k3c * y * (T(4) * zz - xx - yy);
  Y[12] = C::k3d * z * (T(2) * zz - T(3) * xx - T(3) * yy);
  Y[13] = -C::k3c * x * (T(4) * zz - xx - yy);
  Y[14] = C::k3e * z * (xx - yy);
  Y[15] = -C::k3a * x * (xx - T(3) * yy);
}

// d/d(x,y,z) of sum_k w[k] Y_k(x,y,z) (polynomial form), added into g.
template <typename T>
__device__ inline void sh_basis_grad_dot(int deg, T x, T y, T z, const T* w, T* g) {
  using C = ShC<T>;
  if (deg < 1) return;
  g[0] += -C::k1 * w[3];
  g[1] += -C::k1 * w[1];
  g[2] += C::k1 * w[2];
  if (deg < 2) return;
  const T xx = x * x, yy = y * y, zz = z * z;
  g[0] += C::k2a * y * w[4] - C::k2a * z * w[7] - T(2) * C::k2b * x * w[6] + T(2) * C::k2c * x * w[8];
  g[1] += C::k2a * x * w[4] - C::k2a * z * w[5] - T(2) * C::k2b * y * w[6] - T(2) * C::k2c * y * w[8];
  g[2] += -C::k2a * y * w[5] + T(4) * C::k2b * z * w[6] - C::k2a * x * w[7];
  if (deg < 3) return;
  // Y9  = -k3a (3 x^2 y - y^3)       Y10 = k3b x y z
  // Y11 = -k3c (4 y z^2 - x^2 y - y^3)
  // Y12 = k3d (2 z^3 - 3 x^2 z - 3 y^2 z)
  // Y13 = -k3c (4 x z^2 - x^3 - x y^2)
  // Y14 = k3e (x^2 z - y^2 z)        Y15 = -k3a (x^3 - 3 x y^2)
  g[0] += -C::k3a * T(6) * x * y * w[9] + C::k3b * y * z * w[10] + C::k3c * T(2) * x * y * w[11] -
          C::k3d * T(6) * x * z * w[12] - C::k3c * (T(4) * zz - T(3) * xx - yy) * w[13] +
          C::k3e * T(2) * x * z * w[14] - C::k3a * T(3) * (xx - yy) * w[15];
  g[1] += -C::k3a * T(3) * (xx - yy) * w[9] + C::k3b * x * z * w[10] -
          C::k3c * (T(4) * zz - xx - T(3) * yy) * w[11] - C::k3d * T(6) * y * z * w[12] +
          C::k3c * T(2) * x * y * w[13] - C::k3e * T(2) * y * z * w[14] + C::k3a * T(6) * x * y * w[15];
  g[2] += C::k3b * x * y * w[10] - C::k3c * T(8) * y * z * w[11] +
          C::k3d * (T(6) * zz - T(3) * xx - T(3) * yy) * w[12] - C::k3c * T(8) * x * z * w[13] +
          C::k3e * (xx - yy) * w[14];
}

// Finite check without relying on fast-math semantics.
__device__ inline bool finitef(float v) { return isfinite(v); }
__device__ inline bool finitef(double v) { return isfinite(v); }

}  // namespace gs
