// Device-side building blocks shared by the libgs kernels (sm_103a).
//
// Everything here is FP32 device code written for this library; the FP64
// test oracle shares none of it.
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

// Per-slot camera data staged in shared memory by every batched kernel.
struct SlotCam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float campos[3];  // camera centre -R^T t
  float limx, limy; // guard band on x/z, y/z
  int W, H;
  int tiles_x, tiles_y;
  int view;
  int tile_offset;
  long long px_offset;
};

// Loads the B slot cameras of a batch into `sc` (shared); call from all
// threads of the block, followed by __syncthreads().
// Camera index of slot b; an out-of-range id (a caller error the host
// cannot see) is mapped to camera 0 instead of reading out of bounds.
__device__ inline int slot_view(const gs_cameras& cams, const gs_batch& batch, int b) {
  const int v = batch.views[b];
  return ((unsigned)v < (unsigned)cams.n_cams) ? v : 0;
}

__device__ inline void load_slot_cams(const gs_cameras& cams, const gs_batch& batch,
                                      SlotCam* sc) {
  for (int b = threadIdx.x; b < batch.B; b += blockDim.x) {
    const int v = slot_view(cams, batch, b);
    SlotCam c;
    const float* Rt = cams.Rt + 12 * v;
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
    c.limx = kGuard * 0.5f * (float)c.W / c.fx;
    c.limy = kGuard * 0.5f * (float)c.H / c.fy;
    c.tiles_x = (c.W + batch.tile - 1) / batch.tile;
    c.tiles_y = (c.H + batch.tile - 1) / batch.tile;
    c.view = v;
    c.tile_offset = batch.tile_offset[b];
    c.px_offset = batch.px_offset[b];
    sc[b] = c;
  }
}

__device__ inline void set_flag(int32_t* status, int32_t flag) {
  if (status) atomicOr(status, flag);
}

// Real spherical harmonics up to degree 3 in the coefficient order and sign
// convention of the original 3DGS renderer.  Normalisation constants are the
// textbook values sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) (times sqrt 2 for m != 0).
namespace shc {
constexpr float k00 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float k1 = 0.4886025119029199f;     // sqrt(3/(4 pi))
constexpr float k2a = 1.0925484305920792f;    // sqrt(15/pi)/2
constexpr float k2b = 0.31539156525252005f;   // sqrt(5/pi)/4
constexpr float k2c = 0.5462742152960396f;    // sqrt(15/pi)/4
constexpr float k3a = 0.5900435899266435f;    // sqrt(35/(2 pi))/4
constexpr float k3b = 2.890611442640554f;     // sqrt(105/pi)/2
constexpr float k3c = 0.4570457994644658f;    // sqrt(21/(2 pi))/4
constexpr float k3d = 0.3731763325901154f;    // sqrt(7/pi)/4
constexpr float k3e = 1.445305721320277f;     // sqrt(105/pi)/4
}  // namespace shc

// Y[0..K) for unit direction (x, y, z).
__device__ inline void sh_basis(int deg, float x, float y, float z, float* Y) {
  using namespace shc;
  Y[0] = k00;
  if (deg < 1) return;
  Y[1] = -k1 * y;
  Y[2] = k1 * z;
  Y[3] = -k1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = k2a * x * y;
  Y[5] = -k2a * y * z;
  Y[6] = k2b * (2.f * zz - xx - yy);
  Y[7] = -k2a * x * z;
  Y[8] = k2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -k3a * y * (3.f * xx - yy);
  Y[10] = k3b * x * y * z;
  Y[11] = -k3c * y * (4.f * zz - xx - yy);
  Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -k3c * x * (4.f * zz - xx - yy);
  Y[14] = k3e * z * (xx - yy);
  Y[15] = -k3a * x * (xx - 3.f * yy);
}

// d/d(x,y,z) of sum_k w[k] Y_k(x,y,z) (polynomial form), added into g.
__device__ inline void sh_basis_grad_dot(int deg, float x, float y, float z, const float* w,
                                         float* g) {
  using namespace shc;
  if (deg < 1) return;
  g[0] += -k1 * w[3];
  g[1] += -k1 * w[1];
  g[2] += k1 * w[2];
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  g[0] += k2a * y * w[4] - k2a * z * w[7] - 2.f * k2b * x * w[6] + 2.f * k2c * x * w[8];
  g[1] += k2a * x * w[4] - k2a * z * w[5] - 2.f * k2b * y * w[6] - 2.f * k2c * y * w[8];
  g[2] += -k2a * y * w[5] + 4.f * k2b * z * w[6] - k2a * x * w[7];
  if (deg < 3) return;
  // Y9  = -k3a (3 x^2 y - y^3)       Y10 = k3b x y z
  // Y11 = -k3c (4 y z^2 - x^2 y - y^3)
  // Y12 = k3d (2 z^3 - 3 x^2 z - 3 y^2 z)
  // Y13 = -k3c (4 x z^2 - x^3 - x y^2)
  // Y14 = k3e (x^2 z - y^2 z)        Y15 = -k3a (x^3 - 3 x y^2)
  g[0] += -k3a * 6.f * x * y * w[9] + k3b * y * z * w[10] + k3c * 2.f * x * y * w[11] -
          k3d * 6.f * x * z * w[12] - k3c * (4.f * zz - 3.f * xx - yy) * w[13] +
          k3e * 2.f * x * z * w[14] - k3a * 3.f * (xx - yy) * w[15];
  g[1] += -k3a * 3.f * (xx - yy) * w[9] + k3b * x * z * w[10] -
          k3c * (4.f * zz - xx - 3.f * yy) * w[11] - k3d * 6.f * y * z * w[12] +
          k3c * 2.f * x * y * w[13] - k3e * 2.f * y * z * w[14] + k3a * 6.f * x * y * w[15];
  g[2] += k3b * x * y * w[10] - k3c * 8.f * y * z * w[11] +
          k3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12] - k3c * 8.f * x * z * w[13] +
          k3e * (xx - yy) * w[14];
}

// Finite check without relying on fast-math semantics.
__device__ inline bool finitef(float v) { return isfinite(v); }

}  // namespace gs
