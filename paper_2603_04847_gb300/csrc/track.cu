// Feature-track reprojection term of Eq. 6 (Algorithm 1, "Joint BA loss on
// track points"), forward and backward in one pass.
//
// Observations are bucketed by camera (view-CSR), so the batch's
// observations are B contiguous ranges.  A fixed grid walks their
// concatenation; each observation does its projection, Huber weight and
// Jacobians in registers, adds weight * drho/dX to its track point (three
// scalar atomics; a track has few observations, so they rarely collide),
// and its pose-tangent share is reduced warp -> block (shared double) ->
// per-block partial, summed in block order by a second kernel.
#include <algorithm>
#include <mutex>

#include "gs_internal.h"

namespace gs {

namespace {

struct TrackSlot {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  long long start;  // first observation of the slot's camera
  long long pref;   // observations of slots before this one
};

// kDet: a launch over one slot (B == 1), whose sums do not depend on the
// order in which warps and blocks run: each warp keeps its own pose and loss
// sums (lane 0 adds its warp's reduced values in the warp's own order), the
// block adds its warps in warp order, and the block's loss goes to
// loss_partial[block] for a fixed-order sum (track_loss_finalize_kernel).
// The point gradients are still added atomically: within one view a track
// point has one observation, so no two adds of one launch meet.
template <bool kDet>
__global__ void __launch_bounds__(256) track_kernel(const float* __restrict__ X, int n_points,
                                                    const int32_t* __restrict__ obs_point,
                                                    const float2* __restrict__ obs_xy,
                                                    const int64_t* __restrict__ view_obs_offset,
                                                    gs_cameras cams, gs_batch batch, float delta,
                                                    float weight, double* loss, float* grad_X,
                                                    uint32_t* n_masked, double* partial, double* loss_partial) {
  constexpr int kWarps = 256 / 32;
  __shared__ double s_tan_w[kDet ? kWarps : 1][6];
  __shared__ double s_loss_w[kDet ? kWarps : 1];
  __shared__ TrackSlot ts[GS_MAX_BATCH];
  __shared__ long long s_total;
  __shared__ double s_tan[GS_MAX_BATCH * 6];
  __shared__ double s_loss;
  __shared__ uint32_t s_masked;
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int b = 0; b < batch.B; ++b) {
      const int v = slot_view(cams, batch, b);
      const long long s = view_obs_offset[v], e = view_obs_offset[v + 1];
      ts[b].start = s;
      ts[b].pref = acc;
      acc += e > s ? e - s : 0;
    }
    s_total = acc;
    s_loss = 0.0;
    s_masked = 0;
  }
  for (int b = threadIdx.x; b < batch.B; b += blockDim.x) {
    const int v = slot_view(cams, batch, b);
    const float* Rt = cams.Rt + 12 * v;
    for (int i = 0; i < 9; ++i) ts[b].R[i] = Rt[i];
    for (int i = 0; i < 3; ++i) ts[b].t[i] = Rt[9 + i];
    ts[b].fx = cams.K[4 * v];
    ts[b].fy = cams.K[4 * v + 1];
    ts[b].cx = cams.K[4 * v + 2];
    ts[b].cy = cams.K[4 * v + 3];
  }
  for (int i = threadIdx.x; i < batch.B * 6; i += blockDim.x) s_tan[i] = 0.0;
  if constexpr (kDet)
    for (int i = threadIdx.x; i < kWarps * 6; i += blockDim.x) (&s_tan_w[0][0])[i] = 0.0;
  __syncthreads();
  const long long total = s_total;
  const int lane = threadIdx.x & 31;
  const float d2 = delta * delta;
  float lsum = 0.f;
  uint32_t masked = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // every lane of a warp runs the same number of iterations (warp collectives)
  const long long wbase0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  for (long long wbase = wbase0; wbase < total; wbase += stride) {
    const long long i = wbase + lane;
    const bool valid = i < total;
    int b = 0;
    float tan[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
      int lo = 0, hi = batch.B - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ts[mid].pref <= i) lo = mid;
        else hi = mid - 1;
      }
      b = lo;
      const TrackSlot& c = ts[b];
      const long long o = c.start + (i - c.pref);
      const int k = obs_point[o];
      const float2 xy = obs_xy[o];
      const bool in_range = (unsigned)k < (unsigned)n_points;
      const size_t kk = in_range ? (size_t)k : 0;
      const float Xw0 = X[3 * kk], Xw1 = X[3 * kk + 1], Xw2 = X[3 * kk + 2];
      // The projection and residual are formed in double: the residual is a
      // difference of two pixel coordinates of order 1e3 whose FP32 rounding
      // (~1e-4 px) would otherwise dominate the cancelling pose sum.  A few
      // dozen FP64 operations per observation cost nothing here.
      double Xd[3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        Xd[r] = (double)c.R[3 * r] * Xw0 + (double)c.R[3 * r + 1] * Xw1 + (double)c.R[3 * r + 2] * Xw2 +
                (double)c.t[r];
      float Xc[3] = {(float)Xd[0], (float)Xd[1], (float)Xd[2]};
      if (!in_range) {
        // observation of a point that does not exist: ignored
      } else if (Xd[2] <= (double)cams.near_plane) {
        ++masked;
      } else {
        const double izd = 1.0 / Xd[2];
        const float rx = (float)((double)c.fx * Xd[0] * izd + (double)c.cx - (double)xy.x);
        const float ry = (float)((double)c.fy * Xd[1] * izd + (double)c.cy - (double)xy.y);
        const float iz = (float)izd;
        const float s = rx * rx + ry * ry;
        float rho, drho;
        if (s <= d2) {
          rho = s;
          drho = 1.f;
        } else {
          const float rs = sqrtf(s);
          rho = 2.f * delta * rs - d2;
          drho = delta / rs;
        }
        lsum += rho;
        const float vu = weight * 2.f * rx * drho;
        const float vv = weight * 2.f * ry * drho;
        float vX[3];
        vX[0] = vu * c.fx * iz;
        vX[1] = vv * c.fy * iz;
        vX[2] = -(vu * c.fx * Xc[0] + vv * c.fy * Xc[1]) * iz * iz;
        float* gX = grad_X + 3 * kk;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          atomicAdd(gX + a, c.R[a] * vX[0] + c.R[3 + a] * vX[1] + c.R[6 + a] * vX[2]);
        tan[0] = vX[0];
        tan[1] = vX[1];
        tan[2] = vX[2];
        tan[3] = Xc[1] * vX[2] - Xc[2] * vX[1];
        tan[4] = Xc[2] * vX[0] - Xc[0] * vX[2];
        tan[5] = Xc[0] * vX[1] - Xc[1] * vX[0];
      }
    }
    // valid lanes form a prefix of the warp, so lane 0 is valid here
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    if (__all_sync(0xffffffffu, !valid || b == b0)) {
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        float x = tan[a];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) {
          if constexpr (kDet) s_tan_w[threadIdx.x >> 5][a] += (double)x;
          else atomicAdd(&s_tan[6 * b0 + a], (double)x);
        }
      }
    } else if (valid) {
#pragma unroll
      for (int a = 0; a < 6; ++a) atomicAdd(&s_tan[6 * b + a], (double)tan[a]);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    masked += __shfl_xor_sync(0xffffffffu, masked, off);
  }
  if (lane == 0) {
    if constexpr (kDet) s_loss_w[threadIdx.x >> 5] = (double)lsum;
    else atomicAdd(&s_loss, (double)lsum);
    atomicAdd(&s_masked, masked);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if constexpr (kDet) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s_loss_w[w];
      loss_partial[blockIdx.x] = t;
    } else {
      if (loss && s_loss != 0.0) atomicAdd(loss, s_loss);
    }
    if (n_masked && s_masked) atomicAdd(n_masked, s_masked);
  }
  if constexpr (kDet) {
    if (threadIdx.x < 6) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s_tan_w[w][threadIdx.x];
      partial[(size_t)blockIdx.x * 6 + threadIdx.x] = t;
    }
  } else {
    for (int i = threadIdx.x; i < batch.B * 6; i += blockDim.x)
      partial[(size_t)blockIdx.x * batch.B * 6 + i] = s_tan[i];
  }
}

// loss += the blocks' loss sums, in block order.
__global__ void __launch_bounds__(256) track_loss_finalize_kernel(const double* __restrict__ loss_partial,
                                                                  int n_blocks, double* loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < n_blocks; k += blockDim.x) s += loss_partial[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0 && red[0] != 0.0) atomicAdd(loss, red[0]);
}

}  // namespace

int track_blocks() { return 2 * device_sm_count(); }

size_t track_workspace_bytes(const gs_batch& batch) {
  // the pose partials of all slots, or (deterministic form, one slot at a
  // time) one slot's and the blocks' loss sums
  return (size_t)track_blocks() * (size_t)std::max(batch.B * 6, 7) * sizeof(double);
}

cudaError_t launch_track(const float* X, int n_points, const int32_t* obs_point, const float* obs_xy,
                         const int64_t* view_obs_offset, const gs_cameras& cams, const gs_batch& batch,
                         float delta, float weight, double* loss, float* grad_X,
                         double* g_pose_tangent, uint32_t* n_masked, void* ws, cudaStream_t st) {
  const int nb = track_blocks();
  double* partial = reinterpret_cast<double*>(ws);
  track_kernel<false><<<nb, 256, 0, st>>>(X, n_points, obs_point, reinterpret_cast<const float2*>(obs_xy),
                                          view_obs_offset, cams, batch, delta, weight, loss, grad_X, n_masked,
                                          partial, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_pose_partials_finalize(partial, nb, batch, cams.n_cams, g_pose_tangent, st);
}

cudaError_t launch_track_det(const float* X, int n_points, const int32_t* obs_point, const float* obs_xy,
                             const int64_t* view_obs_offset, const gs_cameras& cams, const gs_batch& batch,
                             float delta, float weight, double* loss, float* grad_X, double* g_pose_tangent,
                             uint32_t* n_masked, void* ws, cudaStream_t st) {
  const int nb = track_blocks();
  double* partial = reinterpret_cast<double*>(ws);
  double* loss_partial = partial + (size_t)nb * 6;
  // one slot per launch, in slot order: the additions into a point's
  // gradient, the pose tangent and the loss then come in a fixed order
  for (int b = 0; b < batch.B; ++b) {
    gs_batch one = batch;
    one.B = 1;
    one.views = batch.views + b;
    track_kernel<true><<<nb, 256, 0, st>>>(X, n_points, obs_point, reinterpret_cast<const float2*>(obs_xy),
                                           view_obs_offset, cams, one, delta, weight, loss, grad_X, n_masked,
                                           partial, loss_partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_pose_partials_finalize(partial, nb, one, cams.n_cams, g_pose_tangent, st);
    if (e != cudaSuccess) return e;
    if (loss) track_loss_finalize_kernel<<<1, 256, 0, st>>>(loss_partial, nb, loss);
  }
  return cudaGetLastError();
}

}  // namespace gs

// ---------------------------------------------------------------------------
// Allocation-free variant of track_reproj_fwd_bwd.
//
// Some callers cannot call cudaMalloc when they run this term: real-time
// loops that must not risk the implicit device synchronisation an allocation
// can cause, plug-ins that live inside a host framework's memory pool and may
// not allocate outside it, and processes that reserve all device memory up
// front.  For them the per-block pose partials go to a fixed array in device
// memory that belongs to this library.

// 1 MiB of scratch: enough for the partials of 2 * SMs blocks x 64 views x 6
// doubles on GPUs with up to 170 SMs.  Every GPU that loads the library
// keeps this array until the process exits.
#define GS_TRACK_STATIC_SCRATCH_BYTES (1u << 20)
static __device__ __align__(256) double gs_track_static_scratch[GS_TRACK_STATIC_SCRATCH_BYTES / sizeof(double)];

namespace gs {
namespace {

std::mutex g_track_scratch_mu;
void* g_track_scratch_ptr[64] = {nullptr};

// Device address of the scratch array on the current device.  Host code
// cannot pass the symbol itself to a kernel (on the host it names a host-side
// stand-in); the address is looked up once per device and cached.
cudaError_t track_static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_track_scratch_mu);
  if (g_track_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, gs_track_static_scratch);
    if (e != cudaSuccess) return e;
    g_track_scratch_ptr[dev] = p;
  }
  *out = g_track_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace gs

extern "C" gs_status track_reproj_fwd_bwd_static(const float* X, int32_t n_points, const int32_t* obs_point,
                                                 const float* obs_xy, const int64_t* view_obs_offset,
                                                 const gs_cameras* cams, const gs_batch* batch, float delta,
                                                 float weight, double* loss, float* grad_X,
                                                 double* g_pose_tangent, uint32_t* n_masked,
                                                 gs_stream stream) {
  using namespace gs;
  const char* who = "track_reproj_fwd_bwd_static";
  gs_status s = check_track_call(X, n_points, obs_point, obs_xy, view_obs_offset, cams, batch, delta,
                                 weight, grad_X, g_pose_tangent, who);
  if (s != GS_OK) return s;
  const size_t need = track_workspace_bytes(*batch);
  if (need > GS_TRACK_STATIC_SCRATCH_BYTES)
    return record_error(GS_ERR_CAPACITY,
                        "%s: this batch needs %zu bytes of scratch, more than the %u-byte static array; "
                        "use track_reproj_fwd_bwd with a caller workspace",
                        who, need, (unsigned)GS_TRACK_STATIC_SCRATCH_BYTES);
  void* ws = nullptr;
  cudaError_t e = track_static_scratch(&ws);
  if (e != cudaSuccess) return record_error(GS_ERR_CUDA, "%s: scratch address: %s", who, cudaGetErrorString(e));
  e = launch_track(X, n_points, obs_point, obs_xy, view_obs_offset, *cams, *batch, delta, weight, loss, grad_X,
                   g_pose_tangent, n_masked, ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return record_error(GS_ERR_CUDA, "%s: %s", who, cudaGetErrorString(e));
  return GS_OK;
}

