// C ABI of libgs: argument validation, workspace carving and launches.
// Nothing here allocates device memory and nothing throws across the ABI.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "gs_internal.h"

namespace gs {

namespace {
thread_local char g_err[512] = "";

gs_status fail(gs_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

gs_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

gs_status check_gaussians(const gs_gaussians* g) {
  if (!g) return fail(GS_ERR_ARG, "gaussians: null");
  if (g->n < 0) return fail(GS_ERR_ARG, "gaussians: n < 0");
  if (g->sh_degree < 0 || g->sh_degree > 3) return fail(GS_ERR_ARG, "gaussians: sh_degree must be 0..3");
  if (g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->sh))
    return fail(GS_ERR_ARG, "gaussians: null array");
  if (!aligned(g->quat, 16)) return fail(GS_ERR_ARG, "gaussians: quat must be 16-byte aligned");
  return GS_OK;
}

gs_status check_cameras(const gs_cameras* c) {
  if (!c) return fail(GS_ERR_ARG, "cameras: null");
  if (c->n_cams < 1) return fail(GS_ERR_ARG, "cameras: n_cams < 1");
  if (!c->wh || !c->K || !c->Rt) return fail(GS_ERR_ARG, "cameras: null array");
  if (!std::isfinite(c->near_plane) || !std::isfinite(c->far_plane))
    return fail(GS_ERR_NONFINITE, "cameras: non-finite near/far");
  if (!(c->near_plane > 0.f) || !(c->far_plane > c->near_plane))
    return fail(GS_ERR_ARG, "cameras: need 0 < near < far");
  return GS_OK;
}

gs_status check_batch(const gs_batch* b) {
  if (!b) return fail(GS_ERR_ARG, "batch: null");
  if (b->B < 1 || b->B > GS_MAX_BATCH) return fail(GS_ERR_ARG, "batch: B must be 1..%d", GS_MAX_BATCH);
  if (b->tile != 16 && b->tile != 32) return fail(GS_ERR_UNSUPPORTED, "batch: tile %d unsupported (16 or 32)", b->tile);
  if (!b->views || !b->px_offset || !b->tile_offset) return fail(GS_ERR_ARG, "batch: null array");
  if (b->n_pixels < 0 || b->n_tiles < 0) return fail(GS_ERR_ARG, "batch: negative sizes");
  return GS_OK;
}

gs_status check_projected(const gs_projected* p) {
  if (!p) return fail(GS_ERR_ARG, "projected: null");
  if (!p->splat || !p->rect || !p->n_tiles || !p->depth_key) return fail(GS_ERR_ARG, "projected: null array");
  if (!aligned(p->splat, 16) || !aligned(p->rect, 8) || !aligned(p->depth_key, 16))
    return fail(GS_ERR_ARG, "projected: splat and depth_key must be 16-byte, rect 8-byte aligned");
  return GS_OK;
}

gs_status check_gaussians(const gs_gaussians_f64* g) {
  if (!g) return fail(GS_ERR_ARG, "gaussians: null");
  if (g->n < 0) return fail(GS_ERR_ARG, "gaussians: n < 0");
  if (g->sh_degree < 0 || g->sh_degree > 3) return fail(GS_ERR_ARG, "gaussians: sh_degree must be 0..3");
  if (g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->sh))
    return fail(GS_ERR_ARG, "gaussians: null array");
  if (!aligned(g->quat, 16)) return fail(GS_ERR_ARG, "gaussians: quat must be 16-byte aligned");
  return GS_OK;
}

gs_status check_cameras(const gs_cameras_f64* c) {
  if (!c) return fail(GS_ERR_ARG, "cameras: null");
  if (c->n_cams < 1) return fail(GS_ERR_ARG, "cameras: n_cams < 1");
  if (!c->wh || !c->K || !c->Rt) return fail(GS_ERR_ARG, "cameras: null array");
  if (!std::isfinite(c->near_plane) || !std::isfinite(c->far_plane))
    return fail(GS_ERR_NONFINITE, "cameras: non-finite near/far");
  if (!(c->near_plane > 0.0) || !(c->far_plane > c->near_plane))
    return fail(GS_ERR_ARG, "cameras: need 0 < near < far");
  return GS_OK;
}

gs_status check_projected(const gs_projected_f64* p) {
  if (!p) return fail(GS_ERR_ARG, "projected: null");
  if (!p->splat || !p->rect || !p->n_tiles || !p->depth_key) return fail(GS_ERR_ARG, "projected: null array");
  if (!aligned(p->splat, 16) || !aligned(p->rect, 8) || !aligned(p->depth_key, 16))
    return fail(GS_ERR_ARG, "projected: splat and depth_key must be 16-byte, rect 8-byte aligned");
  return GS_OK;
}

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t v2d_bytes(int N, const gs_batch& b) { return align_up((size_t)b.B * N * 12 * sizeof(float)); }
size_t v2d_bytes_f64(int N, const gs_batch& b) { return align_up((size_t)b.B * N * 12 * sizeof(double)); }
size_t pose_partial_bytes(int N, const gs_batch& b) {
  return align_up((size_t)project_bwd_blocks(N) * b.B * 6 * sizeof(double));
}

}  // namespace

namespace {
gs_tuning g_tuning = {128, 64, 1, 0};  // what the autotuner picks on the benchmark workloads
}

const gs_tuning& tuning() { return g_tuning; }

int device_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
  if (dev < 64 && cache[dev] > 0) return cache[dev];
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    sms = 148;
  if (dev < 64) cache[dev] = sms;
  return sms;
}

}  // namespace gs

using namespace gs;

extern "C" {

int gs_abi_version(void) { return GS_ABI_VERSION; }

const char* gs_last_error(void) { return g_err; }

size_t gs_struct_size(int which) {
  switch (which) {
    case 0: return sizeof(gs_gaussians);
    case 1: return sizeof(gs_gaussian_grads);
    case 2: return sizeof(gs_cameras);
    case 3: return sizeof(gs_batch);
    case 4: return sizeof(gs_projected);
    case 5: return sizeof(gs_adam);
    case 6: return sizeof(gs_tuning);
    case 7: return sizeof(gs_adam_group);
    case 8: return sizeof(gs_gaussians_f64);
    case 9: return sizeof(gs_gaussian_grads_f64);
    case 10: return sizeof(gs_cameras_f64);
    case 11: return sizeof(gs_projected_f64);
    default: return 0;
  }
}

int gs_device_sm_count(void) { return device_sm_count(); }

gs_status gs_set_tuning(const gs_tuning* t) {
  if (!t) return fail(GS_ERR_ARG, "gs_set_tuning: null");
  for (int32_t rb : {t->render_fwd_batch, t->render_bwd_batch})
    if (rb != 64 && rb != 128 && rb != 256)
      return fail(GS_ERR_ARG, "gs_set_tuning: render_fwd_batch and render_bwd_batch must be 64, 128 or 256");
  if (t->sort_blocks_per_sm < 1 || t->sort_blocks_per_sm > 8)
    return fail(GS_ERR_ARG, "gs_set_tuning: sort_blocks_per_sm must be 1..8");
  if (t->sort_spin_limit < -(1 << 20) || t->sort_spin_limit > (1 << 24))
    return fail(GS_ERR_ARG, "gs_set_tuning: sort_spin_limit must be in [-2^20, 2^24]");
  g_tuning = *t;
  return GS_OK;
}

gs_status gs_get_tuning(gs_tuning* t) {
  if (!t) return fail(GS_ERR_ARG, "gs_get_tuning: null");
  *t = g_tuning;
  return GS_OK;
}

gs_status gs_project(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                     const gs_projected* out, int32_t* status, gs_stream stream) {
  gs_status s;
  if ((s = check_gaussians(g)) || (s = check_cameras(cams)) || (s = check_batch(batch)) ||
      (s = check_projected(out)))
    return s;
  if ((unsigned long long)batch->B * (unsigned long long)g->n >= 0xffffffffull)
    return fail(GS_ERR_ARG, "gs_project: B*N must be < 2^32");
  cudaError_t e = launch_project_fwd(*g, *cams, *batch, *out, status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_project");
  return GS_OK;
}

gs_status gs_sort_tiles_workspace(int32_t n_gaussians, const gs_batch* batch, size_t capacity,
                                  size_t* ws_bytes) {
  gs_status s;
  if ((s = check_batch(batch))) return s;
  if (!ws_bytes || n_gaussians < 0) return fail(GS_ERR_ARG, "gs_sort_tiles_workspace: bad argument");
  *ws_bytes = sort_workspace_bytes(n_gaussians, *batch, capacity);
  return GS_OK;
}

gs_status gs_sort_tiles(int32_t n_gaussians, const gs_cameras* cams, const gs_batch* batch,
                        const gs_projected* proj, uint32_t* tiles, uint32_t* vals, size_t capacity,
                        uint32_t* ranges, uint32_t* n_instances, void* ws, size_t ws_bytes,
                        int32_t* status, gs_stream stream) {
  gs_status s;
  if ((s = check_cameras(cams)) || (s = check_batch(batch)) || (s = check_projected(proj))) return s;
  if (n_gaussians < 0 || !tiles || !vals || !ranges || !n_instances || !ws)
    return fail(GS_ERR_ARG, "gs_sort_tiles: null argument");
  if ((unsigned long long)batch->B * (unsigned long long)n_gaussians >= 0xffffffffull)
    return fail(GS_ERR_ARG, "gs_sort_tiles: B*N must be < 2^32");
  if (capacity == 0 || capacity >= 0xffffffffull)
    return fail(GS_ERR_CAPACITY, "gs_sort_tiles: capacity must be in [1, 2^32 - 1)");
  if (!aligned(ws, 256)) return fail(GS_ERR_ARG, "gs_sort_tiles: ws must be 256-byte aligned");
  if (!aligned(tiles, 16)) return fail(GS_ERR_ARG, "gs_sort_tiles: tiles must be 16-byte aligned");
  const size_t need = sort_workspace_bytes(n_gaussians, *batch, capacity);
  if (ws_bytes < need) return fail(GS_ERR_ARG, "gs_sort_tiles: workspace %zu < %zu bytes", ws_bytes, need);
  cudaError_t e = launch_sort_tiles(n_gaussians, *cams, *batch, *proj, tiles, vals, capacity, ranges,
                                    n_instances, ws, status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_sort_tiles");
  return GS_OK;
}

gs_status gs_render_fwd(const gs_batch* batch, const gs_cameras* cams, const gs_projected* proj,
                        const uint32_t* vals, const uint32_t* ranges, const float* bg, float* image,
                        float* T_final, uint32_t* n_contrib, uint32_t* n_added, gs_stream stream) {
  gs_status s;
  if ((s = check_batch(batch)) || (s = check_cameras(cams)) || (s = check_projected(proj))) return s;
  if (!vals || !ranges || !bg || !image || !T_final || !n_contrib)
    return fail(GS_ERR_ARG, "gs_render_fwd: null argument");
  cudaError_t e = launch_render_fwd(*batch, *cams, *proj, vals, ranges, bg, image, T_final, n_contrib,
                                    n_added, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_render_fwd");
  return GS_OK;
}

gs_status gs_render_bwd_workspace(int32_t n_gaussians, const gs_batch* batch, size_t* ws_bytes) {
  gs_status s;
  if ((s = check_batch(batch))) return s;
  if (!ws_bytes || n_gaussians < 0) return fail(GS_ERR_ARG, "gs_render_bwd_workspace: bad argument");
  *ws_bytes = v2d_bytes(n_gaussians, *batch) + pose_partial_bytes(n_gaussians, *batch);
  return GS_OK;
}

namespace {
gs_status check_bwd_common(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                           const gs_projected* proj, void* ws, size_t ws_bytes, const char* who) {
  gs_status s;
  if ((s = check_gaussians(g)) || (s = check_cameras(cams)) || (s = check_batch(batch)) ||
      (s = check_projected(proj)))
    return s;
  if (!ws) return fail(GS_ERR_ARG, "%s: null workspace", who);
  if (!aligned(ws, 256)) return fail(GS_ERR_ARG, "%s: ws must be 256-byte aligned", who);
  const size_t need = v2d_bytes(g->n, *batch) + pose_partial_bytes(g->n, *batch);
  if (ws_bytes < need) return fail(GS_ERR_ARG, "%s: workspace %zu < %zu bytes", who, ws_bytes, need);
  return GS_OK;
}
}  // namespace

namespace {
gs_status raster_bwd(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                     const gs_projected* proj, const uint32_t* vals, const uint32_t* ranges, const float* bg,
                     const float* image, const float* T_final, const uint32_t* n_contrib, const float* v_image,
                     const float* target, float l1_weight, double* loss, void* ws, size_t ws_bytes,
                     gs_stream stream, bool zero, const char* who) {
  gs_status s;
  if ((s = check_bwd_common(g, cams, batch, proj, ws, ws_bytes, who))) return s;
  if (!vals || !ranges || !bg || !T_final || !n_contrib) return fail(GS_ERR_ARG, "%s: null argument", who);
  if (!v_image && (!target || !image))
    return fail(GS_ERR_ARG, "%s: need v_image, or image and target for the fused L1", who);
  if (!v_image && !std::isfinite(l1_weight)) return fail(GS_ERR_NONFINITE, "%s: l1_weight", who);
  cudaStream_t st = (cudaStream_t)stream;
  float* v2d = reinterpret_cast<float*>(ws);
  cudaError_t e;
  if (zero) {
    e = cudaMemsetAsync(v2d, 0, (size_t)batch->B * g->n * 12 * sizeof(float), st);
    if (e != cudaSuccess) return cuda_fail(e, who);
  }
  e = launch_render_bwd(*batch, *cams, *proj, vals, ranges, bg, image, T_final, n_contrib, v_image,
                        target, l1_weight, loss, v2d, st);
  if (e != cudaSuccess) return cuda_fail(e, who);
  return GS_OK;
}
}  // namespace

gs_status gs_raster_bwd(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                        const gs_projected* proj, const uint32_t* vals, const uint32_t* ranges,
                        const float* bg, const float* image, const float* T_final,
                        const uint32_t* n_contrib, const float* v_image, const float* target,
                        float l1_weight, double* loss, void* ws, size_t ws_bytes, gs_stream stream) {
  return raster_bwd(g, cams, batch, proj, vals, ranges, bg, image, T_final, n_contrib, v_image, target, l1_weight,
                    loss, ws, ws_bytes, stream, true, "gs_raster_bwd");
}

gs_status gs_raster_bwd_zeroed(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                               const gs_projected* proj, const uint32_t* vals, const uint32_t* ranges,
                               const float* bg, const float* image, const float* T_final,
                               const uint32_t* n_contrib, const float* v_image, const float* target,
                               float l1_weight, double* loss, void* ws, size_t ws_bytes, gs_stream stream) {
  return raster_bwd(g, cams, batch, proj, vals, ranges, bg, image, T_final, n_contrib, v_image, target, l1_weight,
                    loss, ws, ws_bytes, stream, false, "gs_raster_bwd_zeroed");
}

static gs_status project_bwd_call(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                                  const gs_projected* proj, const gs_gaussian_grads* dg, double* g_pose_tangent,
                                  void* ws, size_t ws_bytes, gs_stream stream, bool clear, const char* who) {
  gs_status s;
  if ((s = check_bwd_common(g, cams, batch, proj, ws, ws_bytes, who))) return s;
  if (!dg || !g_pose_tangent) return fail(GS_ERR_ARG, "gs_project_bwd: null argument");
  if (!dg->mean || !dg->log_scale || !dg->quat || !dg->opacity_logit || !dg->sh)
    return fail(GS_ERR_ARG, "gs_project_bwd: null gradient array");
  if (!aligned(dg->quat, 16)) return fail(GS_ERR_ARG, "gs_project_bwd: grad quat must be 16-byte aligned");
  const size_t vb = v2d_bytes(g->n, *batch);
  float* v2d = reinterpret_cast<float*>(ws);
  double* partial = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + vb);
  cudaError_t e = launch_project_bwd(*g, *cams, *batch, *proj, v2d, *dg, partial, g_pose_tangent, clear,
                                     (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, who);
  return GS_OK;
}

gs_status gs_project_bwd(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                         const gs_projected* proj, const gs_gaussian_grads* dg, double* g_pose_tangent,
                         void* ws, size_t ws_bytes, gs_stream stream) {
  return project_bwd_call(g, cams, batch, proj, dg, g_pose_tangent, ws, ws_bytes, stream, false, "gs_project_bwd");
}

gs_status gs_project_bwd_clearing(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                                  const gs_projected* proj, const gs_gaussian_grads* dg, double* g_pose_tangent,
                                  void* ws, size_t ws_bytes, gs_stream stream) {
  return project_bwd_call(g, cams, batch, proj, dg, g_pose_tangent, ws, ws_bytes, stream, true,
                          "gs_project_bwd_clearing");
}

gs_status gs_render_bwd(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                        const gs_projected* proj, const uint32_t* vals, const uint32_t* ranges,
                        const float* bg, const float* image, const float* T_final,
                        const uint32_t* n_contrib, const float* v_image, const float* target,
                        float l1_weight, double* loss, const gs_gaussian_grads* dg,
                        double* g_pose_tangent, void* ws, size_t ws_bytes, gs_stream stream) {
  if (!dg || !g_pose_tangent) return fail(GS_ERR_ARG, "gs_render_bwd: null argument");
  gs_status s = gs_raster_bwd(g, cams, batch, proj, vals, ranges, bg, image, T_final, n_contrib, v_image,
                              target, l1_weight, loss, ws, ws_bytes, stream);
  if (s != GS_OK) return s;
  return gs_project_bwd(g, cams, batch, proj, dg, g_pose_tangent, ws, ws_bytes, stream);
}

namespace {
size_t det_ws_bytes(int N, const gs_batch& b, size_t capacity) {
  return v2d_bytes(N, b) + pose_partial_bytes(N, b) + render_bwd_det_bytes((size_t)b.B * N, b.n_tiles, capacity);
}
}  // namespace

gs_status gs_render_bwd_det_workspace(int32_t n_gaussians, const gs_batch* batch, size_t capacity,
                                      size_t* ws_bytes) {
  gs_status s;
  if ((s = check_batch(batch))) return s;
  if (!ws_bytes || n_gaussians < 0) return fail(GS_ERR_ARG, "gs_render_bwd_det_workspace: bad argument");
  if (capacity > 0xffffffffull) return fail(GS_ERR_ARG, "gs_render_bwd_det_workspace: capacity above 2^32 - 1");
  *ws_bytes = det_ws_bytes(n_gaussians, *batch, capacity);
  return GS_OK;
}

gs_status gs_raster_bwd_det(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                            const gs_projected* proj, const uint32_t* vals, const uint32_t* ranges,
                            const uint32_t* n_instances, const float* bg, const float* image, const float* T_final,
                            const uint32_t* n_contrib, const float* v_image, const float* target,
                            float l1_weight, double* loss, size_t capacity, void* ws, size_t ws_bytes,
                            gs_stream stream) {
  gs_status s;
  if ((s = check_bwd_common(g, cams, batch, proj, ws, ws_bytes, "gs_raster_bwd_det"))) return s;
  if (!vals || !ranges || !n_instances || !bg || !T_final || !n_contrib)
    return fail(GS_ERR_ARG, "gs_raster_bwd_det: null argument");
  if (!v_image && (!target || !image))
    return fail(GS_ERR_ARG, "gs_raster_bwd_det: need v_image, or image and target for the fused L1");
  if (!v_image && !std::isfinite(l1_weight)) return fail(GS_ERR_NONFINITE, "gs_raster_bwd_det: l1_weight");
  if (capacity > 0xffffffffull) return fail(GS_ERR_ARG, "gs_raster_bwd_det: capacity above 2^32 - 1");
  const size_t need = det_ws_bytes(g->n, *batch, capacity);
  if (ws_bytes < need) return fail(GS_ERR_ARG, "gs_raster_bwd_det: workspace %zu < %zu bytes", ws_bytes, need);
  char* w = static_cast<char*>(ws);
  float* v2d = reinterpret_cast<float*>(w);
  void* det = w + v2d_bytes(g->n, *batch) + pose_partial_bytes(g->n, *batch);
  const cudaError_t e = launch_render_bwd_det(*batch, *cams, *proj, (size_t)batch->B * g->n, vals, ranges,
                                              n_instances, bg, image, T_final, n_contrib, v_image, target,
                                              l1_weight, loss, v2d, det, capacity, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_raster_bwd_det");
  return GS_OK;
}

gs_status gs_render_bwd_det(const gs_gaussians* g, const gs_cameras* cams, const gs_batch* batch,
                            const gs_projected* proj, const uint32_t* vals, const uint32_t* ranges,
                            const uint32_t* n_instances, const float* bg, const float* image, const float* T_final,
                            const uint32_t* n_contrib, const float* v_image, const float* target,
                            float l1_weight, double* loss, size_t capacity, const gs_gaussian_grads* dg,
                            double* g_pose_tangent, void* ws, size_t ws_bytes, gs_stream stream) {
  if (!dg || !g_pose_tangent) return fail(GS_ERR_ARG, "gs_render_bwd_det: null argument");
  gs_status s = gs_raster_bwd_det(g, cams, batch, proj, vals, ranges, n_instances, bg, image, T_final,
                                  n_contrib, v_image, target, l1_weight, loss, capacity, ws, ws_bytes, stream);
  if (s != GS_OK) return s;
  return gs_project_bwd(g, cams, batch, proj, dg, g_pose_tangent, ws, ws_bytes, stream);
}

/* ---- FP64 instantiation of the projection and compositing -------------- */

gs_status gs_project_f64(const gs_gaussians_f64* g, const gs_cameras_f64* cams, const gs_batch* batch,
                         const gs_projected_f64* out, int32_t* status, gs_stream stream) {
  gs_status s;
  if ((s = check_gaussians(g)) || (s = check_cameras(cams)) || (s = check_batch(batch)) ||
      (s = check_projected(out)))
    return s;
  if ((unsigned long long)batch->B * (unsigned long long)g->n >= 0xffffffffull)
    return fail(GS_ERR_ARG, "gs_project_f64: B*N must be < 2^32");
  cudaError_t e = launch_project_fwd_f64(*g, *cams, *batch, *out, status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_project_f64");
  return GS_OK;
}

gs_status gs_sort_tiles_f64(int32_t n_gaussians, const gs_cameras_f64* cams, const gs_batch* batch,
                            const gs_projected_f64* proj, uint32_t* tiles, uint32_t* vals, size_t capacity,
                            uint32_t* ranges, uint32_t* n_instances, void* ws, size_t ws_bytes, int32_t* status,
                            gs_stream stream) {
  gs_status s;
  if ((s = check_cameras(cams)) || (s = check_projected(proj))) return s;
  // the sort reads only the image sizes of the cameras and the rectangles,
  // tile counts and depth keys of the records, which both paths share
  gs_cameras c32{cams->n_cams, cams->wh, reinterpret_cast<const float*>(cams->K),
                 reinterpret_cast<const float*>(cams->Rt), 0.01f, 1e10f};
  gs_projected p32{reinterpret_cast<float*>(proj->splat), proj->rect, proj->n_tiles, proj->depth_key};
  return gs_sort_tiles(n_gaussians, &c32, batch, &p32, tiles, vals, capacity, ranges, n_instances, ws, ws_bytes,
                       status, stream);
}

gs_status gs_render_fwd_f64(const gs_batch* batch, const gs_cameras_f64* cams, const gs_projected_f64* proj,
                            const uint32_t* vals, const uint32_t* ranges, const double* bg, double* image,
                            double* T_final, uint32_t* n_contrib, uint32_t* n_added, gs_stream stream) {
  gs_status s;
  if ((s = check_batch(batch)) || (s = check_cameras(cams)) || (s = check_projected(proj))) return s;
  if (!vals || !ranges || !bg || !image || !T_final || !n_contrib)
    return fail(GS_ERR_ARG, "gs_render_fwd_f64: null argument");
  cudaError_t e = launch_render_fwd_f64(*batch, *cams, *proj, vals, ranges, bg, image, T_final, n_contrib,
                                        n_added, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_render_fwd_f64");
  return GS_OK;
}

gs_status gs_render_bwd_workspace_f64(int32_t n_gaussians, const gs_batch* batch, size_t* ws_bytes) {
  gs_status s;
  if ((s = check_batch(batch))) return s;
  if (!ws_bytes || n_gaussians < 0) return fail(GS_ERR_ARG, "gs_render_bwd_workspace_f64: bad argument");
  *ws_bytes = v2d_bytes_f64(n_gaussians, *batch) + pose_partial_bytes(n_gaussians, *batch);
  return GS_OK;
}

namespace {
gs_status check_bwd_common_f64(const gs_gaussians_f64* g, const gs_cameras_f64* cams, const gs_batch* batch,
                               const gs_projected_f64* proj, void* ws, size_t ws_bytes, const char* who) {
  gs_status s;
  if ((s = check_gaussians(g)) || (s = check_cameras(cams)) || (s = check_batch(batch)) ||
      (s = check_projected(proj)))
    return s;
  if (!ws) return fail(GS_ERR_ARG, "%s: null workspace", who);
  if (!aligned(ws, 256)) return fail(GS_ERR_ARG, "%s: ws must be 256-byte aligned", who);
  const size_t need = v2d_bytes_f64(g->n, *batch) + pose_partial_bytes(g->n, *batch);
  if (ws_bytes < need) return fail(GS_ERR_ARG, "%s: workspace %zu < %zu bytes", who, ws_bytes, need);
  return GS_OK;
}
}  // namespace

gs_status gs_raster_bwd_f64(const gs_gaussians_f64* g, const gs_cameras_f64* cams, const gs_batch* batch,
                            const gs_projected_f64* proj, const uint32_t* vals, const uint32_t* ranges,
                            const double* bg, const double* image, const double* T_final,
                            const uint32_t* n_contrib, const double* v_image, const double* target,
                            double l1_weight, double* loss, void* ws, size_t ws_bytes, gs_stream stream) {
  gs_status s;
  if ((s = check_bwd_common_f64(g, cams, batch, proj, ws, ws_bytes, "gs_raster_bwd_f64"))) return s;
  if (!vals || !ranges || !bg || !T_final || !n_contrib)
    return fail(GS_ERR_ARG, "gs_raster_bwd_f64: null argument");
  if (!v_image && (!target || !image))
    return fail(GS_ERR_ARG, "gs_raster_bwd_f64: need v_image, or image and target for the fused L1");
  if (!v_image && !std::isfinite(l1_weight)) return fail(GS_ERR_NONFINITE, "gs_raster_bwd_f64: l1_weight");
  cudaStream_t st = (cudaStream_t)stream;
  double* v2d = reinterpret_cast<double*>(ws);
  cudaError_t e = cudaMemsetAsync(v2d, 0, (size_t)batch->B * g->n * 12 * sizeof(double), st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_raster_bwd_f64 memset");
  e = launch_render_bwd_f64(*batch, *cams, *proj, vals, ranges, bg, image, T_final, n_contrib, v_image, target,
                            l1_weight, loss, v2d, st);
  if (e != cudaSuccess) return cuda_fail(e, "gs_raster_bwd_f64");
  return GS_OK;
}

gs_status gs_project_bwd_f64(const gs_gaussians_f64* g, const gs_cameras_f64* cams, const gs_batch* batch,
                             const gs_projected_f64* proj, const gs_gaussian_grads_f64* dg, double* g_pose_tangent,
                             void* ws, size_t ws_bytes, gs_stream stream) {
  gs_status s;
  if ((s = check_bwd_common_f64(g, cams, batch, proj, ws, ws_bytes, "gs_project_bwd_f64"))) return s;
  if (!dg || !g_pose_tangent) return fail(GS_ERR_ARG, "gs_project_bwd_f64: null argument");
  if (!dg->mean || !dg->log_scale || !dg->quat || !dg->opacity_logit || !dg->sh)
    return fail(GS_ERR_ARG, "gs_project_bwd_f64: null gradient array");
  if (!aligned(dg->quat, 16)) return fail(GS_ERR_ARG, "gs_project_bwd_f64: grad quat must be 16-byte aligned");
  const size_t vb = v2d_bytes_f64(g->n, *batch);
  double* v2d = reinterpret_cast<double*>(ws);
  double* partial = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + vb);
  cudaError_t e = launch_project_bwd_f64(*g, *cams, *batch, *proj, v2d, *dg, partial, g_pose_tangent,
                                         (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_project_bwd_f64");
  return GS_OK;
}

gs_status gs_render_bwd_f64(const gs_gaussians_f64* g, const gs_cameras_f64* cams, const gs_batch* batch,
                            const gs_projected_f64* proj, const uint32_t* vals, const uint32_t* ranges,
                            const double* bg, const double* image, const double* T_final,
                            const uint32_t* n_contrib, const double* v_image, const double* target,
                            double l1_weight, double* loss, const gs_gaussian_grads_f64* dg,
                            double* g_pose_tangent, void* ws, size_t ws_bytes, gs_stream stream) {
  if (!dg || !g_pose_tangent) return fail(GS_ERR_ARG, "gs_render_bwd_f64: null argument");
  gs_status s = gs_raster_bwd_f64(g, cams, batch, proj, vals, ranges, bg, image, T_final, n_contrib, v_image,
                                  target, l1_weight, loss, ws, ws_bytes, stream);
  if (s != GS_OK) return s;
  return gs_project_bwd_f64(g, cams, batch, proj, dg, g_pose_tangent, ws, ws_bytes, stream);
}

gs_status pose_se3_update_f64(int32_t n_cams, const double* T0, double* xi, const double* g_tangent,
                              double* g_xi, double* m, double* v, const gs_adam* hp, double* Rt_out,
                              gs_stream stream) {
  if (n_cams < 0 || (n_cams > 0 && (!T0 || !xi || !g_tangent || !Rt_out)))
    return fail(GS_ERR_ARG, "pose_se3_update_f64: null argument");
  if (hp) {
    if (!m || !v || !hp->step) return fail(GS_ERR_ARG, "pose_se3_update_f64: Adam needs m, v and step");
    if (!std::isfinite(hp->lr) || !std::isfinite(hp->beta1) || !std::isfinite(hp->beta2) ||
        !std::isfinite(hp->eps))
      return fail(GS_ERR_NONFINITE, "pose_se3_update_f64: non-finite hyperparameter");
  }
  cudaError_t e = launch_pose_update_f64(n_cams, T0, xi, g_tangent, g_xi, m, v, hp, Rt_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pose_se3_update_f64");
  return GS_OK;
}

gs_status track_reproj_workspace(const gs_batch* batch, size_t* ws_bytes) {
  gs_status s;
  if ((s = check_batch(batch))) return s;
  if (!ws_bytes) return fail(GS_ERR_ARG, "track_reproj_workspace: null");
  *ws_bytes = align_up(track_workspace_bytes(*batch));
  return GS_OK;
}

namespace {
gs_status track_call(const float* X, int32_t n_points, const int32_t* obs_point, const float* obs_xy,
                     const int64_t* view_obs_offset, const gs_cameras* cams, const gs_batch* batch, float delta,
                     float weight, double* loss, float* grad_X, double* g_pose_tangent, uint32_t* n_masked,
                     void* ws, size_t ws_bytes, gs_stream stream, bool det, const char* who) {
  gs_status s;
  if ((s = check_cameras(cams)) || (s = check_batch(batch))) return s;
  if (n_points < 0 || !view_obs_offset || !grad_X || !g_pose_tangent || !ws)
    return fail(GS_ERR_ARG, "%s: null argument", who);
  if (n_points > 0 && (!X || !obs_point || !obs_xy)) return fail(GS_ERR_ARG, "%s: null array", who);
  if (obs_xy && !aligned(obs_xy, 8)) return fail(GS_ERR_ARG, "%s: obs_xy must be 8-byte aligned", who);
  if (!std::isfinite(delta) || !std::isfinite(weight))
    return fail(GS_ERR_NONFINITE, "%s: non-finite delta/weight", who);
  if (!(delta > 0.f)) return fail(GS_ERR_ARG, "%s: delta must be > 0", who);
  if (ws_bytes < track_workspace_bytes(*batch)) return fail(GS_ERR_ARG, "%s: workspace too small", who);
  cudaError_t e = (det ? launch_track_det : launch_track)(X, n_points, obs_point, obs_xy, view_obs_offset, *cams,
                                                           *batch, delta, weight, loss, grad_X, g_pose_tangent,
                                                           n_masked, ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, who);
  return GS_OK;
}
}  // namespace

gs_status track_reproj_fwd_bwd(const float* X, int32_t n_points, const int32_t* obs_point,
                               const float* obs_xy, const int64_t* view_obs_offset,
                               const gs_cameras* cams, const gs_batch* batch, float delta,
                               float weight, double* loss, float* grad_X, double* g_pose_tangent,
                               uint32_t* n_masked, void* ws, size_t ws_bytes, gs_stream stream) {
  return track_call(X, n_points, obs_point, obs_xy, view_obs_offset, cams, batch, delta, weight, loss, grad_X,
                    g_pose_tangent, n_masked, ws, ws_bytes, stream, false, "track_reproj_fwd_bwd");
}

gs_status track_reproj_fwd_bwd_det(const float* X, int32_t n_points, const int32_t* obs_point,
                                   const float* obs_xy, const int64_t* view_obs_offset,
                                   const gs_cameras* cams, const gs_batch* batch, float delta,
                                   float weight, double* loss, float* grad_X, double* g_pose_tangent,
                                   uint32_t* n_masked, void* ws, size_t ws_bytes, gs_stream stream) {
  return track_call(X, n_points, obs_point, obs_xy, view_obs_offset, cams, batch, delta, weight, loss, grad_X,
                    g_pose_tangent, n_masked, ws, ws_bytes, stream, true, "track_reproj_fwd_bwd_det");
}

gs_status pose_se3_update(int32_t n_cams, const float* T0, float* xi, const double* g_tangent,
                          float* g_xi, float* m, float* v, const gs_adam* hp, float* Rt_out,
                          gs_stream stream) {
  if (n_cams < 0 || (n_cams > 0 && (!T0 || !xi || !g_tangent || !Rt_out)))
    return fail(GS_ERR_ARG, "pose_se3_update: null argument");
  if (hp) {
    if (!m || !v || !hp->step) return fail(GS_ERR_ARG, "pose_se3_update: Adam needs m, v and step");
    if (!std::isfinite(hp->lr) || !std::isfinite(hp->beta1) || !std::isfinite(hp->beta2) ||
        !std::isfinite(hp->eps))
      return fail(GS_ERR_NONFINITE, "pose_se3_update: non-finite hyperparameter");
  }
  cudaError_t e = launch_pose_update(n_cams, T0, xi, g_tangent, g_xi, m, v, hp, Rt_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pose_se3_update");
  return GS_OK;
}

gs_status gs_adam_update(float* p, const float* g, float* m, float* v, int64_t n, const gs_adam* hp,
                         gs_stream stream) {
  if (n < 0 || !hp || (n > 0 && (!p || !g || !m || !v)) || !hp->step)
    return fail(GS_ERR_ARG, "gs_adam_update: bad argument");
  if (!std::isfinite(hp->lr) || !std::isfinite(hp->beta1) || !std::isfinite(hp->beta2) ||
      !std::isfinite(hp->eps))
    return fail(GS_ERR_NONFINITE, "gs_adam_update: non-finite hyperparameter");
  cudaError_t e = launch_adam(p, g, m, v, n, *hp, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_adam_update");
  return GS_OK;
}

gs_status gs_adam_update_groups(const gs_adam_group* groups, int32_t n_groups, const gs_adam* hp,
                                gs_stream stream) {
  if (!groups || !hp || !hp->step || n_groups < 0 || n_groups > 8)
    return fail(GS_ERR_ARG, "gs_adam_update_groups: bad argument (1..8 groups)");
  if (!std::isfinite(hp->beta1) || !std::isfinite(hp->beta2) || !std::isfinite(hp->eps))
    return fail(GS_ERR_NONFINITE, "gs_adam_update_groups: non-finite hyperparameter");
  for (int i = 0; i < n_groups; ++i) {
    const gs_adam_group& a = groups[i];
    if (a.n < 0 || (a.n > 0 && (!a.p || !a.g || !a.m || !a.v)))
      return fail(GS_ERR_ARG, "gs_adam_update_groups: bad group %d", i);
    if (!std::isfinite(a.lr)) return fail(GS_ERR_NONFINITE, "gs_adam_update_groups: non-finite lr in group %d", i);
  }
  cudaError_t e = launch_adam_groups(groups, n_groups, *hp, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_adam_update_groups");
  return GS_OK;
}

gs_status gs_step_advance(int32_t* step, gs_stream stream) {
  if (!step) return fail(GS_ERR_ARG, "gs_step_advance: null");
  cudaError_t e = launch_step_advance(step, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_step_advance");
  return GS_OK;
}

gs_status gs_batch_layout(const gs_cameras* cams, const gs_batch* batch, int64_t* px_offset,
                          int32_t* tile_offset, int32_t* status, gs_stream stream) {
  gs_status s;
  if ((s = check_cameras(cams)) || (s = check_batch(batch))) return s;
  if (!px_offset || !tile_offset) return fail(GS_ERR_ARG, "gs_batch_layout: null offset array");
  if (!aligned(px_offset, 8) || !aligned(tile_offset, 4))
    return fail(GS_ERR_ARG, "gs_batch_layout: px_offset must be 8-byte, tile_offset 4-byte aligned");
  cudaError_t e = launch_batch_layout(*cams, *batch, px_offset, tile_offset, status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_batch_layout");
  return GS_OK;
}

gs_status gs_photo_loss_workspace(const gs_batch* batch, size_t* ws_bytes) {
  gs_status s;
  if ((s = check_batch(batch))) return s;
  if (!ws_bytes) return fail(GS_ERR_ARG, "gs_photo_loss_workspace: null ws_bytes");
  *ws_bytes = photo_loss_ws_bytes(batch->n_pixels, batch->n_tiles);
  return GS_OK;
}

gs_status gs_photo_loss(const gs_cameras* cams, const gs_batch* batch, const float* image, const float* target,
                        float l1_weight, float ssim_weight, double* loss, float* v_image, void* ws,
                        size_t ws_bytes, gs_stream stream) {
  gs_status s;
  if ((s = check_cameras(cams)) || (s = check_batch(batch))) return s;
  if (!image || !target || !v_image) return fail(GS_ERR_ARG, "gs_photo_loss: null image, target or v_image");
  if (!std::isfinite(l1_weight) || !std::isfinite(ssim_weight) || l1_weight < 0.f || ssim_weight < 0.f)
    return fail(GS_ERR_ARG, "gs_photo_loss: weights must be finite and >= 0");
  // the kernels index a view's values with 32-bit offsets
  if (batch->n_pixels > (int64_t)(INT32_MAX / 3))
    return fail(GS_ERR_UNSUPPORTED, "gs_photo_loss: more than %d pixels in the batch", INT32_MAX / 3);
  const size_t need = photo_loss_ws_bytes(batch->n_pixels, batch->n_tiles);
  if (batch->n_pixels > 0 && (!ws || ws_bytes < need))
    return fail(GS_ERR_ARG, "gs_photo_loss: workspace needs %zu bytes", need);
  if (!aligned(ws, 4)) return fail(GS_ERR_ARG, "gs_photo_loss: workspace must be 4-byte aligned");
  cudaError_t e = launch_photo_loss(*batch, *cams, image, target, l1_weight, ssim_weight, loss, v_image,
                                    reinterpret_cast<float*>(ws), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_photo_loss");
  return GS_OK;
}

gs_status sfm_ba_assemble(const float* X, int32_t n_points, const gs_cameras* cams, const int32_t* obs_point,
                          const int32_t* obs_cam, const float* obs_xy, int64_t n_obs, float delta, double* U,
                          double* Vp, double* gc, double* gp, double* Wo, double* objective, gs_stream stream) {
  gs_status s;
  if ((s = check_cameras(cams))) return s;
  if (n_points < 0 || n_obs < 0) return fail(GS_ERR_ARG, "sfm_ba_assemble: negative sizes");
  if (!U || !gc) return fail(GS_ERR_ARG, "sfm_ba_assemble: null camera blocks");
  if (n_points > 0 && (!X || !Vp || !gp)) return fail(GS_ERR_ARG, "sfm_ba_assemble: null point arrays");
  if (n_obs > 0 && (!obs_point || !obs_cam || !obs_xy || !Wo))
    return fail(GS_ERR_ARG, "sfm_ba_assemble: null observation arrays");
  if (!aligned(obs_xy, 8)) return fail(GS_ERR_ARG, "sfm_ba_assemble: obs_xy must be 8-byte aligned");
  if (!std::isfinite(delta) || delta <= 0.f) return fail(GS_ERR_ARG, "sfm_ba_assemble: delta must be > 0");
  cudaError_t e = launch_ba_assemble(X, n_points, *cams, obs_point, obs_cam, obs_xy, n_obs, delta, U, Vp, gc, gp,
                                     Wo, objective, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sfm_ba_assemble");
  return GS_OK;
}

gs_status sfm_ba_schur(int32_t n_cams, int32_t n_points, int64_t n_obs, const double* U, const double* Vp,
                       const double* gc, const double* gp, const double* Wo, const int32_t* obs_cam,
                       const int64_t* point_obs_offset, const int32_t* point_obs, double lambda,
                       const double* lambda_dev, double* S, double* rhs, double* Vinv, gs_stream stream) {
  if (n_cams < 0 || n_points < 0 || n_obs < 0) return fail(GS_ERR_ARG, "sfm_ba_schur: negative sizes");
  if (n_cams > 0 && (!U || !gc || !S || !rhs)) return fail(GS_ERR_ARG, "sfm_ba_schur: null camera arrays");
  if (n_points > 0 && (!Vp || !gp || !Vinv || !point_obs_offset || (n_obs > 0 && (!Wo || !obs_cam || !point_obs))))
    return fail(GS_ERR_ARG, "sfm_ba_schur: null point or observation arrays");
  if (!lambda_dev && (!std::isfinite(lambda) || lambda < 0.0))
    return fail(GS_ERR_ARG, "sfm_ba_schur: lambda must be >= 0");
  cudaError_t e = launch_ba_schur(n_cams, n_points, n_obs, U, Vp, gc, gp, Wo, obs_cam, point_obs_offset, point_obs,
                                  lambda, lambda_dev, S, rhs, Vinv, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sfm_ba_schur");
  return GS_OK;
}

gs_status sfm_ba_pair_lists(int32_t n_cams, int32_t n_points, int64_t n_obs, const int32_t* obs_cam,
                            const int64_t* point_obs_offset, const int32_t* point_obs, int32_t chunk, int64_t* n_inc,
                            int32_t* n_pairs, int32_t* n_chunks, int32_t* inc, int32_t* pair_cams,
                            int32_t* pair_chunks, int64_t* chunk_start) {
  if (n_cams < 0 || n_points < 0 || n_obs < 0) return fail(GS_ERR_ARG, "sfm_ba_pair_lists: negative sizes");
  if (chunk <= 0) return fail(GS_ERR_ARG, "sfm_ba_pair_lists: chunk must be > 0");
  if (!n_inc || !n_pairs || !n_chunks) return fail(GS_ERR_ARG, "sfm_ba_pair_lists: null size outputs");
  if (n_points > 0 && (!point_obs_offset || (n_obs > 0 && (!obs_cam || !point_obs))))
    return fail(GS_ERR_ARG, "sfm_ba_pair_lists: null inputs");
  const bool fill = inc && pair_cams && pair_chunks && chunk_start;
  *n_inc = gs::ba_pair_plan(n_cams, n_points, n_obs, obs_cam, point_obs_offset, point_obs, chunk, n_pairs, n_chunks,
                            fill ? inc : nullptr, fill ? pair_cams : nullptr, fill ? pair_chunks : nullptr,
                            fill ? chunk_start : nullptr);
  return GS_OK;
}

gs_status sfm_ba_schur_pairs_workspace(int64_t n_obs, int32_t n_chunks, size_t* bytes) {
  if (n_obs < 0 || n_chunks < 0 || !bytes) return fail(GS_ERR_ARG, "sfm_ba_schur_pairs_workspace: bad arguments");
  *bytes = gs::ba_schur_pairs_workspace_bytes(n_obs, n_chunks);
  return GS_OK;
}

gs_status sfm_ba_schur_pairs(int32_t n_cams, int32_t n_points, int64_t n_obs, const double* U, const double* Vp,
                             const double* gc, const double* gp, const double* Wo, const int32_t* obs_cam,
                             const int64_t* point_obs_offset, const int32_t* point_obs, const int32_t* inc,
                             const int32_t* pair_cams, int32_t n_pairs, const int32_t* pair_chunks,
                             const int64_t* chunk_start, int32_t n_chunks, double lambda, const double* lambda_dev,
                             double* S, double* rhs, double* Vinv, void* ws, size_t ws_bytes, gs_stream stream) {
  if (n_cams < 0 || n_points < 0 || n_obs < 0 || n_pairs < 0 || n_chunks < 0)
    return fail(GS_ERR_ARG, "sfm_ba_schur_pairs: negative sizes");
  if (n_cams > 0 && (!U || !gc || !S || !rhs)) return fail(GS_ERR_ARG, "sfm_ba_schur_pairs: null camera arrays");
  if (n_points > 0 && (!Vp || !gp || !Vinv || !point_obs_offset || (n_obs > 0 && (!Wo || !obs_cam || !point_obs))))
    return fail(GS_ERR_ARG, "sfm_ba_schur_pairs: null point or observation arrays");
  if (n_chunks > 0 && (!inc || !pair_cams || !pair_chunks || !chunk_start))
    return fail(GS_ERR_ARG, "sfm_ba_schur_pairs: null plan arrays");
  if (!lambda_dev && (!std::isfinite(lambda) || lambda < 0.0))
    return fail(GS_ERR_ARG, "sfm_ba_schur_pairs: lambda must be >= 0");
  if (n_points > 0 && n_obs > 0 && (!ws || ws_bytes < gs::ba_schur_pairs_workspace_bytes(n_obs, n_chunks)))
    return fail(GS_ERR_ARG, "sfm_ba_schur_pairs: workspace too small");
  cudaError_t e = gs::launch_ba_schur_pairs(n_cams, n_points, n_obs, U, Vp, gc, gp, Wo, obs_cam, point_obs_offset,
                                            point_obs, inc, pair_cams, n_pairs, pair_chunks, chunk_start, n_chunks,
                                            lambda, lambda_dev, S, rhs, Vinv, ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sfm_ba_schur_pairs");
  return GS_OK;
}

gs_status sfm_ba_lm_accept(int32_t n_cams, int32_t n_points, double* objective, double* lambda, float* Rt, float* X,
                           const float* Rt_trial, const float* X_trial, int32_t* n_accepted, double* history,
                           int32_t history_len, int32_t* n_iter, gs_stream stream) {
  if (n_cams < 0 || n_points < 0 || history_len < 0) return fail(GS_ERR_ARG, "sfm_ba_lm_accept: negative sizes");
  if (!objective || !lambda) return fail(GS_ERR_ARG, "sfm_ba_lm_accept: null objective or lambda");
  if ((n_cams > 0 && (!Rt || !Rt_trial)) || (n_points > 0 && (!X || !X_trial)))
    return fail(GS_ERR_ARG, "sfm_ba_lm_accept: null parameter arrays");
  if (history && !n_iter) return fail(GS_ERR_ARG, "sfm_ba_lm_accept: history needs n_iter");
  cudaError_t e = launch_ba_lm_accept(n_cams, n_points, objective, lambda, Rt, X, Rt_trial, X_trial, n_accepted,
                                      history, history_len, n_iter, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sfm_ba_lm_accept");
  return GS_OK;
}

gs_status sfm_ba_objective(const float* X, int32_t n_points, const gs_cameras* cams, const int32_t* obs_point,
                           const int32_t* obs_cam, const float* obs_xy, int64_t n_obs, float delta, double* objective,
                           gs_stream stream) {
  gs_status s;
  if ((s = check_cameras(cams))) return s;
  if (n_points < 0 || n_obs < 0) return fail(GS_ERR_ARG, "sfm_ba_objective: negative sizes");
  if (!objective) return fail(GS_ERR_ARG, "sfm_ba_objective: null objective");
  if (n_obs > 0 && (!obs_point || !obs_cam || !obs_xy || (n_points > 0 && !X)))
    return fail(GS_ERR_ARG, "sfm_ba_objective: null observation arrays");
  if (!aligned(obs_xy, 8)) return fail(GS_ERR_ARG, "sfm_ba_objective: obs_xy must be 8-byte aligned");
  if (!std::isfinite(delta) || delta <= 0.f) return fail(GS_ERR_ARG, "sfm_ba_objective: delta must be > 0");
  cudaError_t e = launch_ba_assemble(X, n_points, *cams, obs_point, obs_cam, obs_xy, n_obs, delta, nullptr, nullptr,
                                     nullptr, nullptr, nullptr, objective, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sfm_ba_objective");
  return GS_OK;
}

gs_status sfm_ba_apply_step(int32_t n_cams, int32_t n_points, const float* Rt, const float* X, const double* dc,
                            const double* dp, float* Rt_out, float* X_out, gs_stream stream) {
  if (n_cams < 0 || n_points < 0) return fail(GS_ERR_ARG, "sfm_ba_apply_step: negative sizes");
  if ((n_cams > 0 && (!Rt || !dc || !Rt_out)) || (n_points > 0 && (!X || !dp || !X_out)))
    return fail(GS_ERR_ARG, "sfm_ba_apply_step: null argument");
  if ((n_cams > 0 && Rt == Rt_out) || (n_points > 0 && X == X_out))
    return fail(GS_ERR_ARG, "sfm_ba_apply_step: outputs alias inputs");
  cudaError_t e = launch_ba_apply(n_cams, n_points, Rt, X, dc, dp, Rt_out, X_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sfm_ba_apply_step");
  return GS_OK;
}

gs_status sfm_ba_solve_cameras(int32_t n_cams, double* S, const double* rhs, double* dc, int32_t* status,
                               gs_stream stream) {
  if (n_cams < 0) return fail(GS_ERR_ARG, "sfm_ba_solve_cameras: negative n_cams");
  if (n_cams > 0 && (!S || !rhs || !dc)) return fail(GS_ERR_ARG, "sfm_ba_solve_cameras: null argument");
  if (n_cams > GS_MAX_BA_CAMERAS)
    return fail(GS_ERR_UNSUPPORTED, "sfm_ba_solve_cameras: more than %d cameras", GS_MAX_BA_CAMERAS);
  cudaError_t e = launch_ba_solve_cameras(n_cams, S, rhs, dc, status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sfm_ba_solve_cameras");
  return GS_OK;
}

gs_status sfm_ba_back_substitute(int32_t n_cams, int32_t n_points, int64_t n_obs, const double* Vinv,
                                 const double* Vp, const double* gp, const double* Wo, const int32_t* obs_cam,
                                 const int64_t* point_obs_offset, const int32_t* point_obs, const double* dc,
                                 double* dp, gs_stream stream) {
  if (n_cams < 0 || n_points < 0 || n_obs < 0) return fail(GS_ERR_ARG, "sfm_ba_back_substitute: negative sizes");
  if (n_points > 0 && (!Vinv || !Vp || !gp || !dp || !point_obs_offset || !dc ||
                       (n_obs > 0 && (!Wo || !obs_cam || !point_obs))))
    return fail(GS_ERR_ARG, "sfm_ba_back_substitute: null argument");
  cudaError_t e = launch_ba_back_substitute(n_cams, n_points, n_obs, Vinv, Vp, gp, Wo, obs_cam, point_obs_offset,
                                            point_obs, dc, dp, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sfm_ba_back_substitute");
  return GS_OK;
}

gs_status gs_mcmc_workspace(int32_t n, size_t* ws_bytes) {
  if (n < 0 || !ws_bytes) return fail(GS_ERR_ARG, "gs_mcmc_workspace: bad argument");
  *ws_bytes = mcmc_ws_bytes(n);
  return GS_OK;
}

gs_status gs_mcmc_relocate(int32_t n, int32_t sh_degree, float* mean, float* log_scale, float* quat,
                           float* opacity_logit, float* sh, const double* u, int32_t n_u, int32_t* src,
                           uint32_t* n_dead, void* ws, size_t ws_bytes, gs_stream stream) {
  if (n < 0 || n_u < 0 || sh_degree < 0 || sh_degree > 3) return fail(GS_ERR_ARG, "gs_mcmc_relocate: bad sizes");
  if (n > 0 && (!mean || !log_scale || !quat || !opacity_logit || !sh || !src || !ws))
    return fail(GS_ERR_ARG, "gs_mcmc_relocate: null argument");
  if (n_u > 0 && !u) return fail(GS_ERR_ARG, "gs_mcmc_relocate: null u");
  if (n > 0 && ws_bytes < mcmc_ws_bytes(n))
    return fail(GS_ERR_ARG, "gs_mcmc_relocate: workspace needs %zu bytes", mcmc_ws_bytes(n));
  if (!aligned(ws, 16)) return fail(GS_ERR_ARG, "gs_mcmc_relocate: workspace must be 16-byte aligned");
  cudaError_t e = launch_mcmc_relocate(n, sh_degree, mean, log_scale, quat, opacity_logit, sh, u, n_u, src, n_dead,
                                       ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_mcmc_relocate");
  return GS_OK;
}

gs_status gs_mcmc_grow(int32_t n, int32_t n_add, int32_t sh_degree, float* mean, float* log_scale, float* quat,
                       float* opacity_logit, float* sh, const double* u, int32_t* src, void* ws, size_t ws_bytes,
                       gs_stream stream) {
  if (n < 0 || n_add < 0 || sh_degree < 0 || sh_degree > 3) return fail(GS_ERR_ARG, "gs_mcmc_grow: bad sizes");
  if ((long long)n + n_add > INT32_MAX) return fail(GS_ERR_ARG, "gs_mcmc_grow: n + n_add must be < 2^31");
  if (n_add > 0 && (!mean || !log_scale || !quat || !opacity_logit || !sh || !u || !src))
    return fail(GS_ERR_ARG, "gs_mcmc_grow: null argument");
  if (n_add > 0 && (!ws || ws_bytes < mcmc_ws_bytes(n)))
    return fail(GS_ERR_ARG, "gs_mcmc_grow: workspace needs %zu bytes", mcmc_ws_bytes(n));
  if (!aligned(ws, 16)) return fail(GS_ERR_ARG, "gs_mcmc_grow: workspace must be 16-byte aligned");
  cudaError_t e = launch_mcmc_grow(n, n_add, sh_degree, mean, log_scale, quat, opacity_logit, sh, u, src, ws,
                                   (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_mcmc_grow");
  return GS_OK;
}

gs_status gs_mcmc_reset_moments(int32_t n_rows, const int32_t* src, int32_t n_src, int32_t row0,
                                const gs_adam_group* groups, int32_t n_groups, gs_stream stream) {
  if (n_rows <= 0 || n_src < 0 || row0 < 0 || n_groups < 0 || n_groups > 8)
    return fail(GS_ERR_ARG, "gs_mcmc_reset_moments: bad sizes (1..8 groups)");
  if (n_src > 0 && (!src || (n_groups > 0 && !groups))) return fail(GS_ERR_ARG, "gs_mcmc_reset_moments: null argument");
  if ((long long)row0 + n_src > n_rows) return fail(GS_ERR_ARG, "gs_mcmc_reset_moments: rows past n_rows");
  for (int g = 0; g < n_groups; ++g) {
    if (!groups[g].m || !groups[g].v) return fail(GS_ERR_ARG, "gs_mcmc_reset_moments: null moments");
    if (groups[g].n <= 0 || groups[g].n % n_rows != 0)
      return fail(GS_ERR_ARG, "gs_mcmc_reset_moments: group %d size is not a multiple of n_rows", g);
  }
  cudaError_t e = launch_mcmc_reset_moments(n_rows, src, n_src, row0, groups, n_groups, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_mcmc_reset_moments");
  return GS_OK;
}

gs_status gs_mcmc_noise(int32_t n, float* mean, const float* log_scale, const float* quat, const float* opacity_logit,
                        const float* eta, float noise_lr, gs_stream stream) {
  if (n < 0) return fail(GS_ERR_ARG, "gs_mcmc_noise: negative n");
  if (n > 0 && (!mean || !log_scale || !quat || !opacity_logit || !eta))
    return fail(GS_ERR_ARG, "gs_mcmc_noise: null argument");
  if (!std::isfinite(noise_lr)) return fail(GS_ERR_ARG, "gs_mcmc_noise: noise_lr");
  if (n > 0 && !aligned(quat, 16)) return fail(GS_ERR_ARG, "gs_mcmc_noise: quat must be 16-byte aligned");
  cudaError_t e = launch_mcmc_noise(n, mean, log_scale, quat, opacity_logit, eta, noise_lr, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_mcmc_noise");
  return GS_OK;
}

gs_status gs_gather_view_pixels(const float* src, const int64_t* src_px_offset, const gs_cameras* cams,
                                const gs_batch* batch, int32_t channels, float* dst, gs_stream stream) {
  gs_status s;
  if ((s = check_cameras(cams)) || (s = check_batch(batch))) return s;
  if (!src || !src_px_offset || !dst || channels < 1)
    return fail(GS_ERR_ARG, "gs_gather_view_pixels: bad argument");
  cudaError_t e = launch_gather_view_pixels(src, src_px_offset, *cams, *batch, channels, dst, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_gather_view_pixels");
  return GS_OK;
}

gs_status gs_zero(void* ptr, size_t bytes, gs_stream stream) {
  if (bytes == 0) return GS_OK;
  if (!ptr) return fail(GS_ERR_ARG, "gs_zero: null");
  cudaError_t e = cudaMemsetAsync(ptr, 0, bytes, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gs_zero");
  return GS_OK;
}

}  // extern "C"

namespace gs {

// Shared helpers for entry points defined in other translation units.
gs_status record_error(gs_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

gs_status check_track_call(const float* X, int32_t n_points, const int32_t* obs_point, const float* obs_xy,
                           const int64_t* view_obs_offset, const gs_cameras* cams, const gs_batch* batch,
                           float delta, float weight, const float* grad_X, const double* g_pose_tangent,
                           const char* who) {
  gs_status s;
  if ((s = check_cameras(cams)) || (s = check_batch(batch))) return s;
  if (n_points < 0 || !view_obs_offset || !grad_X || !g_pose_tangent)
    return fail(GS_ERR_ARG, "%s: null argument", who);
  if (n_points > 0 && (!X || !obs_point || !obs_xy)) return fail(GS_ERR_ARG, "%s: null array", who);
  if (obs_xy && !aligned(obs_xy, 8)) return fail(GS_ERR_ARG, "%s: obs_xy must be 8-byte aligned", who);
  if (!std::isfinite(delta) || !std::isfinite(weight))
    return fail(GS_ERR_NONFINITE, "%s: non-finite delta/weight", who);
  if (!(delta > 0.f)) return fail(GS_ERR_ARG, "%s: delta must be > 0", who);
  return GS_OK;
}

}  // namespace gs
