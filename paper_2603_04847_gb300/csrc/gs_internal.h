// Internal launch interface between the C ABI layer (gs_capi.cu) and the
// kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "gs.h"
#include "gs_common.cuh"

namespace gs {

int device_sm_count();
// Process-wide launch tuning (gs_set_tuning); defaults when never set.
const gs_tuning& tuning();

cudaError_t launch_project_fwd(const gs_gaussians& g, const gs_cameras& cams, const gs_batch& batch,
                               const gs_projected& out, int32_t* status, cudaStream_t st);
int project_bwd_blocks(int n);
cudaError_t launch_project_fwd_f64(const gs_gaussians_f64& g, const gs_cameras_f64& cams, const gs_batch& batch,
                                   const gs_projected_f64& out, int32_t* status, cudaStream_t st);
cudaError_t launch_project_bwd_f64(const gs_gaussians_f64& g, const gs_cameras_f64& cams, const gs_batch& batch,
                                   const gs_projected_f64& proj, const double* v2d, const gs_gaussian_grads_f64& dg,
                                   double* partial, double* g_pose_tangent, cudaStream_t st);
cudaError_t launch_project_bwd(const gs_gaussians& g, const gs_cameras& cams, const gs_batch& batch,
                               const gs_projected& proj, float* v2d, const gs_gaussian_grads& dg,
                               double* partial, double* g_pose_tangent, bool clear_records, cudaStream_t st);

int sort_tile_bits(int n_tiles_total);
size_t sort_workspace_bytes(int N, const gs_batch& batch, size_t capacity);
int sort_kernel_count(const gs_batch& batch);
cudaError_t launch_sort_tiles(int N, const gs_cameras& cams, const gs_batch& batch,
                              const gs_projected& proj, uint32_t* tiles, uint32_t* vals,
                              size_t capacity, uint32_t* ranges, uint32_t* n_instances, void* ws,
                              int32_t* status, cudaStream_t st);

cudaError_t launch_render_fwd(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                              const uint32_t* vals, const uint32_t* ranges, const float* bg,
                              float* image, float* T_final, uint32_t* n_contrib, uint32_t* n_added,
                              cudaStream_t st);
cudaError_t launch_render_bwd(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                              const uint32_t* vals, const uint32_t* ranges, const float* bg,
                              const float* image, const float* T_final, const uint32_t* n_contrib,
                              const float* v_image, const float* target, float l1_weight,
                              double* loss, float* v2d, cudaStream_t st);
// The deterministic backward's scratch (after the v2d records and pose
// partials): per-record slot bases, scan block sums, one slot of 9 floats
// per instance of the capacity, and the tiles' loss sums.
size_t render_bwd_det_bytes(size_t M, int n_tiles, size_t capacity);
cudaError_t launch_render_bwd_det(const gs_batch& batch, const gs_cameras& cams, const gs_projected& proj,
                                  size_t M, const uint32_t* vals, const uint32_t* ranges,
                                  const uint32_t* n_instances, const float* bg, const float* image,
                                  const float* T_final, const uint32_t* n_contrib, const float* v_image,
                                  const float* target, float l1_weight, double* loss, float* v2d, void* det_ws,
                                  size_t capacity, cudaStream_t st);

cudaError_t launch_render_fwd_f64(const gs_batch& batch, const gs_cameras_f64& cams, const gs_projected_f64& proj,
                                  const uint32_t* vals, const uint32_t* ranges, const double* bg, double* image,
                                  double* T_final, uint32_t* n_contrib, uint32_t* n_added, cudaStream_t st);
cudaError_t launch_render_bwd_f64(const gs_batch& batch, const gs_cameras_f64& cams, const gs_projected_f64& proj,
                                  const uint32_t* vals, const uint32_t* ranges, const double* bg,
                                  const double* image, const double* T_final, const uint32_t* n_contrib,
                                  const double* v_image, const double* target, double l1_weight, double* loss,
                                  double* v2d, cudaStream_t st);

int track_blocks();
size_t track_workspace_bytes(const gs_batch& batch);
cudaError_t launch_track(const float* X, int n_points, const int32_t* obs_point, const float* obs_xy,
                         const int64_t* view_obs_offset, const gs_cameras& cams, const gs_batch& batch,
                         float delta, float weight, double* loss, float* grad_X,
                         double* g_pose_tangent, uint32_t* n_masked, void* ws, cudaStream_t st);
cudaError_t launch_track_det(const float* X, int n_points, const int32_t* obs_point, const float* obs_xy,
                         const int64_t* view_obs_offset, const gs_cameras& cams, const gs_batch& batch,
                         float delta, float weight, double* loss, float* grad_X,
                         double* g_pose_tangent, uint32_t* n_masked, void* ws, cudaStream_t st);

cudaError_t launch_pose_partials_finalize(const double* partial, int n_blocks, const gs_batch& batch,
                                          int n_cams, double* g_pose_tangent, cudaStream_t st);
cudaError_t launch_pose_update(int V, const float* T0, float* xi, const double* g_tangent, float* g_xi,
                               float* m, float* v, const gs_adam* hp, float* Rt_out, cudaStream_t st);
cudaError_t launch_pose_update_f64(int V, const double* T0, double* xi, const double* g_tangent, double* g_xi,
                                   double* m, double* v, const gs_adam* hp, double* Rt_out, cudaStream_t st);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, const gs_adam& hp,
                        cudaStream_t st);
cudaError_t launch_adam_groups(const gs_adam_group* groups, int n_groups, const gs_adam& hp, cudaStream_t st);
cudaError_t launch_step_advance(int32_t* step, cudaStream_t st);
cudaError_t launch_batch_layout(const gs_cameras& cams, const gs_batch& batch, int64_t* px_offset,
                                int32_t* tile_offset, int32_t* status, cudaStream_t st);
int64_t ba_pair_plan(int V, int P, int64_t M, const int32_t* obs_cam, const int64_t* off, const int32_t* point_obs,
                     int chunk, int32_t* n_pairs, int32_t* n_chunks, int32_t* inc, int32_t* pair_cams,
                     int32_t* pair_chunks, int64_t* chunk_start);
size_t ba_schur_pairs_workspace_bytes(int64_t M, int n_chunks);
cudaError_t launch_ba_schur_pairs(int V, int P, int64_t M, const double* U, const double* Vp, const double* gc,
                                  const double* gp, const double* Wo, const int32_t* obs_cam,
                                  const int64_t* point_obs_offset, const int32_t* point_obs, const int32_t* inc,
                                  const int32_t* pair_cams, int n_pairs, const int32_t* pair_chunks,
                                  const int64_t* chunk_start, int n_chunks, double lambda, const double* lambda_dev,
                                  double* S, double* rhs, double* Vinv, void* ws, cudaStream_t st);
cudaError_t launch_ba_assemble(const float* X, int n_points, const gs_cameras& cams, const int32_t* obs_point,
                               const int32_t* obs_cam, const float* obs_xy, int64_t n_obs, float delta, double* U,
                               double* Vp, double* gc, double* gp, double* Wo, double* objective,
                               cudaStream_t st);
cudaError_t launch_ba_schur(int V, int P, int64_t M, const double* U, const double* Vp, const double* gc,
                            const double* gp, const double* Wo, const int32_t* obs_cam, const int64_t* point_obs_offset,
                            const int32_t* point_obs, double lambda, const double* lambda_dev, double* S,
                            double* rhs, double* Vinv, cudaStream_t st);
cudaError_t launch_ba_lm_accept(int V, int P, double* obj, double* lambda, float* Rt, float* X, const float* Rt_trial,
                                const float* X_trial, int32_t* n_accepted, double* history, int32_t history_len,
                                int32_t* n_iter, cudaStream_t st);
cudaError_t launch_ba_apply(int V, int P, const float* Rt, const float* X, const double* dc, const double* dp,
                            float* Rt_out, float* X_out, cudaStream_t st);
cudaError_t launch_ba_solve_cameras(int V, double* S, const double* rhs, double* dc, int32_t* status,
                                   cudaStream_t st);
cudaError_t launch_ba_back_substitute(int V, int P, int64_t M, const double* Vinv, const double* Vp, const double* gp,
                                      const double* Wo, const int32_t* obs_cam, const int64_t* point_obs_offset,
                                      const int32_t* point_obs, const double* dc, double* dp, cudaStream_t st);
size_t mcmc_ws_bytes(int n);
cudaError_t launch_mcmc_relocate(int n, int sh_degree, float* mean, float* log_scale, float* quat, float* logit,
                                 float* sh, const double* u, int n_u, int32_t* src, uint32_t* n_dead, void* ws,
                                 cudaStream_t st);
cudaError_t launch_mcmc_grow(int n, int n_add, int sh_degree, float* mean, float* log_scale, float* quat,
                             float* logit, float* sh, const double* u, int32_t* src, void* ws, cudaStream_t st);
cudaError_t launch_mcmc_reset_moments(int n_rows, const int32_t* src, int n_src, int row0,
                                      const gs_adam_group* groups, int n_groups, cudaStream_t st);
cudaError_t launch_mcmc_noise(int n, float* mean, const float* log_scale, const float* quat, const float* logit,
                              const float* eta, float lr, cudaStream_t st);
size_t photo_loss_ws_bytes(int64_t n_pixels, int32_t n_tiles);
cudaError_t launch_photo_loss(const gs_batch& batch, const gs_cameras& cams, const float* image,
                              const float* target, float l1_weight, float ssim_weight, double* loss,
                              float* v_image, float* ws, cudaStream_t st);
cudaError_t launch_gather_view_pixels(const float* src, const int64_t* src_px_offset, const gs_cameras& cams,
                                      const gs_batch& batch, int channels, float* dst, cudaStream_t st);

// Error reporting and argument checks shared with entry points outside
// gs_capi.cu.
gs_status record_error(gs_status code, const char* fmt, ...);
gs_status check_track_call(const float* X, int32_t n_points, const int32_t* obs_point, const float* obs_xy,
                           const int64_t* view_obs_offset, const gs_cameras* cams, const gs_batch* batch,
                           float delta, float weight, const float* grad_X, const double* g_pose_tangent,
                           const char* who);

}  // namespace gs
