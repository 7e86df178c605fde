/*
 * FP64 CPU oracle for the joint photometric + feature-track training step of
 * GloSplat (arXiv 2603.04847, Sec. 3.3, Eq. 5, Eq. 6, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this library: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library; it is a plain, slow restatement of the method:
 *   - projection pi(X) = proj(K (R X + t)) of Sec. 3.2 (Eq. 4 text) and the
 *     "Projection function" bullet after Algorithm 1;
 *   - EWA splatting, SH colour and front-to-back alpha compositing, which the
 *     paper delegates to its rasterizer (Sec. 3.3 "Implementation"); every
 *     point the paper leaves open follows the published 3DGS convention,
 *     stated beside the code that applies it;
 *   - per-pixel brute-force compositing over ALL visible Gaussians of a view,
 *     ordered by (camera depth, index): no tiles;
 *   - hand-derived reverse-mode derivatives of all of the above, the Huber
 *     reprojection term of Eq. 6 and the SE(3) pose composition of
 *     Algorithm 1 (T_i = T_i^(0) (+) dT_i), read as a left perturbation.
 *
 * Conventions (all double precision):
 *   Gaussian j: mean[3], log_scale[3], quat[4] = (w,x,y,z) unnormalised,
 *   opacity_logit, sh[K][3] with K = (deg+1)^2.
 *   Camera: world-to-camera R (row-major 3x3) and t; x_c = R x + t.
 *   Pixel (u,v) has its centre at (u+0.5, v+0.5).
 *   Pose tangent g = (d/d rho, d/d phi) of T <- Exp((rho,phi)) T at 0.
 */
#ifndef GS_ORACLE_H
#define GS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_camera {
  int32_t width, height;
  double fx, fy, cx, cy;
  double R[9];
  double t[3];
  double near_plane, far_plane;
} orc_camera;

typedef struct orc_scene {
  int32_t n;
  int32_t sh_degree;
  const double* mean;          /* [n][3] */
  const double* log_scale;     /* [n][3] */
  const double* quat;          /* [n][4] */
  const double* opacity_logit; /* [n]    */
  const double* sh;            /* [n][K][3] */
} orc_scene;

/* Field offsets of one projected record (orc_project output, doubles). */
enum {
  ORC_P_VISIBLE = 0,
  ORC_P_DEPTH = 1,
  ORC_P_MX = 2, ORC_P_MY = 3,
  ORC_P_COV_XX = 4, ORC_P_COV_XY = 5, ORC_P_COV_YY = 6,
  ORC_P_CON_A = 7, ORC_P_CON_B = 8, ORC_P_CON_C = 9,
  ORC_P_OPACITY = 10,
  ORC_P_R = 11, ORC_P_G = 12, ORC_P_B = 13,
  ORC_P_BOUND_X0 = 14, ORC_P_BOUND_Y0 = 15, ORC_P_BOUND_X1 = 16, ORC_P_BOUND_Y1 = 17,
  ORC_P_PX_X0 = 18, ORC_P_PX_Y0 = 19, ORC_P_PX_X1 = 20, ORC_P_PX_Y1 = 21,
  ORC_P_XC = 22, ORC_P_YC = 23,
  ORC_P_FIELDS = 24
};

/* Knife-edge flag bits of a pixel (orc_render). */
enum {
  ORC_KNIFE_ALPHA_MIN = 1, /* some evaluated o*G within eps of 1/255        */
  ORC_KNIFE_T_MIN = 2,     /* some T' within eps of 1e-4                    */
  ORC_KNIFE_ALPHA_MAX = 4, /* some o*G within eps of 0.99 (gradient only)   */
  ORC_KNIFE_DEPTH = 8      /* two contributors with nearly equal depth      */
};

int orc_sh_eval(int degree, const double dir[3], double* Y, double* dY);
int orc_project(const orc_scene* s, const orc_camera* cam, double* out);
int orc_render(const orc_scene* s, const orc_camera* cam, const double bg[3],
               int64_t npix, const int32_t* pix, double knife_eps,
               double* image, double* T_final, int32_t* last_id,
               int32_t* n_added, int32_t* knife, int64_t* n_pairs);
int orc_render_tiled(const orc_scene* s, const orc_camera* cam,
                     const double bg[3], int tile, double* image,
                     double* T_final);
int orc_render_bwd(const orc_scene* s, const orc_camera* cam,
                   const double bg[3], int64_t npix, const int32_t* pix,
                   const double* v_image, double* v_mean, double* v_log_scale,
                   double* v_quat, double* v_opacity_logit, double* v_sh,
                   double* v_tangent, double* v_tangent_abs, double* v2d);
int orc_track(int32_t n_points, const double* X, int64_t n_obs,
              const int32_t* obs_point, const int32_t* obs_cam,
              const double* obs_xy, int32_t n_cams, const orc_camera* cams,
              double delta, double weight, double* loss, double* grad_X,
              double* tangent, double* tangent_abs, int64_t* n_masked);
void orc_se3_exp(const double xi[6], double T[12]);
void orc_se3_log(const double T[12], double xi[6]);
void orc_se3_left_jacobian(const double xi[6], double J[36]);
void orc_adam(int64_t n, double* p, const double* g, double* m, double* v,
              double lr, double beta1, double beta2, double eps, int step);
void orc_pose_update(int32_t n_cams, const double* T0, double* xi,
                     const double* g_tangent, double* g_xi, double* m,
                     double* v, int use_adam, double lr, double beta1,
                     double beta2, double eps, int step, double* Rt_out);

#ifdef __cplusplus
}
#endif
#endif
