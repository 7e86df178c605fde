// MCMC densification (Sec. 3.3, "stochastic density control via MCMC-based
// densification"; Algorithm 1 "Relocate / add Gaussians"), with the cited
// method's rules:
//  * a Gaussian is dead when sigmoid(logit) <= 0.005;
//  * each dead Gaussian, in index order, takes the parameters of the live one
//    drawn by its uniform u: the first j whose cumulative live opacity
//    exceeds u times the total;
//  * a source drawn c times becomes N = c + 1 identical Gaussians with
//    o_N = 1 - (1 - o)^(1/N) and scales s o / D_N,
//    D_N = sum_{m=1..N} C(N, m) (-1)^(m-1) o_N^m / sqrt(m)
//    (the stacked copies composite to the source's alpha at the centre and
//    to the same alpha integral along a line through it; D_N is the
//    front-to-back double sum over copies and powers collapsed with the
//    hockey-stick identity);
//    the reset opacity is then bounded to [0.005, 1 - 2^-23] (a copy is never
//    born dead and its logit stays finite);
//  * growth: each new Gaussian (appended after the n existing ones) draws a
//    live source like a relocation does, the drawn sources are reset by the
//    same rule and the new ones copy them;
//  * noise on the means: mu += lr sigmoid(-100 (o - 0.005)) Sigma eta.
// Passes: a two-level scan gives the cumulative live opacity (FP64) and each
// dead Gaussian's rank; draws are binary searches with atomic copy counts;
// then the sources are reset and the dead (or new) ones copy them.  A draw
// always lands on a live Gaussian: its target is below cdf[n-1] itself, and
// a search that ends on a dead one (possible only where the two scan levels
// round differently) moves on to the nearest live one.
#include <algorithm>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kThr = 256;
constexpr double kDead = 0.005;
constexpr double kMaxOpacity = 1.0 - 1.1920928955078125e-07;  // 1 - 2^-23

__device__ inline double opacity_of(float logit) { return 1.0 / (1.0 + exp(-(double)logit)); }

struct McmcWs {
  double* cdf;     // [n] inclusive cumulative live opacity
  int32_t* rank;   // [n] rank among the dead, -1 if live
  int32_t* count;  // [n] times drawn as a source
  double* bsum;    // [nb] per block, then exclusive over blocks
  int32_t* bcnt;   // [nb]
  double* total;   // [1]
  int32_t* list;   // [n] the distinct drawn sources, in no particular order
  uint32_t* list_n;  // [1]
};

inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

McmcWs mcmc_layout(void* base, int n, size_t* bytes) {
  const int nb = (n + kThr - 1) / kThr;
  char* p = (char*)base;
  size_t o = 0;
  McmcWs w;
  w.cdf = (double*)(p + o); o += al(8 * (size_t)n);
  w.rank = (int32_t*)(p + o); o += al(4 * (size_t)n);
  w.count = (int32_t*)(p + o); o += al(4 * (size_t)n);
  w.bsum = (double*)(p + o); o += al(8 * (size_t)nb);
  w.bcnt = (int32_t*)(p + o); o += al(4 * (size_t)nb);
  w.total = (double*)(p + o); o += al(8);
  w.list = (int32_t*)(p + o); o += al(4 * (size_t)n);
  w.list_n = (uint32_t*)(p + o); o += al(4);
  if (bytes) *bytes = o;
  return w;
}

// Block-wide inclusive and exclusive scans of a double and exclusive scan of
// an int.  The exclusive double prefix is the inclusive one of the thread
// before (not inclusive - v, which rounds differently).
__device__ inline void block_scan(double v, int c, double* incl, int* excl, double* s_d, int* s_i,
                                  double* excl_d = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double x = v;
  int y = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double a = __shfl_up_sync(0xffffffffu, x, off);
    const int b = __shfl_up_sync(0xffffffffu, y, off);
    if (lane >= off) {
      x += a;
      y += b;
    }
  }
  const double xprev = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 31) {
    s_d[warp] = x;
    s_i[warp] = y;
  }
  __syncthreads();
  double dbase = 0.0;
  int ibase = 0;
  for (int w = 0; w < warp; ++w) {
    dbase += s_d[w];
    ibase += s_i[w];
  }
  *incl = dbase + x;
  *excl = ibase + y - c;
  if (excl_d) *excl_d = lane > 0 ? dbase + xprev : dbase;
}

// The opacity is evaluated once (FP64 exp) and left in cdf[i] for
// mcmc_apply_kernel, which overwrites it with the cumulative sum.
__global__ void __launch_bounds__(kThr) mcmc_reduce_kernel(int n, const float* __restrict__ logit,
                                                           double* __restrict__ bsum, int32_t* __restrict__ bcnt,
                                                           double* __restrict__ o_out) {
  __shared__ double s_d[kThr / 32];
  __shared__ int s_i[kThr / 32];
  const int i = blockIdx.x * kThr + threadIdx.x;
  double v = 0.0;
  int c = 0;
  if (i < n) {
    const double o = opacity_of(logit[i]);
    o_out[i] = o;
    if (o <= kDead) c = 1;
    else v = o;
  }
  double incl;
  int excl;
  block_scan(v, c, &incl, &excl, s_d, s_i);
  if (threadIdx.x == kThr - 1) {
    bsum[blockIdx.x] = incl;
    bcnt[blockIdx.x] = excl + c;
  }
}

// Exclusive scan of the per-block sums in place, by one block with a carry.
__global__ void __launch_bounds__(kThr) mcmc_blocks_kernel(int nb, double* __restrict__ bsum, int32_t* __restrict__ bcnt,
                                                           double* __restrict__ total, uint32_t* __restrict__ n_dead) {
  __shared__ double s_d[kThr / 32];
  __shared__ int s_i[kThr / 32];
  __shared__ double carry_d;
  __shared__ int carry_i;
  if (threadIdx.x == 0) {
    carry_d = 0.0;
    carry_i = 0;
  }
  __syncthreads();
  for (int base = 0; base < nb; base += kThr) {
    const int i = base + threadIdx.x;
    const double v = i < nb ? bsum[i] : 0.0;
    const int c = i < nb ? bcnt[i] : 0;
    double incl, excl_d;
    int excl;
    block_scan(v, c, &incl, &excl, s_d, s_i, &excl_d);
    const double cd = carry_d;
    const int ci = carry_i;
    if (i < nb) {
      bsum[i] = cd + excl_d;
      bcnt[i] = ci + excl;
    }
    __syncthreads();
    if (threadIdx.x == kThr - 1) {
      carry_d = cd + incl;
      carry_i = ci + excl + c;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = carry_d;
    if (n_dead) *n_dead = (uint32_t)carry_i;
  }
}

__global__ void __launch_bounds__(kThr) mcmc_apply_kernel(int n, const float* __restrict__ logit,
                                                          const double* __restrict__ bsum,
                                                          const int32_t* __restrict__ bcnt, double* __restrict__ cdf,
                                                          int32_t* __restrict__ rank, int32_t* __restrict__ count,
                                                          uint32_t* __restrict__ list_n) {
  __shared__ double s_d[kThr / 32];
  __shared__ int s_i[kThr / 32];
  const int i = blockIdx.x * kThr + threadIdx.x;
  if (i == 0) *list_n = 0u;
  double v = 0.0;
  int c = 0;
  if (i < n) {
    const double o = cdf[i];  // the opacity, left there by mcmc_reduce_kernel
    if (o <= kDead) c = 1;
    else v = o;
  }
  double incl;
  int excl;
  block_scan(v, c, &incl, &excl, s_d, s_i);
  if (i < n) {
    cdf[i] = bsum[blockIdx.x] + incl;
    rank[i] = c ? bcnt[blockIdx.x] + excl : -1;
    count[i] = 0;
  }
}

// The live Gaussian that uniform u draws: the first j with cdf[j] > u T,
// T = cdf[n-1] (so some j qualifies for any u in [0, 1)); a dead one there
// (only where the scan's two levels round apart) gives way to the next live
// one, or the previous one at the end.  -1 when no Gaussian is live.
__device__ inline int draw_live(int n, double u, const double* __restrict__ cdf, const int32_t* __restrict__ rank) {
  const double T = cdf[n - 1];
  if (!(T > 0.0)) return -1;
  const double target = u * T;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cdf[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  int s = lo;
  while (s < n && rank[s] >= 0) ++s;
  if (s == n) {
    s = lo;
    while (s >= 0 && rank[s] >= 0) --s;
  }
  return s;
}

__global__ void __launch_bounds__(kThr) mcmc_draw_kernel(int n, const int32_t* __restrict__ rank,
                                                         const double* __restrict__ cdf, const double* __restrict__ u,
                                                         int n_u, int32_t* __restrict__ src,
                                                         int32_t* __restrict__ count, int32_t* __restrict__ list,
                                                         uint32_t* __restrict__ list_n) {
  const int i = blockIdx.x * kThr + threadIdx.x;
  if (i >= n) return;
  const int r = rank[i];
  int s = -1;
  if (r >= 0 && r < n_u) {
    s = draw_live(n, u[r], cdf, rank);
    if (s >= 0 && atomicAdd(&count[s], 1) == 0) list[atomicAdd(list_n, 1u)] = s;
  }
  src[i] = s;
}

// Growth: new Gaussian k (row n + k) draws its source with u[k].
__global__ void __launch_bounds__(kThr) mcmc_grow_draw_kernel(int n, int n_add, const int32_t* __restrict__ rank,
                                                              const double* __restrict__ cdf,
                                                              const double* __restrict__ u, int32_t* __restrict__ src,
                                                              int32_t* __restrict__ count, int32_t* __restrict__ list,
                                                              uint32_t* __restrict__ list_n) {
  const int k = blockIdx.x * kThr + threadIdx.x;
  if (k >= n_add) return;
  const int s = draw_live(n, u[k], cdf, rank);
  if (s >= 0 && atomicAdd(&count[s], 1) == 0) list[atomicAdd(list_n, 1u)] = s;
  src[k] = s;
}

// Over the list of distinct drawn sources (dense warps: the FP64 reset runs
// only where it is needed; each source is reset once, whatever the order of
// the list).
__global__ void __launch_bounds__(kThr) mcmc_reset_kernel(const int32_t* __restrict__ list,
                                                          const uint32_t* __restrict__ list_n,
                                                          float* __restrict__ logit, float* __restrict__ log_scale,
                                                          const int32_t* __restrict__ count) {
  const uint32_t k = blockIdx.x * kThr + threadIdx.x;
  if (k >= *list_n) return;
  const int j = list[k];
  const int N = count[j] + 1;
  const double o = opacity_of(logit[j]);
  const double oN = 1.0 - pow(1.0 - o, 1.0 / N);
  double den = 0.0, binom = 1.0, p = 1.0;
  for (int m = 1; m <= N; ++m) {
    binom = binom * (double)(N - m + 1) / (double)m;
    p *= oN;
    den += ((m & 1) ? 1.0 : -1.0) * binom * p / sqrt((double)m);
  }
  const double oB = fmin(fmax(oN, kDead), kMaxOpacity);   // the scale keeps the unbounded o_N
  logit[j] = (float)log(oB / (1.0 - oB));
  const double ds = log(o / den);
  for (int a = 0; a < 3; ++a) log_scale[3 * (size_t)j + a] = (float)((double)log_scale[3 * (size_t)j + a] + ds);
}

__global__ void __launch_bounds__(kThr) mcmc_copy_kernel(int n, int K3, const int32_t* __restrict__ src,
                                                         float* __restrict__ mean, float* __restrict__ log_scale,
                                                         float* __restrict__ quat, float* __restrict__ logit,
                                                         float* __restrict__ sh) {
  const int i = blockIdx.x * kThr + threadIdx.x;
  if (i >= n) return;
  const int s = src[i];
  if (s < 0) return;
  for (int a = 0; a < 3; ++a) {
    mean[3 * (size_t)i + a] = mean[3 * (size_t)s + a];
    log_scale[3 * (size_t)i + a] = log_scale[3 * (size_t)s + a];
  }
  for (int a = 0; a < 4; ++a) quat[4 * (size_t)i + a] = quat[4 * (size_t)s + a];
  logit[i] = logit[s];
  for (int a = 0; a < K3; ++a) sh[(size_t)K3 * i + a] = sh[(size_t)K3 * s + a];
}

// Growth: row n + k copies the (reset) parameters of its source src[k].
__global__ void __launch_bounds__(kThr) mcmc_grow_copy_kernel(int n, int n_add, int K3, const int32_t* __restrict__ src,
                                                              float* __restrict__ mean, float* __restrict__ log_scale,
                                                              float* __restrict__ quat, float* __restrict__ logit,
                                                              float* __restrict__ sh) {
  const int k = blockIdx.x * kThr + threadIdx.x;
  if (k >= n_add) return;
  const int s = src[k];
  if (s < 0) return;
  const size_t i = (size_t)n + k;
  for (int a = 0; a < 3; ++a) {
    mean[3 * i + a] = mean[3 * (size_t)s + a];
    log_scale[3 * i + a] = log_scale[3 * (size_t)s + a];
  }
  for (int a = 0; a < 4; ++a) quat[4 * i + a] = quat[4 * (size_t)s + a];
  logit[i] = logit[s];
  for (int a = 0; a < K3; ++a) sh[(size_t)K3 * i + a] = sh[(size_t)K3 * s + a];
}

// Zeroes the Adam moments of row row0 + k and of row src[k], for every k
// with src[k] >= 0, in every group (row width = group n / n_rows).
struct MomentGroups {
  float* m[8];
  float* v[8];
  int width[8];
  int n;
};

__global__ void __launch_bounds__(kThr) mcmc_reset_moments_kernel(int n_src, const int32_t* __restrict__ src,
                                                                  int row0, MomentGroups G) {
  // a thread per k reads src[k]; the warp then zeroes the two rows of each
  // of its lanes with src[k] >= 0 in turn, lanes over the row (coalesced)
  const int k = blockIdx.x * kThr + threadIdx.x, lane = threadIdx.x & 31;
  const int s = k < n_src ? src[k] : -1;
  unsigned todo = __ballot_sync(0xffffffffu, s >= 0);
  while (todo) {
    const int l = __ffs(todo) - 1;
    todo &= todo - 1;
    const int kl = __shfl_sync(0xffffffffu, k, l), sl = __shfl_sync(0xffffffffu, s, l);
    for (int r = 0; r < 2; ++r) {
      const size_t row = r ? (size_t)sl : (size_t)row0 + kl;
      for (int g = 0; g < G.n; ++g) {
        const size_t w = (size_t)G.width[g];
        for (int a = lane; a < G.width[g]; a += 32) {
          G.m[g][row * w + a] = 0.f;
          G.v[g][row * w + a] = 0.f;
        }
      }
    }
  }
}

// FP32 throughout (the means are float; the FP64 pipe of this part is a
// small fraction of the FP32 rate, and the noise is a perturbation whose
// float rounding, ~1e-7 relative, is far below its own size).
__global__ void __launch_bounds__(kThr) mcmc_noise_kernel(int n, float* __restrict__ mean,
                                                          const float* __restrict__ log_scale,
                                                          const float* __restrict__ quat,
                                                          const float* __restrict__ logit,
                                                          const float* __restrict__ eta, float lr) {
  const int i = blockIdx.x * kThr + threadIdx.x;
  if (i >= n) return;
  const float o = 1.f / (1.f + expf(-logit[i]));
  const float gate = 1.f / (1.f + expf(100.f * (o - (float)kDead)));
  const float4 q = reinterpret_cast<const float4*>(quat)[i];
  const float iq = 1.f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * iq, x = q.y * iq, y = q.z * iq, z = q.w * iq;
  const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                      2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                      2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
  float s2[3], e[3], Rte[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float sc = expf(log_scale[3 * (size_t)i + a]);
    s2[a] = sc * sc;
    e[a] = eta[3 * (size_t)i + a];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) Rte[a] = R[a] * e[0] + R[3 + a] * e[1] + R[6 + a] * e[2];   // R^T eta
  const float k = lr * gate;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float v = R[3 * a] * s2[0] * Rte[0] + R[3 * a + 1] * s2[1] * Rte[1] + R[3 * a + 2] * s2[2] * Rte[2];
    mean[3 * (size_t)i + a] += k * v;
  }
}

}  // namespace

size_t mcmc_ws_bytes(int n) {
  size_t b = 0;
  mcmc_layout(nullptr, n, &b);
  return b;
}

cudaError_t launch_mcmc_relocate(int n, int sh_degree, float* mean, float* log_scale, float* quat, float* logit,
                                 float* sh, const double* u, int n_u, int32_t* src, uint32_t* n_dead, void* ws,
                                 cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  McmcWs w = mcmc_layout(ws, n, nullptr);
  const int nb = (n + kThr - 1) / kThr;
  const int K3 = 3 * (sh_degree + 1) * (sh_degree + 1);
  mcmc_reduce_kernel<<<nb, kThr, 0, st>>>(n, logit, w.bsum, w.bcnt, w.cdf);
  mcmc_blocks_kernel<<<1, kThr, 0, st>>>(nb, w.bsum, w.bcnt, w.total, n_dead);
  mcmc_apply_kernel<<<nb, kThr, 0, st>>>(n, logit, w.bsum, w.bcnt, w.cdf, w.rank, w.count, w.list_n);
  mcmc_draw_kernel<<<nb, kThr, 0, st>>>(n, w.rank, w.cdf, u, n_u, src, w.count, w.list, w.list_n);
  const int n_sources = std::min(n, std::max(n_u, 0));  // bound on the distinct sources
  if (n_sources > 0)
    mcmc_reset_kernel<<<(n_sources + kThr - 1) / kThr, kThr, 0, st>>>(w.list, w.list_n, logit, log_scale, w.count);
  mcmc_copy_kernel<<<nb, kThr, 0, st>>>(n, K3, src, mean, log_scale, quat, logit, sh);
  return cudaGetLastError();
}

cudaError_t launch_mcmc_grow(int n, int n_add, int sh_degree, float* mean, float* log_scale, float* quat,
                             float* logit, float* sh, const double* u, int32_t* src, void* ws, cudaStream_t st) {
  if (n == 0 || n_add == 0) return cudaSuccess;
  McmcWs w = mcmc_layout(ws, n, nullptr);
  const int nb = (n + kThr - 1) / kThr;
  const int nba = (n_add + kThr - 1) / kThr;
  const int K3 = 3 * (sh_degree + 1) * (sh_degree + 1);
  mcmc_reduce_kernel<<<nb, kThr, 0, st>>>(n, logit, w.bsum, w.bcnt, w.cdf);
  mcmc_blocks_kernel<<<1, kThr, 0, st>>>(nb, w.bsum, w.bcnt, w.total, nullptr);
  mcmc_apply_kernel<<<nb, kThr, 0, st>>>(n, logit, w.bsum, w.bcnt, w.cdf, w.rank, w.count, w.list_n);
  mcmc_grow_draw_kernel<<<nba, kThr, 0, st>>>(n, n_add, w.rank, w.cdf, u, src, w.count, w.list, w.list_n);
  const int n_sources = std::min(n, n_add);
  mcmc_reset_kernel<<<(n_sources + kThr - 1) / kThr, kThr, 0, st>>>(w.list, w.list_n, logit, log_scale, w.count);
  mcmc_grow_copy_kernel<<<nba, kThr, 0, st>>>(n, n_add, K3, src, mean, log_scale, quat, logit, sh);
  return cudaGetLastError();
}

cudaError_t launch_mcmc_reset_moments(int n_rows, const int32_t* src, int n_src, int row0,
                                      const gs_adam_group* groups, int n_groups, cudaStream_t st) {
  if (n_src == 0 || n_groups == 0) return cudaSuccess;
  MomentGroups G;
  G.n = n_groups;
  for (int g = 0; g < n_groups; ++g) {
    G.m[g] = groups[g].m;
    G.v[g] = groups[g].v;
    G.width[g] = (int)(groups[g].n / n_rows);
  }
  mcmc_reset_moments_kernel<<<(n_src + kThr - 1) / kThr, kThr, 0, st>>>(n_src, src, row0, G);
  return cudaGetLastError();
}

cudaError_t launch_mcmc_noise(int n, float* mean, const float* log_scale, const float* quat, const float* logit,
                              const float* eta, float lr, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  mcmc_noise_kernel<<<(n + kThr - 1) / kThr, kThr, 0, st>>>(n, mean, log_scale, quat, logit, eta, lr);
  return cudaGetLastError();
}

}  // namespace gs
