// Kernels shared by both arithmetic paths: initial state, the two-stage fixed-order
// reduction of per-tile column partials, the per-job scalar step (shrink factors,
// penalty schedule), the FP32 col2im gather with the Omega-projection (L-update),
// and the end-of-run scalars.
#include <math.h>
#include "icnnm_internal.h"

namespace icnnm {

namespace {

struct TileVox {
  int jb, tile, t, h, w;
  bool valid;
};

// Voxel of thread threadIdx.x (< TILE_VOX) in global tile blockIdx.x.
__device__ __forceinline__ TileVox tile_voxel(const Shared& sh) {
  TileVox r;
  const int tile_g = blockIdx.x;
  r.jb = job_of_tile(sh.job_tile0, sh.njobs, tile_g);
  const JobDev& J = sh.jobs[r.jb];
  r.tile = tile_g - sh.job_tile0[r.jb];
  const int tw = r.tile % J.ntw, th = (r.tile / J.ntw) % J.nth;
  r.t = r.tile / (J.ntw * J.nth);
  r.h = th * TH + threadIdx.x / TW;
  r.w = tw * TW + threadIdx.x % TW;
  r.valid = r.h < J.H && r.w < J.W;
  return r;
}

// L = P_Omega(M) (the initial iterate, a reading: the paper does not state L0); X = L.
__global__ void init_L_kernel(Shared sh) {
  const TileVox p = tile_voxel(sh);
  if (!p.valid) return;
  const JobDev& J = sh.jobs[p.jb];
  const long long v = ((long long)p.t * J.H + p.h) * J.W + p.w;
  const float x = J.mask[v] ? J.M[v] : 0.f;
  J.L[v] = x;
  if (J.X) J.X[v] = x;
}

// First reduction stage: colseg[seg][c] = sum over the partial rows (PROW per tile or
// per forward CTA slot) of
// segment seg of part[row][c], in FP64; warp w adds rows lo+w, lo+w+8, ... in increasing
// order and the 8 warp sums are combined in warp order. Block = (job, 32 channels, segment).
// With `advance`, one block per job moves theta to theta_next and counts the
// iteration (every kernel of the iteration that reads theta has run by then).
__global__ void reduce_cols_kernel(Shared sh, int advance, int tpr) {
  const JobDev& J = sh.jobs[blockIdx.x];
  const int c = blockIdx.y * 32 + (threadIdx.x & 31);
  const int warp = threadIdx.x >> 5;
  const int seg = blockIdx.z;
  // row groups: tpr > 0 tiles each; tpr == 0: the job's fchunk tiles each; tpr < 0: one per
  // forward CTA slot (-tpr slots), at most one per tile
  const int tp = tpr > 0 ? tpr : J.fchunk;
  const int nrows = (tpr < 0 ? min(-tpr, J.ntiles) : (J.ntiles + tp - 1) / tp) * PROW;
  const int lo = (int)((long long)nrows * seg / NSEG);
  const int hi = (int)((long long)nrows * (seg + 1) / NSEG);
  double acc = 0.0;
  if (c < sh.kc) {
    const float* p = J.part + c;
    int t = lo + warp;
    // four independent loads in flight per step; the sum order is fixed by the tile index
    for (; t + 24 < hi; t += 32) {
      const float a0 = p[(long long)t * sh.kc], a1 = p[(long long)(t + 8) * sh.kc];
      const float a2 = p[(long long)(t + 16) * sh.kc], a3 = p[(long long)(t + 24) * sh.kc];
      acc += (double)a0; acc += (double)a1; acc += (double)a2; acc += (double)a3;
    }
    for (; t < hi; t += 8) acc += (double)p[(long long)t * sh.kc];
  }
  __shared__ double red[8][32];
  red[warp][threadIdx.x & 31] = acc;
  __syncthreads();
  if (warp == 0 && c < sh.kc) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    J.colseg[(long long)seg * sh.kc + c] = s;
  }
  if (advance && blockIdx.y == 0 && seg == 0 && threadIdx.x == 0) {
    J.sc->theta = J.sc->theta_next;
    J.sc->iter += 1;
  }
}

__device__ __forceinline__ double colsq_of(const JobDev& J, int kc, int c) {
  double q = 0.0;
  for (int s0 = 0; s0 < NSEG; s0 += 32) {
    double v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = J.colseg[(long long)(s0 + i) * kc + c];
#pragma unroll
    for (int i = 0; i < 32; ++i) q += v[i];
  }
  return q;
}

// Per-job scalar step at the start of an iteration (the Z-update of Sec. III-D in
// shifted form): s_c = max(0, 1 - 1/||U_c||) (the column-wise l2,1 shrinkage with
// threshold 1/theta applied to -U/theta), D_c = 1 - s_c; theta' = min(rho theta, theta_max).
__global__ void scalars_kernel(Shared sh) {
  // block = (job, 32 channels); warp w sums segments w, w + 8, ... (fixed order), then
  // the 8 warp sums are added in warp order
  const JobDev& J = sh.jobs[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  double q = 0.0;
  if (c < sh.kc) {
#pragma unroll
    for (int i = 0; i < NSEG / 8; ++i) q += J.colseg[(long long)(warp + 8 * i) * sh.kc + c];
  }
  __shared__ double red[8][32];
  red[warp][lane] = q;
  __syncthreads();
  if (warp == 0 && c < sh.kc) {
    double n2 = 0.0;
    for (int w = 0; w < 8; ++w) n2 += red[w][lane];
    const double n = sqrt(n2);
    const double sc = (c < sh.k && n > 1.0) ? 1.0 - 1.0 / n : 0.0;
    J.s[c] = (float)sc;
    J.D[c] = (c < sh.k) ? (float)(1.0 - sc) : 0.f;
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) J.sc->theta_next = fmin(J.rho * J.sc->theta, J.theta_max);
}

// theta0 = 1 / max_c ||A_k(P_Omega M) V_c|| unless the caller gives one (a reading: the
// paper does not state theta0). Column sums come from the norm-only forward pass.
__global__ void theta0_kernel(Shared sh, double theta0_user) {
  const JobDev& J = sh.jobs[blockIdx.x];
  __shared__ double mx[256];
  double m = 0.0;
  for (int c = threadIdx.x; c < sh.k; c += blockDim.x) m = fmax(m, colsq_of(J, sh.kc, c));
  mx[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int i = 0; i < blockDim.x; ++i) mm = fmax(mm, mx[i]);
    const double th = theta0_user > 0 ? theta0_user : (mm > 0 ? 1.0 / sqrt(mm) : 1.0);
    J.sc->theta = th;
    J.sc->theta_next = th;
    J.sc->iter = 0;
  }
}

__global__ void scale_X_kernel(Shared sh) {
  const TileVox p = tile_voxel(sh);
  if (!p.valid) return;
  const JobDev& J = sh.jobs[p.jb];
  const long long v = ((long long)p.t * J.H + p.h) * J.W + p.w;
  J.X[v] = (float)J.sc->theta * J.L[v];
}

// FP32 path L-update. Delta_j = [A_k^*(G)]_j = sum_s G^T[s][(j + s) mod dims] in tap
// order (the adjoint of Eq. ak), then
//   lambda = inf : L'_j = M_j on Omega and L_j + Delta_j/(k theta) off Omega;
//   lambda finite: L'_j = (Delta_j/k + theta L_j + lambda Theta_j M_j)/(lambda Theta_j + theta);
// X_j = (theta + theta') L'_j - theta L_j; L <- L'. Per-tile partial of ||L'||^2.
__global__ void gather_fp32_kernel(Shared sh) {
  const TileVox p = tile_voxel(sh);
  const JobDev& J = sh.jobs[p.jb];
  __shared__ float red[TILE_VOX];
  float l2 = 0.f;
  if (p.valid) {
    const int H = J.H, W = J.W, T = J.T;
    const long long v = ((long long)p.t * H + p.h) * W + p.w;
    float d = 0.f;
    int s = 0;
    for (int st = 0; st < sh.k3; ++st) {
      const int tt = wrapi(p.t + st, T);
      for (int sh_ = 0; sh_ < sh.k1; ++sh_) {
        const long long rowb = ((long long)tt * H + wrapi(p.h + sh_, H)) * W;
        for (int sw = 0; sw < sh.k2; ++sw, ++s) d += J.G[(long long)s * J.m + rowb + wrapi(p.w + sw, W)];
      }
    }
    const float Ln = l_update(J, sh.k, v, d);
    l2 = Ln * Ln;
  }
  red[threadIdx.x] = l2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < TILE_VOX; ++i) s += red[i];
    J.lpart[p.tile] = s;
  }
}

// End-of-pass scalars: what = 1: ||L||^2 and the residual sum of squares from the
// per-tile partials; what = 2: objective sum_c sqrt(colsq_c).
// One block per job. The residual partials (one float per tile and task slot) are summed per
// thread in FP32 (GB300 runs FP64 adds at a small fraction of the FP32 rate, and this sum is
// the stopping test's) and across threads in FP64, all in a fixed order.
constexpr int FIN_THREADS = 1024;
__global__ void __launch_bounds__(FIN_THREADS) finish_kernel(Shared sh, int what) {
  const JobDev& J = sh.jobs[blockIdx.x];
  __shared__ double a[FIN_THREADS / 32], b[FIN_THREADS / 32];
  double x = 0.0, y = 0.0;
  if (what == 2) {
    for (int c = threadIdx.x; c < sh.k; c += blockDim.x) x += sqrt(colsq_of(J, sh.kc, c));
  } else {
    for (int t = threadIdx.x; t < J.nlp; t += blockDim.x) x += J.lpart[t];
    const long long n = (long long)J.ntiles * sh.nrp;
    float yf = 0.f;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) yf += J.rpart[t];
    y = yf;
  }
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  if ((threadIdx.x & 31) == 0) {
    a[threadIdx.x >> 5] = x;
    b[threadIdx.x >> 5] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0, sy = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { sx += a[i]; sy += b[i]; }
    if (what == 2) J.sc->objective = sx;
    else { J.sc->lsq = sx; J.sc->rsq = sy; }
  }
}

// U widened from BF16 to FP32 (exact), for the FP32 finish of a BF16 job.
__global__ void widen_bf16_kernel(const __nv_bfloat16* src, float* dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = __bfloat162float(src[i]);
}

__global__ void check_observed_kernel(const float* M, const uint8_t* mask, long long n, int* out) {
  int cnt = 0, bad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (mask[i] > 1) bad = 1;
    if (mask[i]) { ++cnt; if (!isfinite(M[i])) bad = 1; }
  }
  if (cnt) atomicAdd(out, cnt);
  if (bad) atomicExch(out + 1, 1);
}

// Synthetic input of the tile autotuner: a smooth pattern with about half of the voxels
// observed (a hash of the index decides), deterministic.
__global__ void tune_fill_kernel(float* M, uint8_t* mask, int H, int W, int T) {
  const long long m = (long long)H * W * T;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(i % W), h = (int)((i / W) % H), t = (int)(i / ((long long)W * H));
    M[i] = 0.5f + 0.25f * __sinf(0.37f * w + 0.11f * t) * __cosf(0.23f * h - 0.07f * t);
    unsigned x = (unsigned)i * 2654435761u;
    x ^= x >> 15;
    x *= 2246822519u;
    x ^= x >> 13;
    mask[i] = (x & 1u) ? 1 : 0;
  }
}

}  // namespace

cudaError_t launch_tune_fill(float* M, uint8_t* mask, int H, int W, int T, cudaStream_t st) {
  tune_fill_kernel<<<512, 256, 0, st>>>(M, mask, H, W, T);
  return cudaGetLastError();
}

cudaError_t launch_init_L(const Shared& sh, cudaStream_t st) {
  init_L_kernel<<<sh.total_tiles, TILE_VOX, 0, st>>>(sh);
  return cudaGetLastError();
}

cudaError_t launch_widen_bf16(const __nv_bfloat16* src, float* dst, long long n, cudaStream_t st) {
  widen_bf16_kernel<<<1216, 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_reduce_cols(const Shared& sh, int advance, int tpr, cudaStream_t st) {
  dim3 grid(sh.njobs, (sh.kc + 31) / 32, NSEG);
  reduce_cols_kernel<<<grid, 256, 0, st>>>(sh, advance, tpr);
  return cudaGetLastError();
}

cudaError_t launch_scalars(const Shared& sh, cudaStream_t st) {
  scalars_kernel<<<dim3(sh.njobs, (sh.kc + 31) / 32), 256, 0, st>>>(sh);
  return cudaGetLastError();
}

cudaError_t launch_theta0(const Shared& sh, double theta0_user, cudaStream_t st) {
  theta0_kernel<<<sh.njobs, 256, 0, st>>>(sh, theta0_user);
  return cudaGetLastError();
}

cudaError_t launch_scale_X(const Shared& sh, cudaStream_t st) {
  scale_X_kernel<<<sh.total_tiles, TILE_VOX, 0, st>>>(sh);
  return cudaGetLastError();
}

cudaError_t launch_gather_fp32(const Shared& sh, cudaStream_t st) {
  gather_fp32_kernel<<<sh.total_tiles, TILE_VOX, 0, st>>>(sh);
  return cudaGetLastError();
}

cudaError_t launch_finish(const Shared& sh, int what, cudaStream_t st) {
  finish_kernel<<<sh.njobs, FIN_THREADS, 0, st>>>(sh, what);
  return cudaGetLastError();
}

cudaError_t check_observed(const float* M, const uint8_t* mask, long long n, int* d2, cudaStream_t st) {
  check_observed_kernel<<<256, 256, 0, st>>>(M, mask, n, d2);
  return cudaGetLastError();
}

}  // namespace icnnm
