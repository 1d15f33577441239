// Internal declarations shared by the CUDA translation units of libicnnm.
//
// Algorithm (ADMM of Sec. III-D, run in the shifted-multiplier form
// U = Y - theta*A_k(L)V, which follows from the Z-, L- and Y-updates using
// V V^T = I and A_k^* A_k = k I):
//   s_c  = max(0, 1 - 1/||U_c||),  D = diag(1 - s)                  (Z-update)
//   L'   = P_Omega^perp(L + A_k^*(U D V^T)/(k theta)) + P_Omega(M)   (L-update, lambda = inf)
//        = (A_k^*(U D V^T)/k + theta L + lambda Theta M)/(lambda Theta + theta)   (finite lambda)
//   X    = (theta + theta') L' - theta L,  theta' = min(rho theta, theta_max)
//   U'   = U D - A_k(X) V                                           (Y-update, re-shifted)
// Per iteration: one "adjoint" pass (G = U (D V^T), then col2im), one gather/projection
// pass over m voxels, one "forward" pass (E = A_k(X)V fused with the U update and the
// per-tile column-norm partials of U'), and small per-job reduction/scalar kernels.
#pragma once
#include <math.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

namespace icnnm {

// Voxel tile of the forward/adjoint passes: TW (w) x TH (h) x 1 (t) = 128 voxels.
constexpr int TW = 8;
constexpr int TH = 16;
constexpr int TILE_VOX = TW * TH;
constexpr int NSEG = 128;         // row segments of the first column-reduction stage
// Tiles of a job per column-partial row group of the deterministic BF16 forward pass:
// decided by the job alone (1 for jobs of fewer than 2048 tiles, up to 4 for large ones),
// so that the column sums are grouped the same way whatever other jobs share a launch; small
// chunks keep the CTAs evenly loaded.
__host__ __device__ inline int fwd_chunk_of(int ntiles) {
  const int c = ntiles / 1024;
  return c < 1 ? 1 : (c > 4 ? 4 : c);
}
constexpr int PROW = 4;           // column-partial rows per tile (one per group of 32 voxels)

// Mutable per-job scalars (device memory). Kept apart from JobDev so that a job can
// be listed in several launch lists without its state diverging.
struct JobScal {
  double theta;         // current penalty
  double theta_next;    // penalty of the next iteration
  double lsq;           // ||L||^2 at the last residual check
  double rsq;           // ||Z - A_k(L)V||_F^2 at the last residual check
  double objective;     // ||A_k(L)V||_{2,1} after the run
  int iter;             // iterations completed
  int status;           // 0 ok; nonzero: a bounded device-side wait expired
};

// Per-job device pointers and static info (copied by value into launch lists).
struct JobDev {
  int H, W, T;          // dims
  int nth, ntw;         // voxel tiles along h and w (ceil(H/TH), ceil(W/TW))
  int ntiles;           // nth * ntw * T
  int fchunk;           // fwd_chunk_of(ntiles)
  long long m;          // H*W*T
  double lam;           // INFINITY for the exact projection
  double rho, theta_max;
  JobScal* sc;
  const float* M;       // m, observed values (entries off Omega are ignored)
  const uint8_t* mask;  // m, 1 = observed
  float* L;             // m, current iterate (FP32)
  float* X;             // m, operand of the forward pass (FP32 path)
  __nv_bfloat16* Xc;    // BF16 path: wrap-padded, w-shifted copies of the operand
  void* U;              // m x kc shifted multiplier, row-major [voxel][channel]:
                        //   FP32 (FP32 path) or BF16 (BF16 path)
  float* part;          // column partial sums of ||.||^2: [rows][PROW][kc], one row per
                        //   tile (FP32 passes) or per forward CTA slot (BF16 pass)
  float* rpart;         // per-tile residual partials: [ntiles][nrp]
  float* lpart;         // ||L'||^2 partials: nlp of them (per tile on the FP32 path, per
                        //   1024-voxel block on the BF16 path); room for ntiles
  int nlp;
  double* colseg;       // first-stage column sums: [NSEG][kc]
  float* s;             // kc, shrink factors of this iteration
  float* D;             // kc, 1 - s
  float* G;             // FP32 path: G^T = (V D) U^T, [k][m]; BF16 path: col2im sums Delta [m]
                        //   as 64-bit fixed point (2^-40 units), zero between passes (the
                        //   gather clears what it reads)
  __nv_bfloat16* B2img; // BF16 path: A-operand images of the adjoint pass (V D)
  const void* tmapX;    // BF16 path: TMA map (CUtensorMap, device memory) of Xc, 8 copies
  const void* tmapX2;   // BF16 path: the same with k2 - 8 copies (kernels wider than 8)
  const void* tmapU;    // BF16 path: TMA map of U (box: one tile x 64 channels)
  void* Ulo;            // split forward: the lo part of U (BF16, like U), or null
  const void* tmapUlo;  // split forward: TMA map of Ulo
  int xTp, xHp, xWp;    // BF16 path: dims of each copy in Xc
};

// Shared (per V / per launch list) constants.
struct Shared {
  int k1, k2, k3, k;     // kernel dims along (h, w, t) and k = k1*k2*k3
  int kc;                // channel stride of U (k rounded up to 16)
  int nrp;               // residual partials per tile
  const float* Vf;       // [k taps][kc] FP32, V[s][c] (column c = eigenvector c)
  const __nv_bfloat16* VtImg;  // BF16 forward-pass B images (see k_tc.cu)
  const __nv_bfloat16* VtImgS; // the same for the split forward (hi, then lo), or null
  int njobs;
  const JobDev* jobs;    // device array of njobs
  const int* job_tile0;  // device, njobs + 1 prefix sums of ntiles
  const int* job_chunk0; // device, njobs + 1 prefix sums of ceil(ntiles / fchunk)
  int total_tiles;
  int total_chunks;
  int max_vblk;          // most 1024-voxel blocks of one job in the list
  long long nvox;        // voxels of all jobs in the list (host-side bookkeeping)
};

// Binary search: the job that owns global tile `t`.
__device__ __forceinline__ int job_of_tile(const int* tile0, int njobs, int t) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tile0[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// L-update of Sec. III-D at voxel v, given Delta = [A_k^*(U D V^T)]_v:
//   lambda = inf : L' = M on Omega, L + Delta/(k theta) off Omega;
//   lambda finite: L' = (Delta/k + theta L + lambda Theta M)/(lambda Theta + theta).
// Also writes the next forward operand X = (theta + theta') L' - theta L. Returns L'.
__device__ __forceinline__ float l_update(const JobDev& J, int k, long long v, float d) {
  const float Lo = J.L[v];
  const double th = J.sc->theta;
  const bool obs = J.mask[v] != 0;
  float Ln;
  if (isinf(J.lam)) {
    Ln = obs ? J.M[v] : fmaf(d, (float)(1.0 / (k * th)), Lo);
  } else {
    const double lt = obs ? J.lam : 0.0;
    Ln = (float)(((double)d / k + th * (double)Lo + lt * (obs ? (double)J.M[v] : 0.0)) / (lt + th));
  }
  J.X[v] = fmaf((float)(th + J.sc->theta_next), Ln, -(float)th * Lo);
  J.L[v] = Ln;
  return Ln;
}

// ---------------------------------------------------------------------------------
// Launchers (host). All enqueue on `st` and return cudaGetLastError().
// ---------------------------------------------------------------------------------
// k_common.cu
cudaError_t launch_init_L(const Shared& sh, cudaStream_t st);
// synthetic input of the tile autotuner (smooth values, about half observed)
cudaError_t launch_tune_fill(float* M, uint8_t* mask, int H, int W, int T, cudaStream_t st);
// tpr: tiles per column-partial row group (1: one per tile, the FP32 passes; 0: the job's
// fchunk, the deterministic BF16 forward pass), ceil(ntiles / tpr) row groups per job; tpr
// < 0: one row group per forward CTA slot (-tpr slots, the BF16 forward without
// deterministic reductions), min(-tpr, ntiles) per job.
cudaError_t launch_reduce_cols(const Shared& sh, int advance, int tpr, cudaStream_t st);
cudaError_t launch_theta0(const Shared& sh, double theta0_user, cudaStream_t st);
cudaError_t launch_scale_X(const Shared& sh, cudaStream_t st);
// dst[i] = float(src[i]) (BF16 to FP32 state, for the FP32 finish of a BF16 job)
cudaError_t launch_widen_bf16(const __nv_bfloat16* src, float* dst, long long n, cudaStream_t st);
cudaError_t launch_scalars(const Shared& sh, cudaStream_t st);
cudaError_t launch_gather_fp32(const Shared& sh, cudaStream_t st);
// what: 1 = residual (||L||^2 and residual^2 from the partials), 2 = objective
cudaError_t launch_finish(const Shared& sh, int what, cudaStream_t st);

// k_fp32.cu
// mode: 0 = column norms of A_k(X)V only (no U access); 1 = U' = U D - A_k(X)V;
//       2 = U' = -A_k(X)V (U not read); 3 = residual partials sum (U s/theta + A_k(L)V)^2
//       (no write); 4 = column norms of A_k(L)V (the objective)
cudaError_t launch_fwd_fp32(const Shared& sh, int mode, cudaStream_t st);
cudaError_t launch_adj_gemm_fp32(const Shared& sh, cudaStream_t st);
int fwd_fp32_nrp(int k);

// k_learn.cu
// exact: exact products summed to ~2^-48 relative (diagnostics, column norms); otherwise
// FP32 products summed over 64 voxels, then in FP64.
cudaError_t learn_gram(int b, const float* const* dL, const int* ddims, int k1, int k2, int k3,
                       double* dpart, int nblk, double* dgram, cudaStream_t st, bool exact = false);
// P = V^T G V (dT: k*k scratch), sigma_i = sqrt(P_ii), the support I (sigma_i > tol *
// max(1, max sigma)), S = D P D (D = 1/sigma on I, 0 elsewhere), dout[0] = r_K,
// dout[1] = mu_1(V_I).
cudaError_t diag_spectral(const double* dG, const double* dV, int k, double tol, double* dT, double* dP,
                          double* dsigma, double* dS, double* dout, cudaStream_t st);
size_t learn_smem_bytes(int k1, int k2, int k3);
int learn_max_lags();
cudaError_t learn_eig(double* dA, double* dV, int k, double* devals, double* dVout, int* dinfo,
                      cudaStream_t st);
// The same eigensolver spread over every SM (cooperative launch, grid barriers); dinfo[0]
// = sweeps, dinfo[1] = 1 if a grid barrier timed out. scratch: learn_eig_grid_scratch bytes.
size_t learn_eig_grid_scratch(int dev);
cudaError_t learn_eig_grid(double* dA, double* dV, int k, double* devals, double* dVout, int* dinfo, void* scratch,
                           cudaStream_t st);
// Column norms ||A_k(L) v_c||^2 of one tensor through its Gram (autocorrelations of
// exact products), written into colseg (NSEG x kc: segment 0, the others zero). dpart:
// nblk * (2k1-1)(2k2-1)(2k3-1) doubles, dG: k*k doubles; dV: V column-contiguous (FP64).
cudaError_t gram_colsq(const float* dL, int H, int W, int T, int k1, int k2, int k3, const double* dV, int kc,
                       double* dpart, int nblk, double* dG, double* colseg, cudaStream_t st);
// P = V^T G V (dT: k*k scratch); column j of V is V[j*k ...].
cudaError_t diag_spectral_products(const double* dG, const double* dV, int k, double* dT, double* dP, cudaStream_t st);
cudaError_t check_finite(const float* x, long long n, int* dbad, cudaStream_t st);

// k_cnnm.cu: the CNNM baseline (Eq. cnnm) solved with SVT through the Gram of B.
struct CnnmProblem {
  int H, W, T, k1, k2, k3;
  const float* dM;          // device, m
  const uint8_t* dmask;     // device, m
  float* dL;                // device output, m
  int iters;
  double theta0, rho, theta_max;   // theta0 <= 0: 1/||A_k(P_Omega M)||_2
};
struct CnnmResult {
  double seconds, theta, objective;   // device time; final penalty; ||A_k(L)||_*
  int timed_out;
  int unconverged;   // the eigensolver hit its sweep cap unconverged in some iteration
};
// Pass bracketing for diagnostics: begin(user, pass, kernels, voxels) before the kernels
// of a pass are enqueued, end(user, pass) after. Neither may throw.
struct PassHook {
  void* user = nullptr;
  void (*begin)(void* user, int pass, int nkernels, long long nvox) = nullptr;
  void (*end)(void* user, int pass) = nullptr;
};

// Frequency-domain ICNNM (power-of-two dims; FP32 complex spectra of U and kappa).
// Passes for the hook: 0 = the spectral U update (U' = U D - X^ kappa^), 1 = the spectral
// adjoint sum, 2 = the L-update, 3 = transforms and everything else.
struct FftProblem {
  int device, H, W, T, k1, k2, k3;
  const float* dM;          // device, m
  const uint8_t* dmask;     // device, m
  float* dL;                // device output, m (also the iterate)
  const double* dV;         // device, k*k, eigenvector c at dV[c*k ...]
  int max_iters, check_every;
  double theta0, rho, theta_max, lambda, tol;
  PassHook hook;
};
struct FftResult {
  int iters;
  double residual, objective, theta, seconds;
};
bool fft_supported(int H, int W, int T, std::string* why);
size_t fft_state_bytes(int H, int W, int T, int k);
cudaError_t fft_run(const FftProblem& P, cudaStream_t st, FftResult* res);
size_t cnnm_state_bytes(int H, int W, int T, int k1, int k2, int k3);
cudaError_t cnnm_run(const CnnmProblem& P, cudaStream_t st, CnnmResult* res);
cudaError_t learn_gram_streamed(int b, const float* const* dptrs, const int* ddims, int k1, int k2, int k3,
                                double* dpart, int nblk, double* dlagsum, double* dgram, cudaStream_t st);
cudaError_t check_observed(const float* M, const uint8_t* mask, long long n, int* dcount_bad,
                           cudaStream_t st);

}  // namespace icnnm
