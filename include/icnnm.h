/*
 * icnnm.h — C ABI of the GB300 (sm_103a) ICNNM library (libicnnm.so).
 *
 * ICNNM (Inductive Convolution Nuclear Norm Minimization, arxiv 2604.17001) solves
 * tensor completion with arbitrary sampling (Definition 1, Sec. I): recover
 * L0 (H x W x T) from the entries P_Omega(L0) at an arbitrary sampling set Omega.
 * It solves, for a fixed orthogonal k x k matrix V of pre-learned convolution
 * eigenvectors (the paper's K),
 *
 *     min_L ||A_k(L) V||_{2,1}  s.t. P_Omega(L) = P_Omega(M)          (Eq. InductiveCNNM)
 *  or min_L ||A_k(L) V||_{2,1} + (lambda k / 2)||P_Omega(L - M)||_F^2  (Eq. admm)
 *
 * by ADMM (Sec. III-D), and learns V from reference tensors (Sec. III-C, Eq. A).
 *
 * Conventions shared by every call
 *  - A tensor of dims {H, W, T} is a float array of m = H*W*T entries, w fastest:
 *    index i = (t*H + h)*W + w. An image (ndim = 2) has T = 1 and kdims[2] = 1.
 *  - Kernel dims {k1, k2, k3} run along (h, w, t); k = k1*k2*k3; tap index
 *    s = (st*k1 + sh)*k2 + sw. The convolution is circular in every dimension
 *    (Sec. II-B), and every dim must be at least the kernel's (H >= k1, ...).
 *  - V is k*k doubles, column-major: V[i*k + s] is tap s of eigenvector i
 *    (eigenvector i contiguous), orthonormal to 1e-6.
 *  - Pointer arguments may be host or device memory of the context's device; the
 *    library detects which. The caller owns every buffer. Inputs are copied before
 *    icnnm_solve / icnnm_submit return; outputs are written before the call that
 *    fills them returns.
 *  - Calls never abort the process; every failure is a status code, and
 *    icnnm_last_error() returns a message describing the last failure on the
 *    calling thread's context.
 */
#ifndef ICNNM_H_
#define ICNNM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct icnnm_ctx icnnm_ctx;

typedef enum {
  ICNNM_OK = 0,
  ICNNM_EINVAL = 1,      /* invalid argument: shapes, V, mask, params, non-finite input */
  ICNNM_ENOMEM = 2,      /* the job's device state exceeds the context's HBM budget */
  ICNNM_EAGAIN = 3,      /* icnnm_poll: the job is queued or running */
  ICNNM_ENOTFOUND = 4,   /* unknown job id (or its result was already collected) */
  ICNNM_ECUDA = 5,       /* a CUDA runtime/driver call or a kernel failed */
  ICNNM_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
  ICNNM_ECANCELED = 7,   /* the job was cancelled */
  ICNNM_EUNSUPPORTED = 8, /* a valid request this build does not implement */
  ICNNM_ENOCONV = 9      /* the FP64 Jacobi eigensolver reached its sweep cap with the
                            off-diagonal norm still above 1e-10 of the matrix norm */
} icnnm_status;

typedef enum {
  ICNNM_FP32 = 0,        /* every product in FP32 on CUDA cores (the plain baseline) */
  ICNNM_BF16 = 1,        /* A_k(.)V and A_k^*(. V^T) on tcgen05 tensor cores: BF16
                            operands, FP32 accumulation; L, norms and updates in FP32.
                            With tol > 0 a job finishes in BF16X3 (where built for its
                            kernel, else in FP32), since BF16 rounding floors the residual
                            near 1e-3. Kernels with k <= 512; EUNSUPPORTED above (FP32
                            takes k up to 1024) */
  ICNNM_BF16X3 = 2       /* as BF16, but the forward pass A_k(X)V splits X and V into hi +
                            lo BF16 pairs (three products into one FP32 accumulator, about
                            2^-16 relative) and keeps U as a hi + lo pair; the adjoint stays
                            BF16. About 1e-6 from the FP64 oracle where BF16 is near 1e-3.
                            Built where the split forward fits in shared memory (k up to
                            about 150); EUNSUPPORTED otherwise */
} icnnm_precision;

typedef struct {
  int32_t ndim;          /* 2 (image) or 3 (video) */
  int64_t dims[3];       /* {H, W, T}; T = 1 when ndim == 2 */
  int64_t kdims[3];      /* {k1, k2, k3}; k3 = 1 when ndim == 2 */
} icnnm_shape;

typedef struct {
  double lambda;         /* INFINITY: exact projection P_Omega(L) = P_Omega(M) (Eq.
                            InductiveCNNM); finite > 0: penalised form (Eq. admm, the
                            paper uses 1000) */
  double theta0;         /* initial penalty; <= 0 selects 1/||A_k(P_Omega M) V||_{2,inf} */
  double rho;            /* penalty growth theta <- min(rho*theta, theta_max), rho >= 1 */
  double theta_max;
  int32_t max_iters;     /* iteration cap (>= 1) */
  double tol;            /* stop when ||Z - A_k(L)V||_F/(sqrt(k)||L||_F) <= tol; 0: run
                            exactly max_iters iterations */
  int32_t check_every;   /* residual cadence when tol > 0 (>= 1) */
  int32_t prec;          /* icnnm_precision */
} icnnm_params;

typedef struct {
  int32_t iters;         /* iterations run */
  double residual;       /* ||Z - A_k(L)V||_F/(sqrt(k)||L||_F) at the last check */
  double objective;      /* ||A_k(L)V||_{2,1} of the returned L */
  double theta;          /* final penalty */
  double seconds;        /* blocking solves: device time of the solve (CUDA events);
                            served jobs: seconds from admission to completion */
  double latency;        /* served jobs: seconds from icnnm_submit to completion (queueing
                            included); blocking solves: the same as seconds */
} icnnm_stats;

/* Fill *p with the defaults: lambda = INFINITY, theta0 = 0 (automatic), rho = 1.1,
 * theta_max = 1e10, max_iters = 100, tol = 0, check_every = 10, prec = ICNNM_BF16. */
icnnm_status icnnm_params_default(icnnm_params* p);

/* Create a context on CUDA device `device`. `hbm_budget_bytes` caps the device
 * memory of job state (0: 90% of the free memory at creation). `cuda_stream` is a
 * cudaStream_t the context orders its work on (NULL: the context creates its own).
 * ENOMEM if the budget cannot be reserved, ECUDA on device errors. */
icnnm_status icnnm_create(icnnm_ctx** out, int device, size_t hbm_budget_bytes,
                          void* cuda_stream);

/* Wait for running jobs to finish, cancel queued ones, free everything. NULL-safe. */
void icnnm_destroy(icnnm_ctx* ctx);

/* Static message of a status code. */
const char* icnnm_strerror(icnnm_status st);

/* Message of the last failure of a call on this context ("" if none). */
const char* icnnm_last_error(icnnm_ctx* ctx);

/*
 * Learn V from b reference tensors (Sec. III-C, Definition 3, Eq. A): V's columns
 * are the eigenvectors of A^T A, A = [A_k(L_1); ...; A_k(L_b)], by decreasing
 * eigenvalue. A^T A is accumulated on the GPU (FP32 products, FP64 sums) and its
 * eigendecomposition is computed in FP64 on the GPU. Each column's largest-|.|
 * entry is made positive (ties: lowest index).
 *   kdims   : {k1, k2, k3}
 *   shapes  : b shapes (dims may differ between tensors; kdims in them are ignored)
 *   tensors : b pointers to float tensors (host or device)
 *   V_out   : k*k doubles, column-major as above (caller-owned, host or device)
 *   eig_out : k doubles, the eigenvalues (the ensemble convolution eigenvalues
 *             sigma_i of Definition 3), or NULL
 * EINVAL: b < 1, k < 1, k > 1024, a dim smaller than the kernel, non-finite entry.
 * EUNSUPPORTED: more autocorrelation lags or a larger halo than the Gram kernel takes.
 * ENOCONV: the eigensolver did not converge (V_out and eig_out are then unreliable).
 * ETIMEOUT: a bounded grid barrier of the eigensolver expired.
 */
icnnm_status icnnm_learn_V(icnnm_ctx* ctx, const int64_t kdims[3], int32_t b,
                           const icnnm_shape* shapes, const float* const* tensors,
                           double* V_out, double* eig_out);

/*
 * Solve one completion problem and block until done (Sec. III-D).
 *   shape  : dims and kernel dims
 *   M      : m floats; only entries with mask = 1 are read
 *   mask   : m bytes, 1 = observed (in Omega), 0 = missing
 *   V      : k*k doubles as above
 *   params : NULL for the defaults
 *   L_out  : m floats, the completed tensor; with lambda = INFINITY its observed
 *            entries are bit-identical copies of M
 *   stats  : may be NULL
 * EINVAL: bad shape, V not orthonormal to 1e-6, empty Omega, non-finite M at an
 * observed entry, bad params. ENOMEM: the job's state does not fit the budget.
 */
icnnm_status icnnm_solve(icnnm_ctx* ctx, const icnnm_shape* shape, const float* M,
                         const uint8_t* mask, const double* V, const icnnm_params* params,
                         float* L_out, icnnm_stats* stats);

/*
 * Solve n independent problems of any dims that share kernel dims and V, stepping
 * all of them together (one launch per pass for the whole batch). Arrays hold n
 * entries each; params (NULL: defaults) apply to every problem.
 */
icnnm_status icnnm_solve_batch(icnnm_ctx* ctx, int32_t n, const icnnm_shape* shapes,
                               const float* const* M, const uint8_t* const* mask,
                               const double* V, const icnnm_params* params,
                               float* const* L_out, icnnm_stats* stats);

/*
 * CNNM, the method ICNNM is compared with (Eq. cnnm; Sec. II-C; Tables II and IV):
 *     min_L ||A_k(L)||_*  s.t. P_Omega(L) = P_Omega(M),
 * by the same ADMM iteration with the Z-update done by singular-value thresholding of
 * A_k(L) - Y/theta at 1/theta, i.e. an SVD of an m x k matrix every iteration. On the
 * GPU the SVD goes through the k x k Gram of that matrix (FP64 sums of exact products)
 * and the FP64 Jacobi eigensolver, warm-started from the previous iteration's singular
 * vectors; everything else is plain FP32. theta0 <= 0 selects 1/||A_k(P_Omega M)||_2.
 *   shape, M, mask, L_out : as for icnnm_solve (no V)
 *   params : NULL for the defaults; lambda must be INFINITY, tol 0 (runs exactly
 *            max_iters iterations) and prec ICNNM_FP32, else EUNSUPPORTED
 *   stats  : iters, objective = ||A_k(L)||_* of the result, theta = final penalty,
 *            seconds; residual is 0 (not computed). May be NULL.
 * EINVAL as for icnnm_solve; ENOMEM if the state (two k x m FP32 arrays plus O(m + k^2))
 * exceeds the budget; ETIMEOUT if a bounded grid barrier of the eigensolver expired;
 * ENOCONV if the eigensolver failed to converge in any iteration.
 */
icnnm_status icnnm_cnnm_solve(icnnm_ctx* ctx, const icnnm_shape* shape, const float* M,
                              const uint8_t* mask, const icnnm_params* params, float* L_out,
                              icnnm_stats* stats);

/*
 * Solve one completion problem as icnnm_solve does (Sec. III-D, the same ADMM iteration,
 * initial state and stopping rule), computing in the frequency domain. The convolution
 * of Sec. II-B is circular, so A_k(X)V has the 3-D DFT X^ kappa_c^ in column c (kappa_c:
 * eigenvector c laid out as a k1 x k2 x k3 kernel), A_k^*(U D V^T) has the DFT
 * sum_c D_c U_c^ conj(kappa_c^), and column norms follow from Parseval. Each U_c^ stays a
 * multiple of kappa_c^, so the state is y_c = U_c^ conj(kappa_c^) (FP32 complex) and
 * q_c = |kappa_c^|^2 (FP32) over the H*T*(W/2+1) frequencies of a real transform; an
 * iteration streams y once and y and q once more (about 14*k*m bytes) and transforms one
 * tensor each way, in place of the two m x k x k products.
 *   shape, M, mask, V, L_out : as for icnnm_solve
 *   params : as for icnnm_solve; prec is ignored (the spectra are FP32 complex, the
 *            norms FP64)
 *   stats  : as for icnnm_solve; seconds = device time of the solve including the
 *            transforms of the k kernels
 * EINVAL as for icnnm_solve. EUNSUPPORTED unless H, W, T are powers of two with
 * 2 <= W <= 1024, H <= 1024, T <= 1024 and H*T >= 2. ENOMEM if the state (12 bytes per
 * frequency and eigenvector, k*H*T*(W/2+1) of them, plus O(16 m)) exceeds the budget.
 */
icnnm_status icnnm_solve_fft(icnnm_ctx* ctx, const icnnm_shape* shape, const float* M,
                             const uint8_t* mask, const double* V, const icnnm_params* params,
                             float* L_out, icnnm_stats* stats);

/*
 * Relative convolution diagnostics of a tensor L0 with respect to V (Sec. III-A,
 * Definition 2, Eqs. rkL0 and alphaK; the coherence of Eq. coherence):
 *   sigma_i = ||L0 * kappa_i||_F = ||A_k(L0) v_i||_2   (relative convolution eigenvalues)
 *   r_K     = |I|, I = {i : sigma_i > rank_tol * max(1, max_j sigma_j)}   (the paper counts
 *             the nonzero sigma_i; rank_tol is the numerical reading of "nonzero")
 *   alpha_K = ||A_k(L0) V D|| (operator norm), D_ii = 1/sigma_i on I, 0 elsewhere
 *   mu_K    = mu_1(V_I), V_I the columns of V on I: (k / r_K) max_s sum_{i in I} V[i*k+s]^2
 * Computed on the GPU through G = A_k(L0)^T A_k(L0) (circular autocorrelations of exact
 * products, summed to ~2^-48 relative): sigma_i^2 = v_i^T G v_i, and alpha_K^2 is the
 * largest eigenvalue of D V^T G V D (FP64 Jacobi). Squaring limits the resolution: a sigma_i that is zero
 * in exact arithmetic comes out near sqrt(k * 1e-16) * max sigma, so rank_tol should be
 * at least 1e-6.
 *   shape    : dims and kdims of L0
 *   L0       : m floats (host or device)
 *   V        : k*k doubles as above
 *   rank_tol : in (0, 1)
 *   sigma_out: k doubles in V's column order (host or device), or NULL
 *   r_K, alpha_K, mu_K : host outputs, each may be NULL (alpha_K = mu_K = 0 when I is empty)
 * EINVAL: bad shape, V not orthonormal to 1e-6, non-finite L0, rank_tol outside (0, 1).
 * ETIMEOUT: a bounded grid barrier of the eigensolver expired. ENOCONV: the eigensolver
 * that gives alpha_K did not converge.
 */
icnnm_status icnnm_spectral_diagnostics(icnnm_ctx* ctx, const icnnm_shape* shape, const float* L0,
                                        const double* V, double rank_tol, double* sigma_out,
                                        int32_t* r_K, double* alpha_K, double* mu_K);

/*
 * Serving. icnnm_submit validates and copies the inputs, queues the job and returns
 * at once with its id. A serving thread admits queued jobs while their device state
 * fits the HBM budget, keeps admitted jobs resident, and steps all admitted jobs that
 * share (kdims, V, precision) together, admitting new ones as others finish
 * (continuous batching). ENOMEM only if the job alone exceeds the whole budget.
 */
icnnm_status icnnm_submit(icnnm_ctx* ctx, const icnnm_shape* shape, const float* M,
                          const uint8_t* mask, const double* V, const icnnm_params* params,
                          uint64_t* job_id);

/* EAGAIN while queued or running. On completion copies L into L_out (m floats,
 * may be NULL to drop it), fills stats (may be NULL), forgets the job, returns OK
 * (or the job's failure status). ENOTFOUND for unknown ids. */
icnnm_status icnnm_poll(icnnm_ctx* ctx, uint64_t job_id, float* L_out, icnnm_stats* stats);

/* Like icnnm_poll, but waits up to timeout_ms (< 0: forever) for completion. */
icnnm_status icnnm_wait(icnnm_ctx* ctx, uint64_t job_id, int64_t timeout_ms,
                        float* L_out, icnnm_stats* stats);

/* Cancel a queued or running job; a later poll returns ECANCELED. */
icnnm_status icnnm_cancel(icnnm_ctx* ctx, uint64_t job_id);

/*
 * Diagnostics (no counterpart in the paper). While profiling is enabled the library
 * brackets each pass of the blocking solves with CUDA events on the context's stream
 * and counts every kernel it launches.
 *   icnnm_profile_enable : enable (1) or disable (0); either resets the counters.
 *   icnnm_profile_read   : pass 0 = forward pass A_k(X)V fused with the U update (BF16),
 *                          1 = adjoint pass (V D)U^T with col2im, 2 = gather/projection
 *                          (L-update), 3 = everything else, 4 = forward pass of BF16X3
 *                          jobs, 5 = forward pass of FP32 jobs; ms_total = summed device
 *                          time, launches = kernels of that pass (pass -1: all kernels,
 *                          ms_total = 0). EINVAL for other pass ids.
 */
icnnm_status icnnm_profile_enable(icnnm_ctx* ctx, int32_t enable);
icnnm_status icnnm_profile_read(icnnm_ctx* ctx, int32_t pass, double* ms_total, int64_t* launches);
/* Voxels the launches of a pass processed since profiling was last enabled or disabled
 * (the sum over its launches of the voxels of the jobs each launch stepped); pass ids as
 * for icnnm_profile_read (-1: all passes). Counted whether or not timing is enabled. */
icnnm_status icnnm_profile_voxels(icnnm_ctx* ctx, int32_t pass, int64_t* voxels);

/*
 * Tile configuration of the tensor-core passes for one kernel size (no counterpart in the
 * paper; a performance choice that leaves every result unchanged up to the order of FP32
 * additions). Each field is an upper bound (the widest tile that fits in shared memory
 * below it is taken); 0 keeps the default, the narrow tile (128 / 128 / 2):
 *   adj_tap_width     : columns of an adjoint tap tile, 128 or 256 (256 where the V D image
 *                       of the wider tile fits in shared memory)
 *   fwd_channel_width : channels of a forward channel tile, 128 or 256 (256: one tile of all
 *                       channels when k <= 256 and it fits)
 *   fwd_u_stages      : shared-memory stages of the forward's U tiles, 1 or 2
 */
typedef struct {
  int32_t adj_tap_width;
  int32_t fwd_channel_width;
  int32_t fwd_u_stages;
} icnnm_tile_config;

typedef struct {
  icnnm_tile_config cfg;  /* the candidate (upper bounds as passed to the geometry) */
  int32_t adj_tap_width;  /* what the geometry took: tap-tile columns */
  int32_t fwd_channel_width; /* channel-tile width taken */
  int32_t fwd_u_stages;   /* U stages taken */
  double ms_per_iter;     /* measured device time of one iteration of all the jobs */
} icnnm_tile_result;

/*
 * Deterministic reductions of the BF16 path (on by default; no counterpart in the paper).
 * On: the col2im sums of the adjoint pass are 64-bit fixed point (2^-40 units, whose
 * additions are associative) and the forward pass keeps its column partials per fixed chunk
 * of each job's tiles, so a job's result is the same, bit for bit, alone, in any batch or
 * serving mix, and from run to run. Off: float atomics and a round-robin tile order, faster
 * on large kernels (k = 405: about 20%) but reproducible only to rounding. Applies to V data
 * built after the call (set it before the first BF16 solve of a V).
 */
icnnm_status icnnm_set_deterministic(icnnm_ctx* ctx, int32_t on);

/*
 * Use cfg for BF16 work with these kernel dims from now on in this context (V data built
 * before the call keep their tiles). EINVAL for widths other than 0/128/256 or stages
 * other than 0/1/2.
 */
icnnm_status icnnm_set_tile_config(icnnm_ctx* ctx, const int64_t kdims[3], const icnnm_tile_config* cfg);

/*
 * Autotuner of the tile configuration: for every distinct tile geometry the candidates
 * give, builds the tensor-core data of V, creates n synthetic jobs of the given shapes
 * (smooth values, about half the voxels observed), runs `iters` BF16 iterations of all of
 * them stepped together, and times them with CUDA events on the context's stream. The
 * fastest becomes the context's configuration for these kernel dims (as by
 * icnnm_set_tile_config) and is returned in *best; results (capacity max_results, may be
 * NULL) receive every measured candidate and *n_results their count. Blocking; needs the
 * device memory of the n jobs within the budget.
 */
icnnm_status icnnm_autotune(icnnm_ctx* ctx, const double* V, int32_t n, const icnnm_shape* shapes,
                            int32_t iters, icnnm_tile_config* best, icnnm_tile_result* results,
                            int32_t max_results, int32_t* n_results);

/*
 * Device bytes of the state of one job of this shape in this precision (the amount the
 * HBM budget is charged at admission; a BF16 job with a tolerance may take more for its
 * FP32 finish). For callers that size a context's budget. V is not needed: kdims decide.
 * EINVAL: bad shape or precision; EUNSUPPORTED: BF16 is not built for these kernel dims.
 */
icnnm_status icnnm_job_bytes(icnnm_ctx* ctx, const icnnm_shape* shape, int32_t prec, size_t* bytes);

/*
 * Check of the bounded device-side waits (no counterpart in the paper): one thread block
 * waits, through the same bounded wait as the solve kernels, on a barrier that nothing
 * completes, for limit_ns nanoseconds (1 ms .. 10 s). Returns ETIMEOUT once that wait has
 * given up and the kernel has returned, which is what a solve reports when one of its
 * waits expires; the context stays usable. EINVAL for a limit outside the range.
 */
icnnm_status icnnm_check_bounded_wait(icnnm_ctx* ctx, int64_t limit_ns);

/*
 * Allocation-free learning of V (the paper has no counterpart; this is an interface for
 * callers, not a step of the method). It computes what icnnm_learn_V computes (the same
 * Gram accumulation and FP64 eigensolver, summed in a different fixed order, on one
 * thread block) but never allocates: it calls no cudaMalloc/cudaFree, creates no
 * context, and uses no allocating library routine. It is meant for callers that cannot
 * allocate device memory themselves: code inside a framework that hands out device
 * memory only from its own pool (so a cudaMalloc behind its back would break its
 * accounting or fail against its reservation), and latency-critical code that must avoid
 * the device-wide synchronisation a cudaMalloc/cudaFree can cause.
 *   kdims, b, shapes : as for icnnm_learn_V
 *   tensors          : b pointers to float tensors in device memory of the current device
 *   V_out, eig_out   : as for icnnm_learn_V (host memory, or device memory of the current
 *                      device; eig_out may be NULL)
 *   cuda_stream      : cudaStream_t to run on (NULL: the legacy default stream)
 * All intermediates live in one fixed device array (about 2.1 MiB) that every GPU
 * loading this library keeps until the process exits. Limits: k <= 256,
 * (2k1-1)(2k2-1)(2k3-1) <= 4096, 1 <= b <= 256; larger requests return EINVAL and
 * icnnm_noalloc_last_error() says which limit. A kernel whose Gram halo needs more than
 * 220 KiB of shared memory (for example 256 x 1 x 1) returns EUNSUPPORTED. A pointer on
 * another device returns EINVAL. ENOCONV: the eigensolver did not converge.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and so must not be the first CUDA call of a thread that has no current device. The
 * call is blocking: it synchronises cuda_stream twice (after the finiteness check of the
 * inputs and before returning). Every call reuses the same array and leaves its contents
 * behind, so calls that may overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller.
 */
icnnm_status icnnm_learn_V_noalloc(const int64_t kdims[3], int32_t b, const icnnm_shape* shapes,
                                   const float* const* tensors, double* V_out, double* eig_out,
                                   void* cuda_stream);

/* Message of the last failure of icnnm_learn_V_noalloc on the calling thread. */
const char* icnnm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ICNNM_H_ */
