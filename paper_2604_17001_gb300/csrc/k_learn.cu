// Learning V (Sec. III-C, Definition 3, Eq. A): the eigenvectors of A^T A with
// A = [A_k(L_1); ...; A_k(L_b)].
//
// Entry (u, s) of A_k(L)^T A_k(L) is sum_i L[i-u] L[i-s] = R[u - s], the circular
// autocorrelation R[d] = sum_i L[i] L[i+d] of L at the lag u - s (each coordinate
// in (-k_j, k_j)). So the Gram needs prod_j (2 k_j - 1) autocorrelation lags per
// tensor instead of the k^2 dot products of length m of the direct product; the
// autocorrelations are data-parallel over tensors and voxel bricks (FP32 products,
// summed in FP32 over 64 voxels, then in FP64).
//
// The FP64 eigendecomposition is a parallel cyclic Jacobi method (round-robin pair
// ordering: every round rotates k/2 disjoint pairs, rows first, then columns).
#include <math.h>
#include "icnnm_internal.h"

namespace icnnm {

namespace {

constexpr int BW = 16, BH = 16, BT = 8;      // autocorrelation brick
constexpr int AC_THREADS = 256;
constexpr int AC_MAXLAG_PER_THREAD = 16;     // supports up to 4096 lags

struct LearnArgs {
  int b;
  const float* const* L;     // device array of b device pointers (NULL: the one tensor L1)
  const int* dims;           // device, 3*b: H, W, T
  const float* L1;           // b = 1 without device arrays: the tensor and its dims
  int H1, W1, T1;
  int k1, k2, k3;
  int nl1, nl2, nl3, nlag;   // 2k-1 per dim and their product
  int nblk;                  // blocks per tensor
  double* part;              // [b][nblk][nlag]
};

// Lag index l <-> (dt, dh, dw) with dt in [-(k3-1), k3-1] etc, l = ((dt+k3-1)*nl1 + dh+k1-1)*nl2 + dw+k2-1.
// EXACT: every product kept exactly and summed to about 2^-48 relative (float pairs, see
// below), for the diagnostics and the column norms, whose smallest entries need it.
template <bool EXACT>
__global__ void __launch_bounds__(AC_THREADS) autocorr_kernel(LearnArgs a) {
  extern __shared__ float sL[];
  const int j = blockIdx.x;
  const int H = a.L ? a.dims[3 * j] : a.H1, W = a.L ? a.dims[3 * j + 1] : a.W1, T = a.L ? a.dims[3 * j + 2] : a.T1;
  const float* L = a.L ? a.L[j] : a.L1;
  const int ew = BW + 2 * (a.k2 - 1), eh = BH + 2 * (a.k1 - 1), et = BT + 2 * (a.k3 - 1);
  const int nbw = (W + BW - 1) / BW, nbh = (H + BH - 1) / BH, nbt = (T + BT - 1) / BT;
  const int nbr = nbw * nbh * nbt;
  double acc[AC_MAXLAG_PER_THREAD];
  int lagoff[AC_MAXLAG_PER_THREAD];
  int nmy = 0;
  for (int l = threadIdx.x; l < a.nlag && nmy < AC_MAXLAG_PER_THREAD; l += AC_THREADS) {
    const int dw = l % a.nl2 - (a.k2 - 1);
    const int dh = (l / a.nl2) % a.nl1 - (a.k1 - 1);
    const int dt = l / (a.nl2 * a.nl1) - (a.k3 - 1);
    lagoff[nmy] = (dt * eh + dh) * ew + dw;
    acc[nmy] = 0.0;
    ++nmy;
  }
  for (int br = blockIdx.y; br < nbr; br += gridDim.y) {
    const int bw = br % nbw, bh = (br / nbw) % nbh, bt = br / (nbw * nbh);
    const int w0 = bw * BW - (a.k2 - 1), h0 = bh * BH - (a.k1 - 1), t0 = bt * BT - (a.k3 - 1);
    __syncthreads();
    for (int e = threadIdx.x; e < ew * eh * et; e += AC_THREADS) {
      const int x = e % ew, y = (e / ew) % eh, z = e / (ew * eh);
      sL[e] = L[((long long)wrapi(t0 + z, T) * H + wrapi(h0 + y, H)) * W + wrapi(w0 + x, W)];
    }
    __syncthreads();
    const int vw = min(BW, W - bw * BW), vh = min(BH, H - bh * BH), vt = min(BT, T - bt * BT);
    for (int q = 0; q < nmy; ++q) {
      if (EXACT) {
        // every product a*b is split exactly into p + e (p = a*b rounded, e = fma(a, b, -p))
        // and summed over the brick as an unevaluated float pair hi + lo (Knuth's TwoSum
        // for p, e added to lo): about 2^-48 relative per term, on the FP32 pipe; the pair
        // goes to FP64 once per brick
        float hi = 0.f, lo = 0.f;
        for (int z = 0; z < vt; ++z)
          for (int y = 0; y < vh; ++y) {
            const int base = ((z + a.k3 - 1) * eh + (y + a.k1 - 1)) * ew + (a.k2 - 1);
            for (int x = 0; x < vw; ++x) {
              const float av = sL[base + x], bv = sL[base + x + lagoff[q]];
              const float p = __fmul_rn(av, bv);
              const float e = __fmaf_rn(av, bv, -p);
              const float s = __fadd_rn(hi, p);
              const float bb = __fsub_rn(s, hi);
              const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
              hi = s;
              lo = __fadd_rn(lo, __fadd_rn(err, e));
            }
          }
        acc[q] += (double)hi + (double)lo;
        continue;
      }
      float part = 0.f;
      int cnt = 0;
      for (int z = 0; z < vt; ++z)
        for (int y = 0; y < vh; ++y) {
          const int base = ((z + a.k3 - 1) * eh + (y + a.k1 - 1)) * ew + (a.k2 - 1);
          for (int x = 0; x < vw; ++x) {
            part = fmaf(sL[base + x], sL[base + x + lagoff[q]], part);
            if (++cnt == 64) { acc[q] += (double)part; part = 0.f; cnt = 0; }
          }
        }
      acc[q] += (double)part;
    }
  }
  int q = 0;
  for (int l = threadIdx.x; l < a.nlag && q < AC_MAXLAG_PER_THREAD; l += AC_THREADS, ++q)
    a.part[((long long)j * a.nblk + blockIdx.y) * a.nlag + l] = acc[q];
}

// Gram[u][s] = sum_j sum_blk part[j][blk][lag(u - s)], summed in a fixed order. The
// circular autocorrelation is even, R(d) = R(-d), but the two lags are summed from
// different products, so they agree only to rounding (about 1e-7 relative with FP32
// products); G takes their average, which makes it exactly symmetric (IEEE addition
// commutes), as the symmetric Jacobi eigensolver needs: an antisymmetric part survives
// every rotation and would hold the off-diagonal norm at its size. The lag index of
// s - u is nlag - 1 - lag(u - s).
__global__ void gram_kernel(LearnArgs a, double* gram) {
  const int k = a.k1 * a.k2 * a.k3;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)k * k) return;
  const int u = (int)(idx / k), s = (int)(idx % k);
  const int uw = u % a.k2, uh = (u / a.k2) % a.k1, ut = u / (a.k1 * a.k2);
  const int sw = s % a.k2, shh = (s / a.k2) % a.k1, st = s / (a.k1 * a.k2);
  const int l = ((ut - st + a.k3 - 1) * a.nl1 + (uh - shh + a.k1 - 1)) * a.nl2 + (uw - sw + a.k2 - 1);
  const int lm = a.nlag - 1 - l;
  double g = 0.0, gm = 0.0;
  for (int j = 0; j < a.b; ++j)
    for (int bb = 0; bb < a.nblk; ++bb) {
      g += a.part[((long long)j * a.nblk + bb) * a.nlag + l];
      gm += a.part[((long long)j * a.nblk + bb) * a.nlag + lm];
    }
  gram[idx] = 0.5 * (g + gm);
}

// ---------------------------------------------------------------------------------
// FP64 parallel cyclic Jacobi on one thread block. A (k x k, row-major, symmetric) is
// overwritten; V (k x k) accumulates the rotations. Each sweep runs n-1 rounds of the
// circle (round-robin) schedule on n = k rounded up to even; index k is a dummy.
// Stops when the off-diagonal Frobenius norm is <= tol * ||A||_F or after max_sweeps.
// info[0] = sweeps run, or JACOBI_UNCONVERGED if after max_sweeps the off-diagonal norm
// is still above JACOBI_ACCEPT * ||A||_F (a cyclic Jacobi converges quadratically, so
// that only happens when something is wrong); the flag is sticky while the caller does
// not reset info[0] (CNNM runs the solver every iteration and reads info once).
// ---------------------------------------------------------------------------------
constexpr int JACOBI_UNCONVERGED = -1;
constexpr double JACOBI_ACCEPT = 1e-10;
constexpr int EIG_THREADS = 1024;
constexpr int EIG_MAXK = 1024;

// Sort by decreasing eigenvalue (stable: ties by index), make the largest-|.| entry of each
// eigenvector positive (ties: lowest index), write the vectors column by column. One block.
__device__ void eig_sort_sign(const double* A, const double* V, int k, double* evals_out, double* Vout, double* ev,
                              int* order) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) ev[i] = A[(long long)i * k + i];
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    int rank = 0;
    for (int j = 0; j < k; ++j) rank += (ev[j] > ev[i]) || (ev[j] == ev[i] && j < i);
    order[rank] = i;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < k; o += blockDim.x) {
    const int i = order[o];
    int amax = 0;
    double vmax = -1.0;
    for (int srow = 0; srow < k; ++srow) {
      const double a = fabs(V[(long long)srow * k + i]);
      if (a > vmax) { vmax = a; amax = srow; }
    }
    const double sg = V[(long long)amax * k + i] < 0 ? -1.0 : 1.0;
    for (int srow = 0; srow < k; ++srow) Vout[(long long)o * k + srow] = sg * V[(long long)srow * k + i];
    evals_out[o] = ev[i];
  }
}

__global__ void __launch_bounds__(EIG_THREADS)
jacobi_kernel(double* A, double* V, int k, int max_sweeps, double tol, double* evals_out,
              double* Vout, int* info) {
  __shared__ double cs[EIG_MAXK / 2], sn[EIG_MAXK / 2];
  __shared__ int pp[EIG_MAXK / 2], qq[EIG_MAXK / 2];
  __shared__ double red[EIG_THREADS];
  __shared__ int order[EIG_MAXK];
  __shared__ double ev[EIG_MAXK];
  const int n = (k + 1) & ~1;
  const int npair = n / 2;
  for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x)
    V[e] = (e / k == e % k) ? 1.0 : 0.0;
  __syncthreads();
  // ||A||_F for the stopping test
  double fr = 0.0;
  for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) fr += A[e] * A[e];
  red[threadIdx.x] = fr;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double normA = sqrt(red[0]);
  __syncthreads();
  int sweep = 0;
  bool unconv = false;
  for (;; ++sweep) {
    double off = 0.0;
    for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x)
      if (e / k != e % k) off += A[e] * A[e];
    red[threadIdx.x] = off;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    const double offn = sqrt(red[0]);
    __syncthreads();
    if (offn <= tol * normA) break;
    if (sweep == max_sweeps) {
      unconv = offn > JACOBI_ACCEPT * normA;
      break;
    }
    for (int r = 0; r < n - 1; ++r) {
      for (int i = threadIdx.x; i < npair; i += blockDim.x) {
        int p, q;
        if (i == 0) { p = r; q = n - 1; }
        else { p = (r + i) % (n - 1); q = (r - i + (n - 1)) % (n - 1); }
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < k) {
          const double apq = A[(long long)p * k + q];
          if (apq != 0.0) {
            const double app = A[(long long)p * k + p], aqq = A[(long long)q * k + q];
            const double th = (aqq - app) / (2.0 * apq);
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
      }
      __syncthreads();
      // rows: A[p][:], A[q][:] <- c A[p] - s A[q], s A[p] + c A[q]
      for (long long e = threadIdx.x; e < (long long)npair * k; e += blockDim.x) {
        const int i = (int)(e / k), col = (int)(e % k);
        const int p = pp[i], q = qq[i];
        if (q >= k || sn[i] == 0.0) continue;
        const double c = cs[i], s = sn[i];
        const double ap = A[(long long)p * k + col], aq = A[(long long)q * k + col];
        A[(long long)p * k + col] = c * ap - s * aq;
        A[(long long)q * k + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns of A and of V
      for (long long e = threadIdx.x; e < (long long)npair * k; e += blockDim.x) {
        const int i = (int)(e / k), row = (int)(e % k);
        const int p = pp[i], q = qq[i];
        if (q >= k || sn[i] == 0.0) continue;
        const double c = cs[i], s = sn[i];
        const double ap = A[(long long)row * k + p], aq = A[(long long)row * k + q];
        A[(long long)row * k + p] = c * ap - s * aq;
        A[(long long)row * k + q] = s * ap + c * aq;
        const double vp = V[(long long)row * k + p], vq = V[(long long)row * k + q];
        V[(long long)row * k + p] = c * vp - s * vq;
        V[(long long)row * k + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  eig_sort_sign(A, V, k, evals_out, Vout, ev, order);
  if (threadIdx.x == 0) info[0] = (unconv || info[0] == JACOBI_UNCONVERGED) ? JACOBI_UNCONVERGED : sweep;
}


// Rotation of pair slot i of round r of the round-robin ordering on n (even) indices:
// p < q, and (c, s) zeroing A[p][q] (c = 1, s = 0 for a padding index or A[p][q] = 0).
__device__ __forceinline__ void jacobi_pair(const double* A, int k, int n, int r, int i, int& p, int& q, double& c,
                                            double& s) {
  if (i == 0) { p = r; q = n - 1; }
  else { p = (r + i) % (n - 1); q = (r - i + (n - 1)) % (n - 1); }
  if (p > q) { const int t = p; p = q; q = t; }
  c = 1.0;
  s = 0.0;
  if (q < k) {
    const double apq = __ldcg(A + (long long)p * k + q);
    if (apq != 0.0) {
      const double app = __ldcg(A + (long long)p * k + p), aqq = __ldcg(A + (long long)q * k + q);
      const double th = (aqq - app) / (2.0 * apq);
      const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
      c = 1.0 / sqrt(t * t + 1.0);
      s = t * c;
    }
  }
}

constexpr int JG_THREADS = 256;

// Barrier over all blocks of a cooperative launch: bar[0] arrivals, bar[1] generation,
// bar[2] error. A wait that exceeds ~2 s sets the error; every later barrier is then a
// no-op, so the kernel ends promptly and the host reports the failure.
__device__ __forceinline__ void grid_sync(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* verr = bar + 2;
    if (!*verr) {
      const unsigned g = *vgen;
      __threadfence();
      if (atomicAdd(bar, 1u) == gridDim.x - 1) {
        bar[0] = 0;
        __threadfence();
        atomicExch(bar + 1, g + 1);
      } else {
        unsigned long long t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        while (*vgen == g) {
          if (*verr) break;
          unsigned long long t1;
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
          if (t1 - t0 > 2000000000ull) { atomicExch(bar + 2, 1u); break; }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
}

// Block sum of v (fixed order) -> part[blockIdx.x]; after a grid barrier every block reads
// the total as the in-order sum of part[0..gridDim.x).
__device__ __forceinline__ void block_partial(double v, double* part, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < JG_THREADS / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}
__device__ __forceinline__ double grid_total(const double* part, double* red) {
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(part + b);
    red[0] = t;
  }
  __syncthreads();
  const double t = red[0];
  __syncthreads();
  return t;
}

// The same cyclic Jacobi as jacobi_kernel, spread over every SM (A, V and the partial sums
// are read from L2, as other SMs rewrite them between barriers): each round's rotations
// are computed by every block (into its shared memory, from the matrix as the previous
// round left it), the row updates and the column updates of the round are split over all
// threads, with a grid barrier after each.
__global__ void __launch_bounds__(JG_THREADS)
jacobi_grid_kernel(double* A, double* V, int k, int max_sweeps, double tol, unsigned* bar, double* part,
                   int* info) {
  __shared__ double cs[EIG_MAXK / 2], sn[EIG_MAXK / 2];
  __shared__ int pp[EIG_MAXK / 2], qq[EIG_MAXK / 2];
  __shared__ double red[JG_THREADS / 32];
  const int n = (k + 1) & ~1;
  const int npair = n / 2;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  double fr = 0.0;
  for (long long e = gt; e < (long long)k * k; e += nt) {
    V[e] = (e / k == e % k) ? 1.0 : 0.0;
    const double a0 = __ldcg(A + e);
    fr += a0 * a0;
  }
  block_partial(fr, part, red);
  grid_sync(bar);
  const double normA = sqrt(grid_total(part, red));
  double* offpart = part + gridDim.x;
  int sweep = 0;
  bool unconv = false;
  for (;; ++sweep) {
    double off = 0.0;
    for (long long e = gt; e < (long long)k * k; e += nt)
      if (e / k != e % k) {
        const double a0 = __ldcg(A + e);
        off += a0 * a0;
      }
    block_partial(off, offpart, red);
    grid_sync(bar);
    const double offn = sqrt(grid_total(offpart, red));
    if (offn <= tol * normA) break;
    if (sweep == max_sweeps) {
      unconv = offn > JACOBI_ACCEPT * normA;
      break;
    }
    for (int r = 0; r < n - 1; ++r) {
      for (int i = threadIdx.x; i < npair; i += blockDim.x) jacobi_pair(A, k, n, r, i, pp[i], qq[i], cs[i], sn[i]);
      __syncthreads();
      for (long long e = gt; e < (long long)npair * k; e += nt) {
        const int i = (int)(e / k), col = (int)(e % k);
        const int p = pp[i], q = qq[i];
        if (q >= k || sn[i] == 0.0) continue;
        const double c = cs[i], s = sn[i];
        const double ap = __ldcg(A + (long long)p * k + col), aq = __ldcg(A + (long long)q * k + col);
        A[(long long)p * k + col] = c * ap - s * aq;
        A[(long long)q * k + col] = s * ap + c * aq;
      }
      grid_sync(bar);
      for (long long e = gt; e < (long long)npair * k; e += nt) {
        const int i = (int)(e / k), row = (int)(e % k);
        const int p = pp[i], q = qq[i];
        if (q >= k || sn[i] == 0.0) continue;
        const double c = cs[i], s = sn[i];
        const double ap = __ldcg(A + (long long)row * k + p), aq = __ldcg(A + (long long)row * k + q);
        A[(long long)row * k + p] = c * ap - s * aq;
        A[(long long)row * k + q] = s * ap + c * aq;
        const double vp = __ldcg(V + (long long)row * k + p), vq = __ldcg(V + (long long)row * k + q);
        V[(long long)row * k + p] = c * vp - s * vq;
        V[(long long)row * k + q] = s * vp + c * vq;
      }
      grid_sync(bar);
    }
  }
  if (gt == 0) {
    info[0] = (unconv || info[0] == JACOBI_UNCONVERGED) ? JACOBI_UNCONVERGED : sweep;
    info[1] = (int)bar[2];
  }
}

__global__ void __launch_bounds__(EIG_THREADS)
eig_sort_kernel(const double* A, const double* V, int k, double* evals_out, double* Vout) {
  __shared__ int order[EIG_MAXK];
  __shared__ double ev[EIG_MAXK];
  eig_sort_sign(A, V, k, evals_out, Vout, ev, order);
}

// lagsum[l] += sum_blk part[blk][l] (blocks in order): the running sum over tensors of
// the autocorrelations, one tensor per call.
__global__ void lag_accumulate_kernel(const double* part, int nblk, int nlag, double* lagsum, int first) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlag) return;
  double g = first ? 0.0 : lagsum[l];
  for (int bb = 0; bb < nblk; ++bb) g += part[(long long)bb * nlag + l];
  lagsum[l] = g;
}

// Gram[u][s] = lagsum[lag(u - s)].
__global__ void gram_from_lags_kernel(const double* lagsum, int k1, int k2, int k3, double* gram) {
  const int k = k1 * k2 * k3;
  const int nl1 = 2 * k1 - 1, nl2 = 2 * k2 - 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)k * k) return;
  const int u = (int)(idx / k), s = (int)(idx % k);
  const int uw = u % k2, uh = (u / k2) % k1, ut = u / (k1 * k2);
  const int sw = s % k2, shh = (s / k2) % k1, st = s / (k1 * k2);
  const int l = ((ut - st + k3 - 1) * nl1 + (uh - shh + k1 - 1)) * nl2 + (uw - sw + k2 - 1);
  const int nlag = (2 * k3 - 1) * nl1 * nl2;
  gram[idx] = 0.5 * (lagsum[l] + lagsum[nlag - 1 - l]);    // exactly symmetric (see gram_kernel)
}

// Diagnostics (Sec. III-A, Definition 2). With G = A_k(L0)^T A_k(L0) and K = V:
// P = K^T G K, sigma_i^2 = P_ii, and (A_k(L0) K D)^T (A_k(L0) K D) = D P D.
// T[j][s] = sum_u G[s][u] V[j][u]   (V[j*k + u] = tap u of eigenvector j)
__global__ void gv_kernel(const double* G, const double* V, int k, double* T) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)k * k) return;
  const int j = (int)(idx / k), srow = (int)(idx % k);
  double t = 0.0;
  for (int u = 0; u < k; ++u) t = fma(G[(long long)srow * k + u], V[(long long)j * k + u], t);
  T[idx] = t;
}

// P[i][j] = sum_s V[i][s] T[j][s]
__global__ void vt_kernel(const double* V, const double* T, int k, double* P) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)k * k) return;
  const int i = (int)(idx / k), j = (int)(idx % k);
  double p = 0.0;
  for (int srow = 0; srow < k; ++srow) p = fma(V[(long long)i * k + srow], T[(long long)j * k + srow], p);
  P[idx] = p;
}

// One block: sigma_i = sqrt(max(P_ii, 0)); I = {i : sigma_i > tol * max(1, max sigma)};
// S = D P D (zero outside I) for the eigensolver; out[0] = r_K, out[1] = mu_1(V_I) =
// (k / r) max_s sum_{i in I} V[i][s]^2 (Eq. (coherence); V_I has orthonormal columns).
__global__ void __launch_bounds__(EIG_THREADS)
diag_support_kernel(const double* P, const double* V, int k, double tol, double* sigma, double* S, double* out) {
  __shared__ double red[EIG_THREADS];
  __shared__ double d[EIG_MAXK];
  double mx = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double sg = sqrt(fmax(P[(long long)i * k + i], 0.0));
    sigma[i] = sg;
    d[i] = sg;
    mx = fmax(mx, sg);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const double thr = tol * fmax(1.0, red[0]);
  __syncthreads();
  int cnt = 0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const bool on = d[i] > thr;
    d[i] = on ? 1.0 / d[i] : 0.0;
    cnt += on;
  }
  red[threadIdx.x] = (double)cnt;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  // S = D P D from the symmetric part of P: V^T (G V) is symmetric only to rounding, and
  // the scaling by 1/sigma lifts that asymmetry far above the eigensolver's tolerance
  for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) {
    const int i = (int)(e / k), j = (int)(e % k);
    const double pij = 0.5 * (P[e] + P[(long long)j * k + i]);
    S[e] = d[i] * pij * d[j];
  }
  double rowmax = 0.0;
  for (int srow = threadIdx.x; srow < k; srow += blockDim.x) {
    double q = 0.0;
    for (int i = 0; i < k; ++i)
      if (d[i] != 0.0) q = fma(V[(long long)i * k + srow], V[(long long)i * k + srow], q);
    rowmax = fmax(rowmax, q);
  }
  red[threadIdx.x] = rowmax;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = r;
    out[1] = r > 0 ? (double)k / r * red[0] : 0.0;
  }
}

// colsq[c] = v_c^T G v_c = ||A_k(L) v_c||^2 (G = A_k(L)^T A_k(L), V[c*k + s] = tap s of
// column c), written as the first of the NSEG column segments of a job (the others zero)
// so that the per-job reductions over segments read it like a forward pass's sums. One
// block per channel c < kc (zero past k); FP64, fixed order.
__global__ void gram_colsq_kernel(const double* G, const double* V, int k, int kc, double* colseg) {
  const int c = blockIdx.x;
  __shared__ double red[256];
  double q = 0.0;
  if (c < k)
    for (int srow = threadIdx.x; srow < k; srow += blockDim.x) {
      double y = 0.0;
      for (int u = 0; u < k; ++u) y = fma(G[(long long)srow * k + u], V[(long long)c * k + u], y);
      q = fma(V[(long long)c * k + srow], y, q);
    }
  red[threadIdx.x] = q;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  for (int sg = threadIdx.x; sg < NSEG; sg += blockDim.x) colseg[(long long)sg * kc + c] = (sg == 0) ? red[0] : 0.0;
}

__global__ void finite_check_kernel(const float* x, long long n, int* bad) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) { atomicExch(bad, 1); return; }
}

}  // namespace

// Host launchers -------------------------------------------------------------------
cudaError_t learn_gram(int b, const float* const* dL, const int* ddims, int k1, int k2, int k3,
                       double* dpart, int nblk, double* dgram, cudaStream_t st, bool exact) {
  LearnArgs a;
  a.b = b; a.L = dL; a.dims = ddims; a.k1 = k1; a.k2 = k2; a.k3 = k3;
  a.nl1 = 2 * k1 - 1; a.nl2 = 2 * k2 - 1; a.nl3 = 2 * k3 - 1;
  a.nlag = a.nl1 * a.nl2 * a.nl3;
  a.nblk = nblk; a.part = dpart;
  const int ew = BW + 2 * (k2 - 1), eh = BH + 2 * (k1 - 1), et = BT + 2 * (k3 - 1);
  const size_t smem = sizeof(float) * (size_t)ew * eh * et;
  if (exact) {
    cudaFuncSetAttribute(autocorr_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    autocorr_kernel<true><<<dim3(b, nblk), AC_THREADS, smem, st>>>(a);
  } else {
    cudaFuncSetAttribute(autocorr_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    autocorr_kernel<false><<<dim3(b, nblk), AC_THREADS, smem, st>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long kk = (long long)k1 * k2 * k3;
  gram_kernel<<<(unsigned)((kk * kk + 255) / 256), 256, 0, st>>>(a, dgram);
  return cudaGetLastError();
}

size_t learn_smem_bytes(int k1, int k2, int k3) {
  return sizeof(float) * (size_t)(BW + 2 * (k2 - 1)) * (BH + 2 * (k1 - 1)) * (BT + 2 * (k3 - 1));
}
int learn_max_lags() { return AC_THREADS * AC_MAXLAG_PER_THREAD; }

cudaError_t learn_eig(double* dA, double* dV, int k, double* devals, double* dVout, int* dinfo,
                      cudaStream_t st) {
  jacobi_kernel<<<1, EIG_THREADS, 0, st>>>(dA, dV, k, 30, 1e-15, devals, dVout, dinfo);
  return cudaGetLastError();
}

size_t learn_eig_grid_scratch(int dev) {
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 64 + 2 * (size_t)sms * sizeof(double);
}

cudaError_t learn_eig_grid(double* dA, double* dV, int k, double* devals, double* dVout, int* dinfo, void* scratch,
                           cudaStream_t st) {
  int dev = 0, sms = 1, per = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_grid_kernel, JG_THREADS, 0);
  if (e != cudaSuccess || !coop || per < 1) {
    cudaGetLastError();
    return learn_eig(dA, dV, k, devals, dVout, dinfo, st);       // one block
  }
  unsigned* bar = static_cast<unsigned*>(scratch);
  double* part = reinterpret_cast<double*>(static_cast<char*>(scratch) + 64);
  if ((e = cudaMemsetAsync(bar, 0, 64, st)) != cudaSuccess) return e;
  int maxs = 30;
  double tol = 1e-15;
  void* args[] = {&dA, &dV, &k, &maxs, &tol, &bar, &part, &dinfo};
  // one block per SM: every block is resident, as the grid barriers require
  if (cudaLaunchCooperativeKernel((const void*)jacobi_grid_kernel, dim3(sms), dim3(JG_THREADS), args, 0, st) !=
      cudaSuccess) {
    cudaGetLastError();
    return learn_eig(dA, dV, k, devals, dVout, dinfo, st);       // not co-resident here: one block
  }
  eig_sort_kernel<<<1, EIG_THREADS, 0, st>>>(dA, dV, k, devals, dVout);
  return cudaGetLastError();
}

// Gram accumulation one tensor at a time into caller-provided scratch (no allocation):
// dptrs/ddims are device arrays of b tensor pointers and b (H, W, T) triples.
cudaError_t learn_gram_streamed(int b, const float* const* dptrs, const int* ddims, int k1, int k2, int k3,
                                double* dpart, int nblk, double* dlagsum, double* dgram, cudaStream_t st) {
  LearnArgs a;
  a.b = 1; a.k1 = k1; a.k2 = k2; a.k3 = k3;
  a.nl1 = 2 * k1 - 1; a.nl2 = 2 * k2 - 1; a.nl3 = 2 * k3 - 1;
  a.nlag = a.nl1 * a.nl2 * a.nl3;
  a.nblk = nblk; a.part = dpart;
  const size_t smem = learn_smem_bytes(k1, k2, k3);
  cudaFuncSetAttribute(autocorr_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  for (int j = 0; j < b; ++j) {
    a.L = dptrs + j;
    a.dims = ddims + 3 * j;
    autocorr_kernel<false><<<dim3(1, nblk), AC_THREADS, smem, st>>>(a);
    lag_accumulate_kernel<<<(a.nlag + 255) / 256, 256, 0, st>>>(dpart, nblk, a.nlag, dlagsum, j == 0);
  }
  const long long kk = (long long)k1 * k2 * k3;
  gram_from_lags_kernel<<<(unsigned)((kk * kk + 255) / 256), 256, 0, st>>>(dlagsum, k1, k2, k3, dgram);
  return cudaGetLastError();
}

cudaError_t diag_spectral(const double* dG, const double* dV, int k, double tol, double* dT, double* dP,
                          double* dsigma, double* dS, double* dout, cudaStream_t st) {
  const unsigned nb = (unsigned)(((long long)k * k + 255) / 256);
  gv_kernel<<<nb, 256, 0, st>>>(dG, dV, k, dT);
  vt_kernel<<<nb, 256, 0, st>>>(dV, dT, k, dP);
  diag_support_kernel<<<1, EIG_THREADS, 0, st>>>(dP, dV, k, tol, dsigma, dS, dout);
  return cudaGetLastError();
}

cudaError_t gram_colsq(const float* dL, int H, int W, int T, int k1, int k2, int k3, const double* dV, int kc,
                       double* dpart, int nblk, double* dG, double* colseg, cudaStream_t st) {
  LearnArgs a{};
  a.b = 1; a.L = nullptr; a.dims = nullptr; a.L1 = dL; a.H1 = H; a.W1 = W; a.T1 = T;
  a.k1 = k1; a.k2 = k2; a.k3 = k3;
  a.nl1 = 2 * k1 - 1; a.nl2 = 2 * k2 - 1; a.nl3 = 2 * k3 - 1;
  a.nlag = a.nl1 * a.nl2 * a.nl3;
  a.nblk = nblk; a.part = dpart;
  const size_t smem = learn_smem_bytes(k1, k2, k3);
  cudaFuncSetAttribute(autocorr_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  autocorr_kernel<true><<<dim3(1, nblk), AC_THREADS, smem, st>>>(a);
  const long long kk = (long long)k1 * k2 * k3;
  gram_kernel<<<(unsigned)((kk * kk + 255) / 256), 256, 0, st>>>(a, dG);
  gram_colsq_kernel<<<kc, 256, 0, st>>>(dG, dV, (int)kk, kc, colseg);
  return cudaGetLastError();
}

cudaError_t diag_spectral_products(const double* dG, const double* dV, int k, double* dT, double* dP, cudaStream_t st) {
  const unsigned nb = (unsigned)(((long long)k * k + 255) / 256);
  gv_kernel<<<nb, 256, 0, st>>>(dG, dV, k, dT);
  vt_kernel<<<nb, 256, 0, st>>>(dV, dT, k, dP);
  return cudaGetLastError();
}

cudaError_t check_finite(const float* x, long long n, int* dbad, cudaStream_t st) {
  finite_check_kernel<<<256, 256, 0, st>>>(x, n, dbad);
  return cudaGetLastError();
}

}  // namespace icnnm
