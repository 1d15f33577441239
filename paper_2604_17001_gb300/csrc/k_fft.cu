// Frequency-domain ICNNM: the ADMM iteration of Sec. III-D (in the shifted-multiplier form
// of the implicit-GEMM path: U = Y - theta A_k(L)V, D = 1 - s) with every m x k quantity
// held as discrete Fourier transforms. The convolution of Sec. II-B is circular, so with
// kappa_c the kernel of eigenvector c (tap s = (st, sh, sw) at voxel (t, h, w) = (st, sh, sw)
// of an H x W x T array, zero elsewhere) and ^ the 3-D DFT:
//   (A_k(X) v_c)^         = X^ kappa_c^                       (convolution theorem)
//   (A_k^*(U D V^T))^     = sum_c D_c U_c^ conj(kappa_c^)     (correlation theorem)
//   ||U_c||^2             = (1/m) sum_omega |U_c^(omega)|^2   (Parseval)
// Every column of U stays a multiple of its kernel's spectrum: U_c^ = kappa_c^ w_c with
// w_c' = D_c w_c - X^ (and w_c = -X^ at the start). So the iteration needs only
// q_c = |kappa_c^|^2 and y_c = U_c^ conj(kappa_c^) = q_c w_c:
//   adjoint    Delta^ = sum_c D_c y_c
//   update     y_c'   = D_c y_c - q_c X^,   ||U_c'||^2 = (1/m) sum |y_c'|^2 / q_c
// An iteration streams y once (adjoint) and y and q once more (update: 28 bytes per
// frequency and channel in all) and transforms one tensor each way, in place of two
// m x k x k products.
//
// Every signal is real, so transforms along w keep the W/2 + 1 non-negative frequencies
// (the rest are complex conjugates); in Parseval the interior w-frequencies count twice.
// FFTs are radix-2 over power-of-two lengths, one kernel per axis, LB lines per block staged
// in shared memory, twiddles from FP64 values; in the iteration, the inverse transform along
// w, the L-update and the next operand's transform along w share one kernel and its lines.
// Arithmetic is FP32 complex; norms are summed per thread in FP32 and across threads and
// blocks in FP64, in a fixed order.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "icnnm_internal.h"

namespace icnnm {

namespace {

constexpr int LB = 16;               // lines per FFT block
constexpr int NB = 64;               // frequency blocks per channel in the spectral passes
constexpr int KAPPA_CHUNK = 16;      // eigenvector kernels transformed per batch
constexpr int CG = 4;                // channels per block of the spectral passes

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ int bitrev(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

// In-place radix-2 FFT (decimation in time) of LB lines of length n >= 2 held in shared
// memory in bit-reversed order, line l at s + l*n. tw[j] = exp(-2 pi i j / n), j < n/2;
// inv conjugates the twiddles (no 1/n).
__device__ void fft_smem(float2* s, int n, int logn, const float2* tw, bool inv) {
  const int hn = n >> 1;
  for (int lg = 1; lg <= logn; ++lg) {
    const int half = 1 << (lg - 1);
    const int step = n >> lg;
    __syncthreads();
    for (int b = threadIdx.x; b < LB * hn; b += blockDim.x) {
      const int l = b / hn, bi = b - l * hn;
      const int j = bi & (half - 1);
      const int i0 = ((bi - j) << 1) + j, i1 = i0 + half;
      float2 w = tw[j * step];
      if (inv) w.y = -w.y;
      float2* line = s + l * n;
      const float2 a = line[i0], t = cmul(w, line[i1]);
      line[i0] = make_float2(a.x + t.x, a.y + t.y);
      line[i1] = make_float2(a.x - t.x, a.y - t.y);
    }
  }
  __syncthreads();
}

// Complex FFT in place along a strided axis: line l (< nlines) has element e at
// base(l) + e * stride, base(l) = (l / inner) * outer + (l % inner). Consecutive threads
// take consecutive lines, which are adjacent in memory for the h and t axes.
__global__ void fft_axis_kernel(float2* data, int n, int logn, long long stride, long long inner, long long outer,
                                long long nlines, const float2* tw, int inv) {
  extern __shared__ float2 sm[];
  const long long l0 = (long long)blockIdx.x * LB;
  for (int i = threadIdx.x; i < LB * n; i += blockDim.x) {
    const int l = i % LB, e = i / LB;
    const long long line = l0 + l;
    if (line >= nlines) continue;
    const long long base = (line / inner) * outer + (line % inner);
    sm[l * n + bitrev(e, logn)] = data[base + e * stride];
  }
  fft_smem(sm, n, logn, tw, inv != 0);
  for (int i = threadIdx.x; i < LB * n; i += blockDim.x) {
    const int l = i % LB, e = i / LB;
    const long long line = l0 + l;
    if (line >= nlines) continue;
    const long long base = (line / inner) * outer + (line % inner);
    data[base + e * stride] = sm[l * n + e];
  }
}

// Real rows of length W (x[row * W + w]) -> the first W/2 + 1 DFT values of each row
// (out[row * Wh + omega]).
__global__ void rfft_rows_kernel(const float* x, float2* out, int W, int logw, long long nrows, const float2* tw) {
  extern __shared__ float2 sm[];
  const long long r0 = (long long)blockIdx.x * LB;
  const int Wh = W / 2 + 1;
  for (int i = threadIdx.x; i < LB * W; i += blockDim.x) {
    const int l = i / W, e = i - l * W;
    const long long row = r0 + l;
    sm[l * W + bitrev(e, logw)] = make_float2(row < nrows ? x[row * W + e] : 0.f, 0.f);
  }
  fft_smem(sm, W, logw, tw, false);
  for (int i = threadIdx.x; i < LB * Wh; i += blockDim.x) {
    const int l = i / Wh, e = i - l * Wh;
    const long long row = r0 + l;
    if (row < nrows) out[row * Wh + e] = sm[l * W + e];
  }
}

// Adjoint pass: Dh(omega) = sum_c D_c y_c(omega). A block takes ADJ_P frequency pairs; its
// ADJ_S thread slices each sum every ADJ_S-th channel for one pair, and the slices are added
// in slice order (a fixed order).
constexpr int ADJ_P = 64, ADJ_S = 4;
__global__ void __launch_bounds__(ADJ_P * ADJ_S) fft_adjoint_kernel(const float2* __restrict__ Yh,
                                                                    const float* __restrict__ D, int k, unsigned mh,
                                                                    float2* __restrict__ Dh) {
  extern __shared__ float sDv[];
  __shared__ float4 red[ADJ_S][ADJ_P];
  for (int c = threadIdx.x; c < k; c += blockDim.x) sDv[c] = D[c];
  __syncthreads();
  const unsigned np = mh / 2;
  const int pl = threadIdx.x % ADJ_P, sl = threadIdx.x / ADJ_P;
  for (unsigned p0 = blockIdx.x * ADJ_P; p0 < np; p0 += gridDim.x * ADJ_P) {
    const unsigned p = p0 + pl;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p < np) {
#pragma unroll 8
      for (int c = sl; c < k; c += ADJ_S) {
        const float4 y = __ldcs(reinterpret_cast<const float4*>(Yh + (size_t)c * mh) + p);
        const float d = sDv[c];
        acc.x = fmaf(d, y.x, acc.x);
        acc.y = fmaf(d, y.y, acc.y);
        acc.z = fmaf(d, y.z, acc.z);
        acc.w = fmaf(d, y.w, acc.w);
      }
    }
    red[sl][pl] = acc;
    __syncthreads();
    if (sl == 0 && p < np) {
      float4 t = red[0][pl];
#pragma unroll
      for (int q = 1; q < ADJ_S; ++q) {
        const float4 u = red[q][pl];
        t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
      }
      reinterpret_cast<float4*>(Dh)[p] = t;
    }
    __syncthreads();
  }
}

// Parseval weight of the w-frequency ow: 1 for 0 and W/2, else 2.
__device__ __forceinline__ float pw(unsigned ow, unsigned W) { return (ow == 0 || 2 * ow == W) ? 1.f : 2.f; }

// |r|^2 / q as q |r/q|^2 (r is a multiple of q, so r/q stays of order one where q is tiny); 0
// where q = 0 (there r = 0 too).
__device__ __forceinline__ float norm_over_q(float rx, float ry, float q) {
  if (!(q > 0.f)) return 0.f;
  const float iq = 1.f / q;
  const float wx = rx * iq, wy = ry * iq;
  return q * fmaf(wx, wx, wy * wy);
}

// Spectral pass with q_c = |kappa_c^|^2 and y_c = U_c^ conj(kappa_c^):
//   MODE 1: y_c <- D_c y_c - q_c X^ (stored); sums ||U_c'||^2 = (1/m) sum |y_c'|^2 / q_c
//   MODE 2: y_c <- -q_c X^ (stored); its ||U_c||^2 = (1/m) sum q_c |X^|^2
//   MODE 3: || (s_c / theta) U_c + A_k(X) v_c ||^2 from (s_c / theta) y_c + q_c X^ (the
//           primal residual column)
//   MODE 4: ||A_k(X) v_c||^2 = (1/m) sum q_c |X^|^2
// Work items are (group of CG channels, one of NB ranges of frequency pairs), taken by a
// persistent grid in item order; part[c * NB + range] = the item's Parseval-weighted sum
// for channel c (without the 1/m), each summed in a fixed order.
template <int MODE>
__global__ void __launch_bounds__(256) fft_spectral_kernel(float2* __restrict__ Yh, const float* __restrict__ Qk,
                                                           const float2* __restrict__ Xh, const float* __restrict__ D,
                                                           const float* __restrict__ sc, float inv_theta, int k,
                                                           unsigned mh, unsigned Wh, unsigned W,
                                                           double* __restrict__ part) {
  __shared__ double red[CG][8];
  const unsigned np = mh / 2;
  const unsigned per = (np + NB - 1) / NB;
  const int ngroups = (k + CG - 1) / CG;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int item = blockIdx.x; item < ngroups * NB; item += gridDim.x) {
    const int g = item / NB, rb = item % NB;
    const int c0 = g * CG, ncg = min(CG, k - c0);
    const unsigned lo = per * rb, hi = min(np, lo + per);
    float dc[CG], sct[CG], acc[CG];
    const float2* qp[CG];
    float4* yp[CG];
#pragma unroll
    for (int cc = 0; cc < CG; ++cc) {
      const int c = min(c0 + cc, k - 1);           // past k: re-read the last channel, store nothing
      dc[cc] = MODE == 1 ? D[c] : 0.f;
      sct[cc] = MODE == 3 ? sc[c] * inv_theta : 0.f;
      acc[cc] = 0.f;
      qp[cc] = reinterpret_cast<const float2*>(Qk + (size_t)c * mh);
      yp[cc] = reinterpret_cast<float4*>(Yh + (size_t)c * mh);
    }
    for (unsigned p = lo + threadIdx.x; p < hi; p += blockDim.x) {
      const float4 x = reinterpret_cast<const float4*>(Xh)[p];
      float2 q[CG];
      float4 y[CG];
#pragma unroll
      for (int cc = 0; cc < CG; ++cc) {
        q[cc] = __ldcs(qp[cc] + p);
        if (MODE == 1 || MODE == 3) y[cc] = __ldcs(yp[cc] + p);
      }
      const unsigned ow0 = (2 * p) % Wh, ow1 = ow0 + 1 == Wh ? 0 : ow0 + 1;
      const float w0 = pw(ow0, W), w1 = pw(ow1, W);
      const float x0 = fmaf(x.x, x.x, x.y * x.y), x1 = fmaf(x.z, x.z, x.w * x.w);
#pragma unroll
      for (int cc = 0; cc < CG; ++cc) {
        float n0, n1;
        if (MODE == 1) {
          const float4 r = make_float4(fmaf(dc[cc], y[cc].x, -q[cc].x * x.x), fmaf(dc[cc], y[cc].y, -q[cc].x * x.y),
                                       fmaf(dc[cc], y[cc].z, -q[cc].y * x.z), fmaf(dc[cc], y[cc].w, -q[cc].y * x.w));
          if (cc < ncg) __stcs(yp[cc] + p, r);
          n0 = norm_over_q(r.x, r.y, q[cc].x);
          n1 = norm_over_q(r.z, r.w, q[cc].y);
        } else if (MODE == 2) {
          if (cc < ncg)
            __stcs(yp[cc] + p, make_float4(-q[cc].x * x.x, -q[cc].x * x.y, -q[cc].y * x.z, -q[cc].y * x.w));
          n0 = q[cc].x * x0;
          n1 = q[cc].y * x1;
        } else if (MODE == 3) {
          n0 = norm_over_q(fmaf(sct[cc], y[cc].x, q[cc].x * x.x), fmaf(sct[cc], y[cc].y, q[cc].x * x.y), q[cc].x);
          n1 = norm_over_q(fmaf(sct[cc], y[cc].z, q[cc].y * x.z), fmaf(sct[cc], y[cc].w, q[cc].y * x.w), q[cc].y);
        } else {
          n0 = q[cc].x * x0;
          n1 = q[cc].y * x1;
        }
        acc[cc] = fmaf(w0, n0, fmaf(w1, n1, acc[cc]));
      }
    }
#pragma unroll
    for (int cc = 0; cc < CG; ++cc) {
      double a = acc[cc];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) red[cc][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < ncg) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
      part[(size_t)(c0 + threadIdx.x) * NB + rb] = t;
    }
    __syncthreads();
  }
}

// q_c = |kappa_c^|^2 for the cnt transformed kernels of a batch.
__global__ void kappa_q_kernel(const float2* Ks, float* Q, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = Ks[i];
    Q[i] = fmaf(v.x, v.x, v.y * v.y);
  }
}

// colsq_c = (1/m) sum_b part[c][b] (fixed order). With s, D: the shrink factors of the
// Z-update for the new U, s_c = max(0, 1 - 1/||U_c||), D_c = 1 - s_c.
__global__ void fft_colsq_kernel(const double* part, int k, double inv_m, double* colsq, float* s, float* D) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double t = 0.0;
  for (int b = 0; b < NB; ++b) t += part[(long long)c * NB + b];
  t *= inv_m;
  colsq[c] = t;
  if (s) {
    const double n = sqrt(t);
    const double sv = n > 1.0 ? 1.0 - 1.0 / n : 0.0;
    s[c] = (float)sv;
    D[c] = (float)(1.0 - sv);
  }
}

// One iteration's row stage, LB rows of W voxels per block: the rows of Delta^ (already
// inverse-transformed along t and h) are extended by conjugate symmetry and
// inverse-transformed along w (times 1/m), giving Delta = A_k^*(U D V^T); the L-update is
// applied per voxel (lambda = inf: P_Omega^perp(L + Delta/(k theta)) + P_Omega(M); finite
// lambda: the penalised form); the next forward operand X = (theta + theta') L' - theta L
// is transformed along w in the same shared-memory lines and its W/2 + 1 frequencies
// stored; lpart[block] = the block's ||L'||^2 (FP64, fixed order).
__global__ void fft_row_update_kernel(const float2* __restrict__ Dh, float* __restrict__ L,
                                      const float* __restrict__ M, const uint8_t* __restrict__ mask,
                                      float2* __restrict__ Xh, int W, int logw, long long nrows,
                                      const float2* __restrict__ tw, float scale, double th, double thn, double lam,
                                      int k, double* __restrict__ lpart) {
  extern __shared__ float2 sm[];
  __shared__ double red[32];
  const long long r0 = (long long)blockIdx.x * LB;
  const int Wh = W / 2 + 1;
  for (int i = threadIdx.x; i < LB * W; i += blockDim.x) {
    const int l = i / W, e = i - l * W;
    const long long row = r0 + l;
    float2 v = make_float2(0.f, 0.f);
    if (row < nrows) {
      if (e < Wh) {
        v = Dh[row * Wh + e];
      } else {
        const float2 c = Dh[row * Wh + (W - e)];
        v = make_float2(c.x, -c.y);
      }
    }
    sm[l * W + bitrev(e, logw)] = v;
  }
  fft_smem(sm, W, logw, tw, true);
  const float inv = (float)(1.0 / (k * th));
  const float xa = (float)(th + thn), xb = -(float)th;
  const bool exact = isinf(lam);
  double l2 = 0.0;
  for (int i = threadIdx.x; i < LB * W; i += blockDim.x) {
    const int l = i / W, e = i - l * W;
    const long long row = r0 + l;
    float x = 0.f;
    if (row < nrows) {
      const long long v = row * W + e;
      const float d = sm[i].x * scale;
      const float Lo = L[v];
      const bool obs = mask[v] != 0;
      float Ln;
      if (exact) {
        Ln = obs ? M[v] : fmaf(d, inv, Lo);
      } else {
        const double lt = obs ? lam : 0.0;
        Ln = (float)(((double)d / k + th * (double)Lo + lt * (obs ? (double)M[v] : 0.0)) / (lt + th));
      }
      x = fmaf(xa, Ln, xb * Lo);
      L[v] = Ln;
      l2 += (double)Ln * Ln;
    }
    sm[i] = make_float2(x, 0.f);
  }
  __syncthreads();
  // bit-reversed order for the forward transform (each pair swapped by one thread)
  for (int i = threadIdx.x; i < LB * W; i += blockDim.x) {
    const int l = i / W, e = i - l * W;
    const int r = bitrev(e, logw);
    if (e < r) {
      const float2 a = sm[l * W + e];
      sm[l * W + e] = sm[l * W + r];
      sm[l * W + r] = a;
    }
  }
  fft_smem(sm, W, logw, tw, false);
  for (int i = threadIdx.x; i < LB * Wh; i += blockDim.x) {
    const int l = i / Wh, e = i - l * Wh;
    const long long row = r0 + l;
    if (row < nrows) Xh[row * Wh + e] = sm[l * W + e];
  }
  for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    lpart[blockIdx.x] = t;
  }
}

// L = P_Omega(M), X = th * L.
__global__ void fft_init_kernel(const float* M, const uint8_t* mask, long long m, float* L, float* X, float th) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < m; v += (long long)gridDim.x * blockDim.x) {
    const float x = mask[v] ? M[v] : 0.f;
    L[v] = x;
    X[v] = th * x;
  }
}

// Writes the taps of eigenvectors c0 .. c0+cnt-1 into the zeroed slots x[j*m ...]: tap s of
// eigenvector c at voxel (st, sh, sw). Every slot has its nonzeros at the same k voxels,
// so reusing the slots for the next eigenvectors overwrites all of them.
__global__ void kappa_place_kernel(float* x, long long m, const double* V, int c0, int cnt, int k, int k1, int k2,
                                   int H, int W) {
  const int j = blockIdx.x;
  if (j >= cnt) return;
  for (int s = threadIdx.x; s < k; s += blockDim.x) {
    const int sw = s % k2, sh = (s / k2) % k1, st = s / (k1 * k2);
    x[(long long)j * m + ((long long)st * H + sh) * W + sw] = (float)V[(long long)(c0 + j) * k + s];
  }
}

int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

}  // namespace

bool fft_supported(int H, int W, int T, std::string* why) {
  auto p2 = [](int n) { return n >= 1 && (n & (n - 1)) == 0; };
  if (!p2(H) || !p2(W) || !p2(T)) {
    if (why) *why = "the frequency-domain path takes power-of-two dims only";
    return false;
  }
  if (W < 2 || H > 1024 || W > 1024 || T > 1024 || H * T < 2) {
    if (why) *why = "the frequency-domain path takes W in [2, 1024], H and T up to 1024, and H*T >= 2";
    return false;
  }
  return true;
}

size_t fft_state_bytes(int H, int W, int T, int k) {
  const size_t mh = (size_t)T * H * (W / 2 + 1), m = (size_t)T * H * W;
  const size_t chunk = (size_t)std::min(k, KAPPA_CHUNK);
  return (size_t)k * mh * 12 + chunk * mh * 8 + 2 * mh * 8 + 3 * m * 4 + chunk * m * 4 + (size_t)k * NB * 8 +
         (size_t)k * 24 + 2048 * 8 + 3 * 1024 * 8 + 4096;
}

cudaError_t fft_run(const FftProblem& P, cudaStream_t st, FftResult* res) {
  const int H = P.H, W = P.W, T = P.T, k1 = P.k1, k2 = P.k2, k3 = P.k3, k = k1 * k2 * k3;
  const long long m = (long long)H * W * T;
  const int Wh = W / 2 + 1;
  const long long mh = (long long)T * H * Wh;
  cudaError_t e = cudaSuccess;
  std::vector<void*> mem;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e == cudaSuccess) mem.push_back(p);
    return p;
  };
  const int chunk = std::min(k, KAPPA_CHUNK);
  float2* Yh = (float2*)alloc(sizeof(float2) * (size_t)k * mh);    // y_c = U_c^ conj(kappa_c^)
  float* Qk = (float*)alloc(sizeof(float) * (size_t)k * mh);        // q_c = |kappa_c^|^2
  float2* Ks = (float2*)alloc(sizeof(float2) * (size_t)chunk * mh); // kappa^ of one batch
  float2* Xh = (float2*)alloc(sizeof(float2) * mh);
  float2* Dh = (float2*)alloc(sizeof(float2) * mh);
  float* L = P.dL;
  float* X = (float*)alloc(4 * m);
  float* xs = (float*)alloc(4 * (size_t)chunk * m);
  double* part = (double*)alloc(8 * (size_t)k * NB);
  double* colsq = (double*)alloc(8 * (size_t)k);
  float* sv = (float*)alloc(4 * (size_t)k);
  float* Dv = (float*)alloc(4 * (size_t)k);
  int sms = 152;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P.device);
  const int gblocks = std::max(1, std::min(8 * sms, 2048));
  const int nrb = (int)(((long long)T * H + LB - 1) / LB);        // blocks of the row stage
  double* lpart = (double*)alloc(8 * (size_t)nrb);
  // twiddles exp(-2 pi i j / n) per axis length, from FP64 cos/sin
  const int lens[3] = {W, H, T};
  float2* tws[3] = {nullptr, nullptr, nullptr};
  std::vector<float2> htw[3];
  for (int a = 0; a < 3; ++a) {
    const int n = lens[a];
    htw[a].resize(std::max(1, n / 2));
    for (int j = 0; j < n / 2; ++j) {
      const double ang = -2.0 * M_PI * j / n;
      htw[a][j] = make_float2((float)cos(ang), (float)sin(ang));
    }
    tws[a] = (float2*)alloc(sizeof(float2) * htw[a].size());
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tws[a], htw[a].data(), sizeof(float2) * htw[a].size(), cudaMemcpyHostToDevice, st);
  }
  const int lw = log2i(W), lh = log2i(H), lt = log2i(T);
  const int adj_blocks = (int)std::max(1LL, std::min(16LL * sms, (mh / 2 + ADJ_P - 1) / ADJ_P));
  int spb = 1;                                    // resident blocks per SM of the update pass
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&spb, fft_spectral_kernel<1>, 256, 0);
  const int spec_blocks = std::max(1, spb) * sms;
  const int fthreads = 256;
  const size_t smax = (size_t)LB * std::max(W, std::max(H, T)) * sizeof(float2);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fft_axis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(rfft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_row_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
  // inverse transforms of a half spectrum along t and h (in place); the row stage does w
  auto inv_th = [&](float2* in) {
    if (e != cudaSuccess) return;
    if (T > 1)
      fft_axis_kernel<<<(unsigned)(((long long)H * Wh + LB - 1) / LB), fthreads, LB * T * sizeof(float2), st>>>(
          in, T, lt, (long long)H * Wh, (long long)H * Wh, mh, (long long)H * Wh, tws[2], 1);
    if (H > 1)
      fft_axis_kernel<<<(unsigned)(((long long)T * Wh + LB - 1) / LB), fthreads, LB * H * sizeof(float2), st>>>(
          in, H, lh, Wh, Wh, (long long)H * Wh, (long long)T * Wh, tws[1], 1);
    e = cudaGetLastError();
  };
  // forward transforms along h and t (in place), as in rfft3 after its row stage
  auto fwd_ht = [&](float2* out) {
    if (e != cudaSuccess) return;
    if (H > 1)
      fft_axis_kernel<<<(unsigned)(((long long)T * Wh + LB - 1) / LB), fthreads, LB * H * sizeof(float2), st>>>(
          out, H, lh, Wh, Wh, (long long)H * Wh, (long long)T * Wh, tws[1], 0);
    if (T > 1)
      fft_axis_kernel<<<(unsigned)(((long long)H * Wh + LB - 1) / LB), fthreads, LB * T * sizeof(float2), st>>>(
          out, T, lt, (long long)H * Wh, (long long)H * Wh, mh, (long long)H * Wh, tws[2], 0);
    e = cudaGetLastError();
  };
  // nb real tensors x[b*m ...] -> their half spectra out[b*mh ...]
  auto rfft3 = [&](const float* x, float2* out, int nb) {
    if (e != cudaSuccess) return;
    const long long rows = (long long)nb * T * H;
    rfft_rows_kernel<<<(unsigned)((rows + LB - 1) / LB), fthreads, LB * W * sizeof(float2), st>>>(x, out, W, lw, rows,
                                                                                                 tws[0]);
    if (H > 1) {
      const long long lines = (long long)nb * T * Wh;
      fft_axis_kernel<<<(unsigned)((lines + LB - 1) / LB), fthreads, LB * H * sizeof(float2), st>>>(
          out, H, lh, Wh, Wh, (long long)H * Wh, lines, tws[1], 0);
    }
    if (T > 1) {
      const long long lines = (long long)nb * H * Wh;
      fft_axis_kernel<<<(unsigned)((lines + LB - 1) / LB), fthreads, LB * T * sizeof(float2), st>>>(
          out, T, lt, (long long)H * Wh, (long long)H * Wh, mh, lines, tws[2], 0);
    }
    e = cudaGetLastError();
  };
  // a spectral pass, then the per-column squared norms (and, with shrink, s and D)
  auto spectral = [&](const float2* xh, int mode, double inv_theta, bool shrink) {
    if (e != cudaSuccess) return;
    const int items = ((k + CG - 1) / CG) * NB;
    const int gs = std::max(1, std::min(items, spec_blocks));
    const unsigned umh = (unsigned)mh, uwh = (unsigned)Wh, uw = (unsigned)W;
    const float it_ = (float)inv_theta;
    if (mode == 1)
      fft_spectral_kernel<1><<<gs, 256, 0, st>>>(Yh, Qk, xh, Dv, sv, it_, k, umh, uwh, uw, part);
    else if (mode == 2)
      fft_spectral_kernel<2><<<gs, 256, 0, st>>>(Yh, Qk, xh, Dv, sv, it_, k, umh, uwh, uw, part);
    else if (mode == 3)
      fft_spectral_kernel<3><<<gs, 256, 0, st>>>(Yh, Qk, xh, Dv, sv, it_, k, umh, uwh, uw, part);
    else
      fft_spectral_kernel<4><<<gs, 256, 0, st>>>(Yh, Qk, xh, Dv, sv, it_, k, umh, uwh, uw, part);
    fft_colsq_kernel<<<(k + 127) / 128, 128, 0, st>>>(part, k, 1.0 / (double)m, colsq, shrink ? sv : nullptr,
                                                      shrink ? Dv : nullptr);
    e = cudaGetLastError();
  };
  std::vector<double> hc(k), hl(nrb);
  auto read_back = [&](bool with_l) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), colsq, 8 * (size_t)k, cudaMemcpyDeviceToHost, st);
    if (with_l && e == cudaSuccess)
      e = cudaMemcpyAsync(hl.data(), lpart, 8 * (size_t)nrb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  };
  auto pass_begin = [&](int pass, int nk, long long nvox) {
    if (P.hook.begin) P.hook.begin(P.hook.user, pass, nk, nvox);
  };
  auto pass_end = [&](int pass) {
    if (P.hook.end) P.hook.end(P.hook.user, pass);
  };
  const int nk_fft = 1 + (H > 1) + (T > 1);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  // kappa_c^ of every eigenvector, KAPPA_CHUNK at a time
  if (e == cudaSuccess) e = cudaMemsetAsync(xs, 0, 4 * (size_t)chunk * m, st);
  for (int c0 = 0; c0 < k && e == cudaSuccess; c0 += chunk) {
    const int cnt = std::min(chunk, k - c0);
    kappa_place_kernel<<<cnt, 256, 0, st>>>(xs, m, P.dV, c0, cnt, k, k1, k2, H, W);
    rfft3(xs, Ks, cnt);
    if (e == cudaSuccess) {
      kappa_q_kernel<<<gblocks, 256, 0, st>>>(Ks, Qk + (size_t)c0 * mh, (long long)cnt * mh);
      e = cudaGetLastError();
    }
  }
  // theta0 = 1/max_c ||A_k(P_Omega M) v_c|| (Parseval), then U = -A_k(theta0 P_Omega M) V
  if (e == cudaSuccess) {
    fft_init_kernel<<<gblocks, 256, 0, st>>>(P.dM, P.dmask, m, L, X, 0.f);
    e = cudaGetLastError();
  }
  rfft3(L, Xh, 1);
  spectral(Xh, 4, 0.0, false);
  read_back(false);
  double theta = P.theta0;
  if (!(theta > 0)) {
    double mx = 0.0;
    for (double v : hc) mx = std::max(mx, v);
    theta = mx > 0 ? 1.0 / sqrt(mx) : 1.0;
  }
  if (e == cudaSuccess) {
    fft_init_kernel<<<gblocks, 256, 0, st>>>(P.dM, P.dmask, m, L, X, (float)theta);
    e = cudaGetLastError();
  }
  rfft3(X, Xh, 1);
  spectral(Xh, 2, 0.0, true);
  int it = 0;
  double resid = NAN;
  for (it = 1; it <= P.max_iters && e == cudaSuccess; ++it) {
    const double thn = std::min(P.rho * theta, P.theta_max);
    pass_begin(1, 1, m);
    fft_adjoint_kernel<<<adj_blocks, ADJ_P * ADJ_S, sizeof(float) * k, st>>>(Yh, Dv, k, (unsigned)mh, Dh);
    pass_end(1);
    e = cudaGetLastError();
    pass_begin(3, nk_fft - 1, 0);
    inv_th(Dh);
    pass_end(3);
    if (e == cudaSuccess) {
      // Delta along w, the L-update and the next operand's transform along w, fused
      pass_begin(2, 1, m);
      fft_row_update_kernel<<<nrb, fthreads, LB * W * sizeof(float2), st>>>(
          Dh, L, P.dM, P.dmask, Xh, W, lw, (long long)T * H, tws[0], (float)(1.0 / (double)m), theta, thn, P.lambda,
          k, lpart);
      pass_end(2);
      e = cudaGetLastError();
    }
    const bool periodic = P.tol > 0 && it % P.check_every == 0;
    bool stop = it >= P.max_iters;
    if (periodic || stop) {
      // ||Z - A_k(L')V|| with Z = -(s / theta) U of this iteration's U
      pass_begin(3, nk_fft + 2, 0);
      rfft3(L, Dh, 1);
      spectral(Dh, 3, 1.0 / theta, false);
      pass_end(3);
      read_back(true);
      double rsq = 0.0, lsq = 0.0;
      for (double v : hc) rsq += v;
      for (double v : hl) lsq += v;
      resid = sqrt(rsq) / (sqrt((double)k) * std::max(sqrt(lsq), 1e-300));
      if (periodic && resid <= P.tol) stop = true;
    }
    theta = thn;
    if (stop) break;
    // U' = U D - A_k(X)V and its column norms (X^ along w from the row stage)
    pass_begin(3, nk_fft - 1, 0);
    fwd_ht(Xh);
    pass_end(3);
    pass_begin(0, 2, m);
    spectral(Xh, 1, 0.0, true);
    pass_end(0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  // ||A_k(L)V||_{2,1} of the returned L
  rfft3(L, Xh, 1);
  spectral(Xh, 4, 0.0, false);
  read_back(false);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (res && e == cudaSuccess) {
    res->iters = std::min(it, P.max_iters);
    res->residual = resid;
    res->theta = theta;
    res->seconds = ms * 1e-3;
    double obj = 0.0;
    for (double v : hc) obj += sqrt(std::max(v, 0.0));
    res->objective = obj;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  for (void* p : mem) cudaFree(p);
  return e != cudaSuccess ? e : e2;
}

}  // namespace icnnm
