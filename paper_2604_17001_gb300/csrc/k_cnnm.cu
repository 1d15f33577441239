// CNNM (Eq. cnnm): min ||A_k(L)||_* s.t. P_Omega(L) = P_Omega(M), by the same
// augmented-Lagrangian iteration as ICNNM with the Z-update replaced by singular-value
// thresholding (the method the paper compares ICNNM with, Sec. II-C, Tables II, IV):
//
//   Z = SVT_{1/theta}(A_k(L) - Y/theta)
//   L' = P_Omega^perp(A_k^*(Y + theta Z))/(k theta) + P_Omega(M)
//   Y' = Y + theta (Z - A_k(L')),  theta' = min(rho theta, theta_max).
//
// GPU form. The SVD of the m x k matrix B = A_k(L) - Y/theta goes through its k x k Gram
// C = B^T B = W Sigma^2 W^T (exact products of the FP32 entries of B, summed to about
// 2^-48 relative per tile and in FP64 across tiles, then the FP64 Jacobi eigensolver), so SVT(B) = B Phi with Phi = W diag(max(0, 1 -
// 1/(theta sigma_i))) W^T. The Jacobi method starts each iteration from the previous
// iteration's W (it diagonalises W_prev^T C W_prev, then rotates W_prev), which leaves
// few sweeps once the iteration settles.
//
// Y is never stored: the state is L and W = Y + theta Z of the previous iteration (k x m,
// tap-major), with Y = W - theta_prev A_k(L), so that
//   B = (1 + theta_prev/theta) A_k(L) - W/theta,   W' = W - theta_prev A_k(L) + theta B Phi.
// Per iteration: gram (B^T B partials), reduce, warm-start products, Jacobi, rotation,
// Phi, update (W'), gather (L' = the adjoint of W', projected).
//
// Plain FP32 arithmetic everywhere except the Gram, the eigensolver and Phi (FP64): this
// is the FP32 CNNM baseline, not a tuned path.
#include <math.h>

#include <algorithm>
#include <vector>

#include "icnnm_internal.h"

namespace icnnm {

namespace {

constexpr int CG = 64;            // taps per Gram block side
constexpr int CG_THREADS = 256;   // 16 x 16 threads, 4 x 4 outputs each
constexpr int CG_PITCH = CG + 4;  // voxel-major rows of B in shared memory
constexpr int CU_CT = 64;         // channels per update block
constexpr int CU_THREADS = 128;   // 8 channel groups x 16 voxel rows
constexpr int CU_KCH = 32;        // taps per staged chunk of Phi and W

struct CnnmDev {
  int H, W, T, k1, k2, k3, k, kp;   // kp = k rounded up to CG (row pitch of Phi)
  long long m;
  int ntw, nth, ntiles;
  const float* L;                    // current L (m)
  const float* WT;                   // current W (k x m, tap-major)
  float* WTn;                        // next W
  const float* Phi;                  // k x kp, Phi[s][c]
  const float* M;
  const uint8_t* mask;
  float* Lnew;
};

__device__ __forceinline__ void tile_coords(const CnnmDev& d, int tile, int& t, int& h0, int& w0) {
  const int tw = tile % d.ntw, th = (tile / d.ntw) % d.nth;
  t = tile / (d.ntw * d.nth);
  h0 = th * TH;
  w0 = tw * TW;
}

// Halo of L for one tile: element (bt, bh, bw) = L at (t - (k3-1) + bt, h0 - (k1-1) + bh,
// w0 - (k2-1) + bw), each coordinate wrapped; row v of A_k(L) holds L[v - s] (Sec. II-B).
__device__ __forceinline__ void stage_halo(const CnnmDev& d, float* sX, int t, int h0, int w0, int nthreads) {
  const int Wb = TW + d.k2 - 1, Hb = TH + d.k1 - 1;
  const int n = Wb * Hb * d.k3;
  for (int e = threadIdx.x; e < n; e += nthreads) {
    const int bw = e % Wb, bh = (e / Wb) % Hb, bt = e / (Wb * Hb);
    const int tt = wrapi(t - (d.k3 - 1) + bt, d.T), hh = wrapi(h0 - (d.k1 - 1) + bh, d.H),
              ww = wrapi(w0 - (d.k2 - 1) + bw, d.W);
    sX[e] = d.L[((long long)tt * d.H + hh) * d.W + ww];
  }
}

// A_k(L)[v][s] for tile voxel (vr, wc) from the halo.
__device__ __forceinline__ float halo_at(const CnnmDev& d, const float* sX, int vr, int wc, int s) {
  const int Wb = TW + d.k2 - 1, Hb = TH + d.k1 - 1;
  const int sw = s % d.k2, sh = (s / d.k2) % d.k1, st = s / (d.k1 * d.k2);
  return sX[((d.k3 - 1 - st) * Hb + (vr + d.k1 - 1 - sh)) * Wb + (wc + d.k2 - 1 - sw)];
}

// Partial Gram blocks: block pair (ib <= jb) of 64 taps, over the voxel tiles
// blockIdx.y, blockIdx.y + gridDim.y, ... part[(split * npair + pair) * 4096 + a * 64 + b]
// = sum_v B[v][ib*64 + a] B[v][jb*64 + b] (exact products, summed per tile as float pairs
// and across tiles in FP64).
__global__ void __launch_bounds__(CG_THREADS)
cnnm_gram_kernel(CnnmDev d, float acoef, float inv_th, int nb, double* part) {
  extern __shared__ float smem[];
  int p = blockIdx.x, ib = 0;
  while (p >= nb - ib) { p -= nb - ib; ++ib; }
  const int jb = ib + p;
  const int halo_n = (TW + d.k2 - 1) * (TH + d.k1 - 1) * d.k3;
  float* sX = smem;
  float* sBi = smem + ((halo_n + 3) & ~3);
  float* sBj = sBi + TILE_VOX * CG_PITCH;
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int tile = blockIdx.y; tile < d.ntiles; tile += gridDim.y) {
    int t, h0, w0;
    tile_coords(d, tile, t, h0, w0);
    __syncthreads();
    stage_halo(d, sX, t, h0, w0, CG_THREADS);
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * CG * TILE_VOX; e += CG_THREADS) {
      const int side = e / (CG * TILE_VOX);
      const int r = e % (CG * TILE_VOX);
      const int ss = r / TILE_VOX, vv = r % TILE_VOX;
      const int vr = vv / TW, wc = vv % TW;
      const int h = h0 + vr, w = w0 + wc;
      const int s = (side ? jb : ib) * CG + ss;
      float b = 0.f;
      if (h < d.H && w < d.W && s < d.k) {
        const long long v = ((long long)t * d.H + h) * d.W + w;
        b = fmaf(acoef, halo_at(d, sX, vr, wc, s), -(d.WT[(long long)s * d.m + v] * inv_th));
      }
      (side ? sBj : sBi)[vv * CG_PITCH + ss] = b;
    }
    __syncthreads();
    // the tile's 128 products per output, each split exactly into p + e (p = x*y rounded,
    // e = fma(x, y, -p)) and summed as a float pair hi + lo with Knuth's TwoSum (about
    // 2^-48 relative, on the FP32 pipe), then added into the FP64 sums once per tile
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.f;
    for (int vv = 0; vv < TILE_VOX; ++vv) {
      const float4 bi = *reinterpret_cast<const float4*>(sBi + vv * CG_PITCH + ti * 4);
      const float4 bj = *reinterpret_cast<const float4*>(sBj + vv * CG_PITCH + tj * 4);
      const float xi[4] = {bi.x, bi.y, bi.z, bi.w};
      const float xj[4] = {bj.x, bj.y, bj.z, bj.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float p = __fmul_rn(xi[a], xj[b]);
          const float e = __fmaf_rn(xi[a], xj[b], -p);
          const float sum = __fadd_rn(hi[a][b], p);
          const float bb = __fsub_rn(sum, hi[a][b]);
          const float err = __fadd_rn(__fsub_rn(hi[a][b], __fsub_rn(sum, bb)), __fsub_rn(p, bb));
          hi[a][b] = sum;
          lo[a][b] = __fadd_rn(lo[a][b], __fadd_rn(err, e));
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += (double)hi[a][b] + (double)lo[a][b];
  }
  const int npair = nb * (nb + 1) / 2;
  double* out = part + ((long long)blockIdx.y * npair + blockIdx.x) * (CG * CG);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) out[(ti * 4 + a) * CG + tj * 4 + b] = acc[a][b];
}

// C[i][j] = sum over splits (in order) of the partial block holding (i, j) or (j, i).
__global__ void cnnm_gram_reduce_kernel(const double* part, int k, int nb, int nsplit, double* C) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)k * k) return;
  int i = (int)(idx / k), j = (int)(idx % k);
  if (i / CG > j / CG) { const int x = i; i = j; j = x; }
  const int ib = i / CG, jb = j / CG;
  const int pair = ib * nb - ib * (ib - 1) / 2 + (jb - ib);
  const int npair = nb * (nb + 1) / 2;
  const int off = (i % CG) * CG + (j % CG);
  double c = 0.0;
  for (int sp = 0; sp < nsplit; ++sp) c += part[((long long)sp * npair + pair) * (CG * CG) + off];
  C[idx] = c;
}

// Wn[o][s] = sum_i R[o][i] W[i][s]: the eigenvectors of C from those of W^T C W.
// (Column o of a k x k matrix is stored contiguously: X[o * k + s].)
__global__ void cnnm_rotate_kernel(const double* R, const double* Wv, int k, double* Wn) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)k * k) return;
  const int o = (int)(idx / k), s = (int)(idx % k);
  double x = 0.0;
  for (int i = 0; i < k; ++i) x = fma(R[(long long)o * k + i], Wv[(long long)i * k + s], x);
  Wn[idx] = x;
}

// Phi[s][c] = sum_i W[i][s] f_i W[i][c], f_i = max(0, 1 - 1/(theta sigma_i)), sigma_i =
// sqrt(max(lambda_i, 0)): the singular-value thresholding operator at 1/theta in the
// right singular basis (FP64, stored FP32, zero padding for c >= k).
__global__ void cnnm_phi_kernel(const double* Wv, const double* evals, int k, int kp, double theta, float* Phi) {
  __shared__ double f[1024];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double sg = sqrt(fmax(evals[i], 0.0));
    f[i] = sg * theta > 1.0 ? 1.0 - 1.0 / (theta * sg) : 0.0;
  }
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)k * kp) return;
  const int s = (int)(idx / kp), c = (int)(idx % kp);
  double x = 0.0;
  if (c < k)
    for (int i = 0; i < k; ++i)
      if (f[i] != 0.0) x = fma(Wv[(long long)i * k + s] * f[i], Wv[(long long)i * k + c], x);
  Phi[idx] = (float)x;
}

// W' = W - theta_prev A_k(L) + theta B Phi, B = acoef A_k(L) - W/theta (FP32 FMA chains).
// Block = one voxel tile x 64 channels; thread (cg, vr): channels c0 + 8cg .. +8, voxels
// (h0 + vr, w0 .. w0 + 7).
__global__ void __launch_bounds__(CU_THREADS)
cnnm_update_kernel(CnnmDev d, float acoef, float inv_th, float th, float thp) {
  extern __shared__ float smem[];
  const int tile = blockIdx.x;
  int t, h0, w0;
  tile_coords(d, tile, t, h0, w0);
  const int halo_n = (TW + d.k2 - 1) * (TH + d.k1 - 1) * d.k3;
  float* sX = smem;
  float* sP = smem + ((halo_n + 3) & ~3);   // [CU_KCH][CU_CT]
  float* sW = sP + CU_KCH * CU_CT;          // [CU_KCH][TILE_VOX]
  const int c0 = blockIdx.y * CU_CT;
  stage_halo(d, sX, t, h0, w0, CU_THREADS);
  const int cg = threadIdx.x & 7, vr = threadIdx.x >> 3;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int w = 0; w < 8; ++w) acc[a][w] = 0.f;
  for (int s0 = 0; s0 < d.k; s0 += CU_KCH) {
    __syncthreads();
    for (int e = threadIdx.x; e < CU_KCH * CU_CT; e += CU_THREADS) {
      const int cc = e % CU_CT, ss = e / CU_CT;
      const int s = s0 + ss;
      sP[e] = s < d.k ? d.Phi[(long long)s * d.kp + c0 + cc] : 0.f;
    }
    for (int e = threadIdx.x; e < CU_KCH * TILE_VOX; e += CU_THREADS) {
      const int vv = e % TILE_VOX, ss = e / TILE_VOX;
      const int s = s0 + ss, h = h0 + vv / TW, w = w0 + vv % TW;
      sW[e] = (s < d.k && h < d.H && w < d.W) ? d.WT[(long long)s * d.m + ((long long)t * d.H + h) * d.W + w] : 0.f;
    }
    __syncthreads();
    const int ns = min(CU_KCH, d.k - s0);
    for (int ss = 0; ss < ns; ++ss) {
      float bv[8];
#pragma unroll
      for (int w = 0; w < 8; ++w)
        bv[w] = fmaf(acoef, halo_at(d, sX, vr, w, s0 + ss), -(sW[ss * TILE_VOX + vr * TW + w] * inv_th));
      const float4 pa = *reinterpret_cast<const float4*>(sP + ss * CU_CT + cg * 8);
      const float4 pb = *reinterpret_cast<const float4*>(sP + ss * CU_CT + cg * 8 + 4);
      const float pv[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int w = 0; w < 8; ++w) acc[a][w] = fmaf(bv[w], pv[a], acc[a][w]);
    }
  }
  const int h = h0 + vr;
  if (h >= d.H) return;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int c = c0 + cg * 8 + a;
    if (c >= d.k) continue;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      if (w0 + w >= d.W) continue;
      const long long v = ((long long)t * d.H + h) * d.W + w0 + w;
      const long long o = (long long)c * d.m + v;
      const float y = fmaf(-thp, halo_at(d, sX, vr, w, c), d.WT[o]);
      d.WTn[o] = fmaf(th, acc[a][w], y);
    }
  }
}

// L'[j] = M[j] on Omega, else (sum_s W'[s][j + s]) / (k theta) (the adjoint of Sec. II-B,
// taps summed in order).
__global__ void cnnm_gather_kernel(CnnmDev d, float inv_kth) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < d.m; j += (long long)gridDim.x * blockDim.x) {
    if (d.mask[j]) { d.Lnew[j] = d.M[j]; continue; }
    const int w = (int)(j % d.W), h = (int)((j / d.W) % d.H), t = (int)(j / ((long long)d.W * d.H));
    float acc = 0.f;
    for (int st = 0; st < d.k3; ++st) {
      const int tt = t + st >= d.T ? t + st - d.T : t + st;
      for (int sh = 0; sh < d.k1; ++sh) {
        const int hh = h + sh >= d.H ? h + sh - d.H : h + sh;
        const long long rb = ((long long)tt * d.H + hh) * d.W;
        const int s0 = (st * d.k1 + sh) * d.k2;
        for (int sw = 0; sw < d.k2; ++sw) {
          const int ww = w + sw >= d.W ? w + sw - d.W : w + sw;
          acc += d.WTn[(long long)(s0 + sw) * d.m + rb + ww];
        }
      }
    }
    d.Lnew[j] = acc * inv_kth;
  }
}

__global__ void cnnm_identity_kernel(double* X, int k) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (long long)k * k) X[idx] = (idx / k == idx % k) ? 1.0 : 0.0;
}

__global__ void cnnm_project_kernel(const float* M, const uint8_t* mask, long long m, float* L) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x)
    L[j] = mask[j] ? M[j] : 0.f;
}

// Hand-checked sizes of the launches below (k <= 1024, so k*k < 2^31).
unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t cnnm_state_bytes(int H, int W, int T, int k1, int k2, int k3) {
  const long long m = (long long)H * W * T;
  const int k = k1 * k2 * k3;
  return (size_t)m * (4 * 3 + 1) + (size_t)2 * k * m * 4 + (size_t)12 * k * k * 8;
}

// The whole CNNM solve on one stream. dM, dmask: device inputs; dL: device output (m).
// eig(C) uses the grid-wide Jacobi (measured several times faster than the one-block
// version per round, also at k = 75).
cudaError_t cnnm_run(const CnnmProblem& P, cudaStream_t st, CnnmResult* res) {
  const int k = P.k1 * P.k2 * P.k3;
  const long long m = (long long)P.H * P.W * P.T;
  const int nb = (k + CG - 1) / CG, kp = nb * CG, npair = nb * (nb + 1) / 2;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  CnnmDev d;
  d.H = P.H; d.W = P.W; d.T = P.T; d.k1 = P.k1; d.k2 = P.k2; d.k3 = P.k3; d.k = k; d.kp = kp; d.m = m;
  d.ntw = (P.W + TW - 1) / TW; d.nth = (P.H + TH - 1) / TH; d.ntiles = d.ntw * d.nth * P.T;
  d.M = P.dM; d.mask = P.dmask;
  const int nsplit = std::max(1, std::min(d.ntiles, 2 * sms / npair));
  const int nlag = (2 * P.k1 - 1) * (2 * P.k2 - 1) * (2 * P.k3 - 1);
  const int gblk = 2 * sms;

  std::vector<void*> mem;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, bytes);
    if (p) mem.push_back(p);
    return p;
  };
  float* L0 = (float*)alloc(m * 4);
  float* L1 = (float*)alloc(m * 4);
  float* W0 = (float*)alloc((size_t)k * m * 4);
  float* W1 = (float*)alloc((size_t)k * m * 4);
  double* part = (double*)alloc(sizeof(double) * (size_t)nsplit * npair * CG * CG);
  double* lagpart = (double*)alloc(sizeof(double) * (size_t)gblk * nlag);
  double* C = (double*)alloc(sizeof(double) * k * k);
  double* T = (double*)alloc(sizeof(double) * k * k);
  double* Pm = (double*)alloc(sizeof(double) * k * k);
  double* R = (double*)alloc(sizeof(double) * k * k);
  double* Rout = (double*)alloc(sizeof(double) * k * k);
  double* Wv = (double*)alloc(sizeof(double) * k * k);
  double* Wv2 = (double*)alloc(sizeof(double) * k * k);
  double* evals = (double*)alloc(sizeof(double) * k);
  float* Phi = (float*)alloc(sizeof(float) * (size_t)k * kp);
  int* info = (int*)alloc(2 * sizeof(int));
  void* scr = alloc(learn_eig_grid_scratch(dev));
  const float** dLp = (const float**)alloc(sizeof(float*));
  int* ddims = (int*)alloc(3 * sizeof(int));
  std::vector<double> hev(k);
  if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, 2 * sizeof(int), st);
  auto eig = [&](double* A, double* Vacc, double* Vout) {
    if (e != cudaSuccess) return;
    e = learn_eig_grid(A, Vacc, k, evals, Vout, info, scr, st);
  };
  // Nuclear norm / spectral norm of A_k(X) from the Gram of X (autocorrelations of exact products).
  auto gram_eigs = [&](const float* X) {
    if (e != cudaSuccess) return;
    const float* xp = X;
    const int dims[3] = {P.H, P.W, P.T};
    if ((e = cudaMemcpyAsync(dLp, &xp, sizeof(float*), cudaMemcpyHostToDevice, st)) != cudaSuccess) return;
    if ((e = cudaMemcpyAsync(ddims, dims, sizeof dims, cudaMemcpyHostToDevice, st)) != cudaSuccess) return;
    if ((e = learn_gram(1, dLp, ddims, P.k1, P.k2, P.k3, lagpart, gblk, C, st, true)) != cudaSuccess) return;
    eig(C, R, Rout);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hev.data(), evals, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  };

  const int halo_n = (TW + P.k2 - 1) * (TH + P.k1 - 1) * P.k3;
  const size_t gsm = sizeof(float) * (((halo_n + 3) & ~3) + 2 * TILE_VOX * CG_PITCH);
  const size_t usm = sizeof(float) * (((halo_n + 3) & ~3) + CU_KCH * CU_CT + CU_KCH * TILE_VOX);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(cnnm_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(cnnm_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess && (gsm > 200 * 1024 || usm > 200 * 1024)) e = cudaErrorInvalidValue;

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
  // L0 = P_Omega(M), W = 0 (Y0 = 0, theta_prev = 0), Wv = I
  if (e == cudaSuccess) {
    cnnm_project_kernel<<<gblk, 256, 0, st>>>(P.dM, P.dmask, m, L0);
    e = cudaMemsetAsync(W0, 0, (size_t)k * m * 4, st);
  }
  if (e == cudaSuccess) {
    cnnm_identity_kernel<<<nblocks((long long)k * k, 256), 256, 0, st>>>(Wv, k);
    e = cudaGetLastError();
  }
  double theta = P.theta0;
  if (!(theta > 0)) {
    gram_eigs(L0);                                      // theta0 = 1/||A_k(P_Omega M)||_2
    if (e == cudaSuccess) theta = hev[0] > 0 ? 1.0 / sqrt(hev[0]) : 1.0;
  }
  double thp = 0.0;
  float *Lc = L0, *Ln = L1, *Wc = W0, *Wn = W1;
  double *Wcur = Wv, *Wnext = Wv2;
  for (int it = 0; it < P.iters && e == cudaSuccess; ++it) {
    d.L = Lc; d.WT = Wc; d.WTn = Wn; d.Phi = Phi; d.Lnew = Ln;
    const float acoef = (float)(1.0 + thp / theta), inv_th = (float)(1.0 / theta);
    cnnm_gram_kernel<<<dim3(npair, nsplit), CG_THREADS, gsm, st>>>(d, acoef, inv_th, nb, part);
    cnnm_gram_reduce_kernel<<<nblocks((long long)k * k, 256), 256, 0, st>>>(part, k, nb, nsplit, C);
    // warm start: Pm = Wcur^T C Wcur (T = C Wcur scratch)
    diag_spectral_products(C, Wcur, k, T, Pm, st);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    eig(Pm, R, Rout);
    cnnm_rotate_kernel<<<nblocks((long long)k * k, 256), 256, 0, st>>>(Rout, Wcur, k, Wnext);
    cnnm_phi_kernel<<<nblocks((long long)k * kp, 256), 256, 0, st>>>(Wnext, evals, k, kp, theta, Phi);
    cnnm_update_kernel<<<dim3(d.ntiles, (k + CU_CT - 1) / CU_CT), CU_THREADS, usm, st>>>(d, acoef, inv_th,
                                                                                         (float)theta, (float)thp);
    cnnm_gather_kernel<<<gblk * 2, 256, 0, st>>>(d, (float)(1.0 / (k * theta)));
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    std::swap(Lc, Ln);
    std::swap(Wc, Wn);
    std::swap(Wcur, Wnext);
    thp = theta;
    theta = std::min(P.rho * theta, P.theta_max);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P.dL, Lc, m * 4, cudaMemcpyDeviceToDevice, st);
  int hinfo[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
  res->seconds = ms * 1e-3;
  res->theta = theta;
  res->timed_out = hinfo[1];
  res->unconverged = hinfo[0] < 0;
  // objective ||A_k(L)||_* = sum of the singular values of A_k(L)
  gram_eigs(Lc);
  if (e == cudaSuccess) {
    double nuc = 0.0;
    for (int i = k - 1; i >= 0; --i) nuc += sqrt(std::max(hev[i], 0.0));
    res->objective = nuc;
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  for (void* p : mem) cudaFree(p);
  return e;
}

}  // namespace icnnm
