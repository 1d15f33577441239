// FP32 SIMT kernels of the plain-FP32 ICNNM path (no tensor cores, no reduced
// precision): the forward pass E = A_k(X)V fused with the shifted-multiplier update,
// and the adjoint GEMM G^T = (V D) U^T, written so that each output element is a plain
// FP32 fused-multiply-add chain in a fixed order.
//
// A_k(X) is never materialised: row i of A_k(X) (Sec. II-B, Eq. ak) holds X[i - s]
// for every tap s, read from a circularly wrapped halo of X staged in shared memory.
#include "icnnm_internal.h"

namespace icnnm {

namespace {

constexpr int F_CT = 64;         // channels per block
constexpr int F_THREADS = 128;   // 8 channel groups x 16 voxel rows
constexpr int F_KCH = 32;        // taps per staged chunk of V

// Forward pass. Block = (voxel tile of 8w x 16h at one frame) x (64 channels).
// Thread (cg, vr): channels c0 + 8cg .. +8, voxels (h0 + vr, w0 .. w0+7).
__global__ void __launch_bounds__(F_THREADS)
fwd_fp32_kernel(Shared sh, int mode, const float* __restrict__ dummy) {
  extern __shared__ float smem[];
  const int tile_g = blockIdx.x;
  const int jb = job_of_tile(sh.job_tile0, sh.njobs, tile_g);
  const JobDev& J = sh.jobs[jb];
  const int tile = tile_g - sh.job_tile0[jb];
  const int H = J.H, W = J.W, T = J.T;
  const int tw = tile % J.ntw;
  const int th = (tile / J.ntw) % J.nth;
  const int t = tile / (J.ntw * J.nth);
  const int h0 = th * TH, w0 = tw * TW;
  const int k1 = sh.k1, k2 = sh.k2, k3 = sh.k3, k = sh.k, kc = sh.kc;
  const int c0 = blockIdx.y * F_CT;
  const int Wb = TW + k2 - 1, Hb = TH + k1 - 1;
  const int halo_n = Wb * Hb * k3;
  float* sX = smem;                       // [k3][Hb][Wb]
  float* sV = smem + ((halo_n + 3) & ~3); // [F_KCH][F_CT]
  float* sRed = sV + F_KCH * F_CT;        // [16][F_CT]
  const float* Xsrc = (mode == 3 || mode == 4) ? J.L : J.X;

  // Stage the halo: element (bt, bh, bw) is X at (t - (k3-1) + bt, h0 - (k1-1) + bh,
  // w0 - (k2-1) + bw), each coordinate wrapped (circular convolution, Sec. II-B).
  for (int e = threadIdx.x; e < halo_n; e += F_THREADS) {
    int bw = e % Wb, bh = (e / Wb) % Hb, bt = e / (Wb * Hb);
    int tt = wrapi(t - (k3 - 1) + bt, T), hh = wrapi(h0 - (k1 - 1) + bh, H), ww = wrapi(w0 - (k2 - 1) + bw, W);
    sX[e] = Xsrc[((long long)tt * H + hh) * W + ww];
  }

  const int cg = threadIdx.x & 7, vr = threadIdx.x >> 3;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

  for (int s0 = 0; s0 < k; s0 += F_KCH) {
    __syncthreads();
    for (int e = threadIdx.x; e < F_KCH * F_CT; e += F_THREADS) {
      int cc = e % F_CT, ss = e / F_CT;
      int s = s0 + ss, c = c0 + cc;
      sV[e] = (s < k && c < k) ? sh.Vf[(long long)s * kc + c] : 0.f;
    }
    __syncthreads();
    const int ns = min(F_KCH, k - s0);
    for (int ss = 0; ss < ns; ++ss) {
      const int s = s0 + ss;
      const int sw = s % k2, shh = (s / k2) % k1, st = s / (k1 * k2);
      // voxel (vr, w) reads halo (k3-1-st, vr + k1-1-sh, w + k2-1-sw)
      const float* xr = sX + ((k3 - 1 - st) * Hb + (vr + k1 - 1 - shh)) * Wb + (k2 - 1 - sw);
      float xv[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) xv[w] = xr[w];
      const float4 va = *reinterpret_cast<const float4*>(sV + ss * F_CT + cg * 8);
      const float4 vb = *reinterpret_cast<const float4*>(sV + ss * F_CT + cg * 8 + 4);
      const float vv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int w = 0; w < 8; ++w) acc[a][w] = fmaf(xv[w], vv[a], acc[a][w]);
    }
  }

  // Epilogue.
  const int h = h0 + vr;
  float csum[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) csum[a] = 0.f;
  float rsum = 0.f;
  float* U = reinterpret_cast<float*>(J.U);
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const int ww = w0 + w;
    if (h >= H || ww >= W) continue;
    const long long v = ((long long)t * H + h) * W + ww;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int c = c0 + cg * 8 + a;
      if (c >= k) continue;
      const float e = acc[a][w];
      if (mode == 0 || mode == 4) {
        csum[a] = fmaf(e, e, csum[a]);
      } else if (mode == 1) {
        const float u = U[v * kc + c];
        const float un = fmaf(u, J.D[c], -e);
        U[v * kc + c] = un;
        csum[a] = fmaf(un, un, csum[a]);
      } else if (mode == 2) {
        U[v * kc + c] = -e;
        csum[a] = fmaf(e, e, csum[a]);
      } else {
        const float r = fmaf(U[v * kc + c], (float)(J.s[c] / J.sc->theta), e);
        rsum = fmaf(r, r, rsum);
      }
    }
  }
  // Fixed-order reduction over the 16 voxel rows.
  __syncthreads();
  if (mode != 3) {
#pragma unroll
    for (int a = 0; a < 8; ++a) sRed[vr * F_CT + cg * 8 + a] = csum[a];
    __syncthreads();
    // partial row q covers voxel rows 4q..4q+3 (32 voxels), the same grouping as the
    // tensor-core path
    for (int i = threadIdx.x; i < PROW * F_CT; i += F_THREADS) {
      const int q = i / F_CT, cl = i % F_CT;
      float sum = 0.f;
      for (int r = 4 * q; r < 4 * q + 4; ++r) sum += sRed[r * F_CT + cl];
      const int c = c0 + cl;
      if (c < kc) J.part[((long long)tile * PROW + q) * kc + c] = sum;
    }
  } else {
    sRed[threadIdx.x] = rsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float sum = 0.f;
      for (int r = 0; r < F_THREADS; ++r) sum += sRed[r];
      J.rpart[(long long)tile * sh.nrp + blockIdx.y] = sum;
    }
  }
}

// Adjoint GEMM: G^T[s][v] = sum_c (V D)[s][c] U[v][c] over the voxels of one tile,
// 64 taps per block, K = channels in chunks of 16. Thread tile 4 taps x 8 voxels.
constexpr int A_TS = 64, A_KC = 16, A_THREADS = 256;

__global__ void __launch_bounds__(A_THREADS)
adj_gemm_fp32_kernel(Shared sh) {
  __shared__ float sA[A_KC][A_TS + 4];       // [c][s]
  __shared__ float sB[A_KC][TILE_VOX + 4];   // [c][v]
  const int tile_g = blockIdx.x;
  const int jb = job_of_tile(sh.job_tile0, sh.njobs, tile_g);
  const JobDev& J = sh.jobs[jb];
  const int tile = tile_g - sh.job_tile0[jb];
  const int H = J.H, W = J.W;
  const int tw = tile % J.ntw, th = (tile / J.ntw) % J.nth, t = tile / (J.ntw * J.nth);
  const int h0 = th * TH, w0 = tw * TW;
  const int k = sh.k, kc = sh.kc;
  const int s0 = blockIdx.y * A_TS;
  const float* U = reinterpret_cast<const float*>(J.U);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // voxels 8*tx.., taps 4*ty..
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

  for (int cb = 0; cb < kc; cb += A_KC) {
    __syncthreads();
    for (int e = threadIdx.x; e < A_KC * A_TS; e += A_THREADS) {
      int cc = e % A_KC, ss = e / A_KC;
      int s = s0 + ss, c = cb + cc;
      sA[cc][ss] = (s < k && c < k) ? sh.Vf[(long long)s * kc + c] * J.D[c] : 0.f;
    }
    for (int e = threadIdx.x; e < A_KC * TILE_VOX; e += A_THREADS) {
      int cc = e % A_KC, vv = e / A_KC;
      int h = h0 + vv / TW, w = w0 + vv % TW, c = cb + cc;
      float u = 0.f;
      if (h < H && w < W && c < k) u = U[(((long long)t * H + h) * W + w) * kc + c];
      sB[cc][vv] = u;
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < A_KC; ++cc) {
      float a[4], b[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[cc][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = sB[cc][tx * 8 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  // Store G^T[s][voxel]: the 8 voxels of a thread are one row segment (h fixed).
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int s = s0 + ty * 4 + i;
    if (s >= k) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int vv = tx * 8 + j;
      const int h = h0 + vv / TW, w = w0 + vv % TW;
      if (h < H && w < W) J.G[(long long)s * J.m + ((long long)t * H + h) * W + w] = acc[i][j];
    }
  }
}

}  // namespace

cudaError_t launch_fwd_fp32(const Shared& sh, int mode, cudaStream_t st) {
  const int halo_n = (TW + sh.k2 - 1) * (TH + sh.k1 - 1) * sh.k3;
  size_t smem = sizeof(float) * (((halo_n + 3) & ~3) + F_KCH * F_CT + 16 * F_CT + F_THREADS);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(fwd_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  dim3 grid(sh.total_tiles, (sh.k + F_CT - 1) / F_CT);
  fwd_fp32_kernel<<<grid, F_THREADS, smem, st>>>(sh, mode, nullptr);
  return cudaGetLastError();
}

int fwd_fp32_nrp(int k) { return (k + F_CT - 1) / F_CT; }

cudaError_t launch_adj_gemm_fp32(const Shared& sh, cudaStream_t st) {
  dim3 grid(sh.total_tiles, (sh.k + A_TS - 1) / A_TS);
  adj_gemm_fp32_kernel<<<grid, A_THREADS, 0, st>>>(sh);
  return cudaGetLastError();
}

}  // namespace icnnm
