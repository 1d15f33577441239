// BF16 tensor-core path (sm_103a: tcgen05 MMA with TMEM accumulators, TMA loads and stores).
//
// Forward pass  E = A_k(X) V  (row i of A_k(X) holds X[i - s] for every tap s,
// Sec. II-B Eq. ak), fused with U' = U D - E and the column sums of U'^2.
//   M = 128 voxels (an 8w x 16h tile of one frame), N = the channel tile (128, or all of
//   kc <= 256 in one wide tile), K = taps. B = V^T (one channel tile per persistent CTA,
//   resident in shared memory, SW128 K-major). A = A_k(X) is never formed: the operand is
//   kept as ncopy = min(k2, 8) BF16 copies of X, copy c shifted by c along w and
//   wrap-padded, so that every 8-voxel row segment of every tap starts on a 16-byte
//   boundary. A TMA box of all copies (the tile's halo: Hh = TH + k1 - 1 rows x k3 frames x
//   8 w; the copies keep the k3 frames of a w-segment adjacent) lands in shared memory as
//   16-byte rows indexed rho = h*k3 + t. For a fixed w-tap sw the taps (sh, st) then sit at
//   rows rho = g*k3 + r with r = k1*k3 - 1 - (sh*k3 + st), so the A operand of each MMA is
//   an MN-major no-swizzle matrix whose core matrices overlap (M-groups k3 rows apart,
//   K-rows consecutive). Taps run in sw-runs padded to 16 (the padded taps have zero rows
//   in V^T), so every MMA stays inside one run.
//   BF16X3 (split): X and V as hi + lo BF16 pairs, three MMA chains into one accumulator,
//   U kept as a hi + lo pair.
//
// Adjoint pass  G = U (V D)^T, then col2im  Delta_j = sum_s G[j + s, s]  (the adjoint of
// Eq. ak): M = 128 voxels (the U tile by TMA), N = a tap tile of 128 or 256 columns (whole
// tap rows per 32-column group, spread evenly over the groups), K = channels. The epilogue
// warps pre-sum with shuffles the values of a tile row that land on the same halo column
// and add them into a double-buffered shared-memory halo; while tile i is added, tile i-1's
// halo is flushed into the job's Delta. With deterministic sums (the default) the halo and
// Delta hold 64-bit fixed point, so every sum is independent of the order of warps and
// CTAs; otherwise float atomics.
//
// Warp roles in both kernels: warp 0 issues the TMA loads (and, in the forward pass, the
// TMA stores of U'), warp 1 (one lane) issues tcgen05.mma, warps 2-17 run the epilogue from
// TMEM (warp w reads TMEM lanes 32*(w%4)..+31, i.e. 32 voxels of the tile). Two TMEM
// accumulators let the epilogue of a tile overlap the MMAs of the next. Every mbarrier
// wait is bounded (ptx::mbar_wait) and a timeout is reported through the job status
// instead of hanging.
#include <cuda.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <mutex>
#include <vector>

#include "ptx_sm100.cuh"
#include "tc_api.h"

namespace icnnm {

namespace {

constexpr int EPI_WARPS = 16;        // 4 per TMEM lane quarter, each owning 32 columns
constexpr int TC_THREADS = 64 + 32 * EPI_WARPS;
constexpr int ADJ_STAGES = 4;
constexpr int FWD_USTAGES = 2;      // U tile stages of the forward pass (fewer if short of space)
constexpr int USTAGE = 2 * 16384;    // one U tile: 128 voxels x 128 channels bf16 (two boxes)
constexpr int CHUNK = 16384;         // one SW128 K-chunk: 128 rows x 128 bytes
constexpr uint32_t TMEM_COLS = 256;
constexpr int SMEM_LIMIT = 227 * 1024;
// The col2im sums (the halo buffers and the per-job Delta) are 64-bit fixed point with 40
// fractional bits: integer additions are associative, so the sums do not depend on the
// order in which CTAs and warps add them (results are the same alone and in any batch).
// Range: every column of U D has norm <= 1 (D_c = 1/||U_c|| when ||U_c|| > 1), so each
// entry of G = U D V^T is at most sqrt(k) and |Delta| <= k sqrt(k) < 2^14 for k <= 512,
// well inside 2^63 / 2^40 = 2^23; resolution 2^-40.
constexpr float FX_ONE = 1099511627776.0f;          // 2^40
constexpr double FX_INV = 1.0 / 1099511627776.0;

__device__ __forceinline__ void fx_add(unsigned long long* p, float v) {
  atomicAdd(p, (unsigned long long)__float2ll_rn(v * FX_ONE));
}
// the col2im accumulation: fixed point (deterministic) or float
__device__ __forceinline__ void col_add(unsigned long long* p, float v) { fx_add(p, v); }
__device__ __forceinline__ void col_add(float* p, float v) { atomicAdd(p, v); }

int rup(int x, int a) { return (x + a - 1) / a * a; }
size_t fwd_smem_n(const TcGeom& g, int nus, bool split = false);

size_t adj_smem(const TcGeom& g);

TcGeom make_geom(int k1, int k2, int k3, int gpt_max, int ctw_max = 256, int nus_max = FWD_USTAGES, int det = 1) {
  TcGeom g{};
  g.det = det;
  g.k1 = k1; g.k2 = k2; g.k3 = k3; g.k = k1 * k2 * k3; g.kc = rup(g.k, 16);
  // each w-run of taps is padded to a multiple of 16 (two 8-row K-groups): every MMA then
  // stays inside one run, its K stride is one group and the issuer advances descriptors
  // by register adds
  g.R = k1 * k3; g.R8 = rup(g.R, 16);
  g.ngrp = k2 * (g.R8 / 8);
  g.nmma = (g.ngrp + 1) / 2;
  g.kpad = g.nmma * 16;
  g.nch_f = (g.kpad + 63) / 64;
  g.ncopy = std::min(k2, 8);
  g.nwc = (k2 + 7) / 8;
  g.Hh = TH + k1 - 1;
  g.region_bytes = g.Hh * k3 * 16;
  g.stage_bytes = rup(k2 * g.region_bytes + 16 * 16, 1024);  // k2 copies + 16 zero rows
  g.ctw = 128;
  g.nct = (g.k + 127) / 128;
  g.nct_s = g.nct;
  // adjoint tap columns: whole tap rows per 32-column group for the kernel widths with a
  // compile-time col2im (3, 5, 7, 9, 11, 13), taps in order otherwise
  g.rpg = (k2 == 3 || k2 == 5 || k2 == 7 || k2 == 9 || k2 == 11 || k2 == 13) ? 32 / k2 : 0;
  g.kcp = rup(g.kc, 64);
  g.nch_a = g.kcp / 64;
  g.Hb = TH + k1 - 1;
  g.Wb = TW + k2 - 1;
  g.pitch = rup(g.Wb, 8);
  if ((g.pitch / 8) % 2 == 0) g.pitch += 8;
  g.HBp = k3 * g.Hb * g.pitch;
  // tap tiles of 256 columns (8 groups) where the compile-time col2im applies, the
  // taps need more than one 128-column tile and the wider V D image fits beside the U
  // stages; 128 columns (4 groups) otherwise
  g.gpt = 4;
  if (gpt_max >= 8 && g.rpg && (k1 * k3 + g.rpg - 1) / g.rpg > 4) {
    g.gpt = 8;
    g.nta = 256;
    if (adj_smem(g) > SMEM_LIMIT) g.gpt = 4;
  }
  g.nta = 32 * g.gpt;
  g.ntt = g.rpg ? ((k1 * k3 + g.rpg - 1) / g.rpg + g.gpt - 1) / g.gpt : (g.k + 127) / 128;
  // spread the tap rows evenly over the ntt * gpt groups (fewer rows per group where they
  // do not fill them): every epilogue warp and every tap tile then adds about as many rows
  if (g.rpg) g.rpg = std::min(g.rpg, (k1 * k3 + g.ntt * g.gpt - 1) / (g.ntt * g.gpt));
  // frames (st) each tap tile's taps reach: its col2im partial keeps only those nsl
  // frames of the halo, starting at frame slo[tt]
  g.nsl = 1;
  for (int tt = 0; tt < g.ntt && tt < 16; ++tt) {
    int lo = 1 << 30, hi = -1;
    for (int j = 0; j < g.nta; ++j) {
      int sp = -1;
      if (g.rpg == 0) {
        sp = tt * 128 + j < g.k ? tt * 128 + j : -1;
      } else {
        const int G = tt * g.gpt + j / 32, r = (j % 32) / k2, sw = (j % 32) % k2, TR = G * g.rpg + r;
        sp = (r < g.rpg && TR < k1 * k3) ? TR * k2 + sw : -1;
      }
      if (sp < 0) continue;
      const int st = sp / (k1 * k2);
      lo = std::min(lo, st);
      hi = std::max(hi, st);
    }
    if (hi < 0) lo = hi = 0;
    g.slo[tt] = lo;
    g.nsl = std::max(g.nsl, hi - lo + 1);
  }
  g.HB = g.Hb * g.Wb * g.nsl;
  g.nus = std::max(1, std::min(FWD_USTAGES, nus_max));
  while (g.nus > 1 && fwd_smem_n(g, g.nus) > SMEM_LIMIT) --g.nus;
  // one channel tile of all channels (N = kc rounded up to 32) when 128 < that <= 256 and
  // it fits in shared memory with two U stages: one CTA per voxel tile, so the halo is
  // loaded and the MMAs issued once instead of twice
  {
    const int w = rup(g.kc, 32);
    if (ctw_max >= 256 && w > 128 && w <= 256) {
      TcGeom h = g;
      h.ctw = w;
      h.nct = 1;
      int nu = std::max(1, std::min(FWD_USTAGES, nus_max));
      while (nu > 1 && fwd_smem_n(h, nu) > SMEM_LIMIT) --nu;
      if (fwd_smem_n(h, nu) <= SMEM_LIMIT) {
        g.ctw = w;
        g.nct = 1;
        g.nus = nu;
      }
    }
  }
  // the lo copies start on a 128-byte boundary (tiled TMA destinations must)
  g.lo_off = rup(k2 * g.region_bytes + 16 * 16, 128);
  g.stage_bytes_s = rup(g.lo_off + k2 * g.region_bytes + 16 * 16, 1024);
  g.nus_s = FWD_USTAGES;
  while (g.nus_s > 1 && fwd_smem_n(g, g.nus_s, true) > SMEM_LIMIT) --g.nus_s;
  g.split_ok = fwd_smem_n(g, g.nus_s, true) <= SMEM_LIMIT;
  return g;
}

// Shared memory of the forward pass: B image(s), two halo stages, nus U stages (ubox boxes
// of 64 channels, twice for split), the per-warp scales (two tasks per warp) and the
// shared column-sum accumulators of second tasks (wide channel tiles), descriptors, barriers.
size_t fwd_smem_n(const TcGeom& g, int nus, bool split) {
  const int img = split ? 2 : 1;
  const int ctw = split ? 128 : g.ctw;
  const size_t stage = split ? (size_t)g.stage_bytes_s : (size_t)g.stage_bytes;
  const int ubox = (ctw + 63) / 64;
  const int ng2 = std::max(0, ctw / 32 - 4);          // column groups beyond the first four
  return 1024 + (size_t)img * g.nch_f * (ctw * 128) + 2 * stage + (size_t)nus * img * ubox * CHUNK +
         EPI_WARPS * (ng2 ? 64 : 32) * 4 + (size_t)ng2 * 4 * 32 * 32 * 4 + 64 * 16 + 256;
}
size_t fwd_smem(const TcGeom& g, bool split = false) {
  return split ? fwd_smem_n(g, g.nus_s, true) : fwd_smem_n(g, g.nus);
}
size_t adj_smem(const TcGeom& g) {
  return 1024 + (size_t)g.nch_a * (g.nta * 128) + ADJ_STAGES * (size_t)CHUNK + 2 * (size_t)g.HBp * (g.det ? 8 : 4) +
         128 * 4 + 256;
}

// Byte offset of forward K-group `grp` (8 taps) inside a halo stage.
uint32_t group_off(const TcGeom& g, int grp) {
  const int per = g.R8 / 8;
  const int sw = grp / per, j = grp % per;
  return (uint32_t)(((sw / 8) * g.ncopy + sw % 8) * g.region_bytes + j * 128);
}

struct FwdTab {
  uint32_t boff[64];
  uint32_t kstr[64];
  int reg;       // 1: boff[i] = (i / hp) * region_bytes + (i % hp) * 256 and kstr[i] = 128 for all i
  int hp;        // MMAs per w-run (half the 8-tap groups of a run)
};

struct FwdArgs {
  Shared sh;
  TcGeom g;
  FwdTab tab;
  int mode;
  int cta0[9];   // first CTA of each channel tile (cta0[nct] = grid size)
};

// Voxel-tile coordinates (tw, th, t) of the tiles a thread visits (the adjoint's contiguous
// tile ranges): the next tile of the same job advances them by one (w fastest, then h,
// then t); any other tile divides.
struct TileXY {
  int jb = -1, tile = -1, tw = 0, th = 0, t = 0;
  __device__ __forceinline__ void at(int jb_, int tile_, const JobDev& J) {
    if (jb_ == jb && tile_ == tile + 1) {
      if (++tw == J.ntw) {
        tw = 0;
        if (++th == J.nth) { th = 0; ++t; }
      }
    } else if (jb_ != jb || tile_ != tile) {
      tw = tile_ % J.ntw;
      th = (tile_ / J.ntw) % J.nth;
      t = tile_ / (J.ntw * J.nth);
    }
    jb = jb_;
    tile = tile_;
  }
};

// TMA store of one tile's U' (hi, and lo for the split form) from a U stage.
template <int NIMG>
__device__ __forceinline__ void fwd_store_u(const Shared& sh, uint8_t* stage, size_t uhalf, int jb, int tile, int c0,
                                            int nbox) {
  const JobDev& J = sh.jobs[jb];
  const int tw = tile % J.ntw, th = (tile / J.ntw) % J.nth, t = tile / (J.ntw * J.nth);
  for (int half = 0; half < NIMG; ++half)
    for (int bx = 0; bx < nbox; ++bx)
      ptx::tma_store_4d(half ? J.tmapUlo : J.tmapU, stage + (size_t)half * uhalf + (size_t)bx * CHUNK, c0 + bx * 64,
                        tw * TW, th * TH, t);
}

struct AdjArgs {
  Shared sh;
  TcGeom g;
};

__device__ __forceinline__ uint8_t* align1k(uint8_t* p) {
  return p + ((1024 - (ptx::smem_u32(p) & 1023)) & 1023);
}

__device__ __forceinline__ void set_fail(const Shared& sh) {
  if (sh.njobs > 0) atomicExch(&sh.jobs[0].sc->status, 1);
}

// Sum a[j] (j = 0..31) over the 32 lanes of the warp in a fixed order and store the sum
// for j = lane at dst[lane] (if `ok`): a transpose-reduce in five halving steps, after
// which lane l holds the total of value l.
// n (8, 16, 24 or 32; warp-uniform) consecutive accumulator columns from TMEM into e[0..n).
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&e)[32], int n) {
  if (n == 32) {
    ptx::tmem_ld32(taddr, e);
  } else if (n == 8) {
    ptx::tmem_ld8(taddr, *reinterpret_cast<float(*)[8]>(&e[0]));
  } else {
    ptx::tmem_ld16(taddr, *reinterpret_cast<float(*)[16]>(&e[0]));
    if (n == 24) ptx::tmem_ld8(taddr + 16, *reinterpret_cast<float(*)[8]>(&e[16]));
  }
}

// Address of 8-channel unit cu (channel 8 cu of the tile) in a voxel's row of a U stage:
// 64-channel SW128 boxes of CHUNK bytes, the unit's 16 bytes XOR-swizzled by the row phase.
__device__ __forceinline__ uint8_t* uunit(uint8_t* rowb, int cu, uint32_t usw) {
  return rowb + (size_t)(cu >> 3) * CHUNK + ((((uint32_t)cu & 7u) ^ usw) << 4);
}

__device__ __forceinline__ void warp_colsum_store(float (&a)[32], int lane, float* dst, bool ok) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float snd = (lane & 16) ? a[k] : a[k + 16];
    const float kp = (lane & 16) ? a[k + 16] : a[k];
    a[k] = kp + __shfl_xor_sync(0xffffffffu, snd, 16);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float snd = (lane & 8) ? a[k] : a[k + 8];
    const float kp = (lane & 8) ? a[k + 8] : a[k];
    a[k] = kp + __shfl_xor_sync(0xffffffffu, snd, 8);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float snd = (lane & 4) ? a[k] : a[k + 4];
    const float kp = (lane & 4) ? a[k + 4] : a[k];
    a[k] = kp + __shfl_xor_sync(0xffffffffu, snd, 4);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float snd = (lane & 2) ? a[k] : a[k + 2];
    const float kp = (lane & 2) ? a[k + 2] : a[k];
    a[k] = kp + __shfl_xor_sync(0xffffffffu, snd, 2);
  }
  {
    const float snd = (lane & 1) ? a[0] : a[1];
    const float kp = (lane & 1) ? a[1] : a[0];
    a[0] = kp + __shfl_xor_sync(0xffffffffu, snd, 1);
  }
  if (ok) dst[lane] = a[0];
}

// ---------------------------------------------------------------------------------
// Forward pass
// ---------------------------------------------------------------------------------
// Tile order of a forward CTA: the chunks (fchunk consecutive tiles of one job) of the
// launch list, every nslot-th from `slot`, each chunk's tiles in order. Column partials
// are kept per chunk (row group = chunk index within its job), so the sums are grouped the
// same way whatever other jobs share the launch.
// Without deterministic reductions the CTA takes every nslot-th tile of the list instead,
// with one partial row group per (job, CTA): the round-robin order spreads neighbouring
// tiles over the CTAs, but a job's sums are then grouped by its position in the list.
struct TileSeq {
  const Shared& sh;
  int nslot, det, chg, jb = 0, tile = 0, thi = 0;
  __device__ TileSeq(const Shared& s, int slot, int ns, int d) : sh(s), nslot(ns), det(d), chg(slot - ns) {}
  // key of the column-partial group of the current tile
  __device__ int group() const { return det ? chg : jb; }
  __device__ bool next() {
    if (!det) {
      chg += nslot;                                   // chg is the global tile index here
      if (chg >= sh.total_tiles) return false;
      jb = job_of_tile(sh.job_tile0, sh.njobs, chg);
      tile = chg - sh.job_tile0[jb];
      return true;
    }
    if (++tile < thi) return true;
    chg += nslot;
    if (chg >= sh.total_chunks) return false;
    jb = job_of_tile(sh.job_chunk0, sh.njobs, chg);
    const int fc = sh.jobs[jb].fchunk;
    tile = (chg - sh.job_chunk0[jb]) * fc;
    thi = min(sh.jobs[jb].ntiles, tile + fc);
    return true;
  }
};
// SPLIT: the operand copies, V^T and U come as hi + lo BF16 pairs (lo = bf16(x - hi)),
// and each tile takes three products into one accumulator, A_k(X_hi)V_hi + A_k(X_lo)V_hi
// + A_k(X_hi)V_lo, i.e. A_k(X)V to about 2^-16 relative instead of 2^-8; U' is stored as
// hi = bf16(U'), lo = bf16(U' - hi). The halo stage holds the hi copies (and 16 zero
// rows) and then the lo copies (and 16 zero rows); a U stage holds the hi tile and then
// the lo tile; shared memory holds both V^T images.
// WIDE: channel tiles of g.ctw > 128 channels (some epilogue warps take two 32-channel
// groups); otherwise the tile width is the compile-time 128 and each warp one group.
template <bool SPLIT, bool WIDE>
__global__ void __launch_bounds__(TC_THREADS, 1) fwd_tc_kernel(const __grid_constant__ FwdArgs a) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1k(smraw);
  const TcGeom& g = a.g;
  const Shared& sh = a.sh;
  constexpr int NIMG = SPLIT ? 2 : 1;
  const int ctw = (SPLIT || !WIDE) ? 128 : g.ctw;               // channels per tile (the MMA's N)
  const int nct = SPLIT ? g.nct_s : g.nct;
  const int chunkF = ctw * 128;                                  // one K chunk (64 taps) of the B image
  const int ubox = (ctw + 63) / 64;                              // 64-channel U boxes per tile
  const int ng = ctw / 32;                                       // 32-channel epilogue groups
  const uint32_t tcols = 2 * ctw > 256 ? 512u : TMEM_COLS;
  const int stage_bytes = SPLIT ? g.stage_bytes_s : g.stage_bytes;
  const int nus = SPLIT ? g.nus_s : g.nus;
  const int uhalf = ubox * CHUNK;                                // one U tile (hi or lo) in a stage
  const int ustage = NIMG * uhalf;
  uint8_t* sA = sm;                                              // V^T image(s) of this channel tile
  uint8_t* sH = sA + (size_t)NIMG * g.nch_f * chunkF;            // [2] halo stages
  uint8_t* sU = sH + 2 * (size_t)stage_bytes;                    // [nus] U tiles
  const int sdw = ng > 4 ? 64 : 32;                              // scale slots per warp (one per group)
  float* sD = reinterpret_cast<float*>(sU + (size_t)nus * ustage);   // [EPI_WARPS][sdw] channel scales
  float* sAcc2 = sD + EPI_WARPS * sdw;                           // [ng - 4 groups][4][32][32] second-group sums
  ulonglong2* sDesc = reinterpret_cast<ulonglong2*>(sAcc2 + (size_t)max(0, ng - 4) * 4 * 32 * 32);  // [64]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sDesc + 64);
  uint64_t* full = bars;                   // [2] halo landed
  uint64_t* empty = bars + 2;              // [2] halo consumed by the MMAs
  uint64_t* tfull = bars + 4;              // [2] accumulator ready
  uint64_t* tempty = bars + 6;             // [2] accumulator read out
  uint64_t* ufull = bars + 8;              // [nus] U tile landed
  uint64_t* uempty = bars + 8 + nus;       // [nus] U stage free again (mode 2: the epilogue may write it)
  uint64_t* sready = bars + 8 + 2 * nus;   // [nus] the epilogue is done with the stage (U' written)
  uint64_t* abar = bars + 8 + 3 * nus;
  uint64_t* dbar = abar + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(dbar + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ct = 0;
  while (ct + 1 < nct && (int)blockIdx.x >= a.cta0[ct + 1]) ++ct;
  const int slot = (int)blockIdx.x - a.cta0[ct], nslot = a.cta0[ct + 1] - a.cta0[ct];
  const int mode = a.mode;
  const bool rdU = (mode == 1 || mode == 3);   // U is read (TMA) in these modes
  const bool wrU = (mode == 1 || mode == 2);   // U' is written (TMA store) in these modes
  const int nbox = min(ubox, (sh.kc - ct * ctw + 63) / 64);     // 64-channel boxes of U inside kc

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&full[i], 1);
      ptx::mbar_init(&empty[i], 1);
      ptx::mbar_init(&tfull[i], 1);
      ptx::mbar_init(&tempty[i], EPI_WARPS);
    }
    for (int i = 0; i < nus; ++i) {
      ptx::mbar_init(&ufull[i], 1);
      ptx::mbar_init(&uempty[i], 1);
      ptx::mbar_init(&sready[i], EPI_WARPS);
    }
    ptx::mbar_init(abar, 1);
    ptx::mbar_init(dbar, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tslot, tcols);
    ptx::tmem_relinquish();
  }
  for (int i = threadIdx.x; i < max(0, ng - 4) * 4 * 32 * 32; i += blockDim.x) sAcc2[i] = 0.f;
  // zero rows after the copies of each stage (read by the padded taps, times zero)
  for (int i = threadIdx.x; i < 2 * NIMG * 64; i += blockDim.x) {
    const int st = i / (NIMG * 64), half = (i / 64) % NIMG;
    reinterpret_cast<uint32_t*>(sH + (size_t)st * stage_bytes + (size_t)half * g.lo_off +
                                g.k2 * g.region_bytes)[i % 64] = 0u;
  }
  ptx::fence_proxy_async_smem();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tbase = *tslot;
  bool failed = false;

  if (warp == 0) {
    if (lane == 0) {
      ptx::mbar_arrive_expect_tx(abar, (uint32_t)(NIMG * g.nch_f * chunkF));
      for (int im = 0; im < NIMG; ++im) {
        // image im of channel tile ct (split: the lo images follow the nct hi images)
        const uint8_t* src = reinterpret_cast<const uint8_t*>(SPLIT ? sh.VtImgS : sh.VtImg) +
                             ((size_t)im * nct + ct) * g.nch_f * chunkF;
        for (int c = 0; c < g.nch_f; ++c)
          ptx::bulk_g2s(sA + ((size_t)im * g.nch_f + c) * chunkF, src + (size_t)c * chunkF, (uint32_t)chunkF, abar);
      }
      const uint32_t hbytes = (uint32_t)(NIMG * g.k2 * g.region_bytes);
      int rjb[FWD_USTAGES] = {0}, rtile[FWD_USTAGES] = {0};   // job and tile held by each U stage
      int it = 0;
      TileSeq sq(sh, slot, nslot, g.det);
      for (; sq.next(); ++it) {
        const int s = it & 1;
        const uint32_t ph = (it >> 1) & 1;
        if (!ptx::mbar_wait_abortable(&empty[s], ph ^ 1, abort)) { failed = true; break; }
        const JobDev& J = sh.jobs[sq.jb];
        const int tile = sq.tile;
        const int tw = tile % J.ntw, th = (tile / J.ntw) % J.nth, t = tile / (J.ntw * J.nth);
        ptx::mbar_arrive_expect_tx(&full[s], hbytes);
        // w-chunk q holds the copies of taps sw = 8q .. min(8q + 7, k2 - 1); the last
        // chunk of a kernel wider than 8 uses the map whose box has only k2 - 8 copies
        // (SPLIT: the lo copies are copies ncopy..2 ncopy-1 of the same maps)
        for (int half = 0; half < NIMG; ++half)
          for (int q = 0; q < g.nwc; ++q)
            ptx::tma_load_4d(sH + (size_t)s * stage_bytes + (size_t)half * g.lo_off + (size_t)q * g.ncopy * g.region_bytes,
                             (q > 0) ? J.tmapX2 : J.tmapX, t * 8, th * TH, tw + (g.nwc - 1) - q, half * g.ncopy,
                             &full[s]);
        {
          // U stage us: once the epilogue is done with tile it - nus there, store that tile's
          // U' (this thread issues every store, so that no epilogue warp waits for one) and
          // wait until the store has read the stage; then load tile it's U into it (modes 1
          // and 3) or hand it to the epilogue (mode 2)
          const int us = it % nus;
          if (it >= nus) {
            if (!ptx::mbar_wait_abortable(&sready[us], ((it - nus) / nus) & 1, abort)) { failed = true; ++it; break; }
            if (wrU) {
              fwd_store_u<NIMG>(sh, sU + (size_t)us * ustage, uhalf, rjb[us], rtile[us], ct * ctw, nbox);
              ptx::bulk_commit_group();
              ptx::bulk_wait_group_read0();
            }
          }
          rjb[us] = sq.jb;
          rtile[us] = tile;
          if (rdU) {
            ptx::mbar_arrive_expect_tx(&ufull[us], (uint32_t)(NIMG * nbox * CHUNK));
            for (int half = 0; half < NIMG; ++half)
              for (int bx = 0; bx < nbox; ++bx)
                ptx::tma_load_4d(sU + (size_t)us * ustage + (size_t)half * uhalf + (size_t)bx * CHUNK,
                                 half ? J.tmapUlo : J.tmapU, ct * ctw + bx * 64, tw * TW, th * TH, t, &ufull[us]);
          } else if (it >= nus) {
            ptx::mbar_arrive(&uempty[us]);
          }
        }
      }
      // the U' of the last tiles, once the epilogue is done with them
      if (!failed)
        for (int i = (it > nus ? it - nus : 0); i < it; ++i) {
          const int us = i % nus;
          if (!ptx::mbar_wait_abortable(&sready[us], (i / nus) & 1, abort)) { failed = true; break; }
          if (wrU) {
            fwd_store_u<NIMG>(sh, sU + (size_t)us * ustage, uhalf, rjb[us], rtile[us], ct * ctw, nbox);
            ptx::bulk_commit_group();
          }
        }
      if (wrU) ptx::bulk_wait_group0();   // every U' store is complete before the CTA exits
      // every issued load has landed before the CTA can exit
      for (int i = (it > 2 ? it - 2 : 0); i < it; ++i)
        if (!ptx::mbar_wait(&full[i & 1], (i >> 1) & 1)) failed = true;
      if (rdU)
        for (int i = (it > nus ? it - nus : 0); i < it; ++i)
          if (!ptx::mbar_wait(&ufull[i % nus], (i / nus) & 1)) failed = true;
      if (failed) *abort = 1;
    }
  } else if (warp == 1) {
    // A = halo (voxels x taps, MN-major, overlapping core matrices), B = V^T image
    // (channels x taps, K-major SW128): D[voxel][channel] in TMEM. The descriptors of the
    // nmma MMAs of a tile (halo stage 0) are built once here, so that the issuing thread
    // only loads, offsets and issues: its dependent scalar chain sets the MMA rate.
    {
      const uint32_t aB = ptx::smem_u32(sA), hB = ptx::smem_u32(sH);
      const uint32_t nstride = (uint32_t)g.k3 * 16;
      for (int i = lane; i < g.nmma; i += 32) {
        ulonglong2 dd;
        dd.x = ptx::sdesc(hB + a.tab.boff[i], a.tab.kstr[i], nstride, 0);
        dd.y = ptx::sdesc(aB + (uint32_t)(i >> 2) * (uint32_t)chunkF + (uint32_t)(i & 3) * 32, 16, 1024, 2);
        sDesc[i] = dd;
      }
      __syncwarp();
    }
    if (lane == 0) {
      if (!ptx::mbar_wait_abortable(abar, 0, abort)) failed = true;
      const uint32_t idesc = ptx::idesc_bf16(128, (uint32_t)ctw, 1, 0);
      int it = 0;
      TileSeq sq(sh, slot, nslot, g.det);
      for (; !failed && sq.next(); ++it) {
        const int s = it & 1, b = it & 1;
        const uint32_t ph = (it >> 1) & 1;
        if (!ptx::mbar_wait_abortable(&full[s], ph, abort)) { failed = true; break; }
        if (!ptx::mbar_wait_abortable(&tempty[b], ph ^ 1, abort)) { failed = true; break; }
        ptx::tc_fence_after();
        const uint32_t d = tbase + (uint32_t)(b * ctw);
        const uint64_t sadd = (uint64_t)(((uint32_t)s * (uint32_t)stage_bytes) >> 4);   // start-address field
        // chains: (hi, hi); SPLIT adds (lo halo, hi V^T) and (hi halo, lo V^T)
        for (int chn = 0; chn < (SPLIT ? 3 : 1); ++chn) {
          const uint64_t aoff = chn == 1 ? (uint64_t)(g.lo_off >> 4) : 0;
          const uint64_t boff = chn == 2 ? (uint64_t)((g.nch_f * chunkF) >> 4) : 0;
          if (a.tab.reg) {
            // regular tap layout: both descriptors advance by register adds (no table
            // loads, so the issue rate is the tensor core's): A by 256 bytes inside a
            // w-run and to the next copy's region at its end, B by 32 bytes inside a
            // 64-tap chunk and to the next chunk at its end
            uint64_t ad = sDesc[0].x + sadd + aoff, bd = sDesc[0].y + boff;
            const uint64_t a_run = (uint64_t)((g.region_bytes - (a.tab.hp - 1) * 256) >> 4);
            int jj = 0, bq = 0;
            for (int i = 0; i < g.nmma; ++i) {
              ptx::mma_bf16(d, ad, bd, idesc, (chn > 0 || i > 0) ? 1u : 0u);
              if (++jj == a.tab.hp) { jj = 0; ad += a_run; } else { ad += 16; }
              if (++bq == 4) { bq = 0; bd += (uint64_t)((chunkF >> 4) - 6); } else { bd += 2; }
            }
          } else {
#pragma unroll 4
            for (int i = 0; i < g.nmma; ++i) {
              const ulonglong2 dd = sDesc[i];
              ptx::mma_bf16(d, dd.x + sadd + aoff, dd.y + boff, idesc, (chn > 0 || i > 0) ? 1u : 0u);
            }
          }
        }
        ptx::mma_commit(&empty[s]);
        ptx::mma_commit(&tfull[b]);
      }
      ptx::mma_commit(dbar);
      if (!ptx::mbar_wait(dbar, 0)) failed = true;
      if (failed) *abort = 1;
    }
  } else {
    // Epilogue: 16 warps. Warp w reads TMEM lanes 32q..32q+31 (q = w % 4), i.e. voxels
    // 32q + lane of the tile. Task 0 of the warp is column group jq = (w - 2) / 4 (32
    // channels); in a channel tile wider than 128, task 1 is the warp's equal share of the
    // channels past 128 (E = (ctw - 128) / 4 of them, a multiple of 8), so that the four
    // warps of a voxel quarter carry the same load. U of the tile sits in a shared-memory
    // stage (SW128 boxes of 64 channels, row = voxel), loaded by TMA ahead of time; U' is
    // written back into the stage and stored by TMA. Column sums of U'^2 stay, per voxel
    // lane and channel, in registers (task 0) or in a shared-memory slot of the warp
    // (task 1) across the tiles of a chunk, and are reduced over the warp once per chunk
    // into its partial row group.
    // A failed wait marks the thread failed; it still arrives on every mbarrier that other
    // warps wait on (tempty, sready) but does no more waiting.
    const int q = warp & 3;
    const int ew = warp - 2;
    const int jq = ew >> 2;
    const int E = WIDE ? (ctw - 128) / 4 : 0;
    // first channel (in the tile) and width of task ti
#define TCS(ti) ((ti) == 0 ? 32 * jq : 128 + E * jq)
#define TCW(ti) ((ti) == 0 ? 32 : E)
    const int ntask = E > 0 ? 2 : 1;
    const int vox = q * 32 + lane;
    const uint32_t usw = (uint32_t)(lane & 7);                  // SW128 row phase (vox % 8)
    float* acc2 = sAcc2 + (size_t)ew * E * 32;                 // task 1's sums [j < E][lane]
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    int cur = -1, row0 = 0, curchunk = -1;
    int it = 0;
    TileSeq sq(sh, slot, nslot, g.det);
    for (; sq.next(); ++it) {
      const int jb = sq.jb;
      const JobDev& J = sh.jobs[jb];
      const int tile = sq.tile;
      if (sq.group() != curchunk) {
        if (cur >= 0 && wrU) {
          // flush the previous chunk's column sums into its row group
          const JobDev& P = sh.jobs[cur];
          for (int ti = 0; ti < ntask; ++ti) {
            const int c0 = ct * ctw + TCS(ti);
            if (ti == 1) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                acc[j] = j < E ? acc2[j * 32 + lane] : 0.f;
                if (j < E) acc2[j * 32 + lane] = 0.f;
              }
            }
            warp_colsum_store(acc, lane, P.part + ((size_t)row0 * PROW + q) * sh.kc + c0,
                              c0 + lane < sh.kc && lane < TCW(ti));
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = 0.f;
          }
        }
        cur = jb;
        curchunk = sq.group();
        row0 = g.det ? tile / J.fchunk : tile;
        if (rdU) {
          const float* src = mode == 1 ? J.D : J.s;
          const float sc = mode == 1 ? 1.f : (float)(1.0 / J.sc->theta);
          for (int ti = 0; ti < ntask; ++ti) {
            const int c0 = ct * ctw + TCS(ti);
            sD[ew * sdw + ti * 32 + lane] = (c0 + lane < sh.kc && lane < TCW(ti)) ? src[c0 + lane] * sc : 0.f;
          }
          __syncwarp();
        }
      }
      const int tw = tile % J.ntw, th = (tile / J.ntw) % J.nth, t = tile / (J.ntw * J.nth);
      const int h = th * TH + (vox >> 3), w = tw * TW + (vox & 7);
      const bool valid = h < J.H && w < J.W;
      const int b = it & 1;
      const uint32_t ph = (it >> 1) & 1;
      const int us = it % nus;
      const uint32_t uph = (it / nus) & 1;
      if (!failed)
        failed = !ptx::mbar_wait_abortable(rdU ? &ufull[us] : &uempty[us], rdU ? uph : (uph ^ 1), abort);
      if (!failed) failed = !ptx::mbar_wait_abortable(&tfull[b], ph, abort);
      ptx::tc_fence_after();
      // the groups' accumulator columns are read one after the other into e (the second
      // after the first has been used); the accumulator is released after the last read
      float e[32];
      const uint32_t tl = tbase + (uint32_t)(b * ctw) + ((uint32_t)(q * 32) << 16);
      float rsum = 0.f;
#pragma unroll 1
      for (int ti = 0; ti < ntask; ++ti) {
        tmem_ld_cols(tl + (uint32_t)TCS(ti), e, TCW(ti));
        ptx::tmem_ld_wait();
        if (ti == ntask - 1) {
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&tempty[b]);     // the accumulator is in registers
        }
        const int c0 = ct * ctw + TCS(ti);                        // first channel of this task
        const int nun = max(0, min(TCW(ti) / 8, (sh.kc - c0) / 8));   // 8-channel units inside kc
        const float* sDw = sD + ew * sdw + ti * 32;
        uint8_t* rowb = sU + (size_t)us * ustage + (size_t)vox * 128;   // this voxel's row of the stage
        const int cu0 = TCS(ti) >> 3;                             // first 8-channel unit of the task
        if (mode == 3) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (u < nun) {
              const uint4 x = *reinterpret_cast<const uint4*>(uunit(rowb, cu0 + u, usw));
              uint4 xl = make_uint4(0u, 0u, 0u, 0u);
              if (SPLIT) xl = *reinterpret_cast<const uint4*>(uunit(rowb, cu0 + u, usw) + uhalf);
              const float4 d0 = *reinterpret_cast<const float4*>(sDw + 8 * u);
              const float4 d1 = *reinterpret_cast<const float4*>(sDw + 8 * u + 4);
              const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
              const uint32_t xw[4] = {x.x, x.y, x.z, x.w};
              const uint32_t xlw[4] = {xl.x, xl.y, xl.z, xl.w};
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                float uf = __uint_as_float((j & 1) ? (xw[j >> 1] & 0xffff0000u) : (xw[j >> 1] << 16));
                if (SPLIT) uf += __uint_as_float((j & 1) ? (xlw[j >> 1] & 0xffff0000u) : (xlw[j >> 1] << 16));
                const float r = fmaf(uf, dv[j], e[8 * u + j]);
                rsum = fmaf(r, r, rsum);
              }
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (u < nun) {
              uint4* p = reinterpret_cast<uint4*>(uunit(rowb, cu0 + u, usw));
              uint4* pl = reinterpret_cast<uint4*>(uunit(rowb, cu0 + u, usw) + uhalf);
              float dv[8];
              uint32_t xw[4] = {0u, 0u, 0u, 0u}, xlw[4] = {0u, 0u, 0u, 0u};
              if (mode == 1) {
                const uint4 x = *p;
                xw[0] = x.x; xw[1] = x.y; xw[2] = x.z; xw[3] = x.w;
                if (SPLIT) {
                  const uint4 y = *pl;
                  xlw[0] = y.x; xlw[1] = y.y; xlw[2] = y.z; xlw[3] = y.w;
                }
                const float4 d0 = *reinterpret_cast<const float4*>(sDw + 8 * u);
                const float4 d1 = *reinterpret_cast<const float4*>(sDw + 8 * u + 4);
                dv[0] = d0.x; dv[1] = d0.y; dv[2] = d0.z; dv[3] = d0.w;
                dv[4] = d1.x; dv[5] = d1.y; dv[6] = d1.z; dv[7] = d1.w;
              } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) dv[j] = 0.f;
              }
              uint32_t ow[4], olw[4];
#pragma unroll
              for (int j2 = 0; j2 < 4; ++j2) {
                // the two channels of word j2 (its low and high halves)
                float ua = __uint_as_float(xw[j2] << 16), ub = __uint_as_float(xw[j2] & 0xffff0000u);
                if (SPLIT) {
                  ua += __uint_as_float(xlw[j2] << 16);
                  ub += __uint_as_float(xlw[j2] & 0xffff0000u);
                }
                const float na = fmaf(ua, dv[2 * j2], -e[8 * u + 2 * j2]);
                const float nb = fmaf(ub, dv[2 * j2 + 1], -e[8 * u + 2 * j2 + 1]);
                const __nv_bfloat162 pr = __floats2bfloat162_rn(na, nb);
                ow[j2] = *reinterpret_cast<const uint32_t*>(&pr);
                float ra = __uint_as_float(ow[j2] << 16), rb = __uint_as_float(ow[j2] & 0xffff0000u);
                if (SPLIT) {
                  const __nv_bfloat162 pl2 = __floats2bfloat162_rn(na - ra, nb - rb);
                  olw[j2] = *reinterpret_cast<const uint32_t*>(&pl2);
                  ra += __uint_as_float(olw[j2] << 16);
                  rb += __uint_as_float(olw[j2] & 0xffff0000u);
                }
                const int ja = 8 * u + 2 * j2;
                if (ti == 0) {
                  acc[ja] = valid ? fmaf(ra, ra, acc[ja]) : acc[ja];
                  acc[ja + 1] = valid ? fmaf(rb, rb, acc[ja + 1]) : acc[ja + 1];
                } else if (valid) {
                  acc2[ja * 32 + lane] = fmaf(ra, ra, acc2[ja * 32 + lane]);
                  acc2[(ja + 1) * 32 + lane] = fmaf(rb, rb, acc2[(ja + 1) * 32 + lane]);
                }
              }
              *p = make_uint4(ow[0], ow[1], ow[2], ow[3]);
              if (SPLIT) *pl = make_uint4(olw[0], olw[1], olw[2], olw[3]);
            }
          }
        }
        if (mode == 3) {
          // residual partial of this group (one per (channel group, voxel quarter))
          float r = valid ? rsum : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
          if (lane == 0) J.rpart[(size_t)tile * sh.nrp + (ct * 8 + (ti == 0 ? jq : 4 + jq)) * 4 + q] = r;
          rsum = 0.f;
        }
      }
      // done with the stage: the producer thread stores U' from it (the writes are made
      // visible to the async proxy first) and refills it
      if (wrU) ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&sready[us]);
    }
    if (cur >= 0 && wrU) {
      const JobDev& P = sh.jobs[cur];
      for (int ti = 0; ti < ntask; ++ti) {
        const int c0 = ct * ctw + TCS(ti);
        if (ti == 1) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            acc[j] = j < E ? acc2[j * 32 + lane] : 0.f;
            if (j < E) acc2[j * 32 + lane] = 0.f;
          }
        }
        warp_colsum_store(acc, lane, P.part + ((size_t)row0 * PROW + q) * sh.kc + c0,
                          c0 + lane < sh.kc && lane < TCW(ti));
      }
    }
  }
  if (failed) set_fail(sh);
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tbase, tcols);
  }
}

#undef TCS
#undef TCW

// ---------------------------------------------------------------------------------
// Adjoint pass
// ---------------------------------------------------------------------------------
// Tap columns of the adjoint: column j of tap tile tt belongs to 32-column group
// G = gpt tt + j / 32, which holds rpg <= floor(32 / k2) whole tap rows (st, sh) of k2 taps
// each (row TR = G rpg + r, r = (j % 32) / k2, sw = (j % 32) % k2, TR = st k1 + sh);
// the remaining 32 - rpg k2 columns of a group and the rows past k1 k3 are padding.
// Returns the tap s = TR k2 + sw of a column, or -1 for padding.
// Kernel widths without a compile-time col2im (rpg = 0) keep the taps in order: column
// j of tap tile tt is tap 128 tt + j.
__host__ __device__ __forceinline__ int adj_tap_of_col(const TcGeom& g, int tt, int j) {
  if (g.rpg == 0) {
    const int s = tt * 128 + j;
    return s < g.k ? s : -1;
  }
  const int G = tt * g.gpt + j / 32, r = (j % 32) / g.k2, sw = (j % 32) % g.k2;
  const int TR = G * g.rpg + r;
  if (r >= g.rpg || TR >= g.k1 * g.k3) return -1;
  return TR * g.k2 + sw;
}

// Halo-buffer offset of tap row TR = (st, sh) for a voxel in tile row 0: the contribution
// of voxel (h, w) and tap (st, sh, sw) lands at h*pitch + rowoff(TR) + (w + k2 - 1 - sw).
__device__ __forceinline__ int adj_rowoff(const TcGeom& g, int TR) {
  const int st = TR / g.k1, shh = TR % g.k1;
  return ((g.k3 - 1 - st) * g.Hb + (g.k1 - 1 - shh)) * g.pitch;
}

// col2im of one warp's 32 accumulator columns (K2 = k2 known at compile time): for each
// of its whole tap rows, the 8 lanes of a tile row (w = lane % 8) first sum the values
// that land on the same halo column o = w + k2 - 1 - sw with warp shuffles (lane w keeps
// the outputs o = w + 8j), then add those sums into the halo buffer: 1 + (k2 - 1) / 8
// shared-memory reductions per lane and tap row instead of k2. The sum over the 8 lanes
// runs in a fixed order; the reductions of different warps into one address do not.
template <int K2, typename HT>
__device__ __forceinline__ void adj_col2im_rows(const float (&e)[32], int lane, HT* hb, int hoff,
                                                const TcGeom& g, int G, const int* rtab, int TR0) {
  constexpr int RPG = 32 / K2;            // tap rows a group can hold; it holds g.rpg <= RPG
  constexpr int NJ = (K2 + 14) / 8;      // halo columns 0 .. K2 + 6 over 8 lanes
  const int w = lane & 7;
#pragma unroll
  for (int r = 0; r < RPG; ++r) {
    if (r >= g.rpg) break;                 // warp-uniform: the group's unused rows
    const int TR = G * g.rpg + r;
    if (TR >= g.k1 * g.k3) break;          // warp-uniform: padding rows
    const int base = hoff + rtab[TR - TR0];   // adj_rowoff(g, TR), tabulated per CTA
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      float T = 0.f;
#pragma unroll
      for (int d = -7; d <= 7; ++d) {
        const int idx = d + K2 - 1 - 8 * j;  // tap sw whose value lane w + d sends to o = w + 8j
        if (idx < 0 || idx >= K2) continue;
        const float x = (d == 0) ? e[r * K2 + idx] : __shfl_sync(0xffffffffu, e[r * K2 + idx], (lane + d) & 31);
        if (w + d >= 0 && w + d <= 7) T += x;
      }
      const int o = w + 8 * j;
      if (o <= K2 + 6) col_add(&hb[base + o], T);
    }
  }
}

// Adjoint pass G = U (D V^T) with col2im: per voxel tile and tap tile, the MMA leaves
// G[voxel][tap column] in TMEM; the epilogue adds it into a shared-memory halo buffer
// (Hb x pitch per frame of the k3-frame halo) and flushes the buffer to the tile's halo
// partial, which the gather pass sums. K2 = 0 selects the per-element reduction path
// for kernel widths without a compile-time specialisation.
// WIDE: tap tiles of 256 columns (g.gpt == 8; each epilogue warp takes two column groups);
// otherwise 128 columns as compile-time constants.
template <int K2, bool DET, bool WIDE>
__global__ void __launch_bounds__(TC_THREADS, 1) adj_tc_kernel(const __grid_constant__ AdjArgs a) {
  using HT = typename std::conditional<DET, unsigned long long, float>::type;   // halo entry
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1k(smraw);
  const TcGeom& g = a.g;
  const Shared& sh = a.sh;
  const int nta = WIDE ? 256 : 128;              // tap-tile columns (the MMA's N)
  const int gpt = WIDE ? 8 : 4;
  const int chunkA = nta * 128;                  // one 64-channel chunk of the V D image
  const uint32_t tcols = WIDE ? 512u : TMEM_COLS;   // two accumulators of nta columns
  uint8_t* sA = sm;
  uint8_t* sU = sm + (size_t)g.nch_a * chunkA;
  HT* buf = reinterpret_cast<HT*>(sU + (size_t)ADJ_STAGES * CHUNK);   // [2][HBp]
  int* toff = reinterpret_cast<int*>(buf + 2 * (size_t)g.HBp);              // [128] (K2 = 0)
  uint64_t* bars = reinterpret_cast<uint64_t*>(toff + 128);
  uint64_t* full = bars;                           // [ADJ_STAGES]
  uint64_t* empty = bars + ADJ_STAGES;             // [ADJ_STAGES]
  uint64_t* tfull = bars + 2 * ADJ_STAGES;         // [2]
  uint64_t* tempty = tfull + 2;                    // [2]
  uint64_t* abar = tfull + 4;
  uint64_t* dbar = tfull + 5;
  uint64_t* redbar = tfull + 6;                    // [2] all epilogue warps have added a tile
  uint64_t* zbar = tfull + 8;                      // [2] a halo buffer has been flushed and cleared
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tfull + 10);
  static_assert((2 * ADJ_STAGES + 10) * 8 + 4 <= 256, "adjoint barriers exceed their space");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tt = blockIdx.x % g.ntt;
  const int slot = blockIdx.x / g.ntt, nslot = gridDim.x / g.ntt;
  const int lo = (int)((long long)sh.total_tiles * slot / nslot);
  const int hi = (int)((long long)sh.total_tiles * (slot + 1) / nslot);

  if (threadIdx.x == 0) {
    for (int i = 0; i < ADJ_STAGES; ++i) {
      ptx::mbar_init(&full[i], 1);
      ptx::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&tfull[i], 1);
      ptx::mbar_init(&tempty[i], EPI_WARPS);
      ptx::mbar_init(&redbar[i], EPI_WARPS);
      ptx::mbar_init(&zbar[i], EPI_WARPS);
    }
    ptx::mbar_init(abar, 1);
    ptx::mbar_init(dbar, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tslot, tcols);
    ptx::tmem_relinquish();
  }
  for (int i = threadIdx.x; i < 2 * g.HBp; i += blockDim.x) buf[i] = (HT)0;
  // K2 = 0: halo offset of each tap column (-1 for padding); G[v][j] lands at
  // buf[h_v * pitch + w_v + toff[j]]
  if (K2 == 0 && threadIdx.x < 128) {
    const int s = adj_tap_of_col(g, tt, threadIdx.x);
    int o = -1;
    if (s >= 0) {
      const int sw = s % g.k2, shh = (s / g.k2) % g.k1, st = s / (g.k1 * g.k2);
      o = ((g.k3 - 1 - st) * g.Hb + (g.k1 - 1 - shh)) * g.pitch + (g.k2 - 1 - sw);
    }
    toff[threadIdx.x] = o;
  }
  // compile-time k2: halo offset of each tap row of this tap tile (at most gpt * 32 / k2 <=
  // 80 rows), toff[TR - TR0] for row TR
  if (K2 > 0 && threadIdx.x < 128) {
    const int TR = tt * g.gpt * g.rpg + threadIdx.x;
    toff[threadIdx.x] = TR < g.k1 * g.k3 ? adj_rowoff(g, TR) : 0;
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tbase = *tslot;
  bool failed = false;

  if (warp == 0) {
    if (lane == 0) {
      int cnt = 0;
      for (int tg = lo; tg < hi && !failed; ++tg) {
        const int jb = job_of_tile(sh.job_tile0, sh.njobs, tg);
        const JobDev& J = sh.jobs[jb];
        const int tile = tg - sh.job_tile0[jb];
        const int tw = tile % J.ntw, th = (tile / J.ntw) % J.nth, t = tile / (J.ntw * J.nth);
        for (int c = 0; c < g.nch_a; ++c, ++cnt) {
          const int s = cnt % ADJ_STAGES;
          const uint32_t ph = (cnt / ADJ_STAGES) & 1;
          if (!ptx::mbar_wait(&empty[s], ph ^ 1)) { failed = true; break; }
          ptx::mbar_arrive_expect_tx(&full[s], CHUNK);
          ptx::tma_load_4d(sU + (size_t)s * CHUNK, J.tmapU, c * 64, tw * TW, th * TH, t, &full[s]);
        }
      }
      for (int i = (cnt > ADJ_STAGES ? cnt - ADJ_STAGES : 0); i < cnt; ++i)
        if (!ptx::mbar_wait(&full[i % ADJ_STAGES], (i / ADJ_STAGES) & 1)) failed = true;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // A = U tile (voxels x channels), B = V D image (tap columns x channels), both
      // K-major SW128: G[voxel][tap column] in TMEM.
      const uint32_t idesc = ptx::idesc_bf16(128, (uint32_t)nta, 0, 0);
      // descriptors of U stage 0 and image chunk 0; others differ only in the start address
      const uint64_t ubase = ptx::sdesc(ptx::smem_u32(sU), 16, 1024, 2);
      const uint64_t bbase = ptx::sdesc(ptx::smem_u32(sA), 16, 1024, 2);
      int cur = -1, cnt = 0, i = 0;
      uint32_t aph = 0, dph = 0;
      for (int tg = lo; tg < hi && !failed; ++tg, ++i) {
        const int jb = job_of_tile(sh.job_tile0, sh.njobs, tg);
        if (jb != cur) {
          // the MMAs that read the previous job's image must finish before it is replaced
          if (cur >= 0) {
            ptx::mma_commit(dbar);
            if (!ptx::mbar_wait(dbar, dph)) { failed = true; break; }
            dph ^= 1;
          }
          ptx::mbar_arrive_expect_tx(abar, (uint32_t)(g.nch_a * chunkA));
          const uint8_t* src = reinterpret_cast<const uint8_t*>(sh.jobs[jb].B2img) + (size_t)tt * g.nch_a * chunkA;
          for (int c = 0; c < g.nch_a; ++c)
            ptx::bulk_g2s(sA + (size_t)c * chunkA, src + (size_t)c * chunkA, (uint32_t)chunkA, abar);
          if (!ptx::mbar_wait(abar, aph)) { failed = true; break; }
          aph ^= 1;
          cur = jb;
        }
        const int b = i & 1;
        const uint32_t bph = (i >> 1) & 1;
        if (!ptx::mbar_wait(&tempty[b], bph ^ 1)) { failed = true; break; }
        ptx::tc_fence_after();
        const uint32_t d = tbase + (uint32_t)(b * nta);
        for (int c = 0; c < g.nch_a; ++c, ++cnt) {
          const int s = cnt % ADJ_STAGES;
          const uint32_t ph = (cnt / ADJ_STAGES) & 1;
          if (!ptx::mbar_wait(&full[s], ph)) { failed = true; break; }
          ptx::tc_fence_after();
          const uint64_t ad0 = ubase + (uint64_t)(s * (CHUNK >> 4));
          const uint64_t bd0 = bbase + (uint64_t)(c * (chunkA >> 4));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) ptx::mma_bf16(d, ad0 + 2 * kk, bd0 + 2 * kk, idesc, (c | kk) ? 1u : 0u);
          ptx::mma_commit(&empty[s]);
        }
        if (failed) break;
        ptx::mma_commit(&tfull[b]);
      }
      ptx::mma_commit(dbar);
      if (!ptx::mbar_wait(dbar, dph)) failed = true;
    }
  } else {
    // Epilogue: 16 warps. Warp w reads TMEM lanes 32q..32q+31 (q = w % 4), i.e. voxels
    // 32q + lane (rows 4q..4q+3 of the tile, w = lane % 8), and columns 32g..32g+31
    // (g = (w - 2) / 4), i.e. one group of whole tap rows. Tile i is added into halo
    // buffer i % 2; while tile i is added, the warps flush tile i-1's buffer (write the
    // partial, clear), so the two phases of consecutive tiles overlap.
    const int q = warp & 3;
    const int cg = (warp - 2) >> 2;
    const int ew = warp - 2;
    const int vox = q * 32 + lane;
    const int hoff = (vox >> 3) * g.pitch;
    // The halo entries a thread flushes (p = ew*32 + lane + i*512) are the same for every
    // tile: their buffer index and (frame, row, column) are packed once into one word each
    // (si << 16 | st << 12 | bh << 6 | bw; all-ones: nothing to flush) where they fit
    constexpr int FL_MAX = 4;
    const bool fl_pre = g.HB <= FL_MAX * 32 * EPI_WARPS && g.k3 <= 16 && g.Hb <= 64 && g.Wb <= 64 &&
                        g.HBp <= 65535;
    uint32_t fl[FL_MAX];
#pragma unroll
    for (int f = 0; f < FL_MAX; ++f) {
      const int p = ew * 32 + lane + f * 32 * EPI_WARPS;
      uint32_t code = 0xFFFFFFFFu;
      if (fl_pre && p < g.HB) {
        const int row = p / g.Wb, col = p - row * g.Wb;
        const int j = row / g.Hb, bh = row - j * g.Hb;
        const int st = g.slo[tt] + j;
        if (st < g.k3)
          code = ((uint32_t)(((g.k3 - 1 - st) * g.Hb + bh) * g.pitch + col) << 16) | ((uint32_t)st << 12) |
                 ((uint32_t)bh << 6) | (uint32_t)col;
      }
      fl[f] = code;
    }
    int i = 0;
    int prev_jb = 0, prev_t = 0, prev_h0 = 0, prev_w0 = 0;   // tile flushed next: job, frame, halo origin
    TileXY txy;
    for (int tg = lo; tg <= hi; ++tg, ++i) {
      const bool have = tg < hi;
      HT* hb = buf + (size_t)(i & 1) * g.HBp;
      if (have) {
        // buffer i % 2 was last used by tile i - 2; wait until it has been flushed
        if (i >= 2 && !ptx::mbar_wait(&zbar[i & 1], ((i - 2) >> 1) & 1)) { failed = true; break; }
        const int b = i & 1;
        const uint32_t bph = (i >> 1) & 1;
        if (!ptx::mbar_wait(&tfull[b], bph)) { failed = true; break; }
        ptx::tc_fence_after();
        // the warp's column groups: cg, and cg + 4 in a 256-column tap tile, read from
        // TMEM one after the other into v; the accumulator is released after the last read
        float v[32];
        const uint32_t tl = tbase + (uint32_t)(b * nta) + ((uint32_t)(q * 32) << 16);
        if constexpr (K2 > 0) {
#pragma unroll 1
          for (int gi = 0; gi < (WIDE ? 2 : 1); ++gi) {
            ptx::tmem_ld32(tl + (uint32_t)(cg + 4 * gi) * 32, v);
            ptx::tmem_ld_wait();
            if (gi == (WIDE ? 1 : 0)) {
              ptx::tc_fence_before();
              __syncwarp();
              if (lane == 0) ptx::mbar_arrive(&tempty[b]);
            }
            adj_col2im_rows<K2>(v, lane, hb, hoff, g, tt * gpt + cg + 4 * gi, toff, tt * gpt * g.rpg);
          }
        } else {
          ptx::tmem_ld32(tl + (uint32_t)cg * 32, v);
          ptx::tmem_ld_wait();
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&tempty[b]);
          const int vbase = hoff + (vox & 7);
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int o = toff[cg * 32 + e];
            if (o >= 0) col_add(&hb[vbase + o], v[e]);
          }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&redbar[i & 1]);
      }
      // flush tile i-1: every warp has added it into buffer (i-1) % 2
      if (i >= 1) {
        const int pb = (i - 1) & 1;
        if (!ptx::mbar_wait(&redbar[pb], ((i - 1) >> 1) & 1)) { failed = true; break; }
        HT* src = buf + (size_t)pb * g.HBp;
        // halo entry (frame st, row bh, column bw) belongs to voxel ((t - st) mod T,
        // (th*TH - (k1-1) + bh) mod H, (tw*TW - (k2-1) + bw) mod W); only the nsl frames
        // this tap tile reaches (from slo) can be nonzero
        const JobDev& P = sh.jobs[prev_jb];
        const int PT = P.T, PH = P.H, PW = P.W;
        HT* PG = reinterpret_cast<HT*>(P.G);
        auto flush_one = [&](int si, int st, int bh, int col) {
          const HT v = src[si];
          src[si] = (HT)0;
          int tq = prev_t - st, hq = prev_h0 + bh, wq = prev_w0 + col;
          tq += tq < 0 ? PT : 0;
          hq = hq < 0 ? hq + PH : (hq >= PH ? hq - PH : hq);
          wq = wq < 0 ? wq + PW : (wq >= PW ? wq - PW : wq);
          if (v) atomicAdd(PG + ((size_t)tq * PH + hq) * PW + wq, v);
        };
        if (fl_pre) {
#pragma unroll
          for (int f = 0; f < FL_MAX; ++f) {
            const uint32_t code = fl[f];
            if (code != 0xFFFFFFFFu)
              flush_one((int)(code >> 16), (int)((code >> 12) & 15u), (int)((code >> 6) & 63u), (int)(code & 63u));
          }
        } else {
          for (int p = ew * 32 + lane; p < g.HB; p += 32 * EPI_WARPS) {
            const int row = p / g.Wb, col = p - row * g.Wb;   // row = j * Hb + bh
            const int j = row / g.Hb, bh = row - j * g.Hb;
            const int st = g.slo[tt] + j;
            if (st >= g.k3) continue;
            flush_one(((g.k3 - 1 - st) * g.Hb + bh) * g.pitch + col, st, bh, col);
          }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&zbar[pb]);
      }
      if (have) {
        const int jb = (txy.jb >= 0 && tg < sh.job_tile0[txy.jb + 1]) ? txy.jb
                                                                      : job_of_tile(sh.job_tile0, sh.njobs, tg);
        const JobDev& J = sh.jobs[jb];
        const int tile = tg - sh.job_tile0[jb];
        txy.at(jb, tile, J);
        prev_jb = jb;
        prev_t = txy.t;
        prev_h0 = txy.th * TH - (g.k1 - 1);
        prev_w0 = txy.tw * TW - (g.k2 - 1);
      }
    }
  }
  if (failed) set_fail(sh);
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tbase, tcols);
  }
}

// ---------------------------------------------------------------------------------
// Per-iteration images and gathers
// ---------------------------------------------------------------------------------
// A operand of the adjoint: rows = taps of tile tt, K = channels; value bf16(V[s][c] D[c]).
// SW128 K-major: 16-byte unit j of row r sits at unit j ^ (r % 8) of the 128-byte row.
__global__ void build_B2_kernel(Shared sh, TcGeom g) {
  const JobDev& J = sh.jobs[blockIdx.x];
  const int tt = blockIdx.y / g.nch_a, c = blockIdx.y % g.nch_a;
  uint8_t* img = reinterpret_cast<uint8_t*>(J.B2img) + ((size_t)tt * g.nch_a + c) * (g.nta * 128);
  for (int u = threadIdx.x; u < g.nta * 8; u += blockDim.x) {
    const int r = u >> 3, j = u & 7;
    const int s = adj_tap_of_col(g, tt, r);
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int ch = c * 64 + j * 8 + e;
      const float x = (s >= 0 && ch < sh.k) ? sh.Vf[(size_t)s * sh.kc + ch] * J.D[ch] : 0.f;
      v[e] = __float2bfloat16(x);
    }
    *reinterpret_cast<uint4*>(img + (r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) * 16)) =
        *reinterpret_cast<const uint4*>(v);
  }
}

// Copy c of the forward operand, element (tp, hp, wp), is
//   bf16(src[(tp - (k3-1)) mod T][(hp - (k1-1)) mod H][(wp - 8(nwc-1) - c) mod W]),
// stored as Xc[c][wp / 8][hp][tp][wp % 8]: the k3 frames of a 16-byte w-segment are
// adjacent, so one TMA box row of the tile halo is k3 * 16 bytes. A thread reads the
// NC + 7 source values of one (w-segment, hp, tp) once and writes all NC copies.
// SPLIT: copies NC..2NC-1 hold the lo parts, bf16(x - bf16(x)), of copies 0..NC-1.
template <int NC, bool SPLIT>
__global__ void prepare_X_kernel(Shared sh, TcGeom g, int from_L) {
  const JobDev& J = sh.jobs[blockIdx.y];
  const float* src = from_L ? J.L : J.X;
  const int nwcol = J.xWp / 8;
  const long long nunits = (long long)nwcol * J.xHp * J.xTp;
  const int pw = 8 * (g.nwc - 1);
  const size_t plane = (size_t)nwcol * J.xHp * J.xTp * 8;   // one copy
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < nunits;
       u += (long long)gridDim.x * blockDim.x) {
    const int tp = (int)(u % J.xTp);
    long long r = u / J.xTp;
    const int hp = (int)(r % J.xHp);
    const int wu = (int)(r / J.xHp);
    const long long rowb = ((long long)wrapi(tp - (g.k3 - 1), J.T) * J.H + wrapi(hp - (g.k1 - 1), J.H)) * J.W;
    const int w0 = wu * 8 - pw - (NC - 1);                     // first source column of the window
    float win[NC + 7];
    if (w0 >= 0 && w0 + NC + 6 < J.W) {
#pragma unroll
      for (int i = 0; i < NC + 7; ++i) win[i] = src[rowb + w0 + i];
    } else {
#pragma unroll
      for (int i = 0; i < NC + 7; ++i) win[i] = src[rowb + wrapi(w0 + i, J.W)];
    }
    __nv_bfloat16* dst = J.Xc + (((size_t)wu * J.xHp + hp) * J.xTp + tp) * 8;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      __align__(16) __nv_bfloat16 v[8];
      __align__(16) __nv_bfloat16 vl[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float x = win[NC - 1 - c + e];
        v[e] = __float2bfloat16(x);
        if (SPLIT) vl[e] = __float2bfloat16(x - __bfloat162float(v[e]));
      }
      *reinterpret_cast<uint4*>(dst + (size_t)c * plane) = *reinterpret_cast<const uint4*>(v);
      if (SPLIT) *reinterpret_cast<uint4*>(dst + (size_t)(NC + c) * plane) = *reinterpret_cast<const uint4*>(vl);
    }
  }
}

// L-update from the col2im sums: Delta_j (added into J.G by the adjoint pass, over all
// tap tiles and tiles whose halo covers voxel j) is read and cleared for the next pass,
// then the same projection as the FP32 path. Flat over the voxels: block (b, job) takes
// voxels 1024 b .. 1024 b + 1023 of the job, four per thread with 16-byte accesses; the
// block's ||L'||^2 partial goes to lpart[b].
template <bool DET>
__global__ void __launch_bounds__(256) gather_tc_kernel(Shared sh) {
  const JobDev& J = sh.jobs[blockIdx.y];
  const long long v0 = (long long)blockIdx.x * 1024 + 4 * threadIdx.x;
  if ((long long)blockIdx.x * 1024 >= J.m) return;             // the whole block is past this job
  const double th = J.sc->theta, thn = J.sc->theta_next;
  const float xa = (float)(th + thn), xb = -(float)th;
  const float inv = (float)(1.0 / (sh.k * th));
  float l2 = 0.f;
  unsigned long long* Dx = reinterpret_cast<unsigned long long*>(J.G);   // fixed-point Delta (DET)
  if (v0 + 3 < J.m) {
    float4 d;
    if (DET) {
      const ulonglong2 da = *reinterpret_cast<const ulonglong2*>(Dx + v0);
      const ulonglong2 db = *reinterpret_cast<const ulonglong2*>(Dx + v0 + 2);
      *reinterpret_cast<ulonglong2*>(Dx + v0) = make_ulonglong2(0ull, 0ull);
      *reinterpret_cast<ulonglong2*>(Dx + v0 + 2) = make_ulonglong2(0ull, 0ull);
      d = make_float4((float)((double)(long long)da.x * FX_INV), (float)((double)(long long)da.y * FX_INV),
                      (float)((double)(long long)db.x * FX_INV), (float)((double)(long long)db.y * FX_INV));
    } else {
      d = *reinterpret_cast<const float4*>(J.G + v0);
      *reinterpret_cast<float4*>(J.G + v0) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 lo = *reinterpret_cast<const float4*>(J.L + v0);
    const float4 mv = *reinterpret_cast<const float4*>(J.M + v0);
    const uchar4 ob = *reinterpret_cast<const uchar4*>(J.mask + v0);
    const float dd[4] = {d.x, d.y, d.z, d.w}, ll[4] = {lo.x, lo.y, lo.z, lo.w}, mm[4] = {mv.x, mv.y, mv.z, mv.w};
    const bool oo[4] = {ob.x != 0, ob.y != 0, ob.z != 0, ob.w != 0};
    float ln[4], xn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (isinf(J.lam)) {
        ln[e] = oo[e] ? mm[e] : fmaf(dd[e], inv, ll[e]);
      } else {
        const double lt = oo[e] ? J.lam : 0.0;
        ln[e] = (float)(((double)dd[e] / sh.k + th * (double)ll[e] + lt * (oo[e] ? (double)mm[e] : 0.0)) / (lt + th));
      }
      xn[e] = fmaf(xa, ln[e], xb * ll[e]);
      l2 = fmaf(ln[e], ln[e], l2);
    }
    *reinterpret_cast<float4*>(J.L + v0) = make_float4(ln[0], ln[1], ln[2], ln[3]);
    *reinterpret_cast<float4*>(J.X + v0) = make_float4(xn[0], xn[1], xn[2], xn[3]);
  } else {
    for (long long v = v0; v < J.m; ++v) {
      float d;
      if (DET) {
        d = (float)((double)(long long)Dx[v] * FX_INV);
        Dx[v] = 0ull;
      } else {
        d = J.G[v];
        J.G[v] = 0.f;
      }
      const float Ln = l_update(J, sh.k, v, d);
      l2 = fmaf(Ln, Ln, l2);
    }
  }
  // block partial in a fixed order: warp butterflies, then the 8 warps
  __shared__ float red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
  __syncthreads();
  if (threadIdx.x == 0)
    J.lpart[blockIdx.x] = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
}

// One CTA waits, through the solve kernels' bounded wait, on an mbarrier that nothing
// arrives on; the wait gives up after limit_ns and the kernel reports it in *status (the
// same path a solve kernel takes when a copy or an MMA never completes). Nothing is in
// flight and no tensor memory is held, so the kernel simply returns.
__global__ void bounded_wait_check_kernel(uint64_t limit_ns, int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    abort = 0;
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = ptx::mbar_wait_abortable(&bar, 0, &abort, limit_ns);
    *status = ok ? 0 : 1;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
TcGeom tc_geom(int k1, int k2, int k3, int kc, const TcTiles& t) {
  TcGeom g = make_geom(k1, k2, k3, t.gpt_max, t.ctw_max, t.nus_max, t.det);
  g.kc = kc;
  return g;
}

bool tc_supported(int k1, int k2, int k3, std::string* why) {
  const TcGeom g = make_geom(k1, k2, k3, 4);
  auto no = [&](const char* m) { if (why) *why = m; return false; };
  if (g.k > 512) return no("k > 512");
  if (k2 > 16) return no("k2 > 16");
  if (g.ntt > 16) return no("more than 16 adjoint tap tiles");
  if (g.nmma > 64) return no("padded forward K > 1024");
  if (g.Hh > 256 || k3 > 256) return no("halo box too tall");
  if (fwd_smem(g) > SMEM_LIMIT) return no("forward shared memory exceeds 227 KiB");
  if (adj_smem(g) > SMEM_LIMIT) return no("adjoint shared memory exceeds 227 KiB");
  if (!encoder()) return no("cuTensorMapEncodeTiled unavailable");
  return true;
}

// B image of the forward pass for channel tiles of `ctw` channels: tile ct, K chunk c (64
// taps), row r (channel ct*ctw + r), SW128 K-major (16-byte unit j of row r at unit
// j ^ (r % 8) of its 128-byte row, 8-row groups 1024 bytes apart); the taps in the
// forward K order (w-runs of k1*k3 taps padded to R8). `part` 0: bf16(V), 1: the
// remainder bf16(V - bf16(V)).
static std::vector<uint8_t> fwd_images(const TcGeom& g, const double* V64, int ctw, int nct, int part) {
  const int k = g.k, k1 = g.k1, k3 = g.k3;
  const size_t chunk = (size_t)ctw * 128, per = (size_t)g.nch_f * chunk;
  std::vector<uint8_t> img((size_t)nct * per, 0);
  const int per8 = g.R8 / 8;
  for (int ct = 0; ct < nct; ++ct)
    for (int r = 0; r < ctw; ++r) {
      const int ch = ct * ctw + r;
      if (ch >= k) continue;
      for (int kap = 0; kap < g.kpad; ++kap) {
        const int grp = kap / 8, rin = kap % 8;
        if (grp >= g.ngrp) continue;
        const int sw = grp / per8, rr = (grp % per8) * 8 + rin;
        if (rr >= g.R) continue;
        const int u = g.R - 1 - rr, sh = u / k3, st = u % k3;
        const int s = (st * k1 + sh) * g.k2 + sw;
        const double vd = V64[(size_t)ch * k + s];
        const __nv_bfloat16 hi = __float2bfloat16((float)vd);
        const __nv_bfloat16 b = part == 0 ? hi : __float2bfloat16((float)(vd - (double)__bfloat162float(hi)));
        const int c = kap / 64, col = kap % 64;
        const size_t off = (size_t)ct * per + (size_t)c * chunk + (r / 8) * 1024 + (r % 8) * 128 +
                           (((col / 8) ^ (r % 8)) * 16) + (col % 8) * 2;
        memcpy(&img[off], &b, 2);
      }
    }
  return img;
}

cudaError_t tc_build_vdata(const double* V64, int k1, int k2, int k3, int kc, TcVData* out, const TcTiles& t) {
  TcGeom g = make_geom(k1, k2, k3, t.gpt_max, t.ctw_max, t.nus_max, t.det);
  g.kc = kc;
  out->g = g;
  std::vector<uint8_t> img = fwd_images(g, V64, g.ctw, g.nct, 0);
  for (int i = 0; i < 64; ++i) { out->boff[i] = 0; out->kstr[i] = 0; }
  for (int i = 0; i < g.nmma; ++i) {
    out->boff[i] = group_off(g, 2 * i);
    out->kstr[i] = (2 * i + 1 < g.ngrp) ? group_off(g, 2 * i + 1) - group_off(g, 2 * i) : 0;
  }
  cudaError_t e = cudaMalloc(&out->VtImg, img.size());
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpy(out->VtImg, img.data(), img.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if (g.split_ok) {
    std::vector<uint8_t> hi = fwd_images(g, V64, 128, g.nct_s, 0), lo = fwd_images(g, V64, 128, g.nct_s, 1);
    hi.insert(hi.end(), lo.begin(), lo.end());
    if ((e = cudaMalloc(&out->VtImgS, hi.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(out->VtImgS, hi.data(), hi.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void tc_free_vdata(TcVData* v) {
  if (v->VtImg) cudaFree(v->VtImg);
  if (v->VtImgS) cudaFree(v->VtImgS);
  v->VtImg = nullptr;
  v->VtImgS = nullptr;
}

// residual partials per tile: 8 task slots (4 column groups and 4 shares of the channels
// past 128) x 4 voxel quarters per channel tile (an upper bound for every channel-tile width)
int tc_nrp(int k) {
  const int kc = (k + 15) / 16 * 16;
  return std::max(32 * ((k + 127) / 128), 4 * ((kc + 31) / 32));
}

static void xc_dims(const TcGeom& g, int H, int W, int T, int& Tp, int& Hp, int& Wp) {
  const int nth = (H + TH - 1) / TH, ntw = (W + TW - 1) / TW;
  Tp = T + g.k3 - 1;
  Hp = nth * TH + g.k1 - 1;
  Wp = ntw * TW + 8 * (g.nwc - 1);
}

size_t tc_job_extra_bytes(int H, int W, int T, const TcGeom& g) {
  int Tp, Hp, Wp;
  xc_dims(g, H, W, T, Tp, Hp, Wp);
  const int ntiles = ((H + TH - 1) / TH) * ((W + TW - 1) / TW) * T;
  size_t b = 0;
  auto add = [&](size_t n) { b += (n + 255) / 256 * 256; };
  add((size_t)(g.split_ok ? 2 : 1) * g.ncopy * Tp * Hp * Wp * 2);   // Xc (and its lo copies)
  add((size_t)H * W * T * 8);                          // col2im sums (Delta, 64-bit fixed point)
  add((size_t)g.ntt * g.nch_a * g.nta * 128);          // V D images
  add(4 * sizeof(CUtensorMap));                        // TMA maps
  return b;
}

size_t tc_tmap_bytes() { return 4 * sizeof(CUtensorMap); }

cudaError_t tc_carve_job(JobDev* d, const TcVData& v, char* base, size_t& off, size_t total, void* host_tmp,
                         cudaStream_t st) {
  const TcGeom& g = v.g;
  auto take = [&](size_t n) { void* p = base + off; off += (n + 255) / 256 * 256; return p; };
  int Tp, Hp, Wp;
  xc_dims(g, d->H, d->W, d->T, Tp, Hp, Wp);
  d->xTp = Tp; d->xHp = Hp; d->xWp = Wp;
  const int ncp = (g.split_ok ? 2 : 1) * g.ncopy;        // copies in Xc (hi, then lo)
  d->Xc = (__nv_bfloat16*)take((size_t)ncp * Tp * Hp * Wp * 2);
  d->G = (float*)take((size_t)d->m * 8);             // fixed-point Delta (see FX_ONE)
  d->B2img = (__nv_bfloat16*)take((size_t)g.ntt * g.nch_a * g.nta * 128);
  CUtensorMap* tm = (CUtensorMap*)take(4 * sizeof(CUtensorMap));
  if (off > total) return cudaErrorInvalidValue;
  EncodeTiledFn enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap hm[4];
  memset(hm, 0, sizeof hm);
  const cuuint32_t es[4] = {1, 1, 1, 1};
  // Xc as [c][wc][hp][tp*8]: dim0 = (tp, w%8) flattened, dim1 = hp, dim2 = wc, dim3 = c.
  // Map 0 loads all ncopy copies of a w-chunk; map 1 only the first k2 - 8 (the last
  // w-chunk of a kernel wider than 8).
  for (int mi = 0; mi < 2; ++mi) {
    const int nwcol = Wp / 8;
    const int nc = mi == 0 ? g.ncopy : std::max(1, g.k2 - 8 * (g.nwc - 1));
    cuuint64_t dims[4] = {(cuuint64_t)Tp * 8, (cuuint64_t)Hp, (cuuint64_t)nwcol, (cuuint64_t)ncp};
    cuuint64_t str[3] = {(cuuint64_t)Tp * 16, (cuuint64_t)Hp * Tp * 16, (cuuint64_t)nwcol * Hp * Tp * 16};
    cuuint32_t box[4] = {(cuuint32_t)(8 * g.k3), (cuuint32_t)g.Hh, 1, (cuuint32_t)nc};
    if (enc(&hm[mi], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, d->Xc, dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  // U as [t][h][w][kc]: map 2, box = one tile of 64 channels (64 x 8 w x 16 h), SW128
  // (row = voxel, 128 bytes); used by both tensor-core passes.
  {
    cuuint64_t dims[4] = {(cuuint64_t)g.kc, (cuuint64_t)d->W, (cuuint64_t)d->H, (cuuint64_t)d->T};
    cuuint64_t str[3] = {(cuuint64_t)g.kc * 2, (cuuint64_t)d->W * g.kc * 2, (cuuint64_t)d->H * d->W * g.kc * 2};
    cuuint32_t box[4] = {64, TW, TH, 1};
    if (enc(&hm[2], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, d->U, dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  memcpy(host_tmp, hm, sizeof hm);
  cudaError_t e = cudaMemcpyAsync(tm, host_tmp, sizeof hm, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  d->tmapX = &tm[0];
  d->tmapX2 = &tm[1];
  d->tmapU = &tm[2];
  d->tmapUlo = &tm[3];                     // encoded by tc_attach_ulo
  d->Ulo = nullptr;
  return cudaSuccess;
}

// Give a job the lo part of U (m x kc BF16 at `ulo`, zeroed by the caller when U's value
// is to be kept) and encode its TMA map into the job's fourth map slot.
cudaError_t tc_attach_ulo(JobDev* d, const TcVData& v, void* ulo, void* host_tmp, cudaStream_t st) {
  EncodeTiledFn enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const TcGeom& g = v.g;
  CUtensorMap m;
  const cuuint32_t es[4] = {1, 1, 1, 1};
  cuuint64_t dims[4] = {(cuuint64_t)g.kc, (cuuint64_t)d->W, (cuuint64_t)d->H, (cuuint64_t)d->T};
  cuuint64_t str[3] = {(cuuint64_t)g.kc * 2, (cuuint64_t)d->W * g.kc * 2, (cuuint64_t)d->H * d->W * g.kc * 2};
  cuuint32_t box[4] = {64, TW, TH, 1};
  if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, ulo, dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  memcpy(host_tmp, &m, sizeof m);
  cudaError_t e = cudaMemcpyAsync(const_cast<void*>(d->tmapUlo), host_tmp, sizeof m, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  d->Ulo = ulo;
  return cudaSuccess;
}

template <bool SPLIT>
static void launch_prepare_X_t(const Shared& sh, const TcGeom& g, int from_L, cudaStream_t st) {
  const dim3 grid(608, sh.njobs);
  switch (g.ncopy) {
    case 1: prepare_X_kernel<1, SPLIT><<<grid, 256, 0, st>>>(sh, g, from_L); break;
    case 2: prepare_X_kernel<2, SPLIT><<<grid, 256, 0, st>>>(sh, g, from_L); break;
    case 3: prepare_X_kernel<3, SPLIT><<<grid, 256, 0, st>>>(sh, g, from_L); break;
    case 4: prepare_X_kernel<4, SPLIT><<<grid, 256, 0, st>>>(sh, g, from_L); break;
    case 5: prepare_X_kernel<5, SPLIT><<<grid, 256, 0, st>>>(sh, g, from_L); break;
    case 6: prepare_X_kernel<6, SPLIT><<<grid, 256, 0, st>>>(sh, g, from_L); break;
    case 7: prepare_X_kernel<7, SPLIT><<<grid, 256, 0, st>>>(sh, g, from_L); break;
    default: prepare_X_kernel<8, SPLIT><<<grid, 256, 0, st>>>(sh, g, from_L); break;
  }
}

cudaError_t tc_launch_prepare_X(const Shared& sh, const TcVData& v, int from_L, cudaStream_t st, bool split) {
  if (split) launch_prepare_X_t<true>(sh, v.g, from_L, st);
  else launch_prepare_X_t<false>(sh, v.g, from_L, st);
  return cudaGetLastError();
}

// Per-device launch facts, set up once outside any stream capture: the SM count and the
// shared-memory opt-in of the tcgen05 kernels.
namespace {
constexpr int MAX_DEV = 64;
struct DevFacts {
  bool ready = false;
  int sms = 1;
};
DevFacts g_dev[MAX_DEV];
std::mutex g_dev_mu;

typedef void (*AdjKernel)(AdjArgs);
// compile-time kernel widths of the adjoint col2im (others take the per-element path)
template <bool DET, bool WIDE>
AdjKernel adj_kernel_for_t(const TcGeom& g) {
  if (g.rpg == 0) return adj_tc_kernel<0, DET, false>;
  switch (g.k2) {
    case 3: return adj_tc_kernel<3, DET, WIDE>;
    case 5: return adj_tc_kernel<5, DET, WIDE>;
    case 7: return adj_tc_kernel<7, DET, WIDE>;
    case 9: return adj_tc_kernel<9, DET, WIDE>;
    case 11: return adj_tc_kernel<11, DET, WIDE>;
    case 13: return adj_tc_kernel<13, DET, WIDE>;
    default: return adj_tc_kernel<0, DET, false>;
  }
}
AdjKernel adj_kernel_for(const TcGeom& g) {
  const bool wide = g.gpt == 8;
  if (g.det) return wide ? adj_kernel_for_t<true, true>(g) : adj_kernel_for_t<true, false>(g);
  return wide ? adj_kernel_for_t<false, true>(g) : adj_kernel_for_t<false, false>(g);
}

int dev_sms() {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= MAX_DEV) dev = 0;
  DevFacts& f = g_dev[dev];
  if (!f.ready) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    f.sms = n > 0 ? n : 1;
    cudaFuncSetAttribute(fwd_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    cudaFuncSetAttribute(fwd_tc_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    cudaFuncSetAttribute(fwd_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    for (AdjKernel kf : {adj_tc_kernel<0, true, false>, adj_tc_kernel<0, false, false>,
                         adj_tc_kernel<3, true, false>, adj_tc_kernel<5, true, false>, adj_tc_kernel<7, true, false>,
                         adj_tc_kernel<9, true, false>, adj_tc_kernel<3, false, false>, adj_tc_kernel<5, false, false>,
                         adj_tc_kernel<7, false, false>, adj_tc_kernel<9, false, false>, adj_tc_kernel<3, true, true>,
                         adj_tc_kernel<5, true, true>, adj_tc_kernel<7, true, true>, adj_tc_kernel<9, true, true>,
                         adj_tc_kernel<3, false, true>, adj_tc_kernel<5, false, true>, adj_tc_kernel<7, false, true>,
                         adj_tc_kernel<9, false, true>, adj_tc_kernel<11, true, false>, adj_tc_kernel<13, true, false>,
                         adj_tc_kernel<11, false, false>, adj_tc_kernel<13, false, false>, adj_tc_kernel<11, true, true>,
                         adj_tc_kernel<13, true, true>, adj_tc_kernel<11, false, true>, adj_tc_kernel<13, false, true>})
      cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    f.ready = true;
  }
  return f.sms;
}
}  // namespace

cudaError_t tc_launch_fwd(const Shared& sh, const TcVData& v, int mode, cudaStream_t st, bool split) {
  if (split && !v.g.split_ok) return cudaErrorInvalidValue;
  FwdArgs a;
  a.sh = sh;
  a.g = v.g;
  for (int i = 0; i < 64; ++i) { a.tab.boff[i] = v.boff[i]; a.tab.kstr[i] = v.kstr[i]; }
  a.tab.hp = v.g.R8 / 16;
  a.tab.reg = (v.g.R8 / 8) % 2 == 0 && (v.g.region_bytes % 16) == 0;
  for (int i = 0; a.tab.reg && i < v.g.nmma; ++i)
    if (v.kstr[i] != 128u || v.boff[i] != (uint32_t)((i / a.tab.hp) * v.g.region_bytes + (i % a.tab.hp) * 256))
      a.tab.reg = 0;
  a.mode = mode;
  const size_t smem = fwd_smem(v.g, split);
  const int per = tc_fwd_slots(sh, v, split);
  const int nct = split ? v.g.nct_s : v.g.nct;
  if (nct > 8) return cudaErrorInvalidValue;     // k <= 512 on this path: at most 4 tiles
  // CTAs per channel tile: equal shares, except that the split pass with deterministic
  // partials (rows per chunk, whatever the CTA count) gives each tile CTAs in proportion to
  // an estimate of its work: its MMAs (the same for every tile, weighted as two column
  // groups) plus its epilogue's 32-channel groups
  int cnt[8];
  for (int ct = 0; ct < nct; ++ct) cnt[ct] = per;
  if (split && v.g.det && nct > 1 && nct <= 8) {
    int wsum = 0, w[8];
    for (int ct = 0; ct < nct; ++ct) {
      w[ct] = 2 + std::min(4, (v.g.kc - 128 * ct + 31) / 32);
      wsum += w[ct];
    }
    const int total = per * nct, cap = std::max(1, sh.total_chunks);
    for (int ct = 0; ct < nct; ++ct) cnt[ct] = std::max(1, std::min(cap, total * w[ct] / wsum));
  }
  a.cta0[0] = 0;
  for (int ct = 0; ct < nct; ++ct) a.cta0[ct + 1] = a.cta0[ct] + cnt[ct];
  const int grid = a.cta0[nct];
  if (split) fwd_tc_kernel<true, false><<<grid, TC_THREADS, smem, st>>>(a);
  else if (v.g.ctw > 128) fwd_tc_kernel<false, true><<<grid, TC_THREADS, smem, st>>>(a);
  else fwd_tc_kernel<false, false><<<grid, TC_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

int tc_fwd_slots(const Shared& sh, const TcVData& v, bool split) {
  return std::max(1, std::min(dev_sms() / (split ? v.g.nct_s : v.g.nct), v.g.det ? sh.total_chunks : sh.total_tiles));
}

cudaError_t tc_launch_build_B2(const Shared& sh, const TcVData& v, cudaStream_t st) {
  build_B2_kernel<<<dim3(sh.njobs, v.g.ntt * v.g.nch_a), 256, 0, st>>>(sh, v.g);
  return cudaGetLastError();
}

cudaError_t tc_launch_adj(const Shared& sh, const TcVData& v, cudaStream_t st) {
  AdjArgs a;
  a.sh = sh;
  a.g = v.g;
  const int per = std::max(1, std::min(dev_sms() / v.g.ntt, sh.total_tiles));
  adj_kernel_for(v.g)<<<per * v.g.ntt, TC_THREADS, adj_smem(v.g), st>>>(a);
  return cudaGetLastError();
}

cudaError_t tc_bounded_wait_check(uint64_t limit_ns, int* dstatus, cudaStream_t st) {
  bounded_wait_check_kernel<<<1, 32, 0, st>>>(limit_ns, dstatus);
  return cudaGetLastError();
}

cudaError_t tc_launch_gather(const Shared& sh, const TcVData& v, cudaStream_t st) {
  if (v.g.det) gather_tc_kernel<true><<<dim3(sh.max_vblk, sh.njobs), 256, 0, st>>>(sh);
  else gather_tc_kernel<false><<<dim3(sh.max_vblk, sh.njobs), 256, 0, st>>>(sh);
  return cudaGetLastError();
}

}  // namespace icnnm
