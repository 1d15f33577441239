// Host interface of the BF16 tcgen05 path (k_tc.cu).
#pragma once
#include <string>
#include "icnnm_internal.h"

namespace icnnm {

// Geometry of the tensor-core passes, fixed by the kernel dims.
struct TcGeom {
  int k1, k2, k3, k, kc;
  // forward pass E = P(X) V (M = 128 voxels, N = 128 channels, K = taps)
  int R, R8;        // taps per w-run (k1*k3) and the run padded to a multiple of 16 rows
  int ngrp, nmma;   // K-groups of 8 taps, MMAs of K = 16
  int kpad;         // nmma * 16
  int nch_f;        // 64-wide SW128 chunks of the forward A image
  int ncopy, nwc;   // w-shifted copies of the operand (min(k2, 8)) and 8-wide w-chunks
  int Hh;           // halo height TH + k1 - 1
  int region_bytes; // one copy's halo: Hh * k3 rows of 16 bytes
  int stage_bytes;  // one halo stage (the k2 copies used + 16 zero rows), 1024-aligned
  int ctw;          // channel-tile width of the plain forward: 128, or kc rounded up to 32
                    // (128 < that <= 256) when one tile of all channels fits shared memory
  int nct;          // channel tiles of the plain forward (of ctw channels)
  int nct_s;        // channel tiles of the split forward (of 128 channels)
  // adjoint pass G = U (D V^T) (M = 128 voxels, N = 128 taps, K = channels)
  int gpt;          // 32-column groups per adjoint tap tile: 4 (N = 128) or 8 (N = 256,
                    // when the wider tile's V D image fits in shared memory)
  int nta;          // tap-tile width 32 * gpt: the adjoint MMA's N
  int ntt;          // tap tiles (gpt groups of rpg tap rows each)
  int kcp;          // channels rounded up to 64
  int nch_a;        // 64-wide SW128 chunks of the adjoint A image
  int Hb, Wb, HB;   // col2im halo of a tile: Hb = TH + k1 - 1, Wb = TW + k2 - 1, HB = Hb*Wb*nsl
  int nsl;          // frames of the halo one tap tile reaches (its partial keeps only those)
  int slo[16];      // first frame (st) reached by each tap tile
  int rpg;          // adjoint: whole tap rows (k2 taps) per 32-column group, spread evenly over
                    // the groups (0: taps in order)
  int nus;          // forward U tile stages in shared memory (1 or 2)
  // split forward (ICNNM_BF16X3 and the finish of BF16 jobs): the operand and V^T as
  // hi + lo BF16 pairs, three products per tile, U stored as a hi + lo pair
  int det;          // deterministic reductions (TcTiles::det)
  int split_ok;     // 1: the split forward fits in shared memory for these kernel dims
  int lo_off;       // byte offset of the lo copies in a split halo stage (after hi + 16 zero rows)
  int stage_bytes_s;// one split halo stage: hi copies, 16 zero rows, lo copies, 16 zero rows
  int nus_s;        // U tile stages (each a hi and a lo tile) of the split forward
  int pitch, HBp;   // shared-memory row pitch of the halo buffers (an odd multiple of 8,
                    // >= Wb, so 4 rows x 8 voxels hit 32 banks) and k3*Hb*pitch
};

// Per-V device data of the tensor-core path.
struct TcVData {
  TcGeom g{};
  __nv_bfloat16* VtImg = nullptr;   // plain forward: nct B images of V^T (ctw channels each,
                                    // nch_f chunks of ctw x 128 bytes)
  __nv_bfloat16* VtImgS = nullptr;  // split forward (when g.split_ok): nct_s images of V^T (128
                                    // channels each), then nct_s of V^T - bf16(V^T) (the lo part)
  uint32_t boff[64];                // forward: byte offset of each MMA's first K-group
  uint32_t kstr[64];                // forward: byte distance to its second K-group
};

// Tile choices of the tensor-core passes (upper bounds; a choice that does not fit in
// shared memory falls back to the narrower one): adjoint tap tiles of 32 * gpt_max columns
// (4 or 8), forward channel tiles of up to ctw_max channels (128 or 256), forward U stages
// up to nus_max (1 or 2). The defaults are the narrow tiles; the autotuner (or a table of
// its results) picks wider ones per kernel size.
struct TcTiles {
  int gpt_max = 4;
  int ctw_max = 128;
  int nus_max = 2;
  int det = 1;      // 1: deterministic reductions (fixed-point col2im, forward partials per
                    // fixed chunk of a job's tiles); 0: float atomics, strided tiles
};

bool tc_supported(int k1, int k2, int k3, std::string* why);
// Geometry of the tensor-core passes for these kernel dims (kc: the channel stride).
TcGeom tc_geom(int k1, int k2, int k3, int kc, const TcTiles& tiles = TcTiles());
cudaError_t tc_build_vdata(const double* V64, int k1, int k2, int k3, int kc, TcVData* out,
                           const TcTiles& tiles = TcTiles());
void tc_free_vdata(TcVData* v);
size_t tc_job_extra_bytes(int H, int W, int T, const TcGeom& g);
// Carve the tensor-core buffers of a job from its allocation and encode its TMA maps;
// the maps are written into host_tmp (tc_tmap_bytes(), pinned) and copied to the device
// on `st` (the caller keeps host_tmp until that copy has completed).
size_t tc_tmap_bytes();
cudaError_t tc_carve_job(JobDev* d, const TcVData& v, char* base, size_t& off, size_t total, void* host_tmp,
                         cudaStream_t st);
int tc_nrp(int k);
// split: also write the lo copies (the operand of the split forward)
cudaError_t tc_launch_prepare_X(const Shared& sh, const TcVData& v, int from_L, cudaStream_t st, bool split = false);
// split: the three-product forward with U as a hi + lo pair (needs v.g.split_ok and every
// job's Ulo attached)
cudaError_t tc_launch_fwd(const Shared& sh, const TcVData& v, int mode, cudaStream_t st, bool split = false);
cudaError_t tc_attach_ulo(JobDev* d, const TcVData& v, void* ulo, void* host_tmp, cudaStream_t st);
// CTA slots per channel tile of the forward launch: the update modes write one
// column-partial row group per (slot, job), min(slots, ntiles) groups per job.
int tc_fwd_slots(const Shared& sh, const TcVData& v, bool split = false);
// B = V D image per job (bf16, SW128), then the adjoint GEMM + col2im into halo partials.
cudaError_t tc_launch_build_B2(const Shared& sh, const TcVData& v, cudaStream_t st);
cudaError_t tc_launch_adj(const Shared& sh, const TcVData& v, cudaStream_t st);
cudaError_t tc_launch_gather(const Shared& sh, const TcVData& v, cudaStream_t st);
// A bounded mbarrier wait that nothing completes, given up after limit_ns: *dstatus = 1.
cudaError_t tc_bounded_wait_check(uint64_t limit_ns, int* dstatus, cudaStream_t st);

}  // namespace icnnm
