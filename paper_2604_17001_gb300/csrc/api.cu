// C ABI of libicnnm (include/icnnm.h): contexts, validation, the job engine that steps
// any set of completion jobs sharing (kernel dims, V, precision) together, learn_V,
// the blocking solves, and the continuous-batching serving thread.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/icnnm.h"
#include "icnnm_internal.h"
#include "tc_api.h"

using namespace icnnm;

namespace {

struct CudaFail {
  cudaError_t e;
  const char* what;
};

#define CK(x)                                      \
  do {                                             \
    cudaError_t e__ = (x);                         \
    if (e__ != cudaSuccess) throw CudaFail{e__, #x}; \
  } while (0)

struct StatusFail {
  icnnm_status st;
  std::string msg;
};

[[noreturn]] void fail(icnnm_status st, const std::string& msg) { throw StatusFail{st, msg}; }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int round_up(int x, int a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------------
// Shared per-V device data
// ---------------------------------------------------------------------------------
struct VData {
  int k1, k2, k3, k, kc;
  std::vector<double> V64;   // column-major k x k
  float* dVf = nullptr;      // [k][kc]
  double* dV64 = nullptr;    // V64 on the device (column norms through the Gram)
  TcVData tc;                // BF16 images (tc_api.h)
  std::atomic<bool> tc_ready{false};
};

// ---------------------------------------------------------------------------------
// Jobs
// ---------------------------------------------------------------------------------
enum Phase { QUEUED = 0, ADMITTED, RUNNING, DONE, FAILED, CANCELED };

struct Job {
  uint64_t id = 0;
  int H = 0, W = 0, T = 0;
  long long m = 0;
  icnnm_params p{};
  VData* vd = nullptr;
  void* dstage = nullptr;       // serving: the inputs staged on the device at submit (M, then mask)
  const float* srcM = nullptr;  // caller's buffers (blocking solves)
  const uint8_t* srcmask = nullptr;
  bool src_dev = false;
  void* block = nullptr;        // one device allocation for all of the job's state
  size_t bytes = 0;
  int run_prec = 0;             // arithmetic of the next iterations (BF16 jobs with a tolerance
                                //   finish in BF16X3 where it is built for their kernel, else FP32)
  void* block2 = nullptr;       // FP32 finish: widened U and the FP32 adjoint workspace
  size_t bytes2 = 0;
  double last_resid = INFINITY; // residual at the previous check (BF16 stall detection)
  JobDev dev{};
  Phase phase = QUEUED;
  icnnm_status st = ICNNM_OK;
  std::string err;
  int iters = 0;
  bool converged = false;
  double resid = NAN;
  icnnm_stats stats{};
  float* dres = nullptr;        // serving: the result L on the device until collected
  std::chrono::steady_clock::time_point t_admit;
  std::chrono::steady_clock::time_point t_submit;
  std::atomic<bool> cancel{false};
};

size_t job_bytes(int H, int W, int T, int k, int kc, int prec, int nrp, const TcGeom* tg) {
  const long long m = (long long)H * W * T;
  const int ntiles = ((H + TH - 1) / TH) * ((W + TW - 1) / TW) * T;
  size_t b = 0;
  auto add = [&](size_t n) { b += (n + 255) / 256 * 256; };
  add(sizeof(JobScal));
  add(m * 4);            // M
  add(m);                // mask
  add(m * 4);            // L
  add(m * 4);            // X
  add((size_t)ntiles * PROW * kc * 4);   // part
  add((size_t)ntiles * nrp * 4);  // rpart
  add((size_t)ntiles * 4);        // lpart
  add((size_t)NSEG * kc * 8);     // colseg
  add(kc * 4);           // s
  add(kc * 4);           // D
  if (prec == ICNNM_FP32) {
    add(m * kc * 4);     // U
    add((size_t)k * m * 4);  // G^T
  } else {
    add(m * kc * 2);     // U (bf16)
    if (prec == ICNNM_BF16X3) add(m * kc * 2);   // the lo part of U
    b += tc_job_extra_bytes(H, W, T, *tg);
  }
  return b;
}

}  // namespace

// ---------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------
constexpr int NPASS = 6;   // profiled passes (see icnnm_profile_read)

struct icnnm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  // device bytes of job state in use: charged and released under mu; the serving thread's
  // admission test also reads it under qmu (advisory; alloc_job checks again under mu)
  std::atomic<size_t> used{0};
  std::recursive_mutex mu;         // serialises device work of API calls and the server
  std::mutex err_mu;
  std::string last_err;
  std::map<std::string, std::unique_ptr<VData>> vcache;   // inserted under mu and vmu
  std::mutex vmu;                  // lookups of vcache without mu (the submitting side)
  std::map<std::string, TcTiles> tiles;   // tile configuration per kernel dims ("k1_k2_k3")
  int det = 1;                     // deterministic reductions of the BF16 path
  // serving
  std::mutex qmu;
  std::condition_variable qcv;
  std::deque<std::shared_ptr<Job>> queue;            // submitted, not admitted
  std::map<uint64_t, std::shared_ptr<Job>> jobs;     // all known (until collected)
  std::vector<std::shared_ptr<Job>> active;          // admitted (server thread only)
  std::thread server;
  bool stop = false;
  uint64_t next_id = 1;
  // diagnostics
  bool prof = false;
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  std::vector<std::pair<int, size_t>> pending;   // (pass, index of the start event)
  // passes: 0 forward (BF16), 1 adjoint, 2 gather, 3 other, 4 forward (BF16X3),
  // 5 forward (FP32 lists); index NPASS counts every pass
  double pass_ms[NPASS] = {};
  long long pass_n[NPASS + 1] = {};
  long long pass_vox[NPASS + 1] = {};
  size_t hook_idx = 0;                           // start event of the open hook pass
  // engine scratch
  // device job tables: slot 0 for the main list, slot 1 for a list stepped beside it
  // (the BF16 jobs finishing in FP32), so that both can be live at once. Uploads are
  // stream-ordered, so a slot may be rewritten after the kernels that read it are enqueued.
  JobDev* dlist[2] = {nullptr, nullptr};
  int* dtile0[2] = {nullptr, nullptr};
  int list_cap[2] = {0, 0};
  // device memory of jobs, job tables and scratch: a pool of this context with
  // stream-ordered allocation and release (no device-wide synchronisation)
  cudaMemPool_t pool = nullptr;
  // validation and staging of served inputs, on the submitting thread's side
  cudaStream_t sub_stream = nullptr;
  std::mutex submu;
  // pinned host staging of host-to-device copies (job tables, tensor maps) and of the
  // scalars read back per step; an entry is reused once its last copy has completed
  struct Pinned {
    char* p = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
  };
  std::vector<Pinned> ring;
  size_t ring_next = 0;
  JobScal* hscal = nullptr;      // pinned, hscal_cap entries
  int hscal_cap = 0;
  // scratch of the Gram route to column norms (autocorrelation partials, k x k Gram)
  double* gscr = nullptr;
  size_t gscr_bytes = 0;
};

namespace {

void set_err(icnnm_ctx* c, const std::string& s) {
  std::lock_guard<std::mutex> g(c->err_mu);
  c->last_err = s;
}

// Stream-ordered device memory from the context's pool.
void* dalloc_async(icnnm_ctx* c, size_t bytes, cudaStream_t st) {
  void* p = nullptr;
  CK(cudaMallocFromPoolAsync(&p, std::max<size_t>(bytes, 256), c->pool, st));
  return p;
}
void dfree_async(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// A pinned host buffer of at least n bytes for one host-to-device copy on c->stream:
// the caller fills it, enqueues the copy and calls pinned_done. The ring entry is reused
// only after that copy has completed (usually long before), so no stream sync is needed.
icnnm_ctx::Pinned& pinned_take(icnnm_ctx* c, size_t n) {
  if (c->ring.empty()) c->ring.resize(32);
  icnnm_ctx::Pinned& e = c->ring[c->ring_next++ % c->ring.size()];
  if (e.pending) {
    CK(cudaEventSynchronize(e.ev));
    e.pending = false;
  }
  if (!e.ev) CK(cudaEventCreateWithFlags(&e.ev, cudaEventDisableTiming));
  if (e.cap < n) {
    if (e.p) CK(cudaFreeHost(e.p));
    e.p = nullptr;
    e.cap = 0;
    const size_t cap = std::max<size_t>(n, 64 << 10);
    CK(cudaHostAlloc((void**)&e.p, cap, cudaHostAllocDefault));
    e.cap = cap;
  }
  return e;
}
void pinned_done(icnnm_ctx* c, icnnm_ctx::Pinned& e) {
  CK(cudaEventRecord(e.ev, c->stream));
  e.pending = true;
}
// Host-to-device copy of n bytes through the pinned ring (stream-ordered on c->stream).
void h2d_staged(icnnm_ctx* c, void* dst, const void* src, size_t n) {
  icnnm_ctx::Pinned& e = pinned_take(c, n);
  memcpy(e.p, src, n);
  CK(cudaMemcpyAsync(dst, e.p, n, cudaMemcpyHostToDevice, c->stream));
  pinned_done(c, e);
}

// Diagnostics: bracket a pass with events when profiling, and count launches.
cudaEvent_t pool_event(icnnm_ctx* c) {
  if (c->evnext == c->evpool.size()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c->evpool.push_back(e);
  }
  return c->evpool[c->evnext++];
}

struct PassScope {
  icnnm_ctx* c;
  int pass;
  size_t idx = 0;
  PassScope(icnnm_ctx* c_, int pass_, int nkernels, long long nvox = 0) : c(c_), pass(pass_) {
    c->pass_n[pass] += nkernels;
    c->pass_n[NPASS] += nkernels;
    c->pass_vox[pass] += nvox;
    c->pass_vox[NPASS] += nvox;
    if (c->prof) {
      idx = c->evnext;
      CK(cudaEventRecord(pool_event(c), c->stream));
    }
  }
  ~PassScope() noexcept(false) {
    if (c->prof) {
      CK(cudaEventRecord(pool_event(c), c->stream));
      c->pending.emplace_back(pass, idx);
    }
  }
};

// After a stream synchronisation: fold the recorded pass times into the totals.
void flush_prof(icnnm_ctx* c) {
  for (auto& pr : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->evpool[pr.second], c->evpool[pr.second + 1]) == cudaSuccess)
      c->pass_ms[pr.first] += ms;
  }
  c->pending.clear();
  c->evnext = 0;
}

icnnm_status report(icnnm_ctx* c, const StatusFail& f) {
  set_err(c, f.msg);
  return f.st;
}
icnnm_status report(icnnm_ctx* c, const CudaFail& f) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %d (%s) at %s", (int)f.e, cudaGetErrorString(f.e), f.what);
  set_err(c, buf);
  return ICNNM_ECUDA;
}

// Validation ------------------------------------------------------------------------
void validate_shape(const icnnm_shape* s, int& H, int& W, int& T, int& k1, int& k2, int& k3) {
  if (!s) fail(ICNNM_EINVAL, "shape is NULL");
  if (s->ndim != 2 && s->ndim != 3) fail(ICNNM_EINVAL, "ndim must be 2 or 3");
  H = (int)s->dims[0]; W = (int)s->dims[1]; T = s->ndim == 3 ? (int)s->dims[2] : 1;
  k1 = (int)s->kdims[0]; k2 = (int)s->kdims[1]; k3 = s->ndim == 3 ? (int)s->kdims[2] : 1;
  if (s->ndim == 2 && ((s->dims[2] != 1 && s->dims[2] != 0) || (s->kdims[2] != 1 && s->kdims[2] != 0)))
    fail(ICNNM_EINVAL, "an image (ndim 2) has T = 1 and k3 = 1");
  if (H < 1 || W < 1 || T < 1 || k1 < 1 || k2 < 1 || k3 < 1) fail(ICNNM_EINVAL, "dims and kdims must be >= 1");
  if (s->dims[0] > (1 << 20) || s->dims[1] > (1 << 20) || s->dims[2] > (1 << 20))
    fail(ICNNM_EINVAL, "dims too large");
  if (H < k1 || W < k2 || T < k3) fail(ICNNM_EINVAL, "every dim must be at least the kernel's (Sec. II-B)");
  if ((long long)k1 * k2 * k3 > 1024) fail(ICNNM_EINVAL, "k = k1*k2*k3 must be <= 1024");
}

void validate_params(const icnnm_params& p) {
  if (!(p.lambda > 0)) fail(ICNNM_EINVAL, "lambda must be > 0 (INFINITY for the exact projection)");
  if (!(p.rho >= 1.0) || !isfinite(p.rho)) fail(ICNNM_EINVAL, "rho must be finite and >= 1");
  if (!(p.theta_max > 0)) fail(ICNNM_EINVAL, "theta_max must be > 0");
  if (p.max_iters < 1) fail(ICNNM_EINVAL, "max_iters must be >= 1");
  if (!(p.tol >= 0) || !isfinite(p.tol)) fail(ICNNM_EINVAL, "tol must be finite and >= 0");
  if (p.check_every < 1) fail(ICNNM_EINVAL, "check_every must be >= 1");
  if (p.prec != ICNNM_FP32 && p.prec != ICNNM_BF16 && p.prec != ICNNM_BF16X3) fail(ICNNM_EINVAL, "unknown precision");
  if (!isfinite(p.theta0) && p.theta0 > 0) fail(ICNNM_EINVAL, "theta0 must be finite");
}

std::string v_key(const double* V, int k1, int k2, int k3) {
  // FNV-1a over the bytes of V plus the kernel dims.
  uint64_t h = 1469598103934665603ull;
  const unsigned char* b = reinterpret_cast<const unsigned char*>(V);
  const size_t n = sizeof(double) * (size_t)k1 * k2 * k3 * k1 * k2 * k3;
  for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  char buf[96];
  snprintf(buf, sizeof buf, "%d_%d_%d_%016llx", k1, k2, k3, (unsigned long long)h);
  return buf;
}

std::vector<double> read_V(const double* V, int k) {
  if (!V) fail(ICNNM_EINVAL, "V is NULL");
  std::vector<double> hv((size_t)k * k);
  if (is_device_ptr(V)) CK(cudaMemcpy(hv.data(), V, hv.size() * 8, cudaMemcpyDeviceToHost));
  else memcpy(hv.data(), V, hv.size() * 8);
  return hv;
}

// The cached per-V data if it exists and is ready for `prec` (no device work, no engine
// mutex: the submitting side must not wait for a serving step), else nullptr.
VData* find_vdata_ready(icnnm_ctx* c, const std::string& key, int prec) {
  std::lock_guard<std::mutex> g(c->vmu);
  auto it = c->vcache.find(key);
  if (it == c->vcache.end()) return nullptr;
  VData* vd = it->second.get();
  if (prec != ICNNM_FP32 && !vd->tc_ready) return nullptr;
  if (prec == ICNNM_BF16X3 && !vd->tc.g.split_ok) return nullptr;
  return vd;
}

VData* get_vdata(icnnm_ctx* c, const double* V, int k1, int k2, int k3, int prec) {
  const int k = k1 * k2 * k3;
  std::vector<double> hv = read_V(V, k);
  const std::string key = v_key(hv.data(), k1, k2, k3);
  std::map<std::string, std::unique_ptr<VData>>::iterator it;
  {
    std::lock_guard<std::mutex> g(c->vmu);
    it = c->vcache.find(key);
  }
  VData* vd;
  if (it == c->vcache.end()) {
    for (double x : hv)
      if (!isfinite(x)) fail(ICNNM_EINVAL, "V has a non-finite entry");
    // orthonormality: max |V^T V - I| <= 1e-6
    double worst = 0.0;
    for (int i = 0; i < k; ++i)
      for (int j = i; j < k; ++j) {
        double d = 0.0;
        const double* a = hv.data() + (size_t)i * k;
        const double* b = hv.data() + (size_t)j * k;
        for (int s = 0; s < k; ++s) d += a[s] * b[s];
        worst = std::max(worst, fabs(d - (i == j ? 1.0 : 0.0)));
      }
    if (worst > 1e-6) fail(ICNNM_EINVAL, "V is not orthonormal to 1e-6");
    auto nv = std::make_unique<VData>();
    nv->k1 = k1; nv->k2 = k2; nv->k3 = k3; nv->k = k; nv->kc = round_up(k, 16);
    nv->V64 = std::move(hv);
    std::vector<float> vf((size_t)k * nv->kc, 0.f);
    for (int s = 0; s < k; ++s)
      for (int ch = 0; ch < k; ++ch) vf[(size_t)s * nv->kc + ch] = (float)nv->V64[(size_t)ch * k + s];
    CK(cudaMalloc(&nv->dVf, vf.size() * 4));
    CK(cudaMemcpy(nv->dVf, vf.data(), vf.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&nv->dV64, nv->V64.size() * 8));
    CK(cudaMemcpy(nv->dV64, nv->V64.data(), nv->V64.size() * 8, cudaMemcpyHostToDevice));
    vd = nv.get();
    std::lock_guard<std::mutex> g(c->vmu);
    c->vcache[key] = std::move(nv);
  } else {
    vd = it->second.get();
  }
  return vd;
}

std::string kdims_key(int k1, int k2, int k3) {
  char buf[48];
  snprintf(buf, sizeof buf, "%d_%d_%d", k1, k2, k3);
  return buf;
}

TcTiles tiles_for(icnnm_ctx* c, int k1, int k2, int k3) {
  auto it = c->tiles.find(kdims_key(k1, k2, k3));
  TcTiles t = it == c->tiles.end() ? TcTiles() : it->second;
  t.det = c->det;
  return t;
}

void ensure_tc(icnnm_ctx* c, VData* vd, int prec) {
  const int k1 = vd->k1, k2 = vd->k2, k3 = vd->k3;
  if (prec != ICNNM_FP32 && !vd->tc_ready) {
    std::string why;
    if (!tc_supported(k1, k2, k3, &why)) fail(ICNNM_EUNSUPPORTED, "BF16 path: " + why);
    CK(tc_build_vdata(vd->V64.data(), k1, k2, k3, vd->kc, &vd->tc, tiles_for(c, k1, k2, k3)));
    vd->tc_ready = true;
  }
  if (prec == ICNNM_BF16X3 && !vd->tc.g.split_ok)
    fail(ICNNM_EUNSUPPORTED, "BF16X3: the split forward pass does not fit in shared memory for this kernel");
}

// Engine ---------------------------------------------------------------------------
void alloc_job(icnnm_ctx* c, Job& j) {
  VData* vd = j.vd;
  const int k = vd->k, kc = vd->kc;
  const int nrp = std::max(fwd_fp32_nrp(k), tc_nrp(k));
  j.bytes = job_bytes(j.H, j.W, j.T, k, kc, j.p.prec, nrp, &vd->tc.g);
  j.run_prec = j.p.prec;
  if (c->used + j.bytes > c->budget) fail(ICNNM_ENOMEM, "job state exceeds the HBM budget");
  j.block = dalloc_async(c, j.bytes, c->stream);
  c->used += j.bytes;
  char* b = static_cast<char*>(j.block);
  size_t off = 0;
  auto take = [&](size_t n) { void* p = b + off; off += (n + 255) / 256 * 256; return p; };
  const long long m = j.m;
  JobDev& d = j.dev;
  d = JobDev{};
  d.H = j.H; d.W = j.W; d.T = j.T;
  d.nth = (j.H + TH - 1) / TH; d.ntw = (j.W + TW - 1) / TW;
  d.ntiles = d.nth * d.ntw * j.T;
  d.fchunk = fwd_chunk_of(d.ntiles);
  d.m = m;
  d.lam = j.p.lambda; d.rho = j.p.rho; d.theta_max = j.p.theta_max;
  d.sc = (JobScal*)take(sizeof(JobScal));
  d.M = (const float*)take(m * 4);
  d.mask = (const uint8_t*)take(m);
  d.L = (float*)take(m * 4);
  d.X = (float*)take(m * 4);
  d.part = (float*)take((size_t)d.ntiles * PROW * kc * 4);
  d.rpart = (float*)take((size_t)d.ntiles * nrp * 4);
  d.lpart = (float*)take((size_t)d.ntiles * 4);
  d.nlp = j.p.prec == ICNNM_FP32 ? d.ntiles : (int)((m + 1023) / 1024);   // gather partials
  d.colseg = (double*)take((size_t)NSEG * kc * 8);
  d.s = (float*)take(kc * 4);
  d.D = (float*)take(kc * 4);
  if (j.p.prec == ICNNM_FP32) {
    d.U = take(m * kc * 4);
    d.G = (float*)take((size_t)k * m * 4);
  } else {
    d.U = take(m * kc * 2);
    void* ulo = j.p.prec == ICNNM_BF16X3 ? take(m * kc * 2) : nullptr;
    icnnm_ctx::Pinned& e = pinned_take(c, tc_tmap_bytes());
    CK(tc_carve_job(&d, vd->tc, b, off, j.bytes, e.p, c->stream));
    pinned_done(c, e);
    if (ulo) {
      icnnm_ctx::Pinned& e2 = pinned_take(c, tc_tmap_bytes());
      CK(tc_attach_ulo(&d, vd->tc, ulo, e2.p, c->stream));
      pinned_done(c, e2);
      CK(cudaMemsetAsync(ulo, 0, m * kc * 2, c->stream));
    }
  }
  CK(cudaMemsetAsync(d.sc, 0, sizeof(JobScal), c->stream));
  CK(cudaMemsetAsync(d.U, 0, (size_t)m * kc * (j.p.prec == ICNNM_FP32 ? 4 : 2), c->stream));
  CK(cudaMemsetAsync(d.part, 0, (size_t)d.ntiles * PROW * kc * 4, c->stream));
  CK(cudaMemsetAsync(d.rpart, 0, (size_t)d.ntiles * nrp * 4, c->stream));
  if (j.p.prec != ICNNM_FP32) CK(cudaMemsetAsync(d.G, 0, (size_t)m * 8, c->stream));   // fixed-point Delta
  // inputs: staged on the device at submit (serving), else the caller's buffers
  if (j.dstage) {
    CK(cudaMemcpyAsync((void*)d.M, j.dstage, m * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync((void*)d.mask, static_cast<char*>(j.dstage) + m * 4, m, cudaMemcpyDeviceToDevice, c->stream));
    dfree_async(j.dstage, c->stream);
    j.dstage = nullptr;
  } else {
    CK(cudaMemcpyAsync((void*)d.M, j.srcM, m * 4, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync((void*)d.mask, j.srcmask, m, cudaMemcpyDefault, c->stream));
  }
}

// Stream-ordered release of the job's device state (and of its staged inputs and
// result, if any) on c->stream.
void free_job(icnnm_ctx* c, Job& j) {
  if (j.block) {
    dfree_async(j.block, c->stream);
    c->used -= j.bytes;
    j.block = nullptr;
  }
  if (j.block2) {
    dfree_async(j.block2, c->stream);
    c->used -= j.bytes2;
    j.block2 = nullptr;
  }
  if (j.dstage) {
    dfree_async(j.dstage, c->stream);
    j.dstage = nullptr;
  }
}

// Finish of a BF16 job with a residual tolerance. U is stored in BF16 and the forward
// pass rounds its operands to BF16, so the BF16 residual ||Z - A_k(L)V|| carries a rounding
// floor near 1e-3 relative; a tolerance at or below it cannot be certified in BF16. When
// the BF16 residual is within 4x the tolerance or has stopped falling (less than 10%
// between checks), the job continues in BF16X3 where that path is built for its kernel
// (the forward with hi + lo operand pairs and U kept as a hi + lo pair: only the lo half of
// U is added, zero, so the state the next iteration reads is unchanged), else in FP32 (U
// widened exactly, the FP32 adjoint workspace added). Returns false (the job stays in BF16)
// when the extra state does not fit the budget.
bool bf16_should_finish(const Job& j) {
  return j.run_prec == ICNNM_BF16 && j.p.tol > 0 && (j.resid <= 4 * j.p.tol || j.resid > 0.9 * j.last_resid);
}

bool switch_to_finish(icnnm_ctx* c, Job& j) {
  const size_t m = (size_t)j.m, kc = (size_t)j.vd->kc, k = (size_t)j.vd->k;
  const bool split = j.vd->tc.g.split_ok;
  const size_t ub = (m * kc * (split ? 2 : 4) + 255) / 256 * 256;
  const size_t need = split ? ub : ub + k * m * 4;
  if (c->used + need > c->budget) return false;
  void* b = nullptr;
  if (cudaMallocFromPoolAsync(&b, need, c->pool, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->used += need;
  j.block2 = b;
  j.bytes2 = need;
  // the finishing kernel writes its residual partials into its own slots of rpart, which
  // need not be the slots the BF16 kernel wrote: clear them all so that no stale BF16
  // partial is summed into a later residual
  const int nrp = std::max(fwd_fp32_nrp((int)k), tc_nrp((int)k));
  CK(cudaMemsetAsync(j.dev.rpart, 0, (size_t)j.dev.ntiles * nrp * 4, c->stream));
  if (split) {
    CK(cudaMemsetAsync(b, 0, m * kc * 2, c->stream));
    icnnm_ctx::Pinned& e = pinned_take(c, tc_tmap_bytes());
    CK(tc_attach_ulo(&j.dev, j.vd->tc, b, e.p, c->stream));
    pinned_done(c, e);
    j.run_prec = ICNNM_BF16X3;
    return true;
  }
  float* U32 = static_cast<float*>(b);
  CK(launch_widen_bf16(static_cast<const __nv_bfloat16*>(j.dev.U), U32, (long long)(m * kc), c->stream));
  j.dev.U = U32;
  j.dev.G = reinterpret_cast<float*>(static_cast<char*>(b) + ub);
  j.dev.nlp = j.dev.ntiles;            // the FP32 gather writes one partial per tile
  j.run_prec = ICNNM_FP32;
  return true;
}

struct List {
  Shared sh{};
};

// Upload a launch list of jobs (all sharing vd and precision) and fill the Shared view.
Shared upload_list(icnnm_ctx* c, const std::vector<Job*>& js, int slot = 0) {
  const int n = (int)js.size();
  if (n > c->list_cap[slot]) {
    // stream-ordered: the old tables are released after the kernels that read them
    dfree_async(c->dlist[slot], c->stream);
    dfree_async(c->dtile0[slot], c->stream);
    c->dlist[slot] = nullptr;
    c->dtile0[slot] = nullptr;
    const int cap = std::max(n, 2 * c->list_cap[slot]);
    c->dlist[slot] = (JobDev*)dalloc_async(c, sizeof(JobDev) * std::max(cap, 64), c->stream);
    c->dtile0[slot] = (int*)dalloc_async(c, sizeof(int) * 2 * (std::max(cap, 64) + 1), c->stream);
    c->list_cap[slot] = std::max(cap, 64);
  }
  // one pinned staging buffer: the job table, then the tile and the chunk prefix sums
  const size_t tb = sizeof(JobDev) * n, pb = sizeof(int) * 2 * (n + 1);
  icnnm_ctx::Pinned& e = pinned_take(c, tb + pb);
  JobDev* hd = reinterpret_cast<JobDev*>(e.p);
  int* t0 = reinterpret_cast<int*>(e.p + tb);
  int* c0 = t0 + (n + 1);
  t0[0] = 0;
  c0[0] = 0;
  for (int i = 0; i < n; ++i) {
    hd[i] = js[i]->dev;
    t0[i + 1] = t0[i] + js[i]->dev.ntiles;
    c0[i + 1] = c0[i] + (js[i]->dev.ntiles + js[i]->dev.fchunk - 1) / js[i]->dev.fchunk;
  }
  CK(cudaMemcpyAsync(c->dlist[slot], hd, tb, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->dtile0[slot], t0, pb, cudaMemcpyHostToDevice, c->stream));
  pinned_done(c, e);
  const VData* vd = js[0]->vd;
  Shared sh{};
  sh.k1 = vd->k1; sh.k2 = vd->k2; sh.k3 = vd->k3; sh.k = vd->k; sh.kc = vd->kc;
  sh.nrp = js[0]->run_prec == ICNNM_FP32 ? fwd_fp32_nrp(vd->k) : tc_nrp(vd->k);
  sh.Vf = vd->dVf;
  sh.VtImg = vd->tc_ready ? vd->tc.VtImg : nullptr;
  sh.VtImgS = vd->tc_ready ? vd->tc.VtImgS : nullptr;
  sh.njobs = n;
  sh.jobs = c->dlist[slot];
  sh.job_tile0 = c->dtile0[slot];
  sh.job_chunk0 = c->dtile0[slot] + (n + 1);
  sh.total_tiles = t0[n];
  sh.total_chunks = c0[n];
  sh.max_vblk = 1;
  sh.nvox = 0;
  for (int i = 0; i < n; ++i) {
    sh.max_vblk = std::max(sh.max_vblk, (int)((js[i]->m + 1023) / 1024));
    sh.nvox += js[i]->m;
  }
  return sh;
}

void run_fwd(icnnm_ctx* c, const Shared& sh, int prec, int mode, const TcVData* tcv) {
  // the once-per-solve FP32 passes (theta0, objective) count as "other"
  PassScope ps(c, mode == 0 || mode == 4 ? 3 : (prec == ICNNM_BF16X3 ? 4 : (prec == ICNNM_FP32 ? 5 : 0)), 1, sh.nvox);
  if (prec == ICNNM_FP32 || mode == 0 || mode == 4) CK(launch_fwd_fp32(sh, mode, c->stream));
  else CK(tc_launch_fwd(sh, *tcv, mode, c->stream, prec == ICNNM_BF16X3));
}

// Tiles per column-partial row group of the update pass.
int fwd_slots(const Shared& sh, int prec, const TcVData* tcv) {
  if (prec == ICNNM_FP32) return 1;
  return tcv->g.det ? 0 : -tc_fwd_slots(sh, *tcv, prec == ICNNM_BF16X3);
}

// Column norms ||A_k(L) v_c||^2 of each job's current L into its colseg through the
// Gram A_k(L)^T A_k(L) (autocorrelations of exact products, then v_c^T G v_c in FP64):
// FP64-accurate and far cheaper than the FP32 m x k x k forward pass it replaces for
// theta0 and the objective on large jobs. Returns false (nothing launched) where the
// autocorrelation kernel's limits do not admit the kernel size.
bool gram_colnorms(icnnm_ctx* c, const std::vector<Job*>& js) {
  const VData* vd = js[0]->vd;
  const int k1 = vd->k1, k2 = vd->k2, k3 = vd->k3, k = vd->k;
  const long long nlag = (long long)(2 * k1 - 1) * (2 * k2 - 1) * (2 * k3 - 1);
  if (nlag > learn_max_lags() || learn_smem_bytes(k1, k2, k3) > 220 * 1024) return false;
  int sms = 1;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  const int nblk = 2 * sms;
  const size_t need = sizeof(double) * ((size_t)nblk * nlag + (size_t)k * k);
  if (need > c->gscr_bytes) {
    dfree_async(c->gscr, c->stream);    // stream-ordered: after its last use
    c->gscr = nullptr;
    c->gscr_bytes = 0;
    c->gscr = (double*)dalloc_async(c, need, c->stream);
    c->gscr_bytes = need;
  }
  double* part = c->gscr;
  double* G = part + (size_t)nblk * nlag;
  PassScope ps(c, 3, 3 * (int)js.size());
  for (const Job* j : js)
    CK(gram_colsq(j->dev.L, j->H, j->W, j->T, k1, k2, k3, vd->dV64, vd->kc, part, nblk, G, j->dev.colseg, c->stream));
  return true;
}

// Jobs whose FP32 forward pass would take at least 2^31 multiply-adds (m k^2) take their
// once-per-solve column norms from the Gram; below that the Gram's fixed cost (three
// launches, per-block partial sums) exceeds the pass. Decided per job, so a job takes the
// same route alone and in a batch.
void launch_reduce_cols_counted(icnnm_ctx* c, const Shared& sh) {
  PassScope ps(c, 3, 1);
  CK(launch_reduce_cols(sh, 0, 1, c->stream));
}

bool gram_route(const Job* j) { return (double)j->m * j->vd->k * j->vd->k >= 2147483648.0; }

// Column norms of A_k(L)V for every job of js into its colseg (L = the job's current L):
// the Gram route for the large jobs, the FP32 forward pass (mode 0 or 4) for the rest,
// as a list of its own in the second device job table.
void colnorms_once(icnnm_ctx* c, const std::vector<Job*>& js, int mode) {
  std::vector<Job*> big, small;
  for (Job* j : js) (gram_route(j) ? big : small).push_back(j);
  if (!big.empty() && !gram_colnorms(c, big)) small.insert(small.end(), big.begin(), big.end());
  if (small.empty()) return;
  const Shared shs = upload_list(c, small, 1);
  run_fwd(c, shs, ICNNM_FP32, mode, nullptr);
  launch_reduce_cols_counted(c, shs);
}

#define OTHER(n, expr)            \
  do {                            \
    PassScope ps__(c, 3, (n));    \
    CK(expr);                     \
  } while (0)

// Initial state: L = P_Omega M, theta0, U0 = -theta0 A_k(L)V and its column norms.
// theta0's column norms always come from the FP32 forward pass.
void engine_init(icnnm_ctx* c, const std::vector<Job*>& js) {
  const int prec = js[0]->run_prec;
  const TcVData* tcv = &js[0]->vd->tc;
  Shared sh = upload_list(c, js);
  OTHER(1, launch_init_L(sh, c->stream));
  colnorms_once(c, js, 0);
  OTHER(1, launch_theta0(sh, js[0]->p.theta0, c->stream));
  OTHER(1, launch_scale_X(sh, c->stream));
  if (prec != ICNNM_FP32) OTHER(1, tc_launch_prepare_X(sh, *tcv, /*from_L=*/0, c->stream, prec == ICNNM_BF16X3));
  run_fwd(c, sh, prec, 2, tcv);
  OTHER(1, launch_reduce_cols(sh, 0, fwd_slots(sh, prec, tcv), c->stream));
}

// One ADMM iteration for every job of the list. `check` (per list) adds the residual.
void engine_step(icnnm_ctx* c, const Shared& sh, int prec, const TcVData* tcv, bool check) {
  OTHER(1, launch_scalars(sh, c->stream));
  if (prec != ICNNM_FP32) OTHER(1, tc_launch_build_B2(sh, *tcv, c->stream));
  {
    PassScope ps(c, 1, 1, sh.nvox);
    if (prec == ICNNM_FP32) CK(launch_adj_gemm_fp32(sh, c->stream));
    else CK(tc_launch_adj(sh, *tcv, c->stream));
  }
  {
    PassScope ps(c, 2, 1, sh.nvox);
    if (prec == ICNNM_FP32) CK(launch_gather_fp32(sh, c->stream));
    else CK(tc_launch_gather(sh, *tcv, c->stream));
  }
  if (check) {
    if (prec != ICNNM_FP32) OTHER(1, tc_launch_prepare_X(sh, *tcv, /*from_L=*/1, c->stream, prec == ICNNM_BF16X3));
    run_fwd(c, sh, prec, 3, tcv);
    OTHER(1, launch_finish(sh, 1, c->stream));
  }
  if (prec != ICNNM_FP32) OTHER(1, tc_launch_prepare_X(sh, *tcv, /*from_L=*/0, c->stream, prec == ICNNM_BF16X3));
  run_fwd(c, sh, prec, 1, tcv);
  OTHER(1, launch_reduce_cols(sh, 1, fwd_slots(sh, prec, tcv), c->stream));
}

// ||A_k(L)V||_{2,1} of the returned L, in FP64-accurate arithmetic for every job (not from
// the BF16 forward pass: the l2,1 norm sums k column norms, most of them small for smooth
// data, and BF16 rounding of L lifts each small one in quadrature, +1.5% measured on the
// video-prediction workload).
void engine_objective(icnnm_ctx* c, const std::vector<Job*>& js) {
  const Shared sh = upload_list(c, js);
  colnorms_once(c, js, 4);
  OTHER(1, launch_finish(sh, 2, c->stream));
}

JobScal read_scal(Job& j, cudaStream_t st) {
  JobScal s;
  CK(cudaMemcpyAsync(&s, j.dev.sc, sizeof s, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

// Enqueue the copy of every listed job's scalars into the pinned array c->hscal (entry
// i for js[i]); they are valid after the next synchronisation of c->stream.
void enqueue_scals(icnnm_ctx* c, const std::vector<Job*>& js) {
  if ((int)js.size() > c->hscal_cap) {
    CK(cudaStreamSynchronize(c->stream));        // the old array may still be a copy target
    if (c->hscal) CK(cudaFreeHost(c->hscal));
    c->hscal = nullptr;
    c->hscal_cap = 0;
    const int cap = std::max<int>((int)js.size(), 256);
    CK(cudaHostAlloc((void**)&c->hscal, sizeof(JobScal) * cap, cudaHostAllocDefault));
    c->hscal_cap = cap;
  }
  for (size_t i = 0; i < js.size(); ++i)
    CK(cudaMemcpyAsync(&c->hscal[i], js[i]->dev.sc, sizeof(JobScal), cudaMemcpyDeviceToHost, c->stream));
}

double resid_of(const JobScal& s, int k) {
  return sqrt(s.rsq) / (sqrt((double)k) * std::max(sqrt(s.lsq), 1e-300));
}

// Run a fixed set of jobs to completion (blocking solves).
void run_jobs(icnnm_ctx* c, std::vector<Job*>& js, float* const* outs) {
  int prec = js[0]->p.prec;
  const TcVData* tcv = &js[0]->vd->tc;
  const int k = js[0]->vd->k;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, c->stream));
  engine_init(c, js);
  std::vector<Job*> live = js;
  Shared sh = upload_list(c, live);
  std::vector<Job*> live32;      // BF16 jobs in their finish (see switch_to_finish)
  Shared sh32{};
  int it = 0;
  const icnnm_params& p = js[0]->p;
  // Runs of plain (non-check) iterations are replayed from a CUDA graph of GRAPH_ITERS
  // iterations, captured after one direct iteration (which sets kernel attributes).
  // The legacy default stream cannot be captured; there every iteration is launched directly.
  constexpr int GRAPH_ITERS = 25;
  const bool graphs = c->stream != cudaStreamLegacy && c->stream != nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long graph_counts[NPASS + 1] = {}, graph_vox[NPASS + 1] = {};
  auto is_check = [&](int i) { return i >= p.max_iters || (p.tol > 0 && i % p.check_every == 0); };
  auto plain_run = [&](int from) {          // plain iterations from..from+n-1
    int n = 0;
    while (from + n <= p.max_iters && !is_check(from + n)) ++n;
    return n;
  };
  while (!live.empty()) {
    if (graphs && !c->prof && it >= 1 && live32.empty() && plain_run(it + 1) >= GRAPH_ITERS) {
      if (!gexec) {
        long long before[NPASS + 1], vbefore[NPASS + 1];
        for (int i = 0; i <= NPASS; ++i) before[i] = c->pass_n[i], vbefore[i] = c->pass_vox[i];
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        try {
          for (int i = 0; i < GRAPH_ITERS; ++i) engine_step(c, sh, prec, tcv, false);
        } catch (...) {
          cudaStreamEndCapture(c->stream, &graph);   // leave the stream usable
          if (graph) cudaGraphDestroy(graph);
          cudaGetLastError();
          throw;
        }
        CK(cudaStreamEndCapture(c->stream, &graph));
        const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
        for (int i = 0; i <= NPASS; ++i) {
          graph_counts[i] = c->pass_n[i] - before[i];
          c->pass_n[i] = before[i];
          graph_vox[i] = c->pass_vox[i] - vbefore[i];
          c->pass_vox[i] = vbefore[i];
        }
      }
      CK(cudaGraphLaunch(gexec, c->stream));
      for (int i = 0; i <= NPASS; ++i) c->pass_n[i] += graph_counts[i], c->pass_vox[i] += graph_vox[i];
      it += GRAPH_ITERS;
      continue;
    }
    ++it;
    const bool last = it >= p.max_iters;
    const bool check = is_check(it);
    engine_step(c, sh, prec, tcv, check);
    if (!live32.empty()) {
      const int fp = live32[0]->run_prec;
      engine_step(c, sh32, fp, fp == ICNNM_FP32 ? nullptr : &js[0]->vd->tc, check);
    }
    if (check) {
      std::vector<Job*> keep, keep32;
      bool moved = false;
      std::vector<Job*> all(live);
      all.insert(all.end(), live32.begin(), live32.end());
      enqueue_scals(c, all);
      CK(cudaStreamSynchronize(c->stream));
      size_t ai = 0;
      for (int grp = 0; grp < 2; ++grp)
        for (Job* j : grp == 0 ? live : live32) {
          const JobScal s = c->hscal[ai++];
          j->resid = resid_of(s, k);
          j->iters = it;
          const bool conv = p.tol > 0 && j->resid <= p.tol && it % p.check_every == 0;
          if (conv || last) {
            j->converged = conv;
          } else if (grp == 0 && bf16_should_finish(*j) && switch_to_finish(c, *j)) {
            keep32.push_back(j);
            moved = true;
          } else {
            (grp == 0 ? keep : keep32).push_back(j);
          }
          j->last_resid = j->resid;
        }
      if (keep.size() != live.size() || moved) {
        live = keep;
        if (!live.empty()) sh = upload_list(c, live);
        if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
      }
      if (keep32.size() != live32.size() || moved) {
        live32 = keep32;
        if (!live32.empty()) sh32 = upload_list(c, live32, 1);
      }
      if (live.empty() && !live32.empty()) {   // only FP32 finishers left: they become the main list
        live.swap(live32);
        std::swap(sh, sh32);
        prec = live[0]->run_prec;
        tcv = prec == ICNNM_FP32 ? nullptr : &js[0]->vd->tc;
      }
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  engine_objective(c, js);
  CK(cudaEventRecord(e1, c->stream));
  enqueue_scals(c, js);
  CK(cudaStreamSynchronize(c->stream));
  flush_prof(c);
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t i = 0; i < js.size(); ++i) {
    Job& j = *js[i];
    const JobScal s = c->hscal[i];
    if (s.status) fail(ICNNM_ETIMEOUT, "a bounded device-side wait expired");
    j.stats.iters = j.iters;
    j.stats.residual = j.resid;
    j.stats.objective = s.objective;
    j.stats.theta = s.theta;
    j.stats.seconds = ms * 1e-3;
    j.stats.latency = ms * 1e-3;
    if (outs && outs[i]) CK(cudaMemcpyAsync(outs[i], j.dev.L, j.m * 4, cudaMemcpyDefault, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
}

void prepare_job(icnnm_ctx* c, Job& j, const icnnm_shape* shape, const float* M, const uint8_t* mask,
                 const double* V, const icnnm_params& p) {
  int H, W, T, k1, k2, k3;
  validate_shape(shape, H, W, T, k1, k2, k3);
  validate_params(p);
  if (!M || !mask) fail(ICNNM_EINVAL, "M and mask must not be NULL");
  j.H = H; j.W = W; j.T = T; j.m = (long long)H * W * T;
  j.p = p;
  j.vd = get_vdata(c, V, k1, k2, k3, p.prec);
  // observed-entry checks on the device (inputs may be host or device)
  const bool mdev = is_device_ptr(M), kdev = is_device_ptr(mask);
  const float* dM = M;
  const uint8_t* dK = mask;
  float* tM = nullptr;
  uint8_t* tK = nullptr;
  if (!mdev) {
    tM = (float*)dalloc_async(c, j.m * 4, c->stream);
    CK(cudaMemcpyAsync(tM, M, j.m * 4, cudaMemcpyHostToDevice, c->stream));
    dM = tM;
  }
  if (!kdev) {
    tK = (uint8_t*)dalloc_async(c, j.m, c->stream);
    CK(cudaMemcpyAsync(tK, mask, j.m, cudaMemcpyHostToDevice, c->stream));
    dK = tK;
  }
  int* d2 = (int*)dalloc_async(c, 8, c->stream);
  CK(cudaMemsetAsync(d2, 0, 8, c->stream));
  CK(check_observed(dM, dK, j.m, d2, c->stream));
  int h2[2];
  CK(cudaMemcpyAsync(h2, d2, 8, cudaMemcpyDeviceToHost, c->stream));
  dfree_async(d2, c->stream);
  dfree_async(tM, c->stream);
  dfree_async(tK, c->stream);
  CK(cudaStreamSynchronize(c->stream));
  if (h2[1]) fail(ICNNM_EINVAL, "mask entries must be 0/1 and M must be finite on Omega");
  if (h2[0] == 0) fail(ICNNM_EINVAL, "Omega is empty");
  ensure_tc(c, j.vd, p.prec);
  j.srcM = M;
  j.srcmask = mask;
}

icnnm_params defaults() {
  icnnm_params p;
  icnnm_params_default(&p);
  return p;
}

// Serving thread ---------------------------------------------------------------------
// One step: admit queued jobs in FIFO order while their state fits the budget, initialise
// the admitted ones, run one iteration of every running job (grouped by V and by the
// arithmetic of their next iteration, each group as a plain and a check list), read the
// scalars of the checked jobs back with one stream synchronisation, then retire the jobs
// that converged, hit their cap or were cancelled: their objective is computed, L is kept
// on the device until the caller collects it, and their state is released (stream-ordered).
void server_loop(icnnm_ctx* c) {
  if (cudaSetDevice(c->device) != cudaSuccess) return;
  while (true) {
    std::vector<std::shared_ptr<Job>> admitted;
    {
      std::unique_lock<std::mutex> lk(c->qmu);
      c->qcv.wait(lk, [&] { return c->stop || !c->queue.empty() || !c->active.empty(); });
      if (c->stop && c->queue.empty() && c->active.empty()) return;
      // FIFO admission while the state fits the budget; jobs of other groups (V,
      // precision) are admitted too and stepped as lists of their own
      size_t planned = c->used;
      while (!c->queue.empty()) {
        auto j = c->queue.front();
        if (j->cancel) {
          c->queue.pop_front();
          if (j->dstage) { dfree_async(j->dstage, c->stream); j->dstage = nullptr; }
          j->phase = CANCELED;
          j->st = ICNNM_ECANCELED;
          continue;
        }
        const int nrp = std::max(fwd_fp32_nrp(j->vd->k), tc_nrp(j->vd->k));
        const size_t need = job_bytes(j->H, j->W, j->T, j->vd->k, j->vd->kc, j->p.prec, nrp, &j->vd->tc.g);
        if (planned + need > c->budget) break;
        planned += need;
        c->queue.pop_front();
        admitted.push_back(j);
        c->active.push_back(j);
        j->phase = ADMITTED;
      }
    }
    c->qcv.notify_all();
    std::lock_guard<std::recursive_mutex> g(c->mu);
    try {
      // groups of jobs that can share a launch list: same V and same arithmetic
      auto groups = [](const std::vector<Job*>& js, bool by_run_prec) {
        std::vector<std::vector<Job*>> out;
        for (Job* j : js) {
          const int pr = by_run_prec ? j->run_prec : j->p.prec;
          bool put = false;
          for (auto& gr : out)
            if (gr[0]->vd == j->vd && (by_run_prec ? gr[0]->run_prec : gr[0]->p.prec) == pr) {
              gr.push_back(j);
              put = true;
              break;
            }
          if (!put) out.push_back({j});
        }
        return out;
      };
      std::vector<Job*> fresh;
      for (auto& j : admitted) {
        try {
          alloc_job(c, *j);
          j->t_admit = std::chrono::steady_clock::now();
          fresh.push_back(j.get());
        } catch (StatusFail& f) {
          std::lock_guard<std::mutex> lk(c->qmu);
          free_job(c, *j);
          j->phase = FAILED; j->st = f.st; j->err = f.msg;
        }
      }
      for (auto& gr : groups(fresh, false)) engine_init(c, gr);
      for (Job* j : fresh) j->phase = RUNNING;
      // one iteration for every running job
      std::vector<Job*> run;
      for (auto& j : c->active)
        if (j->phase == RUNNING) run.push_back(j.get());
      std::vector<Job*> chk;
      for (auto& gr : groups(run, true)) {
        const int prec = gr[0]->run_prec;
        std::vector<Job*> plain, chk1;
        for (Job* j : gr) {
          const int it = j->iters + 1;
          const bool check = it >= j->p.max_iters || (j->p.tol > 0 && it % j->p.check_every == 0) || j->cancel;
          (check ? chk1 : plain).push_back(j);
        }
        const TcVData* tcv = prec != ICNNM_FP32 ? &gr[0]->vd->tc : nullptr;
        if (!plain.empty()) engine_step(c, upload_list(c, plain), prec, tcv, false);
        if (!chk1.empty()) engine_step(c, upload_list(c, chk1), prec, tcv, true);
        chk.insert(chk.end(), chk1.begin(), chk1.end());
      }
      for (Job* j : run) j->iters += 1;
      enqueue_scals(c, chk);
      CK(cudaStreamSynchronize(c->stream));          // the one synchronisation of a step
      flush_prof(c);
      std::vector<Job*> fin;
      for (size_t i = 0; i < chk.size(); ++i) {
        Job* j = chk[i];
        const JobScal& sc = c->hscal[i];
        j->resid = resid_of(sc, j->vd->k);
        const bool conv = j->p.tol > 0 && j->resid <= j->p.tol && j->iters % j->p.check_every == 0;
        if (conv || j->iters >= j->p.max_iters || j->cancel || sc.status) {
          j->converged = conv;
          fin.push_back(j);
        } else if (bf16_should_finish(*j)) {
          switch_to_finish(c, *j);
        }
        j->last_resid = j->resid;
      }
      if (!fin.empty()) {
        for (auto& gr : groups(fin, false)) engine_objective(c, gr);
        for (Job* j : fin) {
          j->dres = (float*)dalloc_async(c, (size_t)j->m * 4, c->stream);
          CK(cudaMemcpyAsync(j->dres, j->dev.L, j->m * 4, cudaMemcpyDeviceToDevice, c->stream));
        }
        enqueue_scals(c, fin);
        for (Job* j : fin) free_job(c, *j);
        CK(cudaStreamSynchronize(c->stream));
        const auto now = std::chrono::steady_clock::now();
        std::lock_guard<std::mutex> lk(c->qmu);
        for (size_t i = 0; i < fin.size(); ++i) {
          Job* j = fin[i];
          const JobScal& sc = c->hscal[i];
          j->stats.iters = j->iters;
          j->stats.residual = j->resid;
          j->stats.objective = sc.objective;
          j->stats.theta = sc.theta;
          j->stats.seconds = std::chrono::duration<double>(now - j->t_admit).count();
          j->stats.latency = std::chrono::duration<double>(now - j->t_submit).count();
          if (sc.status) { j->st = ICNNM_ETIMEOUT; j->phase = FAILED; }
          else if (j->cancel) { j->st = ICNNM_ECANCELED; j->phase = CANCELED; }
          else j->phase = DONE;
          if (j->phase != DONE) { dfree_async(j->dres, c->stream); j->dres = nullptr; }
        }
      }
    } catch (CudaFail& f) {
      report(c, f);
      std::lock_guard<std::mutex> lk(c->qmu);
      for (auto& j : c->active) {
        free_job(c, *j);
        if (j->phase < DONE) { j->phase = FAILED; j->st = ICNNM_ECUDA; }
      }
    } catch (StatusFail& f) {
      report(c, f);
      std::lock_guard<std::mutex> lk(c->qmu);
      for (auto& j : c->active) {
        free_job(c, *j);
        if (j->phase < DONE) { j->phase = FAILED; j->st = f.st; j->err = f.msg; }
      }
    }
    {
      std::lock_guard<std::mutex> lk(c->qmu);
      c->active.erase(std::remove_if(c->active.begin(), c->active.end(),
                                     [](const std::shared_ptr<Job>& j) { return j->phase >= DONE; }),
                      c->active.end());
    }
    c->qcv.notify_all();
  }
}

// Submit-side preparation of a served job (its V already looked up): the inputs copied
// into a device staging buffer on the submitting side's stream, where they are checked
// (mask 0/1, M finite on Omega, Omega non-empty) before the job is queued.
void prepare_submit(icnnm_ctx* c, Job& j, const icnnm_shape* shape, const float* M, const uint8_t* mask,
                    const icnnm_params& p) {
  int H, W, T, k1, k2, k3;
  validate_shape(shape, H, W, T, k1, k2, k3);
  if (!M || !mask) fail(ICNNM_EINVAL, "M and mask must not be NULL");
  j.H = H; j.W = W; j.T = T; j.m = (long long)H * W * T;
  j.p = p;
  std::lock_guard<std::mutex> sg(c->submu);
  const size_t mb = (size_t)j.m * 4, kb = (size_t)j.m;
  const size_t flag_off = (mb + kb + 15) / 16 * 16;
  void* st = nullptr;
  CK(cudaMallocFromPoolAsync(&st, flag_off + 8, c->pool, c->sub_stream));
  char* b = static_cast<char*>(st);
  int h2[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(b, M, mb, cudaMemcpyDefault, c->sub_stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + mb, mask, kb, cudaMemcpyDefault, c->sub_stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + flag_off, 0, 8, c->sub_stream);
  if (e == cudaSuccess)
    e = check_observed((const float*)b, (const uint8_t*)(b + mb), j.m, (int*)(b + flag_off), c->sub_stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h2, b + flag_off, 8, cudaMemcpyDeviceToHost, c->sub_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->sub_stream);
  if (e != cudaSuccess || h2[1] || h2[0] == 0) {
    cudaFreeAsync(st, c->sub_stream);
    cudaStreamSynchronize(c->sub_stream);
    if (e != cudaSuccess) throw CudaFail{e, "staging of the submitted inputs"};
    if (h2[1]) fail(ICNNM_EINVAL, "mask entries must be 0/1 and M must be finite on Omega");
    fail(ICNNM_EINVAL, "Omega is empty");
  }
  j.dstage = st;
}

}  // namespace

// =================================================================================
// Exported entry points
// =================================================================================
extern "C" {

icnnm_status icnnm_params_default(icnnm_params* p) {
  if (!p) return ICNNM_EINVAL;
  p->lambda = INFINITY;
  p->theta0 = 0.0;
  p->rho = 1.1;
  p->theta_max = 1e10;
  p->max_iters = 100;
  p->tol = 0.0;
  p->check_every = 10;
  p->prec = ICNNM_BF16;
  return ICNNM_OK;
}

const char* icnnm_strerror(icnnm_status st) {
  switch (st) {
    case ICNNM_OK: return "ok";
    case ICNNM_EINVAL: return "invalid argument";
    case ICNNM_ENOMEM: return "job state exceeds the HBM budget";
    case ICNNM_EAGAIN: return "job not finished";
    case ICNNM_ENOTFOUND: return "unknown job id";
    case ICNNM_ECUDA: return "CUDA error";
    case ICNNM_ETIMEOUT: return "a bounded device-side wait expired";
    case ICNNM_ECANCELED: return "job cancelled";
    case ICNNM_EUNSUPPORTED: return "not supported by this build";
    case ICNNM_ENOCONV: return "the eigensolver did not converge within its sweep cap";
  }
  return "unknown status";
}

const char* icnnm_last_error(icnnm_ctx* c) {
  if (!c) return "";
  std::lock_guard<std::mutex> g(c->err_mu);
  return c->last_err.c_str();
}

icnnm_status icnnm_create(icnnm_ctx** out, int device, size_t budget, void* stream) {
  if (!out) return ICNNM_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return ICNNM_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return ICNNM_ECUDA;
  auto* c = new icnnm_ctx();
  c->device = device;
  if (stream) c->stream = (cudaStream_t)stream;
  else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return ICNNM_ECUDA; }
    c->own_stream = true;
  }
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  c->budget = budget ? budget : (size_t)(0.9 * fr);
  auto undo = [&](icnnm_status st) {
    if (c->sub_stream) cudaStreamDestroy(c->sub_stream);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return st;
  };
  if (budget > fr) return undo(ICNNM_ENOMEM);
  if (cudaStreamCreateWithFlags(&c->sub_stream, cudaStreamNonBlocking) != cudaSuccess) return undo(ICNNM_ECUDA);
  // the context's own pool: memory freed by finished jobs stays reserved (up to the
  // budget) for the next ones instead of going back to the driver at every synchronisation
  cudaMemPoolProps pp{};
  pp.allocType = cudaMemAllocationTypePinned;
  pp.location.type = cudaMemLocationTypeDevice;
  pp.location.id = device;
  if (cudaMemPoolCreate(&c->pool, &pp) != cudaSuccess) { cudaGetLastError(); c->pool = nullptr; return undo(ICNNM_ECUDA); }
  uint64_t keep = c->budget;
  cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  // an allocation on the submitting side's stream must not wait for memory that the
  // serving stream frees later in its own order: no cross-stream reuse dependencies
  int no_deps = 0;
  cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowInternalDependencies, &no_deps);
  *out = c;
  return ICNNM_OK;
}

void icnnm_destroy(icnnm_ctx* c) {
  if (!c) return;
  {
    std::lock_guard<std::mutex> lk(c->qmu);
    c->stop = true;
    for (auto& j : c->queue) j->cancel = true;
  }
  c->qcv.notify_all();
  if (c->server.joinable()) c->server.join();
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->jobs) {
    free_job(c, *kv.second);
    if (kv.second->dres) cudaFreeAsync(kv.second->dres, c->stream);
    kv.second->dres = nullptr;
  }
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  for (auto& kv : c->vcache) {
    if (kv.second->dVf) cudaFree(kv.second->dVf);
    if (kv.second->dV64) cudaFree(kv.second->dV64);
    if (kv.second->tc_ready) tc_free_vdata(&kv.second->tc);
  }
  for (int sl = 0; sl < 2; ++sl) {
    dfree_async(c->dlist[sl], c->stream);
    dfree_async(c->dtile0[sl], c->stream);
  }
  for (int sl = 0; sl < 2; ++sl) c->dlist[sl] = nullptr, c->dtile0[sl] = nullptr;
  dfree_async(c->gscr, c->stream);
  cudaStreamSynchronize(c->stream);
  cudaStreamSynchronize(c->sub_stream);
  for (auto& e : c->ring) {
    if (e.p) cudaFreeHost(e.p);
    if (e.ev) cudaEventDestroy(e.ev);
  }
  if (c->hscal) cudaFreeHost(c->hscal);
  if (c->pool) cudaMemPoolDestroy(c->pool);
  cudaStreamDestroy(c->sub_stream);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

icnnm_status icnnm_learn_V(icnnm_ctx* c, const int64_t kdims[3], int32_t b, const icnnm_shape* shapes,
                           const float* const* tensors, double* V_out, double* eig_out) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  std::vector<void*> tmp;
  try {
    CK(cudaSetDevice(c->device));
    if (!kdims || b < 1 || !shapes || !tensors || !V_out) fail(ICNNM_EINVAL, "NULL argument or b < 1");
    const int k1 = (int)kdims[0], k2 = (int)kdims[1], k3 = (int)kdims[2];
    if (k1 < 1 || k2 < 1 || k3 < 1) fail(ICNNM_EINVAL, "kdims must be >= 1");
    const long long kk = (long long)k1 * k2 * k3;
    if (kk > 1024) fail(ICNNM_EINVAL, "k must be <= 1024");
    if ((long long)(2 * k1 - 1) * (2 * k2 - 1) * (2 * k3 - 1) > learn_max_lags())
      fail(ICNNM_EUNSUPPORTED, "too many autocorrelation lags for this build");
    if (learn_smem_bytes(k1, k2, k3) > 220 * 1024) fail(ICNNM_EUNSUPPORTED, "kernel too large for learn_V");
    const int k = (int)kk;
    std::vector<const float*> dptr(b);
    std::vector<int> dims(3 * b);
    int* dbad;
    CK(cudaMalloc(&dbad, 4));
    tmp.push_back(dbad);
    CK(cudaMemset(dbad, 0, 4));
    for (int j = 0; j < b; ++j) {
      const icnnm_shape& s = shapes[j];
      const int H = (int)s.dims[0], W = (int)s.dims[1], T = s.ndim == 3 ? (int)s.dims[2] : 1;
      if (s.ndim != 2 && s.ndim != 3) fail(ICNNM_EINVAL, "ndim must be 2 or 3");
      if (H < k1 || W < k2 || T < k3) fail(ICNNM_EINVAL, "every dim must be at least the kernel's");
      if (!tensors[j]) fail(ICNNM_EINVAL, "NULL tensor");
      const long long m = (long long)H * W * T;
      dims[3 * j] = H; dims[3 * j + 1] = W; dims[3 * j + 2] = T;
      if (is_device_ptr(tensors[j])) dptr[j] = tensors[j];
      else {
        void* p;
        CK(cudaMalloc(&p, m * 4));
        tmp.push_back(p);
        CK(cudaMemcpyAsync(p, tensors[j], m * 4, cudaMemcpyHostToDevice, c->stream));
        dptr[j] = (const float*)p;
      }
      CK(check_finite(dptr[j], m, dbad, c->stream));
    }
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, dbad, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hbad) fail(ICNNM_EINVAL, "a reference tensor has a non-finite entry");
    const float** dL;
    int* ddims;
    CK(cudaMalloc(&dL, sizeof(float*) * b)); tmp.push_back(dL);
    CK(cudaMalloc(&ddims, sizeof(int) * 3 * b)); tmp.push_back(ddims);
    CK(cudaMemcpyAsync(dL, dptr.data(), sizeof(float*) * b, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(ddims, dims.data(), sizeof(int) * 3 * b, cudaMemcpyHostToDevice, c->stream));
    const int nblk = 16;
    const long long nlag = (long long)(2 * k1 - 1) * (2 * k2 - 1) * (2 * k3 - 1);
    double *dpart, *dgram, *dV, *dev, *dVout;
    int* dinfo;
    CK(cudaMalloc(&dpart, sizeof(double) * b * nblk * nlag)); tmp.push_back(dpart);
    CK(cudaMalloc(&dgram, sizeof(double) * k * k)); tmp.push_back(dgram);
    CK(cudaMalloc(&dV, sizeof(double) * k * k)); tmp.push_back(dV);
    CK(cudaMalloc(&dVout, sizeof(double) * k * k)); tmp.push_back(dVout);
    CK(cudaMalloc(&dev, sizeof(double) * k)); tmp.push_back(dev);
    CK(cudaMalloc(&dinfo, 2 * sizeof(int))); tmp.push_back(dinfo);
    CK(cudaMemsetAsync(dinfo, 0, 2 * sizeof(int), c->stream));
    void* dscr;
    CK(cudaMalloc(&dscr, learn_eig_grid_scratch(c->device))); tmp.push_back(dscr);
    CK(learn_gram(b, dL, ddims, k1, k2, k3, dpart, nblk, dgram, c->stream));
    CK(learn_eig_grid(dgram, dV, k, dev, dVout, dinfo, dscr, c->stream));
    CK(cudaMemcpyAsync(V_out, dVout, sizeof(double) * k * k, cudaMemcpyDefault, c->stream));
    if (eig_out) CK(cudaMemcpyAsync(eig_out, dev, sizeof(double) * k, cudaMemcpyDefault, c->stream));
    int hinfo[2] = {0, 0};
    CK(cudaMemcpyAsync(hinfo, dinfo, sizeof hinfo, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hinfo[1]) fail(ICNNM_ETIMEOUT, "a bounded grid barrier of the eigensolver expired");
    if (hinfo[0] < 0) fail(ICNNM_ENOCONV, "the FP64 Jacobi eigensolver did not converge within 30 sweeps");
    for (void* p : tmp) cudaFree(p);
    return ICNNM_OK;
  } catch (StatusFail& f) {
    for (void* p : tmp) cudaFree(p);
    return report(c, f);
  } catch (CudaFail& f) {
    for (void* p : tmp) cudaFree(p);
    return report(c, f);
  }
}

icnnm_status icnnm_spectral_diagnostics(icnnm_ctx* c, const icnnm_shape* shape, const float* L0, const double* V,
                                        double rank_tol, double* sigma_out, int32_t* r_K, double* alpha_K,
                                        double* mu_K) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  std::vector<void*> tmp;
  try {
    CK(cudaSetDevice(c->device));
    int H, W, T, k1, k2, k3;
    validate_shape(shape, H, W, T, k1, k2, k3);
    if (!L0) fail(ICNNM_EINVAL, "L0 is NULL");
    if (!(rank_tol > 0 && rank_tol < 1)) fail(ICNNM_EINVAL, "rank_tol must be in (0, 1)");
    if ((long long)(2 * k1 - 1) * (2 * k2 - 1) * (2 * k3 - 1) > learn_max_lags())
      fail(ICNNM_EUNSUPPORTED, "too many autocorrelation lags for this build");
    if (learn_smem_bytes(k1, k2, k3) > 220 * 1024) fail(ICNNM_EUNSUPPORTED, "kernel too large");
    VData* vd = get_vdata(c, V, k1, k2, k3, ICNNM_FP32);       // validates V (orthonormal, finite)
    const int k = vd->k;
    const long long m = (long long)H * W * T;
    auto dalloc = [&](size_t bytes) {
      void* p;
      CK(cudaMalloc(&p, bytes));
      tmp.push_back(p);
      return p;
    };
    const float* dL = L0;
    if (!is_device_ptr(L0)) {
      float* p = (float*)dalloc(m * 4);
      CK(cudaMemcpyAsync(p, L0, m * 4, cudaMemcpyHostToDevice, c->stream));
      dL = p;
    }
    int* dbad = (int*)dalloc(4);
    CK(cudaMemsetAsync(dbad, 0, 4, c->stream));
    CK(check_finite(dL, m, dbad, c->stream));
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, dbad, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hbad) fail(ICNNM_EINVAL, "L0 has a non-finite entry");
    const int dims[3] = {H, W, T};
    const float** dLp = (const float**)dalloc(sizeof(float*));
    int* ddims = (int*)dalloc(sizeof dims);
    CK(cudaMemcpyAsync(dLp, &dL, sizeof(float*), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(ddims, dims, sizeof dims, cudaMemcpyHostToDevice, c->stream));
    const size_t kk = (size_t)k * k;
    const long long nlag = (long long)(2 * k1 - 1) * (2 * k2 - 1) * (2 * k3 - 1);
    int sms = 1;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int nblk = 2 * sms;                // b = 1: spread the bricks over every SM
    double* dpart = (double*)dalloc(sizeof(double) * nblk * nlag);
    double* dG = (double*)dalloc(sizeof(double) * kk);
    double* dV = (double*)dalloc(sizeof(double) * kk);
    double* dT = (double*)dalloc(sizeof(double) * kk);
    double* dP = (double*)dalloc(sizeof(double) * kk);
    double* dS = (double*)dalloc(sizeof(double) * kk);
    double* dR = (double*)dalloc(sizeof(double) * kk);
    double* dRout = (double*)dalloc(sizeof(double) * kk);
    double* dsig = (double*)dalloc(sizeof(double) * k);
    double* dev = (double*)dalloc(sizeof(double) * k);
    double* dout = (double*)dalloc(sizeof(double) * 2);
    int* dinfo = (int*)dalloc(2 * sizeof(int));
    void* dscr = dalloc(learn_eig_grid_scratch(c->device));
    CK(cudaMemsetAsync(dinfo, 0, 2 * sizeof(int), c->stream));
    CK(cudaMemcpyAsync(dV, vd->V64.data(), sizeof(double) * kk, cudaMemcpyHostToDevice, c->stream));
    CK(learn_gram(1, dLp, ddims, k1, k2, k3, dpart, nblk, dG, c->stream, true));
    CK(diag_spectral(dG, dV, k, rank_tol, dT, dP, dsig, dS, dout, c->stream));
    CK(learn_eig_grid(dS, dR, k, dev, dRout, dinfo, dscr, c->stream));
    double hout[2] = {0, 0}, lmax = 0;
    int hinfo[2] = {0, 0};
    if (sigma_out) CK(cudaMemcpyAsync(sigma_out, dsig, sizeof(double) * k, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(hout, dout, sizeof hout, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&lmax, dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(hinfo, dinfo, sizeof hinfo, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hinfo[1]) fail(ICNNM_ETIMEOUT, "a bounded grid barrier of the eigensolver expired");
    if (hinfo[0] < 0) fail(ICNNM_ENOCONV, "the FP64 Jacobi eigensolver did not converge within 30 sweeps");
    if (r_K) *r_K = (int32_t)hout[0];
    if (mu_K) *mu_K = hout[1];
    if (alpha_K) *alpha_K = hout[0] > 0 ? sqrt(fmax(lmax, 0.0)) : 0.0;
    for (void* p : tmp) cudaFree(p);
    return ICNNM_OK;
  } catch (StatusFail& f) {
    for (void* p : tmp) cudaFree(p);
    return report(c, f);
  } catch (CudaFail& f) {
    for (void* p : tmp) cudaFree(p);
    return report(c, f);
  }
}

icnnm_status icnnm_cnnm_solve(icnnm_ctx* c, const icnnm_shape* shape, const float* M, const uint8_t* mask,
                              const icnnm_params* params, float* L_out, icnnm_stats* stats) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  std::vector<void*> tmp;
  try {
    CK(cudaSetDevice(c->device));
    int H, W, T, k1, k2, k3;
    validate_shape(shape, H, W, T, k1, k2, k3);
    const icnnm_params p = params ? *params : defaults();
    validate_params(p);
    if (!M || !mask || !L_out) fail(ICNNM_EINVAL, "M, mask and L_out must not be NULL");
    if (!isinf(p.lambda)) fail(ICNNM_EUNSUPPORTED, "CNNM: only lambda = INFINITY (the exact projection)");
    if (p.tol != 0) fail(ICNNM_EUNSUPPORTED, "CNNM: fixed iteration counts only (tol = 0)");
    if (p.prec != ICNNM_FP32) fail(ICNNM_EUNSUPPORTED, "CNNM: FP32 only");
    if (learn_smem_bytes(k1, k2, k3) > 220 * 1024 ||
        (long long)(2 * k1 - 1) * (2 * k2 - 1) * (2 * k3 - 1) > learn_max_lags())
      fail(ICNNM_EUNSUPPORTED, "kernel too large");
    const long long m = (long long)H * W * T;
    if (cnnm_state_bytes(H, W, T, k1, k2, k3) + c->used > c->budget)
      fail(ICNNM_ENOMEM, "CNNM state exceeds the HBM budget");
    auto dalloc = [&](size_t bytes) {
      void* q;
      CK(cudaMalloc(&q, bytes));
      tmp.push_back(q);
      return q;
    };
    float* dM = (float*)dalloc(m * 4);
    uint8_t* dK = (uint8_t*)dalloc(m);
    float* dL = (float*)dalloc(m * 4);
    CK(cudaMemcpyAsync(dM, M, m * 4, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(dK, mask, m, cudaMemcpyDefault, c->stream));
    int* d2 = (int*)dalloc(8);
    CK(cudaMemsetAsync(d2, 0, 8, c->stream));
    CK(check_observed(dM, dK, m, d2, c->stream));
    int h2[2];
    CK(cudaMemcpyAsync(h2, d2, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h2[1]) fail(ICNNM_EINVAL, "mask entries must be 0/1 and M must be finite on Omega");
    if (h2[0] == 0) fail(ICNNM_EINVAL, "Omega is empty");
    CnnmProblem P{H, W, T, k1, k2, k3, dM, dK, dL, p.max_iters, p.theta0, p.rho, p.theta_max};
    CnnmResult r{};
    CK(cnnm_run(P, c->stream, &r));
    if (r.timed_out) fail(ICNNM_ETIMEOUT, "a bounded grid barrier of the eigensolver expired");
    if (r.unconverged) fail(ICNNM_ENOCONV, "the FP64 Jacobi eigensolver did not converge within 30 sweeps");
    CK(cudaMemcpyAsync(L_out, dL, m * 4, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (stats) {
      stats->iters = p.max_iters;
      stats->residual = 0.0;
      stats->objective = r.objective;
      stats->theta = r.theta;
      stats->seconds = r.seconds;
      stats->latency = r.seconds;
    }
    for (void* q : tmp) cudaFree(q);
    return ICNNM_OK;
  } catch (StatusFail& f) {
    for (void* q : tmp) cudaFree(q);
    return report(c, f);
  } catch (CudaFail& f) {
    for (void* q : tmp) cudaFree(q);
    return report(c, f);
  }
}

// PassHook callbacks on a context: the same counters and events as PassScope, without
// throwing (a failed event record only loses that pass's time).
static void fft_hook_begin(void* u, int pass, int nk, long long nvox) {
  icnnm_ctx* c = (icnnm_ctx*)u;
  c->pass_n[pass] += nk;
  c->pass_n[NPASS] += nk;
  c->pass_vox[pass] += nvox;
  c->pass_vox[NPASS] += nvox;
  if (c->prof) {
    try {
      c->hook_idx = c->evnext;
      cudaEventRecord(pool_event(c), c->stream);
    } catch (...) {
      c->hook_idx = (size_t)-1;
    }
  }
}
static void fft_hook_end(void* u, int pass) {
  icnnm_ctx* c = (icnnm_ctx*)u;
  if (c->prof && c->hook_idx != (size_t)-1) {
    try {
      cudaEventRecord(pool_event(c), c->stream);
      c->pending.emplace_back(pass, c->hook_idx);
    } catch (...) {
    }
  }
}

icnnm_status icnnm_solve_fft(icnnm_ctx* c, const icnnm_shape* shape, const float* M, const uint8_t* mask,
                             const double* V, const icnnm_params* params, float* L_out, icnnm_stats* stats) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  std::vector<void*> tmp;
  auto release = [&] {
    for (void* q : tmp) cudaFree(q);
    tmp.clear();
  };
  try {
    CK(cudaSetDevice(c->device));
    int H, W, T, k1, k2, k3;
    validate_shape(shape, H, W, T, k1, k2, k3);
    const icnnm_params p = params ? *params : defaults();
    validate_params(p);
    if (!M || !mask || !L_out) fail(ICNNM_EINVAL, "M, mask and L_out must not be NULL");
    std::string why;
    if (!fft_supported(H, W, T, &why)) fail(ICNNM_EUNSUPPORTED, why);
    VData* vd = get_vdata(c, V, k1, k2, k3, ICNNM_FP32);       // validates V (orthonormal, finite)
    const long long m = (long long)H * W * T;
    if (fft_state_bytes(H, W, T, vd->k) + (size_t)m * 9 + c->used > c->budget)
      fail(ICNNM_ENOMEM, "the spectra of U and of the kernels exceed the HBM budget");
    auto dalloc = [&](size_t bytes) {
      void* q;
      CK(cudaMalloc(&q, bytes));
      tmp.push_back(q);
      return q;
    };
    float* dM = (float*)dalloc(m * 4);
    uint8_t* dK = (uint8_t*)dalloc(m);
    float* dL = (float*)dalloc(m * 4);
    CK(cudaMemcpyAsync(dM, M, m * 4, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(dK, mask, m, cudaMemcpyDefault, c->stream));
    int* d2 = (int*)dalloc(8);
    CK(cudaMemsetAsync(d2, 0, 8, c->stream));
    CK(check_observed(dM, dK, m, d2, c->stream));
    int h2[2];
    CK(cudaMemcpyAsync(h2, d2, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h2[1]) fail(ICNNM_EINVAL, "mask entries must be 0/1 and M must be finite on Omega");
    if (h2[0] == 0) fail(ICNNM_EINVAL, "Omega is empty");
    FftProblem P{c->device, H, W, T, k1, k2, k3, dM, dK, dL, vd->dV64, p.max_iters, p.check_every,
                 p.theta0, p.rho, p.theta_max, p.lambda, p.tol, PassHook{c, fft_hook_begin, fft_hook_end}};
    FftResult r{};
    const cudaError_t fe = fft_run(P, c->stream, &r);
    flush_prof(c);
    CK(fe);
    CK(cudaMemcpyAsync(L_out, dL, m * 4, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (stats) {
      stats->iters = r.iters;
      stats->residual = r.residual;
      stats->objective = r.objective;
      stats->theta = r.theta;
      stats->seconds = r.seconds;
      stats->latency = r.seconds;
    }
    release();
    return ICNNM_OK;
  } catch (StatusFail& f) {
    release();
    return report(c, f);
  } catch (CudaFail& f) {
    release();
    return report(c, f);
  }
}

icnnm_status icnnm_solve_batch(icnnm_ctx* c, int32_t n, const icnnm_shape* shapes, const float* const* M,
                               const uint8_t* const* mask, const double* V, const icnnm_params* params,
                               float* const* L_out, icnnm_stats* stats) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  std::vector<std::unique_ptr<Job>> jobs;
  try {
    CK(cudaSetDevice(c->device));
    if (n < 1 || !shapes || !M || !mask || !L_out) fail(ICNNM_EINVAL, "NULL argument or n < 1");
    const icnnm_params p = params ? *params : defaults();
    std::vector<Job*> js;
    for (int i = 0; i < n; ++i) {
      jobs.push_back(std::make_unique<Job>());
      prepare_job(c, *jobs.back(), &shapes[i], M[i], mask[i], V, p);
      if (i > 0 && (shapes[i].kdims[0] != shapes[0].kdims[0] || shapes[i].kdims[1] != shapes[0].kdims[1] ||
                    shapes[i].kdims[2] != shapes[0].kdims[2]))
        fail(ICNNM_EINVAL, "all problems of a batch share kernel dims");
      js.push_back(jobs.back().get());
    }
    for (Job* j : js) alloc_job(c, *j);
    run_jobs(c, js, L_out);
    if (stats)
      for (int i = 0; i < n; ++i) stats[i] = js[i]->stats;
    for (Job* j : js) free_job(c, *j);
    return ICNNM_OK;
  } catch (StatusFail& f) {
    cudaStreamSynchronize(c->stream);
    for (auto& j : jobs) free_job(c, *j);
    return report(c, f);
  } catch (CudaFail& f) {
    cudaStreamSynchronize(c->stream);
    for (auto& j : jobs) free_job(c, *j);
    return report(c, f);
  }
}

icnnm_status icnnm_solve(icnnm_ctx* c, const icnnm_shape* shape, const float* M, const uint8_t* mask,
                         const double* V, const icnnm_params* params, float* L_out, icnnm_stats* stats) {
  if (!L_out) {
    if (c) set_err(c, "L_out is NULL");
    return ICNNM_EINVAL;
  }
  float* outs[1] = {L_out};
  const float* Ms[1] = {M};
  const uint8_t* Ks[1] = {mask};
  return icnnm_solve_batch(c, 1, shape, Ms, Ks, V, params, outs, stats);
}

icnnm_status icnnm_submit(icnnm_ctx* c, const icnnm_shape* shape, const float* M, const uint8_t* mask,
                          const double* V, const icnnm_params* params, uint64_t* job_id) {
  if (!c || !job_id) return ICNNM_EINVAL;
  auto j = std::make_shared<Job>();
  j->t_submit = std::chrono::steady_clock::now();
  try {
    CK(cudaSetDevice(c->device));
    const icnnm_params p = params ? *params : defaults();
    int H, W, T, k1, k2, k3;
    validate_shape(shape, H, W, T, k1, k2, k3);
    validate_params(p);
    {
      // V: the cached data without the engine's mutex when it is ready; built under it
      // (once per V and precision) otherwise
      const std::vector<double> hv = read_V(V, k1 * k2 * k3);
      VData* vd = find_vdata_ready(c, v_key(hv.data(), k1, k2, k3), p.prec);
      if (!vd) {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        vd = get_vdata(c, hv.data(), k1, k2, k3, p.prec);
        ensure_tc(c, vd, p.prec);
      }
      const int nrp = std::max(fwd_fp32_nrp(vd->k), tc_nrp(vd->k));
      if (job_bytes(H, W, T, vd->k, vd->kc, p.prec, nrp, &vd->tc.g) > c->budget)
        fail(ICNNM_ENOMEM, "the job alone exceeds the HBM budget");
      j->vd = vd;
    }
    prepare_submit(c, *j, shape, M, mask, p);
  } catch (StatusFail& f) {
    return report(c, f);
  } catch (CudaFail& f) {
    return report(c, f);
  }
  {
    std::lock_guard<std::mutex> lk(c->qmu);
    j->id = c->next_id++;
    c->jobs[j->id] = j;
    c->queue.push_back(j);
    if (!c->server.joinable()) c->server = std::thread(server_loop, c);
  }
  c->qcv.notify_all();
  *job_id = j->id;
  return ICNNM_OK;
}

static icnnm_status collect(icnnm_ctx* c, std::shared_ptr<Job> j, float* L_out, icnnm_stats* stats) {
  if (j->phase == DONE) {
    // the server synchronised its stream after writing dres, so a plain copy is ordered
    cudaSetDevice(c->device);
    cudaError_t e = cudaSuccess;
    if (L_out) e = cudaMemcpy(L_out, j->dres, j->m * 4, cudaMemcpyDefault);
    {
      std::lock_guard<std::mutex> sg(c->submu);
      cudaFreeAsync(j->dres, c->sub_stream);
    }
    j->dres = nullptr;
    if (e != cudaSuccess) {
      cudaGetLastError();
      return ICNNM_ECUDA;
    }
    if (stats) *stats = j->stats;
    return ICNNM_OK;
  }
  if (!j->err.empty()) set_err(c, j->err);
  return j->st == ICNNM_OK ? ICNNM_ECUDA : j->st;
}

icnnm_status icnnm_poll(icnnm_ctx* c, uint64_t id, float* L_out, icnnm_stats* stats) {
  return icnnm_wait(c, id, 0, L_out, stats);
}

icnnm_status icnnm_wait(icnnm_ctx* c, uint64_t id, int64_t timeout_ms, float* L_out, icnnm_stats* stats) {
  if (!c) return ICNNM_EINVAL;
  std::shared_ptr<Job> j;
  {
    std::unique_lock<std::mutex> lk(c->qmu);
    auto it = c->jobs.find(id);
    if (it == c->jobs.end()) return ICNNM_ENOTFOUND;
    j = it->second;
    auto done = [&] { return j->phase >= DONE; };
    if (timeout_ms < 0) c->qcv.wait(lk, done);
    else if (timeout_ms > 0) c->qcv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
    if (!done()) return ICNNM_EAGAIN;
    c->jobs.erase(it);
  }
  return collect(c, j, L_out, stats);
}

icnnm_status icnnm_profile_enable(icnnm_ctx* c, int32_t enable) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  c->prof = enable != 0;
  c->pending.clear();
  c->evnext = 0;
  for (int i = 0; i < NPASS; ++i) c->pass_ms[i] = 0;
  for (int i = 0; i <= NPASS; ++i) c->pass_n[i] = 0, c->pass_vox[i] = 0;
  return ICNNM_OK;
}

icnnm_status icnnm_profile_voxels(icnnm_ctx* c, int32_t pass, int64_t* voxels) {
  if (!c || pass < -1 || pass >= NPASS) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  if (voxels) *voxels = c->pass_vox[pass < 0 ? NPASS : pass];
  return ICNNM_OK;
}

icnnm_status icnnm_profile_read(icnnm_ctx* c, int32_t pass, double* ms_total, int64_t* launches) {
  if (!c || pass < -1 || pass >= NPASS) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  if (ms_total) *ms_total = pass < 0 ? 0.0 : c->pass_ms[pass];
  if (launches) *launches = pass < 0 ? c->pass_n[NPASS] : c->pass_n[pass];
  return ICNNM_OK;
}

static bool tile_cfg_ok(const icnnm_tile_config& t) {
  return (t.adj_tap_width == 0 || t.adj_tap_width == 128 || t.adj_tap_width == 256) &&
         (t.fwd_channel_width == 0 || t.fwd_channel_width == 128 || t.fwd_channel_width == 256) &&
         (t.fwd_u_stages >= 0 && t.fwd_u_stages <= 2);
}

static TcTiles tiles_of(const icnnm_tile_config& t) {
  TcTiles r;
  if (t.adj_tap_width) r.gpt_max = t.adj_tap_width / 32;
  if (t.fwd_channel_width) r.ctw_max = t.fwd_channel_width;
  if (t.fwd_u_stages) r.nus_max = t.fwd_u_stages;
  return r;
}

icnnm_status icnnm_set_deterministic(icnnm_ctx* c, int32_t on) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  c->det = on ? 1 : 0;
  return ICNNM_OK;
}

icnnm_status icnnm_set_tile_config(icnnm_ctx* c, const int64_t kdims[3], const icnnm_tile_config* cfg) {
  if (!c || !kdims || !cfg) return ICNNM_EINVAL;
  if (!tile_cfg_ok(*cfg) || kdims[0] < 1 || kdims[1] < 1 || kdims[2] < 1) {
    set_err(c, "tile widths must be 0, 128 or 256 and stages 0, 1 or 2");
    return ICNNM_EINVAL;
  }
  std::lock_guard<std::recursive_mutex> g(c->mu);
  c->tiles[kdims_key((int)kdims[0], (int)kdims[1], (int)kdims[2])] = tiles_of(*cfg);
  return ICNNM_OK;
}

icnnm_status icnnm_autotune(icnnm_ctx* c, const double* V, int32_t n, const icnnm_shape* shapes, int32_t iters,
                            icnnm_tile_config* best, icnnm_tile_result* results, int32_t max_results,
                            int32_t* n_results) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  std::vector<std::unique_ptr<Job>> jobs;
  std::vector<void*> inputs;
  TcVData tmp;
  bool tmp_built = false;
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    for (auto& j : jobs) free_job(c, *j);
    for (void* p : inputs) dfree_async(p, c->stream);
    if (tmp_built) tc_free_vdata(&tmp);
    cudaStreamSynchronize(c->stream);
  };
  try {
    CK(cudaSetDevice(c->device));
    if (n < 1 || !shapes || iters < 1 || !best) fail(ICNNM_EINVAL, "NULL argument, n < 1 or iters < 1");
    int H, W, T, k1, k2, k3;
    validate_shape(&shapes[0], H, W, T, k1, k2, k3);
    VData* vd = get_vdata(c, V, k1, k2, k3, ICNNM_BF16);     // validates V
    std::string why;
    if (!tc_supported(k1, k2, k3, &why)) fail(ICNNM_EUNSUPPORTED, "BF16 path: " + why);
    icnnm_params p = defaults();
    p.prec = ICNNM_BF16;
    p.max_iters = iters + 2;
    // the synthetic jobs (inputs filled on the device)
    for (int i = 0; i < n; ++i) {
      int h, w, t, a, b, e;
      validate_shape(&shapes[i], h, w, t, a, b, e);
      if (a != k1 || b != k2 || e != k3) fail(ICNNM_EINVAL, "all shapes share kernel dims");
      auto j = std::make_unique<Job>();
      j->H = h; j->W = w; j->T = t; j->m = (long long)h * w * t;
      j->p = p;
      float* dM = (float*)dalloc_async(c, (size_t)j->m * 4, c->stream);
      uint8_t* dK = (uint8_t*)dalloc_async(c, (size_t)j->m, c->stream);
      inputs.push_back(dM);
      inputs.push_back(dK);
      CK(launch_tune_fill(dM, dK, h, w, t, c->stream));
      j->srcM = dM;
      j->srcmask = dK;
      jobs.push_back(std::move(j));
    }
    // candidates: every combination of the three bounds; equal geometries are measured once
    std::vector<icnnm_tile_result> res;
    double best_ms = INFINITY;
    icnnm_tile_config best_cfg{};
    for (int aw : {256, 128})
      for (int fw : {256, 128})
        for (int us : {2, 1}) {
          const icnnm_tile_config cfg{aw, fw, us};
          TcTiles tl = tiles_of(cfg);
          tl.det = c->det;
          const TcGeom gg = tc_geom(k1, k2, k3, vd->kc, tl);
          bool seen = false;
          for (const auto& r : res)
            if (r.adj_tap_width == gg.nta && r.fwd_channel_width == gg.ctw && r.fwd_u_stages == gg.nus) seen = true;
          if (seen) continue;
          // V data of this candidate, not cached: the jobs point at a private VData
          VData cand;
          cand.k1 = k1; cand.k2 = k2; cand.k3 = k3; cand.k = vd->k; cand.kc = vd->kc;
          cand.dVf = vd->dVf;
          cand.dV64 = vd->dV64;
          CK(tc_build_vdata(vd->V64.data(), k1, k2, k3, vd->kc, &tmp, tl));
          tmp_built = true;
          cand.tc = tmp;
          cand.tc_ready = true;
          std::vector<Job*> js;
          for (auto& j : jobs) {
            j->vd = &cand;
            alloc_job(c, *j);
            js.push_back(j.get());
          }
          engine_init(c, js);
          const Shared sh = upload_list(c, js);
          for (int w0 = 0; w0 < 2; ++w0) engine_step(c, sh, ICNNM_BF16, &cand.tc, false);
          cudaEvent_t e0, e1;
          CK(cudaEventCreate(&e0));
          CK(cudaEventCreate(&e1));
          CK(cudaEventRecord(e0, c->stream));
          for (int it = 0; it < iters; ++it) engine_step(c, sh, ICNNM_BF16, &cand.tc, false);
          CK(cudaEventRecord(e1, c->stream));
          CK(cudaStreamSynchronize(c->stream));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          enqueue_scals(c, js);
          CK(cudaStreamSynchronize(c->stream));
          for (size_t i = 0; i < js.size(); ++i)
            if (c->hscal[i].status) fail(ICNNM_ETIMEOUT, "a bounded device-side wait expired while tuning");
          for (auto& j : jobs) free_job(c, *j);
          CK(cudaStreamSynchronize(c->stream));
          tc_free_vdata(&tmp);
          tmp_built = false;
          icnnm_tile_result r{cfg, gg.nta, gg.ctw, gg.nus, ms / iters};
          res.push_back(r);
          if (r.ms_per_iter < best_ms) {
            best_ms = r.ms_per_iter;
            best_cfg = cfg;
          }
        }
    for (auto& j : jobs) j->vd = nullptr;
    c->tiles[kdims_key(k1, k2, k3)] = tiles_of(best_cfg);
    *best = best_cfg;
    if (n_results) *n_results = (int32_t)res.size();
    for (int i = 0; results && i < (int)res.size() && i < max_results; ++i) results[i] = res[i];
    cleanup();
    return ICNNM_OK;
  } catch (StatusFail& f) {
    cleanup();
    return report(c, f);
  } catch (CudaFail& f) {
    cleanup();
    return report(c, f);
  }
}

icnnm_status icnnm_job_bytes(icnnm_ctx* c, const icnnm_shape* shape, int32_t prec, size_t* bytes) {
  if (!c || !bytes) return ICNNM_EINVAL;
  try {
    int H, W, T, k1, k2, k3;
    validate_shape(shape, H, W, T, k1, k2, k3);
    if (prec != ICNNM_FP32 && prec != ICNNM_BF16 && prec != ICNNM_BF16X3) fail(ICNNM_EINVAL, "unknown precision");
    const int k = k1 * k2 * k3, kc = round_up(k, 16);
    TcGeom g{};
    if (prec != ICNNM_FP32) {
      std::string why;
      if (!tc_supported(k1, k2, k3, &why)) fail(ICNNM_EUNSUPPORTED, "BF16 path: " + why);
      g = tc_geom(k1, k2, k3, kc, tiles_for(c, k1, k2, k3));
      if (prec == ICNNM_BF16X3 && !g.split_ok) fail(ICNNM_EUNSUPPORTED, "BF16X3 is not built for these kernel dims");
    }
    const int nrp = std::max(fwd_fp32_nrp(k), tc_nrp(k));
    *bytes = job_bytes(H, W, T, k, kc, prec, nrp, &g);
    return ICNNM_OK;
  } catch (StatusFail& f) {
    return report(c, f);
  }
}

icnnm_status icnnm_check_bounded_wait(icnnm_ctx* c, int64_t limit_ns) {
  if (!c) return ICNNM_EINVAL;
  if (limit_ns < 1000000 || limit_ns > 10000000000ll) {
    set_err(c, "limit_ns must be in [1e6, 1e10]");
    return ICNNM_EINVAL;
  }
  std::lock_guard<std::recursive_mutex> g(c->mu);
  try {
    CK(cudaSetDevice(c->device));
    int* d = (int*)dalloc_async(c, sizeof(int), c->stream);
    CK(cudaMemsetAsync(d, 0, sizeof(int), c->stream));
    CK(tc_bounded_wait_check((uint64_t)limit_ns, d, c->stream));
    int h = 0;
    CK(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    dfree_async(d, c->stream);
    CK(cudaStreamSynchronize(c->stream));
    if (h) fail(ICNNM_ETIMEOUT, "the bounded wait expired (expected: nothing completes its barrier)");
    return ICNNM_OK;
  } catch (StatusFail& f) {
    return report(c, f);
  } catch (CudaFail& f) {
    return report(c, f);
  }
}

icnnm_status icnnm_cancel(icnnm_ctx* c, uint64_t id) {
  if (!c) return ICNNM_EINVAL;
  std::lock_guard<std::mutex> lk(c->qmu);
  auto it = c->jobs.find(id);
  if (it == c->jobs.end()) return ICNNM_ENOTFOUND;
  it->second->cancel = true;
  c->qcv.notify_all();
  return ICNNM_OK;
}

}  // extern "C"
