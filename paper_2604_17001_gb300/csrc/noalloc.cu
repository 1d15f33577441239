// icnnm_learn_V_noalloc: learning V (the same Gram accumulation and FP64 Jacobi
// eigensolver as icnnm_learn_V) without allocating any memory.
//
// For callers that cannot call cudaMalloc themselves: code inside a host framework that
// hands out device memory only from its own pool (an allocation behind its back would
// break its accounting or fail against its reservation), or latency-bound code that must
// not trigger the device-wide synchronisation a cudaMalloc/cudaFree can cause. The caller
// passes device-resident inputs and outputs on the current device; every intermediate
// lives in one file-scope device array of fixed size (about 2.1 MiB) that every GPU that
// loads this library holds until the process exits. The call is blocking (it
// synchronises the caller's stream).
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/icnnm.h"
#include "icnnm_internal.h"

namespace {

constexpr int NA_MAXK = 256;      // k = k1*k2*k3
constexpr int NA_MAXLAG = 4096;   // (2k1-1)(2k2-1)(2k3-1)
constexpr int NA_NBLK = 16;       // autocorrelation blocks per tensor
constexpr int NA_MAXB = 256;      // reference tensors per call
constexpr int NA_MAXDEV = 64;

struct Scratch {
  double part[NA_NBLK * NA_MAXLAG];
  double lagsum[NA_MAXLAG];
  double gram[NA_MAXK * NA_MAXK];
  double vacc[NA_MAXK * NA_MAXK];
  double vout[NA_MAXK * NA_MAXK];
  double evals[NA_MAXK];
  const float* ptrs[NA_MAXB];
  int dims[3 * NA_MAXB];
  int info;
  int bad;
};

// The scratch array. In host code `g_scratch` names a host-side stand-in, not device
// memory; kernels get the device address that cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_scratch[sizeof(Scratch)];

std::mutex g_setup_mu;
Scratch* g_addr[NA_MAXDEV] = {};

// Once per device, with that device current: look up the device address of g_scratch.
cudaError_t scratch_address(Scratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAXDEV) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<Scratch*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

thread_local char g_err[256];

icnnm_status fail(icnnm_status st, const char* msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return st;
}

// 1: device (or managed) memory of device `dev`; 0: host memory; -1: device memory of
// another device (the kernels would dereference a peer address).
int where(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return 0;
  return a.device == dev ? 1 : -1;
}

}  // namespace

extern "C" const char* icnnm_noalloc_last_error(void) { return g_err; }

extern "C" icnnm_status icnnm_learn_V_noalloc(const int64_t kdims[3], int32_t b, const icnnm_shape* shapes,
                                             const float* const* tensors, double* V_out, double* eig_out,
                                             void* cuda_stream) {
  using namespace icnnm;
  g_err[0] = 0;
  if (!kdims || !shapes || !tensors || !V_out) return fail(ICNNM_EINVAL, "NULL argument");
  const int k1 = (int)kdims[0], k2 = (int)kdims[1], k3 = (int)kdims[2];
  if (k1 < 1 || k2 < 1 || k3 < 1) return fail(ICNNM_EINVAL, "kdims must be >= 1");
  const long long k = (long long)k1 * k2 * k3;
  const long long nlag = (long long)(2 * k1 - 1) * (2 * k2 - 1) * (2 * k3 - 1);
  if (k > NA_MAXK) return fail(ICNNM_EINVAL, "k = k1*k2*k3 exceeds the static scratch limit of 256");
  if (nlag > NA_MAXLAG) return fail(ICNNM_EINVAL, "(2k1-1)(2k2-1)(2k3-1) exceeds the static scratch limit of 4096");
  if (b < 1 || b > NA_MAXB) return fail(ICNNM_EINVAL, "b must be in [1, 256]");
  if (learn_smem_bytes(k1, k2, k3) > 220 * 1024)
    return fail(ICNNM_EUNSUPPORTED, "the Gram halo of this kernel needs more than 220 KiB of shared memory");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  int ptrsdims[3 * NA_MAXB];
  for (int j = 0; j < b; ++j) {
    const icnnm_shape& s = shapes[j];
    if (s.ndim != 2 && s.ndim != 3) return fail(ICNNM_EINVAL, "ndim must be 2 or 3");
    const int H = (int)s.dims[0], W = (int)s.dims[1], T = s.ndim == 3 ? (int)s.dims[2] : 1;
    if (H < k1 || W < k2 || T < k3) return fail(ICNNM_EINVAL, "every dim must be at least the kernel's");
    if (!tensors[j] || where(tensors[j], dev) != 1)
      return fail(ICNNM_EINVAL, "reference tensors must be device memory of the current device");
    ptrsdims[3 * j] = H; ptrsdims[3 * j + 1] = W; ptrsdims[3 * j + 2] = T;
  }
  const int vw = where(V_out, dev), ew = eig_out ? where(eig_out, dev) : 0;
  if (vw < 0 || ew < 0) return fail(ICNNM_EINVAL, "V_out and eig_out must be host memory or memory of the current device");
  const bool vdev = vw == 1, edev = ew == 1;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Scratch* S = nullptr;
  e = scratch_address(&S);
  if (e != cudaSuccess) return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  // inputs of this call into the shared scratch (plain copies; nothing is allocated)
  if ((e = cudaMemcpyAsync(S->ptrs, tensors, sizeof(float*) * b, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(S->dims, ptrsdims, sizeof(int) * 3 * b, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(&S->bad, 0, sizeof(int), st)) != cudaSuccess)
    return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  for (int j = 0; j < b; ++j) {
    const long long m = (long long)ptrsdims[3 * j] * ptrsdims[3 * j + 1] * ptrsdims[3 * j + 2];
    if ((e = check_finite(tensors[j], m, &S->bad, st)) != cudaSuccess) return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  }
  int bad = 0;
  if ((e = cudaMemcpyAsync(&bad, &S->bad, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  if (bad) return fail(ICNNM_EINVAL, "a reference tensor has a non-finite entry");
  // lagsum starts at zero with the first tensor; the Jacobi kernel initialises vacc
  if ((e = learn_gram_streamed(b, S->ptrs, S->dims, k1, k2, k3, S->part, NA_NBLK, S->lagsum, S->gram, st)) !=
      cudaSuccess)
    return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  double* vdst = vdev ? V_out : S->vout;
  double* edst = edev ? eig_out : S->evals;
  if ((e = cudaMemsetAsync(&S->info, 0, sizeof(int), st)) != cudaSuccess ||
      (e = learn_eig(S->gram, S->vacc, (int)k, edst, vdst, &S->info, st)) != cudaSuccess)
    return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  int info = 0;
  if ((e = cudaMemcpyAsync(&info, &S->info, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  if (!vdev && (e = cudaMemcpyAsync(V_out, S->vout, sizeof(double) * k * k, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  if (eig_out && !edev &&
      (e = cudaMemcpyAsync(eig_out, S->evals, sizeof(double) * k, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(ICNNM_ECUDA, cudaGetErrorString(e));
  if (info < 0) return fail(ICNNM_ENOCONV, "the FP64 Jacobi eigensolver did not converge within 30 sweeps");
  return ICNNM_OK;
}
