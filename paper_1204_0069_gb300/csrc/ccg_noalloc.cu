// ccg_noalloc.cu -- ccg_solve_noalloc: the persistent FP64 solve run on a
// scratch area that lives in a file-scope device array, for callers that
// cannot allocate device memory while they run (their memory may be owned by
// a pool or a fixed budget, or an allocation's implicit synchronisation may
// be unacceptable).  Nothing here calls cudaMalloc, cudaFree, a pinned-host
// allocation or an event constructor.  The kernel is the same one ccg_solve
// launches; only where its scratch comes from differs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "ccg.h"
#include "ccg_internal.h"

namespace {

constexpr int kNoallocMaxCtas = 160;
constexpr size_t kBlockBytes = (size_t)CCG_NOALLOC_MAX_NP * sizeof(double);
constexpr size_t kPartBytes = (size_t)kNoallocMaxCtas * ccg::kPartStride * sizeof(double);
constexpr size_t kStateBytes = (sizeof(ccg::DevState) + 255) / 256 * 256;
constexpr size_t kScratchBytes = 5 * kBlockBytes + kPartBytes + kStateBytes;

// The scratch area (about 10.7 MB).  Every call on a device uses it, in this
// layout: X, R, D0, D1, W (CCG_NOALLOC_MAX_NP doubles each), the per-CTA
// partial sums, then the solver state.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];
std::once_flag g_scratch_once[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];

// Device address of g_scratch on the current device (looked up once per
// device; the name alone is a host-side stand-in, not a device address).
cudaError_t scratch_address(int device, void** out) {
  std::call_once(g_scratch_once[device], [device]() {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    g_scratch_err[device] = e;
    g_scratch_addr[device] = (e == cudaSuccess) ? p : nullptr;
  });
  *out = g_scratch_addr[device];
  return g_scratch_err[device];
}

bool on_device(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) &&
         a.device == device;
}

}  // namespace

extern "C" int ccg_solve_noalloc(int device, void* stream, int64_t n, const double* A,
                                 int64_t lda, const double* b, const double* x0, int p,
                                 double tol, int maxit, double* x_out, ccg_result* res) {
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->agent = -1;
  }
  auto fail = [&](int st) {
    if (res) res->status = st;
    return st;
  };
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return fail(CCG_ERR_CUDA);
  }
  if (device < 0 || device >= ndev || device >= kMaxDevices) return fail(CCG_ERR_INVALID);
  if (n < 1 || p < 1 || p > ccg::kMaxP || p > n || lda < n || !(tol > 0.0) ||
      !std::isfinite(tol) || maxit < 0 || !A || !b || !x_out)
    return fail(CCG_ERR_INVALID);
  if (n * (int64_t)p > CCG_NOALLOC_MAX_NP) return fail(CCG_ERR_INVALID);

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (cudaSetDevice(device) != cudaSuccess) return fail(CCG_ERR_CUDA);
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev};

  for (const void* ptr : {(const void*)A, (const void*)b, (const void*)x0, (const void*)x_out})
    if (ptr && ((reinterpret_cast<uintptr_t>(ptr) % 8) != 0 || !on_device(ptr, device)))
      return fail(CCG_ERR_INVALID);

  void* base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess || base == nullptr) return fail(CCG_ERR_CUDA);
  char* sc = static_cast<char*>(base);

  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return fail(CCG_ERR_CUDA);
  int64_t g = std::min<int64_t>(std::min<int64_t>(sms, kNoallocMaxCtas),
                                (n + ccg::kWarps - 1) / ccg::kWarps);
  const int G = (int)std::max<int64_t>(1, g);
  const int P = ccg::p_bucket(p);
  const bool vec = (lda % 2 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  if (ccg::fp64_ctas_per_sm(P, vec) < 1) return fail(CCG_ERR_CUDA);

  ccg::Params prm{};
  prm.n = n;
  prm.lda = lda;
  prm.A = A;
  prm.b = b;
  prm.x0 = x0;
  prm.X0 = nullptr;
  prm.spread = 1.0;
  prm.seed = 0;
  prm.X = reinterpret_cast<double*>(sc + 0 * kBlockBytes);
  prm.R = reinterpret_cast<double*>(sc + 1 * kBlockBytes);
  prm.D0 = reinterpret_cast<double*>(sc + 2 * kBlockBytes);
  prm.D1 = reinterpret_cast<double*>(sc + 3 * kBlockBytes);
  prm.W = reinterpret_cast<double*>(sc + 4 * kBlockBytes);
  prm.part = reinterpret_cast<double*>(sc + 5 * kBlockBytes);
  prm.st = reinterpret_cast<ccg::DevState*>(sc + 5 * kBlockBytes + kPartBytes);
  prm.x_out = x_out;
  prm.X_out = nullptr;
  prm.p = p;
  prm.maxit = maxit;
  prm.tol = tol;
  prm.rank_tol = 1e-12;
  prm.replacement = 1;
  prm.mode = ccg::MODE_SOLVE;
  prm.timeout_ns = 10000LL * 1000000LL;
  prm.expected_ctas = (unsigned)G;

  // Solver state: zeroed, then the fields that do not start at zero.  The
  // leading part of the state (counters, agent map) is staged through a
  // state object on the stack (about 60 KB; no heap memory).
  constexpr size_t kHead = offsetof(ccg::DevState, s);
  ccg::DevState hstate;
  std::memset(&hstate, 0, sizeof(hstate));
  ccg::DevState* hs = &hstate;
  hs->pk = p;
  hs->prev_pk = p;
  hs->k_replaced = -1;
  for (int j = 0; j < ccg::kMaxP; ++j) hs->agent[j] = j;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(prm.st, 0, sizeof(ccg::DevState), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(prm.st, hs, kHead, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = ccg::launch_fp64(prm, P, vec, G, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs, prm.st, kHead, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CCG_ERR_CUDA);
  }
  const int status = hs->error != 0 ? hs->error : hs->result;
  if (res) {
    res->status = status;
    res->iterations = hs->k;
    res->agent = (hs->error == 0) ? hs->agent[hs->jbest] : -1;
    res->p_final = hs->pk;
    res->replacements = hs->replacements;
    res->drops = hs->drops;
    res->relres_true = hs->relres_true;
    res->relres_recur = hs->relres_recur;
    res->device_ms = 0.f;
    res->ctas = G;
  }
  return status;
}
