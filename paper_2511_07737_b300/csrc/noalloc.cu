// noalloc.cu -- an evaluation entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool
// they do not own, processes whose device memory is reserved up front by
// another runtime, or callers in restricted contexts where a late allocation
// could fail or stall.  tsat_evaluate needs a state buffer from the caller
// for its histogram; this variant evaluates a caller-supplied bit matrix with
// its temporaries in a fixed array that lives in the library's device image
// (one copy per GPU, held until the process exits).
#include <mutex>

#include "internal.h"
#include "kernels.cuh"

namespace tsat {

// Header (64 ints) + histogram + per-sample unsatisfied counts + S values.
constexpr int64_t kNoAllocScratchInts = 1 << 20;   // 4 MiB
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocScratchInts];

constexpr int kMaxDevices = 64;
// Per device: the unique id of the context the address was looked up in, and
// the address.
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  void *ptr = nullptr;
};
static ScratchSlot g_scratch[kMaxDevices];
static std::mutex g_scratch_mu;

// The driver's cuCtxGetCurrent and cuCtxGetId, reached through the runtime (no
// link-time dependency on the driver library).  CUcontext is an opaque
// pointer; a context id is never reused within a process, unlike an address.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
struct CtxFns {
  CtxGetCurrentFn current = nullptr;
  CtxGetIdFn id = nullptr;
};
static const CtxFns &ctx_fns() {
  static const CtxFns fns = [] {
    CtxFns f;
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
        qb == cudaDriverEntryPointSuccess) {
      f.current = reinterpret_cast<CtxGetCurrentFn>(a);
      f.id = reinterpret_cast<CtxGetIdFn>(b);
    }
    return f;
  }();
  return fns;
}

// Id of the context current on this thread, 0 if none.
static unsigned long long current_ctx_id() {
  const CtxFns &f = ctx_fns();
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (!f.current || f.current(&ctx) != 0 || !ctx || f.id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in, never a device address, so the address is looked
// up with cudaGetSymbolAddress with the device current, once per device and
// context: a context torn down and made again (cudaDeviceReset) gets a new
// lookup instead of a pointer into the dead context.
static int scratch_address(int32_t **out) {
  int dev = 0;
  TSAT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device %d beyond the no-alloc table", dev);
    return TSAT_EINVAL;
  }
  if (!ctx_fns().current) {
    set_error("cannot reach cuCtxGetCurrent / cuCtxGetId");
    return TSAT_ECUDA;
  }
  unsigned long long id = current_ctx_id();   // 0: no context current on this thread yet
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  ScratchSlot &slot = g_scratch[dev];
  if (!slot.ptr || id == 0 || slot.ctx_id != id) {
    void *p = nullptr;
    // the lookup makes the device's primary context current if none was
    TSAT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if ((id = current_ctx_id()) == 0) {
      set_error("no CUDA context current after the scratch lookup");
      return TSAT_ECUDA;
    }
    slot.ptr = p;
    slot.ctx_id = id;
  }
  *out = static_cast<int32_t *>(slot.ptr);
  return TSAT_OK;
}

}  // namespace tsat

using namespace tsat;

extern "C" int tsat_evaluate_bits_noalloc(const tsat_problem *p, const uint32_t *d_bits, int32_t n_samples, float tau,
                                          int32_t *d_unsat, uint32_t *d_satmask, float *d_loss, cudaStream_t stream) {
  if (!p || !d_bits || !d_unsat || !d_satmask) {
    set_error("NULL argument");
    return TSAT_EINVAL;
  }
  const int32_t N = n_samples;
  if (N < TSAT_MIN_SAMPLES || N > TSAT_MAX_SAMPLES || (N & (N - 1))) {
    set_error("n_samples must be a power of two in [32, 1024], got %d", N);
    return TSAT_EINVAL;
  }
  if (!(tau > 0.f)) {
    set_error("tau must be positive");
    return TSAT_EINVAL;
  }
  const int64_t lm1 = p->lmax + 1, I = p->n_inst;
  const int64_t need = 64 + I * N * (lm1 + 2);
  if (need > kNoAllocScratchInts) {
    set_error("no-alloc evaluation needs %lld scratch ints (n_inst x N x (lmax + 3)); the fixed maximum is %lld",
              (long long)need, (long long)kNoAllocScratchInts);
    return TSAT_ERANGE;
  }
  // the problem's device arrays live on the device it was loaded on; the
  // scratch array and the launches below belong to the current device
  int dev = -1;
  TSAT_CUDA(cudaGetDevice(&dev));
  if (dev != p->device) {
    set_error("the problem was loaded on device %d but device %d is current", p->device, dev);
    return TSAT_EINVAL;
  }
  int32_t *scr = nullptr;
  int rc = scratch_address(&scr);
  if (rc) return rc;
  // scratch layout: [0, 64) header (t = 0 selects d_bits), histogram, unsat, S
  StateHdr *hdr = reinterpret_cast<StateHdr *>(scr);
  int32_t *hist = scr + 64;
  int32_t *unsat_tmp = hist + I * lm1 * N;
  float *S_tmp = reinterpret_cast<float *>(unsat_tmp + I * N);
  StateDev sd{};
  sd.N = N;
  sd.W = N / 32;
  sd.lm1 = (int32_t)lm1;
  sd.layer = TSAT_LAYER_STE;
  sd.hdr = hdr;
  sd.bits = const_cast<uint32_t *>(d_bits);
  sd.unsat = unsat_tmp;
  sd.S = S_tmp;
  sd.V = p->V;
  const ProbDev &pd = p->dev;
  // the array keeps the previous call's contents: zero what must start at zero
  TSAT_CUDA(cudaMemsetAsync(hdr, 0, sizeof(StateHdr), stream));
  TSAT_CUDA(cudaMemsetAsync(d_unsat, 0, sizeof(int32_t) * I * N, stream));
  cudaError_t e = launch_check(pd, sd, d_unsat, d_satmask, stream);
  if (e != cudaSuccess) return cuda_fail(e, "check");
  if (d_loss) {
    TSAT_CUDA(cudaMemsetAsync(hist, 0, sizeof(int32_t) * I * lm1 * N, stream));
    if ((e = launch_fwd_hist(pd, sd, hist, 0, stream)) != cudaSuccess) return cuda_fail(e, "forward");
    Hyper hy{};
    hy.tau = tau;
    LrSched ls{};
    if ((e = launch_gamma(pd, sd, hy, ls, hist, 0, 0, d_loss, S_tmp, stream)) != cudaSuccess)
      return cuda_fail(e, "loss");
  }
  return TSAT_OK;
}
