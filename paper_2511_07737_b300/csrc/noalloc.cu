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
static void *g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
static int scratch_address(int32_t **out) {
  int dev = 0;
  TSAT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device %d beyond the no-alloc table", dev);
    return TSAT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    TSAT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<int32_t *>(g_scratch_ptr[dev]);
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
