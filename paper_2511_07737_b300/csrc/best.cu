// best.cu -- hand-off selection (Sec. IV-B) for one instance:
//   sample choice (fewest unsatisfied clauses, lowest index), the STE gradient
//   of that sample's current bits, the k variables with the smallest
//   |gradient| (ties to the lower variable) by a 4 x 16-bit radix select on
//   unique 64-bit keys (|G| bits : variable), and the sample's full bits.
#include <algorithm>

#include "kernels.cuh"

namespace tsat {

__device__ __forceinline__ const uint32_t *cur_bits_b(const StateDev &sd) {
  return sd.bits + (size_t)(sd.hdr->t & 1) * (size_t)sd.V * sd.W;
}

// small[0] = chosen sample, small[1] = its unsat count, small[2] = selected count
__global__ void k_pick(const int32_t *unsat, int N, int32_t *small) {
  __shared__ int32_t su[32], si[32];
  int32_t mu = 0x7FFFFFFF, mi = 0x7FFFFFFF;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    int32_t u = unsat[i];
    if (u < mu || (u == mu && i < mi)) { mu = u; mi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    int32_t u2 = __shfl_xor_sync(0xFFFFFFFFu, mu, o), i2 = __shfl_xor_sync(0xFFFFFFFFu, mi, o);
    if (u2 < mu || (u2 == mu && i2 < mi)) { mu = u2; mi = i2; }
  }
  if ((threadIdx.x & 31) == 0) { su[threadIdx.x >> 5] = mu; si[threadIdx.x >> 5] = mi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (su[w] < mu || (su[w] == mu && si[w] < mi)) { mu = su[w]; mi = si[w]; }
    small[0] = mi;
    small[1] = mu;
    small[2] = 0;
  }
}

// Histogram of R_c,i* over the instance's clauses (Eq. 1 for one sample).
__global__ void k_hist1(ProbDev pd, StateDev sd, int inst, const int32_t *small, int32_t *hist1) {
  __shared__ int32_t sh[32];
  if (threadIdx.x < 32) sh[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t *bits = cur_bits_b(sd);
  const int i = small[0], word = i >> 5, bit = i & 31;
  const InstInfo I = pd.inst[inst];
  for (int64_t c = I.c_off + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < I.c_off + I.n_clauses;
       c += (int64_t)gridDim.x * blockDim.x) {
    int r = 0;
    for (int32_t j = pd.cptr[c]; j < pd.cptr[c + 1]; ++j) {
      const int32_t lit = pd.clit[j];
      r += (int)(((bits[(size_t)(lit >> 1) * sd.W + word] >> bit) & 1u) ^ (uint32_t)(lit & 1));
    }
    atomicAdd(&sh[r], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32 && sh[threadIdx.x]) atomicAdd(hist1 + threadIdx.x, sh[threadIdx.x]);
}

// G_v,i* (STE, Sec. III-B) for every variable of the instance.
__global__ void k_gcol(ProbDev pd, StateDev sd, Hyper hy, int inst, const int32_t *small, const int32_t *hist1,
                       float *gcol) {
  __shared__ float gt[32];
  const InstInfo I = pd.inst[inst];
  if (threadIdx.x == 0) {
    float Z = 0.f, Y = 0.f;
    for (int r = 0; r <= I.lmax; ++r) {
      float e = expf(-hy.tau * (float)r), h = (float)hist1[r];
      Z += h * e;
      Y += (float)r * h * e;
    }
    const float S = Y / Z;
    for (int r = 0; r < 32; ++r)
      gt[r] = (r <= I.lmax) ? -(expf(-hy.tau * (float)r) / Z) * (1.0f - hy.tau * ((float)r - S)) : 0.f;
  }
  __syncthreads();
  const uint32_t *bits = cur_bits_b(sd);
  const int i = small[0], word = i >> 5, bit = i & 31;
  for (int64_t vl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; vl < I.n_vars;
       vl += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = I.v_off + vl;
    const uint32_t own = (bits[(size_t)v * sd.W + word] >> bit) & 1u;
    float G = 0.f;
    for (int64_t p = pd.xptr[v]; p < pd.xptr[v + 1];) {
      const int32_t h = pd.xrec[p];
      if (h == 0) break;
      const int len = h >> 1;
      int r = (int)(own ^ (uint32_t)(h & 1));
      for (int q = 1; q < len; ++q) {
        const int32_t lit = pd.xrec[p + q];
        r += (int)(((bits[(size_t)(lit >> 1) * sd.W + word] >> bit) & 1u) ^ (uint32_t)(lit & 1));
      }
      G += (h & 1) ? -gt[r] : gt[r];
      p += pd.rec_stride ? pd.rec_stride : len;
    }
    gcol[vl] = G;
  }
}

__device__ __forceinline__ unsigned long long conf_key(const float *gcol, int64_t vl) {
  return ((unsigned long long)__float_as_uint(fabsf(gcol[vl])) << 32) | (unsigned long long)vl;
}

// selstate[0] = key prefix, selstate[1] = rank still to find (1-based)
__global__ void k_digit_hist(const float *gcol, int64_t n, int pass, const int64_t *selstate, int32_t *digits) {
  const unsigned long long prefix = (unsigned long long)selstate[0];
  const int hi_shift = 64 - 16 * pass;
  const int sh = 48 - 16 * pass;
  for (int64_t vl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; vl < n; vl += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = conf_key(gcol, vl);
    if (pass > 0 && (key >> hi_shift) != (prefix >> hi_shift)) continue;
    atomicAdd(digits + ((key >> sh) & 0xFFFFull), 1);
  }
}

__global__ void k_digit_pick(int32_t *digits, int pass, int64_t *selstate) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x;
  const int64_t krem = selstate[1];
  __syncthreads();
  int64_t s = 0;
  for (int k = 0; k < 64; ++k) s += digits[tid * 64 + k];
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t y = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += y;
    __syncthreads();
  }
  const int64_t excl = part[tid] - s;
  if (excl < krem && part[tid] >= krem) {  // exactly one thread
    int64_t run = excl;
    for (int k = 0; k < 64; ++k) {
      const int64_t d = digits[tid * 64 + k];
      if (run + d >= krem) {
        const unsigned long long digit = (unsigned long long)(tid * 64 + k);
        selstate[0] = (int64_t)((unsigned long long)selstate[0] | (digit << (48 - 16 * pass)));
        selstate[1] = krem - run;
        break;
      }
      run += d;
    }
  }
  __syncthreads();
  for (int k = 0; k < 64; ++k) digits[tid * 64 + k] = 0;
}

__global__ void k_collect(const float *gcol, int64_t n, const int64_t *selstate, unsigned long long *sel,
                          int32_t *small, int k) {
  const unsigned long long T = (unsigned long long)selstate[0];
  for (int64_t vl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; vl < n; vl += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = conf_key(gcol, vl);
    if (key <= T) {
      const int idx = atomicAdd(small + 2, 1);
      if (idx < k) sel[idx] = key;  // keys are unique, so exactly k pass; the host checks the count
    }
  }
}

// rank-order the k selected keys; outputs 1-based variables and their values
__global__ void k_sort_sel(ProbDev pd, StateDev sd, int inst, int k, const unsigned long long *sel,
                           const int32_t *small, int32_t *part_var, uint8_t *part_val) {
  const uint32_t *bits = cur_bits_b(sd);
  const int i = small[0];
  const int64_t v_off = pd.inst[inst].v_off;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
    const unsigned long long key = sel[a];
    int rank = 0;
    for (int b = 0; b < k; ++b) rank += sel[b] < key;
    const int64_t vl = (int64_t)(key & 0xFFFFFFFFull);
    part_var[rank] = (int32_t)(vl + 1);
    part_val[rank] = (uint8_t)((bits[(size_t)(v_off + vl) * sd.W + (i >> 5)] >> (i & 31)) & 1u);
  }
}

__global__ void k_extract_bits(ProbDev pd, StateDev sd, int inst, const int32_t *small, uint32_t *out) {
  const uint32_t *bits = cur_bits_b(sd);
  const int i = small[0];
  const InstInfo I = pd.inst[inst];
  const int64_t nround = ((int64_t)I.n_vars + 31) / 32 * 32;
  for (int64_t vl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; vl < nround;
       vl += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b = 0;
    if (vl < I.n_vars) b = (bits[(size_t)(I.v_off + vl) * sd.W + (i >> 5)] >> (i & 31)) & 1u;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, b);
    if ((threadIdx.x & 31) == 0) out[vl >> 5] = m;
  }
}

// launch wrappers used by tsat_best (api.cu)
cudaError_t best_pick(const int32_t *unsat, int N, int32_t *small, cudaStream_t st) {
  k_pick<<<1, 1024, 0, st>>>(unsat, N, small);
  return cudaGetLastError();
}
cudaError_t best_gcol(const ProbDev &pd, const StateDev &sd, const Hyper &hy, int inst, int n_vars, int n_clauses,
                      const int32_t *small, int32_t *hist1, float *gcol, cudaStream_t st) {
  const int gc = (int)std::min<int64_t>(4096, ((int64_t)n_clauses + 255) / 256);
  k_hist1<<<gc, 256, 0, st>>>(pd, sd, inst, small, hist1);
  const int gv = (int)std::min<int64_t>(4096, ((int64_t)n_vars + 255) / 256);
  k_gcol<<<gv, 256, 0, st>>>(pd, sd, hy, inst, small, hist1, gcol);
  return cudaGetLastError();
}
cudaError_t best_select(const ProbDev &pd, const StateDev &sd, int inst, int n_vars, int k, const float *gcol,
                        unsigned long long *sel, int32_t *digits, int64_t *selstate, int32_t *small,
                        int32_t *part_var, uint8_t *part_val, uint32_t *outbits, cudaStream_t st) {
  const int gv = (int)std::min<int64_t>(4096, ((int64_t)n_vars + 255) / 256);
  for (int pass = 0; pass < 4; ++pass) {
    k_digit_hist<<<gv, 256, 0, st>>>(gcol, n_vars, pass, selstate, digits);
    k_digit_pick<<<1, 1024, 0, st>>>(digits, pass, selstate);
  }
  k_collect<<<gv, 256, 0, st>>>(gcol, n_vars, selstate, sel, small, k);
  k_sort_sel<<<(k + 255) / 256, 256, 0, st>>>(pd, sd, inst, k, sel, small, part_var, part_val);
  k_extract_bits<<<gv, 256, 0, st>>>(pd, sd, inst, small, outbits);
  return cudaGetLastError();
}

}  // namespace tsat
