// Task hashing: Alg. 1 Hash(T) (Sec. 4.1) -- a task and its region
// arguments become one 64-bit token, so that tasks which would be analysed
// identically compare equal.  FNV-1a 64 (Fowler, Noll, Vo; offset basis
// 0xcbf29ce484222325, prime 0x100000001b3) over the little-endian bytes of
// task_id:u32, nargs:u32 and, per argument in issue order, region:u32,
// field_mask:u64, priv:u8.
//
// One thread hashes one task.  FNV is a serial chain per task, so the
// parallelism is across tasks; the descriptor arrays are read once.
#include <algorithm>

#include "apo_internal.cuh"

namespace apo {

namespace {

constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull;
constexpr uint64_t kFnvPrime = 0x100000001b3ull;

template <int kBytes>
__device__ __forceinline__ uint64_t fnv_le(uint64_t h, uint64_t v) {
#pragma unroll
  for (int b = 0; b < kBytes; ++b) {
    h ^= (v >> (8 * b)) & 0xffu;
    h *= kFnvPrime;
  }
  return h;
}

__global__ void __launch_bounds__(256) k_hash_tasks(uint64_t N, const uint32_t *__restrict__ task_id,
                                                    const uint32_t *__restrict__ arg_off,
                                                    const uint32_t *__restrict__ region,
                                                    const uint64_t *__restrict__ mask,
                                                    const uint8_t *__restrict__ priv,
                                                    uint64_t *__restrict__ out) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t lo = arg_off[t], hi = arg_off[t + 1];
    uint64_t h = fnv_le<4>(kFnvBasis, task_id[t]);
    h = fnv_le<4>(h, hi - lo);
    for (uint32_t a = lo; a < hi; ++a) {
      h = fnv_le<4>(h, region[a]);
      h = fnv_le<8>(h, mask[a]);
      h = fnv_le<1>(h, priv[a]);
    }
    out[t] = h;
  }
}

}  // namespace

void launch_hash_tasks(apo_ctx *c, const apo_tasks *t, uint64_t *out, cudaStream_t s) {
  const int sms = c->num_sms;
  const uint64_t N = t->n_tasks;
  const long long blocks = std::min<long long>((long long)((N + 255) / 256), (long long)sms * 8);
  {
    Launch lp_(c, kKHash, N, s);
    k_hash_tasks<<<(int)std::max<long long>(1, blocks), 256, 0, s>>>(
        N, t->task_id, t->arg_off, t->region, t->field_mask, t->priv, out);
  }
}

}  // namespace apo
