// apo_greedy_select_noalloc: the greedy selection loop for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs inside a task runtime which owns all device
// memory through its own pool (and treats any outside cudaMalloc as a
// failure), or code on a latency-critical path that must not pay for
// cudaMalloc / cudaFree, which may synchronise the whole device.  Such a
// caller can still hand over candidate arrays and output buffers it owns;
// the only scratch this routine needs, the mark bitmap over window
// positions, lives in a fixed-size array compiled into the library.
//
// The scratch array below is a file-scope __device__ variable: every GPU that
// loads the library holds its 512 KiB until the process exits.  In host code
// its name is only a host-side stand-in, not a device address, so the host
// asks the runtime for the array's device address once per device and passes
// that to the kernel.  All calls share the array and it keeps the previous
// call's contents; the kernel clears the part it uses before using it.  Two
// calls whose kernels overlap on the GPU (e.g. on two streams) race on it.
#include <mutex>

#include "apo_internal.cuh"

namespace {

constexpr uint32_t kMaxWindow = APO_NOALLOC_MAX_WINDOW;  // positions covered by the bitmap
static __device__ __align__(256) uint32_t g_noalloc_marks[kMaxWindow / 32];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_marks_dev[kMaxDevices] = {};  // device address of g_noalloc_marks, per device

constexpr int kT = 1024;

__device__ __forceinline__ bool is_marked(const uint32_t *bits, uint32_t x) {
  const uint32_t w = *(volatile const uint32_t *)(bits + (x >> 5));
  return (w >> (x & 31)) & 1u;
}

// One block visits the candidates in order, 1024 at a time: those whose first
// or last position is already marked are rejected in parallel (lengths never
// increase along the order, so that test is exact), and one warp settles the
// remaining ones in order, marking each accepted interval.  A length that
// increases along the order breaks that exactness; it is detected and
// reported as a count of 0xffffffff.
__global__ void __launch_bounds__(kT, 1) k_greedy_noalloc(const uint32_t *__restrict__ cl,
                                                          const uint32_t *__restrict__ cs,
                                                          uint32_t m, uint32_t n, uint32_t *bits,
                                                          uint8_t *acc, uint32_t *count) {
  __shared__ uint32_t s_l[kT], s_s[kT], s_k[kT];
  __shared__ uint32_t s_wc[32], s_off[32], s_total;
  __shared__ int s_rising;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_rising = 0;
  for (uint32_t w = tid; w < (n + 31) / 32; w += kT) bits[w] = 0;  // left over from the last call
  uint32_t nacc = 0;
  __syncthreads();
  for (uint32_t base = 0; base < m; base += kT) {
    const uint32_t k = base + tid;
    bool surv = false;
    uint32_t l = 0, s = 0;
    if (k < m) {
      l = cl[k];
      s = cs[k];
      acc[k] = 0;
      if (k > 0 && l > cl[k - 1]) s_rising = 1;
      surv = l > 0 && (uint64_t)s + l <= n && !is_marked(bits, s) && !is_marked(bits, s + l - 1);
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, surv);
    if (lane == 0) s_wc[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
      const uint32_t c = s_wc[lane];
      uint32_t inc = c;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
      }
      s_off[lane] = inc - c;
      if (lane == 31) s_total = inc;
    }
    __syncthreads();
    if (surv) {
      const uint32_t q = s_off[warp] + __popc(bal & ((1u << lane) - 1u));
      s_l[q] = l;
      s_s[q] = s;
      s_k[q] = k;
    }
    __syncthreads();
    if (warp == 0) {
      const uint32_t total = s_total;
      for (uint32_t q = 0; q < total; ++q) {
        const uint32_t qs = s_s[q], qe = qs + s_l[q] - 1;
        if (!is_marked(bits, qs) && !is_marked(bits, qe)) {
          const uint32_t w0 = qs >> 5, w1 = qe >> 5;
          for (uint32_t w = w0 + lane; w <= w1; w += 32) {
            uint32_t msk = 0xffffffffu;
            if (w == w0) msk &= 0xffffffffu << (qs & 31);
            if (w == w1) msk &= 0xffffffffu >> (31 - (qe & 31));
            bits[w] |= msk;
          }
          if (lane == 0) {
            acc[s_k[q]] = 1;
            ++nacc;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (tid == 0) *count = s_rising ? 0xffffffffu : nacc;
}

}  // namespace

extern "C" int apo_greedy_select_noalloc(const uint32_t *cand_len, const uint32_t *cand_start,
                                         uint64_t m, uint64_t n, uint8_t *accepted,
                                         uint32_t *accepted_count, void *stream) {
  if (n > kMaxWindow) {
    apo::set_error("apo_greedy_select_noalloc: window of " + std::to_string(n) +
                   " positions exceeds the fixed maximum of " + std::to_string(kMaxWindow));
    return APO_EINVAL;
  }
  if (m >= 0xffffffffull) {
    apo::set_error("apo_greedy_select_noalloc: too many candidates");
    return APO_EINVAL;
  }
  if (!accepted_count || (m > 0 && (!cand_len || !cand_start || !accepted))) {
    apo::set_error("apo_greedy_select_noalloc: null pointer argument");
    return APO_EINVAL;
  }
  int dev = 0;
  APO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    apo::set_error("apo_greedy_select_noalloc: device ordinal out of range");
    return APO_EINVAL;
  }
  uint32_t *marks = nullptr;
  {
    // Set-up, once per device, on the current device: the device address of
    // the scratch array (its name is not an address in host code).
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_marks_dev[dev]) {
      void *p = nullptr;
      APO_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_marks));
      g_marks_dev[dev] = static_cast<uint32_t *>(p);
    }
    marks = g_marks_dev[dev];
  }
  k_greedy_noalloc<<<1, kT, 0, static_cast<cudaStream_t>(stream)>>>(
      cand_len, cand_start, (uint32_t)m, (uint32_t)n, marks, accepted, accepted_count);
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}
