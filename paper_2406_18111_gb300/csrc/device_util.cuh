// Device helpers: decoupled look-back status words and block-wide scans.
//
// Decoupled look-back (Merrill & Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", NVIDIA TR 2016): each tile publishes its
// aggregate, then walks back over its predecessors' status words until it
// meets an inclusive prefix.  A status word packs the state in bits 63:62
// (0 = not yet published, 1 = aggregate, 2 = inclusive prefix), a 30-bit
// launch epoch in bits 61:32 and a 32-bit value, so one 64-bit store
// publishes both the flag and the payload and the array never needs
// clearing between launches (a word from another launch has another epoch).
#pragma once

#include <stdint.h>

#include "apo_internal.cuh"

namespace apo {

enum : uint32_t { kLbNone = 0, kLbAggregate = 1, kLbInclusive = 2 };

__device__ __forceinline__ uint64_t lb_pack(uint32_t state, uint32_t epoch, uint32_t value) {
  return ((uint64_t)state << 62) | ((uint64_t)(epoch & 0x3fffffffu) << 32) | value;
}

__device__ __forceinline__ void lb_store(uint64_t *p, uint64_t w) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ uint64_t lb_load(const uint64_t *p) {
  uint64_t w;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}

struct OpSum {
  __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; }
};
struct OpMax {
  __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a > b ? a : b; }
};

// Combine the published values of tiles t-1, t-2, ... (words at
// status[j * stride]) until an inclusive one is found, in index order (the
// operator need not commute).  Bounded: after
// kSpinLimit polls of a word that is not ready the wait gives up, records
// kDevTimeout in *err and returns what it has (the launch's results are then
// invalid and the host reports APO_ETIMEOUT).
template <class Op>
__device__ uint32_t lb_exclusive(const uint64_t *status, int stride, uint32_t t, uint32_t epoch,
                                 Op op, uint32_t identity, uint32_t *err) {
  uint32_t acc = identity;
  long long j = (long long)t - 1;
  uint32_t spins = 0;
  while (j >= 0) {
    uint64_t w = lb_load(status + (size_t)j * stride);
    uint32_t st = (uint32_t)(w >> 62);
    uint32_t ep = (uint32_t)(w >> 32) & 0x3fffffffu;
    if (ep != epoch || st == kLbNone) {
      if (++spins > kSpinLimit) {
        atomicExch(err, kDevTimeout);
        break;
      }
      if (spins > 32) __nanosleep(128);
      continue;
    }
    acc = op((uint32_t)w, acc);  // tile j precedes the tiles already combined
    if (st == kLbInclusive) break;
    --j;
  }
  return acc;
}

// The same walk with K predecessor words loaded at once (K loads in flight
// instead of one dependent load per step).  The words nearer than the first
// one that is not ready are combined and the walk moves past them; it ends at
// the first inclusive word.
template <int K, class Op>
__device__ uint32_t lb_exclusive_k(const uint64_t *status, int stride, uint32_t t, uint32_t epoch, Op op,
                                   uint32_t identity, uint32_t *err) {
  uint32_t acc = identity;
  long long hi = (long long)t - 1;
  uint32_t spins = 0;
  while (hi >= 0) {
    uint64_t w[K];
#pragma unroll
    for (int i = 0; i < K; ++i) w[i] = hi - i >= 0 ? lb_load(status + (size_t)(hi - i) * stride) : 0ull;
    uint32_t part = identity;
    int used = 0;
    bool done = false;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (done || used < i) continue;  // stop at the first word not ready
      if (hi - i < 0) {
        done = true;
        continue;
      }
      const uint32_t st = (uint32_t)(w[i] >> 62), ep = (uint32_t)(w[i] >> 32) & 0x3fffffffu;
      if (ep != epoch || st == kLbNone) continue;
      part = op((uint32_t)w[i], part);  // tile hi - i precedes the tiles in part
      used = i + 1;
      if (st == kLbInclusive) done = true;
    }
    acc = op(part, acc);
    if (done) break;
    hi -= used;
    if (used == 0) {
      if (++spins > kSpinLimit) {
        atomicExch(err, kDevTimeout);
        break;
      }
      if (spins > 32) __nanosleep(128);
    }
  }
  return acc;
}

// The same walk by a whole warp, for a commutative operator: lane l reads
// the word of tile hi - l, so 32 predecessors are combined per step instead
// of one.  Every lane of the warp must call it; all receive the result.
// The words nearer than the first inclusive one must all be published
// before the step is taken; otherwise the warp polls them again (bounded as
// above, then kDevTimeout).
template <class Op>
__device__ uint32_t lb_exclusive_warp(const uint64_t *status, int stride, uint32_t t, uint32_t epoch, Op op,
                                      uint32_t identity, uint32_t *err) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t acc = identity;
  long long hi = (long long)t - 1;  // the nearest tile not combined yet
  uint32_t spins = 0;
  while (hi >= 0) {
    const long long j = hi - (long long)lane;
    bool ready = true, incl = true;  // past tile 0: nothing to combine, the walk ends
    uint32_t val = identity;
    if (j >= 0) {
      const uint64_t w = lb_load(status + (size_t)j * stride);
      const uint32_t st = (uint32_t)(w >> 62), ep = (uint32_t)(w >> 32) & 0x3fffffffu;
      ready = ep == epoch && st != kLbNone;
      incl = ready && st == kLbInclusive;
      val = (uint32_t)w;
    }
    const uint32_t incl_mask = __ballot_sync(0xffffffffu, incl);
    const uint32_t first = incl_mask ? (uint32_t)(__ffs(incl_mask) - 1) : 32u;  // nearest inclusive word
    const uint32_t need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
    if (__ballot_sync(0xffffffffu, !ready) & need) {
      if (++spins > kSpinLimit) {
        if (lane == 0) atomicExch(err, kDevTimeout);
        break;
      }
      if (spins > 32) __nanosleep(128);
      continue;
    }
    uint32_t v = (lane <= first && j >= 0) ? val : identity;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    acc = op(acc, v);
    if (first < 32) break;
    hi -= 32;
  }
  return acc;
}

// ---- 1-D bulk copies global -> shared (TMA engine), completed on an
// mbarrier.  Both addresses 16-byte aligned, the size a multiple of 16.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(arrivals) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// The calling thread arrives and announces `bytes` of copies to come.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the barrier to complete.  Bounded: after
// kSpinLimit polls it records kDevTimeout and polls as long again, so that
// a copy still in flight lands before the caller reuses (or gives up) the
// shared memory; the data is then invalid and the host reports the error.
__device__ __forceinline__ void mbar_wait(uint64_t *bar, uint32_t parity, uint32_t *err) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_test(bar, parity)) return;
  atomicExch(err, kDevTimeout);
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_test(bar, parity)) return;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class Op>
__device__ __forceinline__ uint32_t warp_inclusive(uint32_t v, Op op) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v = op(o, v);  // lane - d precedes this lane
  }
  return v;
}

// Block-wide inclusive scan for blocks of NW warps; `scratch` holds NW words.
// Returns the inclusive value; *total receives the block total.
template <int NW, class Op>
__device__ __forceinline__ uint32_t block_inclusive(uint32_t v, Op op, uint32_t identity,
                                                    uint32_t *scratch, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = warp_inclusive(v, op);
  if (lane == 31) scratch[warp] = inc;
  __syncthreads();
  uint32_t pre = identity, tot = identity;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    uint32_t x = scratch[w];
    if (w < warp) pre = op(pre, x);
    tot = op(tot, x);
  }
  __syncthreads();
  *total = tot;
  return op(pre, inc);
}

// Block-wide exclusive scan; *total receives the block total.
template <int NW, class Op>
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, Op op, uint32_t identity,
                                                    uint32_t *scratch, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t inc = warp_inclusive(v, op);
  uint32_t wex = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) wex = identity;
  if (lane == 31) scratch[warp] = inc;
  __syncthreads();
  uint32_t pre = identity, tot = identity;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t x = scratch[w];
    if (w < warp) pre = op(pre, x);
    tot = op(tot, x);
  }
  __syncthreads();
  *total = tot;
  return op(pre, wex);
}

}  // namespace apo
