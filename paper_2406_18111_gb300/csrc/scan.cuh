// Device-wide inclusive scans with an associative (not necessarily
// commutative) operator on 32-bit values: one tile of kGTile elements per
// block, tiles chained by decoupled look-back (device_util.cuh).  Src and Dst
// are functors that produce element i and consume the scanned value of i.
#pragma once

#include <stdint.h>

#include "apo_internal.cuh"
#include "device_util.cuh"

namespace apo {

// Inclusive scan over n elements (in reverse index order when kReverse), one
// kGTile-element tile per block.
constexpr int kGT = 256, kGI = 8, kGTile = kGT * kGI;
template <bool kReverse, class Src, class Op, class Dst>
__global__ void __launch_bounds__(kGT) k_seg_scan(Src src, Dst dst, uint32_t n, Op op, uint32_t ident,
                                                  uint64_t *status, uint32_t *tile_ctr, uint32_t epoch,
                                                  uint32_t *err) {
  __shared__ uint32_t s_tile, s_pre;
  __shared__ uint32_t scr[kGT / 32];
  __shared__ uint32_t sv[kGTile];
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kGTile;
  for (int q = tid; q < kGTile; q += kGT) {
    const uint64_t i = base + q;
    sv[q] = i < n ? src(kReverse ? (uint32_t)(n - 1 - i) : (uint32_t)i) : ident;
  }
  __syncthreads();
  uint32_t run = ident;
#pragma unroll
  for (int i = 0; i < kGI; ++i) run = op(run, sv[tid * kGI + i]);
  uint32_t tot;
  const uint32_t ex = block_exclusive<kGT / 32>(run, op, ident, scr, &tot);
  if (tid == 0) {
    lb_store(&status[t], lb_pack(t == 0 ? kLbInclusive : kLbAggregate, epoch, tot));
    uint32_t pre = ident;
    if (t > 0) {
      pre = lb_exclusive_k<8>(status, 1, t, epoch, op, ident, err);
      lb_store(&status[t], lb_pack(kLbInclusive, epoch, op(pre, tot)));
    }
    s_pre = pre;
  }
  __syncthreads();
  uint32_t r = op(s_pre, ex);
#pragma unroll
  for (int i = 0; i < kGI; ++i) {
    r = op(r, sv[tid * kGI + i]);
    sv[tid * kGI + i] = r;
  }
  __syncthreads();
  for (int q = tid; q < kGTile; q += kGT) {
    const uint64_t i = base + q;
    if (i < n) dst(kReverse ? (uint32_t)(n - 1 - i) : (uint32_t)i, sv[q]);
  }
}

template <bool kReverse, class Src, class Op, class Dst>
int seg_scan(apo_ctx *c, Src src, Dst dst, uint32_t n, Op op, uint32_t ident, cudaStream_t s) {
  if (n == 0) return APO_OK;
  const int tiles = ceil_div(n, kGTile);
  APO_TRY(ensure_lookback(c, tiles));
  uint32_t *ctr = c->ps.counters + kCtrMisc + kMiscCompactTiles;
  APO_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(uint32_t), s));
  Launch lp_(c, kKSegScan, n, s);
  k_seg_scan<kReverse><<<tiles, kGT, 0, s>>>(src, dst, n, op, ident, c->ps.lookback, ctr, next_epoch(c),
                                             c->ps.err);
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

}  // namespace apo
