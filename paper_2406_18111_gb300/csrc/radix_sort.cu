// Onesweep LSD radix sort of (u64 key, u32 value) pairs.
//
// After Adinets & Merrill, "Onesweep: A Faster Least Significant Digit Radix
// Sort for GPUs" (2022): each digit place is scattered by one kernel whose
// tiles learn their global digit offsets through decoupled look-back instead
// of a separate scan pass.  Only the first place's histogram needs its own
// read of the keys; every pass counts the next place's digits of the keys it
// already holds, and each tile turns a histogram into offsets itself.  Within a tile, keys are ranked per warp
// with __match_any_sync (stable: a warp's items are visited in input order),
// staged in shared memory in digit order and written out in runs, so global
// writes are coalesced per digit.
//
// A digit place is described by `place` = shift | (256 if the digit comes
// from the value instead of the key).  Sorting on value digits first and key
// digits after gives a stable sort on the 96-bit composite (key : value).
#include <algorithm>

#include "apo_internal.cuh"
#include "device_util.cuh"

namespace apo {

namespace {

constexpr int kThreads = 256;              // histogram / offsets kernels
constexpr int kWarps = kThreads / 32;
constexpr int kPT = 512;                   // digit-pass kernel: threads per block
constexpr int kPW = kPT / 32;
constexpr int kItems = 8;                  // pairs per thread
constexpr int kTile = kPT * kItems;        // 4096 pairs per tile
constexpr int kRadix = 256;
constexpr int kMaxPass = 12;

struct Places {
  int p[kMaxPass];
  int n;
};

__device__ __forceinline__ uint32_t digit_of(uint64_t k, uint32_t v, int place) {
  const int sh = place & 255;
  return (place & 256) ? ((v >> sh) & 255u) : (uint32_t)((k >> sh) & 255u);
}

// Every place's digit histogram in one read of the keys.  When all lanes of
// a warp hold the same digit (common for the high digits of sorted ranks)
// one add counts the whole warp, so skewed digits do not serialise on one
// shared-memory counter.
__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint64_t *__restrict__ keys,
                                                      const uint32_t *__restrict__ vals, uint32_t n,
                                                      Places pl, uint32_t *__restrict__ hist) {
  __shared__ uint32_t sh[kMaxPass * kRadix];
  for (int i = threadIdx.x; i < pl.n * kRadix; i += kThreads) sh[i] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t b0 = (uint64_t)blockIdx.x * kThreads + (threadIdx.x & ~31u); b0 < n; b0 += stride) {
    const uint64_t i = b0 + lane;
    const bool valid = i < n;
    const uint64_t k = valid ? keys[i] : 0;
    const uint32_t v = valid ? vals[i] : 0;
    for (int p = 0; p < pl.n; ++p) {
      const uint32_t d = valid ? digit_of(k, v, pl.p[p]) : 256u;
      const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
      if (__all_sync(0xffffffffu, d == d0 && d0 < 256u)) {
        if (lane == 0) atomicAdd(&sh[p * kRadix + d0], 32u);
      } else if (valid) {
        atomicAdd(&sh[p * kRadix + d], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < pl.n * kRadix; i += kThreads)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// One digit place.  `gcnt` is this place's global digit histogram (the
// tile turns it into digit offsets itself); when next_place >= 0 the tile
// also counts the next place's digits of its keys into next_cnt, so no
// separate histogram read is needed for any place but the first.
__global__ void __launch_bounds__(kPT, 2) k_rs_pass(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, uint32_t n, int place, const uint32_t *__restrict__ gcnt,
    int next_place, uint32_t *__restrict__ next_cnt, uint64_t *status, uint32_t *tile_ctr,
    uint32_t epoch, uint32_t *err) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(smem);
  uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kTile);
  uint32_t *wc = sv + kTile;            // [kPW][256] per-warp digit counts, then prefixes
  uint32_t *tex = wc + kPW * kRadix;     // [256] exclusive digit prefix within the tile
  uint32_t *gof = tex + kRadix;          // [256] global offset of the tile's digit run, minus tex
  __shared__ uint32_t s_tile;
  __shared__ uint32_t scratch[kPW];
  __shared__ uint32_t s_next[kRadix];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kPW * kRadix; i += kPT) wc[i] = 0;
  if (tid < kRadix) s_next[tid] = 0;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kTile;
  const uint64_t seg = base + (uint64_t)warp * (kItems * 32);

  uint64_t k[kItems];
  uint32_t v[kItems];
  uint32_t rk[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint64_t idx = seg + j * 32 + lane;
    if (idx < n) {
      k[j] = kin[idx];
      v[j] = vin[idx];
    } else {
      k[j] = 0;
      v[j] = 0;
    }
  }
  uint32_t *mywc = wc + warp * kRadix;
  const uint32_t lt = lanemask_lt();
  if (next_place >= 0) {
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const bool valid = seg + j * 32 + lane < n;
      const uint32_t dn = valid ? digit_of(k[j], v[j], next_place) : 256u;
      const uint32_t d0 = __shfl_sync(0xffffffffu, dn, 0);
      if (__all_sync(0xffffffffu, dn == d0 && d0 < 256u)) {
        if (lane == 0) atomicAdd(&s_next[d0], 32u);
      } else if (valid) {
        atomicAdd(&s_next[dn], 1u);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const bool valid = seg + j * 32 + lane < n;
    const uint32_t d = valid ? digit_of(k[j], v[j], place) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t b = 0;
    if (valid) b = mywc[d];
    __syncwarp();
    if (valid) {
      rk[j] = b + __popc(peers & lt);
      if ((peers & lt) == 0) mywc[d] = b + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();

  // Thread d < 256 owns digit d: warp prefixes, tile count, publication,
  // look-back (threads 256.. only join the block scan with zero).
  const int d = tid;
  const bool owner = d < kRadix;
  uint32_t tcnt = 0;
  if (owner) {
#pragma unroll
    for (int w = 0; w < kPW; ++w) {
      const uint32_t c = wc[w * kRadix + d];
      wc[w * kRadix + d] = tcnt;
      tcnt += c;
    }
  }
  uint64_t *st = status + (size_t)t * kRadix;
  if (owner) lb_store(&st[d], lb_pack(t == 0 ? kLbInclusive : kLbAggregate, epoch, tcnt));
  uint32_t tot;
  const uint32_t gc = owner ? gcnt[d] : 0u;
  const uint32_t ginc = block_inclusive<kPW>(gc, OpSum(), 0u, scratch, &tot);
  if (owner && next_place >= 0 && s_next[d]) atomicAdd(&next_cnt[d], s_next[d]);
  const uint32_t inc = block_inclusive<kPW>(tcnt, OpSum(), 0u, scratch, &tot);
  if (owner) {
    tex[d] = inc - tcnt;
    uint32_t excl = 0;
    if (t > 0) {
      excl = lb_exclusive(status + d, kRadix, t, epoch, OpSum(), 0u, err);
      lb_store(&st[d], lb_pack(kLbInclusive, epoch, excl + tcnt));
    }
    gof[d] = (ginc - gc) + excl - (inc - tcnt);
  }
  __syncthreads();

#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    if (seg + j * 32 + lane < n) {
      const uint32_t dd = digit_of(k[j], v[j], place);
      const uint32_t lp = tex[dd] + wc[warp * kRadix + dd] + rk[j];
      sk[lp] = k[j];
      sv[lp] = v[j];
    }
  }
  __syncthreads();
  const uint32_t cnt = (n - base) < (uint64_t)kTile ? (uint32_t)(n - base) : (uint32_t)kTile;
  for (uint32_t q = tid; q < cnt; q += kPT) {
    const uint64_t kk = sk[q];
    const uint32_t vv = sv[q];
    const uint32_t pos = gof[digit_of(kk, vv, place)] + q;
    if (pos < n) {
      kout[pos] = kk;
      vout[pos] = vv;
    } else {
      atomicExch(err, kDevRange);  // only after a failed look-back
    }
  }
}

__global__ void k_key_or(const uint64_t *__restrict__ keys, uint32_t n, unsigned long long *out) {
  uint64_t acc = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc |= keys[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicOr(out, (unsigned long long)acc);
}

constexpr size_t kPassSmem =
    (size_t)kTile * 8 + (size_t)kTile * 4 + (size_t)kPW * kRadix * 4 + 2 * kRadix * 4;

}  // namespace

int radix_sort_init() {
  APO_CUDA_TRY(cudaFuncSetAttribute(k_rs_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kPassSmem));
  return APO_OK;
}

int plan_digits(int lo, int hi, int *places, int start) {
  int n = start;
  for (int s = lo; s < hi; s += 8) places[n++] = s;
  return n;
}

void launch_key_or(apo_ctx *c, const uint64_t *keys, uint32_t n, uint64_t *out_dev, cudaStream_t s) {
  int blocks = n ? std::min(1024, ceil_div(n, 256 * 8)) : 1;
  {
    Launch lp_(c, kKKeyOr, n, s);
    k_key_or<<<blocks, 256, 0, s>>>(keys, n, reinterpret_cast<unsigned long long *>(out_dev));
  }
}

int radix_sort_pairs(apo_ctx *c, SortBuffers &b, uint32_t n, const int *places, int npass,
                     cudaStream_t s) {
  if (n <= 1 || npass == 0) return APO_OK;
  if (npass > kMaxPass) {
    set_error("radix sort: too many digit places");
    return APO_EINVAL;
  }
  const int tiles = ceil_div(n, kTile);
  APO_TRY(ensure_lookback(c, (size_t)tiles * kRadix));
  Places pl;
  pl.n = npass;
  for (int p = 0; p < npass; ++p) pl.p[p] = places[p];
  uint32_t *hist = c->ps.counters + kCtrSortHist;  // [kMaxPass][256]
  uint32_t *tctr = c->ps.counters + kCtrSortTiles;  // [kMaxPass]
  APO_CUDA_TRY(cudaMemsetAsync(hist, 0, (kMaxPass * kRadix + kMaxPass) * sizeof(uint32_t), s));
  const int hblocks = std::min(c->num_sms * 4, ceil_div(n, kThreads * 8));
  {
    Launch lp_(c, kKRsHist, n, s);
    Places first = pl;
    first.n = 1;
    k_rs_hist<<<hblocks, kThreads, 0, s>>>(b.keys[b.cur], b.vals[b.cur], n, first, hist);
  }
  for (int p = 0; p < npass; ++p) {
    const uint32_t ep = next_epoch(c);
    const int nxt = p + 1 < npass ? places[p + 1] : -1;
    {
      Launch lp_(c, kKRsPass, n, s);
      k_rs_pass<<<tiles, kPT, kPassSmem, s>>>(b.keys[b.cur], b.vals[b.cur], b.keys[b.cur ^ 1],
                                                   b.vals[b.cur ^ 1], n, places[p],
                                                   hist + p * kRadix, nxt, hist + (p + 1) * kRadix,
                                                   c->ps.lookback, tctr + p, ep, c->ps.err);
    }
    b.cur ^= 1;
  }
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

}  // namespace apo
