// Onesweep LSD radix sort of (u64 key, u32 value) pairs, with a per-context
// autotuner for its launch shape.
//
// After Adinets & Merrill, "Onesweep: A Faster Least Significant Digit Radix
// Sort for GPUs" (2022): each digit place is scattered by one kernel whose
// tiles learn their global digit offsets through decoupled look-back instead
// of a separate scan pass.  Only the first place's histogram needs its own
// read of the keys; every pass counts the next place's digits of the keys it
// already holds, and each tile turns a histogram into offsets itself.
// Within a tile, keys are ranked per warp with __match_any_sync (stable: a
// warp's items are visited in input order), staged in shared memory in digit
// order and written out in runs, so global writes are coalesced per digit.
//
// A digit place is described by `place` = shift | (kFromValue if the digit
// comes from the value instead of the key).  Sorting on value digits first
// and key digits after gives a stable sort on the 96-bit composite.
//
// Launch shapes.  The pass kernel is instantiated for threads per block,
// pairs per thread and digit width (8 or 9 bits).  Small sorts want small
// tiles (more tiles in flight, shorter look-back chains), large ones want
// wide tiles; a wider digit saves a pass when the key width is just above a
// multiple of 8.  The first sort of each (size class, key bits) in a context
// times every shape on synthetic keys of that size and width and keeps the
// fastest for the rest of the context's life.
#include <algorithm>
#include <mutex>

#include "apo_internal.cuh"
#include "device_util.cuh"

namespace apo {

namespace {

constexpr int kHistThreads = 256;
constexpr int kMaxRadix = 512;
constexpr int kMaxPass = 12;

struct Places {
  int p[kMaxPass];
  int n;
};

template <int BITS>
__device__ __forceinline__ uint32_t digit_of(uint64_t k, uint32_t v, int place) {
  const int sh = place & 255;
  return (place & kFromValue) ? ((v >> sh) & ((1u << BITS) - 1)) : (uint32_t)((k >> sh) & ((1u << BITS) - 1));
}

// The first place's digit histogram.  When all lanes of a warp hold the same
// digit (common for the high digits of sorted ranks) one add counts the whole
// warp, so skewed digits do not serialise on one shared-memory counter.
template <int BITS>
__global__ void __launch_bounds__(kHistThreads) k_rs_hist(const uint64_t *__restrict__ keys,
                                                          const uint32_t *__restrict__ vals, uint32_t n,
                                                          const uint32_t *__restrict__ n_dev, int place,
                                                          uint32_t *__restrict__ hist) {
  constexpr int R = 1 << BITS;
  if (n_dev) n = min(n, *n_dev);
  __shared__ uint32_t sh[R];
  for (int i = threadIdx.x; i < R; i += kHistThreads) sh[i] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * kHistThreads;
  for (uint64_t b0 = (uint64_t)blockIdx.x * kHistThreads + (threadIdx.x & ~31u); b0 < n; b0 += stride) {
    const uint64_t i = b0 + lane;
    const bool valid = i < n;
    const uint32_t d = valid ? digit_of<BITS>(keys[i], vals ? vals[i] : 0u, place) : (uint32_t)R;
    const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
    if (__all_sync(0xffffffffu, d == d0 && d0 < (uint32_t)R)) {
      if (lane == 0) atomicAdd(&sh[d0], 32u);
    } else if (valid) {
      atomicAdd(&sh[d], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < R; i += kHistThreads)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

template <int TPB, int ITEMS, int BITS, bool KO>
struct PassShape {
  static constexpr int kRadix = 1 << BITS;
  static constexpr int kWarps = TPB / 32;
  static constexpr int kTile = TPB * ITEMS;
  static constexpr size_t kSmem = (size_t)kTile * (KO ? 8 : 12) + (size_t)kWarps * kRadix * 2 + 2 * kRadix * 4;
  static_assert(kRadix <= TPB, "each digit needs an owner thread");
  static_assert(kTile <= 65535, "per-warp digit prefixes are 16-bit");
};

// One digit place.  `gcnt` is this place's global digit histogram (the
// tile turns it into digit offsets itself); when next_place >= 0 the tile
// also counts the next place's digits of its keys into next_cnt, so no
// separate histogram read is needed for any place but the first.  A full
// tile arrives in shared memory by two bulk copies (keys, values) that one
// thread issues while the others clear the counters; the ragged last tile
// is loaded by the threads.  KO: keys only (vin, vout unused; no value
// digits).  Without values a thread needs fewer registers and a tile less
// shared memory, so three blocks of 512 threads fit an SM instead of two.
template <int TPB, int ITEMS, int BITS, bool KO>
__global__ void __launch_bounds__(TPB, (KO ? 1536 : 1024) / TPB) k_rs_pass(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, uint32_t n, const uint32_t *__restrict__ n_dev, int place,
    const uint32_t *__restrict__ gcnt, int next_place, uint32_t *__restrict__ next_cnt, uint64_t *status,
    uint32_t *tile_ctr, uint32_t epoch, uint32_t *err) {
  using S = PassShape<TPB, ITEMS, BITS, KO>;
  if (n_dev) n = min(n, *n_dev);  // the launch is sized for an upper bound
  constexpr int R = S::kRadix, NW = S::kWarps, TILE = S::kTile;
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(smem);
  uint32_t *sv = reinterpret_cast<uint32_t *>(sk + TILE);  // (pairs only)
  uint16_t *wc = reinterpret_cast<uint16_t *>(KO ? reinterpret_cast<uint8_t *>(sk + TILE)
                                                 : reinterpret_cast<uint8_t *>(sv + TILE));  // [NW][R] per-warp digit counts, then prefixes
  uint32_t *tex = reinterpret_cast<uint32_t *>(wc + NW * R);  // [R] exclusive digit prefix within the tile
  uint32_t *gof = tex + R;             // [R] global offset of the tile's digit run, minus tex
  __shared__ uint32_t s_tile;
  __shared__ uint32_t scratch[NW];
  __shared__ uint32_t s_next[R];
  __shared__ __align__(8) uint64_t s_bar;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr bool hv = !KO;
  if (tid == 0) {
    s_tile = atomicAdd(tile_ctr, 1u);
    mbar_init(&s_bar, 1);
  }
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * TILE;
  if (base >= n) return;  // a tile past the device-side count (no later tile looks at it)
  const bool bulk = n - base >= (uint64_t)TILE &&
                    ((reinterpret_cast<uintptr_t>(kin) | reinterpret_cast<uintptr_t>(vin)) & 15) == 0;
  if (bulk && tid == 0) {
    mbar_arrive_expect(&s_bar, TILE * (hv ? 12u : 8u));
    bulk_load(sk, kin + base, TILE * 8u, &s_bar);
    if (hv) bulk_load(sv, vin + base, TILE * 4u, &s_bar);
  }
  for (int i = tid; i < NW * R; i += TPB) wc[i] = 0;
  if (tid < R) s_next[tid] = 0;
  const uint64_t seg = base + (uint64_t)warp * (ITEMS * 32);
  const uint32_t wseg = (uint32_t)warp * (ITEMS * 32);

  uint64_t k[ITEMS];
  uint32_t v[ITEMS];
  uint32_t rk[ITEMS];
  if (bulk) {
    mbar_wait(&s_bar, 0, err);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      k[j] = sk[wseg + j * 32 + lane];
      v[j] = hv ? sv[wseg + j * 32 + lane] : 0u;
    }
  } else {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint64_t idx = seg + j * 32 + lane;
      if (idx < n) {
        k[j] = kin[idx];
        v[j] = hv ? vin[idx] : 0u;
      } else {
        k[j] = 0;
        v[j] = 0;
      }
    }
  }
  __syncthreads();  // the counters are clear
  uint16_t *mywc = wc + warp * R;
  const uint32_t lt = lanemask_lt();
  if (next_place >= 0) {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const bool valid = seg + j * 32 + lane < n;
      const uint32_t dn = valid ? digit_of<BITS>(k[j], v[j], next_place) : (uint32_t)R;
      const uint32_t d0 = __shfl_sync(0xffffffffu, dn, 0);
      if (__all_sync(0xffffffffu, dn == d0 && d0 < (uint32_t)R)) {
        if (lane == 0) atomicAdd(&s_next[d0], 32u);
      } else if (valid) {
        atomicAdd(&s_next[dn], 1u);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const bool valid = seg + j * 32 + lane < n;
    const uint32_t d = valid ? digit_of<BITS>(k[j], v[j], place) : (uint32_t)R;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t b = 0;
    if (valid) b = mywc[d];
    __syncwarp();
    if (valid) {
      rk[j] = b + __popc(peers & lt);
      if ((peers & lt) == 0) mywc[d] = (uint16_t)(b + __popc(peers));
    }
    __syncwarp();
  }
  __syncthreads();

  // Thread d < R owns digit d: warp prefixes, tile count, publication,
  // look-back (threads R.. only join the block scan with zero).
  const int d = tid;
  const bool owner = d < R;
  uint32_t tcnt = 0;
  if (owner) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = wc[w * R + d];
      wc[w * R + d] = (uint16_t)tcnt;
      tcnt += c;
    }
  }
  uint64_t *st = status + (size_t)t * R;
  if (owner) lb_store(&st[d], lb_pack(t == 0 ? kLbInclusive : kLbAggregate, epoch, tcnt));
  uint32_t tot;
  const uint32_t gc = owner ? gcnt[d] : 0u;
  const uint32_t ginc = block_inclusive<NW>(gc, OpSum(), 0u, scratch, &tot);
  if (owner && next_place >= 0 && s_next[d]) atomicAdd(&next_cnt[d], s_next[d]);
  const uint32_t inc = block_inclusive<NW>(tcnt, OpSum(), 0u, scratch, &tot);
  if (owner) {
    tex[d] = inc - tcnt;
    uint32_t excl = 0;
    if (t > 0) {
      excl = lb_exclusive(status + d, R, t, epoch, OpSum(), 0u, err);
      lb_store(&st[d], lb_pack(kLbInclusive, epoch, excl + tcnt));
    }
    gof[d] = (ginc - gc) + excl - (inc - tcnt);
  }
  __syncthreads();

#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    if (seg + j * 32 + lane < n) {
      const uint32_t dd = digit_of<BITS>(k[j], v[j], place);
      const uint32_t lp = tex[dd] + wc[warp * R + dd] + rk[j];
      sk[lp] = k[j];
      if (hv) sv[lp] = v[j];
    }
  }
  __syncthreads();
  const uint32_t cnt = (n - base) < (uint64_t)TILE ? (uint32_t)(n - base) : (uint32_t)TILE;
  for (uint32_t q = tid; q < cnt; q += TPB) {
    const uint64_t kk = sk[q];
    const uint32_t vv = hv ? sv[q] : 0u;
    const uint32_t pos = gof[digit_of<BITS>(kk, vv, place)] + q;
    if (pos < n) {
      kout[pos] = kk;
      if (hv) vout[pos] = vv;
    } else {
      atomicExch(err, kDevRange);  // only after a failed look-back
    }
  }
}

// out[0] |= every key, out[1] = max(out[1], every key).
__global__ void k_key_or(const uint64_t *__restrict__ keys, uint32_t n, unsigned long long *out) {
  uint64_t acc = 0, mx = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    acc |= k;
    mx = k > mx ? k : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc |= __shfl_xor_sync(0xffffffffu, acc, o);
    const uint64_t m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = m2 > mx ? m2 : mx;
  }
  if ((threadIdx.x & 31) == 0 && acc) {
    atomicOr(out, (unsigned long long)acc);
    atomicMax(out + 1, (unsigned long long)mx);
  }
}

// Synthetic trial pairs: keys uniform over `bits` bits (splitmix64 of the
// index and a seed), values = index.
__global__ void k_rs_trial_keys(uint64_t *keys, uint32_t *vals, uint32_t n, int bits, uint64_t seed) {
  const uint64_t mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9e3779b97f4a7c15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    keys[i] = z & mask;
    vals[i] = i;
  }
}

// ---------------------------------------------------------------- shapes
using PassFn = void (*)(const uint64_t *, const uint32_t *, uint64_t *, uint32_t *, uint32_t, const uint32_t *,
                        int, const uint32_t *, int, uint32_t *, uint64_t *, uint32_t *, uint32_t, uint32_t *);
using HistFn = void (*)(const uint64_t *, const uint32_t *, uint32_t, const uint32_t *, int, uint32_t *);

struct Shape {
  int threads, items, bits;
  PassFn pass, pass_keys;  // (key, value) pairs; keys only
  HistFn hist;
  size_t smem, smem_keys;
};

template <int TPB, int ITEMS, int BITS>
constexpr Shape shape() {
  return Shape{TPB, ITEMS, BITS, k_rs_pass<TPB, ITEMS, BITS, false>, k_rs_pass<TPB, ITEMS, BITS, true>,
               k_rs_hist<BITS>, PassShape<TPB, ITEMS, BITS, false>::kSmem, PassShape<TPB, ITEMS, BITS, true>::kSmem};
}

// Shape 0 is the default (and the only one used with tuning off).
const Shape kShapes[] = {
    shape<512, 8, 8>(), shape<256, 8, 8>(), shape<512, 4, 8>(), shape<256, 4, 8>(),
    shape<512, 8, 9>(), shape<512, 4, 9>(),
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int plan(const Shape &sh, const DigitRange *ranges, int nranges, Places *pl) {
  pl->n = 0;
  for (int r = 0; r < nranges; ++r)
    for (int s = ranges[r].lo; s < ranges[r].hi; s += sh.bits) {
      if (pl->n >= kMaxPass) return APO_EINVAL;
      pl->p[pl->n++] = s | (ranges[r].from_value ? kFromValue : 0);
    }
  return APO_OK;
}

// All passes of one sort with one shape (b.cur flips once per pass).
int sort_with(apo_ctx *c, const Shape &sh, SortBuffers &b, uint32_t n, const uint32_t *n_dev, const Places &pl,
              bool count, cudaStream_t s, bool hist_ready = false) {
  const int R = 1 << sh.bits;
  const int tile = sh.threads * sh.items;
  const int tiles = ceil_div(n, tile);
  APO_TRY(ensure_lookback(c, (size_t)tiles * R));
  uint32_t *hist = c->ps.counters + kCtrSortHist;   // [kMaxPass][kMaxRadix]
  uint32_t *tctr = c->ps.counters + kCtrSortTiles;  // [kMaxPass]
  if (hist_ready) {  // the first place's counts are in; clear the others and the tile tickets
    APO_CUDA_TRY(cudaMemsetAsync(hist + kMaxRadix, 0, ((kMaxPass - 1) * kMaxRadix + kMaxPass) * sizeof(uint32_t), s));
  } else {
    APO_CUDA_TRY(cudaMemsetAsync(hist, 0, (kMaxPass * kMaxRadix + kMaxPass) * sizeof(uint32_t), s));
    const int hblocks = std::max(1, std::min(c->num_sms * 4, ceil_div(n, kHistThreads * 8)));
    Launch lp_(c, count ? kKRsHist : kKRsTune, n, s);
    sh.hist<<<hblocks, kHistThreads, 0, s>>>(b.keys[b.cur], b.vals[b.cur], n, n_dev, pl.p[0], hist);
  }
  for (int p = 0; p < pl.n; ++p) {
    const uint32_t ep = next_epoch(c);
    const int nxt = p + 1 < pl.n ? pl.p[p + 1] : -1;
    {
      const bool ko = b.vals[b.cur] == nullptr;
      Launch lp_(c, count ? (ko ? kKRsPassKeys : kKRsPass) : kKRsTune, n, s);
      (ko ? sh.pass_keys : sh.pass)<<<tiles, sh.threads, ko ? sh.smem_keys : sh.smem, s>>>(
          b.keys[b.cur], b.vals[b.cur], b.keys[b.cur ^ 1],
                                                 b.vals[b.cur ^ 1], n, n_dev, pl.p[p], hist + p * kMaxRadix, nxt,
                                                 hist + (p + 1) * kMaxRadix, c->ps.lookback, tctr + p, ep,
                                                 c->ps.err);
    }
    b.cur ^= 1;
  }
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

}  // namespace

int radix_sort_init() {
  for (int i = 0; i < kNumShapes; ++i) {
    APO_CUDA_TRY(cudaFuncSetAttribute((const void *)kShapes[i].pass,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kShapes[i].smem));
    APO_CUDA_TRY(cudaFuncSetAttribute((const void *)kShapes[i].pass_keys,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kShapes[i].smem_keys));
  }
  return APO_OK;
}

namespace {
std::mutex g_table_mu;
constexpr int kMaxDevices = 64;
SortTable g_tables[kMaxDevices];
}  // namespace

SortTable &sort_table(int device) { return g_tables[device >= 0 && device < kMaxDevices ? device : 0]; }
void sort_table_lock(bool lock) {
  if (lock) g_table_mu.lock();
  else g_table_mu.unlock();
}

int SortTuner::size_class(uint32_t n) {
  return std::min(std::max(bits_for(n - 1), kTuneMinBits), kTuneMaxBits) - kTuneMinBits;
}

namespace {

// Times every shape on synthetic pairs of the call's size (at most 2^22) and
// key width; keeps the fastest.
int tune(apo_ctx *c, uint32_t n, int bits, int cls, cudaStream_t s) {
  SortTuner &T = c->tuner;
  const uint32_t nt = std::min<uint32_t>(n, 1u << 22);
  const size_t need = (size_t)nt * 24 + 1024;
  if (T.scratch_bytes < need) {
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    if (T.scratch) cudaFree(T.scratch);
    T.scratch = nullptr;
    T.scratch_bytes = 0;
    APO_CUDA_TRY(cudaMalloc(&T.scratch, need));
    T.scratch_bytes = need;
  }
  char *p = static_cast<char *>(T.scratch);
  SortBuffers b;
  b.keys[0] = reinterpret_cast<uint64_t *>(p);
  b.keys[1] = b.keys[0] + nt;
  b.vals[0] = reinterpret_cast<uint32_t *>(b.keys[1] + nt);
  b.vals[1] = b.vals[0] + nt;
  // the trial sorts as many bits as the call (value digits beyond 64 bits)
  const DigitRange trial[2] = {{0, bits > 64 ? bits - 64 : 0, true}, {0, std::min(bits, 64), false}};
  cudaEvent_t e0, e1;
  APO_CUDA_TRY(cudaEventCreate(&e0));
  APO_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f, dflt = 0.f;
  int pick = 0;
  for (int i = 0; i < kNumShapes; ++i) {
    Places pl;
    if (plan(kShapes[i], trial, 2, &pl) != APO_OK) continue;
    float t = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      k_rs_trial_keys<<<std::min(ceil_div(nt, 256), c->num_sms * 8), 256, 0, s>>>(b.keys[0], b.vals[0], nt,
                                                                                  std::min(bits, 64), 0x5eedull + rep);
      b.cur = 0;
      APO_CUDA_TRY(cudaEventRecord(e0, s));
      APO_TRY(sort_with(c, kShapes[i], b, nt, nullptr, pl, false, s));
      APO_CUDA_TRY(cudaEventRecord(e1, s));
      APO_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      APO_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) t = std::min(t, ms);  // the first run warms the shape
    }
    if (i == 0) dflt = t;
    if (t < best) {
      best = t;
      pick = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  APO_TRY(check_device_error(c, s));
  SortTable &tb = sort_table(c->device);
  std::lock_guard<std::mutex> lk(g_table_mu);
  tb.choice[cls][bits] = (int8_t)pick;
  tb.best_ms[cls][bits] = best;
  tb.default_ms[cls][bits] = dflt;
  tb.trial_n[cls][bits] = nt;
  return APO_OK;
}

}  // namespace

void launch_key_or(apo_ctx *c, const uint64_t *keys, uint32_t n, uint64_t *out_dev, cudaStream_t s) {
  int blocks = n ? std::min(1024, ceil_div(n, 256 * 8)) : 1;
  {
    Launch lp_(c, kKKeyOr, n, s);
    k_key_or<<<blocks, 256, 0, s>>>(keys, n, reinterpret_cast<unsigned long long *>(out_dev));
  }
}

int sort_plan(apo_ctx *c, uint32_t n, const DigitRange *ranges, int nranges, SortPlan *out, cudaStream_t s) {
  out->shape = -1;
  int bits = 0;
  for (int r = 0; r < nranges; ++r) bits += std::max(0, ranges[r].hi - ranges[r].lo);
  if (n <= 1 || bits == 0) return APO_OK;
  if (bits >= kTuneBits) {
    set_error("radix sort: more than 96 bits to sort on");
    return APO_EINVAL;
  }
  int shape_id = c->tuner.mode >= 2 ? c->tuner.mode - 2 : 0;  // mode 2 + k: always shape k
  if (c->tuner.mode == 0) {
    const int cls = SortTuner::size_class(n);
    SortTable &tb = sort_table(c->device);
    int id;
    {
      std::lock_guard<std::mutex> lk(g_table_mu);
      id = tb.choice[cls][bits];
    }
    if (id < 0 && c->ext) {
      id = 0;  // a caller workspace: no trial buffers, the default shape until the class is tuned
    } else if (id < 0) {
      APO_TRY(tune(c, n, bits, cls, s));
      std::lock_guard<std::mutex> lk(g_table_mu);
      id = tb.choice[cls][bits];
    }
    shape_id = id;
  }
  Places pl;
  if (plan(kShapes[shape_id], ranges, nranges, &pl) != APO_OK) {
    set_error("radix sort: too many digit places");
    return APO_EINVAL;
  }
  out->shape = shape_id;
  out->bits = kShapes[shape_id].bits;
  out->places = pl.n;
  for (int p = 0; p < pl.n; ++p) out->place[p] = pl.p[p];
  return APO_OK;
}

int sort_first_hist_clear(apo_ctx *c, cudaStream_t s) {
  APO_CUDA_TRY(cudaMemsetAsync(c->ps.counters + kCtrSortHist, 0, kMaxRadix * sizeof(uint32_t), s));
  return APO_OK;
}

uint32_t *sort_first_hist(apo_ctx *c) { return c->ps.counters + kCtrSortHist; }

int radix_sort_planned(apo_ctx *c, SortBuffers &b, uint32_t n, const SortPlan &sp, cudaStream_t s,
                       const uint32_t *n_dev, bool hist_ready) {
  if (sp.shape < 0) return APO_OK;
  Places pl;
  pl.n = sp.places;
  for (int p = 0; p < sp.places; ++p) pl.p[p] = sp.place[p];
  return sort_with(c, kShapes[sp.shape], b, n, n_dev, pl, true, s, hist_ready);
}

int radix_sort_pairs(apo_ctx *c, SortBuffers &b, uint32_t n, const DigitRange *ranges, int nranges,
                     cudaStream_t s, const uint32_t *n_dev) {
  SortPlan sp;
  APO_TRY(sort_plan(c, n, ranges, nranges, &sp, s));
  return radix_sort_planned(c, b, n, sp, s, n_dev, false);
}

int sort_shape_count() { return kNumShapes; }

int sort_shape_info(int id, int *threads, int *items, int *bits) {
  if (id < 0 || id >= kNumShapes) return APO_EINVAL;
  *threads = kShapes[id].threads;
  *items = kShapes[id].items;
  *bits = kShapes[id].bits;
  return APO_OK;
}

}  // namespace apo
