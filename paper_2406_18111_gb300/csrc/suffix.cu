// Suffix array by prefix doubling, and the LCP array by Phi / PLCP.
//
// Alg. 2 starts with SuffixArray(S) -> SA, LCP.  The suffix array is built
// by prefix doubling (Manber & Myers 1993) on the GPU in the style of
// Larsson & Sadakane: a suffix's rank is the SA position where its group of
// suffixes with an equal 2^r-token prefix starts.  Round r sorts only the
// suffixes whose group is not yet a singleton, by the key
// (rank[i], rank[i+h] + 1) with h = 2^r (0 when i + h runs past the end, so
// a proper prefix sorts first), with the onesweep radix sort.  The active
// suffixes are kept in SA order, so the k-th sorted key takes the k-th
// smallest active SA position: no segment bookkeeping is needed.  A single
// refresh kernel then finds the new group heads, writes SA and ranks, and
// compacts the suffixes that still share a group (one decoupled look-back
// max-scan for the head positions, one sum-scan for the compaction).
//
// Each round's rank array is kept ("level" r ranks: equal iff the first 2^r
// tokens are equal).  The LCP array follows Karkkainen, Manzini & Puglisi
// (CPM 2009): Phi[SA[k]] = SA[k-1]; PLCP[i] = lcp(i, Phi[i]) >= PLCP[i-1] - 1
// is computed in chunks with direct token comparison, and a match that keeps
// going is finished in O(levels) steps by binary lifting over the kept ranks;
// finally LCP[k] = PLCP[SA[k+1]] (LCP[k] pairs SA[k] with SA[k+1]).
#include <algorithm>
#include <cstring>

#include "apo_internal.cuh"
#include "device_util.cuh"

namespace apo {

namespace {

constexpr int kRT = 256;            // refresh threads per block
constexpr int kRI = 4;              // consecutive elements per thread
constexpr int kRTile = kRT * kRI;   // 1024
constexpr uint32_t kNone = 0xffffffffu;
constexpr size_t kRefreshSmem = (size_t)(kRTile + 2) * 8 + (size_t)kRTile * 8;

__global__ void k_init_keys(const void *__restrict__ tokens, int tb, uint32_t n,
                            uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    keys[i] = tb == 4 ? (uint64_t) static_cast<const uint32_t *>(tokens)[i]
                      : static_cast<const uint64_t *>(tokens)[i];
    vals[i] = i;
  }
}

// Sorted (key, suffix) pairs of the active suffixes -> new group heads, SA,
// ranks and the next active list.  actpos == nullptr means position = index
// (the first call, where the sorted list is the whole SA).  Only a suffix
// whose group became a singleton has reached its final SA position, so only
// it writes SA; a rank is written only when it changed (with old_sh >= 0 the
// old rank is key >> old_sh; a group's first subgroup keeps its start).
// Both cut scattered 4-byte writes, each of which costs a whole sector.
__global__ void __launch_bounds__(kRT) k_refresh(
    const uint64_t *__restrict__ keys, const uint32_t *__restrict__ idx, uint32_t A,
    const uint32_t *__restrict__ A_dev, const uint32_t *__restrict__ actpos, int old_sh,
    uint32_t *__restrict__ sa, uint32_t *__restrict__ rank, uint32_t *__restrict__ act_next,
    uint32_t *__restrict__ pos_next, uint32_t n, uint32_t *count_out, uint64_t *st_max, uint64_t *st_sum,
    uint32_t *tile_ctr, uint32_t epoch, uint32_t *err) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(smem);           // [kRTile + 2], key[base-1 ..]
  uint32_t *si = reinterpret_cast<uint32_t *>(sk + kRTile + 2);  // [kRTile]
  uint32_t *sp = si + kRTile;                                     // [kRTile]
  __shared__ uint32_t s_tile, s_pmax, s_psum;
  __shared__ uint32_t scr[kRT / 32];
  const int tid = threadIdx.x;
  if (A_dev) A = min(A, *A_dev);  // the launch is sized for an upper bound
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kRTile;
  if (base >= A) return;  // past the device-side count: no later tile looks at it
  const uint32_t cnt = (A - base) < (uint64_t)kRTile ? (uint32_t)(A - base) : (uint32_t)kRTile;
  for (uint32_t q = tid; q < cnt + 2; q += kRT) {
    const long long g = (long long)base - 1 + q;
    sk[q] = (g >= 0 && g < (long long)A) ? keys[g] : 0;
  }
  for (uint32_t q = tid; q < cnt; q += kRT) {
    si[q] = idx[base + q];
    sp[q] = actpos ? actpos[base + q] : (uint32_t)(base + q);
  }
  __syncthreads();

  const uint32_t e0 = tid * kRI;
  uint32_t hb = 0;  // bit i: element e0+i starts a group (bit kRI: the element after)
#pragma unroll
  for (int i = 0; i <= kRI; ++i) {
    const uint32_t local = e0 + i;
    if (local <= cnt) {
      const uint64_t g = base + local;
      if (g == 0 || g == A || sk[local + 1] != sk[local]) hb |= 1u << i;
    }
  }
  uint32_t tmax = 0, tcnt = 0;
  bool thead = false;
#pragma unroll
  for (int i = 0; i < kRI; ++i) {
    if (e0 + i < cnt) {
      const bool h = (hb >> i) & 1u;
      if (h) {
        tmax = sp[e0 + i];
        thead = true;
      }
      if (!(h && ((hb >> (i + 1)) & 1u))) ++tcnt;
    }
  }
  uint32_t tot_max, tot_sum;
  const uint32_t ex_max = block_exclusive<kRT / 32>(tmax, OpMax(), 0u, scr, &tot_max);
  const uint32_t ex_sum = block_exclusive<kRT / 32>(tcnt, OpSum(), 0u, scr, &tot_sum);
  const int any_head = __syncthreads_or(thead);
  if (tid == 0) {
    const bool incl = t == 0 || any_head;
    lb_store(&st_max[t], lb_pack(incl ? kLbInclusive : kLbAggregate, epoch, tot_max));
    uint32_t pm = 0;
    if (t > 0) pm = lb_exclusive(st_max, 1, t, epoch, OpMax(), 0u, err);
    if (!incl) lb_store(&st_max[t], lb_pack(kLbInclusive, epoch, max(pm, tot_max)));
    s_pmax = pm;
  }
  if (tid == 32) {
    lb_store(&st_sum[t], lb_pack(t == 0 ? kLbInclusive : kLbAggregate, epoch, tot_sum));
    uint32_t ps = 0;
    if (t > 0) {
      ps = lb_exclusive(st_sum, 1, t, epoch, OpSum(), 0u, err);
      lb_store(&st_sum[t], lb_pack(kLbInclusive, epoch, ps + tot_sum));
    }
    s_psum = ps;
    if (base + cnt == A) *count_out = ps + tot_sum;
  }
  __syncthreads();
  uint32_t rm = max(s_pmax, ex_max);
  uint32_t rs = s_psum + ex_sum;
#pragma unroll
  for (int i = 0; i < kRI; ++i) {
    const uint32_t local = e0 + i;
    if (local < cnt) {
      const bool h = (hb >> i) & 1u;
      const uint32_t p = sp[local];
      if (h) rm = p;
      const uint32_t id = si[local];
      if (p >= n || id >= n) {
        atomicExch(err, kDevRange);
        continue;
      }
      const bool single = h && ((hb >> (i + 1)) & 1u);
      if (single) sa[p] = id;
      if (old_sh < 0 || (uint32_t)(sk[local + 1] >> old_sh) != rm) rank[id] = rm;
      if (!single) {
        if (rs < A) {
          act_next[rs] = id;
          pos_next[rs] = p;
        } else {
          atomicExch(err, kDevRange);
        }
        ++rs;
      }
    }
  }
}

// ---------------------------------------------------------------- initial keys
// The first sort groups suffixes by their first h0 tokens at once: each
// token gets an order-preserving code 1..sigma (0 = past the window's end),
// h0 codes of cb bits are packed into one key under the window id, so the
// doubling starts at h = h0 instead of 1.  Codes: the token + 1 when the
// tokens are small integers; otherwise the rank of the token among the
// distinct tokens, through a hash dictionary of the distinct tokens.
constexpr uint64_t kDictEmpty = ~0ull;
constexpr uint32_t kDictMaxLog = 23;  // dictionary capacity at most 2^23 slots (sigma <= 2^22)

__device__ __forceinline__ uint64_t dmix(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint64_t token_at(const void *tokens, int tb, uint32_t i) {
  return tb == 4 ? (uint64_t) static_cast<const uint32_t *>(tokens)[i] : static_cast<const uint64_t *>(tokens)[i];
}

// Inserts every token (a token equal to the empty marker gets the last code
// by itself, see k_code_map); counts distinct tokens and gives up (flag)
// past `limit` of them.
__global__ void k_dict_tokens(const void *__restrict__ tokens, int tb, uint32_t n, uint64_t *keys, uint64_t mask,
                              uint32_t limit, uint32_t *distinct, uint32_t *over) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (*(volatile uint32_t *)over) return;
    const uint64_t t = token_at(tokens, tb, i);
    if (t == kDictEmpty) continue;
    uint64_t slot = dmix(t) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      uint64_t cur = keys[slot];
      if (cur == t) break;
      if (cur == kDictEmpty) {
        cur = atomicCAS((unsigned long long *)&keys[slot], (unsigned long long)kDictEmpty,
                        (unsigned long long)t);
        if (cur == kDictEmpty) {
          if (atomicAdd(distinct, 1u) >= limit) atomicExch(over, 1u);
          break;
        }
        if (cur == t) break;
      }
      slot = (slot + 1) & mask;
    }
  }
}

// (token, slot) of every occupied slot, in any order (sorted next).
__global__ void k_dict_list(const uint64_t *__restrict__ keys, uint64_t cap, uint64_t *lk, uint32_t *lv,
                            uint32_t *count) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cap; e += (uint64_t)gridDim.x * blockDim.x) {
    if (keys[e] == kDictEmpty) continue;
    const uint32_t q = atomicAdd(count, 1u);
    lk[q] = keys[e];
    lv[q] = (uint32_t)e;
  }
}

// code of slot = its token's rank among the distinct tokens + 1
__global__ void k_code_scatter(const uint32_t *__restrict__ sorted_slots, uint32_t sigma, uint32_t *code) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < sigma; q += gridDim.x * blockDim.x)
    code[sorted_slots[q]] = q + 1;
}

__global__ void k_code_map(const void *__restrict__ tokens, int tb, uint32_t n, const uint64_t *__restrict__ keys,
                           uint64_t mask, const uint32_t *__restrict__ slot_code, uint32_t top,
                           uint32_t *__restrict__ codes) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t t = token_at(tokens, tb, i);
    uint32_t cd = top;  // the all-ones token: larger than every other token
    if (t != kDictEmpty) {
      uint64_t slot = dmix(t) & mask;
      while (keys[slot] != t) slot = (slot + 1) & mask;
      cd = slot_code[slot];
    }
    codes[i] = cd;
  }
}

// key(i) = (window << (h0 * cb)) | code(i) code(i+1) .. code(i+h0-1), value i.
__global__ void k_pack0(const void *__restrict__ tokens, int tb, const uint32_t *__restrict__ codes, uint32_t n,
                        uint32_t h0, int cb, Windows W, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t we = win_end(W, i, n);
    uint64_t key = 0;
    for (uint32_t j = 0; j < h0; ++j) {
      uint64_t cd = 0;
      if (i + j < we) cd = codes ? codes[i + j] : token_at(tokens, tb, i + j) + 1;
      key = (key << cb) | cd;
    }
    if (W.count > 1) key |= (uint64_t)win_id(W, i) << (h0 * cb);
    keys[i] = key;
    vals[i] = i;
  }
}

// key = (rank[i] << sh) | (i + h < end of i's window ? rank[i + h] + 1 : 0)
// (the second part relative to the window's SA range with several windows),
// value = i, with sh = bits of the longest window (the second part is at
// most its length).
// Also counts the digits of the sort's first place (key bits [shift,
// shift + dbits)) into hist, which saves the sort its own pass over the keys.
__global__ void k_pack(const uint32_t *__restrict__ act, uint32_t A, const uint32_t *__restrict__ A_dev,
                       const uint32_t *__restrict__ rank, uint32_t n, uint64_t h, int sh, Windows W,
                       uint64_t *__restrict__ keys, uint32_t *__restrict__ vals, uint32_t *hist, int shift,
                       int dbits) {
  __shared__ uint32_t cnt[512];
  const uint32_t R = 1u << dbits, lane = threadIdx.x & 31;
  for (uint32_t q = threadIdx.x; q < R; q += blockDim.x) cnt[q] = 0;
  __syncthreads();
  if (A_dev) A = min(A, *A_dev);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t k0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); k0 < A; k0 += stride) {
    const uint32_t k = k0 + lane;
    uint32_t d = R;
    if (k < A) {
      const uint32_t i = act[k];
      const uint64_t j = i + h;
      // the second rank is only compared within a group, i.e. within one
      // window, so it is taken relative to the window's SA range
      uint32_t r2 = 0;
      if (j < win_end(W, i, n)) r2 = rank[j] + 1u - (W.count > 1 ? W.off_dev[W.wid[i]] : 0u);
      const uint64_t key = ((uint64_t)rank[i] << sh) | r2;
      keys[k] = key;
      vals[k] = i;
      d = (uint32_t)(key >> shift) & (R - 1);
    }
    const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
    if (__all_sync(0xffffffffu, d == d0 && d0 < R)) {
      if (lane == 0) atomicAdd(&cnt[d0], 32u);
    } else if (d < R) {
      atomicAdd(&cnt[d], 1u);
    }
  }
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < R; q += blockDim.x)
    if (cnt[q]) atomicAdd(&hist[q], cnt[q]);
}

// Batched first round: key = (window << 32) | rank of the token among all
// tokens, so that suffixes of different windows never share a group.
__global__ void k_wkeys(const uint32_t *__restrict__ rank, Windows W, uint32_t n,
                        uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    keys[i] = ((uint64_t)win_id(W, i) << 32) | rank[i];
    vals[i] = i;
  }
}

__global__ void k_phi(const uint32_t *__restrict__ sa, uint32_t n, Windows W,
                      uint32_t *__restrict__ phi) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t i = sa[k];
    phi[i] = (k && win_id(W, sa[k - 1]) == win_id(W, i)) ? sa[k - 1] : kNone;
  }
}

template <class T>
__device__ __forceinline__ bool long_match(const T *__restrict__ S, uint32_t n, uint32_t i,
                                           uint32_t j, uint32_t &l) {
  // i and j lie in the same window, which ends at n
  uint32_t steps = 0;
  while (i + (uint64_t)l < n && j + (uint64_t)l < n && S[i + l] == S[j + l]) {
    ++l;
    if (++steps == 32) return true;
  }
  return false;
}

// PLCP[i] = lcp(i, Phi[i]) over chunks of consecutive i, kRChunk per thread.
constexpr int kPChunk = 16;
template <class T>
__global__ void k_plcp(const T *__restrict__ S, uint32_t n, Windows W,
                       const uint32_t *__restrict__ phi, const uint32_t *__restrict__ snaps,
                       int levels, uint32_t h0, uint32_t *__restrict__ plcp) {
  const uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * kPChunk;
  if (i0 >= n) return;
  const uint32_t iend = (i0 + kPChunk) < (uint64_t)n ? (uint32_t)(i0 + kPChunk) : n;
  uint32_t l = 0;
  for (uint32_t i = (uint32_t)i0; i < iend; ++i) {
    const uint32_t j = phi[i];
    if (j == kNone) {
      plcp[i] = 0;
      l = 0;
      continue;
    }
    if (i > i0 && win_id(W, i) != win_id(W, i - 1)) l = 0;  // a new window starts
    const uint32_t we = win_end(W, i, n);
    if (long_match(S, we, i, j, l)) {
      // lift: level lev ranks are equal iff the next h0 * 2^lev tokens are
      // equal; what remains is shorter than h0 and is compared directly
      for (int lev = levels - 1; lev >= 0; --lev) {
        const uint64_t a = (uint64_t)i + l, b = (uint64_t)j + l;
        if (a < we && b < we && snaps[(size_t)lev * n + a] == snaps[(size_t)lev * n + b])
          l += h0 << lev;
      }
      for (uint32_t k = 1; k < h0 && i + (uint64_t)l < we && j + (uint64_t)l < we && S[i + l] == S[j + l]; ++k)
        ++l;
    }
    plcp[i] = l;
    l = l ? l - 1 : 0;
  }
}

__global__ void k_lcp_perm(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ plcp,
                           uint32_t n, Windows W, uint32_t *__restrict__ lcp) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    lcp[k] = (k + 1 < n && win_id(W, sa[k + 1]) == win_id(W, sa[k])) ? plcp[sa[k + 1]] : 0u;
}

// Launches the refresh of the (at most A, exactly *A_dev when given) sorted
// active suffixes; the number still active lands in *count_dev (zeroed
// first, so a launch with nothing to do leaves 0).
int refresh_launch(apo_ctx *c, const uint64_t *keys, const uint32_t *idx, uint32_t A, const uint32_t *A_dev,
                   const uint32_t *actpos, int old_sh, uint32_t *sa, uint32_t *rank, uint32_t *act_next,
                   uint32_t *pos_next, uint32_t n, uint32_t *count_dev, cudaStream_t s) {
  const int tiles = std::max(1, ceil_div(A, kRTile));
  APO_TRY(ensure_lookback(c, (size_t)2 * tiles));
  uint32_t *misc = c->ps.counters + kCtrMisc;
  APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscRefreshTiles, 0, sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(count_dev, 0, sizeof(uint32_t), s));
  const uint32_t ep = next_epoch(c);
  {
    Launch lp_(c, kKRefresh, A, s);
    k_refresh<<<tiles, kRT, kRefreshSmem, s>>>(keys, idx, A, A_dev, actpos, old_sh, sa, rank, act_next, pos_next,
                                               n, count_dev, c->ps.lookback, c->ps.lookback + tiles,
                                               misc + kMiscRefreshTiles, ep, c->ps.err);
  }
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

uint64_t dict_capacity(uint32_t n) {
  uint64_t cap = 1;
  while (cap < 2ull * n && cap < (1ull << kDictMaxLog)) cap <<= 1;
  return cap;
}

// Order-preserving dense codes of the tokens (1 .. sigma, sigma + 1 for the
// all-ones u64 token) through a dictionary of the distinct tokens.  begin
// queues the inserts and the read-back of the distinct count and overflow
// flag (pinned words 2 and 3); finish, after the caller's synchronisation,
// leaves *codes_out null when there are more than half the dictionary's
// capacity of distinct tokens.
struct DictCodes {
  uint64_t cap = 0;
  uint64_t *keys = nullptr;
  uint32_t *slot_code = nullptr, *codes = nullptr;
  SortBuffers lb;
  bool ok = false;
};

int dictionary_begin(apo_ctx *c, const void *tokens, int tb, uint32_t n, DictCodes *d, cudaStream_t s) {
  d->cap = dict_capacity(n);
  const uint32_t limit = (uint32_t)(d->cap / 2);
  d->keys = c->arena.take_n<uint64_t>(d->cap);
  d->slot_code = c->arena.take_n<uint32_t>(d->cap);
  d->codes = c->arena.take_n<uint32_t>(n);
  d->lb.keys[0] = c->arena.take_n<uint64_t>(limit);
  d->lb.keys[1] = c->arena.take_n<uint64_t>(limit);
  d->lb.vals[0] = c->arena.take_n<uint32_t>(limit);
  d->lb.vals[1] = c->arena.take_n<uint32_t>(limit);
  d->ok = d->keys && d->slot_code && d->codes && d->lb.keys[0] && d->lb.keys[1] && d->lb.vals[0] && d->lb.vals[1];
  if (!d->ok) return APO_OK;
  uint32_t *misc = c->ps.counters + kCtrMisc;
  APO_CUDA_TRY(cudaMemsetAsync(d->keys, 0xff, d->cap * sizeof(uint64_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscDict, 0, 2 * sizeof(uint32_t), s));
  {
    Launch lp_(c, kKSaDict, n, s);
    k_dict_tokens<<<grid_for(n, 256, c->num_sms), 256, 0, s>>>(tokens, tb, n, d->keys, d->cap - 1, limit,
                                                               misc + kMiscDict, misc + kMiscDict + 1);
  }
  if (!capturing(c))  // read in dictionary_finish (a captured call takes it from its tape there)
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 2, misc + kMiscDict, 8, cudaMemcpyDeviceToHost, s));
  return APO_OK;
}

int dictionary_finish(apo_ctx *c, const void *tokens, int tb, uint32_t n, int tbits, DictCodes *d,
                      uint32_t **codes_out, int *cb_out, cudaStream_t s) {
  *codes_out = nullptr;
  uint32_t *misc = c->ps.counters + kCtrMisc;
  if (!d->ok) return APO_OK;
  uint32_t sv[2];  // distinct tokens, overflow flag
  if (capturing(c)) {
    APO_TRY(tape_take(c, misc + kMiscDict, sv, 2, s));
  } else {
    sv[0] = c->host_pinned[2];
    sv[1] = c->host_pinned[3];
    if (recording(c)) tape_put(c, sv, 2);
  }
  const uint32_t sigma = sv[0];
  if (sv[1] || sigma > d->cap / 2) return APO_OK;
  APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscDict, 0, sizeof(uint32_t), s));
  {
    Launch lp_(c, kKSaDict, d->cap, s);
    k_dict_list<<<grid_for(d->cap, 256, c->num_sms), 256, 0, s>>>(d->keys, d->cap, d->lb.keys[0], d->lb.vals[0],
                                                                  misc + kMiscDict);
  }
  d->lb.cur = 0;
  const DigitRange r{0, tbits, false};
  APO_TRY(radix_sort_pairs(c, d->lb, sigma, &r, 1, s));
  {
    Launch lp_(c, kKSaDict, sigma, s);
    k_code_scatter<<<grid_for(std::max<uint32_t>(sigma, 1), 256, c->num_sms), 256, 0, s>>>(d->lb.vals[d->lb.cur],
                                                                                           sigma, d->slot_code);
  }
  {
    Launch lp_(c, kKSaDict, n, s);
    k_code_map<<<grid_for(n, 256, c->num_sms), 256, 0, s>>>(tokens, tb, n, d->keys, d->cap - 1, d->slot_code,
                                                            sigma + 1, d->codes);
  }
  APO_CUDA_TRY(cudaGetLastError());
  *codes_out = d->codes;
  *cb_out = bits_for(sigma + 1);
  return APO_OK;
}

}  // namespace

int suffix_init() {
  APO_CUDA_TRY(cudaFuncSetAttribute(k_refresh, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kRefreshSmem));
  return APO_OK;
}

size_t suffix_workspace_bytes(uint64_t n) {
  const int levels = bits_for(n) + 2;
  const uint64_t cap = dict_capacity((uint32_t)std::min<uint64_t>(n, 0xffffffffull));
  return (size_t)n * (2 * 8 + 2 * 4 + 4 * 4 + 4 + 4) + (size_t)levels * n * 4 + 16 * 256 +
         (size_t)(cap * 12 + (cap / 2) * 24 + n * 4 + 8 * 256);  // token dictionary
}

int build_suffix_array(apo_ctx *c, const void *tokens, int tb, uint32_t n, SuffixState &st,
                       int max_levels, uint32_t *rounds_out, cudaStream_t s) {
  st.n = n;
  st.levels = 0;
  *rounds_out = 0;
  if (n == 0) return APO_OK;
  SortBuffers b;
  b.keys[0] = c->arena.take_n<uint64_t>(n);
  b.keys[1] = c->arena.take_n<uint64_t>(n);
  b.vals[0] = c->arena.take_n<uint32_t>(n);
  b.vals[1] = c->arena.take_n<uint32_t>(n);
  uint32_t *act[2] = {c->arena.take_n<uint32_t>(n), c->arena.take_n<uint32_t>(n)};
  uint32_t *pos[2] = {c->arena.take_n<uint32_t>(n), c->arena.take_n<uint32_t>(n)};
  if (!b.keys[0] || !b.keys[1] || !b.vals[0] || !b.vals[1] || !act[0] || !act[1] || !pos[0] ||
      !pos[1]) {
    set_error("suffix array: workspace too small");
    return APO_ENOMEM;
  }
  const int g = grid_for(n, 256, c->num_sms);
  {
    Launch lp_(c, kKInitKeys, n, s);
    k_init_keys<<<g, 256, 0, s>>>(tokens, tb, n, b.keys[0], b.vals[0]);
  }
  // how many token bits are populated (for u64 tokens the dictionary of
  // distinct tokens is filled in the same round trip)
  uint32_t *misc = c->ps.counters + kCtrMisc;
  uint64_t *kor = reinterpret_cast<uint64_t *>(misc + kMiscKeyOr);
  APO_CUDA_TRY(cudaMemsetAsync(kor, 0, 2 * sizeof(uint64_t), s));
  launch_key_or(c, b.keys[0], n, kor, s);
  DictCodes dict;
  const bool dict_early = tb == 8 && n >= 4096;
  if (dict_early) APO_TRY(dictionary_begin(c, tokens, tb, n, &dict, s));
  uint64_t orv = 0, maxv = 0;
  // (pinned words 8..11: words 2..3 may be receiving the dictionary's size)
  if (capturing(c)) {
    APO_TRY(tape_take(c, reinterpret_cast<const uint32_t *>(kor), c->host_pinned + 8, 4, s));
  } else {
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 8, kor, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    if (recording(c)) tape_put(c, c->host_pinned + 8, 4);
  }
  memcpy(&orv, c->host_pinned + 8, sizeof(uint64_t));
  memcpy(&maxv, c->host_pinned + 10, sizeof(uint64_t));

  // codes for the packed first keys: token + 1, or dictionary ranks when
  // that packs more tokens per key
  const int wb = st.win.count > 1 ? bits_for(st.win.count - 1) : 0;
  const int tbits = bits_for(orv);
  int cb = tbits <= 32 ? bits_for(maxv + 1) : 0;  // codes token + 1 <= max + 1
  uint32_t h0 = cb ? (uint32_t)((64 - wb) / cb) : 0;
  const uint32_t *codes = nullptr;
  if (h0 < 4 && n >= 4096) {
    uint32_t *code_arr = nullptr;
    int cb_dict = 0;
    if (!dict_early) {
      APO_TRY(dictionary_begin(c, tokens, tb, n, &dict, s));
      if (!capturing(c)) APO_CUDA_TRY(cudaStreamSynchronize(s));
    }
    APO_TRY(dictionary_finish(c, tokens, tb, n, tbits, &dict, &code_arr, &cb_dict, s));
    if (code_arr && (uint32_t)((64 - wb) / cb_dict) > h0) {
      codes = code_arr;
      cb = cb_dict;
      h0 = (uint32_t)((64 - wb) / cb);
    }
  }
  uint32_t A = 0;
  if (h0 >= 2) {
    h0 = std::min<uint32_t>(h0, 32);
    {
      Launch lp_(c, kKInitKeys, n, s);
      k_pack0<<<g, 256, 0, s>>>(tokens, tb, codes, n, h0, cb, st.win, b.keys[0], b.vals[0]);
    }
    b.cur = 0;
    const DigitRange r{0, wb + (int)h0 * cb, false};
    APO_TRY(radix_sort_pairs(c, b, n, &r, 1, s));
    APO_TRY(refresh_launch(c, b.keys[b.cur], b.vals[b.cur], n, nullptr, nullptr, -1, st.sa, st.rank, act[0],
                           pos[0], n, misc + kMiscRefreshCount, s));
    A = n;  // an upper bound: the count stays on the device
  } else {
    h0 = 1;
    {
      const DigitRange r{0, tbits, false};
      APO_TRY(radix_sort_pairs(c, b, n, &r, 1, s));
    }
    APO_TRY(refresh_launch(c, b.keys[b.cur], b.vals[b.cur], n, nullptr, nullptr, -1, st.sa, st.rank, act[0],
                           pos[0], n, misc + kMiscRefreshCount, s));
    A = n;  // an upper bound: the count stays on the device
    if (st.win.count > 1) {
      // group by (window, token): re-sort by the window id over the token ranks
      {
        Launch lp_(c, kKInitKeys, n, s);
        k_wkeys<<<g, 256, 0, s>>>(st.rank, st.win, n, b.keys[0], b.vals[0]);
      }
      b.cur = 0;
      const DigitRange r[2] = {{0, bits_for(n - 1), false}, {32, 32 + wb, false}};
      APO_TRY(radix_sort_pairs(c, b, n, r, 2, s));
      APO_TRY(refresh_launch(c, b.keys[b.cur], b.vals[b.cur], n, nullptr, nullptr, -1, st.sa, st.rank, act[0],
                           pos[0], n, misc + kMiscRefreshCount, s));
    A = n;  // an upper bound: the count stays on the device
    }
  }
  st.h0 = h0;
  APO_CUDA_TRY(cudaMemcpyAsync(st.snaps[0], st.rank, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  st.levels = 1;
  int cur = 0;
  uint32_t rounds = 0;
  // second rank + 1 <= the longest window; first rank < n
  const int minor_bits = bits_for(st.win.count > 1 ? st.win.max_len : n), major_bits = bits_for(n - 1);
  // Round r reads its active count from a device word and writes the next
  // one; the host queues round r+1 before it has read round r's count (an
  // upper bound sizes the launches), and stops one round after the count
  // reaches 0 (that round's kernels find nothing to do and return).
  uint32_t *rc = misc + kMiscRound;
  uint32_t ub = A;  // upper bound on the current round's input count
  for (uint32_t r = 0; A > 0; ++r) {
    if (st.levels >= max_levels) {
      set_error("suffix array: too many doubling rounds");
      return APO_EDEVICE;
    }
    const uint32_t *in = r == 0 ? misc + kMiscRefreshCount : rc + ((r - 1) & 1);
    uint32_t *out = rc + (r & 1);
    const uint64_t h = (uint64_t)h0 << r;
    b.cur = 0;
    const DigitRange dr{0, minor_bits + major_bits, false};
    SortPlan sp;
    APO_TRY(sort_plan(c, ub, &dr, 1, &sp, s));
    APO_TRY(sort_first_hist_clear(c, s));
    {
      Launch lp_(c, kKPack, ub, s);
      const int blocks = std::max(1, std::min(ceil_div(ub, 256), c->num_sms * 4));
      k_pack<<<blocks, 256, 0, s>>>(act[cur], ub, in, st.rank, n, h, minor_bits, st.win, b.keys[0], b.vals[0],
                                    sort_first_hist(c), sp.shape >= 0 ? (sp.place[0] & 255) : 0, sp.bits);
    }
    APO_TRY(radix_sort_planned(c, b, ub, sp, s, in, true));
    APO_TRY(refresh_launch(c, b.keys[b.cur], b.vals[b.cur], ub, in, pos[cur], minor_bits, st.sa, st.rank,
                           act[cur ^ 1], pos[cur ^ 1], n, out, s));
    cur ^= 1;
    APO_CUDA_TRY(cudaMemcpyAsync(st.snaps[st.levels], st.rank, (size_t)n * 4,
                                 cudaMemcpyDeviceToDevice, s));
    ++st.levels;
    const bool cap = capturing(c);
    if (!cap) {
      if (r == 0)  // round 0's input count, also unknown on the host so far
        APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 6, in, 4, cudaMemcpyDeviceToHost, s));
      APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 4 + (r & 1), out, 4, cudaMemcpyDeviceToHost, s));
      APO_CUDA_TRY(cudaEventRecord(c->round_ev[r & 1], s));
    }
    if (r > 0) {
      // (a captured call takes the counts from its tape, checked against the
      // device words -- still unchanged at this point of the stream)
      uint32_t first = 0, a = 0;
      if (r == 1) {
        if (cap) {
          APO_TRY(tape_take(c, misc + kMiscRefreshCount, &first, 1, s));
        } else {
          APO_CUDA_TRY(cudaEventSynchronize(c->round_ev[(r - 1) & 1]));
          first = c->host_pinned[6];
          if (recording(c)) tape_put(c, &first, 1);
        }
        if (first == 0) {  // the first sort left no group: rounds 0 and 1 idle
          st.levels -= 2;
          rounds = 0;
          break;
        }
      }
      if (cap) {
        APO_TRY(tape_take(c, rc + ((r - 1) & 1), &a, 1, s));
      } else {
        if (r > 1) APO_CUDA_TRY(cudaEventSynchronize(c->round_ev[(r - 1) & 1]));
        a = c->host_pinned[4 + ((r - 1) & 1)];  // round r's input count
        if (recording(c)) tape_put(c, &a, 1);
      }
      if (a == 0) {  // round r had nothing to do
        --st.levels;
        break;
      }
      ub = a;
    }
    ++rounds;
  }
  *rounds_out = rounds;
  return APO_OK;
}

int build_lcp(apo_ctx *c, const void *tokens, int tb, const SuffixState &st, uint32_t *lcp,
              cudaStream_t s) {
  const uint32_t n = st.n;
  if (n == 0) return APO_OK;
  uint32_t *phi = c->arena.take_n<uint32_t>(n);
  uint32_t *plcp = c->arena.take_n<uint32_t>(n);
  if (!phi || !plcp) {
    set_error("lcp: workspace too small");
    return APO_ENOMEM;
  }
  const int g = grid_for(n, 256, c->num_sms);
  {
    Launch lp_(c, kKPhi, n, s);
    k_phi<<<g, 256, 0, s>>>(st.sa, n, st.win, phi);
  }
  const int pb = ceil_div(ceil_div(n, kPChunk), 128);
  if (tb == 4)
    {
      Launch lp_(c, kKPlcp, n, s);
      k_plcp<uint32_t><<<pb, 128, 0, s>>>(static_cast<const uint32_t *>(tokens), n, st.win, phi,
                                          st.snaps[0],
                                          st.levels, st.h0, plcp);
    }
  else
    {
      Launch lp_(c, kKPlcp, n, s);
      k_plcp<uint64_t><<<pb, 128, 0, s>>>(static_cast<const uint64_t *>(tokens), n, st.win, phi,
                                          st.snaps[0],
                                          st.levels, st.h0, plcp);
    }
  {
    Launch lp_(c, kKLcpPerm, n, s);
    k_lcp_perm<<<g, 256, 0, s>>>(st.sa, plcp, n, st.win, lcp);
  }
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

}  // namespace apo
