// Suffix array by prefix doubling, and the LCP array by Phi / PLCP.
//
// Alg. 2 starts with SuffixArray(S) -> SA, LCP.  The suffix array is built
// by prefix doubling (Manber & Myers 1993) in the style of Larsson &
// Sadakane: a suffix's level-L rank is the SA slot where its group of
// suffixes sharing the first h0 * 2^L tokens starts, and a suffix alone in
// its group has its final slot.
//
// Level 0 comes from one radix sort of the first h0 tokens of every suffix
// (dense token codes packed into a 64-bit key under the window id).  Each
// later round r refines the groups that are not yet singletons by the minor
// key rank_{r-1}[i + h] + 1 (0 when i + h is past the window's end), h =
// h0 * 2^(r-1).  The groups are already in order, so a round only has to
// sort each group by its minor keys:
//
//   * The active suffixes form a list of (suffix, group head slot) entries,
//     each group contiguous.  k_round cuts the list into tiles of kRdT
//     entries; a tile owns the groups that start in it.  The groups of at
//     most kRdBig entries ("small") are sorted together by (group, minor) in
//     shared memory with a block-wide LSD radix sort and settled by the
//     owner in one pass: no key leaves the chip.  Whether a group is small is
//     read off the entry kRdBig places after its start, so no scan over
//     group sizes is needed.  The minor keys come from k_minor, a streaming
//     pass that keeps many of its dependent gathers in flight.
//   * Larger groups ("big") are written as (big-group ordinal, minor) keys
//     and sorted by the onesweep radix sort; k_split then settles them.
//   * Settled entries go to a holed copy of the list (a suffix that became
//     final leaves a hole), which k_list_compact squeezes into the next
//     round's list.  Every prefix a tile needs from the tiles before it (big
//     entries, big groups, list positions) is a decoupled look-back.
//
// Settling a sorted group: its subgroups of equal minor keys start at the
// slots head + (position in the group); a subgroup of one suffix is final
// (SA, final rank, level recorded in fin[]); the others form the next list.
//
// Level ranks for the LCP.  Every round writes the new level rank of each
// of its active suffixes that stay grouped into that level's snapshot array
// and nothing else, so snaps[L][i] is valid exactly when suffix i is still
// grouped after round L (fin[i] > L); a suffix final at level L or before
// has its level rank -- its final slot -- in rank[i] (a group of one starts
// at its own slot).  level_rank(L, i) therefore reads fin[i] first.  A round
// reads only the previous level and final ranks, which no kernel of the
// same round writes, so rounds need no copies of the rank array.
//
// The LCP array follows Karkkainen, Manzini & Puglisi (CPM 2009):
// Phi[SA[k]] = SA[k-1]; PLCP[i] = lcp(i, Phi[i]) >= PLCP[i-1] - 1 is
// computed in chunks by direct token comparison, and a match that keeps
// going is finished in O(levels) steps by binary lifting over the level
// ranks; finally LCP[k] = PLCP[SA[k+1]] (LCP[k] pairs SA[k] with SA[k+1]).
#include <algorithm>
#include <cstring>

#include "apo_internal.cuh"
#include "device_util.cuh"

namespace apo {

namespace {

constexpr uint32_t kNone = 0xffffffffu;
constexpr uint32_t kHole = 0xfffffffeu;  // head of a place in the holed next list that holds no entry

__global__ void k_init_keys(const void *__restrict__ tokens, int tb, uint32_t n,
                            uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    keys[i] = tb == 4 ? (uint64_t) static_cast<const uint32_t *>(tokens)[i]
                      : static_cast<const uint64_t *>(tokens)[i];
    vals[i] = i;
  }
}

// out[0] |= every token, out[1] = max(out[1], every token).
__global__ void k_token_or(const void *__restrict__ tokens, int tb, uint32_t n, unsigned long long *out) {
  uint64_t acc = 0, mx = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t k = tb == 4 ? (uint64_t) static_cast<const uint32_t *>(tokens)[i]
                               : static_cast<const uint64_t *>(tokens)[i];
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

__device__ __forceinline__ bool bit_at(const uint32_t *__restrict__ bits, uint32_t j) {
  return (__ldg(bits + (j >> 5)) >> (j & 31)) & 1u;
}

// Level-L rank of suffix j: its final slot when it was settled at level L
// or before, else the level's snapshot.
__device__ __forceinline__ uint32_t level_rank(const uint8_t *__restrict__ fin, const uint32_t *__restrict__ rank,
                                               const uint32_t *__restrict__ snap, uint32_t L, uint32_t j) {
  const uint32_t f = fin[j];
  return f <= L ? rank[j] : snap[j];
}

// Decoupled look-back: lb_publish stores the tile's aggregate, lb_sum_warp
// publishes it and resolves the sum over tiles < t with one warp, then stores
// the tile's inclusive prefix.  A tile should resolve right after it
// publishes: a walk back only ends at an inclusive prefix, so tiles that
// resolve late make their successors' walks long.
__device__ __forceinline__ void lb_publish(uint64_t *st, uint32_t t, uint32_t v, uint32_t epoch) {
  lb_store(&st[t], lb_pack(t == 0 ? kLbInclusive : kLbAggregate, epoch, v));
}
// Every lane of the warp calls it; all get the prefix.
__device__ __forceinline__ uint32_t lb_sum_warp(uint64_t *st, uint32_t t, uint32_t v, uint32_t epoch,
                                                uint32_t *err) {
  if ((threadIdx.x & 31) == 0) lb_publish(st, t, v, epoch);
  if (t == 0) return 0;
  const uint32_t p = lb_exclusive_warp(st, 1, t, epoch, OpSum(), 0u, err);
  if ((threadIdx.x & 31) == 0) lb_store(&st[t], lb_pack(kLbInclusive, epoch, p + v));
  return p;
}

// ---------------------------------------------------------------- settling sorted groups
// Sorted (key, suffix) pairs -> groups of equal keys.  Every suffix gets its
// level rank (the slot where its group starts) in snap; with `finals` a
// suffix alone in its group is settled (sa, rank, fin = level).
//   kBig false (the first sort): the slot of sorted element q is q; the
//   suffixes not alone are appended, group by group, to the list (nid, nhd),
//   whose length lands in *count_out.
//   kBig true (big groups sorted by (ordinal o = key >> ord_shift, minor)):
//   group o's sorted elements start at bg_off[o], its slots at bg_head[o],
//   and its list entries at bg_pos[o]; a suffix not alone is written in
//   place to the holed next list (nid, nhd), a singleton's place becomes a
//   hole.
// Decoupled look-backs: the last group start (max) and, for kBig false, the
// list position (sum).
constexpr int kST = 256, kSI = 4, kSTile = kST * kSI;

template <bool kBig>
__global__ void __launch_bounds__(kST) k_split(
    const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, uint32_t ub,
    const uint32_t *__restrict__ n_dev, int ord_shift, const uint32_t *__restrict__ bg_head,
    const uint32_t *__restrict__ bg_off, const uint32_t *__restrict__ bg_pos, uint32_t bg_cap, uint32_t level,
    int finals, uint32_t *__restrict__ snap, uint32_t *__restrict__ sa, uint32_t *__restrict__ rank,
    uint8_t *__restrict__ fin, uint32_t *__restrict__ nid, uint32_t *__restrict__ nhd, uint32_t list_cap,
    uint32_t *count_out, uint32_t n, uint64_t *st_max, uint64_t *st_sum, uint32_t *tile_ctr, uint32_t epoch,
    uint32_t *err, int id_bits) {
  __shared__ uint64_t sk[kSTile + 2];  // key of element base - 1 + q (without the suffix bits)
  __shared__ uint32_t sv[kSTile];
  __shared__ uint32_t s_tile, s_pmax, s_psum;
  __shared__ uint32_t scr[kST / 32];
  const int tid = threadIdx.x;
  const uint32_t N = n_dev ? min(ub, *n_dev) : ub;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kSTile;
  if (base >= N) return;  // past the device-side count: no later tile looks at it
  const uint32_t cnt = (N - base) < (uint64_t)kSTile ? (uint32_t)(N - base) : (uint32_t)kSTile;
  // id_bits > 0: the suffix is the key's low id_bits bits (keys-only sort)
  const uint64_t idmask = id_bits ? (1ull << id_bits) - 1 : 0ull;
  for (uint32_t q = tid; q < cnt + 2; q += kST) {
    const long long g = (long long)base - 1 + q;
    const uint64_t kv = (g >= 0 && g < (long long)N) ? keys[g] : 0;
    sk[q] = kv >> id_bits;
    if (id_bits && q >= 1 && q <= cnt) sv[q - 1] = (uint32_t)(kv & idmask);
  }
  if (!id_bits)
    for (uint32_t q = tid; q < cnt; q += kST) sv[q] = vals[base + q];
  __syncthreads();

  const uint32_t e0 = tid * kSI;
  uint32_t hb = 0;  // bit i: element e0 + i starts a group (bit kSI: the element after)
#pragma unroll
  for (int i = 0; i <= kSI; ++i) {
    const uint32_t local = e0 + i;
    if (local <= cnt) {
      const uint64_t g = base + local;
      if (g == 0 || g == N || sk[local + 1] != sk[local]) hb |= 1u << i;
    }
  }
  uint32_t tmax = 0, tcnt = 0;
  bool thead = false;
#pragma unroll
  for (int i = 0; i < kSI; ++i) {
    if (e0 + i < cnt) {
      const bool h = (hb >> i) & 1u;
      if (h) {
        tmax = (uint32_t)(base + e0 + i);
        thead = true;
      }
      if (!(h && ((hb >> (i + 1)) & 1u))) ++tcnt;
    }
  }
  uint32_t tot_max, tot_sum;
  const uint32_t ex_max = block_exclusive<kST / 32>(tmax, OpMax(), 0u, scr, &tot_max);
  const uint32_t ex_sum = kBig ? 0u : block_exclusive<kST / 32>(tcnt, OpSum(), 0u, scr, &tot_sum);
  const int any_head = __syncthreads_or(thead);
  if (tid < 32) {
    const bool incl = t == 0 || any_head;  // a tile with a group start knows its maximum
    if (tid == 0) lb_store(&st_max[t], lb_pack(incl ? kLbInclusive : kLbAggregate, epoch, tot_max));
    uint32_t pm = 0;
    if (t > 0) pm = lb_exclusive_warp(st_max, 1, t, epoch, OpMax(), 0u, err);
    if (tid == 0) {
      if (!incl) lb_store(&st_max[t], lb_pack(kLbInclusive, epoch, max(pm, tot_max)));
      s_pmax = pm;
    }
  } else if (!kBig && tid < 64) {
    const uint32_t ps = lb_sum_warp(st_sum, t, tot_sum, epoch, err);
    if (tid == 32) {
      s_psum = ps;
      if (finals && base + cnt == N) *count_out = ps + tot_sum;
    }
  }
  __syncthreads();
  uint32_t hq = max(s_pmax, ex_max);  // index of the current group's first element
  uint32_t rs = kBig ? 0u : s_psum + ex_sum;
#pragma unroll
  for (int i = 0; i < kSI; ++i) {
    const uint32_t local = e0 + i;
    if (local >= cnt) break;
    const bool h = (hb >> i) & 1u;
    const uint32_t q = (uint32_t)(base + local);
    if (h) hq = q;
    const uint32_t id = sv[local];
    uint32_t slot = q, head = hq, at = 0;
    if (kBig) {
      const uint32_t o = (uint32_t)(sk[local + 1] >> ord_shift);
      if (o >= bg_cap) {
        atomicExch(err, kDevRange);
        continue;
      }
      const uint32_t hs = bg_head[o], bo = bg_off[o];
      slot = hs + (q - bo);
      head = hs + (hq - bo);
      at = bg_pos[o] + (q - bo);
    }
    if (id >= n || slot >= n || (kBig && at >= list_cap)) {
      atomicExch(err, kDevRange);
      continue;
    }
    const bool alone = finals && h && ((hb >> (i + 1)) & 1u);
    if (!alone) snap[id] = head;  // (a final suffix's level rank is its rank[])
    if (!finals) continue;
    if (alone) {
      sa[slot] = id;
      rank[id] = slot;
      fin[id] = (uint8_t)level;
      if (kBig) nhd[at] = kHole;
    } else if (kBig) {
      nid[at] = id;
      nhd[at] = head;
    } else {
      if (rs < list_cap) {
        nid[rs] = id;
        nhd[rs] = head;
      } else {
        atomicExch(err, kDevRange);
      }
      ++rs;
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
// The keys' lowest hist_bits bits are counted into hist (the sort's first
// digit place), so that the sort needs no histogram read of its own.
__global__ void k_pack0(const void *__restrict__ tokens, int tb, const uint32_t *__restrict__ codes, uint32_t n,
                        uint32_t h0, int cb, Windows W, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                        uint32_t *__restrict__ hist, int hist_bits) {
  __shared__ uint32_t sh[512];
  const uint32_t hmask = (1u << hist_bits) - 1;
  for (uint32_t d = threadIdx.x; d <= hmask; d += blockDim.x) sh[d] = 0;
  __syncthreads();
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
    atomicAdd(&sh[(uint32_t)key & hmask], 1u);
  }
  __syncthreads();
  for (uint32_t d = threadIdx.x; d <= hmask; d += blockDim.x)
    if (sh[d]) atomicAdd(&hist[d], sh[d]);
}

// ---------------------------------------------------------------- a doubling round
constexpr int kRdT = 1024;                     // list entries per tile
constexpr int kRdBig = 128;                    // a group with more entries is sorted globally ("big")
constexpr int kRdThreads = 256;
constexpr int kRdWarps = kRdThreads / 32;
constexpr int kRdDigit = 9;                    // digit bits of the in-tile sort
constexpr int kRdRadix = 1 << kRdDigit;
constexpr int kRdWin = kRdT + kRdBig + 1;      // positions a tile reads: its span and the next kRdBig + 1
constexpr int kRdRows = (kRdWin + kRdThreads - 1) / kRdThreads;  // rows of kRdThreads positions
constexpr int kRdPosBits = 11;                 // bits of a position in a sort key
constexpr int kRdHw0 = kRdBig + 2;             // list heads read before the span
constexpr int kRdHw = kRdWin + kRdHw0;
constexpr int kRdGroups = kRdWin / 2 + 2;      // group starts in the window (groups have two entries or more)
constexpr uint32_t kRdNoGroup = 0xffff;
static_assert(kRdWin <= (1 << kRdPosBits), "positions fit the key");
static_assert(kRdGroups < kRdNoGroup, "group numbers fit 16 bits");
static_assert(kRdRadix % kRdThreads == 0, "each thread owns whole digits");
constexpr size_t kRoundSmem = (size_t)kRdWin * 8 * 2           // sort keys (two buffers)
                              + (size_t)kRdHw * 4               // list heads
                              + (size_t)kRdWin * 4 * 2          // minor keys, suffixes by position
                              + (size_t)(kRdGroups + 1) * 4     // group starts
                              + (size_t)kRdGroups * 4 * 3       // group heads, big indices, first entries
                              + (size_t)kRdWin * 2              // group of each position
                              + (size_t)kRdWarps * kRdRadix * 2;  // per-warp digit counts

struct RoundArgs {
  const uint32_t *lid, *lhd;   // this round's list: suffix, head slot of its group
  const uint32_t *mkey;        // minor key of each entry (k_minor)
  uint32_t ub;                 // launch bound on the list length
  const uint32_t *A_dev;       // the list length
  uint32_t r, h, n;            // round, doubling offset, positions
  const uint32_t *wsb;         // window-start bits (bit n set), null for one window
  const uint32_t *wid, *woff;  // window of each position and window offsets (several windows)
  uint8_t *fin;
  uint32_t *rank, *sa;
  const uint32_t *snap_prev;   // level r - 1
  uint32_t *snap_cur;          // level r
  uint32_t *hid, *hhd;         // the next list with holes: entry k of a small group settled in place
  uint64_t *bkeys;             // big entries: (ordinal << mb) | minor relative to the window
  uint32_t *bvals;
  uint32_t *bg_head, *bg_off, *bg_pos;  // per big group: head slot, first big entry, first list entry
  uint32_t bg_cap;
  int mb;
  int id_bits;                 // > 0: big keys carry the suffix in their low id_bits bits (no values)
  uint32_t *big_hist;          // digit counts of the big keys' lowest hist_bits bits
  int hist_bits;
  uint32_t *words;             // [1] big entries, [3] big groups (of the round)
  uint64_t *st_bc, *st_bs;
  uint32_t *tile_ctr;
  uint32_t epoch;
  uint32_t *err;
};

__device__ __forceinline__ int bits_for_dev(uint32_t v) { return v ? 32 - __clz(v) : 0; }

// Exclusive counts of flags over the tile's rows (item (i, tid) is number
// i * kRdThreads + tid; bit i of `bits` is row i's flag): warp ballots, one
// pass of warp 0 over the (row, warp) counts.  ex[i] receives the flags
// before item (i, tid); *total all of them.
__device__ __forceinline__ void flags_exclusive(uint32_t bits, int rows, uint32_t *rowtot,
                                                uint32_t (&ex)[kRdRows], uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  uint32_t pre[kRdRows];
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= rows) break;
    const uint32_t b = __ballot_sync(0xffffffffu, (bits >> i) & 1u);
    pre[i] = __popc(b & lt);
    if (lane == 0) rowtot[i * kRdWarps + warp] = __popc(b);
  }
  __syncthreads();
  if (warp == 0) {  // (row, warp) counts in row-major order: 2 per lane
    const int m = rows * kRdWarps;
    const uint32_t c0 = 2 * lane < m ? rowtot[2 * lane] : 0u, c1 = 2 * lane + 1 < m ? rowtot[2 * lane + 1] : 0u;
    const uint32_t inc = warp_inclusive(c0 + c1, OpSum());
    if (2 * lane < m) rowtot[2 * lane] = inc - c0 - c1;
    if (2 * lane + 1 < m) rowtot[2 * lane + 1] = inc - c1;
    if (lane == 31) rowtot[kRdRows * kRdWarps] = inc;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= rows) break;
    ex[i] = rowtot[i * kRdWarps + warp] + pre[i];
  }
  *total = rowtot[kRdRows * kRdWarps];
  __syncthreads();
}

// Two flag sets at once (their counts packed in 16-bit halves: a tile's
// totals stay below 2^16): the exclusive counts of both, one scan.
__device__ __forceinline__ void flags_exclusive2(uint32_t bits_a, uint32_t bits_b, int rows, uint32_t *rowtot,
                                                 uint32_t (&ex_a)[kRdRows], uint32_t (&ex_b)[kRdRows],
                                                 uint32_t *total_a, uint32_t *total_b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  uint32_t pre[kRdRows];
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= rows) break;
    const uint32_t ba = __ballot_sync(0xffffffffu, (bits_a >> i) & 1u);
    const uint32_t bb = __ballot_sync(0xffffffffu, (bits_b >> i) & 1u);
    pre[i] = __popc(ba & lt) | (__popc(bb & lt) << 16);
    if (lane == 0) rowtot[i * kRdWarps + warp] = __popc(ba) | (__popc(bb) << 16);
  }
  __syncthreads();
  if (warp == 0) {  // (row, warp) counts in row-major order: 2 per lane
    const int m = rows * kRdWarps;
    const uint32_t c0 = 2 * lane < m ? rowtot[2 * lane] : 0u, c1 = 2 * lane + 1 < m ? rowtot[2 * lane + 1] : 0u;
    const uint32_t inc = warp_inclusive(c0 + c1, OpSum());
    if (2 * lane < m) rowtot[2 * lane] = inc - c0 - c1;
    if (2 * lane + 1 < m) rowtot[2 * lane + 1] = inc - c1;
    if (lane == 31) rowtot[kRdRows * kRdWarps] = inc;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= rows) break;
    const uint32_t e = rowtot[i * kRdWarps + warp] + pre[i];
    ex_a[i] = e & 0xffffu;
    ex_b[i] = e >> 16;
  }
  const uint32_t t = rowtot[kRdRows * kRdWarps];
  *total_a = t & 0xffffu;
  *total_b = t >> 16;
  __syncthreads();
}

// Minor key of every list entry of round r: rank_{r-1}[i + h] + 1, or 0
// when i + h is past the window's end (absolute slots).  A streaming pass
// with independent loads in flight, so that the round kernel reads the keys
// in order instead of chasing three dependent loads per entry.
__global__ void __launch_bounds__(256) k_minor(const uint32_t *__restrict__ lid, uint32_t ub,
                                               const uint32_t *__restrict__ A_dev, uint32_t r, uint32_t h,
                                               uint32_t n, const uint32_t *__restrict__ wsb,
                                               const uint8_t *__restrict__ fin, const uint32_t *__restrict__ rank,
                                               const uint32_t *__restrict__ snap_prev, uint32_t *__restrict__ mout) {
  constexpr int kI = 4;
  const uint32_t A = min(ub, *A_dev);
  for (uint64_t k0 = ((uint64_t)blockIdx.x * blockDim.x) * kI + threadIdx.x; k0 < A;
       k0 += (uint64_t)gridDim.x * blockDim.x * kI) {
    uint32_t j[kI];
#pragma unroll
    for (int u = 0; u < kI; ++u) {
      const uint64_t k = k0 + (uint64_t)u * blockDim.x;
      const uint32_t i = k < A ? lid[k] : n;
      const uint32_t x = i < n ? i + h : n;
      j[u] = (x >= n || (wsb && bit_at(wsb, x))) ? n : x;  // n: past the end
    }
    uint8_t fb[kI];
#pragma unroll
    for (int u = 0; u < kI; ++u) fb[u] = j[u] < n ? fin[j[u]] : 0;
#pragma unroll
    for (int u = 0; u < kI; ++u) {
      const uint64_t k = k0 + (uint64_t)u * blockDim.x;
      if (k < A) mout[k] = j[u] < n ? ((uint32_t)fb[u] <= r - 1 ? rank[j[u]] : snap_prev[j[u]]) + 1 : 0u;
    }
  }
}

__global__ void __launch_bounds__(kRdThreads, 4) k_round(const RoundArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  // positions q of the tile's window are list entries base + q
  uint64_t *ka = reinterpret_cast<uint64_t *>(smem);  // [kRdWin] sort keys of the small groups' entries
  uint64_t *kb = ka + kRdWin;
  uint32_t *hw = reinterpret_cast<uint32_t *>(kb + kRdWin);  // [kRdHw] list heads from base - kRdHw0
  uint32_t *mv = hw + kRdHw;                           // [kRdWin] minor key by position
  uint32_t *sid = mv + kRdWin;                         // [kRdWin] suffix by position
  uint32_t *gst = sid + kRdWin;                        // [kRdGroups + 1] group start positions
  uint32_t *ghd = gst + kRdGroups + 1;                 // [kRdGroups] group head slots
  uint32_t *gbx = ghd + kRdGroups;                     // [kRdGroups] big group: its index; small: kNone
  uint32_t *gfs = gbx + kRdGroups;                     // [kRdGroups] big: first big entry; small: first sorted entry
  uint16_t *gid = reinterpret_cast<uint16_t *>(gfs + kRdGroups);  // [kRdWin] group of each position
  uint16_t *wcs = gid + kRdWin;                        // [kRdWarps][kRdRadix] per-warp digit counts
  __shared__ uint32_t rowtot[kRdRows * kRdWarps + 1];
  __shared__ uint32_t s_tile, s_G, s_BC, s_BS, s_cov, s_mmin, s_mmax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = lanemask_lt();
  if (tid == 0) {
    s_tile = atomicAdd(a.tile_ctr, 1u);
    s_mmin = kNone;
    s_mmax = 0;
  }
  const uint32_t A = min(a.ub, *a.A_dev);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base64 = (uint64_t)t * kRdT;
  if (base64 >= A) return;  // past the list: no later tile looks at it
  const uint32_t base = (uint32_t)base64;
  const uint32_t span_end = min(base + (uint32_t)kRdT, A);
  const uint32_t span = span_end - base;
  const uint32_t lim = min(A - base, span + (uint32_t)kRdBig + 1);  // positions read: [0, lim)
  // list heads of entries base - kRdHw0 .. base + lim - 1; suffixes and
  // minor keys of entries base .. base + lim - 1 (all loads at once)
  {
    constexpr int kHr = (kRdHw + kRdThreads - 1) / kRdThreads;
    uint32_t rh[kHr], ri[kRdRows], rm[kRdRows];
#pragma unroll
    for (int i = 0; i < kHr; ++i) {
      const uint32_t q = i * kRdThreads + tid;
      const long long k = (long long)base - kRdHw0 + q;
      rh[i] = (q < lim + kRdHw0 && k >= 0) ? a.lhd[k] : kNone;
    }
#pragma unroll
    for (int i = 0; i < kRdRows; ++i) {
      const uint32_t q = i * kRdThreads + tid;
      ri[i] = q < lim ? a.lid[base + q] : 0u;
      rm[i] = q < lim ? a.mkey[base + q] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kHr; ++i) {
      const uint32_t q = i * kRdThreads + tid;
      if (q < lim + kRdHw0) hw[q] = rh[i];
    }
#pragma unroll
    for (int i = 0; i < kRdRows; ++i) {
      const uint32_t q = i * kRdThreads + tid;
      if (q < lim) {
        sid[q] = ri[i];
        mv[q] = rm[i];
      }
    }
  }
  __syncthreads();
  // group starts among positions [0, lim), numbered in order
  const int rows = (int)((lim + kRdThreads - 1) / kRdThreads);
  uint32_t stb = 0, gex[kRdRows], gall;
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= rows) break;
    const uint32_t q = i * kRdThreads + tid;
    if (q < lim && hw[q + kRdHw0] != hw[q + kRdHw0 - 1]) stb |= 1u << i;
  }
  flags_exclusive(stb, rows, rowtot, gex, &gall);
  gall = min(gall, (uint32_t)kRdGroups);
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= rows) break;
    const uint32_t q = i * kRdThreads + tid;
    if (q < lim) {
      const uint32_t s = (stb >> i) & 1u;
      if (s && gex[i] < kRdGroups) gst[gex[i]] = q;
      if (s && gex[i] >= kRdGroups) atomicExch(a.err, kDevRange);  // list groups have two entries or more
      gid[q] = gex[i] + s == 0 ? (uint16_t)kRdNoGroup : (uint16_t)min(gex[i] + s - 1, (uint32_t)kRdGroups - 1);
    }
  }
  __syncthreads();
  if (tid == 0) {
    // groups starting in the span, and where the last of them ends: the next
    // start, or the list's end when it lies in the window, else unknown
    uint32_t lo = 0, hi = gall;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) / 2;
      if (gst[mid] < span) lo = mid + 1; else hi = mid;
    }
    s_G = lo;
    gst[gall] = lim == A - base ? lim : kNone;
    // the group covering [0, f): big iff it has more than kRdBig entries, i.e.
    // it covers the whole span or the entry kRdBig places before its end is
    // still in it
    const uint32_t f = lo ? gst[0] : span;
    bool cov = false;
    if (f > 0) {
      if (lo == 0 && span == (uint32_t)kRdT) {
        cov = true;
      } else {
        const long long x = (long long)(lo ? f : A - base) - kRdBig - 1;  // relative to base, >= -kRdBig - 1
        cov = (long long)base + x >= 0 && hw[x + kRdHw0] == hw[kRdHw0];
      }
    }
    s_cov = cov;
  }
  __syncthreads();
  const uint32_t G = s_G;
  const uint32_t f = G ? gst[0] : span;  // entries before f belong to a group that started earlier
  const bool cov_big = s_cov != 0;
  // big groups: more than kRdBig entries (or not ending in the window)
  const int grows = (int)((G + kRdThreads - 1) / kRdThreads);
  uint32_t gbb = 0, gbxe[kRdRows], bs_tile;
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= grows) break;
    const uint32_t g = i * kRdThreads + tid;
    if (g < G) {
      const uint32_t q0 = gst[g], nx = gst[g + 1];
      ghd[g] = hw[q0 + kRdHw0];
      if (nx == kNone || nx - q0 > (uint32_t)kRdBig) gbb |= 1u << i;
    }
  }
  flags_exclusive(gbb, grows, rowtot, gbxe, &bs_tile);
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= grows) break;
    const uint32_t g = i * kRdThreads + tid;
    if (g < G) gbx[g] = ((gbb >> i) & 1u) ? gbxe[i] : kNone;
  }
  __syncthreads();
  // per position: in a small group of this tile (sorted here), or a big
  // entry of the span (keyed for the global sort); their numbers in order
  uint32_t gend = span;
  if (G && gbx[G - 1] == kNone) gend = max(gend, gst[G]);
  const int mrows = (int)((gend + kRdThreads - 1) / kRdThreads);
  uint32_t smb = 0, bgb = 0;
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= mrows) break;
    const uint32_t q = i * kRdThreads + tid;
    if (q < gend) {
      if (q < f) {
        if (cov_big) bgb |= 1u << i;
      } else {
        const uint32_t g = gid[q];
        if (g < G && gbx[g] == kNone) smb |= 1u << i;
        else if (g < G && q < span) bgb |= 1u << i;
      }
    }
  }
  uint32_t sx[kRdRows], bx[kRdRows], S, bc;
  flags_exclusive2(smb, bgb, mrows, rowtot, sx, bx, &S, &bc);
  // the tile's big entries and big groups are known: their prefixes over the
  // tiles before, resolved at once so that inclusive prefixes spread through
  // the tiles in flight and every walk back stays short
  if (warp == 0) {
    const uint32_t p = lb_sum_warp(a.st_bc, t, bc, a.epoch, a.err);
    if (lane == 0) s_BC = p;
  } else if (warp == 1) {
    const uint32_t p = lb_sum_warp(a.st_bs, t, bs_tile, a.epoch, a.err);
    if (lane == 0) s_BS = p;
  }
  // a group's first small or big entry
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= mrows) break;
    const uint32_t q = i * kRdThreads + tid;
    if (q >= f && q < gend && ((stb >> i) & 1u)) {
      const uint32_t g = gid[q];
      if (g < G) gfs[g] = ((smb >> i) & 1u) ? sx[i] : bx[i];
    }
  }

  // the small groups' minor key range
  {
    uint32_t lmin = kNone, lmax = 0;
#pragma unroll
    for (int i = 0; i < kRdRows; ++i) {
      if (i >= mrows) break;
      if ((smb >> i) & 1u) {
        const uint32_t m = mv[i * kRdThreads + tid];
        lmin = min(lmin, m);
        lmax = max(lmax, m);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
      lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    }
    if (lane == 0 && lmin != kNone) {
      atomicMin(&s_mmin, lmin);
      atomicMax(&s_mmax, lmax);
    }
  }
  __syncthreads();

  // ---- the small groups' entries sorted by (group, minor), block-wide LSD
  // radix with kRdDigit-bit digits, stable: warp w ranks the contiguous
  // entries [w * R, (w + 1) * R) in order
  const uint32_t mmin = s_mmin;
  const int mbits = S ? bits_for_dev(s_mmax - mmin) : 0;
  const int gbits = bits_for_dev(G ? G - 1 : 0);
  const int B = gbits + mbits;
#pragma unroll
  for (int i = 0; i < kRdRows; ++i) {
    if (i >= mrows) break;
    const uint32_t q = i * kRdThreads + tid;
    if ((smb >> i) & 1u)
      ka[sx[i]] = ((((uint64_t)gid[q] << mbits) | (uint64_t)(mv[q] - mmin)) << kRdPosBits) | q;
  }
  __syncthreads();
  uint64_t *src = ka, *dst = kb;
  const int srows = (int)((S + kRdThreads - 1) / kRdThreads);  // rows of 32 per warp
  const uint32_t R = (uint32_t)srows * 32;
  for (int sh = kRdPosBits; sh < kRdPosBits + B && S > 1; sh += kRdDigit) {
    uint16_t *mywc = wcs + warp * kRdRadix;
    for (int d = lane; d < kRdRadix; d += 32) mywc[d] = 0;
    __syncwarp();
    uint32_t rk[kRdRows], dg[kRdRows];
    uint64_t kr[kRdRows];
#pragma unroll
    for (int j = 0; j < kRdRows; ++j) {
      if (j >= srows) break;
      const uint32_t p = warp * R + j * 32 + lane;
      const bool v = p < S;
      kr[j] = v ? src[p] : 0ull;
      const uint32_t d = v ? (uint32_t)(kr[j] >> sh) & (kRdRadix - 1) : (uint32_t)kRdRadix;
      dg[j] = d;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t b = 0;
      if (v) b = mywc[d];
      __syncwarp();
      rk[j] = 0;
      if (v) {
        rk[j] = b + __popc(peers & lt);
        if ((peers & lt) == 0) mywc[d] = (uint16_t)(b + __popc(peers));
      }
      __syncwarp();
    }
    __syncthreads();
    // thread tid owns digits 2 tid, 2 tid + 1: warp-major prefixes, then the bases
    uint32_t run = 0;
#pragma unroll
    for (int dd = 0; dd < kRdRadix / kRdThreads; ++dd) {
      const int d = tid * (kRdRadix / kRdThreads) + dd;
#pragma unroll
      for (int w = 0; w < kRdWarps; ++w) {
        const uint32_t c = wcs[w * kRdRadix + d];
        wcs[w * kRdRadix + d] = (uint16_t)run;
        run += c;
      }
    }
    uint32_t tot;
    const uint32_t dbase = block_exclusive<kRdWarps>(run, OpSum(), 0u, rowtot, &tot);
#pragma unroll
    for (int dd = 0; dd < kRdRadix / kRdThreads; ++dd) {
      const int d = tid * (kRdRadix / kRdThreads) + dd;
#pragma unroll
      for (int w = 0; w < kRdWarps; ++w) wcs[w * kRdRadix + d] += (uint16_t)dbase;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRdRows; ++j) {
      if (j >= srows) break;
      const uint32_t p = warp * R + j * 32 + lane;
      if (p < S) dst[mywc[dg[j]] + rk[j]] = kr[j];
    }
    __syncthreads();
    uint64_t *x = src;
    src = dst;
    dst = x;
  }

  // ---- settle the sorted entries: subgroups of equal (group, minor)
  {
    const int csh = kRdPosBits;
    uint32_t stf = 0, enf = 0;
#pragma unroll
    for (int i = 0; i < kRdRows; ++i) {
      if (i >= srows) break;
      const uint32_t p = i * kRdThreads + tid;
      if (p < S) {
        const uint64_t c = src[p] >> csh;
        const uint32_t g = (uint32_t)(c >> mbits);
        if (p == 0 || (src[p - 1] >> csh) != c || gfs[g] == p) stf |= 1u << i;
        if (p + 1 == S || (src[p + 1] >> csh) != c) enf |= 1u << i;
      }
    }
    // the last subgroup start at or before each entry: ballots in a row, the
    // (row, warp) carry through warp 0
#pragma unroll
    for (int i = 0; i < kRdRows; ++i) {
      if (i >= srows) break;
      const uint32_t b = __ballot_sync(0xffffffffu, (stf >> i) & 1u);
      if (lane == 0) rowtot[i * kRdWarps + warp] = b ? i * kRdThreads + warp * 32 + (31 - __clz(b)) + 1 : 0u;
    }
    __syncthreads();
    if (warp == 0) {
      const int m = srows * kRdWarps;
      uint32_t c0 = 2 * lane < m ? rowtot[2 * lane] : 0u, c1 = 2 * lane + 1 < m ? rowtot[2 * lane + 1] : 0u;
      const uint32_t inc = warp_inclusive(max(c0, c1), OpMax());
      const uint32_t before = __shfl_up_sync(0xffffffffu, inc, 1);
      const uint32_t ex0 = lane ? before : 0u;
      if (2 * lane < m) rowtot[2 * lane] = ex0;
      if (2 * lane + 1 < m) rowtot[2 * lane + 1] = max(ex0, c0);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRdRows; ++i) {
      if (i >= srows) break;
      const uint32_t p = i * kRdThreads + tid;
      const uint32_t b = __ballot_sync(0xffffffffu, (stf >> i) & 1u) & (lt | (1u << lane));
      if (p >= S) continue;
      const uint32_t hp = b ? i * kRdThreads + warp * 32 + (31 - __clz(b)) : rowtot[i * kRdWarps + warp] - 1;
      const uint64_t key = src[p];
      const uint32_t q = (uint32_t)key & ((1u << kRdPosBits) - 1);
      const uint32_t g = (uint32_t)(key >> (csh + mbits));
      if (g >= G) {
        atomicExch(a.err, kDevRange);
        continue;
      }
      const uint32_t id = sid[q], k = p - gfs[g], hk = hp - gfs[g];
      const uint32_t slot = ghd[g] + k, head = ghd[g] + hk, at = base + gst[g] + k;
      if (id >= a.n || slot >= a.n || at >= a.ub) {
        atomicExch(a.err, kDevRange);
        continue;
      }
      if (((stf >> i) & 1u) && ((enf >> i) & 1u)) {  // alone in its subgroup: final
        a.sa[slot] = id;
        a.rank[id] = slot;
        a.fin[id] = (uint8_t)a.r;
        a.hhd[at] = kHole;
      } else {
        a.snap_cur[id] = head;
        a.hid[at] = id;
        a.hhd[at] = head;
      }
    }
  }

  // ---- big entries of the span: (ordinal, minor relative to the window),
  // and each big group's head, first big entry and first list entry
  const uint32_t BC = s_BC, BS = s_BS;  // (read after the barriers since they were set)
  if (bc) {
    // kb may hold the sorted keys the settle just read: every warp is done
    // with them before it becomes the digit counts of the big keys
    __syncthreads();
    uint32_t *hcnt = reinterpret_cast<uint32_t *>(kb);
    const uint32_t hmask = (1u << a.hist_bits) - 1;
    for (uint32_t d = tid; d <= hmask; d += kRdThreads) hcnt[d] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRdRows; ++i) {
      if (i >= mrows) break;
      if (!((bgb >> i) & 1u)) continue;
      const uint32_t q = i * kRdThreads + tid;
      const uint32_t o = q < f ? BS - 1 : BS + gbx[gid[q]];
      const uint32_t i2 = sid[q];
      uint32_t m = mv[q];
      if (m && a.woff && i2 < a.n) m -= a.woff[a.wid[i2]];
      const uint64_t key = ((uint64_t)o << a.mb) | m;
      const uint32_t j = BC + bx[i];
      if (j < a.ub && o < a.bg_cap && i2 < a.n) {
        if (a.id_bits) {
          a.bkeys[j] = (key << a.id_bits) | i2;
        } else {
          a.bkeys[j] = key;
          a.bvals[j] = i2;
        }
        atomicAdd(&hcnt[(uint32_t)key & hmask], 1u);
      } else {
        atomicExch(a.err, kDevRange);
      }
    }
    for (uint32_t g = tid; g < G; g += kRdThreads) {
      if (gbx[g] == kNone) continue;
      const uint32_t o = BS + gbx[g];
      if (o < a.bg_cap) {
        a.bg_head[o] = ghd[g];
        a.bg_off[o] = BC + gfs[g];
        a.bg_pos[o] = base + gst[g];
      } else {
        atomicExch(a.err, kDevRange);
      }
    }
    __syncthreads();
    for (uint32_t d = tid; d <= hmask; d += kRdThreads)
      if (hcnt[d]) atomicAdd(&a.big_hist[d], hcnt[d]);
  }
  if (tid == 0 && span_end == A) {
    a.words[1] = BC + bc;
    a.words[3] = BS + bs_tile;
  }
}

// The holed next list (entries settled in place, holes where a suffix became
// final) -> the dense next list, order kept; its length lands in *count_out.
constexpr int kLcT = 256, kLcI = 8, kLcTile = kLcT * kLcI;
__global__ void __launch_bounds__(kLcT) k_list_compact(const uint32_t *__restrict__ hid,
                                                       const uint32_t *__restrict__ hhd, uint32_t ub,
                                                       const uint32_t *__restrict__ A_dev,
                                                       uint32_t *__restrict__ nid, uint32_t *__restrict__ nhd,
                                                       uint32_t n, uint32_t *count_out, uint64_t *status,
                                                       uint32_t *tile_ctr, uint32_t epoch, uint32_t *err) {
  __shared__ uint32_t s_tile, s_pre;
  __shared__ uint32_t scr[kLcT / 32];
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  const uint32_t A = min(ub, *A_dev);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kLcTile;
  if (base >= A) return;
  uint32_t hd[kLcI], cnt = 0;
#pragma unroll
  for (int i = 0; i < kLcI; ++i) {
    const uint64_t k = base + (uint64_t)tid * kLcI + i;
    hd[i] = k < A ? hhd[k] : kHole;
    cnt += hd[i] != kHole;
  }
  uint32_t tot;
  const uint32_t ex = block_exclusive<kLcT / 32>(cnt, OpSum(), 0u, scr, &tot);
  if (tid < 32) {
    const uint32_t p = lb_sum_warp(status, t, tot, epoch, err);
    if (tid == 0) {
      s_pre = p;
      if (base + kLcTile >= A) *count_out = p + tot;
    }
  }
  __syncthreads();
  uint32_t rs = s_pre + ex;
#pragma unroll
  for (int i = 0; i < kLcI; ++i) {
    if (hd[i] == kHole) continue;
    const uint64_t k = base + (uint64_t)tid * kLcI + i;
    if (rs < n) {
      nid[rs] = hid[k];
      nhd[rs] = hd[i];
    } else {
      atomicExch(err, kDevRange);
    }
    ++rs;
  }
}

// Window-start bits: bit off[w] for w >= 1, and bit n.
__global__ void k_wsb(const uint32_t *__restrict__ off, uint32_t count, uint32_t n, uint32_t *bits) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w <= count; w += gridDim.x * blockDim.x) {
    const uint32_t j = w < count ? off[w + 1] : n;
    if (w < count && j >= n) continue;
    atomicOr(&bits[j >> 5], 1u << (j & 31));
  }
}

// Batched first round: key = (window << 32) | level-0 rank of the token among
// all tokens, so that suffixes of different windows never share a group.
__global__ void k_wkeys(const uint32_t *__restrict__ r0, Windows W, uint32_t n,
                        uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    keys[i] = ((uint64_t)win_id(W, i) << 32) | r0[i];
    vals[i] = i;
  }
}

// Phi[SA[k]] = SA[k-1] within a window (a window's first slot has none).
__global__ void k_phi(const uint32_t *__restrict__ sa, uint32_t n, const uint32_t *__restrict__ wsb,
                      uint32_t *__restrict__ phi) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t i = sa[k];
    const bool first = k == 0 || (wsb && bit_at(wsb, k));
    if (i < n) phi[i] = first ? kNone : sa[k - 1];
  }
}

// PLCP[i] = lcp(i, Phi[i]) over chunks of kPChunk consecutive i per thread.
// Tokens are compared directly for up to kPDirect steps; a match that keeps
// going is finished by lifting over the level ranks: level lev ranks are
// equal iff the next h0 * 2^lev tokens are, from the top level down (level
// lev's snapshot at snap0 + lev * n).
constexpr int kPChunk = 16;
constexpr uint32_t kPDirect = 256;
template <class T>
__global__ void k_plcp(const T *__restrict__ S, uint32_t n, Windows W, const uint32_t *__restrict__ wsb,
                       const uint32_t *__restrict__ phi, const uint8_t *__restrict__ fin,
                       const uint32_t *__restrict__ rank, const uint32_t *__restrict__ snap0, int levels,
                       uint32_t h0, uint32_t *__restrict__ plcp) {
  const uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * kPChunk;
  if (i0 >= n) return;
  const uint32_t iend = (i0 + kPChunk) < (uint64_t)n ? (uint32_t)(i0 + kPChunk) : n;
  uint32_t l = 0;
  for (uint32_t i = (uint32_t)i0; i < iend; ++i) {
    const uint32_t j = phi[i];
    if (i > i0 && wsb && bit_at(wsb, i)) l = 0;  // a new window starts
    if (j >= n) {
      plcp[i] = 0;
      l = 0;
      continue;
    }
    const uint32_t we = win_end(W, i, n);  // i and j lie in the same window
    // tokens left to compare in both suffixes (0 if j is not before the
    // window's end: only a suffix array from a replay whose checks failed,
    // and whose results are discarded, can hold such a pair)
    const uint32_t lim = max(i, j) < we ? we - max(i, j) : 0u;
    uint32_t steps = 0;
    // four token pairs per step (eight independent loads in flight), then
    // one at a time near the window's end
    for (bool more = true; more && steps < kPDirect;) {
      if (l + 4 <= lim) {
        const T a0 = S[i + l], a1 = S[i + l + 1], a2 = S[i + l + 2], a3 = S[i + l + 3];
        const T b0 = S[j + l], b1 = S[j + l + 1], b2 = S[j + l + 2], b3 = S[j + l + 3];
        if (a0 != b0) {
          more = false;
        } else if (a1 != b1) {
          l += 1;
          more = false;
        } else if (a2 != b2) {
          l += 2;
          more = false;
        } else if (a3 != b3) {
          l += 3;
          more = false;
        } else {
          l += 4;
          steps += 4;
        }
      } else if (l < lim && S[i + l] == S[j + l]) {
        ++l;
        ++steps;
      } else {
        more = false;
      }
    }
    if (steps >= kPDirect) {
      for (int lev = levels - 1; lev >= 0; --lev) {
        const uint64_t x = (uint64_t)i + l, y = (uint64_t)j + l;
        if (x < we && y < we &&
            level_rank(fin, rank, snap0 + (size_t)lev * n, (uint32_t)lev, (uint32_t)x) ==
                level_rank(fin, rank, snap0 + (size_t)lev * n, (uint32_t)lev, (uint32_t)y))
          l += h0 << lev;
      }
      // what remains is shorter than h0 tokens
      for (uint32_t k = 1; k < h0 && i + (uint64_t)l < we && j + (uint64_t)l < we && S[i + l] == S[j + l]; ++k)
        ++l;
    }
    plcp[i] = l;
    l = l ? l - 1 : 0;
  }
}

__global__ void k_lcp_perm(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ plcp, uint32_t n,
                           const uint32_t *__restrict__ wsb, uint32_t *__restrict__ lcp) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const bool last = k + 1 >= n || (wsb && bit_at(wsb, k + 1));
    const uint32_t x = last ? 0u : sa[k + 1];
    lcp[k] = (last || x >= n) ? 0u : plcp[x];
  }
}

// Launches k_split over ub sorted pairs (exactly *n_dev when given).  With
// big = false the slot of sorted element q is q and the list length lands in
// *count_out; with big = true the groups' tables place slots and list entries.
int split_launch(apo_ctx *c, bool big, const uint64_t *keys, const uint32_t *vals, uint32_t ub,
                 const uint32_t *n_dev, int ord_shift, const uint32_t *bg_head, const uint32_t *bg_off,
                 const uint32_t *bg_pos, uint32_t bg_cap, uint32_t level, bool finals, uint32_t *snap,
                 SuffixState &st, uint32_t *nid, uint32_t *nhd, uint32_t *count_out, cudaStream_t s,
                 int id_bits = 0) {
  const int tiles = std::max(1, ceil_div(ub, kSTile));
  APO_TRY(ensure_lookback(c, (size_t)2 * tiles));
  uint32_t *misc = c->ps.counters + kCtrMisc;
  APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscRefreshTiles, 0, sizeof(uint32_t), s));
  const uint32_t ep = next_epoch(c);
  Launch lp_(c, kKSplit, ub, s);
  if (big)
    k_split<true><<<tiles, kST, 0, s>>>(keys, vals, ub, n_dev, ord_shift, bg_head, bg_off, bg_pos, bg_cap, level,
                                        finals, snap, st.sa, st.rank, st.fin, nid, nhd, st.n, count_out, st.n,
                                        c->ps.lookback, c->ps.lookback + tiles, misc + kMiscRefreshTiles, ep,
                                        c->ps.err, id_bits);
  else
    k_split<false><<<tiles, kST, 0, s>>>(keys, vals, ub, n_dev, 0, nullptr, nullptr, nullptr, 0, level, finals,
                                         snap, st.sa, st.rank, st.fin, nid, nhd, st.n, count_out, st.n,
                                         c->ps.lookback, c->ps.lookback + tiles, misc + kMiscRefreshTiles, ep,
                                         c->ps.err, 0);
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
  APO_CUDA_TRY(cudaFuncSetAttribute(k_round, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRoundSmem));
  return APO_OK;
}

size_t suffix_workspace_bytes(uint64_t n) {
  const int levels = bits_for(n) + 2;
  const uint64_t cap = dict_capacity((uint32_t)std::min<uint64_t>(n, 0xffffffffull));
  return (size_t)n * (2 * 8 + 2 * 4)        // sort pairs
         + (size_t)n * 4 * 6                // two lists of (suffix, head), the holed list
         + (size_t)n * (1 + 4 + 4)          // fin; phi and plcp
         + (size_t)(n / 32 + 2) * 4         // window-start bits
         + (size_t)(n / (kRdBig + 1) + 2) * 12  // big-group table
         + (size_t)levels * n * 4 + 16 * 256 +
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
  uint32_t *lid[2] = {c->arena.take_n<uint32_t>(n), c->arena.take_n<uint32_t>(n)};
  uint32_t *lhd[2] = {c->arena.take_n<uint32_t>(n), c->arena.take_n<uint32_t>(n)};
  const uint32_t bg_cap = n / (kRdBig + 1) + 2;  // big groups have more than kRdBig entries
  uint32_t *bg_head = c->arena.take_n<uint32_t>(bg_cap);
  uint32_t *bg_off = c->arena.take_n<uint32_t>(bg_cap);
  uint32_t *bg_pos = c->arena.take_n<uint32_t>(bg_cap);
  uint32_t *mkey = c->arena.take_n<uint32_t>(n);  // minor keys of a round's list
  uint32_t *hid = c->arena.take_n<uint32_t>(n);  // the holed next list of a round
  uint32_t *hhd = c->arena.take_n<uint32_t>(n);
  st.fin = c->arena.take_n<uint8_t>(n);
  const size_t wsb_words = (size_t)n / 32 + 2;
  st.wsb = st.win.count > 1 ? c->arena.take_n<uint32_t>(wsb_words) : nullptr;
  if (!b.keys[0] || !b.keys[1] || !b.vals[0] || !b.vals[1] || !lid[0] || !lid[1] || !lhd[0] || !lhd[1] ||
      !bg_head || !bg_off || !bg_pos || !mkey || !hid || !hhd || !st.fin || (st.win.count > 1 && !st.wsb)) {
    set_error("suffix array: workspace too small");
    return APO_ENOMEM;
  }
  const int g = grid_for(n, 256, c->num_sms);
  APO_CUDA_TRY(cudaMemsetAsync(st.fin, 0xff, n, s));
  if (st.wsb) {
    APO_CUDA_TRY(cudaMemsetAsync(st.wsb, 0, wsb_words * 4, s));
    Launch lp_(c, kKWsb, st.win.count, s);
    k_wsb<<<grid_for(st.win.count + 1, 256, c->num_sms), 256, 0, s>>>(st.win.off_dev, st.win.count, n, st.wsb);
  }
  // how many token bits are populated (for u64 tokens the dictionary of
  // distinct tokens is filled in the same round trip)
  uint32_t *misc = c->ps.counters + kCtrMisc;
  uint64_t *kor = reinterpret_cast<uint64_t *>(misc + kMiscKeyOr);
  APO_CUDA_TRY(cudaMemsetAsync(kor, 0, 2 * sizeof(uint64_t), s));
  {
    Launch lp_(c, kKKeyOr, n, s);
    k_token_or<<<std::min(1024, ceil_div(n, 256 * 8)), 256, 0, s>>>(tokens, tb, n,
                                                                     reinterpret_cast<unsigned long long *>(kor));
  }
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
  // level 0: groups of equal first h0 tokens (within a window)
  uint32_t *first_count = misc + kMiscRefreshCount;
  if (h0 >= 2) {
    h0 = std::min<uint32_t>(h0, 32);
    const DigitRange r{0, wb + (int)h0 * cb, false};
    SortPlan sp;
    APO_TRY(sort_plan(c, n, &r, 1, &sp, s));
    APO_TRY(sort_first_hist_clear(c, s));
    {
      Launch lp_(c, kKInitKeys, n, s);
      k_pack0<<<g, 256, 0, s>>>(tokens, tb, codes, n, h0, cb, st.win, b.keys[0], b.vals[0], sort_first_hist(c),
                                sp.shape >= 0 ? sp.bits : 8);
    }
    b.cur = 0;
    APO_TRY(radix_sort_planned(c, b, n, sp, s, nullptr, true));
  } else {
    h0 = 1;
    {
      Launch lp_(c, kKInitKeys, n, s);
      k_init_keys<<<g, 256, 0, s>>>(tokens, tb, n, b.keys[0], b.vals[0]);
    }
    b.cur = 0;
    const DigitRange r{0, tbits, false};
    APO_TRY(radix_sort_pairs(c, b, n, &r, 1, s));
    if (st.win.count > 1) {
      // group by (window, token): the token's rank among all tokens, then a
      // re-sort by the window id over those ranks
      APO_TRY(split_launch(c, false, b.keys[b.cur], b.vals[b.cur], n, nullptr, 0, nullptr, nullptr, nullptr, 0, 0,
                           false, st.snaps[0], st, lid[0], lhd[0], first_count, s));
      {
        Launch lp_(c, kKInitKeys, n, s);
        k_wkeys<<<g, 256, 0, s>>>(st.snaps[0], st.win, n, b.keys[0], b.vals[0]);
      }
      b.cur = 0;
      const DigitRange r2[2] = {{0, bits_for(n - 1), false}, {32, 32 + wb, false}};
      APO_TRY(radix_sort_pairs(c, b, n, r2, 2, s));
    }
  }
  APO_TRY(split_launch(c, false, b.keys[b.cur], b.vals[b.cur], n, nullptr, 0, nullptr, nullptr, nullptr, 0, 0,
                       true, st.snaps[0], st, lid[0], lhd[0], first_count, s));
  st.h0 = h0;
  st.levels = 1;

  // Rounds r = 1, 2, ...: round r reads list (r - 1) & 1 and writes the
  // level-r snapshot and list r & 1: k_round settles the small groups into
  // the holed list (hid, hhd) and writes the big entries' keys; the big
  // entries are sorted and k_split settles them into the holed list; then
  // k_list_compact drops the holes.  The round's device words (next list
  // length, big entries, -, big groups) alternate between two slots.  The host queues round r + 1 before it has read round r's
  // length (an upper bound sizes the launches), and stops one round after
  // the length reaches 0 (that round's kernels find nothing to do).  A round
  // with no big entries has no big groups after it, so from then on the big
  // path is not queued.
  const int mb = bits_for(st.win.count > 1 ? st.win.max_len : n);
  const int idb = std::max(1, bits_for(n - 1));  // bits of a suffix index
  uint32_t ub = n;      // bound on the current round's list length
  uint32_t big_ub = n;  // bound on its big entries (a round has no more than the round before)
  bool big_possible = true;
  // per round: the bounds its launches were sized for (units recorded by
  // the profiler), corrected to the exact counts when those are read
  struct RoundBounds {
    uint32_t ub = 0, big_ub = 0;
    int places = 0;
    bool keys = false;
  };
  std::vector<RoundBounds> rb(2);
  auto exact_list = [&](uint32_t rr, uint32_t len) {  // round rr's list held len entries
    const int64_t d = (int64_t)len - (int64_t)rb[rr].ub;
    for (int id : {(int)kKMinor, (int)kKRound, (int)kKListCompact}) c->prof.adjust(id, d);
  };
  auto exact_big = [&](uint32_t rr, uint32_t cnt) {  // round rr had cnt big entries
    if (!rb[rr].places) return;
    const int64_t d = (int64_t)cnt - (int64_t)rb[rr].big_ub;
    c->prof.adjust(rb[rr].keys ? kKRsPassKeys : kKRsPass, d * rb[rr].places);
    c->prof.adjust(kKSplit, d);
  };
  for (uint32_t r = 1;; ++r) {
    if (st.levels >= max_levels) {
      // a device wait that gave up or an index out of range leaves counts
      // that never reach 0: report that first
      if (!capturing(c)) APO_TRY(check_device_error(c, s));
      set_error("suffix array: too many doubling rounds");
      return APO_EDEVICE;
    }
    const int cur = (r - 1) & 1, nxt = r & 1;
    const uint32_t *in = r == 1 ? first_count : misc + kMiscRoundW + 4 * ((r - 1) & 1);
    uint32_t *words = misc + kMiscRoundW + 4 * (r & 1);
    const uint64_t h64 = (uint64_t)h0 << (r - 1);
    const uint32_t h = (uint32_t)std::min<uint64_t>(h64, n);  // no suffix is active once h reaches n
    const int tiles = std::max(1, ceil_div(ub, kRdT));
    const int ctiles = std::max(1, ceil_div(ub, kLcTile));
    APO_TRY(ensure_lookback(c, std::max<size_t>((size_t)2 * tiles, ctiles)));
    SortPlan sp;
    big_ub = std::min(big_ub, ub);
    // the big keys carry the suffix in their low bits when it fits: a
    // keys-only sort moves 16 instead of 24 bytes per entry and pass
    const int kbits = bits_for(big_ub / (kRdBig + 1) + 1) + mb;
    const int id_bits = idb + kbits <= 64 ? idb : 0;
    if (big_possible) {
      const DigitRange dr{id_bits, id_bits + kbits, false};
      APO_TRY(sort_plan(c, big_ub, &dr, 1, &sp, s));
      APO_TRY(sort_first_hist_clear(c, s));
    }
    APO_CUDA_TRY(cudaMemsetAsync(words, 0, 4 * sizeof(uint32_t), s));
    APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscRoundTiles, 0, sizeof(uint32_t), s));
    {
      Launch lp_(c, kKMinor, ub, s);
      k_minor<<<std::max(1, std::min(ceil_div(ub, 256 * 4), c->num_sms * 8)), 256, 0, s>>>(
          lid[cur], ub, in, r, h, n, st.wsb, st.fin, st.rank, st.snaps[r - 1], mkey);
    }
    {
      RoundArgs a;
      a.mkey = mkey;
      a.lid = lid[cur];
      a.lhd = lhd[cur];
      a.ub = ub;
      a.A_dev = in;
      a.r = r;
      a.h = h;
      a.n = n;
      a.wsb = st.wsb;
      a.wid = st.win.count > 1 ? st.win.wid : nullptr;
      a.woff = st.win.count > 1 ? st.win.off_dev : nullptr;
      a.fin = st.fin;
      a.rank = st.rank;
      a.sa = st.sa;
      a.snap_prev = st.snaps[r - 1];
      a.snap_cur = st.snaps[r];
      a.hid = hid;
      a.hhd = hhd;
      a.bkeys = b.keys[0];
      a.bvals = b.vals[0];
      a.bg_head = bg_head;
      a.bg_off = bg_off;
      a.bg_pos = bg_pos;
      a.bg_cap = bg_cap;
      a.mb = mb;
      a.id_bits = id_bits;
      a.big_hist = sort_first_hist(c);
      a.hist_bits = big_possible && sp.shape >= 0 ? sp.bits : 8;
      a.words = words;
      a.st_bc = c->ps.lookback;
      a.st_bs = c->ps.lookback + tiles;
      a.tile_ctr = misc + kMiscRoundTiles;
      a.epoch = next_epoch(c);
      a.err = c->ps.err;
      Launch lp_(c, kKRound, ub, s);
      k_round<<<tiles, kRdThreads, kRoundSmem, s>>>(a);
    }
    APO_CUDA_TRY(cudaGetLastError());
    rb.resize(r + 1);
    rb[r].ub = ub;
    if (big_possible && sp.shape >= 0) {
      rb[r].big_ub = big_ub;
      rb[r].places = sp.places;
      rb[r].keys = id_bits != 0;
      SortBuffers bb = b;
      bb.cur = 0;
      if (id_bits) bb.vals[0] = bb.vals[1] = nullptr;
      APO_TRY(radix_sort_planned(c, bb, big_ub, sp, s, words + 1, true));
      APO_TRY(split_launch(c, true, bb.keys[bb.cur], bb.vals[bb.cur], big_ub, words + 1, mb, bg_head, bg_off,
                           bg_pos, bg_cap, r, true, st.snaps[r], st, hid, hhd, nullptr, s, id_bits));
    }
    APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscRoundTiles, 0, sizeof(uint32_t), s));
    {
      Launch lp_(c, kKListCompact, ub, s);
      k_list_compact<<<ctiles, kLcT, 0, s>>>(hid, hhd, ub, in, lid[nxt], lhd[nxt], n, words, c->ps.lookback,
                                             misc + kMiscRoundTiles, next_epoch(c), c->ps.err);
    }
    APO_CUDA_TRY(cudaGetLastError());
    ++st.levels;
    const bool cap = capturing(c);
    if (!cap) {
      if (r == 1) APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 6, first_count, 4, cudaMemcpyDeviceToHost, s));
      APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 16 + 2 * (r & 1), words, 8, cudaMemcpyDeviceToHost, s));
      APO_CUDA_TRY(cudaEventRecord(c->round_ev[r & 1], s));
    }
    if (r == 1) continue;
    // round r - 1's results (a captured call takes them from its tape,
    // checked against the device words -- still unchanged at this point)
    if (r == 2) {
      uint32_t first = 0;
      if (cap) {
        APO_TRY(tape_take(c, first_count, &first, 1, s));
      } else {
        APO_CUDA_TRY(cudaEventSynchronize(c->round_ev[1]));
        first = c->host_pinned[6];
        if (recording(c)) tape_put(c, &first, 1);
      }
      if (!cap) exact_list(1, first);
      if (first == 0) {  // the first sort left no group: rounds 1 and 2 idle
        if (!cap) {
          exact_list(2, 0);
          exact_big(1, 0);
          exact_big(2, 0);
        }
        st.levels = 1;
        break;
      }
    }
    uint32_t w2[2];
    if (cap) {
      APO_TRY(tape_take(c, misc + kMiscRoundW + 4 * ((r - 1) & 1), w2, 2, s));
    } else {
      if (r > 2) APO_CUDA_TRY(cudaEventSynchronize(c->round_ev[(r - 1) & 1]));
      w2[0] = c->host_pinned[16 + 2 * ((r - 1) & 1)];
      w2[1] = c->host_pinned[17 + 2 * ((r - 1) & 1)];
      if (recording(c)) tape_put(c, w2, 2);
    }
    if (!cap) {
      exact_list(r, w2[0]);
      exact_big(r - 1, w2[1]);
    }
    if (w2[0] == 0) {  // round r had nothing to do: levels 0 .. r - 1
      if (!cap) exact_big(r, 0);
      st.levels = (int)r;
      break;
    }
    ub = w2[0];
    big_ub = std::min(big_ub, w2[1]);
    if (w2[1] == 0) big_possible = false;
  }
  *rounds_out = (uint32_t)(st.levels - 1);
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
    k_phi<<<g, 256, 0, s>>>(st.sa, n, st.wsb, phi);
  }
  const int pb = ceil_div(ceil_div(n, kPChunk), 128);
  {
    Launch lp_(c, kKPlcp, n, s);
    if (tb == 4)
      k_plcp<uint32_t><<<pb, 128, 0, s>>>(static_cast<const uint32_t *>(tokens), n, st.win, st.wsb, phi, st.fin,
                                          st.rank, st.snaps[0], st.levels, st.h0, plcp);
    else
      k_plcp<uint64_t><<<pb, 128, 0, s>>>(static_cast<const uint64_t *>(tokens), n, st.win, st.wsb, phi, st.fin,
                                          st.rank, st.snaps[0], st.levels, st.h0, plcp);
  }
  {
    Launch lp_(c, kKLcpPerm, n, s);
    k_lcp_perm<<<g, 256, 0, s>>>(st.sa, plcp, n, st.wsb, lcp);
  }
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

}  // namespace apo
