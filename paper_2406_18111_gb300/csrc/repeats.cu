// Alg. 2 after the suffix array: candidates, their order, the greedy
// non-overlapping selection and the deduplicated result R.
//
//  candidates  one thread per adjacent SA pair (Alg. 2's first loop),
//              candidates shorter than min_len dropped on the spot.
//  ids         Sec. 4.2 replaces the sub-string in a candidate by a unique ID
//              so that the sort and the deduplication are cheap.  The ID used
//              here is the left end of the LCP interval that holds the pair:
//              id = 1 + max{ j < i : LCP[j] < l } (0 if none), i.e. the SA index
//              of the first suffix starting with the sub-string.  Equal-length
//              distinct sub-strings occupy disjoint SA ranges in lexicographic
//              order, so id order is sub-string order and the sort needs no
//              token comparison.  The "previous smaller value" query walks a
//              32-ary min-tree over LCP (up one level until a block with a
//              smaller minimum lies to the left, then down into it).
//  sort        (length desc, id asc, start asc): the onesweep radix sort over
//              one (window, length, id, start) key when it fits 64 bits, else
//              over the start digits (value) then the (window, length, id)
//              digits (key).
//  dedup       identical (length, start) pairs are adjacent after the sort and
//              are kept once (order-preserving compaction).
//  greedy      the second loop of Alg. 2 is sequential by definition; it runs
//              in one block (1024 threads for a single window, 256 per window
//              in a batch) with the mark array of Sec. 4.2 as a bitmap (in
//              shared memory when the window fits).  Because the candidates
//              come in non-increasing length, a candidate meets an accepted
//              interval iff its first or last position is marked.  Each round
//              takes 4 candidates per thread, drops in parallel those whose
//              ends are already marked, and warp 0 settles the survivors 32
//              at a time, in order, marking the accepted intervals.  A single
//              window runs in phases of growing length; between them the
//              whole GPU drops the remaining candidates with a marked end.
//  R           accepted candidates in order; a new trace starts where (length,
//              id) changes; selected intervals are re-sorted by start.
#include <algorithm>
#include <cstring>
#include <vector>

#include "apo_internal.cuh"
#include "device_util.cuh"
#include "lcp_tree.cuh"

namespace apo {

namespace {


// Alg. 2 first loop.  Each kept pair writes two (key, start) entries with
// key = (window << (bl + bi)) | ((lmax - l) << bi) | id, shifted left by ks
// with the start in the low ks bits when everything fits one 64-bit key
// (ks = 0 otherwise: the start is sorted as the value).  Pairs that straddle
// two windows have LCP 0 and are dropped with the other short candidates.
// Alg. 2's candidates of the SA pair (s1, s2) with common prefix p: length
// l and the two starts a, b.
__device__ __forceinline__ void pair_cand(uint32_t s1, uint32_t s2, uint32_t p, uint32_t *l, uint32_t *a,
                                          uint32_t *b) {
  const uint32_t lo = min(s1, s2), hi = max(s1, s2);
  if (hi - lo >= p) {  // [s1, s1+p) and [s2, s2+p) are disjoint
    *l = p;
    *a = s1;
    *b = s2;
  } else {             // the common prefix is a run of S[lo, lo + d)
    const uint32_t d = hi - lo;
    uint64_t h = ((uint64_t)p + d) / 2;
    h -= h % d;
    *l = (uint32_t)h;
    *a = lo;
    *b = lo + *l;
  }
}

__global__ void k_cand_gen(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ lcp,
                           uint32_t n, uint32_t min_len, MinTree T, int bi, int bl, uint32_t lmax, int ks,
                           Windows W, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                           uint32_t *count, uint32_t *err, uint32_t *__restrict__ hist, int hist_bits) {
  // the sort's first digit place (the key's lowest hist_bits bits when the
  // key holds the start, else the value's): counted here for the sort
  __shared__ uint32_t sh[512];
  const uint32_t hmask = (1u << hist_bits) - 1;
  for (uint32_t d = threadIdx.x; d <= hmask; d += blockDim.x) sh[d] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n - 1; base += stride) {
    const uint32_t k = base + threadIdx.x;
    bool ok = false, ok_b = false;
    uint32_t l = 0, a = 0, b = 0;
    if (k < n - 1) {
      pair_cand(sa[k], sa[k + 1], lcp[k], &l, &a, &b);
      ok = l >= min_len && l > 0;
      // pair k + 1's first candidate is often this pair's second one (equal
      // LCPs along a run of the SA): leave it to pair k + 1
      ok_b = ok;
      if (ok && k + 1 < n - 1) {
        uint32_t l2, a2, b2;
        pair_cand(sa[k + 1], sa[k + 2], lcp[k + 1], &l2, &a2, &b2);
        if (l2 == l && a2 == b) ok_b = false;
      }
    }
    uint64_t key = 0;
    if (ok) {
      // with several windows, the id and the start are relative to the
      // window (its suffixes occupy a contiguous SA range starting at its
      // offset), which keeps the key and value digits to the longest window
      // (the pair's SA slots and suffixes lie in the same window: its id is
      // read at slot k, next to the other threads' reads)
      const uint32_t w = win_id(W, k), wbase = W.off_dev ? W.off_dev[w] : 0u;
      const uint32_t wlen = (W.off_dev ? W.off_dev[w + 1] : n) - wbase;
      if (a < wbase || b < wbase || a - wbase + (uint64_t)l > wlen || b - wbase + (uint64_t)l > wlen) {
        // (only a suffix array or LCP from a replay whose checks failed)
        atomicExch(err, kDevRange);
        ok = ok_b = false;
      }
      const long long j = prev_less(T, k, l, err);
      key = ((uint64_t)w << (bl + bi)) | ((uint64_t)(lmax - l) << bi) | (uint64_t)(j + 1 - wbase);
      a -= wbase;
      b -= wbase;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, ok), bal_b = __ballot_sync(0xffffffffu, ok_b);
    if (bal == 0) continue;
    const int leader = __ffs(bal) - 1;
    uint32_t slot0 = 0;
    if ((int)lane == leader) slot0 = atomicAdd(count, __popc(bal) + __popc(bal_b));
    slot0 = __shfl_sync(0xffffffffu, slot0, leader);
    if (ok) {
      const uint32_t lt = lanemask_lt();
      const uint32_t slot = slot0 + __popc(bal & lt) + __popc(bal_b & lt);
      if (slot + (ok_b ? 1u : 0u) >= 2 * (n - 1)) {
        atomicExch(err, kDevRange);
        continue;
      }
      const uint64_t ka = ks ? (key << ks) | a : key, kb = ks ? (key << ks) | b : key;
      keys[slot] = ka;
      if (ok_b) keys[slot + 1] = kb;
      // the first digit: of the key when it holds the start, else of the value
      atomicAdd(&sh[(ks ? (uint32_t)ka : a) & hmask], 1u);
      if (ok_b) atomicAdd(&sh[(ks ? (uint32_t)kb : b) & hmask], 1u);
      if (!ks) {  // the start is the value (otherwise it is the key's low digits)
        vals[slot] = a;
        if (ok_b) vals[slot + 1] = b;
      }
    }
  }
  __syncthreads();
  for (uint32_t d = threadIdx.x; d <= hmask; d += blockDim.x)
    if (sh[d]) atomicAdd(&hist[d], sh[d]);
}

// Order-preserving compaction of the indices k < m with pred(k) (one
// decoupled look-back sum-scan).
constexpr int kCT = 256, kCI = 8, kCTile = kCT * kCI;

struct PredFirstOfRun {  // k starts a run of identical (key, value) pairs (vals == nullptr: keys)
  const uint64_t *keys;
  const uint32_t *vals;
  __device__ bool operator()(uint32_t k) const {
    return k == 0 || keys[k] != keys[k - 1] || (vals && vals[k] != vals[k - 1]);
  }
};
struct PredFlag {
  const uint8_t *f;
  __device__ bool operator()(uint32_t k) const { return f[k] != 0; }
};

// Where the r-th kept k goes: out[r] = k.
struct PutIndex {
  uint32_t *out;
  __device__ __forceinline__ void operator()(uint32_t r, uint32_t k) const { out[r] = k; }
};

template <class Pred, class Put>
__global__ void __launch_bounds__(kCT) k_compact(Pred pred, uint32_t m, const uint32_t *m_dev, uint32_t m_sub,
                                                 Put put, uint32_t *count_out, uint64_t *status,
                                                 uint32_t *tile_ctr, uint32_t epoch, uint32_t *err) {
  __shared__ uint32_t s_tile, s_pre;
  __shared__ uint32_t scr[kCT / 32];
  const int tid = threadIdx.x;
  if (m_dev) {  // the launch is sized for an upper bound; the count is *m_dev - m_sub
    const uint32_t v = *m_dev;
    m = min(m, v > m_sub ? v - m_sub : 0u);
  }
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kCTile;
  if (t > 0 && base >= m) return;  // past the count (no earlier tile looks at it)
  const uint64_t e0 = base + (uint64_t)tid * kCI;
  uint32_t fb = 0;
#pragma unroll
  for (int i = 0; i < kCI; ++i)
    if (e0 + i < m && pred((uint32_t)(e0 + i))) fb |= 1u << i;
  uint32_t tot;
  const uint32_t ex = block_exclusive<kCT / 32>(__popc(fb), OpSum(), 0u, scr, &tot);
  if (tid == 0) {
    lb_store(&status[t], lb_pack(t == 0 ? kLbInclusive : kLbAggregate, epoch, tot));
    uint32_t pre = 0;
    if (t > 0) {
      pre = lb_exclusive_k<8>(status, 1, t, epoch, OpSum(), 0u, err);
      lb_store(&status[t], lb_pack(kLbInclusive, epoch, pre + tot));
    }
    s_pre = pre;
    if (base + kCTile >= m) *count_out = pre + tot;
  }
  __syncthreads();
  uint32_t r = s_pre + ex;
#pragma unroll
  for (int i = 0; i < kCI; ++i) {
    if ((fb >> i) & 1u) {
      if (r < m) put(r, (uint32_t)(e0 + i)); else atomicExch(err, kDevRange);
      ++r;
    }
  }
}

__global__ void k_cand_gather(const uint32_t *__restrict__ sel, uint32_t m, const uint32_t *m_dev,
                              const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                              int bi, int bl, uint32_t lmax, int ks, const uint32_t *__restrict__ woff,
                              uint32_t nwin, uint32_t *__restrict__ cl, uint32_t *__restrict__ cid,
                              uint32_t *__restrict__ cs, uint32_t *err) {
  m = min(m, *m_dev);  // m: an upper bound
  const uint64_t idmask = (bi >= 64) ? ~0ull : ((1ull << bi) - 1);
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
    const uint32_t k = sel[q];
    const uint64_t full = keys[k], key = full >> ks;
    const uint64_t w = key >> (bl + bi);
    if (woff && w >= nwin) {  // (only keys of a replay whose checks failed)
      atomicExch(err, kDevRange);
      continue;
    }
    const uint32_t base = woff ? woff[(uint32_t)w] : 0u;  // back to global positions
    cl[q] = lmax - (uint32_t)((key >> bi) & lmax);
    cid[q] = (uint32_t)(key & idmask) + base;
    cs[q] = (ks ? (uint32_t)(full & ((1ull << ks) - 1)) : vals[k]) + base;
  }
}

// ---------------------------------------------------------------- greedy
constexpr int kGI = 4;  // candidates per thread per round
constexpr uint32_t kGreedyFirstPhase = 1u << 16;  // candidates settled before the first drop
constexpr uint32_t kGWideWin = 1u << 16;  // batched windows of this many tokens or more: 1024-thread blocks
constexpr int glist_bytes(int threads) { return threads * kGI * 16; }

template <bool kSmem>
__device__ __forceinline__ bool marked(const uint32_t *bits, uint32_t x) {
  uint32_t w;
  if (kSmem)
    w = bits[x >> 5];
  else
    w = *(volatile const uint32_t *)(bits + (x >> 5));
  return (w >> (x & 31)) & 1u;
}

// One block per window runs Alg. 2's second loop over the window's
// candidates [cand_off[w], cand_off[w+1]).  Each round takes the next kT * 4
// candidates (base + i*kT + tid for item i of thread tid), drops those whose
// first or last position is already marked, compacts the rest in candidate
// order, and warp 0 settles them 32 at a time, marking accepted intervals.
// The accepted flags must be zero on entry.  The mark bitmap covers the
// window in shared memory (positions relative to the window start), or all
// positions in global memory (zeroed by the caller).
//
// Single window, in phases: `corig` maps list positions to candidate indices
// (null: the identity) when the list is a compacted remainder, and with
// `persist` the shared-memory bitmap is loaded from gbits at the start and
// stored back at the end, so that a later phase continues the same marks.
template <int kT, bool kSmem>
__global__ void __launch_bounds__(kT) k_greedy(const uint32_t *__restrict__ cl,
                                               const uint32_t *__restrict__ cs,
                                               const uint32_t *__restrict__ cand_off, uint32_t m,
                                               const uint32_t *__restrict__ woff, uint32_t n,
                                               uint32_t *gbits, uint8_t *acc, uint32_t *acc_count,
                                               const uint32_t *__restrict__ corig, int persist,
                                               const uint32_t *m_dev, uint32_t *err, uint32_t len_lo = 0,
                                               uint32_t len_hi = 0xffffffffu) {
  constexpr int kGT = kT;
  constexpr int kGRound = kT * kGI;
  extern __shared__ __align__(16) uint32_t gsm[];
  const uint32_t w = blockIdx.x;
  if (m_dev) m = min(m, *m_dev);  // single window: m bounds the list, *m_dev is its length
  const uint32_t cb = cand_off ? cand_off[w] : 0u, ce = cand_off ? cand_off[w + 1] : m;
  const uint32_t ws = woff ? woff[w] : 0u, we = woff ? woff[w + 1] : n;
  if (we - ws < len_lo || we - ws >= len_hi) return;  // a window for the other launch
  const uint32_t shift = kSmem ? ws : 0u;  // bitmap coordinate = position - shift
  const uint32_t words = kSmem ? ((we - ws + 31) / 32 + 3) & ~3u : 0;
  uint32_t *bits = kSmem ? gsm : gbits;
  if (ce <= cb) return;
  cl += cb;
  cs += cb;
  acc += cb;
  m = ce - cb;
  uint32_t *sl = gsm + words, *ss = sl + kGRound, *sk = ss + kGRound, *sov = sk + kGRound;
  __shared__ uint32_t s_cnt[2][kGI][32];  // survivors per (item, warp), by round parity
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (kSmem)
    for (uint32_t x = tid; x < words; x += kGT) gsm[x] = persist ? gbits[x] : 0u;
  uint32_t nacc = 0;
  uint32_t nl[kGI], ns[kGI], no[kGI];  // the next round's candidates, loaded a round ahead
#pragma unroll
  for (int i = 0; i < kGI; ++i) {
    const uint32_t k = i * kGT + tid;
    nl[i] = k < m ? cl[k] : 0u;
    ns[i] = k < m ? cs[k] : 0u;
    no[i] = corig && k < m ? corig[k] : k;
  }
  __syncthreads();
  uint32_t par = 0;
  for (uint32_t base = 0; base < m; base += kGRound, par ^= 1u) {
    uint32_t l[kGI], s[kGI], o[kGI], bal[kGI];
    bool surv[kGI];
#pragma unroll
    for (int i = 0; i < kGI; ++i) {
      l[i] = nl[i];
      s[i] = ns[i];
      o[i] = no[i];
      const uint64_t kn = (uint64_t)base + kGRound + i * kGT + tid;  // prefetch the next round
      if (kn < m) {
        nl[i] = cl[kn];
        ns[i] = cs[kn];
        no[i] = corig ? corig[kn] : (uint32_t)kn;
      }
    }
#pragma unroll
    for (int i = 0; i < kGI; ++i) {
      const uint32_t k = base + i * kGT + tid;
      surv[i] = false;
      if (k < m) {
        if (l[i] == 0 || s[i] < ws || (uint64_t)s[i] + l[i] > we) {
          atomicExch(err, kDevRange);
        } else {
          s[i] -= shift;
          surv[i] = !(marked<kSmem>(bits, s[i]) | marked<kSmem>(bits, s[i] + l[i] - 1));
        }
      }
      bal[i] = __ballot_sync(0xffffffffu, surv[i]);
      if (lane == 0) s_cnt[par][i][warp] = __popc(bal[i]);
    }
    __syncthreads();
    // Survivor offsets in (item, warp) order = candidate order, scanned by
    // every warp for itself.  The counts are double-buffered by round
    // parity: a round without survivors skips the barriers below, and a
    // warp may write the next round's counts while another still reads these.
    uint32_t off[kGI], s_total = 0;
#pragma unroll
    for (int i = 0; i < kGI; ++i) {
      const uint32_t c = lane < kGT / 32 ? s_cnt[par][i][lane] : 0u;
      const uint32_t inc = warp_inclusive(c, OpSum());
      off[i] = s_total + __shfl_sync(0xffffffffu, inc - c, warp);
      s_total += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (s_total == 0) continue;  // the same in every warp; no mark changes
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kGI; ++i) {
      if (surv[i]) {
        const uint32_t q = off[i] + __popc(bal[i] & lt);
        sl[q] = l[i];
        ss[q] = s[i];
        sk[q] = o[i];
      }
    }
    __syncthreads();
    // Overlap masks of the survivor batches, by every warp (they depend on
    // the intervals only): sov[q] bit j = survivor q0 + j of q's batch of 32
    // (q0 = q rounded down to 32), j before q's lane, meets survivor q.
    for (uint32_t q = tid; q < s_total; q += kGT) {
      const uint32_t q0 = q & ~31u, nb = min(32u, s_total - q0);
      const uint32_t qs = ss[q], qe = qs + sl[q] - 1;
      uint32_t ov = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const uint32_t js = ss[q0 + j], je = js + sl[q0 + j] - 1;  // list has room past total
        if (j < lane && (uint32_t)j < nb && js <= qe && qs <= je) ov |= 1u << j;
      }
      sov[q] = ov;
    }
    __syncthreads();
    if (warp == 0 && s_total) {
      // Settle the survivors 32 at a time: lane j holds survivor q0 + j.  A
      // lane is out if its ends are marked by an earlier batch; among the
      // rest, a lane is accepted once no earlier lane that overlaps it is
      // accepted or undecided, and rejected once one that overlaps it is
      // accepted (the batch's greedy order, settled a few ballots at a time).
      const uint32_t total = s_total;
      // the lane's survivor of the next batch, read one batch ahead (the
      // survivor lists do not change during the settle; only the marks do)
      uint32_t ps = 0, pl = 1, pov = 0, pk = 0;
      if (lane < total) {
        ps = ss[lane];
        pl = sl[lane];
        pov = sov[lane];
        pk = sk[lane];
      }
      for (uint32_t q0 = 0; q0 < total; q0 += 32) {
        const uint32_t q = q0 + lane;
        const uint32_t qs = ps, qe = ps + pl - 1;
        const uint32_t ov = pov, qk = pk;  // ov: earlier lanes of the batch meeting this one
        if (q + 32 < total) {
          ps = ss[q + 32];
          pl = sl[q + 32];
          pov = sov[q + 32];
          pk = sk[q + 32];
        }
        const bool free = q < total && !(marked<kSmem>(bits, qs) | marked<kSmem>(bits, qe));
        uint32_t und = __ballot_sync(0xffffffffu, free), accm = 0;
        if (und == 0) continue;  // every survivor of the batch met an accepted interval meanwhile
        while (und) {
          const bool mine = (und >> lane) & 1u;
          const uint32_t take = __ballot_sync(0xffffffffu, mine && (ov & (und | accm)) == 0);
          accm |= take;
          und &= ~take;
          const uint32_t drop = __ballot_sync(0xffffffffu, ((und >> lane) & 1u) && (ov & accm) != 0);
          und &= ~drop;
        }
        // mark accepted intervals: short ones by their own lane, long ones warp-wide
        const bool mine = (accm >> lane) & 1u;
        bool lng = false;
        if (mine) {
          acc[qk] = 1;
          const uint32_t w0 = qs >> 5, w1 = qe >> 5;
          if (w1 - w0 < 8) {
            for (uint32_t w = w0; w <= w1; ++w) {
              uint32_t msk = 0xffffffffu;
              if (w == w0) msk &= 0xffffffffu << (qs & 31);
              if (w == w1) msk &= 0xffffffffu >> (31 - (qe & 31));
              atomicOr(&bits[w], msk);
            }
          } else {
            lng = true;
          }
        }
        for (uint32_t am = __ballot_sync(0xffffffffu, lng); am; am &= am - 1) {
          const int j = __ffs(am) - 1;
          const uint32_t js = __shfl_sync(0xffffffffu, qs, j);
          const uint32_t je = __shfl_sync(0xffffffffu, qe, j);
          const uint32_t w0 = js >> 5, w1 = je >> 5;
          for (uint32_t w = w0 + lane; w <= w1; w += 32) {
            uint32_t msk = 0xffffffffu;
            if (w == w0) msk &= 0xffffffffu << (js & 31);
            if (w == w1) msk &= 0xffffffffu >> (31 - (je & 31));
            atomicOr(&bits[w], msk);
          }
        }
        nacc += __popc(accm);
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (tid == 0) atomicAdd(acc_count, nacc);  // lane 0 of warp 0 counted every batch
  if (kSmem && persist) {
    __syncthreads();
    for (uint32_t x = tid; x < words; x += kGT) gbits[x] = gsm[x];
  }
}

// Candidates of the list remainder [from, len) whose first and last
// positions are both unmarked (the others can never be accepted: marks only
// accumulate, and a candidate meets an accepted interval iff an end of it is
// marked).
struct PredUnmarked {
  const uint32_t *l, *s, *bits;
  uint32_t from;
  __device__ bool operator()(uint32_t k) const {
    const uint32_t a = s[from + k], b = a + l[from + k] - 1;
    return !((bits[a >> 5] >> (a & 31)) & 1u) && !((bits[b >> 5] >> (b & 31)) & 1u);
  }
};

// The drop's output: the r-th kept remainder entry k (list position from + k)
// becomes entry r of the next list.
struct PutList {
  const uint32_t *l, *st, *orig;
  uint32_t from;
  uint32_t *l2, *s2, *o2;
  __device__ __forceinline__ void operator()(uint32_t r, uint32_t k) const {
    const uint32_t q = from + k;
    l2[r] = l[q];
    s2[r] = st[q];
    o2[r] = orig ? orig[q] : q;
  }
};

// Accepted candidates (compacted, in order) -> R and the keys of the
// selected intervals.  A new trace starts wherever (length, id) changes; the
// trace index of an accepted candidate is the number of such starts up to it,
// minus one (a decoupled look-back sum over tiles of 4096).
__global__ void __launch_bounds__(kCT) k_traces(const uint32_t *__restrict__ accidx, uint32_t K,
                                                const uint32_t *__restrict__ cl,
                                                const uint32_t *__restrict__ cid,
                                                const uint32_t *__restrict__ cs,
                                                uint32_t *__restrict__ tl, uint32_t *__restrict__ ts,
                                                uint64_t *__restrict__ skeys,
                                                uint32_t *__restrict__ svals, uint32_t *tcount,
                                                uint64_t *status, uint32_t *tile_ctr, uint32_t epoch,
                                                uint32_t *err) {
  __shared__ uint32_t s_tile, s_pre;
  __shared__ uint32_t scr[kCT / 32];
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kCTile;
  const uint64_t e0 = base + (uint64_t)tid * kCI;
  uint32_t fb = 0;
#pragma unroll
  for (int i = 0; i < kCI; ++i) {
    const uint64_t q = e0 + i;
    if (q < K) {
      const uint32_t k = accidx[q];
      bool f = q == 0;
      if (!f) {
        const uint32_t kp = accidx[q - 1];
        f = cl[k] != cl[kp] || cid[k] != cid[kp];
      }
      if (f) fb |= 1u << i;
    }
  }
  uint32_t tot;
  const uint32_t ex = block_exclusive<kCT / 32>(__popc(fb), OpSum(), 0u, scr, &tot);
  if (tid == 0) {
    lb_store(&status[t], lb_pack(t == 0 ? kLbInclusive : kLbAggregate, epoch, tot));
    uint32_t pre = 0;
    if (t > 0) {
      pre = lb_exclusive_k<8>(status, 1, t, epoch, OpSum(), 0u, err);
      lb_store(&status[t], lb_pack(kLbInclusive, epoch, pre + tot));
    }
    s_pre = pre;
    if (base + kCTile >= K) *tcount = pre + tot;
  }
  __syncthreads();
  uint32_t run = s_pre + ex;  // trace starts before element e0
#pragma unroll
  for (int i = 0; i < kCI; ++i) {
    const uint64_t q = e0 + i;
    if (q < K) {
      const uint32_t k = accidx[q];
      const bool f = (fb >> i) & 1u;
      run += f;
      const uint32_t tr = run - 1;  // index of this candidate's trace
      if (f) {
        tl[tr] = cl[k];
        ts[tr] = cs[k];
      }
      skeys[q] = ((uint64_t)cs[k] << 32) | cl[k];
      svals[q] = tr;
    }
  }
}

__global__ void k_sel_out(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                          uint32_t K, uint32_t *__restrict__ ss, uint32_t *__restrict__ sl,
                          uint32_t *__restrict__ st) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < K; q += gridDim.x * blockDim.x) {
    const uint64_t key = keys[q];
    ss[q] = (uint32_t)(key >> 32);
    sl[q] = (uint32_t)key;
    st[q] = vals[q];
  }
}

// First index of each window in a list sorted by window (the window of entry
// k is the window of position pos[k]); out[count] = m.
__global__ void k_window_bounds(const uint32_t *__restrict__ pos, uint32_t m, Windows W, uint32_t n,
                                uint32_t *__restrict__ out, const uint32_t *m_dev = nullptr) {
  if (m_dev) m = min(m, *m_dev);  // m: an upper bound
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w <= W.count; w += gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = m;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      const uint32_t p = pos[mid];
      if ((p < n ? win_id(W, p) : W.count) < w) lo = mid + 1; else hi = mid;
    }
    out[w] = lo;
  }
}

// Window-relative outputs: starts minus the window start, trace indices
// minus the window's first trace.
__global__ void k_relativize(uint32_t *__restrict__ start, uint32_t *__restrict__ trace, uint32_t k,
                             Windows W, const uint32_t *__restrict__ trace_off) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < k; q += gridDim.x * blockDim.x) {
    const uint32_t w = win_id(W, start[q]);
    if (trace) trace[q] -= trace_off[w];
    start[q] -= W.off_dev ? W.off_dev[w] : 0u;
  }
}

int g_greedy_smem_max = 0;  // dynamic shared memory available to k_greedy<*, true>

// A device count (and optionally a second one) and the error word in one
// synchronisation (a captured call takes them from its tape).
int read_u32(apo_ctx *c, const uint32_t *dev, uint32_t *host, cudaStream_t s, const uint32_t *dev2 = nullptr,
             uint32_t *host2 = nullptr) {
  if (capturing(c)) {
    uint32_t e = 0;
    APO_TRY(tape_take(c, dev, host, 1, s));
    if (dev2) APO_TRY(tape_take(c, dev2, host2, 1, s));
    return tape_take(c, c->ps.err, &e, 1, s);
  }
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (dev2) APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 1, dev2, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + kPinnedErr, c->ps.err, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  if (recording(c)) {
    tape_put(c, c->host_pinned, 1);
    if (dev2) tape_put(c, c->host_pinned + 1, 1);
    tape_put(c, c->host_pinned + kPinnedErr, 1);
  }
  APO_TRY(device_error_status(c, s));
  if (dev2) *host2 = c->host_pinned[1];
  *host = c->host_pinned[0];
  return APO_OK;
}

// Compacts the k < m (or, with m_dev, k < min(m, *m_dev - m_sub)) for which
// pred(k) holds: the r-th of them goes to put(r, k) (out[r] = k with an
// index array); their number lands in *count_dev.
template <class Pred, class Put>
int compact_to(apo_ctx *c, Pred pred, Put put, uint32_t m, uint32_t *count_dev, cudaStream_t s,
               const uint32_t *m_dev = nullptr, uint32_t m_sub = 0) {
  const int tiles = std::max(1, ceil_div(m, kCTile));
  APO_TRY(ensure_lookback(c, tiles));
  uint32_t *tctr = c->ps.counters + kCtrMisc + kMiscCompactTiles;
  APO_CUDA_TRY(cudaMemsetAsync(tctr, 0, sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(count_dev, 0, sizeof(uint32_t), s));
  {
    Launch lp_(c, kKCompact, m, s);
    k_compact<<<tiles, kCT, 0, s>>>(pred, m, m_dev, m_sub, put, count_dev, c->ps.lookback, tctr,
                                    next_epoch(c), c->ps.err);
  }
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

template <class Pred>
int compact(apo_ctx *c, Pred pred, uint32_t m, uint32_t *out, uint32_t *count_dev, cudaStream_t s) {
  return compact_to(c, pred, PutIndex{out}, m, count_dev, s);
}

template <class T>
int copy_out(T *dst, const T *src, uint64_t count, uint64_t cap, bool *over, cudaStream_t s) {
  if (!dst) return APO_OK;
  if (count > cap) *over = true;
  const uint64_t k = std::min(count, cap);
  if (k) APO_CUDA_TRY(cudaMemcpyAsync(dst, src, k * sizeof(T), cudaMemcpyDeviceToDevice, s));
  return APO_OK;
}

}  // namespace

__global__ void k_min32(const uint32_t *__restrict__ in, uint32_t nin, uint32_t *__restrict__ out,
                        uint32_t nout) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nout; b += warps) {
    const uint32_t i = b * 32 + lane;
    uint32_t v = i < nin ? in[i] : 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) out[b] = v;
  }
}

int build_min_tree(apo_ctx *c, const uint32_t *lcp, uint32_t n, MinTree *T, cudaStream_t s) {
  T->lv[0] = lcp;
  T->cnt[0] = n;
  T->nlev = 1;
  while (T->cnt[T->nlev - 1] > 32) {
    if (T->nlev >= kMaxTree) {
      set_error("LCP min-tree: array too large");
      return APO_EINVAL;
    }
    const uint32_t nin = T->cnt[T->nlev - 1], nout = (nin + 31) / 32;
    uint32_t *o = c->arena.take_n<uint32_t>(nout);
    if (!o) return APO_ENOMEM;
    {
      Launch lp_(c, kKMin32, nin, s);
      const int blocks = std::max(1, std::min(ceil_div((long long)nout * 32, 256), c->num_sms * 16));
      k_min32<<<blocks, 256, 0, s>>>(T->lv[T->nlev - 1], nin, o, nout);
    }
    T->lv[T->nlev] = o;
    T->cnt[T->nlev] = nout;
    ++T->nlev;
  }
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

int repeats_init(int smem_optin) {
  // k_greedy: dynamic = bitmap (shared-memory variants) + survivor list;
  // static = 2 * 4 * 32 + 1 words
  g_greedy_smem_max = smem_optin - 2048;
  APO_CUDA_TRY(cudaFuncSetAttribute(k_greedy<1024, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    g_greedy_smem_max));
  APO_CUDA_TRY(cudaFuncSetAttribute(k_greedy<1024, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    glist_bytes(1024)));
  APO_CUDA_TRY(cudaFuncSetAttribute(k_greedy<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    g_greedy_smem_max));
  APO_CUDA_TRY(cudaFuncSetAttribute(k_greedy<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    glist_bytes(256)));
  return APO_OK;
}

size_t repeats_workspace_bytes(uint64_t n, uint64_t windows) {
  const uint64_t M = n ? 2 * (n - 1) : 0;
  return (size_t)M * (2 * 8 + 2 * 4)  // sort buffers
         + (size_t)M * (4 * 3 + 4 + 1)  // candidate arrays, compaction indices, flags
         + (size_t)M * (4 * 6)           // single window: greedy lists (two sets of three arrays)
         + (size_t)n * 20                // R and the selected intervals (5 arrays of <= n)
         + (size_t)n * 4 / 16 + (size_t)n / 8 + 16 + (size_t)(windows + 1) * 12 + 64 * 256;
}

int find_repeats_from_sa(apo_ctx *c, const void *tokens, int tb, const SuffixState &st,
                         const uint32_t *lcp, uint32_t min_len, apo_repeats_out *out,
                         const BatchOffsets *boff, cudaStream_t s) {
  ScopeGuard scope_(c, kScopeRepeats);
  (void)tokens;
  (void)tb;
  const uint32_t n = st.n;
  const Windows &W = st.win;
  uint64_t *counts = out->counts;
  counts[0] = counts[1] = counts[2] = 0;
  auto zero_offsets = [&]() {
    if (!boff) return;
    for (uint32_t w = 0; w <= W.count; ++w) {
      if (boff->cand_off) boff->cand_off[w] = 0;
      if (boff->sel_off) boff->sel_off[w] = 0;
      if (boff->trace_off) boff->trace_off[w] = 0;
    }
  };
  zero_offsets();
  // The call's last step: the device error word, read behind everything
  // queued so far (one synchronisation), or checked against the tape.
  auto err_check = [&]() -> int {
    if (capturing(c)) {
      uint32_t e = 0;
      return tape_take(c, c->ps.err, &e, 1, s);
    }
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + kPinnedErr, c->ps.err, sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, s));
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    if (recording(c)) tape_put(c, c->host_pinned + kPinnedErr, 1);
    return device_error_status(c, s);
  };
  if (n < 2) return err_check();
  uint32_t *misc = c->ps.counters + kCtrMisc;
  const int g = grid_for(n, 256, c->num_sms);

  // bits of the (window, length, id) key: after the last doubling round no
  // two suffixes share h0 * 2^rounds tokens, so every LCP is below that
  const uint64_t lcp_bound = ((uint64_t)st.h0 << std::max(0, st.levels - 1)) - 1;
  const int bl = std::max(1, bits_for(std::min<uint64_t>(lcp_bound, n)));
  const uint32_t lmax = (uint32_t)((1ull << bl) - 1);
  // ids and starts are window-relative with several windows
  const int bi = std::max(1, bits_for((W.count > 1 ? W.max_len : n) - 1));
  const int bs = bi;
  const int bw = W.count > 1 ? bits_for(W.count - 1) : 0;
  if (bw + bl + bi > 64) {
    set_error("repeats: windows, lengths and ids do not fit a 64-bit sort key");
    return APO_EINVAL;
  }
  // the start joins the key when it fits: one digit range instead of two
  const int ks = bw + bl + bi + bs <= 64 ? bs : 0;

  // 32-ary min-tree over LCP
  MinTree T;
  APO_TRY(build_min_tree(c, lcp, n, &T, s));

  // candidates
  const uint64_t M = 2ull * (n - 1);
  SortBuffers b;
  b.keys[0] = c->arena.take_n<uint64_t>(M);
  b.keys[1] = c->arena.take_n<uint64_t>(M);
  b.vals[0] = c->arena.take_n<uint32_t>(M);
  b.vals[1] = c->arena.take_n<uint32_t>(M);
  uint32_t *sel = c->arena.take_n<uint32_t>(M);
  uint32_t *cl = c->arena.take_n<uint32_t>(M);
  uint32_t *cid = c->arena.take_n<uint32_t>(M);
  uint32_t *cs = c->arena.take_n<uint32_t>(M);
  uint8_t *acc = c->arena.take_n<uint8_t>(M);
  const size_t gwords = (size_t)(n + 31) / 32 + 4;  // the shared-memory bitmap rounds up to 4 words
  uint32_t *gbits = c->arena.take_n<uint32_t>(gwords);
  uint32_t *cand_off = c->arena.take_n<uint32_t>(W.count + 1);
  uint32_t *sel_off = c->arena.take_n<uint32_t>(W.count + 1);
  uint32_t *trace_off = c->arena.take_n<uint32_t>(W.count + 1);
  if (!b.keys[0] || !b.keys[1] || !b.vals[0] || !b.vals[1] || !sel || !cl || !cid || !cs || !acc ||
      !gbits || !cand_off || !sel_off || !trace_off) {
    set_error("repeats: workspace too small");
    return APO_ENOMEM;
  }
  // the candidate sort is planned for the bound M, so that candidate
  // generation can count its first digit place (the start's low digits)
  const DigitRange r[2] = {{0, bs, true}, {0, bw + bl + bi, false}};
  const DigitRange rk{0, bw + bl + bi + bs, false};
  SortPlan sp;
  if (ks)
    APO_TRY(sort_plan(c, (uint32_t)M, &rk, 1, &sp, s));
  else
    APO_TRY(sort_plan(c, (uint32_t)M, r, 2, &sp, s));
  APO_TRY(sort_first_hist_clear(c, s));
  APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscCandCount, 0, sizeof(uint32_t), s));
  {
    Launch lp_(c, kKCandGen, n, s);
    k_cand_gen<<<g, 256, 0, s>>>(st.sa, lcp, n, min_len, T, bi, bl, lmax, ks, W, b.keys[0], b.vals[0],
                                 misc + kMiscCandCount, c->ps.err, sort_first_hist(c),
                                 sp.shape >= 0 ? sp.bits : 8);
  }
  APO_CUDA_TRY(cudaGetLastError());
  uint32_t mraw = 0;
  APO_TRY(read_u32(c, misc + kMiscCandCount, &mraw, s));
  // m, the candidates left after deduplication, stays on the device (m_dev)
  // until it is read with the greedy's count; launches before that are sized
  // by mu = mraw >= m
  uint32_t m = 0, mu = 0;
  const uint32_t *m_dev = misc + kMiscCandUnique;
  if (mraw) {
    // (window, length, id, start): one key, or start digits (the value)
    // first and then the (window, length, id) key
    b.cur = 0;
    if (ks) {  // the key holds every field: a keys-only sort (two thirds of the bytes per pass)
      SortBuffers kb = b;
      kb.vals[0] = kb.vals[1] = nullptr;
      APO_TRY(radix_sort_planned(c, kb, mraw, sp, s, nullptr, true));
      b.cur = kb.cur;
    } else {
      APO_TRY(radix_sort_planned(c, b, mraw, sp, s, nullptr, true));
    }
    PredFirstOfRun pr{b.keys[b.cur], ks ? nullptr : b.vals[b.cur]};
    APO_TRY(compact(c, pr, mraw, sel, misc + kMiscCandUnique, s));
    mu = mraw;
    {
      Launch lp_(c, kKCandGather, mu, s);
      k_cand_gather<<<grid_for(mu, 256, c->num_sms), 256, 0, s>>>(sel, mu, m_dev, b.keys[b.cur], b.vals[b.cur],
                                                                  bi, bl, lmax, ks, W.count > 1 ? W.off_dev : nullptr,
                                                                  W.count, cl, cid, cs, c->ps.err);
    }
  }

  // greedy selection, one block per window
  uint32_t K = 0;
  if (mu) {
    {
      Launch lp_(c, kKSlices, W.count + 1, s);
      k_window_bounds<<<ceil_div(W.count + 1, 256), 256, 0, s>>>(cs, mu, W, n, cand_off, m_dev);
    }
    APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscAccCount, 0, sizeof(uint32_t), s));
    APO_CUDA_TRY(cudaMemsetAsync(acc, 0, mu, s));
    const uint32_t maxw = W.count > 1 ? W.max_len : n;
    const size_t bm_bytes = (size_t)((((maxw + 31) / 32) + 3) & ~3u) * 4;
    const bool big = W.count == 1;  // one window: one wide block
    const size_t list = glist_bytes(big ? 1024 : 256);
    const uint32_t *coff = W.count > 1 ? cand_off : nullptr;
    const bool smem = (long long)(bm_bytes + list) <= g_greedy_smem_max;
    if (!smem) APO_CUDA_TRY(cudaMemsetAsync(gbits, 0, gwords * 4, s));
    uint32_t *glist[2][3] = {};
    if (big) {
      for (auto &g : glist)
        for (auto &a : g) a = c->arena.take_n<uint32_t>(mu);
      if (!glist[1][2]) return APO_ENOMEM;
    }
    if (big) {
      // Phases: the one block settles a prefix of the list; then every
      // remaining candidate with a marked end is dropped by the whole GPU
      // and the survivors form the next list.  Long candidates come first,
      // so a short prefix marks most of the window; each prefix is twice the
      // last (a drop costs far less than the block's rounds over candidates
      // that a drop would have removed).  The list lengths after the drops
      // stay on the device (two alternating words): the host sizes every
      // launch for an upper bound -- the list before its drops -- and queues
      // phases until that bound is used up; a phase past the real end finds
      // an empty list and returns at once.
      if (smem) APO_CUDA_TRY(cudaMemsetAsync(gbits, 0, gwords * 4, s));
      const uint32_t *pl = cl, *ps = cs, *po = nullptr;
      const uint32_t *len_dev = m_dev;  // the current list's length
      uint32_t len = mu, prefix = kGreedyFirstPhase;  // len: an upper bound of that length
      for (int phase = 0;; ++phase) {
        const uint32_t take = std::min(prefix, len);
        {
          Launch lp_(c, kKGreedy, take, s);
          if (smem)
            k_greedy<1024, true><<<1, 1024, bm_bytes + list, s>>>(pl, ps, nullptr, take, W.off_dev, n, gbits,
                                                                  acc, misc + kMiscAccCount, po, 1, len_dev,
                                                                  c->ps.err);
          else
            k_greedy<1024, false><<<1, 1024, list, s>>>(pl, ps, nullptr, take, W.off_dev, n, gbits, acc,
                                                         misc + kMiscAccCount, po, 0, len_dev, c->ps.err);
        }
        APO_CUDA_TRY(cudaGetLastError());
        if (take == len) break;
        uint32_t *kept_dev = misc + kMiscPhaseLen + (phase & 1);
        uint32_t *l2 = glist[phase & 1][0], *s2 = glist[phase & 1][1], *o2 = glist[phase & 1][2];
        PredUnmarked pu{pl, ps, gbits, take};
        APO_TRY(compact_to(c, pu, PutList{pl, ps, po, take, l2, s2, o2}, len - take, kept_dev, s, len_dev,
                           take));
        pl = l2;
        ps = s2;
        po = o2;
        len -= take;
        len_dev = kept_dev;
        prefix *= 2;
      }
    } else {
      // windows of kGWideWin tokens and more get blocks of 1024 threads (4x
      // the candidates per round: their long sequences of rounds bound the
      // launch), the others blocks of 256; each launch skips the other's
      const bool wide = W.max_len >= kGWideWin;
      const uint32_t hi = wide ? kGWideWin : 0xffffffffu;
      if (wide) {  // on the context's second stream, beside the narrow windows' launch
        const size_t list_w = glist_bytes(1024);
        const bool smem_w = (long long)(bm_bytes + list_w) <= g_greedy_smem_max;
        if (!smem_w && smem) APO_CUDA_TRY(cudaMemsetAsync(gbits, 0, gwords * 4, s));
        cudaStream_t s2 = c->aux;
        APO_CUDA_TRY(cudaEventRecord(c->fork_ev[0], s));
        APO_CUDA_TRY(cudaStreamWaitEvent(s2, c->fork_ev[0], 0));
        {
          Launch lp_(c, kKGreedy, mu, s2);
          if (smem_w)
            k_greedy<1024, true><<<W.count, 1024, bm_bytes + list_w, s2>>>(cl, cs, coff, mu, W.off_dev, n,
                                                                          nullptr, acc, misc + kMiscAccCount,
                                                                          nullptr, 0, nullptr, c->ps.err, hi);
          else
            k_greedy<1024, false><<<W.count, 1024, list_w, s2>>>(cl, cs, coff, mu, W.off_dev, n, gbits, acc,
                                                                misc + kMiscAccCount, nullptr, 0, nullptr,
                                                                c->ps.err, hi);
        }
        APO_CUDA_TRY(cudaGetLastError());
        APO_CUDA_TRY(cudaEventRecord(c->fork_ev[1], s2));
      }
      {
        Launch lp_(c, kKGreedy, mu, s);
        if (smem)
          k_greedy<256, true><<<W.count, 256, bm_bytes + list, s>>>(cl, cs, coff, mu, W.off_dev, n,
                                                                    nullptr, acc, misc + kMiscAccCount,
                                                                    nullptr, 0, nullptr, c->ps.err, 0u, hi);
        else
          k_greedy<256, false><<<W.count, 256, list, s>>>(cl, cs, coff, mu, W.off_dev, n, gbits, acc,
                                                          misc + kMiscAccCount, nullptr, 0, nullptr, c->ps.err,
                                                          0u, hi);
      }
      if (wide) APO_CUDA_TRY(cudaStreamWaitEvent(s, c->fork_ev[1], 0));  // join
    }
    APO_CUDA_TRY(cudaGetLastError());
    APO_TRY(read_u32(c, misc + kMiscAccCount, &K, s, m_dev, &m));
  }

  // R and the selected intervals
  uint32_t Tn = 0;
  uint32_t *tl = c->arena.take_n<uint32_t>(std::max<uint32_t>(K, 1));
  uint32_t *ts = c->arena.take_n<uint32_t>(std::max<uint32_t>(K, 1));
  uint32_t *ss = c->arena.take_n<uint32_t>(std::max<uint32_t>(K, 1));
  uint32_t *sl = c->arena.take_n<uint32_t>(std::max<uint32_t>(K, 1));
  uint32_t *sq = c->arena.take_n<uint32_t>(std::max<uint32_t>(K, 1));
  if (!tl || !ts || !ss || !sl || !sq) return APO_ENOMEM;
  if (K) {
    PredFlag pf{acc};
    APO_TRY(compact(c, pf, m, sel, misc + kMiscCompactCount, s));
    SortBuffers sb;
    sb.keys[0] = b.keys[0];
    sb.keys[1] = b.keys[1];
    sb.vals[0] = b.vals[0];
    sb.vals[1] = b.vals[1];
    sb.cur = 0;
    {
      const int tiles = ceil_div(K, kCTile);
      APO_TRY(ensure_lookback(c, tiles));
      APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscCompactTiles, 0, sizeof(uint32_t), s));
      Launch lp_(c, kKTraces, K, s);
      k_traces<<<tiles, kCT, 0, s>>>(sel, K, cl, cid, cs, tl, ts, sb.keys[0], sb.vals[0],
                                     misc + kMiscTraceCount, c->ps.lookback,
                                     misc + kMiscCompactTiles, next_epoch(c), c->ps.err);
    }
    const DigitRange r{32, 32 + bits_for(n - 1), false};
    APO_TRY(radix_sort_pairs(c, sb, K, &r, 1, s));
    {
      Launch lp_(c, kKSelOut, K, s);
      k_sel_out<<<grid_for(K, 256, c->num_sms), 256, 0, s>>>(sb.keys[sb.cur], sb.vals[sb.cur], K, ss,
                                                             sl, sq);
    }
    APO_CUDA_TRY(cudaGetLastError());
    APO_TRY(read_u32(c, misc + kMiscTraceCount, &Tn, s));
    if (W.count > 1) {  // per-window offsets, then window-relative values
      {
        Launch lp_(c, kKSlices, W.count + 1, s);
        k_window_bounds<<<ceil_div(W.count + 1, 256), 256, 0, s>>>(ss, K, W, n, sel_off);
        k_window_bounds<<<ceil_div(W.count + 1, 256), 256, 0, s>>>(ts, Tn, W, n, trace_off);
      }
      {
        Launch lp_(c, kKSelOut, K, s);
        k_relativize<<<grid_for(K, 256, c->num_sms), 256, 0, s>>>(ss, sq, K, W, trace_off);
        k_relativize<<<grid_for(Tn, 256, c->num_sms), 256, 0, s>>>(ts, nullptr, Tn, W, trace_off);
      }
    }
  }
  if (W.count > 1 && m && out->cand_start) {
    // window-relative candidate starts for the caller (greedy is done with them)
    Launch lp_(c, kKSelOut, m, s);
    k_relativize<<<grid_for(m, 256, c->num_sms), 256, 0, s>>>(cs, nullptr, m, W, trace_off);
  }

  bool over = false;
  APO_TRY(copy_out(out->cand_len, cl, m, out->cand_cap, &over, s));
  APO_TRY(copy_out(out->cand_id, cid, m, out->cand_cap, &over, s));
  APO_TRY(copy_out(out->cand_start, cs, m, out->cand_cap, &over, s));
  APO_TRY(copy_out(out->cand_accepted, acc, m, out->cand_cap, &over, s));
  APO_TRY(copy_out(out->sel_start, ss, K, out->sel_cap, &over, s));
  APO_TRY(copy_out(out->sel_len, sl, K, out->sel_cap, &over, s));
  APO_TRY(copy_out(out->sel_trace, sq, K, out->sel_cap, &over, s));
  APO_TRY(copy_out(out->trace_len, tl, Tn, out->trace_cap, &over, s));
  APO_TRY(copy_out(out->trace_start, ts, Tn, out->trace_cap, &over, s));
  if (boff && W.count > 1 && capturing(c)) {
    // a replay copies the offsets to the tape's pinned stage (zeros where
    // there is nothing), the host reads them after the replay
    uint32_t *h = c->tape->stage;
    const size_t wb = (size_t)(W.count + 1) * 4;
    if (m) APO_CUDA_TRY(cudaMemcpyAsync(h, cand_off, wb, cudaMemcpyDeviceToHost, s));
    else memset(h, 0, wb);
    if (K) {
      APO_CUDA_TRY(cudaMemcpyAsync(h + (W.count + 1), sel_off, wb, cudaMemcpyDeviceToHost, s));
      APO_CUDA_TRY(cudaMemcpyAsync(h + 2 * (W.count + 1), trace_off, wb, cudaMemcpyDeviceToHost, s));
    } else {
      memset(h + (W.count + 1), 0, 2 * wb);
    }
  } else if (boff && W.count > 1) {
    std::vector<uint32_t> h(3 * (size_t)(W.count + 1), 0);
    if (m) APO_CUDA_TRY(cudaMemcpyAsync(h.data(), cand_off, (W.count + 1) * 4, cudaMemcpyDeviceToHost, s));
    if (K) {
      APO_CUDA_TRY(cudaMemcpyAsync(h.data() + (W.count + 1), sel_off, (W.count + 1) * 4,
                                   cudaMemcpyDeviceToHost, s));
      APO_CUDA_TRY(cudaMemcpyAsync(h.data() + 2 * (W.count + 1), trace_off, (W.count + 1) * 4,
                                   cudaMemcpyDeviceToHost, s));
    }
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    for (uint32_t w = 0; w <= W.count; ++w) {
      if (boff->cand_off) boff->cand_off[w] = h[w];
      if (boff->sel_off) boff->sel_off[w] = h[(W.count + 1) + w];
      if (boff->trace_off) boff->trace_off[w] = h[2 * (W.count + 1) + w];
    }
  } else if (boff) {
    if (boff->cand_off) boff->cand_off[1] = m;
    if (boff->sel_off) boff->sel_off[1] = K;
    if (boff->trace_off) boff->trace_off[1] = Tn;
  }
  APO_TRY(err_check());
  counts[0] = m;
  counts[1] = K;
  counts[2] = Tn;
  if (over) {
    set_error("find_repeats: an output capacity is too small (counts written)");
    return APO_ECAPACITY;
  }
  return APO_OK;
}

}  // namespace apo
