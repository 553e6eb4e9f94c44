// Candidate matching (Sec. 4.3): the candidate traces are ingested into a
// trie and the stream is followed through it; a trace is reported whenever
// a pointer reaches its end.  All pointers at once are exactly the state of
// an Aho-Corasick automaton (Aho & Corasick, CACM 1975): the goto trie, a
// failure link per node (longest proper suffix that is also in the trie) and
// an output link per node (nearest pattern end on the failure chain).
//
// Symbols.  Tokens (u32 or u64) are mapped to dense 32-bit symbols through an
// open-addressed dictionary filled from the pattern tokens (a token's symbol
// is its slot); a stream token missing from the dictionary matches nothing.
//
// Build without a level-by-level walk.  The patterns are laid out as one
// text T = P_0 #_0 P_1 #_1 ... whose separators #_p are distinct and smaller
// than every symbol, and T gets a suffix array and an LCP array (the same
// prefix-doubling and Phi/PLCP kernels as the window analysis).  With that:
//
//  nodes   a trie node is a distinct pattern prefix x.  Its id is the
//          position in T of the last symbol of x inside the first pattern,
//          in suffix order, that starts with x.  Pattern starts in suffix
//          order, with slcp[j] = lcp(start j-1, start j), give that pattern
//          as rep(j, |x|) = the largest j' <= j with slcp[j'] < |x|.  So the
//          prefix of length d of the pattern at start j is its own node iff
//          d > slcp[j], and a node's child on its own next symbol is simply
//          the next position of T ("primary" edge, stored nowhere).  Only
//          the depth slcp[j] + 1 node of each pattern hangs off another
//          pattern's node, so the goto hash table holds at most one edge per
//          pattern.
//  fail    M(q) = the longest common prefix of suffix q with any pattern
//          start (the nearer start on either side in suffix order, two
//          segmented min-scans over LCP).  The suffix of length k of the
//          node ending at e is a node iff M(e - k) >= k, so the failure depth
//          of that node is e - q* with q* the first position after the
//          pattern's start whose reach q + M(q) is >= e: a binary search over
//          the segmented running maximum of the reach.  Its node id follows
//          from a pattern start that shares that prefix (the nearer start on
//          the side where M was attained) and rep().
//  totals  match count per node = own pattern ends + the failure link's
//          count, and the output link, by pointer jumping along failure
//          links (a fixed number of in-place rounds: the chain shrinks by at
//          least half per round).
//
// Match.  The stream is cut into short chunks and each thread runs the
// automaton over its chunk from the root, writing the state of every
// position (only the first chunk is exact).  Repair passes then give each
// group of chunks (4, or 8 on streams of 2^22 tokens and more) one warp that
// restarts from the predecessor's end state and stops at the first position
// whose state agrees with the recorded one -- from there on the
// deterministic automaton repeats the recorded run.  When a pass changes no
// end state all states are exact (after k passes groups 0..k are, by
// induction); passes are queued two at a time, and one behind a pass without
// changes returns at once.  The per-node match totals turn the output
// offsets into one prefix sum over positions; each output record's chain is
// flattened once, and a final kernel per position copies its matches.
// Where the patterns are slices of the stream itself and long (deep
// states over much of the stream), one exact pass replaces the chunks and
// repairs: a warp per segment starts its walk one longest-pattern length
// before the segment, from the root, and follows failure chains 32 nodes
// at a time through lifting tables of the skip links.
// Output order: end ascending, then pattern length descending (the output
// chain's order), then pattern id ascending.
#include <algorithm>
#include <cstring>
#include <vector>

#include "apo_internal.cuh"
#include "device_util.cuh"
#include "lcp_tree.cuh"
#include "scan.cuh"

namespace apo {

namespace {

constexpr uint32_t kNil = 0xffffffffu;  // no node; also the symbol of a token no pattern has
constexpr uint32_t kSep = 0xfffffffeu;  // symbol slot of a pattern separator in T
constexpr uint64_t kEmpty = ~0ull;
constexpr uint32_t kFlag = 0x80000000u;  // segment-start flag of a packed scan value
constexpr int kTsymPad = 40;            // separators after the pattern text (warp-wide reads)
constexpr uint64_t kMaxFlat = 1ull << 28;  // longest flattened output chains (entries)

__device__ __forceinline__ uint64_t mix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Open addressing with linear probing, capacity a power of two.  A goto entry
// is 16 bytes (key, child id, pad) so that one 128-bit load reads both.
struct Table {
  uint64_t *keys;  // entry e: keys[2e] = key, keys[2e+1] low word = value
  uint64_t mask;
};

__device__ __forceinline__ uint32_t table_lookup(const Table &g, uint32_t u, uint32_t c) {
  const uint64_t key = ((uint64_t)u << 32) | c;
  uint64_t slot = mix64(key) & g.mask;
  while (true) {
    const ulonglong2 e = *reinterpret_cast<const ulonglong2 *>(g.keys + 2 * slot);
    if (e.x == key) return (uint32_t)e.y;
    if (e.x == kEmpty) return kNil;
    slot = (slot + 1) & g.mask;
  }
}

// goto(v, c): the primary edge when T continues with c after v, else the
// branch table.
__device__ __forceinline__ uint32_t ac_goto(const uint32_t *__restrict__ tsym, const Table &g,
                                            uint32_t v, uint32_t c, uint32_t root) {
  if (v != root && tsym[v + 1] == c) return v + 1;
  return table_lookup(g, v, c);
}

// ---------------------------------------------------------------- symbols
struct Dict {
  uint64_t *keys;  // a token's symbol is its slot
  uint64_t mask;
};

template <class T>
__global__ void k_dict_insert(const T *__restrict__ tok, uint64_t m, Dict d) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = (uint64_t)tok[i];
    if (t == kEmpty) continue;  // mapped to a reserved symbol instead
    uint64_t slot = mix64(t) & d.mask;
    for (uint64_t probe = 0; probe <= d.mask; ++probe) {
      uint64_t cur = d.keys[slot];
      if (cur == t) break;
      if (cur == kEmpty) {
        cur = atomicCAS((unsigned long long *)&d.keys[slot], (unsigned long long)kEmpty,
                        (unsigned long long)t);
        if (cur == kEmpty || cur == t) break;
      }
      slot = (slot + 1) & d.mask;
    }
  }
}

template <class T>
__device__ __forceinline__ uint32_t dict_symbol(const Dict &d, T tok) {
  const uint64_t t = (uint64_t)tok;
  if (t == kEmpty) return (uint32_t)(d.mask + 1);  // reserved symbol of the all-ones token
  uint64_t slot = mix64(t) & d.mask;
  while (true) {
    const uint64_t k = d.keys[slot];
    if (k == t) return (uint32_t)slot;
    if (k == kEmpty) return kNil;
    slot = (slot + 1) & d.mask;
  }
}

template <class T>
__global__ void k_dict_map(const T *__restrict__ tok, uint64_t m, Dict d, uint32_t *__restrict__ sym) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x)
    sym[i] = dict_symbol(d, tok[i]);
}

// max length, max end and total length of slice-form patterns; flags empty ones
__global__ void k_slices(const uint32_t *__restrict__ pstart, const uint32_t *__restrict__ plen,
                         uint32_t P, uint32_t *maxlen, uint32_t *maxend,
                         unsigned long long *total, uint32_t *err) {
  uint32_t ml = 0, me = 0;
  unsigned long long tot = 0;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const uint32_t l = plen[p];
    if (l == 0) atomicExch(err, kDevRange);
    ml = max(ml, l);
    me = max(me, pstart[p] + l);
    tot += l;
  }
  atomicMax(maxlen, ml);
  atomicMax(maxend, me);
  atomicAdd(total, tot);
}

// ---------------------------------------------------------------- pattern text
// T position of pattern p's first symbol: tstart[p] = sum of earlier lengths + p.
// One warp per pattern writes its symbols and its separator: tsym (symbol,
// kSep at the separator) and tkey (the suffix-sort token: separator p -> p,
// symbol c -> P + c, so separators are distinct and below every symbol).
template <class T>
__global__ void k_pat_layout(const T *__restrict__ tok, const uint32_t *__restrict__ pstart,
                             const uint32_t *__restrict__ plen, const uint32_t *__restrict__ tstart,
                             uint32_t P, uint32_t N, Dict d, uint32_t *__restrict__ tsym,
                             uint64_t *__restrict__ tkey, uint32_t *__restrict__ tpid) {
  if (blockIdx.x == 0 && threadIdx.x < kTsymPad) tsym[N + threadIdx.x] = kSep;  // past the text
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < P; p += warps) {
    const uint32_t src = pstart[p], len = plen[p], dst = tstart[p];
    for (uint32_t k = lane; k <= len; k += 32) {
      uint32_t c = kSep;
      uint64_t key = p;
      if (k < len) {
        c = dict_symbol(d, tok[src + k]);
        key = (uint64_t)P + c;
      }
      tsym[dst + k] = c;
      tkey[dst + k] = key;
      tpid[dst + k] = p;
    }
  }
}

// ---------------------------------------------------------------- segmented scans
// Packed value: bit 31 = "a segment starts in this range", bits 30:0 = value.
struct OpSegMin {  // running minimum since the last segment start
  __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const {
    if (b & kFlag) return b;
    return (a & kFlag) | min(a & ~kFlag, b);
  }
};
struct OpSegMax {  // running maximum since the last segment start
  __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const {
    if (b & kFlag) return b;
    return (a & kFlag) | max(a & ~kFlag, b);
  }
};
constexpr uint32_t kSegMinId = 0x7fffffffu, kSegMaxId = 0u;

// Element k of the left scan over suffix order: lcp(SA[k-1], SA[k]), a
// segment start when SA[k-1] is a pattern start.  Output: the lcp of SA[k]
// with the nearest pattern start before it in suffix order (0 if none).
struct SrcLeft {
  const uint32_t *lcp;
  const uint8_t *is_start;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const {
    if (k == 0) return kSegMinId;
    return (is_start[k - 1] ? kFlag : 0u) | lcp[k - 1];
  }
};
// Element k of the right scan (run from the end): lcp(SA[k], SA[k+1]), a
// segment start when SA[k+1] is a pattern start.
struct SrcRight {
  const uint32_t *lcp;
  const uint8_t *is_start;
  uint32_t n;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const {
    if (k + 1 >= n) return kSegMinId;
    return (is_start[k + 1] ? kFlag : 0u) | lcp[k];
  }
};
struct DstFlagged {  // value where a segment start was seen, else 0
  uint32_t *out;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t v) const {
    out[k] = (v & kFlag) ? (v & ~kFlag) : 0u;
  }
};
// Element q of the reach scan over T: reach(q) = q + M(q), M(q) the longer of
// the two lcps of suffix q with its nearest pattern starts; a segment starts
// (with value 0) at each pattern's first position.
struct SrcReach {
  const uint64_t *tkey;
  const uint32_t *rank, *left, *right;
  uint32_t P;
  __device__ __forceinline__ uint32_t operator()(uint32_t q) const {
    if (q == 0 || tkey[q - 1] < P) return kFlag;
    const uint32_t r = rank[q];
    return q + max(left[r], right[r]);
  }
};
struct DstValue {
  uint32_t *out;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t v) const { out[k] = v & ~kFlag; }
};

// ---------------------------------------------------------------- pattern starts
// (rank of pattern p's first suffix, p) for the sort into suffix order.
__global__ void k_start_keys(const uint32_t *__restrict__ tstart, const uint32_t *__restrict__ rank,
                             uint32_t P, uint64_t *keys, uint32_t *vals) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    keys[p] = rank[tstart[p]];
    vals[p] = p;
  }
}

// After the sort: sorted start j is SA index sr[j] of pattern sp[j].  Marks
// the start suffixes and records each pattern's position j.
__global__ void k_start_mark(const uint64_t *__restrict__ skeys, const uint32_t *__restrict__ svals,
                             uint32_t P, uint32_t *sr, uint32_t *jpos, uint8_t *is_start) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)skeys[j];
    sr[j] = r;
    jpos[svals[j]] = j;
    is_start[r] = 1;
  }
}

// slcp[j] = lcp(start j-1, start j) in suffix order (0 for j = 0): the left
// scan's value at the start's own SA index.
__global__ void k_slcp(const uint32_t *__restrict__ sr, const uint32_t *__restrict__ left, uint32_t P,
                       uint32_t *slcp) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += gridDim.x * blockDim.x)
    slcp[j] = j ? left[sr[j]] : 0u;
}

// Sparse table of minima over windows ending at j: lev l, entry j =
// min(slcp[max(0, j - 2^l + 1) .. j]).
__global__ void k_sparse_level(const uint32_t *__restrict__ prev, uint32_t P, uint32_t half,
                               uint32_t *__restrict__ next) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < P; j += gridDim.x * blockDim.x)
    next[j] = j >= half ? min(prev[j], prev[j - half]) : prev[j];
}

// All levels 1 .. nlev-1 in one block (level l at base + l * P), for a short
// table: one launch instead of one per level.
constexpr uint32_t kSparseOneBlock = 1u << 15;
__global__ void __launch_bounds__(1024) k_sparse_all(uint32_t *base, uint32_t P, int nlev) {
  for (int l = 1; l < nlev; ++l) {
    const uint32_t *prev = base + (size_t)(l - 1) * P;
    uint32_t *next = base + (size_t)l * P;
    const uint32_t half = 1u << (l - 1);
    for (uint32_t j = threadIdx.x; j < P; j += blockDim.x)
      next[j] = j >= half ? min(prev[j], prev[j - half]) : prev[j];
    __syncthreads();
  }
}

constexpr int kMaxSparse = 33;
struct Sparse {
  const uint32_t *lev[kMaxSparse];
  int nlev;
};

// rep(j, d): the largest j' <= j with slcp[j'] < d (d >= 1; slcp[0] = 0).
__device__ __forceinline__ uint32_t rep_of(const Sparse &S, uint32_t j, uint32_t d) {
  if (S.lev[0][j] < d) return j;
  long long y = (long long)j - 1;  // every entry in (y, j] is >= d
  for (int l = S.nlev - 1; l >= 0; --l) {
    const long long w = 1ll << l;
    if (y - w + 1 >= 0 && S.lev[l][y] >= d) y -= w;
  }
  return (uint32_t)max(0ll, y);
}

// The end of the block of sorted patterns that share d symbols with pattern
// j: the smallest j' > j with slcp[j'] < d, or P.
__device__ __forceinline__ uint32_t block_end(const Sparse &S, uint32_t j, uint32_t d, uint32_t P) {
  uint32_t x = j + 1;  // every entry in (j, x) is >= d
  for (int l = S.nlev - 1; l >= 0; --l) {
    const uint64_t e = (uint64_t)x + (1u << l) - 1;
    if (e < P && S.lev[l][e] >= d) x += 1u << l;
  }
  return x;
}

// ---------------------------------------------------------------- source mode
// The patterns are slices of a source whose suffix array and LCP array are
// given.  A pattern's key is (left end of its string's LCP interval in the
// source, length): sorting by it is sorting the pattern strings (disjoint
// intervals are in string order; a proper prefix has the enclosing interval
// and sorts first at an equal left end).
__global__ void k_isa(const uint32_t *__restrict__ sa, uint32_t n, uint32_t *__restrict__ rank, uint32_t *err) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t i = sa[k];
    if (i < n) rank[i] = k;
    else atomicExch(err, kDevRange);
  }
}

__global__ void k_src_pat_keys(const uint32_t *__restrict__ pstart, const uint32_t *__restrict__ plen, uint32_t P,
                               const uint32_t *__restrict__ rank, MinTree T, int lenbits, uint64_t *keys,
                               uint32_t *vals, uint32_t *startlen, uint32_t *err) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const uint32_t st = pstart[p], len = plen[p];
    const long long j = prev_less(T, rank[st], len, err);
    keys[p] = ((uint64_t)(j + 1) << lenbits) | len;
    vals[p] = p;
    atomicMax(&startlen[st], len);
  }
}

// slcp[j] = lcp of the sorted patterns j-1 and j (direct comparison, one
// warp per j); jpos[p] = sorted position of pattern p.
template <class T>
__global__ void k_src_slcp(const T *__restrict__ tok, const uint32_t *__restrict__ pstart,
                           const uint32_t *__restrict__ plen, const uint32_t *__restrict__ sp, uint32_t P,
                           uint32_t *slcp, uint32_t *jpos) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < P; j += warps) {
    const uint32_t b = sp[j];
    if (lane == 0) jpos[b] = j;
    uint32_t l = 0;
    if (j > 0) {
      const uint32_t a = sp[j - 1];
      const uint32_t m = min(plen[a], plen[b]);
      const T *x = tok + pstart[a], *y = tok + pstart[b];
      for (uint32_t k0 = 0; k0 < m; k0 += 32) {
        const uint32_t k = k0 + lane;
        const uint32_t miss = __ballot_sync(0xffffffffu, k < m && x[k] != y[k]);
        if (miss) {
          l = k0 + __ffs(miss) - 1;
          break;
        }
        l = min(m, k0 + 32);
      }
    }
    if (lane == 0) slcp[j] = l;
  }
}

// F(k) = max over pattern starts at suffix ranks <= k (resp. >= k) of
// min(pattern length, LCP of the two suffixes): the scan element of rank k is
// the map x -> max(s_k, min(x, l_k)) (s_k: longest pattern starting at SA[k],
// l_k: the LCP towards the previous rank), and these maps compose into maps
// of the same form, (s, l) then (s', l') = (max(s', min(s, l')), min(l, l')).
// Both parts are clamped to 16 bits (to the longest pattern, below 2^16).
struct OpClampCompose {
  __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const {
    const uint32_t as = a >> 16, al = a & 0xffffu, bs = b >> 16, bl = b & 0xffffu;
    return (max(bs, min(as, bl)) << 16) | min(al, bl);
  }
};
constexpr uint32_t kClampId = 0x0000ffffu;
struct SrcFnLeft {
  const uint32_t *sa, *lcp, *startlen;
  uint32_t cap;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const {
    const uint32_t sv = min(startlen[sa[k]], cap), lv = k ? min(lcp[k - 1], cap) : 0u;
    return (sv << 16) | lv;
  }
};
struct SrcFnRight {
  const uint32_t *sa, *lcp, *startlen;
  uint32_t cap, n;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const {
    const uint32_t sv = min(startlen[sa[k]], cap), lv = k + 1 < n ? min(lcp[k], cap) : 0u;
    return (sv << 16) | lv;
  }
};
struct DstFnLeft {
  uint32_t *out;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t v) const { out[k] = v >> 16; }
};
struct DstFnRight {  // M of source position SA[k] = the better of both sides
  const uint32_t *sa, *left;
  uint32_t *mw;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t v) const { mw[sa[k]] = max(left[k], v >> 16); }
};
// reach(q) = q + M(q) over T, M(q) = min(the pattern's remaining length,
// M of the source position), a segment starting at each pattern
struct SrcReachSrc {
  const uint32_t *tsym, *tpid, *tstart, *plen, *pstart, *mw;
  __device__ __forceinline__ uint32_t operator()(uint32_t q) const {
    if (q == 0 || tsym[q - 1] == kSep) return kFlag;
    const uint32_t p = tpid[q], o = q - tstart[p], rem = plen[p] - o;
    return q + (rem ? min(rem, mw[pstart[p] + o]) : 0u);
  }
};

// ---------------------------------------------------------------- nodes and links
struct NodeArgs {
  const uint32_t *tstart, *plen, *tsym;
  const uint32_t *jpos, *sp, *sr;  // sorted starts: pattern sp[j] at SA index sr[j]
  const uint32_t *rank, *left, *reach;
  Sparse S;  // minima over slcp
  uint32_t P, root;
  Table g;
  uint32_t *fail, *own, *end_node;
  uint8_t *has_branch;  // [nodes] 1 if a branch-table edge leaves the node
  unsigned long long *pref;  // [nodes] preferred child (null: not wanted), zeroed
  uint32_t *err;
  // source mode (the patterns are slices of a source with a known suffix
  // array): failure nodes are found through the source's LCP intervals
  bool src;
  const uint32_t *pstart, *src_rank;
  const uint64_t *skey;  // sorted pattern keys (LCP-interval left end << lenbits | length)
  MinTree T;             // over the source LCP
  int lenbits;
};

__device__ __forceinline__ void table_insert(const Table &g, uint32_t u, uint32_t c, uint32_t v,
                                             uint32_t *err) {
  const uint64_t key = ((uint64_t)u << 32) | c;
  uint64_t slot = mix64(key) & g.mask;
  for (uint64_t probe = 0; probe <= g.mask; ++probe) {
    uint64_t *ek = g.keys + 2 * slot;
    const uint64_t cur = atomicCAS((unsigned long long *)ek, (unsigned long long)kEmpty,
                                   (unsigned long long)key);
    if (cur == kEmpty) {
      ek[1] = v;
      return;
    }
    slot = (slot + 1) & g.mask;
  }
  atomicExch(err, kDevRange);
}

// Node id of the pattern prefix of length d shared with sorted start j.
__device__ __forceinline__ uint32_t node_of(const NodeArgs &a, uint32_t j, uint32_t d) {
  return a.tstart[a.sp[rep_of(a.S, j, d)]] + d - 1;
}

// One warp per pattern, one lane per depth d = 1 .. len + 1 (len + 1 is the
// separator after the pattern).  A depth-d prefix that is its own node gets
// its failure link, and the branch edge into it when it hangs off another
// pattern's node; the pattern's end node counts one more pattern end.  With
// `pref`, every node also gets its preferred child: the one that the most
// patterns pass through (for slices of the stream itself, the way the stream
// most likely continues; ties to the larger node id).  The preferred
// children are wanted by the halo pass only, which is when kPref is set.
template <bool kPref>
__global__ void k_ac_nodes(NodeArgs a) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.P; i += warps) {
    const uint32_t S = a.tstart[i], len = a.plen[i], j = a.jpos[i];
    const uint32_t sl = a.S.lev[0][j];
    for (uint32_t d = lane + 1; d <= len + 1; d += 32) {
      const uint32_t v = S + d - 1;
      uint32_t f = a.root;
      if (d <= len && d > sl) {
        const uint32_t e = S + d;
        if (d >= 2 && a.reach[e - 1] >= e) {
          uint32_t lo = S + 1, hi = e - 1;  // first q in (S, e) with reach >= e
          while (lo < hi) {
            const uint32_t mid = lo + ((hi - lo) >> 1);
            if (a.reach[mid] >= e) hi = mid;
            else lo = mid + 1;
          }
          const uint32_t fd = e - lo;
          if (a.src) {
            // the string's LCP interval in the source; the first pattern in
            // sorted order whose key is not below (left end, fd) starts with it
            const uint32_t r = a.src_rank[a.pstart[i] + (lo - S)];
            const uint64_t key = ((uint64_t)(prev_less(a.T, r, fd, a.err) + 1) << a.lenbits) | fd;
            uint32_t jl = 0, jh = a.P;
            while (jl < jh) {
              const uint32_t mid = (jl + jh) >> 1;
              if (a.skey[mid] < key) jl = mid + 1;
              else jh = mid;
            }
            if (jl >= a.P) atomicExch(a.err, kDevRange);
            else f = a.tstart[a.sp[jl]] + fd - 1;
          } else {
            const uint32_t k = a.rank[lo];
            uint32_t cnt = 0, hi2 = a.P;  // starts before SA index k
            while (cnt < hi2) {
              const uint32_t mid = (cnt + hi2) >> 1;
              if (a.sr[mid] < k) cnt = mid + 1;
              else hi2 = mid;
            }
            const uint32_t jj = (a.left[k] >= fd) ? cnt - 1 : cnt;
            if (jj >= a.P) {
              atomicExch(a.err, kDevRange);
            } else {
              f = node_of(a, jj, fd);
            }
          }
        }
        if (d == sl + 1) {
          const uint32_t parent = d == 1 ? a.root : node_of(a, j, d - 1);
          table_insert(a.g, parent, a.tsym[v], v, a.err);
          a.has_branch[parent] = 1;
          if (kPref && d > 1)  // v as a child of parent, weighed by the patterns through it
            atomicMax(&a.pref[parent], ((unsigned long long)(block_end(a.S, j, d, a.P) - j) << 32) | v);
        }
        if (kPref && d < len)  // v's own next position as its child
          atomicMax(&a.pref[v], ((unsigned long long)(block_end(a.S, j, d + 1, a.P) - j) << 32) | (v + 1));
      }
      a.fail[v] = f;
      if (d == len) {
        const uint32_t en = node_of(a, j, len);
        a.end_node[i] = en;
        atomicAdd(&a.own[en], 1u);
      }
    }
  }
}

// Pointer jumping along failure links, in place.  w[v] = (pointer << 32) |
// sum of own over the chain from v up to the pointer (exclusive); jl[v] =
// the first node with own > 0 found so far on the chain after v.  Every
// value read is a valid state of its owner, so a round may see another
// node's update of the same round.  The last round writes the totals, each
// node's first output record and each record's successor (the record of the
// output link).
// Skip links for matching: sk[v] = the first node u on v's failure chain that
// could have a transition v's own primary symbol cannot rule out, i.e. the
// root, a node with branch-table edges, or a node whose primary symbol
// differs from v's.  A failure step is only taken after v's primary edge did
// not match, so the nodes skipped (no branch edges, the same primary symbol)
// cannot match either.  sk[u] of a skipped u has the same criterion as sk[v],
// which makes the jumps composable.
__global__ void k_ac_jump(uint64_t *w, uint32_t *jl, uint32_t *sk, const uint32_t *__restrict__ own,
                          const uint32_t *__restrict__ tsym, const uint8_t *__restrict__ has_branch,
                          uint32_t nodes, uint32_t root, int last, uint32_t *total,
                          const uint32_t *__restrict__ recidx, uint32_t *firstrec, uint4 *rec, uint32_t *err) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nodes; v += gridDim.x * blockDim.x) {
    uint32_t u = sk[v];
    const uint32_t a = v != root ? tsym[v + 1] : kNil;
    const bool skippable = u != root && !has_branch[u] && tsym[u + 1] == a;
    if (skippable) {
      u = *(volatile uint32_t *)&sk[u];
      sk[v] = u;
    }
    if (last && u != root && !has_branch[u] && tsym[u + 1] == a) atomicExch(err, kDevRange);
    uint64_t x = w[v];
    uint32_t p = (uint32_t)(x >> 32);
    if (p != root) {
      const uint64_t y = *(volatile uint64_t *)&w[p];
      x = (y & 0xffffffff00000000ull) | (uint32_t)((uint32_t)x + (uint32_t)y);
      w[v] = x;
      p = (uint32_t)(x >> 32);
    }
    uint32_t o = jl[v];
    if (o != root && own[o] == 0) {
      o = *(volatile uint32_t *)&jl[o];
      jl[v] = o;
    }
    if (last) {
      if (p != root || (o != root && own[o] == 0)) atomicExch(err, kDevRange);
      total[v] = (uint32_t)x;
      const uint32_t ro = o != root ? recidx[o] : kNil;  // output record of the output link
      if (v != root && own[v] != 0) {
        const uint32_t r = recidx[v];
        rec[r].z = ro;
        firstrec[v] = r;
      } else {
        firstrec[v] = ro;
      }
    }
  }
}

__global__ void k_jump_init(const uint32_t *__restrict__ fail, const uint32_t *__restrict__ own,
                            uint32_t nodes, uint32_t root, uint64_t *w, uint32_t *jl, uint32_t *sk) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nodes; v += gridDim.x * blockDim.x) {
    const uint32_t f = v == root ? root : fail[v];
    sk[v] = f;
    w[v] = ((uint64_t)f << 32) | own[v];
    jl[v] = f;
  }
}

__global__ void k_table_init(uint64_t *keys, uint64_t entries) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < entries;
       e += (uint64_t)gridDim.x * blockDim.x) {
    keys[2 * e] = kEmpty;
    keys[2 * e + 1] = 0;
  }
}

__global__ void k_end_pairs(const uint32_t *__restrict__ end_node, uint32_t P, uint64_t *keys,
                            uint32_t *vals) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    keys[p] = end_node[p];
    vals[p] = p;
  }
}

// Output records: one per node where patterns end, in node order after the
// sort of (end node, pattern id): rec = (first sorted index, patterns ending
// there, next record down the output chain); recidx[node] = its record.
struct SrcRunStart {
  const uint64_t *keys;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const {
    return (k == 0 || keys[k] != keys[k - 1]) ? 1u : 0u;
  }
};
struct DstRecord {
  const uint64_t *keys;
  const uint32_t *own;
  uint32_t *recidx;
  uint4 *rec;      // (first sorted index, patterns ending there, next record, node)
  uint32_t P;
  uint32_t *count;  // number of records
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t v) const {
    if (k == 0 || keys[k] != keys[k - 1]) {
      const uint32_t node = (uint32_t)keys[k];
      recidx[node] = v - 1;
      rec[v - 1] = make_uint4(k, own[node], kNil, node);
    }
    if (k == P - 1) *count = v;
  }
};

// Flattened output chains: record r's chain (all its matches, in report
// order) is flat[flat_off[r] .. + rtot[r]).  rtot[r] = the match total of
// the record's node for r < *R_dev, 0 for the rest of the P-entry bound.
__global__ void k_rec_totals(const uint4 *__restrict__ rec, const uint32_t *__restrict__ total, uint32_t P,
                             const uint32_t *R_dev, uint32_t *rtot) {
  const uint32_t R = min(P, *R_dev);
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < P; r += gridDim.x * blockDim.x)
    rtot[r] = r < R ? total[rec[r].w] : 0u;
}

struct SrcU32 {
  const uint32_t *a;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const { return a[k]; }
};
struct DstExclusive {  // out[k] = inclusive - a[k]; *sum = the grand total
  const uint32_t *a;
  uint32_t *out, *sum;
  uint32_t n;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t v) const {
    out[k] = v - a[k];
    if (k == n - 1) *sum = v;
  }
};

// One warp per record walks its chain and writes the ids.
__global__ void k_flat_chains(const uint4 *__restrict__ rec, uint32_t R, const uint32_t *__restrict__ flat_off,
                              const uint32_t *__restrict__ evals, uint32_t *__restrict__ flat) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < R; r += warps) {
    uint32_t o = flat_off[r];
    uint32_t cur = r;
    while (cur != kNil) {
      const uint4 q = rec[cur];
      for (uint32_t k = lane; k < q.y; k += 32) flat[o + k] = evals[q.x + k];
      o += q.y;
      cur = q.z;
    }
  }
}

// Pass B over flattened chains: one warp per 32 positions; lane j fetches
// position x0+j's chain; short chains are copied by their own lane, long ones
// by the whole warp in position order (contiguous reads and writes).
constexpr uint32_t kFillOwn = 4;
__global__ void k_ac_fill_flat(const uint32_t *__restrict__ state, uint32_t n, const uint32_t *__restrict__ off,
                               const uint32_t *__restrict__ firstrec, const uint32_t *__restrict__ rtot,
                               const uint32_t *__restrict__ flat_off, const uint32_t *__restrict__ flat,
                               uint32_t *mend, uint32_t *mid, uint64_t cap) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint64_t x0 = (uint64_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; x0 < n;
       x0 += (uint64_t)warps * 32) {
    const uint64_t x = x0 + lane;
    uint32_t cnt = 0, src = 0, dst = 0;
    if (x < n) {
      const uint32_t r = firstrec[state[x]];
      if (r != kNil) {
        cnt = rtot[r];
        src = flat_off[r];
        dst = off[x];
      }
    }
    if (cnt <= kFillOwn) {  // short chains: each lane copies its own
      for (uint32_t k = 0; k < cnt; ++k) {
        if (dst + (uint64_t)k < cap) {
          mend[dst + k] = (uint32_t)x;
          mid[dst + k] = flat[src + k];
        }
      }
    }
    for (uint32_t busy = __ballot_sync(0xffffffffu, cnt > kFillOwn); busy; busy &= busy - 1) {
      const int j = __ffs(busy) - 1;
      const uint32_t c = __shfl_sync(0xffffffffu, cnt, j);
      const uint32_t sj = __shfl_sync(0xffffffffu, src, j);
      const uint64_t dj = __shfl_sync(0xffffffffu, dst, j);
      const uint32_t xj = (uint32_t)(x0 + j);
      for (uint32_t k = lane; k < c; k += 32) {
        if (dj + k < cap) {
          mend[dj + k] = xj;
          mid[dj + k] = flat[sj + k];
        }
      }
    }
  }
}

// ---------------------------------------------------------------- match
// One warp runs the automaton over one chunk.  Along a primary edge the next
// state is the next position of T, so the warp compares up to 32 stream
// symbols with the 32 symbols of T after the current state at once and
// takes the whole agreeing run in one step; a mismatch is settled by one
// lane with the goto table and the failure chain.
constexpr int kLift = 5;  // skip^(2^k), k < kLift: 32 chain nodes per warp-wide step
struct Automaton {
  const uint32_t *tsym;  // padded with kTsymPad separators past the text
  const uint8_t *has_branch;
  Table g;
  const uint32_t *skip;  // failure steps taken after the primary edge did not match
  uint32_t root;
  const uint32_t *lift[kLift];  // lift[k][u] = skip^(2^k)(u) (warp-wide walks only)
  uint32_t batches;             // bound on the 32-node steps of one walk (chains end at the root)
  const uint32_t *heavy[kLift];  // heavy[k][u] = hc^(2^k)(u), hc = preferred child (halo pass)
};
constexpr int kStateWarps = 4;

// Runs positions [x, x1) from state v.  With `recorded`, stops at the first
// position whose new state equals the state already stored there (the run
// from there on is the stored one) and returns true.  *v_out: the state after
// the last position run.
template <bool kCheck>
__device__ __forceinline__ bool run_chunk(const uint32_t *__restrict__ ssym, uint64_t x, uint64_t x1,
                                          uint32_t v, const Automaton &A, uint32_t *__restrict__ state,
                                          uint32_t *v_out) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t root = A.root;
  while (x < x1) {
    uint32_t m = 0;
    if (v != root) {
      const uint64_t xi = x + lane;
      const bool ok = xi < x1 && ssym[xi] == A.tsym[v + 1 + lane];
      const uint32_t miss = __ballot_sync(0xffffffffu, !ok);
      m = miss ? (uint32_t)(__ffs(miss) - 1) : 32u;
    }
    else {
      // from the root: positions whose symbol starts no pattern stay at the
      // root, so the first of the next 32 that does is found at once
      const uint64_t xi = x + lane;
      uint32_t r = kNil;
      if (xi < x1) r = table_lookup(A.g, root, ssym[xi]);
      const uint32_t hit = __ballot_sync(0xffffffffu, r != kNil || xi >= x1);
      const uint32_t h = hit ? (uint32_t)(__ffs(hit) - 1) : 32u;  // positions staying at the root
      if (h > 0) {
        if (kCheck) {
          const uint32_t ab = __ballot_sync(0xffffffffu, lane < h && state[xi] == root);
          if (ab) {
            const uint32_t first = __ffs(ab) - 1;
            if (lane < first) state[xi] = root;
            return true;
          }
        }
        if (lane < h) state[xi] = root;
        x += h;
        continue;
      }
      // position x leaves the root on its own symbol
      const uint32_t nv = __shfl_sync(0xffffffffu, r, 0);
      if (kCheck && __shfl_sync(0xffffffffu, lane == 0 ? state[x] : 0u, 0) == nv) return true;
      if (lane == 0) state[x] = nv;
      v = nv;
      ++x;
      continue;
    }
    if (m > 0) {
      if (kCheck) {
        const bool agree = lane < m && state[x + lane] == v + 1 + lane;
        const uint32_t ab = __ballot_sync(0xffffffffu, agree);
        if (ab) {
          const uint32_t first = __ffs(ab) - 1;
          if (lane < first) state[x + lane] = v + 1 + lane;
          return true;
        }
      }
      if (lane < m) state[x + lane] = v + 1 + lane;
      v += m;
      x += m;
      continue;
    }
    uint32_t nv = root;
    if (lane == 0) {
      const uint32_t c = ssym[x];
      uint32_t cur = v;
      while (true) {
        const uint32_t nx = ac_goto(A.tsym, A.g, cur, c, root);
        if (nx != kNil) {
          nv = nx;
          break;
        }
        if (cur == root) break;
        cur = A.skip[cur];
      }
      if (kCheck && state[x] == nv) nv = kNil;  // agreement
      else state[x] = nv;
    }
    nv = __shfl_sync(0xffffffffu, nv, 0);
    if (kCheck && nv == kNil) return true;
    v = nv;
    ++x;
  }
  *v_out = v;
  return false;
}

// Pass A1: chunk t = positions [t*chunk, (t+1)*chunk) from the root state,
// one lane per chunk (short chunks, many of them: the first pass is mostly
// short runs and failure steps, which independent lanes overlap best).  One
// goto probe or one failure step per loop iteration, so that the lanes of a
// warp advance through their chunks independently.  Chunk 0 is exact; the
// others may start in the wrong state.
__global__ void k_ac_states(const uint32_t *__restrict__ ssym, uint64_t n, uint64_t chunk, Automaton A,
                            uint32_t *__restrict__ state_out) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t cs = t * chunk;
  if (cs >= n) return;
  const uint64_t ce = min(n, cs + chunk);
  const uint32_t root = A.root;
  uint32_t state = root, cur = root;  // cur: where the transition for x is being looked up
  uint64_t x = cs;
  uint32_t c = ssym[x];
  while (x < ce) {
    const uint32_t nx = ac_goto(A.tsym, A.g, cur, c, root);
    if (nx != kNil || cur == root) {
      state = nx != kNil ? nx : root;
      state_out[x] = state;
      cur = state;
      if (++x < ce) c = ssym[x];
    } else {
      cur = A.skip[cur];
    }
  }
}

// Pass A2 (repeated until nothing changes), one warp per group of `group`
// consecutive first-pass chunks: the group restarts from the state stored at
// its predecessor's last position, and each of its chunks re-runs until its
// state equals the stored one (the rest of that chunk was stored by a
// continuous run, so it already agrees), then the next chunk continues from
// the stored end state.  The start state may be read while the predecessor
// is still rewriting it; then the predecessor's end state changes in this
// pass and the host runs another.  When no group's end state changes, every
// group continues its predecessor exactly and all states are exact.
__global__ void __launch_bounds__(32 * kStateWarps)
    k_ac_fix(const uint32_t *__restrict__ ssym, uint64_t n, uint64_t chunk, uint32_t group, Automaton A,
             uint32_t *__restrict__ state, const uint32_t *prev_changed, uint32_t *changed) {
  // a pass queued behind one that changed nothing has nothing to do
  if (prev_changed && *(volatile const uint32_t *)prev_changed == 0) return;
  const uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t g0 = t * chunk * group;
  if (g0 >= n) return;
  const uint64_t ce = min(n, g0 + chunk * group);
  const uint64_t cs = g0 == 0 ? chunk : g0;  // the first chunk of all is exact
  if (cs >= ce) return;
  const uint32_t rec_end = state[ce - 1];
  uint32_t v = *(volatile uint32_t *)&state[cs - 1];
  for (uint64_t fs = cs; fs < ce; fs += chunk) {
    const uint64_t fe = min(ce, fs + chunk);
    if (run_chunk<true>(ssym, fs, fe, v, A, state, &v)) {
      __syncwarp();
      v = state[fe - 1];
    }
  }
  if ((threadIdx.x & 31) == 0 && v != rec_end) atomicAdd(changed, 1u);
}

// Pass A with a halo (exact in one pass).  The state at x is the longest
// suffix of the stream up to x that is a trie node, so its depth is at most
// the longest pattern length H.  A walk from the root that starts H
// positions before g0 has read every symbol that state can span, and from
// g0 on its states are the exact ones: each warp takes a segment [g0, g0 +
// seg), starts at g0 - H and writes the states of its segment only.  The
// halo costs H extra positions per segment; it pays where states are deep
// (long patterns that the stream contains), which makes the chunked first
// pass wrong over most positions and its repairs long.

// The transition from v (not the root) on c after v's preferred child did
// not match: v's next position in T or a branch edge of v, else the first
// node on v's skip chain with an edge on c (the root, with or without one,
// ends every chain).  The chain is taken 32 nodes at a time: lane j gets
// skip^j(u0) in five doubling rounds (lanes [2^k, 2^(k+1)) apply
// skip^(2^k) to the node of lane j - 2^k), the lanes test their nodes at
// once and the first hit in chain order wins.
__device__ __forceinline__ uint32_t fail_walk_warp(const Automaton &A, uint32_t v, uint32_t c,
                                                   uint32_t *err) {
  const uint32_t lane = threadIdx.x & 31, root = A.root;
  uint32_t u0 = A.skip[v];
  if (A.tsym[v + 1] == c) return v + 1;  // when the preferred child was another one
  if (A.has_branch[v]) {
    const uint32_t r = table_lookup(A.g, v, c);
    if (r != kNil) return r;
  }
  for (uint32_t step = 0; step < A.batches; ++step) {
    uint32_t u = u0;
#pragma unroll
    for (int k = 0; k < kLift; ++k) {
      const uint32_t from = __shfl_up_sync(0xffffffffu, u, 1u << k);
      if (lane >= (1u << k) && lane < (2u << k)) u = A.lift[k][from];
    }
    uint32_t r = kNil;
    bool hit = false;
    if (u == root) {
      r = table_lookup(A.g, root, c);
      if (r == kNil) r = root;
      hit = true;
    } else {
      const uint32_t p = A.tsym[u + 1];
      const uint8_t b = A.has_branch[u];
      if (p == c) {
        r = u + 1;
        hit = true;
      } else if (b) {
        r = table_lookup(A.g, u, c);
        hit = r != kNil;
      }
    }
    const uint32_t h = __ballot_sync(0xffffffffu, hit);
    if (h) return __shfl_sync(0xffffffffu, r, __ffs(h) - 1);
    u0 = A.skip[__shfl_sync(0xffffffffu, u, 31)];  // skip^32 of this step's first node
  }
  if (lane == 0) atomicExch(err, kDevRange);  // a chain longer than the deepest node
  return root;
}

// One warp runs positions [x, x1) from the root and writes the states of
// [wfrom, x1): down the path of preferred children 32 positions per step,
// from the root the positions that start no pattern 32 at a time, a
// mismatch by the warp-wide failure walk.
__device__ __forceinline__ void run_exact(const uint32_t *__restrict__ ssym, uint64_t x, uint64_t wfrom,
                                          uint64_t x1, const Automaton &A, uint32_t *__restrict__ state,
                                          uint32_t *err) {
  const uint32_t lane = threadIdx.x & 31, root = A.root;
  uint32_t v = root;
  while (x < x1) {
    const uint64_t xi = x + lane;
    const uint32_t sy = xi < x1 ? ssym[xi] : kNil;
    if (v != root) {
      // down the path of preferred children: lane j tests node hc^(j+1)(v)
      // (doubling rounds as in the failure walk), whose own symbol is the
      // one that leads into it
      uint32_t u = A.heavy[0][v];
#pragma unroll
      for (int k = 0; k < kLift; ++k) {
        const uint32_t from = __shfl_up_sync(0xffffffffu, u, 1u << k);
        if (lane >= (1u << k) && lane < (2u << k)) u = A.heavy[k][from];
      }
      const bool ok = xi < x1 && sy == A.tsym[u];
      const uint32_t miss = __ballot_sync(0xffffffffu, !ok);
      const uint32_t m = miss ? (uint32_t)(__ffs(miss) - 1) : 32u;
      if (m > 0) {
        if (lane < m && xi >= wfrom) state[xi] = u;
        v = __shfl_sync(0xffffffffu, u, m - 1);
        x += m;
        continue;
      }
      v = fail_walk_warp(A, v, __shfl_sync(0xffffffffu, sy, 0), err);
    } else {
      const uint32_t r = xi < x1 ? table_lookup(A.g, root, sy) : kNil;
      const uint32_t hit = __ballot_sync(0xffffffffu, r != kNil || xi >= x1);
      const uint32_t h = hit ? (uint32_t)(__ffs(hit) - 1) : 32u;  // positions staying at the root
      if (h > 0) {
        if (lane < h && xi >= wfrom) state[xi] = root;
        x += h;
        continue;
      }
      v = __shfl_sync(0xffffffffu, r, 0);
    }
    if (lane == 0 && x >= wfrom) state[x] = v;
    ++x;
  }
}

__global__ void __launch_bounds__(32 * kStateWarps)
    k_ac_halo(const uint32_t *__restrict__ ssym, uint64_t n, uint64_t seg, uint64_t halo, Automaton A,
              uint32_t *__restrict__ state, uint32_t *err) {
  const uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // the same in the warp
  const uint64_t g0 = t * seg;
  if (g0 >= n) return;
  run_exact(ssym, g0 > halo ? g0 - halo : 0, g0, min(n, g0 + seg), A, state, err);
}

// hc[t] over T positions and the root: a node's preferred child (its next
// position in T when no preference was recorded), a separator and the root
// map to themselves -- a separator's symbol matches no stream symbol, so a
// walk down the path stops there.
__global__ void k_heavy_init(const uint32_t *__restrict__ tsym, const unsigned long long *__restrict__ pref,
                             uint32_t N, uint32_t *__restrict__ hc) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= N; t += gridDim.x * blockDim.x) {
    uint32_t h = t;
    if (t < N && tsym[t] != kSep) h = pref[t] ? (uint32_t)pref[t] : t + 1;
    hc[t] = h;
  }
}

// next[v] = prev[prev[v]] for two tables at once: the lifting tables of the
// skip links and of the preferred children, one doubling each
__global__ void k_lift(const uint32_t *__restrict__ prev_a, uint32_t *__restrict__ next_a,
                       const uint32_t *__restrict__ prev_b, uint32_t *__restrict__ next_b, uint32_t nodes) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nodes; v += gridDim.x * blockDim.x) {
    next_a[v] = prev_a[prev_a[v]];
    next_b[v] = prev_b[prev_b[v]];
  }
}

// Exclusive prefix sum of total[state[x]] over stream positions (the first
// output slot of each position), decoupled look-back.
constexpr int kST = 256, kSI = 8, kSTile = kST * kSI;
__global__ void __launch_bounds__(kST) k_match_offsets(const uint32_t *__restrict__ state,
                                                       const uint32_t *__restrict__ total, uint32_t n,
                                                       uint32_t *__restrict__ off, uint32_t *sum_out,
                                                       uint64_t *status, uint32_t *tile_ctr,
                                                       uint32_t epoch, uint32_t *err) {
  __shared__ uint32_t s_tile, s_pre;
  __shared__ uint32_t scr[kST / 32];
  __shared__ uint32_t sv[kSTile];
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t base = (uint64_t)t * kSTile;
  for (int q = tid; q < kSTile; q += kST) sv[q] = base + q < n ? total[state[base + q]] : 0u;
  __syncthreads();
  uint32_t run = 0;
#pragma unroll
  for (int i = 0; i < kSI; ++i) run += sv[tid * kSI + i];
  uint32_t tot;
  const uint32_t ex = block_exclusive<kST / 32>(run, OpSum(), 0u, scr, &tot);
  if (tid == 0) {
    lb_store(&status[t], lb_pack(t == 0 ? kLbInclusive : kLbAggregate, epoch, tot));
    uint32_t pre = 0;
    if (t > 0) {
      pre = lb_exclusive_k<8>(status, 1, t, epoch, OpSum(), 0u, err);
      lb_store(&status[t], lb_pack(kLbInclusive, epoch, pre + tot));
    }
    s_pre = pre;
    if (base + kSTile >= n) *sum_out = pre + tot;
  }
  __syncthreads();
  uint32_t r = s_pre + ex;
#pragma unroll
  for (int i = 0; i < kSI; ++i) {  // exclusive offsets back into the tile, then written coalesced
    const uint32_t v = sv[tid * kSI + i];
    sv[tid * kSI + i] = r;
    r += v;
  }
  __syncthreads();
  for (int q = tid; q < kSTile; q += kST)
    if (base + q < n) off[base + q] = sv[q];
}

// Pass B: the matches of position x, down the output chain from its state
// (deepest first), ids ascending within a node.  The chain is walked over
// the compact output records (one 16-byte load per node that ends patterns).
__global__ void k_ac_fill(const uint32_t *__restrict__ state, uint32_t n, const uint32_t *__restrict__ off,
                          const uint32_t *__restrict__ firstrec, const uint4 *__restrict__ rec,
                          const uint32_t *__restrict__ evals, uint32_t *mend, uint32_t *mid, uint64_t cap) {
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    uint32_t r = firstrec[state[x]];
    uint64_t o = off[x];
    while (r != kNil) {
      const uint4 q = rec[r];
      for (uint32_t k = q.x; k < q.x + q.y; ++k) {
        if (o < cap) {
          mend[o] = x;
          mid[o] = evals[k];
        }
        ++o;
      }
      r = q.z;
    }
  }
}

}  // namespace

int match_init(int sms) {
  (void)sms;
  return APO_OK;
}

size_t suffix_workspace_bytes(uint64_t n);

namespace {
uint64_t pow2_at_least(uint64_t x) {
  uint64_t t = 1;
  while (t < x) t <<= 1;
  return t;
}
int sa_levels(uint64_t maxlen) { return bits_for(maxlen + 1) + 3; }
}  // namespace

size_t match_workspace_bytes(uint64_t total_tokens, uint64_t P, uint64_t n, uint64_t extent,
                             uint64_t maxlen, uint64_t src_n) {
  const uint64_t N = total_tokens + P;  // pattern text with separators
  const uint64_t tbl = pow2_at_least(2 * (P + 1));
  const uint64_t dct = pow2_at_least(2 * (extent + 1));
  const uint64_t sparse = (uint64_t)(bits_for(P) + 1) * P;
  // pattern text (symbols, sort tokens, pattern ids, reach) and the per-node
  // arrays (with the halo pass's preferred children and lifting tables)
  uint64_t bytes = N * (8 + 4 + 4) + (N + kTsymPad) * (4 + 4 + 8 + 4 + 4 + 4 + 4 + 4 + 1 + 16 + 8 + 20) +
                   P * (16 + 8) +
                   tbl * 16 + dct * 8 + P * (4 * 8 + 24) + sparse * 4 + (extent + n) * 4 + n * 8 + 96 * 256 +
                   P * 8;  // record totals and flattened-chain offsets
  if (src_n)  // source ranks, start lengths, both interval scans, the LCP min-tree
    bytes += src_n * 16 + (src_n / 31 + 1) * 4 + kMaxTree * 256;
  else  // the suffix array, LCP and nearest-start scans of the pattern text
    bytes += suffix_workspace_bytes(N) + (uint64_t)sa_levels(maxlen) * N * 4 + N * (4 + 1 + 4 + 4);
  return bytes;
}

namespace {


// Exclusive prefix of plen[p] + 1 (pattern p's first position in T).
struct SrcPlen {
  const uint32_t *plen;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const { return plen[k] + 1; }
};
struct DstTstart {
  const uint32_t *plen;
  uint32_t *out;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t v) const { out[k] = v - plen[k] - 1; }
};


}  // namespace

int match_patterns(apo_ctx *c, const apo_patterns *pp, const void *stream, uint64_t n,
                   uint32_t *match_end, uint32_t *match_id, uint64_t cap, uint64_t *count,
                   cudaStream_t s, uint32_t *aux_order, uint32_t *aux_slcp) {
  ScopeGuard scope_(c, kScopeMatch);
  const uint32_t P = (uint32_t)pp->n_patterns;
  const int tb = pp->token_bytes;
  uint32_t *misc = c->ps.counters + kCtrMisc;
  unsigned long long *cnt64 = reinterpret_cast<unsigned long long *>(misc + kMiscKeyOr);
  const int sms = c->num_sms;
  // pattern p = tokens[pstart[p] .. pstart[p] + plen[p])
  const uint32_t *pstart = pp->pat_start, *plen = pp->pat_len;
  uint64_t total = 0, maxlen = 0, extent = 0;
  if (pp->pat_off) {
    for (uint32_t p = 0; p < P; ++p) maxlen = std::max(maxlen, pp->pat_off[p + 1] - pp->pat_off[p]);
    total = pp->pat_off[P];
    extent = total;
  } else {
    APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscMaxLen, 0, 2 * sizeof(uint32_t), s));
    APO_CUDA_TRY(cudaMemsetAsync(cnt64, 0, 8, s));
    {
      Launch lp_(c, kKSlices, P, s);
      k_slices<<<grid_for(P, 256, sms), 256, 0, s>>>(pstart, plen, P, misc + kMiscMaxLen,
                                                      misc + kMiscMaxLen + 1, cnt64, c->ps.err);
    }
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, misc + kMiscMaxLen, 8, cudaMemcpyDeviceToHost, s));
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 2, cnt64, 8, cudaMemcpyDeviceToHost, s));
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + kPinnedErr, c->ps.err, sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, s));
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    if (device_error_status(c, s) != APO_OK) {
      set_error("match_candidates: empty pattern");
      return APO_EINVAL;
    }
    maxlen = c->host_pinned[0];
    extent = c->host_pinned[1];
    memcpy(&total, c->host_pinned + 2, 8);
  }
  // T positions and reach values live in 31 bits; dictionary slots below 2^31
  if (total + P >= 0x7fffffffull || extent >= (1ull << 30)) {
    set_error("match_candidates: at most 2^30 pattern source tokens and 2^31 - 1 pattern tokens "
              "plus patterns");
    return APO_EINVAL;
  }
  // source mode: the slices' source comes with its suffix and LCP arrays
  bool srcm = !pp->pat_off && pp->src_sa && pp->src_lcp;
  if (srcm && (pp->src_n < extent || pp->src_n >= 0xffffffffull)) {
    set_error("match_candidates: src_n does not cover the pattern slices");
    return APO_EINVAL;
  }
  if (srcm && maxlen >= 0xffff) srcm = false;  // the interval scans hold lengths in 16 bits
  const uint32_t src_n = srcm ? (uint32_t)pp->src_n : 0u;
  // Pass A's shape.  A chunk per lane in the first pass, about 64 per SM; a
  // repair pass moves exact states one group of chunks further (chunks of 32
  // positions and 256 lanes per SM on the 2^20-token window: first pass 0.28
  // -> about 0.1 ms, repairs 0.45 -> 0.79 ms).
  const uint64_t chunk = std::max<uint64_t>(64, std::min<uint64_t>(512, n / ((uint64_t)sms * 64)));
  const uint64_t nch = (n + chunk - 1) / chunk;
  // chunks per repair warp: longer groups settle in fewer passes, shorter
  // ones keep more warps busy on a short stream
  const uint32_t group = n >= (1ull << 22) ? 8u : 4u;
  const uint64_t nch2 = (nch + group - 1) / group;
  // The halo pass instead where states are deep: the patterns are slices of
  // the stream itself (each occurs at least at its own slice), they cover a
  // quarter of it or more, and the longest is longer than a chunk -- so the
  // chunked pass would be wrong over most covered positions -- but at most
  // four segments long (the halo's extra walk).  Segments of 128 to 1024
  // positions, about 24 warps per SM.
  uint64_t seg = 128;
  while (seg < 1024 && seg * 2 * 24 * (uint64_t)sms <= n) seg *= 2;
  const bool self_slices = !pp->pat_off && pp->tokens == stream;
  const bool halo = n && self_slices && 4 * total >= n && maxlen > chunk && maxlen <= 4 * seg;
  APO_TRY(c->arena.reserve(match_workspace_bytes(total, P, n, extent, maxlen, src_n)));
  const uint32_t N = (uint32_t)(total + P);  // pattern text with separators
  const uint32_t root = N;                   // node ids are T positions; the root is N
  const uint64_t tbl = pow2_at_least(2 * (P + 1));
  const uint64_t dct = pow2_at_least(2 * (extent + 1));
  const int levels = sa_levels(maxlen);
  const int nsparse = std::max(1, bits_for(P));

  Table g{c->arena.take_n<uint64_t>(2 * tbl), tbl - 1};
  Dict d{c->arena.take_n<uint64_t>(dct), dct - 1};
  uint32_t *pbuf = pp->pat_off ? c->arena.take_n<uint32_t>(2 * (size_t)P) : nullptr;
  uint32_t *tstart = c->arena.take_n<uint32_t>(P);
  uint32_t *tsym = c->arena.take_n<uint32_t>((size_t)N + kTsymPad);
  uint64_t *tkey = c->arena.take_n<uint64_t>(N);
  uint32_t *tpid = c->arena.take_n<uint32_t>(N);
  uint32_t *reach = c->arena.take_n<uint32_t>(N);
  // pattern-text suffix array (not in source mode)
  uint32_t *lcp = srcm ? nullptr : c->arena.take_n<uint32_t>(N);
  uint8_t *is_start = srcm ? nullptr : c->arena.take_n<uint8_t>(N);
  uint32_t *left = srcm ? nullptr : c->arena.take_n<uint32_t>(N);
  uint32_t *right = srcm ? nullptr : c->arena.take_n<uint32_t>(N);
  // source mode
  uint32_t *src_rank = srcm ? c->arena.take_n<uint32_t>(src_n) : nullptr;
  uint32_t *startlen = srcm ? c->arena.take_n<uint32_t>(src_n) : nullptr;
  uint32_t *fl = srcm ? c->arena.take_n<uint32_t>(src_n) : nullptr;
  uint32_t *mw = srcm ? c->arena.take_n<uint32_t>(src_n) : nullptr;
  uint32_t *fail = c->arena.take_n<uint32_t>((size_t)N + 1);
  uint32_t *own = c->arena.take_n<uint32_t>((size_t)N + 1);
  uint64_t *wj = c->arena.take_n<uint64_t>((size_t)N + 1);
  uint32_t *jl = c->arena.take_n<uint32_t>((size_t)N + 1);
  uint32_t *mtotal = c->arena.take_n<uint32_t>((size_t)N + 1);
  uint32_t *skip = c->arena.take_n<uint32_t>((size_t)N + 1);
  uint8_t *has_branch = c->arena.take_n<uint8_t>((size_t)N + 1);
  unsigned long long *pref = halo ? c->arena.take_n<unsigned long long>((size_t)N + 1) : nullptr;
  uint32_t *recidx = c->arena.take_n<uint32_t>((size_t)N + 1);
  uint32_t *firstrec = c->arena.take_n<uint32_t>((size_t)N + 1);
  uint4 *rec = c->arena.take_n<uint4>(P);
  uint32_t *sr = c->arena.take_n<uint32_t>(P);
  uint32_t *jpos = c->arena.take_n<uint32_t>(P);
  uint32_t *end_node = c->arena.take_n<uint32_t>(P);
  uint32_t *sparse = c->arena.take_n<uint32_t>((size_t)nsparse * P);
  SuffixState st;
  st.n = N;
  st.sa = srcm ? nullptr : c->arena.take_n<uint32_t>(N);
  st.rank = srcm ? nullptr : c->arena.take_n<uint32_t>(N);
  uint32_t *snap_base = srcm ? nullptr : c->arena.take_n<uint32_t>((size_t)levels * N);
  SortBuffers b, be;
  for (SortBuffers *x : {&b, &be}) {
    x->keys[0] = c->arena.take_n<uint64_t>(P);
    x->keys[1] = c->arena.take_n<uint64_t>(P);
    x->vals[0] = c->arena.take_n<uint32_t>(P);
    x->vals[1] = c->arena.take_n<uint32_t>(P);
  }
  const bool sa_mode_ok = srcm || (lcp && is_start && left && right && st.sa && st.rank && snap_base);
  const bool src_mode_ok = !srcm || (src_rank && startlen && fl && mw);
  if (!g.keys || !d.keys || (pp->pat_off && !pbuf) || !tstart || !tsym || !tkey || !tpid || !reach ||
      !sa_mode_ok || !src_mode_ok || !fail || !own || !wj || !jl || !mtotal || !skip || !has_branch || !recidx ||
      !firstrec || (halo && !pref) || !rec || !sr || !jpos || !end_node || !sparse || !b.keys[0] || !b.keys[1] || !b.vals[0] ||
      !b.vals[1] || !be.keys[0] || !be.keys[1] || !be.vals[0] || !be.vals[1]) {
    set_error("match: workspace too small");
    return APO_ENOMEM;
  }
  if (pp->pat_off) {  // CSR on the host -> (start, len) on the device
    std::vector<uint32_t> h(2 * (size_t)P);
    for (uint32_t p = 0; p < P; ++p) {
      h[p] = (uint32_t)pp->pat_off[p];
      h[P + p] = (uint32_t)(pp->pat_off[p + 1] - pp->pat_off[p]);
    }
    APO_CUDA_TRY(cudaMemcpyAsync(pbuf, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s));
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    pstart = pbuf;
    plen = pbuf + P;
  }

  // symbols: the dictionary of pattern tokens, the pattern text, the stream
  APO_CUDA_TRY(cudaMemsetAsync(d.keys, 0xff, dct * sizeof(uint64_t), s));
  uint32_t *ssym = c->arena.take_n<uint32_t>(std::max<uint64_t>(n, 1));
  if (!ssym) return APO_ENOMEM;
  APO_TRY(seg_scan<false>(c, SrcPlen{plen}, DstTstart{plen, tstart}, P, OpSum(), 0u, s));
  {
    Launch lp_(c, kKDictInsert, extent, s);
    if (tb == 4)
      k_dict_insert<<<grid_for(extent, 256, sms), 256, 0, s>>>(static_cast<const uint32_t *>(pp->tokens),
                                                                extent, d);
    else
      k_dict_insert<<<grid_for(extent, 256, sms), 256, 0, s>>>(static_cast<const uint64_t *>(pp->tokens),
                                                                extent, d);
  }
  {
    Launch lp_(c, kKPatLayout, N, s);
    const int blocks = std::max(1, std::min(ceil_div(P, 8), sms * 16));
    if (tb == 4)
      k_pat_layout<<<blocks, 256, 0, s>>>(static_cast<const uint32_t *>(pp->tokens), pstart, plen, tstart,
                                          P, N, d, tsym, tkey, tpid);
    else
      k_pat_layout<<<blocks, 256, 0, s>>>(static_cast<const uint64_t *>(pp->tokens), pstart, plen, tstart,
                                          P, N, d, tsym, tkey, tpid);
  }
  if (n) {
    Launch lp_(c, kKDictMap, n, s);
    if (tb == 4)
      k_dict_map<<<grid_for(n, 256, sms), 256, 0, s>>>(static_cast<const uint32_t *>(stream), n, d, ssym);
    else
      k_dict_map<<<grid_for(n, 256, sms), 256, 0, s>>>(static_cast<const uint64_t *>(stream), n, d, ssym);
  }
  APO_CUDA_TRY(cudaGetLastError());

  const uint32_t *sp = nullptr;
  const uint64_t *skey = nullptr;
  MinTree src_tree;
  const int lenbits = std::max(1, bits_for(maxlen));
  if (srcm) {
    // the patterns in string order by their LCP intervals in the source, the
    // start-to-start lcps, and M over the source positions
    const int g = grid_for(src_n, 256, sms);
    {
      Launch lp_(c, kKStarts, src_n, s);
      k_isa<<<g, 256, 0, s>>>(pp->src_sa, src_n, src_rank, c->ps.err);
    }
    APO_TRY(build_min_tree(c, pp->src_lcp, src_n, &src_tree, s));
    APO_CUDA_TRY(cudaMemsetAsync(startlen, 0, (size_t)src_n * 4, s));
    {
      Launch lp_(c, kKStarts, P, s);
      k_src_pat_keys<<<grid_for(P, 256, sms), 256, 0, s>>>(pstart, plen, P, src_rank, src_tree, lenbits,
                                                           b.keys[0], b.vals[0], startlen, c->ps.err);
    }
    b.cur = 0;
    {
      const DigitRange r{0, bits_for(src_n - 1) + lenbits, false};
      APO_TRY(radix_sort_pairs(c, b, P, &r, 1, s));
    }
    sp = b.vals[b.cur];
    skey = b.keys[b.cur];
    {
      Launch lp_(c, kKStarts, P, s);
      const int blocks = std::max(1, std::min(ceil_div(P, 8), sms * 16));
      if (tb == 4)
        k_src_slcp<<<blocks, 256, 0, s>>>(static_cast<const uint32_t *>(pp->tokens), pstart, plen, sp, P, sparse,
                                          jpos);
      else
        k_src_slcp<<<blocks, 256, 0, s>>>(static_cast<const uint64_t *>(pp->tokens), pstart, plen, sp, P, sparse,
                                          jpos);
    }
    const uint32_t capv = (uint32_t)maxlen;
    APO_TRY(seg_scan<false>(c, SrcFnLeft{pp->src_sa, pp->src_lcp, startlen, capv}, DstFnLeft{fl}, src_n,
                            OpClampCompose(), kClampId, s));
    APO_TRY(seg_scan<true>(c, SrcFnRight{pp->src_sa, pp->src_lcp, startlen, capv, src_n},
                           DstFnRight{pp->src_sa, fl, mw}, src_n, OpClampCompose(), kClampId, s));
    APO_TRY(seg_scan<false>(c, SrcReachSrc{tsym, tpid, tstart, plen, pstart, mw}, DstValue{reach}, N,
                            OpSegMax(), kSegMaxId, s));
  } else {
    // suffix array and LCP of the pattern text
    {
      uint32_t *snaps[64];
      for (int k = 0; k < levels; ++k) snaps[k] = snap_base + (size_t)k * N;
      st.snaps = snaps;
      uint32_t rounds = 0;
      APO_TRY(build_suffix_array(c, tkey, 8, N, st, levels, &rounds, s));
      APO_TRY(build_lcp(c, tkey, 8, st, lcp, s));
    }

    // pattern starts in suffix order
    {
      Launch lp_(c, kKStarts, P, s);
      k_start_keys<<<grid_for(P, 256, sms), 256, 0, s>>>(tstart, st.rank, P, b.keys[0], b.vals[0]);
    }
    b.cur = 0;
    {
      const DigitRange r{0, bits_for(N - 1), false};
      APO_TRY(radix_sort_pairs(c, b, P, &r, 1, s));
    }
    sp = b.vals[b.cur];
    APO_CUDA_TRY(cudaMemsetAsync(is_start, 0, N, s));
    {
      Launch lp_(c, kKStarts, P, s);
      k_start_mark<<<grid_for(P, 256, sms), 256, 0, s>>>(b.keys[b.cur], sp, P, sr, jpos, is_start);
    }
    // lcp with the nearest pattern start on each side in suffix order, the
    // start-to-start lcps, and the running maximum of the reach over T
    APO_TRY(seg_scan<false>(c, SrcLeft{lcp, is_start}, DstFlagged{left}, N, OpSegMin(), kSegMinId, s));
    {
      Launch lp_(c, kKStarts, P, s);
      k_slcp<<<grid_for(P, 256, sms), 256, 0, s>>>(sr, left, P, sparse);
    }
    APO_TRY(seg_scan<true>(c, SrcRight{lcp, is_start, N}, DstFlagged{right}, N, OpSegMin(), kSegMinId, s));
    APO_TRY(seg_scan<false>(c, SrcReach{tkey, st.rank, left, right, P}, DstValue{reach}, N, OpSegMax(),
                            kSegMaxId, s));
  }
  if (aux_order) APO_CUDA_TRY(cudaMemcpyAsync(aux_order, sp, (size_t)P * 4, cudaMemcpyDeviceToDevice, s));
  if (aux_slcp) APO_CUDA_TRY(cudaMemcpyAsync(aux_slcp, sparse, (size_t)P * 4, cudaMemcpyDeviceToDevice, s));
  Sparse S;
  S.nlev = nsparse;
  S.lev[0] = sparse;
  if (P <= kSparseOneBlock) {
    if (nsparse > 1) {
      Launch lp_(c, kKSparse, P, s);
      k_sparse_all<<<1, 1024, 0, s>>>(sparse, P, nsparse);
    }
    for (int l = 1; l < nsparse; ++l) S.lev[l] = sparse + (size_t)l * P;
  } else {
    for (int l = 1; l < nsparse; ++l) {
      uint32_t *lv = sparse + (size_t)l * P;
      Launch lp_(c, kKSparse, P, s);
      k_sparse_level<<<grid_for(P, 256, sms), 256, 0, s>>>(S.lev[l - 1], P, 1u << (l - 1), lv);
      S.lev[l] = lv;
    }
  }

  // nodes: failure links, branch edges, pattern ends
  {
    Launch lp_(c, kKTableInit, tbl, s);
    k_table_init<<<grid_for(tbl, 256, sms), 256, 0, s>>>(g.keys, tbl);
  }
  APO_CUDA_TRY(cudaMemsetAsync(own, 0, ((size_t)N + 1) * sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(has_branch, 0, (size_t)N + 1, s));
  if (pref) APO_CUDA_TRY(cudaMemsetAsync(pref, 0, ((size_t)N + 1) * sizeof(unsigned long long), s));
  {
    NodeArgs a;
    a.tstart = tstart;
    a.plen = plen;
    a.tsym = tsym;
    a.jpos = jpos;
    a.sp = sp;
    a.sr = sr;
    a.rank = st.rank;
    a.left = left;
    a.reach = reach;
    a.S = S;
    a.P = P;
    a.root = root;
    a.g = g;
    a.fail = fail;
    a.own = own;
    a.end_node = end_node;
    a.has_branch = has_branch;
    a.pref = pref;
    a.err = c->ps.err;
    a.src = srcm;
    a.pstart = pstart;
    a.src_rank = src_rank;
    a.skey = skey;
    a.T = src_tree;
    a.lenbits = lenbits;
    Launch lp_(c, kKAcNodes, N, s);
    if (pref)
      k_ac_nodes<true><<<std::max(1, std::min(ceil_div(P, 8), sms * 16)), 256, 0, s>>>(a);
    else
      k_ac_nodes<false><<<std::max(1, std::min(ceil_div(P, 8), sms * 16)), 256, 0, s>>>(a);
  }
  // pattern ids grouped by end node
  {
    Launch lp_(c, kKEndPairs, P, s);
    k_end_pairs<<<grid_for(P, 256, sms), 256, 0, s>>>(end_node, P, be.keys[0], be.vals[0]);
  }
  be.cur = 0;
  {
    const DigitRange r{0, bits_for(root), false};
    APO_TRY(radix_sort_pairs(c, be, P, &r, 1, s));
  }
  const uint64_t *ek = be.keys[be.cur];
  const uint32_t *ev = be.vals[be.cur];
  APO_TRY(seg_scan<false>(c, SrcRunStart{ek}, DstRecord{ek, own, recidx, rec, P, misc + kMiscTraceCount},
                          P, OpSum(), 0u, s));
  // match totals and output links
  {
    Launch lp_(c, kKAcJump, (uint64_t)N + 1, s);
    k_jump_init<<<grid_for((uint64_t)N + 1, 256, sms), 256, 0, s>>>(fail, own, N + 1, root, wj, jl, skip);
  }
  const int jumps = bits_for(maxlen) + 1;
  for (int r = 0; r < jumps; ++r) {
    Launch lp_(c, kKAcJump, (uint64_t)N + 1, s);
    k_ac_jump<<<grid_for((uint64_t)N + 1, 256, sms), 256, 0, s>>>(wj, jl, skip, own, tsym, has_branch, N + 1,
                                                                  root, r == jumps - 1, mtotal, recidx,
                                                                  firstrec, rec, c->ps.err);
  }
  APO_CUDA_TRY(cudaGetLastError());
  if (n == 0) return check_device_error(c, s);  // synchronises

  // record totals and flattened-chain offsets: they depend on the automaton
  // only, so they are queued now over the bound P >= records, and their
  // total is read with the match total below
  uint32_t *rtot = c->arena.take_n<uint32_t>(P), *flat_off = c->arena.take_n<uint32_t>(P);
  const bool flat_ok = rtot && flat_off;
  if (flat_ok) {
    {
      Launch lp_(c, kKMarkEnds, P, s);
      k_rec_totals<<<grid_for(P, 256, sms), 256, 0, s>>>(rec, mtotal, P, misc + kMiscTraceCount, rtot);
    }
    APO_TRY(seg_scan<false>(c, SrcU32{rtot}, DstExclusive{rtot, flat_off, misc + kMiscFlatTotal, P}, P, OpSum(),
                            0u, s));
  }

  // pass A: the state of every stream position (pass shape chosen above)
  Automaton A{tsym, has_branch, g, skip, root, {skip}, (uint32_t)(maxlen / 32 + 2), {}};
  uint32_t *state = c->arena.take_n<uint32_t>(n);
  uint32_t *off = c->arena.take_n<uint32_t>(n);
  if (!state || !off) return APO_ENOMEM;
  if (halo) {
    // lifting tables of the skip links and of the preferred children
    uint32_t *hc = c->arena.take_n<uint32_t>((size_t)N + 1);
    if (!hc) return APO_ENOMEM;
    {
      Launch lp_(c, kKAcJump, (uint64_t)N + 1, s);
      k_heavy_init<<<grid_for((uint64_t)N + 1, 256, sms), 256, 0, s>>>(tsym, pref, N, hc);
    }
    A.heavy[0] = hc;
    for (int k = 1; k < kLift; ++k) {
      uint32_t *t = c->arena.take_n<uint32_t>((size_t)N + 1), *h = c->arena.take_n<uint32_t>((size_t)N + 1);
      if (!t || !h) return APO_ENOMEM;
      Launch lp_(c, kKAcJump, 2 * ((uint64_t)N + 1), s);
      k_lift<<<grid_for((uint64_t)N + 1, 256, sms), 256, 0, s>>>(A.lift[k - 1], t, A.heavy[k - 1], h, N + 1);
      A.lift[k] = t;
      A.heavy[k] = h;
    }
    const uint64_t nseg = (n + seg - 1) / seg;
    Launch lp_(c, kKAcHalo, n, s);
    k_ac_halo<<<ceil_div(nseg, kStateWarps), 32 * kStateWarps, 0, s>>>(ssym, n, seg, maxlen, A, state,
                                                                        c->ps.err);
  } else {
    Launch lp_(c, kKAcStates, n, s);
    k_ac_states<<<ceil_div(nch, 64), 64, 0, s>>>(ssym, n, chunk, A, state);
  }
  // Repair passes two at a time: pass p counts its changes in word p & 1,
  // and a pass after one without changes returns at once, so the host reads
  // a count only after every second pass.
  uint32_t *chg = misc + kMiscFixChanged;
  for (uint64_t pass = 0; !halo && pass < nch2;) {
    const uint64_t last = std::min<uint64_t>(pass + 2, nch2);
    for (; pass < last; ++pass) {
      APO_CUDA_TRY(cudaMemsetAsync(chg + (pass & 1), 0, sizeof(uint32_t), s));
      Launch lp_(c, kKAcFix, n, s);
      k_ac_fix<<<ceil_div(nch2, kStateWarps), 32 * kStateWarps, 0, s>>>(
          ssym, n, chunk, group, A, state, pass ? chg + ((pass - 1) & 1) : nullptr, chg + (pass & 1));
    }
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, chg + ((pass - 1) & 1), 4, cudaMemcpyDeviceToHost, s));
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    if (c->host_pinned[0] == 0) break;
  }
  // output offsets and total
  const int tiles = ceil_div(n, kSTile);
  APO_TRY(ensure_lookback(c, tiles));
  APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscCompactTiles, 0, 2 * sizeof(uint32_t), s));
  {
    Launch lp_(c, kKMatchOffsets, n, s);
    k_match_offsets<<<tiles, kST, 0, s>>>(state, mtotal, (uint32_t)n, off, misc + kMiscCompactCount,
                                          c->ps.lookback, misc + kMiscCompactTiles, next_epoch(c),
                                          c->ps.err);
  }
  APO_CUDA_TRY(cudaGetLastError());
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, misc + kMiscCompactCount, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 1, misc + kMiscTraceCount, 4, cudaMemcpyDeviceToHost, s));
  if (flat_ok)
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 2, misc + kMiscFlatTotal, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + kPinnedErr, c->ps.err, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  APO_TRY(device_error_status(c, s));
  const uint64_t total_m = c->host_pinned[0];
  *count = total_m;
  if (total_m > cap) {
    set_error("match_candidates: more matches than cap (count written)");
    return APO_ECAPACITY;
  }
  if (total_m) {
    // flatten each output record's chain once (sum over records of their
    // chain lengths, usually far below the match count), then copy chains
    // per position; very long flattened chains fall back to walking
    const uint32_t R = c->host_pinned[1];
    const uint64_t flat_total = flat_ok && R ? c->host_pinned[2] : ~0ull;
    uint32_t *flat = nullptr;
    if (flat_total <= kMaxFlat) {
      APO_TRY(ensure_side(c, std::max<uint64_t>(flat_total, 1) * 4, s));
      flat = static_cast<uint32_t *>(c->side);
    }
    if (flat) {
      {
        Launch lp_(c, kKAcFill, flat_total, s);
        k_flat_chains<<<std::max(1, std::min(ceil_div(R, 8), sms * 16)), 256, 0, s>>>(rec, R, flat_off, ev, flat);
      }
      Launch lp_(c, kKAcFill, n, s);
      k_ac_fill_flat<<<std::max(1, std::min(ceil_div(n, 256), sms * 32)), 256, 0, s>>>(
          state, (uint32_t)n, off, firstrec, rtot, flat_off, flat, match_end, match_id, cap);
    } else {
      Launch lp_(c, kKAcFill, n, s);
      k_ac_fill<<<grid_for(n, 256, sms), 256, 0, s>>>(state, (uint32_t)n, off, firstrec, rec, ev, match_end,
                                                      match_id, cap);
    }
  }
  APO_CUDA_TRY(cudaGetLastError());
  return check_device_error(c, s);  // synchronises
}

}  // namespace apo
