// Trace replay over a whole stream -- Alg. 1 "TraceReplayer", Sec. 4.3.
//
// The replayer of the paper works task by task: the candidate traces sit in
// a trie that grows as analyses are ingested, every task starts a pointer at
// the root and moves the live pointers one edge down, a pointer standing at
// the end of a trace completes it, and when some trace completes the best
// one by score is replayed (it ends at the current task) and every pointer is
// dropped.  The score of a completed trace is its length times its
// appearance count (capped), decayed by the tasks since its previous
// appearance, raised when the trace was replayed before.
//
// Here the same decisions are computed for all tasks at once:
//
//  pieces      a trace longer than the maximum trace length enters as
//              consecutive pieces (Sec. 6.2); piece ids in input order.
//  occurrences every (end, piece) with stream[end - len + 1 .. end] equal to
//              the piece: the Aho-Corasick matcher of ac.cu, which also
//              returns the pieces in string order with neighbour lcps.
//  need(t)     a pointer started at task s survives to complete t iff for
//              every prefix t[:j], j < |t|, some piece starting with t[:j]
//              was ingested by task s + j - 1, and t itself by task
//              s + |t| - 1.  So the occurrence is followed iff
//              s >= need(t) = max(max_{j<|t|} B(t[:j]) - j + 1, E(t) - |t| + 1)
//              with B(u) the earliest ingestion of a piece starting with u and
//              E(t) that of t.  The pieces starting with t[:j] are an interval
//              of the string order (lcp >= j); the walk over the enclosing
//              intervals takes range minima of the ingestion times.
//  replay ends after a replay ending at x, the next one ends at the first
//              task e with a followed occurrence starting after x:
//              nxt(x) = min{e : PM(e) >= x + 2}, PM the running maximum of
//              (largest followed start ending at e) + 1.  The chain from
//              x = -1 is found by pointer doubling on nxt (tables J_k =
//              nxt^(2^k)), a short walk at the top level and a refinement
//              down the levels.  The chain does not depend on which trace is
//              chosen, since every chosen trace ends at the replay task.
//  appearances the followed occurrences ending at a replay task and
//              starting after the previous replay: the set D of that task.
//              Sorted by trace (stable), they give each appearance its count
//              and the task of the trace's previous appearance.
//  selection   a task's winner depends on flags "replayed before" only; a
//              task whose best candidate wins under every flag assignment is
//              decided at once.  The rest are solved as the fixed point of
//              "flags from the current winners, winners from the flags",
//              iterated in one block; the fixed point is unique (the first
//              task where two fixed points differ would see the same flags)
//              and each round fixes at least the first wrong task.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/apo.h"
#include "apo_internal.cuh"
#include "device_util.cuh"
#include "scan.cuh"

namespace apo {

namespace {

constexpr uint32_t kNone = 0xffffffffu;
constexpr int kSelectThreads = 1024;

#define RP_FOR(i, n) \
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (n); i += (uint64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- pieces
// Pieces per trace; flags an empty trace or one past the stream's end.
__global__ void k_piece_count(const uint32_t *__restrict__ start, const uint32_t *__restrict__ len, uint32_t P,
                              uint64_t n, uint32_t M, uint32_t *__restrict__ cnt, uint32_t *bad) {
  RP_FOR(q, P) {
    const uint32_t l = len[q];
    if (l == 0 || (uint64_t)start[q] + l > n) {
      atomicOr(bad, 1u);
      cnt[q] = 0;
    } else {
      cnt[q] = M ? (l - 1) / M + 1 : 1u;
    }
  }
}

struct SrcU32 {
  const uint32_t *v;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const { return v[k]; }
};
// exclusive offsets from the inclusive sum; the last element also writes the total
struct DstExclusive {
  const uint32_t *v;
  uint32_t *out;
  uint32_t n;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t s) const {
    out[k] = s - v[k];
    if (k == n - 1) out[n] = s;
  }
};
struct DstU32 {
  uint32_t *out;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t s) const { out[k] = s; }
};

__global__ void k_piece_write(const uint32_t *__restrict__ start, const uint32_t *__restrict__ len,
                              const uint32_t *__restrict__ ingest, uint32_t P, uint32_t M, uint32_t n,
                              const uint32_t *__restrict__ poff, uint32_t *__restrict__ pstart,
                              uint32_t *__restrict__ plen, uint32_t *__restrict__ ptau) {
  RP_FOR(q, P) {
    const uint32_t off = poff[q], k = poff[q + 1] - off, l = len[q], a = start[q];
    const uint32_t tau = min(ingest[q], n);  // at n or later: never in the trie
    for (uint32_t i = 0; i < k; ++i) {
      const uint32_t rest = l - i * M;
      pstart[off + i] = a + i * M;
      plen[off + i] = (M && rest > M) ? M : rest;
      ptau[off + i] = tau;
    }
  }
}

// ---------------------------------------------------------------- equal pieces
// Equal strings (the same trace found by several analyses) are matched once:
// pieces are sorted by a hash of their string, each piece is compared with
// the first piece of its hash run, and equal ones merge into it, keeping the
// smallest piece number and the earliest ingestion (all that need() and the
// reported trace number use).  A piece that differs from its run's first
// (a hash collision) stays on its own; equal strings left apart that way are
// still told apart later (k_need's runs).
__device__ __forceinline__ uint64_t mix_rp(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

template <class T>
__global__ void k_piece_hash(const T *__restrict__ tok, const uint32_t *__restrict__ pstart,
                             const uint32_t *__restrict__ plen, uint32_t Q, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ vals) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t q = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; q < Q; q += warps) {
    const uint32_t a = pstart[q], L = plen[q];
    uint64_t h = 0;
    for (uint32_t k = lane; k < L; k += 32) h += mix_rp((uint64_t)tok[a + k] * 0x9e3779b97f4a7c15ull + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if (lane == 0) {
      keys[q] = mix_rp(h ^ ((uint64_t)L << 40)) >> 24;  // 40 bits
      vals[q] = (uint32_t)q;
    }
  }
}

// One warp per sorted position: rep[piece] = the run's first piece if the
// strings are equal, else the piece itself; the representative keeps the
// smallest piece number and ingestion task of its members.
template <class T>
__global__ void k_piece_dups(const T *__restrict__ tok, const uint32_t *__restrict__ pstart,
                             const uint32_t *__restrict__ plen, const uint32_t *__restrict__ ptau,
                             const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, uint32_t Q,
                             uint32_t *__restrict__ rep, uint32_t *tau_min, uint32_t *pid_min) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t j = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; j < Q; j += warps) {
    const uint64_t key = keys[j];
    uint32_t lo = 0, hi = (uint32_t)j;  // the run's first position
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (keys[mid] < key) lo = mid + 1;
      else hi = mid;
    }
    const uint32_t a = vals[j], b = vals[lo];
    bool same = plen[a] == plen[b];
    if (same && a != b) {
      const uint32_t L = plen[a], sa = pstart[a], sb = pstart[b];
      for (uint32_t k0 = 0; k0 < L && same; k0 += 32) {
        const uint32_t k = k0 + lane;
        same = __all_sync(0xffffffffu, k >= L || tok[sa + k] == tok[sb + k]);
      }
    }
    if (lane == 0) {
      const uint32_t r = same ? b : a;
      rep[a] = r;
      atomicMin(&tau_min[r], ptau[a]);
      atomicMin(&pid_min[r], a);
    }
  }
}

struct SrcIsRep {
  const uint32_t *rep;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const { return rep[k] == k ? 1u : 0u; }
};
struct DstRepOffset {
  const uint32_t *rep;
  uint32_t *out;
  uint32_t n;
  __device__ __forceinline__ void operator()(uint32_t k, uint32_t s) const {
    out[k] = s - (rep[k] == k ? 1u : 0u);
    if (k == n - 1) out[n] = s;
  }
};

__global__ void k_unique_write(const uint32_t *__restrict__ rep, const uint32_t *__restrict__ uoff, uint32_t Q,
                               const uint32_t *__restrict__ pstart, const uint32_t *__restrict__ plen,
                               const uint32_t *__restrict__ tau_min, const uint32_t *__restrict__ pid_min,
                               uint32_t *__restrict__ ust, uint32_t *__restrict__ uln, uint32_t *__restrict__ uta,
                               uint32_t *__restrict__ upi) {
  RP_FOR(q, Q) {
    if (rep[q] != q) continue;
    const uint32_t i = uoff[q];
    ust[i] = pstart[q];
    uln[i] = plen[q];
    uta[i] = tau_min[q];
    upi[i] = pid_min[q];
  }
}

// ---------------------------------------------------------------- need(t)
// Sparse tables of minima over windows ending at j (clipped at 0): level 0
// is slcp (the lcp with the previous piece in string order) and the
// ingestion times in string order.
__global__ void k_tables0(const uint32_t *__restrict__ sp, const uint32_t *__restrict__ ptau, uint32_t Q,
                          uint32_t *__restrict__ tau_sorted) {
  RP_FOR(j, Q) tau_sorted[j] = ptau[sp[j]];
}

__global__ void k_tables_level(const uint32_t *__restrict__ la, const uint32_t *__restrict__ ta, uint32_t Q,
                               uint32_t half, uint32_t *__restrict__ lb, uint32_t *__restrict__ tb) {
  RP_FOR(j, Q) {
    uint32_t x = la[j], y = ta[j];
    if (j >= half) {
      x = min(x, la[j - half]);
      y = min(y, ta[j - half]);
    }
    lb[j] = x;
    tb[j] = y;
  }
}

// Level 0's ingestion times and every level above in one block (level l's
// arrays at lev + 2 (l - 1) Q), for a short table: one launch instead of one
// per level.
constexpr uint32_t kTablesOneBlock = 1u << 15;
__global__ void __launch_bounds__(1024) k_tables_all(const uint32_t *__restrict__ sp,
                                                     const uint32_t *__restrict__ ptau, const uint32_t *slcp,
                                                     uint32_t Q, int nlev, uint32_t *tau_sorted, uint32_t *lev) {
  for (uint32_t j = threadIdx.x; j < Q; j += blockDim.x) tau_sorted[j] = ptau[sp[j]];
  __syncthreads();
  const uint32_t *la = slcp, *ta = tau_sorted;
  for (int l = 1; l < nlev; ++l) {
    uint32_t *lb = lev + (size_t)(2 * (l - 1)) * Q, *tb = lb + Q;
    const uint32_t half = 1u << (l - 1);
    for (uint32_t j = threadIdx.x; j < Q; j += blockDim.x) {
      uint32_t x = la[j], y = ta[j];
      if (j >= half) {
        x = min(x, la[j - half]);
        y = min(y, ta[j - half]);
      }
      lb[j] = x;
      tb[j] = y;
    }
    __syncthreads();
    la = lb;
    ta = tb;
  }
}

struct Tables {
  const uint32_t *lcp[32];  // window minima of slcp, level l covers 2^l entries
  const uint32_t *tau[32];  // window minima of the ingestion times
  int nlev;
  uint32_t Q;
};

__device__ __forceinline__ int floor_log2(uint32_t v) { return 31 - __clz(v); }

// minimum ingestion time over string positions [a, b]
__device__ __forceinline__ uint32_t tau_min(const Tables &T, uint32_t a, uint32_t b) {
  const int l = floor_log2(b - a + 1);
  return min(T.tau[l][b], T.tau[l][a + (1u << l) - 1]);
}

// largest j <= lo with slcp[j] < d (d >= 1; slcp[0] = 0)
__device__ __forceinline__ uint32_t left_bound(const Tables &T, uint32_t lo, uint32_t d) {
  uint32_t j = lo;
  for (int l = T.nlev - 1; l >= 0; --l)
    if (T.lcp[l][j] >= d) j -= 1u << l;  // a clipped window holds slcp[0] = 0 < d
  return j;
}

// smallest j > hi with slcp[j] < d, or Q
__device__ __forceinline__ uint32_t right_bound(const Tables &T, uint32_t hi, uint32_t d) {
  uint32_t j = hi + 1;
  for (int l = T.nlev - 1; l >= 0; --l) {
    const uint64_t e = (uint64_t)j + (1u << l) - 1;
    if (e < T.Q && T.lcp[l][e] >= d) j += 1u << l;
  }
  return j;
}

// One thread per string position; the first position of each run of equal
// strings handles the run: its entry with the smallest piece number becomes
// the canonical one of every entry in it, and gets need().
__global__ void k_need(Tables T, const uint32_t *__restrict__ sp, const uint32_t *__restrict__ plen,
                       const uint32_t *__restrict__ upid, const uint32_t *__restrict__ tau_sorted,
                       uint32_t *__restrict__ canon, uint32_t *__restrict__ need) {
  const uint32_t Q = T.Q;
  const uint32_t *slcp = T.lcp[0];
  RP_FOR(h64, Q) {
    const uint32_t h = (uint32_t)h64;
    const uint32_t L = plen[sp[h]];
    if (h > 0 && plen[sp[h - 1]] == L && slcp[h] >= L) continue;  // not a run head
    uint32_t r = h, cmin = sp[h], tb = tau_sorted[h];
    while (r + 1 < Q && slcp[r + 1] >= L && plen[sp[r + 1]] == L) {
      ++r;
      if (upid[sp[r]] < upid[cmin]) cmin = sp[r];  // the entry with the smallest piece number
      tb = min(tb, tau_sorted[r]);
    }
    for (uint32_t j = h; j <= r; ++j) canon[sp[j]] = cmin;
    // the pointer completes t at task s + L - 1: s >= E(t) - L + 1
    long long best = (long long)tb - L + 1;
    // pieces that start with t: the run and the longer pieces after it
    uint32_t lo = h, hi = right_bound(T, r, L) - 1;
    uint32_t B = tau_min(T, lo, hi);
    uint32_t dcur = L;
    bool first = true;
    while (true) {
      const uint32_t dl = slcp[lo], dr = hi + 1 < Q ? slcp[hi + 1] : 0u;
      const uint32_t dn = max(dl, dr);  // the interval holds for depths dn+1 .. dcur
      const uint32_t jhi = first ? L - 1 : dcur;
      if (dn + 1 <= jhi) best = max(best, (long long)B - (long long)dn);  // at depth j = dn + 1
      if (dn == 0 || (long long)B <= best) break;  // deeper terms are below B
      const uint32_t nlo = left_bound(T, lo, dn), nhi = right_bound(T, hi, dn) - 1;
      if (nlo < lo) B = min(B, tau_min(T, nlo, lo - 1));
      if (nhi > hi) B = min(B, tau_min(T, hi + 1, nhi));
      lo = nlo;
      hi = nhi;
      dcur = dn;
      first = false;
    }
    need[cmin] = best < 0 ? 0u : (uint32_t)best;
  }
}

__device__ __forceinline__ bool followed(uint32_t e, uint32_t t, const uint32_t *canon, const uint32_t *need,
                                         const uint32_t *plen, uint32_t *start) {
  if (canon[t] != t) return false;
  const uint32_t s = e + 1 - plen[t];
  *start = s;
  return s >= need[t];
}

// ms1[e] = 1 + the largest start of a followed occurrence ending at e (0: none);
// first[e] = index of the first occurrence ending at e (occurrences come
// sorted by end; entries of tasks without one are not written).
__global__ void k_valid_ends(const uint32_t *__restrict__ oend, const uint32_t *__restrict__ oid, uint32_t O,
                             const uint32_t *__restrict__ canon, const uint32_t *__restrict__ need,
                             const uint32_t *__restrict__ plen, uint32_t *__restrict__ ms1,
                             uint32_t *__restrict__ first) {
  RP_FOR(i, O) {
    const uint32_t e = oend[i];
    if (i == 0 || oend[i - 1] != e) first[e] = (uint32_t)i;
    uint32_t s;
    if (followed(e, oid[i], canon, need, plen, &s)) atomicMax(&ms1[e], s + 1);
  }
}

// ---------------------------------------------------------------- replay ends
// Nodes i = x + 1 for x = -1 .. n-1, plus the end node n + 1.
// J0[i] = nxt(i - 1) + 1 = 1 + first e with pm[e] >= i + 1, or n + 1.
__global__ void k_jump0(const uint32_t *__restrict__ pm, uint32_t n, uint32_t *__restrict__ J) {
  RP_FOR(i64, (uint64_t)n + 2) {
    const uint32_t i = (uint32_t)i64;
    uint32_t r = n + 1;
    if (i <= n && n > 0 && pm[n - 1] >= i + 1) {
      uint32_t lo = 0, hi = n - 1;  // first e with pm[e] >= i + 1
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pm[mid] >= i + 1) hi = mid;
        else lo = mid + 1;
      }
      r = lo + 1;
    }
    J[i] = r;
  }
}

__global__ void k_jump_level(const uint32_t *__restrict__ Jp, uint32_t n, uint32_t *__restrict__ Jn) {
  RP_FOR(i, (uint64_t)n + 2) Jn[i] = Jp[Jp[i]];
}

// The chain from node 0 at stride 2^K, walked by one thread (each step moves
// at least 2^K nodes ahead, so at most (n + 1) / 2^K + 1 steps; K is chosen
// to keep that near 2^8).
__global__ void k_chain_top(const uint32_t *__restrict__ JK, uint32_t n, uint32_t *__restrict__ list,
                            uint32_t *__restrict__ len_out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t i = 0, cnt = 0;
  while (i <= n) {
    list[cnt++] = i;
    i = JK[i];
  }
  *len_out = cnt;
}

// Level k from level k + 1: between chain nodes 2^(k+1) steps apart lies the
// node J_k of the first one.
__global__ void k_chain_refine(const uint32_t *__restrict__ lin, const uint32_t *__restrict__ len_in,
                               const uint32_t *__restrict__ Jk, uint32_t n, uint32_t *__restrict__ lout,
                               uint32_t *__restrict__ len_out) {
  const uint32_t m = *len_in;
  RP_FOR(j, m) {
    const uint32_t v = lin[j], w = Jk[v];
    lout[2 * j] = v;
    if (w <= n) lout[2 * j + 1] = w;
    if (j == m - 1) *len_out = 2 * m - (w <= n ? 0u : 1u);
  }
}

// ---------------------------------------------------------------- appearances
// Replay r (0-based) ends at task chain[r + 1] - 1; the appearances are the
// followed occurrences ending there and starting at chain[r] or later (a
// replay task always has an occurrence, so first[] is written there).
template <bool kWrite>
__global__ void k_appear(const uint32_t *__restrict__ chain, uint32_t R, const uint32_t *__restrict__ first,
                         const uint32_t *__restrict__ oend,
                         const uint32_t *__restrict__ oid, uint32_t O, const uint32_t *__restrict__ canon,
                         const uint32_t *__restrict__ need, const uint32_t *__restrict__ plen,
                         uint32_t *__restrict__ acnt, const uint32_t *__restrict__ aoff,
                         uint32_t *__restrict__ app_t, uint32_t *__restrict__ app_r) {
  RP_FOR(r, R) {
    const uint32_t e = chain[r + 1] - 1, c = chain[r];
    uint32_t k = first[e], cnt = 0;
    uint32_t w = kWrite ? aoff[r] : 0u;
    for (; k < O && oend[k] == e; ++k) {
      uint32_t s;
      const uint32_t t = oid[k];
      if (!followed(e, t, canon, need, plen, &s) || s < c) continue;
      if (kWrite) {
        app_t[w] = t;
        app_r[w] = (uint32_t)r;
        ++w;
      } else {
        ++cnt;
      }
    }
    if (!kWrite) acnt[r] = cnt;
  }
}

__global__ void k_app_keys(const uint32_t *__restrict__ app_t, const uint32_t *__restrict__ n_dev,
                           uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  RP_FOR(a, *n_dev) {
    keys[a] = app_t[a];
    vals[a] = (uint32_t)a;
  }
}

struct ScoreParams {
  uint32_t cap, half_life, num, den;
};

__device__ __forceinline__ uint64_t score_of(uint64_t x, uint32_t sh, uint32_t mult) {
  return sh >= 64 ? 0ull : (x * mult) >> sh;
}

// After the stable sort by trace: the appearance at sorted position q is the
// (q - first position of its trace + 1)-th of its trace, and the one before
// it (if any) is its previous appearance.
__global__ void k_app_score(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                            const uint32_t *__restrict__ n_dev, const uint32_t *__restrict__ app_r,
                            const uint32_t *__restrict__ chain, const uint32_t *__restrict__ plen, ScoreParams p,
                            uint64_t *__restrict__ app_x, uint32_t *__restrict__ app_sh) {
  const uint32_t A = *n_dev;
  RP_FOR(q64, A) {
    const uint32_t q = (uint32_t)q64;
    const uint64_t t = keys[q];
    uint32_t lo = 0, hi = q;  // first position with key t
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (keys[mid] < t) lo = mid + 1;
      else hi = mid;
    }
    const uint32_t a = vals[q];
    const uint64_t count = (uint64_t)(q - lo) + 1;
    uint32_t sh = 0;
    if (q > lo && p.half_life) {
      const uint32_t e = chain[app_r[a] + 1] - 1, ep = chain[app_r[vals[q - 1]] + 1] - 1;
      sh = min((e - ep) / p.half_life, 64u);
    }
    const uint64_t c = (p.cap && count > p.cap) ? (uint64_t)p.cap : count;
    app_x[a] = (uint64_t)plen[t] * c;
    app_sh[a] = sh;
  }
}

// ---------------------------------------------------------------- selection
// A replay task is decided when its best candidate by the lower score (flags
// least favourable to it) beats every other candidate's higher score.
__global__ void k_decide(uint32_t R, const uint32_t *__restrict__ aoff, const uint32_t *__restrict__ app_t,
                         const uint64_t *__restrict__ app_x, const uint32_t *__restrict__ app_sh,
                         const uint32_t *__restrict__ plen, ScoreParams p, uint32_t *__restrict__ winner,
                         uint32_t *__restrict__ first_dec, uint32_t *__restrict__ und, uint32_t *ucnt) {
  const uint32_t mlo = min(p.num, p.den), mhi = max(p.num, p.den);
  RP_FOR(r, R) {
    const uint32_t a0 = aoff[r], a1 = aoff[r + 1];
    uint32_t w = kNone, wl = 0;
    uint64_t ws = 0;
    for (uint32_t a = a0; a < a1; ++a) {
      const uint32_t t = app_t[a], L = plen[t];
      const uint64_t s = score_of(app_x[a], app_sh[a], mlo);
      if (w == kNone || s > ws || (s == ws && L > wl)) {
        w = t;
        ws = s;
        wl = L;
      }
    }
    bool decided = true;
    for (uint32_t a = a0; a < a1 && decided; ++a) {
      const uint32_t t = app_t[a], L = plen[t];
      if (t == w) continue;
      const uint64_t s = score_of(app_x[a], app_sh[a], mhi);
      if (s > ws || (s == ws && L > wl)) decided = false;
    }
    if (w == kNone) {  // a replay task always has a candidate
      winner[r] = kNone;
      continue;
    }
    if (decided) {
      winner[r] = w;
      atomicMin(&first_dec[w], (uint32_t)r);
    } else {
      winner[r] = kNone;
      und[atomicAdd(ucnt, 1u)] = (uint32_t)r;
    }
  }
}

// The undecided tasks, in one block: round after round, every undecided task
// takes the winner under the flags of the previous round's winners
// ("replayed before r" = a decided or undecided task before r chose it),
// until a round changes nothing.  fu[t] = the earliest undecided task whose
// current winner is t.  At most U + 1 rounds are needed; the loop gives up
// (error word) after U + 2.
__global__ void __launch_bounds__(kSelectThreads)
    k_select(const uint32_t *__restrict__ und, const uint32_t *__restrict__ ucnt, const uint32_t *__restrict__ aoff,
             const uint32_t *__restrict__ app_t, const uint64_t *__restrict__ app_x,
             const uint32_t *__restrict__ app_sh, const uint32_t *__restrict__ plen,
             const uint32_t *__restrict__ first_dec, uint32_t *fu, uint32_t *wcur, uint32_t *wnew, ScoreParams p,
             uint32_t *__restrict__ winner, uint32_t *rounds_out, uint32_t *err) {
  const uint32_t U = *ucnt;
  const int tid = threadIdx.x;
  for (uint32_t i = tid; i < U; i += blockDim.x) wcur[i] = kNone;
  __syncthreads();
  uint32_t round = 0;
  while (true) {
    int changed = 0;
    for (uint32_t i = tid; i < U; i += blockDim.x) {
      const uint32_t r = und[i];
      uint32_t w = kNone, wl = 0;
      uint64_t ws = 0;
      for (uint32_t a = aoff[r]; a < aoff[r + 1]; ++a) {
        const uint32_t t = app_t[a], L = plen[t];
        const bool before = min(first_dec[t], fu[t]) < r;
        const uint64_t s = score_of(app_x[a], app_sh[a], before ? p.num : p.den);
        if (w == kNone || s > ws || (s == ws && L > wl)) {
          w = t;
          ws = s;
          wl = L;
        }
      }
      wnew[i] = w;
      if (w != wcur[i]) changed = 1;
    }
    ++round;
    if (!__syncthreads_or(changed)) break;
    if (round > U + 2) {
      if (tid == 0) atomicExch(err, kDevTimeout);
      break;
    }
    for (uint32_t i = tid; i < U; i += blockDim.x) {
      if (wcur[i] != kNone) fu[wcur[i]] = kNone;
      if (wnew[i] != kNone) fu[wnew[i]] = kNone;
    }
    __syncthreads();
    for (uint32_t i = tid; i < U; i += blockDim.x) {
      wcur[i] = wnew[i];
      if (wnew[i] != kNone) atomicMin(&fu[wnew[i]], und[i]);
    }
    __syncthreads();
  }
  for (uint32_t i = tid; i < U; i += blockDim.x) winner[und[i]] = wnew[i];
  if (tid == 0) *rounds_out = round;
}

// ---------------------------------------------------------------- outputs
// One warp per replay: the replay record, the traced tasks, the traced total.
__global__ void k_replay_out(uint32_t R, const uint32_t *__restrict__ chain, const uint32_t *__restrict__ winner,
                             const uint32_t *__restrict__ plen, const uint32_t *__restrict__ upid,
                             uint32_t *rep_end, uint32_t *rep_len,
                             uint32_t *rep_trace, uint64_t rcap, uint8_t *traced,
                             unsigned long long *traced_total, uint32_t *err) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; r < R; r += warps) {
    const uint32_t w = winner[r], e = chain[r + 1] - 1;
    if (w == kNone) {  // no winner: the selection gave up (error word set) or a task had no candidate
      if (lane == 0) atomicCAS(err, kDevOk, kDevRange);
      continue;
    }
    const uint32_t L = plen[w];
    if (lane == 0) {
      if (r < rcap) {
        rep_end[r] = e;
        rep_len[r] = L;
        rep_trace[r] = upid[w];
      }
      atomicAdd(traced_total, (unsigned long long)L);
    }
    if (traced)
      for (uint32_t j = lane; j < L; j += 32) traced[e + 1 - L + j] = 1;
  }
}

struct SrcU8 {
  const uint8_t *v;
  __device__ __forceinline__ uint32_t operator()(uint32_t k) const { return v[k]; }
};

// traced tasks among the `window` tasks ending at k (fewer at the start)
__global__ void k_curve(const uint32_t *__restrict__ pre, uint32_t n, uint32_t window, uint32_t *__restrict__ curve) {
  RP_FOR(k, n) curve[k] = pre[k] - (k >= window ? pre[k - window] : 0u);
}

#undef RP_FOR

// Grow-only buffers of the replayer: 0 = trace staging (sized by the traces),
// 1 = pieces and per-task arrays, 2 = occurrences and appearances.
int ensure_rp(apo_ctx *c, int which, size_t bytes, cudaStream_t s) {
  if (bytes <= c->rp_bytes[which]) return APO_OK;
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  if (c->rp[which]) cudaFree(c->rp[which]);
  c->rp[which] = nullptr;
  c->rp_bytes[which] = 0;
  const size_t want = std::max<size_t>(bytes + bytes / 4, (size_t)1 << 20);
  APO_CUDA_TRY(cudaMalloc(&c->rp[which], want));
  c->rp_bytes[which] = want;
  return APO_OK;
}

// Hands out 256-byte aligned pieces of a buffer; with base == nullptr it only
// adds up the size.
struct Carve {
  char *base;
  size_t used = 0;
  template <class T>
  T *take(size_t n) {
    T *r = base ? reinterpret_cast<T *>(base + used) : nullptr;
    used += (n * sizeof(T) + 255) & ~(size_t)255;
    return r;
  }
};

struct Ws1 {
  uint32_t *pstart, *plen, *ptau, *sp, *slcp, *tau_sorted, *lev, *canon, *need, *first_dec, *fu;
  uint64_t *hk0, *hk1;
  uint32_t *hv0, *hv1, *rep, *tmin, *pmin, *uoff, *ust, *uln, *uta, *upi;
  uint32_t *ms1, *pm, *first, *J, *la, *lb, *acnt, *aoff, *winner, *und, *wcur, *wnew, *pre, *small;
  uint8_t *traced;
};

Ws1 carve1(Carve &cv, uint64_t n, uint32_t Q, int nlev, int K) {
  Ws1 w;
  w.pstart = cv.take<uint32_t>(Q);
  w.plen = cv.take<uint32_t>(Q);
  w.ptau = cv.take<uint32_t>(Q);
  w.sp = cv.take<uint32_t>(Q);
  w.slcp = cv.take<uint32_t>(Q);
  w.tau_sorted = cv.take<uint32_t>(Q);
  w.lev = cv.take<uint32_t>(2 * (size_t)std::max(0, nlev - 1) * Q + 1);
  w.canon = cv.take<uint32_t>(Q);
  w.need = cv.take<uint32_t>(Q);
  w.first_dec = cv.take<uint32_t>(Q);
  w.fu = cv.take<uint32_t>(Q);
  w.hk0 = cv.take<uint64_t>(Q);
  w.hk1 = cv.take<uint64_t>(Q);
  w.hv0 = cv.take<uint32_t>(Q);
  w.hv1 = cv.take<uint32_t>(Q);
  w.rep = cv.take<uint32_t>(Q);
  w.tmin = cv.take<uint32_t>(Q);
  w.pmin = cv.take<uint32_t>(Q);
  w.uoff = cv.take<uint32_t>((size_t)Q + 1);
  w.ust = cv.take<uint32_t>(Q);
  w.uln = cv.take<uint32_t>(Q);
  w.uta = cv.take<uint32_t>(Q);
  w.upi = cv.take<uint32_t>(Q);
  w.ms1 = cv.take<uint32_t>(n + 1);
  w.pm = cv.take<uint32_t>(n + 1);
  w.first = cv.take<uint32_t>(n + 1);
  w.J = cv.take<uint32_t>((size_t)(K + 1) * (n + 2));
  w.la = cv.take<uint32_t>(n + 2);
  w.lb = cv.take<uint32_t>(n + 2);
  w.acnt = cv.take<uint32_t>(n + 2);
  w.aoff = cv.take<uint32_t>(n + 2);
  w.winner = cv.take<uint32_t>(n + 1);
  w.und = cv.take<uint32_t>(n + 1);
  w.wcur = cv.take<uint32_t>(n + 1);
  w.wnew = cv.take<uint32_t>(n + 1);
  w.pre = cv.take<uint32_t>(n + 1);
  w.traced = cv.take<uint8_t>(n + 1);
  w.small = cv.take<uint32_t>(64);
  return w;
}

struct Ws2 {
  uint32_t *oend, *oid, *app_t, *app_r, *vals0, *vals1, *app_sh;
  uint64_t *keys0, *keys1, *app_x;
};

Ws2 carve2(Carve &cv, uint64_t cap) {
  Ws2 w;
  w.oend = cv.take<uint32_t>(cap);
  w.oid = cv.take<uint32_t>(cap);
  w.app_t = cv.take<uint32_t>(cap);
  w.app_r = cv.take<uint32_t>(cap);
  w.vals0 = cv.take<uint32_t>(cap);
  w.vals1 = cv.take<uint32_t>(cap);
  w.app_sh = cv.take<uint32_t>(cap);
  w.keys0 = cv.take<uint64_t>(cap);
  w.keys1 = cv.take<uint64_t>(cap);
  w.app_x = cv.take<uint64_t>(cap);
  return w;
}

// small words of Ws1
enum : int { kSmLens = 0, kSmUcnt = 40, kSmRounds = 41, kSmBad = 42, kSmTraced = 44 /* u64 */ };

}  // namespace

int replay_stream(apo_ctx *c, const void *tokens, uint64_t n, int tb, const apo_replay_traces *tr,
                  const apo_replay_params *prm, apo_replay_out *out, cudaStream_t s) {
  uint64_t *counts = out->counts;
  for (int k = 0; k < 8; ++k) counts[k] = 0;
  const uint32_t P = (uint32_t)tr->n_traces;
  const uint32_t M = prm->max_trace_len;
  const int sms = c->num_sms;
  if (P == 0 || n == 0) {
    if (P > 0) {
      set_error("apo_replay: a trace is empty or runs past the stream");
      return APO_EINVAL;
    }
    if (out->traced && n) APO_CUDA_TRY(cudaMemsetAsync(out->traced, 0, n, s));
    if (out->curve && n) APO_CUDA_TRY(cudaMemsetAsync(out->curve, 0, n * 4, s));
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    return APO_OK;
  }
  const uint32_t nn = (uint32_t)n;
  // pieces
  APO_TRY(ensure_rp(c, 0, ((size_t)2 * P + 8) * 4 + 512, s));
  uint32_t *cnt = static_cast<uint32_t *>(c->rp[0]);
  uint32_t *poff = cnt + P;
  uint32_t *bad = poff + P + 1;
  APO_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, s));
  {
    Launch lp_(c, kKRpPieces, P, s);
    k_piece_count<<<grid_for(P, 256, sms), 256, 0, s>>>(tr->start, tr->len, P, n, M, cnt, bad);
  }
  APO_TRY(seg_scan<false>(c, SrcU32{cnt}, DstExclusive{cnt, poff, P}, P, OpSum(), 0u, s));
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, poff + P, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 1, bad, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + kPinnedErr, c->ps.err, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  APO_TRY(device_error_status(c, s));
  if (c->host_pinned[1]) {
    set_error("apo_replay: a trace is empty or runs past the stream");
    return APO_EINVAL;
  }
  const uint32_t Q = c->host_pinned[0];
  counts[2] = Q;
  if (Q >= 0x7fffffffu) {
    set_error("apo_replay: more than 2^31 - 1 pieces");
    return APO_EINVAL;
  }
  const int nlev = std::max(1, bits_for(Q));
  const int K = std::max(0, bits_for(n + 1) - 8);  // the top-level walk takes at most ~2^8 steps
  Carve sz{nullptr};
  carve1(sz, n, Q, nlev, K);
  APO_TRY(ensure_rp(c, 1, sz.used, s));
  Carve cv1{static_cast<char *>(c->rp[1])};
  const Ws1 w = carve1(cv1, n, Q, nlev, K);
  {
    Launch lp_(c, kKRpPieces, P, s);
    k_piece_write<<<grid_for(P, 256, sms), 256, 0, s>>>(tr->start, tr->len, tr->ingest, P, M, nn, poff, w.pstart,
                                                        w.plen, w.ptau);
  }
  APO_CUDA_TRY(cudaGetLastError());

  // one entry per distinct string
  {
    const int hb = grid_for((uint64_t)Q * 32, 256, sms);
    Launch lp_(c, kKRpPieces, Q, s);
    if (tb == 4)
      k_piece_hash<<<hb, 256, 0, s>>>(static_cast<const uint32_t *>(tokens), w.pstart, w.plen, Q, w.hk0, w.hv0);
    else
      k_piece_hash<<<hb, 256, 0, s>>>(static_cast<const uint64_t *>(tokens), w.pstart, w.plen, Q, w.hk0, w.hv0);
  }
  SortBuffers hb;
  hb.keys[0] = w.hk0;
  hb.keys[1] = w.hk1;
  hb.vals[0] = w.hv0;
  hb.vals[1] = w.hv1;
  hb.cur = 0;
  {
    const DigitRange hr{0, 40, false};
    APO_TRY(radix_sort_pairs(c, hb, Q, &hr, 1, s));
  }
  APO_CUDA_TRY(cudaMemsetAsync(w.tmin, 0xff, (size_t)Q * 4, s));
  APO_CUDA_TRY(cudaMemsetAsync(w.pmin, 0xff, (size_t)Q * 4, s));
  {
    const int db = grid_for((uint64_t)Q * 32, 256, sms);
    Launch lp_(c, kKRpPieces, Q, s);
    if (tb == 4)
      k_piece_dups<<<db, 256, 0, s>>>(static_cast<const uint32_t *>(tokens), w.pstart, w.plen, w.ptau,
                                      hb.keys[hb.cur], hb.vals[hb.cur], Q, w.rep, w.tmin, w.pmin);
    else
      k_piece_dups<<<db, 256, 0, s>>>(static_cast<const uint64_t *>(tokens), w.pstart, w.plen, w.ptau,
                                      hb.keys[hb.cur], hb.vals[hb.cur], Q, w.rep, w.tmin, w.pmin);
  }
  APO_TRY(seg_scan<false>(c, SrcIsRep{w.rep}, DstRepOffset{w.rep, w.uoff, Q}, Q, OpSum(), 0u, s));
  {
    Launch lp_(c, kKRpPieces, Q, s);
    k_unique_write<<<grid_for(Q, 256, sms), 256, 0, s>>>(w.rep, w.uoff, Q, w.pstart, w.plen, w.tmin, w.pmin, w.ust,
                                                         w.uln, w.uta, w.upi);
  }
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, w.uoff + Q, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  const uint32_t Qd = c->host_pinned[0];  // distinct strings (entries from here on)
  const uint32_t *plen = w.uln, *ptau = w.uta, *upid = w.upi;
  const int nlevd = std::max(1, bits_for(Qd));

  // occurrences of the entries, and the entries in string order
  apo_patterns pp;
  memset(&pp, 0, sizeof(pp));
  pp.n_patterns = Qd;
  pp.tokens = tokens;
  pp.token_bytes = tb;
  pp.pat_start = w.ust;
  pp.pat_len = w.uln;
  uint64_t cap = std::max<uint64_t>(c->rp_cap, std::max<uint64_t>(1 << 20, n));
  uint64_t O = 0;
  Ws2 v;
  for (int attempt = 0; attempt < 2; ++attempt) {
    Carve sz2{nullptr};
    carve2(sz2, cap);
    APO_TRY(ensure_rp(c, 2, sz2.used, s));
    c->rp_cap = std::max(c->rp_cap, cap);
    Carve cv2{static_cast<char *>(c->rp[2])};
    v = carve2(cv2, cap);
    const int r = match_patterns(c, &pp, tokens, n, v.oend, v.oid, cap, &O, s, w.sp, w.slcp);
    if (r == APO_ECAPACITY && attempt == 0) {
      cap = O;
      continue;
    }
    APO_TRY(r);
    break;
  }
  counts[3] = O;
  if (O >= 0x7fffffffull) {
    set_error("apo_replay: more than 2^31 - 1 occurrences");
    return APO_EINVAL;
  }
  const uint32_t O32 = (uint32_t)O;

  // need(t) and canonical piece ids
  Tables T;
  T.nlev = nlevd;
  T.Q = Qd;
  T.lcp[0] = w.slcp;
  T.tau[0] = w.tau_sorted;
  if (Qd <= kTablesOneBlock) {
    {
      Launch lp_(c, kKRpNeed, Qd, s);
      k_tables_all<<<1, 1024, 0, s>>>(w.sp, ptau, w.slcp, Qd, nlevd, w.tau_sorted, w.lev);
    }
    for (int l = 1; l < nlevd; ++l) {
      T.lcp[l] = w.lev + (size_t)(2 * (l - 1)) * Qd;
      T.tau[l] = T.lcp[l] + Qd;
    }
  } else {
    {
      Launch lp_(c, kKRpNeed, Qd, s);
      k_tables0<<<grid_for(Qd, 256, sms), 256, 0, s>>>(w.sp, ptau, Qd, w.tau_sorted);
    }
    for (int l = 1; l < nlevd; ++l) {
      uint32_t *lb = w.lev + (size_t)(2 * (l - 1)) * Qd, *tbv = lb + Qd;
      Launch lp_(c, kKRpNeed, Qd, s);
      k_tables_level<<<grid_for(Qd, 256, sms), 256, 0, s>>>(T.lcp[l - 1], T.tau[l - 1], Qd, 1u << (l - 1), lb,
                                                               tbv);
      T.lcp[l] = lb;
      T.tau[l] = tbv;
    }
  }
  {
    Launch lp_(c, kKRpNeed, Qd, s);
    k_need<<<grid_for(Qd, 128, sms), 128, 0, s>>>(T, w.sp, plen, upid, w.tau_sorted, w.canon, w.need);
  }

  // replay ends
  APO_CUDA_TRY(cudaMemsetAsync(w.ms1, 0, n * 4, s));
  if (O32) {
    Launch lp_(c, kKRpChain, O32, s);
    k_valid_ends<<<grid_for(O32, 256, sms), 256, 0, s>>>(v.oend, v.oid, O32, w.canon, w.need, plen, w.ms1,
                                                         w.first);
  }
  APO_TRY(seg_scan<false>(c, SrcU32{w.ms1}, DstU32{w.pm}, nn, OpMax(), 0u, s));
  {
    Launch lp_(c, kKRpChain, n + 2, s);
    k_jump0<<<grid_for(n + 2, 256, sms), 256, 0, s>>>(w.pm, nn, w.J);
  }
  for (int k = 1; k <= K; ++k) {
    Launch lp_(c, kKRpChain, n + 2, s);
    k_jump_level<<<grid_for(n + 2, 256, sms), 256, 0, s>>>(w.J + (size_t)(k - 1) * (n + 2), nn,
                                                            w.J + (size_t)k * (n + 2));
  }
  uint32_t *lens = w.small + kSmLens;
  uint32_t *lin = (K % 2 == 0) ? w.la : w.lb, *lout = (K % 2 == 0) ? w.lb : w.la;
  {
    Launch lp_(c, kKRpChain, 1, s);
    k_chain_top<<<1, 32, 0, s>>>(w.J + (size_t)K * (n + 2), nn, lin, lens + K);
  }
  for (int k = K - 1; k >= 0; --k) {
    const uint64_t ub = std::min<uint64_t>(n + 2, ((n + 1) >> (k + 1)) + (1ull << (K - k - 1)) + 1);
    Launch lp_(c, kKRpChain, ub, s);
    k_chain_refine<<<grid_for(ub, 256, sms), 256, 0, s>>>(lin, lens + k + 1, w.J + (size_t)k * (n + 2), nn, lout,
                                                           lens + k);
    std::swap(lin, lout);
  }
  const uint32_t *chain = lin;  // node 0, then 1 + the end task of each replay
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, lens, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  const uint32_t R = c->host_pinned[0] - 1;
  counts[0] = R;
  counts[7] = (uint64_t)K;

  uint8_t *traced = out->traced ? out->traced : (out->curve ? w.traced : nullptr);
  if (traced) APO_CUDA_TRY(cudaMemsetAsync(traced, 0, n, s));
  unsigned long long *traced_total = reinterpret_cast<unsigned long long *>(w.small + kSmTraced);
  APO_CUDA_TRY(cudaMemsetAsync(w.small + kSmUcnt, 0, 8 * 4, s));
  if (R > 0) {
    const ScoreParams sp{prm->count_cap, prm->half_life, prm->bonus_num, prm->bonus_den};
    // appearances: the set D of each replay task
    {
      Launch lp_(c, kKRpAppear, R, s);
      k_appear<false><<<grid_for(R, 128, sms), 128, 0, s>>>(chain, R, w.first, v.oend, v.oid, O32, w.canon, w.need,
                                                            plen,
                                                            w.acnt, nullptr, nullptr, nullptr);
    }
    APO_TRY(seg_scan<false>(c, SrcU32{w.acnt}, DstExclusive{w.acnt, w.aoff, R}, R, OpSum(), 0u, s));
    {
      Launch lp_(c, kKRpAppear, R, s);
      k_appear<true><<<grid_for(R, 128, sms), 128, 0, s>>>(chain, R, w.first, v.oend, v.oid, O32, w.canon, w.need,
                                                           plen,
                                                           nullptr, w.aoff, v.app_t, v.app_r);
    }
    // count and previous appearance per trace: stable sort by trace
    const uint32_t *A_dev = w.aoff + R;
    {
      Launch lp_(c, kKRpAppear, O32, s);
      k_app_keys<<<grid_for(O32, 256, sms), 256, 0, s>>>(v.app_t, A_dev, v.keys0, v.vals0);
    }
    SortBuffers b;
    b.keys[0] = v.keys0;
    b.keys[1] = v.keys1;
    b.vals[0] = v.vals0;
    b.vals[1] = v.vals1;
    b.cur = 0;
    const DigitRange rg{0, std::max(1, bits_for(Qd - 1)), false};
    APO_TRY(radix_sort_pairs(c, b, O32, &rg, 1, s, A_dev));
    {
      Launch lp_(c, kKRpAppear, O32, s);
      k_app_score<<<grid_for(O32, 256, sms), 256, 0, s>>>(b.keys[b.cur], b.vals[b.cur], A_dev, v.app_r, chain,
                                                          plen, sp, v.app_x, v.app_sh);
    }
    // selection
    APO_CUDA_TRY(cudaMemsetAsync(w.first_dec, 0xff, (size_t)Qd * 4, s));
    APO_CUDA_TRY(cudaMemsetAsync(w.fu, 0xff, (size_t)Qd * 4, s));
    {
      Launch lp_(c, kKRpSelect, R, s);
      k_decide<<<grid_for(R, 128, sms), 128, 0, s>>>(R, w.aoff, v.app_t, v.app_x, v.app_sh, plen, sp, w.winner,
                                                     w.first_dec, w.und, w.small + kSmUcnt);
    }
    {
      Launch lp_(c, kKRpSelect, R, s);
      k_select<<<1, kSelectThreads, 0, s>>>(w.und, w.small + kSmUcnt, w.aoff, v.app_t, v.app_x, v.app_sh, plen,
                                            w.first_dec, w.fu, w.wcur, w.wnew, sp, w.winner, w.small + kSmRounds,
                                            c->ps.err);
    }
    {
      Launch lp_(c, kKRpOut, R, s);
      k_replay_out<<<grid_for((uint64_t)R * 32, 256, sms), 256, 0, s>>>(R, chain, w.winner, plen, upid, out->rep_end,
                                                                        out->rep_len, out->rep_trace, out->rep_cap,
                                                                        traced, traced_total, c->ps.err);
    }
  }
  if (out->curve) {
    APO_TRY(seg_scan<false>(c, SrcU8{traced}, DstU32{w.pre}, nn, OpSum(), 0u, s));
    Launch lp_(c, kKRpOut, n, s);
    k_curve<<<grid_for(n, 256, sms), 256, 0, s>>>(w.pre, nn, prm->window ? prm->window : nn, out->curve);
  }
  APO_CUDA_TRY(cudaGetLastError());
  // counts
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, w.small + kSmUcnt, 2 * 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 2, traced_total, 8, cudaMemcpyDeviceToHost, s));
  if (R > 0) APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + 4, w.aoff + R, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + kPinnedErr, c->ps.err, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  APO_TRY(device_error_status(c, s));
  uint64_t tt;
  memcpy(&tt, c->host_pinned + 2, 8);
  counts[1] = tt;
  counts[4] = R > 0 ? c->host_pinned[4] : 0;
  counts[5] = c->host_pinned[0];
  counts[6] = c->host_pinned[1];
  if (R > out->rep_cap) {
    set_error("apo_replay: more replays than rep_cap");
    return APO_ECAPACITY;
  }
  return APO_OK;
}

}  // namespace apo
