// Oracle for the trace finder's string analysis -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, sequential CPU restatement of what the hot path computes,
// used by the test-suite, the smoke check and the CPU-baseline leg of the
// benchmark to check the CUDA library.  Nothing in the library may call it.
// Every routine states the definition or the published step it follows.
// Tokens are handled as unsigned 64-bit integers (u32 tokens are widened,
// which keeps their order).
//
//   ora_fnv1a64 / ora_hash_tasks   Alg. 1 "Hash(T)", Sec. 4.1: a task and its
//                                  ordered region arguments -> one token.
//   ora_suffix_array               Alg. 2 "SuffixArray(S)": suffixes sorted by
//                                  direct lexicographic comparison.
//   ora_suffix_array_doubling      the same array by Manber-Myers prefix
//                                  doubling with a comparison sort (for inputs
//                                  whose long repeats make direct comparison slow).
//   ora_lcp_direct / ora_lcp_kasai LCP of adjacent SA entries: by direct scan,
//                                  and by Kasai et al. (CPM 2001).
//   ora_find_repeats               Alg. 2 "FindRepeats": candidate loop, sort by
//                                  (length desc, sub-string asc, start asc),
//                                  greedy non-overlapping selection, dedup;
//                                  sub-strings compared token by token or, for
//                                  long windows, by LCE queries (range minima
//                                  of the LCP array).
//   ora_match                      every occurrence of every candidate trace in
//                                  a stream (Sec. 4.3: a pointer that reaches the
//                                  end of a trace in the trie is a match).
//   ora_replay                     Alg. 1 "TraceReplayer" (Sec. 4.3) task by
//                                  task: a growing trie, pointers advanced per
//                                  task, completed candidates scored, the best
//                                  one replayed.
//   ora_optimum                    the optimisation problem of Sec. 3 (with
//                                  every trace repeated) by exhaustive
//                                  enumeration of the interval sets.
//
// Parity notes (readings where the paper is silent):
//   * a suffix that is a proper prefix of another sorts first;
//   * LCP[i] pairs SA[i] with SA[i+1] (Alg. 2 indexes it that way), LCP[n-1] = 0;
//   * (p + d) / 2 is integer division; the "symmetric" case swaps so that
//     s1 = min(SA[i], SA[i+1]);
//   * [s1, s1+p) and [s2, s2+p) are disjoint iff |s1 - s2| >= p;
//   * a candidate is kept iff its length >= min_len;
//   * identical (length, start) candidates are kept once;
//   * the task hash is FNV-1a 64 over task_id:u32, nargs:u32, then per
//     argument region:u32, field_mask:u64, priv:u8, all little-endian.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <set>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

const uint64_t kFnvOffset = 0xcbf29ce484222325ULL;  // FNV-1a 64 offset basis
const uint64_t kFnvPrime = 0x100000001b3ULL;        // FNV 64-bit prime

void put_le(std::vector<uint8_t> &b, uint64_t v, int bytes) {
  for (int k = 0; k < bytes; ++k) b.push_back((uint8_t)(v >> (8 * k)));
}

// Lexicographic order of suffixes S[a..n) and S[b..n); a proper prefix is smaller.
bool suffix_less(const uint64_t *S, uint64_t n, uint64_t a, uint64_t b) {
  while (a < n && b < n) {
    if (S[a] != S[b]) return S[a] < S[b];
    ++a;
    ++b;
  }
  return a == n && b != n;
}

// Compare S[a..a+l) with S[b..b+l) (both in bounds): <0, 0, >0.
int substr_cmp(const uint64_t *S, uint64_t a, uint64_t b, uint64_t l) {
  for (uint64_t k = 0; k < l; ++k) {
    if (S[a + k] != S[b + k]) return S[a + k] < S[b + k] ? -1 : 1;
  }
  return 0;
}

// Is the length-l prefix of suffix j lexicographically smaller than S[r..r+l)?
// A suffix shorter than l that matches as far as it goes is smaller.
bool prefix_less(const uint64_t *S, uint64_t n, uint64_t j, uint64_t r, uint64_t l) {
  for (uint64_t k = 0; k < l; ++k) {
    if (j + k >= n) return true;
    if (S[j + k] != S[r + k]) return S[j + k] < S[r + k];
  }
  return false;
}

struct Cand {
  uint64_t l, s;
};

// Longest common extension of two suffixes from the LCP array: the LCP of
// suffixes a and b is the minimum of LCP over the SA positions between them
// (a range-minimum query), answered by a sparse table of minima over
// power-of-two ranges (Bender & Farach-Colton 2000, the O(n log n) table).
struct Lce {
  uint64_t n = 0;
  std::vector<uint32_t> isa;
  std::vector<std::vector<uint32_t>> tab;  // tab[k][i] = min LCP[i .. i + 2^k)
  Lce(const uint32_t *sa, const uint32_t *lcp, uint64_t n_) : n(n_), isa(n_) {
    for (uint64_t k = 0; k < n; ++k) isa[sa[k]] = (uint32_t)k;
    tab.emplace_back(lcp, lcp + n);
    for (uint64_t w = 1; 2 * w <= n; w *= 2) {
      const std::vector<uint32_t> &prev = tab.back();
      std::vector<uint32_t> next(n - 2 * w + 1);
      for (uint64_t i = 0; i + 2 * w <= n; ++i) next[i] = std::min(prev[i], prev[i + w]);
      tab.push_back(std::move(next));
    }
  }
  // lcp of the suffixes starting at a and b
  uint64_t operator()(uint64_t a, uint64_t b) const {
    if (a == b) return n - a;
    uint64_t x = isa[a], y = isa[b];
    if (x > y) std::swap(x, y);
    // min LCP[x .. y - 1]: LCP[k] pairs SA[k] with SA[k + 1]
    uint64_t len = y - x, k = 0;
    while ((2ull << k) <= len) ++k;
    return std::min(tab[k][x], tab[k][y - (1ull << k)]);
  }
};

// substr_cmp and prefix_less through LCE queries instead of token loops.
int substr_cmp_lce(const uint64_t *S, const Lce &E, uint64_t a, uint64_t b, uint64_t l) {
  const uint64_t e = E(a, b);
  if (e >= l) return 0;
  return S[a + e] < S[b + e] ? -1 : 1;
}

bool prefix_less_lce(const uint64_t *S, uint64_t n, const Lce &E, uint64_t j, uint64_t r, uint64_t l) {
  const uint64_t e = E(j, r);
  if (e >= l) return false;
  if (j + e >= n) return true;  // suffix j ends first: a proper prefix is smaller
  return S[j + e] < S[r + e];
}

}  // namespace

extern "C" {

uint64_t ora_fnv1a64(const uint8_t *p, uint64_t n) {
  uint64_t h = kFnvOffset;
  for (uint64_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= kFnvPrime;
  }
  return h;
}

// Canonical byte string of one task (Sec. 2: a task id and its ordered region
// arguments; the region, the fields it touches and the privilege all matter).
uint64_t ora_serialize_task(uint64_t t, const uint32_t *task_id, const uint32_t *arg_off,
                            const uint32_t *region, const uint64_t *field_mask,
                            const uint8_t *priv, uint8_t *out, uint64_t cap) {
  std::vector<uint8_t> b;
  put_le(b, task_id[t], 4);
  uint32_t lo = arg_off[t], hi = arg_off[t + 1];
  put_le(b, hi - lo, 4);
  for (uint32_t a = lo; a < hi; ++a) {
    put_le(b, region[a], 4);
    put_le(b, field_mask[a], 8);
    put_le(b, priv[a], 1);
  }
  if (out && cap >= b.size()) memcpy(out, b.data(), b.size());
  return b.size();
}

void ora_hash_tasks(uint64_t N, const uint32_t *task_id, const uint32_t *arg_off,
                    const uint32_t *region, const uint64_t *field_mask, const uint8_t *priv,
                    uint64_t *out) {
  std::vector<uint8_t> b;
  for (uint64_t t = 0; t < N; ++t) {
    uint64_t len = ora_serialize_task(t, task_id, arg_off, region, field_mask, priv, nullptr, 0);
    b.resize(len);
    ora_serialize_task(t, task_id, arg_off, region, field_mask, priv, b.data(), len);
    out[t] = ora_fnv1a64(b.data(), len);
  }
}

// Alg. 2 SuffixArray(S): the start positions sorted by their suffixes.
void ora_suffix_array(const uint64_t *S, uint64_t n, uint32_t *sa) {
  std::vector<uint32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0u);
  std::sort(idx.begin(), idx.end(),
            [&](uint32_t a, uint32_t b) { return suffix_less(S, n, a, b); });
  std::copy(idx.begin(), idx.end(), sa);
}

// Manber & Myers (1993) prefix doubling with a comparison sort: after the
// round with step h the ranks order the suffixes by their first 2h tokens.
void ora_suffix_array_doubling(const uint64_t *S, uint64_t n, uint32_t *sa) {
  if (n == 0) return;
  std::vector<uint32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0u);
  std::sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
    return S[a] != S[b] ? S[a] < S[b] : a < b;
  });
  std::vector<uint64_t> rank(n), tmp(n);
  uint64_t r = 1;
  for (uint64_t k = 0; k < n; ++k) {
    if (k > 0 && S[idx[k]] != S[idx[k - 1]]) ++r;
    rank[idx[k]] = r;
  }
  for (uint64_t h = 1; r < n; h *= 2) {
    auto key2 = [&](uint32_t i) -> uint64_t { return i + h < n ? rank[i + h] : 0; };
    std::sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
      if (rank[a] != rank[b]) return rank[a] < rank[b];
      if (key2(a) != key2(b)) return key2(a) < key2(b);
      return a < b;
    });
    r = 1;
    for (uint64_t k = 0; k < n; ++k) {
      if (k > 0 && (rank[idx[k]] != rank[idx[k - 1]] || key2(idx[k]) != key2(idx[k - 1]))) ++r;
      tmp[idx[k]] = r;
    }
    rank.swap(tmp);
  }
  std::copy(idx.begin(), idx.end(), sa);
}

// LCP[i] = length of the longest common prefix of suffixes SA[i] and SA[i+1].
void ora_lcp_direct(const uint64_t *S, uint64_t n, const uint32_t *sa, uint32_t *lcp) {
  for (uint64_t i = 0; i + 1 < n; ++i) {
    uint64_t a = sa[i], b = sa[i + 1], k = 0;
    while (a + k < n && b + k < n && S[a + k] == S[b + k]) ++k;
    lcp[i] = (uint32_t)k;
  }
  if (n) lcp[n - 1] = 0;
}

// Kasai, Lee, Arimura, Arikawa, Park (2001): visiting suffixes in text order,
// the LCP with the SA predecessor drops by at most one per step.
void ora_lcp_kasai(const uint64_t *S, uint64_t n, const uint32_t *sa, uint32_t *lcp) {
  if (n == 0) return;
  std::vector<uint32_t> rank(n);
  for (uint64_t k = 0; k < n; ++k) rank[sa[k]] = (uint32_t)k;
  uint64_t h = 0;
  for (uint64_t i = 0; i < n; ++i) {
    if (rank[i] == 0) {
      h = 0;
      continue;
    }
    uint64_t j = sa[rank[i] - 1];
    while (i + h < n && j + h < n && S[i + h] == S[j + h]) ++h;
    lcp[rank[i] - 1] = (uint32_t)h;
    if (h > 0) --h;
  }
  lcp[n - 1] = 0;
}

// Alg. 2 candidate loop over adjacent SA pairs, before filtering and sorting.
// Writes up to 2(n-1) (length, start) pairs; returns their number.
uint64_t ora_candidates_raw(uint64_t n, const uint32_t *sa, const uint32_t *lcp,
                            uint32_t *l_out, uint32_t *s_out) {
  uint64_t m = 0;
  for (uint64_t i = 0; i + 1 < n; ++i) {
    uint64_t s1 = sa[i], s2 = sa[i + 1], p = lcp[i];
    uint64_t lo = std::min(s1, s2), hi = std::max(s1, s2);
    if (hi >= lo + p) {  // [s1, s1+p) and [s2, s2+p) do not intersect
      l_out[m] = (uint32_t)p; s_out[m++] = (uint32_t)s1;
      l_out[m] = (uint32_t)p; s_out[m++] = (uint32_t)s2;
    } else {             // overlap: the shared prefix is a run of S[lo, lo+d)
      uint64_t d = hi - lo;
      uint64_t l = (p + d) / 2;
      l -= l % d;
      l_out[m] = (uint32_t)l; s_out[m++] = (uint32_t)lo;
      l_out[m] = (uint32_t)l; s_out[m++] = (uint32_t)(lo + l);
    }
  }
  return m;
}

// LCE queries (for the tests): out[k] = lcp of the suffixes at a[k] and b[k],
// through the sparse table over the given SA and LCP.
void ora_lce(const uint32_t *sa, const uint32_t *lcp, uint64_t n, const uint32_t *a, const uint32_t *b,
             uint64_t q, uint64_t *out) {
  if (n == 0) return;
  Lce E(sa, lcp, n);
  for (uint64_t k = 0; k < q; ++k) out[k] = E(a[k], b[k]);
}

// Greedy selection over candidates already in priority order (Alg. 2's second
// loop).  variant 0: an ordered set of the accepted intervals; 1: the literal
// scan over every accepted interval; 2: the mark array of Sec. 4.2 (mark every
// covered position, test only the candidate's first and last position).
void ora_greedy(uint64_t n, uint64_t m, const uint32_t *l, const uint32_t *s,
                uint8_t *accepted, int variant) {
  if (variant == 0) {
    std::set<std::pair<uint64_t, uint64_t>> I;  // (start, end) half-open
    for (uint64_t k = 0; k < m; ++k) {
      uint64_t a = s[k], b = (uint64_t)s[k] + l[k];
      bool hit = false;
      auto it = I.lower_bound({a, 0});
      if (it != I.end() && it->first < b) hit = true;
      if (it != I.begin() && std::prev(it)->second > a) hit = true;
      accepted[k] = !hit && b > a;
      if (accepted[k]) I.insert({a, b});
    }
  } else if (variant == 1) {
    std::vector<std::pair<uint64_t, uint64_t>> I;
    for (uint64_t k = 0; k < m; ++k) {
      uint64_t a = s[k], b = (uint64_t)s[k] + l[k];
      bool hit = false;
      for (auto &iv : I)
        if (a < iv.second && iv.first < b) hit = true;
      accepted[k] = !hit && b > a;
      if (accepted[k]) I.push_back({a, b});
    }
  } else {
    std::vector<uint8_t> mark(n, 0);
    for (uint64_t k = 0; k < m; ++k) {
      uint64_t a = s[k], e = (uint64_t)s[k] + l[k] - 1;
      accepted[k] = l[k] > 0 && !mark[a] && !mark[e];
      if (accepted[k])
        for (uint64_t x = a; x <= e; ++x) mark[x] = 1;
    }
  }
}

// Alg. 2 FindRepeats(S) from a given SA and LCP.
//
// Outputs (caller-allocated, capacity 2n each for candidates, n for the rest):
//   cand_l/cand_id/cand_s   candidates with length >= min_len, sorted by
//                           (length desc, sub-string asc, start asc), one per
//                           distinct (length, start); cand_id is the number of
//                           suffixes whose first `length` tokens are smaller
//                           than the sub-string (= the SA index of its first
//                           occurrence), which orders same-length sub-strings
//   accepted                1 where the greedy loop took the candidate
//   sel_start/len/trace     the accepted intervals by increasing start, with
//                           the index of their sub-string in R
//   trace_len/start         R: distinct accepted sub-strings in the order the
//                           loop first took them; start = smallest accepted start
//   counts[0..2]            #candidates, #accepted, |R|
// cmp_method: how sub-strings are compared in the sort and the id search:
// 0 token by token, 1 by LCE queries over the given SA and LCP (O(1) per
// comparison, for windows whose long repeats make token loops quadratic),
// 2 token by token up to 2^16 tokens and by LCE above.
void ora_find_repeats(const uint64_t *S, uint64_t n, const uint32_t *sa, const uint32_t *lcp,
                      uint32_t min_len, int greedy_variant, int cmp_method, uint32_t *cand_l, uint32_t *cand_id,
                      uint32_t *cand_s, uint8_t *accepted, uint32_t *sel_start, uint32_t *sel_len,
                      uint32_t *sel_trace, uint32_t *trace_len, uint32_t *trace_start,
                      uint64_t *counts) {
  counts[0] = counts[1] = counts[2] = 0;
  if (n < 2) return;
  std::vector<uint32_t> rl(2 * n), rs(2 * n);
  uint64_t m_raw = ora_candidates_raw(n, sa, lcp, rl.data(), rs.data());
  std::vector<Cand> C;
  for (uint64_t k = 0; k < m_raw; ++k)
    if (rl[k] >= min_len && rl[k] > 0) C.push_back({rl[k], rs[k]});
  const bool use_lce = cmp_method == 1 || (cmp_method == 2 && n > (1u << 16));
  Lce *E = nullptr;
  if (use_lce) E = new Lce(sa, lcp, n);
  // Sort by decreasing length, then increasing sub-string, then increasing start.
  std::sort(C.begin(), C.end(), [&](const Cand &a, const Cand &b) {
    if (a.l != b.l) return a.l > b.l;
    int c = E ? substr_cmp_lce(S, *E, a.s, b.s, a.l) : substr_cmp(S, a.s, b.s, a.l);
    if (c != 0) return c < 0;
    return a.s < b.s;
  });
  std::vector<Cand> D;
  for (auto &c : C)
    if (D.empty() || D.back().l != c.l || D.back().s != c.s) D.push_back(c);
  uint64_t m = D.size();
  for (uint64_t k = 0; k < m; ++k) {
    cand_l[k] = (uint32_t)D[k].l;
    cand_s[k] = (uint32_t)D[k].s;
    // First SA index whose length-l prefix is not smaller than the sub-string.
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
      uint64_t mid = (lo + hi) / 2;
      const bool less = E ? prefix_less_lce(S, n, *E, sa[mid], D[k].s, D[k].l)
                          : prefix_less(S, n, sa[mid], D[k].s, D[k].l);
      if (less) lo = mid + 1; else hi = mid;
    }
    cand_id[k] = (uint32_t)lo;
  }
  delete E;
  ora_greedy(n, m, cand_l, cand_s, accepted, greedy_variant);
  // R: distinct accepted sub-strings, keyed by their tokens, in first-acceptance order.
  std::map<std::vector<uint64_t>, uint32_t> Rix;
  std::vector<std::pair<uint64_t, uint64_t>> sel;  // (start, k)
  std::vector<uint32_t> tr_of(m, 0);
  uint64_t ntr = 0;
  for (uint64_t k = 0; k < m; ++k) {
    if (!accepted[k]) continue;
    std::vector<uint64_t> key(S + cand_s[k], S + cand_s[k] + cand_l[k]);
    auto it = Rix.find(key);
    uint32_t t;
    if (it == Rix.end()) {
      t = (uint32_t)ntr++;
      Rix.emplace(std::move(key), t);
      trace_len[t] = cand_l[k];
      trace_start[t] = cand_s[k];
    } else {
      t = it->second;
      trace_start[t] = std::min(trace_start[t], cand_s[k]);
    }
    tr_of[k] = t;
    sel.push_back({cand_s[k], k});
  }
  std::sort(sel.begin(), sel.end());
  for (uint64_t q = 0; q < sel.size(); ++q) {
    uint64_t k = sel[q].second;
    sel_start[q] = cand_s[k];
    sel_len[q] = cand_l[k];
    sel_trace[q] = tr_of[k];
  }
  counts[0] = m;
  counts[1] = sel.size();
  counts[2] = ntr;
}

// All (end, pattern) pairs with stream[end-len+1 .. end] == pattern, ordered
// by end ascending, pattern length descending, pattern id ascending.  naive != 0 tries every pattern at every position; otherwise
// only the patterns whose first token equals stream[pos].  Returns the count
// (entries beyond cap are not written).
uint64_t ora_match(const uint64_t *pat_tok, const uint64_t *pat_off, uint64_t P,
                   const uint64_t *stream, uint64_t n, int naive, uint32_t *end_out,
                   uint32_t *id_out, uint64_t cap) {
  struct Hit {
    uint64_t end, len, p;
  };
  std::vector<Hit> hits;
  auto try_at = [&](uint64_t pos, uint64_t p) {
    uint64_t len = pat_off[p + 1] - pat_off[p];
    if (len == 0 || pos + len > n) return;
    for (uint64_t k = 0; k < len; ++k)
      if (stream[pos + k] != pat_tok[pat_off[p] + k]) return;
    hits.push_back({pos + len - 1, len, p});
  };
  if (naive) {
    for (uint64_t pos = 0; pos < n; ++pos)
      for (uint64_t p = 0; p < P; ++p) try_at(pos, p);
  } else {
    std::unordered_map<uint64_t, std::vector<uint64_t>> first;
    for (uint64_t p = 0; p < P; ++p)
      if (pat_off[p + 1] > pat_off[p]) first[pat_tok[pat_off[p]]].push_back(p);
    for (uint64_t pos = 0; pos < n; ++pos) {
      auto it = first.find(stream[pos]);
      if (it == first.end()) continue;
      for (uint64_t p : it->second) try_at(pos, p);
    }
  }
  std::sort(hits.begin(), hits.end(), [](const Hit &a, const Hit &b) {
    if (a.end != b.end) return a.end < b.end;
    if (a.len != b.len) return a.len > b.len;
    return a.p < b.p;
  });
  for (uint64_t k = 0; k < hits.size() && k < cap; ++k) {
    end_out[k] = (uint32_t)hits[k].end;
    id_out[k] = (uint32_t)hits[k].p;
  }
  return hits.size();
}

// Alg. 1 "TraceReplayer" with Sec. 4.3's trie, pointers and scoring, one
// task at a time.  Candidate trace q is the slice S[tr_start[q] ..
// tr_start[q] + tr_len[q]) and enters the trie when task tr_ingest[q] is
// processed (IngestCandidates runs first in TraceReplayer).  A trace longer
// than max_len (0 = no limit) enters as consecutive pieces of max_len tokens,
// the last one shorter (the maximum trace length of Sec. 6.2); pieces are
// numbered in input order, and a replay reports the smallest piece number
// with its string.  For task k (token S[k]):
//   AdvanceActiveCandidates / FilterInvalidCandidates: every pointer moves
//     along the edge S[k] if the trie has it and is dropped otherwise; a new
//     pointer starts at the root and moves along S[k] the same way;
//   FilterCompletedCandidates: D = the pointers standing at the end of a
//     trace; every trace in D counts one more appearance;
//   SelectReplayTrace: if D is not empty, the trace with the highest score
//     (the longer one on a tie) is replayed -- it ends at k -- and
//   ExecuteAndReplay: the tasks before it run untraced, its tasks are the
//     replay, and every pointer is dropped (each one has consumed task k,
//     which the replay took).
// score = (len * min(count, cap) * (replayed before ? bonus_num : bonus_den))
//         >> ((k - previous appearance) / half_life)
// with count including this appearance; no shift at a trace's first
// appearance or with half_life = 0, a shift of 64 or more gives 0, cap = 0
// means no cap.  Writes up to rcap replays (end task, length, trace number)
// and traced[k] = 1 for the tasks inside replays; returns the replay count.
uint64_t ora_replay(const uint64_t *S, uint64_t n, uint64_t P, const uint64_t *tr_start,
                    const uint64_t *tr_len, const uint64_t *tr_ingest, uint64_t max_len, uint64_t cap,
                    uint64_t half_life, uint64_t bonus_num, uint64_t bonus_den, uint32_t *rep_end,
                    uint32_t *rep_len, uint32_t *rep_trace, uint64_t rcap, uint8_t *traced) {
  struct Piece {
    uint64_t start, len, ingest, id;
  };
  std::vector<Piece> pieces;
  for (uint64_t q = 0; q < P; ++q) {
    uint64_t off = 0;
    do {
      uint64_t l = tr_len[q] - off;
      if (max_len && l > max_len) l = max_len;
      pieces.push_back({tr_start[q] + off, l, tr_ingest[q], (uint64_t)pieces.size()});
      off += l;
    } while (off < tr_len[q]);
  }
  // smallest piece number per string
  std::map<std::vector<uint64_t>, uint64_t> first_id;
  for (const Piece &pc : pieces) {
    std::vector<uint64_t> str(S + pc.start, S + pc.start + pc.len);
    auto it = first_id.find(str);
    if (it == first_id.end()) first_id.emplace(std::move(str), pc.id);
  }
  struct Node {
    std::map<uint64_t, uint32_t> child;
    int64_t trace = -1;  // trace number if a trace ends here
    uint64_t len = 0, count = 0;
    int64_t last = -1;
    bool replayed = false;
  };
  std::vector<Node> trie(1);
  auto ingest = [&](const Piece &pc) {
    uint32_t v = 0;
    for (uint64_t j = 0; j < pc.len; ++j) {
      const uint64_t c = S[pc.start + j];
      auto it = trie[v].child.find(c);
      if (it == trie[v].child.end()) {
        trie.emplace_back();
        const uint32_t w = (uint32_t)(trie.size() - 1);
        trie[v].child.emplace(c, w);
        v = w;
      } else {
        v = it->second;
      }
    }
    if (trie[v].trace < 0) {
      std::vector<uint64_t> str(S + pc.start, S + pc.start + pc.len);
      trie[v].trace = (int64_t)first_id[str];
      trie[v].len = pc.len;
    }
  };
  std::vector<uint64_t> order(pieces.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint64_t a, uint64_t b) { return pieces[a].ingest < pieces[b].ingest; });
  uint64_t next_piece = 0, nrep = 0;
  std::vector<uint32_t> A, A2;  // pointers: trie nodes (a node's depth fixes its start)
  for (uint64_t k = 0; k < n; ++k) {
    traced[k] = 0;
    while (next_piece < order.size() && pieces[order[next_piece]].ingest <= k) ingest(pieces[order[next_piece++]]);
    A2.clear();
    for (uint32_t v : A) {
      auto it = trie[v].child.find(S[k]);
      if (it != trie[v].child.end()) A2.push_back(it->second);
    }
    {
      auto it = trie[0].child.find(S[k]);
      if (it != trie[0].child.end()) A2.push_back(it->second);
    }
    A.swap(A2);
    int64_t best = -1;
    uint64_t best_score = 0;
    for (uint32_t v : A) {
      Node &t = trie[v];
      if (t.trace < 0) continue;
      uint64_t shift = 0;
      if (t.last >= 0 && half_life) shift = (k - (uint64_t)t.last) / half_life;
      t.count += 1;
      t.last = (int64_t)k;
      const uint64_t c = cap ? std::min(t.count, cap) : t.count;
      const uint64_t x = t.len * c * (t.replayed ? bonus_num : bonus_den);
      const uint64_t score = shift >= 64 ? 0 : (x >> shift);
      if (best < 0 || score > best_score || (score == best_score && t.len > trie[best].len)) {
        best = v;
        best_score = score;
      }
    }
    if (best >= 0) {
      Node &t = trie[best];
      t.replayed = true;
      if (nrep < rcap) {
        rep_end[nrep] = (uint32_t)k;
        rep_len[nrep] = (uint32_t)t.len;
        rep_trace[nrep] = (uint32_t)t.trace;
      }
      ++nrep;
      for (uint64_t j = k + 1 - t.len; j <= k; ++j) traced[j] = 1;
      A.clear();
    }
  }
  return nrep;
}

// Sec. 3's problem: traces T (sub-strings of S of length >= min_len) and
// for each trace a set of intervals of S holding it, all intervals disjoint;
// maximise the coverage (sum of interval lengths), then the number of
// intervals, then minimise |T|.  As stated the problem is solved by T = {S}
// (one interval covering everything), so every trace is required to match at
// least two intervals: the traces must repeat.  Exhaustive: every set of
// disjoint intervals of length >= min_len is enumerated (positions left to
// right: uncovered, or the start of an interval of each admissible length);
// a set is feasible iff each of its distinct strings occurs in it at least
// twice, and T is then its set of distinct strings.  Writes the optimum
// (coverage, intervals, |T|) and one optimal set (the first met in the
// enumeration order; wstart/wlen, n entries each) and returns its size.
uint64_t ora_optimum(const uint64_t *S, uint64_t n, uint64_t min_len, uint64_t *best3, uint32_t *wstart,
                     uint32_t *wlen) {
  std::vector<std::pair<uint64_t, uint64_t>> cur, best;
  int64_t bcov = -1, bcnt = -1, bdist = -1;
  auto evaluate = [&]() {
    std::map<std::vector<uint64_t>, int> groups;
    int64_t cov = 0;
    for (auto &iv : cur) {
      groups[std::vector<uint64_t>(S + iv.first, S + iv.first + iv.second)] += 1;
      cov += (int64_t)iv.second;
    }
    for (auto &g : groups)
      if (g.second < 2) return;
    const int64_t cnt = (int64_t)cur.size(), dist = (int64_t)groups.size();
    if (cov > bcov || (cov == bcov && (cnt > bcnt || (cnt == bcnt && dist < bdist)))) {
      bcov = cov;
      bcnt = cnt;
      bdist = dist;
      best = cur;
    }
  };
  std::function<void(uint64_t)> go = [&](uint64_t p) {
    if (p >= n) {
      evaluate();
      return;
    }
    go(p + 1);  // position p uncovered
    for (uint64_t L = std::max<uint64_t>(min_len, 1); p + L <= n; ++L) {
      cur.push_back({p, L});
      go(p + L);
      cur.pop_back();
    }
  };
  go(0);
  best3[0] = (uint64_t)bcov;
  best3[1] = (uint64_t)bcnt;
  best3[2] = (uint64_t)bdist;
  for (uint64_t k = 0; k < best.size(); ++k) {
    wstart[k] = (uint32_t)best[k].first;
    wlen[k] = (uint32_t)best[k].second;
  }
  return best.size();
}

}  // extern "C"
