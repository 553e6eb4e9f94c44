// The optimum of Sec. 3's trace-selection problem for many short windows --
// the yardstick that Alg. 2, a heuristic (Sec. 4.2), is measured against.
//
// Problem (Sec. 3): traces T, sub-strings of S of length >= min_len, each
// with a set of intervals of S that hold it, all intervals disjoint;
// maximise the coverage (summed interval lengths), then the number of
// intervals, then minimise |T|.  As stated, T = {S} covers everything, so
// each trace must match at least two intervals (the traces must repeat).
//
// One thread per window, exhaustive: a depth-first walk over the interval
// sets, positions left to right, each one either uncovered or the start of
// an interval of length min_len, min_len + 1, ...  Per string a counter of
// its intervals in the current set gives "every string at least twice"
// (no counter at 1) and |T| (counters above 0) at every leaf in O(1).
// Two cuts that leave the first optimal set in the walk order unchanged:
// an interval whose string has no second, disjoint occurrence in the window
// is never tried (every set holding it is infeasible), and a subtree whose
// coverage bound -- coverage so far plus the positions ahead that some
// repeatable interval covers -- is below the best coverage found is skipped
// (none of its sets can reach it).
#include <algorithm>
#include <vector>

#include "../../include/apo.h"
#include "apo_internal.cuh"

namespace apo {

namespace {

constexpr int kOptMax = 24;                // longest window
constexpr int kIdStride = kOptMax + 1;     // string id = first start * kIdStride + length
constexpr uint64_t kOptLeaves = 1ull << 24;  // largest admissible enumeration
constexpr uint32_t kOptGuard = 1u << 30;     // node visits after which a walk gives up

template <class T>
__global__ void __launch_bounds__(128)
    k_optimum(const T *__restrict__ tok, const uint32_t *__restrict__ off, uint32_t W, uint32_t m,
              uint32_t *__restrict__ best, uint32_t *__restrict__ wstart, uint32_t *__restrict__ wlen,
              uint32_t *__restrict__ wcount, uint32_t *err) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x) {
    const uint32_t a0 = off[w];
    const int n = (int)(off[w + 1] - a0);
    T s[kOptMax];
    for (int i = 0; i < n; ++i) s[i] = tok[a0 + i];
    // sid[a][L] = the first start of the length-L string at a
    uint8_t sid[kOptMax][kOptMax + 1];
    for (int a = 0; a < n; ++a) {
      for (int L = 1; L <= n - a; ++L) sid[a][L] = (uint8_t)a;
      for (int b = a - 1; b >= 0; --b) {
        int l = 0;
        while (a + l < n && s[b + l] == s[a + l]) ++l;
        for (int L = 1; L <= l; ++L) sid[a][L] = (uint8_t)b;
      }
    }
    // rep[a] bit L: the length-L string at a occurs again, disjoint from it;
    // ahead[p]: positions >= p inside some repeatable interval
    uint32_t rep[kOptMax];
    for (int a = 0; a < n; ++a) rep[a] = 0;
    for (int a = 0; a < n; ++a)
      for (int b = a + 1; b < n; ++b) {
        int l = 0;
        while (b + l < n && s[a + l] == s[b + l]) ++l;
        const int lim = min(l, b - a);  // disjoint: L <= b - a
        for (int L = 1; L <= lim; ++L) {
          rep[a] |= 1u << L;
          rep[b] |= 1u << L;
        }
      }
    uint8_t ahead[kOptMax + 1];
    {
      uint32_t covered = 0;  // bit i: position i inside a repeatable interval of length >= m
      for (int a = 0; a < n; ++a)
        for (int L = (m < 1 ? 1 : (int)m); a + L <= n; ++L)
          if (rep[a] >> L & 1u) covered |= ((L == 32 ? 0u : (1u << L)) - 1u) << a;
      ahead[n] = 0;
      for (int p = n - 1; p >= 0; --p) ahead[p] = (uint8_t)(ahead[p + 1] + ((covered >> p) & 1u));
    }
    uint8_t cnt[kOptMax * kIdStride];
    for (int i = 0; i < kOptMax * kIdStride; ++i) cnt[i] = 0;
    uint8_t pos[kOptMax + 1], ch[kOptMax + 1];  // ch: 0xff unvisited, 0 uncovered, else interval length
    uint8_t bs[kOptMax], bl[kOptMax];
    int bk = 0, bcov = -1, bcnt = -1, bdist = 1 << 30;
    int cov = 0, icnt = 0, singles = 0, distinct = 0;
    const int m1 = m < 1 ? 1 : (int)m;
    int d = 0;
    pos[0] = 0;
    ch[0] = 0xff;
    uint32_t guard = 0;
    while (d >= 0) {
      if (++guard > kOptGuard) {
        atomicExch(err, kDevTimeout);
        break;
      }
      const int p = pos[d];
      if (ch[d] == 0xff) {
        if (p == n) {  // a complete interval set
          if (singles == 0 &&
              (cov > bcov || (cov == bcov && (icnt > bcnt || (icnt == bcnt && distinct < bdist))))) {
            bcov = cov;
            bcnt = icnt;
            bdist = distinct;
            bk = 0;
            for (int k = 0; k < d; ++k)
              if (ch[k]) {
                bs[bk] = pos[k];
                bl[bk] = ch[k];
                ++bk;
              }
          }
          --d;
          continue;
        }
        if (cov + ahead[p] < bcov) {  // cannot reach the best coverage
          --d;
          continue;
        }
        ch[d] = 0;  // position p uncovered
        pos[d + 1] = (uint8_t)(p + 1);
        ch[d + 1] = 0xff;
        ++d;
        continue;
      }
      // back from a child: take the interval of the last choice out, try the next length
      const int L = ch[d];
      if (L) {
        const int id = sid[p][L] * kIdStride + L;
        const int c = --cnt[id];
        if (c == 1) ++singles;
        else if (c == 0) {
          --singles;
          --distinct;
        }
        cov -= L;
        --icnt;
      }
      int nx = L ? L + 1 : m1;
      while (p + nx <= n && !(rep[p] >> nx & 1u)) ++nx;  // only strings that can repeat
      if (p + nx > n) {
        --d;
        continue;
      }
      ch[d] = (uint8_t)nx;
      {
        const int id = sid[p][nx] * kIdStride + nx;
        const int c = ++cnt[id];
        if (c == 1) {
          ++singles;
          ++distinct;
        } else if (c == 2) {
          --singles;
        }
        cov += nx;
        ++icnt;
      }
      pos[d + 1] = (uint8_t)(p + nx);
      ch[d + 1] = 0xff;
      ++d;
    }
    best[3 * w] = (uint32_t)bcov;
    best[3 * w + 1] = (uint32_t)bcnt;
    best[3 * w + 2] = (uint32_t)bdist;
    for (int k = 0; k < bk; ++k) {
      wstart[a0 + k] = bs[k];
      wlen[a0 + k] = bl[k];
    }
    wcount[w] = (uint32_t)bk;
  }
}

// Interval sets of a length-n window with pieces of at least m: f(n) =
// f(n - 1) + sum_{L >= m} f(n - L), f(0) = 1 (capped).
uint64_t interval_sets(int n, int m) {
  std::vector<uint64_t> f(n + 1, 0);
  f[0] = 1;
  for (int k = 1; k <= n; ++k) {
    uint64_t v = f[k - 1];
    for (int L = std::max(m, 1); L <= k; ++L) v = std::min<uint64_t>(v + f[k - L], 1ull << 62);
    f[k] = v;
  }
  return f[n];
}

}  // namespace

int optimum_batched(apo_ctx *c, const apo_windows *ws, uint32_t min_len, uint32_t *best, uint32_t *wstart,
                    uint32_t *wlen, uint32_t *wcount, cudaStream_t s) {
  const uint64_t W = ws->n_windows;
  uint64_t maxn = 0;
  for (uint64_t w = 0; w < W; ++w) maxn = std::max(maxn, ws->win_off[w + 1] - ws->win_off[w]);
  if (maxn > (uint64_t)kOptMax) {
    set_error("apo_optimum_batched: windows of at most 24 tokens");
    return APO_EINVAL;
  }
  if (interval_sets((int)maxn, (int)min_len) > kOptLeaves) {
    set_error("apo_optimum_batched: the exhaustive search is too large (more than 2^24 interval sets "
              "for the longest window at this min_len)");
    return APO_EINVAL;
  }
  APO_TRY(ensure_side(c, (W + 1) * 4, s));
  uint32_t *off = static_cast<uint32_t *>(c->side);
  std::vector<uint32_t> h(W + 1);
  for (uint64_t w = 0; w <= W; ++w) h[w] = (uint32_t)ws->win_off[w];
  APO_CUDA_TRY(cudaMemcpyAsync(off, h.data(), (W + 1) * 4, cudaMemcpyHostToDevice, s));
  const int threads = 128;
  const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((W + threads - 1) / threads,
                                                                   (uint64_t)c->num_sms * 64));
  {
    Launch lp_(c, kKOptimum, W, s);
    if (ws->token_bytes == 4)
      k_optimum<<<blocks, threads, 0, s>>>(static_cast<const uint32_t *>(ws->tokens), off, (uint32_t)W, min_len,
                                           best, wstart, wlen, wcount, c->ps.err);
    else
      k_optimum<<<blocks, threads, 0, s>>>(static_cast<const uint64_t *>(ws->tokens), off, (uint32_t)W, min_len,
                                           best, wstart, wlen, wcount, c->ps.err);
  }
  APO_CUDA_TRY(cudaGetLastError());
  return check_device_error(c, s);  // synchronises: the host array h is released on return
}

}  // namespace apo
