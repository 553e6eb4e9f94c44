// Candidate matching (Sec. 4.3): the candidate traces are ingested into a
// trie and the stream is followed through it; a trace is reported whenever
// a pointer reaches its end.  All pointers at once are exactly the state of
// an Aho-Corasick automaton (Aho & Corasick, CACM 1975): the goto trie, a
// failure link per node (longest proper suffix that is also in the trie) and
// an output link per node (nearest pattern end on the failure chain).
//
// Build.  Tokens become 32-bit symbols (u32 tokens as they are; u64 tokens
// by their index in the sorted list of distinct pattern tokens, a stream
// token outside that list matching nothing).  The goto function is one
// open-addressed hash table keyed by (node << 32 | symbol); one thread per
// pattern inserts its path, claiming slots with atomicCAS (a node id is
// published after its parent/depth/symbol).  Nodes are ordered by depth with
// the radix sort, and failure and output links are computed level by level.
//
// Match.  A node's state depends only on the last (max pattern length)
// tokens, so the stream is cut into chunks and each thread runs the
// automaton over its chunk after a halo of (max length - 1) tokens, writing
// the state of every position.  The number of matches a state reports
// (its own pattern ends plus those down its output chain) is precomputed per
// node during the level-by-level link pass, so the output offsets are one
// prefix sum over positions; a final kernel per position then writes its
// matches.  Output order: end ascending, then pattern length descending (the
// output chain's order), then pattern id ascending.
#include <algorithm>
#include <cstring>
#include <vector>

#include "apo_internal.cuh"
#include "device_util.cuh"

namespace apo {

namespace {

constexpr uint32_t kNil = 0xffffffffu;
constexpr uint64_t kEmpty = ~0ull;

__device__ __forceinline__ uint64_t mix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

struct Goto {
  uint64_t *keys;
  uint32_t *vals;
  uint64_t mask;
};

__device__ __forceinline__ uint32_t goto_lookup(const Goto &g, uint32_t u, uint32_t c) {
  const uint64_t key = ((uint64_t)u << 32) | c;
  uint64_t slot = mix64(key) & g.mask;
  while (true) {
    const uint64_t k = g.keys[slot];
    if (k == key) return g.vals[slot];
    if (k == kEmpty) return kNil;
    slot = (slot + 1) & g.mask;
  }
}

__device__ __forceinline__ uint32_t to_sym(const void *tok, int tb, uint64_t i, const uint64_t *dict,
                                           uint32_t sigma) {
  if (tb == 4) return static_cast<const uint32_t *>(tok)[i];
  const uint64_t t = static_cast<const uint64_t *>(tok)[i];
  uint32_t lo = 0, hi = sigma;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (dict[mid] < t) lo = mid + 1; else hi = mid;
  }
  return (lo < sigma && dict[lo] == t) ? lo : kNil;
}

__global__ void k_trie_insert(const void *pat_tok, int tb, const uint32_t *__restrict__ pstart,
                              const uint32_t *__restrict__ plen, uint32_t P, const uint64_t *dict,
                              uint32_t sigma, Goto g,
                              uint32_t *node_ctr, uint32_t *parent, uint32_t *depth, uint32_t *nsym,
                              uint32_t *end_node, uint32_t *err) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  uint32_t u = 0;
  const uint64_t off = pstart[p], len = plen[p];
  for (uint64_t d = 0; d < len; ++d) {
    const uint32_t c = to_sym(pat_tok, tb, off + d, dict, sigma);
    const uint64_t key = ((uint64_t)u << 32) | c;
    uint64_t slot = mix64(key) & g.mask;
    uint32_t v = kNil;
    for (uint64_t probe = 0; probe <= g.mask; ++probe) {
      uint64_t cur = *(volatile uint64_t *)&g.keys[slot];
      if (cur == kEmpty) {
        cur = atomicCAS((unsigned long long *)&g.keys[slot], (unsigned long long)kEmpty,
                        (unsigned long long)key);
        if (cur == kEmpty) {  // this thread created the node
          v = atomicAdd(node_ctr, 1u) + 1u;
          parent[v] = u;
          depth[v] = (uint32_t)d + 1;
          nsym[v] = c;
          __threadfence();
          *(volatile uint32_t *)&g.vals[slot] = v;
          break;
        }
      }
      if (cur == key) {  // wait until the creator publishes the id
        uint32_t spins = 0;
        while ((v = *(volatile uint32_t *)&g.vals[slot]) == 0) {
          if (++spins > kSpinLimit) {
            atomicExch(err, kDevTimeout);
            return;
          }
          __nanosleep(64);
        }
        __threadfence();
        break;
      }
      slot = (slot + 1) & g.mask;
    }
    if (v == kNil) {
      atomicExch(err, kDevRange);
      return;
    }
    u = v;
  }
  end_node[p] = u;
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

__global__ void k_depth_keys(const uint32_t *__restrict__ depth, uint32_t N, uint64_t *keys,
                             uint32_t *vals, uint32_t *level_cnt) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    const uint32_t d = v == 0 ? 0 : depth[v];
    keys[v] = d;
    vals[v] = v;
    atomicAdd(&level_cnt[d], 1u);
  }
}

__global__ void k_end_pairs(const uint32_t *__restrict__ end_node, uint32_t P, uint64_t *keys,
                            uint32_t *vals) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    keys[p] = end_node[p];
    vals[p] = p;
  }
}

__global__ void k_mark_ends(const uint64_t *__restrict__ skeys, uint32_t P, uint32_t *end_first) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x)
    if (k == 0 || skeys[k] != skeys[k - 1]) end_first[(uint32_t)skeys[k]] = k;
}

// Failure and output links of the nodes order[lo, hi) (all of one depth).
__global__ void k_fail_level(const uint32_t *__restrict__ order, uint32_t lo, uint32_t hi,
                             uint32_t d, Goto g, const uint32_t *__restrict__ parent,
                             const uint32_t *__restrict__ nsym, const uint32_t *__restrict__ end_first,
                             const uint32_t *__restrict__ own, uint32_t *fail, uint32_t *outl,
                             uint32_t *total) {
  for (uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x) {
    const uint32_t v = order[i];
    uint32_t f = 0;
    if (d > 1) {
      const uint32_t c = nsym[v];
      uint32_t w = fail[parent[v]];
      while (true) {
        const uint32_t x = goto_lookup(g, w, c);
        if (x != kNil) {
          f = x;
          break;
        }
        if (w == 0) break;
        w = fail[w];
      }
    }
    fail[v] = f;
    const uint32_t o = (f != 0 && end_first[f] != kNil) ? f : outl[f];
    outl[v] = o;
    total[v] = own[v] + total[o];  // matches reported when the automaton is in v
  }
}

// own[v] = number of patterns ending exactly at node v.
__global__ void k_own_counts(const uint64_t *__restrict__ skeys, uint32_t P, uint32_t *own) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x)
    atomicAdd(&own[(uint32_t)skeys[k]], 1u);
}

// Pass A: automaton state after every stream position.  Thread t owns
// positions [t*chunk, (t+1)*chunk) and starts from the root `halo` tokens
// earlier (a state only depends on the last max-length tokens).
__global__ void k_ac_states(const void *stream, int tb, uint64_t n, uint64_t chunk, uint64_t halo,
                            const uint64_t *dict, uint32_t sigma, Goto g,
                            const uint32_t *__restrict__ fail, uint32_t *__restrict__ state_out) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t cs = t * chunk;
  if (cs >= n) return;
  const uint64_t ce = min(n, cs + chunk);
  uint64_t x = cs > halo ? cs - halo : 0;
  uint32_t state = 0;
  for (; x < ce; ++x) {
    const uint32_t c = to_sym(stream, tb, x, dict, sigma);
    while (true) {
      const uint32_t nx = (c == kNil && tb == 8) ? kNil : goto_lookup(g, state, c);
      if (nx != kNil) {
        state = nx;
        break;
      }
      if (state == 0) break;
      state = fail[state];
    }
    if (x >= cs) state_out[x] = state;
  }
}

// Exclusive prefix sum of total[state[x]] over stream positions (the first
// output slot of each position), decoupled look-back.
constexpr int kST = 256, kSI = 16, kSTile = kST * kSI;
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
  for (int q = tid; q < kSTile; q += kST)
    sv[q] = base + q < n ? total[state[base + q]] : 0u;
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
      pre = lb_exclusive(status, 1, t, epoch, OpSum(), 0u, err);
      lb_store(&status[t], lb_pack(kLbInclusive, epoch, pre + tot));
    }
    s_pre = pre;
    if (base + kSTile >= n) *sum_out = pre + tot;
  }
  __syncthreads();
  uint32_t r = s_pre + ex;
#pragma unroll
  for (int i = 0; i < kSI; ++i) {
    const uint64_t x = base + (uint64_t)tid * kSI + i;
    if (x < n) off[x] = r;
    r += sv[tid * kSI + i];
  }
}

// Pass B: the matches of position x, following the output chain from its
// state (deepest first), ids ascending within a node.
__global__ void k_ac_fill(const uint32_t *__restrict__ state, uint32_t n,
                          const uint32_t *__restrict__ off, const uint32_t *__restrict__ outl,
                          const uint32_t *__restrict__ end_first, const uint64_t *__restrict__ ekeys,
                          const uint32_t *__restrict__ evals, uint32_t P, uint32_t *mend,
                          uint32_t *mid, uint64_t cap) {
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const uint32_t s0 = state[x];
    uint64_t o = off[x];
    uint32_t v = end_first[s0] != kNil ? s0 : outl[s0];
    while (v != 0) {
      for (uint32_t k = end_first[v]; k < P && (uint32_t)ekeys[k] == v; ++k) {
        if (o < cap) {
          mend[o] = x;
          mid[o] = evals[k];
        }
        ++o;
      }
      v = outl[v];
    }
  }
}

__global__ void k_u64_keys(const uint64_t *__restrict__ t, uint64_t m, uint64_t *keys, uint32_t *vals) {
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    keys[q] = t[q];
    vals[q] = 0;
  }
}

__global__ void k_unique_u64(const uint64_t *__restrict__ s, uint64_t m, uint64_t *out,
                             unsigned long long *cnt) {
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    if (q == 0 || s[q] != s[q - 1]) out[atomicAdd(cnt, 1ull)] = s[q];  // sorted again after
  }
}

inline int grid_for(uint64_t n, int threads, int sms) {
  long long b = (long long)((n + threads - 1) / threads);
  return (int)std::max<long long>(1, std::min<long long>(b, (long long)sms * 16));
}

}  // namespace

size_t match_workspace_bytes(uint64_t total_tokens, uint64_t P, uint64_t n, uint64_t cap) {
  uint64_t tbl = 1;
  while (tbl < 2 * (total_tokens + 1)) tbl <<= 1;
  const uint64_t N = total_tokens + 1;
  (void)cap;
  const uint64_t M = std::max<uint64_t>(std::max<uint64_t>(N, total_tokens), P);
  return tbl * 12 + N * 4 * 9 + P * 24 + (P + 1) * 8 + total_tokens * 12 + M * 24 + n * 8 +
         64 * 256;
}

int match_patterns(apo_ctx *c, const apo_patterns *pp, const void *stream, uint64_t n,
                   uint32_t *match_end, uint32_t *match_id, uint64_t cap, uint64_t *count,
                   cudaStream_t s) {
  const uint32_t P = (uint32_t)pp->n_patterns;
  const int tb = pp->token_bytes;
  uint32_t *misc = c->ps.counters + kCtrMisc;
  unsigned long long *cnt64 = reinterpret_cast<unsigned long long *>(misc + kMiscKeyOr);
  const int sms = c->num_sms;
  // pattern p = tokens[pstart[p] .. pstart[p] + plen[p])
  const uint32_t *pstart = pp->pat_start, *plen = pp->pat_len;
  uint64_t total = 0, maxlen = 0, extent = 0;
  uint32_t *hostbuf = nullptr;
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
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    if (check_device_error(c, s) != APO_OK) {
      set_error("match_candidates: empty pattern");
      return APO_EINVAL;
    }
    maxlen = c->host_pinned[0];
    extent = c->host_pinned[1];
    memcpy(&total, c->host_pinned + 2, 8);
  }
  (void)hostbuf;
  if (total >= 0xffffffffull || extent >= 0xffffffffull) {
    set_error("match_candidates: more than 2^32 - 1 pattern tokens");
    return APO_EINVAL;
  }
  APO_TRY(c->arena.reserve(match_workspace_bytes(std::max(total, extent), P, n, cap)));
  const uint64_t N = total + 1;  // node bound (root included)
  uint64_t tbl = 1;
  while (tbl < 2 * N) tbl <<= 1;
  Goto g;
  g.keys = c->arena.take_n<uint64_t>(tbl);
  g.vals = c->arena.take_n<uint32_t>(tbl);
  g.mask = tbl - 1;
  uint32_t *pbuf = pp->pat_off ? c->arena.take_n<uint32_t>(2 * (size_t)P) : nullptr;
  uint32_t *parent = c->arena.take_n<uint32_t>(N);
  uint32_t *depth = c->arena.take_n<uint32_t>(N);
  uint32_t *nsym = c->arena.take_n<uint32_t>(N);
  uint32_t *fail = c->arena.take_n<uint32_t>(N);
  uint32_t *outl = c->arena.take_n<uint32_t>(N);
  uint32_t *end_first = c->arena.take_n<uint32_t>(N);
  uint32_t *end_node = c->arena.take_n<uint32_t>(P);
  uint32_t *own = c->arena.take_n<uint32_t>(N);
  uint32_t *mtotal = c->arena.take_n<uint32_t>(N);
  uint32_t *levels = c->arena.take_n<uint32_t>(maxlen + 2);
  const uint64_t M = std::max<uint64_t>(std::max<uint64_t>(N, extent), P);
  SortBuffers b;
  b.keys[0] = c->arena.take_n<uint64_t>(M);
  b.keys[1] = c->arena.take_n<uint64_t>(M);
  b.vals[0] = c->arena.take_n<uint32_t>(M);
  b.vals[1] = c->arena.take_n<uint32_t>(M);
  uint64_t *dict = c->arena.take_n<uint64_t>(std::max<uint64_t>(extent, 1));
  if (!g.keys || !g.vals || (pp->pat_off && !pbuf) || !parent || !depth || !nsym || !fail || !outl || !end_first || !own || !mtotal ||
      !end_node || !levels || !b.keys[0] || !b.keys[1] || !b.vals[0] || !b.vals[1] || !dict) {
    set_error("match: workspace too small");
    return APO_ENOMEM;
  }
  if (M >= 0xffffffffull || N >= 0xffffffffull || n >= 0xffffffffull) {
    set_error("match: more than 2^32 - 1 nodes, stream tokens or matches");
    return APO_EINVAL;
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
  APO_CUDA_TRY(cudaMemsetAsync(g.keys, 0xff, tbl * sizeof(uint64_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(g.vals, 0, tbl * sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(end_first, 0xff, N * sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(own, 0, N * sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(mtotal, 0, N * sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(levels, 0, (maxlen + 2) * sizeof(uint32_t), s));
  // u64 tokens: dictionary of distinct pattern tokens
  uint32_t sigma = 0;
  if (tb == 8) {
    {
      Launch lp_(c, kKU64Keys, 0, s);
      k_u64_keys<<<grid_for(extent, 256, sms), 256, 0, s>>>(static_cast<const uint64_t *>(pp->tokens),
                                                            extent, b.keys[0], b.vals[0]);
    }
    b.cur = 0;
    int places[8];
    const int np = plan_digits(0, 64, places, 0);
    APO_TRY(radix_sort_pairs(c, b, (uint32_t)extent, places, np, s));
    APO_CUDA_TRY(cudaMemsetAsync(cnt64, 0, 8, s));
    {
      Launch lp_(c, kKUnique, extent, s);
      k_unique_u64<<<grid_for(extent, 256, sms), 256, 0, s>>>(b.keys[b.cur], extent, dict, cnt64);
    }
    unsigned long long sg = 0;
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, cnt64, 8, cudaMemcpyDeviceToHost, s));
    APO_CUDA_TRY(cudaStreamSynchronize(s));
    memcpy(&sg, c->host_pinned, 8);
    sigma = (uint32_t)sg;
    // distinct values were appended in arbitrary order: sort them
    {
      Launch lp_(c, kKU64Keys, 0, s);
      k_u64_keys<<<grid_for(sigma, 256, sms), 256, 0, s>>>(dict, sigma, b.keys[0], b.vals[0]);
    }
    b.cur = 0;
    APO_TRY(radix_sort_pairs(c, b, sigma, places, np, s));
    APO_CUDA_TRY(cudaMemcpyAsync(dict, b.keys[b.cur], sigma * sizeof(uint64_t),
                                 cudaMemcpyDeviceToDevice, s));
  }

  // trie
  APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscMatchCount, 0, sizeof(uint32_t), s));
  {
    Launch lp_(c, kKTrieInsert, total, s);
    k_trie_insert<<<ceil_div(P, 128), 128, 0, s>>>(pp->tokens, tb, pstart, plen, P, dict, sigma, g,
                                                   misc + kMiscMatchCount, parent, depth, nsym,
                                                   end_node, c->ps.err);
  }
  APO_CUDA_TRY(cudaGetLastError());
  uint32_t nodes = 0;
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, misc + kMiscMatchCount, 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  APO_TRY(check_device_error(c, s));
  nodes = c->host_pinned[0] + 1;

  // pattern ends: (end node, pattern id) sorted by node
  uint64_t *ek;
  uint32_t *ev;
  {
    Launch lp_(c, kKEndPairs, P, s);
    k_end_pairs<<<grid_for(P, 256, sms), 256, 0, s>>>(end_node, P, b.keys[0], b.vals[0]);
  }
  b.cur = 0;
  {
    int places[8];
    const int np = plan_digits(0, bits_for(nodes), places, 0);
    APO_TRY(radix_sort_pairs(c, b, P, places, np, s));
  }
  // keep the sorted end pairs where the depth sort below will not overwrite them
  ek = c->arena.take_n<uint64_t>(P);
  ev = c->arena.take_n<uint32_t>(P);
  if (!ek || !ev) return APO_ENOMEM;
  APO_CUDA_TRY(cudaMemcpyAsync(ek, b.keys[b.cur], P * 8, cudaMemcpyDeviceToDevice, s));
  APO_CUDA_TRY(cudaMemcpyAsync(ev, b.vals[b.cur], P * 4, cudaMemcpyDeviceToDevice, s));
  {
    Launch lp_(c, kKMarkEnds, P, s);
    k_mark_ends<<<grid_for(P, 256, sms), 256, 0, s>>>(ek, P, end_first);
  }
  {
    Launch lp_(c, kKOwn, P, s);
    k_own_counts<<<grid_for(P, 256, sms), 256, 0, s>>>(ek, P, own);
  }

  // BFS order by depth
  {
    Launch lp_(c, kKDepthKeys, nodes, s);
    k_depth_keys<<<grid_for(nodes, 256, sms), 256, 0, s>>>(depth, nodes, b.keys[0], b.vals[0], levels);
  }
  b.cur = 0;
  {
    int places[8];
    const int np = plan_digits(0, bits_for(maxlen), places, 0);
    APO_TRY(radix_sort_pairs(c, b, nodes, places, np, s));
  }
  std::vector<uint32_t> lc(maxlen + 1);
  APO_CUDA_TRY(cudaMemcpyAsync(lc.data(), levels, (maxlen + 1) * 4, cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  const uint32_t *order = b.vals[b.cur];
  APO_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaMemsetAsync(outl, 0, sizeof(uint32_t), s));
  uint32_t lo = lc[0];
  for (uint64_t d = 1; d <= maxlen; ++d) {
    const uint32_t hi = lo + lc[d];
    if (hi > lo) {
      Launch lp_(c, kKFailLevel, hi - lo, s);
      k_fail_level<<<grid_for(hi - lo, 128, sms), 128, 0, s>>>(order, lo, hi, (uint32_t)d, g, parent,
                                                              nsym, end_first, own, fail, outl,
                                                              mtotal);
    }
    lo = hi;
  }
  APO_CUDA_TRY(cudaGetLastError());
  if (n == 0) return APO_OK;

  // pass A: states
  uint32_t *state = c->arena.take_n<uint32_t>(n);
  uint32_t *off = c->arena.take_n<uint32_t>(n);
  if (!state || !off) return APO_ENOMEM;
  const uint64_t halo = maxlen ? maxlen - 1 : 0;
  const uint64_t chunk = std::max<uint64_t>(64, n / ((uint64_t)sms * 32));
  const uint64_t threads = (n + chunk - 1) / chunk;
  {
    Launch lp_(c, kKAcMatch, n, s);
    k_ac_states<<<ceil_div(threads, 128), 128, 0, s>>>(stream, tb, n, chunk, halo, dict, sigma, g,
                                                       fail, state);
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
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  APO_TRY(check_device_error(c, s));
  const uint64_t total_m = c->host_pinned[0];
  *count = total_m;
  if (total_m > cap) {
    set_error("match_candidates: more matches than cap (count written)");
    return APO_ECAPACITY;
  }
  if (total_m) {
    Launch lp_(c, kKAcFill, n, s);
    k_ac_fill<<<grid_for(n, 256, sms), 256, 0, s>>>(state, (uint32_t)n, off, outl, end_first, ek, ev, P,
                                                    match_end, match_id, cap);
  }
  APO_CUDA_TRY(cudaGetLastError());
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(c, s);
}

}  // namespace apo
