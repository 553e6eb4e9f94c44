// Candidate matching (Sec. 4.3): the candidate traces are ingested into a
// trie and the stream is followed through it; a trace is reported whenever
// a pointer reaches its end.  All pointers at once are exactly the state of
// an Aho-Corasick automaton (Aho & Corasick, CACM 1975): the goto trie, a
// failure link per node (longest proper suffix that is also in the trie) and
// an output link per node (nearest pattern end on the failure chain).
//
// Symbols.  u32 tokens are their own symbols.  u64 tokens are mapped to 32-bit
// symbols through an open-addressed dictionary filled from the pattern tokens
// (a token's symbol is its slot); a stream token missing from the dictionary
// matches nothing.  Both the pattern source and the stream are mapped once,
// in parallel, before any sequential work.
//
// Build.  One cooperative kernel builds the trie level by level: at level d
// every pattern longer than d inserts its (d+1)-th node into the goto hash
// table (keyed by node << 32 | symbol, slots claimed with atomicCAS; a node's
// id is its slot), while the depth-d nodes get their failure link, output
// link and match total (own pattern ends plus those down the output chain),
// each computed by the pattern that created the node.  A bounded grid
// barrier separates levels.
//
// Match.  The stream is cut into short chunks and each thread runs the
// automaton over its chunk from the root, writing the state of every
// position (only the first chunk is exact).  Repair passes then restart each
// chunk from its predecessor's end state and stop at the first position whose
// state agrees with the recorded one -- from there on the deterministic
// automaton repeats the recorded run.  When a pass changes no end state all
// states are exact (after k passes chunks 0..k are, by induction).  The
// per-node match totals turn the output offsets into one prefix sum over
// positions; a final kernel per position writes its matches.  Output order:
// end ascending, then pattern length descending (the output chain's order),
// then pattern id ascending.
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

// Open addressing with linear probing, capacity a power of two.  A goto entry
// is 16 bytes (key, child id, pad) so that one 128-bit load reads both.
struct Table {
  uint64_t *keys;  // entry e: keys[2e] = key, keys[2e+1] low word = value
  uint64_t mask;
};

__device__ __forceinline__ uint32_t goto_lookup(const Table &g, uint32_t u, uint32_t c) {
  const uint64_t key = ((uint64_t)u << 32) | c;
  uint64_t slot = mix64(key) & g.mask;
  while (true) {
    const ulonglong2 e = *reinterpret_cast<const ulonglong2 *>(g.keys + 2 * slot);
    if (e.x == key) return (uint32_t)e.y;
    if (e.x == kEmpty) return kNil;
    slot = (slot + 1) & g.mask;
  }
}

// ---------------------------------------------------------------- symbols
struct Dict {
  uint64_t *keys;  // a token's symbol is its slot
  uint64_t mask;
};

__global__ void k_dict_insert(const uint64_t *__restrict__ tok, uint64_t m, Dict d) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = tok[i];
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

__global__ void k_dict_map(const uint64_t *__restrict__ tok, uint64_t m, Dict d,
                           uint32_t *__restrict__ sym) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = tok[i];
    uint32_t s = kNil;
    if (t == kEmpty) {
      s = (uint32_t)(d.mask + 1);  // reserved symbol of the all-ones token
    } else {
      uint64_t slot = mix64(t) & d.mask;
      while (true) {
        const uint64_t k = d.keys[slot];
        if (k == t) {
          s = (uint32_t)slot;
          break;
        }
        if (k == kEmpty) break;
        slot = (slot + 1) & d.mask;
      }
    }
    sym[i] = s;
  }
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

// ---------------------------------------------------------------- build
struct GridBarrier {
  uint32_t *count;
  uint32_t *gen;
};

// All blocks of a cooperative launch meet here.  Bounded: a block that waits
// too long records kDevTimeout and leaves (the caller then stops).
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ void grid_sync(const GridBarrier &b, uint32_t *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t g0 = ld_acquire(b.gen);
    __threadfence();  // this block's writes before its arrival
    if (atomicAdd(b.count, 1u) == gridDim.x - 1) {
      *(volatile uint32_t *)b.count = 0;
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      uint32_t spins = 0;
      while (ld_acquire(b.gen) == g0) {
        if (++spins > kSpinLimit) {
          atomicExch(err, kDevTimeout);
          break;
        }
      }
    }
  }
  __syncthreads();
}

// A node's id is the goto-table slot of the edge that leads to it (every
// node but the root has exactly one incoming edge); the root's id is the
// table capacity.  Node arrays therefore hold capacity + 1 entries.
struct BuildArgs {
  const uint32_t *psym;    // symbols of the pattern source tokens
  const uint32_t *pstart;  // pattern p = psym[pstart[p] .. pstart[p] + plen[p])
  const uint32_t *plen;
  uint32_t P;
  uint32_t maxlen;
  uint32_t root;
  Table g;
  uint32_t *cur[2];    // [P] node of each pattern at depth d (parity of d)
  uint8_t *made[2];    // [P] 1 if the pattern created that node
  uint32_t *parent;    // [nodes]
  uint32_t *nsym;      // [nodes] symbol on the edge into the node
  uint32_t *fail;      // [nodes]
  uint32_t *outl;      // [nodes] nearest pattern end on the failure chain (root = none)
  uint32_t *own;       // [nodes] patterns ending exactly here
  uint32_t *total;     // [nodes] matches reported in this state
  uint32_t *end_node;  // [P]
  GridBarrier bar;
  uint32_t *err;
};

constexpr int kBuildThreads = 512;

// Level d: inserter p creates or finds its depth-(d+1) node; linker p, if
// pattern p created its depth-d node one level earlier, computes that node's
// failure link, output link and match total (all shallower nodes and all
// depth-d nodes exist after the previous barrier).
__global__ void __launch_bounds__(kBuildThreads) k_ac_build(BuildArgs a) {
  const uint32_t half = gridDim.x * blockDim.x / 2;
  const uint32_t gt0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool inserter = gt0 < half;
  const uint32_t gt = inserter ? gt0 : gt0 - half;
  const uint32_t root = a.root;
  for (uint32_t d = 0; d <= a.maxlen; ++d) {
    const int par = d & 1;
    for (uint32_t p = gt; p < a.P; p += half) {
      const uint32_t L = a.plen[p];
      if (inserter) {
        if (d >= L) continue;
        const uint32_t u = d ? a.cur[par][p] : root;
        const uint32_t c = a.psym[a.pstart[p] + d];
        const uint64_t key = ((uint64_t)u << 32) | c;
        uint64_t slot = mix64(key) & a.g.mask;
        uint32_t v = kNil;
        uint8_t made = 0;
        for (uint64_t probe = 0; probe <= a.g.mask; ++probe) {
          uint64_t *ek = a.g.keys + 2 * slot;
          uint64_t cur = *(volatile uint64_t *)ek;
          if (cur == kEmpty) {
            cur = atomicCAS((unsigned long long *)ek, (unsigned long long)kEmpty,
                            (unsigned long long)key);
            if (cur == kEmpty) {  // this pattern creates the node
              v = (uint32_t)slot;
              made = 1;
              ek[1] = v;
              a.parent[v] = u;
              a.nsym[v] = c;
              break;
            }
          }
          if (cur == key) {
            v = (uint32_t)slot;
            break;
          }
          slot = (slot + 1) & a.g.mask;
        }
        if (v == kNil) {
          atomicExch(a.err, kDevRange);
          continue;
        }
        a.cur[par ^ 1][p] = v;
        a.made[par ^ 1][p] = made;
        if (d + 1 == L) {
          a.end_node[p] = v;
          atomicAdd(&a.own[v], 1u);
        }
      } else {
        if (d == 0 || d > L || !a.made[par][p]) continue;
        const uint32_t v = a.cur[par][p];
        uint32_t f = root;
        if (d > 1) {
          const uint32_t c = a.nsym[v];
          uint32_t w = a.fail[a.parent[v]];
          while (true) {
            const uint32_t x = goto_lookup(a.g, w, c);
            if (x != kNil) {
              f = x;
              break;
            }
            if (w == root) break;
            w = a.fail[w];
          }
        }
        a.fail[v] = f;
        // total[f] = own[f] + total[outl[f]], so whichever of f and outl[f]
        // is v's output link, the matches reported down it number total[f]
        const uint32_t of = a.own[f];
        a.outl[v] = (f != root && of != 0) ? f : a.outl[f];
        a.total[v] = a.own[v] + a.total[f];
      }
    }
    grid_sync(a.bar, a.err);
    if (*(volatile uint32_t *)a.err != kDevOk) return;
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

__global__ void k_mark_ends(const uint64_t *__restrict__ skeys, uint32_t P, uint32_t *end_first) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x)
    if (k == 0 || skeys[k] != skeys[k - 1]) end_first[(uint32_t)skeys[k]] = k;
}

// ---------------------------------------------------------------- match
// One goto probe or one failure step per loop iteration, so that the lanes
// of a warp advance through their chunks independently instead of waiting at
// every token for the lane with the longest failure chain.

// Pass A1: chunk t = positions [t*chunk, (t+1)*chunk) from the root state.
// Chunk 0 is exact; the others may start in the wrong state.
__global__ void k_ac_states(const uint32_t *__restrict__ ssym, uint64_t n, uint64_t chunk, Table g,
                            const uint32_t *__restrict__ fail, uint32_t *__restrict__ state_out,
                            uint32_t *__restrict__ end_state) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t cs = t * chunk;
  if (cs >= n) return;
  const uint64_t ce = min(n, cs + chunk);
  const uint32_t root = (uint32_t)(g.mask + 1);
  uint32_t state = root, cur = root;  // cur: where the transition for x is being looked up
  uint64_t x = cs;
  uint32_t c = ssym[x];
  while (x < ce) {
    const uint32_t nx = goto_lookup(g, cur, c);
    if (nx != kNil || cur == root) {
      state = nx != kNil ? nx : root;
      state_out[x] = state;
      cur = state;
      if (++x < ce) c = ssym[x];
    } else {
      cur = fail[cur];
    }
  }
  end_state[t] = state;
}

// Pass A2 (repeated until nothing changes): chunk t restarts from the end
// state of chunk t-1 and re-runs until its state equals the recorded one
// (the automaton is deterministic, so the rest of the chunk already agrees).
// After k passes chunks 0..k are exact; the host stops when no end state
// changed.
__global__ void k_ac_fix(const uint32_t *__restrict__ ssym, uint64_t n, uint64_t chunk, Table g,
                         const uint32_t *__restrict__ fail, uint32_t *__restrict__ state_out,
                         const uint32_t *__restrict__ end_in, uint32_t *__restrict__ end_out,
                         uint32_t *changed) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t cs = t * chunk;
  if (cs >= n) return;
  if (t == 0) {
    end_out[0] = end_in[0];
    return;
  }
  const uint64_t ce = min(n, cs + chunk);
  const uint32_t root = (uint32_t)(g.mask + 1);
  uint32_t state = end_in[t - 1], cur = state;
  uint64_t x = cs;
  uint32_t c = ssym[x];
  while (x < ce) {
    const uint32_t nx = goto_lookup(g, cur, c);
    if (nx != kNil || cur == root) {
      state = nx != kNil ? nx : root;
      if (state_out[x] == state) {
        end_out[t] = end_in[t];
        return;
      }
      state_out[x] = state;
      cur = state;
      if (++x < ce) c = ssym[x];
    } else {
      cur = fail[cur];
    }
  }
  end_out[t] = state;
  if (state != end_in[t]) atomicAdd(changed, 1u);
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

// Pass B: the matches of position x, down the output chain from its state
// (deepest first), ids ascending within a node.
__global__ void k_ac_fill(const uint32_t *__restrict__ state, uint32_t n,
                          const uint32_t *__restrict__ off, const uint32_t *__restrict__ own,
                          const uint32_t *__restrict__ outl, const uint32_t *__restrict__ end_first,
                          const uint32_t *__restrict__ evals, uint32_t *mend, uint32_t *mid,
                          uint64_t cap, uint32_t root) {
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const uint32_t s0 = state[x];
    uint64_t o = off[x];
    uint32_t v = own[s0] != 0 ? s0 : outl[s0];
    while (v != root) {
      const uint32_t k0 = end_first[v], k1 = k0 + own[v];
      for (uint32_t k = k0; k < k1; ++k) {
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

inline int grid_for(uint64_t n, int threads, int sms) {
  long long b = (long long)((n + threads - 1) / threads);
  return (int)std::max<long long>(1, std::min<long long>(b, (long long)sms * 16));
}

int g_build_blocks = 0;  // most co-resident blocks of k_ac_build for a cooperative launch

}  // namespace

int match_init(int sms) {
  // The level barrier's cost grows with the number of arriving blocks, so
  // launches use no more blocks than the pattern count needs.
  int per_sm = 0;
  APO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ac_build, kBuildThreads, 0));
  g_build_blocks = std::max(1, per_sm * sms);
  return APO_OK;
}

size_t match_workspace_bytes(uint64_t total_tokens, uint64_t P, uint64_t n, uint64_t extent) {
  uint64_t tbl = 1;
  while (tbl < 2 * (total_tokens + 1)) tbl <<= 1;
  uint64_t dct = 1;
  while (dct < 2 * (extent + 1)) dct <<= 1;
  const uint64_t N = tbl + 1;
  const uint64_t chunks = n / 32 + 2;
  return tbl * 16 + dct * 12 + N * 4 * 8 + P * 64 + (extent + n) * 4 + n * 8 + chunks * 8 +
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
  if (total >= 0xffffffffull || extent >= 0xffffffffull) {
    set_error("match_candidates: more than 2^32 - 1 pattern tokens");
    return APO_EINVAL;
  }
  APO_TRY(c->arena.reserve(match_workspace_bytes(total, P, n, extent)));
  const uint64_t N0 = total + 1;  // node bound (root included)
  uint64_t tbl = 1;
  while (tbl < 2 * N0) tbl <<= 1;
  const uint64_t N = tbl + 1;     // node ids are goto slots; the root is `tbl`
  const uint32_t root = (uint32_t)tbl;

  Table g;
  g.keys = c->arena.take_n<uint64_t>(2 * tbl);
  g.mask = tbl - 1;
  uint32_t *pbuf = pp->pat_off ? c->arena.take_n<uint32_t>(2 * (size_t)P) : nullptr;
  uint32_t *parent = c->arena.take_n<uint32_t>(N);
  uint32_t *nsym = c->arena.take_n<uint32_t>(N);
  uint32_t *fail = c->arena.take_n<uint32_t>(N);
  uint32_t *outl = c->arena.take_n<uint32_t>(N);
  uint32_t *own = c->arena.take_n<uint32_t>(N);
  uint32_t *mtotal = c->arena.take_n<uint32_t>(N);
  uint32_t *end_first = c->arena.take_n<uint32_t>(N);
  uint32_t *cur = c->arena.take_n<uint32_t>(2 * (size_t)P);
  uint8_t *made = c->arena.take_n<uint8_t>(2 * (size_t)P);
  uint32_t *end_node = c->arena.take_n<uint32_t>(P);
  SortBuffers b;
  b.keys[0] = c->arena.take_n<uint64_t>(P);
  b.keys[1] = c->arena.take_n<uint64_t>(P);
  b.vals[0] = c->arena.take_n<uint32_t>(P);
  b.vals[1] = c->arena.take_n<uint32_t>(P);
  if (!g.keys || (pp->pat_off && !pbuf) || !parent || !nsym || !fail || !outl || !own ||
      !mtotal || !end_first || !cur || !made || !end_node || !b.keys[0] || !b.keys[1] || !b.vals[0] ||
      !b.vals[1]) {
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
  {  // every entry: key = empty, value = 0
    Launch lp_(c, kKDepthKeys, tbl, s);
    k_table_init<<<grid_for(tbl, 256, sms), 256, 0, s>>>(g.keys, tbl);
  }
  APO_CUDA_TRY(cudaMemsetAsync(own, 0, N * sizeof(uint32_t), s));
  {  // the root fails to itself, has no output link and reports nothing
    const uint32_t rv[3] = {root, root, 0u};
    APO_CUDA_TRY(cudaMemcpyAsync(fail + root, &rv[0], 4, cudaMemcpyHostToDevice, s));
    APO_CUDA_TRY(cudaMemcpyAsync(outl + root, &rv[1], 4, cudaMemcpyHostToDevice, s));
    APO_CUDA_TRY(cudaMemcpyAsync(mtotal + root, &rv[2], 4, cudaMemcpyHostToDevice, s));
    APO_CUDA_TRY(cudaStreamSynchronize(s));
  }

  // symbols of the pattern source and of the stream
  const uint32_t *psym = nullptr, *ssym = nullptr;
  if (tb == 4) {
    psym = static_cast<const uint32_t *>(pp->tokens);
    ssym = static_cast<const uint32_t *>(stream);
  } else {
    uint64_t dct = 1;
    while (dct < 2 * (extent + 1)) dct <<= 1;
    Dict d;
    d.keys = c->arena.take_n<uint64_t>(dct);
    d.mask = dct - 1;
    const bool same = pp->tokens == stream && n >= extent;
    uint32_t *ps = c->arena.take_n<uint32_t>(std::max<uint64_t>(same ? n : extent, 1));
    uint32_t *ss = same ? ps : c->arena.take_n<uint32_t>(std::max<uint64_t>(n, 1));
    if (!d.keys || !ps || !ss) return APO_ENOMEM;
    APO_CUDA_TRY(cudaMemsetAsync(d.keys, 0xff, dct * sizeof(uint64_t), s));
    const uint64_t *pt = static_cast<const uint64_t *>(pp->tokens);
    {
      Launch lp_(c, kKU64Keys, extent, s);
      k_dict_insert<<<grid_for(extent, 256, sms), 256, 0, s>>>(pt, extent, d);
    }
    {
      Launch lp_(c, kKUnique, same ? n : extent, s);
      k_dict_map<<<grid_for(same ? n : extent, 256, sms), 256, 0, s>>>(pt, same ? n : extent, d, ps);
    }
    if (!same) {
      Launch lp_(c, kKUnique, n, s);
      k_dict_map<<<grid_for(n, 256, sms), 256, 0, s>>>(static_cast<const uint64_t *>(stream), n, d, ss);
    }
    psym = ps;
    ssym = ss;
  }

  // trie, failure / output links and match totals, level by level
  APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscMatchCount, 0, 3 * sizeof(uint32_t), s));
  {
    BuildArgs a;
    a.psym = psym;
    a.pstart = pstart;
    a.plen = plen;
    a.P = P;
    a.maxlen = (uint32_t)maxlen;
    a.g = g;
    a.root = root;
    a.cur[0] = cur;
    a.cur[1] = cur + P;
    a.made[0] = made;
    a.made[1] = made + P;
    a.parent = parent;
    a.nsym = nsym;
    a.fail = fail;
    a.outl = outl;
    a.own = own;
    a.total = mtotal;
    a.end_node = end_node;
    a.bar.count = misc + kMiscMatchCount + 1;
    a.bar.gen = misc + kMiscMatchCount + 2;
    a.err = c->ps.err;
    void *args[] = {&a};
    Launch lp_(c, kKTrieInsert, total, s);
    // one inserter and one linker thread per pattern where possible, at least
    // 32 blocks, at most what is co-resident (larger sets loop)
    const int blocks = std::min<int>(g_build_blocks, std::max<int>(32, ceil_div(2ull * P, kBuildThreads)));
    APO_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_ac_build, blocks, kBuildThreads, args, 0, s));
  }
  APO_CUDA_TRY(cudaGetLastError());
  // pattern ids grouped by end node
  {
    Launch lp_(c, kKEndPairs, P, s);
    k_end_pairs<<<grid_for(P, 256, sms), 256, 0, s>>>(end_node, P, b.keys[0], b.vals[0]);
  }
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  APO_TRY(check_device_error(c, s));
  b.cur = 0;
  {
    int places[8];
    const int np = plan_digits(0, bits_for(root), places, 0);
    APO_TRY(radix_sort_pairs(c, b, P, places, np, s));
  }
  const uint64_t *ek = b.keys[b.cur];
  const uint32_t *ev = b.vals[b.cur];
  {
    Launch lp_(c, kKMarkEnds, P, s);
    k_mark_ends<<<grid_for(P, 256, sms), 256, 0, s>>>(ek, P, end_first);
  }
  if (n == 0) return APO_OK;

  // pass A: states, chunked without a halo, then repaired until stable
  uint32_t *state = c->arena.take_n<uint32_t>(n);
  uint32_t *off = c->arena.take_n<uint32_t>(n);
  // short chunks: a chunk is a chain of dependent lookups, so its length is
  // the pass time; repair passes cost little once chunks end in a reset
  const uint64_t chunk = std::max<uint64_t>(32, std::min<uint64_t>(512, n / ((uint64_t)sms * 64)));
  const uint64_t nch = (n + chunk - 1) / chunk;
  uint32_t *ends[2] = {c->arena.take_n<uint32_t>(nch), c->arena.take_n<uint32_t>(nch)};
  if (!state || !off || !ends[0] || !ends[1]) return APO_ENOMEM;
  {
    Launch lp_(c, kKAcMatch, n, s);
    k_ac_states<<<ceil_div(nch, 64), 64, 0, s>>>(ssym, n, chunk, g, fail, state, ends[0]);
  }
  for (uint64_t pass = 0, e = 0; pass < nch; ++pass, e ^= 1) {
    APO_CUDA_TRY(cudaMemsetAsync(misc + kMiscAccCount, 0, sizeof(uint32_t), s));
    {
      Launch lp_(c, kKFailLevel, n, s);
      k_ac_fix<<<ceil_div(nch, 64), 64, 0, s>>>(ssym, n, chunk, g, fail, state, ends[e], ends[e ^ 1],
                                                   misc + kMiscAccCount);
    }
    APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned, misc + kMiscAccCount, 4, cudaMemcpyDeviceToHost, s));
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
    k_ac_fill<<<grid_for(n, 256, sms), 256, 0, s>>>(state, (uint32_t)n, off, own, outl, end_first, ev,
                                                    match_end, match_id, cap, root);
  }
  APO_CUDA_TRY(cudaGetLastError());
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(c, s);
}

}  // namespace apo
