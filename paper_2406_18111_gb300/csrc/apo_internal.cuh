// Internal declarations shared by the libapo translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/apo.h"

namespace apo {

// ---------------------------------------------------------------- errors
// Device error word values (set by kernels, read by the host at sync points).
enum : uint32_t {
  kDevOk = 0,
  kDevTimeout = 1,   // a bounded spin gave up
  kDevRange = 2,     // an index fell outside its array
};

// Iterations after which a device-side spin wait gives up (with back-off this
// bounds a wait to well under a second).
constexpr uint32_t kSpinLimit = 1u << 22;

void set_error(const std::string &msg);

#define APO_CUDA_TRY(expr)                                                         \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::apo::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));        \
      return APO_ECUDA;                                                            \
    }                                                                              \
  } while (0)

#define APO_TRY(expr)          \
  do {                         \
    int r_ = (expr);           \
    if (r_ != APO_OK) return r_; \
  } while (0)

// ---------------------------------------------------------------- workspace
// A bump allocator over one device buffer owned by the context.  reserve()
// grows the buffer (cudaMalloc) only between calls, never inside a stream's
// pending work; take() hands out 256-byte aligned slices.
struct Arena {
  char *base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  uint64_t moves = 0;  // reallocations so far
  bool external = false;  // base/cap lie in a caller-owned workspace: never reallocated
  int reserve(size_t bytes);
  void reset() { used = 0; }
  void *take(size_t bytes);
  template <class T>
  T *take_n(size_t n) { return static_cast<T *>(take(n * sizeof(T))); }
};

// Layout of the context's small device counter buffer (u32 words).
enum : int {
  kCtrSortHist = 0,       // radix sort digit histograms, 12 places x 512 digits
  kCtrSortTiles = 6144,   // radix sort tile tickets, 12
  kCtrMisc = 6208,        // per-kernel tile tickets and totals, see kMisc*
  kCtrWords = 8192,
};
enum : int {
  kMiscRefreshTiles = 0, kMiscRefreshCount, kMiscCompactTiles, kMiscCompactCount,
  kMiscCandCount, kMiscMaxLen, kMiscAccCount, kMiscTraceCount, kMiscMatchCount,
  kMiscKeyOr = 16,        // two u64 (four words): OR and maximum of keys
  kMiscRound = 20,        // two words: active-suffix counts of consecutive doubling rounds
  kMiscDict = 22,         // two words: distinct tokens, dictionary overflow flag
  kMiscPhaseLen = 24,     // two words: list lengths of consecutive greedy phases
  kMiscFixChanged = 26,   // two words: changes of consecutive automaton repair passes
  kMiscFlatTotal = 28,    // length of the flattened output chains
  kMiscCandUnique = 29,   // candidates left after deduplication
  kMiscRoundTiles = 30,   // tile tickets of a doubling round
  kMiscRoundW = 32,       // 2 x 4 words of consecutive doubling rounds (see build_suffix_array)
  kMiscCount = 64,
};

// Per-context persistent device state.
struct Persistent {
  uint32_t *err = nullptr;        // device error word
  uint64_t *lookback = nullptr;   // decoupled look-back status words
  size_t lookback_words = 0;
  uint32_t *counters = nullptr;   // small scratch counters (tile ids, totals)
  uint32_t epoch = 0;             // look-back epoch, bumped per launch
};

// ---------------------------------------------------------------- instrumentation
enum KernelId : int {
  kKHash, kKInitKeys, kKKeyOr, kKRsHist, kKRsOffsets, kKRsPass, kKRefresh, kKPack, kKPhi,
  kKPlcp, kKLcpPerm, kKMin32, kKMax, kKCandGen, kKCompact, kKCandGather, kKGreedy, kKTraces,
  kKSelOut, kKPatLayout, kKTableInit, kKEndPairs, kKMarkEnds, kKAcFix, kKAcStates,
  kKAcFill, kKDictInsert, kKDictMap, kKSlices, kKMatchOffsets, kKSegScan, kKStarts, kKSparse,
  kKAcNodes, kKAcJump, kKRsTune, kKRpPieces, kKRpNeed, kKRpChain, kKRpAppear, kKRpSelect, kKRpOut,
  kKOptimum, kKSaDict, kKRound, kKSplit, kKWsb, kKListCompact, kKMinor, kKRsPassKeys, kKAcHalo, kKCount
};
extern const char *const kKernelNames[kKCount];

// Launch records are kept per scope, so that the same kernel on different
// stages never mixes: scope 0 is the call's own path (hashing, the suffix
// array and LCP of the analysed windows, the replayer), scope 1 everything
// the matcher launches ("ac." prefix), scope 2 the repeat selection after
// the LCP ("rep." prefix: candidates, their sort, greedy loop, R).
constexpr int kScopes = 3;
enum : int { kScopeOwn = 0, kScopeMatch = 1, kScopeRepeats = 2 };

struct Profiler {
  bool timing = false;
  int scope = 0;
  uint64_t launches[kScopes * kKCount] = {};
  uint64_t units[kScopes * kKCount] = {};
  double ms[kScopes * kKCount] = {};
  struct Pending {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  // A launch sized for an upper bound records the bound as its units; once
  // the exact count is known the difference is taken off again.
  void adjust(int id, int64_t delta) { units[id + scope * kKCount] += (uint64_t)delta; }
  cudaEvent_t get();
  int resolve();
  void release();
};

}  // namespace apo

namespace apo {

// Radix-sort launch shape per (size class, key bits): chosen by timing every
// shape the first time a class is sorted on a device (mode 0), always the
// default shape (mode 1), or always shape k (mode 2 + k).  The choices are shared by all contexts of the
// process on the same device (sort_table()).
constexpr int kTuneMinBits = 10, kTuneMaxBits = 23;  // size classes: n <= 2^10 .. n > 2^22
constexpr int kTuneClasses = kTuneMaxBits - kTuneMinBits + 1;
constexpr int kTuneBits = 97;  // sorted bits 0..96 (key and value digits together)
struct SortTable {
  int8_t choice[kTuneClasses][kTuneBits];
  float best_ms[kTuneClasses][kTuneBits] = {};
  float default_ms[kTuneClasses][kTuneBits] = {};
  uint32_t trial_n[kTuneClasses][kTuneBits] = {};
  SortTable() {
    for (auto &row : choice)
      for (auto &x : row) x = -1;
  }
};
// The device's table; `lock` guards every read and write of it.
SortTable &sort_table(int device);
void sort_table_lock(bool lock);
struct SortTuner {
  int mode = 0;
  void *scratch = nullptr;  // trial pairs
  size_t scratch_bytes = 0;
  static int size_class(uint32_t n);
};

}  // namespace apo

namespace apo {
// Host reads of a call, for replaying the call as a CUDA graph.  While a call
// is recorded, every value the host reads back from the device (a count, a
// code width, the error word) is appended to `vals`; while the same call is
// captured into a graph, those reads take the recorded values in the same
// order and queue a check of the device words at that point of the stream
// instead (a difference counts into the device word `bad`: the replay's
// results are then discarded).  `stage` (pinned) receives the per-window
// output offsets a capture copies back, `upload` (pinned) holds the window
// offsets a capture copies in.
struct Tape {
  int mode = 0;
  std::vector<uint32_t> vals;
  size_t pos = 0;
  uint32_t *dev_vals = nullptr;
  uint32_t *bad = nullptr;
  uint32_t *stage = nullptr;
  uint32_t *upload = nullptr;
};
enum : int { kTapeOff = 0, kTapeRecord = 1, kTapeCapture = 2 };
struct GraphCache;
}  // namespace apo

struct apo_ctx {
  int device = 0;
  int num_sms = 0;
  apo::Arena arena;
  apo::Persistent ps;
  apo::Profiler prof;
  apo::SortTuner tuner;
  uint32_t *host_pinned = nullptr;  // small pinned staging buffer (counts)
  void *side = nullptr;             // grow-only buffer for sizes known only mid-call
  size_t side_bytes = 0;
  cudaEvent_t round_ev[2] = {nullptr, nullptr};  // doubling-round count read-backs
  cudaStream_t aux = nullptr;                     // a second stream for independent launches
  cudaEvent_t fork_ev[2] = {nullptr, nullptr};    // fork to it, join back
  void *rp[3] = {nullptr, nullptr, nullptr};     // trace replay buffers (grow-only)
  size_t rp_bytes[3] = {0, 0, 0};
  uint64_t rp_cap = 0;                            // occurrences the replay buffers hold
  apo::Tape *tape = nullptr;                      // active tape of a recorded or captured call
  uint64_t gen = 0;                               // bumped when a workspace buffer moves
  int graph_mode = 0;                             // replay batched calls as CUDA graphs
  apo::GraphCache *graphs = nullptr;
  // A caller-owned workspace (apo_set_workspace): look-back words at its
  // start (zeroed up to ext_lb_bytes), the arena after them.  While one is
  // attached the context's own arena and look-back array are set aside here.
  char *ext = nullptr;
  size_t ext_bytes = 0, ext_lb_bytes = 0;
  char *own_base = nullptr;
  size_t own_cap = 0;
  uint64_t *own_lookback = nullptr;
  size_t own_lookback_words = 0;
};

namespace apo {

// Launches counted under `scope` while alive (restores the previous scope).
struct ScopeGuard {
  apo_ctx *c;
  int prev;
  ScopeGuard(apo_ctx *c_, int scope);
  ~ScopeGuard();
  ScopeGuard(const ScopeGuard &) = delete;
  ScopeGuard &operator=(const ScopeGuard &) = delete;
};

// Counts one kernel launch and, with timing enabled, brackets it with CUDA
// events on the launch stream.  Construct it right before the launch.
class Launch {
 public:
  Launch(apo_ctx *c, int id, uint64_t units, cudaStream_t s);
  ~Launch();
  Launch(const Launch &) = delete;
  Launch &operator=(const Launch &) = delete;

 private:
  apo_ctx *c_;
  int id_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

}  // namespace apo

namespace apo {

// Next look-back epoch (30 bits, never 0).
inline uint32_t next_epoch(apo_ctx *c) {
  c->ps.epoch = (c->ps.epoch + 1) & 0x3fffffffu;
  if (c->ps.epoch == 0) c->ps.epoch = 1;
  return c->ps.epoch;
}

int ensure_lookback(apo_ctx *c, size_t words);
// Sizes the call's scratch: an arena of arena_bytes and a look-back array of
// lb_words (grown with cudaMalloc, or laid out in the caller's workspace).
int reserve_workspace(apo_ctx *c, size_t arena_bytes, size_t lb_words, cudaStream_t s);
// Scratch of apo_find_repeats / _batched over n tokens in `windows` windows.
void find_repeats_need(uint64_t n, uint64_t windows, size_t *arena_bytes, size_t *lb_words);
// Grows the context's side buffer to `bytes` (waits for the stream first).
int ensure_side(apo_ctx *c, size_t bytes, cudaStream_t s);
int check_device_error(apo_ctx *c, cudaStream_t s);
// Pinned slot that receives the device error word alongside a count read.
constexpr int kPinnedErr = 15;
int device_error_status(apo_ctx *c, cudaStream_t s);

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
// Blocks for a grid-stride loop over n elements: enough for one element per
// thread, at most 16 blocks per SM.
inline int grid_for(uint64_t n, int threads, int sms) {
  long long b = (long long)((n + threads - 1) / threads);
  return (int)std::max<long long>(1, std::min<long long>(b, (long long)sms * 16));
}
inline int bits_for(uint64_t v) {  // number of bits to represent values 0..v
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

// ---------------------------------------------------------------- radix sort
// Stable LSD sort of (key u64, value u32) pairs on the bit ranges listed in
// `ranges`, least significant first (a range of value bits sorts by the
// value).  The result lands in (*keys, *vals); the other buffer of each pair
// is scratch.  The digit width and tile shape come from the context's tuner.
struct SortBuffers {
  uint64_t *keys[2];
  uint32_t *vals[2];
  int cur = 0;  // index of the buffer holding the current data
};
struct DigitRange {
  int lo, hi;       // bits [lo, hi) of the key (or of the value)
  bool from_value;
};
constexpr int kFromValue = 256;  // place flag: the digit comes from the value
// With n_dev, the element count is the device word *n_dev and n only bounds
// the launch (so a sort can be queued before its count reaches the host).
int radix_sort_pairs(apo_ctx *c, SortBuffers &b, uint32_t n, const DigitRange *ranges, int nranges,
                     cudaStream_t s, const uint32_t *n_dev = nullptr);
// The same in two steps, for a caller that counts the first digit place
// while it writes the keys: sort_plan picks the shape (tuning it if needed)
// and the places; the caller clears sort_first_hist() (sort_first_hist_clear),
// adds the counts of place[0] (digit width `bits`) into it, and runs
// radix_sort_planned with hist_ready.
struct SortPlan {
  int shape = -1, bits = 8, places = 0;
  int place[12];
};
int sort_plan(apo_ctx *c, uint32_t n, const DigitRange *ranges, int nranges, SortPlan *out, cudaStream_t s);
int sort_first_hist_clear(apo_ctx *c, cudaStream_t s);
uint32_t *sort_first_hist(apo_ctx *c);
int radix_sort_planned(apo_ctx *c, SortBuffers &b, uint32_t n, const SortPlan &sp, cudaStream_t s,
                       const uint32_t *n_dev, bool hist_ready);
// OR of all keys (how many digits are populated) in out_dev[0] and their
// maximum in out_dev[1]; both words must be zero on entry.
void launch_key_or(apo_ctx *c, const uint64_t *keys, uint32_t n, uint64_t *out_dev, cudaStream_t s);
int radix_sort_init();
int sort_shape_info(int id, int *threads, int *items, int *bits);
int sort_shape_count();

// ---------------------------------------------------------------- windows
// Several windows analysed at once are concatenated; position i belongs to
// window wid[i], which ends at wend[i] (exclusive, in concatenated
// coordinates).  Null arrays mean one window spanning all positions.
struct Windows {
  uint32_t count = 1;
  const uint32_t *wid = nullptr;    // [N]
  const uint32_t *wend = nullptr;   // [N]
  const uint64_t *off_host = nullptr;  // [count + 1] window offsets (host)
  const uint32_t *off_dev = nullptr;   // [count + 1] window offsets (device)
  uint32_t max_len = 0;             // longest window
};

__device__ __forceinline__ uint32_t win_end(const Windows &w, uint32_t i, uint32_t n) {
  return w.wend ? w.wend[i] : n;
}
__device__ __forceinline__ uint32_t win_id(const Windows &w, uint32_t i) {
  return w.wid ? w.wid[i] : 0u;
}

// ---------------------------------------------------------------- suffix array
struct SuffixState {
  uint32_t n;        // positions over all windows
  uint32_t *sa;      // global SA: window w's suffixes occupy [off[w], off[w+1])
  uint32_t *rank;
  uint32_t **snaps;  // host array of device pointers, snaps[k] = snaps[0] + k * n: level-k ranks
                     // of the suffixes still grouped at the start of round k (fin >= k)
  int levels;        // number of levels written
  Windows win;
  uint32_t h0 = 1;   // tokens per initial key: level k ranks are equal iff h0 * 2^k tokens are
  uint8_t *fin = nullptr;    // level at which each suffix became final (0xff: not yet)
  uint32_t *wsb = nullptr;   // window-start bits (bit n set), null for one window
};
int build_suffix_array(apo_ctx *c, const void *tokens, int token_bytes, uint32_t n,
                       SuffixState &st, int max_levels, uint32_t *rounds_out, cudaStream_t s);
int build_lcp(apo_ctx *c, const void *tokens, int token_bytes, const SuffixState &st,
              uint32_t *lcp, cudaStream_t s);

// ---------------------------------------------------------------- repeats
// Per-window outputs of a batched call (HOST offset arrays, count + 1 each).
struct BatchOffsets {
  uint64_t *cand_off = nullptr;
  uint64_t *sel_off = nullptr;
  uint64_t *trace_off = nullptr;
};
int find_repeats_from_sa(apo_ctx *c, const void *tokens, int token_bytes, const SuffixState &st,
                         const uint32_t *lcp, uint32_t min_len, apo_repeats_out *out,
                         const BatchOffsets *boff, cudaStream_t s);

// ---------------------------------------------------------------- hashing
void launch_hash_tasks(apo_ctx *c, const apo_tasks *t, uint64_t *out, cudaStream_t s);

// ---------------------------------------------------------------- served form
int server_token_bytes(apo_server *s);

// ---------------------------------------------------------------- matching
// With aux_order / aux_slcp (device, P entries each) it also returns the
// patterns in string order (aux_order[j] = pattern id; equal strings by
// increasing id) and aux_slcp[j] = lcp of the patterns at j - 1 and j
// (aux_slcp[0] = 0).
int match_patterns(apo_ctx *c, const apo_patterns *p, const void *stream_tokens, uint64_t n,
                   uint32_t *match_end, uint32_t *match_id, uint64_t cap, uint64_t *count,
                   cudaStream_t s, uint32_t *aux_order = nullptr, uint32_t *aux_slcp = nullptr);

// ---------------------------------------------------------------- call tapes
inline bool capturing(const apo_ctx *c) { return c->tape && c->tape->mode == kTapeCapture; }
inline bool recording(const apo_ctx *c) { return c->tape && c->tape->mode == kTapeRecord; }
// Recording: append `words` values the host has read.
void tape_put(apo_ctx *c, const uint32_t *vals, int words);
// Capturing: the next `words` recorded values into host[], and a check that
// the device words at `dev` hold them at this point of the stream.
int tape_take(apo_ctx *c, const uint32_t *dev, uint32_t *host, int words, cudaStream_t s);
void graph_cache_free(apo_ctx *c);
void graph_stats(apo_ctx *c, uint64_t *replays, uint64_t *captures, uint64_t *discarded);
namespace drv {
int find_repeats_driver(apo_ctx *c, const void *tokens, int tb, uint64_t total, const uint64_t *win_off,
                        uint32_t nwin, const apo_repeats_params *p, apo_repeats_out *out, cudaStream_t s);
}
int graph_batched(apo_ctx *c, const apo_windows *ws, const apo_repeats_params *p, apo_repeats_out *out,
                  cudaStream_t s);

// ---------------------------------------------------------------- trace replay
int replay_stream(apo_ctx *c, const void *tokens, uint64_t n, int token_bytes, const apo_replay_traces *tr,
                  const apo_replay_params *prm, apo_replay_out *out, cudaStream_t s);

// ---------------------------------------------------------------- Sec. 3 optimum
int optimum_batched(apo_ctx *c, const apo_windows *ws, uint32_t min_len, uint32_t *best, uint32_t *wstart,
                    uint32_t *wlen, uint32_t *wcount, cudaStream_t s);

}  // namespace apo
