/*
 * apo.h -- C ABI of libapo, the GPU trace finder.
 *
 * The library computes the string analysis at the heart of automatic trace
 * identification (Yadav et al., "Automatic Tracing in Task-Based Runtime
 * Systems", ASPLOS 2025): task descriptors are hashed to tokens (Alg. 1,
 * Sec. 4.1), a window of tokens is turned into non-overlapping repeated
 * sub-strings (Alg. 2, Sec. 4.2), and the resulting candidate traces are
 * matched against a token stream (Sec. 4.3).  All work runs in CUDA kernels
 * on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Array arguments are DEVICE pointers owned by the caller unless a
 *     function says otherwise; the library never frees them.
 *   - Calls are issued on the CUDA stream `stream` (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream).  Functions that must learn a
 *     data-dependent size before they can continue synchronise that stream;
 *     each function documents whether it returns before the work finishes.
 *   - Every function returns an apo_status.  On failure, apo_last_error()
 *     returns a message for the calling thread.  Errors detected inside a
 *     kernel (a device wait that gave up, an index out of range) are
 *     reported by the next call that synchronises, as APO_ETIMEOUT or
 *     APO_EDEVICE.
 *   - Sizes: a window holds at most 2^31 - 1 tokens.
 *   - A context owns the device scratch memory ("workspace") of the calls
 *     made with it and grows it on demand with cudaMalloc; it is bound to
 *     the device that was current when it was created.  A context must not
 *     be used by two host threads at the same time.
 */
#ifndef APO_H
#define APO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  APO_OK = 0,
  APO_EINVAL = -1,     /* a bad argument (null pointer, bad size or token width) */
  APO_ENOMEM = -2,     /* device memory could not be allocated */
  APO_ECAPACITY = -3,  /* an output array is too small; the needed count is still written */
  APO_ECUDA = -4,      /* a CUDA runtime call failed */
  APO_ETIMEOUT = -5,   /* a bounded device-side wait gave up (the results are invalid) */
  APO_EDEVICE = -6,    /* a kernel detected an inconsistency (the results are invalid) */
  APO_EAGAIN = -7      /* not ready yet (a served request still in flight) */
} apo_status;

typedef struct apo_ctx apo_ctx;

/* Create a context on `device` (a CUDA ordinal).  The device becomes current
 * for the calling thread. */
int apo_create(apo_ctx **ctx, int device);

/* Release a context and the workspace it owns.  NULL is accepted. */
int apo_destroy(apo_ctx *ctx);

/* Message describing the last failure on the calling thread ("" if none). */
const char *apo_last_error(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int apo_version(void);

/* ------------------------------------------------------------------------
 * Task hashing -- Alg. 1 "Hash(T)", Sec. 4.1; what a task is: Sec. 2
 * (a task id plus its ordered region arguments, whose regions, fields and
 * privileges all affect the dependence analysis).
 *
 * token[t] = FNV-1a-64 over the little-endian bytes
 *     task_id[t]:u32, nargs:u32,
 *     then for a in arg_off[t] .. arg_off[t+1]-1:
 *         region[a]:u32, field_mask[a]:u64, priv[a]:u8
 * where nargs = arg_off[t+1] - arg_off[t].
 * ---------------------------------------------------------------------- */
typedef struct {
  uint64_t n_tasks;           /* N */
  const uint32_t *task_id;    /* [N] */
  const uint32_t *arg_off;    /* [N+1], non-decreasing CSR offsets into the argument arrays */
  const uint32_t *region;     /* [arg_off[N]] */
  const uint64_t *field_mask; /* [arg_off[N]] */
  const uint8_t *priv;        /* [arg_off[N]] */
} apo_tasks;

/* Hash N task descriptors to tokens_out[N] (device).  Asynchronous: returns
 * after enqueueing.  N = 0 is a no-op.  APO_EINVAL if a pointer needed for
 * N > 0 is NULL. */
int apo_hash_tasks(apo_ctx *ctx, const apo_tasks *tasks, uint64_t *tokens_out, void *stream);

/* ------------------------------------------------------------------------
 * Repeat finding -- Alg. 2 "FindRepeats(S)", Sec. 4.2.
 *
 * For one window S of n tokens (u32 or u64, compared as unsigned integers):
 *   SA   suffix array; a suffix that is a proper prefix of another sorts first.
 *   LCP  LCP[i] = longest common prefix of suffixes SA[i] and SA[i+1];
 *        LCP[n-1] = 0.
 *   candidates  for every adjacent pair i (s1 = SA[i], s2 = SA[i+1],
 *        p = LCP[i]): if [s1, s1+p) and [s2, s2+p) are disjoint (|s1-s2| >= p)
 *        the pair (p, s1), (p, s2); otherwise, with lo = min(s1, s2) and
 *        d = |s1 - s2|, l = floor((p + d) / 2) - (floor((p + d) / 2) mod d)
 *        and the pair (l, lo), (l, lo + l).  Candidates shorter than min_len
 *        are dropped, identical (length, start) pairs are kept once, and the
 *        rest are ordered by length descending, sub-string ascending
 *        (lexicographic over the tokens), start ascending.  A candidate's
 *        id is the SA index of the first suffix that starts with its
 *        sub-string, so equal ids (at equal length) mean equal sub-strings
 *        and id order is sub-string order.
 *   greedy selection  candidates are visited in that order; one is accepted
 *        iff [start, start+len) meets no interval accepted before it.
 *   R    the distinct accepted sub-strings ("traces") in the order of their
 *        first acceptance; trace_start = smallest accepted start of the trace.
 *   selected intervals  the accepted intervals by increasing start, with the
 *        index into R of their sub-string.
 * ---------------------------------------------------------------------- */
typedef struct {
  uint64_t n;          /* tokens in the window */
  const void *tokens;  /* device, n tokens of token_bytes each */
  int token_bytes;     /* 4 (uint32) or 8 (uint64) */
} apo_window;

typedef struct {
  uint32_t min_len;    /* minimum trace length, >= 1 (Sec. 3: traces must be long enough
                          to amortise the replay cost) */
  uint32_t flags;      /* reserved, must be 0 */
} apo_repeats_params;

typedef struct {
  /* Optional stage outputs; NULL skips the copy. */
  uint32_t *sa;              /* [n] */
  uint32_t *lcp;             /* [n] */
  uint32_t *cand_len;        /* [cand_cap] candidates in greedy order */
  uint32_t *cand_id;         /* [cand_cap] */
  uint32_t *cand_start;      /* [cand_cap] */
  uint8_t *cand_accepted;    /* [cand_cap] 1 = accepted by the greedy loop */
  uint64_t cand_cap;
  /* Results. */
  uint32_t *sel_start;       /* [sel_cap] accepted intervals by increasing start */
  uint32_t *sel_len;         /* [sel_cap] */
  uint32_t *sel_trace;       /* [sel_cap] index into the trace arrays */
  uint64_t sel_cap;
  uint32_t *trace_len;       /* [trace_cap] R in first-acceptance order */
  uint32_t *trace_start;     /* [trace_cap] smallest accepted start of the trace */
  uint64_t trace_cap;
  /* HOST array of 4 counts, written before the call returns:
   * [0] candidates, [1] accepted intervals, [2] traces, [3] doubling rounds. */
  uint64_t *counts;
  /* Batched calls only (HOST, n_windows + 1 entries each, or NULL): where
   * each window's candidates, selected intervals and traces start in the
   * arrays above. */
  uint64_t *cand_off;
  uint64_t *sel_off;
  uint64_t *trace_off;
} apo_repeats_out;

/* Run Alg. 2 on one window.  Synchronises `stream` (the suffix sorting loop
 * and the output sizes are data-dependent); all outputs are complete when it
 * returns APO_OK.  APO_ECAPACITY if cand_cap (when cand_* is requested),
 * sel_cap or trace_cap is too small: counts are still written and nothing
 * beyond a capacity is touched.  Capacities that always suffice:
 * cand_cap = 2(n-1), sel_cap = trace_cap = floor(n / min_len).
 * n = 0 or 1 gives no candidates. */
int apo_find_repeats(apo_ctx *ctx, const apo_window *window, const apo_repeats_params *params,
                     apo_repeats_out *out, void *stream);

/* ------------------------------------------------------------------------
 * Batched repeat finding -- Alg. 2 applied to many independent windows in one
 * call (Alg. 1 analyses many history slices asynchronously, Sec. 4.2 and 4.4).
 *
 * The windows are concatenated in `tokens`; window w is tokens[win_off[w] ..
 * win_off[w+1]).  Every window gets exactly the results apo_find_repeats
 * would give it alone: the suffix sorting, the candidates and the greedy
 * selection never mix windows.  Outputs are concatenated window by window:
 * sa/lcp (optional, sum of window lengths entries, values relative to the
 * window start), candidates, selected intervals and traces (starts relative
 * to their window, sel_trace relative to the window's first trace), with
 * out->cand_off / sel_off / trace_off (HOST) giving each window's range.
 * cand_id values are SA indices in the concatenated array (they order a
 * window's sub-strings; only equality and order within a window matter).
 * Synchronises `stream`.  Capacities that always suffice: cand_cap = 2 *
 * total tokens, sel_cap = trace_cap = total tokens / min_len.
 * ---------------------------------------------------------------------- */
typedef struct {
  uint64_t n_windows;       /* W >= 1 */
  const void *tokens;       /* device, win_off[W] tokens */
  int token_bytes;          /* 4 or 8 */
  const uint64_t *win_off;  /* HOST [W+1], win_off[0] = 0, non-decreasing; each window
                               holds at most 2^31 - 1 tokens, all together < 2^31 */
} apo_windows;

int apo_find_repeats_batched(apo_ctx *ctx, const apo_windows *windows,
                             const apo_repeats_params *params, apo_repeats_out *out, void *stream);

/* ------------------------------------------------------------------------
 * Workspace of the repeat-finding calls (the scratch of Alg. 2's stages:
 * sort buffers, doubling-round lists, level ranks, candidate arrays).
 *
 * apo_find_repeats_workspace: *bytes (HOST) receives the device bytes that
 * apo_find_repeats (one window: n_windows = 1, win_off = {0, n}) or
 * apo_find_repeats_batched needs for `windows` -- an upper bound that depends
 * only on the total token count and the window count.  It allocates and
 * launches nothing and needs no GPU (ctx may be NULL).  APO_EINVAL for a
 * null windows or bytes pointer, no windows, or more than 2^31 - 1 tokens.
 *
 * apo_set_workspace: from now on the context takes all scratch of its repeat
 * calls from `workspace` (DEVICE, `bytes` long, 256-byte aligned, at least
 * 4096 bytes, owned by the caller and not freed by the library) instead of
 * growing its own with cudaMalloc; a call that needs more than is attached
 * fails with APO_ENOMEM before it launches anything, with the size it needs
 * in apo_last_error().  Radix-sort shapes are not tuned by trial runs while a
 * workspace is attached (the default shape, or a choice made earlier in the
 * process).  workspace = NULL returns to the context's own scratch.  The
 * caller makes sure that the context's earlier work has finished before it
 * attaches, replaces or detaches a workspace (the call does not wait), and
 * does not reuse the workspace's memory while calls on the context may still
 * run.
 * Calls that need scratch of another kind (matching's flattened output
 * chains, the replayer, the optimum) fail with APO_ENOMEM while a workspace
 * is attached.
 * ---------------------------------------------------------------------- */
int apo_find_repeats_workspace(apo_ctx *ctx, const apo_windows *windows, uint64_t *bytes);
int apo_set_workspace(apo_ctx *ctx, void *workspace, uint64_t bytes);

/* Graph mode for apo_find_repeats and apo_find_repeats_batched (off by
 * default).  The first call with given arguments (token pointer and width,
 * window offsets, min_len,
 * output pointers and capacities) runs as usual while the values the host
 * reads back between its kernels are recorded; the call is then captured
 * into a CUDA graph that takes those values as given and checks each on the
 * device where it would have been read.  Later calls with the same arguments
 * replay the graph, one launch for the whole call; when a check fails (the
 * token contents led to other counts) the replay is discarded and the call
 * runs as usual and is recorded again.  Results are the same either way.
 * Calls while the context's workspace has moved since the capture run as
 * usual (and are recorded again).  enable = 0 turns it off and frees the
 * graphs. */
int apo_graph_mode(apo_ctx *ctx, int enable);
/* Since graph mode was turned on: calls answered by a graph replay, graphs
 * captured, replays discarded because a check failed (HOST outputs). */
int apo_graph_stats(apo_ctx *ctx, uint64_t *replays, uint64_t *captures, uint64_t *discarded);

/* ------------------------------------------------------------------------
 * Served repeat finding -- Alg. 1 launches an asynchronous FindRepeats for
 * each history slice while the application keeps issuing tasks, and ingests
 * each result when it completes (Sec. 4.2, 4.3).  A server accepts such
 * analysis requests at any time and batches them continuously: each of its
 * `lanes` (a context and a stream of its own) repeatedly takes the requests
 * that are waiting, in arrival order, runs apo_find_repeats_batched on them
 * and publishes each request's results.  Batches of different lanes overlap
 * on the device; requests that arrive meanwhile join the next batch a lane
 * forms.  A request's results are the ones apo_find_repeats gives its window
 * alone.
 *
 * Admission is by device-memory footprint: the server holds one pool of
 * hbm_budget bytes, and a batch takes a slice of it for its tokens, outputs
 * and analysis scratch (apo_find_repeats_workspace of its windows).  A lane
 * adds waiting requests to its batch while the larger footprint still fits
 * in a free slice, within max_batch_tokens and max_batch_windows; when not
 * even the first waiting request fits beside the batches in flight, it waits
 * until one of them finishes and returns its slice.  A request whose
 * footprint exceeds the whole budget completes with status APO_ECAPACITY.
 * ---------------------------------------------------------------------- */
typedef struct apo_server apo_server;

typedef struct {
  uint32_t min_len;            /* as apo_repeats_params */
  int token_bytes;             /* 4 or 8 */
  uint64_t max_batch_tokens;   /* most tokens per batch (a larger request runs alone) */
  uint32_t max_batch_windows;  /* most requests per batch */
  uint32_t lanes;              /* batches in flight at once, >= 1 */
  uint64_t hbm_budget;         /* device bytes all batches in flight may hold together (one pool,
                                  allocated at creation); 0 = 16 GiB */
} apo_server_config;

typedef struct {
  int status;                  /* APO_OK or the batch's error */
  uint64_t n;                  /* tokens of the request */
  uint64_t n_selected, n_traces;
  const uint32_t *sel_start;   /* HOST, owned by the server until apo_server_release */
  const uint32_t *sel_len;
  const uint32_t *sel_trace;
  const uint32_t *trace_len;
  const uint32_t *trace_start;
  double t_submit, t_start, t_done;  /* seconds on the server's steady clock */
  uint64_t batch_windows;      /* requests in the batch that served it */
} apo_request_result;

/* Start a server on `device` with cfg->lanes worker threads. */
int apo_server_create(apo_server **srv, int device, const apo_server_config *cfg);
/* Queue a request; `tokens` (HOST, n tokens) is copied before the call
 * returns.  *id identifies the request. */
int apo_server_submit(apo_server *srv, const void *tokens, uint64_t n, uint64_t *id);
/* APO_OK and *out filled if request `id` is done, APO_EAGAIN if not yet. */
int apo_server_poll(apo_server *srv, uint64_t id, apo_request_result *out);
/* Block until request `id` is done, then as apo_server_poll. */
int apo_server_wait(apo_server *srv, uint64_t id, apo_request_result *out);
/* Drop a finished request's results (its pointers become invalid). */
int apo_server_release(apo_server *srv, uint64_t id);
/* Seconds on the server's steady clock (the clock of the t_* fields). */
double apo_server_now(apo_server *srv);
/* The pool's size, the bytes batches in flight hold now, and the most they
 * have held at once (HOST outputs; NULL skips one). */
int apo_server_memory(apo_server *srv, uint64_t *budget, uint64_t *held, uint64_t *held_max);
/* Finish the queued requests, stop the lanes and free everything. */
int apo_server_destroy(apo_server *srv);

/* ------------------------------------------------------------------------
 * Online trace finder -- Alg. 1's TraceFinder with Sec. 4.4's sampling of
 * the history buffer by the exponentiated ruler function.
 *
 * Tokens arrive in issue order (apo_finder_push, any chunk sizes).  The
 * finder keeps the most recent `buffer_tokens` of them.  After every `unit`
 * tokens (analysis point i = 1, 2, ...) it hands the most recent
 * unit * 2^ruler(i) tokens (ruler(i): how many times 2 divides i), at most
 * the buffer and at most what has arrived, to the server as one
 * asynchronous FindRepeats (Alg. 2) request.  Completed analyses come back
 * in analysis order through apo_finder_poll, with trace starts in stream
 * coordinates (token index since the first push).  Total tokens analysed
 * over a stream of n tokens grow as n log(buffer/unit), so the work is
 * O(n log^2 n) for Alg. 2's O(n log n) per slice (Sec. 4.4).
 * ---------------------------------------------------------------------- */
typedef struct apo_finder apo_finder;

typedef struct {
  uint64_t buffer_tokens;  /* history buffer size (the paper uses 5000) */
  uint64_t unit;           /* analysis period and smallest slice (250 or 500) */
} apo_finder_config;

typedef struct {
  uint64_t index;          /* analysis point i (1-based) */
  uint64_t slice_start;    /* stream position of the slice's first token */
  uint64_t slice_len;
  int status;              /* the request's status */
  uint64_t n_traces;
  const uint32_t *trace_len;    /* HOST, valid until the next poll or destroy */
  const uint64_t *trace_start;  /* stream coordinates */
  double t_submit, t_done;      /* server clock */
} apo_finder_result;

/* A finder feeding `server` (tokens of the server's token width, min_len of
 * the server).  APO_EINVAL for unit = 0 or buffer_tokens < unit. */
int apo_finder_create(apo_finder **out, apo_server *server, const apo_finder_config *cfg);
/* Append n tokens (HOST, copied); submits the analyses whose points are
 * reached.  *submitted (optional) receives how many were submitted. */
int apo_finder_push(apo_finder *f, const void *tokens, uint64_t n, uint64_t *submitted);
/* The oldest submitted analysis not yet returned: APO_OK and *out filled
 * if it is done, APO_EAGAIN if it is still running, APO_ECAPACITY if there
 * is none outstanding.  With wait != 0, blocks until it is done. */
int apo_finder_poll(apo_finder *f, int wait, apo_finder_result *out);
/* Totals so far: tokens pushed, analyses submitted, tokens analysed. */
int apo_finder_stats(apo_finder *f, uint64_t *pushed, uint64_t *analyses, uint64_t *analysed_tokens);
/* Releases the outstanding requests (waiting for them) and frees the finder;
 * the server stays. */
int apo_finder_destroy(apo_finder *f);

/* ------------------------------------------------------------------------
 * Candidate matching -- Sec. 4.3: the candidate traces are ingested into a
 * trie, and pointers advanced through the trie as tokens arrive report a
 * trace whenever one ends.  Computed here with an Aho-Corasick automaton
 * (goto trie, failure and output links) over the whole stream at once.
 *
 * Reports every (end, id) with stream[end - len(id) + 1 .. end] == pattern id,
 * for all patterns (overlapping occurrences included; a pattern listed twice
 * is reported under both ids), ordered by end ascending, then pattern length
 * descending, then id ascending.  At most 2^32 - 1 matches per call.
 * ---------------------------------------------------------------------- */
typedef struct {
  uint64_t n_patterns;       /* P >= 1 */
  const void *tokens;        /* device token array the patterns are taken from */
  int token_bytes;           /* 4 or 8, same width as the stream */
  /* Either CSR form: pattern p = tokens[pat_off[p] .. pat_off[p+1]) with
   * pat_off a HOST array of P+1 offsets (pat_start/pat_len NULL) ... */
  const uint64_t *pat_off;
  /* ... or slice form (pat_off NULL): pattern p = tokens[pat_start[p] ..
   * pat_start[p] + pat_len[p]) with DEVICE arrays, e.g. the trace_start /
   * trace_len outputs of apo_find_repeats over the same tokens. */
  const uint32_t *pat_start;
  const uint32_t *pat_len;
  /* Optional, slice form only: the suffix array and LCP array of the
   * pattern source tokens[0 .. src_n) (DEVICE arrays of src_n entries, as
   * apo_find_repeats writes them for one window: lcp[k] pairs sa[k] with
   * sa[k+1], lcp[src_n-1] = 0).  Every slice must lie inside the source.
   * With them the trie, failure links and match totals are read off the
   * source's suffix array; without them (NULL) the library builds one over
   * the patterns.  The results are the same; APO_EINVAL if src_n does not
   * cover the slices, APO_EDEVICE if sa is not a permutation. */
  const uint32_t *src_sa;
  const uint32_t *src_lcp;
  uint64_t src_n;
} apo_patterns;

/* Match `patterns` against stream[n] (device, same token width).  Writes the
 * matches to match_end/match_id (device, `cap` entries each) and their total
 * number to *count (HOST).  Synchronises `stream`.  APO_ECAPACITY if the total
 * exceeds cap (*count is exact, the arrays' contents are then unspecified).
 * APO_EINVAL for an empty pattern, P = 0, or token_bytes not 4 or 8.
 * Performance only, the results are the same either way: when the slices are
 * taken from the stream itself (patterns->tokens == stream_tokens) and are
 * long, the automaton's states are computed in one exact pass that starts
 * each segment of the stream one longest-pattern length early; otherwise in
 * short chunks from the root, repaired until they agree. */
int apo_match_candidates(apo_ctx *ctx, const apo_patterns *patterns, const void *stream_tokens,
                         uint64_t n, uint32_t *match_end, uint32_t *match_id, uint64_t cap,
                         uint64_t *count, void *stream);

/* ------------------------------------------------------------------------
 * Trace replay -- Alg. 1 "TraceReplayer", Sec. 4.3, for a whole stream.
 *
 * The replayer the paper runs per task: candidate traces are ingested into
 * a trie; each task advances every live pointer along its token (dropping
 * those the trie does not continue) and starts a new one at the root; a
 * pointer standing at the end of a trace completes it, which counts one
 * appearance of that trace; when traces complete, the one with the highest
 * score is replayed -- it ends at the current task, the tasks before it run
 * untraced -- and every pointer is dropped (each has consumed the replayed
 * task).  Score of a completed trace t at task k:
 *     (len(t) * min(count(t), count_cap) * (t replayed before ? bonus_num : bonus_den))
 *         >> ((k - previous appearance of t) / half_life)
 * in unsigned 64-bit arithmetic (wrapping), count(t) including this
 * appearance; no shift at a first appearance or with half_life = 0; a shift
 * of 64 or more gives 0; count_cap = 0 means no cap; a tie goes to the longer
 * trace.  (The paper names these ingredients -- length times a capped count,
 * exponential decay with the tasks since the trace last appeared, a small
 * raise for a trace already replayed -- without constants; the halving per
 * half_life tasks and the integer form are this library's.)
 *
 * Trace q is the slice stream[start[q] .. start[q] + len[q]) and enters the
 * trie when task ingest[q] is processed (before that task's token; at
 * ingest >= n never).  A trace longer than max_trace_len (0 = no limit)
 * enters as consecutive pieces of max_trace_len tokens, the last one shorter
 * (the maximum trace length of Sec. 6.2).  Pieces are numbered in trace
 * order; a replay reports the smallest piece number with its string.
 * ---------------------------------------------------------------------- */
typedef struct {
  uint64_t n_traces;       /* P (0 allowed: nothing is replayed) */
  const uint32_t *start;   /* [P] device */
  const uint32_t *len;     /* [P] device, >= 1, start + len <= n */
  const uint32_t *ingest;  /* [P] device: task index at which the trace enters the trie */
} apo_replay_traces;

typedef struct {
  uint32_t max_trace_len;  /* 0 = no limit */
  uint32_t count_cap;      /* 0 = no cap */
  uint32_t half_life;      /* tasks per halving of the score; 0 = no decay */
  uint32_t bonus_num;      /* factor for a trace replayed before, 1 .. 65535 */
  uint32_t bonus_den;      /* factor otherwise, 1 .. 65535 */
  uint32_t window;         /* curve window in tasks (0 = every task so far) */
} apo_replay_params;

typedef struct {
  uint32_t *rep_end;       /* [rep_cap] device: task where each replay ends, ascending */
  uint32_t *rep_len;       /* [rep_cap] its length */
  uint32_t *rep_trace;     /* [rep_cap] the smallest piece number of its string */
  uint64_t rep_cap;
  uint8_t *traced;         /* [n] device or NULL: 1 for a task inside a replay */
  uint32_t *curve;         /* [n] device or NULL: traced tasks among the `window`
                              tasks ending at each task (the paper's Fig. 10 view) */
  /* HOST array of 8 counts, written before the call returns: [0] replays,
   * [1] traced tasks, [2] pieces, [3] occurrences of the pieces, [4]
   * appearances, [5] replay tasks not decided by the lower/upper score
   * bound, [6] rounds of the fixed-point selection, [7] jump levels. */
  uint64_t *counts;
} apo_replay_out;

/* Replay decisions for stream[n] (device tokens of token_bytes 4 or 8).
 * Synchronises `stream`.  APO_EINVAL for a bad argument or trace;
 * APO_ECAPACITY if the replays exceed rep_cap (counts are still written). */
int apo_replay(apo_ctx *ctx, const void *stream_tokens, uint64_t n, int token_bytes,
               const apo_replay_traces *traces, const apo_replay_params *params, apo_replay_out *out,
               void *stream);

/* ------------------------------------------------------------------------
 * Optimal trace selection for short windows -- the optimisation problem of
 * Sec. 3, the yardstick for Alg. 2 (a heuristic, Sec. 4.2).
 *
 * For each window S: choose traces T (sub-strings of S, length >= min_len)
 * and for each trace a set of intervals of S holding it, all intervals
 * disjoint, every trace matching at least two intervals (as stated in the
 * paper the problem is solved by T = {S}, one interval over everything; the
 * traces must repeat).  Maximise the coverage (summed interval lengths),
 * then the number of intervals, then minimise |T|.
 *
 * Exhaustive search per window (one GPU thread each), positions left to
 * right, each uncovered or starting an interval of length min_len,
 * min_len + 1, ...; the witness is the first optimal set in that order.
 * Windows hold at most 24 tokens, and the number of interval sets of the
 * longest window at this min_len must not exceed 2^24 (e.g. 24 tokens at
 * min_len 2, 16 at min_len 1); APO_EINVAL otherwise.
 * ---------------------------------------------------------------------- */
/* best: [3 * n_windows] device: coverage, intervals, |T| per window.
 * wit_start / wit_len: [win_off[n_windows]] device: window w's optimal
 * intervals at [win_off[w], win_off[w] + wit_count[w]), by start, in
 * window coordinates.  wit_count: [n_windows] device.  Synchronises. */
int apo_optimum_batched(apo_ctx *ctx, const apo_windows *windows, uint32_t min_len, uint32_t *best,
                        uint32_t *wit_start, uint32_t *wit_len, uint32_t *wit_count, void *stream);

/* ------------------------------------------------------------------------
 * Greedy selection without allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code
 * running inside a task runtime that owns all device memory through its own
 * pool, or on a latency-critical path that must not pay for cudaMalloc /
 * cudaFree (which may synchronise the whole device).  It needs no context.
 *
 * Contract: the m candidates are visited in the order given, and
 * accepted[k] = 1 iff [cand_start[k], cand_start[k] + cand_len[k]) meets no
 * interval accepted before it (else 0).  cand_len must not increase along
 * the order -- apo_find_repeats's candidate order (length descending)
 * satisfies this -- because the test that a candidate meets an accepted
 * interval looks only at its first and last position, which is exact only
 * then.  When a length does increase, the flags are undefined and
 * *accepted_count is set to 0xffffffff; otherwise *accepted_count (DEVICE
 * u32) receives the number accepted.  Intervals must lie in [0, n); one that
 * does not is never accepted.  All arguments are device pointers owned by the
 * caller (cand_len, cand_start and accepted with m entries); the call only
 * enqueues work on `stream` and returns.  m = 0 writes *accepted_count = 0.
 *
 * Its scratch is a fixed bitmap of APO_NOALLOC_MAX_WINDOW bits (512 KiB)
 * compiled into the library as a static device array, which every GPU that
 * loads the library holds until the process exits.  A window larger than
 * that is rejected with APO_EINVAL.  The first call on a device looks up the
 * array's device address (once per device, on the current device); make that
 * first call before any stream capture.  Every call shares the array and it
 * keeps the last call's contents (each call clears the part it uses first);
 * calls whose work overlaps on the GPU race on it, so do not run two at once.
 * ---------------------------------------------------------------------- */
#define APO_NOALLOC_MAX_WINDOW (1u << 22)
int apo_greedy_select_noalloc(const uint32_t *cand_len, const uint32_t *cand_start, uint64_t m,
                              uint64_t n, uint8_t *accepted, uint32_t *accepted_count, void *stream);

/* ------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper; used to report per-kernel
 * device time against the hardware roofline).
 *
 * Every kernel launch of the library is counted per kernel.  With timing
 * enabled, each launch is also bracketed by two CUDA events recorded on its
 * launch stream, and the elapsed device time is accumulated when the entry
 * is read.  `units` accumulates the elements each launch processed (keys for
 * a radix-sort pass, list entries for a doubling round, tokens for a match), from which
 * a caller derives algorithmic bytes.  The same kernel on different stages
 * is kept in separate entries: everything the matcher launches (including
 * the suffix array of its pattern text) carries the prefix "ac.", the
 * repeat selection after the LCP (candidates, their sort, the greedy loop,
 * R) the prefix "rep."; unprefixed entries are the call's own path (task
 * hashing, the suffix array and LCP of the analysed windows with its token
 * dictionary "sa_dict", the replayer).
 * ---------------------------------------------------------------------- */
int apo_profile_enable(apo_ctx *ctx, int enable_timing);
int apo_profile_reset(apo_ctx *ctx);
/* Entry `index` (0-based): its kernel name (NUL-terminated, truncated to
 * name_cap), launches, accumulated milliseconds (0 without timing) and units.
 * Synchronises the events still pending.  APO_EINVAL when index is past the
 * last entry. */
int apo_profile_read(apo_ctx *ctx, int index, char *name, size_t name_cap, uint64_t *launches,
                     double *ms, uint64_t *units);

/* ------------------------------------------------------------------------
 * Radix-sort launch shapes (no counterpart in the paper: a property of this
 * GPU implementation).
 *
 * Every sort (the prefix-doubling rounds, the candidate order, the pattern
 * starts) runs the onesweep digit pass in one of several shapes: threads per
 * block, pairs per thread and digit width (8 or 9 bits).  In mode 0 (the
 * default) the first sort of each size class (n rounded up to a power of
 * two, 2^10 .. 2^23 and above) and key width on a device times every shape
 * on synthetic keys of that size (at most 2^22 pairs) and width, on the
 * call's stream, and keeps the fastest for the process's lifetime; that
 * first call is slower by the trials.  Mode 1 always uses the default shape
 * (512 threads, 8 pairs each, 8-bit digits) and never times anything; mode
 * 2 + k always uses shape k (0: 512 x 8 pairs, 8-bit; 1: 256 x 8, 8-bit;
 * 2: 512 x 4, 8-bit; 3: 256 x 4, 8-bit; 4: 512 x 8, 9-bit; 5: 512 x 4,
 * 9-bit), for reproducible profiles.  Other modes: APO_EINVAL.
 * The choices are kept per device and shared by every context of the
 * process (a served lane benefits from another lane's trials); the mode is
 * per context.
 * Results never depend on the shape: the sort is stable and exact.
 * ---------------------------------------------------------------------- */
int apo_sort_tuning(apo_ctx *ctx, int mode);
/* Tuned entry `index` (0-based, in class then key-width order): size class
 * (log2 of the class's largest n), key bits, trial size, the chosen shape
 * and the trial times (ms per sort) of the chosen and the default shape.
 * APO_EINVAL when index is past the last tuned entry. */
int apo_sort_tuning_read(apo_ctx *ctx, int index, uint32_t *size_log2, uint32_t *key_bits,
                         uint32_t *trial_n, int *threads, int *items, int *digit_bits, double *best_ms,
                         double *default_ms);

#ifdef __cplusplus
}
#endif

#endif /* APO_H */
