// Batched calls replayed as CUDA graphs.
//
// A batched call (apo_find_repeats_batched) queues about a hundred kernels
// and reads a handful of values back on the host between them: the token code
// width, the active-suffix count of each doubling round, the candidate and
// selection counts.  Those reads decide the launches that follow (how many
// rounds, how many elements each sort covers, how many bytes each copy
// moves), so a call cannot be captured into a graph as it stands.  With graph
// mode on, the first call on a batch runs as usual while a tape records every
// value the host reads; the same call is then captured into a graph with the
// reads answered from the tape, each answer checked on the device at that
// point of the stream by a one-thread kernel.  Later calls with the same
// arguments replay the graph (one launch for the whole call); if any checked
// word differs -- the batch's contents led elsewhere -- the replay's results
// are discarded and the call runs again as usual, recording a new tape.
//
// A graph bakes in the device addresses of the context's workspace and the
// look-back epochs of its kernels: it is dropped when a workspace buffer
// moves, and every replay starts by clearing the look-back status words (an
// epoch from the previous replay of the same graph would otherwise be
// mistaken for a fresh one).
#include <cstring>
#include <unordered_map>
#include <vector>

#include "../../include/apo.h"
#include "apo_internal.cuh"

namespace apo {

namespace {

// bad += number of words at dev[0..words) that differ from want[0..words)
__global__ void k_tape_check(const uint32_t *__restrict__ dev, const uint32_t *__restrict__ want, int words,
                             uint32_t *bad) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    uint32_t d = 0;
    for (int i = 0; i < words; ++i) d += dev[i] != want[i];
    if (d) atomicAdd(bad, d);
  }
}

}  // namespace

void tape_put(apo_ctx *c, const uint32_t *vals, int words) {
  if (!recording(c)) return;
  c->tape->vals.insert(c->tape->vals.end(), vals, vals + words);
}

int tape_take(apo_ctx *c, const uint32_t *dev, uint32_t *host, int words, cudaStream_t s) {
  Tape *t = c->tape;
  if (t->pos + words > t->vals.size()) {
    set_error("graph capture: the call read more values than it recorded");
    return APO_EDEVICE;
  }
  memcpy(host, t->vals.data() + t->pos, (size_t)words * 4);
  k_tape_check<<<1, 32, 0, s>>>(dev, t->dev_vals + t->pos, words, t->bad);
  t->pos += words;
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  uint64_t gen = 0, moves = 0;   // workspace state the graph was captured with
  std::vector<uint32_t> win_off; // the call's arguments, compared on every hit
  std::vector<const void *> ptrs;
  std::vector<uint64_t> caps;
  uint32_t *dev_vals = nullptr;  // recorded values (device)
  uint32_t *bad = nullptr;       // mismatch counter (device)
  uint32_t *stage = nullptr;     // pinned: per-window output offsets
  uint32_t *upload = nullptr;    // pinned: window offsets copied in
  uint32_t *bad_host = nullptr;  // pinned
  uint64_t counts[4] = {0, 0, 0, 0};
  uint64_t launches[kScopes * kKCount] = {};
};

struct GraphCache {
  std::unordered_map<uint64_t, GraphEntry> entries;
  uint64_t replays = 0, captures = 0, discarded = 0;
  cudaStream_t stream = nullptr;     // graphs are captured and replayed on a stream of their own
  cudaEvent_t in = nullptr, out = nullptr;
};

namespace {

void free_entry(GraphEntry &e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.dev_vals) cudaFree(e.dev_vals);
  if (e.bad) cudaFree(e.bad);
  if (e.stage) cudaFreeHost(e.stage);
  if (e.upload) cudaFreeHost(e.upload);
  if (e.bad_host) cudaFreeHost(e.bad_host);
  e = GraphEntry();
}

uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

// Everything a call's launches depend on besides the device contents.
void call_key(const apo_windows *ws, const apo_repeats_params *p, const apo_repeats_out *o,
              std::vector<uint32_t> *win, std::vector<const void *> *ptrs, std::vector<uint64_t> *caps) {
  win->assign(ws->n_windows + 1, 0);
  for (uint64_t w = 0; w <= ws->n_windows; ++w) (*win)[w] = (uint32_t)ws->win_off[w];
  *ptrs = {ws->tokens, o->sa, o->lcp, o->cand_len, o->cand_id, o->cand_start, o->cand_accepted, o->sel_start,
           o->sel_len, o->sel_trace, o->trace_len, o->trace_start};
  *caps = {(uint64_t)ws->token_bytes, p->min_len, p->flags, o->cand_cap, o->sel_cap, o->trace_cap,
           o->cand_off != nullptr, o->sel_off != nullptr, o->trace_off != nullptr};
}

uint64_t key_hash(const std::vector<uint32_t> &win, const std::vector<const void *> &ptrs,
                  const std::vector<uint64_t> &caps) {
  uint64_t h = 0x6a09e667f3bcc909ull;
  for (uint32_t v : win) h = mix(h, v);
  for (const void *q : ptrs) h = mix(h, (uint64_t)(uintptr_t)q);
  for (uint64_t v : caps) h = mix(h, v);
  return h;
}

void write_offsets(const GraphEntry &e, uint32_t W, apo_repeats_out *out) {
  for (uint32_t w = 0; w <= W; ++w) {
    if (out->cand_off) out->cand_off[w] = e.stage[w];
    if (out->sel_off) out->sel_off[w] = e.stage[(W + 1) + w];
    if (out->trace_off) out->trace_off[w] = e.stage[2 * (W + 1) + w];
  }
}

int ensure_cache(apo_ctx *c) {
  if (c->graphs) return APO_OK;
  GraphCache *g = new GraphCache();
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete g;
    set_error("graph mode: stream or event creation failed");
    return APO_ECUDA;
  }
  c->graphs = g;
  return APO_OK;
}

}  // namespace

void graph_cache_free(apo_ctx *c) {
  GraphCache *g = c->graphs;
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (auto &kv : g->entries) free_entry(kv.second);
  if (g->in) cudaEventDestroy(g->in);
  if (g->out) cudaEventDestroy(g->out);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
  c->graphs = nullptr;
}

int graph_batched(apo_ctx *c, const apo_windows *ws, const apo_repeats_params *p, apo_repeats_out *out,
                  cudaStream_t s) {
  const uint32_t W = (uint32_t)ws->n_windows;
  const uint64_t total = ws->win_off[W];
  auto eager = [&]() {
    return drv::find_repeats_driver(c, ws->tokens, ws->token_bytes, total, ws->win_off, W, p, out, s);
  };
  if (total == 0) return eager();
  APO_TRY(ensure_cache(c));
  GraphCache *g = c->graphs;
  std::vector<uint32_t> win;
  std::vector<const void *> ptrs;
  std::vector<uint64_t> caps;
  call_key(ws, p, out, &win, &ptrs, &caps);
  const uint64_t key = key_hash(win, ptrs, caps);

  // replay
  auto it = g->entries.find(key);
  if (it != g->entries.end()) {
    GraphEntry &e = it->second;
    if (e.gen == c->gen && e.moves == c->arena.moves && e.win_off == win && e.ptrs == ptrs && e.caps == caps) {
      APO_CUDA_TRY(cudaEventRecord(g->in, s));
      APO_CUDA_TRY(cudaStreamWaitEvent(g->stream, g->in, 0));
      APO_CUDA_TRY(cudaGraphLaunch(e.exec, g->stream));
      APO_CUDA_TRY(cudaMemcpyAsync(e.bad_host, e.bad, 4, cudaMemcpyDeviceToHost, g->stream));
      APO_CUDA_TRY(cudaEventRecord(g->out, g->stream));
      APO_CUDA_TRY(cudaStreamWaitEvent(s, g->out, 0));
      APO_CUDA_TRY(cudaStreamSynchronize(g->stream));
      if (*e.bad_host == 0) {
        ++g->replays;
        for (int k = 0; k < 4; ++k) out->counts[k] = e.counts[k];
        write_offsets(e, W, out);
        for (int k = 0; k < kScopes * kKCount; ++k) c->prof.launches[k] += e.launches[k];
        return APO_OK;
      }
      // the batch led elsewhere (or a check of the error word failed): run it as usual
      ++g->discarded;
      APO_CUDA_TRY(cudaMemsetAsync(c->ps.err, 0, sizeof(uint32_t), s));
    }
    free_entry(e);
    g->entries.erase(it);
  }

  // record: the call as usual, keeping every value the host reads
  Tape rec;
  rec.mode = kTapeRecord;
  c->tape = &rec;
  const int r = eager();
  c->tape = nullptr;
  if (r != APO_OK) return r;
  uint64_t counts[4];
  for (int k = 0; k < 4; ++k) counts[k] = out->counts[k];

  // capture the same call with the reads answered from the tape
  GraphEntry e;
  e.gen = c->gen;
  e.moves = c->arena.moves;
  e.win_off = win;
  e.ptrs = ptrs;
  e.caps = caps;
  for (int k = 0; k < 4; ++k) e.counts[k] = counts[k];
  const size_t nv = std::max<size_t>(rec.vals.size(), 1);
  bool ok = cudaMalloc(&e.dev_vals, nv * 4) == cudaSuccess && cudaMalloc(&e.bad, 4) == cudaSuccess &&
            cudaMallocHost(&e.stage, 3 * (size_t)(W + 1) * 4) == cudaSuccess &&
            cudaMallocHost(&e.upload, (size_t)(W + 1) * 4) == cudaSuccess &&
            cudaMallocHost(&e.bad_host, 4) == cudaSuccess;
  if (ok && !rec.vals.empty())
    ok = cudaMemcpy(e.dev_vals, rec.vals.data(), rec.vals.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {  // no graph; the recorded call's results stand
    cudaGetLastError();
    free_entry(e);
    return APO_OK;
  }
  Tape cap;
  cap.mode = kTapeCapture;
  cap.vals = std::move(rec.vals);
  cap.dev_vals = e.dev_vals;
  cap.bad = e.bad;
  cap.stage = e.stage;
  cap.upload = e.upload;
  uint64_t before[kScopes * kKCount], ubefore[kScopes * kKCount];
  memcpy(before, c->prof.launches, sizeof(before));
  memcpy(ubefore, c->prof.units, sizeof(ubefore));
  apo_repeats_out o2 = *out;
  uint64_t cnt2[4];
  o2.counts = cnt2;
  o2.cand_off = o2.sel_off = o2.trace_off = nullptr;  // a replay fills them from the stage
  cudaGraph_t graph = nullptr;
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  APO_CUDA_TRY(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
  int rc = APO_OK;
  if (cudaMemsetAsync(e.bad, 0, 4, g->stream) != cudaSuccess ||
      cudaMemsetAsync(c->ps.lookback, 0, c->ps.lookback_words * sizeof(uint64_t), g->stream) != cudaSuccess)
    rc = APO_ECUDA;
  if (rc == APO_OK) {
    c->tape = &cap;
    rc = drv::find_repeats_driver(c, ws->tokens, ws->token_bytes, total, ws->win_off, W, p, &o2, g->stream);
    c->tape = nullptr;
  }
  const cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
  for (int k = 0; k < kScopes * kKCount; ++k) {  // the capture launched nothing
    e.launches[k] = c->prof.launches[k] - before[k];
    c->prof.launches[k] = before[k];
    c->prof.units[k] = ubefore[k];
  }
  if (rc != APO_OK || ce != cudaSuccess || !graph || cap.pos != cap.vals.size() ||
      cudaGraphInstantiate(&e.exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    free_entry(e);
    return APO_OK;  // no graph this time; the recorded call's results stand
  }
  cudaGraphDestroy(graph);
  g->entries.emplace(key, std::move(e));
  ++g->captures;
  return APO_OK;
}

void graph_stats(apo_ctx *c, uint64_t *replays, uint64_t *captures, uint64_t *discarded) {
  GraphCache *g = c->graphs;
  *replays = g ? g->replays : 0;
  *captures = g ? g->captures : 0;
  *discarded = g ? g->discarded : 0;
}

}  // namespace apo
