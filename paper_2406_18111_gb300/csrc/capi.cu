// The C ABI of libapo: contexts, workspace, argument checks and the three
// entry points (apo_hash_tasks, apo_find_repeats, apo_match_candidates).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "apo_internal.cuh"

namespace apo {

size_t suffix_workspace_bytes(uint64_t n);
size_t repeats_workspace_bytes(uint64_t n, uint64_t windows);
int suffix_init();
int repeats_init(int smem_optin);
int match_init(int sms);

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }

int Arena::reserve(size_t bytes) {
  used = 0;
  if (bytes <= cap) return APO_OK;
  if (external) {
    set_error("workspace: the call needs " + std::to_string(bytes) + " bytes of scratch, the attached "
              "workspace leaves " + std::to_string(cap));
    return APO_ENOMEM;
  }
  if (base) {
    cudaDeviceSynchronize();
    cudaFree(base);
    base = nullptr;
    cap = 0;
  }
  const size_t want = std::max<size_t>(bytes, (size_t)1 << 24);
  ++moves;
  if (cudaMalloc(&base, want) != cudaSuccess) {
    cudaGetLastError();
    base = nullptr;
    set_error("workspace: cudaMalloc of " + std::to_string(want) + " bytes failed");
    return APO_ENOMEM;
  }
  cap = want;
  return APO_OK;
}

void *Arena::take(size_t bytes) {
  const size_t a = (used + 255) & ~(size_t)255;
  if (a + bytes > cap) return nullptr;
  used = a + bytes;
  return base + a;
}

int ensure_lookback(apo_ctx *c, size_t words) {
  if (words <= c->ps.lookback_words) return APO_OK;
  if (c->ext) {
    set_error("workspace: a launch needs " + std::to_string(words) + " look-back words, the attached "
              "workspace's reservation holds " + std::to_string(c->ps.lookback_words));
    return APO_ENOMEM;
  }
  // Growing frees the old array: wait for launches that may still read it.
  APO_CUDA_TRY(cudaDeviceSynchronize());
  if (c->ps.lookback) cudaFree(c->ps.lookback);
  c->ps.lookback = nullptr;
  c->ps.lookback_words = 0;
  const size_t w = std::max<size_t>(words, 1 << 16);
  APO_CUDA_TRY(cudaMalloc(&c->ps.lookback, w * sizeof(uint64_t)));
  APO_CUDA_TRY(cudaMemset(c->ps.lookback, 0, w * sizeof(uint64_t)));
  c->ps.lookback_words = w;
  ++c->gen;
  return APO_OK;
}

int reserve_workspace(apo_ctx *c, size_t arena_bytes, size_t lb_words, cudaStream_t s) {
  if (!c->ext) {
    APO_TRY(ensure_lookback(c, lb_words));
    return c->arena.reserve(arena_bytes);
  }
  const size_t lb_bytes = (lb_words * 8 + 255) & ~(size_t)255;
  if (lb_bytes + arena_bytes > c->ext_bytes) {
    set_error("workspace: the call needs " + std::to_string(lb_bytes + arena_bytes) + " bytes, " +
              std::to_string(c->ext_bytes) + " are attached (apo_find_repeats_workspace gives the size)");
    return APO_ENOMEM;
  }
  if (lb_bytes > c->ext_lb_bytes) {
    // the look-back words must start out clear (earlier calls may have used
    // these bytes as arena); queued ahead of the call's kernels
    APO_CUDA_TRY(cudaMemsetAsync(c->ext, 0, lb_bytes, s));
    c->ext_lb_bytes = lb_bytes;
    ++c->gen;
  }
  c->ps.lookback = reinterpret_cast<uint64_t *>(c->ext);
  c->ps.lookback_words = c->ext_lb_bytes / 8;
  c->arena.base = c->ext + c->ext_lb_bytes;
  c->arena.cap = c->ext_bytes - c->ext_lb_bytes;
  c->arena.used = 0;
  return arena_bytes <= c->arena.cap ? APO_OK : c->arena.reserve(arena_bytes);
}

void find_repeats_need(uint64_t n, uint64_t windows, size_t *arena_bytes, size_t *lb_words) {
  *arena_bytes = suffix_workspace_bytes(n) + repeats_workspace_bytes(n, windows) + (size_t)n * 24 +
                 (size_t)(windows + 1) * 4 + ((size_t)1 << 20);  // + slack for 256-byte alignment
  // the widest look-back of the call: a radix pass over at most 2n pairs in
  // tiles of at least 1024 with 512 digits
  *lb_words = ((size_t)(2 * n + 1023) / 1024 + 2) * 512 + ((size_t)1 << 16);
}

int ensure_side(apo_ctx *c, size_t bytes, cudaStream_t s) {
  if (bytes <= c->side_bytes) return APO_OK;
  if (c->ext) {
    set_error("workspace: this call needs scratch outside the attached workspace (" + std::to_string(bytes) +
              " bytes); detach it with apo_set_workspace(ctx, NULL, 0)");
    return APO_ENOMEM;
  }
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  if (c->side) cudaFree(c->side);
  c->side = nullptr;
  c->side_bytes = 0;
  const size_t want = std::max<size_t>(bytes + bytes / 4, (size_t)1 << 20);
  APO_CUDA_TRY(cudaMalloc(&c->side, want));
  c->side_bytes = want;
  ++c->gen;
  return APO_OK;
}

ScopeGuard::ScopeGuard(apo_ctx *c_, int scope) : c(c_), prev(c_->prof.scope) { c->prof.scope = scope; }
ScopeGuard::~ScopeGuard() { c->prof.scope = prev; }

const char *const kKernelNames[kKCount] = {
    "hash_tasks", "init_keys", "key_or", "rs_hist", "rs_offsets", "rs_pass", "refresh", "pack",
    "phi", "plcp", "lcp_perm", "min32", "max", "cand_gen", "compact", "cand_gather", "greedy",
    "traces", "sel_out", "pat_layout", "table_init", "end_pairs", "mark_ends", "ac_fix",
    "ac_states", "ac_fill", "dict_insert", "dict_map", "slices", "match_offsets", "seg_scan",
    "starts", "sparse", "ac_nodes", "ac_jump", "rs_tune", "rp_pieces", "rp_need", "rp_chain",
    "rp_appear", "rp_select", "rp_out", "optimum", "sa_dict", "round", "split", "wsb", "list_compact", "minor",
    "rs_pass_keys", "ac_halo"};

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int Profiler::resolve() {
  for (auto &p : pending) {
    float t = 0.f;
    cudaEventSynchronize(p.b);
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.id] += t;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
  return APO_OK;
}

void Profiler::release() {
  resolve();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

Launch::Launch(apo_ctx *c, int id, uint64_t units, cudaStream_t s)
    : c_(c), id_(id + c->prof.scope * kKCount), s_(s) {
  c->prof.launches[id_] += 1;
  c->prof.units[id_] += units;
  if (c->prof.timing && !capturing(c)) {
    if (c->prof.pending.size() > 8192) c->prof.resolve();
    a_ = c->prof.get();
    b_ = c->prof.get();
    cudaEventRecord(a_, s);
  }
}

Launch::~Launch() {
  if (a_) {
    cudaEventRecord(b_, s_);
    c_->prof.pending.push_back({id_, a_, b_});
  }
}

// Reads the device error word on the call's stream (after everything queued
// before it); clears it when set.
int check_device_error(apo_ctx *c, cudaStream_t s) {
  APO_CUDA_TRY(cudaMemcpyAsync(c->host_pinned + kPinnedErr, c->ps.err, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  return device_error_status(c, s);
}

// The error word already copied to the pinned slot by the caller's last
// synchronised read.
int device_error_status(apo_ctx *c, cudaStream_t s) {
  const uint32_t e = c->host_pinned[kPinnedErr];
  if (e == kDevOk) return APO_OK;
  c->host_pinned[kPinnedErr] = kDevOk;
  APO_CUDA_TRY(cudaMemsetAsync(c->ps.err, 0, sizeof(uint32_t), s));
  APO_CUDA_TRY(cudaStreamSynchronize(s));
  if (e == kDevTimeout) {
    set_error("a bounded device-side wait gave up");
    return APO_ETIMEOUT;
  }
  set_error("a kernel detected an out-of-range index");
  return APO_EDEVICE;
}

}  // namespace apo

using namespace apo;

extern "C" {

int apo_version(void) { return 100; }

const char *apo_last_error(void) { return g_last_error.c_str(); }

int apo_create(apo_ctx **out, int device) {
  if (!out) {
    set_error("apo_create: null output pointer");
    return APO_EINVAL;
  }
  *out = nullptr;
  APO_CUDA_TRY(cudaSetDevice(device));
  apo_ctx *c = new apo_ctx();
  c->device = device;
  int sms = 0, optin = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->num_sms = sms > 0 ? sms : 1;
  int r = APO_OK;
  // (per-device kernel attributes and occupancy; cheap to redo per context)
  if ((r = radix_sort_init()) != APO_OK || (r = suffix_init()) != APO_OK ||
      (r = repeats_init(optin)) != APO_OK || (r = match_init(c->num_sms)) != APO_OK) {
    delete c;
    return r;
  }
  if (cudaMalloc(&c->ps.err, sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&c->ps.counters, kCtrWords * sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost(&c->host_pinned, 256) != cudaSuccess) {
    cudaGetLastError();
    apo_destroy(c);
    set_error("apo_create: device allocation failed");
    return APO_ENOMEM;
  }
  if (cudaEventCreateWithFlags(&c->round_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->round_ev[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork_ev[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    apo_destroy(c);
    set_error("apo_create: event creation failed");
    return APO_ECUDA;
  }
  cudaMemset(c->ps.err, 0, sizeof(uint32_t));
  cudaMemset(c->ps.counters, 0, kCtrWords * sizeof(uint32_t));
  if (ensure_lookback(c, 1 << 16) != APO_OK) {
    apo_destroy(c);
    return APO_ENOMEM;
  }
  *out = c;
  return APO_OK;
}

int apo_destroy(apo_ctx *c) {
  if (!c) return APO_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  graph_cache_free(c);
  if (c->ext) apo_set_workspace(c, nullptr, 0);  // frees the context's own buffers, not the caller's
  if (c->arena.base) cudaFree(c->arena.base);
  if (c->ps.err) cudaFree(c->ps.err);
  if (c->ps.lookback) cudaFree(c->ps.lookback);
  if (c->ps.counters) cudaFree(c->ps.counters);
  if (c->host_pinned) cudaFreeHost(c->host_pinned);
  if (c->tuner.scratch) cudaFree(c->tuner.scratch);
  if (c->side) cudaFree(c->side);
  for (void *p : c->rp)
    if (p) cudaFree(p);
  for (auto e : c->round_ev)
    if (e) cudaEventDestroy(e);
  for (auto e : c->fork_ev)
    if (e) cudaEventDestroy(e);
  if (c->aux) cudaStreamDestroy(c->aux);
  c->prof.release();
  delete c;
  return APO_OK;
}

int apo_find_repeats_workspace(apo_ctx *c, const apo_windows *ws, uint64_t *bytes) {
  (void)c;  // the size depends on the windows only
  if (!ws || !bytes || !ws->win_off || ws->n_windows == 0) {
    set_error("apo_find_repeats_workspace: null argument or no windows");
    return APO_EINVAL;
  }
  const uint64_t n = ws->win_off[ws->n_windows];
  if (n > 0x7fffffffull) {
    set_error("apo_find_repeats_workspace: at most 2^31 - 1 tokens per call");
    return APO_EINVAL;
  }
  size_t arena_bytes = 0, lb_words = 0;
  find_repeats_need(n, ws->n_windows, &arena_bytes, &lb_words);
  *bytes = ((lb_words * 8 + 255) & ~(size_t)255) + arena_bytes;
  return APO_OK;
}

int apo_set_workspace(apo_ctx *c, void *workspace, uint64_t bytes) {
  if (!c || (workspace && bytes < 4096) || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("apo_set_workspace: null context, a workspace under 4096 bytes or not 256-byte aligned");
    return APO_EINVAL;
  }
  APO_CUDA_TRY(cudaSetDevice(c->device));
  if (!c->ext && workspace) {  // set the context's own buffers aside
    c->own_base = c->arena.base;
    c->own_cap = c->arena.cap;
    c->own_lookback = c->ps.lookback;
    c->own_lookback_words = c->ps.lookback_words;
  }
  if (c->ext && !workspace) {  // back to the context's own buffers
    c->arena.base = c->own_base;
    c->arena.cap = c->own_cap;
    c->ps.lookback = c->own_lookback;
    c->ps.lookback_words = c->own_lookback_words;
    c->own_base = nullptr;
    c->own_lookback = nullptr;
  }
  c->ext = static_cast<char *>(workspace);
  c->ext_bytes = workspace ? bytes : 0;
  c->ext_lb_bytes = 0;
  c->arena.external = workspace != nullptr;
  if (workspace) {
    c->arena.base = c->ext;
    c->arena.cap = c->ext_bytes;
    c->ps.lookback = nullptr;
    c->ps.lookback_words = 0;
  }
  c->arena.used = 0;
  ++c->arena.moves;
  ++c->gen;
  return APO_OK;
}

int apo_hash_tasks(apo_ctx *c, const apo_tasks *t, uint64_t *tokens_out, void *stream) {
  if (!c || !t) {
    set_error("apo_hash_tasks: null context or task list");
    return APO_EINVAL;
  }
  if (t->n_tasks == 0) return APO_OK;
  if (!t->task_id || !t->arg_off || !tokens_out) {
    set_error("apo_hash_tasks: null task_id, arg_off or output");
    return APO_EINVAL;
  }
  launch_hash_tasks(c, t, tokens_out, static_cast<cudaStream_t>(stream));
  APO_CUDA_TRY(cudaGetLastError());
  return APO_OK;
}

}  // extern "C"

namespace apo {
namespace drv {

__global__ void k_fill_windows(const uint32_t *__restrict__ off, uint32_t count, uint32_t *wid,
                               uint32_t *wend) {
  for (uint32_t w = blockIdx.x; w < count; w += gridDim.x) {
    const uint32_t a = off[w], b = off[w + 1];
    for (uint32_t i = a + threadIdx.x; i < b; i += blockDim.x) {
      wid[i] = w;
      wend[i] = b;
    }
  }
}

__global__ void k_sa_relative(const uint32_t *__restrict__ sa, uint32_t n, const uint32_t *__restrict__ wid,
                              const uint32_t *__restrict__ off, uint32_t *__restrict__ out) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    out[k] = sa[k] - off[wid[sa[k]]];
}

// Shared driver of apo_find_repeats (one window) and apo_find_repeats_batched.
int find_repeats_driver(apo_ctx *c, const void *tokens, int tb, uint64_t total,
                        const uint64_t *win_off, uint32_t nwin, const apo_repeats_params *p,
                        apo_repeats_out *out, cudaStream_t s) {
  for (int k = 0; k < 4; ++k) out->counts[k] = 0;
  if (tb != 4 && tb != 8) {
    set_error("find_repeats: token_bytes must be 4 or 8");
    return APO_EINVAL;
  }
  if (p->min_len == 0 || p->flags != 0) {
    set_error("find_repeats: min_len must be >= 1 and flags 0");
    return APO_EINVAL;
  }
  if (total > 0x7fffffffull) {
    set_error("find_repeats: at most 2^31 - 1 tokens per call");
    return APO_EINVAL;
  }
  if (total > 0 && !tokens) {
    set_error("find_repeats: null tokens");
    return APO_EINVAL;
  }
  const uint32_t n = (uint32_t)total;
  BatchOffsets boff;
  boff.cand_off = out->cand_off;
  boff.sel_off = out->sel_off;
  boff.trace_off = out->trace_off;
  if (n == 0) {
    for (uint32_t w = 0; w <= nwin; ++w) {
      if (boff.cand_off) boff.cand_off[w] = 0;
      if (boff.sel_off) boff.sel_off[w] = 0;
      if (boff.trace_off) boff.trace_off[w] = 0;
    }
    return APO_OK;
  }
  APO_CUDA_TRY(cudaSetDevice(c->device));
  {
    size_t arena_bytes = 0, lb_words = 0;
    find_repeats_need(n, nwin, &arena_bytes, &lb_words);
    APO_TRY(reserve_workspace(c, arena_bytes, lb_words, s));
  }
  SuffixState st;
  st.n = n;
  st.sa = c->arena.take_n<uint32_t>(n);
  st.rank = c->arena.take_n<uint32_t>(n);
  const int max_levels = bits_for(n) + 2;
  uint32_t *snap_base = c->arena.take_n<uint32_t>((size_t)max_levels * n);
  uint32_t *lcp = c->arena.take_n<uint32_t>(n);
  if (!st.sa || !st.rank || !snap_base || !lcp) {
    set_error("find_repeats: workspace too small");
    return APO_ENOMEM;
  }
  st.win.count = nwin;
  if (nwin > 1) {
    uint32_t *wid = c->arena.take_n<uint32_t>(n);
    uint32_t *wend = c->arena.take_n<uint32_t>(n);
    uint32_t *off = c->arena.take_n<uint32_t>(nwin + 1);
    if (!wid || !wend || !off) return APO_ENOMEM;
    std::vector<uint32_t> h(nwin + 1);
    uint32_t maxlen = 0;
    for (uint32_t w = 0; w <= nwin; ++w) {
      h[w] = (uint32_t)win_off[w];
      if (w) maxlen = std::max(maxlen, h[w] - h[w - 1]);
    }
    if (capturing(c)) {  // a graph copies from a pinned buffer that outlives this call
      memcpy(c->tape->upload, h.data(), (nwin + 1) * 4);
      APO_CUDA_TRY(cudaMemcpyAsync(off, c->tape->upload, (nwin + 1) * 4, cudaMemcpyHostToDevice, s));
    } else {
      APO_CUDA_TRY(cudaMemcpyAsync(off, h.data(), (nwin + 1) * 4, cudaMemcpyHostToDevice, s));
    }
    {
      Launch lp_(c, kKInitKeys, n, s);
      k_fill_windows<<<std::min<uint32_t>(nwin, 4096), 256, 0, s>>>(off, nwin, wid, wend);
    }
    if (!capturing(c)) APO_CUDA_TRY(cudaStreamSynchronize(s));  // h goes out of scope
    st.win.wid = wid;
    st.win.wend = wend;
    st.win.off_host = win_off;
    st.win.off_dev = off;
    st.win.max_len = maxlen;
  } else {
    st.win.max_len = n;
  }
  uint32_t *snaps[40];
  for (int k = 0; k < max_levels; ++k) snaps[k] = snap_base + (size_t)k * n;
  st.snaps = snaps;
  uint32_t rounds = 0;
  APO_TRY(build_suffix_array(c, tokens, tb, n, st, max_levels, &rounds, s));
  APO_TRY(build_lcp(c, tokens, tb, st, lcp, s));
  if (out->sa) {
    if (nwin > 1) {
      Launch lp_(c, kKSelOut, n, s);
      k_sa_relative<<<std::max(1, std::min(ceil_div(n, 256), c->num_sms * 16)), 256, 0, s>>>(
          st.sa, n, st.win.wid, st.win.off_dev, out->sa);
    } else {
      APO_CUDA_TRY(cudaMemcpyAsync(out->sa, st.sa, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (out->lcp) APO_CUDA_TRY(cudaMemcpyAsync(out->lcp, lcp, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  // find_repeats_from_sa ends by reading the device error word (a replay
  // checks that it is still clear)
  const int r = find_repeats_from_sa(c, tokens, tb, st, lcp, p->min_len, out, &boff, s);
  out->counts[3] = rounds;
  return r;
}

}  // namespace drv
}  // namespace apo

extern "C" {

int apo_find_repeats(apo_ctx *c, const apo_window *w, const apo_repeats_params *p,
                     apo_repeats_out *out, void *stream) {
  if (!c || !w || !p || !out || !out->counts) {
    set_error("apo_find_repeats: null argument");
    return APO_EINVAL;
  }
  const uint64_t off[2] = {0, w->n};
  apo_repeats_out o = *out;
  o.cand_off = o.sel_off = o.trace_off = nullptr;
  int r;
  if (c->graph_mode) {  // a repeated call on the same buffers replays as one graph
    const apo_windows ws{1, w->tokens, w->token_bytes, off};
    r = graph_batched(c, &ws, p, &o, static_cast<cudaStream_t>(stream));
  } else {
    r = drv::find_repeats_driver(c, w->tokens, w->token_bytes, w->n, off, 1, p, &o,
                                 static_cast<cudaStream_t>(stream));
  }
  for (int k = 0; k < 4; ++k) out->counts[k] = o.counts[k];
  return r;
}

int apo_find_repeats_batched(apo_ctx *c, const apo_windows *ws, const apo_repeats_params *p,
                             apo_repeats_out *out, void *stream) {
  if (!c || !ws || !p || !out || !out->counts || !ws->win_off) {
    set_error("apo_find_repeats_batched: null argument");
    return APO_EINVAL;
  }
  if (ws->n_windows == 0 || ws->n_windows > 0x7fffffffull || ws->win_off[0] != 0) {
    set_error("apo_find_repeats_batched: need 1 <= n_windows and win_off[0] == 0");
    return APO_EINVAL;
  }
  for (uint64_t w = 0; w < ws->n_windows; ++w) {
    if (ws->win_off[w + 1] < ws->win_off[w]) {
      set_error("apo_find_repeats_batched: win_off must be non-decreasing");
      return APO_EINVAL;
    }
  }
  if (c->graph_mode) return graph_batched(c, ws, p, out, static_cast<cudaStream_t>(stream));
  return drv::find_repeats_driver(c, ws->tokens, ws->token_bytes, ws->win_off[ws->n_windows], ws->win_off,
                             (uint32_t)ws->n_windows, p, out, static_cast<cudaStream_t>(stream));
}

int apo_graph_stats(apo_ctx *c, uint64_t *replays, uint64_t *captures, uint64_t *discarded) {
  if (!c || !replays || !captures || !discarded) {
    set_error("apo_graph_stats: null argument");
    return APO_EINVAL;
  }
  graph_stats(c, replays, captures, discarded);
  return APO_OK;
}

int apo_graph_mode(apo_ctx *c, int enable) {
  if (!c) {
    set_error("apo_graph_mode: null context");
    return APO_EINVAL;
  }
  APO_CUDA_TRY(cudaSetDevice(c->device));
  c->graph_mode = enable != 0;
  if (!enable) graph_cache_free(c);
  return APO_OK;
}

int apo_match_candidates(apo_ctx *c, const apo_patterns *p, const void *stream_tokens, uint64_t n,
                         uint32_t *match_end, uint32_t *match_id, uint64_t cap, uint64_t *count,
                         void *stream) {
  if (!c || !p || !count) {
    set_error("apo_match_candidates: null argument");
    return APO_EINVAL;
  }
  *count = 0;
  if (p->n_patterns == 0 || (p->token_bytes != 4 && p->token_bytes != 8)) {
    set_error("apo_match_candidates: need at least one pattern and token_bytes 4 or 8");
    return APO_EINVAL;
  }
  if (p->n_patterns >= 0xffffffffull || n >= 0xffffffffull) {
    set_error("apo_match_candidates: too many patterns or stream tokens");
    return APO_EINVAL;
  }
  if (p->pat_off) {
    if (p->pat_off[0] != 0) {
      set_error("apo_match_candidates: pat_off[0] must be 0");
      return APO_EINVAL;
    }
    for (uint64_t q = 0; q < p->n_patterns; ++q) {
      if (p->pat_off[q + 1] <= p->pat_off[q]) {
        set_error("apo_match_candidates: empty pattern or decreasing offsets");
        return APO_EINVAL;
      }
    }
  } else if (!p->pat_start || !p->pat_len) {
    set_error("apo_match_candidates: give pat_off (host CSR) or pat_start and pat_len (device)");
    return APO_EINVAL;
  }
  if (!p->tokens || (n > 0 && !stream_tokens) || (cap > 0 && (!match_end || !match_id))) {
    set_error("apo_match_candidates: null tokens or outputs");
    return APO_EINVAL;
  }
  APO_CUDA_TRY(cudaSetDevice(c->device));
  return match_patterns(c, p, stream_tokens, n, match_end, match_id, cap, count,
                        static_cast<cudaStream_t>(stream));
}

int apo_replay(apo_ctx *c, const void *stream_tokens, uint64_t n, int token_bytes,
               const apo_replay_traces *tr, const apo_replay_params *prm, apo_replay_out *out, void *stream) {
  if (!c || !tr || !prm || !out || !out->counts) {
    set_error("apo_replay: null context, traces, params or outputs");
    return APO_EINVAL;
  }
  if (token_bytes != 4 && token_bytes != 8) {
    set_error("apo_replay: token_bytes must be 4 or 8");
    return APO_EINVAL;
  }
  if (n >= 0x7fffffffull || tr->n_traces >= 0x7fffffffull) {
    set_error("apo_replay: at most 2^31 - 2 tasks and 2^31 - 2 traces");
    return APO_EINVAL;
  }
  if (prm->bonus_num < 1 || prm->bonus_num > 65535 || prm->bonus_den < 1 || prm->bonus_den > 65535) {
    set_error("apo_replay: bonus_num and bonus_den must lie in 1 .. 65535");
    return APO_EINVAL;
  }
  if ((n > 0 && !stream_tokens) || (tr->n_traces > 0 && (!tr->start || !tr->len || !tr->ingest)) ||
      (out->rep_cap > 0 && (!out->rep_end || !out->rep_len || !out->rep_trace))) {
    set_error("apo_replay: null stream, trace arrays or replay outputs");
    return APO_EINVAL;
  }
  APO_CUDA_TRY(cudaSetDevice(c->device));
  return replay_stream(c, stream_tokens, n, token_bytes, tr, prm, out, static_cast<cudaStream_t>(stream));
}

int apo_optimum_batched(apo_ctx *c, const apo_windows *ws, uint32_t min_len, uint32_t *best, uint32_t *wit_start,
                        uint32_t *wit_len, uint32_t *wit_count, void *stream) {
  if (!c || !ws || !ws->win_off || !best || !wit_start || !wit_len || !wit_count) {
    set_error("apo_optimum_batched: null context, windows or outputs");
    return APO_EINVAL;
  }
  if (ws->token_bytes != 4 && ws->token_bytes != 8) {
    set_error("apo_optimum_batched: token_bytes must be 4 or 8");
    return APO_EINVAL;
  }
  if (ws->n_windows == 0 || ws->n_windows > 0x7fffffffull || ws->win_off[0] != 0 || min_len == 0) {
    set_error("apo_optimum_batched: need 1 <= n_windows, win_off[0] == 0 and min_len >= 1");
    return APO_EINVAL;
  }
  for (uint64_t w = 0; w < ws->n_windows; ++w) {
    if (ws->win_off[w + 1] < ws->win_off[w]) {
      set_error("apo_optimum_batched: win_off must be non-decreasing");
      return APO_EINVAL;
    }
  }
  if (ws->win_off[ws->n_windows] >= 0x7fffffffull || (ws->win_off[ws->n_windows] > 0 && !ws->tokens)) {
    set_error("apo_optimum_batched: null tokens or too many tokens");
    return APO_EINVAL;
  }
  APO_CUDA_TRY(cudaSetDevice(c->device));
  return optimum_batched(c, ws, min_len, best, wit_start, wit_len, wit_count, static_cast<cudaStream_t>(stream));
}

int apo_profile_enable(apo_ctx *c, int enable) {
  if (!c) {
    set_error("apo_profile_enable: null context");
    return APO_EINVAL;
  }
  c->prof.resolve();
  c->prof.timing = enable != 0;
  return APO_OK;
}

int apo_profile_reset(apo_ctx *c) {
  if (!c) {
    set_error("apo_profile_reset: null context");
    return APO_EINVAL;
  }
  c->prof.resolve();
  for (int k = 0; k < kScopes * kKCount; ++k) {
    c->prof.launches[k] = 0;
    c->prof.units[k] = 0;
    c->prof.ms[k] = 0;
  }
  return APO_OK;
}

int apo_profile_read(apo_ctx *c, int index, char *name, size_t name_cap, uint64_t *launches,
                     double *ms, uint64_t *units) {
  if (!c || index < 0 || index >= kScopes * kKCount) {
    set_error("apo_profile_read: null context or index out of range");
    return APO_EINVAL;
  }
  c->prof.resolve();
  if (name && name_cap) {
    static const char *const kPrefix[kScopes] = {"", "ac.", "rep."};
    const std::string nm = std::string(kPrefix[index / kKCount]) + kKernelNames[index % kKCount];
    strncpy(name, nm.c_str(), name_cap - 1);
    name[name_cap - 1] = 0;
  }
  if (launches) *launches = c->prof.launches[index];
  if (ms) *ms = c->prof.ms[index];
  if (units) *units = c->prof.units[index];
  return APO_OK;
}

int apo_sort_tuning(apo_ctx *c, int mode) {
  if (!c || mode < 0 || mode >= 2 + sort_shape_count()) {
    set_error("apo_sort_tuning: null context or mode not 0, 1 or 2 + a shape index");
    return APO_EINVAL;
  }
  c->tuner.mode = mode;
  return APO_OK;
}

int apo_sort_tuning_read(apo_ctx *c, int index, uint32_t *size_log2, uint32_t *key_bits, uint32_t *trial_n,
                         int *threads, int *items, int *digit_bits, double *best_ms, double *default_ms) {
  if (!c || index < 0) {
    set_error("apo_sort_tuning_read: null context or negative index");
    return APO_EINVAL;
  }
  int k = 0;
  const SortTable &tb = sort_table(c->device);
  sort_table_lock(true);
  for (int cls = 0; cls < kTuneClasses; ++cls)
    for (int bits = 0; bits < kTuneBits; ++bits) {
      const int id = tb.choice[cls][bits];
      if (id < 0) continue;
      if (k++ != index) continue;
      int th = 0, it = 0, db = 0;
      sort_shape_info(id, &th, &it, &db);
      if (size_log2) *size_log2 = (uint32_t)(cls + kTuneMinBits);
      if (key_bits) *key_bits = (uint32_t)bits;
      if (trial_n) *trial_n = tb.trial_n[cls][bits];
      if (threads) *threads = th;
      if (items) *items = it;
      if (digit_bits) *digit_bits = db;
      if (best_ms) *best_ms = tb.best_ms[cls][bits];
      if (default_ms) *default_ms = tb.default_ms[cls][bits];
      sort_table_lock(false);
      return APO_OK;
    }
  sort_table_lock(false);
  set_error("apo_sort_tuning_read: index past the last tuned entry");
  return APO_EINVAL;
}

}  // extern "C"
