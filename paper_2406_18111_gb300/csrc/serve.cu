// The served form: continuous batching of repeat-finding requests, admitted
// by device-memory footprint.
//
// Alg. 1 hands each history slice to an asynchronous FindRepeats while the
// application keeps issuing tasks, and ingests results as they complete.
// Here requests arrive through apo_server_submit at any time.  Each lane (a
// worker thread with its own context and stream) repeatedly takes the
// requests waiting at that moment, in arrival order, concatenates them into
// pinned memory, runs the batched analysis and publishes each request's slice
// of the results.  With several lanes, one batch computes while the next is
// being formed and copied, and their kernels overlap on the device; a request
// arriving while batches run joins the next batch any lane forms.
//
// Admission by footprint.  The server owns one device pool of hbm_budget
// bytes, allocated once.  A batch's footprint is its tokens, its output
// arrays and the scratch apo_find_repeats_workspace reports for its windows;
// a lane carves one slice of that size from the pool (first fit) and hands
// the scratch part to its context with apo_set_workspace, so the batches in
// flight never hold more than the budget together.  A lane grows its batch
// request by request while the bigger footprint still fits in a free slice
// (and within max_batch_tokens / max_batch_windows); when not even the first
// waiting request fits, the lane waits until a finishing batch returns its
// slice.  A request whose footprint exceeds the whole budget fails with
// APO_ECAPACITY.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "apo_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  std::vector<uint8_t> tokens;  // n * token_bytes
  uint64_t n = 0;
  bool done = false;
  int status = APO_OK;
  std::vector<uint32_t> sel_start, sel_len, sel_trace, trace_len, trace_start;
  double t_submit = 0, t_start = 0, t_done = 0;
  uint64_t batch_windows = 0;
};

// First-fit allocator over the pool (offsets, 256-byte granules); free
// ranges are coalesced with their neighbours.
struct Pool {
  uint64_t cap = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> size
  void init(uint64_t bytes) {
    cap = bytes;
    free_.clear();
    if (bytes) free_[0] = bytes;
  }
  bool take(uint64_t bytes, uint64_t *off) {
    bytes = (bytes + 255) & ~255ull;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t rest = it->second - bytes;
      const uint64_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      return true;
    }
    return false;
  }
  void give(uint64_t off, uint64_t bytes) {
    bytes = (bytes + 255) & ~255ull;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

struct apo_server {
  int device = 0;
  apo_server_config cfg{};
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_id = 1;
  bool stopping = false;
  std::vector<std::thread> lanes;
  char *pool_base = nullptr;
  Pool pool;
  uint64_t in_flight = 0;           // batches holding a slice
  uint64_t held = 0, held_max = 0;  // bytes held by them (now, most so far)
  uint64_t pool_gen = 0;            // bumped whenever a slice is returned

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void lane_main();
  uint64_t footprint(const std::vector<uint64_t> &win_off) const;
};

// Tokens, five output arrays of total / min_len + 1 entries, and the
// analysis scratch of these windows (each part 256-byte aligned).
uint64_t apo_server::footprint(const std::vector<uint64_t> &win_off) const {
  const uint64_t W = win_off.size() - 1, total = win_off[W];
  const uint64_t K = total / std::max<uint32_t>(cfg.min_len, 1) + 1;
  apo_windows ws{W, nullptr, cfg.token_bytes, win_off.data()};
  uint64_t scratch = 0;
  apo_find_repeats_workspace(nullptr, &ws, &scratch);
  auto al = [](uint64_t b) { return (b + 255) & ~255ull; };
  return al(total * cfg.token_bytes + 16) + al(5 * K * 4) + al(scratch);
}

void apo_server::lane_main() {
  cudaSetDevice(device);
  apo_ctx *ctx = nullptr;
  if (apo_create(&ctx, device) != APO_OK) ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  const int tb = cfg.token_bytes;
  uint8_t *host_in = nullptr;
  size_t host_cap = 0;
  std::vector<uint32_t> h_out;
  std::vector<uint64_t> win_off, trial, sel_off, trace_off;
  while (true) {
    std::vector<std::shared_ptr<Request>> batch;
    std::vector<std::shared_ptr<Request>> refused;
    uint64_t slice_off = 0, slice_bytes = 0;
    {
      std::unique_lock<std::mutex> lk(mu);
      while (true) {
        cv_work.wait(lk, [&] { return stopping || !pending.empty(); });
        if (pending.empty()) break;  // stopping and drained
        // grow the batch in arrival order while its footprint still fits
        win_off.assign(1, 0);
        uint64_t fit = 0, off = 0;
        size_t take = 0;
        while (take < pending.size() && take < cfg.max_batch_windows) {
          const uint64_t n = pending[take]->n;
          if (take > 0 && win_off.back() + n > cfg.max_batch_tokens) break;
          trial = win_off;
          trial.push_back(win_off.back() + n);
          const uint64_t need = footprint(trial);
          if (take == 0 && need > pool.cap) {  // can never fit: refuse it
            refused.push_back(pending.front());
            pending.pop_front();
            continue;
          }
          if (take > 0) pool.give(off, fit);  // the larger slice replaces the smaller one
          uint64_t o = 0;
          if (!pool.take(need, &o)) {
            if (take > 0 && !pool.take(fit, &off)) take = 0;  // (cannot fail: that space was just free)
            break;
          }
          off = o;
          fit = need;
          win_off.swap(trial);
          ++take;
        }
        if (take == 0) {
          if (!refused.empty()) break;  // publish the refusals
          // the first waiting request does not fit next to the batches in
          // flight: wait until one of them returns its slice
          const uint64_t g0 = pool_gen;
          cv_work.wait(lk, [&] { return in_flight == 0 || pool_gen != g0; });
          continue;
        }
        for (size_t k = 0; k < take; ++k) {
          batch.push_back(pending.front());
          pending.pop_front();
        }
        slice_off = off;
        slice_bytes = fit;
        ++in_flight;
        held += fit;
        held_max = std::max(held_max, held);
        break;
      }
    }
    if (!refused.empty()) {
      const double t = now();
      std::lock_guard<std::mutex> lk(mu);
      for (auto &r : refused) {
        r->status = APO_ECAPACITY;
        r->t_start = r->t_done = t;
        r->done = true;
        r->tokens.clear();
        r->tokens.shrink_to_fit();
      }
      cv_done.notify_all();
    }
    if (batch.empty()) {
      if (refused.empty()) break;  // stopping and drained
      continue;
    }
    const double t_start = now();
    const size_t W = batch.size();
    const uint64_t total = win_off[W];
    const uint64_t K = total / std::max<uint32_t>(cfg.min_len, 1) + 1;
    auto al = [](uint64_t b) { return (b + 255) & ~255ull; };
    char *slice = pool_base + slice_off;
    uint8_t *d_tok = reinterpret_cast<uint8_t *>(slice);
    uint32_t *d_out = reinterpret_cast<uint32_t *>(slice + al(total * tb + 16));
    char *scratch = slice + al(total * tb + 16) + al(5 * K * 4);
    const uint64_t scratch_bytes = slice_bytes - (uint64_t)(scratch - slice);
    int st = ctx ? APO_OK : APO_ECUDA;
    if (st == APO_OK && total * tb > host_cap) {
      if (host_in) cudaFreeHost(host_in);
      host_cap = std::max<size_t>(total * tb, 1 << 20);
      if (cudaMallocHost(&host_in, host_cap) != cudaSuccess) {
        cudaGetLastError();
        host_in = nullptr;
        host_cap = 0;
        st = APO_ENOMEM;
      }
    }
    if (st == APO_OK) st = apo_set_workspace(ctx, scratch, scratch_bytes);
    uint64_t counts[4] = {0, 0, 0, 0};
    if (st == APO_OK) {
      for (size_t w = 0; w < W; ++w)
        memcpy(host_in + win_off[w] * tb, batch[w]->tokens.data(), batch[w]->n * tb);
      if (cudaMemcpyAsync(d_tok, host_in, total * tb, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        st = APO_ECUDA;
    }
    if (st == APO_OK) {
      sel_off.assign(W + 1, 0);
      trace_off.assign(W + 1, 0);
      apo_windows ws{W, d_tok, tb, win_off.data()};
      apo_repeats_params pr{cfg.min_len, 0};
      apo_repeats_out o{};
      o.sel_start = d_out;
      o.sel_len = d_out + K;
      o.sel_trace = d_out + 2 * K;
      o.trace_len = d_out + 3 * K;
      o.trace_start = d_out + 4 * K;
      o.sel_cap = o.trace_cap = K;
      o.counts = counts;
      o.sel_off = sel_off.data();
      o.trace_off = trace_off.data();
      st = apo_find_repeats_batched(ctx, &ws, &pr, &o, stream);
    }
    if (st == APO_OK) {
      h_out.resize(5 * K);
      for (int a = 0; a < 5 && st == APO_OK; ++a)
        if (cudaMemcpyAsync(h_out.data() + a * K, d_out + a * K,
                            (a < 3 ? counts[1] : counts[2]) * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            stream) != cudaSuccess)
          st = APO_ECUDA;
      if (cudaStreamSynchronize(stream) != cudaSuccess) st = APO_ECUDA;
    }
    if (ctx) apo_set_workspace(ctx, nullptr, 0);  // the stream is idle: the slice goes back
    const double t_done = now();
    std::lock_guard<std::mutex> lk(mu);
    for (size_t w = 0; w < W; ++w) {
      Request &r = *batch[w];
      r.status = st;
      if (st == APO_OK) {
        const uint64_t s0 = sel_off[w], s1 = sel_off[w + 1], t0_ = trace_off[w], t1 = trace_off[w + 1];
        r.sel_start.assign(h_out.begin() + s0, h_out.begin() + s1);
        r.sel_len.assign(h_out.begin() + K + s0, h_out.begin() + K + s1);
        r.sel_trace.assign(h_out.begin() + 2 * K + s0, h_out.begin() + 2 * K + s1);
        r.trace_len.assign(h_out.begin() + 3 * K + t0_, h_out.begin() + 3 * K + t1);
        r.trace_start.assign(h_out.begin() + 4 * K + t0_, h_out.begin() + 4 * K + t1);
      }
      r.t_start = t_start;
      r.t_done = t_done;
      r.batch_windows = W;
      r.done = true;
      r.tokens.clear();
      r.tokens.shrink_to_fit();
    }
    pool.give(slice_off, slice_bytes);
    --in_flight;
    held -= slice_bytes;
    ++pool_gen;
    cv_done.notify_all();
    cv_work.notify_all();  // lanes waiting for memory
  }
  if (host_in) cudaFreeHost(host_in);
  if (stream) cudaStreamDestroy(stream);
  apo_destroy(ctx);
}

namespace {

void fill(const Request &r, apo_request_result *o) {
  o->status = r.status;
  o->n = r.n;
  o->n_selected = r.sel_start.size();
  o->n_traces = r.trace_len.size();
  o->sel_start = r.sel_start.data();
  o->sel_len = r.sel_len.data();
  o->sel_trace = r.sel_trace.data();
  o->trace_len = r.trace_len.data();
  o->trace_start = r.trace_start.data();
  o->t_submit = r.t_submit;
  o->t_start = r.t_start;
  o->t_done = r.t_done;
  o->batch_windows = r.batch_windows;
}

}  // namespace

namespace apo {
int server_token_bytes(apo_server *s) { return s->cfg.token_bytes; }
}  // namespace apo

extern "C" {

int apo_server_create(apo_server **out, int device, const apo_server_config *cfg) {
  if (!out || !cfg || cfg->lanes == 0 || cfg->min_len == 0 || cfg->max_batch_windows == 0 ||
      (cfg->token_bytes != 4 && cfg->token_bytes != 8)) {
    apo::set_error("apo_server_create: bad argument (lanes, min_len, max_batch_windows >= 1; "
                   "token_bytes 4 or 8)");
    return APO_EINVAL;
  }
  APO_CUDA_TRY(cudaSetDevice(device));
  auto *s = new apo_server();
  s->device = device;
  s->cfg = *cfg;
  if (s->cfg.hbm_budget == 0) s->cfg.hbm_budget = (uint64_t)16 << 30;
  if (cudaMalloc(&s->pool_base, s->cfg.hbm_budget) != cudaSuccess) {
    cudaGetLastError();
    apo::set_error("apo_server_create: cudaMalloc of the " + std::to_string(s->cfg.hbm_budget) +
                   "-byte pool failed");
    delete s;
    return APO_ENOMEM;
  }
  s->pool.init(s->cfg.hbm_budget);
  s->t0 = Clock::now();
  for (uint32_t l = 0; l < cfg->lanes; ++l) s->lanes.emplace_back([s] { s->lane_main(); });
  *out = s;
  return APO_OK;
}

int apo_server_submit(apo_server *s, const void *tokens, uint64_t n, uint64_t *id) {
  if (!s || !id || (n > 0 && !tokens) || n > 0x7fffffffull) {
    apo::set_error("apo_server_submit: bad argument");
    return APO_EINVAL;
  }
  auto r = std::make_shared<Request>();
  r->n = n;
  r->tokens.resize(n * s->cfg.token_bytes);
  if (n) memcpy(r->tokens.data(), tokens, n * s->cfg.token_bytes);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
      apo::set_error("apo_server_submit: server is stopping");
      return APO_EINVAL;
    }
    r->id = s->next_id++;
    r->t_submit = s->now();
    s->all[r->id] = r;
    s->pending.push_back(r);
    *id = r->id;
  }
  s->cv_work.notify_one();
  return APO_OK;
}

int apo_server_poll(apo_server *s, uint64_t id, apo_request_result *o) {
  if (!s || !o) return APO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) {
    apo::set_error("apo_server_poll: unknown request");
    return APO_EINVAL;
  }
  if (!it->second->done) return APO_EAGAIN;
  fill(*it->second, o);
  return APO_OK;
}

int apo_server_wait(apo_server *s, uint64_t id, apo_request_result *o) {
  if (!s || !o) return APO_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) {
    apo::set_error("apo_server_wait: unknown request");
    return APO_EINVAL;
  }
  auto r = it->second;
  s->cv_done.wait(lk, [&] { return r->done; });
  fill(*r, o);
  return APO_OK;
}

int apo_server_release(apo_server *s, uint64_t id) {
  if (!s) return APO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end() || !it->second->done) {
    apo::set_error("apo_server_release: unknown or unfinished request");
    return APO_EINVAL;
  }
  s->all.erase(it);
  return APO_OK;
}

double apo_server_now(apo_server *s) { return s ? s->now() : 0.0; }

int apo_server_memory(apo_server *s, uint64_t *budget, uint64_t *held, uint64_t *held_max) {
  if (!s) return APO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (budget) *budget = s->cfg.hbm_budget;
  if (held) *held = s->held;
  if (held_max) *held_max = s->held_max;
  return APO_OK;
}

int apo_server_destroy(apo_server *s) {
  if (!s) return APO_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->lanes) t.join();
  cudaSetDevice(s->device);
  if (s->pool_base) cudaFree(s->pool_base);
  delete s;
  return APO_OK;
}

}  // extern "C"
