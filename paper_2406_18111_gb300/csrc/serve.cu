// The served form: continuous batching of repeat-finding requests.
//
// Alg. 1 hands each history slice to an asynchronous FindRepeats while the
// application keeps issuing tasks, and ingests results as they complete.
// Here requests arrive through apo_server_submit at any time.  Each lane (a
// worker thread with its own context and stream) repeatedly takes the
// requests waiting at that moment, in arrival order, up to the admission
// budget (tokens per batch, which bounds the batch's device footprint) and a
// window count, concatenates them into pinned memory, runs the batched
// analysis and publishes each request's slice of the results.  With several
// lanes, one batch computes while the next is being formed and copied, and
// their kernels overlap on the device; a request arriving while batches run
// joins the next batch any lane forms.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
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

template <class T>
struct DevBuf {  // grow-only device buffer
  T *p = nullptr;
  size_t cap = 0;
  int ensure(size_t n) {
    if (n <= cap) return APO_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return APO_ENOMEM;
    }
    cap = n;
    return APO_OK;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
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

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void lane_main();
};

void apo_server::lane_main() {
  cudaSetDevice(device);
  apo_ctx *ctx = nullptr;
  if (apo_create(&ctx, device) != APO_OK) ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  const int tb = cfg.token_bytes;
  uint8_t *host_in = nullptr;
  size_t host_cap = 0;
  DevBuf<uint8_t> d_tok;
  DevBuf<uint32_t> d_out;
  std::vector<uint32_t> h_out;
  std::vector<uint64_t> win_off, sel_off, trace_off;
  while (true) {
    std::vector<std::shared_ptr<Request>> batch;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stopping || !pending.empty(); });
      if (pending.empty()) break;  // stopping and drained
      uint64_t tokens = 0;
      while (!pending.empty() && batch.size() < cfg.max_batch_windows) {
        const auto &r = pending.front();
        if (!batch.empty() && tokens + r->n > cfg.max_batch_tokens) break;
        tokens += r->n;
        batch.push_back(r);
        pending.pop_front();
      }
    }
    const double t_start = now();
    const size_t W = batch.size();
    win_off.assign(W + 1, 0);
    for (size_t w = 0; w < W; ++w) win_off[w + 1] = win_off[w] + batch[w]->n;
    const uint64_t total = win_off[W];
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
    const uint64_t K = total / std::max<uint32_t>(cfg.min_len, 1) + 1;
    if (st == APO_OK) st = d_tok.ensure(total * tb + 1);
    if (st == APO_OK) st = d_out.ensure(5 * K);
    uint64_t counts[4] = {0, 0, 0, 0};
    if (st == APO_OK) {
      for (size_t w = 0; w < W; ++w)
        memcpy(host_in + win_off[w] * tb, batch[w]->tokens.data(), batch[w]->n * tb);
      if (cudaMemcpyAsync(d_tok.p, host_in, total * tb, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        st = APO_ECUDA;
    }
    if (st == APO_OK) {
      sel_off.assign(W + 1, 0);
      trace_off.assign(W + 1, 0);
      apo_windows ws{W, d_tok.p, tb, win_off.data()};
      apo_repeats_params pr{cfg.min_len, 0};
      apo_repeats_out o{};
      o.sel_start = d_out.p;
      o.sel_len = d_out.p + K;
      o.sel_trace = d_out.p + 2 * K;
      o.trace_len = d_out.p + 3 * K;
      o.trace_start = d_out.p + 4 * K;
      o.sel_cap = o.trace_cap = K;
      o.counts = counts;
      o.sel_off = sel_off.data();
      o.trace_off = trace_off.data();
      st = apo_find_repeats_batched(ctx, &ws, &pr, &o, stream);
    }
    if (st == APO_OK) {
      h_out.resize(5 * K);
      for (int a = 0; a < 5 && st == APO_OK; ++a)
        if (cudaMemcpyAsync(h_out.data() + a * K, d_out.p + a * K,
                            (a < 3 ? counts[1] : counts[2]) * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            stream) != cudaSuccess)
          st = APO_ECUDA;
      if (cudaStreamSynchronize(stream) != cudaSuccess) st = APO_ECUDA;
    }
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
    cv_done.notify_all();
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
  auto *s = new apo_server();
  s->device = device;
  s->cfg = *cfg;
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

int apo_server_destroy(apo_server *s) {
  if (!s) return APO_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->lanes) t.join();
  delete s;
  return APO_OK;
}

}  // extern "C"
