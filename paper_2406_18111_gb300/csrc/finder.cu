// The online trace finder: Alg. 1's TraceFinder over a stream of tokens,
// sampling its history buffer by the exponentiated ruler function (Sec. 4.4)
// and running each sampled slice as an asynchronous FindRepeats (Alg. 2) on
// the served form.  Host-side runtime only: the analyses are GPU requests of
// the server.
#include <cstring>
#include <deque>
#include <vector>

#include "apo_internal.cuh"

namespace {

struct Pending {
  uint64_t index, start, len, id;
};

}  // namespace

struct apo_finder {
  apo_server *srv = nullptr;
  apo_finder_config cfg{};
  int tb = 4;
  std::vector<uint8_t> ring;  // the most recent buffer_tokens tokens, position p at p % buffer_tokens
  uint64_t pushed = 0;        // tokens so far
  uint64_t points = 0;        // analysis points reached
  uint64_t analysed = 0;      // tokens handed to analyses
  std::deque<Pending> pending;
  std::vector<uint8_t> slice;
  std::vector<uint32_t> out_len;
  std::vector<uint64_t> out_start;
  bool has_out = false;
  uint64_t out_id = 0;
};

namespace apo {

// How many times 2 divides i (i >= 1): the ruler function.
inline int ruler(uint64_t i) {
  int r = 0;
  while ((i & 1) == 0) {
    i >>= 1;
    ++r;
  }
  return r;
}

}  // namespace apo

using namespace apo;

extern "C" {

int apo_finder_create(apo_finder **out, apo_server *server, const apo_finder_config *cfg) {
  if (!out || !server || !cfg || cfg->unit == 0 || cfg->buffer_tokens < cfg->unit ||
      cfg->buffer_tokens > (1ull << 31)) {
    set_error("apo_finder_create: bad argument (unit >= 1, unit <= buffer_tokens <= 2^31)");
    return APO_EINVAL;
  }
  auto *f = new apo_finder();
  f->srv = server;
  f->cfg = *cfg;
  f->tb = server_token_bytes(server);
  f->ring.resize(cfg->buffer_tokens * f->tb);
  *out = f;
  return APO_OK;
}

int apo_finder_push(apo_finder *f, const void *tokens, uint64_t n, uint64_t *submitted) {
  if (!f || (n && !tokens)) {
    set_error("apo_finder_push: bad argument");
    return APO_EINVAL;
  }
  const uint64_t B = f->cfg.buffer_tokens, c = f->cfg.unit;
  const int tb = f->tb;
  const uint8_t *src = static_cast<const uint8_t *>(tokens);
  uint64_t done = 0, subs = 0;
  while (done < n) {
    // copy up to the next analysis point
    const uint64_t next_point = (f->pushed / c + 1) * c;
    const uint64_t take = std::min(n - done, next_point - f->pushed);
    for (uint64_t k = 0; k < take;) {
      const uint64_t pos = (f->pushed + k) % B;
      const uint64_t run = std::min(take - k, B - pos);
      memcpy(f->ring.data() + pos * tb, src + (done + k) * tb, run * tb);
      k += run;
    }
    f->pushed += take;
    done += take;
    if (f->pushed % c) continue;
    // analysis point i: the most recent c * 2^ruler(i) tokens
    const uint64_t i = ++f->points;
    const int r = ruler(i);
    uint64_t len = r >= 63 ? B : c << r;
    len = std::min(len, std::min(B, f->pushed));
    const uint64_t start = f->pushed - len;
    f->slice.resize(len * tb);
    for (uint64_t k = 0; k < len;) {
      const uint64_t pos = (start + k) % B;
      const uint64_t run = std::min(len - k, B - pos);
      memcpy(f->slice.data() + k * tb, f->ring.data() + pos * tb, run * tb);
      k += run;
    }
    uint64_t id = 0;
    const int st = apo_server_submit(f->srv, f->slice.data(), len, &id);
    if (st != APO_OK) return st;
    f->pending.push_back({i, start, len, id});
    f->analysed += len;
    ++subs;
  }
  if (submitted) *submitted = subs;
  return APO_OK;
}

int apo_finder_poll(apo_finder *f, int wait, apo_finder_result *out) {
  if (!f || !out) {
    set_error("apo_finder_poll: bad argument");
    return APO_EINVAL;
  }
  if (f->has_out) {  // the previous result's arrays are released now
    apo_server_release(f->srv, f->out_id);
    f->has_out = false;
  }
  if (f->pending.empty()) return APO_ECAPACITY;
  const Pending p = f->pending.front();
  apo_request_result r{};
  const int st = wait ? apo_server_wait(f->srv, p.id, &r) : apo_server_poll(f->srv, p.id, &r);
  if (st == APO_EAGAIN) return APO_EAGAIN;
  if (st != APO_OK) return st;
  f->pending.pop_front();
  f->out_len.assign(r.trace_len, r.trace_len + r.n_traces);
  f->out_start.resize(r.n_traces);
  for (uint64_t t = 0; t < r.n_traces; ++t) f->out_start[t] = p.start + r.trace_start[t];
  out->index = p.index;
  out->slice_start = p.start;
  out->slice_len = p.len;
  out->status = r.status;
  out->n_traces = r.n_traces;
  out->trace_len = f->out_len.data();
  out->trace_start = f->out_start.data();
  out->t_submit = r.t_submit;
  out->t_done = r.t_done;
  f->has_out = true;
  f->out_id = p.id;
  return APO_OK;
}

int apo_finder_stats(apo_finder *f, uint64_t *pushed, uint64_t *analyses, uint64_t *analysed_tokens) {
  if (!f) return APO_EINVAL;
  if (pushed) *pushed = f->pushed;
  if (analyses) *analyses = f->points;
  if (analysed_tokens) *analysed_tokens = f->analysed;
  return APO_OK;
}

int apo_finder_destroy(apo_finder *f) {
  if (!f) return APO_OK;
  if (f->has_out) apo_server_release(f->srv, f->out_id);
  for (const Pending &p : f->pending) {
    apo_request_result r{};
    apo_server_wait(f->srv, p.id, &r);
    apo_server_release(f->srv, p.id);
  }
  delete f;
  return APO_OK;
}

}  // extern "C"
