// Served atlasing with continuous batching.  Clients (sessions) keep their mesh
// and output buffers on the device and send view requests at any time; the paper
// targets streaming-shading servers that re-atlas every client frame (Sec. 1,
// Sec. 6).  The server owns slots, each a context plus a stream; the number of
// slots is fixed at creation by a device-memory budget.  A request is queued on
// submission and dispatched to the first free slot as soon as its session has no
// request on the GPU, so requests that arrive while others run are admitted as
// slots free up and their work overlaps on the device.  Every request is the same
// launch sequence as fa_atlas_frame, so its results do not depend on what else
// runs.  Host-side and single-threaded: the caller drives it with submit / poll.
#include <chrono>
#include <deque>
#include <new>
#include <vector>

#include "fa_internal.cuh"

namespace {

struct Request {
  uint64_t ticket;
  uint32_t session;
  fa_frame_params params;
  fa_frame_out out;
  double submit_ms;
};

struct Slot {
  fa_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  Request req{};
  double dispatch_ms = 0.0;
};

struct Session {
  bool open = false;
  bool in_flight = false;
  fa_mesh* mesh = nullptr;
  fa_frame_out out{};
  uint64_t bytes = 0;  // device memory the session's registration took
};

struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

size_t free_bytes() {
  size_t f = 0, t = 0;
  if (cudaMemGetInfo(&f, &t) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return f;
}

}  // namespace

struct fa_server {
  fa_config cfg;
  int device = 0;
  uint64_t budget = 0;  // device bytes for slots and sessions
  uint64_t used = 0;
  std::vector<Slot> slots;
  std::vector<Session> sessions;
  std::deque<Request> queue;
  uint64_t next_ticket = 1;
  std::chrono::steady_clock::time_point t0;
  uint32_t max_in_flight = 0;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Dispatch queued requests (FIFO, skipping sessions with a request on the GPU)
// into free slots.
fa_status dispatch(fa_server* s) {
  for (Slot& sl : s->slots) {
    if (sl.busy) continue;
    auto it = s->queue.begin();
    while (it != s->queue.end() && s->sessions[it->session].in_flight) ++it;
    if (it == s->queue.end()) break;
    Request r = *it;
    s->queue.erase(it);
    Session& se = s->sessions[r.session];
    fa_status st = fa::enqueue_frame(sl.ctx, se.mesh, &r.params, nullptr, &r.out, sl.stream);
    if (st == FA_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = FA_E_CUDA;
    if (st != FA_OK) return st;
    sl.busy = true;
    sl.req = r;
    sl.dispatch_ms = s->now_ms();
    se.in_flight = true;
  }
  uint32_t n = 0;
  for (const Slot& sl : s->slots) n += sl.busy;
  if (n > s->max_in_flight) s->max_in_flight = n;
  return FA_OK;
}

}  // namespace

extern "C" {

void fa_server_destroy(fa_server* s) {
  if (!s) return;
  Guard g(s->device);
  cudaDeviceSynchronize();
  for (Session& se : s->sessions)
    if (se.mesh) fa_mesh_release(se.mesh);
  for (Slot& sl : s->slots) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  for (Slot& sl : s->slots)
    if (sl.ctx) fa_destroy(sl.ctx);
  delete s;
}

fa_status fa_server_create(fa_server** out, const fa_config* cfg, uint32_t max_slots, uint64_t budget_bytes,
                           uint32_t* n_slots) {
  if (!out) return FA_E_INVALID_ARG;
  *out = nullptr;
  if (!cfg || max_slots == 0 || max_slots > FA_SERVER_MAX_SLOTS) return FA_E_INVALID_ARG;
  fa_server* s = new (std::nothrow) fa_server;
  if (!s) return FA_E_OUT_OF_MEMORY;
  s->cfg = *cfg;
  s->device = cfg->device;
  s->budget = budget_bytes;
  s->t0 = std::chrono::steady_clock::now();
  Guard g(s->device);
  // slots while they fit the budget (the first one must)
  for (uint32_t i = 0; i < max_slots; ++i) {
    const size_t before = free_bytes();
    Slot sl;
    fa_status st = fa_create(&sl.ctx, cfg);
    if (st == FA_OK && (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      st = FA_E_CUDA;
    }
    const size_t after = free_bytes();
    const uint64_t cost = before > after ? before - after : 0;
    if (st == FA_OK && s->used + cost > s->budget) st = FA_E_OUT_OF_MEMORY;
    if (st != FA_OK) {
      if (sl.done) cudaEventDestroy(sl.done);
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.ctx) fa_destroy(sl.ctx);
      if (i == 0) {
        fa_server_destroy(s);
        return st;
      }
      break;
    }
    s->used += cost;
    s->slots.push_back(sl);
  }
  if (fa::pack_set_smem_limit() != FA_OK) {
    cudaGetLastError();
    fa_server_destroy(s);
    return FA_E_CUDA;
  }
  for (Slot& sl : s->slots) sl.ctx->pack_smem_set = 1;
  if (n_slots) *n_slots = (uint32_t)s->slots.size();
  *out = s;
  return FA_OK;
}

fa_status fa_server_session_open(fa_server* s, const float* d_pos, uint32_t V, const uint32_t* d_idx, uint32_t T,
                                 const fa_frame_out* out, uint32_t* session) {
  if (!s || !session) return FA_E_INVALID_ARG;
  Guard g(s->device);
  const size_t before = free_bytes();
  fa_mesh* m = nullptr;
  fa_status st = fa_mesh_register(s->slots[0].ctx, d_pos, V, d_idx, T, &m, nullptr);
  if (st != FA_OK) return st;
  if (cudaStreamSynchronize(nullptr) != cudaSuccess) {
    cudaGetLastError();
    fa_mesh_release(m);
    return FA_E_CUDA;
  }
  const size_t after = free_bytes();
  const uint64_t cost = before > after ? before - after : 0;
  if (s->used + cost > s->budget) {  // admission: the session does not fit the budget
    fa_mesh_release(m);
    return FA_E_OUT_OF_MEMORY;
  }
  s->used += cost;
  Session se;
  se.open = true;
  se.mesh = m;
  se.bytes = cost;
  if (out) se.out = *out;
  s->sessions.push_back(se);
  *session = (uint32_t)(s->sessions.size() - 1);
  return FA_OK;
}

fa_status fa_server_session_close(fa_server* s, uint32_t session) {
  if (!s || session >= s->sessions.size() || !s->sessions[session].open) return FA_E_INVALID_ARG;
  Session& se = s->sessions[session];
  if (se.in_flight) return FA_E_INVALID_ARG;
  for (const Request& r : s->queue)
    if (r.session == session) return FA_E_INVALID_ARG;
  Guard g(s->device);
  fa_mesh_release(se.mesh);
  se.mesh = nullptr;
  se.open = false;
  s->used -= se.bytes;
  return FA_OK;
}

fa_status fa_server_submit(fa_server* s, uint32_t session, const fa_frame_params* params, const fa_frame_out* out,
                           uint64_t* ticket) {
  if (!s || !params || session >= s->sessions.size() || !s->sessions[session].open) return FA_E_INVALID_ARG;
  Session& se = s->sessions[session];
  Request r;
  r.session = session;
  r.params = *params;
  r.out = out ? *out : se.out;
  fa_status st = fa::check_frame(s->slots[0].ctx, se.mesh, &r.params, nullptr, &r.out);
  if (st != FA_OK) return st;
  r.ticket = s->next_ticket++;
  r.submit_ms = s->now_ms();
  s->queue.push_back(r);
  if (ticket) *ticket = r.ticket;
  Guard g(s->device);
  return dispatch(s);
}

fa_status fa_server_poll(fa_server* s, fa_server_done* done, uint32_t max_done, uint32_t* n_done) {
  if (!s || !n_done || (max_done && !done)) return FA_E_INVALID_ARG;
  *n_done = 0;
  Guard g(s->device);
  for (Slot& sl : s->slots) {
    if (!sl.busy || *n_done >= max_done) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) {
      cudaGetLastError();
      return FA_E_CUDA;
    }
    fa_server_done& d = done[(*n_done)++];
    d.ticket = sl.req.ticket;
    d.session = sl.req.session;
    d.slot = (uint32_t)(&sl - s->slots.data());
    d.submit_ms = sl.req.submit_ms;
    d.dispatch_ms = sl.dispatch_ms;
    d.done_ms = s->now_ms();
    sl.busy = false;
    s->sessions[sl.req.session].in_flight = false;
  }
  return dispatch(s);
}

fa_status fa_server_stats(const fa_server* s, uint32_t* queued, uint32_t* running, uint32_t* max_running,
                          uint64_t* used_bytes) {
  if (!s) return FA_E_INVALID_ARG;
  uint32_t run = 0;
  for (const Slot& sl : s->slots) run += sl.busy;
  if (queued) *queued = (uint32_t)s->queue.size();
  if (running) *running = run;
  if (max_running) *max_running = s->max_in_flight;
  if (used_bytes) *used_bytes = s->used;
  return FA_OK;
}

double fa_server_now_ms(const fa_server* s) { return s ? s->now_ms() : 0.0; }

}  // extern "C"
