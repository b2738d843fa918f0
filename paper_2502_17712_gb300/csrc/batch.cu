// Batched multi-view atlasing.  Views are independent problems (one atlas per view,
// Sec. 3), and a single view's frame is a chain of small, latency-bound launches
// that leaves most of the GPU idle.  A batch therefore runs its views on lanes:
// each lane is a context (scratch sized for the batch's maxima) with its own
// stream; the lanes fork from the caller's stream through an event and join back
// into it, so one call is stream-ordered and a CUDA graph captured from it
// atlases the whole batch in one launch, with the lanes as parallel branches.
// The schedule (number of lanes, assignment of views to lanes) changes only
// timing, never results; fa_batch_tune picks it by timing captured graphs.
#include <algorithm>
#include <new>
#include <vector>

#include "fa_internal.cuh"

namespace {

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

// Work estimate of a view for the longest-first assignment: triangles (raster
// front end, chart passes) plus viewport pixels (depth buffer, marking).
uint64_t view_cost(const fa_mesh* m, const fa_frame_params& p) {
  return (uint64_t)m->T + (uint64_t)p.width * p.height;
}

// Views of each lane, in the order the lane runs them.
std::vector<std::vector<uint32_t>> assign(const fa_batch* b, uint32_t n, const fa_mesh* const* meshes,
                                          const fa_frame_params* params) {
  std::vector<std::vector<uint32_t>> lanes(b->active);
  if (b->policy == FA_BATCH_ROUND_ROBIN) {
    for (uint32_t i = 0; i < n; ++i) lanes[i % b->active].push_back(i);
    return lanes;
  }
  std::vector<uint32_t> ord(n);
  for (uint32_t i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t c) {
    return view_cost(meshes[a], params[a]) > view_cost(meshes[c], params[c]);
  });
  std::vector<uint64_t> load(b->active, 0);
  for (uint32_t i : ord) {
    const uint32_t l = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[l].push_back(i);
    load[l] += view_cost(meshes[i], params[i]);
  }
  return lanes;
}

fa_status enqueue_batch(fa_batch* b, uint32_t n, const fa_mesh* const* meshes, const fa_frame_params* params,
                        const fa_frame_out* outs, cudaStream_t s) {
  // every view is checked before anything is enqueued, so a bad view leaves no
  // half-forked lanes behind
  for (uint32_t i = 0; i < n; ++i) {
    fa_status st = fa::check_frame(b->ctx[0], meshes[i], &params[i], nullptr, &outs[i]);
    if (st != FA_OK) return st;
  }
  const auto lanes = assign(b, n, meshes, params);
  FA_CUDA_TRY(cudaEventRecord(b->fork, s));
  for (uint32_t l = 0; l < b->active; ++l) {
    if (lanes[l].empty()) continue;
    FA_CUDA_TRY(cudaStreamWaitEvent(b->stream[l], b->fork, 0));
    fa_status st = FA_OK;
    for (uint32_t i : lanes[l]) {
      st = fa::enqueue_frame(b->ctx[l], meshes[i], &params[i], nullptr, &outs[i], b->stream[l]);
      if (st != FA_OK) break;
    }
    // join even after a failed launch, so that a capture in progress stays joined
    FA_CUDA_TRY(cudaEventRecord(b->join[l], b->stream[l]));
    FA_CUDA_TRY(cudaStreamWaitEvent(s, b->join[l], 0));
    if (st != FA_OK) return st;
  }
  return FA_OK;
}

}  // namespace

extern "C" {

void fa_batch_destroy(fa_batch* b) {
  if (!b) return;
  Guard g(b->device);
  cudaDeviceSynchronize();
  for (fa_ctx* c : b->ctx) fa_destroy(c);
  for (cudaStream_t s : b->stream)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

fa_status fa_batch_create(fa_batch** out, const fa_config* cfg, uint32_t n_lanes) {
  if (!out) return FA_E_INVALID_ARG;
  *out = nullptr;
  if (!cfg || n_lanes == 0 || n_lanes > FA_BATCH_MAX_LANES) return FA_E_INVALID_ARG;
  fa_batch* b = new (std::nothrow) fa_batch;
  if (!b) return FA_E_OUT_OF_MEMORY;
  b->cfg = *cfg;
  b->device = cfg->device;
  b->active = n_lanes;
  for (uint32_t l = 0; l < n_lanes; ++l) {
    fa_ctx* c = nullptr;
    fa_status st = fa_create(&c, cfg);
    if (st != FA_OK) {
      fa_batch_destroy(b);
      return st;
    }
    b->ctx.push_back(c);
  }
  Guard g(b->device);
  // the push kernel's shared-memory limit is set now, not inside a later capture
  if (fa::pack_set_smem_limit() != FA_OK) {
    cudaGetLastError();
    fa_batch_destroy(b);
    return FA_E_CUDA;
  }
  for (fa_ctx* c : b->ctx) c->pack_smem_set = 1;
  b->stream.assign(n_lanes, nullptr);
  b->join.assign(n_lanes, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (uint32_t l = 0; ok && l < n_lanes; ++l) {
    ok = cudaStreamCreateWithFlags(&b->stream[l], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[l], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    fa_batch_destroy(b);
    return FA_E_CUDA;
  }
  *out = b;
  return FA_OK;
}

fa_status fa_batch_mesh_register(fa_batch* b, const float* d_pos, uint32_t V, const uint32_t* d_idx, uint32_t T,
                                 fa_mesh** out, fa_stream_t stream) {
  if (!b) return FA_E_INVALID_ARG;
  return fa_mesh_register(b->ctx[0], d_pos, V, d_idx, T, out, stream);
}

fa_status fa_batch_set_schedule(fa_batch* b, uint32_t lanes, uint32_t policy) {
  if (!b || lanes == 0 || lanes > b->ctx.size() || policy > FA_BATCH_LONGEST_FIRST) return FA_E_INVALID_ARG;
  b->active = lanes;
  b->policy = policy;
  return FA_OK;
}

fa_status fa_batch_get_schedule(const fa_batch* b, uint32_t* lanes, uint32_t* policy) {
  if (!b || !lanes || !policy) return FA_E_INVALID_ARG;
  *lanes = b->active;
  *policy = b->policy;
  return FA_OK;
}

fa_status fa_atlas_batch(fa_batch* b, uint32_t n_views, const fa_mesh* const* meshes,
                         const fa_frame_params* params, const fa_frame_out* outs, fa_stream_t stream) {
  if (!b || (n_views && (!meshes || !params || !outs))) return FA_E_INVALID_ARG;
  Guard g(b->device);
  return enqueue_batch(b, n_views, meshes, params, outs, (cudaStream_t)stream);
}

fa_status fa_batch_tune(fa_batch* b, uint32_t n_views, const fa_mesh* const* meshes, const fa_frame_params* params,
                        const fa_frame_out* outs, uint32_t reps, float* best_ms) {
  if (!b || n_views == 0 || !meshes || !params || !outs) return FA_E_INVALID_ARG;
  for (uint32_t i = 0; i < n_views; ++i) {
    fa_status st = fa::check_frame(b->ctx[0], meshes[i], &params[i], nullptr, &outs[i]);
    if (st != FA_OK) return st;
  }
  if (reps == 0) reps = 3;
  Guard g(b->device);
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    return FA_E_CUDA;
  }
  const uint32_t max_lanes = (uint32_t)b->ctx.size();
  std::vector<uint32_t> cand;
  for (uint32_t l = 1; l < max_lanes; l <<= 1) cand.push_back(l);
  cand.push_back(max_lanes);
  float best = -1.0f;
  uint32_t best_l = b->active, best_p = b->policy, best_m = b->ctx[0]->mid_max_pix,
           best_f = b->ctx[0]->raster_flags, best_u = b->ctx[0]->uf_threads, best_q = b->ctx[0]->push_threads;
  fa_status st = FA_OK;
  // one schedule: capture the batch as the caller would run it (one graph), time it
  auto trial = [&](uint32_t l, uint32_t pol, uint32_t mid, uint32_t fl, uint32_t uf, uint32_t pu) {
    if (st != FA_OK) return;
    b->active = l;
    b->policy = pol;
    for (fa_ctx* c : b->ctx) {
      c->mid_max_pix = mid;
      c->raster_flags = fl;
      c->uf_threads = uf;
      c->push_threads = pu;
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = FA_E_CUDA;
      return;
    }
    fa_status est = enqueue_batch(b, n_views, meshes, params, outs, s);
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (est != FA_OK || ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      st = est != FA_OK ? est : FA_E_CUDA;
      return;
    }
    float ms = 0.0f;
    bool ok = cudaGraphLaunch(exec, s) == cudaSuccess;  // warm-up
    for (uint32_t r = 0; ok && r < reps; ++r) {
      float t = 0.0f;
      ok = cudaEventRecord(e0, s) == cudaSuccess && cudaGraphLaunch(exec, s) == cudaSuccess &&
           cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
      if (ok && (r == 0 || t < ms)) ms = t;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (!ok) {
      cudaGetLastError();
      st = FA_E_CUDA;
      return;
    }
    if (best < 0.0f || ms < best) {
      best = ms;
      best_l = l;
      best_p = pol;
      best_m = mid;
      best_f = fl;
      best_u = uf;
      best_q = pu;
    }
  };
  // the raster schedule first (at the current lanes, policy and kernel shapes), then
  // the chart/pack kernel shapes, then lanes x policy
  const uint32_t l0 = b->active, p0 = b->policy, u0 = best_u, q0 = best_q;
  const uint32_t mids[] = {FA_RASTER_MID_OFF, 64};
  for (uint32_t mid : mids)
    for (uint32_t fl = 0; fl <= FA_RASTER_HIZ; ++fl) trial(l0, p0, mid, fl, u0, q0);
  const uint32_t rm = best_m, rf = best_f;
  const uint32_t shapes[] = {256, 512, 1024};
  for (uint32_t uf : shapes)
    for (uint32_t pu : shapes)
      if (uf != u0 || pu != q0) trial(l0, p0, rm, rf, uf, pu);
  const uint32_t ru = best_u, rq = best_q;
  for (uint32_t l : cand)
    for (uint32_t pol = FA_BATCH_ROUND_ROBIN; pol <= FA_BATCH_LONGEST_FIRST; ++pol) {
      if (l == 1 && pol == FA_BATCH_LONGEST_FIRST) continue;  // same schedule as round robin
      trial(l, pol, rm, rf, ru, rq);
    }
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->active = best_l;
  b->policy = best_p;
  for (fa_ctx* c : b->ctx) {
    c->mid_max_pix = best_m;
    c->raster_flags = best_f;
    c->uf_threads = best_u;
    c->push_threads = best_q;
  }
  if (best_ms) *best_ms = best;
  return st;
}

fa_status fa_batch_get_kernel_schedule(const fa_batch* b, fa_kernel_schedule* out) {
  if (!b || !out || b->ctx.empty()) return FA_E_INVALID_ARG;
  return fa_get_kernel_schedule(b->ctx[0], out);
}

uint64_t fa_batch_launch_count(const fa_batch* b) {
  if (!b) return 0;
  uint64_t n = 0;
  for (const fa_ctx* c : b->ctx) n += fa_launch_count(c);
  return n;
}

}  // extern "C"
