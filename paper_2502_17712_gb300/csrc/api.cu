// C ABI of libfastatlas: argument checks, context / mesh lifetime and the
// stream-ordered launch sequences.  All compute happens in the kernels of the
// other translation units.
#include <cstdlib>
#include <cstring>

#include "fa_internal.cuh"

using namespace fa;

namespace fa {
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("FA_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}
}  // namespace fa

namespace {

bool is_pow2(uint32_t x) { return x && !(x & (x - 1)); }

Mat4 to_mat(const float* m) {
  Mat4 M;
  std::memcpy(M.m, m, sizeof(M.m));
  return M;
}

template <class T>
fa_status alloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return FA_E_OUT_OF_MEMORY;
  }
  return FA_OK;
}

fa_status check_view(const fa_ctx* ctx, const float* M, uint32_t W, uint32_t H) {
  if (!M || W == 0 || H == 0 || W > ctx->cfg.max_width || H > ctx->cfg.max_height) return FA_E_INVALID_ARG;
  return FA_OK;
}

fa_status check_charts(const fa_charts* ch) {
  if (!ch || !ch->root || !ch->bbox || !ch->fa || !ch->fb || !ch->rot || !ch->count) return FA_E_INVALID_ARG;
  return FA_OK;
}

fa_status check_pack(const fa_ctx* ctx, uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode) {
  if (atlas_log2 < 1 || atlas_log2 > ctx->cfg.max_atlas_log2) return FA_E_INVALID_ARG;
  if (!is_pow2(n_scales) || n_scales > (uint32_t)kMaxScales) return FA_E_INVALID_ARG;
  if (select_mode > FA_SELECT_LARGEST_K) return FA_E_INVALID_ARG;
  return FA_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

uint32_t fa_version(void) { return 10000u; }

const char* fa_status_string(fa_status s) {
  switch (s) {
    case FA_OK: return "FA_OK";
    case FA_E_INVALID_ARG: return "FA_E_INVALID_ARG";
    case FA_E_OUT_OF_MEMORY: return "FA_E_OUT_OF_MEMORY";
    case FA_E_CAPACITY: return "FA_E_CAPACITY";
    case FA_E_PACK_FAILED: return "FA_E_PACK_FAILED";
    case FA_E_TIMEOUT: return "FA_E_TIMEOUT";
    case FA_E_CUDA: return "FA_E_CUDA";
  }
  return "FA_E_UNKNOWN";
}

void fa_destroy(fa_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->prof_on)
    for (int i = 0; i <= kMaxProf; ++i) cudaEventDestroy(ctx->prof_ev[i]);
  const PackScratch& p = ctx->pack;
  void* ptrs[] = {ctx->ctr, ctx->zbuf, ctx->zmax, ctx->queue, ctx->tile_owner, ctx->cand, ctx->surv, ctx->surv_count, ctx->surv_clip, ctx->clip, ctx->clip_count,
                  ctx->label, ctx->wordroots, ctx->blockcnt, ctx->viscnt, ctx->vis, ctx->xedge, ctx->xcnt, ctx->tile_flag, ctx->tile_list,
                  ctx->box_enc, ctx->box_full, p.ord_counts, p.ord_rank, p.ord_total,
                  p.order, p.fs, p.rec8, p.segs, p.scan_state, p.m, p.xy, p.cand, ctx->psched};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  std::free(ctx);
}

fa_status fa_create(fa_ctx** out, const fa_config* cfg) {
  if (!out) return FA_E_INVALID_ARG;
  *out = nullptr;
  if (!cfg) return FA_E_INVALID_ARG;
  const fa_config& c = *cfg;
  if (c.max_tris == 0 || c.max_verts == 0 || c.max_charts == 0 || c.max_width == 0 || c.max_height == 0)
    return FA_E_INVALID_ARG;
  if (c.max_width > 16384 || c.max_height > 16384 || c.max_atlas_log2 < 1 || c.max_atlas_log2 > 14)
    return FA_E_INVALID_ARG;
  if (c.max_charts > (1u << 22) || (uint64_t)c.max_tris + c.max_verts > 0x7FFFFFFFull) return FA_E_INVALID_ARG;
  if (c.min_box < 1 || c.min_box > 4096 || c.gutter > 4096) return FA_E_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return FA_E_CUDA;
  }
  if (c.device < 0 || c.device >= ndev) return FA_E_INVALID_ARG;
  DeviceGuard g(c.device);
  fa_ctx* ctx = (fa_ctx*)std::calloc(1, sizeof(fa_ctx));
  if (!ctx) return FA_E_OUT_OF_MEMORY;
  ctx->cfg = c;
  ctx->device = c.device;
  ctx->loop_cap = kLoopCap;
  ctx->wait_ns = kWaitNs;
  ctx->mid_max_pix = FA_RASTER_MID_OFF;
  ctx->uf_threads = 1024;
  ctx->push_threads = kDefaultPushThreads;
  fa_status st = FA_OK;
  const uint64_t T = c.max_tris, V = c.max_verts, C = c.max_charts;
  ctx->queue_cap = (uint32_t)(T < (1u << 20) ? T + 1024 : (1u << 20));
  PackScratch& pk = ctx->pack;
  pk.max_boxes = (uint32_t)C;
  pk.max_tiles = (uint32_t)((C + kOrderTile - 1) / kOrderTile);
  pk.max_chunks = (uint32_t)((C + kChunk - 1) / kChunk);
  const uint64_t nblocks = (T + 1023) / 1024 + 1;
#define FA_ALLOC(ptr, n) \
  if (st == FA_OK) st = alloc(&ptr, (size_t)(n));
  FA_ALLOC(ctx->ctr, 1);
  FA_ALLOC(ctx->zbuf, (uint64_t)c.max_width * c.max_height);
  FA_ALLOC(ctx->zmax, (uint64_t)((c.max_width + 15) / 16) * ((c.max_height + 15) / 16));
  FA_ALLOC(ctx->queue, ctx->queue_cap);
  ctx->tile_cap = 4u * ctx->queue_cap;
  FA_ALLOC(ctx->tile_owner, ctx->tile_cap);
  // survivor regions (one per raster front block, each rounded up to 512 slots) and
  // then the clipped-path candidate records
  ctx->surv_cap = (uint32_t)(T + (uint64_t)fa::kMaxFrontBlocks * 512ull);
  ctx->cand_cap = ctx->surv_cap + 65536u;
  if (st == FA_OK) st = alloc((unsigned char**)&ctx->cand, (size_t)ctx->cand_cap * 48);
  FA_ALLOC(ctx->surv, ctx->surv_cap);
  FA_ALLOC(ctx->surv_count, fa::kMaxFrontBlocks);
  if (st == FA_OK) st = alloc((float4**)&ctx->surv_clip, (size_t)ctx->surv_cap * 3);
  FA_ALLOC(ctx->clip, ctx->surv_cap);
  FA_ALLOC(ctx->clip_count, fa::kMaxFrontBlocks);
  FA_ALLOC(ctx->label, T + V);
  FA_ALLOC(ctx->wordroots, (T + 31) / 32);
  FA_ALLOC(ctx->blockcnt, nblocks + 1);
  FA_ALLOC(ctx->viscnt, nblocks + 1);
  FA_ALLOC(ctx->xedge, nblocks * 3072);
  FA_ALLOC(ctx->xcnt, nblocks);
  FA_ALLOC(ctx->tile_flag, nblocks);
  FA_ALLOC(ctx->tile_list, nblocks);
  FA_ALLOC(ctx->vis, T);
  FA_ALLOC(ctx->box_enc, 4 * C);
  FA_ALLOC(ctx->box_full, C);
  FA_ALLOC(pk.ord_counts, (uint64_t)kMaxH * pk.max_tiles);
  FA_ALLOC(pk.ord_rank, C);
  FA_ALLOC(pk.ord_total, kMaxH);
  FA_ALLOC(pk.order, C);
  FA_ALLOC(pk.fs, (uint64_t)pk.max_chunks * kChunk);
  FA_ALLOC(pk.rec8, (uint64_t)kMaxScales * pk.max_chunks * kChunk);
  FA_ALLOC(pk.segs, (uint64_t)kMaxScales * pk.max_chunks * kSegStride);
  FA_ALLOC(pk.scan_state, (uint64_t)kMaxScales * pk.max_chunks);
  FA_ALLOC(pk.m, kMaxScales);
  FA_ALLOC(pk.xy, (uint64_t)kMaxScales * C);
  FA_ALLOC(pk.cand, kMaxScales);
  FA_ALLOC(ctx->psched, kPschedWords);
#undef FA_ALLOC
  pk.ctr = ctx->ctr;
  pk.count = nullptr;
  if (st == FA_OK && cudaMemset(ctx->ctr, 0, sizeof(DevCounters)) != cudaSuccess) st = FA_E_CUDA;
  if (st == FA_OK && cudaMemset(pk.ord_total, 0, kMaxH * sizeof(uint32_t)) != cudaSuccess) st = FA_E_CUDA;
  if (st == FA_OK && cudaMemset(ctx->psched, 0, kPschedWords * sizeof(uint32_t)) != cudaSuccess) st = FA_E_CUDA;
  if (st == FA_OK && cudaDeviceSynchronize() != cudaSuccess) st = FA_E_CUDA;
  if (st != FA_OK) {
    fa_destroy(ctx);
    return st;
  }
  *out = ctx;
  return FA_OK;
}

fa_status fa_mesh_register(fa_ctx* ctx, const float* d_pos, uint32_t V, const uint32_t* d_idx, uint32_t T,
                           fa_mesh** out, fa_stream_t stream) {
  if (!out) return FA_E_INVALID_ARG;
  *out = nullptr;
  if (!ctx || !d_pos || !d_idx || V == 0 || T == 0) return FA_E_INVALID_ARG;
  if (T > ctx->cfg.max_tris || V > ctx->cfg.max_verts) return FA_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  fa_mesh* m = (fa_mesh*)std::calloc(1, sizeof(fa_mesh));
  if (!m) return FA_E_OUT_OF_MEMORY;
  m->ctx = ctx;
  m->pos = d_pos;
  m->idx = d_idx;
  m->V = V;
  m->T = T;
  fa_status st = build_adjacency(ctx, m, (cudaStream_t)stream);
  if (st != FA_OK) {
    std::free(m);
    return st;
  }
  *out = m;
  return FA_OK;
}

void fa_mesh_release(fa_mesh* m) {
  if (!m) return;
  DeviceGuard g(m->ctx->device);
  cudaDeviceSynchronize();
  if (m->adj) cudaFree(m->adj);
  if (m->nm_off) cudaFree(m->nm_off);
  if (m->nm_list) cudaFree(m->nm_list);
  std::free(m);
}

fa_status fa_visibility(fa_ctx* ctx, const fa_mesh* mesh, const float view_proj[16], uint32_t width,
                        uint32_t height, uint32_t flags, uint32_t* d_vt, fa_stream_t stream) {
  if (!ctx || !mesh || !d_vt || mesh->ctx != ctx) return FA_E_INVALID_ARG;
  if (flags & ~FA_VIS_CONSERVATIVE) return FA_E_INVALID_ARG;
  fa_status st = check_view(ctx, view_proj, width, height);
  if (st != FA_OK) return st;
  DeviceGuard g(ctx->device);
  trace_begin(ctx);
  st = launch_visibility(ctx, mesh, to_mat(view_proj), width, height, d_vt, false, (cudaStream_t)stream, nullptr,
                         (flags & FA_VIS_CONSERVATIVE) != 0);
  trace_end(ctx, (cudaStream_t)stream);
  return st;
}

fa_status fa_chartify(fa_ctx* ctx, const fa_mesh* mesh, const uint32_t* d_vt, uint32_t mode,
                      int32_t* d_tri_chart, int32_t* d_vert_chart, const fa_charts* charts,
                      fa_stream_t stream) {
  if (!ctx || !mesh || !d_vt || !d_tri_chart || mesh->ctx != ctx) return FA_E_INVALID_ARG;
  if (mode > FA_CHARTS_VERTEX) return FA_E_INVALID_ARG;
  if (!charts || !charts->root || !charts->count) return FA_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  trace_begin(ctx);
  fa_status st = launch_chartify(ctx, mesh, d_vt, mode, d_tri_chart, d_vert_chart, charts, (cudaStream_t)stream);
  trace_end(ctx, (cudaStream_t)stream);
  return st;
}

// The box and UV kernels walk the context's visible-triangle list; the standalone
// calls build it from tri_chart so that they need no extra argument.
fa_status fa_parameterize(fa_ctx* ctx, const fa_mesh* mesh, const float view_proj[16], uint32_t width,
                          uint32_t height, float ratio, const int32_t* d_tri_chart, const fa_charts* charts,
                          uint32_t flags, uint32_t* d_partial, fa_stream_t stream) {
  if (!ctx || !mesh || !d_tri_chart || mesh->ctx != ctx) return FA_E_INVALID_ARG;
  if (flags & ~FA_BOX_FRUSTUM_CLIP) return FA_E_INVALID_ARG;
  fa_status st = check_view(ctx, view_proj, width, height);
  if (st == FA_OK) st = check_charts(charts);
  if (st != FA_OK) return st;
  if (!(ratio > 0.0f && ratio <= 64.0f)) return FA_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  trace_begin(ctx);
  st = launch_vis_list(ctx, mesh, d_tri_chart, s);
  if (st == FA_OK)
    st = launch_parameterize(ctx, mesh, to_mat(view_proj), width, height, ratio, d_tri_chart, charts, true, flags,
                             d_partial, s);
  trace_end(ctx, s);
  return st;
}

fa_status fa_pack(fa_ctx* ctx, const uint32_t* d_fa, const uint32_t* d_fb, const uint32_t* d_count,
                  uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode, uint32_t* d_order,
                  fa_placement* d_place, fa_pack_result* d_res, uint32_t lowres_log2, fa_stream_t stream) {
  if (!ctx || !d_fa || !d_fb || !d_count || !d_place || !d_res || lowres_log2 > 7) return FA_E_INVALID_ARG;
  fa_status st = check_pack(ctx, atlas_log2, n_scales, select_mode);
  if (st != FA_OK) return st;
  DeviceGuard g(ctx->device);
  trace_begin(ctx);
  st = launch_pack(ctx, d_fa, d_fb, d_count, atlas_log2, n_scales, select_mode, d_order, d_place, d_res,
                   (cudaStream_t)stream, lowres_log2);
  trace_end(ctx, (cudaStream_t)stream);
  return st;
}

fa_status fa_uv(fa_ctx* ctx, const fa_mesh* mesh, const float view_proj[16], uint32_t width, uint32_t height,
                float ratio, const int32_t* d_tri_chart, const fa_charts* charts, const fa_placement* d_place,
                const fa_pack_result* d_res, uint32_t atlas_log2, uint32_t n_scales, float* d_uv,
                float* d_affine, fa_stream_t stream) {
  if (!ctx || !mesh || !d_tri_chart || !d_place || !d_res || mesh->ctx != ctx) return FA_E_INVALID_ARG;
  if (!d_uv && !d_affine) return FA_E_INVALID_ARG;
  fa_status st = check_view(ctx, view_proj, width, height);
  if (st == FA_OK) st = check_charts(charts);
  if (st == FA_OK) st = check_pack(ctx, atlas_log2, n_scales, 0);
  if (st != FA_OK) return st;
  if (!(ratio > 0.0f && ratio <= 64.0f)) return FA_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  trace_begin(ctx);
  st = launch_vis_list(ctx, mesh, d_tri_chart, s);
  if (st == FA_OK)
    st = launch_uv(ctx, mesh, to_mat(view_proj), width, height, ratio, d_tri_chart, charts, d_place, d_res,
                   atlas_log2, n_scales, d_uv, d_affine, s);
  trace_end(ctx, s);
  return st;
}



}  // extern "C"

namespace fa {

// Host-side checks of one frame on ctx (the mesh may belong to another context of
// the same device when its sizes fit this one's maxima).
fa_status check_frame(const fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p, const float* d_view_proj,
                      const fa_frame_out* o) {
  if (!ctx || !mesh || !p || !o || !mesh->ctx || mesh->ctx->device != ctx->device) return FA_E_INVALID_ARG;
  if (mesh->T > ctx->cfg.max_tris || mesh->V > ctx->cfg.max_verts) return FA_E_INVALID_ARG;
  if (!o->vt || !o->tri_chart || !o->place || !o->result) return FA_E_INVALID_ARG;
  fa_status st = check_view(ctx, d_view_proj ? d_view_proj : p->view_proj, p->width, p->height);
  if (st == FA_OK) st = check_charts(&o->charts);
  if (st == FA_OK) st = check_pack(ctx, p->atlas_log2, p->n_scales, p->select_mode);
  if (st != FA_OK) return st;
  if (p->chart_mode > FA_CHARTS_VERTEX || !(p->ratio > 0.0f && p->ratio <= 64.0f)) return FA_E_INVALID_ARG;
  if (p->flags & ~(FA_BOX_FRUSTUM_CLIP | FA_VIS_CONSERVATIVE | FA_LOWRES(7) | FA_FRAME_PERSISTENT))
    return FA_E_INVALID_ARG;
  if (d_view_proj && (reinterpret_cast<uintptr_t>(d_view_proj) & 15u)) return FA_E_INVALID_ARG;
  return FA_OK;
}

// The launch sequence of one checked frame (the device must be current); the
// matrix is p->view_proj, or read on the device from d_view_proj.
fa_status enqueue_frame(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p, const float* d_view_proj,
                        const fa_frame_out* o, cudaStream_t s) {
  if (p->flags & FA_FRAME_PERSISTENT) return enqueue_frame_persistent(ctx, mesh, p, d_view_proj, o, s);
  fa_status st;
  const Mat4 M = d_view_proj ? Mat4{} : to_mat(p->view_proj);
  const float* Md = d_view_proj;
  trace_begin(ctx);
  // the raster front end (first kernel) clears the status word; it also sets
  // tri_chart to -1 (16-byte stores) when it is 16-byte aligned, and the chart-id
  // pass then writes only the listed tiles
  const bool tri_init = (reinterpret_cast<uintptr_t>(o->tri_chart) & 15u) == 0;
  if ((st = launch_visibility(ctx, mesh, M, p->width, p->height, o->vt, true, s, Md,
                              (p->flags & FA_VIS_CONSERVATIVE) != 0, tri_init ? o->tri_chart : nullptr)) != FA_OK)
    return st;
  if ((st = launch_chartify(ctx, mesh, o->vt, p->chart_mode, o->tri_chart, o->vert_chart, &o->charts, s,
                            true, tri_init)) != FA_OK)
    return st;
  // the chart-id pass already reset the chart-box accumulators; the footprints
  // are computed by the first order kernel
  if ((st = launch_parameterize(ctx, mesh, M, p->width, p->height, p->ratio, o->tri_chart, &o->charts,
                                false, p->flags, o->partial, s, Md, false)) != FA_OK)
    return st;
  const FootArgs foot = foot_args(ctx, p->width, p->height, p->ratio, &o->charts);
  // with UVs, the UV kernel also writes the placements
  const bool uv = o->uv || o->affine;
  if ((st = launch_pack(ctx, o->charts.fa, o->charts.fb, o->charts.count, p->atlas_log2, p->n_scales,
                        p->select_mode, o->order, o->place, o->result, s, (p->flags >> 8) & 7u, &foot,
                        !uv)) != FA_OK)
    return st;
  if (uv) {
    if ((st = launch_uv(ctx, mesh, M, p->width, p->height, p->ratio, o->tri_chart, &o->charts, o->place,
                        o->result, p->atlas_log2, p->n_scales, o->uv, o->affine, s, Md, true)) != FA_OK)
      return st;
  }
  trace_end(ctx, s);
  return FA_OK;
}

}  // namespace fa

namespace {

fa_status atlas_frame(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p, const float* d_view_proj,
                      const fa_frame_out* o, fa_stream_t stream) {
  if (!mesh || mesh->ctx != ctx) return FA_E_INVALID_ARG;
  fa_status st = check_frame(ctx, mesh, p, d_view_proj, o);
  if (st != FA_OK) return st;
  DeviceGuard g(ctx->device);
  return enqueue_frame(ctx, mesh, p, d_view_proj, o, (cudaStream_t)stream);
}

}  // namespace

extern "C" {

fa_status fa_atlas_frame(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p, const fa_frame_out* o,
                         fa_stream_t stream) {
  return atlas_frame(ctx, mesh, p, nullptr, o, stream);
}

fa_status fa_atlas_frame_dev_matrix(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p,
                                    const float* d_view_proj, const fa_frame_out* o, fa_stream_t stream) {
  if (!d_view_proj) return FA_E_INVALID_ARG;
  return atlas_frame(ctx, mesh, p, d_view_proj, o, stream);
}

fa_status fa_last_device_status(fa_ctx* ctx, fa_stream_t stream, int32_t* out) {
  if (!ctx || !out) return FA_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  int32_t v = 0;
  if (cudaMemcpyAsync(&v, &ctx->ctr->status, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return FA_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FA_E_CUDA;
  if (v != 0) {
    if (cudaMemsetAsync(&ctx->ctr->status, 0, sizeof(int32_t), s) != cudaSuccess) return FA_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FA_E_CUDA;
  }
  *out = v;
  return FA_OK;
}

uint64_t fa_launch_count(const fa_ctx* ctx) { return ctx ? ctx->launches : 0; }

static bool schedule_threads_ok(uint32_t n) { return n == 256 || n == 512 || n == 1024; }

fa_status fa_set_chart_pack_schedule(fa_ctx* ctx, uint32_t uf_threads, uint32_t push_threads) {
  if (!ctx || !schedule_threads_ok(uf_threads) || !schedule_threads_ok(push_threads)) return FA_E_INVALID_ARG;
  ctx->uf_threads = uf_threads;
  ctx->push_threads = push_threads;
  return FA_OK;
}

fa_status fa_get_kernel_schedule(const fa_ctx* ctx, fa_kernel_schedule* out) {
  if (!ctx || !out) return FA_E_INVALID_ARG;
  *out = fa_kernel_schedule{ctx->mid_max_pix, ctx->raster_flags, ctx->uf_threads, ctx->push_threads};
  return FA_OK;
}

fa_status fa_set_raster_schedule(fa_ctx* ctx, uint32_t mid_max_pix, uint32_t flags) {
  if (!ctx || mid_max_pix < FA_RASTER_MID_OFF || mid_max_pix > FA_RASTER_MID_MAX || (flags & ~FA_RASTER_HIZ))
    return FA_E_INVALID_ARG;
  ctx->mid_max_pix = mid_max_pix;
  ctx->raster_flags = flags;
  return FA_OK;
}

fa_status fa_set_wait_limits(fa_ctx* ctx, uint32_t loop_cap, uint64_t wait_ns) {
  if (!ctx) return FA_E_INVALID_ARG;
  ctx->loop_cap = loop_cap;
  ctx->wait_ns = (unsigned long long)wait_ns;
  return FA_OK;
}

fa_status fa_frame_stats_read(fa_ctx* ctx, fa_stream_t stream, fa_frame_stats* out) {
  if (!ctx || !out) return FA_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  const cudaStream_t s = (cudaStream_t)stream;
  fa::DevCounters c{};
  uint32_t per[fa::kMaxFrontBlocks] = {}, perc[fa::kMaxFrontBlocks] = {};
  const uint32_t nb = ctx->front_blocks < fa::kMaxFrontBlocks ? ctx->front_blocks : fa::kMaxFrontBlocks;
  FA_CUDA_TRY(cudaMemcpyAsync(&c, ctx->ctr, sizeof(c), cudaMemcpyDeviceToHost, s));
  if (nb) {
    FA_CUDA_TRY(cudaMemcpyAsync(per, ctx->surv_count, nb * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    FA_CUDA_TRY(cudaMemcpyAsync(perc, ctx->clip_count, nb * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  }
  FA_CUDA_TRY(cudaStreamSynchronize(s));
  fa_frame_stats r{};
  for (uint32_t i = 0; i < nb; ++i) {
    r.survivors += per[i];
    r.clipped += perc[i];
  }
  r.clip_records = c.ncand;
  r.big_entries = (uint32_t)(c.big >> 40);
  r.big_tiles = c.big & ((1ull << 40) - 1);
  r.visible = c.n_vis;
  r.charts = c.chart_count;
  r.visible_tiles = c.n_vtiles;
  *out = r;
  return FA_OK;
}

fa_status fa_profile_enable(fa_ctx* ctx, int enable) {
  if (!ctx) return FA_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (enable && !ctx->prof_on) {
    for (int i = 0; i <= kMaxProf; ++i) {
      if (cudaEventCreate(&ctx->prof_ev[i]) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->prof_ev[j]);
        return FA_E_CUDA;
      }
    }
    ctx->prof_on = 1;
    ctx->prof_n = 0;
  } else if (!enable && ctx->prof_on) {
    cudaDeviceSynchronize();
    for (int i = 0; i <= kMaxProf; ++i) cudaEventDestroy(ctx->prof_ev[i]);
    ctx->prof_on = 0;
    ctx->prof_n = 0;
  }
  return FA_OK;
}

fa_status fa_profile_read(fa_ctx* ctx, int max_n, float* ms, const char** names, int* n_out) {
  if (!ctx || !n_out || max_n < 0 || (max_n > 0 && (!ms || !names))) return FA_E_INVALID_ARG;
  *n_out = 0;
  if (!ctx->prof_on || ctx->prof_n == 0) return FA_OK;
  DeviceGuard g(ctx->device);
  if (cudaEventSynchronize(ctx->prof_ev[ctx->prof_n]) != cudaSuccess) return FA_E_CUDA;
  const int n = ctx->prof_n < max_n ? ctx->prof_n : max_n;
  for (int i = 0; i < n; ++i) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, ctx->prof_ev[i], ctx->prof_ev[i + 1]) != cudaSuccess) return FA_E_CUDA;
    ms[i] = t;
    names[i] = ctx->prof_name[i];
  }
  *n_out = ctx->prof_n;
  return FA_OK;
}

}  // extern "C"
