// The persistent frame kernel: every stage of the per-frame path (visibility,
// charts, boxes, order, packing, UVs; Sec. 3-5, App. A) for one view or many
// independent views (one atlas each, Sec. 3) in ONE cooperative launch.
//
// The launch is a grid of 1024-thread CTAs, one per SM, that drain a device work
// queue.  A work item is (view, stage, worker j of n): it runs the stage's body with
// the virtual block index j of a virtual grid of n blocks, the same bodies the
// 15-kernel launch sequence runs (raster.cuh, chartify.cuh, param.cuh, pack.cuh), so
// results are identical.  Items are claimed in a fixed order from one counter; an
// item first waits until every worker of the group it depends on (the previous stage
// of its view, or the last stage of the view before it on the same context) has
// finished.  Every dependency lies earlier in the claim order and all CTAs are
// resident (cooperative launch), so the claimed items always make progress.  The
// waits are bounded in time: one that runs out sets an abort flag, every later item
// skips its body, and every view of the launch reports FA_E_TIMEOUT.  The last CTA
// to leave resets the queue for the next launch.
//
// Why: a frame is a chain of dependent stages, most of them latency bound.  As
// separate launches each stage costs a launch and a drain (about 5.5 us on a small
// frame); here a stage boundary is one counter, and with many views in flight the
// idle SMs of one view's latency-bound stages run other views' stages.
#include <algorithm>
#include <cstring>
#include <new>

#include "chartify.cuh"
#include "pack.cuh"
#include "param.cuh"
#include "raster.cuh"

namespace fa {
namespace {

constexpr int kPT = 1024;           // threads per CTA
constexpr int kMaxStages = 24;      // stages of one view (at most 20 are used)
constexpr int kInlineGroups = 24;   // stage groups of a single-view launch (kernel parameter)

enum Stage : uint8_t {
  S_FRONT, S_EXACT, S_DEPTH_BIG, S_ZMAX, S_MARK, S_INIT_V, S_LOCAL, S_HOOK, S_HOOK_V, S_HOOK_NM, S_FLATTEN, S_SCAN,
  S_TRI_CHART, S_VERT_CHART, S_BBOX, S_ORDER_TILE, S_ORDER_SCATTER, S_PACK_SCAN, S_PUSH, S_PLACE, S_UV
};

// Everything the stages of one view read: the per-stage arguments of the launch
// sequence, built by the same host helpers.
struct ViewArgs {
  rs::RasterArgs ra;
  cf::UfArgs uf;
  pm::BoxArgs box;
  pm::UvArgs uv;
  PackScratch ps;
  pk::PackArgs pa;
  FootArgs foot;
  uint32_t* blockcnt;
  uint32_t* viscnt;
  uint2* wordroots;
  int32_t* tri_chart;
  int32_t* vert_chart;
  uint32_t* roots;
  uint32_t* box_enc;
  uint32_t* box_full;
  uint2* vis;
  uint32_t* count_out;
  const uint32_t* nm_off;
  const uint32_t* nm_list;
  const uint32_t* fa;
  const uint32_t* fb;
  uint32_t* order;
  uint32_t max_charts, nb, n_nm, n_scales;
  uint32_t vm, devm, cons, list_tri_chart;
};

// One stage of one view: its items are [start, start + workers) of the claim order.
struct Group {
  uint32_t start;
  uint32_t workers;
  int32_t dep;  // group that must have finished first, or -1
  uint16_t view;
  uint8_t stage;
  uint8_t pad;
};

struct PersistParams {
  const ViewArgs* views;  // device array, or null: the inline view
  const Group* groups;    // device array, or null: the inline groups
  uint32_t n_views, n_groups, n_items;
  uint32_t* sched;        // [4 + n_groups]: next item, exits, abort, -, done per group
  unsigned long long wait_ns;
  Group inline_groups[kInlineGroups];
  ViewArgs inline_view;
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits until *cnt >= target; false when the launch was aborted or the wait ran out
// (which aborts it).
__device__ bool wait_count(const uint32_t* cnt, uint32_t target, uint32_t* abort, unsigned long long limit_ns) {
  if (ld_acquire(cnt) >= target) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (ld_acquire(cnt) >= target) return true;
    if (ld_acquire(abort)) return false;
    if (gtimer() - t0 > limit_ns) {
      atomicExch(abort, 1u);
      return false;
    }
    __nanosleep(64);
  }
}

// One function per stage variant, not inlined: each keeps its own register
// allocation inside the kernel's budget.
template <bool DEV_M>
__device__ __noinline__ void st_front(const ViewArgs& v, uint32_t j, uint32_t n) {
  rs::front_body<DEV_M>(v.ra, j, n);
}
template <bool DEV_M>
__device__ __noinline__ void st_exact(const ViewArgs& v, uint32_t j, uint32_t n) {
  rs::exact_body<DEV_M, kPT>(v.ra, j, n);
}
__device__ __noinline__ void st_depth_big(const ViewArgs& v, uint32_t j, uint32_t n) { rs::depth_big_body(v.ra, j, n); }
__device__ __noinline__ void st_zmax(const ViewArgs& v, uint32_t j, uint32_t n) { rs::zmax_body(v.ra, j, n); }
template <bool CONS>
__device__ __noinline__ void st_mark(const ViewArgs& v, uint32_t j, uint32_t n) {
  rs::mark_body<CONS, kPT>(v.ra, j, n);
}
__device__ __noinline__ void st_init_v(const ViewArgs& v, uint32_t j, uint32_t n) {
  cf::init_v_body(v.uf.label, v.uf.T, v.uf.V, j, n);
}
__device__ __noinline__ void st_local(const ViewArgs& v, uint32_t j, uint32_t n) { cf::local_body<true, kPT>(v.uf, j, n); }
__device__ __noinline__ void st_hook(const ViewArgs& v, uint32_t j, uint32_t n) {
  cf::hook_body<true, 128>(v.uf, j, n);  // eight tiles at a time per CTA
}
__device__ __noinline__ void st_hook_v(const ViewArgs& v, uint32_t j, uint32_t n) { cf::hook_v_body(v.uf, j, n); }
__device__ __noinline__ void st_hook_nm(const ViewArgs& v, uint32_t j, uint32_t n) {
  cf::hook_nm_body(v.uf, v.nm_off, v.nm_list, v.n_nm, j, n);
}
__device__ __noinline__ void st_flatten(const ViewArgs& v, uint32_t j, uint32_t n) {
  cf::flatten_body<true, kPT>(v.uf, v.blockcnt, v.viscnt, v.wordroots, j, n);
}
__device__ __noinline__ void st_scan(const ViewArgs& v) {
  cf::scan_blocks_body(v.blockcnt, v.viscnt, v.nb, v.count_out, v.max_charts, v.ra.ctr);
}
__device__ __noinline__ void st_tri_chart(const ViewArgs& v, uint32_t j, uint32_t n) {
  if (v.list_tri_chart)
    cf::tri_chart_body<true, kPT>(v.uf, v.blockcnt, v.wordroots, v.tri_chart, v.roots, v.box_enc, v.box_full,
                                  v.max_charts, v.viscnt, v.vis, j, n);
  else
    cf::tri_chart_body<false, kPT>(v.uf, v.blockcnt, v.wordroots, v.tri_chart, v.roots, v.box_enc, v.box_full,
                                   v.max_charts, v.viscnt, v.vis, j, n);
}
__device__ __noinline__ void st_vert_chart(const ViewArgs& v, uint32_t j, uint32_t n) {
  cf::vert_chart_body(v.uf, v.blockcnt, v.wordroots, v.vert_chart, (int)v.vm, j, n);
}
template <bool DEV_M>
__device__ __noinline__ void st_bbox(const ViewArgs& v, uint32_t j, uint32_t n) {
  pm::bbox_body<DEV_M>(v.box, j, n);
}
__device__ __noinline__ void st_order_tile(const ViewArgs& v, uint32_t j, unsigned char* smem) {
  pk::order_tile_body<true>(v.ps, v.fb, v.foot, j, reinterpret_cast<uint32_t*>(smem));
}
__device__ __noinline__ void st_order_scatter(const ViewArgs& v, uint32_t j, unsigned char* smem) {
  pk::order_scatter_body(v.ps, v.fa, v.fb, v.order, j, reinterpret_cast<uint32_t*>(smem));
}
__device__ __noinline__ void st_pack_scan(const ViewArgs& v, uint32_t j, uint32_t n) {
  pk::pack_scan_body<kPT, false>(v.ps, v.pa, v.n_scales, j, n);  // one candidate per item
}
__device__ __noinline__ void st_push(const ViewArgs& v, uint32_t j, uint32_t n, unsigned char* smem) {
  pk::push_body<kPT>(v.ps, v.pa, j, n, smem);
}
__device__ __noinline__ void st_place(const ViewArgs& v, uint32_t j, uint32_t n) { pk::pack_place_body(v.ps, v.pa, j, n); }
template <bool DEV_M>
__device__ __noinline__ void st_uv(const ViewArgs& v, uint32_t j, uint32_t n) {
  pm::uv_body<DEV_M>(v.uv, j, n);
}

// Single-view launches: the bodies inlined on the kernel parameter itself, so that
// the arguments are constant-bank operands as in the separate kernels (through a
// pointer they would take registers, and the raster stages would spill).
__device__ void run_stage(const ViewArgs& v, uint32_t stage, uint32_t j, uint32_t n, unsigned char* smem);

__device__ __forceinline__ void run_stage_inline(const ViewArgs& v, uint32_t stage, uint32_t j, uint32_t n,
                                                 unsigned char* smem) {
  // (the device-matrix and conservative variants, and the other stages, keep their
  // own register allocation in the non-inlined wrappers)
  if (stage == S_FRONT && !v.devm) rs::front_body<false>(v.ra, j, n);
  else if (stage == S_EXACT && !v.devm) rs::exact_body<false, kPT>(v.ra, j, n);
  else if (stage == S_MARK && !v.cons) rs::mark_body<false, kPT>(v.ra, j, n);
  else run_stage(v, stage, j, n, smem);
}

__device__ void run_stage(const ViewArgs& v, uint32_t stage, uint32_t j, uint32_t n, unsigned char* smem) {
  switch (stage) {
    case S_FRONT: v.devm ? st_front<true>(v, j, n) : st_front<false>(v, j, n); break;
    case S_EXACT: v.devm ? st_exact<true>(v, j, n) : st_exact<false>(v, j, n); break;
    case S_DEPTH_BIG: st_depth_big(v, j, n); break;
    case S_ZMAX: st_zmax(v, j, n); break;
    case S_MARK: v.cons ? st_mark<true>(v, j, n) : st_mark<false>(v, j, n); break;
    case S_INIT_V: st_init_v(v, j, n); break;
    case S_LOCAL: st_local(v, j, n); break;
    case S_HOOK: st_hook(v, j, n); break;
    case S_HOOK_V: st_hook_v(v, j, n); break;
    case S_HOOK_NM: st_hook_nm(v, j, n); break;
    case S_FLATTEN: st_flatten(v, j, n); break;
    case S_SCAN: st_scan(v); break;
    case S_TRI_CHART: st_tri_chart(v, j, n); break;
    case S_VERT_CHART: st_vert_chart(v, j, n); break;
    case S_BBOX: v.devm ? st_bbox<true>(v, j, n) : st_bbox<false>(v, j, n); break;
    case S_ORDER_TILE: st_order_tile(v, j, smem); break;
    case S_ORDER_SCATTER: st_order_scatter(v, j, smem); break;
    case S_PACK_SCAN: st_pack_scan(v, j, n); break;
    case S_PUSH: st_push(v, j, n, smem); break;
    case S_PLACE: st_place(v, j, n); break;
    case S_UV: v.devm ? st_uv<true>(v, j, n) : st_uv<false>(v, j, n); break;
    default: break;
  }
}

// SINGLE: one view, its arguments in the kernel parameter (P.views is null);
// otherwise the views' arguments are in device memory.
template <bool SINGLE>
__global__ void __launch_bounds__(kPT, 1) k_persist(const __grid_constant__ PersistParams P) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  // the loop keeps nothing in registers across a stage body (every value is re-read
  // from shared memory or the parameter), so that a body has the whole budget
  __shared__ uint32_t s_item, s_g, s_skip;
  for (;;) {
    if (threadIdx.x == 0) {
      const Group* groups = SINGLE ? P.inline_groups : P.groups;
      uint32_t* abort = P.sched + 2;
      const uint32_t item = atomicAdd(P.sched, 1u);
      uint32_t g = 0, skip = 1;
      if (item < P.n_items) {
        uint32_t lo = 0, hi = P.n_groups;  // the last group starting at or before item
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (groups[mid].start <= item) lo = mid;
          else hi = mid;
        }
        g = lo;
        const int32_t dep = groups[g].dep;
        skip = ld_acquire(abort) ? 1u : 0u;
        if (!skip && dep >= 0)
          skip = wait_count(P.sched + 4 + dep, groups[dep].workers, abort, P.wait_ns) ? 0u : 1u;
        __threadfence();
      }
      s_item = item;
      s_g = g;
      s_skip = skip;
    }
    __syncthreads();
    if (s_item >= P.n_items) break;
    if (!s_skip) {
      const Group* groups = SINGLE ? P.inline_groups : P.groups;
      const uint32_t g = s_g;
      const uint32_t stage = groups[g].stage, j = s_item - groups[g].start, n = groups[g].workers;
      if (SINGLE) run_stage_inline(P.inline_view, stage, j, n, smem_dyn);
      else run_stage(P.views[groups[g].view], stage, j, n, smem_dyn);
    }
    __syncthreads();  // the item's writes precede its completion count
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(P.sched + 4 + s_g, 1u);
    }
  }
  // the last CTA to leave reports an abort to every view and resets the schedule
  if (threadIdx.x == 0) {
    uint32_t* exited = P.sched + 1;
    uint32_t* abort = P.sched + 2;
    __threadfence();
    if (atomicAdd(exited, 1u) == gridDim.x - 1u) {
      __threadfence();
      if (ld_acquire(abort)) {
        for (uint32_t vi = 0; vi < P.n_views; ++vi) {
          const ViewArgs* v = SINGLE ? &P.inline_view : P.views + vi;
          set_status(v->ra.ctr, FA_E_TIMEOUT);
          v->pa.res->status = FA_E_TIMEOUT;
        }
      }
      for (uint32_t g = 0; g < P.n_groups; ++g) P.sched[4 + g] = 0u;
      P.sched[0] = 0u;
      *abort = 0u;
      __threadfence();
      *exited = 0u;
    }
  }
}

Mat4 to_mat4(const float* m) {
  Mat4 M;
  std::memcpy(M.m, m, sizeof(M.m));
  return M;
}

uint32_t clampu(uint64_t x, uint32_t lo, uint32_t hi) {
  return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(x, lo), hi);
}

// One view of a launch on context ctx: its arguments and its stages with their
// worker counts (G resident CTAs; scale_pct scales the data-sized counts).
struct ViewPlan {
  ViewArgs va;
  uint32_t n_stages;
  uint8_t stage[kMaxStages];
  uint32_t workers[kMaxStages];
  uint32_t front_cap;
};

void build_view(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p, const float* d_view_proj,
                const fa_frame_out* o, uint32_t G, uint32_t scale_pct, ViewPlan* vp) {
  ViewArgs& v = vp->va;
  std::memset(&v, 0, sizeof(v));
  const Mat4 M = d_view_proj ? Mat4{} : to_mat4(p->view_proj);
  const uint32_t W = p->width, H = p->height, T = mesh->T;
  const bool tri_init = (reinterpret_cast<uintptr_t>(o->tri_chart) & 15u) == 0;
  const bool vm = p->chart_mode == FA_CHARTS_VERTEX;
  const bool uv = o->uv || o->affine;
  // worker counts: at most G, else one worker per kUnit units of what the stage walks
  // (a few warps of work per SM, so that small frames spread over every SM)
  auto wk = [&](uint64_t units, uint64_t per) {
    const uint64_t p = std::max<uint64_t>(1, per * 100u / std::max<uint32_t>(scale_pct, 1u));
    return clampu((units + p - 1) / p, 1, G);
  };
  const uint64_t chart_cap = std::min<uint64_t>(ctx->cfg.max_charts, T);
  const uint32_t ntiles = (T + 1023) / 1024;
  const uint64_t pix = (uint64_t)W * H;
  const uint32_t n_front = std::min<uint32_t>(wk(T, 128), kMaxFrontBlocks);
  const uint32_t n_tri = wk(T, 128);
  const uint32_t n_pix = wk(pix, 2048);
  const uint32_t n_tiles = clampu(ntiles, 1, G);
  const uint32_t order_tiles = (uint32_t)std::max<uint64_t>(1, (chart_cap + kOrderTile - 1) / kOrderTile);
  const uint32_t chunks = (uint32_t)std::max<uint64_t>(1, (chart_cap + kChunk - 1) / kChunk);
  v.ra = rs::make_raster_args(ctx, mesh, M, W, H, o->vt, true, d_view_proj, (p->flags & FA_VIS_CONSERVATIVE) != 0,
                              tri_init ? o->tri_chart : nullptr, n_front, kPT);
  v.ra.partial_clear = o->partial;
  v.uf = cf::make_uf_args(ctx, mesh, o->vt);
  v.box = pm::make_box_args(ctx, mesh, M, o->tri_chart, p->flags, o->partial, d_view_proj);
  v.foot = foot_args(ctx, W, H, p->ratio, &o->charts);
  v.ps = ctx->pack;
  v.ps.count = o->charts.count;
  v.order = o->order ? o->order : v.ps.order;
  v.pa = pk::make_pack_args(ctx, v.order, p->atlas_log2, p->n_scales, p->select_mode, ctx->cfg.min_box,
                            ctx->cfg.gutter, (p->flags >> 8) & 7u, o->place, o->result);
  v.uv = pm::make_uv_args(ctx, mesh, M, W, H, p->ratio, o->tri_chart, &o->charts, o->place, o->result, p->atlas_log2,
                          p->n_scales, o->uv, o->affine, d_view_proj, true);
  v.blockcnt = ctx->blockcnt;
  v.viscnt = ctx->viscnt;
  v.wordroots = ctx->wordroots;
  v.tri_chart = o->tri_chart;
  v.vert_chart = o->vert_chart;
  v.roots = o->charts.root;
  v.box_enc = ctx->box_enc;
  v.box_full = ctx->box_full;
  v.vis = ctx->vis;
  v.count_out = o->charts.count;
  v.nm_off = mesh->nm_off;
  v.nm_list = mesh->nm_list;
  v.fa = o->charts.fa;
  v.fb = o->charts.fb;
  v.max_charts = ctx->cfg.max_charts;
  v.nb = std::max<uint32_t>(ntiles, 1);
  v.n_nm = mesh->n_nm;
  v.n_scales = p->n_scales;
  v.vm = vm ? 1u : 0u;
  v.devm = d_view_proj ? 1u : 0u;
  v.cons = (p->flags & FA_VIS_CONSERVATIVE) ? 1u : 0u;
  v.list_tri_chart = tri_init ? 1u : 0u;
  vp->front_cap = v.pa.front_cap;

  uint32_t n = 0;
  auto add = [&](Stage s, uint32_t w) {
    vp->stage[n] = (uint8_t)s;
    vp->workers[n] = w;
    ++n;
  };
  add(S_FRONT, n_front);
  // (twice the front end's workers: a small frame's survivors then get the raster's
  // lane groups, one group per survivor)
  const uint32_t n_rast = wk(T, 64);
  add(S_EXACT, n_rast);
  add(S_DEPTH_BIG, n_pix);
  if (v.ra.zmax) add(S_ZMAX, wk(pix, 8192));
  add(S_MARK, std::max(n_rast, n_pix));
  if (vm) add(S_INIT_V, wk(mesh->V, 128));
  add(S_LOCAL, n_tiles);
  add(vm ? S_HOOK_V : S_HOOK, vm ? n_tri : clampu((ntiles + 7) / 8, 1, G));
  if (!vm && mesh->n_nm) add(S_HOOK_NM, wk(mesh->n_nm, 128));
  add(S_FLATTEN, n_tiles);
  add(S_SCAN, 1);
  add(S_TRI_CHART, n_tiles);
  if (o->vert_chart) add(S_VERT_CHART, wk(mesh->V, 128));
  add(S_BBOX, n_tri);
  add(S_ORDER_TILE, order_tiles);  // one tile of boxes per worker
  add(S_ORDER_SCATTER, order_tiles);
  add(S_PACK_SCAN, clampu((uint64_t)chunks * p->n_scales, 1, G));
  add(S_PUSH, p->n_scales);  // one candidate per worker; the last one selects
  if (!uv) add(S_PLACE, wk(chart_cap, 128));
  else add(S_UV, n_tri);
  vp->n_stages = n;
}

size_t persist_smem(uint32_t front_cap) {
  return std::max<size_t>((size_t)kMaxH * 4u, pk::push_smem_bytes(front_cap));
}

// Resident CTAs of the launch (one per SM at 1024 threads and this shared memory),
// and the kernel's shared-memory limit, set once per process.
fa_status persist_grid(int device, uint32_t* G) {
  static int set = -1;
  if (set != device) {
    FA_CUDA_TRY(cudaFuncSetAttribute(k_persist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)persist_smem(kFrontCap)));
    FA_CUDA_TRY(cudaFuncSetAttribute(k_persist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)persist_smem(kFrontCap)));
    set = device;
  }
  int sms = 0, per = 0, per1 = 0;
  FA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  FA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persist<false>, kPT, persist_smem(kFrontCap)));
  FA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_persist<true>, kPT, persist_smem(kFrontCap)));
  per = std::min(per, per1);
  if (per < 1) return FA_E_CUDA;
  *G = (uint32_t)(sms * per);
  return FA_OK;
}

fa_status launch_persist(const PersistParams& P, uint32_t G, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kPT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (P.views) FA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_persist<false>, P));
  else FA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_persist<true>, P));
  return FA_OK;
}

}  // namespace

// One checked frame as one persistent launch (FA_FRAME_PERSISTENT).
fa_status enqueue_frame_persistent(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p,
                                   const float* d_view_proj, const fa_frame_out* o, cudaStream_t s) {
  uint32_t G = 0;
  fa_status st = persist_grid(ctx->device, &G);
  if (st != FA_OK) return st;
  PersistParams* P = new (std::nothrow) PersistParams;
  if (!P) return FA_E_OUT_OF_MEMORY;
  ViewPlan* vp = new (std::nothrow) ViewPlan;
  if (!vp) {
    delete P;
    return FA_E_OUT_OF_MEMORY;
  }
  build_view(ctx, mesh, p, d_view_proj, o, G, 100u, vp);
  std::memset(P, 0, sizeof(*P));
  P->inline_view = vp->va;
  uint32_t start = 0;
  for (uint32_t i = 0; i < vp->n_stages; ++i) {
    Group& g = P->inline_groups[i];
    g.start = start;
    g.workers = vp->workers[i];
    g.dep = i ? (int32_t)(i - 1) : -1;
    g.view = 0;
    g.stage = vp->stage[i];
    start += vp->workers[i];
  }
  P->views = nullptr;
  P->groups = nullptr;
  P->n_views = 1;
  P->n_groups = vp->n_stages;
  P->n_items = start;
  P->sched = ctx->psched;
  P->wait_ns = ctx->wait_ns;
  ctx->front_blocks = vp->va.ra.front_blocks;
  trace_begin(ctx);
  mark(ctx, "k_persist", s);
  st = launch_persist(*P, G, persist_smem(vp->front_cap), s);
  trace_end(ctx, s);
  delete vp;
  delete P;
  return st;
}

}  // namespace fa

// ------------------------------------------------------------------ batch plans

struct fa_batch_plan {
  fa_batch* batch;
  uint32_t n_views;
  std::vector<const fa_mesh*> meshes;
  std::vector<fa_frame_params> params;
  std::vector<const float*> dmat;
  std::vector<fa_frame_out> outs;
  fa_plan_schedule sched;
  uint32_t G = 0;
  size_t smem = 0;
  uint32_t n_groups = 0, n_items = 0;
  fa::ViewArgs* d_views = nullptr;
  fa::Group* d_groups = nullptr;
  uint32_t* d_sched = nullptr;
  uint32_t max_groups = 0;
};

namespace {

using fa::Group;
using fa::ViewArgs;
using fa::ViewPlan;

// Views of each lane in the order the lane runs them (the batch's assignment
// policies: round robin, or longest first onto the least-loaded lane).
std::vector<std::vector<uint32_t>> plan_lanes(const fa_batch_plan* pl, uint32_t lanes, uint32_t policy) {
  std::vector<std::vector<uint32_t>> out(lanes);
  const uint32_t n = pl->n_views;
  auto cost = [&](uint32_t i) {
    return (uint64_t)pl->meshes[i]->T + (uint64_t)pl->params[i].width * pl->params[i].height;
  };
  if (policy == FA_BATCH_ROUND_ROBIN) {
    for (uint32_t i = 0; i < n; ++i) out[i % lanes].push_back(i);
    return out;
  }
  std::vector<uint32_t> ord(n);
  for (uint32_t i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t c) { return cost(a) > cost(c); });
  std::vector<uint64_t> load(lanes, 0);
  for (uint32_t i : ord) {
    const uint32_t l = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
    out[l].push_back(i);
    load[l] += cost(i);
  }
  return out;
}

// Builds the views' arguments on their lanes and the claim order of the stage
// groups for the plan's schedule, and uploads both (synchronous: set-up).  Order:
// round r (the r-th view of every lane), then stage position, then lane; a view's
// first stage waits for the last stage of the lane's previous view.
fa_status plan_build(fa_batch_plan* pl) {
  fa_batch* b = pl->batch;
  const uint32_t lanes = pl->sched.lanes, n = pl->n_views;
  const auto assign = plan_lanes(pl, lanes, pl->sched.policy);
  std::vector<ViewPlan> vps(n);
  std::vector<ViewArgs> va(n);
  uint32_t front_cap = 0;
  for (uint32_t l = 0; l < lanes; ++l)
    for (uint32_t i : assign[l]) {
      fa::build_view(b->ctx[l], pl->meshes[i], &pl->params[i], pl->dmat[i], &pl->outs[i], pl->G,
                     pl->sched.worker_pct, &vps[i]);
      vps[i].va.ra.mid_max_pix = pl->sched.mid_max_pix;
      if (!(pl->sched.raster_flags & FA_RASTER_HIZ)) {
        vps[i].va.ra.zmax = nullptr;  // and no tile-depth stage
        uint32_t k = 0;
        for (uint32_t q = 0; q < vps[i].n_stages; ++q)
          if (vps[i].stage[q] != fa::S_ZMAX) {
            vps[i].stage[k] = vps[i].stage[q];
            vps[i].workers[k] = vps[i].workers[q];
            ++k;
          }
        vps[i].n_stages = k;
      } else if (!vps[i].va.ra.zmax) {
        vps[i].va.ra.zmax = b->ctx[l]->zmax;  // and a tile-depth stage before the marking
        uint32_t q = 0;
        while (q < vps[i].n_stages && vps[i].stage[q] != fa::S_MARK) ++q;
        for (uint32_t k = vps[i].n_stages; k > q; --k) {
          vps[i].stage[k] = vps[i].stage[k - 1];
          vps[i].workers[k] = vps[i].workers[k - 1];
        }
        const uint64_t pix = (uint64_t)pl->params[i].width * pl->params[i].height;
        vps[i].stage[q] = fa::S_ZMAX;
        vps[i].workers[q] = (uint32_t)std::min<uint64_t>(pl->G, std::max<uint64_t>(1, (pix + 8191) / 8192));
        ++vps[i].n_stages;
      }
      va[i] = vps[i].va;
      front_cap = std::max(front_cap, vps[i].front_cap);
    }
  std::vector<Group> groups;
  std::vector<int32_t> last(lanes, -1);  // last group of the lane's previous view
  std::vector<int32_t> prev(n, -1);      // previous group of each view
  uint32_t rounds = 0;
  for (const auto& a : assign) rounds = std::max<uint32_t>(rounds, (uint32_t)a.size());
  uint32_t start = 0;
  for (uint32_t r = 0; r < rounds; ++r) {
    uint32_t max_st = 0;
    for (uint32_t l = 0; l < lanes; ++l)
      if (r < assign[l].size()) max_st = std::max(max_st, vps[assign[l][r]].n_stages);
    for (uint32_t k = 0; k < max_st; ++k)
      for (uint32_t l = 0; l < lanes; ++l) {
        if (r >= assign[l].size()) continue;
        const uint32_t vi = assign[l][r];
        const ViewPlan& vp = vps[vi];
        if (k >= vp.n_stages) continue;
        Group g;
        g.start = start;
        g.workers = vp.workers[k];
        g.dep = k ? prev[vi] : last[l];
        g.view = (uint16_t)vi;
        g.stage = vp.stage[k];
        g.pad = 0;
        prev[vi] = (int32_t)groups.size();
        groups.push_back(g);
        start += g.workers;
        if (k + 1 == vp.n_stages) last[l] = prev[vi];
      }
  }
  if (groups.size() > pl->max_groups) return FA_E_CAPACITY;
  pl->n_groups = (uint32_t)groups.size();
  pl->n_items = start;
  pl->smem = fa::persist_smem(front_cap);
  FA_CUDA_TRY(cudaMemcpy(pl->d_views, va.data(), n * sizeof(ViewArgs), cudaMemcpyHostToDevice));
  FA_CUDA_TRY(cudaMemcpy(pl->d_groups, groups.data(), groups.size() * sizeof(Group), cudaMemcpyHostToDevice));
  return FA_OK;
}

}  // namespace

extern "C" {

void fa_batch_plan_destroy(fa_batch_plan* pl) {
  if (!pl) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(pl->batch->device);
  cudaDeviceSynchronize();
  if (pl->d_views) cudaFree(pl->d_views);
  if (pl->d_groups) cudaFree(pl->d_groups);
  if (pl->d_sched) cudaFree(pl->d_sched);
  if (prev >= 0) cudaSetDevice(prev);
  delete pl;
}

fa_status fa_batch_plan_create(fa_batch* b, uint32_t n_views, const fa_mesh* const* meshes,
                               const fa_frame_params* params, const float* const* d_view_proj,
                               const fa_frame_out* outs, fa_batch_plan** out) {
  if (!out) return FA_E_INVALID_ARG;
  *out = nullptr;
  if (!b || n_views == 0 || n_views > FA_PLAN_MAX_VIEWS || !meshes || !params || !outs) return FA_E_INVALID_ARG;
  for (uint32_t i = 0; i < n_views; ++i) {
    const float* dm = d_view_proj ? d_view_proj[i] : nullptr;
    fa_status st = fa::check_frame(b->ctx[0], meshes[i], &params[i], dm, &outs[i]);
    if (st != FA_OK) return st;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(b->device) != cudaSuccess) return FA_E_CUDA;
  fa_batch_plan* pl = new (std::nothrow) fa_batch_plan;
  if (!pl) return FA_E_OUT_OF_MEMORY;
  pl->batch = b;
  pl->n_views = n_views;
  pl->meshes.assign(meshes, meshes + n_views);
  pl->params.assign(params, params + n_views);
  pl->outs.assign(outs, outs + n_views);
  pl->dmat.assign(n_views, nullptr);
  if (d_view_proj) pl->dmat.assign(d_view_proj, d_view_proj + n_views);
  pl->sched.lanes = (uint32_t)b->ctx.size();
  pl->sched.policy = FA_BATCH_LONGEST_FIRST;
  pl->sched.worker_pct = 100;
  pl->sched.mid_max_pix = b->ctx[0]->mid_max_pix;
  pl->sched.raster_flags = b->ctx[0]->raster_flags;
  pl->max_groups = n_views * (uint32_t)fa::kMaxStages;
  fa_status st = fa::persist_grid(b->device, &pl->G);
  if (st == FA_OK && (cudaMalloc(&pl->d_views, n_views * sizeof(fa::ViewArgs)) != cudaSuccess ||
                      cudaMalloc(&pl->d_groups, pl->max_groups * sizeof(fa::Group)) != cudaSuccess ||
                      cudaMalloc(&pl->d_sched, (4 + pl->max_groups) * sizeof(uint32_t)) != cudaSuccess)) {
    cudaGetLastError();
    st = FA_E_OUT_OF_MEMORY;
  }
  if (st == FA_OK && cudaMemset(pl->d_sched, 0, (4 + pl->max_groups) * sizeof(uint32_t)) != cudaSuccess)
    st = FA_E_CUDA;
  if (st == FA_OK) st = plan_build(pl);
  if (st == FA_OK && cudaDeviceSynchronize() != cudaSuccess) st = FA_E_CUDA;
  if (prev >= 0) cudaSetDevice(prev);
  if (st != FA_OK) {
    fa_batch_plan_destroy(pl);
    return st;
  }
  *out = pl;
  return FA_OK;
}

fa_status fa_batch_plan_launch(fa_batch_plan* pl, fa_stream_t stream) {
  if (!pl) return FA_E_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != pl->batch->device && cudaSetDevice(pl->batch->device) != cudaSuccess) return FA_E_CUDA;
  fa::PersistParams* P = new (std::nothrow) fa::PersistParams;
  if (!P) return FA_E_OUT_OF_MEMORY;
  std::memset(P, 0, sizeof(*P));
  P->views = pl->d_views;
  P->groups = pl->d_groups;
  P->n_views = pl->n_views;
  P->n_groups = pl->n_groups;
  P->n_items = pl->n_items;
  P->sched = pl->d_sched;
  unsigned long long w = 0;
  for (fa_ctx* c : pl->batch->ctx) w = std::max(w, c->wait_ns);
  P->wait_ns = w;
  pl->batch->ctx[0]->launches++;
  fa_status st = fa::launch_persist(*P, pl->G, pl->smem, (cudaStream_t)stream);
  delete P;
  if (prev >= 0 && prev != pl->batch->device) cudaSetDevice(prev);
  return st;
}

fa_status fa_batch_plan_get_schedule(const fa_batch_plan* pl, fa_plan_schedule* s) {
  if (!pl || !s) return FA_E_INVALID_ARG;
  *s = pl->sched;
  return FA_OK;
}

fa_status fa_batch_plan_set_schedule(fa_batch_plan* pl, const fa_plan_schedule* s) {
  if (!pl || !s || s->lanes == 0 || s->lanes > pl->batch->ctx.size() || s->policy > FA_BATCH_LONGEST_FIRST ||
      s->worker_pct < 10 || s->worker_pct > 1000 || s->mid_max_pix < FA_RASTER_MID_OFF ||
      s->mid_max_pix > FA_RASTER_MID_MAX || (s->raster_flags & ~FA_RASTER_HIZ))
    return FA_E_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(pl->batch->device) != cudaSuccess) return FA_E_CUDA;
  fa_status st = cudaDeviceSynchronize() == cudaSuccess ? FA_OK : FA_E_CUDA;  // no launch reads the old plan
  if (st == FA_OK) {
    pl->sched = *s;
    st = plan_build(pl);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

fa_status fa_batch_plan_tune(fa_batch_plan* pl, uint32_t reps, float* best_ms) {
  if (!pl) return FA_E_INVALID_ARG;
  if (reps == 0) reps = 3;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(pl->batch->device) != cudaSuccess) return FA_E_CUDA;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (prev >= 0) cudaSetDevice(prev);
    return FA_E_CUDA;
  }
  const uint32_t max_lanes = (uint32_t)pl->batch->ctx.size();
  std::vector<uint32_t> lanes;
  for (uint32_t l = 1; l < max_lanes; l <<= 1) lanes.push_back(l);
  lanes.push_back(max_lanes);
  fa_plan_schedule best = pl->sched;
  float best_t = -1.0f;
  fa_status st = FA_OK;
  auto trial = [&](const fa_plan_schedule& c) {
    if (st != FA_OK) return;
    st = fa_batch_plan_set_schedule(pl, &c);
    if (st != FA_OK) return;
    float ms = 0.0f;
    bool ok = fa_batch_plan_launch(pl, s) == FA_OK;  // warm-up
    for (uint32_t r = 0; ok && r < reps; ++r) {
      float t = 0.0f;
      ok = cudaEventRecord(e0, s) == cudaSuccess && fa_batch_plan_launch(pl, s) == FA_OK &&
           cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
      if (ok && (r == 0 || t < ms)) ms = t;
    }
    if (!ok) {
      cudaGetLastError();
      st = FA_E_CUDA;
      return;
    }
    if (best_t < 0.0f || ms < best_t) {
      best_t = ms;
      best = c;
    }
  };
  // the raster schedule first (at the plan's lanes, policy and worker counts), then
  // lanes x policy x worker counts with the best raster schedule
  const fa_plan_schedule start = pl->sched;
  const uint32_t mids[] = {FA_RASTER_MID_OFF, 64};
  for (uint32_t mid : mids)
    for (uint32_t fl = 0; fl <= FA_RASTER_HIZ; ++fl) trial(fa_plan_schedule{start.lanes, start.policy,
                                                                             start.worker_pct, mid, fl});
  const uint32_t best_mid = best.mid_max_pix, best_fl = best.raster_flags;
  const uint32_t pcts[] = {50, 100, 200};
  for (uint32_t l : lanes)
    for (uint32_t pol = FA_BATCH_ROUND_ROBIN; pol <= FA_BATCH_LONGEST_FIRST; ++pol)
      for (uint32_t pct : pcts) {
        if (l == 1 && pol == FA_BATCH_LONGEST_FIRST) continue;  // the same order as round robin
        trial(fa_plan_schedule{l, pol, pct, best_mid, best_fl});
      }
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == FA_OK) st = fa_batch_plan_set_schedule(pl, &best);
  if (best_ms) *best_ms = best_t;
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

}  // extern "C"
