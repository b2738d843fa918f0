// Chart kernels (Sec. 5.1; App. A "GPU Union Find", Alg. 1): the launch wrappers
// of the stage bodies in chartify.cuh, the standalone visible-list kernels and the
// launch sequence of one chart pass.
#include <algorithm>

#include "chartify.cuh"

namespace fa {
namespace {

using cf::UfArgs;
using cf::kBlock;
using cf::kPerBlock;
using cf::kTile;

template <bool LIST, int NT>
__global__ void __launch_bounds__(NT) k_uf_local(UfArgs a) {
  pdl_wait();
  cf::local_body<LIST, NT>(a, blockIdx.x, gridDim.x);
}

// The local union-find with the context's tile shape (NT threads per tile; listed
// tiles: a grid of the resident blocks, 2048 / NT per SM).
template <bool LIST>
void launch_local(uint32_t nt, uint32_t ntiles, cudaStream_t s, const UfArgs& a) {
  auto grid = [&](uint32_t per_sm) { return LIST ? std::min(ntiles, 152u * per_sm) : ntiles; };
  if (nt == 256)
    launch_k(k_uf_local<LIST, 256>, grid(8), 256, 0, s, a);
  else if (nt == 512)
    launch_k(k_uf_local<LIST, 512>, grid(4), 512, 0, s, a);
  else
    launch_k(k_uf_local<LIST, 1024>, grid(2), 1024, 0, s, a);
}

__global__ void k_uf_init_v(int32_t* label, uint32_t T, uint32_t V) {
  pdl_wait();
  cf::init_v_body(label, T, V, blockIdx.x, gridDim.x);
}

template <bool LIST>
__global__ void __launch_bounds__(128) k_uf_hook(UfArgs a) {
  pdl_wait();
  cf::hook_body<LIST>(a, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kBlock) k_uf_hook_v(UfArgs a) {
  pdl_wait();
  cf::hook_v_body(a, blockIdx.x, gridDim.x);
}

__global__ void k_uf_hook_nm(UfArgs a, const uint32_t* nm_off, const uint32_t* nm_list, uint32_t n_nm) {
  pdl_wait();
  cf::hook_nm_body(a, nm_off, nm_list, n_nm, blockIdx.x, gridDim.x);
}

template <bool LIST>
__global__ void __launch_bounds__(kBlock) k_uf_flatten(UfArgs a, uint32_t* blockcnt, uint32_t* viscnt,
                                                       uint2* wordroots) {
  pdl_wait();
  cf::flatten_body<LIST, kBlock>(a, blockcnt, viscnt, wordroots, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t* blockcnt, uint32_t* viscnt, uint32_t nblocks,
                                                      uint32_t* count_out, uint32_t max_charts,
                                                      DevCounters* ctr) {
  pdl_wait();
  cf::scan_blocks_body(blockcnt, viscnt, nblocks, count_out, max_charts, ctr);
}

__global__ void __launch_bounds__(1024) k_scan_vis(uint32_t* viscnt, uint32_t nblocks, DevCounters* ctr) {
  pdl_wait();
  cf::scan_vis_body(viscnt, nblocks, ctr);
}

template <bool LIST>
__global__ void __launch_bounds__(kBlock) k_tri_chart(UfArgs a, const uint32_t* blockcnt, const uint2* wordroots,
                                                      int32_t* tri_chart, uint32_t* roots, uint32_t* box_enc,
                                                      uint32_t* box_full, uint32_t max_charts,
                                                      const uint32_t* visstart, uint2* vis) {
  pdl_wait();
  cf::tri_chart_body<LIST, kBlock>(a, blockcnt, wordroots, tri_chart, roots, box_enc, box_full, max_charts,
                                   visstart, vis, blockIdx.x, gridDim.x);
}

__global__ void k_vert_chart(UfArgs a, const uint32_t* blockcnt, const uint2* wordroots, int32_t* vert_chart,
                             int vertex_mode) {
  pdl_wait();
  cf::vert_chart_body(a, blockcnt, wordroots, vert_chart, vertex_mode, blockIdx.x, gridDim.x);
}

// Standalone path: visible counts per block from a caller's tri_chart ...
__global__ void __launch_bounds__(kBlock) k_vis_count(const int32_t* tri_chart, uint32_t T, uint32_t* viscnt) {
  pdl_wait();
  __shared__ uint32_t vc[kBlock / 32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t v = 0;
#pragma unroll
  for (uint32_t k = 0; k < kPerBlock / kBlock; ++k) {
    const uint32_t t = blockIdx.x * kPerBlock + (k * (kBlock / 32) + wid) * 32 + lane;
    v += __popc(__ballot_sync(0xFFFFFFFFu, t < T && tri_chart[t] >= 0));
  }
  if (lane == 0) vc[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int i = 0; i < kBlock / 32; ++i) s += vc[i];
    viscnt[blockIdx.x] = s;
  }
}

// ... and the list itself, after k_scan_vis.
__global__ void __launch_bounds__(kBlock) k_vis_fill(const int32_t* tri_chart, uint32_t T, const uint32_t* visstart,
                                                     uint2* vis) {
  pdl_wait();
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t words[kPerBlock / kBlock];
  int32_t chart[kPerBlock / kBlock];
#pragma unroll
  for (uint32_t k = 0; k < kPerBlock / kBlock; ++k) {
    const uint32_t t = blockIdx.x * kPerBlock + (k * (kBlock / 32) + wid) * 32 + lane;
    chart[k] = t < T ? tri_chart[t] : -1;
    words[k] = __ballot_sync(0xFFFFFFFFu, chart[k] >= 0);
  }
  cf::put_visible<kBlock>(words, __ldcg(visstart + blockIdx.x), chart, vis, blockIdx.x);
}

}  // namespace

fa_status launch_chartify(fa_ctx* ctx, const fa_mesh* mesh, const uint32_t* vt, uint32_t mode,
                          int32_t* tri_chart, int32_t* vert_chart, const fa_charts* ch, cudaStream_t s,
                          bool tile_list, bool tri_chart_cleared) {
  const UfArgs a = cf::make_uf_args(ctx, mesh, vt);
  const int vm = mode == FA_CHARTS_VERTEX;
  const unsigned gw = grid_for((uint64_t)((mesh->T + 31) / 32) * 32, kBlock, 152 * 16);
  if (vm) {
    mark(ctx, "k_uf_init_v", s);
    launch_k(k_uf_init_v, grid_for(mesh->V, 256, 152 * 8), 256, 0, s, ctx->label, mesh->T, mesh->V);
  }
  const uint32_t ntiles = (mesh->T + kTile - 1) / kTile;
  mark(ctx, "k_uf_local", s);
  if (tile_list)
    launch_local<true>(ctx->uf_threads, ntiles, s, a);
  else
    launch_local<false>(ctx->uf_threads, ntiles, s, a);
  mark(ctx, "k_uf_hook", s);
  if (vm)
    launch_k(k_uf_hook_v, gw, kBlock, 0, s, a);
  else if (tile_list)
    launch_k(k_uf_hook<true>, ntiles < 152u * 8u ? ntiles : 152u * 8u, 128, 0, s, a);
  else
    launch_k(k_uf_hook<false>, ntiles, 128, 0, s, a);
  if (!vm && mesh->n_nm) {
    mark(ctx, "k_uf_hook_nm", s);
    launch_k(k_uf_hook_nm, grid_for(mesh->n_nm, 256), 256, 0, s, a, mesh->nm_off, mesh->nm_list, mesh->n_nm);
  }
  const uint32_t nb = (mesh->T + kPerBlock - 1) / kPerBlock;
  mark(ctx, "k_uf_flatten", s);
  if (tile_list)
    launch_k(k_uf_flatten<true>, nb < 152u * 8u ? (nb ? nb : 1u) : 152u * 8u, kBlock, 0, s, a, ctx->blockcnt,
             ctx->viscnt, ctx->wordroots);
  else
    launch_k(k_uf_flatten<false>, nb ? nb : 1, kBlock, 0, s, a, ctx->blockcnt, ctx->viscnt, ctx->wordroots);
  mark(ctx, "k_scan_blocks", s);
  launch_k(k_scan_blocks, 1, 1024, 0, s, ctx->blockcnt, ctx->viscnt, nb ? nb : 1, ch->count, ctx->cfg.max_charts,
           ctx->ctr);
  mark(ctx, "k_tri_chart", s);
  if (tile_list && tri_chart_cleared)
    launch_k(k_tri_chart<true>, nb < 152u * 8u ? (nb ? nb : 1u) : 152u * 8u, kBlock, 0, s, a, ctx->blockcnt,
             ctx->wordroots, tri_chart, ch->root, ctx->box_enc, ctx->box_full, ctx->cfg.max_charts, ctx->viscnt,
             ctx->vis);
  else
    launch_k(k_tri_chart<false>, nb ? nb : 1, kBlock, 0, s, a, ctx->blockcnt, ctx->wordroots, tri_chart, ch->root,
             ctx->box_enc, ctx->box_full, ctx->cfg.max_charts, ctx->viscnt, ctx->vis);
  if (vert_chart) {
    mark(ctx, "k_vert_chart", s);
    launch_k(k_vert_chart, grid_for(mesh->V, 256, 152 * 8), 256, 0, s, a, ctx->blockcnt, ctx->wordroots,
             vert_chart, vm);
  }
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
}

fa_status launch_vis_list(fa_ctx* ctx, const fa_mesh* mesh, const int32_t* tri_chart, cudaStream_t s) {
  const uint32_t nb = (mesh->T + kPerBlock - 1) / kPerBlock;
  mark(ctx, "k_vis_count", s);
  launch_k(k_vis_count, nb ? nb : 1, kBlock, 0, s, tri_chart, mesh->T, ctx->viscnt);
  mark(ctx, "k_scan_vis", s);
  launch_k(k_scan_vis, 1, 1024, 0, s, ctx->viscnt, nb ? nb : 1, ctx->ctr);
  mark(ctx, "k_vis_fill", s);
  launch_k(k_vis_fill, nb ? nb : 1, kBlock, 0, s, tri_chart, mesh->T, ctx->viscnt, ctx->vis);
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
}

}  // namespace fa
