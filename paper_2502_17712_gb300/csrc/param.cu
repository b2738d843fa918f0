// Chart boxes, footprints and UVs (Sec. 5.2, Sec. 4.1, Sec. 3 / App. A): the
// launch wrappers of the stage bodies in param.cuh and their launch sequences.
#include "param.cuh"

namespace fa {
namespace {

using pm::BoxArgs;
using pm::UvArgs;

template <bool DEV_M>
__global__ void __launch_bounds__(256) k_bbox(BoxArgs a) {
  pdl_wait();
  pm::bbox_body<DEV_M>(a, blockIdx.x, gridDim.x);
}

template <bool DEV_M>
__global__ void __launch_bounds__(256) k_uv(UvArgs a) {
  pdl_wait();
  pm::uv_body<DEV_M>(a, blockIdx.x, gridDim.x);
}

__global__ void k_box_reset(const uint32_t* count, uint32_t max_charts, uint32_t* box_enc, uint32_t* box_full) {
  pdl_wait();
  const uint32_t C = min(__ldcg(count), max_charts);
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    reinterpret_cast<uint4*>(box_enc)[c] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
    box_full[c] = 0u;
  }
}

__global__ void k_footprint(const uint32_t* count, uint32_t max_charts, FootArgs f, DevCounters* ctr) {
  pdl_wait();
  if (__ldcg(&ctr->status) != 0) return;
  const uint32_t C = min(__ldcg(count), max_charts);
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
    chart_footprint(f, c);
}

}  // namespace

FootArgs foot_args(fa_ctx* ctx, uint32_t W, uint32_t H, float ratio, const fa_charts* ch) {
  FootArgs f;
  f.box_enc = ctx->box_enc;
  f.box_full = ctx->box_full;
  f.hx = 0.5f * (float)W;
  f.hy = 0.5f * (float)H;
  f.s256 = 256.0f * ratio;
  f.bbox = ch->bbox;
  f.fa = ch->fa;
  f.fb = ch->fb;
  f.rot = ch->rot;
  return f;
}

fa_status launch_parameterize(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W, uint32_t H,
                              float ratio, const int32_t* tri_chart, const fa_charts* ch, bool reset_boxes,
                              uint32_t flags, uint32_t* partial, cudaStream_t s, const float* Mdev,
                              bool footprint) {
  if (partial) FA_CUDA_TRY(cudaMemsetAsync(partial, 0, (size_t)((mesh->T + 31) / 32) * 4, s));
  if (reset_boxes) {
    mark(ctx, "k_box_reset", s);
    launch_k(k_box_reset, grid_for(ctx->cfg.max_charts, 256, 152 * 4), 256, 0, s, ch->count, ctx->cfg.max_charts,
                                                                            ctx->box_enc, ctx->box_full);
  }
  const BoxArgs a = pm::make_box_args(ctx, mesh, M, tri_chart, flags, partial, Mdev);
  mark(ctx, "k_bbox", s);
  if (Mdev)
    launch_k(k_bbox<true>, grid_for(mesh->T, 256, 152 * 8), 256, 0, s, a);
  else
    launch_k(k_bbox<false>, grid_for(mesh->T, 256, 152 * 8), 256, 0, s, a);
  if (footprint) {
    mark(ctx, "k_footprint", s);
    launch_k(k_footprint, grid_for(ctx->cfg.max_charts, 256, 152 * 4), 256, 0, s, ch->count, ctx->cfg.max_charts,
             foot_args(ctx, W, H, ratio, ch), ctx->ctr);
  }
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
}

fa_status launch_uv(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W, uint32_t H, float ratio,
                    const int32_t* tri_chart, const fa_charts* ch,
                    const fa_placement* place, const fa_pack_result* res, uint32_t atlas_log2,
                    uint32_t n_scales, float* uv, float* affine, cudaStream_t s, const float* Mdev,
                    bool from_candidates) {
  const UvArgs a = pm::make_uv_args(ctx, mesh, M, W, H, ratio, tri_chart, ch, place, res, atlas_log2, n_scales, uv,
                                    affine, Mdev, from_candidates);
  mark(ctx, "k_uv", s);
  if (Mdev)
    launch_k(k_uv<true>, grid_for(mesh->T, 256, 152 * 8), 256, 0, s, a);
  else
    launch_k(k_uv<false>, grid_for(mesh->T, 256, 152 * 8), 256, 0, s, a);
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
}

}  // namespace fa
