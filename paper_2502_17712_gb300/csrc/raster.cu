// Visibility kernels (Sec. 5.1; App. A "Detecting Visible Triangles"): the launch
// wrappers of the stage bodies in raster.cuh and the launch sequence of one
// visibility pass.
#include <algorithm>

#include "raster.cuh"

namespace fa {
namespace {

using rs::RasterArgs;

template <bool DEV_M>
__global__ void __launch_bounds__(rs::kFrontThreads, 2) k_raster_front(RasterArgs A) {
  pdl_wait();
  rs::front_body<DEV_M>(A, blockIdx.x, gridDim.x);
}

template <bool DEV_M>
__global__ void __launch_bounds__(256, 4) k_raster_exact(RasterArgs A) {
  pdl_wait();
  rs::exact_body<DEV_M, 256>(A, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_raster_depth_big(RasterArgs A) {
  pdl_wait();
  rs::depth_big_body(A, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_raster_zmax(RasterArgs A) {
  pdl_wait();
  rs::zmax_body(A, blockIdx.x, gridDim.x);
}

template <bool CONS>
__global__ void __launch_bounds__(256, 4) k_raster_mark(RasterArgs A) {
  pdl_wait();
  rs::mark_body<CONS, 256>(A, blockIdx.x, gridDim.x);
}

}  // namespace

fa_status launch_visibility(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W, uint32_t H,
                            uint32_t* vt, bool reset_status, cudaStream_t s, const float* Mdev, bool cons,
                            int32_t* tri_chart_init) {
  // one wave (two resident blocks per SM): half the survivor regions of two waves,
  // so the passes that look regions up scan fewer counts
  // (and enough blocks for the clears: at most 16 depth-buffer pixels per thread)
  const uint32_t fb = std::max(grid_for(mesh->T, rs::kFrontThreads, 152u * 2u),
                               grid_for((uint64_t)W * H, rs::kFrontThreads * 16u, 152u * 2u));
  const RasterArgs A = rs::make_raster_args(ctx, mesh, M, W, H, vt, reset_status, Mdev, cons, tri_chart_init, fb,
                                            rs::kFrontThreads);
  ctx->front_blocks = A.front_blocks;
  const unsigned gb = 152 * 8;
  mark(ctx, "k_raster_front", s);
  if (Mdev)
    launch_k(k_raster_front<true>, A.front_blocks, rs::kFrontThreads, 0, s, A);
  else
    launch_k(k_raster_front<false>, A.front_blocks, rs::kFrontThreads, 0, s, A);
  mark(ctx, "k_raster_exact", s);
  if (Mdev)
    launch_k(k_raster_exact<true>, 152 * 8, 256, 0, s, A);
  else
    launch_k(k_raster_exact<false>, 152 * 8, 256, 0, s, A);
  mark(ctx, "k_raster_depth_big", s);
  launch_k(k_raster_depth_big, gb, 256, 0, s, A);
  if (A.zmax) {
    mark(ctx, "k_raster_zmax", s);
    launch_k(k_raster_zmax, grid_for((uint64_t)A.ztx * ((H + 15) / 16) * 32, 256, 152 * 8), 256, 0, s, A);
  }
  mark(ctx, "k_raster_mark", s);
  // one wave of four resident blocks per SM: each block scans the region counts once
  if (cons)
    launch_k(k_raster_mark<true>, 152 * 4, 256, 0, s, A);
  else
    launch_k(k_raster_mark<false>, 152 * 4, 256, 0, s, A);
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
}

}  // namespace fa
