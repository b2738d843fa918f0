// Box order and packing (Sec. 4.1-4.3): the launch wrappers of the stage bodies in
// pack.cuh, the launch sequence of one packing, and the allocation-free packing
// entry point.
#include "pack.cuh"

namespace fa {
namespace {

using pk::PackArgs;

template <bool FOOT>
__global__ void __launch_bounds__(kOrderTile) k_order_tile(PackScratch p, const uint32_t* __restrict__ fb,
                                                           FootArgs foot) {
  pdl_wait();
  __shared__ uint32_t hist[kMaxH];
  pk::order_tile_body<FOOT>(p, fb, foot, blockIdx.x, hist);
}

__global__ void __launch_bounds__(kOrderTile) k_order_scatter(PackScratch p, const uint32_t* __restrict__ fa,
                                                              const uint32_t* __restrict__ fb, uint32_t* order) {
  pdl_wait();
  __shared__ uint32_t binstart[kMaxH];
  pk::order_scatter_body(p, fa, fb, order, blockIdx.x, binstart);
}

__global__ void __launch_bounds__(pk::kScanThreads, 2) k_pack_scan(PackScratch p, PackArgs a, uint32_t n_scales) {
  pdl_wait();
  pk::pack_scan_body<pk::kScanThreads>(p, a, n_scales, blockIdx.x, gridDim.x);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_pack_push(PackScratch p, PackArgs a) {
  pdl_wait();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pk::push_body<NT>(p, a, blockIdx.x, gridDim.x, smem_raw);
}

__global__ void __launch_bounds__(256) k_pack_place(PackScratch p, PackArgs a) {
  pdl_wait();
  pk::pack_place_body(p, a, blockIdx.x, gridDim.x);
}

}  // namespace

fa_status launch_pack_kernels(fa_ctx* ctx, const PackScratch& p, const uint32_t* fa_, const uint32_t* fb,
                              uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode, uint32_t min_box,
                              uint32_t gutter, uint32_t* order, fa_placement* place, fa_pack_result* res,
                              cudaStream_t s, uint32_t lowres_log2, const FootArgs* foot, bool write_place) {
  uint32_t* ord = order ? order : p.order;
  if (ctx) mark(ctx, "k_order_tile", s);
  if (foot)
    launch_k(k_order_tile<true>, p.max_tiles, kOrderTile, 0, s, p, fb, *foot);
  else
    launch_k(k_order_tile<false>, p.max_tiles, kOrderTile, 0, s, p, fb, FootArgs{});
  if (ctx) mark(ctx, "k_order_scatter", s);
  launch_k(k_order_scatter, p.max_tiles, kOrderTile, 0, s, p, fa_, fb, ord);
  const PackArgs a = pk::make_pack_args(ctx, ord, atlas_log2, n_scales, select_mode, min_box, gutter, lowres_log2,
                                        place, res);
  const uint32_t items = p.max_chunks * n_scales;
  const unsigned g2 = items < 152u * 2u ? items : 152u * 2u;  // two 512-thread CTAs per SM
  if (ctx) mark(ctx, "k_pack_scan", s);
  launch_k(k_pack_scan, g2, pk::kScanThreads, 0, s, p, a, n_scales);
  if (ctx) mark(ctx, "k_pack_push", s);
  // one CTA per candidate, of the context's push shape (the allocation-free entry,
  // without a context, takes the default)
  const uint32_t pt = ctx ? ctx->push_threads : (uint32_t)pk::kPushThreads;
  const size_t psm = pk::push_smem_bytes(a.front_cap);
  if (pt == 256)
    launch_k(k_pack_push<256>, n_scales, 256, psm, s, p, a);
  else if (pt == 512)
    launch_k(k_pack_push<512>, n_scales, 512, psm, s, p, a);
  else
    launch_k(k_pack_push<1024>, n_scales, 1024, psm, s, p, a);
  if (write_place) {
    if (ctx) mark(ctx, "k_pack_place", s);
    launch_k(k_pack_place, 152 * 2, 256, 0, s, p, a);
  }
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
}

fa_status pack_set_smem_limit() {
  FA_CUDA_TRY(cudaFuncSetAttribute(k_pack_push<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)pk::push_smem_bytes(kFrontCap)));
  FA_CUDA_TRY(cudaFuncSetAttribute(k_pack_push<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)pk::push_smem_bytes(kFrontCap)));
  FA_CUDA_TRY(cudaFuncSetAttribute(k_pack_push<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)pk::push_smem_bytes(kFrontCap)));
  return FA_OK;
}

fa_status launch_pack(fa_ctx* ctx, const uint32_t* fa_, const uint32_t* fb, const uint32_t* count,
                      uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode, uint32_t* order,
                      fa_placement* place, fa_pack_result* res, cudaStream_t s, uint32_t lowres_log2,
                      const FootArgs* foot, bool write_place) {
  if (!ctx->pack_smem_set) {
    fa_status st = pack_set_smem_limit();
    if (st != FA_OK) return st;
    ctx->pack_smem_set = 1;
  }
  PackScratch p = ctx->pack;
  p.count = count;
  return launch_pack_kernels(ctx, p, fa_, fb, atlas_log2, n_scales, select_mode, ctx->cfg.min_box,
                             ctx->cfg.gutter, order, place, res, s, lowres_log2, foot, write_place);
}

}  // namespace fa

// ------------------------------------------------------------------ allocation-free packing
//
// fa_pack_noalloc runs the same order and pack kernels as fa_pack, but its scratch
// is one file-scope device array instead of context memory, so the call itself never
// allocates.  It exists for callers that are not allowed to allocate device memory
// at the point where they pack: code running inside a host application's frame
// callback or plugin slot whose device memory is owned and budgeted by the host,
// and real-time loops that must not hit cudaMalloc's implicit device
// synchronization.  The array (about 4.8 MiB, for up to 4096 boxes) stays resident
// on every GPU that loads the library, until the process exits.

#include <mutex>

namespace fa {
namespace {

constexpr uint32_t kNoAllocMaxBoxes = 4096;
constexpr uint32_t kNoAllocTiles = kNoAllocMaxBoxes / kOrderTile;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCtr = 0;
constexpr size_t kOffCount = align256(kOffCtr + sizeof(DevCounters));
constexpr size_t kOffCand = align256(kOffCount + sizeof(uint32_t));
constexpr size_t kOffM = align256(kOffCand + sizeof(PackCand) * kMaxScales);
constexpr size_t kOffCounts = align256(kOffM + sizeof(uint32_t) * kMaxScales);
constexpr size_t kOffRank = align256(kOffCounts + sizeof(uint32_t) * kMaxH * kNoAllocTiles);
constexpr size_t kOffTotal = align256(kOffRank + sizeof(uint32_t) * kNoAllocMaxBoxes);
constexpr size_t kOffOrder = align256(kOffTotal + sizeof(uint32_t) * kMaxH);
constexpr size_t kOffFs = align256(kOffOrder + sizeof(uint32_t) * kNoAllocMaxBoxes);
constexpr size_t kOffRec8 = align256(kOffFs + sizeof(uint2) * kNoAllocMaxBoxes);
constexpr size_t kOffSegs = align256(kOffRec8 + sizeof(uint2) * kMaxScales * kNoAllocMaxBoxes);
constexpr size_t kOffState = align256(kOffSegs + sizeof(uint16_t) * kMaxScales * kSegStride);
constexpr size_t kOffXY = align256(kOffState + sizeof(unsigned long long) * kMaxScales);
constexpr size_t kNoAllocBytes = align256(kOffXY + sizeof(uint2) * kMaxScales * kNoAllocMaxBoxes);

// The scratch of fa_pack_noalloc.  Host code must not use this name as a device
// address: it is a host-side shadow there; the device address comes from
// cudaGetSymbolAddress in noalloc_scratch() below.
static __device__ __align__(256) unsigned char g_pack_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Once per device, with that device current: the array's device address, and the
// push kernel's shared-memory limit.
fa_status noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return FA_E_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pack_scratch) != cudaSuccess) {
      cudaGetLastError();
      return FA_E_CUDA;
    }
    if (pack_set_smem_limit() != FA_OK) {
      cudaGetLastError();
      return FA_E_CUDA;
    }
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return FA_OK;
}

// Clears what the kernels expect at zero (status word, finished-candidate counter,
// bin totals) and stores the box count where the kernels read it.
__global__ void k_noalloc_reset(DevCounters* ctr, uint32_t* count, uint32_t* total, uint32_t n) {
  pdl_wait();
  if (threadIdx.x == 0) {
    ctr->status = 0;
    ctr->pack_done = 0;
    *count = n;
  }
  for (uint32_t b = threadIdx.x; b < kMaxH; b += blockDim.x) total[b] = 0;
}

}  // namespace
}  // namespace fa

extern "C" fa_status fa_pack_noalloc(const uint32_t* d_fa, const uint32_t* d_fb, uint32_t n,
                                     uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode,
                                     uint32_t min_box, uint32_t gutter, uint32_t* d_order,
                                     fa_placement* d_place, fa_pack_result* d_res, fa_stream_t stream) {
  using namespace fa;
  if (!d_fa || !d_fb || !d_place || !d_res) return FA_E_INVALID_ARG;
  if (atlas_log2 < 1 || atlas_log2 > 14) return FA_E_INVALID_ARG;
  if (n_scales == 0 || (n_scales & (n_scales - 1)) || n_scales > (uint32_t)kMaxScales) return FA_E_INVALID_ARG;
  if (select_mode > FA_SELECT_LARGEST_K) return FA_E_INVALID_ARG;
  if (min_box < 1 || min_box > 4096 || gutter > 4096) return FA_E_INVALID_ARG;
  if (n > kNoAllocMaxBoxes) return FA_E_CAPACITY;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FA_E_CUDA;
  }
  unsigned char* base = nullptr;
  fa_status st = noalloc_scratch(dev, &base);
  if (st != FA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  PackScratch p;
  p.ctr = (DevCounters*)(base + kOffCtr);
  p.count = (uint32_t*)(base + kOffCount);
  p.max_boxes = kNoAllocMaxBoxes;
  p.max_tiles = kNoAllocTiles;
  p.ord_counts = (uint32_t*)(base + kOffCounts);
  p.ord_rank = (uint32_t*)(base + kOffRank);
  p.ord_total = (uint32_t*)(base + kOffTotal);
  p.order = (uint32_t*)(base + kOffOrder);
  p.max_chunks = kNoAllocMaxBoxes / kChunk;
  p.fs = (uint2*)(base + kOffFs);
  p.rec8 = (uint2*)(base + kOffRec8);
  p.segs = (uint16_t*)(base + kOffSegs);
  p.scan_state = (unsigned long long*)(base + kOffState);
  p.m = (uint32_t*)(base + kOffM);
  p.xy = (uint2*)(base + kOffXY);
  p.cand = (PackCand*)(base + kOffCand);
  launch_k(k_noalloc_reset, 1, 256, 0, s, p.ctr, (uint32_t*)p.count, p.ord_total, n);
  return launch_pack_kernels(nullptr, p, d_fa, d_fb, atlas_log2, n_scales, select_mode, min_box, gutter, d_order,
                             d_place, d_res, s, 0u, nullptr, true);
}
