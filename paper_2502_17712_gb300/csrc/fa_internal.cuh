// Internal declarations shared by the CUDA translation units of libfastatlas.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fastatlas.h"

namespace fa {

// ----------------------------------------------------------------- constants

constexpr float kGuard = 64.0f;     // guard band |x|,|y| <= kGuard * w
constexpr int kSub = 256;           // sub-pixel steps per pixel (1/256 px snapping)
constexpr uint32_t kMaxH = 8192;    // height buckets of the box order (Sec. 4.1)
constexpr int kMaxScales = 64;      // candidate scales (Sec. 4.2)
constexpr uint32_t kFrontCap = 32768;  // frontline entries per candidate (smem)
constexpr int kBigTile = 16;        // tile side of the large-triangle raster
constexpr int kSmallMaxPix = 16;    // in-thread raster when the pixel box has <= this
// boxes of up to mid_max_pix pixels (a per-context schedule knob, fa_set_raster_schedule)
// are also rasterized in-thread when that costs the warp less than the tiles:
constexpr uint32_t kMidSampleCost = 2;  // relative cost of one in-thread sample
constexpr uint32_t kMidStepCost = 3;    // of one warp step of a tile
constexpr uint32_t kMidTriCost = 10;    // of one queued triangle's record and set-up
constexpr int kOrderTile = 1024;    // boxes per tile of the stable order
constexpr uint32_t kLoopCap = FA_DEFAULT_LOOP_CAP;  // device iteration cap (FA_E_TIMEOUT)
constexpr unsigned long long kWaitNs = FA_DEFAULT_WAIT_NS;  // device time limit of a bulk-copy wait

// ----------------------------------------------------------------- device state

// Small counters that live in device memory (one struct per context).
constexpr uint32_t kMaxFrontBlocks = 152 * 4;  // raster front-end blocks (survivor regions)
constexpr uint32_t kDefaultPushThreads = 512;  // threads of a candidate's push CTA (fa_set_chart_pack_schedule)
constexpr uint32_t kPschedWords = 64;          // schedule state of a single-view persistent launch

struct DevCounters {
  int32_t status;          // sticky fa_status of the context
  uint32_t pad0;
  unsigned long long big;  // big-triangle queue: entries << 40 | tiles
  uint32_t pack_done;      // candidate CTAs finished (last one selects)
  uint32_t ncand;          // small sub-triangles recorded by the depth pre-pass
  uint32_t order_tiles;    // tiles of the current order pass
  uint32_t chart_count;    // scratch copy of the frame's chart count
  uint32_t n_groups[kMaxScales];
  uint32_t n_vis;          // entries of the visible-triangle list
  uint32_t n_vtiles;       // 1024-triangle tiles with a visible triangle (listed by the marking pass)
  uint32_t uf_item;        // next listed tile of the local union-find
};

// One queued (large) sub-triangle of the raster: snapped vertices, depths and its
// clamped pixel box; tiles [tile0, tile0 + ntiles) of the queue belong to it.
struct BigTri {
  int32_t X[3], Y[3];
  float zn[3];
  int32_t px0, py0, px1, py1;
  uint32_t tri;
  uint32_t tile0;
  uint32_t pad;
};
static_assert(sizeof(BigTri) == 64, "BigTri is one 64-byte record");

struct PackCand {
  uint32_t ok;      // 1 = fits
  uint32_t omega;   // Omega
  uint32_t height;  // H
  int32_t status;   // FA_OK / FA_E_CAPACITY
};

// Boxes per pack chunk: the unit of the width scan (one work item per candidate and
// chunk) and of the push's shared-memory staging.
constexpr uint32_t kChunk = 4096;
// uint16 entries of one chunk's row-segment list: [0] = segment count s,
// [1 .. s] = chunk-relative first box of each segment, [s + 1] = boxes in the chunk
// (padded so that every list starts on a 16-byte boundary).
constexpr uint32_t kSegStride = kChunk + 8;

// Scratch of the order + pack kernels (context memory, or the static array of
// fa_pack_noalloc).
struct PackScratch {
  DevCounters* ctr;
  const uint32_t* count;        // device box count
  uint32_t max_boxes;
  uint32_t max_tiles;           // ceil(max_boxes / 1024)
  uint32_t* ord_counts;         // [max_tiles][kMaxH]
  uint32_t* ord_rank;           // [max_boxes]
  uint32_t* ord_total;          // [kMaxH], zero between calls
  uint32_t* order;              // [max_boxes] when the caller passes none
  uint32_t max_chunks;          // ceil(max_boxes / kChunk)
  uint2* fs;                    // [max_chunks * kChunk] footprints (fa, fb) in box order
  uint2* rec8;                  // [kMaxScales][max_chunks * kChunk] push records
  uint16_t* segs;               // [kMaxScales][max_chunks][kSegStride] row segments per chunk
  unsigned long long* scan_state;  // [kMaxScales][max_chunks] look-back state of the width scan
  uint32_t* m;                  // [kMaxScales] largest overflow
  uint2* xy;                    // [kMaxScales][max_boxes]
  PackCand* cand;               // [kMaxScales]
};

}  // namespace fa

constexpr int kMaxProf = 64;

struct fa_ctx {
  fa_config cfg;
  int device;
  uint64_t launches;
  uint32_t front_blocks;  // raster front-end blocks of the last visibility pass
  // per-kernel event trace of the last public call (fa_profile_enable)
  int prof_on;
  int prof_n;
  cudaEvent_t prof_ev[kMaxProf + 1];
  const char* prof_name[kMaxProf];
  // scratch
  fa::DevCounters* ctr;
  uint32_t* zbuf;        // [max_w * max_h]
  uint32_t* zmax;        // [ceil(max_w / 16) * ceil(max_h / 16)] largest depth key per 16x16 tile
  uint32_t* tile_flag;   // [ceil(max_tris / 1024)] tile has a visible triangle (this frame)
  uint32_t* tile_list;   // [ceil(max_tris / 1024)] those tiles, in the order the marking found them
  fa::BigTri* queue;     // [queue_cap]
  uint32_t queue_cap;
  uint32_t* tile_owner;  // [tile_cap] queue record of each 16x16 tile
  uint32_t tile_cap;
  void* cand;            // [cand_cap] 48-byte records of small sub-triangles
  uint32_t cand_cap;
  uint32_t* surv;        // [surv_cap] raster survivors (per-block regions)
  uint32_t* surv_count;  // [608] survivors of each raster front block
  uint32_t surv_cap;
  void* surv_clip;       // [max_tris][3] float4 clip coordinates of the survivors
  uint32_t* clip;        // [surv_cap] triangles to clip, a region per raster front block
  uint32_t* clip_count;  // [kMaxFrontBlocks] their count per region
  int32_t* label;        // [max_tris + max_verts]
  uint2* wordroots;      // [ceil(max_tris / 32)] per VT word: root bits, roots before it in its block
  uint32_t* blockcnt;    // [n_blocks + 1]
  uint2* xedge;          // [n_blocks][3072] cross-tile edges of the local union-find
  uint32_t* xcnt;        // [n_blocks] their counts
  uint32_t* viscnt;      // [n_blocks + 1] visible triangles per 1024-triangle block, then their starts
  uint2* vis;            // [max_tris] (triangle, chart) of the visible triangles, triangle order
  uint32_t* box_enc;     // [max_charts * 4] ordered-int chart boxes
  uint32_t* box_full;    // [max_charts]
  fa::PackScratch pack;  // order + pack scratch (count filled per call)
  int pack_smem_set;
  // limits of the device-side waits of later launches (fa_set_wait_limits)
  uint32_t loop_cap;
  unsigned long long wait_ns;
  uint32_t mid_max_pix;  // fa_set_raster_schedule
  uint32_t raster_flags;
  uint32_t uf_threads;    // fa_set_chart_pack_schedule: threads per tile of the local union-find
  uint32_t push_threads;  // threads of each candidate's push CTA
  // schedule state of the persistent frame kernel (FA_FRAME_PERSISTENT): work-item
  // counter, exit counter, abort flag and one completion counter per stage group;
  // zero between launches
  uint32_t* psched;
};

// A batch: lanes (contexts of one configuration), each with its own stream.
struct fa_batch {
  fa_config cfg;
  int device = 0;
  uint32_t active = 1;  // lanes in use
  uint32_t policy = FA_BATCH_ROUND_ROBIN;
  std::vector<fa_ctx*> ctx;
  std::vector<cudaStream_t> stream;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};

struct fa_mesh {
  fa_ctx* ctx;
  const float* pos;      // caller-owned [V][3]
  const uint32_t* idx;   // caller-owned [T][3]
  uint32_t V, T;
  int32_t* adj;          // [T][3]: neighbour across edge j (v_j, v_j+1), -1 boundary,
                         // -2 - e for non-manifold edge e
  uint32_t n_nm;         // non-manifold edges
  uint32_t* nm_off;      // [n_nm + 1]
  uint32_t* nm_list;     // incident triangles of the non-manifold edges
};

namespace fa {

// ----------------------------------------------------------------- helpers

struct Mat4 {
  float m[16];
};

// The view-projection matrix read on the device (16 floats, row-major), for frames
// whose camera is set in device memory when the kernels run.
__device__ __forceinline__ Mat4 load_mat(const float* __restrict__ p) {
  Mat4 M;
#pragma unroll
  for (int i = 0; i < 16; ++i) M.m[i] = __ldg(p + i);
  return M;
}

#define FA_CUDA_TRY(expr)                         \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return FA_E_CUDA;      \
  } while (0)

// Pinned fp32 evaluation of clip = M . [p, 1]: ((m0 x + m1 y) + m2 z) + m3 per row,
// one rounding per operation (no contraction).
__device__ __forceinline__ float4 transform(const Mat4& M, float x, float y, float z) {
  float r[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float acc = __fmul_rn(M.m[4 * i + 0], x);
    acc = __fadd_rn(acc, __fmul_rn(M.m[4 * i + 1], y));
    acc = __fadd_rn(acc, __fmul_rn(M.m[4 * i + 2], z));
    acc = __fadd_rn(acc, M.m[4 * i + 3]);
    r[i] = acc;
  }
  return make_float4(r[0], r[1], r[2], r[3]);
}

__device__ __forceinline__ float4 load_clip(const Mat4& M, const float* __restrict__ pos, uint32_t v) {
  const float* p = pos + 3 * (size_t)v;
  return transform(M, __ldg(p), __ldg(p + 1), __ldg(p + 2));
}

// int64 -> fp32 with round-to-nearest-even, on the integer and fp32 pipes (the
// hardware 64-bit conversion runs on the fp64 units, which this GPU has few of).
// Exact: the same value as a correctly rounded conversion.
__device__ __forceinline__ float ll2float_rn(long long v) {
  if (v >= -2147483648ll && v <= 2147483647ll) return __int2float_rn((int)v);
  const bool neg = v < 0;
  unsigned long long u = neg ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll(u);
  int shift = 40 - lz;  // bits dropped so that 24 remain (u >= 2^31, so shift > 0)
  unsigned long long mant = u >> shift;
  const unsigned long long rem = u & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (mant & 1ull))) ++mant;
  if (mant == (1ull << 24)) {
    mant >>= 1;
    ++shift;
  }
  const float m = __uint2float_rn((unsigned)mant);              // exact: mant < 2^24
  const float scale = __uint_as_float((unsigned)(127 + shift) << 23);  // 2^shift
  const float r = m * scale;                                     // exact power-of-two scaling
  return neg ? -r : r;
}

// Order-preserving map float -> uint32 (with -0 folded onto +0).
__device__ __forceinline__ uint32_t ordered(float f) {
  uint32_t u = __float_as_uint(f);
  if (u == 0x80000000u) u = 0u;
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(u);
}

// Footprint of chart c from its box accumulators (Sec. 5.2, Sec. 4.1): the box
// (full: [-1, 1]^2), its viewport size scaled by 256 * ratio and rounded up to 1/256
// texel, rotated to stand tall.  Written to bbox / fa / fb / rot; returns fb.
struct FootArgs {
  const uint32_t* box_enc;
  const uint32_t* box_full;
  float hx, hy, s256;
  float* bbox;
  uint32_t* fa;
  uint32_t* fb;
  uint8_t* rot;
};

__device__ __forceinline__ uint32_t chart_footprint(const FootArgs& f, uint32_t c) {
  float x0, y0, x1, y1;
  if (__ldcg(f.box_full + c)) {
    x0 = y0 = -1.0f;
    x1 = y1 = 1.0f;
  } else {
    const uint4 e = __ldcg(reinterpret_cast<const uint4*>(f.box_enc) + c);
    x0 = unordered(e.x);
    y0 = unordered(e.y);
    x1 = unordered(e.z);
    y1 = unordered(e.w);
  }
  reinterpret_cast<float4*>(f.bbox)[c] = make_float4(x0, y0, x1, y1);
  const float wpx = __fmul_rn(__fsub_rn(x1, x0), f.hx);
  const float hpx = __fmul_rn(__fsub_rn(y1, y0), f.hy);
  const uint32_t fw = __float2uint_rz(ceilf(__fmul_rn(f.s256, wpx)));
  const uint32_t fh = __float2uint_rz(ceilf(__fmul_rn(f.s256, hpx)));
  const bool r = fw > fh;
  f.rot[c] = r ? 1 : 0;
  f.fa[c] = r ? fh : fw;
  f.fb[c] = r ? fw : fh;
  return r ? fw : fh;
}

__device__ __forceinline__ void set_status(DevCounters* c, int32_t s) {
  atomicCAS(&c->status, 0, s);
}

__device__ __forceinline__ bool vt_bit(const uint32_t* vt, uint32_t t) {
  return (__ldcg(vt + (t >> 5)) >> (t & 31)) & 1u;
}

inline unsigned grid_for(uint64_t n, unsigned block, unsigned cap = 152u * 16u) {
  uint64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// Event record that stays a real (timeable) record when the stream is being
// captured into a CUDA graph.
inline void record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}
// Called right before every kernel launch: counts the launch and, when tracing is
// on, records the event that opens this kernel's slot.
inline void mark(fa_ctx* ctx, const char* name, cudaStream_t s) {
  ctx->launches++;
  if (ctx->prof_on && ctx->prof_n < kMaxProf) {
    record_event(ctx->prof_ev[ctx->prof_n], s);
    ctx->prof_name[ctx->prof_n] = name;
    ctx->prof_n++;
  }
}
// Start / close the trace of one public call.
inline void trace_begin(fa_ctx* ctx) { ctx->prof_n = 0; }
inline void trace_end(fa_ctx* ctx, cudaStream_t s) {
  if (ctx->prof_on && ctx->prof_n > 0) record_event(ctx->prof_ev[ctx->prof_n], s);
}

// Programmatic dependent launch: every per-frame kernel is launched with
// programmatic stream serialization.  Each kernel's first statement lets the next
// kernel be scheduled as soon as all of this kernel's blocks have started (so the
// next kernel's blocks take the resources this one leaves and are resident when it
// ends; none of this kernel's blocks can be kept out by them), then waits until
// the previous grid has completed and its writes are visible.  Both are no-ops
// without the attribute.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

bool pdl_enabled();  // FA_PDL=0 in the environment turns it off

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ----------------------------------------------------------------- launchers
// Each returns FA_OK or FA_E_CUDA (launch error) and bumps ctx->launches.

fa_status launch_visibility(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W,
                            uint32_t H, uint32_t* vt, bool reset_status, cudaStream_t s,
                            const float* Mdev = nullptr, bool conservative = false,
                            int32_t* tri_chart_init = nullptr);
// tile_list: the marking pass of the same frame listed the tiles with a visible
// triangle (and the raster front end zeroed the per-tile counts and set tri_chart
// to -1), so the union-find and chart-id passes visit only those
fa_status launch_chartify(fa_ctx* ctx, const fa_mesh* mesh, const uint32_t* vt, uint32_t mode,
                          int32_t* tri_chart, int32_t* vert_chart, const fa_charts* ch,
                          cudaStream_t s, bool tile_list = false, bool tri_chart_cleared = false);
// launch_parameterize and launch_uv read the context's visible-triangle list (built
// by chartify, or by launch_vis_list).
fa_status launch_parameterize(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W,
                              uint32_t H, float ratio, const int32_t* tri_chart,
                              const fa_charts* ch, bool reset_boxes, uint32_t flags, uint32_t* partial,
                              cudaStream_t s, const float* Mdev = nullptr, bool footprint = true);
// Footprint inputs / outputs of the charts of ch (fused into the first order kernel
// on the frame path).
FootArgs foot_args(fa_ctx* ctx, uint32_t W, uint32_t H, float ratio, const fa_charts* ch);
fa_status launch_pack(fa_ctx* ctx, const uint32_t* fa_, const uint32_t* fb, const uint32_t* count,
                      uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode,
                      uint32_t* order, fa_placement* place, fa_pack_result* res, cudaStream_t s,
                      uint32_t lowres_log2 = 0, const FootArgs* foot = nullptr, bool write_place = true);
fa_status launch_uv(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W, uint32_t H,
                    float ratio, const int32_t* tri_chart, const fa_charts* ch,
                    const fa_placement* place, const fa_pack_result* res, uint32_t atlas_log2,
                    uint32_t n_scales, float* uv, float* affine, cudaStream_t s,
                    const float* Mdev = nullptr, bool from_candidates = false);
fa_status build_adjacency(fa_ctx* ctx, fa_mesh* mesh, cudaStream_t s);
// The visible-triangle list from a caller's tri_chart (standalone box / UV calls).
fa_status launch_vis_list(fa_ctx* ctx, const fa_mesh* mesh, const int32_t* tri_chart, cudaStream_t s);
// One whole frame on ctx: host-side checks, then the launch sequence.
fa_status check_frame(const fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p, const float* d_view_proj,
                      const fa_frame_out* o);
fa_status enqueue_frame(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p, const float* d_view_proj,
                        const fa_frame_out* o, cudaStream_t s);
fa_status launch_pack_kernels(fa_ctx* ctx, const PackScratch& p, const uint32_t* fa_, const uint32_t* fb,
                              uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode, uint32_t min_box,
                              uint32_t gutter, uint32_t* order, fa_placement* place, fa_pack_result* res,
                              cudaStream_t s, uint32_t lowres_log2, const FootArgs* foot, bool write_place);
fa_status pack_set_smem_limit();
// fa_atlas_frame with FA_FRAME_PERSISTENT: the checked frame as one launch of the
// persistent frame kernel (persist.cu).
fa_status enqueue_frame_persistent(fa_ctx* ctx, const fa_mesh* mesh, const fa_frame_params* p,
                                   const float* d_view_proj, const fa_frame_out* o, cudaStream_t s);

}  // namespace fa
