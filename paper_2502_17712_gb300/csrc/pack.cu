// Box order and packing (Sec. 4.1-4.3).
//
// Order: stable counting sort of the boxes by integer height
//   h0 = clamp(ceil(fb / 256), 1, 8192), tallest first, ties by box index (the
//   boxes arrive numbered by ascending root, so this is the paper's
//   (height, lowest triangle id) order).  Three kernels: per 1024-box tile a
//   bitonic sort of (bin, index) keys gives stable in-tile ranks and a per-bin
//   count row; one block scans the counts over tiles and bins; a scatter writes the
//   order.  This replaces the paper's cuckoo-hash bucketing with the same result
//   contract (deterministic, identical for identical frames).
//
// Pack: one CTA per candidate scale k / n (Sec. 4.2).  Phase 1 computes the scaled
//   integer boxes, the exclusive prefix sum P of the widths (block scan, 64-bit),
//   rows P >> log2(omega), in-row offsets and the largest overflow m (Sec. 4.3);
//   Omega = omega + m.  Phase 2 pushes the rows up against a frontline kept in
//   shared memory: a row's texels are processed in parallel, each thread finding
//   its box by binary search over the row's staged offsets, a shared-memory
//   atomicMax giving each box its resting height, then the frontline is
//   overwritten with the box tops.  The last CTA to finish selects the candidate
//   and writes the placements.
#include "fa_internal.cuh"

namespace fa {
namespace {

constexpr int kPackThreads = 1024;
constexpr int kStage = 2048;  // boxes staged per row chunk

__device__ __forceinline__ uint32_t height_bin(uint32_t fb) {
  uint32_t h = (uint32_t)(((uint64_t)fb + 255u) >> 8);
  h = h < 1u ? 1u : (h > kMaxH ? kMaxH : h);
  return kMaxH - h;  // ascending bin = descending height
}

// ------------------------------------------------------------------ order

__global__ void __launch_bounds__(kOrderTile) k_order_tile(const uint32_t* __restrict__ fb,
                                                           const uint32_t* count, uint32_t max_charts,
                                                           uint32_t* counts, uint32_t* rank,
                                                           DevCounters* ctr) {
  __shared__ uint32_t key[kOrderTile];
  __shared__ uint32_t cnt[kMaxH];
  __shared__ uint16_t first[kMaxH];
  if (__ldcg(&ctr->status) != 0) return;
  const uint32_t C = __ldcg(count);
  if (C > max_charts) return;
  const uint32_t ntiles = (C + kOrderTile - 1) / kOrderTile;
  if (blockIdx.x >= ntiles) return;
  const uint32_t tid = threadIdx.x;
  const uint32_t i = blockIdx.x * kOrderTile + tid;
  key[tid] = i < C ? (height_bin(__ldg(fb + i)) << 10) | tid : 0xFFFFFFFFu;
  for (uint32_t b = tid; b < kMaxH; b += kOrderTile) cnt[b] = 0;
  __syncthreads();
  // bitonic sort, ascending
  for (uint32_t size = 2; size <= kOrderTile; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      const uint32_t j = tid ^ stride;
      if (j > tid) {
        const uint32_t a = key[tid], b = key[j];
        const bool up = (tid & size) == 0;
        if ((a > b) == up) {
          key[tid] = b;
          key[j] = a;
        }
      }
      __syncthreads();
    }
  }
  const uint32_t k = key[tid];
  const bool valid = k != 0xFFFFFFFFu;
  const uint32_t bin = k >> 10;
  if (valid && (tid == 0 || (key[tid - 1] >> 10) != bin)) first[bin] = (uint16_t)tid;
  __syncthreads();
  if (valid) {
    const uint32_t r = tid - first[bin];
    rank[blockIdx.x * kOrderTile + (k & 1023u)] = r;
    if (tid == kOrderTile - 1 || (key[tid + 1] >> 10) != bin) cnt[bin] = r + 1;
  }
  __syncthreads();
  uint32_t* row = counts + (size_t)blockIdx.x * kMaxH;
  for (uint32_t b = tid; b < kMaxH; b += kOrderTile) row[b] = cnt[b];
}

// counts[t][b] -> exclusive prefix over tiles; binstart[b] = exclusive prefix over bins.
__global__ void __launch_bounds__(1024) k_order_scan(const uint32_t* count, uint32_t max_charts,
                                                     uint32_t* counts, uint32_t* binstart,
                                                     DevCounters* ctr) {
  __shared__ uint32_t wt[32];
  if (__ldcg(&ctr->status) != 0) return;
  const uint32_t C = __ldcg(count);
  if (C > max_charts) return;
  const uint32_t ntiles = (C + kOrderTile - 1) / kOrderTile;
  constexpr uint32_t kPer = kMaxH / 1024;
  uint32_t tot[kPer];
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    const uint32_t b = threadIdx.x * kPer + j;
    uint32_t run = 0;
    for (uint32_t t = 0; t < ntiles; ++t) {
      uint32_t* p = counts + (size_t)t * kMaxH + b;
      const uint32_t c = *p;
      *p = run;
      run += c;
    }
    tot[j] = run;
    sum += run;
  }
  // block exclusive scan of the per-thread sums
  uint32_t x = sum;
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) wt[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = wt[threadIdx.x];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (threadIdx.x >= (unsigned)o) v += y;
    }
    wt[threadIdx.x] = v;
  }
  __syncthreads();
  uint32_t run = (threadIdx.x >= 32 ? wt[(threadIdx.x >> 5) - 1] : 0) + x - sum;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    binstart[threadIdx.x * kPer + j] = run;
    run += tot[j];
  }
}

__global__ void __launch_bounds__(kOrderTile) k_order_scatter(const uint32_t* __restrict__ fb,
                                                              const uint32_t* count, uint32_t max_charts,
                                                              const uint32_t* counts, const uint32_t* rank,
                                                              const uint32_t* binstart, uint32_t* order,
                                                              DevCounters* ctr) {
  if (__ldcg(&ctr->status) != 0) return;
  const uint32_t C = __ldcg(count);
  if (C > max_charts) return;
  const uint32_t i = blockIdx.x * kOrderTile + threadIdx.x;
  if (i >= C) return;
  const uint32_t bin = height_bin(__ldg(fb + i));
  const uint32_t pos = __ldcg(binstart + bin) + __ldcg(counts + (size_t)blockIdx.x * kMaxH + bin) + __ldcg(rank + i);
  if (pos < C) order[pos] = i;
}

// ------------------------------------------------------------------ pack

struct PackArgs {
  const uint32_t* fa;
  const uint32_t* fb;
  const uint32_t* count;
  const uint32_t* order;
  uint32_t max_charts;
  uint32_t atlas_log2;
  uint32_t n_scales;
  uint32_t shift;  // log2(256 * n_scales)
  uint32_t min_box;
  uint32_t gutter;
  uint32_t select_mode;
  uint32_t front_cap;
  unsigned long long* P;  // [n_scales][max_charts]
  uint2* wh;
  uint2* xy;
  uint32_t* rows;
  PackCand* cand;
  DevCounters* ctr;
  fa_placement* place;
  fa_pack_result* res;
};

// Block-wide inclusive scan (1024 threads) of a 64-bit value; returns the
// inclusive prefix and writes the block total to *total.
template <typename T>
__device__ __forceinline__ T block_scan_incl(T v, T* warp_sums, T* total) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T s = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= (unsigned)o) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  const T r = x + (wid ? warp_sums[wid - 1] : (T)0);
  *total = warp_sums[31];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kPackThreads) k_pack(PackArgs a) {
  extern __shared__ uint32_t smem[];
  uint32_t* F = smem;                      // [front_cap]
  uint32_t* s_xr = F + a.front_cap;        // [kStage]
  uint32_t* s_w = s_xr + kStage;
  uint32_t* s_h = s_w + kStage;
  uint32_t* s_y = s_h + kStage;
  __shared__ unsigned long long ws64[32];
  __shared__ uint32_t ws32[32];
  __shared__ uint32_t s_flag;
  __shared__ uint32_t s_last;

  const uint32_t k = blockIdx.x + 1;
  const uint32_t tid = threadIdx.x;
  const int32_t st0 = __ldcg(&a.ctr->status);
  if (st0 != 0) {
    if (blockIdx.x == 0 && tid == 0) {
      a.res->k = 0;
      a.res->omega = 0;
      a.res->height = 0;
      a.res->status = st0;
      a.res->count = 0;
    }
    return;
  }
  const uint32_t C = __ldcg(a.count);
  const uint32_t om = 1u << a.atlas_log2;
  unsigned long long* P = a.P + (size_t)blockIdx.x * a.max_charts;
  uint2* wh = a.wh + (size_t)blockIdx.x * a.max_charts;
  uint2* xy = a.xy + (size_t)blockIdx.x * a.max_charts;
  uint32_t* rows = a.rows + (size_t)blockIdx.x * a.max_charts;
  int32_t status = FA_OK;
  uint32_t Om = om, H = 0, ok = 0;
  if (C > a.max_charts) {
    status = FA_E_CAPACITY;
  } else {
    // ---- phase 1: scaled boxes, prefix sum, rows, overflow
    unsigned long long carry = 0;
    uint32_t gcarry = 0;
    unsigned long long prev_row = ~0ull;
    uint32_t m = 0;
    const uint32_t g2 = 2u * a.gutter;
    for (uint32_t base = 0; base < C; base += kPackThreads) {
      const uint32_t i = base + tid;
      uint32_t w = 0, h = 0;
      if (i < C) {
        const uint32_t b = __ldg(a.order + i);
        const unsigned long long d = (1ull << a.shift) - 1ull;
        uint32_t sw = (uint32_t)(((unsigned long long)k * __ldg(a.fa + b) + d) >> a.shift);
        uint32_t sh = (uint32_t)(((unsigned long long)k * __ldg(a.fb + b) + d) >> a.shift);
        w = (sw > a.min_box ? sw : a.min_box) + g2;
        h = (sh > a.min_box ? sh : a.min_box) + g2;
      }
      unsigned long long tot;
      const unsigned long long incl = block_scan_incl<unsigned long long>(w, ws64, &tot);
      const unsigned long long Pi = carry + incl - w;
      const unsigned long long row = Pi >> a.atlas_log2;
      // row of the previous box (across the chunk boundary via prev_row)
      unsigned long long rprev = __shfl_up_sync(0xFFFFFFFFu, row, 1);
      if ((tid & 31) == 0) rprev = 0;  // fixed below
      __shared__ unsigned long long s_lastrow[32];
      if ((tid & 31) == 31) s_lastrow[tid >> 5] = row;
      __syncthreads();
      if ((tid & 31) == 0) rprev = (tid == 0) ? prev_row : s_lastrow[(tid >> 5) - 1];
      const uint32_t start = (i < C && row != rprev) ? 1u : 0u;
      uint32_t gtot;
      const uint32_t gincl = block_scan_incl<uint32_t>(start, ws32, &gtot);
      if (i < C) {
        const uint32_t xr = (uint32_t)(Pi & (om - 1));
        if (xr + w > om) m = max(m, xr + w - om);
        P[i] = Pi;
        wh[i] = make_uint2(w, h);
        if (start) rows[gcarry + gincl - 1] = i;
      }
      carry += tot;
      gcarry += gtot;
      __syncthreads();
      const uint32_t last = min(C - base, (uint32_t)kPackThreads) - 1;
      if (tid == last) s_lastrow[0] = row;
      __syncthreads();
      prev_row = s_lastrow[0];
      __syncthreads();
    }
    // ---- overflow -> Omega
    m = __reduce_max_sync(0xFFFFFFFFu, m);
    if ((tid & 31) == 0) ws32[tid >> 5] = m;
    __syncthreads();
    if (tid < 32) {
      uint32_t v = __reduce_max_sync(0xFFFFFFFFu, ws32[tid]);
      if (tid == 0) ws32[0] = v;
    }
    __syncthreads();
    m = ws32[0];
    __syncthreads();
    Om = om + m;
    const uint32_t G = gcarry;
    if (Om > a.front_cap) {
      status = FA_E_CAPACITY;
    } else {
      // ---- phase 2: push rows up against the frontline
      for (uint32_t x = tid; x < Om; x += kPackThreads) F[x] = 0;
      if (tid == 0) s_flag = 0;
      uint32_t Hloc = 0;
      __syncthreads();
      for (uint32_t g = 0; g < G && !s_flag; ++g) {
        const uint32_t s0 = __ldcg(rows + g);
        const uint32_t e0 = (g + 1 < G) ? __ldcg(rows + g + 1) : C;
        const unsigned long long q = __ldcg(P + s0) >> a.atlas_log2;
        const unsigned long long qbase = q << a.atlas_log2;
        const bool l2r = (q % 3ull) == 0ull;
        for (uint32_t cs = s0; cs < e0; cs += kStage) {
          const uint32_t n = min(e0 - cs, (uint32_t)kStage);
          for (uint32_t j = tid; j < n; j += kPackThreads) {
            const uint2 v = __ldcg(wh + cs + j);
            s_xr[j] = (uint32_t)(__ldcg(P + cs + j) - qbase);
            s_w[j] = v.x;
            s_h[j] = v.y;
            s_y[j] = 0;
          }
          __syncthreads();
          const uint32_t o0 = s_xr[0];
          const uint32_t L = s_xr[n - 1] + s_w[n - 1] - o0;
          // pass A: resting height of each box = max frontline under it
          for (uint32_t u = tid; u < L; u += kPackThreads) {
            const uint32_t o = o0 + u;
            uint32_t lo = 0, hi = n;  // last j with s_xr[j] <= o
            while (hi - lo > 1) {
              const uint32_t mid = (lo + hi) >> 1;
              if (s_xr[mid] <= o) lo = mid;
              else hi = mid;
            }
            const uint32_t x = l2r ? o : Om - 1 - o;
            atomicMax(s_y + lo, F[x]);
          }
          __syncthreads();
          // pass B: frontline := top of the box; record the placement
          for (uint32_t u = tid; u < L; u += kPackThreads) {
            const uint32_t o = o0 + u;
            uint32_t lo = 0, hi = n;
            while (hi - lo > 1) {
              const uint32_t mid = (lo + hi) >> 1;
              if (s_xr[mid] <= o) lo = mid;
              else hi = mid;
            }
            const uint32_t x = l2r ? o : Om - 1 - o;
            F[x] = s_y[lo] + s_h[lo];
          }
          for (uint32_t j = tid; j < n; j += kPackThreads) {
            const uint32_t y = s_y[j], top = y + s_h[j];
            const uint32_t x = l2r ? s_xr[j] : Om - s_xr[j] - s_w[j];
            xy[cs + j] = make_uint2(x, y);
            Hloc = max(Hloc, top);
            if (top > Om) s_flag = 1;
          }
          __syncthreads();
        }
      }
      Hloc = __reduce_max_sync(0xFFFFFFFFu, Hloc);
      if ((tid & 31) == 0) ws32[tid >> 5] = Hloc;
      __syncthreads();
      if (tid < 32) {
        uint32_t v = __reduce_max_sync(0xFFFFFFFFu, ws32[tid]);
        if (tid == 0) ws32[0] = v;
      }
      __syncthreads();
      H = ws32[0];
      ok = (!s_flag && H <= Om) ? 1u : 0u;
    }
  }
  // ---- publish this candidate; the last CTA selects
  if (tid == 0) {
    a.cand[blockIdx.x] = PackCand{ok, Om, H, status};
    __threadfence();
    const uint32_t done = atomicAdd(&a.ctr->pack_done, 1u);
    s_last = (done == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ uint32_t s_best;
  __shared__ int32_t s_status;
  if (tid == 0) {
    uint32_t best = 0;
    int32_t pst = FA_OK;
    uint32_t bestOm = 0;
    for (uint32_t kk = 1; kk <= gridDim.x; ++kk) {
      const uint4 cv = __ldcg(reinterpret_cast<const uint4*>(a.cand) + (kk - 1));
      const PackCand c{cv.x, cv.y, cv.z, (int32_t)cv.w};
      if (c.status != FA_OK) pst = c.status;
      if (!c.ok) continue;
      if (best == 0 || a.select_mode == FA_SELECT_LARGEST_K ||
          (unsigned long long)kk * bestOm >= (unsigned long long)best * c.omega) {
        best = kk;
        bestOm = c.omega;
      }
    }
    if (pst == FA_OK && best == 0) pst = FA_E_PACK_FAILED;
    s_best = pst == FA_OK ? best : 0;
    s_status = pst;
    fa_pack_result r;
    r.count = C;
    r.status = pst;
    if (pst == FA_OK) {
      const uint4 cv = __ldcg(reinterpret_cast<const uint4*>(a.cand) + (best - 1));
      const PackCand c{cv.x, cv.y, cv.z, (int32_t)cv.w};
      r.k = best;
      r.omega = c.omega;
      r.height = c.height;
    } else {
      r.k = 0;
      r.omega = 0;
      r.height = 0;
    }
    *a.res = r;
    a.ctr->pack_done = 0;
  }
  __syncthreads();
  if (s_status != FA_OK) return;
  const uint32_t kb = s_best - 1;
  const uint2* bxy = a.xy + (size_t)kb * a.max_charts;
  const uint2* bwh = a.wh + (size_t)kb * a.max_charts;
  for (uint32_t i = tid; i < C; i += kPackThreads) {
    const uint32_t b = __ldcg(a.order + i);
    const uint2 p = __ldcg(bxy + i), s = __ldcg(bwh + i);
    a.place[b] = fa_placement{(int32_t)p.x, (int32_t)p.y, (int32_t)s.x, (int32_t)s.y};
  }
}

}  // namespace

fa_status launch_pack(fa_ctx* ctx, const uint32_t* fa_, const uint32_t* fb, const uint32_t* count,
                      uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode, uint32_t* order,
                      fa_placement* place, fa_pack_result* res, cudaStream_t s) {
  const uint32_t maxc = ctx->cfg.max_charts;
  const uint32_t ntiles = (maxc + kOrderTile - 1) / kOrderTile;
  uint32_t* ord = order ? order : ctx->order;
  mark(ctx, "k_order_tile", s);
  k_order_tile<<<ntiles, kOrderTile, 0, s>>>(fb, count, maxc, ctx->ord_counts, ctx->ord_rank, ctx->ctr);
  mark(ctx, "k_order_scan", s);
  k_order_scan<<<1, 1024, 0, s>>>(count, maxc, ctx->ord_counts, ctx->ord_binstart, ctx->ctr);
  mark(ctx, "k_order_scatter", s);
  k_order_scatter<<<ntiles, kOrderTile, 0, s>>>(fb, count, maxc, ctx->ord_counts, ctx->ord_rank,
                                                ctx->ord_binstart, ord, ctx->ctr);
  PackArgs a;
  a.fa = fa_;
  a.fb = fb;
  a.count = count;
  a.order = ord;
  a.max_charts = maxc;
  a.atlas_log2 = atlas_log2;
  a.n_scales = n_scales;
  uint32_t sh = 8;
  while ((1u << (sh - 8)) < n_scales) ++sh;
  a.shift = sh;
  a.min_box = ctx->cfg.min_box;
  a.gutter = ctx->cfg.gutter;
  a.select_mode = select_mode;
  const uint32_t om = 1u << atlas_log2;
  a.front_cap = (8u * om < kFrontCap) ? 8u * om : kFrontCap;
  a.P = ctx->cand_P;
  a.wh = ctx->cand_wh;
  a.xy = ctx->cand_xy;
  a.rows = ctx->cand_rows;
  a.cand = ctx->cand;
  a.ctr = ctx->ctr;
  a.place = place;
  a.res = res;
  const size_t smem = (size_t)a.front_cap * 4 + (size_t)kStage * 16;
  static bool attr_set = false;
  if (!attr_set) {
    FA_CUDA_TRY(cudaFuncSetAttribute(k_pack, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((size_t)kFrontCap * 4 + (size_t)kStage * 16)));
    attr_set = true;
  }
  mark(ctx, "k_pack", s);
  k_pack<<<n_scales, kPackThreads, smem, s>>>(a);
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
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
// synchronization.  The array (about 7.2 MiB, for up to 4096 boxes) stays resident
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
constexpr size_t kOffCounts = align256(kOffCand + sizeof(PackCand) * kMaxScales);
constexpr size_t kOffRank = align256(kOffCounts + sizeof(uint32_t) * kMaxH * kNoAllocTiles);
constexpr size_t kOffBinstart = align256(kOffRank + sizeof(uint32_t) * kNoAllocMaxBoxes);
constexpr size_t kOffOrder = align256(kOffBinstart + sizeof(uint32_t) * kMaxH);
constexpr size_t kOffP = align256(kOffOrder + sizeof(uint32_t) * kNoAllocMaxBoxes);
constexpr size_t kOffWH = align256(kOffP + sizeof(unsigned long long) * kMaxScales * kNoAllocMaxBoxes);
constexpr size_t kOffXY = align256(kOffWH + sizeof(uint2) * kMaxScales * kNoAllocMaxBoxes);
constexpr size_t kOffRows = align256(kOffXY + sizeof(uint2) * kMaxScales * kNoAllocMaxBoxes);
constexpr size_t kNoAllocBytes = align256(kOffRows + sizeof(uint32_t) * kMaxScales * kNoAllocMaxBoxes);

// The scratch of fa_pack_noalloc.  Host code must not use this name as a device
// address: it is a host-side shadow there; the device address comes from
// cudaGetSymbolAddress in noalloc_scratch() below.
static __device__ __align__(256) unsigned char g_pack_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Once per device, with that device current: the array's device address, and the
// pack kernel's shared-memory limit.
fa_status noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return FA_E_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pack_scratch) != cudaSuccess) {
      cudaGetLastError();
      return FA_E_CUDA;
    }
    if (cudaFuncSetAttribute(k_pack, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)kFrontCap * 4 + (size_t)kStage * 16)) != cudaSuccess) {
      cudaGetLastError();
      return FA_E_CUDA;
    }
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return FA_OK;
}

// Clears what the kernels expect at zero (status word, finished-candidate counter)
// and stores the box count where the kernels read it.
__global__ void k_noalloc_reset(DevCounters* ctr, uint32_t* count, uint32_t n) {
  ctr->status = 0;
  ctr->pack_done = 0;
  *count = n;
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
  DevCounters* ctr = (DevCounters*)(base + kOffCtr);
  uint32_t* count = (uint32_t*)(base + kOffCount);
  uint32_t* counts = (uint32_t*)(base + kOffCounts);
  uint32_t* rank = (uint32_t*)(base + kOffRank);
  uint32_t* binstart = (uint32_t*)(base + kOffBinstart);
  uint32_t* ord = d_order ? d_order : (uint32_t*)(base + kOffOrder);
  k_noalloc_reset<<<1, 1, 0, s>>>(ctr, count, n);
  k_order_tile<<<kNoAllocTiles, kOrderTile, 0, s>>>(d_fb, count, kNoAllocMaxBoxes, counts, rank, ctr);
  k_order_scan<<<1, 1024, 0, s>>>(count, kNoAllocMaxBoxes, counts, binstart, ctr);
  k_order_scatter<<<kNoAllocTiles, kOrderTile, 0, s>>>(d_fb, count, kNoAllocMaxBoxes, counts, rank, binstart,
                                                       ord, ctr);
  PackArgs a;
  a.fa = d_fa;
  a.fb = d_fb;
  a.count = count;
  a.order = ord;
  a.max_charts = kNoAllocMaxBoxes;
  a.atlas_log2 = atlas_log2;
  a.n_scales = n_scales;
  uint32_t sh = 8;
  while ((1u << (sh - 8)) < n_scales) ++sh;
  a.shift = sh;
  a.min_box = min_box;
  a.gutter = gutter;
  a.select_mode = select_mode;
  const uint32_t om = 1u << atlas_log2;
  a.front_cap = (8u * om < kFrontCap) ? 8u * om : kFrontCap;
  a.P = (unsigned long long*)(base + kOffP);
  a.wh = (uint2*)(base + kOffWH);
  a.xy = (uint2*)(base + kOffXY);
  a.rows = (uint32_t*)(base + kOffRows);
  a.cand = (PackCand*)(base + kOffCand);
  a.ctr = ctr;
  a.place = d_place;
  a.res = d_res;
  const size_t smem = (size_t)a.front_cap * 4 + (size_t)kStage * 16;
  k_pack<<<n_scales, kPackThreads, smem, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return FA_E_CUDA;
  return FA_OK;
}
