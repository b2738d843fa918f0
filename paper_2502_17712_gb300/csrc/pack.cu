// Box order and packing (Sec. 4.1-4.3).
//
// Order: stable counting sort of the boxes by integer height
//   h0 = clamp(ceil(fb / 256), 1, 8192), tallest first, ties by box index (the
//   boxes arrive numbered by ascending root, so this is the paper's
//   (height, lowest triangle id) order).  k_order_tile bitonic-sorts the
//   (bin, index) keys of each 1024-box tile, giving stable in-tile ranks, a per-bin
//   count row per tile and global bin totals; k_order_binscan scans the totals;
//   k_order_scatter adds, for each box, the counts of its bin in earlier tiles.
//   This replaces the paper's cuckoo-hash bucketing with the same result contract
//   (deterministic, identical for identical frames).
//
// Pack: candidates k / n, k = 1..n (Sec. 4.2).  The per-box work is spread over
//   (tile, candidate) CTAs: k_pack_boxes computes the scaled integer boxes and
//   tile-local exclusive prefix sums of the widths; k_pack_fix adds the tile's
//   offset (a block reduction over the preceding tile totals), giving P, and
//   reduces the largest overflow m past omega (Sec. 4.3).  Then one CTA per
//   candidate (k_pack_push) pushes the rows up against a frontline in shared
//   memory: boxes are read 4096 at a time into shared-memory x / w / h arrays, the
//   rows inside a chunk are found by a block scan, and each row segment is processed
//   box-parallel (a group of 32 .. 1 threads per box, by the row's box count):
//   resting height = max of the frontline under the box, then the frontline takes
//   the box top, one barrier per segment.  Segments of one row never overlap in x,
//   so a row may span two chunks.  The last CTA to finish selects the candidate;
//   k_pack_place writes the placements with all CTAs.
#include "fa_internal.cuh"

namespace fa {
namespace {

constexpr int kThreads = 1024;

__device__ __forceinline__ uint32_t height_bin(uint32_t fb) {
  uint32_t h = (uint32_t)(((uint64_t)fb + 255u) >> 8);
  h = h < 1u ? 1u : (h > kMaxH ? kMaxH : h);
  return kMaxH - h;  // ascending bin = descending height
}

// Block-wide inclusive scan (1024 threads); writes the block total to *total.
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

template <typename T>
__device__ __forceinline__ T block_max(T v, T* warp_vals) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T y = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = v > y ? v : y;
  }
  if ((threadIdx.x & 31) == 0) warp_vals[threadIdx.x >> 5] = v;
  __syncthreads();
  T r = warp_vals[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = r > warp_vals[w] ? r : warp_vals[w];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ order

__global__ void __launch_bounds__(kOrderTile) k_order_tile(PackScratch p, const uint32_t* __restrict__ fb) {
  pdl_wait();
  __shared__ uint32_t key[kOrderTile];
  __shared__ uint16_t first[kMaxH];
  if (__ldcg(&p.ctr->status) != 0) return;
  const uint32_t C = __ldcg(p.count);
  if (C > p.max_boxes) return;
  const uint32_t ntiles = (C + kOrderTile - 1) / kOrderTile;
  if (blockIdx.x >= ntiles) return;
  const uint32_t tid = threadIdx.x;
  const uint32_t i = blockIdx.x * kOrderTile + tid;
  key[tid] = i < C ? (height_bin(__ldg(fb + i)) << 10) | tid : 0xFFFFFFFFu;
  uint32_t* row = p.ord_counts + (size_t)blockIdx.x * kMaxH;
  for (uint32_t b = tid; b < kMaxH; b += kOrderTile) row[b] = 0;
  __syncthreads();
  for (uint32_t size = 2; size <= kOrderTile; size <<= 1) {  // bitonic sort, ascending
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      const uint32_t j = tid ^ stride;
      if (j > tid) {
        const uint32_t a = key[tid], b = key[j];
        if ((a > b) == ((tid & size) == 0)) {
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
    p.ord_rank[blockIdx.x * kOrderTile + (k & 1023u)] = r;
    if (tid == kOrderTile - 1 || (key[tid + 1] >> 10) != bin) {
      row[bin] = r + 1;
      atomicAdd(p.ord_total + bin, r + 1);
    }
  }
}

// binstart = exclusive scan of the bin totals; the totals are cleared for the next call.
__global__ void __launch_bounds__(1024) k_order_binscan(PackScratch p) {
  pdl_wait();
  __shared__ uint32_t wt[32];
  if (__ldcg(&p.ctr->status) != 0) return;
  constexpr uint32_t kPer = kMaxH / 1024;
  uint4* t4 = reinterpret_cast<uint4*>(p.ord_total) + threadIdx.x * (kPer / 4);
  uint32_t v[kPer];
#pragma unroll
  for (uint32_t j = 0; j < kPer / 4; ++j) {
    const uint4 q = __ldcg(t4 + j);
    v[4 * j] = q.x;
    v[4 * j + 1] = q.y;
    v[4 * j + 2] = q.z;
    v[4 * j + 3] = q.w;
    t4[j] = make_uint4(0, 0, 0, 0);
  }
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) sum += v[j];
  uint32_t tot;
  const uint32_t incl = block_scan_incl<uint32_t>(sum, wt, &tot);
  uint32_t run = incl - sum;
  uint4* b4 = reinterpret_cast<uint4*>(p.ord_binstart) + threadIdx.x * (kPer / 4);
#pragma unroll
  for (uint32_t j = 0; j < kPer / 4; ++j) {
    uint4 q;
    q.x = run; run += v[4 * j];
    q.y = run; run += v[4 * j + 1];
    q.z = run; run += v[4 * j + 2];
    q.w = run; run += v[4 * j + 3];
    b4[j] = q;
  }
}

__global__ void __launch_bounds__(kOrderTile) k_order_scatter(PackScratch p, const uint32_t* __restrict__ fb,
                                                              uint32_t* order) {
  pdl_wait();
  if (__ldcg(&p.ctr->status) != 0) return;
  const uint32_t C = __ldcg(p.count);
  if (C > p.max_boxes) return;
  const uint32_t i = blockIdx.x * kOrderTile + threadIdx.x;
  if (i >= C) return;
  const uint32_t bin = height_bin(__ldg(fb + i));
  uint32_t pos = __ldcg(p.ord_binstart + bin) + __ldcg(p.ord_rank + i);
  uint32_t t = 0;
  for (; t + 4 <= blockIdx.x; t += 4) {
    const uint32_t* c = p.ord_counts + (size_t)t * kMaxH + bin;
    pos += __ldcg(c) + __ldcg(c + kMaxH) + __ldcg(c + 2 * kMaxH) + __ldcg(c + 3 * kMaxH);
  }
  for (; t < blockIdx.x; ++t) pos += __ldcg(p.ord_counts + (size_t)t * kMaxH + bin);
  if (pos < C) order[pos] = i;
}

// ------------------------------------------------------------------ pack

struct PackArgs {
  const uint32_t* fa;
  const uint32_t* fb;
  const uint32_t* order;
  uint32_t atlas_log2;
  uint32_t shift;  // log2(256 * n_scales)
  uint32_t min_box;
  uint32_t gutter;
  uint32_t select_mode;
  uint32_t front_cap;
  fa_placement* place;
  fa_pack_result* res;
};

// Scaled boxes and tile-local exclusive prefix of the widths.  Persistent grid over
// (tile, candidate) work items.
__global__ void __launch_bounds__(kThreads) k_pack_boxes(PackScratch p, PackArgs a, uint32_t n_scales) {
  pdl_wait();
  __shared__ unsigned long long ws[32];
  if (__ldcg(&p.ctr->status) != 0) return;
  const uint32_t C = __ldcg(p.count);
  if (C > p.max_boxes) return;
  if (blockIdx.x == 0 && threadIdx.x < n_scales) p.m[threadIdx.x] = 0;
  const uint32_t ntiles = (C + kThreads - 1) / kThreads;
  const unsigned long long d = (1ull << a.shift) - 1ull;
  for (uint32_t item = blockIdx.x; item < ntiles * n_scales; item += gridDim.x) {
    const uint32_t kidx = item / ntiles, tile = item % ntiles, k = kidx + 1;
    const uint32_t i = tile * kThreads + threadIdx.x;
    uint32_t w = 0, h = 0;
    if (i < C) {
      const uint32_t b = __ldg(a.order + i);
      const uint32_t sw = (uint32_t)(((unsigned long long)k * __ldg(a.fa + b) + d) >> a.shift);
      const uint32_t sh = (uint32_t)(((unsigned long long)k * __ldg(a.fb + b) + d) >> a.shift);
      w = (sw > a.min_box ? sw : a.min_box) + 2u * a.gutter;
      h = (sh > a.min_box ? sh : a.min_box) + 2u * a.gutter;
    }
    unsigned long long tot;
    const unsigned long long incl = block_scan_incl<unsigned long long>(w, ws, &tot);
    BoxRec* rec = p.rec + (size_t)kidx * p.max_boxes;
    if (i < C) rec[i] = BoxRec{incl - w, w, h};
    if (threadIdx.x == 0) p.tile_tot[(size_t)kidx * p.max_tiles + tile] = tot;
  }
}

// Global prefix P (tile offset + local) and the largest overflow past omega.
__global__ void __launch_bounds__(kThreads) k_pack_fix(PackScratch p, PackArgs a, uint32_t n_scales) {
  pdl_wait();
  __shared__ unsigned long long ws[32];
  __shared__ uint32_t wm[32];
  if (__ldcg(&p.ctr->status) != 0) return;
  const uint32_t C = __ldcg(p.count);
  if (C > p.max_boxes) return;
  const uint32_t ntiles = (C + kThreads - 1) / kThreads;
  const uint32_t om = 1u << a.atlas_log2;
  for (uint32_t item = blockIdx.x; item < ntiles * n_scales; item += gridDim.x) {
    const uint32_t kidx = item / ntiles, tile = item % ntiles;
    const unsigned long long* tt = p.tile_tot + (size_t)kidx * p.max_tiles;
    unsigned long long off = 0;
    for (uint32_t t = threadIdx.x; t < tile; t += kThreads) off += __ldcg(tt + t);
    unsigned long long total;
    block_scan_incl<unsigned long long>(off, ws, &total);
    const uint32_t i = tile * kThreads + threadIdx.x;
    uint32_t m = 0;
    if (i < C) {
      BoxRec* r = p.rec + (size_t)kidx * p.max_boxes + i;
      BoxRec v = *r;
      v.P += total;
      r->P = v.P;
      const uint32_t xr = (uint32_t)(v.P & (om - 1));
      if (xr + v.w > om) m = xr + v.w - om;
    }
    m = block_max<uint32_t>(m, wm);
    if (threadIdx.x == 0 && m) atomicMax(p.m + kidx, m);
  }
}

// Row push of one candidate per CTA, then the last CTA selects.
constexpr int kPushThreads = 1024;
constexpr int kChunk = 4096;                        // boxes per chunk
constexpr int kPerThread = kChunk / kPushThreads;   // consecutive boxes per thread

__global__ void __launch_bounds__(kPushThreads) k_pack_push(PackScratch p, PackArgs a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* s_x = reinterpret_cast<uint32_t*>(smem_raw);  // [kChunk] box x in its row's direction
  uint32_t* s_w = s_x + kChunk;                            // [kChunk]
  uint32_t* s_h = s_w + kChunk;                            // [kChunk]
  uint32_t* s_seg = s_h + kChunk;                          // [kChunk + 1] first box of each segment
  uint32_t* F = s_seg + kChunk + 4;                        // [front_cap]
  __shared__ uint32_t ws32[32];
  __shared__ uint32_t s_flag, s_nseg, s_last;

  const uint32_t kidx = blockIdx.x;
  const uint32_t tid = threadIdx.x;
  const int32_t st0 = __ldcg(&p.ctr->status);
  if (st0 != 0) {
    if (kidx == 0 && tid == 0) *a.res = fa_pack_result{0, 0, 0, st0, 0};
    return;
  }
  const uint32_t C = __ldcg(p.count);
  const uint32_t om = 1u << a.atlas_log2;
  int32_t status = FA_OK;
  uint32_t Om = om, H = 0, ok = 0;
  if (C > p.max_boxes) {
    status = FA_E_CAPACITY;
  } else {
    Om = om + __ldcg(p.m + kidx);
    if (Om > a.front_cap) {
      status = FA_E_CAPACITY;
    } else {
      const BoxRec* rec = p.rec + (size_t)kidx * p.max_boxes;
      uint2* xy = p.xy + (size_t)kidx * p.max_boxes;
      for (uint32_t x = tid; x < Om; x += kPushThreads) F[x] = 0;
      if (tid == 0) s_flag = 0;
      uint32_t Hloc = 0;
      const uint32_t nchunks = (C + kChunk - 1) / kChunk;
      // thread tid owns boxes kPerThread * tid .. + kPerThread - 1 of each chunk; the
      // next chunk's records are loaded into registers while this one is pushed
      const uint32_t j0t = tid * kPerThread;
      BoxRec nxt[kPerThread];
      unsigned long long nprev = 0;
#pragma unroll
      for (int e = 0; e < kPerThread; ++e)
        if (j0t + e < C) nxt[e] = rec[j0t + e];
      if (j0t > 0 && j0t - 1 < C) nprev = __ldcg(&rec[j0t - 1].P);
      for (uint32_t c = 0; c < nchunks; ++c) {
        const uint32_t base = c * kChunk;
        const uint32_t n = min(C - base, (uint32_t)kChunk);
        BoxRec r[kPerThread];
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) r[e] = nxt[e];
        unsigned long long qprev = (j0t > 0) ? (nprev >> a.atlas_log2) : ~0ull;
        if (c + 1 < nchunks) {
          const uint32_t nb = base + kChunk;
#pragma unroll
          for (int e = 0; e < kPerThread; ++e)
            if (nb + j0t + e < C) nxt[e] = rec[nb + j0t + e];
          if (j0t > 0 && nb + j0t - 1 < C) nprev = __ldcg(&rec[nb + j0t - 1].P);
        }
        uint32_t flags = 0, cnt = 0;
#pragma unroll
        for (int e = 0; e < kPerThread; ++e) {
          const uint32_t j = j0t + e;
          if (j < n) {
            const unsigned long long q = r[e].P >> a.atlas_log2;
            const uint32_t xr = (uint32_t)(r[e].P & (om - 1));
            s_x[j] = (q % 3ull == 0ull) ? xr : Om - xr - r[e].w;
            s_w[j] = r[e].w;
            s_h[j] = r[e].h;
            if (j == 0 || q != qprev) {
              flags |= 1u << e;
              ++cnt;
            }
            qprev = q;
          }
        }
        uint32_t nseg;
        uint32_t at = block_scan_incl<uint32_t>(cnt, ws32, &nseg) - cnt;
#pragma unroll
        for (int e = 0; e < kPerThread; ++e)
          if (flags & (1u << e)) s_seg[at++] = j0t + e;
        if (tid == 0) {
          s_seg[nseg] = n;
          s_nseg = nseg;
        }
        __syncthreads();
        for (uint32_t sgi = 0; sgi < s_nseg; ++sgi) {
          const uint32_t j0 = s_seg[sgi], nbx = s_seg[sgi + 1] - j0;
          if (nbx > (uint32_t)kPushThreads) {
            // a thread per box, several boxes per thread
            for (uint32_t jj = tid; jj < nbx; jj += kPushThreads) {
              const uint32_t j = j0 + jj, x = s_x[j], w = s_w[j];
              uint32_t mx = 0;
              for (uint32_t u = 0; u < w; ++u) mx = max(mx, F[x + u]);
              const uint32_t top = mx + s_h[j];
              for (uint32_t u = 0; u < w; ++u) F[x + u] = top;
              xy[base + j] = make_uint2(x, mx);
              Hloc = max(Hloc, top);
              if (top > Om) s_flag = 1;
            }
          } else {
            // a group of g threads per box, g = 32 for <= 32 boxes ... 1 for > 512:
            // 1024 / g >= nbx, so every box has a group.  A box's group reads and then
            // writes only that box's texels, which no other box of the row touches.
            const int lgb = nbx > 1 ? 32 - __clz(nbx - 1) : 0;  // ceil(log2(nbx))
            const int lg = min(max(10 - lgb, 0), 5);
            const uint32_t g = 1u << lg;
            const uint32_t jj = tid >> lg, li = tid & (g - 1u);
            uint32_t mx = 0, x = 0, w = 0;
            if (jj < nbx) {
              x = s_x[j0 + jj];
              w = s_w[j0 + jj];
              for (uint32_t u = li; u < w; u += g) mx = max(mx, F[x + u]);
            }
            for (uint32_t o = 1; o < g; o <<= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
            if (jj < nbx) {
              const uint32_t top = mx + s_h[j0 + jj];
              for (uint32_t u = li; u < w; u += g) F[x + u] = top;
              if (li == 0) {
                xy[base + j0 + jj] = make_uint2(x, mx);
                Hloc = max(Hloc, top);
                if (top > Om) s_flag = 1;
              }
            }
          }
          __syncthreads();
          if (s_flag) break;
        }
        if (s_flag) break;
      }
      H = block_max<uint32_t>(Hloc, ws32);
      ok = (!s_flag && H <= Om) ? 1u : 0u;
    }
  }
  // publish this candidate; the last CTA selects
  if (tid == 0) {
    p.cand[kidx] = PackCand{ok, Om, H, status};
    __threadfence();
    const uint32_t done = atomicAdd(&p.ctr->pack_done, 1u);
    s_last = (done == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid == 0) {
    uint32_t best = 0, bestOm = 0;
    int32_t pst = FA_OK;
    for (uint32_t kk = 1; kk <= gridDim.x; ++kk) {
      const uint4 cv = __ldcg(reinterpret_cast<const uint4*>(p.cand) + (kk - 1));
      if ((int32_t)cv.w != FA_OK) pst = (int32_t)cv.w;
      if (!cv.x) continue;
      if (best == 0 || a.select_mode == FA_SELECT_LARGEST_K ||
          (unsigned long long)kk * bestOm >= (unsigned long long)best * cv.y) {
        best = kk;
        bestOm = cv.y;
      }
    }
    if (pst == FA_OK && best == 0) pst = FA_E_PACK_FAILED;
    fa_pack_result r{0, 0, 0, pst, C};
    if (pst == FA_OK) {
      const uint4 cv = __ldcg(reinterpret_cast<const uint4*>(p.cand) + (best - 1));
      r.k = best;
      r.omega = cv.y;
      r.height = cv.z;
    }
    *a.res = r;
    p.ctr->pack_done = 0;
  }
}

// Placements of the selected candidate, in chart order (all CTAs).
__global__ void __launch_bounds__(256) k_pack_place(PackScratch p, PackArgs a) {
  pdl_wait();
  if (__ldcg(&a.res->status) != FA_OK) return;
  const uint32_t C = __ldcg(&a.res->count), kb = __ldcg(&a.res->k) - 1;
  const uint2* bxy = p.xy + (size_t)kb * p.max_boxes;
  const BoxRec* brec = p.rec + (size_t)kb * p.max_boxes;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    const uint32_t b = __ldcg(a.order + i);
    const uint2 q = __ldcg(bxy + i);
    const uint2 wh = __ldcg(reinterpret_cast<const uint2*>(brec + i) + 1);
    a.place[b] = fa_placement{(int32_t)q.x, (int32_t)q.y, (int32_t)wh.x, (int32_t)wh.y};
  }
}

size_t push_smem_bytes(uint32_t front_cap) {
  return (size_t)(4 * kChunk + 4) * 4 + (size_t)front_cap * 4;
}

}  // namespace

fa_status launch_pack_kernels(fa_ctx* ctx, const PackScratch& p, const uint32_t* fa_, const uint32_t* fb,
                              uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode, uint32_t min_box,
                              uint32_t gutter, uint32_t* order, fa_placement* place, fa_pack_result* res,
                              cudaStream_t s) {
  uint32_t* ord = order ? order : p.order;
  if (ctx) mark(ctx, "k_order_tile", s);
  launch_k(k_order_tile, p.max_tiles, kOrderTile, 0, s, p, fb);
  if (ctx) mark(ctx, "k_order_binscan", s);
  launch_k(k_order_binscan, 1, 1024, 0, s, p);
  if (ctx) mark(ctx, "k_order_scatter", s);
  launch_k(k_order_scatter, p.max_tiles, kOrderTile, 0, s, p, fb, ord);
  PackArgs a;
  a.fa = fa_;
  a.fb = fb;
  a.order = ord;
  a.atlas_log2 = atlas_log2;
  uint32_t sh = 8;
  while ((1u << (sh - 8)) < n_scales) ++sh;
  a.shift = sh;
  a.min_box = min_box;
  a.gutter = gutter;
  a.select_mode = select_mode;
  const uint32_t om = 1u << atlas_log2;
  a.front_cap = (8u * om < kFrontCap) ? 8u * om : kFrontCap;
  a.place = place;
  a.res = res;
  const uint32_t items = p.max_tiles * n_scales;
  const unsigned g2 = items < 152u * 2u ? items : 152u * 2u;
  if (ctx) mark(ctx, "k_pack_boxes", s);
  launch_k(k_pack_boxes, g2, kThreads, 0, s, p, a, n_scales);
  if (ctx) mark(ctx, "k_pack_fix", s);
  launch_k(k_pack_fix, g2, kThreads, 0, s, p, a, n_scales);
  if (ctx) mark(ctx, "k_pack_push", s);
  launch_k(k_pack_push, n_scales, kPushThreads, push_smem_bytes(a.front_cap), s, p, a);
  if (ctx) mark(ctx, "k_pack_place", s);
  launch_k(k_pack_place, 152 * 2, 256, 0, s, p, a);
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
}

fa_status pack_set_smem_limit() {
  FA_CUDA_TRY(cudaFuncSetAttribute(k_pack_push, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)push_smem_bytes(kFrontCap)));
  return FA_OK;
}

fa_status launch_pack(fa_ctx* ctx, const uint32_t* fa_, const uint32_t* fb, const uint32_t* count,
                      uint32_t atlas_log2, uint32_t n_scales, uint32_t select_mode, uint32_t* order,
                      fa_placement* place, fa_pack_result* res, cudaStream_t s) {
  if (!ctx->pack_smem_set) {
    fa_status st = pack_set_smem_limit();
    if (st != FA_OK) return st;
    ctx->pack_smem_set = 1;
  }
  PackScratch p = ctx->pack;
  p.count = count;
  return launch_pack_kernels(ctx, p, fa_, fb, atlas_log2, n_scales, select_mode, ctx->cfg.min_box,
                             ctx->cfg.gutter, order, place, res, s);
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
constexpr size_t kOffM = align256(kOffCand + sizeof(PackCand) * kMaxScales);
constexpr size_t kOffCounts = align256(kOffM + sizeof(uint32_t) * kMaxScales);
constexpr size_t kOffRank = align256(kOffCounts + sizeof(uint32_t) * kMaxH * kNoAllocTiles);
constexpr size_t kOffTotal = align256(kOffRank + sizeof(uint32_t) * kNoAllocMaxBoxes);
constexpr size_t kOffBinstart = align256(kOffTotal + sizeof(uint32_t) * kMaxH);
constexpr size_t kOffOrder = align256(kOffBinstart + sizeof(uint32_t) * kMaxH);
constexpr size_t kOffTileTot = align256(kOffOrder + sizeof(uint32_t) * kNoAllocMaxBoxes);
constexpr size_t kOffRec = align256(kOffTileTot + sizeof(unsigned long long) * kMaxScales * kNoAllocTiles);
constexpr size_t kOffXY = align256(kOffRec + sizeof(BoxRec) * kMaxScales * kNoAllocMaxBoxes);
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
  p.ord_binstart = (uint32_t*)(base + kOffBinstart);
  p.order = (uint32_t*)(base + kOffOrder);
  p.tile_tot = (unsigned long long*)(base + kOffTileTot);
  p.rec = (BoxRec*)(base + kOffRec);
  p.m = (uint32_t*)(base + kOffM);
  p.xy = (uint2*)(base + kOffXY);
  p.cand = (PackCand*)(base + kOffCand);
  launch_k(k_noalloc_reset, 1, 256, 0, s, p.ctr, (uint32_t*)p.count, p.ord_total, n);
  return launch_pack_kernels(nullptr, p, d_fa, d_fb, atlas_log2, n_scales, select_mode, min_box, gutter, d_order,
                             d_place, d_res, s);
}
