// Box order and packing (Sec. 4.1-4.3).
//
// Order: stable counting sort of the boxes by integer height
//   h0 = clamp(ceil(fb / 256), 1, 8192), tallest first, ties by box index (the
//   boxes arrive numbered by ascending root, so this is the paper's
//   (height, lowest triangle id) order).  k_order_tile ranks the boxes of each
//   1024-box tile stably inside their height bin (a shared-memory histogram the
//   warps update in index order) and writes a per-bin count row per tile and the
//   global bin totals; k_order_scatter scans the totals (every block) and adds, for
//   each box, the counts of its bin in earlier tiles.
//   This replaces the paper's cuckoo-hash bucketing with the same result contract
//   (deterministic, identical for identical frames).
//
// Pack: candidates k / n, k = 1..n (Sec. 4.2).  k_order_scatter also writes the
//   footprints in box order.  k_pack_scan takes (one or two candidates, 4096-box
//   chunk) work items: scaled integer boxes, the exclusive prefix P of the widths
//   (chunk-local scan plus a decoupled look-back over the preceding chunks), the largest
//   overflow m past omega (Sec. 4.3), and per box a push-ready record (x inside the
//   row, w, h, row direction) plus per chunk the list of row segments.  Then one CTA
//   per candidate (k_pack_push) pushes the rows up against a frontline in shared
//   memory, with the chunks staged by bulk asynchronous copies; segments of one
//   row never overlap in x, so a row may span two chunks.  The last CTA to finish
//   selects the candidate.  The placements are written by the UV kernel on the frame
//   path and by k_pack_place (all CTAs) for a standalone packing.
#pragma once
#include "fa_internal.cuh"

namespace fa {
namespace pk {
namespace {

__device__ __forceinline__ uint32_t height_bin(uint32_t fb) {
  uint32_t h = (uint32_t)(((uint64_t)fb + 255u) >> 8);
  h = h < 1u ? 1u : (h > kMaxH ? kMaxH : h);
  return kMaxH - h;  // ascending bin = descending height
}

// Block-wide inclusive scan (any whole number of warps up to 1024 threads); writes
// the block total to *total.
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
  const uint32_t nw = blockDim.x >> 5;
  if (wid == 0) {
    T s = lane < nw ? warp_sums[lane] : (T)0;
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

// FOOT: the charts' footprints are computed here from their box accumulators
// (written out, and their heights used as the keys) instead of read from fb.
// hist: kMaxH words of shared memory (boxes of each height bin seen so far in the tile).
template <bool FOOT>
__device__ __forceinline__ void order_tile_body(const PackScratch& p, const uint32_t* __restrict__ fb,
                                                const FootArgs& foot, uint32_t bid, uint32_t* hist) {
  if (__ldcg(&p.ctr->status) != 0) return;
  const uint32_t C = __ldcg(p.count);
  if (C > p.max_boxes) return;
  const uint32_t ntiles = (C + kOrderTile - 1) / kOrderTile;
  if (bid >= ntiles) return;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t i = bid * kOrderTile + tid;
  uint32_t fbi = 0;
  if (i < C) fbi = FOOT ? chart_footprint(foot, i) : __ldg(fb + i);
  const uint32_t bin = i < C ? height_bin(fbi) : kMaxH;  // kMaxH: no box
  for (uint32_t b = tid; b < kMaxH; b += kOrderTile) hist[b] = 0;
  // stable rank inside the tile: the warps take their turn in index order; inside a
  // warp, the lanes with the same bin are ranked by lane
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, bin);
  const uint32_t before = __popc(peers & ((1u << lane) - 1u));
  const bool leader = before == 0u;
  uint32_t r = 0;
  for (uint32_t w = 0; w < (uint32_t)(kOrderTile / 32); ++w) {
    __syncthreads();
    if (wid == w && bin < kMaxH) {
      r = hist[bin] + before;
      __syncwarp(peers);
      if (leader) hist[bin] = r + __popc(peers);
    }
  }
  __syncthreads();
  if (bin < kMaxH) p.ord_rank[i] = r;
  uint32_t* row = p.ord_counts + (size_t)bid * kMaxH;
  for (uint32_t b = tid; b < kMaxH; b += kOrderTile) {
    const uint32_t c = hist[b];
    row[b] = c;
    if (c) atomicAdd(p.ord_total + b, c);
  }
}

// Each block scans the bin totals itself (exclusive, in shared memory), then places
// its boxes: bin start + the bin's boxes in earlier tiles + the rank in the tile.
// Block 0 also clears the width scan's look-back state and overflows (k_pack_scan
// runs next; it clears the bin totals for the next call).
// binstart: kMaxH words of shared memory.
__device__ __forceinline__ void order_scatter_body(const PackScratch& p, const uint32_t* __restrict__ fa,
                                                   const uint32_t* __restrict__ fb, uint32_t* order, uint32_t bid,
                                                   uint32_t* binstart) {
  __shared__ uint32_t wt[32];
  if (__ldcg(&p.ctr->status) != 0) return;
  const uint32_t C = __ldcg(p.count);
  if (C > p.max_boxes) return;
  if (bid == 0) {  // also with no boxes: the push reads the overflows
    for (uint32_t i = threadIdx.x; i < kMaxScales * p.max_chunks; i += blockDim.x) p.scan_state[i] = 0ull;
    if (threadIdx.x < kMaxScales) p.m[threadIdx.x] = 0u;
  }
  if (bid * kOrderTile >= C) return;
  constexpr uint32_t kPer = kMaxH / kOrderTile;
  const uint4* t4 = reinterpret_cast<const uint4*>(p.ord_total) + threadIdx.x * (kPer / 4);
  uint32_t v[kPer];
#pragma unroll
  for (uint32_t j = 0; j < kPer / 4; ++j) {
    const uint4 q = __ldcg(t4 + j);
    v[4 * j] = q.x;
    v[4 * j + 1] = q.y;
    v[4 * j + 2] = q.z;
    v[4 * j + 3] = q.w;
  }
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) sum += v[j];
  uint32_t tot;
  uint32_t run = block_scan_incl<uint32_t>(sum, wt, &tot) - sum;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    binstart[threadIdx.x * kPer + j] = run;
    run += v[j];
  }
  __syncthreads();
  const uint32_t i = bid * kOrderTile + threadIdx.x;
  if (i >= C) return;
  const uint32_t bin = height_bin(__ldcg(fb + i));
  uint32_t pos = binstart[bin] + p.ord_rank[i];
  // the bin's boxes in earlier tiles: sixteen independent loads per round
  for (uint32_t t = 0; t < bid; t += 16) {
    const uint32_t* c = p.ord_counts + (size_t)t * kMaxH + bin;
    uint32_t q[16];
#pragma unroll
    for (uint32_t j = 0; j < 16; ++j) q[j] = t + j < bid ? __ldcg(c + (size_t)j * kMaxH) : 0u;
#pragma unroll
    for (uint32_t j = 0; j < 16; ++j) pos += q[j];
  }
  if (pos < C) {
    order[pos] = i;
    p.fs[pos] = make_uint2(__ldcg(fa + i), __ldcg(fb + i));
  }
  p.ord_rank[i] = pos;  // from here on: the box's position in the order
}

// ------------------------------------------------------------------ pack

struct PackArgs {
  const uint32_t* order;
  uint32_t atlas_log2;
  uint32_t lowres_log2;  // > 0: the packing must also serve the atlas scaled by 2^-lowres_log2
  uint32_t shift;  // log2(256 * n_scales)
  uint32_t min_box;
  uint32_t gutter;
  uint32_t select_mode;
  uint32_t front_cap;
  uint32_t loop_cap;          // polls (at most kLookbackPolls) of an unpublished earlier chunk before
                              // the look-back sums that chunk itself
  unsigned long long wait_ns;  // time limit of the push's wait for a staged chunk
  fa_placement* place;
  fa_pack_result* res;
};

// Width scan: one work item per (KC candidates, chunk of kChunk boxes), taken by CTA
// index (items bid, bid + nblk, ...).  Each item computes the scaled boxes (Sec.
// 4.2), scans the widths, and takes its chunk's offset P by a decoupled look-back
// over the preceding chunks' published sums (one warp per candidate); an earlier
// chunk that has published nothing after a few polls is summed by the looking warp
// itself, so no item waits on a CTA that may not be resident.  It then writes, per
// box, the push record
//   x: xr = P mod omega (bits 0-15) | w (bits 16-31)
//   y: h (bits 0-30) | row runs left to right (bit 31: row q = P / omega, q mod 3 == 0)
// (w and h saturate; a candidate whose box exceeds 16 bits of width has Omega above
// the frontline capacity and never reaches the push), the chunk's list of row
// segments (first box of each row inside the chunk; the chunk's first box always
// starts one), and folds the largest overflow past omega into m (Sec. 4.3).
constexpr int kScanThreads = 512;
constexpr unsigned long long kStAgg = 1ull << 62;  // chunk sum published
constexpr unsigned long long kStInc = 2ull << 62;  // inclusive prefix published
constexpr unsigned long long kStVal = (1ull << 62) - 1ull;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* q) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(q) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* q, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(q), "l"(v) : "memory");
}

// Block-wide inclusive scans of KC values at once (warp q scans the warp sums of
// value q); total[q] is value q's block total.
template <int KC>
__device__ __forceinline__ void block_scan_incl_n(const unsigned long long (&v)[KC], unsigned long long (*warp_sums)[32],
                                                  unsigned long long (&incl)[KC], unsigned long long (&total)[KC]) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long x[KC];
#pragma unroll
  for (int q = 0; q < KC; ++q) x[q] = v[q];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x[q], o);
      if (lane >= (unsigned)o) x[q] += y;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int q = 0; q < KC; ++q) warp_sums[q][wid] = x[q];
  __syncthreads();
  const uint32_t nw = blockDim.x >> 5;
  if (wid < (uint32_t)KC) {
    unsigned long long t = lane < nw ? warp_sums[wid][lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= (unsigned)o) t += y;
    }
    warp_sums[wid][lane] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < KC; ++q) {
    incl[q] = x[q] + (wid ? warp_sums[q][wid - 1] : 0ull);
    total[q] = warp_sums[q][31];
  }
}

// Scaled width and height of a footprint for candidate k (Sec. 4.2).
__device__ __forceinline__ uint32_t scaled_side(unsigned long long k, uint32_t f, const PackArgs& a,
                                                unsigned long long d) {
  const uint32_t s = (uint32_t)((k * f + d) >> a.shift);
  return (s > a.min_box ? s : a.min_box) + 2u * a.gutter;
}

// Polls of an unpublished earlier chunk before the look-back sums it itself (the
// context's loop_cap, if lower).
constexpr uint32_t kLookbackPolls = 256;

// Sum of candidate k's scaled widths over chunk j (one warp; the look-back's
// fallback when chunk j's item has published nothing).
__device__ __forceinline__ unsigned long long chunk_width_sum(const PackScratch& p, const PackArgs& a, uint32_t C,
                                                              uint32_t j, unsigned long long k,
                                                              unsigned long long d) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t base = j * kChunk, n = min(C - base, kChunk);
  const uint4* f4 = reinterpret_cast<const uint4*>(p.fs + base);  // padded to whole chunks
  unsigned long long s = 0;
#pragma unroll 4
  for (uint32_t i = lane; i < kChunk / 2; i += 32) {
    const uint4 v = __ldcg(f4 + i);
    if (2u * i < n) s += scaled_side(k, v.x, a, d);
    if (2u * i + 1u < n) s += scaled_side(k, v.z, a, d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  return s;
}

// The items of C boxes with KC candidates each.  KC = 2: the candidates of item
// (g, c) are k = 2g + 1 and 2g + 2, so one item loads its chunk's footprints once
// for both, and twice as many chunks fit one wave of the grid; each candidate keeps
// its own scan state.
template <int NT, int KC>
__device__ __forceinline__ void pack_scan_items(const PackScratch& p, const PackArgs& a, uint32_t n_scales,
                                                uint32_t C, uint32_t bid, uint32_t nblk) {
  constexpr int kScanPer = kChunk / NT;  // consecutive boxes per thread
  __shared__ unsigned long long ws64[KC][32];
  __shared__ uint32_t ws32[KC][32];
  __shared__ uint32_t s_lastw[KC][NT / 32];
  __shared__ uint32_t s_wmax[KC][NT / 32];
  __shared__ unsigned long long s_prefix[KC];
  const uint32_t nch = (C + kChunk - 1) / kChunk;
  const uint32_t items = nch * ((n_scales + KC - 1) / KC);
  const uint32_t om = 1u << a.atlas_log2;
  const unsigned long long d = (1ull << a.shift) - 1ull;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const size_t rstride = (size_t)p.max_chunks * kChunk;
  for (uint32_t item = bid; item < items; item += nblk) {
    __syncthreads();  // the shared memory of the previous item is free
    const uint32_t grp = item / nch, c = item % nch;
    const uint32_t base = c * kChunk, n = min(C - base, kChunk);
    const uint32_t j0 = tid * kScanPer;
    // this thread's footprints (the footprint array is padded to whole chunks)
    const uint4* f4 = reinterpret_cast<const uint4*>(p.fs + base + j0);
    uint32_t fa[kScanPer], fb[kScanPer];
#pragma unroll
    for (int q = 0; q < kScanPer / 2; ++q) {
      const uint4 v = __ldcg(f4 + q);
      fa[2 * q] = v.x;
      fb[2 * q] = v.y;
      fa[2 * q + 1] = v.z;
      fb[2 * q + 1] = v.w;
    }
    unsigned long long sum[KC], incl[KC], tot[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      const unsigned long long k = (unsigned long long)grp * KC + q + 1;
      sum[q] = 0;
      uint32_t w = 0;
#pragma unroll
      for (int e = 0; e < kScanPer; ++e) {
        w = j0 + e < n ? scaled_side(k, fa[e], a, d) : 0u;
        sum[q] += w;
      }
      if (lane == 31) s_lastw[q][wid] = w;
    }
    block_scan_incl_n<KC>(sum, ws64, incl, tot);
    // chunk offsets by decoupled look-back (warp q for the item's candidate q)
    if (wid < (uint32_t)KC && grp * KC + wid < n_scales) {
      const uint32_t kidx = grp * KC + wid;
      unsigned long long* st = p.scan_state + (size_t)kidx * p.max_chunks;
      unsigned long long prefix = 0, tq = 0;
#pragma unroll
      for (int q = 0; q < KC; ++q)
        if (wid == (uint32_t)q) tq = tot[q];
      if (c == 0) {
        if (lane == 0) st_relaxed_u64(st, kStInc | tq);
      } else {
        if (lane == 0) st_relaxed_u64(st + c, kStAgg | tq);
        int jn = (int)c - 1;  // nearest chunk not yet folded in
        const uint32_t max_polls = min(a.loop_cap, kLookbackPolls);
        uint32_t polls = 0;
        for (;;) {
          const int t = jn - (int)lane;
          const unsigned long long v = t >= 0 ? ld_relaxed_u64(st + t) : kStInc;
          const uint32_t inc = __ballot_sync(0xFFFFFFFFu, (v >> 62) == 2ull);
          const uint32_t none = __ballot_sync(0xFFFFFFFFu, (v >> 62) == 0ull);
          const uint32_t ui = inc ? (uint32_t)(__ffs(inc) - 1) : 32u;
          const uint32_t un = none ? (uint32_t)(__ffs(none) - 1) : 32u;
          // fold in the sums before the first unpublished chunk, up to and with the
          // first inclusive prefix
          const uint32_t upto = ui < un ? ui + 1u : un;
          unsigned long long x = lane < upto ? (v & kStVal) : 0ull;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
          prefix += x;
          if (ui < un) break;
          jn -= (int)upto;
          if (upto) polls = 0;
          if (un == 32u) continue;
          // chunk jn has published nothing yet: poll it again, or (its item may not
          // have started: CTAs need not be resident together) sum its widths here
          if (++polls > max_polls) {
            prefix += chunk_width_sum(p, a, C, (uint32_t)jn, kidx + 1ull, d);
            jn -= 1;
            polls = 0;
          }
        }
        if (lane == 0) st_relaxed_u64(st + c, kStInc | ((prefix + tq) & kStVal));
      }
      if (lane == 0) s_prefix[wid] = prefix;
    }
    __syncthreads();
    // the item's candidates side by side: push records, row starts and overflow
    uint32_t u[KC], starts[KC], cnt[KC], mo[KC], wlast[KC], q0m3[KC];
    bool first_start[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      const unsigned long long k = (unsigned long long)grp * KC + q + 1;
      // previous box's width, for the row test of this thread's first box
      uint32_t wprev = __shfl_up_sync(0xFFFFFFFFu, j0 + kScanPer - 1 < n ? scaled_side(k, fa[kScanPer - 1], a, d) : 0u, 1);
      if (lane == 0) wprev = wid ? s_lastw[q][wid - 1] : 0u;
      // the thread's boxes in 32-bit arithmetic relative to its first box: row
      // q0 + (u >> log2 omega) and offset u & (omega - 1) for u = P - q0 omega (u stays
      // below 2^28: a box is at most 2^24 wide)
      const unsigned long long P0 = s_prefix[q] + incl[q] - sum[q];
      const unsigned long long q0 = P0 >> a.atlas_log2;
      q0m3[q] = (uint32_t)(q0 % 3ull);
      u[q] = (uint32_t)(P0 & (om - 1u));
      // first box: does a row start here (the previous box begins in an earlier row)?
      first_start[q] = j0 == 0 || ((P0 - wprev) >> a.atlas_log2) != q0;
      starts[q] = cnt[q] = mo[q] = wlast[q] = 0u;
    }
#pragma unroll
    for (int e2 = 0; e2 < kScanPer / 2; ++e2) {
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        const uint32_t kidx = grp * KC + q;
        if (kidx >= n_scales) break;  // (the same for the whole CTA)
        const unsigned long long k = kidx + 1;
        uint32_t r[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int e = 2 * e2 + h2;
          uint32_t w = 0;
          if (j0 + e < n) {
            w = scaled_side(k, fa[e], a, d);
            const uint32_t h = scaled_side(k, fb[e], a, d);
            const uint32_t dq = u[q] >> a.atlas_log2;
            const uint32_t xr = u[q] & (om - 1u);
            const bool st = e ? ((u[q] - wlast[q]) >> a.atlas_log2) != dq : first_start[q];
            if (st) {
              starts[q] |= 1u << e;
              ++cnt[q];
            }
            if (xr + w > om) mo[q] = max(mo[q], xr + w - om);
            const uint32_t ws = w < 0xFFFFu ? w : 0xFFFFu;
            const uint32_t hs = h < 0x7FFFFFFFu ? h : 0x7FFFFFFFu;
            r[2 * h2] = xr | (ws << 16);
            r[2 * h2 + 1] = hs | (((q0m3[q] + dq % 3u) % 3u == 0u) ? 0x80000000u : 0u);
          }
          u[q] += w;
          wlast[q] = w;
        }
        reinterpret_cast<uint4*>(p.rec8 + kidx * rstride + base + j0)[e2] = make_uint4(r[0], r[1], r[2], r[3]);
      }
    }
    // one block pass for all of them: the exclusive prefix of the row starts and the
    // largest overflow
    uint32_t x[KC], mx[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      x[q] = cnt[q];
      mx[q] = mo[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x[q], o), z = __shfl_xor_sync(0xFFFFFFFFu, mx[q], o);
        if (lane >= (unsigned)o) x[q] += y;
        mx[q] = max(mx[q], z);
      }
      if (lane == 31) {
        ws32[q][wid] = x[q];
        s_wmax[q][wid] = mx[q];
      }
    }
    __syncthreads();
    if (wid < (uint32_t)KC) {
      const uint32_t nw = NT / 32;
      uint32_t t = lane < nw ? ws32[wid][lane] : 0u, m2 = lane < nw ? s_wmax[wid][lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o), z = __shfl_xor_sync(0xFFFFFFFFu, m2, o);
        if (lane >= (unsigned)o) t += y;
        m2 = max(m2, z);
      }
      ws32[wid][lane] = t;
      if (lane == 0) s_wmax[wid][0] = m2;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      const uint32_t kidx = grp * KC + q;
      if (kidx >= n_scales) break;
      const uint32_t nseg = ws32[q][31];
      uint32_t at = x[q] - cnt[q] + (wid ? ws32[q][wid - 1] : 0u);
      uint16_t* sg = p.segs + ((size_t)kidx * p.max_chunks + c) * kSegStride;
#pragma unroll
      for (int e = 0; e < kScanPer; ++e)
        if (starts[q] & (1u << e)) sg[1 + at++] = (uint16_t)(j0 + e);
      if (tid == 0) {
        sg[0] = (uint16_t)nseg;
        sg[1 + nseg] = (uint16_t)n;
        if (s_wmax[q][0]) atomicMax(p.m + kidx, s_wmax[q][0]);
      }
    }
  }
}

// nblk: the CTAs that take items.  PAIRS: two candidates per item where one per item
// would take more than one wave of them.
template <int NT, bool PAIRS = true>
__device__ __forceinline__ void pack_scan_body(const PackScratch& p, const PackArgs& a, uint32_t n_scales,
                                               uint32_t bid, uint32_t nblk) {
  // the order's bin totals were last read by k_order_scatter: clear them for the next call
  if (bid == 0)
    for (uint32_t b = threadIdx.x; b < kMaxH; b += blockDim.x) p.ord_total[b] = 0u;
  __shared__ int32_t s_status;
  // one read of the status word for the whole CTA (another CTA's time-out can set
  // it meanwhile, and every thread must take the same branch before the barriers)
  if (threadIdx.x == 0) s_status = __ldcg(&p.ctr->status);
  __syncthreads();
  if (s_status != 0) return;
  const uint32_t C = __ldcg(p.count);
  if (C > p.max_boxes || C == 0) return;
  if (PAIRS && (unsigned long long)((C + kChunk - 1) / kChunk) * n_scales > nblk)
    pack_scan_items<NT, 2>(p, a, n_scales, C, bid, nblk);
  else
    pack_scan_items<NT, 1>(p, a, n_scales, C, bid, nblk);
}

// Row push of one candidate per CTA, then the last CTA selects.  The chunks' push
// records and segment lists are staged into shared memory by bulk asynchronous
// copies, two chunks in flight; every row segment is processed box-parallel (with NT
// threads: a group of 2 .. 32 threads per box in segments of at most NT / 4 boxes,
// else one thread per box): resting height =
// max of the frontline under the box, then the frontline takes the box top, one
// barrier per segment.  Segments of one row never overlap in x, so a row may span
// two chunks.
constexpr int kPushThreads = (int)kDefaultPushThreads;  // the push kernel's CTA without a context
constexpr uint32_t kStageBytes = kChunk * 8u + kSegStride * 2u;  // records + segment list
static_assert(kStageBytes % 16u == 0u, "bulk copies move multiples of 16 bytes");

__device__ __forceinline__ uint32_t smem_addr(const void* q) { return (uint32_t)__cvta_generic_to_shared(q); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Waits at most limit_ns for the phase of the given parity; false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool better_cand(uint32_t k1, uint32_t o1, uint32_t k2, uint32_t o2, uint32_t mode) {
  if (k1 == 0u) return false;
  if (k2 == 0u) return true;
  if (mode == FA_SELECT_LARGEST_K) return k1 > k2;
  const unsigned long long l = (unsigned long long)k1 * o2, r = (unsigned long long)k2 * o1;
  return l > r || (l == r && k1 > k2);  // larger effective scale, ties to the larger k
}

// smem_raw: push_smem_bytes(a.front_cap) bytes of shared memory (128-byte aligned).
// NT: threads of the CTA (a power of two, 64 .. 1024).
template <int NT>
__device__ __forceinline__ void push_body(const PackScratch& p, const PackArgs& a, uint32_t bid, uint32_t nblk,
                                          unsigned char* smem_raw) {
  uint32_t* F = reinterpret_cast<uint32_t*>(smem_raw + 2 * kStageBytes);  // [front_cap]
  __shared__ __align__(8) unsigned long long s_bar[2];
  __shared__ uint32_t ws32[32];
  __shared__ uint32_t s_last;
  __shared__ int32_t s_st0;
  const uint32_t kidx = bid;
  const uint32_t tid = threadIdx.x;
  // an error of an earlier kernel (or of another candidate that already timed out):
  // no work, but every CTA still publishes and counts itself, so that the last one
  // selects and resets the counter.  One read for the whole CTA: every thread must
  // take the same branch before the barriers below.
  if (tid == 0) s_st0 = __ldcg(&p.ctr->status);
  __syncthreads();
  const int32_t st0 = s_st0;
  const uint32_t C = __ldcg(p.count);
  const uint32_t om = 1u << a.atlas_log2;
  int32_t status = FA_OK;
  uint32_t Om = om, H = 0, ok = 0;
  if (st0 != 0) {
    status = st0;
  } else if (C > p.max_boxes) {
    status = FA_E_CAPACITY;
  } else {
    Om = om + __ldcg(p.m + kidx);
    if (Om > a.front_cap) {
      status = FA_E_CAPACITY;
    } else {
      const uint2* rec = p.rec8 + (size_t)kidx * p.max_chunks * kChunk;
      const uint16_t* sgg = p.segs + (size_t)kidx * p.max_chunks * kSegStride;
      uint2* xy = p.xy + (size_t)kidx * p.max_boxes;
      const uint32_t nchunks = (C + kChunk - 1) / kChunk;
      uint32_t issued = 0;  // chunks whose copies were issued (thread 0)
      auto issue = [&](uint32_t c) {
        unsigned char* dst = smem_raw + (c & 1u) * kStageBytes;
        const uint32_t nb = min(C - c * kChunk, kChunk);
        const uint32_t rbytes = ((nb + 1u) & ~1u) * 8u;  // whole 16-byte units (padded chunk)
        mbar_expect_tx(&s_bar[c & 1u], rbytes + kSegStride * 2u);
        bulk_g2s(dst, rec + (size_t)c * kChunk, rbytes, &s_bar[c & 1u]);
        bulk_g2s(dst + kChunk * 8u, sgg + (size_t)c * kSegStride, kSegStride * 2u, &s_bar[c & 1u]);
      };
      for (uint32_t x = tid; x < Om; x += NT) F[x] = 0;
      if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (; issued < nchunks && issued < 2u; ++issued) issue(issued);
      }
      __syncthreads();
      uint32_t Hloc = 0, consumed = 0;
      bool fail = false, timed_out = false;
      for (uint32_t c = 0; c < nchunks; ++c) {
        const uint32_t stg = c & 1u;
        const bool got = mbar_wait_bounded(&s_bar[stg], (c >> 1) & 1u, a.wait_ns);
        if (__syncthreads_or(!got)) {
          timed_out = true;
          break;
        }
        consumed = c + 1;
        const uint2* s_rec = reinterpret_cast<const uint2*>(smem_raw + stg * kStageBytes);
        const uint16_t* s_sg = reinterpret_cast<const uint16_t*>(smem_raw + stg * kStageBytes + kChunk * 8u);
        // (the clamps keep every shared-memory index inside the stage whatever the list holds)
        const uint32_t nseg = min((uint32_t)s_sg[0], kChunk), base = c * kChunk;
        for (uint32_t sgi = 0; sgi < nseg; ++sgi) {
          const uint32_t j0 = min((uint32_t)s_sg[1 + sgi], kChunk), j1 = min((uint32_t)s_sg[2 + sgi], kChunk);
          const uint32_t nbx = j1 > j0 ? j1 - j0 : 0u;
          bool bad = false;
          if (nbx > (uint32_t)NT / 4u) {
            // a thread per box (several boxes per thread past NT).  Boxes of such rows
            // are mostly a few texels wide: the first four texels are read with
            // independent loads before any is used, the rest in a loop.
            for (uint32_t jj = tid; jj < nbx; jj += NT) {
              const uint2 r = s_rec[j0 + jj];
              const uint32_t xr = r.x & 0xFFFFu, w = r.x >> 16, h = r.y & 0x7FFFFFFFu;
              uint32_t* Fx = F + ((r.y >> 31) ? xr : Om - xr - w);
              uint32_t m0 = w > 0u ? Fx[0] : 0u;
              const uint32_t m1 = w > 1u ? Fx[1] : 0u, m2 = w > 2u ? Fx[2] : 0u, m3 = w > 3u ? Fx[3] : 0u;
              for (uint32_t u = 4; u < w; ++u) m0 = max(m0, Fx[u]);
              const uint32_t mx = max(max(m0, m1), max(m2, m3)), top = mx + h;
              if (w > 0u) Fx[0] = top;
              if (w > 1u) Fx[1] = top;
              if (w > 2u) Fx[2] = top;
              if (w > 3u) Fx[3] = top;
              for (uint32_t u = 4; u < w; ++u) Fx[u] = top;
              xy[base + j0 + jj] = make_uint2((uint32_t)(Fx - F), mx);
              Hloc = max(Hloc, top);
              bad |= top > Om;
            }
          } else {
            // a group of g threads per box, g = min(32, NT / 2^ceil(log2 nbx)) >= 2:
            // NT / g >= nbx, so every box has a group.  A box's group reads and then
            // writes only that box's texels, which no other box of the row touches.
            const int lgb = nbx > 1 ? 32 - __clz(nbx - 1) : 0;  // ceil(log2(nbx))
            const int lg = min(max((31 - __clz(NT)) - lgb, 0), 5);
            const uint32_t g = 1u << lg;
            const uint32_t jj = tid >> lg, li = tid & (g - 1u);
            uint32_t mx = 0, x = 0, w = 0, h = 0;
            if (jj < nbx) {
              const uint2 r = s_rec[j0 + jj];
              const uint32_t xr = r.x & 0xFFFFu;
              w = r.x >> 16;
              h = r.y & 0x7FFFFFFFu;
              x = (r.y >> 31) ? xr : Om - xr - w;
              for (uint32_t u = li; u < w; u += g) mx = max(mx, F[x + u]);
            }
            for (uint32_t o = 1; o < g; o <<= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
            if (jj < nbx) {
              const uint32_t top = mx + h;
              for (uint32_t u = li; u < w; u += g) F[x + u] = top;
              if (li == 0) {
                xy[base + j0 + jj] = make_uint2(x, mx);
                Hloc = max(Hloc, top);
                bad = top > Om;
              }
            }
          }
          fail |= bad;
          __syncthreads();
        }
        // a candidate that no longer fits stops at the end of the chunk (one
        // reduction per chunk; a box may rest above Omega meanwhile, which only
        // raises later rests: every index stays inside [0, Omega))
        if (__syncthreads_or(fail)) {
          fail = true;
          break;
        }
        // every thread is past this chunk's last barrier: its stage is free
        if (tid == 0 && issued < nchunks) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(issued);
          ++issued;
        }
      }
      // copies still in flight land before the CTA leaves (with the full limit, also
      // after a time-out: the shared memory they write must outlive them)
      if (tid == 0)
        for (uint32_t c = consumed; c < issued; ++c) mbar_wait_bounded(&s_bar[c & 1u], (c >> 1) & 1u, kWaitNs);
      if (timed_out) {
        if (tid == 0) set_status(p.ctr, FA_E_TIMEOUT);
        status = FA_E_TIMEOUT;
      }
      H = block_max<uint32_t>(Hloc, ws32);  // (also: every wait on the barriers is over)
      if (tid == 0) {  // the CTA may run another candidate's push next
        mbar_inval(&s_bar[0]);
        mbar_inval(&s_bar[1]);
      }
      ok = (!fail && !timed_out && H <= Om) ? 1u : 0u;
      // one packing, two atlases (Sec. 7): contents at least 2 gutter * alpha texels
      // apart stay a whole texel apart at 2^-d when 2 * gutter * omega >= Omega * 2^d
      if (a.lowres_log2 && ((unsigned long long)Om << a.lowres_log2) > 2ull * a.gutter * om) ok = 0u;
    }
  }
  // publish this candidate; the last CTA selects
  if (tid == 0) {
    p.cand[kidx] = PackCand{ok, Om, H, status};
    __threadfence();
    const uint32_t done = atomicAdd(&p.ctr->pack_done, 1u);
    s_last = (done == nblk - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < 32) {
    // candidate kk = lane + 1, lane + 33, ...: the best fitting one, and the error
    // status of the largest kk that reported one
    uint32_t bk = 0, bOm = 0, bH = 0, ek = 0;
    int32_t est = FA_OK;
    for (uint32_t kk = tid + 1; kk <= nblk; kk += 32) {
      const uint4 cv = __ldcg(reinterpret_cast<const uint4*>(p.cand) + (kk - 1));
      if ((int32_t)cv.w != FA_OK) {
        ek = kk;
        est = (int32_t)cv.w;
      }
      if (cv.x && better_cand(kk, cv.y, bk, bOm, a.select_mode)) {
        bk = kk;
        bOm = cv.y;
        bH = cv.z;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t ok2 = __shfl_xor_sync(0xFFFFFFFFu, bk, o), oO = __shfl_xor_sync(0xFFFFFFFFu, bOm, o);
      const uint32_t oH = __shfl_xor_sync(0xFFFFFFFFu, bH, o), oek = __shfl_xor_sync(0xFFFFFFFFu, ek, o);
      const int32_t oest = __shfl_xor_sync(0xFFFFFFFFu, est, o);
      if (better_cand(ok2, oO, bk, bOm, a.select_mode)) {
        bk = ok2;
        bOm = oO;
        bH = oH;
      }
      if (oek > ek) {
        ek = oek;
        est = oest;
      }
    }
    if (tid == 0) {
      int32_t pst = est;
      if (pst == FA_OK && bk == 0) pst = FA_E_PACK_FAILED;
      fa_pack_result r{0, 0, 0, pst, st0 != 0 ? 0u : C};
      if (pst == FA_OK) {
        r.k = bk;
        r.omega = bOm;
        r.height = bH;
      }
      *a.res = r;
      p.ctr->pack_done = 0;
    }
  }
}

// Placements of the selected candidate, in chart order (all CTAs).
__device__ __forceinline__ void pack_place_body(const PackScratch& p, const PackArgs& a, uint32_t bid,
                                                uint32_t nblk) {
  if (__ldcg(&a.res->status) != FA_OK) return;
  const uint32_t C = __ldcg(&a.res->count), kb = __ldcg(&a.res->k) - 1;
  const uint2* bxy = p.xy + (size_t)kb * p.max_boxes;
  const uint2* brec = p.rec8 + (size_t)kb * p.max_chunks * kChunk;
  for (uint32_t i = bid * blockDim.x + threadIdx.x; i < C; i += nblk * blockDim.x) {
    const uint32_t b = __ldcg(a.order + i);
    const uint2 q = __ldcg(bxy + i);
    const uint2 r = __ldcg(brec + i);
    a.place[b] = fa_placement{(int32_t)q.x, (int32_t)q.y, (int32_t)(r.x >> 16), (int32_t)(r.y & 0x7FFFFFFFu)};
  }
}

size_t push_smem_bytes(uint32_t front_cap) { return 2 * (size_t)kStageBytes + (size_t)front_cap * 4; }

// The pack arguments (host side).
inline PackArgs make_pack_args(const fa_ctx* ctx, uint32_t* order, uint32_t atlas_log2, uint32_t n_scales,
                               uint32_t select_mode, uint32_t min_box, uint32_t gutter, uint32_t lowres_log2,
                               fa_placement* place, fa_pack_result* res) {
  PackArgs a;
  a.order = order;
  a.atlas_log2 = atlas_log2;
  a.lowres_log2 = lowres_log2;
  uint32_t sh = 8;
  while ((1u << (sh - 8)) < n_scales) ++sh;
  a.shift = sh;
  a.min_box = min_box;
  a.gutter = gutter;
  a.select_mode = select_mode;
  const uint32_t om = 1u << atlas_log2;
  a.front_cap = (8u * om < kFrontCap) ? 8u * om : kFrontCap;
  a.loop_cap = ctx ? ctx->loop_cap : kLoopCap;
  a.wait_ns = ctx ? ctx->wait_ns : kWaitNs;
  a.place = place;
  a.res = res;
  return a;
}

}  // namespace
}  // namespace pk
}  // namespace fa
