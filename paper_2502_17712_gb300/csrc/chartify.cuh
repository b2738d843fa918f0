// Charts: connected components of the visible triangles (Sec. 5.1) by union-find
// with pointer hooking in the style of ECL-CC (App. A "GPU Union Find", Alg. 1):
// initialise each visible triangle to the smallest visible neighbour, hook roots
// with atomicCAS so the larger root always points to the smaller one, then flatten.
// The root of a component is therefore its smallest triangle id.  Charts are
// numbered by ascending root: the flatten pass counts the roots per 1024-triangle
// block and records each VT word's root bits, a scan gives each block's first chart,
// and a root's chart is that plus the roots before it inside its block.
//
// Edge mode joins triangles across shared edges (the adjacency built at mesh
// registration, plus the incidence lists of non-manifold edges).  Vertex mode
// (the vertex merge of App. A) joins each visible triangle with its three vertices:
// vertices are extra nodes T + v, so every component's smallest node is a triangle.
//
// Visible triangles are found from the VT words: a warp owns 32 consecutive
// triangles and skips the whole word when it is zero.
#pragma once
#include "fa_internal.cuh"

namespace fa {
namespace cf {
namespace {

constexpr int kBlock = 256;
constexpr int kPerBlock = 1024;  // triangles per counting block (4 per thread)

// The representatives of a and of b, walked side by side (each step loads both next
// labels at once) with path halving (labels only decrease: parents are smaller, and
// a label only ever moves to an ancestor).
__device__ __forceinline__ void find_rep2(volatile int32_t* label, int32_t a, int32_t b, int32_t& ra, int32_t& rb) {
  int32_t ca = label[a], cb = label[b], pa = a, pb = b;
  bool wa = ca != a, wb = cb != b;  // still walking
  while (wa || wb) {
    const int32_t na = wa ? label[ca] : ca, nb = wb ? label[cb] : cb;
    if (wa) {
      if (ca > na) {
        label[pa] = na;
        pa = ca;
        ca = na;
      } else {
        wa = false;
      }
    }
    if (wb) {
      if (cb > nb) {
        label[pb] = nb;
        pb = cb;
        cb = nb;
      } else {
        wb = false;
      }
    }
  }
  ra = ca;
  rb = cb;
}

// Root without writing: used once hooking is over.  (Path halving here would race
// with the final store of another thread: a halving write can replace a label that
// was just set to the root by a non-root ancestor.)
__device__ __forceinline__ int32_t find_root(const volatile int32_t* label, int32_t x) {
  int32_t cur = x, next;
  while ((next = label[cur]) != cur) cur = next;
  return cur;
}

// Hook the components of a and b: the larger root is CASed onto the smaller.
__device__ __forceinline__ void unite(int32_t* label, int32_t a, int32_t b, DevCounters* ctr, uint32_t cap) {
  volatile int32_t* vl = label;
  int32_t ra, rb;
  find_rep2(vl, a, b, ra, rb);
  uint32_t guard = 0;
  while (ra != rb) {
    if (++guard > cap) {
      set_status(ctr, FA_E_TIMEOUT);
      return;
    }
    int32_t hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
    int32_t old = atomicCAS(label + hi, hi, lo);
    if (old == hi) return;
    // hi stopped being a root; retry from the current representatives
    find_rep2(vl, old, lo, ra, rb);
  }
}

struct UfArgs {
  const uint32_t* vt;
  const uint32_t* idx;
  const int32_t* adj;
  uint32_t T, V;
  int32_t* label;
  uint2* xedge;    // per tile: the edges (t, n > t) of its visible triangles that leave it
  uint32_t* xcnt;  // per tile: their count
  const uint32_t* tile_list;  // tiles with a visible triangle (count in ctr->n_vtiles)
  DevCounters* ctr;
  uint32_t loop_cap;  // CAS retries of one hooking step before FA_E_TIMEOUT
};

// Union of the edges inside one tile of kTile consecutive triangles, in shared
// memory, then label[t] = the tile-local root (its smallest triangle).  Replaces the
// global init: afterwards every visible triangle points to a root, and only edges that
// leave the tile remain for the global hooking.
constexpr int kTile = 1024;
constexpr uint32_t kXCap = 3 * kTile;  // cross-tile edge slots per tile

__device__ __forceinline__ int32_t lfind(volatile int32_t* lab, int32_t x) {
  int32_t cur = lab[x];
  if (cur != x) {
    int32_t prev = x, next;
    while (cur > (next = lab[cur])) {
      lab[prev] = next;
      prev = cur;
      cur = next;
    }
  }
  return cur;
}

// One tile (all threads of the block; the caller separates tiles by a barrier).
// NT: the threads that take triangles (kTile / NT each); threads past NT of a larger
// block only pass the barriers.
template <int NT>
__device__ __forceinline__ void local_tile(const UfArgs& a, uint32_t tile) {
  static_assert(kTile % NT == 0 && NT >= 32, "whole triangles per thread");
  const bool act = threadIdx.x < (uint32_t)NT;
  __shared__ int32_t lab[kTile];
  __shared__ uint32_t vis[kTile / 32];
  const uint32_t base = tile * kTile;
  uint32_t v = 0;
  if (threadIdx.x < kTile / 32) {
    const uint32_t w = (base >> 5) + threadIdx.x;
    v = w < ((a.T + 31) >> 5) ? __ldcg(a.vt + w) : 0u;
    vis[threadIdx.x] = v;
  }
  __shared__ uint32_t s_xc;
  if (threadIdx.x == 0) s_xc = 0;
  if (!__syncthreads_or(v != 0u)) {  // no visible triangle in this tile
    if (threadIdx.x == 0) a.xcnt[tile] = 0;
    return;
  }
  volatile int32_t* vl = lab;
  uint2* xe = a.xedge + (size_t)tile * kXCap;
  // start from the smallest visible neighbour inside the tile (Alg. 1, first loop)
  int32_t nb[kTile / NT][3];
#pragma unroll
  for (int k = 0; k < kTile / NT; ++k) {
    if (!act) break;
    const uint32_t i = threadIdx.x + k * NT;
    int32_t l = (int32_t)i;
#pragma unroll
    for (int j = 0; j < 3; ++j) nb[k][j] = -1;
    if ((vis[i >> 5] >> (i & 31)) & 1u) {
      const uint32_t t = base + i;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int32_t n = __ldg(a.adj + 3 * (size_t)t + j);
        if (n < (int32_t)base || (uint32_t)n >= base + kTile) {
          // leaves the tile: hooked globally (once, from the lower end) if n is visible
          if (n > (int32_t)t) xe[atomicAdd(&s_xc, 1u)] = make_uint2(t, (uint32_t)n);
          continue;
        }
        const uint32_t ni = (uint32_t)n - base;
        if (!((vis[ni >> 5] >> (ni & 31)) & 1u)) continue;
        nb[k][j] = (int32_t)ni;
        if ((int32_t)ni < l) l = (int32_t)ni;
      }
    }
    lab[i] = l;
  }
  __syncthreads();
  // the initial labels form trees (every label is a smaller visible neighbour); a few
  // rounds of pointer jumping make them shallow before the hooking walks them (a
  // jump only replaces a label by one of its ancestors, so the rounds need no barrier)
#pragma unroll
  for (int k = 0; k < kTile / NT; ++k) {
    if (!act) break;
    const uint32_t i = threadIdx.x + k * NT;
    if (!((vis[i >> 5] >> (i & 31)) & 1u)) continue;
#pragma unroll 1
    for (int r = 0; r < 4; ++r) vl[i] = vl[vl[i]];
  }
  __syncthreads();
  // hook every in-tile edge once, from its lower end
#pragma unroll
  for (int k = 0; k < kTile / NT; ++k) {
    if (!act) break;
    const int32_t i = (int32_t)(threadIdx.x + k * NT);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int32_t ni = nb[k][j];
      if (ni <= i) continue;
      int32_t ra = lfind(vl, i), rb = lfind(vl, ni);
      while (ra != rb) {
        const int32_t hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
        const int32_t old = atomicCAS(lab + hi, hi, lo);
        if (old == hi) break;
        ra = lfind(vl, old);
        rb = lfind(vl, lo);
      }
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; act && i < kTile; i += NT) {
    if (!((vis[i >> 5] >> (i & 31)) & 1u)) continue;
    // (path halving: the walks of other threads shorten too; the result goes to the
    // global labels, so no halving write can overwrite it)
    a.label[base + i] = (int32_t)base + lfind(vl, (int32_t)i);
  }
  if (threadIdx.x == 0) a.xcnt[tile] = s_xc;  // all appends precede the last barrier
}

// Every tile (a block each), or only the tiles that the marking pass listed (a
// persistent grid over the list).
template <bool LIST, int NT>
__device__ __forceinline__ void local_body(const UfArgs& a, uint32_t bid, uint32_t nblk) {
  if (!LIST) {
    const uint32_t ntiles = (a.T + kTile - 1) / kTile;
    for (uint32_t t = bid; t < ntiles; t += nblk) {
      __syncthreads();  // the shared memory of the previous tile is free
      local_tile<NT>(a, t);
    }
    return;
  }
  // the first tile by block index, the others handed out by a counter, so that a
  // block that drew light tiles takes more (their costs differ by an order of
  // magnitude) and the blocks do not all queue on the counter at once
  const uint32_t n = __ldcg(&a.ctr->n_vtiles);
  __shared__ uint32_t s_i;
  for (uint32_t i = bid; i < n;) {
    local_tile<NT>(a, __ldcg(a.tile_list + i));
    __syncthreads();  // the shared memory of this tile is free, and s_i was read
    if (threadIdx.x == 0) s_i = nblk + atomicAdd(&a.ctr->uf_item, 1u);
    __syncthreads();
    i = s_i;
  }
}

__device__ __forceinline__ void init_v_body(int32_t* label, uint32_t T, uint32_t V, uint32_t bid, uint32_t nblk) {
  for (uint32_t v = bid * blockDim.x + threadIdx.x; v < V; v += nblk * blockDim.x)
    label[T + v] = (int32_t)(T + v);
}

// Hooking (Alg. 1, second loop), edge mode: the edges that leave a tile, each once
// from its lower end, when the other end is visible too (edges inside a tile were
// joined by k_uf_local).  One block per tile.
// t0 / nt: this thread's index in the group of threads that hooks the tile, and the
// group's size (the block, or a slice of it).
__device__ __forceinline__ void hook_tile(const UfArgs& a, uint32_t tile, uint32_t t0, uint32_t nt) {
  const uint32_t n = min(__ldcg(a.xcnt + tile), kXCap);
  const uint2* xe = a.xedge + (size_t)tile * kXCap;
  for (uint32_t i = t0; i < n; i += nt) {
    const uint2 e = __ldcg(xe + i);
    if (e.y < a.T && vt_bit(a.vt, e.y)) unite(a.label, (int32_t)e.x, (int32_t)e.y, a.ctr, a.loop_cap);
  }
}

// Each tile is hooked by a group of GT threads (GT divides the block; no barriers),
// so that a large block hooks several tiles at once.
template <bool LIST, uint32_t GT = 0>
__device__ __forceinline__ void hook_body(const UfArgs& a, uint32_t bid, uint32_t nblk) {
  const uint32_t gt = GT ? GT : blockDim.x, per = blockDim.x / gt;
  const uint32_t grp = bid * per + threadIdx.x / gt, ngrp = nblk * per, t0 = threadIdx.x % gt;
  if (!LIST) {
    const uint32_t ntiles = (a.T + kTile - 1) / kTile;
    for (uint32_t t = grp; t < ntiles; t += ngrp) hook_tile(a, t, t0, gt);
    return;
  }
  const uint32_t n = __ldcg(&a.ctr->n_vtiles);
  for (uint32_t i = grp; i < n; i += ngrp) hook_tile(a, __ldcg(a.tile_list + i), t0, gt);
}

// Vertex mode: every visible triangle joins its three vertex nodes T + v.
__device__ __forceinline__ void hook_v_body(const UfArgs& a, uint32_t bid, uint32_t nblk) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwords = (a.T + 31) >> 5;
  for (uint32_t w = (bid * blockDim.x + threadIdx.x) >> 5; w < nwords; w += (nblk * blockDim.x) >> 5) {
    const uint32_t word = __ldcg(a.vt + w);
    if (word == 0) continue;
    const uint32_t t = (w << 5) + lane;
    if (!((word >> lane) & 1u)) continue;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      uint32_t v = __ldg(a.idx + 3 * (size_t)t + j);
      unite(a.label, (int32_t)t, (int32_t)(a.T + v), a.ctr, a.loop_cap);
    }
  }
}

// Non-manifold edges: join consecutive visible triangles of each incidence list.
__device__ __forceinline__ void hook_nm_body(const UfArgs& a, const uint32_t* nm_off, const uint32_t* nm_list,
                                             uint32_t n_nm, uint32_t bid, uint32_t nblk) {
  for (uint32_t e = bid * blockDim.x + threadIdx.x; e < n_nm; e += nblk * blockDim.x) {
    int32_t prev = -1;
    for (uint32_t i = nm_off[e]; i < nm_off[e + 1]; ++i) {
      uint32_t t = nm_list[i];
      if (!vt_bit(a.vt, t)) continue;
      if (prev >= 0 && prev != (int32_t)t) unite(a.label, prev, (int32_t)t, a.ctr, a.loop_cap);
      prev = (int32_t)t;
    }
  }
}

// Flatten visible triangles to their root and count roots per block of
// kPerBlock triangles: with NT threads, warp w of the block owns VT words w, w + NT / 32, ...
template <int NT>
__device__ __forceinline__ void flatten_tile(const UfArgs& a, uint32_t tile, uint32_t* blockcnt,
                                             uint32_t* viscnt, uint2* wordroots) {
  __shared__ uint32_t wc[kPerBlock / 32], vcnt[NT / 32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t nwords = (a.T + 31) >> 5;
  constexpr uint32_t kK = kPerBlock / NT;
  uint32_t vis = 0, rb[kK], words[kK];
  int32_t cur[kK];
  // the thread's kK triangles walk to their roots side by side, one round of
  // independent label loads per step (every label read on the way is an ancestor on
  // the same path: the only writes meanwhile are other walks' compressions to roots)
#pragma unroll
  for (uint32_t k = 0; k < kK; ++k) {
    const uint32_t w = tile * (kPerBlock / 32) + k * (NT / 32) + wid;
    words[k] = w < nwords ? __ldcg(a.vt + w) : 0u;
    vis += __popc(words[k]);
  }
  uint32_t walking = 0;  // bit k: triangle k has not reached its root yet
#pragma unroll
  for (uint32_t k = 0; k < kK; ++k) {
    const uint32_t t = ((tile * (kPerBlock / 32) + k * (NT / 32) + wid) << 5) + lane;
    cur[k] = -1;
    if ((words[k] >> lane) & 1u) {
      cur[k] = __ldcg(a.label + t);
      if (cur[k] != (int32_t)t) walking |= 1u << k;
    }
  }
  while (walking) {
    int32_t nxt[kK];
#pragma unroll
    for (uint32_t k = 0; k < kK; ++k) nxt[k] = (walking >> k) & 1u ? __ldcg(a.label + cur[k]) : cur[k];
#pragma unroll
    for (uint32_t k = 0; k < kK; ++k) {
      if (!((walking >> k) & 1u)) continue;
      if (nxt[k] == cur[k]) walking &= ~(1u << k);
      else cur[k] = nxt[k];
    }
  }
#pragma unroll
  for (uint32_t k = 0; k < kK; ++k) {
    const uint32_t wl = k * (NT / 32) + wid;
    const uint32_t t = ((tile * (kPerBlock / 32) + wl) << 5) + lane;
    bool root = false;
    if ((words[k] >> lane) & 1u) {
      a.label[t] = cur[k];
      root = cur[k] == (int32_t)t;
    }
    rb[k] = __ballot_sync(0xFFFFFFFFu, root);
    if (lane == 0) wc[wl] = __popc(rb[k]);
  }
  if (lane == 0) vcnt[wid] = vis;  // every lane counted the same words
  __syncthreads();
  // the exclusive prefix of the words' root counts (one warp scan)
  if (wid == 0) {
    const uint32_t c = wc[lane];
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= (unsigned)o) x += y;
    }
    wc[lane] = x - c;
    if (lane == 31) {
      uint32_t v = 0;
      for (int i = 0; i < NT / 32; ++i) v += vcnt[i];
      blockcnt[tile] = x;
      viscnt[tile] = v;
    }
  }
  __syncthreads();
  // per VT word: its root bits and the roots of the block's earlier words
#pragma unroll
  for (uint32_t k = 0; k < kPerBlock / NT; ++k) {
    const uint32_t wl = k * (NT / 32) + wid;
    const uint32_t w = tile * (kPerBlock / 32) + wl;
    if (lane == 0 && w < nwords) wordroots[w] = make_uint2(rb[k], wc[wl]);
  }
}

// Every counting block (a block each), or only the tiles that the marking pass
// listed (a persistent grid; the clear zeroed the counts of the others).
template <bool LIST, int NT>
__device__ __forceinline__ void flatten_body(const UfArgs& a, uint32_t* blockcnt, uint32_t* viscnt,
                                             uint2* wordroots, uint32_t bid, uint32_t nblk) {
  const uint32_t n = LIST ? __ldcg(&a.ctr->n_vtiles) : (a.T + kPerBlock - 1) / kPerBlock;
  for (uint32_t i = bid; i < n; i += nblk) {
    __syncthreads();  // the shared memory of the previous tile is free
    flatten_tile<NT>(a, LIST ? __ldcg(a.tile_list + i) : i, blockcnt, viscnt, wordroots);
  }
}

// Chart of root triangle r: the roots before its block (scanned block counts),
// before its word inside the block, and before it inside its word.
__device__ __forceinline__ uint32_t chart_of_root(const uint32_t* blockcnt, const uint2* wordroots, uint32_t r) {
  const uint2 wr = __ldcg(wordroots + (r >> 5));
  return __ldcg(blockcnt + r / kPerBlock) + wr.y + __popc(wr.x & ((1u << (r & 31)) - 1u));
}

// In-place exclusive scans of the per-block counts a[0..n) and, when given,
// b[0..n) (one 1024-thread block, both at once): thread t owns the `per` consecutive
// entries from t per (per a multiple of 4, so whole groups move as 16-byte vectors);
// one block scan of the owners' sums.  The totals go to a[n], b[n], *ta and *tb.
__device__ __forceinline__ uint4 load4(const uint32_t* a, uint32_t i, uint32_t n) {
  if (i + 4u <= n) return __ldcg(reinterpret_cast<const uint4*>(a + i));
  return make_uint4(i < n ? a[i] : 0u, i + 1u < n ? a[i + 1] : 0u, i + 2u < n ? a[i + 2] : 0u,
                    i + 3u < n ? a[i + 3] : 0u);
}
__device__ __forceinline__ void store4(uint32_t* a, uint32_t i, uint32_t n, uint4 v) {
  if (i + 4u <= n) {
    *reinterpret_cast<uint4*>(a + i) = v;
    return;
  }
  if (i < n) a[i] = v.x;
  if (i + 1u < n) a[i + 1] = v.y;
  if (i + 2u < n) a[i + 2] = v.z;
}
__device__ __forceinline__ uint4 excl4(uint4 v, uint32_t& run) {
  const uint4 o = make_uint4(run, run + v.x, run + v.x + v.y, run + v.x + v.y + v.z);
  run += v.x + v.y + v.z + v.w;
  return o;
}
__device__ void scan_counts(uint32_t* a, uint32_t* b, uint32_t n, uint32_t* ta, uint32_t* tb) {
  __shared__ uint2 warp_tot[32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t per = 4u * ((n + 4095u) / 4096u);
  const uint32_t i0 = threadIdx.x * per;
  uint2 v = make_uint2(0u, 0u);
  uint4 a0 = make_uint4(0u, 0u, 0u, 0u), b0 = a0;  // the first group stays in registers
  for (uint32_t i = i0; i < i0 + per && i < n; i += 4u) {
    const uint4 x = load4(a, i, n);
    v.x += x.x + x.y + x.z + x.w;
    if (i == i0) a0 = x;
    if (b) {
      const uint4 y = load4(b, i, n);
      v.y += y.x + y.y + y.z + y.w;
      if (i == i0) b0 = y;
    }
  }
  uint2 x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y0 = __shfl_up_sync(0xFFFFFFFFu, x.x, o), y1 = __shfl_up_sync(0xFFFFFFFFu, x.y, o);
    if (lane >= (unsigned)o) {
      x.x += y0;
      x.y += y1;
    }
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint2 t = warp_tot[threadIdx.x];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y0 = __shfl_up_sync(0xFFFFFFFFu, t.x, o), y1 = __shfl_up_sync(0xFFFFFFFFu, t.y, o);
      if (threadIdx.x >= (unsigned)o) {
        t.x += y0;
        t.y += y1;
      }
    }
    warp_tot[threadIdx.x] = t;
  }
  __syncthreads();
  const uint2 wp = wid ? warp_tot[wid - 1] : make_uint2(0u, 0u);
  uint32_t ra = wp.x + x.x - v.x, rb = wp.y + x.y - v.y;
  for (uint32_t i = i0; i < i0 + per && i < n; i += 4u) {
    store4(a, i, n, excl4(i == i0 ? a0 : load4(a, i, n), ra));
    if (b) store4(b, i, n, excl4(i == i0 ? b0 : load4(b, i, n), rb));
  }
  if (threadIdx.x == 1023) {
    a[n] = wp.x + x.x;
    *ta = wp.x + x.x;
    if (b) {
      b[n] = wp.y + x.y;
      *tb = wp.y + x.y;
    }
  }
  __syncthreads();
}

// Exclusive scans of the per-block root counts (chart numbering) and visible
// counts (the visible-triangle list); writes the chart count.
__device__ __forceinline__ void scan_blocks_body(uint32_t* blockcnt, uint32_t* viscnt, uint32_t nblocks,
                                                 uint32_t* count_out, uint32_t max_charts, DevCounters* ctr) {
  __shared__ uint32_t charts;
  scan_counts(blockcnt, viscnt, nblocks, &charts, &ctr->n_vis);
  if (threadIdx.x == 0) {
    ctr->chart_count = charts;
    *count_out = charts;
    if (charts > max_charts) set_status(ctr, FA_E_CAPACITY);
  }
}

// Scan of the visible counts alone (the standalone box / UV calls).
__device__ __forceinline__ void scan_vis_body(uint32_t* viscnt, uint32_t nblocks, DevCounters* ctr) {
  scan_counts(viscnt, nullptr, nblocks, &ctr->n_vis, nullptr);
}

// The entries of one 1024-triangle block's visible triangles in the list, in
// triangle order: entry = list start of the block + the visible triangles before
// it.  words[k] is VT word k * (NT / 32) + warp of the block.
template <int NT>
__device__ __forceinline__ void put_visible(const uint32_t (&words)[kPerBlock / NT], uint32_t start,
                                            const int32_t (&chart)[kPerBlock / NT], uint2* vis,
                                            uint32_t tile) {
  __shared__ uint32_t wpop[kPerBlock / 32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (uint32_t k = 0; k < kPerBlock / NT; ++k)
    if (lane == 0) wpop[k * (NT / 32) + wid] = __popc(words[k]);
  __syncthreads();
  if (wid == 0) {  // the exclusive prefix of the words' visible counts
    const uint32_t c = wpop[lane];
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= (unsigned)o) x += y;
    }
    wpop[lane] = x - c;
  }
  __syncthreads();
#pragma unroll
  for (uint32_t k = 0; k < kPerBlock / NT; ++k) {
    const uint32_t wl = k * (NT / 32) + wid;
    if (!((words[k] >> lane) & 1u)) continue;
    const uint32_t pre = start + wpop[wl] + __popc(words[k] & ((1u << lane) - 1u));
    const uint32_t t = ((tile * (kPerBlock / 32) + wl) << 5) + lane;
    vis[pre] = make_uint2(t, (uint32_t)chart[k]);
  }
}

// Chart id of every triangle (-1 invisible; charts numbered by ascending root) and
// the visible-triangle list (same blocking as k_uf_flatten); each root records
// itself as its chart's root and resets the chart's box accumulators.
template <int NT>
__device__ __forceinline__ void chart_tile(const UfArgs& a, uint32_t tile, const uint32_t* blockcnt,
                                           const uint2* wordroots, int32_t* tri_chart, uint32_t* roots,
                                           uint32_t* box_enc, uint32_t* box_full, uint32_t max_charts,
                                           const uint32_t* visstart, uint2* vis) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t nwords = (a.T + 31) >> 5;
  constexpr uint32_t kK = kPerBlock / NT;
  uint32_t words[kK], rt[kK];
  int32_t chart[kK];
  // the loads of the thread's kK triangles in rounds (VT words, roots, the roots'
  // counts), each round independent, before any store
#pragma unroll
  for (uint32_t k = 0; k < kK; ++k) {
    const uint32_t w = tile * (kPerBlock / 32) + k * (NT / 32) + wid;
    words[k] = w < nwords ? __ldcg(a.vt + w) : 0u;
  }
#pragma unroll
  for (uint32_t k = 0; k < kK; ++k) {
    const uint32_t t = ((tile * (kPerBlock / 32) + k * (NT / 32) + wid) << 5) + lane;
    rt[k] = (words[k] >> lane) & 1u ? (uint32_t)__ldcg(a.label + t) : 0u;
  }
#pragma unroll
  for (uint32_t k = 0; k < kK; ++k)
    chart[k] = (words[k] >> lane) & 1u ? (int32_t)chart_of_root(blockcnt, wordroots, rt[k]) : -1;
#pragma unroll
  for (uint32_t k = 0; k < kK; ++k) {
    const uint32_t w = tile * (kPerBlock / 32) + k * (NT / 32) + wid;
    const uint32_t t = (w << 5) + lane;
    if (chart[k] >= 0 && rt[k] == t && (uint32_t)chart[k] < max_charts) {
      const uint32_t c = (uint32_t)chart[k];
      roots[c] = t;
      reinterpret_cast<uint4*>(box_enc)[c] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
      box_full[c] = 0u;
    }
    if (w < nwords && t < a.T) tri_chart[t] = chart[k];
  }
  put_visible<NT>(words, __ldcg(visstart + tile), chart, vis, tile);
}

// Every counting block (a block each; invisible triangles get -1), or, when the
// raster front end already set tri_chart to -1, only the listed tiles (a persistent
// grid over the list).
template <bool LIST, int NT>
__device__ __forceinline__ void tri_chart_body(const UfArgs& a, const uint32_t* blockcnt, const uint2* wordroots,
                                               int32_t* tri_chart, uint32_t* roots, uint32_t* box_enc,
                                               uint32_t* box_full, uint32_t max_charts, const uint32_t* visstart,
                                               uint2* vis, uint32_t bid, uint32_t nblk) {
  __shared__ int32_t s_status;
  if (threadIdx.x == 0) s_status = __ldcg(&a.ctr->status);
  __syncthreads();
  if (s_status != 0) return;
  const uint32_t n = LIST ? __ldcg(&a.ctr->n_vtiles) : (a.T + kPerBlock - 1) / kPerBlock;
  for (uint32_t i = bid; i < n; i += nblk) {
    __syncthreads();  // the shared memory of the previous tile is free
    chart_tile<NT>(a, LIST ? __ldcg(a.tile_list + i) : i, blockcnt, wordroots, tri_chart, roots, box_enc, box_full,
                   max_charts, visstart, vis);
  }
}

__device__ __forceinline__ void vert_chart_body(const UfArgs& a, const uint32_t* blockcnt, const uint2* wordroots,
                                                int32_t* vert_chart, int vertex_mode, uint32_t bid, uint32_t nblk) {
  if (__ldcg(&a.ctr->status) != 0) return;
  for (uint32_t v = bid * blockDim.x + threadIdx.x; v < a.V; v += nblk * blockDim.x) {
    int32_t out = -1;
    if (vertex_mode) {
      int32_t r = find_root(a.label, (int32_t)(a.T + v));
      if (r < (int32_t)a.T) out = (int32_t)chart_of_root(blockcnt, wordroots, (uint32_t)r);
    }
    vert_chart[v] = out;
  }
}

// The union-find arguments of one chart pass on ctx (host side).
inline UfArgs make_uf_args(fa_ctx* ctx, const fa_mesh* mesh, const uint32_t* vt) {
  UfArgs a;
  a.vt = vt;
  a.idx = mesh->idx;
  a.adj = mesh->adj;
  a.T = mesh->T;
  a.V = mesh->V;
  a.label = ctx->label;
  a.xedge = ctx->xedge;
  a.xcnt = ctx->xcnt;
  a.tile_list = ctx->tile_list;
  a.ctr = ctx->ctr;
  a.loop_cap = ctx->loop_cap;
  return a;
}

}  // namespace
}  // namespace cf
}  // namespace fa
