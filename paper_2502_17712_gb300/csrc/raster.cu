// Visibility: depth pre-pass and "<=" marking pass (Sec. 5.1; App. A "Detecting
// Visible Triangles") as a software rasterizer.
//
// Per triangle (one thread, warps over 32 consecutive triangles so that the
// visible bits of a warp form one VT word):
//   transform (pinned fp32) -> trivial reject when all three vertices are outside
//   one side plane or behind the near plane -> Sutherland-Hodgman against the
//   near plane and the guard band |x|,|y| <= 64 w, only when a vertex is outside
//   -> project, snap to 1/256 px (round half even) -> fan sub-triangles -> cull
//   A <= 0 -> pixel-centre samples with the top-left rule -> z/w interpolated by
//   ((E0 z0 + E1 z1) + E2 z2) * (1/A), kept when -1 <= d <= 1.
// Sub-triangles whose clamped pixel box has more than kSmallMaxPix pixels are
// queued (pass 0) and rasterized by a warp per 16x16 tile in a second kernel.
#include "fa_internal.cuh"

namespace fa {
namespace {

struct CV {
  float x, y, z, w;
};

struct SV {
  int64_t X, Y;
  float zn;
};

__device__ __forceinline__ float plane_dist(const CV& c, int pl) {
  switch (pl) {
    case 0: return __fadd_rn(c.z, c.w);
    case 1: return __fsub_rn(__fmul_rn(kGuard, c.w), c.x);
    case 2: return __fadd_rn(__fmul_rn(kGuard, c.w), c.x);
    case 3: return __fsub_rn(__fmul_rn(kGuard, c.w), c.y);
    default: return __fadd_rn(__fmul_rn(kGuard, c.w), c.y);
  }
}

__device__ __forceinline__ CV intersect(const CV& a, const CV& b, float da, float db) {
  float t = __fdiv_rn(da, __fsub_rn(da, db));
  CV r;
  r.x = __fadd_rn(a.x, __fmul_rn(t, __fsub_rn(b.x, a.x)));
  r.y = __fadd_rn(a.y, __fmul_rn(t, __fsub_rn(b.y, a.y)));
  r.z = __fadd_rn(a.z, __fmul_rn(t, __fsub_rn(b.z, a.z)));
  r.w = __fadd_rn(a.w, __fmul_rn(t, __fsub_rn(b.w, a.w)));
  return r;
}

constexpr int kMaxPoly = 16;

// Full Sutherland-Hodgman sequence (near, then the four guard planes).  A convex
// triangle gains at most one vertex per plane (<= 8); rounding on nearly
// plane-aligned input could add more, so the buffer holds kMaxPoly and an overflow
// is reported (returns -1) instead of being truncated.
__device__ __forceinline__ int clip_polygon(CV* poly, int n) {
  CV tmp[kMaxPoly];
  for (int pl = 0; pl < 5 && n >= 3; ++pl) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
      const CV c = poly[i];
      const CV nx = poly[(i + 1) % n];
      float dc = plane_dist(c, pl), dn = plane_dist(nx, pl);
      bool ic = dc >= 0.0f, in_ = dn >= 0.0f;
      if (m + 2 > kMaxPoly) return -1;
      if (ic) tmp[m++] = c;
      if (ic != in_) tmp[m++] = ic ? intersect(c, nx, dc, dn) : intersect(nx, c, dn, dc);
    }
    for (int i = 0; i < m; ++i) poly[i] = tmp[i];
    n = m;
  }
  return n;
}

__device__ __forceinline__ SV project(const CV& c, float hx, float hy) {
  float nx = __fdiv_rn(c.x, c.w), ny = __fdiv_rn(c.y, c.w), zn = __fdiv_rn(c.z, c.w);
  float xs = __fmul_rn(__fadd_rn(nx, 1.0f), hx);
  float ys = __fmul_rn(__fadd_rn(ny, 1.0f), hy);
  SV s;
  s.X = __float2ll_rn(__fmul_rn(xs, 256.0f));
  s.Y = __float2ll_rn(__fmul_rn(ys, 256.0f));
  s.zn = zn;
  return s;
}

__device__ __forceinline__ bool top_left(int64_t ax, int64_t ay, int64_t bx, int64_t by) {
  int64_t dx = bx - ax, dy = by - ay;
  return dy < 0 || (dy == 0 && dx < 0);
}

// Setup of one sub-triangle: area, 1/A, clamped pixel box.
struct Setup {
  int64_t A;
  int px0, py0, px1, py1;
};

__device__ __forceinline__ Setup setup(const SV& a, const SV& b, const SV& c, int W, int H) {
  Setup s;
  s.A = (b.X - a.X) * (c.Y - a.Y) - (c.X - a.X) * (b.Y - a.Y);
  int64_t xmn = min(a.X, min(b.X, c.X)), xmx = max(a.X, max(b.X, c.X));
  int64_t ymn = min(a.Y, min(b.Y, c.Y)), ymx = max(a.Y, max(b.Y, c.Y));
  // first / last pixel whose centre 256 p + 128 lies in [min, max]
  int64_t px0 = -((128 - xmn) >> 8), px1 = (xmx - 128) >> 8;
  int64_t py0 = -((128 - ymn) >> 8), py1 = (ymx - 128) >> 8;
  s.px0 = (int)(px0 > 0 ? px0 : 0);
  s.py0 = (int)(py0 > 0 ? py0 : 0);
  s.px1 = (int)(px1 < W - 1 ? px1 : W - 1);
  s.py1 = (int)(py1 < H - 1 ? py1 : H - 1);
  return s;
}

// Visit covered samples of a sub-triangle over pixel rect [px0..px1] x [py0..py1].
// PASS 0: atomicMin the depth key.  PASS 1: return true on the first sample whose
// key <= zbuf.
template <int PASS>
__device__ bool raster_rect(const SV& a, const SV& b, const SV& c, float invA, int px0, int py0,
                            int px1, int py1, uint32_t* __restrict__ zbuf, int W) {
  const bool tl0 = top_left(b.X, b.Y, c.X, c.Y);
  const bool tl1 = top_left(c.X, c.Y, a.X, a.Y);
  const bool tl2 = top_left(a.X, a.Y, b.X, b.Y);
  for (int py = py0; py <= py1; ++py) {
    const int64_t sy = (int64_t)py * 256 + 128;
    for (int px = px0; px <= px1; ++px) {
      const int64_t sx = (int64_t)px * 256 + 128;
      int64_t e0 = (c.X - b.X) * (sy - b.Y) - (c.Y - b.Y) * (sx - b.X);
      int64_t e1 = (a.X - c.X) * (sy - c.Y) - (a.Y - c.Y) * (sx - c.X);
      int64_t e2 = (b.X - a.X) * (sy - a.Y) - (b.Y - a.Y) * (sx - a.X);
      bool in = (e0 > 0 || (e0 == 0 && tl0)) && (e1 > 0 || (e1 == 0 && tl1)) &&
                (e2 > 0 || (e2 == 0 && tl2));
      if (!in) continue;
      float s = __fmul_rn(__ll2float_rn(e0), a.zn);
      s = __fadd_rn(s, __fmul_rn(__ll2float_rn(e1), b.zn));
      s = __fadd_rn(s, __fmul_rn(__ll2float_rn(e2), c.zn));
      float d = __fmul_rn(s, invA);
      if (!(d >= -1.0f && d <= 1.0f)) continue;
      uint32_t key = ordered(d);
      uint32_t* z = zbuf + (size_t)py * W + px;
      if (PASS == 0) {
        if (key < *z) atomicMin(z, key);
      } else {
        if (key <= __ldcg(z)) return true;
      }
    }
  }
  return false;
}

struct RasterArgs {
  Mat4 M;
  const float* pos;
  const uint32_t* idx;
  uint32_t T;
  int W, H;
  float hx, hy;
  uint32_t* zbuf;
  uint32_t* bigbits;
  BigTri* queue;
  uint32_t queue_cap;
  uint32_t* tile_owner;  // queue record of each reserved tile
  uint32_t tile_cap;
  DevCounters* ctr;
  uint32_t* vt;
};

// Rasterize the fan (sv[0], sv[i], sv[i+1]) of one mesh triangle t.
// PASS 0: depth pre-pass; returns whether the sub-triangles went to the big queue.
// PASS 1: marking pass of a triangle not in the queue; returns visibility.
template <int PASS>
__device__ bool raster_fan(const RasterArgs& A, uint32_t t, const SV* sv, int n) {
  if (PASS == 0) {
    int nq = 0;
    uint64_t tiles = 0;
    bool big = false;
    for (int i = 1; i + 1 < n; ++i) {
      Setup s = setup(sv[0], sv[i], sv[i + 1], A.W, A.H);
      if (s.A <= 0 || s.px1 < s.px0 || s.py1 < s.py0) continue;
      int w = s.px1 - s.px0 + 1, h = s.py1 - s.py0 + 1;
      if (w * h > kSmallMaxPix) big = true;
      ++nq;
      tiles += (uint64_t)((w + kBigTile - 1) / kBigTile) * (uint64_t)((h + kBigTile - 1) / kBigTile);
    }
    if (big) {
      unsigned long long old =
          atomicAdd(&A.ctr->big, ((unsigned long long)nq << 40) | (unsigned long long)tiles);
      uint64_t e0 = old >> 40, tile = old & ((1ull << 40) - 1);
      if (e0 + nq <= A.queue_cap && tile + tiles <= A.tile_cap) {
        int q = 0;
        for (int i = 1; i + 1 < n; ++i) {
          Setup s = setup(sv[0], sv[i], sv[i + 1], A.W, A.H);
          if (s.A <= 0 || s.px1 < s.px0 || s.py1 < s.py0) continue;
          BigTri bt;
          bt.X[0] = (int32_t)sv[0].X; bt.X[1] = (int32_t)sv[i].X; bt.X[2] = (int32_t)sv[i + 1].X;
          bt.Y[0] = (int32_t)sv[0].Y; bt.Y[1] = (int32_t)sv[i].Y; bt.Y[2] = (int32_t)sv[i + 1].Y;
          bt.zn[0] = sv[0].zn; bt.zn[1] = sv[i].zn; bt.zn[2] = sv[i + 1].zn;
          bt.px0 = s.px0; bt.py0 = s.py0; bt.px1 = s.px1; bt.py1 = s.py1;
          bt.tri = t;
          bt.tile0 = (uint32_t)tile;
          bt.pad = 0;
          A.queue[e0 + q] = bt;
          const int w = s.px1 - s.px0 + 1, h = s.py1 - s.py0 + 1;
          const uint64_t nt = (uint64_t)((w + kBigTile - 1) / kBigTile) * (uint64_t)((h + kBigTile - 1) / kBigTile);
          for (uint64_t j = 0; j < nt; ++j) A.tile_owner[tile + j] = (uint32_t)(e0 + q);
          tile += nt;
          ++q;
        }
        return true;
      }
      // queue or tile table full: reserved records become empty, reserved tiles get
      // no owner, and the triangle is rasterized here instead
      for (uint64_t e = e0; e < e0 + nq && e < A.queue_cap; ++e) {
        BigTri bt = {};
        bt.px0 = 1; bt.px1 = 0; bt.py0 = 1; bt.py1 = 0;
        bt.tile0 = (uint32_t)tile;
        A.queue[e] = bt;
      }
      for (uint64_t j = tile; j < tile + tiles && j < A.tile_cap; ++j) A.tile_owner[j] = 0xFFFFFFFFu;
    }
  }
  for (int i = 1; i + 1 < n; ++i) {
    Setup s = setup(sv[0], sv[i], sv[i + 1], A.W, A.H);
    if (s.A <= 0 || s.px1 < s.px0 || s.py1 < s.py0) continue;
    float invA = __fdiv_rn(1.0f, __ll2float_rn(s.A));
    if (raster_rect<PASS>(sv[0], sv[i], sv[i + 1], invA, s.px0, s.py0, s.px1, s.py1, A.zbuf, A.W))
      return true;
  }
  return false;
}

// Triangles that cross the near plane or the guard band (rare): clip first.
template <int PASS>
__device__ __noinline__ bool raster_clipped(const RasterArgs& A, uint32_t t, float4 c0, float4 c1,
                                            float4 c2) {
  CV poly[kMaxPoly];
  poly[0] = CV{c0.x, c0.y, c0.z, c0.w};
  poly[1] = CV{c1.x, c1.y, c1.z, c1.w};
  poly[2] = CV{c2.x, c2.y, c2.z, c2.w};
  int n = clip_polygon(poly, 3);
  if (n < 0) {
    set_status(A.ctr, FA_E_CAPACITY);
    return false;
  }
  if (n < 3) return false;
  for (int i = 0; i < n; ++i)
    if (!(poly[i].w > 0.0f)) return false;
  SV sv[kMaxPoly];
  for (int i = 0; i < n; ++i) sv[i] = project(poly[i], A.hx, A.hy);
  return raster_fan<PASS>(A, t, sv, n);
}

// Returns: PASS 0 -> whether the triangle went to the big queue;
//          PASS 1 -> whether an in-thread sample passed the depth test.
template <int PASS>
__device__ bool raster_triangle(const RasterArgs& A, uint32_t t) {
  const uint32_t* f = A.idx + 3 * (size_t)t;
  const uint32_t i0 = __ldg(f), i1 = __ldg(f + 1), i2 = __ldg(f + 2);
  float4 c0 = load_clip(A.M, A.pos, i0), c1 = load_clip(A.M, A.pos, i1), c2 = load_clip(A.M, A.pos, i2);
  // trivial reject: all vertices outside one side plane, or all behind the near plane
  // (no sample can be covered then: see the design notes on exactness)
  if ((c0.x > c0.w && c1.x > c1.w && c2.x > c2.w) || (c0.x < -c0.w && c1.x < -c1.w && c2.x < -c2.w) ||
      (c0.y > c0.w && c1.y > c1.w && c2.y > c2.w) || (c0.y < -c0.w && c1.y < -c1.w && c2.y < -c2.w) ||
      (__fadd_rn(c0.z, c0.w) < 0.0f && __fadd_rn(c1.z, c1.w) < 0.0f && __fadd_rn(c2.z, c2.w) < 0.0f))
    return false;
  const CV v0{c0.x, c0.y, c0.z, c0.w}, v1{c1.x, c1.y, c1.z, c1.w}, v2{c2.x, c2.y, c2.z, c2.w};
  bool outside = false;
#pragma unroll
  for (int pl = 0; pl < 5; ++pl)
    outside |= !(plane_dist(v0, pl) >= 0.0f) || !(plane_dist(v1, pl) >= 0.0f) ||
               !(plane_dist(v2, pl) >= 0.0f);
  if (outside) return raster_clipped<PASS>(A, t, c0, c1, c2);
  if (!(v0.w > 0.0f) || !(v1.w > 0.0f) || !(v2.w > 0.0f)) return false;
  SV sv[3] = {project(v0, A.hx, A.hy), project(v1, A.hx, A.hy), project(v2, A.hx, A.hy)};
  return raster_fan<PASS>(A, t, sv, 3);
}

__global__ void k_clear(uint32_t* __restrict__ zbuf, uint32_t n, DevCounters* ctr, int reset_status) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctr->big = 0ull;
    if (reset_status) ctr->status = 0;
  }
  uint4* z4 = reinterpret_cast<uint4*>(zbuf);
  const uint4 ff = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
  uint32_t n4 = n / 4;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) z4[i] = ff;
  for (uint32_t i = n4 * 4 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    zbuf[i] = 0xFFFFFFFFu;
}

// Small-triangle pass: warp w handles triangles [32 w', 32 w' + 32) for w' = w,
// w + nwarps, ...  PASS 0 writes the big-queue bits, PASS 1 the VT words.
template <int PASS>
__global__ void __launch_bounds__(256) k_raster(RasterArgs A) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t nwords = (A.T + 31) >> 5;
  if (PASS == 1 && __ldcg(&A.ctr->status) != 0) {
    for (uint32_t w = warp; w < nwords; w += nwarps)
      if (lane == 0) A.vt[w] = 0u;
    return;
  }
  for (uint32_t w = warp; w < nwords; w += nwarps) {
    const uint32_t t = (w << 5) + lane;
    bool flag = false;
    if (t < A.T) {
      if (PASS == 0) {
        flag = raster_triangle<0>(A, t);
      } else {
        const bool big = (__ldg(A.bigbits + w) >> lane) & 1u;
        if (!big) flag = raster_triangle<1>(A, t);
      }
    }
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, flag);
    if (lane == 0) {
      if (PASS == 0) A.bigbits[w] = bits;
      else A.vt[w] = bits;
    }
  }
}

// Large sub-triangles: one warp per 16x16 tile of a queued record.
template <int PASS>
__global__ void __launch_bounds__(256) k_raster_big(RasterArgs A) {
  if (PASS == 1 && __ldcg(&A.ctr->status) != 0) return;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const unsigned long long st = __ldcg(&A.ctr->big);
  const uint64_t n_ent = (st >> 40) < A.queue_cap ? (st >> 40) : A.queue_cap;
  const uint64_t n_tiles = st & ((1ull << 40) - 1);
  if (n_ent == 0) return;
  const uint64_t n_used = n_tiles < A.tile_cap ? n_tiles : A.tile_cap;
  for (uint64_t g = warp; g < n_used; g += nwarps) {
    const uint32_t lo = __ldg(A.tile_owner + g);
    if (lo >= n_ent) continue;
    const BigTri& q = A.queue[lo];
    const int px0 = q.px0, py0 = q.py0, px1 = q.px1, py1 = q.py1;
    if (px1 < px0 || py1 < py0) continue;
    const uint32_t tx_n = (uint32_t)((px1 - px0 + kBigTile) / kBigTile);
    const uint32_t ty_n = (uint32_t)((py1 - py0 + kBigTile) / kBigTile);
    const uint64_t local = g - q.tile0;
    if (local >= (uint64_t)tx_n * ty_n) continue;
    const int bx = px0 + (int)(local % tx_n) * kBigTile, by = py0 + (int)(local / tx_n) * kBigTile;
    SV a{q.X[0], q.Y[0], q.zn[0]}, b{q.X[1], q.Y[1], q.zn[1]}, c{q.X[2], q.Y[2], q.zn[2]};
    const int64_t Ar = (b.X - a.X) * (c.Y - a.Y) - (c.X - a.X) * (b.Y - a.Y);
    const float invA = __fdiv_rn(1.0f, __ll2float_rn(Ar));
    bool vis = false;
#pragma unroll 1
    for (int j = lane; j < kBigTile * kBigTile; j += 32) {
      const int px = bx + (j % kBigTile), py = by + (j / kBigTile);
      if (px > px1 || py > py1) continue;
      vis |= raster_rect<PASS>(a, b, c, invA, px, py, px, py, A.zbuf, A.W);
    }
    if (PASS == 1) {
      if (__any_sync(0xFFFFFFFFu, vis) && lane == 0) atomicOr(A.vt + (q.tri >> 5), 1u << (q.tri & 31));
    }
  }
}

}  // namespace

fa_status launch_visibility(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W, uint32_t H,
                            uint32_t* vt, cudaStream_t s) {
  RasterArgs A;
  A.M = M;
  A.pos = mesh->pos;
  A.idx = mesh->idx;
  A.T = mesh->T;
  A.W = (int)W;
  A.H = (int)H;
  A.hx = 0.5f * (float)W;
  A.hy = 0.5f * (float)H;
  A.zbuf = ctx->zbuf;
  A.bigbits = ctx->bigbits;
  A.queue = ctx->queue;
  A.queue_cap = ctx->queue_cap;
  A.tile_owner = ctx->tile_owner;
  A.tile_cap = ctx->tile_cap;
  A.ctr = ctx->ctr;
  A.vt = vt;
  const uint32_t npix = W * H;
  mark(ctx, "k_clear", s);
  k_clear<<<grid_for(npix / 4 + 1, 256, 152 * 4), 256, 0, s>>>(ctx->zbuf, npix, ctx->ctr, 0);
  const uint32_t nwords = (mesh->T + 31) / 32;
  const unsigned g = grid_for((uint64_t)nwords * 32, 256, 152 * 16);
  const unsigned gb = 152 * 8;
  mark(ctx, "k_raster_depth", s);
  k_raster<0><<<g, 256, 0, s>>>(A);
  mark(ctx, "k_raster_depth_big", s);
  k_raster_big<0><<<gb, 256, 0, s>>>(A);
  mark(ctx, "k_raster_mark", s);
  k_raster<1><<<g, 256, 0, s>>>(A);
  mark(ctx, "k_raster_mark_big", s);
  k_raster_big<1><<<gb, 256, 0, s>>>(A);
  FA_CUDA_TRY(cudaGetLastError());
  return FA_OK;
}

}  // namespace fa
