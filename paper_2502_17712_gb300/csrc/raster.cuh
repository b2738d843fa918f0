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
//
// Kernels: k_raster_front (the per-triangle front end above; it also clears the
// per-frame state for the kernels after it), k_raster_exact (the exact set-up of
// the survivors; small sub-triangles rasterized in-thread, or by a group of 16
// lanes each when the survivors are few for the grid, a 48-byte record kept for the
// marking pass), k_raster_depth_big (the queued tiles) and k_raster_mark (the queued
// tiles, then the records, grouped in the same way; it also lists the 1024-triangle
// tiles that hold a visible triangle for the chart passes).  Edge values that stay
// below 2^24 over a box are stepped as exact fp32 integers.
#pragma once
#include "fa_internal.cuh"

namespace fa {
namespace rs {
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
  // |xs * 256| < 2^28 inside the guard band |x|, |y| <= 64 w, so the rounded value
  // fits an int32 (and the 32-bit conversion avoids the fp64 units)
  s.X = __float2int_rn(__fmul_rn(xs, 256.0f));
  s.Y = __float2int_rn(__fmul_rn(ys, 256.0f));
  s.zn = zn;
  return s;
}


// Setup of one sub-triangle: area, 1/A, clamped pixel box.
struct Setup {
  int64_t A;
  int px0, py0, px1, py1;
};

__device__ __forceinline__ Setup setup(const SV& a, const SV& b, const SV& c, int W, int H, bool cons) {
  Setup s;
  s.A = (b.X - a.X) * (c.Y - a.Y) - (c.X - a.X) * (b.Y - a.Y);
  int64_t xmn = min(a.X, min(b.X, c.X)), xmx = max(a.X, max(b.X, c.X));
  int64_t ymn = min(a.Y, min(b.Y, c.Y)), ymx = max(a.Y, max(b.Y, c.Y));
  // sample rule: first / last pixel whose centre 256 p + 128 lies in [min, max];
  // conservative marking: first / last pixel whose square [256 p, 256 p + 256] meets it
  int64_t px0 = -((128 - xmn) >> 8), px1 = (xmx - 128) >> 8;
  int64_t py0 = -((128 - ymn) >> 8), py1 = (ymx - 128) >> 8;
  if (cons) {
    px0 = -((-xmn) >> 8) - 1;
    px1 = xmx >> 8;
    py0 = -((-ymn) >> 8) - 1;
    py1 = ymx >> 8;
  }
  s.px0 = (int)(px0 > 0 ? px0 : 0);
  s.py0 = (int)(py0 > 0 ? py0 : 0);
  s.px1 = (int)(px1 < W - 1 ? px1 : W - 1);
  s.py1 = (int)(py1 < H - 1 ? py1 : H - 1);
  return s;
}

// Edge functions of a sub-triangle at the sample of pixel (px, py) and their steps
// per pixel in x and y (exact int64; E is affine in the sample position).
struct Edges {
  int64_t e[3];   // E0 (edge b->c), E1 (c->a), E2 (a->b) at the sample
  int64_t dx[3];  // change per +1 pixel in x
  int64_t dy[3];  // change per +1 pixel in y
  bool tl[3];
};

__device__ __forceinline__ Edges edges_at(const SV& a, const SV& b, const SV& c, int px, int py) {
  Edges E;
  const int64_t sx = (int64_t)px * 256 + 128, sy = (int64_t)py * 256 + 128;
  const SV* v0[3] = {&b, &c, &a};
  const SV* v1[3] = {&c, &a, &b};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int64_t ex = v1[i]->X - v0[i]->X, ey = v1[i]->Y - v0[i]->Y;
    E.e[i] = ex * (sy - v0[i]->Y) - ey * (sx - v0[i]->X);
    E.dx[i] = -ey * 256;
    E.dy[i] = ex * 256;
    E.tl[i] = ey < 0 || (ey == 0 && ex < 0);
  }
  return E;
}

// Test and shade one pixel with edge values e at its sample.  PASS 0: covered (top-
// left rule) with a depth in [-1, 1]: atomicMin the depth key.  PASS 1: the same
// test, return key <= zbuf.  PASS 2 (conservative marking, App. A): the pixel's
// closed square meets the closed triangle (each edge function is >= 0 at the
// square corner where it is largest: e + (|dx| + |dy|) / 2, a half pixel each way);
// the depth is the sample's where the sample rule covers the centre, else the plane
// at the centre clamped to [zmin, zmax]; return key <= zbuf when it is in [-1, 1].
template <int PASS>
__device__ __forceinline__ bool sample(const Edges& E, const int64_t* e, const SV& a, const SV& b, const SV& c,
                                       float invA, uint32_t* __restrict__ z, float zmin = 0.0f,
                                       float zmax = 0.0f) {
  const bool in = (e[0] > 0 || (e[0] == 0 && E.tl[0])) && (e[1] > 0 || (e[1] == 0 && E.tl[1])) &&
                  (e[2] > 0 || (e[2] == 0 && E.tl[2]));
  if (PASS == 2) {
    bool meets = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t ax = E.dx[i] < 0 ? -E.dx[i] : E.dx[i], ay = E.dy[i] < 0 ? -E.dy[i] : E.dy[i];
      meets = meets && (e[i] + ((ax + ay) >> 1) >= 0);
    }
    if (!meets) return false;
  } else if (!in) {
    return false;
  }
  float s = __fmul_rn(ll2float_rn(e[0]), a.zn);
  s = __fadd_rn(s, __fmul_rn(ll2float_rn(e[1]), b.zn));
  s = __fadd_rn(s, __fmul_rn(ll2float_rn(e[2]), c.zn));
  float d = __fmul_rn(s, invA);
  if (PASS == 2 && !in) d = fminf(fmaxf(d, zmin), zmax);
  if (!(d >= -1.0f && d <= 1.0f)) return false;
  const uint32_t key = ordered(d);
  if (PASS == 0) {
    atomicMin(z, key);  // result unused: a fire-and-forget reduction
    return false;
  }
  return key <= __ldcg(z);
}

// Visit the samples of a sub-triangle over pixel rect [px0..px1] x [py0..py1],
// stepping the edge functions.  PASS 1 returns true at the first visible sample.
// sample() on edge values held exactly as floats (integers below 2^24), PASS 0 or 1.
template <int PASS>
__device__ __forceinline__ bool sample_f(float e0, float e1, float e2, const bool* tl, float z0, float z1,
                                         float z2, float invA, uint32_t* __restrict__ z) {
  const bool in = (e0 > 0.0f || (e0 == 0.0f && tl[0])) && (e1 > 0.0f || (e1 == 0.0f && tl[1])) &&
                  (e2 > 0.0f || (e2 == 0.0f && tl[2]));
  if (!in) return false;
  float s = __fmul_rn(e0, z0);
  s = __fadd_rn(s, __fmul_rn(e1, z1));
  s = __fadd_rn(s, __fmul_rn(e2, z2));
  const float d = __fmul_rn(s, invA);
  if (!(d >= -1.0f && d <= 1.0f)) return false;
  const uint32_t key = ordered(d);
  if (PASS == 0) {
    atomicMin(z, key);  // result unused: a fire-and-forget reduction
    return false;
  }
  return key <= __ldcg(z);
}

// raster_rect for boxes whose edge values all stay below 2^24 in magnitude (checked
// by the caller): those integers are exact in fp32, so the edge functions are kept
// and stepped as floats (every sum is again such an integer, hence exact), the
// coverage tests compare the same values and the depth multiplies the same
// correctly rounded conversions as sample() does: the same samples and keys, with
// no 64-bit arithmetic or conversion per sample.  PASS 0 or 1.
template <int PASS>
__device__ __forceinline__ bool raster_rect_f32(const Edges& E, const SV& a, const SV& b, const SV& c, float invA,
                                                int px0, int py0, int px1, int py1, uint32_t* __restrict__ zbuf,
                                                int W) {
  float er[3], fdx[3], fdy[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    er[i] = (float)(int32_t)E.e[i];
    fdx[i] = (float)(int32_t)E.dx[i];
    fdy[i] = (float)(int32_t)E.dy[i];
  }
  bool vis = false;  // PASS 1 stops at the first sample that passes the depth test
  for (int py = py0; py <= py1; ++py) {
    float e0 = er[0], e1 = er[1], e2 = er[2];
    uint32_t* zrow = zbuf + (size_t)py * W;
#pragma unroll 2
    for (int px = px0; px <= px1; ++px) {
      vis |= sample_f<PASS>(e0, e1, e2, E.tl, a.zn, b.zn, c.zn, invA, zrow + px);
      if (PASS == 1 && vis) break;
      e0 = __fadd_rn(e0, fdx[0]);
      e1 = __fadd_rn(e1, fdx[1]);
      e2 = __fadd_rn(e2, fdx[2]);
    }
    if (PASS == 1 && vis) break;
    er[0] = __fadd_rn(er[0], fdy[0]);
    er[1] = __fadd_rn(er[1], fdy[1]);
    er[2] = __fadd_rn(er[2], fdy[2]);
  }
  return vis;
}

template <int PASS>
__device__ bool raster_rect(const SV& a, const SV& b, const SV& c, float invA, int px0, int py0,
                            int px1, int py1, uint32_t* __restrict__ zbuf, int W) {
  const Edges E = edges_at(a, b, c, px0, py0);
  if (PASS != 2 && px1 >= px0 && py1 >= py0) {
    // |E| over the box <= |E(px0, py0)| + |dx| (px1 - px0) + |dy| (py1 - py0)
    bool small = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t ax = E.dx[i] < 0 ? -E.dx[i] : E.dx[i], ay = E.dy[i] < 0 ? -E.dy[i] : E.dy[i];
      const int64_t ae = E.e[i] < 0 ? -E.e[i] : E.e[i];
      small = small && ax < (1ll << 24) && ay < (1ll << 24) &&
              ae + ax * (int64_t)(px1 - px0) + ay * (int64_t)(py1 - py0) < (1ll << 24);
    }
    if (small) return raster_rect_f32<PASS>(E, a, b, c, invA, px0, py0, px1, py1, zbuf, W);
  }
  const float zmin = fminf(a.zn, fminf(b.zn, c.zn)), zmax = fmaxf(a.zn, fmaxf(b.zn, c.zn));
  int64_t er[3] = {E.e[0], E.e[1], E.e[2]};
  bool vis = false;  // PASS 1: no early exit, so the depth loads can overlap
  for (int py = py0; py <= py1; ++py) {
    int64_t e[3] = {er[0], er[1], er[2]};
    uint32_t* zrow = zbuf + (size_t)py * W;
#pragma unroll 2
    for (int px = px0; px <= px1; ++px) {
      vis |= sample<PASS>(E, e, a, b, c, invA, zrow + px, zmin, zmax);
      e[0] += E.dx[0];
      e[1] += E.dx[1];
      e[2] += E.dx[2];
    }
    er[0] += E.dy[0];
    er[1] += E.dy[1];
    er[2] += E.dy[2];
  }
  return vis;
}

// One small sub-triangle that passed the depth pre-pass set-up: its snapped
// vertices, depths and clamped pixel box, kept so that the marking pass does not
// redo the set-up.  48 bytes: {X0, Y0, X1, Y1}, {X2, Y2, px0 | py0 << 16,
// px1 | py1 << 16}, {z0, z1, z2, triangle}.
struct CandTri {
  int4 a;
  int4 b;
  float4 c;
};
static_assert(sizeof(CandTri) == 48, "CandTri is 48 bytes");

constexpr int kFrontThreads = 512;

struct RasterArgs {
  Mat4 M;
  int cons;  // conservative marking (FA_VIS_CONSERVATIVE): conservative pixel boxes
  const float* Mdev;  // when set, the matrix is read here on the device instead of M
  const float* pos;
  const uint32_t* idx;
  uint32_t T;
  int W, H;
  float hx, hy;
  uint32_t* zbuf;
  BigTri* queue;
  uint32_t queue_cap;
  uint32_t* tile_owner;  // queue record of each reserved tile
  uint32_t tile_cap;
  CandTri* cand;
  uint32_t cand_cap;
  uint32_t* surv;  // triangles that need the exact set-up, one region per front block
  uint32_t* surv_count;  // [front_blocks] survivors per region
  uint32_t surv_per_block;
  uint32_t front_blocks;
  uint32_t clip_base;  // first candidate slot of the clipped path
  float4* surv_clip;  // [T][3] their clip coordinates
  uint32_t* tile_flag;  // per 1024-triangle tile: listed in tile_list
  uint32_t* tile_list;
  uint32_t* clip_count;  // [front_blocks] clipped triangles per region of `clip`
  uint32_t* blockcnt;    // per-tile counts of the chart passes (cleared here)
  uint32_t* viscnt;
  uint32_t ntiles;
  int reset_status;      // the front end clears the device status word first
  int32_t* tri_chart;    // when set, the front end sets it to -1 (the chart pass writes visible ones)
  uint32_t* partial_clear;  // when set, the front end also clears these ceil(T/32) words
  uint32_t mid_max_pix;     // boxes up to this size may be rasterized in-thread (<= kSmallMaxPix: off)
  uint32_t* zmax;           // [ztx * ceil(H / 16)] largest depth key of each 16x16 pixel tile, or
                            // null: no tile-depth pass (FA_RASTER_HIZ off)
  int ztx;                  // tiles per row, ceil(W / 16)
  uint32_t* clip;  // triangles that need clipping, one region per front block like surv
  DevCounters* ctr;
  uint32_t* vt;
};

__device__ __forceinline__ CandTri make_cand(const SV& a, const SV& b, const SV& c, const Setup& s, uint32_t t) {
  CandTri r;
  r.a = make_int4((int)a.X, (int)a.Y, (int)b.X, (int)b.Y);
  r.b = make_int4((int)c.X, (int)c.Y, s.px0 | (s.py0 << 16), s.px1 | (s.py1 << 16));
  r.c = make_float4(a.zn, b.zn, c.zn, __uint_as_float(t));
  return r;
}

__device__ __forceinline__ void store_cand(const RasterArgs& A, uint32_t slot, const CandTri& r) {
  if (slot < A.cand_cap) {
    float4* d = reinterpret_cast<float4*>(A.cand + slot);
    d[0] = make_float4(__int_as_float(r.a.x), __int_as_float(r.a.y), __int_as_float(r.a.z), __int_as_float(r.a.w));
    d[1] = make_float4(__int_as_float(r.b.x), __int_as_float(r.b.y), __int_as_float(r.b.z), __int_as_float(r.b.w));
    d[2] = r.c;
  } else {
    set_status(A.ctr, FA_E_CAPACITY);
  }
}

// Depth pre-pass of the fan (sv[0], sv[i], sv[i+1]) of one mesh triangle t.  Large
// sub-triangles go to the tile queue; small ones are rasterized here and, when
// `out` is given and the fan has a single sub-triangle, returned for the candidate
// list (otherwise appended one by one).  Returns the number of records in `out`.
__device__ int depth_fan(const RasterArgs& A, uint32_t t, const SV* sv, int n, CandTri* out) {
  int nq = 0;
  uint64_t tiles = 0;
  bool big = false;
  for (int i = 1; i + 1 < n; ++i) {
    Setup s = setup(sv[0], sv[i], sv[i + 1], A.W, A.H, A.cons);
    if (s.A <= 0 || s.px1 < s.px0 || s.py1 < s.py0) continue;
    int w = s.px1 - s.px0 + 1, h = s.py1 - s.py0 + 1;
    if (w * h > kSmallMaxPix) big = true;
    ++nq;
    tiles += (uint64_t)((w + kBigTile - 1) / kBigTile) * (uint64_t)((h + kBigTile - 1) / kBigTile);
  }
  if (nq == 0) return 0;
  if (big) {
    unsigned long long old = atomicAdd(&A.ctr->big, ((unsigned long long)nq << 40) | (unsigned long long)tiles);
    uint64_t e0 = old >> 40, tile = old & ((1ull << 40) - 1);
    if (e0 + nq <= A.queue_cap && tile + tiles <= A.tile_cap) {
      int q = 0;
      for (int i = 1; i + 1 < n; ++i) {
        Setup s = setup(sv[0], sv[i], sv[i + 1], A.W, A.H, A.cons);
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
      return 0;
    }
    // queue or tile table full: the reserved records become empty, the reserved
    // tiles get no owner, and the sub-triangles are handled here instead
    for (uint64_t e = e0; e < e0 + nq && e < A.queue_cap; ++e) {
      BigTri bt = {};
      bt.px0 = 1; bt.px1 = 0; bt.py0 = 1; bt.py1 = 0;
      bt.tile0 = (uint32_t)tile;
      A.queue[e] = bt;
    }
    for (uint64_t j = tile; j < tile + tiles && j < A.tile_cap; ++j) A.tile_owner[j] = 0xFFFFFFFFu;
  }
  int nout = 0;
  for (int i = 1; i + 1 < n; ++i) {
    Setup s = setup(sv[0], sv[i], sv[i + 1], A.W, A.H, A.cons);
    if (s.A <= 0 || s.px1 < s.px0 || s.py1 < s.py0) continue;
    float invA = __fdiv_rn(1.0f, ll2float_rn(s.A));
    raster_rect<0>(sv[0], sv[i], sv[i + 1], invA, s.px0, s.py0, s.px1, s.py1, A.zbuf, A.W);
    const CandTri r = make_cand(sv[0], sv[i], sv[i + 1], s, t);
    if (out && nq == 1) {
      *out = r;
      nout = 1;
    } else {
      store_cand(A, A.clip_base + atomicAdd(&A.ctr->ncand, 1u), r);
    }
  }
  return nout;
}

// Triangles that cross the near plane or the guard band (rare): clip first.
__device__ __noinline__ void depth_clipped(const RasterArgs& A, uint32_t t, float4 c0, float4 c1, float4 c2) {
  CV poly[kMaxPoly];
  poly[0] = CV{c0.x, c0.y, c0.z, c0.w};
  poly[1] = CV{c1.x, c1.y, c1.z, c1.w};
  poly[2] = CV{c2.x, c2.y, c2.z, c2.w};
  int n = clip_polygon(poly, 3);
  if (n < 0) {
    set_status(A.ctr, FA_E_CAPACITY);
    return;
  }
  if (n < 3) return;
  for (int i = 0; i < n; ++i)
    if (!(poly[i].w > 0.0f)) return;
  SV sv[kMaxPoly];
  for (int i = 0; i < n; ++i) sv[i] = project(poly[i], A.hx, A.hy);
  depth_fan(A, t, sv, n, nullptr);
}

// Conservative test on approximate screen positions (correctly rounded 1/w, then
// the same screen mapping): true when the triangle surely covers no sample or is
// surely back-facing.  m bounds, per axis, the distance between the approximate
// position and the exact snapped vertex: 1/512 px of snapping plus
// (|ndc| + 1) * (size / 2) * 2^-20 for the different rounding of x * (1/w) and x / w
// followed by the same +1 and scale.  Both tests only drop triangles the exact path
// would drop, so results are unchanged.
__device__ __forceinline__ bool surely_empty(const RasterArgs& A, const float4& c0, const float4& c1, const float4& c2) {
  const float r0 = __frcp_rn(c0.w), r1 = __frcp_rn(c1.w), r2 = __frcp_rn(c2.w);
  const float nx0 = c0.x * r0, nx1 = c1.x * r1, nx2 = c2.x * r2;
  const float ny0 = c0.y * r0, ny1 = c1.y * r1, ny2 = c2.y * r2;
  const float x0 = (nx0 + 1.0f) * A.hx, x1 = (nx1 + 1.0f) * A.hx, x2 = (nx2 + 1.0f) * A.hx;
  const float y0 = (ny0 + 1.0f) * A.hy, y1 = (ny1 + 1.0f) * A.hy, y2 = (ny2 + 1.0f) * A.hy;
  const float ax = fmaxf(fabsf(nx0), fmaxf(fabsf(nx1), fabsf(nx2))) + 1.0f;
  const float ay = fmaxf(fabsf(ny0), fmaxf(fabsf(ny1), fabsf(ny2))) + 1.0f;
  const float mx = 0.001953125f + ax * A.hx * 9.5367431640625e-7f + 1e-6f;
  const float my = 0.001953125f + ay * A.hy * 9.5367431640625e-7f + 1e-6f;
  // pixel centres p + 0.5 inside the widened box, clamped to the viewport
  const float lo_x = fminf(x0, fminf(x1, x2)) - mx, hi_x = fmaxf(x0, fmaxf(x1, x2)) + mx;
  const float lo_y = fminf(y0, fminf(y1, y2)) - my, hi_y = fmaxf(y0, fmaxf(y1, y2)) + my;
  // (conservative marking: pixels whose squares meet the widened box)
  const float px0 = fmaxf(A.cons ? ceilf(lo_x) - 1.0f : ceilf(lo_x - 0.5f), 0.0f);
  const float px1 = fminf(A.cons ? floorf(hi_x) : floorf(hi_x - 0.5f), (float)(A.W - 1));
  const float py0 = fmaxf(A.cons ? ceilf(lo_y) - 1.0f : ceilf(lo_y - 0.5f), 0.0f);
  const float py1 = fminf(A.cons ? floorf(hi_y) : floorf(hi_y - 0.5f), (float)(A.H - 1));
  if (px0 > px1 || py0 > py1) return true;
  // signed doubled area in px^2 against its error bound
  const float e1x = x1 - x0, e1y = y1 - y0, e2x = x2 - x0, e2y = y2 - y0;
  const float p1 = e1x * e2y, p2 = e1y * e2x;
  const float area = p1 - p2;
  const float m = fmaxf(mx, my);
  const float bound = 2.0f * m * (fabsf(e1x) + fabsf(e1y) + fabsf(e2x) + fabsf(e2y)) + 24.0f * m * m +
                      2.384185791015625e-7f * (fabsf(p1) + fabsf(p2)) + 1e-6f;
  return area < -bound;
}

// Front end of the depth pre-pass for one mesh triangle: transform, trivial reject,
// route to the clipped list, conservative reject.  Returns 1 when the triangle needs
// the exact set-up (unclipped; its clip coordinates are left in c[3]), 2 when it must
// be clipped first, 0 when dropped.
struct TriPos {
  float p[9];  // the three corners' world positions
};

__device__ __forceinline__ uint3 load_tri(const uint32_t* __restrict__ idx, uint32_t t) {
  const uint32_t* f = idx + 3 * (size_t)t;
  return make_uint3(__ldg(f), __ldg(f + 1), __ldg(f + 2));
}

__device__ __forceinline__ TriPos load_pos(const float* __restrict__ pos, uint3 i) {
  TriPos q;
  const uint32_t v[3] = {i.x, i.y, i.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float* p = pos + 3 * (size_t)v[k];
    q.p[3 * k] = __ldg(p);
    q.p[3 * k + 1] = __ldg(p + 1);
    q.p[3 * k + 2] = __ldg(p + 2);
  }
  return q;
}

__device__ __forceinline__ int front_triangle(const RasterArgs& A, const Mat4& M, const TriPos& q, float4* c) {
  const float4 c0 = transform(M, q.p[0], q.p[1], q.p[2]), c1 = transform(M, q.p[3], q.p[4], q.p[5]),
               c2 = transform(M, q.p[6], q.p[7], q.p[8]);
  // trivial reject: all vertices outside one side plane, or all behind the near plane
  // (no sample can be covered then: see the design notes on exactness)
  if ((c0.x > c0.w && c1.x > c1.w && c2.x > c2.w) || (c0.x < -c0.w && c1.x < -c1.w && c2.x < -c2.w) ||
      (c0.y > c0.w && c1.y > c1.w && c2.y > c2.w) || (c0.y < -c0.w && c1.y < -c1.w && c2.y < -c2.w) ||
      (__fadd_rn(c0.z, c0.w) < 0.0f && __fadd_rn(c1.z, c1.w) < 0.0f && __fadd_rn(c2.z, c2.w) < 0.0f))
    return 0;
  const CV v0{c0.x, c0.y, c0.z, c0.w}, v1{c1.x, c1.y, c1.z, c1.w}, v2{c2.x, c2.y, c2.z, c2.w};
  bool outside = false;
#pragma unroll
  for (int pl = 0; pl < 5; ++pl)
    outside |= !(plane_dist(v0, pl) >= 0.0f) || !(plane_dist(v1, pl) >= 0.0f) || !(plane_dist(v2, pl) >= 0.0f);
  if (outside) return 2;
  if (!(v0.w > 0.0f) || !(v1.w > 0.0f) || !(v2.w > 0.0f)) return 0;
  if (surely_empty(A, c0, c1, c2)) return 0;
  c[0] = c0;
  c[1] = c1;
  c[2] = c2;
  return 1;
}

// Snapped vertices and set-up of an unclipped triangle from its clip coordinates,
// all in registers (the fan of an unclipped triangle is the triangle itself).
struct Exact {
  SV a, b, c;
  Setup s;
};

__device__ __forceinline__ Exact exact_setup(const RasterArgs& A, const float4& c0, const float4& c1,
                                             const float4& c2) {
  Exact E;
  E.a = project(CV{c0.x, c0.y, c0.z, c0.w}, A.hx, A.hy);
  E.b = project(CV{c1.x, c1.y, c1.z, c1.w}, A.hx, A.hy);
  E.c = project(CV{c2.x, c2.y, c2.z, c2.w}, A.hx, A.hy);
  E.s = setup(E.a, E.b, E.c, A.W, A.H, A.cons);
  return E;
}

// Depth pre-pass, front end: one thread per triangle; survivors go to a compact list
// (warp-aggregated appends) so that the exact set-up runs on full warps.
// Also clears, for the kernels after it, the depth buffer, VT, the counters and the
// per-tile flags and counts of the visible-tile list (none of which it reads).
template <bool DEV_M>
__device__ __forceinline__ void front_body(const RasterArgs& A, uint32_t bid, uint32_t nblk) {
  const Mat4 M = DEV_M ? load_mat(A.Mdev) : A.M;
  __shared__ uint32_t s_count, s_nclip;
  if (threadIdx.x == 0) {
    s_count = 0;
    s_nclip = 0;
    if (bid == 0) {
      if (A.reset_status) A.ctr->status = 0;
      A.ctr->big = 0ull;
      A.ctr->ncand = 0u;
      A.ctr->n_vtiles = 0u;
      A.ctr->uf_item = 0u;
    }
  }
  {
    const uint32_t gstride = nblk * blockDim.x, g0 = bid * blockDim.x + threadIdx.x;
    const uint32_t npix = (uint32_t)A.W * (uint32_t)A.H, n4 = npix / 4, nwords = (A.T + 31) / 32;
    uint4* z4 = reinterpret_cast<uint4*>(A.zbuf);
    const uint4 ff = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    for (uint32_t i = g0; i < n4; i += gstride) z4[i] = ff;
    for (uint32_t i = n4 * 4 + g0; i < npix; i += gstride) A.zbuf[i] = 0xFFFFFFFFu;
    for (uint32_t i = g0; i < nwords; i += gstride) A.vt[i] = 0u;
    for (uint32_t i = g0; i < A.ntiles; i += gstride) {
      A.tile_flag[i] = 0u;
      A.blockcnt[i] = 0u;
      A.viscnt[i] = 0u;
    }
    if (A.partial_clear)
      for (uint32_t i = g0; i < nwords; i += gstride) A.partial_clear[i] = 0u;
    if (A.tri_chart) {
      int4* t4 = reinterpret_cast<int4*>(A.tri_chart);
      for (uint32_t i = g0; i < A.T / 4; i += gstride) t4[i] = make_int4(-1, -1, -1, -1);
      for (uint32_t i = (A.T / 4) * 4 + g0; i < A.T; i += gstride) A.tri_chart[i] = -1;
    }
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  // block b owns survivor slots [b * surv_per_block, (b + 1) * surv_per_block): it sees
  // at most that many triangles, so its region cannot overflow
  const uint32_t region = bid * A.surv_per_block;
  // software pipeline over this thread's triangles t, t + stride, ...: the indices
  // are loaded two iterations ahead and the corner positions one iteration ahead, so
  // that each iteration waits on no dependent load of its own
  const uint32_t stride = nblk * blockDim.x;
  const uint32_t t0 = bid * blockDim.x + threadIdx.x;
  uint3 idx1 = t0 + stride < A.T ? load_tri(A.idx, t0 + stride) : make_uint3(0u, 0u, 0u);
  TriPos pos0 = load_pos(A.pos, t0 < A.T ? load_tri(A.idx, t0) : make_uint3(0u, 0u, 0u));
  for (uint32_t base = bid * blockDim.x; base < A.T; base += stride) {
    const uint32_t t = base + threadIdx.x;
    const TriPos cur = pos0;
    pos0 = load_pos(A.pos, idx1);
    idx1 = t + 2u * stride < A.T ? load_tri(A.idx, t + 2u * stride) : make_uint3(0u, 0u, 0u);
    float4 c[3];
    const int r = t < A.T ? front_triangle(A, M, cur, c) : 0;
    const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, r == 1), b2 = __ballot_sync(0xFFFFFFFFu, r == 2);
    if (b1) {
      uint32_t o = 0;
      if (lane == 0) o = atomicAdd(&s_count, (uint32_t)__popc(b1));
      o = __shfl_sync(0xFFFFFFFFu, o, 0);
      if (r == 1) {
        const uint32_t slot = region + o + __popc(b1 & ((1u << lane) - 1u));
        A.surv[slot] = t;
        float4* sc = A.surv_clip + 3 * (size_t)slot;
        sc[0] = c[0];
        sc[1] = c[1];
        sc[2] = c[2];
      }
    }
    if (b2) {  // rare: the block's clipped region, like the survivors'
      uint32_t o = 0;
      if (lane == 0) o = atomicAdd(&s_nclip, (uint32_t)__popc(b2));
      o = __shfl_sync(0xFFFFFFFFu, o, 0);
      if (r == 2) A.clip[region + o + __popc(b2 & ((1u << lane) - 1u))] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    A.surv_count[bid] = s_count;
    A.clip_count[bid] = s_nclip;
  }
}

// Exclusive prefix of the front blocks' per-region counts (survivors or clipped
// triangles) into shared memory (front_blocks <= kMaxFrontBlocks); returns the
// total.  Called by every thread of a block of exactly NT threads.
template <int NT>
__device__ uint32_t region_prefix(const RasterArgs& A, const uint32_t* counts, uint32_t* pre) {
  constexpr uint32_t kPer = (kMaxFrontBlocks + NT - 1) / NT;
  __shared__ uint32_t s_warp[NT / 32];
  const uint32_t nb = A.front_blocks, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t c[kPer], sum = 0;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    const uint32_t b = threadIdx.x * kPer + j;
    c[j] = b < nb ? __ldcg(counts + b) : 0u;
    sum += c[j];
  }
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  uint32_t wpre = 0, tot = 0;
#pragma unroll
  for (uint32_t k = 0; k < (uint32_t)(NT / 32); ++k) {
    const uint32_t x = s_warp[k];
    wpre += k < w ? x : 0u;
    tot += x;
  }
  uint32_t run = wpre + inc - sum;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    const uint32_t b = threadIdx.x * kPer + j;
    if (b <= nb) pre[b] = run;
    run += c[j];
  }
  __syncthreads();
  return tot;
}
template <int NT>
__device__ __forceinline__ uint32_t surv_prefix(const RasterArgs& A, uint32_t* pre) {
  return region_prefix<NT>(A, A.surv_count, pre);
}

// Survivor slot of dense index v: block b with pre[b] <= v < pre[b + 1].
// Slot of dense index v in the front blocks' regions (survivors or clipped
// triangles, as pre was built): block b with pre[b] <= v < pre[b + 1].  vfirst <=
// v is the warp's first index, the same in every lane: its search reads the same
// shared words in all lanes (broadcasts), and a lane searches on its own only when
// v lies in a later region than vfirst.
__device__ __forceinline__ uint32_t surv_slot(const RasterArgs& A, const uint32_t* pre, uint32_t v,
                                              uint32_t vfirst) {
  uint32_t lo = 0, hi = A.front_blocks;  // pre[lo] <= vfirst < pre[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= vfirst) lo = mid;
    else hi = mid;
  }
  if (v >= pre[lo + 1]) {
    hi = A.front_blocks;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (pre[mid] <= v) lo = mid;
      else hi = mid;
    }
  }
  return lo * A.surv_per_block + (v - pre[lo]);
}

// The samples of one sub-triangle per group of kRasterGroup lanes: the group's
// leader (its first lane) holds the snapped vertices, area and pixel box, and `go`;
// every lane of the group takes the box's samples sub, sub + kRasterGroup, ...  PASS
// as in sample(): 0 writes the depth keys; 1 and 2 return whether a sample of the
// leader's sub-triangle passed the depth test (in every lane of the group).  All
// lanes of the warp call it.
constexpr uint32_t kRasterGroup = 16;
template <int PASS>
__device__ __forceinline__ bool group_raster(const SV& a0, const SV& b0, const SV& c0, int64_t A0, int qx0, int qy0,
                                             int qx1, int qy1, bool go0, uint32_t* __restrict__ zbuf, int W) {
  const uint32_t lane = threadIdx.x & 31, src = lane & ~(kRasterGroup - 1u), sub = lane - src;
  // every lane of the warp takes part in every shuffle (the groups' leaders differ in
  // `go`, so no shuffle may sit under it)
  const bool go = __shfl_sync(0xFFFFFFFFu, go0, src);
  const SV a{__shfl_sync(0xFFFFFFFFu, (int32_t)a0.X, src), __shfl_sync(0xFFFFFFFFu, (int32_t)a0.Y, src),
             __shfl_sync(0xFFFFFFFFu, a0.zn, src)};
  const SV b{__shfl_sync(0xFFFFFFFFu, (int32_t)b0.X, src), __shfl_sync(0xFFFFFFFFu, (int32_t)b0.Y, src),
             __shfl_sync(0xFFFFFFFFu, b0.zn, src)};
  const SV c{__shfl_sync(0xFFFFFFFFu, (int32_t)c0.X, src), __shfl_sync(0xFFFFFFFFu, (int32_t)c0.Y, src),
             __shfl_sync(0xFFFFFFFFu, c0.zn, src)};
  const int64_t Ar = (int64_t)(((uint64_t)__shfl_sync(0xFFFFFFFFu, (uint32_t)((uint64_t)A0 >> 32), src) << 32) |
                               (uint64_t)__shfl_sync(0xFFFFFFFFu, (uint32_t)A0, src));
  const int px0 = __shfl_sync(0xFFFFFFFFu, qx0, src), py0 = __shfl_sync(0xFFFFFFFFu, qy0, src);
  const int px1 = __shfl_sync(0xFFFFFFFFu, qx1, src), py1 = __shfl_sync(0xFFFFFFFFu, qy1, src);
  bool vis = false;
  if (go) {
    const float invA = __fdiv_rn(1.0f, ll2float_rn(Ar));
    const float zmin = fminf(a.zn, fminf(b.zn, c.zn)), zmax = fmaxf(a.zn, fmaxf(b.zn, c.zn));
    const int w = px1 - px0 + 1, npix = w * (py1 - py0 + 1);
    for (int s = (int)sub; s < npix; s += (int)kRasterGroup) {
      const int px = px0 + s % w, py = py0 + s / w;
      const Edges E = edges_at(a, b, c, px, py);
      vis |= sample<PASS>(E, E.e, a, b, c, invA, zbuf + (size_t)py * W + px, zmin, zmax);
    }
  }
  if (PASS == 0) return false;
  const uint32_t gmask = ((1u << kRasterGroup) - 1u) << src;
  return (__ballot_sync(0xFFFFFFFFu, vis) & gmask) != 0u;
}

// Depth pre-pass, exact part: survivors of the front end.  Survivor i writes its
// candidate record (or an empty marker) at slot i, so no counter is needed; clipped
// triangles append theirs after slot T.
template <bool DEV_M, int NT>
__device__ __forceinline__ void exact_body(const RasterArgs& A, uint32_t bid, uint32_t nblk) {
  __shared__ uint32_t pre[kMaxFrontBlocks + 1];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n = surv_prefix<NT>(A, pre);
  const uint32_t stride = nblk * blockDim.x;
  // Few survivors for the grid (a small frame): each gets a group of kRasterGroup
  // lanes, its leader doing the set-up and the group sharing the box's samples, so
  // that the grid's warps are not each waiting on one thread's sample loop.  The
  // same samples get the same keys either way.
  const bool grouped = (uint64_t)n * kRasterGroup <= (uint64_t)stride;
  const uint32_t sub = lane & (kRasterGroup - 1u);
  for (uint32_t wbase = bid * blockDim.x + (threadIdx.x & ~31u); (grouped ? wbase / kRasterGroup : wbase) < n;
       wbase += stride) {
    const uint32_t vfirst = grouped ? wbase / kRasterGroup : wbase;
    // (in a group only the leader sets up; the others take no survivor here)
    const uint32_t v = grouped ? (sub == 0u ? vfirst + lane / kRasterGroup : n) : wbase + lane;
    const uint32_t i = v < n ? surv_slot(A, pre, v, vfirst) : 0u;
    Exact E = {};
    uint32_t t = 0, tiles = 0;
    int kind = 0;  // 0 nothing, 1 small, 2 large
    bool mid = false;  // large, but at most kMidMaxPix pixels
    uint32_t mid_pix = 0, mid_cost = 0;
    if (v < n) {
      const float4* sc = A.surv_clip + 3 * (size_t)i;
      t = __ldcg(A.surv + i);
      E = exact_setup(A, __ldcs(sc), __ldcs(sc + 1), __ldcs(sc + 2));
      if (E.s.A > 0 && E.s.px1 >= E.s.px0 && E.s.py1 >= E.s.py0) {
        const int w = E.s.px1 - E.s.px0 + 1, h = E.s.py1 - E.s.py0 + 1;
        if (w * h > kSmallMaxPix) {
          kind = 2;
          tiles = (uint32_t)(((w + kBigTile - 1) / kBigTile) * ((h + kBigTile - 1) / kBigTile));
          mid = w * h <= (int)A.mid_max_pix;
          if (mid) {
            mid_pix = (uint32_t)(w * h);
            // the tile path: two rows per warp step in each 16-pixel-wide tile
            // column, plus the queue record and its set-up
            mid_cost = kMidStepCost * (uint32_t)((w + kBigTile - 1) / kBigTile) * (uint32_t)((h + 1) / 2) +
                       kMidTriCost;
          }
        } else {
          kind = 1;
        }
      }
    }
    // Mid-size boxes are rasterized in-thread when that is cheaper for the warp: the
    // in-thread loop lasts as long as the warp's largest box (the small boxes' 16
    // samples are paid anyway), the tile path costs each such triangle its tile
    // steps and its queue record.  Either way the same samples get the same keys.
    {
      const uint32_t smax = __reduce_max_sync(0xFFFFFFFFu, mid_pix);
      const uint32_t tsum = __reduce_add_sync(0xFFFFFFFFu, mid_cost);
      if (mid && (smax - (uint32_t)kSmallMaxPix) * kMidSampleCost < tsum) {
        kind = 1;
        tiles = 0;
      }
    }
    // large triangles of the warp reserve queue records and tiles with one atomic
    const uint32_t bigs = __ballot_sync(0xFFFFFFFFu, kind == 2);
    if (bigs) {
      uint32_t tpre = tiles;  // inclusive prefix of tiles over the warp
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, tpre, o);
        if (lane >= (unsigned)o) tpre += y;
      }
      const uint32_t ttot = __shfl_sync(0xFFFFFFFFu, tpre, 31);
      unsigned long long old = 0;
      if (lane == 0)
        old = atomicAdd(&A.ctr->big, ((unsigned long long)__popc(bigs) << 40) | (unsigned long long)ttot);
      old = __shfl_sync(0xFFFFFFFFu, old, 0);
      if (kind == 2) {
        const uint64_t e = (old >> 40) + __popc(bigs & ((1u << lane) - 1u));
        const uint64_t tile = (old & ((1ull << 40) - 1)) + (tpre - tiles);
        if (e < A.queue_cap && tile + tiles <= A.tile_cap) {
          BigTri bt;
          bt.X[0] = (int32_t)E.a.X; bt.X[1] = (int32_t)E.b.X; bt.X[2] = (int32_t)E.c.X;
          bt.Y[0] = (int32_t)E.a.Y; bt.Y[1] = (int32_t)E.b.Y; bt.Y[2] = (int32_t)E.c.Y;
          bt.zn[0] = E.a.zn; bt.zn[1] = E.b.zn; bt.zn[2] = E.c.zn;
          bt.px0 = E.s.px0; bt.py0 = E.s.py0; bt.px1 = E.s.px1; bt.py1 = E.s.py1;
          bt.tri = t;
          bt.tile0 = (uint32_t)tile;
          bt.pad = 0;
          A.queue[e] = bt;
          for (uint32_t j = 0; j < tiles; ++j) A.tile_owner[tile + j] = (uint32_t)e;
          kind = 0;
        } else {
          // queue or tile table full: empty record, no owners, rasterized here
          if (e < A.queue_cap) {
            BigTri bt = {};
            bt.px0 = 1; bt.px1 = 0; bt.py0 = 1; bt.py1 = 0;
            bt.tile0 = (uint32_t)tile;
            A.queue[e] = bt;
          }
          for (uint64_t j = tile; j < tile + tiles && j < A.tile_cap; ++j) A.tile_owner[j] = 0xFFFFFFFFu;
          kind = 1;
        }
      }
    }
    if (v < n) {
      if (kind == 1) {
        if (!grouped) {
          const float invA = __fdiv_rn(1.0f, ll2float_rn(E.s.A));
          raster_rect<0>(E.a, E.b, E.c, invA, E.s.px0, E.s.py0, E.s.px1, E.s.py1, A.zbuf, A.W);
        }
        store_cand(A, i, make_cand(E.a, E.b, E.c, E.s, t));
      } else {
        reinterpret_cast<uint32_t*>(A.cand + i)[6] = 0xFFFFFFFFu;  // empty: px0 = py0 = 0xFFFF
      }
    }
    if (grouped) group_raster<0>(E.a, E.b, E.c, E.s.A, E.s.px0, E.s.py0, E.s.px1, E.s.py1, kind == 1, A.zbuf, A.W);
  }
  // then the (rare) triangles that need clipping, from the front blocks' regions
  __syncthreads();  // pre is reused
  const uint32_t nc = region_prefix<NT>(A, A.clip_count, pre);
  for (uint32_t i = bid * blockDim.x + threadIdx.x; i < nc; i += stride) {
    const uint32_t t = __ldcg(A.clip + surv_slot(A, pre, i, i));
    const uint32_t* f = A.idx + 3 * (size_t)t;
    const Mat4 M = DEV_M ? load_mat(A.Mdev) : A.M;
    const float4 c0 = load_clip(M, A.pos, __ldg(f)), c1 = load_clip(M, A.pos, __ldg(f + 1)),
                 c2 = load_clip(M, A.pos, __ldg(f + 2));
    depth_clipped(A, t, c0, c1, c2);
  }
}

// Occlusion test of the marking pass on the final depth buffer (exact): a
// sub-triangle whose every sample depth is above the largest depth key of every
// 16x16 tile that its pixel box [px0, px1] x [py0, py1] touches cannot mark.  A
// sample depth is the rounded barycentric combination of the vertex depths; it
// lies within 7 * 2^-24 * max |z| of the exact value (three rounded terms, their
// two sums, 1 / A and the product), which lies in [zmin, zmax] (the clamped depth
// of conservative marking too), so zmin - 1e-6 max |z|, rounded down, bounds it
// from below.
__device__ __forceinline__ bool hidden_by_tiles(const RasterArgs& A, float z0, float z1, float z2, int px0, int py0,
                                                int px1, int py1) {
  if (!A.zmax) return false;
  const float zmin = fminf(z0, fminf(z1, z2));
  const float zabs = fmaxf(fabsf(z0), fmaxf(fabsf(z1), fabsf(z2)));
  const float lo = __fsub_rd(zmin, __fmaf_ru(zabs, 1e-6f, 1e-37f));
  const uint32_t klo = ordered(lo);
  uint32_t zm = 0u;
  for (int ty = py0 >> 4; ty <= (py1 >> 4); ++ty)
    for (int tx = px0 >> 4; tx <= (px1 >> 4); ++tx) zm = max(zm, __ldcg(A.zmax + ty * A.ztx + tx));
  return klo > zm;
}

// The largest depth key of each 16x16 pixel tile of the final depth buffer: a
// warp per tile, a half warp per row.
__device__ __forceinline__ void zmax_body(const RasterArgs& A, uint32_t bid, uint32_t nblk) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t zty = (uint32_t)((A.H + 15) / 16), ntile = (uint32_t)A.ztx * zty;
  const uint32_t nwarps = (nblk * blockDim.x) >> 5;
  for (uint32_t g = (bid * blockDim.x + threadIdx.x) >> 5; g < ntile; g += nwarps) {
    const int x = (int)(g % (uint32_t)A.ztx) * 16 + (int)(lane & 15);
    const int y0 = (int)(g / (uint32_t)A.ztx) * 16 + (int)(lane >> 4);
    uint32_t m = 0u;
    uint32_t k[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int y = y0 + 2 * r;
      k[r] = (x < A.W && y < A.H) ? __ldcg(A.zbuf + (size_t)y * A.W + x) : 0u;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) m = max(m, k[r]);
    m = __reduce_max_sync(0xFFFFFFFFu, m);
    if (lane == 0) A.zmax[g] = m;
  }
}

// The marking pass lists each 1024-triangle tile in which it marks a triangle, once.
__device__ __forceinline__ void note_tile(const RasterArgs& A, uint32_t tile) {
  if (!__ldcg(A.tile_flag + tile) && atomicExch(A.tile_flag + tile, 1u) == 0u)
    A.tile_list[atomicAdd(&A.ctr->n_vtiles, 1u)] = tile;
}

// Large sub-triangles: one warp per 16x16 tile of a queued record (grid-stride).
template <int PASS>
__device__ __forceinline__ void big_tiles(const RasterArgs& A, uint32_t bid, uint32_t nblk) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)bid * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)nblk * blockDim.x) >> 5;
  const unsigned long long st = __ldcg(&A.ctr->big);
  const uint64_t n_ent = (st >> 40) < A.queue_cap ? (st >> 40) : A.queue_cap;
  const uint64_t n_tiles = st & ((1ull << 40) - 1);
  if (n_ent == 0) return;
  const uint64_t n_used = n_tiles < A.tile_cap ? n_tiles : A.tile_cap;
  for (uint64_t g = warp; g < n_used; g += nwarps) {
    const uint32_t lo = __ldcg(A.tile_owner + g);
    if (lo >= n_ent) continue;
    const BigTri& q = A.queue[lo];
    const int px0 = q.px0, py0 = q.py0, px1 = q.px1, py1 = q.py1;
    if (px1 < px0 || py1 < py0) continue;
    const uint32_t tx_n = (uint32_t)((px1 - px0 + kBigTile) / kBigTile);
    const uint32_t ty_n = (uint32_t)((py1 - py0 + kBigTile) / kBigTile);
    const uint64_t local = g - q.tile0;
    if (local >= (uint64_t)tx_n * ty_n) continue;
    // marking: another tile of the sub-triangle may have marked its triangle already
    if (PASS >= 1 && ((__ldcg(A.vt + (q.tri >> 5)) >> (q.tri & 31)) & 1u)) continue;
    const int bx = px0 + (int)(local % tx_n) * kBigTile, by = py0 + (int)(local / tx_n) * kBigTile;
    if (PASS >= 1 && hidden_by_tiles(A, q.zn[0], q.zn[1], q.zn[2], bx, by, min(bx + kBigTile - 1, px1),
                                     min(by + kBigTile - 1, py1)))
      continue;
    SV a{q.X[0], q.Y[0], q.zn[0]}, b{q.X[1], q.Y[1], q.zn[1]}, c{q.X[2], q.Y[2], q.zn[2]};
    const int64_t Ar = (b.X - a.X) * (c.Y - a.Y) - (c.X - a.X) * (b.Y - a.Y);
    const float invA = __fdiv_rn(1.0f, ll2float_rn(Ar));
    const float zmin = fminf(a.zn, fminf(b.zn, c.zn)), zmax = fmaxf(a.zn, fmaxf(b.zn, c.zn));
    bool vis = false;
    const int px = bx + (int)(lane % kBigTile), py_first = by + (int)(lane / kBigTile);
    const Edges E = edges_at(a, b, c, px, py_first);
    int64_t e[3] = {E.e[0], E.e[1], E.e[2]};
    // only the tile's rows inside the box (the last tile row of a box is often
    // short); the same trip count in every lane
    const int rows = min(by + kBigTile - 1, py1) - by + 1;
    const int steps = (rows + 32 / kBigTile - 1) / (32 / kBigTile);
#pragma unroll 1
    for (int k = 0; k < steps; ++k) {
      const int py = py_first + k * (32 / kBigTile);
      if (px <= px1 && py <= py1)
        vis |= sample<PASS>(E, e, a, b, c, invA, A.zbuf + (size_t)py * A.W + px, zmin, zmax);
      if (PASS >= 1 && __any_sync(0xFFFFFFFFu, vis)) break;
      e[0] += E.dy[0] * (32 / kBigTile);
      e[1] += E.dy[1] * (32 / kBigTile);
      e[2] += E.dy[2] * (32 / kBigTile);
    }
    if (PASS >= 1) {
      if (__any_sync(0xFFFFFFFFu, vis) && lane == 0) {
        atomicOr(A.vt + (q.tri >> 5), 1u << (q.tri & 31));
        note_tile(A, q.tri >> 10);
      }
    }
  }
}

// Marking pass: first the tiles of the large sub-triangles, then the candidate
// list (a record is visible when one of its samples has key <= the depth buffer;
// visible bits are OR-ed per VT word and warp).  One launch for both, so blocks
// that finish their share of the tiles early take candidate records.
template <bool CONS, int NT>
__device__ __forceinline__ void mark_body(const RasterArgs& A, uint32_t bid, uint32_t nblk) {
  __shared__ uint32_t pre[kMaxFrontBlocks + 1];
  __shared__ int32_t s_status;
  if (threadIdx.x == 0) s_status = __ldcg(&A.ctr->status);
  __syncthreads();
  if (s_status != 0) return;
  big_tiles<CONS ? 2 : 1>(A, bid, nblk);
  const uint32_t ns = surv_prefix<NT>(A, pre);
  const uint32_t nc = min(__ldcg(&A.ctr->ncand), A.cand_cap - A.clip_base);
  const uint32_t n = ns + nc;  // survivor records, then the clipped-path records
  const uint32_t stride = nblk * blockDim.x;
  // few records for the grid: a group of kRasterGroup lanes per record (as in the
  // exact pass), its samples tested together instead of one after the other
  const bool grouped = (uint64_t)n * kRasterGroup <= (uint64_t)stride;
  const uint32_t sub = threadIdx.x & (kRasterGroup - 1u);
  for (uint32_t base = bid * blockDim.x; (grouped ? base / kRasterGroup : base) < n; base += stride) {
    const uint32_t wb = base + (threadIdx.x & ~31u);  // the warp's first thread
    const uint32_t kfirst = grouped ? wb / kRasterGroup : wb;
    const uint32_t k = grouped ? (sub == 0u ? kfirst + (threadIdx.x & 31u) / kRasterGroup : n) : base + threadIdx.x;
    bool vis = false, go = false;
    uint32_t t = 0xFFFFFFFFu;
    SV ga{0, 0, 0.0f}, gb{0, 0, 0.0f}, gc{0, 0, 0.0f};
    int64_t gA = 0;
    int gx0 = 0, gy0 = 0, gx1 = -1, gy1 = -1;
    if (k < n) {
      const uint32_t i = k < ns ? surv_slot(A, pre, k, kfirst) : A.clip_base + (k - ns);
      const float4* s = reinterpret_cast<const float4*>(A.cand + i);
      const float4 fb = __ldcs(s + 1);
      const uint32_t b0 = __float_as_uint(fb.z), b1 = __float_as_uint(fb.w);
      if (b0 != 0xFFFFFFFFu) {
        const float4 fa = __ldcs(s), fc = __ldcs(s + 2);
        const SV a{__float_as_int(fa.x), __float_as_int(fa.y), fc.x};
        const SV b{__float_as_int(fa.z), __float_as_int(fa.w), fc.y};
        const SV c{__float_as_int(fb.x), __float_as_int(fb.y), fc.z};
        t = __float_as_uint(fc.w);
        const int px0 = (int)(b0 & 0xFFFFu), py0 = (int)(b0 >> 16), px1 = (int)(b1 & 0xFFFFu), py1 = (int)(b1 >> 16);
        if (!hidden_by_tiles(A, fc.x, fc.y, fc.z, px0, py0, px1, py1)) {
          const int64_t Ar = (b.X - a.X) * (c.Y - a.Y) - (c.X - a.X) * (b.Y - a.Y);
          if (grouped) {
            go = true;
            ga = a;
            gb = b;
            gc = c;
            gA = Ar;
            gx0 = px0;
            gy0 = py0;
            gx1 = px1;
            gy1 = py1;
          } else {
            const float invA = __fdiv_rn(1.0f, ll2float_rn(Ar));
            vis = raster_rect<CONS ? 2 : 1>(a, b, c, invA, px0, py0, px1, py1, A.zbuf, A.W);
          }
        }
      }
    }
    if (grouped) {
      const bool gv = group_raster<CONS ? 2 : 1>(ga, gb, gc, gA, gx0, gy0, gx1, gy1, go, A.zbuf, A.W);
      vis = sub == 0u && k < n && gv;
    }
    const uint32_t word = vis ? (t >> 5) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, word);
    const uint32_t bits = __reduce_or_sync(peers, vis ? (1u << (t & 31)) : 0u);
    if (vis && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) {
      atomicOr(A.vt + word, bits);
      note_tile(A, word >> 5);
    }
  }
}

// Depth pre-pass of the large sub-triangles.
__device__ __forceinline__ void depth_big_body(const RasterArgs& A, uint32_t bid, uint32_t nblk) {
  big_tiles<0>(A, bid, nblk);
}

// The arguments of one visibility pass on ctx (host side).  front_blocks blocks of
// `threads` threads run the front end; each owns a survivor region large enough for
// every triangle it can see.
inline RasterArgs make_raster_args(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W, uint32_t H,
                                   uint32_t* vt, bool reset_status, const float* Mdev, bool cons,
                                   int32_t* tri_chart_init, uint32_t front_blocks, uint32_t threads) {
  RasterArgs A;
  A.cons = cons ? 1 : 0;
  A.Mdev = Mdev;
  A.M = M;
  A.pos = mesh->pos;
  A.idx = mesh->idx;
  A.T = mesh->T;
  A.W = (int)W;
  A.H = (int)H;
  A.hx = 0.5f * (float)W;
  A.hy = 0.5f * (float)H;
  A.zbuf = ctx->zbuf;
  A.queue = ctx->queue;
  A.queue_cap = ctx->queue_cap;
  A.tile_owner = ctx->tile_owner;
  A.tile_cap = ctx->tile_cap;
  A.cand = reinterpret_cast<CandTri*>(ctx->cand);
  A.cand_cap = ctx->cand_cap;
  A.surv = ctx->surv;
  A.surv_count = ctx->surv_count;
  A.front_blocks = front_blocks;
  {
    const uint32_t iters = (mesh->T + front_blocks * threads - 1) / (front_blocks * threads);
    A.surv_per_block = iters * threads;
  }
  A.clip_base = A.front_blocks * A.surv_per_block;
  A.surv_clip = reinterpret_cast<float4*>(ctx->surv_clip);
  A.tile_flag = ctx->tile_flag;
  A.tile_list = ctx->tile_list;
  A.clip_count = ctx->clip_count;
  A.blockcnt = ctx->blockcnt;
  A.viscnt = ctx->viscnt;
  A.ntiles = (mesh->T + 1023) / 1024;
  A.reset_status = reset_status ? 1 : 0;
  A.tri_chart = tri_chart_init;
  A.partial_clear = nullptr;
  A.mid_max_pix = ctx->mid_max_pix;
  A.zmax = (ctx->raster_flags & FA_RASTER_HIZ) ? ctx->zmax : nullptr;
  A.ztx = (int)((W + 15) / 16);
  A.clip = ctx->clip;
  A.ctr = ctx->ctr;
  A.vt = vt;
  return A;
}

}  // namespace
}  // namespace rs
}  // namespace fa
