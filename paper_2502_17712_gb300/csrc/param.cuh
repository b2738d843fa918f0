// Chart boxes, footprints and UVs.
//
// k_bbox (Sec. 5.2): per visible triangle, clip against the near plane when it
//   crosses it (otherwise, with FA_BOX_FRUSTUM_CLIP, against the one frustum plane
//   that shrinks its box most), clamp each vertex to [-w, w] and divide (Blinn's
//   estimator); optionally the partial-visibility bits (Sec. 6); then
//   a warp-segmented min / max per chart (__match_any_sync + __reduce_*_sync) and one
//   atomic per chart and warp on order-preserving integer encodings (exact and
//   order independent).
// k_footprint (Sec. 5.2, Sec. 4.1): viewport size of the box, scaled by the
//   texel-to-pixel ratio, quantized up to 1/256 texel, rotated to stand tall.
// k_uv (Sec. 3, App. A): projection of each visible corner into its chart's atlas
//   box in compensated fp32 ("double-float": Knuth TwoSum, FMA TwoProd), rounded
//   once at the end.
#pragma once
#include "fa_internal.cuh"

namespace fa {
namespace pm {
namespace {

struct CV {
  float x, y, z, w;
};

__device__ __forceinline__ CV lerp_in_out(const CV& a, const CV& b, float da, float db) {
  float t = __fdiv_rn(da, __fsub_rn(da, db));
  CV r;
  r.x = __fadd_rn(a.x, __fmul_rn(t, __fsub_rn(b.x, a.x)));
  r.y = __fadd_rn(a.y, __fmul_rn(t, __fsub_rn(b.y, a.y)));
  r.z = __fadd_rn(a.z, __fmul_rn(t, __fsub_rn(b.z, a.z)));
  r.w = __fadd_rn(a.w, __fmul_rn(t, __fsub_rn(b.w, a.w)));
  return r;
}

struct Box {
  float xmin, ymin, xmax, ymax;
  bool full;
};

__device__ __forceinline__ void box_add(Box& b, const CV& c) {
  if (!(c.w > 0.0f)) {
    b.full = true;
    return;
  }
  float x = c.x, y = c.y;
  const float nw = -c.w;
  if (x < nw) x = nw;
  if (x > c.w) x = c.w;
  if (y < nw) y = nw;
  if (y > c.w) y = c.w;
  float nx = __fdiv_rn(x, c.w), ny = __fdiv_rn(y, c.w);
  if (nx == 0.0f) nx = 0.0f;
  if (ny == 0.0f) ny = 0.0f;
  b.xmin = fminf(b.xmin, nx);
  b.ymin = fminf(b.ymin, ny);
  b.xmax = fmaxf(b.xmax, nx);
  b.ymax = fmaxf(b.ymax, ny);
}

struct BoxArgs {
  Mat4 M;
  uint32_t frustum_clip;  // FA_BOX_FRUSTUM_CLIP
  uint32_t* partial;      // partial-visibility bits, or null
  const float* Mdev;  // when set, the matrix is read here on the device instead of M
  const float* pos;
  const uint32_t* idx;
  const uint2* vis;  // (triangle, chart) of the visible triangles
  const int32_t* tri_chart;
  uint32_t T;
  uint32_t* box_enc;
  uint32_t* box_full;
  uint32_t max_charts;
  DevCounters* ctr;
};

// Signed distance to frustum plane pl (inside iff >= 0): 0 left x >= -w, 1 right
// x <= w, 2 bottom y >= -w, 3 top y <= w, 4 far z <= w.
__device__ __forceinline__ float frustum_dist(const CV& c, int pl) {
  switch (pl) {
    case 0: return __fadd_rn(c.x, c.w);
    case 1: return __fsub_rn(c.w, c.x);
    case 2: return __fadd_rn(c.y, c.w);
    case 3: return __fsub_rn(c.w, c.y);
    default: return __fsub_rn(c.w, c.z);
  }
}

// Box of a triangle that does not cross the near plane, clipped first against the
// one frustum plane whose clip gives the smallest Blinn box (fp32 area, ties to the
// first plane in the order above; a plane the triangle does not cross leaves it
// whole; a plane it lies wholly outside of is no candidate).
__device__ __forceinline__ void box_frustum(Box& b, const CV (&v)[3]) {
  const float inf = __int_as_float(0x7f800000);
  Box best{inf, inf, -inf, -inf, false};
  float best_area = inf;
  bool have = false;
#pragma unroll
  for (int pl = 0; pl < 5; ++pl) {
    const float d[3] = {frustum_dist(v[0], pl), frustum_dist(v[1], pl), frustum_dist(v[2], pl)};
    Box cb{inf, inf, -inf, -inf, false};
    int np = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int nx = (i + 1) % 3;
      const bool ic = d[i] >= 0.0f, in_ = d[nx] >= 0.0f;
      if (ic) {
        box_add(cb, v[i]);
        ++np;
      }
      if (ic != in_) {
        box_add(cb, ic ? lerp_in_out(v[i], v[nx], d[i], d[nx]) : lerp_in_out(v[nx], v[i], d[nx], d[i]));
        ++np;
      }
    }
    if (np < 3) continue;
    const float area = cb.full ? inf : __fmul_rn(__fsub_rn(cb.xmax, cb.xmin), __fsub_rn(cb.ymax, cb.ymin));
    if (!have || area < best_area) {
      have = true;
      best_area = area;
      best = cb;
    }
  }
  if (!have) {
    box_add(b, v[0]);
    box_add(b, v[1]);
    box_add(b, v[2]);
  } else if (best.full) {
    b.full = true;
  } else {
    b.xmin = fminf(b.xmin, best.xmin);
    b.ymin = fminf(b.ymin, best.ymin);
    b.xmax = fmaxf(b.xmax, best.xmax);
    b.ymax = fmaxf(b.ymax, best.ymax);
  }
}

template <bool DEV_M>
__device__ __forceinline__ void bbox_body(const BoxArgs& a, uint32_t bid, uint32_t nblk) {
  const Mat4 M = DEV_M ? load_mat(a.Mdev) : a.M;
  if (__ldcg(&a.ctr->status) != 0) return;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n = __ldcg(&a.ctr->n_vis);
  const uint32_t stride = nblk * blockDim.x;
  for (uint32_t base = bid * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
    const uint32_t i = base + lane;
    uint32_t t = 0;
    int32_t c = -1;
    Box b{__int_as_float(0x7f800000), __int_as_float(0x7f800000), __int_as_float(0xff800000),
          __int_as_float(0xff800000), false};
    bool pv = false;  // partially visible (Sec. 6): a vertex with max(|x|, |y|) >= w
    if (i < n) {
      const uint2 e = __ldcg(a.vis + i);
      t = e.x;
      c = (int32_t)e.y;
      if ((uint32_t)c >= a.max_charts || t >= a.T) c = -1;  // not a chart of this context: ignored
    }
    if (c >= 0) {
      const uint32_t* f = a.idx + 3 * (size_t)t;
      float4 p0 = load_clip(M, a.pos, __ldg(f)), p1 = load_clip(M, a.pos, __ldg(f + 1)),
             p2 = load_clip(M, a.pos, __ldg(f + 2));
      CV v[3] = {{p0.x, p0.y, p0.z, p0.w}, {p1.x, p1.y, p1.z, p1.w}, {p2.x, p2.y, p2.z, p2.w}};
      float d[3] = {__fadd_rn(p0.z, p0.w), __fadd_rn(p1.z, p1.w), __fadd_rn(p2.z, p2.w)};
      const bool all_in = d[0] >= 0.0f && d[1] >= 0.0f && d[2] >= 0.0f;
      if (a.partial) {
        pv = fmaxf(fabsf(p0.x), fabsf(p0.y)) >= p0.w || fmaxf(fabsf(p1.x), fabsf(p1.y)) >= p1.w ||
             fmaxf(fabsf(p2.x), fabsf(p2.y)) >= p2.w;
      }
      if (all_in && a.frustum_clip) {
        box_frustum(b, v);
      } else if (all_in) {
        box_add(b, v[0]);
        box_add(b, v[1]);
        box_add(b, v[2]);
      } else {
        // Sutherland-Hodgman against the near plane only (3 -> 3 or 4 vertices)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const int nx = (i + 1) % 3;
          const bool ic = d[i] >= 0.0f, in_ = d[nx] >= 0.0f;
          if (ic) box_add(b, v[i]);
          if (ic != in_) box_add(b, ic ? lerp_in_out(v[i], v[nx], d[i], d[nx]) : lerp_in_out(v[nx], v[i], d[nx], d[i]));
        }
      }
    }
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, c);
    const uint32_t e0 = __reduce_min_sync(peers, ordered(b.xmin));
    const uint32_t e1 = __reduce_min_sync(peers, ordered(b.ymin));
    const uint32_t e2 = __reduce_max_sync(peers, ordered(b.xmax));
    const uint32_t e3 = __reduce_max_sync(peers, ordered(b.ymax));
    const uint32_t fl = __reduce_or_sync(peers, b.full ? 1u : 0u);
    if (c >= 0 && (__ffs(peers) - 1) == (int)lane) {
      uint32_t* be = a.box_enc + 4 * (size_t)c;
      atomicMin(be + 0, e0);
      atomicMin(be + 1, e1);
      atomicMax(be + 2, e2);
      atomicMax(be + 3, e3);
      if (fl) atomicOr(a.box_full + c, 1u);
    }
    if (a.partial) {  // OR the bits of one word once per warp
      const uint32_t word = pv ? (t >> 5) : 0xFFFFFFFFu;
      const uint32_t wp = __match_any_sync(0xFFFFFFFFu, word);
      const uint32_t bits = __reduce_or_sync(wp, pv ? (1u << (t & 31)) : 0u);
      if (pv && (__ffs(wp) - 1) == (int)lane) atomicOr(a.partial + word, bits);
    }
  }
}

// ------------------------------------------------------------ compensated fp32

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF{s, err};
}
__device__ __forceinline__ DF quick_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  DF t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  const float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return quick_two_sum(p, lo);
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.hi, b, -p);
  return quick_two_sum(p, __fmaf_rn(a.lo, b, e));
}
// a / b for fp32 a, b: the remainder a - q b is exact for the rounded quotient q.
__device__ __forceinline__ DF df_div(float a, float b) {
  const float q = __fdiv_rn(a, b);
  const float r = __fmaf_rn(-q, b, a);
  return quick_two_sum(q, __fdiv_rn(r, b));
}

struct UvArgs {
  Mat4 M;
  const float* Mdev;  // when set, the matrix is read here on the device instead of M
  const float* pos;
  const uint32_t* idx;
  const uint2* vis;  // (triangle, chart) of the visible triangles
  const int32_t* tri_chart;
  uint32_t T;
  float hx, hy;
  float ratio;
  uint32_t atlas_log2;
  uint32_t n_scales;
  uint32_t gutter;
  const uint32_t* count;
  uint32_t max_charts;
  const float* bbox;
  const uint8_t* rot;
  const fa_placement* place;
  const fa_pack_result* res;
  float* uv;
  float* affine;
  DevCounters* ctr;
  // frame path: placements straight from the selected candidate's records (box b at
  // sorted position pos_of[b]), and written out to place_out
  const uint2* cand_xy;
  const uint2* cand_rec;
  size_t xy_stride, rec_stride;
  const uint32_t* pos_of;
  fa_placement* place_out;
};

__device__ __forceinline__ fa_placement placement_of(const UvArgs& a, uint32_t c, uint32_t kb) {
  if (!a.cand_xy) return a.place[c];
  const uint32_t pos = __ldcg(a.pos_of + c);
  const uint2 q = __ldcg(a.cand_xy + kb * a.xy_stride + pos);
  const uint2 r = __ldcg(a.cand_rec + kb * a.rec_stride + pos);
  return fa_placement{(int32_t)q.x, (int32_t)q.y, (int32_t)(r.x >> 16), (int32_t)(r.y & 0x7FFFFFFFu)};
}

template <bool DEV_M>
__device__ __forceinline__ void uv_body(const UvArgs& a, uint32_t bid, uint32_t nblk) {
  const Mat4 M = DEV_M ? load_mat(a.Mdev) : a.M;
  if (__ldcg(&a.ctr->status) != 0 || __ldcg(&a.res->status) != FA_OK) return;
  const uint32_t k = __ldcg(&a.res->k);
  const float om = (float)(1u << a.atlas_log2), Om = (float)__ldcg(&a.res->omega);
  const DF alpha = df_div(om, Om);
  DF g = quick_two_sum(__fmul_rn(a.ratio, (float)k), __fmaf_rn(a.ratio, (float)k, -__fmul_rn(a.ratio, (float)k)));
  const float inv_n = 1.0f / (float)a.n_scales;  // power of two: exact
  g.hi = __fmul_rn(g.hi, inv_n);
  g.lo = __fmul_rn(g.lo, inv_n);
  const float gut = (float)a.gutter;

  const uint32_t kb = k - 1u;
  // the last blocks take the charts, the others the visible triangles, so that no
  // thread waits on both chains of dependent loads
  // (a one-block grid does both)
  const bool per_chart = a.affine || a.place_out;
  const uint32_t chart_blocks = (per_chart && a.uv && nblk >= 2u) ? max(nblk / 8u, 1u) : 0u;
  const uint32_t tri_blocks = nblk - chart_blocks;
  // per chart: the placement (frame path) and the affine (uv = A . ndc + b)
  if (per_chart && (chart_blocks == 0u || bid >= tri_blocks)) {
    const uint32_t C = min(__ldcg(a.count), a.max_charts);
    const uint32_t c0 = (chart_blocks ? bid - tri_blocks : bid) * blockDim.x + threadIdx.x;
    const uint32_t cstride = (chart_blocks ? chart_blocks : nblk) * blockDim.x;
    for (uint32_t c = c0; c < C; c += cstride) {
      const fa_placement pl = placement_of(a, c, kb);
      if (a.place_out) a.place_out[c] = pl;
      if (!a.affine) continue;
      const float4 bb = reinterpret_cast<const float4*>(a.bbox)[c];
      const DF X = two_sum((float)pl.x, gut), Y = two_sum((float)pl.y, gut);
      const DF agx = df_mul(df_mul_f(alpha, a.hx), g), agy = df_mul(df_mul_f(alpha, a.hy), g);
      const DF gx = df_mul_f(g, a.hx), gy = df_mul_f(g, a.hy);
      float* o = a.affine + 6 * (size_t)c;
      if (__ldcg(a.rot + c)) {
        o[0] = 0.0f;
        o[1] = agy.hi;
        o[2] = df_mul(alpha, df_add(X, df_neg(df_mul_f(gy, bb.y)))).hi;
        o[3] = -agx.hi;
        o[4] = 0.0f;
        o[5] = df_mul(alpha, df_add(Y, df_mul_f(gx, bb.z))).hi;
      } else {
        o[0] = agx.hi;
        o[1] = 0.0f;
        o[2] = df_mul(alpha, df_add(X, df_neg(df_mul_f(gx, bb.x)))).hi;
        o[3] = 0.0f;
        o[4] = agy.hi;
        o[5] = df_mul(alpha, df_add(Y, df_neg(df_mul_f(gy, bb.y)))).hi;
      }
    }
  }
  if (!a.uv || bid >= tri_blocks) return;
  const uint32_t n = __ldcg(&a.ctr->n_vis);
  const uint32_t C = min(__ldcg(a.count), a.max_charts);
  for (uint32_t i = bid * blockDim.x + threadIdx.x; i < n; i += tri_blocks * blockDim.x) {
    const uint2 e = __ldcg(a.vis + i);
    const uint32_t t = e.x;
    const int32_t c = (int32_t)e.y;
    if (c < 0 || (uint32_t)c >= C || t >= a.T) continue;
    const float4 bb = reinterpret_cast<const float4*>(a.bbox)[c];
    const fa_placement pl = placement_of(a, c, kb);
    const bool r = __ldcg(a.rot + c) != 0;
    const DF X = two_sum((float)pl.x, gut), Y = two_sum((float)pl.y, gut);
    const DF wpx = df_mul_f(two_sum(bb.z, -bb.x), a.hx);
    const uint32_t* f = a.idx + 3 * (size_t)t;
    float2* o = reinterpret_cast<float2*>(a.uv + 6 * (size_t)t);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float4 cc = load_clip(M, a.pos, __ldg(f + j));
      if (!(cc.w > 0.0f)) {
        o[j] = make_float2(__int_as_float(0x7fffffff), __int_as_float(0x7fffffff));
        continue;
      }
      const DF nx = df_div(cc.x, cc.w), ny = df_div(cc.y, cc.w);
      const DF px = df_mul_f(df_add(nx, DF{-bb.x, 0.0f}), a.hx);
      const DF py = df_mul_f(df_add(ny, DF{-bb.y, 0.0f}), a.hy);
      DF lu, lv;
      if (r) {
        lu = df_mul(py, g);
        lv = df_mul(df_add(wpx, df_neg(px)), g);
      } else {
        lu = df_mul(px, g);
        lv = df_mul(py, g);
      }
      const DF u = df_mul(df_add(X, lu), alpha), v = df_mul(df_add(Y, lv), alpha);
      o[j] = make_float2(__fadd_rn(u.hi, u.lo), __fadd_rn(v.hi, v.lo));
    }
  }
}

// The box-pass arguments on ctx (host side); the pass walks the context's
// visible-triangle list.
inline BoxArgs make_box_args(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, const int32_t* tri_chart,
                             uint32_t flags, uint32_t* partial, const float* Mdev) {
  BoxArgs a;
  a.M = M;
  a.Mdev = Mdev;
  a.frustum_clip = (flags & FA_BOX_FRUSTUM_CLIP) ? 1u : 0u;
  a.partial = partial;
  a.pos = mesh->pos;
  a.idx = mesh->idx;
  a.vis = ctx->vis;
  a.tri_chart = tri_chart;
  a.T = mesh->T;
  a.box_enc = ctx->box_enc;
  a.box_full = ctx->box_full;
  a.max_charts = ctx->cfg.max_charts;
  a.ctr = ctx->ctr;
  return a;
}

// The UV-pass arguments on ctx (host side).  from_candidates: the frame path, where
// the placements are read from the selected candidate's records and written out.
inline UvArgs make_uv_args(fa_ctx* ctx, const fa_mesh* mesh, const Mat4& M, uint32_t W, uint32_t H, float ratio,
                           const int32_t* tri_chart, const fa_charts* ch, const fa_placement* place,
                           const fa_pack_result* res, uint32_t atlas_log2, uint32_t n_scales, float* uv,
                           float* affine, const float* Mdev, bool from_candidates) {
  UvArgs a;
  a.M = M;
  a.Mdev = Mdev;
  a.pos = mesh->pos;
  a.idx = mesh->idx;
  a.vis = ctx->vis;
  a.tri_chart = tri_chart;
  a.T = mesh->T;
  a.hx = 0.5f * (float)W;
  a.hy = 0.5f * (float)H;
  a.ratio = ratio;
  a.atlas_log2 = atlas_log2;
  a.n_scales = n_scales;
  a.gutter = ctx->cfg.gutter;
  a.count = ch->count;
  a.max_charts = ctx->cfg.max_charts;
  a.bbox = ch->bbox;
  a.rot = ch->rot;
  a.place = place;
  a.res = res;
  a.uv = uv;
  a.affine = affine;
  a.ctr = ctx->ctr;
  a.cand_xy = nullptr;
  a.cand_rec = nullptr;
  a.pos_of = nullptr;
  a.place_out = nullptr;
  a.xy_stride = a.rec_stride = 0;
  if (from_candidates) {
    a.cand_xy = ctx->pack.xy;
    a.cand_rec = ctx->pack.rec8;
    a.xy_stride = ctx->pack.max_boxes;
    a.rec_stride = (size_t)ctx->pack.max_chunks * kChunk;
    a.pos_of = ctx->pack.ord_rank;
    a.place_out = const_cast<fa_placement*>(place);
  }
  return a;
}

}  // namespace
}  // namespace pm
}  // namespace fa
