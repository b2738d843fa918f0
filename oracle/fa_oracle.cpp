// FastAtlas per-frame atlasing: plain CPU oracle.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
// CPU-baseline leg load this library.  It shares no code, header, table or
// constant with the CUDA path; it restates the method from the paper
// (FastAtlas, Vining et al., EG 2025) and from the readings written down for the
// places where the paper is silent.  Single-threaded, no blocking, no fusion.
// Build: g++ -O2 -std=c++17 -ffp-contract=off (no fast-math): every fp32
// expression below is evaluated in the order it is written, one rounding per op.
//
// Steps (paper section in brackets):
//   transform        clip = M . [p, 1]                           [Sec. 5.2]
//   visibility       depth pre-pass + "<=" marking pass           [Sec. 5.1, App. A]
//   chartify         connected components of visible triangles    [Sec. 5.1, App. A, Alg. 1]
//   parameterize     near-clip (or best single frustum plane) + Blinn-clamped NDC
//                    box, viewport; partial-visibility bits
//                    size, quantized footprint, rotate tall        [Sec. 5.2, Sec. 4.1]
//   order            (height desc, root asc)                      [Sec. 4.1]
//   pack             64 candidate scales: prefix-sum fold, overflow
//                    rescale, push-up; select                      [Sec. 4.2, 4.3]
//   uv               projection parameterization into the atlas   [Sec. 3, App. A]
//
// Parity status: every function here is pinned by tests under tests/ against
// values the mathematics fixes (brute force, textbook routines, invariants).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <utility>
#include <vector>

namespace {

// Guard band for the visibility raster: the clipped polygon keeps |x|,|y| <= 64 w,
// which bounds the 1/256-pixel fixed-point coordinates well inside int64 products.
const float kGuard = 64.0f;
const int64_t kSub = 256;           // sub-pixel steps per pixel
const uint32_t kMaxH = 8192;        // height buckets (Sec. 4.1, max_H)

struct Clip {
  float x, y, z, w;
};

// clip = M . [p, 1], M row-major; each row as ((m0 x + m1 y) + m2 z) + m3.
Clip transform(const float* M, const float* p) {
  float r[4];
  for (int i = 0; i < 4; ++i) {
    float acc = M[4 * i + 0] * p[0];
    acc = acc + M[4 * i + 1] * p[1];
    acc = acc + M[4 * i + 2] * p[2];
    acc = acc + M[4 * i + 3];
    r[i] = acc;
  }
  return Clip{r[0], r[1], r[2], r[3]};
}

// Signed distance to clip plane `pl` (inside iff >= 0).
//   0: near plane z >= -w (OpenGL convention)
//   1..4: guard band x <= G w, x >= -G w, y <= G w, y >= -G w
float plane_dist(const Clip& c, int pl) {
  switch (pl) {
    case 0: return c.z + c.w;
    case 1: return kGuard * c.w - c.x;
    case 2: return kGuard * c.w + c.x;
    case 3: return kGuard * c.w - c.y;
    default: return kGuard * c.w + c.y;
  }
}

// Signed distance to frustum plane `pl` of the box variant (inside iff >= 0):
//   0 left x >= -w, 1 right x <= w, 2 bottom y >= -w, 3 top y <= w, 4 far z <= w.
float frustum_dist(const Clip& c, int pl) {
  switch (pl) {
    case 0: return c.x + c.w;
    case 1: return c.w - c.x;
    case 2: return c.y + c.w;
    case 3: return c.w - c.y;
    default: return c.w - c.z;
  }
}

// Point on segment a->b where the plane is crossed; a is the inside end.
Clip intersect(const Clip& a, const Clip& b, float da, float db) {
  float t = da / (da - db);
  Clip r;
  r.x = a.x + t * (b.x - a.x);
  r.y = a.y + t * (b.y - a.y);
  r.z = a.z + t * (b.z - a.z);
  r.w = a.w + t * (b.w - a.w);
  return r;
}

// Sutherland-Hodgman against one plane.
std::vector<Clip> clip_poly(const std::vector<Clip>& in, int pl) {
  std::vector<Clip> out;
  size_t n = in.size();
  for (size_t i = 0; i < n; ++i) {
    const Clip& c = in[i];
    const Clip& nx = in[(i + 1) % n];
    float dc = plane_dist(c, pl), dn = plane_dist(nx, pl);
    bool ic = dc >= 0.0f, in_ = dn >= 0.0f;
    if (ic) out.push_back(c);
    if (ic != in_) {
      if (ic) out.push_back(intersect(c, nx, dc, dn));
      else out.push_back(intersect(nx, c, dn, dc));
    }
  }
  return out;
}

// Sutherland-Hodgman against one frustum plane of the box variant.
std::vector<Clip> clip_frustum(const std::vector<Clip>& in, int pl) {
  std::vector<Clip> out;
  size_t n = in.size();
  for (size_t i = 0; i < n; ++i) {
    const Clip& c = in[i];
    const Clip& nx = in[(i + 1) % n];
    float dc = frustum_dist(c, pl), dn = frustum_dist(nx, pl);
    bool ic = dc >= 0.0f, in_ = dn >= 0.0f;
    if (ic) out.push_back(c);
    if (ic != in_) {
      if (ic) out.push_back(intersect(c, nx, dc, dn));
      else out.push_back(intersect(nx, c, dn, dc));
    }
  }
  return out;
}

struct SVert {
  int64_t X, Y;  // 1/256 pixel, y up
  float zn;      // z / w
};

int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

int64_t edge_fn(const SVert& a, const SVert& b, int64_t px, int64_t py) {
  return (b.X - a.X) * (py - a.Y) - (b.Y - a.Y) * (px - a.X);
}

bool top_left(const SVert& a, const SVert& b) {
  int64_t dx = b.X - a.X, dy = b.Y - a.Y;
  return dy < 0 || (dy == 0 && dx < 0);
}

uint32_t depth_key(float d) {
  uint32_t u;
  std::memcpy(&u, &d, 4);
  if (u == 0x80000000u) u = 0u;  // -0 -> +0
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Visit every covered sample of one mesh triangle: clip against the near plane and
// the guard band, project, snap to 1/256 px (round half even), fan-triangulate,
// cull back faces / zero area, test pixel centres with the top-left rule, and
// interpolate z/w.  fn(px, py, key) is called per covered sample with a valid depth.
template <class Fn>
void raster_triangle(const float* M, const float* p0, const float* p1, const float* p2,
                     int Wv, int Hv, Fn&& fn) {
  std::vector<Clip> poly = {transform(M, p0), transform(M, p1), transform(M, p2)};
  for (int pl = 0; pl < 5 && poly.size() >= 3; ++pl) poly = clip_poly(poly, pl);
  if (poly.size() < 3) return;
  for (const Clip& c : poly)
    if (!(c.w > 0.0f)) return;
  const float hx = 0.5f * (float)Wv, hy = 0.5f * (float)Hv;
  std::vector<SVert> sv;
  for (const Clip& c : poly) {
    float nx = c.x / c.w, ny = c.y / c.w, zn = c.z / c.w;
    float xs = (nx + 1.0f) * hx, ys = (ny + 1.0f) * hy;
    SVert s;
    s.X = (int64_t)std::llrint((double)(xs * 256.0f));
    s.Y = (int64_t)std::llrint((double)(ys * 256.0f));
    s.zn = zn;
    sv.push_back(s);
  }
  for (size_t i = 1; i + 1 < sv.size(); ++i) {
    const SVert& a = sv[0];
    const SVert& b = sv[i];
    const SVert& c = sv[i + 1];
    int64_t A = (b.X - a.X) * (c.Y - a.Y) - (c.X - a.X) * (b.Y - a.Y);
    if (A <= 0) continue;  // back face or zero area
    float invA = 1.0f / (float)A;
    int64_t xmn = std::min({a.X, b.X, c.X}), xmx = std::max({a.X, b.X, c.X});
    int64_t ymn = std::min({a.Y, b.Y, c.Y}), ymx = std::max({a.Y, b.Y, c.Y});
    int64_t px0 = -floor_div(-(xmn - kSub / 2), kSub), px1 = floor_div(xmx - kSub / 2, kSub);
    int64_t py0 = -floor_div(-(ymn - kSub / 2), kSub), py1 = floor_div(ymx - kSub / 2, kSub);
    px0 = std::max<int64_t>(px0, 0);
    py0 = std::max<int64_t>(py0, 0);
    px1 = std::min<int64_t>(px1, Wv - 1);
    py1 = std::min<int64_t>(py1, Hv - 1);
    bool tl0 = top_left(b, c), tl1 = top_left(c, a), tl2 = top_left(a, b);
    for (int64_t py = py0; py <= py1; ++py) {
      for (int64_t px = px0; px <= px1; ++px) {
        int64_t sx = px * kSub + kSub / 2, sy = py * kSub + kSub / 2;
        int64_t e0 = edge_fn(b, c, sx, sy);
        int64_t e1 = edge_fn(c, a, sx, sy);
        int64_t e2 = edge_fn(a, b, sx, sy);
        bool in = (e0 > 0 || (e0 == 0 && tl0)) && (e1 > 0 || (e1 == 0 && tl1)) &&
                  (e2 > 0 || (e2 == 0 && tl2));
        if (!in) continue;
        float f0 = (float)e0, f1 = (float)e1, f2 = (float)e2;
        float s = f0 * a.zn;
        s = s + f1 * b.zn;
        s = s + f2 * c.zn;
        float d = s * invA;
        if (!(d >= -1.0f && d <= 1.0f)) continue;
        fn((int)px, (int)py, depth_key(d));
      }
    }
  }
}

// Conservative coverage of one mesh triangle for the marking pass (App. A marks with
// conservative rasterization): the same clipping, snapping, fan and culling as
// raster_triangle; a pixel is covered when its closed square meets the closed
// sub-triangle (for each edge, the edge function at the square corner where it is
// largest is >= 0; the pixel range is that of the sub-triangle's bounding box).
// Depth: at a pixel whose centre the sample rule covers, the pre-pass depth there;
// otherwise the plane extrapolated to the centre, clamped to the sub-triangle's
// vertex depths.  fn(px, py, key) per covered pixel with a depth in [-1, 1].
template <class Fn>
void raster_conservative(const float* M, const float* p0, const float* p1, const float* p2,
                         int Wv, int Hv, Fn&& fn) {
  std::vector<Clip> poly = {transform(M, p0), transform(M, p1), transform(M, p2)};
  for (int pl = 0; pl < 5 && poly.size() >= 3; ++pl) poly = clip_poly(poly, pl);
  if (poly.size() < 3) return;
  for (const Clip& c : poly)
    if (!(c.w > 0.0f)) return;
  const float hx = 0.5f * (float)Wv, hy = 0.5f * (float)Hv;
  std::vector<SVert> sv;
  for (const Clip& c : poly) {
    float nx = c.x / c.w, ny = c.y / c.w, zn = c.z / c.w;
    float xs = (nx + 1.0f) * hx, ys = (ny + 1.0f) * hy;
    SVert s;
    s.X = (int64_t)std::llrint((double)(xs * 256.0f));
    s.Y = (int64_t)std::llrint((double)(ys * 256.0f));
    s.zn = zn;
    sv.push_back(s);
  }
  for (size_t i = 1; i + 1 < sv.size(); ++i) {
    const SVert& a = sv[0];
    const SVert& b = sv[i];
    const SVert& c = sv[i + 1];
    int64_t A = (b.X - a.X) * (c.Y - a.Y) - (c.X - a.X) * (b.Y - a.Y);
    if (A <= 0) continue;  // back face or zero area
    float invA = 1.0f / (float)A;
    const float zmin = std::min({a.zn, b.zn, c.zn}), zmax = std::max({a.zn, b.zn, c.zn});
    int64_t xmn = std::min({a.X, b.X, c.X}), xmx = std::max({a.X, b.X, c.X});
    int64_t ymn = std::min({a.Y, b.Y, c.Y}), ymx = std::max({a.Y, b.Y, c.Y});
    // squares [px, px + 1] meeting [xmn, xmx] (in pixels): ceil(xmn) - 1 .. floor(xmx)
    int64_t px0 = -floor_div(-xmn, kSub) - 1, px1 = floor_div(xmx, kSub);
    int64_t py0 = -floor_div(-ymn, kSub) - 1, py1 = floor_div(ymx, kSub);
    px0 = std::max<int64_t>(px0, 0);
    py0 = std::max<int64_t>(py0, 0);
    px1 = std::min<int64_t>(px1, Wv - 1);
    py1 = std::min<int64_t>(py1, Hv - 1);
    bool tl0 = top_left(b, c), tl1 = top_left(c, a), tl2 = top_left(a, b);
    const SVert* ea[3] = {&b, &c, &a};
    const SVert* eb[3] = {&c, &a, &b};
    for (int64_t py = py0; py <= py1; ++py) {
      for (int64_t px = px0; px <= px1; ++px) {
        bool meets = true;
        for (int k = 0; k < 3 && meets; ++k) {
          const SVert& u = *ea[k];
          const SVert& v = *eb[k];
          // E(x, y) = (v.X - u.X)(y - u.Y) - (v.Y - u.Y)(x - u.X): largest at the corner
          // with x high iff -(v.Y - u.Y) > 0 and y high iff (v.X - u.X) > 0
          const int64_t cx = (u.Y - v.Y) > 0 ? (px + 1) * kSub : px * kSub;
          const int64_t cy = (v.X - u.X) > 0 ? (py + 1) * kSub : py * kSub;
          meets = edge_fn(u, v, cx, cy) >= 0;
        }
        if (!meets) continue;
        int64_t sx = px * kSub + kSub / 2, sy = py * kSub + kSub / 2;
        int64_t e0 = edge_fn(b, c, sx, sy);
        int64_t e1 = edge_fn(c, a, sx, sy);
        int64_t e2 = edge_fn(a, b, sx, sy);
        bool in = (e0 > 0 || (e0 == 0 && tl0)) && (e1 > 0 || (e1 == 0 && tl1)) &&
                  (e2 > 0 || (e2 == 0 && tl2));
        float f0 = (float)e0, f1 = (float)e1, f2 = (float)e2;
        float s = f0 * a.zn;
        s = s + f1 * b.zn;
        s = s + f2 * c.zn;
        float d = s * invA;
        if (!in) d = std::min(std::max(d, zmin), zmax);
        if (!(d >= -1.0f && d <= 1.0f)) continue;
        fn((int)px, (int)py, depth_key(d));
      }
    }
  }
}

// Near-plane clip (only), then Blinn's clamp x,y to [-w, w] and divide.
// Returns false when a vertex with w <= 0 survives (box becomes [-1,1]^2).
// Blinn's estimator over a polygon: clamp x, y to [-w, w], divide by w, and widen
// box[4] = (xmin, ymin, xmax, ymax).  False when a vertex has w <= 0.
bool blinn_add(const std::vector<Clip>& poly, float box[4]) {
  for (const Clip& c : poly) {
    if (!(c.w > 0.0f)) return false;
    float x = c.x, y = c.y;
    if (x < -c.w) x = -c.w;
    if (x > c.w) x = c.w;
    if (y < -c.w) y = -c.w;
    if (y > c.w) y = c.w;
    float nx = x / c.w, ny = y / c.w;
    if (nx == 0.0f) nx = 0.0f;  // -0 -> +0
    if (ny == 0.0f) ny = 0.0f;
    box[0] = std::min(box[0], nx);
    box[1] = std::min(box[1], ny);
    box[2] = std::max(box[2], nx);
    box[3] = std::max(box[3], ny);
  }
  return true;
}

// Conservative NDC box of one visible triangle (Sec. 5.2), widening box[4]: clip
// against the near plane when the triangle crosses it, then Blinn's clamp.  With
// frustum_clip, a triangle that does not cross the near plane is instead clipped
// against the one frustum plane (left, right, bottom, top, far) whose single-plane
// clip gives the smallest Blinn box, area (xmax - xmin) * (ymax - ymin) in fp32,
// ties to the first plane in that order (a plane the triangle does not cross leaves
// it whole).  False when the box must become [-1, 1]^2 (a vertex with w <= 0).
bool blinn_box(const float* M, const float* p0, const float* p1, const float* p2, float box[4],
               bool* any, bool frustum_clip) {
  std::vector<Clip> tri = {transform(M, p0), transform(M, p1), transform(M, p2)};
  const bool crosses_near = plane_dist(tri[0], 0) < 0.0f || plane_dist(tri[1], 0) < 0.0f ||
                            plane_dist(tri[2], 0) < 0.0f;
  std::vector<Clip> poly = clip_poly(tri, 0);
  *any = poly.size() >= 3;
  if (!frustum_clip || crosses_near) return blinn_add(poly, box);
  const float inf = std::numeric_limits<float>::infinity();
  float best[4] = {inf, inf, -inf, -inf};
  bool best_ok = true, have = false;
  float best_area = 0.0f;
  for (int pl = 0; pl < 5; ++pl) {
    std::vector<Clip> cp = clip_frustum(tri, pl);
    if (cp.size() < 3) continue;  // wholly outside this plane: not a candidate
    float b[4] = {inf, inf, -inf, -inf};
    const bool ok = blinn_add(cp, b);
    const float area = ok ? (b[2] - b[0]) * (b[3] - b[1]) : inf;
    if (!have || area < best_area) {
      have = true;
      best_area = area;
      best_ok = ok;
      for (int k = 0; k < 4; ++k) best[k] = b[k];
    }
  }
  if (!have) return blinn_add(tri, box);
  if (!best_ok) return false;
  for (int k = 0; k < 2; ++k) box[k] = std::min(box[k], best[k]);
  for (int k = 2; k < 4; ++k) box[k] = std::max(box[k], best[k]);
  return true;
}

// Partial visibility (Sec. 6, temporal re-use): a vertex with max(|x|, |y|) >= w in
// clip coordinates.
bool partially_visible(const float* M, const float* p0, const float* p1, const float* p2) {
  const float* p[3] = {p0, p1, p2};
  for (int k = 0; k < 3; ++k) {
    const Clip c = transform(M, p[k]);
    if (std::max(std::fabs(c.x), std::fabs(c.y)) >= c.w) return true;
  }
  return false;
}

}  // namespace

extern "C" {

struct or_pack_result {
  uint32_t k;       // chosen candidate scale numerator (scale = k / n_scales)
  uint32_t omega;   // virtual atlas side Omega = omega + m of the chosen candidate
  uint32_t height;  // H of the chosen candidate (<= Omega)
  int32_t status;   // 0 ok, 4 = no candidate fits
  uint32_t count;   // number of boxes
};

int or_version() { return 1; }

void or_transform(const float* M, const float* pos, int V, float* clip) {
  for (int v = 0; v < V; ++v) {
    Clip c = transform(M, pos + 3 * v);
    clip[4 * v + 0] = c.x;
    clip[4 * v + 1] = c.y;
    clip[4 * v + 2] = c.z;
    clip[4 * v + 3] = c.w;
  }
}

// Coverage of a single triangle: cover[py*Wv+px] = 1 and key[...] = min depth key;
// sample coverage, or the conservative coverage of the marking pass.
void or_raster_triangle(const float* M, const float* p0, const float* p1, const float* p2, int Wv,
                        int Hv, uint8_t* cover, uint32_t* key, int conservative) {
  for (int i = 0; i < Wv * Hv; ++i) {
    cover[i] = 0;
    key[i] = 0xFFFFFFFFu;
  }
  auto put = [&](int px, int py, uint32_t k) {
    size_t o = (size_t)py * Wv + px;
    cover[o] = 1;
    key[o] = std::min(key[o], k);
  };
  if (conservative)
    raster_conservative(M, p0, p1, p2, Wv, Hv, put);
  else
    raster_triangle(M, p0, p1, p2, Wv, Hv, put);
}

// Depth pre-pass then marking pass with the "<=" test (App. A, Detecting Visible
// Triangles).  vt: ceil(T/32) words, bit t%32 of word t/32.  zbuf may be null.
void or_visibility(const float* M, const float* pos, const uint32_t* idx, int T, int Wv, int Hv,
                   uint32_t* vt, uint32_t* zbuf_out, int conservative) {
  std::vector<uint32_t> zb((size_t)Wv * Hv, 0xFFFFFFFFu);
  for (int t = 0; t < T; ++t) {
    const uint32_t* f = idx + 3 * (size_t)t;
    raster_triangle(M, pos + 3 * f[0], pos + 3 * f[1], pos + 3 * f[2], Wv, Hv,
                    [&](int px, int py, uint32_t k) {
                      size_t o = (size_t)py * Wv + px;
                      if (k < zb[o]) zb[o] = k;
                    });
  }
  int nw = (T + 31) / 32;
  for (int i = 0; i < nw; ++i) vt[i] = 0;
  for (int t = 0; t < T; ++t) {
    const uint32_t* f = idx + 3 * (size_t)t;
    bool vis = false;
    auto test = [&](int px, int py, uint32_t k) {
      if (k <= zb[(size_t)py * Wv + px]) vis = true;
    };
    if (conservative)
      raster_conservative(M, pos + 3 * f[0], pos + 3 * f[1], pos + 3 * f[2], Wv, Hv, test);
    else
      raster_triangle(M, pos + 3 * f[0], pos + 3 * f[1], pos + 3 * f[2], Wv, Hv, test);
    if (vis) vt[t >> 5] |= 1u << (t & 31);
  }
  if (zbuf_out) std::memcpy(zbuf_out, zb.data(), zb.size() * 4);
}

// Charts = connected components of the visible triangles (Sec. 5.1): under shared
// undirected edges {a, b}, a != b, of the index buffer (mode 0), or under shared
// vertices (mode 1, the vertex merge of App. A).  Root = smallest triangle id of the
// component; charts are numbered by ascending root.  Invisible triangles get -1.
// Returns the chart count, or -1 if it exceeds max_charts.
int or_chartify(const uint32_t* idx, int T, int V, const uint32_t* vt, int mode,
                int32_t* tri_chart, uint32_t* roots, int max_charts, int32_t* vert_chart) {
  auto visible = [&](int t) { return (vt[t >> 5] >> (t & 31)) & 1u; };
  // group visible triangles by key (edge or vertex), chain each group
  std::vector<std::pair<uint64_t, int>> keyed;
  for (int t = 0; t < T; ++t) {
    if (!visible(t)) continue;
    const uint32_t* f = idx + 3 * (size_t)t;
    for (int j = 0; j < 3; ++j) {
      if (mode == 0) {
        uint32_t a = f[j], b = f[(j + 1) % 3];
        if (a == b) continue;
        uint64_t k = ((uint64_t)std::min(a, b) << 32) | std::max(a, b);
        keyed.push_back({k, t});
      } else {
        keyed.push_back({(uint64_t)f[j], t});
      }
    }
  }
  std::sort(keyed.begin(), keyed.end());
  std::vector<std::vector<int>> nbr(T);
  for (size_t i = 1; i < keyed.size(); ++i) {
    if (keyed[i].first == keyed[i - 1].first && keyed[i].second != keyed[i - 1].second) {
      nbr[keyed[i].second].push_back(keyed[i - 1].second);
      nbr[keyed[i - 1].second].push_back(keyed[i].second);
    }
  }
  for (int t = 0; t < T; ++t) tri_chart[t] = -1;
  int C = 0;
  std::vector<int> queue;
  for (int t = 0; t < T; ++t) {
    if (!visible(t) || tri_chart[t] >= 0) continue;
    if (C >= max_charts) return -1;
    roots[C] = (uint32_t)t;
    tri_chart[t] = C;
    queue.assign(1, t);
    for (size_t q = 0; q < queue.size(); ++q) {
      for (int n : nbr[queue[q]]) {
        if (tri_chart[n] < 0) {
          tri_chart[n] = C;
          queue.push_back(n);
        }
      }
    }
    ++C;
  }
  if (vert_chart) {
    for (int v = 0; v < V; ++v) vert_chart[v] = -1;
    if (mode == 1) {
      for (int t = 0; t < T; ++t) {
        if (tri_chart[t] < 0) continue;
        for (int j = 0; j < 3; ++j) vert_chart[idx[3 * (size_t)t + j]] = tri_chart[t];
      }
    }
  }
  return C;
}

// Per-chart conservative NDC box and quantized footprint (Sec. 5.2, Sec. 4.1).
// bbox[c] = (xmin, ymin, xmax, ymax).  fa <= fb are the 1/256-texel footprint
// sides after the rotate-tall step, rot[c] = 1 when the box was rotated 90 degrees.
void or_parameterize(const float* M, const float* pos, const uint32_t* idx, int T, int Wv, int Hv,
                     float ratio, const int32_t* tri_chart, int C, float* bbox, uint32_t* fa,
                     uint32_t* fb, uint8_t* rot, uint32_t flags, uint32_t* partial) {
  const float inf = std::numeric_limits<float>::infinity();
  std::vector<uint8_t> full(C, 0);
  for (int c = 0; c < C; ++c) {
    bbox[4 * c + 0] = inf;
    bbox[4 * c + 1] = inf;
    bbox[4 * c + 2] = -inf;
    bbox[4 * c + 3] = -inf;
  }
  if (partial)
    for (int w = 0; w < (T + 31) / 32; ++w) partial[w] = 0u;
  for (int t = 0; t < T; ++t) {
    int c = tri_chart[t];
    if (c < 0) continue;
    const uint32_t* f = idx + 3 * (size_t)t;
    bool any;
    if (!blinn_box(M, pos + 3 * f[0], pos + 3 * f[1], pos + 3 * f[2], bbox + 4 * c, &any, (flags & 1u) != 0))
      full[c] = 1;
    if (partial && partially_visible(M, pos + 3 * f[0], pos + 3 * f[1], pos + 3 * f[2]))
      partial[t >> 5] |= 1u << (t & 31);
  }
  const float hx = 0.5f * (float)Wv, hy = 0.5f * (float)Hv, s = 256.0f * ratio;
  for (int c = 0; c < C; ++c) {
    if (full[c]) {
      bbox[4 * c + 0] = -1.0f;
      bbox[4 * c + 1] = -1.0f;
      bbox[4 * c + 2] = 1.0f;
      bbox[4 * c + 3] = 1.0f;
    }
    float wpx = (bbox[4 * c + 2] - bbox[4 * c + 0]) * hx;
    float hpx = (bbox[4 * c + 3] - bbox[4 * c + 1]) * hy;
    uint32_t fw = (uint32_t)std::ceil(s * wpx);
    uint32_t fh = (uint32_t)std::ceil(s * hpx);
    rot[c] = fw > fh ? 1 : 0;
    fa[c] = rot[c] ? fh : fw;
    fb[c] = rot[c] ? fw : fh;
  }
}

// Box order (Sec. 4.1): integer height h0 = ceil(fb / 256) in [1, 8192], descending;
// ties by the box index (charts are numbered by ascending root triangle).
void or_order(const uint32_t* fb, int C, uint32_t* order) {
  std::vector<uint32_t> h0(C);
  for (int c = 0; c < C; ++c) {
    uint32_t h = (uint32_t)(((uint64_t)fb[c] + 255) / 256);
    h0[c] = std::min(std::max(h, 1u), kMaxH);
  }
  for (int c = 0; c < C; ++c) order[c] = (uint32_t)c;
  std::stable_sort(order, order + C, [&](uint32_t a, uint32_t b) { return h0[a] > h0[b]; });
}

// One candidate scale k / n (Sec. 4.3): scaled integer boxes in `order`, exclusive
// prefix sum of widths, row = P >> log2(omega), in-row offset = P & (omega-1),
// overflow m, virtual width Omega = omega + m, rows q with q % 3 == 0 run left to
// right and the others right to left mirrored in Omega, then the row-by-row push
// against the frontline.  Accepted iff H <= Omega.  x, y, w, h are in box order.
void or_pack_candidate(const uint32_t* fa, const uint32_t* fb, const uint32_t* order, int C,
                       int atlas_log2, int k, int n_scales, int min_box, int gutter, uint32_t* x,
                       uint32_t* y, uint32_t* w, uint32_t* h, uint64_t* omega_out,
                       uint64_t* height_out, int* accepted) {
  const uint64_t om = 1ull << atlas_log2, D = 256ull * (uint64_t)n_scales;
  std::vector<uint64_t> P(C), ww(C), hh(C);
  uint64_t acc = 0;
  for (int i = 0; i < C; ++i) {
    uint32_t b = order[i];
    uint64_t sw = ((uint64_t)k * fa[b] + D - 1) / D, sh = ((uint64_t)k * fb[b] + D - 1) / D;
    ww[i] = std::max<uint64_t>(sw, (uint64_t)min_box) + 2ull * gutter;
    hh[i] = std::max<uint64_t>(sh, (uint64_t)min_box) + 2ull * gutter;
    P[i] = acc;
    acc += ww[i];
  }
  uint64_t m = 0;
  for (int i = 0; i < C; ++i) {
    uint64_t xr = P[i] & (om - 1);
    if (xr + ww[i] > om) m = std::max(m, xr + ww[i] - om);
  }
  const uint64_t Om = om + m;
  std::vector<uint64_t> xx(C), yy(C), F(Om, 0);
  for (int i = 0; i < C; ++i) {
    uint64_t q = P[i] >> atlas_log2, xr = P[i] & (om - 1);
    xx[i] = (q % 3 == 0) ? xr : Om - xr - ww[i];
  }
  uint64_t H = 0;
  int i = 0;
  while (i < C) {
    int j = i;
    uint64_t q = P[i] >> atlas_log2;
    while (j < C && (P[j] >> atlas_log2) == q) ++j;
    for (int b = i; b < j; ++b) {
      uint64_t mx = 0;
      for (uint64_t t = xx[b]; t < xx[b] + ww[b]; ++t) mx = std::max(mx, F[t]);
      yy[b] = mx;
    }
    for (int b = i; b < j; ++b) {
      for (uint64_t t = xx[b]; t < xx[b] + ww[b]; ++t) F[t] = yy[b] + hh[b];
      H = std::max(H, yy[b] + hh[b]);
    }
    i = j;
  }
  for (int b = 0; b < C; ++b) {
    x[b] = (uint32_t)xx[b];
    y[b] = (uint32_t)yy[b];
    w[b] = (uint32_t)ww[b];
    h[b] = (uint32_t)hh[b];
  }
  *omega_out = Om;
  *height_out = H;
  *accepted = H <= Om ? 1 : 0;
}

// Scale search and selection (Sec. 4.2): all n_scales candidates, keep those that
// fit; select_mode 0 maximises the effective scale (k / n) * omega / Omega (exact
// integer compare, ties to the larger k), select_mode 1 takes the largest fitting k.
// place[c] = (x, y, w, h) in the chosen candidate's virtual Omega x Omega grid, in
// chart order.  cand_* (optional, n_scales entries) report every candidate.
// Multi-atlas from one packing (Sec. 7, depth of field / foveated rendering): with
// lowres_log2 = d > 0 the packing must also serve an atlas scaled by 2^-d.  Two
// charts' contents are at least 2 gutter virtual texels apart, alpha * 2 * gutter
// atlas texels, 2^-d of that in the low-resolution atlas; they share no
// low-resolution texel when that gap is >= 1, i.e. 2 * gutter * omega >= Omega * 2^d,
// which a candidate must then satisfy besides H <= Omega.
void or_pack(const uint32_t* fa, const uint32_t* fb, int C, int atlas_log2, int n_scales,
             int min_box, int gutter, int select_mode, int32_t* place, or_pack_result* res,
             uint64_t* cand_omega, uint64_t* cand_height, int32_t* cand_ok, int lowres_log2) {
  std::vector<uint32_t> order(C);
  or_order(fb, C, order.data());
  std::vector<uint64_t> Om(n_scales + 1), Hk(n_scales + 1);
  std::vector<int> ok(n_scales + 1);
  std::vector<uint32_t> x(C), y(C), w(C), h(C);
  for (int k = 1; k <= n_scales; ++k) {
    or_pack_candidate(fa, fb, order.data(), C, atlas_log2, k, n_scales, min_box, gutter, x.data(),
                      y.data(), w.data(), h.data(), &Om[k], &Hk[k], &ok[k]);
    if (lowres_log2 > 0 && (Om[k] << lowres_log2) > 2ull * (uint64_t)gutter * (1ull << atlas_log2)) ok[k] = 0;
    if (cand_omega) cand_omega[k - 1] = Om[k];
    if (cand_height) cand_height[k - 1] = Hk[k];
    if (cand_ok) cand_ok[k - 1] = ok[k];
  }
  int best = 0;
  for (int k = 1; k <= n_scales; ++k) {
    if (!ok[k]) continue;
    if (best == 0) {
      best = k;
    } else if (select_mode == 1) {
      best = k;
    } else if ((unsigned __int128)k * Om[best] >= (unsigned __int128)best * Om[k]) {
      best = k;
    }
  }
  res->count = (uint32_t)C;
  if (best == 0) {
    res->k = 0;
    res->omega = 0;
    res->height = 0;
    res->status = 4;
    return;
  }
  or_pack_candidate(fa, fb, order.data(), C, atlas_log2, best, n_scales, min_box, gutter, x.data(),
                    y.data(), w.data(), h.data(), &Om[best], &Hk[best], &ok[best]);
  for (int i = 0; i < C; ++i) {
    uint32_t b = order[i];
    place[4 * b + 0] = (int32_t)x[i];
    place[4 * b + 1] = (int32_t)y[i];
    place[4 * b + 2] = (int32_t)w[i];
    place[4 * b + 3] = (int32_t)h[i];
  }
  res->k = (uint32_t)best;
  res->omega = (uint32_t)Om[best];
  res->height = (uint32_t)Hk[best];
  res->status = 0;
}

// Projection parameterization (Sec. 3, App. A "Shading and Rasterization"): each
// visible corner maps to alpha * ((x + g, y + g) + local), alpha = omega / Omega,
// local = s * ((ndc - box_min) * viewport / 2), s = ratio * k / n_scales, and for a
// rotated chart local = (s * py, s * (Wpx - px)).  fp64 from the fp32 clip values.
// uv[t][j] = (u, v) in atlas texels; NaN for w <= 0; untouched for invisible t.
// affine[c] = (a11, a12, b1, a21, a22, b2): uv = A . ndc + b.
void or_uv(const float* M, const float* pos, const uint32_t* idx, int T, int Wv, int Hv,
           float ratio, const int32_t* tri_chart, int C, const float* bbox, const uint8_t* rot,
           const int32_t* place, const or_pack_result* res, int atlas_log2, int n_scales, int gutter,
           double* uv, double* affine) {
  if (res->status != 0) return;
  const double alpha = (double)(1u << atlas_log2) / (double)res->omega;
  const double g = (double)ratio * (double)res->k / (double)n_scales;
  const double hx = 0.5 * Wv, hy = 0.5 * Hv;
  for (int t = 0; t < T; ++t) {
    int c = tri_chart[t];
    if (c < 0) continue;
    const double X = place[4 * c + 0] + gutter, Y = place[4 * c + 1] + gutter;
    const double xmin = bbox[4 * c + 0], ymin = bbox[4 * c + 1], xmax = bbox[4 * c + 2];
    for (int j = 0; j < 3; ++j) {
      Clip cc = transform(M, pos + 3 * (size_t)idx[3 * (size_t)t + j]);
      double* o = uv + 6 * (size_t)t + 2 * j;
      if (!(cc.w > 0.0f)) {
        o[0] = o[1] = std::numeric_limits<double>::quiet_NaN();
        continue;
      }
      double ndx = (double)cc.x / (double)cc.w, ndy = (double)cc.y / (double)cc.w;
      double px = (ndx - xmin) * hx, py = (ndy - ymin) * hy;
      double lu, lv;
      if (rot[c]) {
        lu = py * g;
        lv = ((xmax - xmin) * hx - px) * g;
      } else {
        lu = px * g;
        lv = py * g;
      }
      o[0] = alpha * (X + lu);
      o[1] = alpha * (Y + lv);
    }
  }
  for (int c = 0; c < C; ++c) {
    const double X = place[4 * c + 0] + gutter, Y = place[4 * c + 1] + gutter;
    const double xmin = bbox[4 * c + 0], ymin = bbox[4 * c + 1], xmax = bbox[4 * c + 2];
    double* a = affine + 6 * (size_t)c;
    if (rot[c]) {
      a[0] = 0.0;
      a[1] = alpha * g * hy;
      a[2] = alpha * (X - g * hy * ymin);
      a[3] = -alpha * g * hx;
      a[4] = 0.0;
      a[5] = alpha * (Y + g * hx * xmax);
    } else {
      a[0] = alpha * g * hx;
      a[1] = 0.0;
      a[2] = alpha * (X - g * hx * xmin);
      a[3] = 0.0;
      a[4] = alpha * g * hy;
      a[5] = alpha * (Y - g * hy * ymin);
    }
  }
}

}  // extern "C"
