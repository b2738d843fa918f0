"""Pins for the oracle's visibility step (Sec. 5.1, App. A "Detecting Visible
Triangles"), checked against things the oracle's code does not compute itself:
hand-derived coverage tables, closed-form sample counts, an fp64 ray caster and
geometric special cases."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2502_17712_gb300 import scenes as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")
I4 = np.eye(4, dtype=np.float32)


def screen_to_ndc(p, W, H):
    return np.array([p[0] / (W / 2.0) - 1.0, p[1] / (H / 2.0) - 1.0, 0.0], np.float32)


def key_to_depth(k):
    k = np.asarray(k, np.uint32)
    u = np.where(k & 0x80000000, k & 0x7FFFFFFF, ~k)
    return u.astype(np.uint32).view(np.float32)


# ------------------------------------------------------------------ coverage


def test_golden_coverage_tables():
    g = json.load(open(os.path.join(GOLD, "coverage_tables.json")))
    W, H = g["viewport"]
    for case in g["cases"]:
        v = [screen_to_ndc(p, W, H) for p in case["screen_vertices"]]
        cover, _ = O.raster_triangle(I4, v[0], v[1], v[2], W, H)
        want = np.array([[c == "#" for c in row] for row in case["rows_top_to_bottom"]])[::-1]
        assert (cover == want).all(), case["name"]
        assert cover.sum() == case["count"]


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16])
def test_right_triangle_closed_form_count(n):
    # corners on pixel corners (0,0),(n,0),(0,n): centres strictly below the hypotenuse
    # number n(n-1)/2; centres on it (i + j = n - 1) are excluded by the top-left rule.
    W = H = 32
    v = [screen_to_ndc(p, W, H) for p in [(0, 0), (n, 0), (0, n)]]
    cover, _ = O.raster_triangle(I4, *v, W, H)
    assert cover.sum() == n * (n - 1) // 2


def test_shared_edges_cover_each_centre_once():
    # A pixel-aligned square split along both diagonals into 4 triangles and an
    # off-grid fan: every sample inside the union is covered by exactly one triangle.
    W = H = 16
    rng = np.random.default_rng(3)
    for trial in range(20):
        c = rng.uniform(2, 14, size=2).round(3)
        ring = [(1.0, 1.0), (15.0, 1.0), (15.0, 15.0), (1.0, 15.0)]
        if trial % 2:
            ring = [tuple(rng.uniform(0, 16, 2).round(2)) for _ in range(6)]
            ang = np.arctan2([p[1] - c[1] for p in ring], [p[0] - c[0] for p in ring])
            ring = [ring[i] for i in np.argsort(ang)]
        total = np.zeros((H, W), int)
        for a, b in zip(ring, ring[1:] + ring[:1]):
            tri = [screen_to_ndc(c, W, H), screen_to_ndc(a, W, H), screen_to_ndc(b, W, H)]
            cover, _ = O.raster_triangle(I4, *tri, W, H)
            total += cover
        assert total.max() <= 1
        if trial % 2 == 0:
            # the square [1,15]^2 holds centres 1.5 .. 14.5: 14 x 14 of them
            assert total.sum() == 14 * 14


def test_back_face_and_zero_area_are_culled():
    W = H = 16
    a, b, c = (screen_to_ndc(p, W, H) for p in [(1, 1), (12, 2), (3, 11)])
    assert O.raster_triangle(I4, a, b, c, W, H)[0].sum() > 0
    assert O.raster_triangle(I4, a, c, b, W, H)[0].sum() == 0  # clockwise
    assert O.raster_triangle(I4, a, b, (a + b) / 2, W, H)[0].sum() == 0


def test_fronto_parallel_depth_is_constant():
    W = H = 16
    z = np.float32(0.375)
    v = [screen_to_ndc(p, W, H) for p in [(0.3, 0.7), (15.2, 1.1), (4.4, 15.9)]]
    for p in v:
        p[2] = z
    cover, key = O.raster_triangle(I4, *v, W, H)
    d = key_to_depth(key[cover])
    assert np.all(np.abs(d.astype(np.float64) - 0.375) <= 4 * np.spacing(np.float32(0.375)))


def test_depth_matches_plane_in_fp64():
    # ortho, vertices on the 1/256-pixel grid (snapping is exact): zn is affine in
    # screen space, so the interpolated depth equals the fp64 plane to fp32 accuracy
    W = H = 32
    rng = np.random.default_rng(5)
    for _ in range(10):
        sp = rng.integers(0, 32 * 256, size=(3, 2)) / 256.0
        e1, e2 = sp[1] - sp[0], sp[2] - sp[0]
        if e1[0] * e2[1] - e1[1] * e2[0] < 0:
            sp = sp[[0, 2, 1]]
        z = rng.uniform(-0.9, 0.9, 3)
        v = [screen_to_ndc(p, W, H) for p in sp]
        for p, zz in zip(v, z):
            p[2] = zz
        cover, key = O.raster_triangle(I4, *v, W, H)
        ys, xs = np.nonzero(cover)
        A = np.array([[v[i][0], v[i][1], 1.0] for i in range(3)], np.float64)
        coef = np.linalg.solve(A, np.array([v[i][2] for i in range(3)], np.float64))
        nx = (xs + 0.5) / (W / 2) - 1
        ny = (ys + 0.5) / (H / 2) - 1
        want = coef[0] * nx + coef[1] * ny + coef[2]
        got = key_to_depth(key[ys, xs]).astype(np.float64)
        assert np.all(np.abs(got - want) < 4e-7)


# ------------------------------------------------------------------ z-buffer logic


def _mesh(tris):
    pos = np.array([p for t in tris for p in t], np.float32)
    idx = np.arange(len(pos), dtype=np.uint32).reshape(-1, 3)
    return pos, idx


def test_occluded_triangle_is_invisible_and_coplanar_duplicates_both_visible():
    W = H = 16
    big_near = [(-0.9, -0.9, 0.1), (0.9, -0.9, 0.1), (-0.9, 0.9, 0.1)]
    small_far = [(-0.5, -0.5, 0.5), (0.0, -0.5, 0.5), (-0.5, 0.0, 0.5)]
    pos, idx = _mesh([big_near, small_far, big_near])
    vis = O.vt_to_bool(O.visibility(I4, pos, idx, W, H), 3)
    assert vis.tolist() == [True, False, True]


def test_behind_near_plane_is_invisible_and_crossing_triangle_clipped():
    W = H = 16
    behind = [(-0.5, -0.5, -1.5), (0.5, -0.5, -1.5), (0.0, 0.5, -1.5)]  # z < -w: in front of near
    pos, idx = _mesh([behind])
    assert not O.vt_to_bool(O.visibility(I4, pos, idx, W, H), 1)[0]
    # a triangle whose top part is behind the near plane keeps only its bottom samples
    cross = [(-0.9, -0.9, 0.0), (0.9, -0.9, 0.0), (0.0, 0.9, -2.0)]
    cover, _ = O.raster_triangle(I4, *[np.array(p, np.float32) for p in cross], W, H)
    rows = np.nonzero(cover.any(1))[0]
    # z + w = 1 + z crosses zero halfway up (y = 0): no sample above screen row 8
    assert rows.max() <= 8 and rows.min() == 1


# ------------------------------------------------------------------ fp64 ray caster


def raycast(M, pos, idx, W, H, eps_b=0.03, eps_t=1e-4):
    """Nearest front-facing hit per pixel centre by ray casting in fp64.
    Returns (nearest triangle id or -1 per pixel, per-pixel set of 'ambiguous' ids)."""
    Minv = np.linalg.inv(M.astype(np.float64))
    ys, xs = np.mgrid[0:H, 0:W]
    nx = (xs.ravel() + 0.5) / (W / 2) - 1
    ny = (ys.ravel() + 0.5) / (H / 2) - 1
    P0 = np.stack([nx, ny, -np.ones_like(nx), np.ones_like(nx)], 1) @ Minv.T
    P1 = np.stack([nx, ny, np.ones_like(nx), np.ones_like(nx)], 1) @ Minv.T
    o = P0[:, :3] / P0[:, 3:]
    d = P1[:, :3] / P1[:, 3:] - o
    p = pos.astype(np.float64)[idx.astype(np.int64)]
    e1 = p[:, 1] - p[:, 0]
    e2 = p[:, 2] - p[:, 0]
    n = np.cross(e1, e2)
    npx = o.shape[0]
    best = np.full(npx, -1)
    amb = [set() for _ in range(npx)]
    hits = []
    for t in range(idx.shape[0]):
        front = d @ n[t] < 0
        h = np.cross(d, e2[t])
        a = h @ e1[t]
        with np.errstate(divide="ignore", invalid="ignore"):
            f = 1.0 / a
            s = o - p[t, 0]
            u = f * np.einsum("ij,ij->i", s, h)
            q = np.cross(s, e1[t])
            v = f * np.einsum("ij,ij->i", d, q)
            tt = f * (q @ e2[t])
        bmin = np.minimum(np.minimum(u, v), 1 - u - v)
        ok = front & (tt > 0) & (tt < 1)
        hit = ok & (bmin > eps_b)
        near_edge = ok & (np.abs(bmin) <= eps_b)
        for i in np.nonzero(near_edge | (front & (np.abs(tt) < 1e-3)) & (bmin > -eps_b))[0]:
            amb[i].add(t)
        hits.append((t, hit, tt))
    ts = np.full((idx.shape[0], npx), np.inf)
    for t, hit, tt in hits:
        ts[t, hit] = tt[hit]
    order = np.argsort(ts, axis=0)
    t1 = ts[order[0], np.arange(npx)]
    t2 = ts[order[1], np.arange(npx)] if idx.shape[0] > 1 else np.full(npx, np.inf)
    for i in range(npx):
        if np.isfinite(t1[i]):
            best[i] = order[0, i]
            if t2[i] - t1[i] < eps_t:
                amb[i].update([int(order[0, i]), int(order[1, i])])
    return best, amb


@pytest.mark.parametrize("seed", range(6))
def test_visibility_matches_fp64_ray_caster(seed):
    rng = np.random.default_rng(100 + seed)
    W, H = 40, 30
    M = S.view_proj((0, 0, 0), (0, 0, -1), (0, 1, 0), W, H, near=0.05, far=100.0)
    tris = []
    for i in range(24):
        c = np.array([rng.uniform(-1.2, 1.2), rng.uniform(-0.9, 0.9), rng.uniform(-4, -1)])
        c[:2] *= -c[2] * 0.5
        tri = c + rng.normal(scale=0.35 * -c[2] * 0.4, size=(3, 3))
        if i % 6 == 0:
            tri[0, 2] = 0.4  # behind the camera: crosses the near plane
        tris.append(tri)
    pos, idx = _mesh(tris)
    vis = O.vt_to_bool(O.visibility(M, pos, idx, W, H), len(tris))
    best, amb = raycast(M, pos, idx, W, H)
    seen = set()
    for i in range(W * H):
        if best[i] >= 0 and not amb[i]:
            assert vis[best[i]], f"triangle {best[i]} is nearest at pixel {i} but not marked"
        if best[i] >= 0:
            seen.add(int(best[i]))
        seen.update(amb[i])
    for t in np.nonzero(vis)[0]:
        assert t in seen, f"triangle {t} marked visible but never nearest nor ambiguous"
    assert vis.sum() >= 3


def test_convex_icosphere_visible_set_is_front_facing_covering_triangles():
    # On a closed convex surface seen from outside nothing occludes a front face, so
    # the z-buffer passes mark exactly the triangles that cover at least one sample.
    v, f = S.icosphere(2)
    pos = v.astype(np.float32)
    idx = f.astype(np.uint32)
    W, H = 48, 36
    M = S.view_proj((0.3, -2.5, 1.2), (0, 0, 0), (0, 0, 1), W, H)
    vis = O.vt_to_bool(O.visibility(M, pos, idx, W, H), idx.shape[0])
    covers = np.array([O.raster_triangle(M, *pos[t], W, H)[0].any() for t in idx])
    assert (vis == covers).all()
    assert vis.sum() > 30
    # and no back face is ever marked
    p = pos.astype(np.float64)[idx.astype(np.int64)]
    eye = np.array([0.3, -2.5, 1.2])
    nrm = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    facing = np.einsum("ij,ij->i", nrm, eye - p[:, 0]) > 0
    assert not (vis & ~facing).any()


def test_grid_frame_is_deterministic_and_mostly_visible():
    sc, M, prm = S.heightfield_frame(1)
    a = O.visibility(M, sc.pos, sc.idx, prm["width"], prm["height"])
    b = O.visibility(M, sc.pos, sc.idx, prm["width"], prm["height"])
    assert (a == b).all()
    assert O.vt_to_bool(a, sc.T).sum() > 0.5 * sc.T


def test_transform_exact_on_dyadic_inputs():
    # with small dyadic entries every product and sum is exact in fp32, so the pinned
    # fp32 evaluation equals the exact matrix product
    rng = np.random.default_rng(7)
    M = (rng.integers(-64, 64, size=(4, 4)) / 16.0).astype(np.float32)
    pos = (rng.integers(-512, 512, size=(100, 3)) / 64.0).astype(np.float32)
    want = np.c_[pos.astype(np.float64), np.ones(100)] @ M.astype(np.float64).T
    assert (O.transform(M, pos).astype(np.float64) == want).all()
    assert (O.transform(np.eye(4, dtype=np.float32), pos)[:, :3] == pos).all()
