"""Pins for the oracle's chartify step (Sec. 5.1, App. A "GPU Union Find", Alg. 1)
and parameterize step (Sec. 5.2 bounding boxes, Sec. 4.1 rotate tall)."""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle as O
from paper_2502_17712_gb300 import scenes as S


def components_scipy(idx, vis, mode):
    """Textbook connected components (scipy) of the visible triangles."""
    T = idx.shape[0]
    rows, cols = [], []
    groups = {}
    for t in np.nonzero(vis)[0]:
        f = [int(x) for x in idx[t]]
        keys = []
        if mode == 0:
            for j in range(3):
                a, b = f[j], f[(j + 1) % 3]
                if a != b:
                    keys.append((min(a, b), max(a, b)))
        else:
            keys = [(v,) for v in f]
        for k in keys:
            groups.setdefault(k, []).append(int(t))
    for members in groups.values():
        for m in members[1:]:
            rows.append(members[0])
            cols.append(m)
    g = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(T, T))
    n, lab = connected_components(g, directed=False)
    # canonical numbering: visible components by ascending smallest member
    out = np.full(T, -1, np.int64)
    vis_t = np.nonzero(vis)[0]
    mins = {}
    for t in vis_t:
        mins.setdefault(lab[t], t)
    order = sorted(mins.values())
    rank = {lab[r]: i for i, r in enumerate(order)}
    for t in vis_t:
        out[t] = rank[lab[t]]
    return out, np.array(order, np.int64)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("frac", [0.2, 0.5, 0.8])
def test_chartify_matches_scipy_components(mode, frac):
    sc = S.grid_scene(2, n=24)
    rng = np.random.default_rng(int(frac * 10) + mode)
    vis = rng.random(sc.T) < frac
    vt = O.bool_to_vt(vis)
    ch = O.chartify(sc.idx, sc.V, vt, mode)
    want, roots = components_scipy(sc.idx, vis, mode)
    assert (ch.tri_chart == want).all()
    assert (ch.roots == roots).all()
    if mode == 1:
        # vertToChart: every vertex of a visible triangle maps to that triangle's chart
        for t in np.nonzero(vis)[0]:
            assert (ch.vert_chart[sc.idx[t]] == ch.tri_chart[t]).all()


def test_chartify_special_cases():
    sc = S.grid_scene(2, n=16)
    full = np.ones(sc.T, bool)
    ch = O.chartify(sc.idx, sc.V, O.bool_to_vt(full), 0)
    assert ch.C == 1 and ch.roots.tolist() == [0] and (ch.tri_chart == 0).all()
    # checkerboard: even triangles only share edges with odd ones
    even = np.arange(sc.T) % 2 == 0
    ch = O.chartify(sc.idx, sc.V, O.bool_to_vt(even), 0)
    assert ch.C == sc.T // 2 + (sc.T % 2)
    assert (ch.roots == np.arange(0, sc.T, 2)).all()
    ch = O.chartify(sc.idx, sc.V, O.bool_to_vt(even), 1)
    assert ch.C == 1
    none = np.zeros(sc.T, bool)
    ch = O.chartify(sc.idx, sc.V, O.bool_to_vt(none), 0)
    assert ch.C == 0 and (ch.tri_chart == -1).all()


def test_chartify_non_manifold_and_degenerate():
    # four triangles fan around edge (0,1); triangles 4 and 5 are degenerate
    # (0,0,5), (0,0,7): {0,0} is not an edge, so they share no edge with anything,
    # but they share vertex 0 with the fan.
    idx = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4], [1, 0, 6], [0, 0, 5], [0, 0, 7]], np.uint32)
    vis = np.array([1, 0, 1, 1, 1, 1], bool)
    ch = O.chartify(idx, 8, O.bool_to_vt(vis), 0)
    assert ch.tri_chart.tolist() == [0, -1, 0, 0, 1, 2]
    ch = O.chartify(idx, 8, O.bool_to_vt(vis), 1)
    assert ch.tri_chart.tolist() == [0, -1, 0, 0, 0, 0]


def test_chartify_charts_are_connected_and_disjoint_on_frame():
    sc, M, p = S.heightfield_frame(3)
    vt = O.visibility(M, sc.pos, sc.idx, p["width"], p["height"])
    vis = O.vt_to_bool(vt, sc.T)
    for mode in (0, 1):
        ch = O.chartify(sc.idx, sc.V, vt, mode)
        want, _ = components_scipy(sc.idx, vis, mode)
        assert (ch.tri_chart == want).all()
        assert ((ch.tri_chart >= 0) == vis).all()


# ---------------------------------------------------------------- parameterize


def frustum_clip_fp64(clip_tri):
    """Exact-ish (fp64) Sutherland-Hodgman of a clip-space triangle against all six
    frustum planes; returns the NDC x,y of the clipped polygon (may be empty)."""
    poly = [np.asarray(c, np.float64) for c in clip_tri]
    planes = [lambda c: c[3] + c[2], lambda c: c[3] - c[2], lambda c: c[3] - c[0],
              lambda c: c[3] + c[0], lambda c: c[3] - c[1], lambda c: c[3] + c[1]]
    for pl in planes:
        out = []
        for i in range(len(poly)):
            a, b = poly[i], poly[(i + 1) % len(poly)]
            da, db = pl(a), pl(b)
            if da >= 0:
                out.append(a)
            if (da >= 0) != (db >= 0):
                out.append(a + (da / (da - db)) * (b - a))
        poly = out
        if not poly:
            return np.zeros((0, 2))
    P = np.array(poly)
    return P[:, :2] / P[:, 3:4]


def test_blinn_box_single_triangle_closed_form():
    # fully inside the frustum: the box is the min/max of the projected vertices
    W, H = 64, 48
    M = S.view_proj((0, 0, 3), (0, 0, 0), (0, 1, 0), W, H)
    pos = np.array([[-0.5, -0.4, 0.1], [0.6, -0.2, -0.3], [0.1, 0.5, 0.2]], np.float32)
    idx = np.array([[0, 1, 2]], np.uint32)
    fp = O.parameterize(M, pos, idx, W, H, 1.0, np.array([0], np.int32), 1)
    c = np.c_[pos.astype(np.float64), np.ones(3)] @ M.astype(np.float64).T
    ndc = c[:, :2] / c[:, 3:]
    want = np.r_[ndc.min(0), ndc.max(0)]
    assert np.allclose(fp.bbox[0], want, rtol=0, atol=1e-6)
    # footprint: ceil(256 * r * viewport size) in 1/256 texel, tall after rotation
    wpx = (want[2] - want[0]) * W / 2
    hpx = (want[3] - want[1]) * H / 2
    lo, hi = sorted([wpx, hpx])
    assert abs(fp.fa[0] / 256.0 - lo) <= 1 / 256 + 1e-4 and fp.fa[0] >= 256 * lo - 0.05
    assert abs(fp.fb[0] / 256.0 - hi) <= 1 / 256 + 1e-4 and fp.fb[0] >= 256 * hi - 0.05
    assert fp.rot[0] == (wpx > hpx)


@pytest.mark.parametrize("seed", range(8))
def test_box_is_conservative_and_within_screen(seed):
    """Box contains the exact 6-plane clip of every chart triangle, lies in [-1,1]^2,
    and the near-clipped box is inside the box of Blinn's clamp without clipping."""
    rng = np.random.default_rng(seed)
    W, H = 64, 48
    M = S.view_proj((0, 0, 0), (0, 0, -1), (0, 1, 0), W, H)
    n = 6
    pos = rng.normal(scale=1.5, size=(3 * n, 3)) + np.array([0, 0, -2.0])
    pos[::5, 2] = 0.5  # some vertices behind the camera
    pos = pos.astype(np.float32)
    idx = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    tc = np.zeros(n, np.int32)
    fp = O.parameterize(M, pos, idx, W, H, 1.0, tc, 1)
    box = fp.bbox[0].astype(np.float64)
    assert box[0] >= -1 and box[1] >= -1 and box[2] <= 1 and box[3] <= 1
    c = np.c_[pos.astype(np.float64), np.ones(3 * n)] @ M.astype(np.float64).T
    exact = []
    for t in range(n):
        P = frustum_clip_fp64(c[3 * t:3 * t + 3])
        if len(P):
            exact.append(P)
    if exact:
        E = np.concatenate(exact)
        tol = 1e-5
        assert (E[:, 0] >= box[0] - tol).all() and (E[:, 0] <= box[2] + tol).all()
        assert (E[:, 1] >= box[1] - tol).all() and (E[:, 1] <= box[3] + tol).all()
    # Blinn without the near clip, only possible when every w > 0 (Fig. "bbox_clip_alt")
    if (c[:, 3] > 0).all():
        cx = np.clip(c[:, 0], -c[:, 3], c[:, 3]) / c[:, 3]
        cy = np.clip(c[:, 1], -c[:, 3], c[:, 3]) / c[:, 3]
        assert box[0] >= cx.min() - 1e-6 and box[2] <= cx.max() + 1e-6
        assert box[1] >= cy.min() - 1e-6 and box[3] <= cy.max() + 1e-6


def test_near_clip_shrinks_box_of_triangle_through_near_plane():
    # The apex sits between the eye and the near plane (0 < w < near), on the view
    # axis.  Blinn's clamp alone keeps the apex's projection (the screen centre); the
    # near-plane clip replaces it by the near-plane cross-section, whose projection is
    # well below the centre, so the box is tighter (Fig. "bbox_clip_alt").
    W, H = 64, 48
    M = S.view_proj((0, 0, 0), (0, 0, -1), (0, 1, 0), W, H, near=0.05)
    pos = np.array([[-0.3, -0.3, -1.0], [0.3, -0.3, -1.0], [0.0, 0.0, -0.01]], np.float32)
    fp = O.parameterize(M, pos, np.array([[0, 1, 2]], np.uint32), W, H, 1.0, np.array([0], np.int32), 1)
    c = np.c_[pos.astype(np.float64), np.ones(3)] @ M.astype(np.float64).T
    assert (c[:, 3] > 0).all() and c[2, 2] < -c[2, 3]  # apex in front of the eye, behind near
    P = frustum_clip_fp64(c)
    box = fp.bbox[0]
    assert box[0] <= P[:, 0].min() + 1e-6 and box[2] >= P[:, 0].max() - 1e-6
    assert box[1] <= P[:, 1].min() + 1e-6 and box[3] >= P[:, 1].max() - 1e-6
    blinn_ymax = (np.clip(c[:, 1], -c[:, 3], c[:, 3]) / c[:, 3]).max()
    assert abs(blinn_ymax) < 1e-6 and box[3] < -0.5
    # the near-plane points: t = 0.95 / 0.99 along each base-to-apex edge
    t = 0.95 / 0.99
    yn = -0.3 * (1 - t) * M[1, 1] / 0.05
    assert abs(box[3] - yn) < 1e-4


def test_footprint_rotation_and_ratio_scaling():
    sc, M, p = S.heightfield_frame(4)
    vt = O.visibility(M, sc.pos, sc.idx, p["width"], p["height"])
    ch = O.chartify(sc.idx, sc.V, vt, 0)
    base = O.parameterize(M, sc.pos, sc.idx, p["width"], p["height"], 1.0, ch.tri_chart, ch.C)
    assert (base.fa <= base.fb).all()
    for r in (0.5, 2.0, 0.25):
        fp = O.parameterize(M, sc.pos, sc.idx, p["width"], p["height"], r, ch.tri_chart, ch.C)
        assert (fp.bbox == base.bbox).all() and (fp.rot == base.rot).all()
        # scaling by a power of two is exact before the ceiling
        wpx = (base.bbox[:, 2].astype(np.float64) - base.bbox[:, 0]) * p["width"] / 2
        hpx = (base.bbox[:, 3].astype(np.float64) - base.bbox[:, 1]) * p["height"] / 2
        side = np.where(base.rot == 1, hpx, wpx)
        assert np.all(fp.fa >= np.floor(256 * r * side * (1 - 1e-6)))
        assert np.all(fp.fa <= np.ceil(256 * r * side * (1 + 1e-6)))
