"""Pins for the oracle's parameterization (Sec. 3: charts are parameterized by
their view projection, so a constant number of texels maps to each pixel; App. A
"Shading and Rasterization": uniform scale S then a per-chart rigid placement)."""
import numpy as np
import pytest

import oracle as O
from paper_2502_17712_gb300 import scenes as S


def frame(seed, ratio=1.0, atlas_log2=10, mode=0, width=480, height=270):
    sc = S.grid_scene(seed)
    M = S.hemisphere_camera(seed, width, height)
    fr = O.atlas_frame(M, sc.pos, sc.idx, width, height, ratio, atlas_log2, mode=mode)
    return sc, M, fr


def screen_xy(M, pos, idx, W, H):
    # from the fp32 clip coordinates the path works with (transform is pinned separately)
    c = O.transform(M, pos).astype(np.float64)
    ndc = c[:, :2] / c[:, 3:]
    xy = (ndc + 1.0) * np.array([W / 2.0, H / 2.0])
    return xy[idx.astype(np.int64)], c[:, 3][idx.astype(np.int64)]


def signed_area(p):
    a, b, c = p[:, 0], p[:, 1], p[:, 2]
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))


@pytest.mark.parametrize("seed,ratio,log2", [(1, 1.0, 10), (2, 0.5, 9), (3, 2.0, 10), (4, 1.0, 8)])
def test_constant_texel_to_pixel_ratio(seed, ratio, log2):
    """Atlas area / screen area equals (alpha * r * k / n)^2 for every visible triangle
    (uniform stretch, L2 = Linf, Tab. 'stretch_fixed_sr'), orientation preserved."""
    W, H = 480, 270
    sc, M, fr = frame(seed, ratio, log2)
    vis = fr.charts.tri_chart >= 0
    xy, w = screen_xy(M, sc.pos, sc.idx, W, H)
    ok = vis & (w > 0).all(1)
    sa = signed_area(xy[ok])
    ua = signed_area(fr.uv[ok])
    big = np.abs(sa) > 1e-3
    s = (1 << log2) / fr.pk.omega * ratio * fr.pk.k / 64
    assert np.allclose(ua[big] / sa[big], s * s, rtol=1e-9, atol=0)
    # when everything fits at scale 1 with no overflow the ratio is exactly r^2
    if fr.pk.k == 64 and fr.pk.omega == (1 << log2):
        assert np.isclose(s, ratio)


def test_covered_pixel_centres_map_into_the_chart_rectangle():
    W, H = 480, 270
    sc, M, fr = frame(5, 1.0, 9)
    om = 1 << 9
    alpha = om / fr.pk.omega
    checked = 0
    for t in np.nonzero(fr.charts.tri_chart >= 0)[0][::7]:
        c = fr.charts.tri_chart[t]
        cover, _ = O.raster_triangle(M, *sc.pos[sc.idx[t]], W, H)
        ys, xs = np.nonzero(cover)
        if len(xs) == 0:
            continue
        # map the pixel centres with the chart's affine (fp64)
        ndc = np.stack([(xs + 0.5) / (W / 2) - 1, (ys + 0.5) / (H / 2) - 1], 1)
        a = fr.affine[c]
        u = a[0] * ndc[:, 0] + a[1] * ndc[:, 1] + a[2]
        v = a[3] * ndc[:, 0] + a[4] * ndc[:, 1] + a[5]
        x, y, w, h = fr.pk.place[c]
        tol = 1e-9
        assert (u >= alpha * x - tol).all() and (u <= alpha * (x + w) + tol).all()
        assert (v >= alpha * y - tol).all() and (v <= alpha * (y + h) + tol).all()
        checked += len(xs)
    assert checked > 100


def test_affine_reproduces_corner_uvs_and_rotation_is_proper():
    W, H = 480, 270
    for seed in (6, 7, 8):
        sc, M, fr = frame(seed, 1.0, 9, mode=0)
        c = O.transform(M, sc.pos).astype(np.float64)
        vis = np.nonzero(fr.charts.tri_chart >= 0)[0]
        for t in vis[::11]:
            ch = fr.charts.tri_chart[t]
            a = fr.affine[ch]
            for j in range(3):
                cc = c[sc.idx[t, j]]
                if cc[3] <= 0:
                    continue
                nx, ny = cc[0] / cc[3], cc[1] / cc[3]
                assert abs(a[0] * nx + a[1] * ny + a[2] - fr.uv[t, j, 0]) < 1e-9
                assert abs(a[3] * nx + a[4] * ny + a[5] - fr.uv[t, j, 1]) < 1e-9
        det = fr.affine[:, 0] * fr.affine[:, 4] - fr.affine[:, 1] * fr.affine[:, 3]
        assert (det > 0).all()
        rot = fr.fp.rot.astype(bool)
        assert (fr.affine[rot][:, [0, 4]] == 0).all() and (fr.affine[~rot][:, [1, 3]] == 0).all()


def test_rotated_chart_fits_its_box():
    # a wide strip: its box is rotated, and the chart still lies inside the placement
    W, H = 256, 64
    pos = np.array([[-0.9, -0.2, 0], [0.9, -0.2, 0], [0.9, 0.2, 0], [-0.9, 0.2, 0]], np.float32)
    idx = np.array([[0, 1, 2], [0, 2, 3]], np.uint32)
    I4 = np.eye(4, dtype=np.float32)
    fr = O.atlas_frame(I4, pos, idx, W, H, 1.0, 8)
    assert fr.charts.C == 1 and fr.fp.rot[0] == 1
    x, y, w, h = fr.pk.place[0]
    alpha = 256 / fr.pk.omega
    u, v = fr.uv[..., 0], fr.uv[..., 1]
    assert (u >= alpha * x - 1e-9).all() and (u <= alpha * (x + w) + 1e-9).all()
    assert (v >= alpha * y - 1e-9).all() and (v <= alpha * (y + h) + 1e-9).all()
    assert h > w
