"""Pins for the oracle's conservative marking coverage (App. A: the marking pass is
rasterized conservatively).  Screen positions are chosen so that the snapped
1/256-pixel coordinates are exact integers (W = H = 16, clip = (x, y, z, 1)):
x = X / 2048 - 1 snaps to X.  The reference is an exact separating-axis test of the
closed triangle against each closed pixel square in integer arithmetic.
"""
import numpy as np
import pytest

import oracle as O

W = H = 16
EYE = np.eye(4, dtype=np.float32)


def world(X, Y, z=0.0):
    return np.array([X / 2048.0 - 1.0, Y / 2048.0 - 1.0, z], np.float32)


def sat_meets(P, px, py):
    """Closed triangle P (3 integer points) meets the closed square of pixel (px, py)."""
    sq = [(256 * px, 256 * py), (256 * (px + 1), 256 * py), (256 * (px + 1), 256 * (py + 1)),
          (256 * px, 256 * (py + 1))]
    axes = [(1, 0), (0, 1)]
    for k in range(3):
        (x0, y0), (x1, y1) = P[k], P[(k + 1) % 3]
        axes.append((-(y1 - y0), x1 - x0))
    for ax, ay in axes:
        a = [ax * x + ay * y for x, y in P]
        b = [ax * x + ay * y for x, y in sq]
        if max(a) < min(b) or max(b) < min(a):
            return False
    return True


def ccw(P):
    (ax, ay), (bx, by), (cx, cy) = P
    return (bx - ax) * (cy - ay) - (cx - ax) * (by - ay) > 0


def test_conservative_coverage_equals_exact_sat():
    rng = np.random.default_rng(7)
    checked = 0
    for trial in range(300):
        if trial % 3 == 0:  # vertices on pixel corners and edges
            P = [(int(rng.integers(0, 17)) * 256, int(rng.integers(0, 17)) * 128) for _ in range(3)]
        elif trial % 3 == 1:  # tiny triangles
            c = rng.integers(256, 15 * 256, size=2)
            P = [(int(c[0] + rng.integers(-90, 90)), int(c[1] + rng.integers(-90, 90))) for _ in range(3)]
        else:
            P = [(int(rng.integers(0, 16 * 256)), int(rng.integers(0, 16 * 256))) for _ in range(3)]
        if not ccw(P):
            P = [P[0], P[2], P[1]]
        if not ccw(P):
            continue
        cov, _ = O.raster_triangle(EYE, *(world(x, y) for x, y in P), W, H, conservative=True)
        want = np.array([[sat_meets(P, px, py) for px in range(W)] for py in range(H)])
        assert (cov == want).all(), f"trial {trial}: {P}"
        checked += 1
    assert checked > 200


def test_conservative_contains_sample_coverage_with_equal_keys():
    rng = np.random.default_rng(8)
    for _ in range(100):
        p = [world(*rng.integers(0, 16 * 256, size=2), z=float(rng.uniform(-0.5, 0.5))) for _ in range(3)]
        cs, ks = O.raster_triangle(EYE, *p, W, H)
        cc, kc = O.raster_triangle(EYE, *p, W, H, conservative=True)
        assert (cc | ~cs).all()  # every sample-covered pixel is conservatively covered
        assert (kc[cs] == ks[cs]).all()  # with the pre-pass depth there


def key_of(d):
    u = int(np.float32(d).view(np.uint32))
    return (~u) & 0xFFFFFFFF if u & 0x80000000 else u | 0x80000000


def test_extrapolated_depth_is_clamped_to_vertex_range():
    # depth rises along x (z = X / 4096 - 0.5 at the vertices); the left edge lies on
    # the pixel boundary x = 1280, so the squares of pixel column 4 touch it
    Q = [(5 * 256, 2 * 256), (12 * 256, 2 * 256), (5 * 256, 12 * 256)]
    zq = [x / 4096.0 - 0.5 for x, _ in Q]
    q = [world(x, y, zz) for (x, y), zz in zip(Q, zq)]
    cs, _ = O.raster_triangle(EYE, *q, W, H)
    cc, kc = O.raster_triangle(EYE, *q, W, H, conservative=True)
    assert cc[5, 4] and not cs[5, 4]
    # plane at the centre x = 1152 gives -0.21875, below the smallest vertex depth
    # -0.1875: clamped to it
    assert int(kc[5, 4]) == key_of(min(zq))
    # pixel (5, 1): the square [512, 768] x [256, 512] touches the bottom edge y = 512;
    # the plane at its centre x = 1408 is -0.15625, inside the range: not clamped
    assert cc[1, 5] and not cs[1, 5]
    assert int(kc[1, 5]) == key_of(1408 / 4096 - 0.5)


def test_marking_pass_conservative_vs_sample():
    # a big background triangle at z = 0.5 and a tiny one in front that covers no
    # pixel centre: visible only with conservative marking; behind the background it
    # stays hidden in both modes
    bg = [(0, 0), (16 * 256 * 2, 0), (0, 16 * 256 * 2)]
    tiny = [(6 * 256 + 20, 6 * 256 + 20), (6 * 256 + 60, 6 * 256 + 20), (6 * 256 + 20, 6 * 256 + 60)]
    for z_tiny, expect_cons in ((0.2, True), (0.8, False)):
        pos = np.array([world(x, y, 0.5) for x, y in bg] + [world(x, y, z_tiny) for x, y in tiny],
                       np.float32)
        idx = np.arange(6, dtype=np.uint32).reshape(2, 3)
        vs = O.vt_to_bool(O.visibility(EYE, pos, idx, W, H), 2)
        vc = O.vt_to_bool(O.visibility(EYE, pos, idx, W, H, conservative=True), 2)
        assert vs[0] and vc[0]
        assert not vs[1]
        assert vc[1] == expect_cons


@pytest.mark.parametrize("seed", [1, 2])
def test_conservative_vt_contains_sample_vt_on_frames(seed):
    from paper_2502_17712_gb300 import scenes as S
    sc, M, p = S.heightfield_frame(seed)
    vs = O.vt_to_bool(O.visibility(M, sc.pos, sc.idx, p["width"], p["height"]), sc.T)
    vc = O.vt_to_bool(O.visibility(M, sc.pos, sc.idx, p["width"], p["height"], conservative=True), sc.T)
    assert (vc | ~vs).all() and vc.sum() > vs.sum()
