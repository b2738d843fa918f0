"""Pins for the oracle's box variant and partial-visibility bits.

- Frustum-plane box (Sec. 5.2: a triangle that does not cross the near plane is
  clipped against the frustum plane that reduces its box the most, before Blinn's
  clamp): closed forms for a right-plane and a far-plane clip, the chosen box is
  inside the near-only Blinn box and still contains the exact 6-plane fp64 clip.
- Partial visibility (Sec. 6 temporal re-use: a vertex with max(|x|,|y|) >= w):
  hand cases, boundary, invisible triangles untouched.
"""
import numpy as np
import pytest

import oracle as O
from paper_2502_17712_gb300 import scenes as S
from test_oracle_charts import frustum_clip_fp64

EYE = np.eye(4, dtype=np.float32)  # clip = (x, y, z, 1)


def box_of(pos, flags, M=EYE, W=64, H=64):
    pos = np.asarray(pos, np.float32)
    idx = np.arange(3, dtype=np.uint32).reshape(1, 3)
    return O.parameterize(M, pos, idx, W, H, 1.0, np.array([0], np.int32), 1, flags).bbox[0]


def test_right_plane_clip_closed_form():
    # C lies far right of x = w; Blinn clamps it to (1, 0.5) and keeps y up to 0.5,
    # but the triangle meets x = 1 only at y in [1/12, 1/10]
    tri = [[0, 0, 0], [0.2, 0, 0], [5, 0.5, 0]]
    assert np.allclose(box_of(tri, 0), [0, 0, 1, 0.5], atol=1e-7)
    assert np.allclose(box_of(tri, O.BOX_FRUSTUM_CLIP), [0, 0, 1, 0.1], atol=1e-6)


def test_far_plane_clip_closed_form():
    # C is beyond the far plane z = w: the visible part ends at t = 0.2 along AC, BC
    tri = [[0, 0, 0.5], [0.5, 0, 0.5], [0, 0.8, 3]]
    assert np.allclose(box_of(tri, 0), [0, 0, 0.5, 0.8], atol=1e-7)
    assert np.allclose(box_of(tri, O.BOX_FRUSTUM_CLIP), [0, 0, 0.5, 0.16], atol=1e-6)


def test_inside_triangle_unchanged_and_near_crossing_uses_near_clip():
    inside = [[-0.3, -0.2, 0.1], [0.4, -0.1, 0.2], [0.0, 0.5, -0.3]]
    assert (box_of(inside, 0) == box_of(inside, O.BOX_FRUSTUM_CLIP)).all()
    # crosses the near plane z = -w: both modes take the near clip only
    near = [[0.2, 0.1, -3.0], [0.5, 0.2, 0.5], [0.1, 0.6, 0.2]]
    assert (box_of(near, 0) == box_of(near, O.BOX_FRUSTUM_CLIP)).all()


@pytest.mark.parametrize("seed", range(6))
def test_frustum_box_inside_blinn_box_and_conservative(seed):
    rng = np.random.default_rng(100 + seed)
    W, H = 64, 48
    M = S.view_proj((0, 0, 0), (0, 0, -1), (0, 1, 0), W, H, near=0.5, far=6.0)
    n = 40
    pos = (rng.normal(scale=2.5, size=(3 * n, 3)) + np.array([0, 0, -4.0])).astype(np.float32)
    idx = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    tc = np.arange(n, dtype=np.int32)  # one chart per triangle
    b0 = O.parameterize(M, pos, idx, W, H, 1.0, tc, n, 0).bbox.astype(np.float64)
    b1 = O.parameterize(M, pos, idx, W, H, 1.0, tc, n, O.BOX_FRUSTUM_CLIP).bbox.astype(np.float64)
    c = np.c_[pos.astype(np.float64), np.ones(3 * n)] @ M.astype(np.float64).T
    tighter = 0
    for t in range(n):
        if not np.isfinite(b1[t]).all():
            continue
        # never larger than the near-only Blinn box
        assert b1[t, 0] >= b0[t, 0] - 1e-7 and b1[t, 1] >= b0[t, 1] - 1e-7
        assert b1[t, 2] <= b0[t, 2] + 1e-7 and b1[t, 3] <= b0[t, 3] + 1e-7
        tighter += bool((np.abs(b1[t] - b0[t]) > 1e-6).any())
        # still contains the exact visible part
        P = frustum_clip_fp64(c[3 * t:3 * t + 3])
        if len(P):
            tol = 1e-5
            assert (P[:, 0] >= b1[t, 0] - tol).all() and (P[:, 0] <= b1[t, 2] + tol).all()
            assert (P[:, 1] >= b1[t, 1] - tol).all() and (P[:, 1] <= b1[t, 3] + tol).all()
    assert tighter > 0


def test_partial_visibility_hand_cases():
    pos = np.array([[-0.5, -0.5, 0], [0.5, -0.5, 0], [0, 0.5, 0],     # inside: 0
                    [-0.5, -0.5, 0], [1.0, -0.5, 0], [0, 0.5, 0],     # x == w: 1
                    [-0.5, -1.5, 0], [0.5, -0.5, 0], [0, 0.5, 0],     # y < -w: 1
                    [-3.0, 0.0, 0], [0.5, -0.5, 0], [0, 0.5, 0]],     # x < -w but invisible: 0
                   np.float32)
    idx = np.arange(12, dtype=np.uint32).reshape(4, 3)
    tc = np.array([0, 0, 1, -1], np.int32)
    fp = O.parameterize(EYE, pos, idx, 64, 64, 1.0, tc, 2)
    assert fp.partial.shape == (1,)
    assert int(fp.partial[0]) == 0b0110
