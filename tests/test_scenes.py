"""The seeded input generators: sizes, structure and determinism of the synthetic
workloads that stand in for the paper's scene archive (Sec. 6, App. B).

These inputs feed both the CUDA path and the oracle, so they are checked here on
their own: mesh sizes as documented, closed and consistently oriented meshes,
front faces where the cameras look, and the same arrays for the same seed.
"""
import numpy as np
import pytest

from paper_2502_17712_gb300 import scenes as S


def _edges(idx):
    e = np.concatenate([idx[:, [0, 1]], idx[:, [1, 2]], idx[:, [2, 0]]]).astype(np.int64)
    return e


@pytest.mark.parametrize("level", [0, 1, 3])
def test_icosphere_closed_outward_manifold(level):
    v, f = S.icosphere(level)
    assert v.shape == (10 * 4 ** level + 2, 3) and f.shape == (20 * 4 ** level, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    e = _edges(f)
    # every directed edge once and its reverse once: closed, consistently oriented
    d = e[:, 0] * len(v) + e[:, 1]
    r = e[:, 1] * len(v) + e[:, 0]
    assert np.unique(d).size == d.size
    assert np.array_equal(np.sort(d), np.sort(r))
    # Euler characteristic of a sphere
    assert len(v) - d.size // 2 + len(f) == 2
    # counter-clockwise seen from outside: normals point away from the centre
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    assert (np.einsum("ij,ij->i", n, a + b + c) > 0).all()


def test_icosphere_frame_sizes_and_determinism():
    sc, M, p = S.icosphere_frame(1)
    assert (sc.T, sc.V) == (4_096_000, 2_048_400)
    assert sc.pos.dtype == np.float32 and sc.idx.dtype == np.uint32
    assert sc.idx.max() < sc.V and np.isfinite(sc.pos).all()
    # radii 0.5-2 times a displaced unit sphere, centres inside the 48^3 box
    assert np.abs(sc.pos).max() < 24.0 + 2.0 * 1.2
    assert (p["width"], p["height"], p["atlas_log2"], p["ratio"]) == (1920, 1080, 11, 1.0)
    assert M.shape == (4, 4) and np.isfinite(M).all()
    sc2, M2, _ = S.icosphere_frame(1, n_spheres=3)
    assert np.array_equal(sc2.pos, sc.pos[:3 * 10242]) and np.array_equal(sc2.idx, sc.idx[:3 * 20480])
    assert np.array_equal(M2, M)
    sc3, _, _ = S.icosphere_frame(2, n_spheres=3)
    assert not np.array_equal(sc3.pos, sc2.pos)


def test_heightfield_faces_up_and_camera_sees_it():
    sc, M, p = S.heightfield_frame(1)
    assert (sc.T, sc.V) == (2 * 63 * 63, 64 * 64)
    a, b, c = (sc.pos[sc.idx[:, k]].astype(np.float64) for k in range(3))
    assert (np.cross(b - a, c - a)[:, 2] > 0).all()
    clip = np.c_[sc.pos.astype(np.float64), np.ones(sc.V)] @ M.astype(np.float64).T
    assert (clip[:, 3] > 0).all()
    ndc = clip[:, :2] / clip[:, 3:]
    assert (np.abs(ndc) <= 1).all(1).mean() > 0.5
    assert (p["width"], p["height"], p["atlas_log2"]) == (480, 270, 10)


def test_camera_path_is_closed_and_distinct():
    sc, cams, p = S.camera_path_frames(1, 300)
    assert len(cams) == 300 and (p["width"], p["height"]) == (1920, 1080)
    cams = np.asarray(cams, np.float64)
    assert np.isfinite(cams).all()
    assert len({c.tobytes() for c in cams}) == 300


def test_batch_views_workload():
    views = S.batch_views(7)
    assert len(views) == 64
    assert sum(sc.T for sc, _, _ in views) == 108_314_010
    for sc, M, p in views:
        assert (p["width"], p["height"]) in S.BATCH_RESOLUTIONS and p["atlas_log2"] in S.BATCH_ATLAS_LOG2
        n = sc.T // (2 * 63 * 63)
        assert sc.T == n * 2 * 63 * 63 and 50 <= n <= 400 and sc.idx.max() < sc.V


def test_lognormal_boxes():
    fa, fb = S.lognormal_boxes(1, 10000)
    assert fa.dtype == np.uint32 and (fb >= fa).all()
    assert fa.min() >= 64 and fb.max() <= 1024 * 256
    fa2, fb2 = S.lognormal_boxes(1, 10000)
    assert np.array_equal(fa, fa2) and np.array_equal(fb, fb2)
    # median side near the requested mean of the log-normal (12 texels)
    assert 9 * 256 < np.median(np.r_[fa, fb]) < 16 * 256


def test_value_noise_range_and_lattice():
    rng = np.random.default_rng(0)
    p = rng.uniform(-50, 50, size=(20000, 3))
    n = S.value_noise(p, 5)
    assert (np.abs(n) <= 1).all() and n.std() > 0.1
    # at lattice points the noise is the lattice hash itself
    q = np.floor(p[:100])
    h = S._hash3(q[:, 0].astype(np.int64), q[:, 1].astype(np.int64), q[:, 2].astype(np.int64), 5)
    assert np.allclose(S.value_noise(q, 5), h)
