"""Batched multi-view atlasing through the C ABI (fa_atlas_batch).

Every view of a batch must equal its solo fa_atlas_frame result bit for bit,
whatever the schedule (lanes, assignment policy), eagerly and from one captured
CUDA graph, and after the schedule autotuner; two views are also checked against
the oracle.  Views: instanced heightfield floors with mixed resolutions
(640x360 .. 2560x1440) and atlas sides (1024 .. 4096).
"""
import numpy as np
import pytest

from paper_2502_17712_gb300 import scenes as S
from test_gpu_parity import F, compare_frame  # noqa: F401  (fixture + checker)

pytestmark = pytest.mark.gpu


def _same_frame(a, b):
    import torch
    C = int(a.count[0])
    assert C == int(b.count[0])
    for name in ("vt", "tri_chart", "result", "count"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    for name in ("place", "fa", "fb", "rot", "order", "root", "bbox", "affine"):
        assert torch.equal(getattr(a, name)[:C], getattr(b, name)[:C]), name
    vis = a.tri_chart >= 0
    ua, ub = a.uv[vis], b.uv[vis]
    assert torch.equal(torch.isnan(ua), torch.isnan(ub))
    assert torch.equal(torch.nan_to_num(ua), torch.nan_to_num(ub))


def _clear(bufs):
    for b in bufs:
        for name in ("vt", "tri_chart", "result", "count", "place", "fa", "fb", "rot", "order", "root",
                     "bbox", "affine"):
            getattr(b, name).zero_()
        b.uv.fill_(float("nan"))


@pytest.fixture(scope="module")
def setup(F):
    views = S.batch_views(3, n_views=10, min_instances=2, max_instances=12)
    maxT = max(sc.T for sc, _, _ in views)
    maxV = max(sc.V for sc, _, _ in views)
    kw = dict(max_tris=maxT, max_verts=maxV, max_charts=1 << 16, max_width=2560, max_height=1440,
              max_atlas_log2=12)
    batch = F.Batch(4, **kw)
    solo = F.Context(**kw)
    mb = [F.BatchMesh(batch, sc.pos, sc.idx) for sc, _, _ in views]
    ms = [F.Mesh(solo, sc.pos, sc.idx) for sc, _, _ in views]
    params = [F.frame_params(M, p["width"], p["height"], p["ratio"], p["atlas_log2"]) for _, M, p in views]
    ref = [F.FrameBuffers.allocate(m.T, m.V, kw["max_charts"]) for m in ms]
    for (sc, M, p), m, b in zip(views, ms, ref):
        F.atlas_frame(solo, m, b, M, p["width"], p["height"], p["ratio"], p["atlas_log2"])
    import torch
    torch.cuda.synchronize()
    assert solo.device_status() == 0
    for b in ref:
        assert int(b.result[3]) == 0
    out = [F.FrameBuffers.allocate(m.T, m.V, kw["max_charts"]) for m in mb]
    yield views, batch, mb, params, ref, out
    for m in mb + ms:
        m.close()
    batch.close()
    solo.close()


@pytest.mark.parametrize("lanes,policy", [(4, 0), (3, 1), (1, 0), (2, 1)])
def test_batch_equals_solo(F, setup, lanes, policy):
    import torch
    views, batch, mb, params, ref, out = setup
    batch.set_schedule(lanes, policy)
    assert batch.schedule() == (lanes, policy)
    _clear(out)
    F.atlas_batch(batch, mb, params, out)
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        _same_frame(a, b)


def test_batch_graph_replay_equals_solo(F, setup):
    import torch
    views, batch, mb, params, ref, out = setup
    batch.set_schedule(4, 1)
    F.atlas_batch(batch, mb, params, out)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.atlas_batch(batch, mb, params, out)
    for _ in range(2):
        _clear(out)
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(out, ref):
            _same_frame(a, b)


def test_batch_tune_then_equal(F, setup):
    import torch
    views, batch, mb, params, ref, out = setup
    lanes, policy, ms = F.batch_tune(batch, mb, params, out, reps=2)
    assert 1 <= lanes <= 4 and policy in (0, 1) and ms > 0
    _clear(out)
    F.atlas_batch(batch, mb, params, out)
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        _same_frame(a, b)


def test_batch_views_against_oracle(F, setup):
    import torch
    views, batch, mb, params, ref, out = setup
    batch.set_schedule(4, 0)
    _clear(out)
    F.atlas_batch(batch, mb, params, out)
    torch.cuda.synchronize()
    for i in (0, 5):
        sc, M, p = views[i]
        compare_frame(sc, M, p["width"], p["height"], p["ratio"], p["atlas_log2"], out[i], 0)


def test_batch_rejects_bad_view_before_enqueue(F, setup):
    views, batch, mb, params, ref, out = setup
    bad = list(params)
    bad[3] = F.frame_params(views[3][1], 4096, 4096, 1.0, 11)  # above the batch's viewport maxima
    with pytest.raises(F.FastAtlasError):
        F.atlas_batch(batch, mb, bad, out)
