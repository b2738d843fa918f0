"""Served atlasing with continuous batching (fa_server_*): requests of several
sessions submitted together run overlapped on several slots, and every request's
results equal the same request run alone (fa_atlas_frame on its own context), bit
for bit; one request is also checked against the oracle.  Admission by the
device-memory budget: slots and sessions beyond the budget are refused.
"""
import numpy as np
import pytest

from paper_2502_17712_gb300 import scenes as S
from test_gpu_parity import F, compare_frame  # noqa: F401  (fixture + checker)

pytestmark = pytest.mark.gpu

RES = ((1280, 720), (1920, 1080), (2560, 1440))


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


def _sessions(n=6):
    out = []
    for i in range(n):
        sc = S.instanced_grid_scene(40 + i, 2 + i)
        reqs = []
        for j in range(2):
            W, H = RES[(i + j) % len(RES)]
            M = S.hemisphere_camera(400 + 10 * i + j, W, H, radius=10.0)
            reqs.append((M, dict(width=W, height=H, ratio=1.0, atlas_log2=11 + (i + j) % 2)))
        out.append((sc, reqs))
    return out


def test_served_mix_equals_alone(F):
    import torch
    sess = _sessions()
    maxT = max(sc.T for sc, _ in sess)
    maxV = max(sc.V for sc, _ in sess)
    kw = dict(max_tris=maxT, max_verts=maxV, max_charts=1 << 15, max_width=2560, max_height=1440,
              max_atlas_log2=12)
    server = F.Server(3, 1 << 40, **kw)
    assert server.n_slots == 3
    sids = [server.open_session(sc.pos, sc.idx) for sc, _ in sess]
    jobs = []
    for sid, (sc, reqs) in zip(sids, sess):
        for M, p in reqs:
            bufs = F.FrameBuffers.allocate(sc.T, sc.V, kw["max_charts"])
            jobs.append((sid, sc, M, p, bufs))
    # the mix: everything submitted at once, then polled to completion
    tickets = [server.submit(sid, F.frame_params(M, p["width"], p["height"], p["ratio"], p["atlas_log2"]), bufs)
               for sid, sc, M, p, bufs in jobs]
    done = []
    for _ in range(200000):
        done += server.poll()
        if len(done) == len(jobs):
            break
    assert sorted(d["ticket"] for d in done) == sorted(tickets)
    st = server.stats()
    assert st["queued"] == 0 and st["running"] == 0
    assert st["max_running"] >= 2  # requests did run side by side
    # a session never has two requests on the GPU at once
    by_sid = {}
    for d in sorted(done, key=lambda d: d["dispatch_ms"]):
        prev = by_sid.get(d["session"])
        if prev is not None:
            assert d["dispatch_ms"] >= prev["done_ms"]
        by_sid[d["session"]] = d
    torch.cuda.synchronize()
    # alone: each request on its own context, nothing else running
    alone = F.Context(**kw)
    for sid, sc, M, p, bufs in jobs:
        mesh = F.Mesh(alone, sc.pos, sc.idx)
        ref = F.FrameBuffers.allocate(sc.T, sc.V, kw["max_charts"])
        F.atlas_frame(alone, mesh, ref, M, p["width"], p["height"], p["ratio"], p["atlas_log2"])
        torch.cuda.synchronize()
        assert alone.device_status() == 0
        assert int(ref.result[3]) == 0
        _same_frame(bufs, ref)
        mesh.close()
    sid, sc, M, p, bufs = jobs[3]
    compare_frame(sc, M, p["width"], p["height"], p["ratio"], p["atlas_log2"], bufs, 0)
    alone.close()
    server.close()


def test_server_budget_admission(F):
    small = S.instanced_grid_scene(7, 2)
    big = S.instanced_grid_scene(8, 200)  # 1,587,600 triangles: adjacency about 19 MB
    kw = dict(max_tris=big.T, max_verts=big.V, max_charts=1 << 14, max_width=1280, max_height=720,
              max_atlas_log2=11)
    probe = F.Server(1, 1 << 40, **kw)
    slot_bytes = probe.stats()["used_bytes"]
    probe.close()
    assert slot_bytes > 0
    two = F.Server(4, int(2.5 * slot_bytes), **kw)
    assert two.n_slots == 2
    two.close()
    with pytest.raises(F.FastAtlasError):
        F.Server(4, slot_bytes // 2, **kw)  # not even one slot
    tight = F.Server(1, slot_bytes + (8 << 20), **kw)
    assert tight.n_slots == 1
    with pytest.raises(F.FastAtlasError):
        tight.open_session(big.pos, big.idx)  # the session does not fit the rest of the budget
    tight.close()
    roomy = F.Server(1, slot_bytes + (256 << 20), **kw)
    sid = roomy.open_session(small.pos, small.idx)
    roomy.close_session(sid)
    roomy.close()
