"""Per-kernel tracing and the work counts of a frame, through the C ABI.

The traced frame is the documented launch sequence; every kernel in it has a
compulsory-bytes entry in the benchmark's roofline table; the work counts agree
with the outputs (visible triangles, charts) and with the oracle's visibility.
"""
import numpy as np
import pytest

import oracle as O
from paper_2502_17712_gb300 import scenes as S

pytestmark = pytest.mark.gpu

FRAME_KERNELS = ["k_raster_front", "k_raster_exact", "k_raster_depth_big", "k_raster_mark",
                 "k_uf_local", "k_uf_hook", "k_uf_flatten", "k_scan_blocks", "k_tri_chart", "k_bbox",
                 "k_order_tile", "k_order_scatter", "k_pack_scan", "k_pack_push", "k_uv"]


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2502_17712_gb300 import build, fastatlas
    build.build()
    fastatlas.load()
    return fastatlas


def test_trace_and_work_counts(F):
    import torch
    import bench
    # ~500-pixel triangles: the queued tile rasterizer has work too
    sc = S.grid_scene(7)
    W, H = 1920, 1080
    M = S.spline_cameras(7, 5, W, H)[2]
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 15, max_width=W, max_height=H,
                    max_atlas_log2=11)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    bufs = F.FrameBuffers.allocate(mesh.T, mesh.V, ctx.cfg.max_charts)
    F.fa_profile_enable(ctx.handle, True)
    n0 = ctx.launches
    F.atlas_frame(ctx, mesh, bufs, M, W, H, 1.0, 11, 0)
    trace = F.fa_profile_read(ctx.handle)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    names = [n for n, _ in trace]
    assert names == FRAME_KERNELS
    # the benchmark's stage table (which also lists the optional tile-depth pass)
    assert names == [k for ks in bench.STAGES.values() for k in ks if k != "k_raster_zmax"]
    assert ctx.launches - n0 == len(FRAME_KERNELS)
    assert all(ms >= 0.0 for _, ms in trace)
    # with the tile-depth marking on, that pass runs right before the marking pass
    ctx.set_raster_schedule(16, F.FA_RASTER_HIZ)
    ref_vt = bufs.vt.clone()
    F.atlas_frame(ctx, mesh, bufs, M, W, H, 1.0, 11, 0)
    hiz_names = [n for n, _ in F.fa_profile_read(ctx.handle)]
    ctx.set_raster_schedule()
    assert hiz_names == [k for ks in bench.STAGES.values() for k in ks]
    assert torch.equal(bufs.vt, ref_vt) and ctx.device_status() == 0
    F.atlas_frame(ctx, mesh, bufs, M, W, H, 1.0, 11, 0)

    work = ctx.frame_stats()
    vt = bufs.vt.cpu().numpy().view(np.uint32)
    assert (vt == O.visibility(M, sc.pos, sc.idx, W, H)).all()
    T_vis = int(np.unpackbits(vt.view(np.uint8)).sum())
    C = int(bufs.count[0])
    assert work["visible"] == T_vis
    assert work["charts"] == C
    # a visible triangle passed the front end, directly or through the clipping path
    assert 0 < T_vis <= work["survivors"] + work["clipped"] <= sc.T
    assert work["big_entries"] > 0 and work["big_tiles"] >= work["big_entries"]
    # the tiles of 1024 triangles that hold a visible one, as the marking pass listed them
    tiles = np.zeros(((sc.T + 1023) // 1024) * 1024, bool)
    tiles[:sc.T] = np.unpackbits(vt.view(np.uint8), bitorder="little")[:sc.T].astype(bool)
    assert work["visible_tiles"] == int(tiles.reshape(-1, 1024).any(1).sum())
    for n in names:
        assert bench.algorithmic_bytes(n, sc.T, sc.V, W, H, T_vis, C, work) is not None, n
    F.fa_profile_enable(ctx.handle, False)
    mesh.close()
    ctx.close()


def test_unaligned_tri_chart_output(F):
    """A tri_chart buffer that is not 16-byte aligned takes the path that writes every
    triangle's chart id in the chart pass: same outputs as an aligned buffer."""
    import torch
    sc, M, p = S.heightfield_frame(2)
    W, H = p["width"], p["height"]
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 15, max_width=W, max_height=H,
                    max_atlas_log2=12)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    outs = []
    for offset in (0, 1):
        bufs = F.FrameBuffers.allocate(mesh.T, mesh.V, ctx.cfg.max_charts)
        big = torch.full((sc.T + 4,), 7, dtype=torch.int32, device="cuda")
        bufs.tri_chart = big[offset:offset + sc.T]
        assert (bufs.tri_chart.data_ptr() % 16 == 0) == (offset == 0)
        F.atlas_frame(ctx, mesh, bufs, M, W, H, p["ratio"], p["atlas_log2"], 0)
        torch.cuda.synchronize()
        assert ctx.device_status() == 0
        outs.append({k: getattr(bufs, k).cpu().numpy().view(np.uint8).copy()
                     for k in ("vt", "tri_chart", "root", "order", "place", "result", "uv")})
        if offset:  # nothing written outside the view
            assert int(big[0]) == 7 and (big[offset + sc.T:].cpu().numpy() == 7).all()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    fr = O.atlas_frame(M, sc.pos, sc.idx, W, H, p["ratio"], p["atlas_log2"])
    assert (outs[1]["tri_chart"].view(np.int32) == fr.charts.tri_chart).all()
    mesh.close()
    ctx.close()
