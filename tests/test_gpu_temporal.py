"""Re-atlasing along a camera path: the 64x64 heightfield over a 300-frame
Catmull-Rom camera spline at 1920x1080 into a 2048^2 atlas, every frame atlased by
replaying ONE captured CUDA graph whose view-projection matrix is read on the
device (fa_atlas_frame_dev_matrix).  Every frame must equal the eager
fa_atlas_frame result bit for bit; sampled frames are checked against the oracle.
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
    assert torch.equal(a.vt, b.vt)
    assert torch.equal(a.tri_chart, b.tri_chart)
    assert torch.equal(a.result, b.result)
    assert torch.equal(a.place[:C], b.place[:C])
    assert torch.equal(a.fa[:C], b.fa[:C]) and torch.equal(a.fb[:C], b.fb[:C])
    vis = a.tri_chart >= 0
    ua, ub = a.uv[vis], b.uv[vis]
    assert torch.equal(torch.isnan(ua), torch.isnan(ub))
    assert torch.equal(torch.nan_to_num(ua), torch.nan_to_num(ub))


def test_camera_path_graph_replay(F):
    import torch
    n_frames = 300
    sc, cams, p = S.camera_path_frames(1, n_frames)
    W, H, r, L = p["width"], p["height"], p["ratio"], p["atlas_log2"]
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 15, max_width=W, max_height=H,
                    max_atlas_log2=L)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    g_bufs = F.FrameBuffers.allocate(mesh.T, mesh.V, ctx.cfg.max_charts)
    e_bufs = F.FrameBuffers.allocate(mesh.T, mesh.V, ctx.cfg.max_charts)
    d_M = torch.empty(16, dtype=torch.float32, device="cuda")
    host = torch.from_numpy(np.stack([np.asarray(c, np.float32).reshape(16) for c in cams])).pin_memory()
    d_M.copy_(host[0])
    F.atlas_frame_dev_matrix(ctx, mesh, g_bufs, d_M, W, H, r, L)  # warm-up outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        F.atlas_frame_dev_matrix(ctx, mesh, g_bufs, d_M, W, H, r, L)
    oracle_frames = {0, 77, 150, 299}
    for f in range(n_frames):
        d_M.copy_(host[f], non_blocking=True)
        graph.replay()
        F.atlas_frame(ctx, mesh, e_bufs, cams[f], W, H, r, L)
        torch.cuda.synchronize()
        assert ctx.device_status() == 0, f"frame {f}"
        _same_frame(g_bufs, e_bufs)
        if f in oracle_frames:
            compare_frame(sc, cams[f], W, H, r, L, g_bufs, 0)
    mesh.close()
    ctx.close()


def test_dev_matrix_frame_equals_frame_on_icospheres(F):
    import torch
    sc, M, p = S.icosphere_frame(2, 40)
    W, H, r, L = p["width"], p["height"], p["ratio"], p["atlas_log2"]
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 17, max_width=W, max_height=H,
                    max_atlas_log2=L)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    a = F.FrameBuffers.allocate(mesh.T, mesh.V, ctx.cfg.max_charts)
    b = F.FrameBuffers.allocate(mesh.T, mesh.V, ctx.cfg.max_charts)
    d_M = torch.from_numpy(np.asarray(M, np.float32).reshape(16).copy()).cuda()
    F.atlas_frame(ctx, mesh, a, M, W, H, r, L)
    F.atlas_frame_dev_matrix(ctx, mesh, b, d_M, W, H, r, L)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    _same_frame(a, b)
    mesh.close()
    ctx.close()
