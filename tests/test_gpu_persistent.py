"""The persistent frame kernel: one cooperative launch per frame
(FA_FRAME_PERSISTENT) and one per batch (batch plans) give the launch sequence's
results bit for bit, and equal the oracle; a dependency wait that runs out aborts
the launch with FA_E_TIMEOUT and the next launch is clean."""
import numpy as np
import pytest

from paper_2502_17712_gb300 import scenes as S
from test_gpu_parity import F, compare_frame, run_gpu  # noqa: F401  (fixture + checker)

pytestmark = pytest.mark.gpu

FIELDS = ("vt", "tri_chart", "root", "bbox", "fa", "fb", "rot", "count", "order", "place", "result", "affine")


def assert_same(a, b, C=None, visible_uv_only=False):
    """Every output of a equals b's (UVs of invisible triangles are left untouched by
    a frame, so with reused buffers only the visible ones are compared)."""
    import torch
    for name in FIELDS:
        x, y = getattr(a, name), getattr(b, name)
        if name in ("root", "bbox", "fa", "fb", "rot", "order", "place", "affine") and C is not None:
            x, y = x[:C], y[:C]
        assert torch.equal(x, y), name
    for name in ("vert_chart", "partial"):
        x, y = getattr(a, name), getattr(b, name)
        if x is not None and y is not None:
            assert torch.equal(x, y), name
    if a.uv is not None:
        ua, ub = torch.nan_to_num(a.uv, 7.0), torch.nan_to_num(b.uv, 7.0)
        if visible_uv_only:
            vis = a.tri_chart >= 0
            ua, ub = ua[vis], ub[vis]
        assert torch.equal(ua, ub)


@pytest.fixture(scope="module")
def pctx(F):
    ctx = F.Context(max_tris=1 << 16, max_verts=1 << 16, max_charts=1 << 15, max_width=1920, max_height=1080,
                    max_atlas_log2=12)
    yield ctx
    ctx.close()


def both(F, ctx, mesh, M, W, H, r, L, mode=0, n_scales=64, sel=0, flags=0):
    a, sa = run_gpu(F, ctx, mesh, M, W, H, r, L, mode, n_scales, sel, flags=flags)
    b, sb = run_gpu(F, ctx, mesh, M, W, H, r, L, mode, n_scales, sel, flags=flags | F.FA_FRAME_PERSISTENT)
    assert sa == sb
    assert_same(a, b, int(a.count[0]))
    return b, sb


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("mode", [0, 1])
def test_persistent_frame_equals_launch_sequence_and_oracle(F, pctx, seed, mode):
    sc, M, p = S.heightfield_frame(seed)
    mesh = F.Mesh(pctx, sc.pos, sc.idx)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    b, st = both(F, pctx, mesh, M, *args, mode)
    compare_frame(sc, M, *args, b, st, mode)
    mesh.close()


@pytest.mark.parametrize("flags_name", ["FA_BOX_FRUSTUM_CLIP", "FA_VIS_CONSERVATIVE"])
def test_persistent_flags(F, pctx, flags_name):
    sc, M, p = S.heightfield_frame(2)
    mesh = F.Mesh(pctx, sc.pos, sc.idx)
    flags = getattr(F, flags_name)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    b, st = both(F, pctx, mesh, M, *args, flags=flags)
    compare_frame(sc, M, *args, b, st, flags=flags)
    mesh.close()


def test_persistent_variants_big_triangles_near_plane_scales(F, pctx):
    sc = S.grid_scene(7)
    M = S.spline_cameras(7, 5, 1920, 1080)[2]  # large triangles: the tile rasterizer
    mesh = F.Mesh(pctx, sc.pos, sc.idx)
    b, st = both(F, pctx, mesh, M, 1920, 1080, 1.0, 11)
    compare_frame(sc, M, 1920, 1080, 1.0, 11, b, st)
    b, st = both(F, pctx, mesh, M, 1920, 1080, 2.0, 10, 0, 16, 1)  # 16 scales, largest k
    compare_frame(sc, M, 1920, 1080, 2.0, 10, b, st, 0, 16, 1)
    mesh.close()
    sc = S.instanced_grid_scene(3, 6, n=24)  # near plane and guard band crossings
    W, H = 640, 360
    mesh = F.Mesh(pctx, sc.pos, sc.idx)
    for eye in [(0.1, 0.2, 0.12), (-0.5, 0.3, 0.06)]:
        M = S.view_proj(eye, (eye[0] + 1.0, eye[1] + 0.4, -0.2), (0, 0, 1), W, H, near=0.05)
        b, st = both(F, pctx, mesh, M, W, H, 1.0, 10)
        compare_frame(sc, M, W, H, 1.0, 10, b, st)
    mesh.close()


def test_persistent_non_manifold_and_lowres(F):
    pos = np.array([[-0.5, -0.5, 0.0], [0.5, -0.5, 0.0], [0.0, 0.5, 0.0], [0.0, -0.9, 0.1],
                    [0.3, 0.6, -0.1], [-0.6, 0.2, 0.05], [0.6, 0.1, 0.2], [-0.8, -0.8, 0.0],
                    [-0.7, -0.8, 0.0], [-0.75, -0.7, 0.0]], np.float32)
    idx = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4], [0, 1, 6], [0, 0, 5], [2, 2, 2], [7, 8, 9],
                    [1, 2, 6]], np.uint32)
    ctx = F.Context(max_tris=64, max_verts=64, max_charts=64, max_width=64, max_height=64, max_atlas_log2=8,
                    gutter=4)
    mesh = F.Mesh(ctx, pos, idx)
    M = np.eye(4, dtype=np.float32)
    for mode in (0, 1):
        b, st = both(F, ctx, mesh, M, 64, 64, 1.0, 8, mode)
        compare_frame(S.Scene(pos, idx), M, 64, 64, 1.0, 8, b, st, mode, gutter=4)
    mesh.close()
    ctx.close()
    sc, M, p = S.heightfield_frame(2)
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 14, max_width=p["width"],
                    max_height=p["height"], max_atlas_log2=p["atlas_log2"], gutter=4)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    b, st = both(F, ctx, mesh, M, *args, flags=F.FA_LOWRES(3))
    compare_frame(sc, M, *args, b, st, flags=F.FA_LOWRES(3), gutter=4)
    mesh.close()
    ctx.close()


def test_persistent_full_size_icospheres(F):
    """The 4,096,000-triangle frame (1920x1080, 2048^2 atlas) as one launch."""
    sc, M, p = S.icosphere_frame(1)
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 17, max_width=1920, max_height=1080,
                    max_atlas_log2=11)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    b, st = both(F, ctx, mesh, M, *args)
    fr = compare_frame(sc, M, *args, b, st)
    assert fr.pk.status == 0 and fr.uv_err_inside <= 1e-4
    mesh.close()
    ctx.close()


def test_persistent_camera_path_graph(F, pctx):
    """One graph captured from a persistent fa_atlas_frame_dev_matrix call serves a
    camera path; every frame equals the launch sequence's."""
    import torch
    sc, cams, p = S.camera_path_frames(1, 300)
    W, H, r, L = p["width"], p["height"], p["ratio"], p["atlas_log2"]
    mesh = F.Mesh(pctx, sc.pos, sc.idx)
    dm = torch.zeros(16, dtype=torch.float32, device="cuda")
    g_bufs = F.FrameBuffers.allocate(mesh.T, mesh.V, pctx.cfg.max_charts)
    dm.copy_(torch.as_tensor(np.asarray(cams[0], np.float32).reshape(16)))
    F.atlas_frame_dev_matrix(pctx, mesh, g_bufs, dm, W, H, r, L, flags=F.FA_FRAME_PERSISTENT)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.atlas_frame_dev_matrix(pctx, mesh, g_bufs, dm, W, H, r, L, flags=F.FA_FRAME_PERSISTENT)
    for f in range(0, 300, 37):
        dm.copy_(torch.as_tensor(np.asarray(cams[f], np.float32).reshape(16)))
        g.replay()
        ref, st = run_gpu(F, pctx, mesh, cams[f], W, H, r, L)
        assert st == 0
        assert_same(ref, g_bufs, int(ref.count[0]), visible_uv_only=True)
    del g
    mesh.close()


def test_batch_plan_equals_solo(F):
    """Twelve views of mixed scenes, resolutions and atlas sides in one launch: every
    view equals its own fa_atlas_frame, under several schedules and in a graph."""
    import torch
    views = []
    for i in range(12):
        if i % 3 == 0:
            sc, M, p = S.heightfield_frame(10 + i)
        elif i % 3 == 1:
            sc = S.instanced_grid_scene(20 + i, 6, n=6 + i)
            W, H = (640, 360) if i % 2 else (1280, 720)
            M = S.hemisphere_camera(i, W, H, radius=4.0)
            p = {"width": W, "height": H, "ratio": 1.0, "atlas_log2": 10 + i % 3}
        else:
            sc, M, p = S.icosphere_frame(30 + i, 3)
        views.append((sc, M, p))
    maxT = max(sc.T for sc, _, _ in views)
    maxV = max(sc.V for sc, _, _ in views)
    kw = dict(max_tris=maxT, max_verts=maxV, max_charts=1 << 15, max_width=1920, max_height=1080, max_atlas_log2=12)
    batch = F.Batch(4, **kw)
    solo = F.Context(**kw)
    meshes = [F.BatchMesh(batch, sc.pos, sc.idx) for sc, _, _ in views]
    smeshes = [F.Mesh(solo, sc.pos, sc.idx) for sc, _, _ in views]
    params = [F.frame_params(M, p["width"], p["height"], p["ratio"], p["atlas_log2"]) for _, M, p in views]
    out = [F.FrameBuffers.allocate(m.T, m.V, kw["max_charts"]) for m in meshes]
    ref = []
    for (sc, M, p), m in zip(views, smeshes):
        b, st = run_gpu(F, solo, m, M, p["width"], p["height"], p["ratio"], p["atlas_log2"])
        assert st == 0
        ref.append(b)
    plan = F.BatchPlan(batch, meshes, params, out)

    def check():
        torch.cuda.synchronize()
        for r, o in zip(ref, out):
            assert_same(r, o, int(r.count[0]))
        for o in out:
            o.vt.zero_()
            o.result.fill_(-1)

    plan.launch()
    check()
    for lanes, pol, pct, mid, rfl in [(1, 0, 100, 16, 0), (2, 1, 50, 64, 1), (4, 0, 200, 256, 0), (3, 1, 100, 16, 1)]:
        plan.set_schedule(lanes, pol, pct, mid, rfl)
        plan.launch()
        check()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        plan.launch()
    g.replay()
    check()
    lanes, pol, pct, mid, rfl, ms = plan.tune(reps=1)
    assert 1 <= lanes <= 4 and ms > 0 and mid in (16, 64) and rfl in (0, F.FA_RASTER_HIZ)
    plan.launch()
    check()
    del g
    plan.close()
    for m in meshes + smeshes:
        m.close()
    batch.close()
    solo.close()
    # one view of the plan compared with the oracle
    sc, M, p = views[1]
    compare_frame(sc, M, p["width"], p["height"], p["ratio"], p["atlas_log2"], ref[1], 0)


def test_persistent_wait_runs_out_then_next_launch_is_clean(F):
    sc, M, p = S.icosphere_frame(5, 10)
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 15, max_width=p["width"],
                    max_height=p["height"], max_atlas_log2=p["atlas_log2"])
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    ctx.set_wait_limits(wait_ns=0)
    b, st = run_gpu(F, ctx, mesh, M, *args, flags=F.FA_FRAME_PERSISTENT)
    assert st == F.FA_E_TIMEOUT
    assert int(b.result[3]) == F.FA_E_TIMEOUT
    ctx.set_wait_limits()
    b, st = run_gpu(F, ctx, mesh, M, *args, flags=F.FA_FRAME_PERSISTENT)
    compare_frame(sc, M, *args, b, st)
    mesh.close()
    ctx.close()
