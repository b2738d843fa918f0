"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bit-exact: VT bits, chart ids, roots, chart count, NDC boxes (fp32 bits),
footprints, rotations, the packing order, placements and the chosen candidate.
UVs: |GPU - fp64 oracle| <= 1e-4 texel flat wherever fp32 can hold the value to
1e-4 (|uv| < 2048 texels, which is every corner inside an atlas of side <= 2048);
larger values (corners in 4096^2 atlases, off-screen corners of partially visible
triangles) must be the correctly rounded fp32 value (half an ulp, plus 2^-30 |uv|
for the compensated arithmetic before the final rounding).
"""
import numpy as np
import pytest

import oracle as O
from paper_2502_17712_gb300 import scenes as S

pytestmark = pytest.mark.gpu

UV_TOL = 1e-4


def uv_tolerance(o):
    """Accepted |GPU - oracle| for UV components whose fp64 oracle value is o."""
    a = np.abs(np.asarray(o, np.float64))
    _, e = np.frexp(np.maximum(a, 1.0))
    half_ulp = np.ldexp(1.0, e - 25)  # half the fp32 spacing in a's binade
    return np.where(a < 2048.0, UV_TOL, np.maximum(UV_TOL, half_ulp + 2.0 ** -30 * a))


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2502_17712_gb300 import build, fastatlas
    build.build()
    fastatlas.load()
    return fastatlas


def run_gpu(F, ctx, mesh, M, W, H, ratio, log2, mode=0, n_scales=64, select_mode=0, bufs=None, flags=0):
    import torch
    if bufs is None:
        bufs = F.FrameBuffers.allocate(mesh.T, mesh.V, ctx.cfg.max_charts, vert_chart=True, partial=True)
    F.atlas_frame(ctx, mesh, bufs, M, W, H, ratio, log2, mode, n_scales, select_mode, flags=flags)
    torch.cuda.synchronize()
    st = ctx.device_status()
    return bufs, st


def to_np(t):
    return t.cpu().numpy()


def compare_frame(sc, M, W, H, ratio, log2, bufs, status, mode=0, n_scales=64, select_mode=0, vt=None,
                  flags=0, gutter=0):
    fr = O.atlas_frame(M, sc.pos, sc.idx, W, H, ratio, log2, mode=mode, n_scales=n_scales,
                       select_mode=select_mode, vt=vt, flags=flags, gutter=gutter)
    assert status == 0
    T = sc.T
    gvt = to_np(bufs.vt).view(np.uint32)
    if vt is None:
        assert (gvt == fr.vt).all(), f"VT differs in {int((gvt != fr.vt).sum())} words"
    C = int(to_np(bufs.count)[0])
    assert C == fr.charts.C
    assert (to_np(bufs.tri_chart) == fr.charts.tri_chart).all()
    assert (to_np(bufs.root)[:C].view(np.uint32) == fr.charts.roots).all()
    if mode == 1:
        assert (to_np(bufs.vert_chart) == fr.charts.vert_chart).all()
    gb = to_np(bufs.bbox)[:C]
    assert (gb.view(np.uint32) == fr.fp.bbox.view(np.uint32)).all()
    assert (to_np(bufs.fa)[:C].view(np.uint32) == fr.fp.fa).all()
    assert (to_np(bufs.fb)[:C].view(np.uint32) == fr.fp.fb).all()
    assert (to_np(bufs.rot)[:C] == fr.fp.rot).all()
    if bufs.partial is not None:
        gp = to_np(bufs.partial).view(np.uint32)
        assert (gp == fr.fp.partial).all(), f"partial bits differ in {int((gp != fr.fp.partial).sum())} words"
    assert (to_np(bufs.order)[:C].view(np.uint32) == fr.order).all()
    res = to_np(bufs.result).view(np.uint32)
    assert int(res[3]) == fr.pk.status
    if fr.pk.status == 0:
        assert (int(res[0]), int(res[1]), int(res[2])) == (fr.pk.k, fr.pk.omega, fr.pk.height)
        assert (to_np(bufs.place)[:C] == fr.pk.place).all()
        u = to_np(bufs.uv).astype(np.float64)
        vis = fr.charts.tri_chart >= 0
        ou = fr.uv[vis]
        gu = u[vis]
        nan = np.isnan(ou)
        assert (np.isnan(gu) == nan).all()
        o = ou[~nan]
        err = np.abs(gu[~nan] - o)
        tol = uv_tolerance(o)
        assert (err <= tol).all(), f"UV error {err[err > tol].max():.3g} above its tolerance"
        inside = np.abs(o) < float(1 << log2)
        fr.uv_err_inside = float(err[inside].max()) if inside.any() else 0.0
        fr.uv_err_max = float(err.max()) if err.size else 0.0
        fr.uv_outside = int((~inside).sum())
        ga = to_np(bufs.affine)[:C].astype(np.float64)
        assert np.allclose(ga, fr.affine, rtol=1e-6, atol=2e-4)
    return fr


@pytest.fixture(scope="module")
def small_ctx(F):
    return F.Context(max_tris=1 << 16, max_verts=1 << 16, max_charts=1 << 15, max_width=1920,
                     max_height=1080, max_atlas_log2=12)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("mode", [0, 1])
def test_heightfield_frame(F, small_ctx, seed, mode):
    sc, M, p = S.heightfield_frame(seed)
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    bufs, st = run_gpu(F, small_ctx, mesh, M, p["width"], p["height"], p["ratio"], p["atlas_log2"], mode)
    compare_frame(sc, M, p["width"], p["height"], p["ratio"], p["atlas_log2"], bufs, st, mode)


@pytest.mark.parametrize("ratio,log2,n_scales,sel", [(0.5, 9, 64, 0), (2.0, 10, 32, 0), (1.0, 8, 16, 1),
                                                     (4.0, 9, 64, 0)])
def test_heightfield_variants(F, small_ctx, ratio, log2, n_scales, sel):
    sc = S.grid_scene(5)
    W, H = 1280, 720
    M = S.hemisphere_camera(5, W, H, radius=2.2)
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    bufs, st = run_gpu(F, small_ctx, mesh, M, W, H, ratio, log2, 0, n_scales, sel)
    compare_frame(sc, M, W, H, ratio, log2, bufs, st, 0, n_scales, sel)


def test_big_triangles_full_hd(F, small_ctx):
    # ~500-pixel triangles exercise the queued tile rasterizer
    for seed in (7, 8):
        sc = S.grid_scene(seed)
        M = S.spline_cameras(seed, 5, 1920, 1080)[seed % 5]
        mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
        bufs, st = run_gpu(F, small_ctx, mesh, M, 1920, 1080, 1.0, 11)
        compare_frame(sc, M, 1920, 1080, 1.0, 11, bufs, st)


def test_near_plane_and_guard_band_clipping(F, small_ctx):
    # camera inside a field of instanced patches, close to the surface
    sc = S.instanced_grid_scene(3, 6, n=24)
    W, H = 640, 360
    for i, eye in enumerate([(0.1, 0.2, 0.12), (-0.5, 0.3, 0.06), (1.0, -1.0, 0.3)]):
        M = S.view_proj(eye, (eye[0] + 1.0, eye[1] + 0.4, -0.2), (0, 0, 1), W, H, near=0.05)
        mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
        bufs, st = run_gpu(F, small_ctx, mesh, M, W, H, 1.0, 10)
        compare_frame(sc, M, W, H, 1.0, 10, bufs, st)


def test_nothing_visible(F, small_ctx):
    sc = S.grid_scene(1)
    M = S.view_proj((0, 0, 3), (0, 0, 6), (0, 1, 0), 320, 240)  # looking away
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    bufs, st = run_gpu(F, small_ctx, mesh, M, 320, 240, 1.0, 10)
    fr = compare_frame(sc, M, 320, 240, 1.0, 10, bufs, st)
    assert fr.charts.C == 0 and int(to_np(bufs.count)[0]) == 0


def test_non_manifold_and_degenerate_mesh(F, small_ctx):
    # a fan of four triangles on one edge, degenerate triangles, an isolated one
    pos = np.array([[-0.5, -0.5, 0.0], [0.5, -0.5, 0.0], [0.0, 0.5, 0.0], [0.0, -0.9, 0.1],
                    [0.3, 0.6, -0.1], [-0.6, 0.2, 0.05], [0.6, 0.1, 0.2], [-0.8, -0.8, 0.0],
                    [-0.7, -0.8, 0.0], [-0.75, -0.7, 0.0]], np.float32)
    idx = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4], [0, 1, 6], [0, 0, 5], [2, 2, 2], [7, 8, 9],
                    [1, 2, 6]], np.uint32)
    M = np.eye(4, dtype=np.float32)
    mesh = F.Mesh(small_ctx, pos, idx)
    for mode in (0, 1):
        # visibility from the GPU; also force a VT that keeps the fan visible
        bufs, st = run_gpu(F, small_ctx, mesh, M, 64, 64, 1.0, 8, mode)
        compare_frame(S.Scene(pos, idx), M, 64, 64, 1.0, 8, bufs, st, mode)


def test_standalone_calls_equal_frame(F, small_ctx):
    import torch
    sc, M, p = S.heightfield_frame(4)
    W, H, r, L = p["width"], p["height"], p["ratio"], p["atlas_log2"]
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    ref, st = run_gpu(F, small_ctx, mesh, M, W, H, r, L)
    b = F.FrameBuffers.allocate(mesh.T, mesh.V, small_ctx.cfg.max_charts)
    h = small_ctx.handle
    F.fa_visibility(h, mesh.handle, M, W, H, b.vt)
    ch = b.charts()
    F.fa_chartify(h, mesh.handle, b.vt, 0, b.tri_chart, None, ch)
    F.fa_parameterize(h, mesh.handle, M, W, H, r, b.tri_chart, ch)
    F.fa_pack(h, b.fa, b.fb, b.count, L, 64, 0, b.order, b.place, b.result)
    F.fa_uv(h, mesh.handle, M, W, H, r, b.tri_chart, ch, b.place, b.result, L, 64, b.uv, b.affine)
    torch.cuda.synchronize()
    assert small_ctx.device_status() == 0
    for name in ("vt", "tri_chart", "count", "bbox", "fa", "fb", "rot", "place", "result", "affine"):
        assert torch.equal(getattr(ref, name), getattr(b, name)), name
    assert torch.equal(torch.nan_to_num(ref.uv, 7.0), torch.nan_to_num(b.uv, 7.0))


def test_deterministic_repeat(F, small_ctx):
    import torch
    sc, M, p = S.heightfield_frame(6)
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    a, _ = run_gpu(F, small_ctx, mesh, M, p["width"], p["height"], 1.0, 10)
    b, _ = run_gpu(F, small_ctx, mesh, M, p["width"], p["height"], 1.0, 10)
    for name in ("vt", "tri_chart", "bbox", "place", "result"):
        assert torch.equal(getattr(a, name), getattr(b, name))
    assert torch.equal(torch.nan_to_num(a.uv, 7.0), torch.nan_to_num(b.uv, 7.0))


# ------------------------------------------------------------------ packing alone


@pytest.mark.parametrize("n,log2,seed", [(1, 4, 0), (3, 5, 1), (1000, 10, 2), (1023, 9, 3), (1025, 11, 4),
                                         (12000, 11, 5), (40000, 12, 6)])
def test_pack_matches_oracle(F, n, log2, seed):
    import torch
    ctx = F.Context(max_tris=1024, max_verts=1024, max_charts=1 << 16, max_width=64, max_height=64,
                    max_atlas_log2=12)
    fa, fb = S.lognormal_boxes(seed, n, mean_texels=6 if n > 5000 else 12)
    d_fa = torch.as_tensor(fa.view(np.int32)).cuda()
    d_fb = torch.as_tensor(fb.view(np.int32)).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    order = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    place = torch.zeros(1 << 16, 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    for sel in (0, 1):
        F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, 64, sel, order, place, res)
        torch.cuda.synchronize()
        pk = O.pack(fa, fb, log2, select_mode=sel)
        r = to_np(res).view(np.uint32)
        assert int(r[3]) == pk.status
        assert (to_np(order)[:n].view(np.uint32) == O.order(fb)).all()
        if pk.status == 0:
            assert (int(r[0]), int(r[1]), int(r[2])) == (pk.k, pk.omega, pk.height)
            assert (to_np(place)[:n] == pk.place).all()
    ctx.close()


@pytest.mark.parametrize("n_scales,mean_texels,fits", [(1, 5, True), (1, 16, False), (2, 16, True),
                                                      (4, 16, True), (8, 16, True)])
def test_pack_few_scales_matches_oracle(F, n_scales, mean_texels, fits):
    """Short scale ladders (Sec. 4.2: candidates k / n, k = 1..n), on three 4096-box
    chunks and a ragged tail: the width scan takes two candidates per work item, so
    n = 1 leaves the second slot of its only item empty.  At 16 texels per box the
    largest candidates overflow (the oracle picks k = 1, 2, 5 of 2, 4, 8) and the
    single candidate of n = 1 fails."""
    import torch
    n, log2 = 13001, 11
    ctx = F.Context(max_tris=1024, max_verts=1024, max_charts=1 << 16, max_width=64, max_height=64,
                    max_atlas_log2=12)
    fa, fb = S.lognormal_boxes(40 + n_scales, n, mean_texels=mean_texels)
    d_fa = torch.as_tensor(fa.view(np.int32)).cuda()
    d_fb = torch.as_tensor(fb.view(np.int32)).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    place = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    for sel in (0, 1):
        F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, n_scales, sel, None, place, res)
        torch.cuda.synchronize()
        pk = O.pack(fa, fb, log2, n_scales, select_mode=sel)
        r = to_np(res).view(np.uint32)
        assert int(r[3]) == pk.status
        assert (pk.status == 0) == fits
        if fits:
            assert (int(r[0]), int(r[1]), int(r[2])) == (pk.k, pk.omega, pk.height)
            assert (to_np(place) == pk.place).all()
    ctx.close()


def test_pack_one_scale_past_one_wave(F):
    """One candidate (n = 1) on 305 chunks of 4096 boxes plus a ragged tail: more
    chunks than the width scan's CTAs, so the scan pairs candidates per work item and
    every item's second slot is empty."""
    import torch
    n, log2 = 305 * 4096 + 77, 12
    ctx = F.Context(max_tris=64, max_verts=64, max_charts=1 << 21, max_atlas_log2=log2)
    fa, fb = S.lognormal_boxes(77, n, mean_texels=1)
    d_fa = torch.as_tensor(fa.view(np.int32)).cuda()
    d_fb = torch.as_tensor(fb.view(np.int32)).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    place = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    for sel in (0, 1):
        F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, 1, sel, None, place, res)
        torch.cuda.synchronize()
        pk = O.pack(fa, fb, log2, 1, select_mode=sel)
        r = to_np(res).view(np.uint32)
        assert pk.status == 0 and int(r[3]) == 0
        assert (int(r[0]), int(r[1]), int(r[2]), int(r[4])) == (pk.k, pk.omega, pk.height, n)
        assert (to_np(place) == pk.place).all()
    ctx.close()


@pytest.mark.parametrize("n,log2,mean_texels,seed", [(1, 1, 1, 0), (2, 1, 1, 1), (1, 2, 1, 2), (40, 3, 1, 3),
                                                       (60000, 14, 800, 4)])
def test_pack_extreme_atlas_sizes(F, n, log2, mean_texels, seed):
    """The smallest atlases (2^1 .. 2^3 texels: one box fits a 2x2 atlas, two do not)
    and the largest one (2^14, with boxes so large that only k = 6 of 64 fits and the
    frontline spans 16,479 texels)."""
    import torch
    ctx = F.Context(max_tris=64, max_verts=64, max_charts=1 << 16, max_atlas_log2=14)
    fa, fb = S.lognormal_boxes(seed, n, mean_texels=mean_texels)
    d_fa = torch.as_tensor(fa.view(np.int32)).cuda()
    d_fb = torch.as_tensor(fb.view(np.int32)).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    place = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    for sel in (0, 1):
        F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, 64, sel, None, place, res)
        torch.cuda.synchronize()
        pk = O.pack(fa, fb, log2, select_mode=sel)
        r = to_np(res).view(np.uint32)
        assert int(r[3]) == pk.status
        if pk.status == 0:
            assert (int(r[0]), int(r[1]), int(r[2])) == (pk.k, pk.omega, pk.height)
            assert (to_np(place) == pk.place).all()
    ctx.close()


def test_pack_failure_and_capacity(F):
    import torch
    ctx = F.Context(max_tris=1024, max_verts=1024, max_charts=1024, max_width=64, max_height=64,
                    max_atlas_log2=12)
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    place = torch.zeros(1024, 4, dtype=torch.int32, device="cuda")
    # a single box far taller than the atlas: no candidate fits
    fa = torch.tensor([256 * 100], dtype=torch.int32, device="cuda")
    fb = torch.tensor([256 * 100000], dtype=torch.int32, device="cuda")
    cnt = torch.tensor([1], dtype=torch.int32, device="cuda")
    F.fa_pack(ctx.handle, fa, fb, cnt, 6, 64, 0, None, place, res)
    torch.cuda.synchronize()
    assert int(res[3]) == F.FA_E_PACK_FAILED
    # a box wider than 8 omega overflows the frontline capacity
    fa = torch.tensor([256 * 1000], dtype=torch.int32, device="cuda")
    fb = torch.tensor([256 * 1000], dtype=torch.int32, device="cuda")
    F.fa_pack(ctx.handle, fa, fb, cnt, 6, 64, 0, None, place, res)
    torch.cuda.synchronize()
    assert int(res[3]) == F.FA_E_CAPACITY
    # more boxes than max_charts
    cnt = torch.tensor([5000], dtype=torch.int32, device="cuda")
    F.fa_pack(ctx.handle, fa, fb, cnt, 6, 64, 0, None, place, res)
    torch.cuda.synchronize()
    assert int(res[3]) == F.FA_E_CAPACITY
    # host-side argument errors
    with pytest.raises(F.FastAtlasError):
        F.fa_pack(ctx.handle, fa, fb, cnt, 13, 64, 0, None, place, res)  # above max_atlas_log2
    with pytest.raises(F.FastAtlasError):
        F.fa_pack(ctx.handle, fa, fb, cnt, 6, 48, 0, None, place, res)  # not a power of two
    ctx.close()


def test_chart_capacity_error(F):
    sc, M, p = S.heightfield_frame(2)
    ctx = F.Context(max_tris=1 << 14, max_verts=1 << 13, max_charts=4, max_width=480, max_height=270,
                    max_atlas_log2=10)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    # vertex-disjoint checkerboard-like visibility through many charts: use edge mode on
    # a frame whose edge charts exceed 4 by forcing a sparse VT
    import torch
    b = F.FrameBuffers.allocate(mesh.T, mesh.V, 4)
    vis = np.zeros(sc.T, bool)
    vis[::2] = True
    b.vt.copy_(torch.as_tensor(O.bool_to_vt(vis).view(np.int32)))
    F.fa_chartify(ctx.handle, mesh.handle, b.vt, 0, b.tri_chart, None, b.charts())
    torch.cuda.synchronize()
    assert ctx.device_status() == F.FA_E_CAPACITY
    assert int(b.count[0]) == sc.T // 2
    assert ctx.device_status() == 0  # read-and-clear


# ------------------------------------------------------------------ the 4.1M-triangle frame


@pytest.fixture(scope="module")
def sphere_frame():
    return S.icosphere_frame(1)


@pytest.mark.parametrize("mode,ratio", [(0, 1.0), (1, 1.0), (0, 0.5), (0, 2.0)])
def test_icosphere_frame_full_size(F, sphere_frame, mode, ratio):
    """200 icospheres (4,096,000 triangles), 1920x1080, 2048^2 atlas: the whole frame
    at full size, every output compared (the oracle takes ~10 s here), at the
    texel-to-pixel ratios 1 (both chart modes), 0.5 and 2 (edge charts; each ratio
    selects a different candidate, so the push takes a different path)."""
    sc, M, p = sphere_frame
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 17, max_width=1920, max_height=1080,
                    max_atlas_log2=11)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    bufs, st = run_gpu(F, ctx, mesh, M, p["width"], p["height"], ratio, p["atlas_log2"], mode)
    fr = compare_frame(sc, M, p["width"], p["height"], ratio, p["atlas_log2"], bufs, st, mode)
    assert fr.pk.status == 0
    print(f"ratio {ratio} mode {mode}: k={fr.pk.k} Omega={fr.pk.omega} charts={fr.charts.C} "
          f"max |duv| inside the atlas {fr.uv_err_inside:.3g} texel, overall {fr.uv_err_max:.3g} "
          f"({fr.uv_outside} components outside)")
    assert fr.uv_err_inside <= UV_TOL
    mesh.close()
    ctx.close()


# ---------------------------------------------------------------- box variant, partial bits

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_frustum_clip_boxes_heightfield(F, small_ctx, seed):
    sc, M, p = S.heightfield_frame(seed)
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    bufs, st = run_gpu(F, small_ctx, mesh, M, *args, flags=F.FA_BOX_FRUSTUM_CLIP)
    compare_frame(sc, M, *args, bufs, st, flags=F.FA_BOX_FRUSTUM_CLIP)


def test_frustum_clip_boxes_icospheres(F):
    sc, M, p = S.icosphere_frame(3, 30)
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 16, max_width=1920, max_height=1080,
                    max_atlas_log2=11)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    for flags in (0, F.FA_BOX_FRUSTUM_CLIP):
        bufs, st = run_gpu(F, ctx, mesh, M, *args, flags=flags)
        fr = compare_frame(sc, M, *args, bufs, st, flags=flags)
        assert int(fr.fp.partial.astype(np.uint64).sum()) > 0  # the view cuts some charts
    mesh.close()
    ctx.close()


def test_standalone_parameterize_flags_and_partial(F, small_ctx):
    import torch
    sc = S.grid_scene(9)
    W, H = 640, 360
    M = S.hemisphere_camera(9, W, H, radius=1.6)  # close: the view cuts the floor
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    bufs, st = run_gpu(F, small_ctx, mesh, M, W, H, 1.0, 10)
    assert st == 0
    tc = bufs.tri_chart.clone()
    C = int(bufs.count[0])
    for flags in (0, F.FA_BOX_FRUSTUM_CLIP):
        b = F.FrameBuffers.allocate(mesh.T, mesh.V, small_ctx.cfg.max_charts, partial=True)
        b.count.copy_(bufs.count)
        F.fa_parameterize(small_ctx.handle, mesh.handle, M, W, H, 1.0, tc, b.charts(), flags=flags,
                          partial=b.partial)
        torch.cuda.synchronize()
        assert small_ctx.device_status() == 0
        fp = O.parameterize(M, sc.pos, sc.idx, W, H, 1.0, to_np(tc), C, flags)
        assert (to_np(b.bbox)[:C].view(np.uint32) == fp.bbox.view(np.uint32)).all()
        assert (to_np(b.fa)[:C].view(np.uint32) == fp.fa).all()
        assert (to_np(b.fb)[:C].view(np.uint32) == fp.fb).all()
        assert (to_np(b.partial).view(np.uint32) == fp.partial).all()
        assert int(fp.partial.astype(np.uint64).sum()) > 0
    mesh.close()


# ---------------------------------------------------------------- conservative marking

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_conservative_marking_heightfield(F, small_ctx, seed):
    sc, M, p = S.heightfield_frame(seed)
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    bufs, st = run_gpu(F, small_ctx, mesh, M, *args, flags=F.FA_VIS_CONSERVATIVE)
    fr = compare_frame(sc, M, *args, bufs, st, flags=F.FA_VIS_CONSERVATIVE)
    plain = O.visibility(M, sc.pos, sc.idx, p["width"], p["height"])
    assert int(np.unpackbits(fr.vt.view(np.uint8)).sum()) > int(np.unpackbits(plain.view(np.uint8)).sum())


def test_conservative_marking_big_and_clipped(F, small_ctx):
    flags = F.FA_VIS_CONSERVATIVE | F.FA_BOX_FRUSTUM_CLIP
    sc = S.grid_scene(7)
    M = S.spline_cameras(7, 5, 1920, 1080)[2]  # large triangles: the tile rasterizer
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    bufs, st = run_gpu(F, small_ctx, mesh, M, 1920, 1080, 1.0, 11, flags=flags)
    compare_frame(sc, M, 1920, 1080, 1.0, 11, bufs, st, flags=flags)
    sc = S.instanced_grid_scene(3, 6, n=24)  # near plane and guard band crossings
    W, H = 640, 360
    for eye in [(0.1, 0.2, 0.12), (-0.5, 0.3, 0.06)]:
        M = S.view_proj(eye, (eye[0] + 1.0, eye[1] + 0.4, -0.2), (0, 0, 1), W, H, near=0.05)
        mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
        bufs, st = run_gpu(F, small_ctx, mesh, M, W, H, 1.0, 10, flags=flags)
        compare_frame(sc, M, W, H, 1.0, 10, bufs, st, flags=flags)


def test_conservative_marking_icospheres_and_standalone(F):
    import torch
    sc, M, p = S.icosphere_frame(4, 20)
    W, H = p["width"], p["height"]
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 16, max_width=W, max_height=H,
                    max_atlas_log2=11)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    bufs, st = run_gpu(F, ctx, mesh, M, W, H, 1.0, 11, flags=F.FA_VIS_CONSERVATIVE)
    compare_frame(sc, M, W, H, 1.0, 11, bufs, st, flags=F.FA_VIS_CONSERVATIVE)
    vt = torch.zeros_like(bufs.vt)
    F.fa_visibility(ctx.handle, mesh.handle, M, W, H, vt, flags=F.FA_VIS_CONSERVATIVE)
    torch.cuda.synchronize()
    assert torch.equal(vt, bufs.vt)
    mesh.close()
    ctx.close()


# ---------------------------------------------------------------- one packing, two atlases

@pytest.mark.parametrize("d,gutter,seed", [(2, 2, 0), (3, 4, 1), (3, 8, 2)])
def test_pack_lowres_matches_oracle(F, d, gutter, seed):
    import torch
    fa, fb = S.lognormal_boxes(seed, 2000, mean_texels=30.0)
    n, L = len(fa), 12
    ctx = F.Context(max_tris=64, max_verts=64, max_charts=4096, max_atlas_log2=L, gutter=gutter)
    d_fa = torch.as_tensor(fa.view(np.int32)).cuda()
    d_fb = torch.as_tensor(fb.view(np.int32)).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    place = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    F.fa_pack(ctx.handle, d_fa, d_fb, cnt, L, 64, 0, None, place, res, lowres_log2=d)
    torch.cuda.synchronize()
    pk = O.pack(fa, fb, L, 64, 2, gutter, 0, d)
    r = to_np(res).view(np.uint32)
    assert (int(r[3]), int(r[0]), int(r[1]), int(r[2])) == (pk.status, pk.k, pk.omega, pk.height)
    assert (to_np(place) == pk.place).all()
    assert (pk.omega << d) <= 2 * gutter * (1 << L)
    ctx.close()


def test_lowres_frame_matches_oracle(F):
    sc, M, p = S.heightfield_frame(2)
    gutter, flags = 4, F.FA_LOWRES(3)
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 14, max_width=p["width"],
                    max_height=p["height"], max_atlas_log2=p["atlas_log2"], gutter=gutter)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    args = (p["width"], p["height"], p["ratio"], p["atlas_log2"])
    bufs, st = run_gpu(F, ctx, mesh, M, *args, flags=flags)
    fr = compare_frame(sc, M, *args, bufs, st, flags=flags, gutter=gutter)
    assert fr.pk.status == 0 and (fr.pk.omega << 3) <= 2 * gutter * (1 << p["atlas_log2"])
    mesh.close()
    ctx.close()


# ---------------------------------------------------------------- depth ties

def test_coplanar_duplicates_tie_exactly(F, small_ctx):
    """Duplicated triangles give equal depth keys at the same pixels: every copy of a
    visible triangle is visible (the "<=" test); two and three copies."""
    sc = S.grid_scene(4)
    rng = np.random.default_rng(4)
    dup2 = rng.choice(sc.T, 300, replace=False)
    dup3 = rng.choice(sc.T, 100, replace=False)
    idx = np.concatenate([sc.idx, sc.idx[dup2], sc.idx[dup3], sc.idx[dup3]]).astype(np.uint32)
    M = S.hemisphere_camera(4, 640, 360)
    mesh = F.Mesh(small_ctx, sc.pos, idx)
    bufs, st = run_gpu(F, small_ctx, mesh, M, 640, 360, 1.0, 10)
    sc2 = S.Scene(sc.pos, idx)
    fr = compare_frame(sc2, M, 640, 360, 1.0, 10, bufs, st)
    vis = O.vt_to_bool(fr.vt, idx.shape[0])
    T = sc.T
    assert (vis[T:T + 300] == vis[dup2]).all() and vis[dup2].any()
    assert (vis[T + 300:T + 400] == vis[dup3]).all() and (vis[T + 400:] == vis[dup3]).all()
    mesh.close()


# ---------------------------------------------------------------- edge cases

def test_pack_empty_box_set(F):
    import torch
    ctx = F.Context(max_tris=64, max_verts=64, max_charts=4096, max_atlas_log2=11)
    d = torch.zeros(4096, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    place = torch.full((4096, 4), -7, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    for sel in (0, 1):
        F.fa_pack(ctx.handle, d, d, cnt, 11, 64, sel, None, place, res)
        torch.cuda.synchronize()
        pk = O.pack(np.zeros(0, np.uint32), np.zeros(0, np.uint32), 11, 64, 2, 0, sel)
        r = to_np(res).view(np.uint32)
        assert (int(r[3]), int(r[0]), int(r[1]), int(r[2]), int(r[4])) == (pk.status, pk.k, pk.omega, pk.height, 0)
    assert (to_np(place) == -7).all()  # nothing written
    ctx.close()


def test_single_triangle_mesh_and_charts_at_capacity(F):
    # one triangle filling part of the view: one chart, at max_charts = 1 exactly
    pos = np.array([[-0.5, -0.5, 0.0], [0.5, -0.4, 0.1], [0.0, 0.6, -0.1]], np.float32)
    idx = np.array([[0, 1, 2]], np.uint32)
    M = S.view_proj((0, 0, 2), (0, 0, 0), (0, 1, 0), 320, 240)
    ctx = F.Context(max_tris=1, max_verts=3, max_charts=1, max_width=320, max_height=240, max_atlas_log2=9)
    mesh = F.Mesh(ctx, pos, idx)
    bufs, st = run_gpu(F, ctx, mesh, M, 320, 240, 1.0, 9)
    fr = compare_frame(S.Scene(pos, idx), M, 320, 240, 1.0, 9, bufs, st)
    assert fr.charts.C == 1 and fr.pk.status == 0
    mesh.close()
    ctx.close()


def test_chart_count_one_above_capacity(F, small_ctx):
    # two separate triangles but room for one chart: the count is reported, status
    # FA_E_CAPACITY, no chart writes beyond the capacity
    import torch
    pos = np.array([[-0.9, -0.5, 0], [-0.4, -0.5, 0], [-0.6, 0.2, 0],
                    [0.4, -0.5, 0], [0.9, -0.5, 0], [0.6, 0.2, 0]], np.float32)
    idx = np.array([[0, 1, 2], [3, 4, 5]], np.uint32)
    M = np.eye(4, dtype=np.float32)
    ctx = F.Context(max_tris=2, max_verts=6, max_charts=1, max_width=64, max_height=64, max_atlas_log2=8)
    mesh = F.Mesh(ctx, pos, idx)
    b = F.FrameBuffers.allocate(2, 6, 1)
    F.atlas_frame(ctx, mesh, b, M, 64, 64, 1.0, 8)
    torch.cuda.synchronize()
    assert ctx.device_status() == F.FA_E_CAPACITY
    assert int(b.count[0]) == 2
    r = to_np(b.result).view(np.uint32)
    assert int(r[3]) == F.FA_E_CAPACITY
    mesh.close()
    ctx.close()


# ---------------------------------------------------------------- raster schedule

@pytest.mark.parametrize("mid,flags", [(64, 0), (256, 0), (16, 1), (64, 1)])
def test_raster_schedule_changes_no_result(F, small_ctx, mid, flags):
    """Mid-size sub-triangles rasterized in-thread instead of in 16x16 tiles, and the
    marking pass skipping what the tile depths show hidden (fa_set_raster_schedule),
    give the same frame, bit for bit, and the oracle's."""
    import torch
    # (the third scene has more survivors than the raster's lane groups take: its
    # mid-size boxes go to whole warps)
    cases = [(S.grid_scene(7), S.spline_cameras(7, 5, 1920, 1080)[2], 1920, 1080, 11),
             (S.instanced_grid_scene(11, 8, n=24), S.hemisphere_camera(11, 1280, 720, radius=4.0), 1280, 720, 11),
             (S.instanced_grid_scene(13, 24, n=32, half=3.0), S.hemisphere_camera(13, 1920, 1080, radius=4.0),
              1920, 1080, 11)]
    for ci, (sc, M, W, H, L) in enumerate(cases):
        mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
        a, sa = run_gpu(F, small_ctx, mesh, M, W, H, 1.0, L)
        if ci == 2:
            assert small_ctx.frame_stats()["survivors"] > 9728
        small_ctx.set_raster_schedule(mid, flags)
        try:
            b, sb = run_gpu(F, small_ctx, mesh, M, W, H, 1.0, L)
        finally:
            small_ctx.set_raster_schedule()
        assert sa == sb == 0
        for name in ("vt", "tri_chart", "place", "result", "bbox"):
            assert torch.equal(getattr(a, name), getattr(b, name)), name
        assert torch.equal(torch.nan_to_num(a.uv, 7.0), torch.nan_to_num(b.uv, 7.0))
        compare_frame(sc, M, W, H, 1.0, L, b, sb)
        mesh.close()


@pytest.mark.parametrize("uf,push", [(256, 256), (512, 512), (256, 1024), (1024, 1024)])
def test_chart_pack_schedule_changes_no_result(F, small_ctx, uf, push):
    """Other tile shapes of the local union-find and CTA sizes of the push
    (fa_set_chart_pack_schedule) give the same frame, bit for bit, and the oracle's;
    so does fa_pack alone on 40,000 boxes."""
    import torch
    with pytest.raises(F.FastAtlasError):
        small_ctx.set_chart_pack_schedule(128, 1024)
    assert small_ctx.kernel_schedule()["uf_threads"] == 1024
    cases = [(S.grid_scene(7), S.spline_cameras(7, 5, 1920, 1080)[2], 1920, 1080, 11),
             (S.instanced_grid_scene(11, 8, n=24), S.hemisphere_camera(11, 1280, 720, radius=4.0), 1280, 720, 11)]
    for sc, M, W, H, L in cases:
        mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
        a, sa = run_gpu(F, small_ctx, mesh, M, W, H, 1.0, L)
        small_ctx.set_chart_pack_schedule(uf, push)
        try:
            assert small_ctx.kernel_schedule() == {"mid_max_pix": F.FA_RASTER_MID_OFF, "raster_flags": 0,
                                                   "uf_threads": uf, "push_threads": push}
            b, sb = run_gpu(F, small_ctx, mesh, M, W, H, 1.0, L)
        finally:
            small_ctx.set_chart_pack_schedule()
        assert sa == sb == 0
        for name in ("vt", "tri_chart", "place", "result", "bbox"):
            assert torch.equal(getattr(a, name), getattr(b, name)), name
        assert torch.equal(torch.nan_to_num(a.uv, 7.0), torch.nan_to_num(b.uv, 7.0))
        compare_frame(sc, M, W, H, 1.0, L, b, sb)
        mesh.close()
    n, log2 = 40000, 12
    fa, fb = S.lognormal_boxes(6, n, mean_texels=6)
    d_fa = torch.as_tensor(fa.view(np.int32)).cuda()
    d_fb = torch.as_tensor(fb.view(np.int32)).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    ctx = F.Context(max_tris=1024, max_verts=1024, max_charts=1 << 16, max_width=64, max_height=64,
                    max_atlas_log2=12)
    ctx.set_chart_pack_schedule(uf, push)
    place = torch.zeros(1 << 16, 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, 64, 0, None, place, res)
    torch.cuda.synchronize()
    pk = O.pack(fa, fb, log2)
    r = res.cpu().numpy().view(np.uint32)
    assert (int(r[0]), int(r[1]), int(r[2]), int(r[3])) == (pk.k, pk.omega, pk.height, 0)
    assert (place[:n].cpu().numpy() == pk.place).all()
    ctx.close()


@pytest.mark.parametrize("seed", range(6))
def test_grouped_raster_random_views(F, small_ctx, seed):
    """Small meshes (a few thousand survivors: the exact and marking passes give each
    survivor a group of lanes) under seeded views, resolutions and raster options:
    conservative marking, mid-size boxes in-thread, tile-depth marking.  Every frame
    equals the oracle's."""
    rng = np.random.default_rng([seed, 0x6A0])
    n_inst = int(rng.integers(1, 5))
    sc = S.instanced_grid_scene(100 + seed, n_inst, n=int(rng.choice([16, 24, 32])), half=2.0)
    W, H = [(640, 360), (1280, 720), (1920, 1080), (480, 270)][seed % 4]
    M = S.hemisphere_camera(200 + seed, W, H, radius=float(rng.uniform(1.5, 4.0)))
    flags = F.FA_VIS_CONSERVATIVE if seed % 2 else 0
    mid, hiz = [(16, 0), (64, 0), (256, F.FA_RASTER_HIZ)][seed % 3]
    mesh = F.Mesh(small_ctx, sc.pos, sc.idx)
    small_ctx.set_raster_schedule(mid, hiz)
    try:
        bufs, st = run_gpu(F, small_ctx, mesh, M, W, H, 1.0, 11, flags=flags)
    finally:
        small_ctx.set_raster_schedule()
    compare_frame(sc, M, W, H, 1.0, 11, bufs, st, flags=flags)
    mesh.close()
