"""Failure detection on the device: every loop that waits on other threads has a
limit (fa_set_wait_limits), and running it out gives FA_E_TIMEOUT in the device
status word and the pack result, never a trap or a hang; the next frame on the
same context is clean and equals the oracle.

The limits are lowered on purpose here.  With a hooking cap of 0, the first
union-find hooking step that finds two different roots gives up: on the
heightfield frame the visible patch spans several 1024-triangle tiles, so the
cross-tile hooking always meets such a step.  The push's bulk-copy wait is run
with a limit of 0 as well; whether it runs out depends on timing, so that case
checks that the outcome is one of the two consistent ones and that the context
recovers.  The packing width scan's look-back never gives up: with a poll limit
of 0 every item sums the earlier chunks that have not published yet itself, and
the packing still equals the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2502_17712_gb300 import scenes as S
from test_gpu_parity import F, compare_frame, run_gpu  # noqa: F401  (fixture + checker)

pytestmark = pytest.mark.gpu


def test_hooking_cap_runs_out_then_next_frame_is_clean(F):
    import torch
    sc, M, p = S.heightfield_frame(1)
    W, H, r, L = p["width"], p["height"], p["ratio"], p["atlas_log2"]
    ctx = F.Context(max_tris=sc.T, max_verts=sc.V, max_charts=1 << 14, max_width=W, max_height=H,
                    max_atlas_log2=L)
    mesh = F.Mesh(ctx, sc.pos, sc.idx)
    bufs, st = run_gpu(F, ctx, mesh, M, W, H, r, L)
    assert st == F.FA_OK
    assert (sc.T + 1023) // 1024 > 1
    ctx.set_wait_limits(loop_cap=0)
    bufs, st = run_gpu(F, ctx, mesh, M, W, H, r, L)
    assert st == F.FA_E_TIMEOUT
    assert int(bufs.result[3]) == F.FA_E_TIMEOUT  # the pack saw the word and skipped its work
    assert ctx.device_status() == F.FA_OK         # read and cleared
    ctx.set_wait_limits()                          # defaults again
    bufs, st = run_gpu(F, ctx, mesh, M, W, H, r, L)
    compare_frame(sc, M, W, H, r, L, bufs, st)
    torch.cuda.synchronize()
    mesh.close()
    ctx.close()


def test_pack_waits_with_zero_limits_stay_consistent_and_recover(F):
    import torch
    n, log2 = 40000, 12
    fa, fb = S.lognormal_boxes(6, n, mean_texels=6)
    ctx = F.Context(max_tris=1024, max_verts=1024, max_charts=1 << 16, max_width=64, max_height=64,
                    max_atlas_log2=12)
    d_fa = torch.as_tensor(fa.view(np.int32)).cuda()
    d_fb = torch.as_tensor(fb.view(np.int32)).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    place = torch.zeros(1 << 16, 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    pk = O.pack(fa, fb, log2)
    ctx.set_wait_limits(loop_cap=0, wait_ns=0)
    for _ in range(3):
        F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, 64, 0, None, place, res)
        torch.cuda.synchronize()
        st = ctx.device_status()
        r = res.cpu().numpy().view(np.uint32)
        assert st in (F.FA_OK, F.FA_E_TIMEOUT)
        if st == F.FA_OK:
            assert (int(r[0]), int(r[1]), int(r[3])) == (pk.k, pk.omega, 0)
        else:
            assert int(r[3]) == F.FA_E_TIMEOUT
    ctx.set_wait_limits()
    F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, 64, 0, None, place, res)
    torch.cuda.synchronize()
    assert ctx.device_status() == F.FA_OK
    r = res.cpu().numpy().view(np.uint32)
    assert (int(r[0]), int(r[1]), int(r[2]), int(r[3])) == (pk.k, pk.omega, pk.height, 0)
    assert (place[:n].cpu().numpy() == pk.place).all()
    ctx.close()


@pytest.mark.parametrize("n", [12000, 40000])
def test_scan_look_back_sums_unpublished_chunks_itself(F, n):
    """loop_cap = 0: the width scan polls no earlier chunk, so each item adds up the
    widths of the chunks before it that have published nothing yet (the fallback
    that lets the scan finish whichever of its CTAs are resident).  12,000 boxes are
    3 chunks (one candidate per item, one wave); 40,000 are 10 chunks (two
    candidates per item, and some CTAs take a second item)."""
    import torch
    log2 = 12
    fa, fb = S.lognormal_boxes(6, n, mean_texels=6)
    ctx = F.Context(max_tris=1024, max_verts=1024, max_charts=1 << 16, max_width=64, max_height=64,
                    max_atlas_log2=12)
    d_fa = torch.as_tensor(fa.view(np.int32)).cuda()
    d_fb = torch.as_tensor(fb.view(np.int32)).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    place = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int32, device="cuda")
    ctx.set_wait_limits(loop_cap=0)
    for sel in (0, 1):
        pk = O.pack(fa, fb, log2, select_mode=sel)
        F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, 64, sel, None, place, res)
        torch.cuda.synchronize()
        assert ctx.device_status() == F.FA_OK
        r = res.cpu().numpy().view(np.uint32)
        assert (int(r[0]), int(r[1]), int(r[2]), int(r[3])) == (pk.k, pk.omega, pk.height, 0)
        assert (place.cpu().numpy() == pk.place).all()
    ctx.close()
