"""The allocation-free packing entry point (fa_pack_noalloc) gives the same
results as fa_pack with a context.

fa_pack_noalloc serves callers that may not allocate device memory where they
pack (a host application's frame callback or plugin slot with host-owned device
memory, or a real-time loop that must not pay cudaMalloc's device
synchronization); its scratch is a static device array inside the library.  The
test calls it through the C ABI twice in a row, on different box sets, and compares
every output with fa_pack's, bit for bit (all outputs are integers); the second
call must leave the device's free memory unchanged, and an empty box set must give
fa_pack's result too.  This file is collected last so that a first failure here
comes after every other test.
"""
import numpy as np
import pytest

from paper_2502_17712_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def test_pack_noalloc_matches_pack_twice_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2502_17712_gb300 import build, fastatlas as F
    build.build()
    F.load()
    ctx = F.Context(max_tris=1024, max_verts=1024, max_charts=4096, max_width=64, max_height=64,
                    max_atlas_log2=12)
    cases = [(3000, 11, 64, 0, 11), (777, 9, 32, 1, 12), (0, 10, 64, 0, 13)]  # n, log2, scales, select, seed
    for i, (n, log2, ns, sel, seed) in enumerate(cases):
        fa, fb = S.lognormal_boxes(seed, n, mean_texels=8)
        d_fa = torch.zeros(4096, dtype=torch.int32, device="cuda")  # room for 4096 (non-NULL when n = 0)
        d_fb = torch.zeros(4096, dtype=torch.int32, device="cuda")
        d_fa[:n] = torch.as_tensor(fa.view(np.int32)).cuda()
        d_fb[:n] = torch.as_tensor(fb.view(np.int32)).cuda()
        cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
        want_order = torch.zeros(4096, dtype=torch.int32, device="cuda")
        want_place = torch.zeros(4096, 4, dtype=torch.int32, device="cuda")
        want_res = torch.zeros(5, dtype=torch.int32, device="cuda")
        F.fa_pack(ctx.handle, d_fa, d_fb, cnt, log2, ns, sel, want_order, want_place, want_res)
        got_order = torch.full((4096,), -1, dtype=torch.int32, device="cuda")
        got_place = torch.full((4096, 4), -1, dtype=torch.int32, device="cuda")
        got_res = torch.full((5,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        F.fa_pack_noalloc(d_fa, d_fb, n, log2, ns, sel, 2, 0, got_order, got_place, got_res)
        torch.cuda.synchronize()
        if i > 0:  # after the first call's one-time set-up: no device memory taken
            assert torch.cuda.mem_get_info()[0] == free0
        assert int(want_res[3]) == F.FA_OK
        assert torch.equal(got_res, want_res)
        assert torch.equal(got_order[:n], want_order[:n])
        assert torch.equal(got_place[:n], want_place[:n])
    # sizes beyond the static array are rejected up front
    with pytest.raises(F.FastAtlasError) as e:
        F.fa_pack_noalloc(d_fa, d_fb, 4097, 11, 64, 0, 2, 0, None, got_place, got_res)
    assert e.value.status == F.FA_E_CAPACITY
    ctx.close()
