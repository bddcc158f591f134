"""fmm2d_keys_sort_noalloc: keys and stable sort for callers that cannot
allocate GPU memory (the entry point's scratch is a static device array).

Its output must equal what the allocating path (fmm2d_build, read back with
fmm2d_debug_export) produces for the same points - bit for bit, as for all
integer work in these tests - on two calls in a row, the second with a
different point set, so that stale scratch contents would show.  This file
is collected last on purpose.
"""
import numpy as np
import pytest

from gpu_util import _torch
from paper_1204_3105_gb300.inputs import uniform_square

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    torch = _torch()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()
    return fmm2d


@pytest.mark.parametrize("tiling,levels", [("quad", 7), ("sept", 6), ("tri", 8), ("sept", 9)])
def test_noalloc_matches_build_two_calls(fm, tiling, levels):
    torch = _torch()
    dev = torch.device("cuda:0")
    for call, (n, seed) in enumerate([(300007, 11), (1 << 20, 12)]):
        xy, _ = uniform_square(n, seed=seed, dtype=np.float32)
        x_d = torch.from_numpy(xy).to(dev)
        keys = torch.empty(n, dtype=torch.int32, device=dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        # leaf_scale 0: the septree leaf radius of `levels` is the library's own
        fm.fmm2d_keys_sort_noalloc(tiling, levels, 0.0, None, x_d, n, fm.IN_F32, keys, perm)
        plan = fm.Plan(tiling, levels=levels, p=4, flags=fm.PREC_MIXED | fm.IN_F32)
        plan.build(x_d, n, x_d, n)
        want_perm = plan.export("src_perm")
        want_keys = plan.export("src_keys")[want_perm]
        leaf_scale = plan.query()["leaf_scale"]
        plan.close()
        if tiling == "sept":   # the plan's own leaf radius is accepted, another one is not
            k2 = torch.empty_like(keys)
            p2 = torch.empty_like(perm)
            fm.fmm2d_keys_sort_noalloc(tiling, levels, leaf_scale, None, x_d, n, fm.IN_F32, k2, p2)
            assert torch.equal(k2, keys) and torch.equal(p2, perm)
            with pytest.raises(fm.FMM2DError) as e:
                fm.fmm2d_keys_sort_noalloc(tiling, levels, leaf_scale * 1.001, None, x_d, n,
                                           fm.IN_F32, k2, p2)
            assert e.value.status == fm.EINVAL
        got_perm = perm.cpu().numpy().astype(np.int64)
        got_keys = keys.cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.array_equal(got_perm, want_perm), (tiling, call)
        assert np.array_equal(got_keys, want_keys), (tiling, call)


def test_noalloc_rejects_sizes_beyond_maximum(fm):
    torch = _torch()
    dev = torch.device("cuda:0")
    small = torch.zeros(16, dtype=torch.float64, device=dev)
    out = torch.zeros(16, dtype=torch.int32, device=dev)
    with pytest.raises(fm.FMM2DError) as e:
        fm.fmm2d_keys_sort_noalloc("quad", 5, 0.0, None, small, (1 << 20) + 1, 0, out, out)
    assert e.value.status == fm.EINVAL
    assert "1048576" in str(e.value)
