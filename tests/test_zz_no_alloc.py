"""kl_render_noalloc: the render for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they render, for instance code
embedded in an application that owns the whole device heap through its own
pool, or a render loop held to a fixed device-memory budget.  This entry point
keeps its tables in a scratch array compiled into the library, so such a
caller passes only the image and the counters.  The test checks, through the
C ABI, that two calls in a row give exactly what kl_render gives with a
caller-allocated workspace (same arithmetic, so the same hits), and that a
job larger than the array is refused.  It lives in a file of its own that
pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import klsynth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device for a gpu-marked test")
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


@pytest.mark.parametrize("group,depth,size,window", [
    (klsynth.GASKET, 14, 2048, (-1.5, 1.5, -1.5, 1.5)),
    (klsynth.NEAR_CUSP, 13, 1536, (-2.0, 2.0, -2.0, 2.0)),
])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_render_twice(kl, group, depth, size, window, precision):
    import torch
    prec = kl.FP64 if precision == "fp64" else kl.MIXED
    p = kl.params_init(group.ta, group.tb, depth, size, size, window, prec)
    assert kl.workspace_bytes(p) <= kl.binding.KL_STATIC_SCRATCH_BYTES
    ref_img, ref_cnt = kl.render(p)
    ref = ref_img.cpu().numpy().view(np.uint32).copy()
    ref_c = ref_cnt.cpu().numpy().copy()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        img = torch.full((size, size), 7, dtype=torch.int32, device="cuda")
        cnt = torch.full((kl.KL_N_COUNTERS,), 3, dtype=torch.int64, device="cuda")
        st = kl.lib().kl_render_noalloc(ctypes.byref(p), img.data_ptr(), cnt.data_ptr(), stream)
        assert st == 0, kl.status_string(st)
        torch.cuda.synchronize()
        assert np.array_equal(img.cpu().numpy().view(np.uint32), ref)
        assert np.array_equal(cnt.cpu().numpy(), ref_c)
    assert int(ref_c[0]) + int(ref_c[1]) == kl.word_count(depth)


def test_noalloc_refuses_jobs_larger_than_its_array(kl):
    import torch
    c = klsynth.C3   # length 20: its tables exceed the 32 MiB array
    p = kl.params_init(c.group.ta, c.group.tb, c.depth, 1024, 1024, c.window, kl.MIXED)
    assert kl.workspace_bytes(p) > kl.binding.KL_STATIC_SCRATCH_BYTES
    img = torch.zeros((1024, 1024), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(kl.KL_N_COUNTERS, dtype=torch.int64, device="cuda")
    st = kl.lib().kl_render_noalloc(ctypes.byref(p), img.data_ptr(), cnt.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == 4   # KL_ENOSPACE
