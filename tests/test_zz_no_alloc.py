"""The allocation-free entry point (sunb_integrate_robertson_noalloc).

It serves callers that own all device memory and may not allocate once
their time loop runs; its scratch is a static device array shared by every
call.  Its results must equal those of the context-based entry point
(sunb_integrate on a Robertson context), on two calls in a row -- the
second call finds the first call's counter and counters in the shared
array and must not be affected by them.  The file is named to be collected
last.
"""
import numpy as np
import pytest

import synth
from gpu_util import dev, need_gpu, sb, torch

pytestmark = pytest.mark.gpu
RTOL, ATOL = 1e-6, 1e-10


def test_noalloc_matches_context_entry_point_twice():
    need_gpu()
    m = sb()
    w = synth.workloads.robertson(1024)
    k = dev(w["params"])
    # reference: the existing entry point
    it = m.from_workload(w)
    it.set_params(k)
    y_ref = dev(w["y0"])
    st_ref = torch.zeros(1024, dtype=torch.int32, device="cuda")
    it.integrate(y_ref, w["t0"], w["tout"], st_ref)
    y_ref, st_ref = y_ref.cpu().numpy(), st_ref.cpu().numpy()
    assert np.all(st_ref == 0)
    for call in range(2):
        y = dev(w["y0"])
        st = torch.full((1024,), 99, dtype=torch.int32, device="cuda")
        m.integrate_robertson_noalloc(k, y, w["t0"], w["tout"], RTOL, [ATOL] * 3, status=st)
        torch.cuda.synchronize()
        y, st = y.cpu().numpy(), st.cpu().numpy()
        np.testing.assert_array_equal(st, st_ref)
        # same kernel arithmetic: equal to rounding (the tolerance the GPU
        # tests use for identical computations is bitwise; allow 1e-12)
        np.testing.assert_allclose(y, y_ref, rtol=1e-12, atol=1e-300)
        assert np.max(np.abs(y.sum(axis=1) - 1.0)) < 1e-9


def test_noalloc_rejects_batches_beyond_its_static_scratch():
    need_gpu()
    m = sb()
    n = 65537
    k = torch.ones((n, 3), dtype=torch.float64, device="cuda")
    y = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(m.SunbError) as e:
        m.integrate_robertson_noalloc(k, y, 0.0, 1.0, RTOL, [ATOL] * 3)
    assert e.value.code == m.ILL_INPUT
    assert "65536" in str(e.value)
