"""The allocation-free entry point (sunb_integrate_robertson_noalloc).

It serves callers that own all device memory and may not allocate once
their time loop runs; its scratch is a static device array shared by every
call.  Its results must equal those of the context-based entry point
(sunb_integrate on a Robertson context) bit for bit -- both launch the same
thread-per-cell kernel, so every cell's arithmetic is the same -- on two
calls in a row: the second call finds the first call's counter and
counters in the shared array and must not be affected by them.  A warm call
must not change the device's free memory.  The file is named to be
collected last.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from gpu_util import dev, need_gpu, sb, torch

pytestmark = pytest.mark.gpu
RTOL, ATOL = 1e-6, 1e-10
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _context_run(m, w, n):
    k = dev(w["params"][:n])
    it = m.Integrator(m.ROBERTSON, n)
    it.set_tolerances(RTOL, ATOL)
    it.set_params(k)
    y = dev(w["y0"][:n])
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    it.integrate(y, w["t0"], w["tout"], st)
    return y.cpu().numpy(), st.cpu().numpy()


def test_noalloc_matches_context_entry_point_twice():
    need_gpu()
    m = sb()
    w = synth.workloads.robertson(1024)
    y_ref, st_ref = _context_run(m, w, 1024)
    assert np.all(st_ref == 0)
    k = dev(w["params"])
    for call in range(2):
        y = dev(w["y0"])
        st = torch.full((1024,), 99, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        m.integrate_robertson_noalloc(k, y, w["t0"], w["tout"], RTOL, [ATOL] * 3, status=st)
        torch.cuda.synchronize()
        if call == 1:     # warm: the module and its static array are loaded
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_reserved() == reserved0
        y, st = y.cpu().numpy(), st.cpu().numpy()
        np.testing.assert_array_equal(st, st_ref)
        np.testing.assert_array_equal(y, y_ref)          # same kernel, same bits
        assert np.max(np.abs(y.sum(axis=1) - 1.0)) < 1e-9


_FRESH = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import synth, paper_2405_01713_b300 as m
w = synth.workloads.robertson(1000)
k = torch.tensor(w["params"], device="cuda")
y = torch.tensor(w["y0"], device="cuda")
# the first CUDA work of this process: the allocation-free call, ragged, no status
m.integrate_robertson_noalloc(k, y, w["t0"], w["tout"], 1e-6, [1e-10] * 3)
torch.cuda.synchronize()
yn = y.cpu().numpy()
it = m.Integrator(m.ROBERTSON, 1000)
it.set_tolerances(1e-6, 1e-10)
it.set_params(k)
y2 = torch.tensor(w["y0"], device="cuda")
it.integrate(y2, w["t0"], w["tout"])
assert np.array_equal(yn, y2.cpu().numpy()), "allocation-free result differs"
assert it.totals()["worst_status"] == 0
print("fresh ok")
"""


def test_noalloc_first_in_a_fresh_process_ragged_without_status():
    need_gpu()
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=ROOT)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


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


def test_noalloc_binding_checks_its_tensors():
    need_gpu()
    m = sb()
    y = torch.zeros((8, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):      # k shorter than y
        m.integrate_robertson_noalloc(torch.ones((4, 3), dtype=torch.float64, device="cuda"), y,
                                      0.0, 1.0, RTOL, [ATOL] * 3)
    with pytest.raises(TypeError):       # k in float32
        m.integrate_robertson_noalloc(torch.ones((8, 3), dtype=torch.float32, device="cuda"), y,
                                      0.0, 1.0, RTOL, [ATOL] * 3)
    with pytest.raises(TypeError):       # status in int64
        m.integrate_robertson_noalloc(torch.ones((8, 3), dtype=torch.float64, device="cuda"), y,
                                      0.0, 1.0, RTOL, [ATOL] * 3,
                                      status=torch.zeros(8, dtype=torch.int64, device="cuda"))
