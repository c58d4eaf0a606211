"""CUDA-graph outer steps (hot-path row a15): a captured graph of several
outer steps, re-timed and replayed, gives the same bytes as the same steps
launched one by one through sunb_integrate."""
import numpy as np
import pytest

import synth
from gpu_util import dev, need_gpu, sb, torch

pytestmark = pytest.mark.gpu


def _flat(w):
    if w["kind"] == "mixed":
        return (np.concatenate([w["e0"].ravel(), w["y0_mech"].ravel()]),
                np.concatenate([w["cosmo_params"].ravel(), w["mech_params"].ravel()]))
    return w["y0"].ravel(), w["params"].ravel()


@pytest.mark.parametrize("name", ["mech22", "mixed", "robertson"])
def test_graph_replay_equals_step_by_step(name):
    need_gpu()
    m = sb()
    if name == "mech22":
        w, dt = synth.workloads.mech22(40), 2e-7
    elif name == "mixed":
        w, dt = synth.workloads.mixed(n_cosmo=2000, n_mech=24), 2e-7
    else:
        w, dt = synth.workloads.robertson(64), 10.0
    Y, P = _flat(w)
    p = dev(P)
    steps = 3
    ref = dev(Y)
    it = m.from_workload(w, precision=1 if name != "robertson" else 0, lanes_per_cell=16)
    it.set_params(p)
    for t0 in (0.0, 5 * dt):
        ref.copy_(dev(Y))
        for k in range(steps):
            it.integrate(ref, t0 + k * dt, t0 + (k + 1) * dt)
        torch.cuda.synchronize()
        expect = ref.cpu().numpy()
        it2 = m.from_workload(w, precision=1 if name != "robertson" else 0, lanes_per_cell=16)
        it2.set_params(p)
        y = dev(Y)
        it2.graph_capture(y, 0.0, dt, steps)
        y.copy_(dev(Y))
        it2.graph_launch(t0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(y.cpu().numpy(), expect)
        assert it2.totals()["worst_status"] == 0
        # launching again from the same start repeats the result
        y.copy_(dev(Y))
        it2.graph_launch(t0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(y.cpu().numpy(), expect)


def test_graph_rejects_adjoint_contexts_and_missing_capture():
    need_gpu()
    m = sb()
    w = synth.workloads.adjoint(4)
    it = m.Integrator(m.MECHANISM, 4, mech=w["mech"], record_adjoint=64)
    it.set_params(dev(w["params"]))
    with pytest.raises(m.SunbError):
        it.graph_capture(dev(w["y0"]), 0.0, 1e-6, 2)
    it2 = m.Integrator(m.MECHANISM, 4, mech=w["mech"])
    with pytest.raises(m.SunbError):
        it2.graph_launch(0.0)
