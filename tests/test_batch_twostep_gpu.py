"""Batched two-step passes (lbm_batch_set_twostep: the frame + rolling
launches over every instance at once).  Each instance must be bit-identical
to the same instance run alone through the single-domain path -- over every
storage the pass serves, BGK and MRT, far fields at rest and in a stream
(the batch then stores every instance shifted), and step counts that mix
graph replays, direct passes and a last single step -- on ragged instance
sizes and on the 256-instance workload."""
import numpy as np
import pytest

from paper_2005_08674_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import lbm as m
    return m


def ragged_batch():
    ws = inputs.batch_instances(count=8, lo=8, hi=300)
    ws += [inputs.Workload("smallest", 8, 8, 0.7, 0, kind="pulse",
                           params=dict(amplitude=1e-3, half_width=1.5, centres=[(3.5, 3.5)])),
           inputs.Workload("thin", 517, 9, 0.6, 0, farfield_u=(0.02, 0.0), kind="pulse",
                           params=dict(amplitude=1e-3, half_width=3.0, centres=[(100.0, 4.0)])),
           inputs.Workload("tall", 131, 700, 0.55, 0, farfield_u=(0.0, 0.03), kind="pulse",
                           params=dict(amplitude=1e-3, half_width=6.0, centres=[(60.0, 650.0)]))]
    return ws


def single(lbm, w, storage, steps, **kw):
    with lbm.Simulation(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, storage=storage, **kw) as s:
        return s.init(*w.fields()).step(steps).macros()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
def test_batch_twostep_bit_identical_to_single_runs(lbm, storage, collision):
    ws = ragged_batch()
    kw = dict(collision=collision, mrt_rates=(1.4, 1.4, 1.2), beta=0.05)
    with lbm.Batch(ws, storage=storage, **kw) as b:
        for k, w in enumerate(ws):
            b.init(k, *w.fields())
        b.set_twostep(True)
        assert b.twostep
        for n in (2, 16, 3, 16):  # direct passes, a graph of 16, passes + a single step, a graph
            b.step(n)
        b.status()
        for k, w in enumerate(ws):
            ref = single(lbm, w, storage, 37, **kw)
            for a, c in zip(b.macros(k), ref):
                assert np.array_equal(a, c), (w.name, w.nx, w.ny)


def test_batch_twostep_refused_below_8x8(lbm):
    ws = ragged_batch()[:3] + [inputs.Workload("tiny", 7, 30, 0.7, 0, kind="pulse",
                                               params=dict(amplitude=1e-3, half_width=1.0, centres=[(3.0, 9.0)]))]
    with lbm.Batch(ws, storage="f32") as b:
        with pytest.raises(Exception):
            b.set_twostep(True)
        assert not b.twostep
    with lbm.Batch(ragged_batch()[:2], storage="f64") as b:
        with pytest.raises(Exception):
            b.set_twostep(True)


def test_batch_twostep_256_sampled(lbm):
    """The 256-instance workload (sizes 64..1024, pulses and vortices) in
    two-step passes: sampled instances equal their single-domain runs after
    200 steps, and every instance stays finite."""
    ws = inputs.batch_instances()
    with lbm.Batch(ws, storage="f32") as b:
        for k, w in enumerate(ws):
            b.init(k, *w.fields())
        b.set_twostep(True)
        b.step(200)
        b.status()
        for k in (0, 1, 77, 128, 255):
            ref = single(lbm, ws[k], "f32", 200)
            for a, c in zip(b.macros(k), ref):
                assert np.array_equal(a, c), k
        assert all(b.unstable_nodes(k) == 0 for k in range(len(ws)))
