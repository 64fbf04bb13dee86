"""Batched mode: many instances of uneven sizes stepped by one persistent
launch per step.  Each instance must be bit-identical to the same instance
run alone through the single-domain path (same storage and collision), and
the f64 batch must match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2005_08674_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import lbm as m
    return m


def small_batch():
    ws = inputs.batch_instances(count=8, lo=3, hi=200)
    ws += [inputs.Workload("tiny", 3, 3, 0.7, 0, kind="pulse",
                           params=dict(amplitude=1e-3, half_width=1.0, centres=[(1.0, 1.0)])),
           inputs.Workload("thin", 517, 4, 0.6, 0, farfield_u=(0.02, 0.0), kind="pulse",
                           params=dict(amplitude=1e-3, half_width=3.0, centres=[(100.0, 1.5)]))]
    return ws


def single(lbm, w, storage, steps, **kw):
    with lbm.Simulation(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, storage=storage, **kw) as s:
        return s.init(*w.fields()).step(steps).macros()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
@pytest.mark.parametrize("launch", [None, (128, 1, -1, 0, 0, 0)])
def test_batch_bit_identical_to_single_runs(lbm, storage, collision, launch):
    """Default launch (the producer/consumer form) and the register path."""
    ws = small_batch()
    kw = dict(collision=collision, mrt_rates=(1.4, 1.4, 1.2), beta=0.05)
    with lbm.Batch(ws, storage=storage, **kw) as b:
        for k, w in enumerate(ws):
            b.init(k, *w.fields())
        if launch:
            b.set_launch(*launch)
        b.step(37)  # two graph replays of 16 and five direct launches
        for k, w in enumerate(ws):
            ref = single(lbm, w, storage, 37, **kw)
            got = b.macros(k)
            for a, c in zip(got, ref):
                assert np.array_equal(a, c), (w.name, w.nx, w.ny)


def test_batch_f64_matches_oracle(lbm):
    ws = small_batch()[:5]
    with lbm.Batch(ws, storage="f64", beta=0.1) as b:
        for k, w in enumerate(ws):
            b.init(k, *w.fields())
        b.step(60)
        for k, w in enumerate(ws):
            o = oracle.Oracle(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, beta=0.1).init(*w.fields())
            ref = o.step(60).macros()
            err = max(float(np.abs(a - c).max()) for a, c in zip(b.macros(k), ref))
            assert err <= 1e-12, (w.name, err)


@pytest.mark.parametrize("shape", [(64, 1, 0, 0, 0, 0), (128, 2, 0, 1, 1, 0), (256, 4, 152, 0, 0, 0), (64, 4, 7, 64, 1, 0), (128, 1, 0, 0, 1, 128), (128, 1, 0, 0, 1, 256), (256, 1, 0, 0, 1, 256),
                                   (128, 4, -1, 1, 0, 0), (256, 1, -1, 0, 1, 0),
                                   (128, 3, 0, 0, 0, 128), (128, 4, 0, 2, 0, 128), (128, 3, 5, 2, 0, 128)])
def test_batch_launch_shapes_agree(lbm, shape):
    """Every tile shape, grid size (one block per item, persistent waves, a
    grid far smaller than the work list) and prefetch gives the same bits."""
    ws = small_batch()
    outs = []
    for sh in [(128, 1, -1, 0, 0, 0), shape]:
        with lbm.Batch(ws, storage="f32") as b:
            for k, w in enumerate(ws):
                b.init(k, *w.fields())
            b.set_launch(*sh)
            b.step(21)
            outs.append([b.macros(k) for k in range(len(ws))])
    for x, y in zip(*outs):
        for a, c in zip(x, y):
            assert np.array_equal(a, c)


def test_full_batch_256_sampled(lbm):
    """The 256-instance workload (sizes 64..1024, pulses and vortices) after
    autotuning: sampled instances equal their single-domain runs, and every
    instance stays finite over 200 steps."""
    ws = inputs.batch_instances()
    with lbm.Batch(ws, storage="f32") as b:
        for k, w in enumerate(ws):
            b.init(k, *w.fields())
        b.autotune()
        b.step(200)
        for k in (0, 1, 77, 128, 255):
            ref = single(lbm, ws[k], "f32", 200)
            for a, c in zip(b.macros(k), ref):
                assert np.array_equal(a, c), k
        assert all(b.unstable_nodes(k) == 0 for k in range(len(ws)))


def test_batch_with_edge_types_bit_identical(lbm):
    ws = small_batch()[:6]
    edges = [("velocity", 0.03, 0.0), "nsbc", "periodic", "periodic"]
    kw = dict(collision="mrt", mrt_rates=(1.4, 1.4, 1.2), edges=edges)
    with lbm.Batch(ws, storage="f32", **kw) as b:
        for k, w in enumerate(ws):
            b.init(k, *w.fields())
        b.step(33)
        for k, w in enumerate(ws):
            ref = single(lbm, w, "f32", 33, **kw)
            for a, c in zip(b.macros(k), ref):
                assert np.array_equal(a, c), w.name


def test_bounded_wait_gives_up_and_context_survives(lbm):
    """Failure detection without a fault: a wait on a barrier nothing arrives on
    gives up after its budget (~1 ms here) and reports LBM_ETIMEOUT; the context
    stays usable and a staged-tile batch then steps normally with a clean status."""
    assert lbm.lbm_wait_selftest(2_000_000) == lbm.LBM_ETIMEOUT
    ws = small_batch()[:4]
    with lbm.Batch(ws, storage="f32") as b:
        for k, w in enumerate(ws):
            b.init(k, *w.fields())
        b.set_launch(128, 1, 0, 0, 0, 128)
        b.step(20)
        b.status()
        ref = single(lbm, ws[0], "f32", 20)
        for a, c in zip(b.macros(0), ref):
            assert np.array_equal(a, c)
