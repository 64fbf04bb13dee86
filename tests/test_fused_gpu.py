"""Fused one-launch step (the bulk grid and the NSBC quads in one kernel):
the same device functions as the bulk + NSBC kernel pair, so every run must
be bit-identical to the pair's run of the same case (which the parity tests
pin to the FP64 oracle), for every launch shape, storage, collision model and
edge type; f64 runs are also checked against the oracle directly."""
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


def run(lbm, nx, ny, tau, fields, storage, steps, shape, fused, **kw):
    with lbm.Simulation(nx, ny, tau, storage=storage, **kw) as s:
        s.init(*fields)
        s.set_launch(*shape)
        if fused:
            s.set_fused(True)
            assert s.fused and s.staged == 0
        s.step(steps)
        return s.macros(), s.populations()


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a[0], b[0])) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
@pytest.mark.parametrize("shape", [(128, 1, 0), (64, 4, 3), (512, 2, 1)])
def test_bit_identical_to_kernel_pair(lbm, storage, collision, shape):
    w = inputs.pulse_200()
    kw = dict(collision=collision, mrt_rates=(1.4, 1.4, 1.2), beta=0.05)
    ref = run(lbm, w.nx, w.ny, w.tau, w.fields(), storage, 53, shape, False, **kw)
    got = run(lbm, w.nx, w.ny, w.tau, w.fields(), storage, 53, shape, True, **kw)
    assert same(got, ref)


@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 7), (65, 3), (131, 67), (1031, 9), (128, 128)])
@pytest.mark.parametrize("edges", [None, [("velocity", 0.03, 0.0), "nsbc", "periodic", "periodic"]])
def test_ragged_sizes_and_edges(lbm, nx, ny, edges):
    f = inputs.acoustic_pulse(nx, ny, 1e-3, 2.0, [((nx - 1) / 2, (ny - 1) / 2)])
    kw = dict(edges=edges, grad_order=2) if edges else {}
    ref = run(lbm, nx, ny, 0.6, f, "f32", 37, (128, 1, 0), False, **kw)
    got = run(lbm, nx, ny, 0.6, f, "f32", 37, (128, 1, 0), True, **kw)
    assert same(got, ref)


def test_f64_against_oracle(lbm):
    w = inputs.pulse_200()
    ref = oracle.Oracle(w.nx, w.ny, w.tau, beta=0.1).init(*w.fields()).step(250).macros()
    got, _ = run(lbm, w.nx, w.ny, w.tau, w.fields(), "f64", 250, (256, 1, 0), True, beta=0.1)
    assert max(float(np.abs(a - b).max()) for a, b in zip(got, ref)) <= 1e-12


def test_profiled_steps_count_one_kernel(lbm):
    """Per-launch timing in fused mode: one kernel per step, no NSBC launch."""
    w = inputs.pulse_200()
    with lbm.Simulation(w.nx, w.ny, w.tau, storage="f32") as s:
        s.init(*w.fields())
        s.set_fused(True)
        lbm.lbm_profile(s.h, True)
        s.step(10)
        ms, n, nsbc_ms, n_nsbc = lbm.lbm_profile_read(s.h)
        lbm.lbm_profile(s.h, False)
        assert n == 10 and n_nsbc == 0 and ms > 0
        s.set_staged(3)
        assert not s.fused
        s.set_fused(True)
        s.set_launch(128, 1, 0)
        assert not s.fused and s.staged == 0


def test_autotuned_small_domain_matches_pair(lbm):
    """The autotuner may pick any form for a small domain; the result is the pair's."""
    w = inputs.pulse_200()
    ref = run(lbm, w.nx, w.ny, w.tau, w.fields(), "f32", 64, (128, 1, 0), False)
    with lbm.Simulation(w.nx, w.ny, w.tau, storage="f32") as s:
        s.init(*w.fields())
        s.autotune()
        s.step(64)
        got = s.macros(), s.populations()
    assert same(got, ref)
