"""lbm_reduce_noalloc: the reduction for callers that cannot allocate device
memory when they need it (e.g. a hook running inside another framework's step
loop, where that framework owns the device memory).  Called through the C ABI,
it must give the same sums as lbm_reduce, call after call, although its
partial sums live in one fixed array that every call on the device shares.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2005_08674_gb300 import inputs


@pytest.fixture(scope="module")
def lbm():
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import lbm as m
    return m


def _close(a, b):
    for x, y in zip(a, b):
        assert abs(x - y) <= 1e-12 * max(abs(x), abs(y)) + 1e-300, (a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_noalloc_matches_reduce_on_consecutive_calls(lbm, storage):
    import torch
    w = inputs.pulse_square(600, margin=120, half_width=30.0)
    big = 700  # a padded reference domain: node (0, 0) of the test run sits at (50, 50)
    ref_w = inputs.pulse_square(big, margin=170, half_width=30.0)
    sim = lbm.Simulation(w.nx, w.ny - 37, w.tau, storage=storage)
    rho, ux, uy = (a[:w.ny - 37] for a in w.fields())
    sim.init(rho, ux, uy)
    ref_sim = lbm.Simulation(big, big, ref_w.tau, storage="f64").init(*ref_w.fields())
    seen = []
    for k in range(2):  # two calls in a row, the state moving on between them
        sim.step(40 + 13 * k)
        ref_sim.step(40 + 13 * k)
        a = lbm.lbm_reduce(sim.h)
        b = lbm.lbm_reduce_noalloc(sim.h)
        _close(a, b)
        mac = ref_sim.macros_device()
        win = mac[:, 50:, 50:]
        args = (win[0].data_ptr(), win[1].data_ptr(), win[2].data_ptr(), big)
        a = lbm.lbm_reduce(sim.h, *args)
        b = lbm.lbm_reduce_noalloc(sim.h, *args)
        _close(a, b)
        seen.append(b)
        torch.cuda.synchronize()
    assert seen[0] != seen[1]  # the second call did not just return the first call's sums
    sim.close()
    ref_sim.close()


@pytest.mark.gpu
def test_noalloc_on_a_small_domain_after_a_large_one(lbm):
    """Stale partials of an earlier, larger call are never read."""
    fields = [a[:1500] for a in inputs.pulse_square(2048, margin=300).fields()]
    big = lbm.Simulation(2048, 1500, 0.6, storage="f32").init(*fields)
    _ = lbm.lbm_reduce_noalloc(big.h)
    small_fields = inputs.acoustic_pulse(50, 40, 1e-3, 5.0, [(20.0, 20.0)])
    small = lbm.Simulation(50, 40, 0.6, storage="f64").init(*small_fields).step(7)
    _close(lbm.lbm_reduce(small.h), lbm.lbm_reduce_noalloc(small.h))
    big.close()
    small.close()


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny", [(65536, 5), (8193, 8192)])
def test_noalloc_wide_and_large_domains(lbm, nx, ny):
    """A domain wider than it is tall (65,536 x 5: five blocks, one per row)
    and one with more rows than the array has block slots (8193 x 8192: 4096
    blocks, two rows each) give lbm_reduce's sums."""
    import torch
    fields = inputs.acoustic_pulse(nx, ny, 1e-3, 3.0, [(nx / 3, ny / 2)])
    with lbm.Simulation(nx, ny, 0.6, storage="f32") as sim:
        sim.init(*fields).step(3)
        _close(lbm.lbm_reduce(sim.h), lbm.lbm_reduce_noalloc(sim.h))
    del fields
    torch.cuda.empty_cache()
