"""Two-step pass (two time steps per launch, the step in between kept on
chip except on the frame): it runs the same device arithmetic as the single-step
kernels and rounds the intermediate step to the storage type as a single step
stores it, so every run must be bit-identical to the kernel pair's -- over
ragged sizes (one strip and many, bands of rows, narrow last strips), every
storage it serves, BGK and MRT, a far field at rest and in a stream, both
orders of Eq. nes_2, both corner readings, velocity edges, and step counts
that mix graph replays, two-step launches and a last single step.  The f32
path is also checked against the FP64 oracle directly, at 200^2 and at the
bench's 8192^2 with disturbances on every edge and corner."""
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


def _fields(nx, ny, seed, u0=0.0):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    rho = 1 + 1e-3 * np.sin(0.45 * x + 0.3 * y + rng.uniform(0, 6))
    ux = u0 + 0.02 * np.cos(0.3 * x - 0.35 * y + rng.uniform(0, 6))
    uy = 0.02 * np.sin(0.25 * x + 0.4 * y + rng.uniform(0, 6))
    return rho, ux, uy


def _run(lbm, nx, ny, storage, two, steps, fields, farfield_u=(0.0, 0.0), **kw):
    with lbm.Simulation(nx, ny, 0.6, 1.0, farfield_u, storage=storage, **kw) as s:
        s.init(*fields)
        if two:
            s.set_twostep(True)
            assert s.twostep
        else:
            s.set_launch(128, 1, 0)
        for n in (steps if isinstance(steps, (list, tuple)) else [steps]):
            s.step(n)
        s.status()
        return s.populations()


SIZES = [(8, 8), (9, 11), (64, 64), (131, 67), (257, 41), (258, 9), (513, 70), (700, 500), (1031, 9)]


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_bit_identical_to_kernel_pair(lbm, nx, ny, storage):
    f = _fields(nx, ny, nx + 7 * ny)
    ref = _run(lbm, nx, ny, storage, False, 37, f, beta=0.1)
    got = _run(lbm, nx, ny, storage, True, [2, 16, 3, 16], f, beta=0.1)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
@pytest.mark.parametrize("readings", [dict(grad_order=1, corner_mode=0), dict(grad_order=2, corner_mode=1),
                                      dict(grad_order=2, corner_mode=0, kappa=1.0)])
def test_readings_and_mean_flow(lbm, storage, collision, readings):
    nx, ny = 300, 77
    f = _fields(nx, ny, 3, u0=0.03)
    kw = dict(collision=collision, mrt_rates=(1.4, 1.4, 1.2), beta=0.05, farfield_u=(0.03, 0.0), **readings)
    ref = _run(lbm, nx, ny, storage, False, 34, f, **kw)
    got = _run(lbm, nx, ny, storage, True, 34, f, **kw)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("edges", [[("velocity", 0.04, 0.0), "nsbc", "nsbc", "nsbc"],
                                   ["nsbc", ("velocity", 0.03, 0.01), ("velocity", 0.02, 0.0), "nsbc"]])
def test_velocity_edges(lbm, edges):
    nx, ny = 270, 45
    f = _fields(nx, ny, 9, u0=0.03)
    kw = dict(beta=0.1, farfield_u=(0.03, 0.0), edges=edges)
    assert np.array_equal(_run(lbm, nx, ny, "f32", True, 20, f, **kw), _run(lbm, nx, ny, "f32", False, 20, f, **kw))


def test_refused_where_it_does_not_apply(lbm):
    with lbm.Simulation(64, 64, 0.6, storage="f64") as s:
        with pytest.raises(lbm.LbmError):
            s.set_twostep(True)
    with lbm.Simulation(7, 64, 0.6, storage="f32") as s:
        with pytest.raises(lbm.LbmError):
            s.set_twostep(True)
    with lbm.Simulation(64, 64, 0.6, storage="f32", edges=["nsbc", "nsbc", "periodic", "periodic"]) as s:
        with pytest.raises(lbm.LbmError):
            s.set_twostep(True)


def test_pulse_200_against_oracle(lbm):
    w = inputs.pulse_200()
    ref = oracle.Oracle(w.nx, w.ny, w.tau, openmp=True).init(*w.fields()).step(1000).macros()
    with lbm.Simulation(w.nx, w.ny, w.tau, storage="f32") as s:
        got = s.init(*w.fields()).set_twostep(True).step(1000).macros()
    assert max(float(np.abs(a - b).max()) for a, b in zip(got, ref)) <= 1e-6


def test_full_size_8192_edges_and_corners(lbm):
    """The bench's size in the two-step form: narrow pulses next to every edge
    and corner, sampled windows against the oracle at 1e-6."""
    import torch
    import test_parity_gpu as tp
    nx = ny = 8192
    fields = inputs.acoustic_pulse(nx, ny, 1e-3, 8.0, tp.EDGE_CENTRES_8192)
    sim = lbm.Simulation(nx, ny, 0.55, storage="f32")
    sim.init(*fields)
    sim.set_twostep(True)
    sim.step(tp.EDGE_K)
    sim.status()
    worst, weakest = tp._sampled_error(sim, fields, nx, ny, 0.55, tp.EDGE_K, tp.EDGE_SAMPLES_8192, disturbance=True)
    sim.close()
    del fields
    torch.cuda.empty_cache()
    assert weakest >= 1e-5 and worst <= 1e-6, (worst, weakest)
