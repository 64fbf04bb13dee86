"""The second corner reading on the GPU (Sec. 5 says nothing about corners):
with corner_mode = 1 a corner node gets the mean of the two blended states
m_c (Eqs. nes_2, nes_3) of the edges meeting there.  The CUDA path is checked
against the FP64 oracle (which the brute-force restatement and the corner-state
pin fix) at 1e-12 in f64 and 1e-6 in f32, and every launch form (kernel pair,
fused, staged, batched) must give the same bits as the kernel pair."""
import numpy as np
import pytest

import oracle
from paper_2005_08674_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-6}


@pytest.fixture(scope="module")
def lbm():
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import lbm as m
    return m


def _fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    rho = 1 + 1e-3 * np.sin(0.6 * x + 0.25 * y + rng.uniform(0, 6))
    ux = 0.02 + 0.02 * np.cos(0.35 * x - 0.45 * y + rng.uniform(0, 6))
    uy = -0.01 + 0.02 * np.sin(0.3 * x + 0.2 * y + rng.uniform(0, 6))
    return rho, ux, uy


def _max_err(a, b):
    return max(float(np.abs(x - y).max()) for x, y in zip(a, b))


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 3), (5, 7), (33, 17), (131, 67)])
@pytest.mark.parametrize("order", [1, 2])
def test_corner_mean_matches_oracle(lbm, storage, nx, ny, order):
    if order == 2 and min(nx, ny) < 3:
        pytest.skip("no second interior point")
    fields = _fields(nx, ny, nx * 100 + ny)
    kw = dict(gamma=0.55, beta=0.2, grad_order=order, corner_mode=1)
    ref = oracle.Oracle(nx, ny, 0.58, 1.0, (0.01, -0.005), **kw).init(*fields).step(37).macros()
    with lbm.Simulation(nx, ny, 0.58, 1.0, (0.01, -0.005), storage=storage, **kw) as s:
        got = s.init(*fields).step(37).macros()
    assert _max_err(got, ref) <= TOL[storage]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_corner_mean_pulse_200(lbm, storage):
    """pulse-200 for 1000 steps: the wave crosses all four corners."""
    w = inputs.pulse_200()
    ref = oracle.Oracle(w.nx, w.ny, w.tau, openmp=True, corner_mode=1).init(*w.fields()).step(1000).macros()
    with lbm.Simulation(w.nx, w.ny, w.tau, storage=storage, corner_mode=1) as s:
        got = s.init(*w.fields()).step(1000).macros()
    assert _max_err(got, ref) <= TOL[storage]


def test_corner_mean_with_velocity_edges(lbm):
    """A velocity edge meeting NSBC edges and another velocity edge at corners."""
    nx, ny = 41, 29
    fields = _fields(nx, ny, 3)
    ref = oracle.Oracle(nx, ny, 0.62, 1.0, (0.03, 0.0), beta=0.1, corner_mode=1,
                        velocity_edges={0: (0.04, 0.0), 2: (0.02, 0.0)}).init(*fields).step(40).macros()
    with lbm.Simulation(nx, ny, 0.62, 1.0, (0.03, 0.0), storage="f64", beta=0.1, corner_mode=1,
                        edges=[("velocity", 0.04, 0.0), "nsbc", ("velocity", 0.02, 0.0), "nsbc"]) as s:
        got = s.init(*fields).step(40).macros()
    assert _max_err(got, ref) <= 1e-12


def _run(lbm, nx, ny, storage, form, fields, steps=41, **kw):
    with lbm.Simulation(nx, ny, 0.6, 1.0, (0.02, 0.0), storage=storage, corner_mode=1, grad_order=2, **kw) as s:
        s.init(*fields)
        if form == "pair":
            s.set_launch(128, 1, 0)
        elif form == "fused":
            s.set_launch(128, 1, 0)
            s.set_fused(True)
        else:
            s.set_staged(int(form[-1]))
        s.step(steps)
        s.status()
        return s.populations()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("form", ["fused", "staged3", "staged4"])
def test_forms_bit_identical(lbm, storage, form):
    nx, ny = 131, 67
    fields = _fields(nx, ny, 8)
    ref = _run(lbm, nx, ny, storage, "pair", fields, collision="mrt", mrt_rates=(1.4, 1.4, 1.2))
    got = _run(lbm, nx, ny, storage, form, fields, collision="mrt", mrt_rates=(1.4, 1.4, 1.2))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_bit_identical_to_single_runs(lbm, storage):
    ws = [inputs.Workload(f"c{k}", nx, ny, tau, 0, farfield_u=u)
          for k, (nx, ny, tau, u) in enumerate([(64, 80, 0.6, (0.0, 0.0)), (97, 66, 0.55, (0.03, 0.0)),
                                                (3, 3, 0.7, (0.0, 0.01)), (200, 31, 0.52, (0.02, -0.01))])]
    fields = [_fields(w.nx, w.ny, 40 + k) for k, w in enumerate(ws)]
    with lbm.Batch(ws, storage=storage, corner_mode=1, beta=0.05) as b:
        for k, f in enumerate(fields):
            b.init(k, *f)
        b.step(33)
        b.status()
        got = [b.macros(k) for k in range(len(ws))]
    for w, f, g in zip(ws, fields, got):
        with lbm.Simulation(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, storage=storage, corner_mode=1,
                            beta=0.05) as s:
            s.set_launch(128, 1, 0)
            ref = s.init(*f).step(33).macros()
        assert all(np.array_equal(x, y) for x, y in zip(g, ref))
