"""Single-domain staged step kernel (producer/consumer, tiles staged into
shared memory by bulk copies): it runs the same device arithmetic as the bulk
+ NSBC kernel pair, so every run must be bit-identical to the kernel-pair run
of the same case (which the parity tests pin to the FP64 oracle); f64 runs
are also checked against the oracle directly."""
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


def _fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    rho = 1 + 1e-3 * np.sin(0.5 * x + 0.2 * y + rng.uniform(0, 6))
    ux = 0.03 + 0.02 * np.cos(0.3 * x - 0.4 * y + rng.uniform(0, 6))
    uy = 0.02 * np.sin(0.25 * x + 0.35 * y + rng.uniform(0, 6))
    return rho, ux, uy


def run(lbm, w, storage, steps, stages, fields=None, chunks=None, **kw):
    with lbm.Simulation(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, storage=storage, **kw) as s:
        s.init(*(fields or w.fields()))
        if stages:
            s.set_staged(stages)
        else:
            s.set_launch(128, 1, 0)
        for n in (chunks or [steps]):
            s.step(n)
        s.status()
        return s.macros(), s.populations()


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a[0], b[0])) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
@pytest.mark.parametrize("stages", [3, 4])
def test_bit_identical_to_kernel_pair(lbm, storage, collision, stages):
    w = inputs.pulse_200()
    kw = dict(collision=collision, mrt_rates=(1.4, 1.4, 1.2), beta=0.05)
    ref = run(lbm, w, storage, 101, 0, **kw)
    got = run(lbm, w, storage, 101, stages, **kw)
    assert same(got, ref)


@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 7), (65, 3), (131, 67), (1031, 9), (700, 500), (64, 64)])
def test_ragged_sizes(lbm, nx, ny):
    """Fewer items than blocks, tiles spanning several rows and the padding
    columns, one interior row, a pitch with no padding."""
    w = inputs.Workload("ragged", nx, ny, 0.6, 0, farfield_u=(0.03, 0.0))
    f = _fields(nx, ny, 5)
    ref = run(lbm, w, "f32", 37, 0, fields=f, grad_order=2)
    got = run(lbm, w, "f32", 37, 3, fields=f, grad_order=2, chunks=[1, 16, 20])
    assert same(got, ref)


@pytest.mark.parametrize("edges", [[("velocity", 0.04, 0.01), "nsbc", "periodic", "periodic"],
                                   ["periodic", "periodic", "periodic", "periodic"],
                                   ["nsbc", ("velocity", 0.03, 0.0), "nsbc", ("velocity", 0.02, 0.0)]])
def test_edge_types(lbm, edges):
    w = inputs.Workload("edges", 97, 66, 0.6, 0, farfield_u=(0.03, 0.0))
    f = _fields(97, 66, 21)
    ref = run(lbm, w, "f32", 40, 0, fields=f, beta=0.1, edges=edges)
    got = run(lbm, w, "f32", 40, 3, fields=f, beta=0.1, edges=edges)
    assert same(got, ref)


def test_f64_against_oracle(lbm):
    w = inputs.Workload("small", 45, 31, 0.7, 0, farfield_u=(0.02, 0.01))
    f = _fields(45, 31, 9)
    (got, _) = run(lbm, w, "f64", 300, 3, fields=f, chunks=[1, 299])
    o = oracle.Oracle(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u).init(*f)
    ref = o.step(300).macros()
    err = max(float(np.abs(a - c).max()) for a, c in zip(got, ref))
    assert err <= 1e-12, err


def test_profiled_steps_count_one_kernel(lbm):
    """Per-launch timing in staged mode: one step kernel per step, no NSBC launch."""
    w = inputs.pulse_200()
    with lbm.Simulation(w.nx, w.ny, w.tau, storage="f32") as s:
        s.init(*w.fields())
        s.set_staged(3)
        lbm.lbm_profile(s.h, True)
        s.step(10)
        ms, n, nsbc_ms, n_nsbc = lbm.lbm_profile_read(s.h)
        lbm.lbm_profile(s.h, False)
        assert n == 10 and n_nsbc == 0 and ms > 0
        s.status()
