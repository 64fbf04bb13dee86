"""Domains with a mean flow store their populations as deviations from the
far-field equilibrium and run the shifted form of every step kernel.  The
three single-domain forms (bulk + NSBC pair, fused one-launch step, staged
producer/consumer step) must give the same bits there too, for every
storage and both collision models; the pair itself is pinned to the FP64
oracle by the parity tests (test_vortex_in_stream)."""
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


def run(lbm, form, storage, collision, fields, nx, ny, u0, steps):
    with lbm.Simulation(nx, ny, 0.6, 1.0, (u0, 0.0), storage=storage, collision=collision,
                        mrt_rates=(1.4, 1.4, 1.2), beta=0.05) as s:
        s.init(*fields)
        if form == "staged":
            s.set_staged(3)
        else:
            s.set_launch(128, 1, 0)
            s.set_fused(form == "fused")
        s.step(steps)
        return s.macros(), s.populations()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
def test_forms_agree_with_a_mean_flow(lbm, storage, collision):
    nx, ny, u0 = 131, 67, 0.05
    f = inputs.convected_vortex(nx, ny, u0, 0.02, 8.0, 40.0, 33.0)
    ref = run(lbm, "pair", storage, collision, f, nx, ny, u0, 37)
    for form in ("fused", "staged"):
        got = run(lbm, form, storage, collision, f, nx, ny, u0, 37)
        assert all(np.array_equal(a, b) for a, b in zip(got[0], ref[0])), form
        assert np.array_equal(got[1], ref[1]), form
