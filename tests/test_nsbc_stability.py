"""Linear stability of the NSBC in a mean stream (oracle, FP64).  A uniform
stream equal to the far field (Ma 0.1 along +x, 200^2, tau 0.505) is an exact
fixed point of the scheme (Sec. 5: zero gradients, m_c = m0); these tests
seed it with white noise of 1e-12 and watch the noise:

  * MRT with the rates of Sec. 7 and the first-order difference of Eq. nes_2
    (the configuration of the paper's vortex test): the noise does not grow;
  * the same with the second-order one-sided difference: it grows about 75x
    per 100 steps on the inflow edge (x = 0, 1) -- the second-order reading
    of Eq. nes_2 is unstable where the stream enters;
  * BGK with the first-order difference at this viscosity (nu = 0.0017): it
    grows about 25x per 100 steps next to the outflow edge -- the blow-up of
    the 400^2 BGK vortex workload is this instability, not the vortex.

Any mistake that changed the boundary operator (a sign, a stencil weight, a
normal) would move or remove these growth rates.
"""
import numpy as np
import pytest

import oracle
from paper_2005_08674_gb300 import inputs

N, TAU = 200, 0.505
U0 = 0.1 * inputs.CS
MRT = [1.0, 1.4, 1.4, 1.0, 1.2, 1.0, 1.2, 1.0 / TAU, 1.0 / TAU]


def noisy_stream(seed=1, amp=1e-12):
    rng = np.random.default_rng(seed)
    return (1 + amp * rng.standard_normal((N, N)), U0 + amp * rng.standard_normal((N, N)),
            amp * rng.standard_normal((N, N)))


def amplitude(fields):
    rho, ux, uy = fields
    d = np.maximum(np.maximum(np.abs(rho - 1), np.abs(ux - U0)), np.abs(uy))
    d = np.nan_to_num(d, nan=np.inf)
    j = np.unravel_index(np.argmax(d), d.shape)
    return float(d.max()), int(j[1])  # amplitude, x of its largest value


def run(steps, **kw):
    o = oracle.Oracle(N, N, TAU, 1.0, (U0, 0.0), openmp=True, **kw).init(*noisy_stream())
    return amplitude(o.step(steps).macros())


def test_mrt_first_order_is_stable():
    a, _ = run(800, collision="mrt", mrt_rates=MRT, grad_order=1)
    assert a < 1e-11


def test_mrt_second_order_is_unstable_on_the_inflow_edge():
    a4, x4 = run(400, collision="mrt", mrt_rates=MRT, grad_order=2)
    a5, x5 = run(500, collision="mrt", mrt_rates=MRT, grad_order=2)
    assert a4 > 1e-7 and 30 < a5 / a4 < 200, (a4, a5)
    assert x4 <= 1 and x5 <= 1


@pytest.mark.parametrize("corner", [0, 1])
def test_bgk_first_order_is_unstable_next_to_the_outflow_edge(corner):
    a5, x5 = run(500, grad_order=1, corner_mode=corner)
    a6, x6 = run(600, grad_order=1, corner_mode=corner)
    assert a5 > 1e-7 and 10 < a6 / a5 < 60, (a5, a6)
    assert x5 >= N - 3 and x6 >= N - 3
