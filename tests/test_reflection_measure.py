"""The reflection measure (oracle/reflection.py) against what defines it:
E is the acoustic energy of a difference (zero for equal fields, symmetric,
the closed form on a single-node disturbance), and the padding P is wide
enough that the padded reference seen through the test window is, to
round-off, what an even wider padding gives over the run -- while a padding
well below the round-trip distance is not."""
import math

import numpy as np

import oracle
from oracle import reflection as R
from paper_2005_08674_gb300 import inputs


def test_energy_definition():
    rng = np.random.default_rng(1)
    a = [1 + 1e-3 * rng.standard_normal((5, 6)), 1e-3 * rng.standard_normal((5, 6)), 1e-3 * rng.standard_normal((5, 6))]
    b = [1 + 1e-3 * rng.standard_normal((5, 6)), 1e-3 * rng.standard_normal((5, 6)), 1e-3 * rng.standard_normal((5, 6))]
    assert R.energy(*a, *a) == 0.0
    assert R.energy(*a, *b) == R.energy(*b, *a)
    # one node: drho = 2e-3, du = (3e-3, -4e-3), rho0 = 1.25
    z = np.zeros((3, 3))
    ra, ua, va = z + 1.25, z.copy(), z.copy()
    ra[1, 1] += 2e-3
    ua[1, 1] = 3e-3
    va[1, 1] = -4e-3
    want = 0.5 * ((1.0 / 3.0) * (2e-3) ** 2 / 1.25 + 1.25 * ((3e-3) ** 2 + (4e-3) ** 2))
    assert math.isclose(R.energy(ra, ua, va, z + 1.25, z, z, rho0=1.25), want, rel_tol=1e-15)


def test_embed_and_window_are_inverse():
    f = inputs.acoustic_pulse(7, 5, 1e-3, 2.0, [(3.0, 2.0)])
    big = R.embed(f, 4, (1.0, 0.02, 0.0))
    assert big[0].shape == (13, 15)
    assert np.all(big[1][:4] == 0.02) and np.all(big[0][:, :4] == 1.0)
    back = R.window(big, 4, 7, 5)
    assert all(np.array_equal(x, y) for x, y in zip(back, f))


def _windows(n, steps, pad, tau=0.6):
    f = inputs.acoustic_pulse(n, n, 1e-3, 3.0, [((n - 1) / 2, (n - 1) / 2)])
    o = oracle.Oracle(n + 2 * pad, n + 2 * pad, tau).init(*R.embed(f, pad, (1.0, 0.0, 0.0)))
    out = []
    for _ in range(steps // 10):
        out.append(R.window(o.step(10).macros(), pad, n, n))
    return out


def test_padding_keeps_the_edge_out_of_the_window():
    """Through the window, the reference with padding P equals one with P + 30
    to round-off over the whole run (the lattice's own precursors, which move
    at one node per step rather than c_s, stay at the 1e-15 level); a padding of
    2 nodes lets the reference's edge reflections in at a level that R would
    see (energy ratio above 1e-6 of the initial disturbance)."""
    n, steps = 40, 60
    P = R.padding_for(steps)
    assert P == math.ceil(steps / math.sqrt(3.0) / 2.0) + 8
    f = inputs.acoustic_pulse(n, n, 1e-3, 3.0, [((n - 1) / 2, (n - 1) / 2)])
    z = np.zeros_like(f[0])
    e0 = R.energy(*f, np.ones_like(z), z, z)
    near = _windows(n, steps, P)
    far = _windows(n, steps, P + 30)
    for a, b in zip(near, far):
        assert max(float(np.abs(x - y).max()) for x, y in zip(a, b)) <= 1e-12
        assert R.energy(*a, *b) / e0 <= 1e-15
    short = _windows(n, steps, 2)
    assert max(R.energy(*a, *b) / e0 for a, b in zip(short, far)) > 1e-6
