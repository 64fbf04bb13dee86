"""Brute force on tiny grids: the FP64 oracle against a second, independently
structured restatement of one time step, written here node by node with
plain Python loops from the paper's definitions (Sec. 3 pull streaming
Eq. lbe_0 and BGK Eqs. lbe_1/feq_1; Sec. 4 MRT Eq. mrt_lbe with the moment
basis of Eq. mrt_rm, inverted numerically here; Sec. 5 NSBC Eqs.
nes_0..nes_4) and the readings the oracle states (outward one-sided normal
difference, at a corner either the diagonal normal of length sqrt(2) or the
mean of the two edges' predictions, both equilibria of the mirror at m_c, a
doubly unknown pair set to equilibrium, correction factor kappa, left/right
velocity edges winning at corners).  It shares nothing with
the oracle but the lattice table of Fig. 1 (read from tests/golden).

4x4, 5x3 and 6x5 grids are almost all boundary: every corner and edge rule
is exercised, so a wrong normal, sign, index, pair or dropped term in the
oracle shows up within a few steps.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lattice():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "d2q9_lattice.txt"))
            if l.strip() and not l.startswith("#")]
    c = [(int(r[1]), int(r[2])) for r in rows]
    w = [int(r[3]) / int(r[4]) for r in rows]
    opp = [c.index((-cx, -cy)) for cx, cy in c]
    return c, w, opp


C, W, OPP = _lattice()


def feq(i, rho, ux, uy):
    cu = C[i][0] * ux + C[i][1] * uy
    return W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))


def moments(f):
    rho = sum(f)
    jx = sum(C[i][0] * f[i] for i in range(9))
    jy = sum(C[i][1] * f[i] for i in range(9))
    return rho, jx / rho, jy / rho


def mrt_matrix():
    """Rows of Eq. mrt_rm as polynomials of c: rho, e, eps, jx, qx, jy, qy, pxx, pxy."""
    rows = []
    for poly in (lambda x, y: 1.0,
                 lambda x, y: -4.0 + 3.0 * (x * x + y * y),
                 lambda x, y: 4.0 - 10.5 * (x * x + y * y) + 4.5 * (x * x + y * y) ** 2,
                 lambda x, y: float(x),
                 lambda x, y: (-5.0 + 3.0 * (x * x + y * y)) * x,
                 lambda x, y: float(y),
                 lambda x, y: (-5.0 + 3.0 * (x * x + y * y)) * y,
                 lambda x, y: float(x * x - y * y),
                 lambda x, y: float(x * y)):
        rows.append([poly(cx, cy) for cx, cy in C])
    return np.array(rows)


def brute_step(f, nx, ny, tau, m0, gamma, beta, kappa, order, periodic=(False, False), vel=None, rates=None,
               corner_mode=0):
    """One step on f[(x, y)] = list of 9 populations; returns the new dict."""
    vel = vel or {}

    def predicted(x, y, nxn, nyn):
        """m_c of Eqs. nes_2 and nes_3 at (x, y) for the outward normal (nxn, nyn)."""
        length = math.sqrt(nxn * nxn + nyn * nyn)
        mb = moments(f[x, y])
        m1 = moments(f[x - nxn, y - nyn])
        if order == 1:
            dn = [(mb[k] - m1[k]) / length for k in range(3)]
        else:
            m2 = moments(f[x - 2 * nxn, y - 2 * nyn])
            dn = [(3 * mb[k] - 4 * m1[k] + m2[k]) / (2 * length) for k in range(3)]
        mp = [mb[k] - gamma * dn[k] for k in range(3)]
        return [(1 - beta) * mp[k] + beta * m0[k] for k in range(3)]

    def inside(x, y):
        return 0 <= x < nx and 0 <= y < ny

    def wrap(x, y):
        if periodic[0]:
            x %= nx
        if periodic[1]:
            y %= ny
        return x, y

    # 1. pull streaming; unknown where the source lies outside
    g, unknown = {}, {}
    for y in range(ny):
        for x in range(nx):
            g[x, y], unknown[x, y] = [0.0] * 9, set()
            for i in range(9):
                sx, sy = wrap(x - C[i][0], y - C[i][1])
                if inside(sx, sy):
                    g[x, y][i] = f[sx, sy][i]
                else:
                    unknown[x, y].add(i)
    # 2. NSBC at every edge node with an outward normal
    for (x, y), u in unknown.items():
        nxn = 0 if periodic[0] else (-1 if x == 0 else (1 if x == nx - 1 else 0))
        nyn = 0 if periodic[1] else (-1 if y == 0 else (1 if y == ny - 1 else 0))
        if nxn == 0 and nyn == 0:
            continue
        if corner_mode == 1 and nxn != 0 and nyn != 0:
            # a corner read as the mean of its two edges' predictions
            mc = [(a + b) / 2 for a, b in zip(predicted(x, y, nxn, 0), predicted(x, y, 0, nyn))]
        else:
            mc = predicted(x, y, nxn, nyn)
        side = next((s for s, hit in ((0, x == 0), (1, x == nx - 1), (2, y == 0), (3, y == ny - 1))
                     if hit and s in vel), None)
        if side is not None:
            mc[1], mc[2] = vel[side]
        gb = g[x, y]
        known_before = list(gb)
        for i in u:
            e_i = feq(i, *mc)
            gb[i] = e_i + (known_before[OPP[i]] - feq(OPP[i], *mc)) if OPP[i] not in u else e_i
        rho = sum(gb)
        jx = sum(C[i][0] * gb[i] for i in range(9))
        jy = sum(C[i][1] * gb[i] for i in range(9))
        d_rho, d_jx, d_jy = rho - mc[0], jx - mc[0] * mc[1], jy - mc[0] * mc[2]
        for i in range(9):
            gb[i] -= W[i] * (d_rho + kappa * (C[i][0] * d_jx + C[i][1] * d_jy))
    # 3. collision at every node
    out = {}
    if rates is not None:
        M = mrt_matrix()
        Minv = np.linalg.inv(M)
        S = np.diag(rates)
    for key, gn in g.items():
        rho, ux, uy = moments(gn)
        e = [feq(i, rho, ux, uy) for i in range(9)]
        if rates is None:
            out[key] = [gn[i] - (gn[i] - e[i]) / tau for i in range(9)]
        else:
            out[key] = list(np.array(gn) - Minv @ S @ (M @ (np.array(gn) - np.array(e))))
    return out


def _to_dict(fa):
    _, ny, nx = fa.shape
    return {(x, y): [float(fa[i, y, x]) for i in range(9)] for y in range(ny) for x in range(nx)}


def _to_array(fd, nx, ny):
    a = np.zeros((9, ny, nx))
    for (x, y), v in fd.items():
        a[:, y, x] = v
    return a


def _fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    return (1.0 + 0.01 * rng.standard_normal((ny, nx)), 0.03 + 0.02 * rng.standard_normal((ny, nx)),
            -0.01 + 0.02 * rng.standard_normal((ny, nx)))


CASES = [
    dict(nx=4, ny=4, tau=0.7, gamma=0.6, beta=0.0, kappa=3.0, order=1),
    dict(nx=5, ny=3, tau=0.56, gamma=0.6, beta=0.1, kappa=3.0, order=1),
    dict(nx=6, ny=5, tau=0.9, gamma=0.45, beta=0.2, kappa=1.0, order=2),
    dict(nx=5, ny=6, tau=0.62, gamma=0.6, beta=0.0, kappa=3.0, order=1, periodic=(False, True)),
    dict(nx=6, ny=4, tau=0.75, gamma=0.3, beta=0.0, kappa=3.0, order=2, periodic=(True, False)),
    dict(nx=6, ny=5, tau=0.66, gamma=0.6, beta=0.0, kappa=3.0, order=1, vel={0: (0.05, 0.01), 2: (0.02, 0.0)}),
    dict(nx=5, ny=5, tau=0.6, gamma=0.6, beta=0.05, kappa=3.0, order=1, rates=(1.4, 1.4, 1.2)),
    dict(nx=4, ny=5, tau=0.7, gamma=0.6, beta=0.1, kappa=3.0, order=1, corner_mode=1),
    dict(nx=6, ny=5, tau=0.8, gamma=0.45, beta=0.0, kappa=1.0, order=2, corner_mode=1),
    dict(nx=6, ny=5, tau=0.66, gamma=0.6, beta=0.0, kappa=3.0, order=1, corner_mode=1,
         vel={0: (0.05, 0.01), 2: (0.02, 0.0)}),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['nx']}x{c['ny']}-corner{c.get('corner_mode', 0)}")
def test_oracle_matches_brute_force(case):
    case = dict(case)
    nx, ny, tau = case.pop("nx"), case.pop("ny"), case.pop("tau")
    periodic = case.get("periodic", (False, False))
    vel = case.get("vel")
    mrt = case.get("rates")
    m0 = (1.002, 0.03, -0.01)
    fields = _fields(nx, ny, nx * 10 + ny)
    corner_mode = case.get("corner_mode", 0)
    kw = dict(gamma=case["gamma"], beta=case["beta"], kappa=case["kappa"], grad_order=case["order"],
              periodic=periodic, velocity_edges=vel, corner_mode=corner_mode)
    rates9 = None
    if mrt:
        e, eps, q = mrt
        rates9 = [1.0, e, eps, 1.0, q, 1.0, q, 1.0 / tau, 1.0 / tau]
        kw.update(collision="mrt", mrt_rates=rates9)
    o = oracle.Oracle(nx, ny, tau, m0[0], m0[1:], **kw).init(*fields)
    f = _to_dict(o.get_f())
    for _ in range(6):
        f = brute_step(f, nx, ny, tau, m0, case["gamma"], case["beta"], case["kappa"], case["order"],
                       periodic, vel, rates9, corner_mode)
    got = o.step(6).get_f()
    err = float(np.abs(got - _to_array(f, nx, ny)).max())
    assert err < 1e-13, err
