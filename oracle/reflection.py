"""Reflection measure for open-boundary runs (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper judges reflections from figures only (close to zero for the
acoustic test of Sec. 6, complete absorption for the vortex of Sec. 7), so the
number used here is defined for this project:

  E[a, b] = sum over the window of  ( cs^2 (rho_a - rho_b)^2 / rho0 + rho0 |u_a - u_b|^2 ) / 2

is the linear acoustic energy of the difference between two fields.  A run
on the test domain D is compared with a run of the same initial state on an
extended domain D' = D padded by P nodes on every side (padding at the far
field) that is large enough that nothing reflected at the edge of D' can
re-enter D by the final time.  Then R(t) = E[test(t), ref(t)] / E[ref(0), m0],
and R_max = max over sampled t.

The measure itself is pinned by its closed forms (zero for equal fields,
symmetry, the one-node disturbance, padding and windowing as inverses).  The
values of R_max it gives for the paper's experiments are parity unpinned
against the paper, which prints no reflection numbers.
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0


def energy(rho_a, ux_a, uy_a, rho_b, ux_b, uy_b, rho0: float = 1.0) -> float:
    d_rho = np.asarray(rho_a, np.float64) - rho_b
    d_ux = np.asarray(ux_a, np.float64) - ux_b
    d_uy = np.asarray(uy_a, np.float64) - uy_b
    return float(0.5 * np.sum(CS2 * d_rho * d_rho / rho0 + rho0 * (d_ux * d_ux + d_uy * d_uy)))


def padding_for(steps: int, farfield_speed: float = 0.0, extra: int = 8) -> int:
    """Padding P such that a disturbance leaving D at time 0 and reflected at the
    edge of D' cannot come back into D within `steps` (round trip 2P at speed
    cs + |u|)."""
    return int(math.ceil((1.0 / math.sqrt(3.0) + abs(farfield_speed)) * steps / 2.0)) + extra


def embed(fields, pad: int, farfield):
    """Embed (rho, ux, uy) in a domain padded by `pad` on every side with the far field."""
    rho, ux, uy = fields
    ny, nx = rho.shape
    out = []
    for a, v in zip((rho, ux, uy), farfield):
        b = np.full((ny + 2 * pad, nx + 2 * pad), float(v))
        b[pad:pad + ny, pad:pad + nx] = a
        out.append(b)
    return tuple(out)


def window(fields, pad: int, nx: int, ny: int):
    return tuple(np.ascontiguousarray(a[pad:pad + ny, pad:pad + nx]) for a in fields)
