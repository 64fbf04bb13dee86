"""Reflection measurements shared by the ablation tests: the reflected-energy
ratio R (oracle/reflection.py) of a run with given NSBC readings, against one
oracle run of the same initial state on a padded domain.

Workloads (seeded, synthetic; the paper's own experiments are figures only):
  pulse-1024    the 8192^2 pulse recipe at 1024^2 (four pulses A = 1e-3,
                HWHM 64, tau 0.55), 2000 steps;
  pulse-256     the same recipe at 256^2 (HWHM 16), 500 steps (CPU-sized);
  vortex-exit   a convected vortex crossing the outflow edge: 200^2, tau
                0.505, MRT rates of Sec. 7, Ma 0.1 stream, swirl 0.05 cs,
                Rc 10, centre (150, 100), 800 steps;
  plane-wave    Sec. 6: 128^2, 60 degrees, zeta 0.01, lambda l/32, MRT
                rates 1.9, tau 0.5001 for tau = 0.5, 240 steps.
Variants are NSBC readings of Sec. 5 where the paper leaves a choice: the
one-sided difference of Eq. nes_2 (grad_order 1 or 2) and the corner reading
(corner_mode 0: diagonal normal; 1: mean of the two edges' m_c).

TEST INFRASTRUCTURE: imports the oracle; the product path never does.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

import oracle
from oracle import reflection as R
from paper_2005_08674_gb300 import inputs


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    tau: float
    steps: int
    every: int
    fields: tuple
    farfield_u: tuple = (0.0, 0.0)
    rates: tuple | None = None  # MRT (omega_e, omega_eps, omega_q), or BGK
    pad_extra: int = 8
    meta: dict = field(default_factory=dict)

    def oracle_kw(self):
        if self.rates is None:
            return {}
        e, eps, q = self.rates
        return dict(collision="mrt", mrt_rates=[1.0, e, eps, 1.0, q, 1.0, q, 1.0 / self.tau, 1.0 / self.tau])

    def gpu_kw(self):
        return {} if self.rates is None else dict(collision="mrt", mrt_rates=self.rates)


def pulse(n: int, steps: int) -> Case:
    w = inputs.pulse_square(n, steps=steps, half_width=n / 16, margin=n // 4)
    return Case(f"pulse-{n}", n, n, w.tau, steps, 20, w.fields(), meta=dict(recipe=w.name))


def vortex_exit() -> Case:
    u0 = 0.1 * inputs.CS
    f0 = inputs.convected_vortex(200, 200, u0, 0.05 * inputs.CS, 10.0, 150.0, 100.0)
    return Case("vortex-exit", 200, 200, 0.505, 800, 20, f0, farfield_u=(u0, 0.0), rates=(1.4, 1.4, 1.2),
                pad_extra=40)


def plane_wave() -> Case:
    n = 128
    return Case("plane-wave", n, n, 0.5001, 240, 20, inputs.plane_wave(n, n, 0.01, n / 32, 60.0),
                rates=(1.9, 1.9, 1.9))


VARIANTS = {"order1_diagonal": dict(grad_order=1, corner_mode=0), "order2_diagonal": dict(grad_order=2, corner_mode=0),
            "order1_mean": dict(grad_order=1, corner_mode=1), "order2_mean": dict(grad_order=2, corner_mode=1)}


def reference(case: Case, openmp: bool = True):
    """Oracle fields on the padded domain, windowed to the test domain, every
    `every` steps, and the initial disturbance energy."""
    u0 = case.farfield_u
    P = R.padding_for(case.steps, math.hypot(*u0), extra=case.pad_extra)
    big = oracle.Oracle(case.nx + 2 * P, case.ny + 2 * P, case.tau, 1.0, u0, openmp=openmp, **case.oracle_kw())
    big.init(*R.embed(case.fields, P, (1.0, u0[0], u0[1])))
    refs = [R.window(big.step(case.every).macros(), P, case.nx, case.ny) for _ in range(case.steps // case.every)]
    z = np.zeros((case.ny, case.nx))
    e0 = R.energy(*case.fields, z + 1.0, z + u0[0], z + u0[1])
    return refs, e0


def r_series(step_and_macros, refs, e0, every):
    return [R.energy(*step_and_macros(every), *ref) / e0 for ref in refs]


def oracle_rmax(case: Case, refs, e0, variant: dict, openmp: bool = True, **extra) -> float:
    o = oracle.Oracle(case.nx, case.ny, case.tau, 1.0, case.farfield_u, openmp=openmp, **case.oracle_kw(),
                      **variant, **extra).init(*case.fields)
    return max(r_series(lambda n: o.step(n).macros(), refs, e0, case.every))


def gpu_rmax(lbm, case: Case, refs, e0, variant: dict, storage: str = "f32", **extra) -> float:
    """R_max of the CUDA path (through the C ABI) with the given readings,
    against the same oracle reference."""
    with lbm.Simulation(case.nx, case.ny, case.tau, 1.0, case.farfield_u, storage=storage, **case.gpu_kw(),
                        **variant, **extra) as s:
        s.init(*case.fields)
        return max(r_series(lambda n: s.step(n).macros(), refs, e0, case.every))
