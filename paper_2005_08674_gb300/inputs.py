"""Seeded synthetic workloads (initial density and velocity fields).

This module holds only input generation: random draws and the initial
macroscopic fields of the test flows.  It contains none of the
lattice-Boltzmann or boundary arithmetic, and it is the one module that both
the FP64 oracle's tests and the CUDA path's tests and benchmark take their
inputs from.  It depends on numpy only and never loads the CUDA library.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds and a final xor-shift; a uniform double is
(z >> 11) * 2^-53.  Master seed 20050867; instance k of a batch draws from
state seed + k.

The flows:
  * acoustic pulse: fluid at rest, rho = rho0 (1 + sum_k A exp(-ln2 r_k^2 / b^2)),
    b the half-width at half maximum, u = 0 (the paper's acoustic test, Sec. 6,
    uses a plane wave; a Gaussian pulse exercises every edge and corner);
  * convected vortex (Sec. 7, Eqs. cv_u, cv_v, cv_d, cv_r), with r the distance
    to the centre, Gaussian factor exp(-r^2 / (2 Rc^2)) on the swirl,
    exp(-r^2 / Rc^2) in the density, gas constant (d+2)/d = 2 and
    C_v = (d/2) cs^2 = 1/3 for d = 2;
  * plane wave (Sec. 6, Eqs. pw_p, pw_s) at an angle, condensation
    s = sqrt(e) zeta / (rho0 lam) xi exp(-xi^2 / (2 lam^2)) along xi = x cos(a) + y sin(a),
    rho = rho0 (1 + s), u = cs s along the propagation direction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
MASTER_SEED = 20050867
CS = 1.0 / math.sqrt(3.0)


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1)."""
        return (self.next_u64() >> 11) * (2.0 ** -53)

    def uniform_in(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def int_in(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1))


def _grid(nx: int, ny: int):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    return x, y


def acoustic_pulse(nx: int, ny: int, amplitude, half_width: float, centres,
                   rho0: float = 1.0, background_u=(0.0, 0.0)):
    """Gaussian density pulse(s) on a uniform background.  Returns (rho, ux, uy) [ny][nx]."""
    amps = np.broadcast_to(np.asarray(amplitude, dtype=np.float64), (len(centres),))
    rho = np.ones((ny, nx))
    ln2_b2 = math.log(2.0) / (half_width * half_width)
    xs = np.arange(nx, dtype=np.float64)
    ys = np.arange(ny, dtype=np.float64)
    for a, (cx, cy) in zip(amps, centres):
        gx = np.exp(-ln2_b2 * (xs - cx) ** 2)  # separable Gaussian
        gy = np.exp(-ln2_b2 * (ys - cy) ** 2)
        rho += a * np.outer(gy, gx)
    rho *= rho0
    ux = np.full((ny, nx), float(background_u[0]))
    uy = np.full((ny, nx), float(background_u[1]))
    return rho, ux, uy


def convected_vortex(nx: int, ny: int, u0: float, beta_u0: float, rc: float,
                     x0: float, y0: float):
    """Isentropic (Lamb-Oseen type) vortex in a uniform stream u0 along +x."""
    x, y = _grid(nx, ny)
    dx, dy = x - x0, y - y0
    r2 = dx * dx + dy * dy
    g = np.exp(-r2 / (2.0 * rc * rc))
    ux = u0 - beta_u0 * dy / rc * g
    uy = beta_u0 * dx / rc * g
    d = 2
    gamma_gas = (d + 2) / d
    c_v = d / 2 * CS * CS
    rho = (1.0 - beta_u0 ** 2 / (2.0 * c_v) * np.exp(-r2 / (rc * rc))) ** (1.0 / (gamma_gas - 1.0))
    return rho, ux, uy


def plane_wave(nx: int, ny: int, zeta: float, lam: float, angle_deg: float,
               origin=None, rho0: float = 1.0):
    """Gaussian plane wave travelling along angle_deg, centred on origin."""
    x, y = _grid(nx, ny)
    if origin is None:
        origin = ((nx - 1) / 2.0, (ny - 1) / 2.0)
    a = math.radians(angle_deg)
    xi = (x - origin[0]) * math.cos(a) + (y - origin[1]) * math.sin(a)
    s = math.sqrt(math.e) * zeta / (rho0 * lam) * xi * np.exp(-xi * xi / (2.0 * lam * lam))
    rho = rho0 * (1.0 + s)
    ux = CS * s * math.cos(a)
    uy = CS * s * math.sin(a)
    return rho, ux, uy


@dataclass
class Workload:
    """One named synthetic case: domain, relaxation, far field and initial fields."""
    name: str
    nx: int
    ny: int
    tau: float
    steps: int
    farfield_rho: float = 1.0
    farfield_u: tuple = (0.0, 0.0)
    kind: str = "pulse"
    params: dict = field(default_factory=dict)

    def fields(self):
        p = self.params
        if self.kind == "pulse":
            return acoustic_pulse(self.nx, self.ny, p["amplitude"], p["half_width"], p["centres"])
        if self.kind == "vortex":
            return convected_vortex(self.nx, self.ny, p["u0"], p["beta_u0"], p["rc"], p["x0"], p["y0"])
        if self.kind == "plane":
            return plane_wave(self.nx, self.ny, p["zeta"], p["lam"], p["angle"])
        raise ValueError(self.kind)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def pulse_centres(count: int, lo: float, hi: float, seed: int = MASTER_SEED):
    rng = SplitMix64(seed)
    return [(rng.uniform_in(lo, hi), rng.uniform_in(lo, hi)) for _ in range(count)]


def pulse_200(steps: int = 500) -> Workload:
    """200^2 cells, tau 0.6, one pulse A = 1e-3, HWHM 10, at the domain centre, far field at rest."""
    return Workload("pulse-200", 200, 200, 0.6, steps, kind="pulse",
                    params=dict(amplitude=1e-3, half_width=10.0, centres=[(99.5, 99.5)]))


def vortex_400(steps: int = 4000) -> Workload:
    """400^2 cells, tau 0.505, Ma 0.1 stream along +x, vortex Rc 20 at (100, 200)."""
    u0 = 0.1 * CS
    return Workload("vortex-400", 400, 400, 0.505, steps, farfield_u=(u0, 0.0), kind="vortex",
                    params=dict(u0=u0, beta_u0=0.05 * CS, rc=20.0, x0=100.0, y0=200.0))


def pulse_square(n: int, steps: int = 2000, tau: float = 0.55, half_width: float = 64.0,
                 amplitude: float = 1e-3, margin: int = 256) -> Workload:
    """n^2 cells, four pulses A = 1e-3 at seeded centres in [margin, n - margin]^2."""
    return Workload(f"pulse-{n}", n, n, tau, steps, kind="pulse",
                    params=dict(amplitude=amplitude, half_width=half_width,
                                centres=pulse_centres(4, margin, n - margin)))


def pulse_8192(steps: int = 2000) -> Workload:
    return pulse_square(8192, steps)


def pulse_1024(steps: int = 2000) -> Workload:
    return pulse_square(1024, steps)


def batch_instances(count: int = 256, seed: int = MASTER_SEED, lo: int = 64, hi: int = 1024,
                    steps: int = 1000):
    """Independent instances of uneven sizes: even k a pulse, odd k a convected vortex."""
    out = []
    for k in range(count):
        rng = SplitMix64(seed + k)
        nx = rng.int_in(lo, hi)
        ny = rng.int_in(lo, hi)
        tau = rng.uniform_in(0.51, 0.8)
        m = min(nx, ny)
        if k % 2 == 0:
            amp = 10.0 ** rng.uniform_in(-4.0, -2.0)
            out.append(Workload(f"batch-{k}-pulse", nx, ny, tau, steps, kind="pulse",
                                params=dict(amplitude=amp, half_width=m / 20.0,
                                            centres=[((nx - 1) / 2.0, (ny - 1) / 2.0)])))
        else:
            ma = rng.uniform_in(0.05, 0.15)
            u0 = ma * CS
            out.append(Workload(f"batch-{k}-vortex", nx, ny, tau, steps, farfield_u=(u0, 0.0),
                                kind="vortex",
                                params=dict(u0=u0, beta_u0=0.5 * u0, rc=max(4.0, m / 20.0),
                                            x0=nx / 4.0, y0=ny / 2.0)))
    return out
