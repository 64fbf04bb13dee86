"""The seeded input generators shared by the oracle's and the CUDA path's
tests: SplitMix64 against its published test vector (seed 0), the uniform
draw's definition, and the initial fields against their defining properties
(a pulse's half width at half maximum, a vortex's stream at its centre and
its swirl's sense, a plane wave's peak condensation)."""
import math

import numpy as np

from paper_2005_08674_gb300 import inputs


def test_splitmix64_reference_vector():
    g = inputs.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_is_the_top_53_bits():
    a, b = inputs.SplitMix64(7), inputs.SplitMix64(7)
    for _ in range(5):
        z = a.next_u64()
        assert b.uniform() == (z >> 11) * 2.0 ** -53
    u = [inputs.SplitMix64(k).uniform() for k in range(200)]
    assert all(0.0 <= x < 1.0 for x in u)


def test_pulse_half_width_at_half_maximum():
    A, b = 1e-3, 4.0
    rho, ux, uy = inputs.acoustic_pulse(41, 31, A, b, [(20.0, 15.0)])
    assert math.isclose(rho[15, 20] - 1.0, A, rel_tol=1e-12)
    assert math.isclose(rho[15, 24] - 1.0, A / 2, rel_tol=1e-12)   # distance b along x
    assert math.isclose(rho[11, 20] - 1.0, A / 2, rel_tol=1e-12)   # distance b along y
    assert np.all(ux == 0) and np.all(uy == 0)


def test_vortex_stream_and_swirl():
    u0, bu, rc = 0.05, 0.02, 6.0
    rho, ux, uy = inputs.convected_vortex(61, 41, u0, bu, rc, 30.0, 20.0)
    assert math.isclose(ux[20, 30], u0, rel_tol=1e-14) and uy[20, 30] == 0.0
    # counter-clockwise swirl: +y velocity to the right of the centre, -x above it
    assert uy[20, 36] > 0 and ux[26, 30] < u0
    # density dips at the centre and returns to 1 far away
    assert rho[20, 30] < 1.0 and math.isclose(rho[0, 0], 1.0, abs_tol=1e-12)


def test_vortex_swirl_profile_and_radial_balance():
    """The swirl v_theta = beta u0 (r / R_c) exp(-r^2 / 2 R_c^2) reaches
    beta u0 e^(-1/2) at r = R_c; the density satisfies the radial momentum
    balance of a steady vortex to first order, cs^2 d(rho)/dr = v_theta^2 / r
    (central differences along the x axis, within 1 %), and its integral from
    the centre to the far field, cs^2 (1 - rho(0)) = (beta u0)^2 / 2."""
    u0, bu, rc = 0.05, 0.02, 12.0
    rho, ux, uy = inputs.convected_vortex(121, 101, u0, bu, rc, 60.0, 50.0)
    assert math.isclose(uy[50, 72], bu * math.exp(-0.5), rel_tol=1e-13) and ux[50, 72] == u0
    assert math.isclose(ux[62, 60], u0 - bu * math.exp(-0.5), rel_tol=1e-13) and uy[62, 60] == 0.0
    for r in (6, 12, 18):
        v = uy[50, 60 + r]
        drho = (rho[50, 61 + r] - rho[50, 59 + r]) / 2.0
        assert math.isclose(inputs.CS ** 2 * drho, v * v / r, rel_tol=0.01), r
    assert math.isclose(inputs.CS ** 2 * (1.0 - rho[50, 60]), bu * bu / 2.0, rel_tol=1e-12)


def test_plane_wave_peak_and_direction():
    """Along the propagation direction the condensation peaks at zeta / rho0 one
    width lam ahead of the origin (xi exp(-xi^2 / 2 lam^2) peaks at xi = lam),
    and the velocity is cs times the condensation along that direction."""
    zeta, lam = 0.01, 4.0
    rho, ux, uy = inputs.plane_wave(64, 64, zeta, lam, 0.0, origin=(20.0, 10.0))
    assert math.isclose(rho[5, 24] - 1.0, zeta, rel_tol=1e-12)       # xi = x - 20 = lam
    assert math.isclose(rho[5, 16] - 1.0, -zeta, rel_tol=1e-12)      # xi = -lam
    assert float(np.max(rho - 1.0)) <= zeta * (1 + 1e-12)
    assert np.allclose(ux, inputs.CS * (rho - 1.0), rtol=0, atol=1e-15) and np.all(uy == 0)
    rho60, ux60, uy60 = inputs.plane_wave(64, 64, zeta, lam, 60.0)
    s = rho60 - 1.0
    assert np.allclose(ux60, inputs.CS * s * 0.5, atol=1e-15)
    assert np.allclose(uy60, inputs.CS * s * math.sqrt(3) / 2, atol=1e-15)


def test_batch_recipe():
    """256 instances: sides uniform in [64, 1024], tau in [0.51, 0.8], even k a
    centred pulse (amplitude log-uniform in [1e-4, 1e-2], HWHM min side / 20),
    odd k a vortex in a stream of Mach 0.05..0.15 (swirl half the stream speed,
    R_c = max(4, min side / 20), centre (nx / 4, ny / 2)); each instance draws
    from its own SplitMix64 stream, so instance k does not depend on the count."""
    ws = inputs.batch_instances()
    assert len(ws) == 256
    for k, w in enumerate(ws):
        assert 64 <= w.nx <= 1024 and 64 <= w.ny <= 1024
        assert 0.51 <= w.tau < 0.8
        m = min(w.nx, w.ny)
        if k % 2 == 0:
            assert w.kind == "pulse" and w.farfield_u == (0.0, 0.0)
            assert 1e-4 <= w.params["amplitude"] < 1e-2
            assert w.params["half_width"] == m / 20.0
            assert w.params["centres"] == [((w.nx - 1) / 2.0, (w.ny - 1) / 2.0)]
        else:
            u0 = w.params["u0"]
            assert w.kind == "vortex" and w.farfield_u == (u0, 0.0)
            assert 0.05 * inputs.CS <= u0 < 0.15 * inputs.CS
            assert w.params["beta_u0"] == 0.5 * u0 and w.params["rc"] == max(4.0, m / 20.0)
            assert (w.params["x0"], w.params["y0"]) == (w.nx / 4.0, w.ny / 2.0)
    assert len({(w.nx, w.ny) for w in ws}) > 200  # uneven sizes
    few = inputs.batch_instances(count=5)
    assert [(w.nx, w.ny, w.tau) for w in few] == [(w.nx, w.ny, w.tau) for w in ws[:5]]
