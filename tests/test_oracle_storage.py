"""The oracle's storage emulation (a test instrument: populations kept as
deviations rounded through a narrower format, all arithmetic in double).

Pinned against independent roundings (numpy's binary16, torch's bfloat16),
then used to show on the oracle alone -- no GPU -- what the CUDA path's
16-bit error figures come from: on a vortex leaving the domain in a Ma 0.1
stream, storing deviations from the far-field equilibrium keeps binary16's
density error an order of magnitude below storing deviations from w_i."""
import numpy as np
import pytest

import oracle
from paper_2005_08674_gb300 import inputs


def _lattice_w():
    return np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_off_is_the_plain_oracle():
    f = inputs.acoustic_pulse(30, 20, 1e-3, 3.0, [(14.5, 9.5)])
    a = oracle.Oracle(30, 20, 0.6).init(*f).step(25).macros()
    b = oracle.Oracle(30, 20, 0.6).storage("f64").init(*f).step(25).macros()
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_rounding_matches_independent_implementations():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    w = _lattice_w()[:, None, None]
    dev = rng.standard_normal((9, 6, 7)) * 10.0 ** rng.uniform(-7, -2, (9, 6, 7))
    f = w + dev
    for fmt in ("f32", "f16", "bf16"):
        o = oracle.Oracle(7, 6, 0.6).set_f(f).storage(fmt, far_field_shift=False)
        got = o.get_f() - w
        v32 = dev.astype(np.float32)
        if fmt == "f32":
            want = v32.astype(np.float64)
        elif fmt == "f16":
            want = (dev * 4096.0).astype(np.float32).astype(np.float16).astype(np.float64) / 4096.0
        else:
            want = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
        # (w + q) - w recovers q exactly: q is far smaller than w and both are exact in double
        assert np.allclose(got, want, rtol=0, atol=1e-17), fmt


def test_far_field_shift_keeps_binary16_accurate_in_a_stream():
    u0 = 0.1 * inputs.CS
    f0 = inputs.convected_vortex(200, 200, u0, 0.05 * inputs.CS, 10.0, 150.0, 100.0)
    rates = [1.0, 1.4, 1.4, 1.0, 1.2, 1.0, 1.2, 1 / 0.505, 1 / 0.505]

    def run(fmt=None, ff=True):
        o = oracle.Oracle(200, 200, 0.505, 1.0, (u0, 0.0), collision="mrt", mrt_rates=rates, openmp=True)
        if fmt:
            o.storage(fmt, ff)
        return o.init(*f0).step(800).macros()

    ref = run()
    err = {k: float(np.abs(run(*k)[0] - ref[0]).max()) for k in (("f16", True), ("f16", False), ("bf16", True))}
    assert err[("f16", True)] <= 5e-5, err
    assert err[("f16", False)] >= 5 * err[("f16", True)], err
    assert err[("bf16", True)] <= 3e-4, err
