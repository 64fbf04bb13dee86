"""16-bit shifted storage (f16, bf16) against the FP64 oracle.

Workload: the 8192^2 pulse recipe at 1024^2 (four pulses A = 1e-3, half-width
64, centres in [256, 768]^2, tau 0.55), 2000 steps.  Bars: density error
<= 1e-4 and a change of the reflection coefficient R_max of at most 1 %
relative to the oracle's.  R(t) = E[run(t), ref(t)] / E[ref(0), m0] with E the
acoustic energy of the difference and ref an oracle run on the domain padded
by P nodes of far field on every side, so that nothing comes back from its
edge within the run; R_max over samples every 20 steps.  The f32 path is
measured the same way, and a convected vortex crossing the outflow edge
(200^2, MRT, 800 steps) is measured likewise with its mean flow through the
edges.  If LBM_RESULTS_DIR is
set, the figures are written there as JSON.

f32 and f16 are held to the bars.  bf16 does not meet them: on both flows its
8 significant bits alone -- the oracle with only its stored populations
rounded through bfloat16, all arithmetic in double -- already miss a bar
(R_max by 1.2 % on the pulse, density by 1.4e-4 on the vortex).  Its tests
record whether the bars are met (they are not) and hold the GPU to what the
format loses: density error and R_max change within 3x of that storage
emulation's.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import reflection as R
from paper_2005_08674_gb300 import inputs

pytestmark = pytest.mark.gpu

STEPS, EVERY = 2000, 20


@pytest.fixture(scope="module")
def lbm():
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import lbm as m
    return m


@pytest.fixture(scope="module")
def reference():
    """Oracle on the test domain and on the padded domain: fields every EVERY steps."""
    w = inputs.pulse_1024()
    f0 = w.fields()
    P = R.padding_for(STEPS)
    big = oracle.Oracle(w.nx + 2 * P, w.ny + 2 * P, w.tau, openmp=True).init(*R.embed(f0, P, (1.0, 0.0, 0.0)))
    test = oracle.Oracle(w.nx, w.ny, w.tau, openmp=True).init(*f0)
    z = np.zeros_like(f0[0])
    e0 = R.energy(*f0, np.ones_like(z), z, z)
    # what each 16-bit format alone loses: the oracle with its stored
    # populations rounded through that format, arithmetic in double
    emul = {fmt: oracle.Oracle(w.nx, w.ny, w.tau, openmp=True).storage(fmt, True).init(*f0)
            for fmt in ("f16", "bf16")}
    refs, rs = [], []
    rs_emul = {fmt: [] for fmt in emul}
    for _ in range(STEPS // EVERY):
        big.step(EVERY)
        test.step(EVERY)
        ref = R.window(big.macros(), P, w.nx, w.ny)
        refs.append(ref)
        rs.append(R.energy(*test.macros(), *ref) / e0)
        for fmt, o in emul.items():
            rs_emul[fmt].append(R.energy(*o.step(EVERY).macros(), *ref) / e0)
    final = test.macros()
    emulated = {fmt: dict(drho=float(np.abs(o.macros()[0] - final[0]).max()),
                          r_change=abs(max(rs_emul[fmt]) - max(rs)) / max(rs)) for fmt, o in emul.items()}
    return dict(w=w, f0=f0, refs=refs, e0=e0, r_max=max(rs), final=final, emulated=emulated)


def _check(res, storage, rho_tol, r_tol, emulated):
    """f32 / f16: the bars.  bf16: within 3x of what the format alone loses
    (its storage emulation), with the bar verdict recorded."""
    res["meets_bar"] = bool(res["max_abs_drho"] <= rho_tol and res["r_change"] <= r_tol)
    out = os.environ.get("LBM_RESULTS_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, f"{res['case']}_{storage}.json"), "w") as f:
            json.dump(res, f)
    print(res)
    if storage == "bf16":
        e = emulated["bf16"]
        assert res["max_abs_drho"] <= 3.0 * e["drho"], res
        assert res["r_change"] <= 3.0 * max(e["r_change"], 1e-3), res
    else:
        assert res["meets_bar"], res
        if storage in emulated:
            assert res["max_abs_drho"] <= 3.0 * emulated[storage]["drho"], res


# Bars: density error 1e-4 and reflection change 1 % for the 16-bit forms
# (f32: 1e-6).  bf16 misses the R_max bar here (emulated: 1.2 %).
@pytest.mark.parametrize("storage,rho_tol,r_tol", [("f16", 1e-4, 0.01), ("bf16", 1e-4, 0.01), ("f32", 1e-6, 0.01)])
def test_storage_error_and_reflection(lbm, reference, storage, rho_tol, r_tol):
    w = reference["w"]
    sim = lbm.Simulation(w.nx, w.ny, w.tau, storage=storage).init(*reference["f0"])
    rs = []
    for ref in reference["refs"]:
        sim.step(EVERY)
        rs.append(R.energy(*sim.macros(), *ref) / reference["e0"])
    got = sim.macros()
    sim.close()
    ref_final = reference["final"]
    d_rho = float(np.abs(got[0] - ref_final[0]).max())
    d_u = float(max(np.abs(got[1] - ref_final[1]).max(), np.abs(got[2] - ref_final[2]).max()))
    r_max = max(rs)
    change = abs(r_max - reference["r_max"]) / reference["r_max"]
    emulated = reference["emulated"]
    res = dict(case="mixed", storage=storage, workload="pulse-1024, 2000 steps", max_abs_drho=d_rho,
               max_abs_du=d_u, r_max=r_max, r_max_oracle=reference["r_max"], r_change=change,
               oracle_storage_emulation=emulated.get(storage))
    _check(res, storage, rho_tol, r_tol, emulated)


# A convected vortex leaving the domain (Sec. 7's situation): 200^2, tau 0.505,
# Ma 0.1 stream along +x, swirl 0.05 cs, Rc 10, centre (150, 100), MRT rates
# of Sec. 7; in 800 steps the centre moves to x = 196, so the vortex crosses
# the outflow edge.  (On the 400^2 vortex workload the vortex is still far from
# every edge after 1000 steps: R there is ~1e-9, below the f32 rounding noise,
# and says nothing about the boundary.)  The padded oracle reference is
# 788^2 nodes.
V_N, V_STEPS, V_EVERY = 200, 800, 20
VORTEX_RATES = (1.4, 1.4, 1.2)
V_TAU = 0.505


@pytest.fixture(scope="module")
def vortex_reference():
    u0 = 0.1 * inputs.CS
    f0 = inputs.convected_vortex(V_N, V_N, u0, 0.05 * inputs.CS, 10.0, 150.0, 100.0)
    rates = [1.0, VORTEX_RATES[0], VORTEX_RATES[1], 1.0, VORTEX_RATES[2], 1.0, VORTEX_RATES[2],
             1.0 / V_TAU, 1.0 / V_TAU]
    P = R.padding_for(V_STEPS, u0, extra=4 * 10)
    kw = dict(collision="mrt", mrt_rates=rates, openmp=True)
    big = oracle.Oracle(V_N + 2 * P, V_N + 2 * P, V_TAU, 1.0, (u0, 0.0), **kw)
    big.init(*R.embed(f0, P, (1.0, u0, 0.0)))
    test = oracle.Oracle(V_N, V_N, V_TAU, 1.0, (u0, 0.0), **kw).init(*f0)
    z = np.zeros_like(f0[0])
    e0 = R.energy(*f0, np.ones_like(z), z + u0, z)
    refs, rs = [], []
    for _ in range(V_STEPS // V_EVERY):
        big.step(V_EVERY)
        test.step(V_EVERY)
        ref = R.window(big.macros(), P, V_N, V_N)
        refs.append(ref)
        rs.append(R.energy(*test.macros(), *ref) / e0)
    final = test.macros()
    # what the storage format alone loses: the oracle with its populations
    # rounded through that format (deviations from the far-field equilibrium)
    emulated = {}
    for fmt in ("f16", "bf16"):
        o = oracle.Oracle(V_N, V_N, V_TAU, 1.0, (u0, 0.0), **kw).storage(fmt, True).init(*f0)
        re = [R.energy(*o.step(V_EVERY).macros(), *r) / e0 for r in refs]
        emulated[fmt] = dict(drho=float(np.abs(o.macros()[0] - final[0]).max()),
                             r_change=abs(max(re) - max(rs)) / max(rs))
    return dict(u0=u0, f0=f0, refs=refs, e0=e0, r_max=max(rs), final=final, emulated=emulated)


# Bars: density error 1e-4 for 16-bit storage (f32: 1e-6), R_max change 1 %.
# bf16 misses the density bar on this flow (emulated: 1.4e-4).
@pytest.mark.parametrize("storage,rho_tol,r_tol", [("f32", 1e-6, 0.01), ("f16", 1e-4, 0.01), ("bf16", 1e-4, 0.01)])
def test_vortex_storage_error_and_reflection(lbm, vortex_reference, storage, rho_tol, r_tol):
    ref = vortex_reference
    sim = lbm.Simulation(V_N, V_N, V_TAU, 1.0, (ref["u0"], 0.0), storage=storage, collision="mrt",
                         mrt_rates=VORTEX_RATES).init(*ref["f0"])
    rs = []
    for r in ref["refs"]:
        sim.step(V_EVERY)
        rs.append(R.energy(*sim.macros(), *r) / ref["e0"])
    got = sim.macros()
    sim.close()
    d_rho = float(np.abs(got[0] - ref["final"][0]).max())
    d_u = float(max(np.abs(got[1] - ref["final"][1]).max(), np.abs(got[2] - ref["final"][2]).max()))
    r_max = max(rs)
    change = abs(r_max - ref["r_max"]) / ref["r_max"]
    emulated = ref["emulated"]
    res = dict(case="vortex", storage=storage, workload=f"vortex leaving a {V_N}^2 domain, MRT, {V_STEPS} steps",
               max_abs_drho=d_rho, max_abs_du=d_u, r_max=r_max, r_max_oracle=ref["r_max"], r_change=change,
               oracle_storage_emulation=emulated.get(storage))
    # the 16-bit error is the storage format's: within a factor of 3 of the
    # oracle run that loses only what that storage loses
    _check(res, storage, rho_tol, r_tol, emulated)
