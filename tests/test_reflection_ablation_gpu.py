"""The reflection ablation on the FP32 CUDA path: for each NSBC reading the
paper leaves open (Eq. nes_2 first- or second-order difference; diagonal or
mean corner treatment) and each workload of tests/reflection_cases.py --
pulse-1024 (the mixed-precision workload), the vortex leaving a 200^2
domain and the Sec. 6 plane wave -- the GPU's R_max against the padded
oracle reference is within 1 % of the oracle's own (stored in
tests/golden/reflection_ablation.json by an oracle-only script), so the
orderings the oracle shows hold on the GPU path too.

One comparison is left out: the second-order difference on the exiting
vortex.  That reading is linearly unstable on the inflow edge
(tests/test_nsbc_stability.py), so the run's fate depends on the noise that
seeds it there: the oracle rounds absolute populations (about 1e-16 of noise
in the uniform inflow every step) and blows up by step 800, while the CUDA
path computes in deviations from the far field, keeps the uniform inflow
exactly steady, and is still bounded at step 800.  Instead, the instability
itself is checked on the GPU: from the same noisy uniform stream, the f64
path's noise grows at the oracle's rate, on the same edge.  With
LBM_RESULTS_DIR set, the table is written there as JSON."""
import json
import os

import numpy as np
import pytest

import oracle
import reflection_cases as rc
import test_nsbc_stability as st

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "reflection_ablation.json")


@pytest.fixture(scope="module")
def lbm():
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import lbm as m
    return m


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)["r_max"]


@pytest.mark.parametrize("make", [lambda: rc.pulse(1024, 2000), rc.vortex_exit, rc.plane_wave],
                         ids=["pulse-1024", "vortex-exit", "plane-wave"])
def test_gpu_reflection_per_reading(lbm, golden, make):
    case = make()
    refs, e0 = rc.reference(case)
    got = {k: rc.gpu_rmax(lbm, case, refs, e0, v) for k, v in rc.VARIANTS.items()}
    want = golden[case.name]
    out = os.environ.get("LBM_RESULTS_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, f"ablation_{case.name}.json"), "w") as f:
            json.dump({"case": case.name, "gpu_f32": got, "oracle": want}, f)
    print(case.name, got, want)
    for k in rc.VARIANTS:
        if case.name == "vortex-exit" and k.startswith("order2"):
            continue  # seed-dependent: see the module docstring
        assert abs(got[k] - want[k]) <= 0.01 * want[k], (k, got[k], want[k])


@pytest.mark.parametrize("kw,steps", [(dict(collision="mrt", grad_order=2), 500), (dict(grad_order=1), 600)],
                         ids=["mrt-order2-inflow", "bgk-order1-outflow"])
def test_gpu_instability_matches_oracle(lbm, kw, steps):
    """The NSBC instabilities of a Ma 0.1 stream at tau 0.505, on the f64 CUDA
    path from the oracle's noisy initial state: same amplitude within 1 % and
    the same place (the noise, 1e-12, dominates both sides' rounding)."""
    okw = dict(kw)
    gkw = dict(kw)
    if kw.get("collision") == "mrt":
        okw["mrt_rates"] = st.MRT
        gkw["mrt_rates"] = (1.4, 1.4, 1.2)
    fields = st.noisy_stream()
    ref = st.amplitude(oracle.Oracle(st.N, st.N, st.TAU, 1.0, (st.U0, 0.0), openmp=True, **okw)
                       .init(*fields).step(steps).macros())
    with lbm.Simulation(st.N, st.N, st.TAU, 1.0, (st.U0, 0.0), storage="f64", **gkw) as s:
        got = st.amplitude(s.init(*fields).step(steps).macros())
    assert ref[0] > 1e-7
    assert abs(got[0] - ref[0]) <= 0.01 * ref[0], (got, ref)
    assert abs(got[1] - ref[1]) <= 1, (got, ref)
