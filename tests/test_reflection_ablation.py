"""The NSBC readings the paper leaves open, compared by the reflection they
leave (oracle, FP64): the one-sided difference of Eq. nes_2 (first or second
order) and the corner treatment (Sec. 5 is silent on corners: the diagonal
normal, or the mean of the two edges' predictions).  The stored values in
tests/golden/reflection_ablation.json are written by
tests/golden/make_reflection_ablation.py from the oracle alone; this file
recomputes the CPU-sized ones and pins the orderings they show:

  * a radial pulse (pulse-256): the second-order difference reflects more
    than the first-order one, and the corner mean a little less than the
    diagonal normal;
  * the Sec. 6 plane wave at 60 degrees (MRT 1.9): the second-order
    difference reflects a little less, and the corner reading makes no
    difference (the wave's energy has left before it matters);
  * the vortex leaving a 200^2 domain (MRT, tau 0.505): with the first-order
    difference R stays below 0.2 and the corner reading changes it by under
    0.1 %; with the second-order one the oracle run grows without bound by
    step 800 -- not because of the vortex: the second-order difference is
    unstable on the inflow edge (tests/test_nsbc_stability.py), and the
    oracle's rounding of absolute populations there seeds it;
  * the 400^2 BGK vortex at tau 0.505 blows up under every reading, more than
    twice as soon with the second-order difference, and the corner reading
    moves the step by at most 2 %: it does not cure the instability.
"""
import json
import os

import pytest

import reflection_cases as rc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "reflection_ablation.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def measured():
    out = {}
    for case in (rc.pulse(256, 500), rc.plane_wave(), rc.vortex_exit()):
        refs, e0 = rc.reference(case)
        out[case.name] = {k: rc.oracle_rmax(case, refs, e0, v) for k, v in rc.VARIANTS.items()}
    return out


def test_stored_values_reproduce(golden, measured):
    for name, row in measured.items():
        for k, v in row.items():
            assert v == pytest.approx(golden["r_max"][name][k], rel=1e-9), (name, k)
    assert set(golden["r_max"]) >= {"pulse-256", "plane-wave", "vortex-exit", "pulse-1024"}


def test_orderings(measured):
    p, w, v = measured["pulse-256"], measured["plane-wave"], measured["vortex-exit"]
    assert p["order2_diagonal"] > 1.02 * p["order1_diagonal"]
    assert p["order1_mean"] < p["order1_diagonal"] < p["order2_mean"] < p["order2_diagonal"]
    assert w["order2_diagonal"] < 0.99 * w["order1_diagonal"]
    assert w["order1_mean"] == pytest.approx(w["order1_diagonal"], rel=1e-6)
    assert v["order1_diagonal"] < 0.2
    assert v["order1_mean"] == pytest.approx(v["order1_diagonal"], rel=1e-3)
    assert v["order2_diagonal"] > 10 and v["order2_mean"] > 10


def test_large_pulse_orderings(golden):
    """The same pulse ordering at 1024^2 (stored: several minutes of oracle)."""
    p = golden["r_max"]["pulse-1024"]
    assert p["order1_mean"] < p["order1_diagonal"] < p["order2_mean"] < p["order2_diagonal"]


def test_bgk_blowup_steps(golden):
    """Recomputes the stored steps: BGK at tau 0.505 with a Ma 0.1 stream blows
    up whatever the reading, the second-order difference sooner, and the
    corner reading hardly moves the step."""
    import make_reflection_ablation as mk  # noqa: E402  (tests/golden is on the path below)
    steps = {k: mk.bgk_blowup_step(int(k[5]), 1 if k.endswith("mean") else 0)
             for k in golden["bgk_vortex_400_blowup_step"]}
    assert steps == golden["bgk_vortex_400_blowup_step"]
    assert all(s is not None for s in steps.values())
    assert steps["order2_diagonal"] < 0.5 * steps["order1_diagonal"]
    for order in (1, 2):  # the corner reading moves the step by at most 2 %
        a, b = steps[f"order{order}_mean"], steps[f"order{order}_diagonal"]
        assert abs(a - b) <= 0.02 * b
