"""Write reflection_ablation.json: the FP64 oracle's reflected-energy ratio
R_max for the NSBC readings the paper leaves open (Sec. 5: the one-sided
difference of Eq. nes_2, first or second order; the corner treatment, on
which the paper is silent), on the workloads of tests/reflection_cases.py,
and the step at which the 400^2 convected vortex with BGK at tau 0.505 (Ma
0.1) first shows a non-finite or grossly wrong density under each reading.
Calls only the oracle and the shared input generators.

  python tests/golden/make_reflection_ablation.py [--skip-large]

(--skip-large leaves out pulse-1024, which takes several minutes.)
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import reflection_cases as rc  # noqa: E402
from paper_2005_08674_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "reflection_ablation.json")


def bgk_blowup_step(order: int, corner: int, limit: int = 3000, every: int = 10):
    """First multiple of `every` steps at which the 400^2 BGK vortex has a
    non-finite density or |rho - 1| > 0.5 anywhere (None if not by `limit`)."""
    w = inputs.vortex_400()
    o = oracle.Oracle(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, openmp=True, grad_order=order,
                      corner_mode=corner).init(*w.fields())
    for k in range(every, limit + 1, every):
        r = o.step(every).macros()[0]
        if not np.isfinite(r).all() or np.abs(r - 1).max() > 0.5:
            return k
    return None


def main():
    skip_large = "--skip-large" in sys.argv
    cases = [rc.pulse(256, 500), rc.plane_wave(), rc.vortex_exit()] + ([] if skip_large else [rc.pulse(1024, 2000)])
    old = json.load(open(OUT)) if os.path.exists(OUT) else {}
    r_max = dict(old.get("r_max", {}))
    for case in cases:
        refs, e0 = rc.reference(case)
        r_max[case.name] = {k: rc.oracle_rmax(case, refs, e0, v) for k, v in rc.VARIANTS.items()}
        print(case.name, r_max[case.name], flush=True)
    blowup = {f"order{o}_{'mean' if c else 'diagonal'}": bgk_blowup_step(o, c) for o in (1, 2) for c in (0, 1)}
    print("bgk blow-up", blowup, flush=True)
    out = {"what": "oracle R_max (reflection measure of oracle/reflection.py) per NSBC reading; "
                   "BGK vortex-400 (tau 0.505, Ma 0.1) blow-up step per reading",
           "variants": rc.VARIANTS, "r_max": r_max, "bgk_vortex_400_blowup_step": blowup}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
