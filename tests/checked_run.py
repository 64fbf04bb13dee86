"""Driver for the bounds-checked library (run in a child process with
LBM_CHECKED=1 by test_checked_build_gpu.py; not collected by pytest).

Steps every launch form of the single-domain (kernel pair, fused, staged,
two-step where it applies) and batched paths on small, odd-sized domains (all storages, BGK and MRT,
first- and second-order NSBC differences, periodic and velocity edges, far
fields at rest and in a stream, i.e. the plain and shifted kernels) and
prints one JSON line: whether the loaded library is the checked build, how
many accesses its checker rejected, the first rejected address, and the
largest f64 difference from the oracle (the checked build must still compute
the same results)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_2005_08674_gb300 import inputs, lbm  # noqa: E402

STEPS = 21
SIZES = [(3, 3), (5, 7), (33, 17), (65, 4), (517, 4), (4, 129), (130, 66), (9, 8), (300, 41)]
LAUNCHES = [("pair", (64, 1, 0)), ("pair", (128, 2, 1)), ("pair", (256, 1, 3)), ("pair", (512, 8, 64)),
            ("fused", (128, 1, 0)), ("fused", (64, 4, 3)), ("staged", 3), ("staged", 4), ("twostep", None)]
BATCH_LAUNCHES = [(128, 1, -1, 0, 0, 0), (64, 1, 0, 0, 0, 0), (128, 2, 0, 1, 1, 0), (256, 4, 152, 0, 0, 0),
                  (64, 4, 7, 64, 1, 0), (128, 1, 0, 0, 1, 128), (128, 1, 0, 0, 1, 256), (256, 1, 0, 0, 1, 256),
                  (128, 4, -1, 1, 0, 0), (256, 1, -1, 0, 1, 0), (128, 3, 0, 0, 0, 128), (128, 4, 0, 2, 0, 128),
                  (128, 3, 5, 2, 0, 128)]


def err(a, b):
    return max(float(np.abs(x - y).max()) for x, y in zip(a, b))


def main():
    torch.cuda.set_device(0)
    worst = 0.0
    kws = [dict(beta=0.1), dict(collision="mrt", mrt_rates=(1.4, 1.4, 1.2), grad_order=2),
           dict(edges=[("velocity", 0.03, 0.0), "nsbc", "periodic", "periodic"]),
           # a far field with a mean flow: the shifted form of every step kernel
           dict(farfield_rho=1.001, farfield_u=(0.04, -0.01), beta=0.1, collision="mrt", mrt_rates=(1.4, 1.4, 1.2)),
           # the second corner reading (an out-of-line second prediction at corners)
           dict(farfield_u=(0.02, 0.01), corner_mode=1, grad_order=2)]
    for nx, ny in SIZES:
        fields = inputs.acoustic_pulse(nx, ny, 1e-3, 2.0, [((nx - 1) / 2, (ny - 1) / 2)])
        ref = oracle.Oracle(nx, ny, 0.6, beta=0.1).init(*fields).step(STEPS).macros()
        for storage in ("f64", "f32", "f16", "bf16"):
            for kind, arg in LAUNCHES:
                for i, kw in enumerate(kws):
                    with lbm.Simulation(nx, ny, 0.6, storage=storage, **kw) as s:
                        s.init(*fields)
                        if kind == "twostep":
                            if storage == "f64" or nx < 8 or ny < 8 or "edges" in kw:
                                continue  # the two-step kernel does not serve these
                            s.set_twostep(True)
                        elif kind == "staged":
                            s.set_staged(arg)
                        else:
                            s.set_launch(*arg)
                            s.set_fused(kind == "fused")
                        got = s.step(STEPS).macros()
                        s.reduce(allow_unstable=True)
                    if storage == "f64" and i == 0:
                        worst = max(worst, err(got, ref))
    ws = inputs.batch_instances(count=6, lo=3, hi=90)
    ws += [inputs.Workload("thin", 517, 4, 0.6, 0, farfield_u=(0.02, 0.0), kind="pulse",
                           params=dict(amplitude=1e-3, half_width=3.0, centres=[(100.0, 1.5)]))]
    for storage in ("f64", "f32", "f16"):
        for j, launch in enumerate(BATCH_LAUNCHES):
            with lbm.Batch(ws, storage=storage, beta=0.05, corner_mode=j % 2) as b:
                for k, w in enumerate(ws):
                    b.init(k, *w.fields())
                b.set_launch(*launch)
                b.step(STEPS)
                b.status()
                for k in range(len(ws)):
                    b.macros(k)
    torch.cuda.synchronize()
    checked, rejected, first = lbm.lbm_check_read()
    print(json.dumps(dict(checked=checked, rejected=rejected, first=hex(first), max_err_f64=worst)), flush=True)


if __name__ == "__main__":
    main()
