"""The bounds-checked build (liblbm_check.so, compiled with LBM_CHECK) stands
in for a device memory checker: every global access of the step kernels and
every shared-memory tile access is checked against the buffers the host
registered, and an access that fails is counted and not made.  The runs of
tests/checked_run.py (every launch form, odd sizes, batched) must reject
nothing and still match the oracle; with every buffer registered 1 KB short,
the checker must reject accesses (to memory that is still valid)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checked_lib():
    from paper_2005_08674_gb300 import build
    return build.build(check=True)


def run_checked(extra_env=None):
    env = dict(os.environ, LBM_CHECKED="1", **(extra_env or {}))
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_no_access_leaves_its_buffer(checked_lib):
    res = run_checked()
    assert res["checked"] is True, res
    assert res["rejected"] == 0, res
    assert res["max_err_f64"] <= 1e-12, res


def test_checker_rejects_accesses_past_a_shortened_buffer(checked_lib):
    res = run_checked({"LBM_CHECK_SHRINK": "1024"})
    assert res["checked"] is True, res
    assert res["rejected"] > 0, res
