"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lbm.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2005_08674_gb300 import build
    return build.build()


def test_header_declares_the_core_entry_points():
    names = declared_symbols()
    for core in ["lbm_create", "lbm_init", "lbm_step", "lbm_get_macros", "lbm_destroy"]:
        assert core in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2005_08674_gb300 import lbm
    assert set(lbm.EXPORTED) == declared_symbols()


def test_host_side_argument_checks(lib_path):
    """Argument validation happens on the host, before any device work."""
    from paper_2005_08674_gb300 import lbm
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(2, 10, 0.6)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(10, 10, 0.5)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(10, 10, 0.6, farfield_rho=0.0)
    h = lbm.lbm_create(200, 100, 0.6)
    try:
        assert lbm.lbm_buffer_bytes(h) == 9 * 100 * 256 * 4  # pitch 200 -> 256, f32
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_nsbc(h, 0.6, 0.0, 3.0, grad_order=3)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_nsbc(h, 0.6, 0.0, 3.0, corner_mode=2)
        lbm.lbm_set_nsbc(h, 0.6, 0.0, 3.0, corner_mode=1, grad_order=2)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_precision(h, 7)
        lbm.lbm_set_precision(h, "f16")
        assert lbm.lbm_buffer_bytes(h) == 9 * 100 * 256 * 2
        with pytest.raises(lbm.LbmError):
            lbm.lbm_step(h, 1)  # not initialised
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_launch(h, 96, 1, 0)
        assert lbm.lbm_get_staged(h) == 0
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_staged(h, 2)
        lbm.lbm_set_staged(h, 3)
        assert lbm.lbm_get_staged(h) == 3
        lbm.lbm_set_launch(h, 128, 1, 0)  # back to the kernel pair
        assert lbm.lbm_get_staged(h) == 0
        import numpy as np
        with pytest.raises(lbm.LbmError, match="bytes given"):
            lbm.lbm_load_state(h, np.zeros(100, dtype=np.uint8))
        with pytest.raises(lbm.LbmError, match="not a checkpoint record"):
            lbm.lbm_load_state(h, np.zeros(lbm.lbm_state_bytes(h), dtype=np.uint8))
        lbm.lbm_status(h)  # nothing launched yet: OK without touching the device
        assert lbm.lbm_steps_done(h) == 0
    finally:
        lbm.lbm_destroy(h)
    lbm.lbm_destroy(None)


def _record(lbm, h, storage, nx, ny, pitch, steps, m0):
    """A checkpoint record of lbm_state_bytes(h) bytes with the given header."""
    import struct
    import numpy as np
    buf = np.zeros(lbm.lbm_state_bytes(h), dtype=np.uint8)
    head = struct.pack("<8s6iq3d", b"LBMSTAT1", 1, storage, nx, ny, pitch, 0, steps, *m0)
    buf[:64] = np.frombuffer(head, dtype=np.uint8)
    return buf


def test_checkpoint_record_is_checked_before_any_device_work():
    """A record saved from an f16 handle has the byte count of a bf16 one of the
    same size; loading it there would continue on garbage, so the header is
    checked first (storage, size, pitch, far field, step count).  Host-only."""
    from paper_2005_08674_gb300 import lbm
    h = lbm.lbm_create(200, 100, 0.6, farfield_rho=1.0, farfield_u=(0.02, 0.0))
    try:
        lbm.lbm_set_precision(h, "bf16")
        assert lbm.lbm_state_bytes(h) == 64 + lbm.lbm_buffer_bytes(h)
        m0 = (1.0, 0.02, 0.0)
        with pytest.raises(lbm.LbmError, match="storage") as e:
            lbm.lbm_load_state(h, _record(lbm, h, lbm.LBM_F16, 200, 100, 256, 5, m0))
        assert e.value.code == lbm.LBM_EINVAL
        with pytest.raises(lbm.LbmError, match="storage"):
            lbm.lbm_load_state(h, _record(lbm, h, lbm.LBM_BF16, 100, 200, 256, 5, m0))
        with pytest.raises(lbm.LbmError, match="far field"):
            lbm.lbm_load_state(h, _record(lbm, h, lbm.LBM_BF16, 200, 100, 256, 5, (1.0, 0.0, 0.0)))
        with pytest.raises(lbm.LbmError, match="step count"):
            lbm.lbm_load_state(h, _record(lbm, h, lbm.LBM_BF16, 200, 100, 256, -1, m0))
    finally:
        lbm.lbm_destroy(h)


def test_ordinary_build_reports_no_checker(lib_path):
    """lbm_check_read exists in every build; the ordinary one has no checker."""
    from paper_2005_08674_gb300 import lbm
    if lbm.CHECKED:
        pytest.skip("the bounds-checked library is loaded")
    assert lbm.lbm_check_read() == (False, 0, 0)


def test_dims_and_host_array_checks(lib_path):
    """The binding sizes every host array from lbm_get_dims / lbm_batch_get_dims
    and refuses a wrong shape, dtype or layout before the library reads or
    writes a byte (these checks run on the host, without a GPU)."""
    import numpy as np
    from paper_2005_08674_gb300 import lbm
    h = lbm.lbm_create(37, 11, 0.6)
    try:
        assert lbm.lbm_get_dims(h) == (37, 11)
        good = np.ones((11, 37))
        for bad in (np.ones((11, 36)), np.ones((37, 11)), np.ones(11 * 37)):
            with pytest.raises(lbm.LbmError, match="shape"):
                lbm.lbm_init(h, bad, good, good)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_get_macros(h, good, good, np.ones((11, 37), dtype=np.float32))
        with pytest.raises(lbm.LbmError):
            lbm.lbm_get_macros(h, good, good, np.ones((37, 11)).T)  # not C-contiguous
        ro = np.ones((11, 37))
        ro.flags.writeable = False
        with pytest.raises(lbm.LbmError):
            lbm.lbm_get_macros(h, good, good, ro)
        with pytest.raises(lbm.LbmError, match="shape"):
            lbm.lbm_set_populations(h, np.ones((8, 11, 37)))
        with pytest.raises(lbm.LbmError):
            lbm.lbm_get_populations(h, np.ones((11, 37)))
    finally:
        lbm.lbm_destroy(h)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_get_dims(None)
    b = lbm.lbm_batch_create([(5, 7, 0.6, 1.0, 0.0, 0.0), (64, 3, 0.7, 1.0, 0.01, 0.0)], "f32")
    try:
        assert lbm.lbm_batch_get_dims(b, 0) == (5, 7)
        assert lbm.lbm_batch_get_dims(b, 1) == (64, 3)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_batch_get_dims(b, 2)
        with pytest.raises(lbm.LbmError, match="shape"):
            lbm.lbm_batch_init(b, 1, np.ones((7, 5)), np.ones((3, 64)), np.ones((3, 64)))
        with pytest.raises(lbm.LbmError):
            lbm.lbm_batch_get_macros(b, 0, np.ones((7, 5)), np.ones((7, 5)), np.ones((5, 7)))
    finally:
        lbm.lbm_batch_destroy(b)


def test_simulation_checks_reference_tensors_on_the_host(lib_path):
    """Simulation.reduce refuses a reference field that does not cover the
    domain or whose planes end before the last row the kernel would read,
    before any call reaches the library (CPU tensors stand in for device
    ones; the object is built without a device)."""
    import torch
    from paper_2005_08674_gb300 import lbm
    s = lbm.Simulation.__new__(lbm.Simulation)
    s.nx, s.ny, s.h = 20, 10, None
    s._a = torch.empty(1, dtype=torch.uint8)
    f64 = dict(dtype=torch.float64)
    bad = [(torch.zeros(3, 9, 24, **f64), {}), (torch.zeros(3, 10, 19, **f64), {}),
           (torch.zeros(3, 10, 24), {}), (torch.zeros(10, 24, **f64), {}),
           (torch.zeros(3, 30, 40, **f64)[:, 5:, 35:], {}),
           (torch.zeros(3, 10, 24, **f64), dict(ref_pitch=10)), (torch.zeros(3, 10, 24, **f64), dict(ref_pitch=30))]
    for ref, kw in bad:
        with pytest.raises(lbm.LbmError, match="reduce: ref"):
            s.reduce(ref, **kw)
    # a well-formed reference (a padded pitch, or a window of a larger field)
    # passes the checks and reaches the library, which refuses the NULL handle
    for ref in (torch.zeros(3, 10, 24, **f64), torch.zeros(3, 30, 40, **f64)[:, 5:, 7:]):
        with pytest.raises(lbm.LbmError, match="lbm_reduce: NULL"):
            s.reduce(ref)
    with pytest.raises(lbm.LbmError, match="init_device"):
        s.init_device(*(torch.zeros(20, 10, **f64),) * 3)


def test_binding_fails_loudly_without_the_library(tmp_path):
    """With the CUDA library absent the binding refuses to import: there is no
    CPU path to fall back to.  (A copy of the binding in a package with no
    library beside it, imported in a child process.)"""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_2005_08674_gb300"
    pkg.mkdir()
    (pkg / "__init__.py").write_text("")
    shutil.copy(os.path.join(ROOT, "paper_2005_08674_gb300", "lbm.py"), pkg / "lbm.py")
    r = subprocess.run([sys.executable, "-c", "import paper_2005_08674_gb300.lbm"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300,
                       env={k: v for k, v in os.environ.items() if k not in ("PYTHONPATH", "LBM_CHECKED")})
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "is not built" in r.stderr, r.stderr[-1000:]
