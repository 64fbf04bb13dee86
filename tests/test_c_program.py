"""The boundary is a plain C ABI: include/lbm.h compiles as C11, and a C
program compiled with gcc and linked against liblbm.so runs the host-side
entry points (creation, argument checks, sizes, settings) without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2005_08674_gb300")

C_SOURCE = r"""
#include <stdio.h>
#include <string.h>
#include "lbm.h"

int main(void) {
  const double u[2] = {0.0, 0.0};
  if (lbm_create(2, 10, 0.6, 1.0, u) != NULL) return 1;          /* nx < 3 is refused */
  if (strstr(lbm_last_error(), "nx=2") == NULL) return 2;
  lbm_t* h = lbm_create(200, 100, 0.6, 1.0, u);
  if (!h) return 3;
  if (lbm_buffer_bytes(h) != (size_t)9 * 100 * 256 * 4) return 4; /* f32, pitch 256 */
  if (lbm_set_precision(h, LBM_F16) != LBM_OK) return 5;
  if (lbm_buffer_bytes(h) != (size_t)9 * 100 * 256 * 2) return 6;
  if (lbm_set_nsbc(h, 0.6, 0.1, 3.0, LBM_CORNER_MEAN, 2) != LBM_OK) return 7;
  if (lbm_set_nsbc(h, 0.6, 0.0, 3.0, LBM_CORNER_DIAGONAL, 3) != LBM_EINVAL) return 8; /* order 3 does not exist */
  if (lbm_set_nsbc(h, 0.6, 0.0, 3.0, 2, 1) != LBM_EINVAL) return 8; /* no third corner reading */
  if (lbm_step(h, 1) != LBM_ESTATE) return 9;                     /* not initialised */
  if (lbm_set_staged(h, 3) != LBM_OK || lbm_get_staged(h) != 3) return 10;
  if (lbm_set_fused(h, 1) != LBM_OK || lbm_get_fused(h) != 1 || lbm_get_staged(h) != 0) return 11;
  if (lbm_steps_done(h) != 0) return 12;
  int32_t nx = 0, ny = 0;
  if (lbm_get_dims(h, &nx, &ny) != LBM_OK || nx != 200 || ny != 100) return 13;
  if (lbm_get_dims(h, NULL, &ny) != LBM_EINVAL) return 14;
  lbm_destroy(h);
  lbm_destroy(NULL);
  printf("ok\n");
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_header_is_c11():
    r = subprocess.run(["gcc", "-fsyntax-only", "-x", "c", "-std=c11", "-Wall", "-Wextra", "-Werror",
                        os.path.join(ROOT, "include", "lbm.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c_program_uses_the_library(tmp_path):
    from paper_2005_08674_gb300 import build
    build.build()
    src = tmp_path / "host_calls.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "host_calls"
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", PKG, "-l:liblbm.so", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=PKG + os.pathsep + os.environ.get("LD_LIBRARY_PATH", ""))
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
