"""Host logic of the staged kernels, compiled with nvcc and run on the CPU (no
GPU needed): the work list of one instance covers every interior vector with
exactly one tile and every perimeter node with exactly one NSBC chunk, and
puts each chunk after the tile that stages the last row it reads; the
multiply-and-shift row divisor gives the exact quotient."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_08674_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "lbm_staged.cuh"

static int check_instance(int nx, int ny, int V, int tile, int chunk) {
  lbmk::InstDev d{};
  d.nx = nx;
  d.ny = ny;
  d.pitch = ((nx + V - 1) / V) * V;
  lbmk::set_row_divisor(d, V);
  std::vector<int4> items;
  lbmk::staged_instance_items(5, d, V, tile, chunk, items);
  const int nvec = d.pitch / V, total = (ny - 2) * nvec, perim = 2 * nx + 2 * (ny - 2);
  std::vector<int> vec_seen(total, 0), node_seen(perim, 0), tile_of_vec(total, -1);
  for (size_t p = 0; p < items.size(); ++p) {
    const int4 w = items[p];
    if (w.x >= 0) {
      if (w.x != 5 || w.z < 1 || w.z > tile) return 10;
      for (int j = w.y; j < w.y + w.z; ++j) {
        if (j < 0 || j >= total) return 11;
        ++vec_seen[j];
        tile_of_vec[j] = (int)p;
      }
    } else {
      if (~w.x != 5 || w.z < 1 || w.z > chunk) return 12;
      int last = 0;
      for (int n = w.y; n < w.y + w.z; ++n) {
        if (n < 0 || n >= perim) return 13;
        ++node_seen[n];
        const int r = lbmk::perimeter_row(n, nx, ny);
        last = std::max(last, std::min(r + 2, ny - 1));
      }
      // every interior row up to `last` is staged by a tile placed before the chunk
      const int R = std::min(last, ny - 2);
      if (R >= 1) {
        const int j = (R - 1) * nvec;
        if (tile_of_vec[j] < 0 || tile_of_vec[j] > (int)p) return 14;
      }
    }
  }
  for (int v : vec_seen) if (v != 1) return 15;
  for (int v : node_seen) if (v != 1) return 16;
  return 0;
}

static int check_divisor() {
  for (int nvec = 1; nvec <= 5000; nvec += (nvec < 300 ? 1 : 37)) {
    lbmk::InstDev d{};
    d.pitch = nvec * 4;
    lbmk::set_row_divisor(d, 4);
    for (long long j = 0; j < 4000000; j += (j < 20000 ? 1 : 997)) {
      const unsigned hi = (unsigned)(((unsigned long long)d.vec_mul * (unsigned long long)j) >> 32);
      const long long q = (long long)((hi + (unsigned)j) >> d.vec_shift);
      if (q != j / nvec) return 20;
    }
  }
  return 0;
}

int main() {
  const int sizes[][2] = {{3, 3}, {4, 5}, {17, 9}, {64, 64}, {65, 33}, {130, 7}, {1031, 12}, {8, 300}};
  const int forms[][3] = {{4, 128, 32}, {8, 128, 32}, {2, 128, 64}, {4, 16, 8}, {8, 3, 5}};
  for (auto& s : sizes)
    for (auto& f : forms) {
      const int rc = check_instance(s[0], s[1], f[0], f[1], f[2]);
      if (rc) {
        std::printf("instance %dx%d V=%d tile=%d chunk=%d: check %d failed\n", s[0], s[1], f[0], f[1], f[2], rc);
        return 1;
      }
    }
  const int rc = check_divisor();
  if (rc) {
    std::printf("row divisor: check %d failed\n", rc);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
"""


def _nvcc():
    return shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)


@pytest.mark.skipif(_nvcc() is None, reason="no nvcc")
def test_work_list_and_row_divisor(tmp_path):
    src = tmp_path / "work_list.cu"
    src.write_text(DRIVER)
    exe = tmp_path / "work_list"
    r = subprocess.run([_nvcc(), "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-gencode",
                        "arch=compute_103a,code=sm_103a", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.stdout, r.stderr)
