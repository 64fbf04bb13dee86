"""The autotuner cache file (csrc/lbm_tune_cache.h), on the CPU: a host
program built with g++ from the header checks the key's size classes and
fields, the round trip through the file, replacement of an entry, and the
fallbacks -- a missing, malformed or truncated file reads as empty and an
unwritable path makes store() report failure without touching anything.
The library's own entry points (lbm_set_tune_cache, lbm_tune_cache_stats) are
host-only and are called here too."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_08674_gb300", "csrc")

PROGRAM = r"""
#include "lbm_tune_cache.h"
#include <cassert>
#include <cstdio>
using namespace lbmtune;
#define CHECK(c) do { if (!(c)) { std::printf("FAILED line %d: %s\n", __LINE__, #c); return 1; } } while (0)
int main(int argc, char** argv) {
  const std::string dir = argv[1];
  // size classes: ceil(log2 n)
  CHECK(size_class(1) == 0 && size_class(2) == 1 && size_class(3) == 2 && size_class(256) == 8);
  CHECK(size_class(257) == 9 && size_class(8192) == 13 && size_class(8193) == 14);
  // keys: every field matters, sizes only through their class
  const std::string k = make_key("NVIDIA GB300", 13000, 13000, "abc", "domain", 1, 0, false, {8192, 8192});
  CHECK(k == make_key("NVIDIA GB300", 13000, 13000, "abc", "domain", 1, 0, false, {8000, 4097}));
  CHECK(k != make_key("NVIDIA GB300", 13000, 13000, "abc", "domain", 1, 0, false, {8192, 4096}));
  CHECK(k != make_key("NVIDIA GB300", 13000, 13000, "abc", "domain", 2, 0, false, {8192, 8192}));
  CHECK(k != make_key("NVIDIA GB300", 13000, 13000, "abc", "domain", 1, 1, false, {8192, 8192}));
  CHECK(k != make_key("NVIDIA GB300", 13000, 13000, "abc", "domain", 1, 0, true, {8192, 8192}));
  CHECK(k != make_key("NVIDIA GB300", 13000, 13000, "abd", "domain", 1, 0, false, {8192, 8192}));
  CHECK(k != make_key("NVIDIA GB300", 13010, 13000, "abc", "domain", 1, 0, false, {8192, 8192}));
  CHECK(k != make_key("NVIDIA GB200", 13000, 13000, "abc", "domain", 1, 0, false, {8192, 8192}));
  CHECK(k != make_key("NVIDIA GB300", 13000, 13000, "abc", "batch", 1, 0, false, {8192, 8192}));
  CHECK(make_key("a\"b\\c", 1, 1, "x", "domain", 0, 0, false, {3}).find('"') == std::string::npos);
  // missing file: empty, lookup misses
  const std::string path = dir + "/tune.json";
  Entry e;
  CHECK(load(path).empty() && !lookup(path, k, &e));
  // round trip, a second entry, replacement
  CHECK(store(path, Entry{k, {{"threads_x", 128}, {"rows", 1}, {"ms_per_step", 0.6982}}}));
  const std::string k2 = make_key("NVIDIA GB300", 13000, 13000, "abc", "batch", 2, 0, true, {256, 74800000});
  CHECK(store(path, Entry{k2, {{"tma_tile", 128}, {"ms_per_step", 0.5228}}}));
  double v = 0;
  CHECK(lookup(path, k, &e) && e.get("threads_x", &v) && v == 128 && e.get("ms_per_step", &v) && v == 0.6982);
  CHECK(!e.get("tma_tile", &v));
  CHECK(store(path, Entry{k, {{"threads_x", 256}, {"rows", 2}, {"ms_per_step", 0.7}}}));
  CHECK(load(path).size() == 2);
  CHECK(lookup(path, k, &e) && e.get("threads_x", &v) && v == 256);
  CHECK(lookup(path, k2, &e) && e.get("tma_tile", &v) && v == 128);
  // malformed and truncated files read as empty, and are rewritten by store
  const char* bad[] = {"", "{", "not json", "{\"lbm_tune_cache\": 2, \"entries\": []}",
                       "{\"lbm_tune_cache\": 1, \"entries\": [{\"key\": \"x\", \"a\": }]}",
                       "{\"lbm_tune_cache\": 1, \"entries\": [{\"key\": \"x\", \"a\": 1}", "[1, 2, 3]",
                       "{\"lbm_tune_cache\": 1, \"entries\": [{\"key\": \"x\", \"a\": nan}]}"};
  for (const char* text : bad) {
    FILE* f = std::fopen(path.c_str(), "wb");
    std::fputs(text, f);
    std::fclose(f);
    CHECK(load(path).empty() && !lookup(path, k, &e));
  }
  CHECK(store(path, Entry{k, {{"rows", 4}}}) && lookup(path, k, &e) && e.get("rows", &v) && v == 4);
  std::vector<Entry> parsed;
  CHECK(parse("{\"lbm_tune_cache\": 1, \"entries\": []}", parsed) && parsed.empty());
  // an unwritable location: store reports failure, nothing is created
  CHECK(!store(dir + "/no/such/dir/tune.json", Entry{k, {{"rows", 1}}}));
  std::printf("OK\n");
  return 0;
}
"""


def test_cache_file_logic(tmp_path):
    src = tmp_path / "tune_cache_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "tune_cache_check"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-Wall", "-I", CSRC, str(src), "-o", str(exe)])
    r = subprocess.run([str(exe), str(tmp_path)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr


def test_library_entry_points_are_host_only(tmp_path):
    """lbm_set_tune_cache / lbm_tune_cache_stats need no GPU: counts start at
    zero and a path can be set and cleared."""
    lbm = pytest.importorskip("paper_2005_08674_gb300.lbm")
    hits, misses = lbm.lbm_tune_cache_stats()
    assert hits >= 0 and misses >= 0
    lbm.lbm_set_tune_cache(str(tmp_path / "tune.json"))
    lbm.lbm_set_tune_cache(None)
    assert lbm.lbm_tune_cache_stats() == (hits, misses)
