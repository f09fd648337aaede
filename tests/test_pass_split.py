"""The bench's FLOP model follows the library's m-pass split (CPU).

bench.py restates the accumulation kernel's cost-balanced split of the m
columns into passes; this compiles a small host program against the
library's own constexpr split (csrc/ctb_internal.cuh) and compares them for
every l_max.
"""
import os
import shutil
import subprocess

import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

PROGRAM = r"""
#include <cstdio>
#include "ctb_internal.cuh"
using namespace ctb;
int main() {
  for (int L = 0; L <= kLmaxCap; ++L) {
    printf("%d", L);
    for (int m0 = 0; m0 <= L;) {
      const int m1 = pass_end(L, m0, pass_cap(L, m0));
      printf(" %d-%d", m0, m1);
      m0 = m1 + 1;
    }
    printf("\n");
  }
  return 0;
}
"""


def test_bench_pass_split_matches_library(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "split.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "split"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-o", str(exe), str(src),
                    "-I", os.path.join(ROOT, "paper_2604_08855_gb300", "csrc"), "-I", os.path.join(ROOT, "include")],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    lib = {}
    for line in out:
        if line.strip():
            parts = line.split()
            lib[int(parts[0])] = [tuple(int(v) for v in p.split("-")) for p in parts[1:]]
    assert sorted(lib) == list(range(21))
    for L, passes in lib.items():
        assert bench.pass_split(L) == passes, L
    assert lib[10] == [(0, 10)]
    assert lib[20] == [(0, 2), (3, 7), (8, 20)]
