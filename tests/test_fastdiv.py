"""The multiply-high integer division used for index decoding in the Hartree kernel is
exact: compared with C integer division over the grid sizes in use and random operands."""
import os
import shutil
import subprocess

import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2410_09189_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include <random>
#include "fastdiv.h"
using namespace rmgtd;
int main() {
  std::mt19937_64 rng(241009189);
  long bad = 0;
  const int ds[] = {1, 2, 3, 4, 5, 6, 7, 8, 12, 16, 24, 27, 32, 48, 56, 64, 72, 80, 88, 96, 128,
                    192, 216, 512, 1728, 4096, 13824, 32768, 110592, 262144, 884736, 2097152,
                    7077888, 1000003, 2147483647};
  for (int d : ds) {
    const FastDiv f = make_fastdiv(d);
    for (int x = 0; x < 1000000; ++x) bad += fdiv(x, f) != x / d;
    for (int k = 0; k < 200000; ++k) {
      const int x = (int)(rng() % 2147483648ull);
      bad += fdiv(x, f) != x / d;
    }
    bad += fdiv(2147483647, f) != 2147483647 / d;
  }
  for (int k = 0; k < 2000000; ++k) {
    const int d = 1 + (int)(rng() % 2147483647ull), x = (int)(rng() % 2147483648ull);
    bad += fdiv(x, make_fastdiv(d)) != x / d;
  }
  std::printf("%ld\n", bad);
  return bad != 0;
}
"""


def test_fastdiv_exact(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "fd.cpp"
    src.write_text(SRC)
    exe = tmp_path / "fd"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "0", out.stdout
