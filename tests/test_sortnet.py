"""The sorting network of the short-row sweep (csrc/sortnet.h, Batcher's
odd-even merge network) compiled for the host: by the 0-1 principle (Knuth,
TAOCP vol. 3, 5.3.4, Theorem Z) a comparator network sorts every input when
it sorts every 0-1 input, checked exhaustively for the widths the sweep
uses; plus seeded float inputs with ties and -inf against std::sort, and the
comparator counts of Batcher's construction."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_07777_gb300", "csrc")

PROGRAM = r"""
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <functional>
#include <random>
#include "sortnet.h"

template <int N>
static void apply(float (&v)[N]) {
  constexpr auto P = dlm::Batcher<N>::pairs();
  for (int t = 0; t < dlm::Batcher<N>::kCount; ++t) {
    const float x = v[P.lo[t]], y = v[P.hi[t]];
    v[P.lo[t]] = std::fmax(x, y);
    v[P.hi[t]] = std::fmin(x, y);
  }
}

template <int N>
static bool check() {
  for (unsigned bits = 0; bits < (1u << N); ++bits) {
    float v[N];
    for (int t = 0; t < N; ++t) v[t] = static_cast<float>((bits >> t) & 1u);
    apply<N>(v);
    for (int t = 0; t + 1 < N; ++t)
      if (v[t] < v[t + 1]) return false;
  }
  std::mt19937 rng(7);
  for (int trial = 0; trial < 20000; ++trial) {
    float v[N], w[N];
    for (int t = 0; t < N; ++t) {
      const unsigned r = rng() % 16;
      v[t] = r == 0 ? -INFINITY : static_cast<float>(static_cast<int>(rng() % 9) - 4) * 0.25f;
      w[t] = v[t];
    }
    apply<N>(v);
    std::sort(w, w + N, std::greater<float>());
    for (int t = 0; t < N; ++t)
      if (v[t] != w[t]) return false;
  }
  std::printf("%d %d\n", N, dlm::Batcher<N>::kCount);
  return true;
}

int main() {
  return (check<4>() && check<6>() && check<8>() && check<10>() && check<12>() && check<16>()) ? 0 : 1;
}
"""


def test_batcher_network_sorts(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "sortnet_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "sortnet_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    counts = dict(tuple(map(int, line.split())) for line in r.stdout.split("\n") if line.strip())
    # Batcher's odd-even merge sort: 5, 19 comparators for 4, 8 inputs (Knuth
    # 5.3.4), 63 for 16; its restrictions to 6, 10 and 12 inputs keep 12, 32
    # and 42 (the comparators that touch no input past n)
    assert counts == {4: 5, 6: 12, 8: 19, 10: 32, 12: 42, 16: 63}
