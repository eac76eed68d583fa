"""The sorting network of the short-row sweep (csrc/sortnet.h, Batcher's
odd-even merge network) compiled for the host: by the 0-1 principle (Knuth,
TAOCP vol. 3, 5.3.4, Theorem Z) a comparator network sorts every input when
it sorts every 0-1 input, checked exhaustively for every width class of the
sweep up to 24 wires (64 inputs at a time for 24) and on 2^26 sampled 0-1
inputs for 32; plus seeded float inputs with ties and -inf against
std::sort, and the comparator counts of Batcher's construction."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_07777_gb300", "csrc")

PROGRAM = r"""
#include <algorithm>
#include <cmath>
#include <cstdint>
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

// 0-1 inputs 64 at a time: word t holds wire t of inputs base .. base + 63
// (input number n sets wire t to bit t of n); a comparator puts OR on its
// upper wire and AND on its lower one, so sortedness is w[t] >= w[t + 1]
// lane by lane.  Every input when all, else `words` random blocks of 64.
template <int N>
static bool check01_wide(bool all, unsigned words) {
  constexpr auto P = dlm::Batcher<N>::pairs();
  const uint64_t low[6] = {0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull, 0xF0F0F0F0F0F0F0F0ull,
                           0xFF00FF00FF00FF00ull, 0xFFFF0000FFFF0000ull, 0xFFFFFFFF00000000ull};
  std::mt19937_64 rng(11);
  const uint64_t blocks = all ? (uint64_t(1) << (N - 6)) : words;
  for (uint64_t blk = 0; blk < blocks; ++blk) {
    const uint64_t base = (all ? blk : (rng() & ((uint64_t(1) << (N - 6)) - 1))) << 6;
    uint64_t w[N];
    for (int t = 0; t < N; ++t) w[t] = t < 6 ? low[t] : (((base >> t) & 1u) ? ~0ull : 0ull);
    for (int c = 0; c < dlm::Batcher<N>::kCount; ++c) {
      const uint64_t x = w[P.lo[c]], y = w[P.hi[c]];
      w[P.lo[c]] = x | y;
      w[P.hi[c]] = x & y;
    }
    for (int t = 0; t + 1 < N; ++t)
      if (w[t + 1] & ~w[t]) return false;
  }
  return true;
}

// the wide classes: every 0-1 input for 24 wires, 2^26 of them for 32, and
// seeded float inputs against std::sort
template <int N>
static bool check_wide(bool all) {
  if (!check01_wide<N>(all, 1u << 20)) return false;
  std::mt19937 rng(9);
  for (int trial = 0; trial < 20000; ++trial) {
    float v[N], w[N];
    for (int t = 0; t < N; ++t) {
      const unsigned r = rng() % 16;
      v[t] = r == 0 ? -INFINITY : static_cast<float>(static_cast<int>(rng() % 17) - 8) * 0.125f;
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
  return (check<4>() && check<6>() && check<8>() && check<10>() && check<12>() && check<16>() &&
          check_wide<24>(true) && check_wide<32>(false)) ? 0 : 1;
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
    # 5.3.4), 63 for 16, 191 for 32; its restrictions to 6, 10, 12 and 24
    # inputs keep 12, 32, 42 and 132 (the comparators that touch no input
    # past n)
    assert counts == {4: 5, 6: 12, 8: 19, 10: 32, 12: 42, 16: 63, 24: 132, 32: 191}
