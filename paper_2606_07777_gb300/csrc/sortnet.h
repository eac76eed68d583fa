// sortnet.h -- Batcher's odd-even merge sorting network on N inputs (Batcher
// 1968; the loop form of Knuth, TAOCP vol. 3, 5.3.4), listed at compile time
// as comparator pairs (lo, hi): applying the comparators in order, each
// putting the larger of v[lo], v[hi] at lo, sorts v into descending order.
// Plain C++17 (no CUDA), so that host tests check the same table the short-row
// sweep uses (sweep_short.cu).
#pragma once

namespace dlm {

template <int N>
struct Batcher {
  template <class F>
  static constexpr void each(F f) {
    for (int p = 1; p < N; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < N; j += 2 * k)
          for (int i = 0; i < k && i + j + k < N; ++i)
            if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) f(i + j, i + j + k);
  }
  static constexpr int count() {
    int c = 0;
    each([&](int, int) { ++c; });
    return c;
  }
  static constexpr int kCount = count();
  struct Pairs {
    int lo[kCount], hi[kCount];
  };
  static constexpr Pairs pairs() {
    Pairs r{};
    int c = 0;
    each([&](int a, int b) {
      r.lo[c] = a;
      r.hi[c] = b;
      ++c;
    });
    return r;
  }
};

}  // namespace dlm
