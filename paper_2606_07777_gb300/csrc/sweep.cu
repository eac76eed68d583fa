// sweep.cu -- the fused dual sweep (the per-iteration hot path).
//
// For every user i and dual point y (Sec. 3.2, Eq. primal-recovery):
//     u_ik = -(c_ik + a_ik * y_j(k))                 (v = u / gamma)
//     x_i  = Proj_C_i(u_i / gamma)
// and per item j (Eq. dual-gradient): (A x)_j = sum_i a_ij x_ij.
// With STATS it also accumulates per item sum c x and sum x^2 and the
// objective sum (c x + gamma/2 x^2) for the dual value and the certified gap,
// and optionally writes x in the caller's edge order.
//
// Layout and mapping: users sit in degree-sorted slices of 32 (layout.cu);
// lane t of a warp owns user t of its slice and walks the user's edges four
// at a time with 128-bit loads (512 contiguous bytes per warp load).  The item dual y lives in
// shared memory (gathered by item index); item sums are accumulated in
// shared memory and flushed once per CTA.
//
// Simplex projection (Sec. 4.3 gets the threshold by sorting the whole row;
// no sort here).  In u-space the threshold tau solves
// sum max(u - tau, 0) = gamma z.  One pass over the row keeps its four
// largest u in a sorted register network, with the positions of the first
// three; the sort-based rule applied to those four either fixes the active
// set (at most three edges active: nearly every row at the paper's gammas,
// and for one edge x = z on it exactly) or shows that at least four are
// active.  With at most three, the threshold is recomputed over the recorded
// edges in float-pair arithmetic, so that x = (u - tau) / gamma keeps full
// FP32 relative accuracy when u and tau nearly cancel, and x is deposited on
// them: no second pass over the row.  With four or more the lane (or the
// whole warp, when few lanes need it) runs the iteration
// tau <- (sum_{u > tau} u - gamma z) / #{u > tau} from tau_4 (Michelot 1986;
// monotone from below, it stops when the active set stops changing), the
// pair-arithmetic refinement and a deposit pass.  The inequality simplex
// takes max(tau, 0) (the early exit of Sec. 4.3).  Box: x = clip(u / gamma,
// 0, z).
//
// Determinism: item sums are 64-bit fixed point (value * 2^s rounded, s chosen
// at set-up so no sum can overflow), exact and order independent; slices are
// dealt to warps statically and the FP64 objective is summed per warp in
// slice order, per CTA in warp order and across CTAs in task order.
#include <cuda_bf16.h>

#include <algorithm>

#include "dlm_impl.cuh"
#include "sweep_common.cuh"

namespace dlm {
namespace {

// The same value layouts for instances with a global count constraint: the
// count dual mu floors the threshold and every deposit adds x to the count.
// (A separate instantiation, so that instances without one keep the plain
// code: the register and comparison cost measured 4 % on the sweep.)
template <class Base>
struct Counted : Base {
  static constexpr bool kCount = true;
};

// Threshold of user t of the slice computed by the whole warp: lane l takes
// edges l, l + 32, ... of the user (re-read from L1/L2; the warp has just
// streamed them), the Michelot sums and the pair-arithmetic refinement are
// warp reductions in a fixed order, and every lane deposits the x of its own
// edges.  tau0 is the starting threshold (a lower bound on the equality
// threshold); with `exact` it is already the threshold of the final active
// set and the iteration is skipped.  Returns the threshold (tau, taul) and
// whether the inequality simplex took tau = 0.
template <class P, bool STATS>
__device__ __forceinline__ void coop_user(const Seg& S, const float* __restrict__ ys, unsigned long long* accG,
                                          unsigned long long* accC, unsigned long long* accQ,
                                          const typename P::IX* __restrict__ cp0, const typename P::T* __restrict__ vp0,
                                          int w, int w4, int t, float tau0, bool exact, float& tau, float& taul,
                                          bool& zero, float& ob, unsigned long long& cn) {
  const int lane = threadIdx.x & 31;
  const bool box = S.kind == DLM_BOX;
  const bool eq = S.kind == DLM_SIMPLEX_EQ;
  auto uval = [&](int k, int& j, float& c, float& a) {
    const int e = sell_el(k, t, w4);
    j = static_cast<int>(__ldg(cp0 + e));
    P::get(__ldg(vp0 + e), c, a);
    return -fmaf(a, ys[j], c);
  };
  tau = 0.f;
  taul = 0.f;
  zero = box;
  if (!box) {
    tau = tau0;
    if (!exact) {
      int prevn = -1;
      for (int it = 0; it < 256; ++it) {
        float sm = 0.f;
        int n = 0;
        for (int k = lane; k < w; k += 32) {
          int j;
          float c, a;
          const float u = uval(k, j, c, a);
          if (u > tau) {
            sm += u;
            ++n;
          }
        }
        sm = warp_sum(sm);
        n = warp_sumi(n);
        if (n == prevn || n == 0) break;
        prevn = n;
        const float tn = __fdiv_rn(sm - S.gz, static_cast<float>(n));
        if (tn == tau) break;
        tau = tn;
      }
    }
    zero = !eq && tau <= (P::kCount ? S.mu : 0.f);
    if (!zero) {
      F2 sum{0.f, 0.f};
      int n = 0;
      for (int k = lane; k < w; k += 32) {
        int j;
        float c, a;
        if (uval(k, j, c, a) > tau) {
          sum = f2_add(sum, u_pair(c, a, ys[j]));
          ++n;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const F2 other{__shfl_xor_sync(kFull, sum.h, o), __shfl_xor_sync(kFull, sum.l, o)};
        sum = f2_add(sum, other);
        n += __shfl_xor_sync(kFull, n, o);
      }
      const F2 t2 = f2_threshold(sum, S.gz, S.gzl, n > 0 ? n : 1);
      if (!eq && t2.h + t2.l <= (P::kCount ? S.mu : 0.f)) {
        zero = true;
      } else {
        tau = t2.h;
        taul = t2.l;
      }
    }
  }
  if (zero) {
    tau = (P::kCount ? S.mu : 0.f);
    taul = 0.f;
  }
  for (int k = lane; k < w; k += 32) {
    int j;
    float c, a;
    if (uval(k, j, c, a) > tau) {
      const float x = x_general(S, box, tau, taul, c, a, ys[j]);
      if (x > 0.f) deposit<P, STATS>(S, j, c, a, x, accG, accC, accQ, ob, cn);
    }
  }
}

// A row whose simplex active set is the r <= 3 recorded edges (on the
// inequality simplex with tau <= 0: those of them with u > 0): load them once,
// compute the threshold over them in pair arithmetic, deposit x on each.
// Returns (tau, taul, zero, objective part).  Used by the iteration sweeps
// (same arithmetic, in the same order, as the re-reading path the certificate
// sweeps take): it saves a re-read (4 % on the 64-instance batch, 6 % on the
// appendix instance once its rows have several active edges; no change on
// the precision sweep).
template <class P, bool STATS, int K>
__device__ __forceinline__ float4 rows_upto(const Seg S, const float* __restrict__ ys, unsigned long long* accG,
                                         unsigned long long* accC, unsigned long long* accQ,
                                         const typename P::IX* __restrict__ col0, const typename P::T* __restrict__ ca0,
                                         int w4, int r, const int (&pos)[K - 1], float tau, bool eq,
                                         unsigned long long& cn) {
  const int lane = threadIdx.x & 31;
  int jr[K - 1];
  float cr[K - 1], ar[K - 1];
#pragma unroll
  for (int i = 0; i < K - 1; ++i) {
    jr[i] = 0;
    cr[i] = ar[i] = 0.f;
    if (i < r) {
      const int el = sell_el(pos[i], lane, w4);
      jr[i] = static_cast<int>(__ldg(col0 + el));
      P::get(__ldg(ca0 + el), cr[i], ar[i]);
    }
  }
  bool zero = !eq && tau <= (P::kCount ? S.mu : 0.f);
  float taul = 0.f;
  if (!zero) {
    F2 sum{0.f, 0.f};
#pragma unroll
    for (int i = 0; i < K - 1; ++i)
      if (i < r) sum = f2_add(sum, u_pair(cr[i], ar[i], ys[jr[i]]));
    const F2 t2 = f2_threshold(sum, S.gz, S.gzl, r);
    if (!eq && t2.h + t2.l <= (P::kCount ? S.mu : 0.f)) {
      zero = true;
    } else {
      tau = t2.h;
      taul = t2.l;
    }
  }
  if (zero) {
    tau = (P::kCount ? S.mu : 0.f);
    taul = 0.f;
  }
  float ob = 0.f;
#pragma unroll
  for (int i = 0; i < K - 1; ++i) {
    if (i < r) {
      const float x = x_general(S, false, tau, taul, cr[i], ar[i], ys[jr[i]]);
      if (x > 0.f) deposit<P, STATS>(S, jr[i], cr[i], ar[i], x, accG, accC, accQ, ob, cn);
    }
  }
  return make_float4(tau, taul, zero ? 1.f : 0.f, ob);
}

// Users of a slice whose active set is larger than the four tracked values
// (mode 3 below) are handled by the whole warp, one after another, unless at
// least coop_max of the 32 need it (then each lane runs its own user, which
// keeps the lanes busy).  coop_max is a tuning parameter (0: always per lane,
// 33: always cooperative).

// The K largest u of a row (v[0] >= ... >= v[K-1]) and the edge positions
// id[0..K-2] of the first K - 1.  K = 4 for most instances; K = 8 resolves
// rows with up to seven active edges without the threshold iteration.
template <int K>
struct TopK {
  float v[K];
  int id[K - 1];
};
template <int K>
__device__ __forceinline__ TopK<K> topk_empty() {
  TopK<K> t;
#pragma unroll
  for (int q = 0; q < K; ++q) t.v[q] = -INFINITY;
#pragma unroll
  for (int q = 0; q < K - 1; ++q) t.id[q] = 0;
  return t;
}
// Sorted insertion of edge k with value u (strict comparisons: among equal
// values the earlier edge ranks first; for K = 4 the network of top4_insert).
template <int K>
__device__ __forceinline__ void topk_insert(float u, int k, TopK<K>& t) {
  float x = u;
  int xi = k;
#pragma unroll
  for (int q = 0; q < K - 1; ++q) {
    const bool c = x > t.v[q];
    const float lo = c ? t.v[q] : x;
    const int loi = c ? t.id[q] : xi;
    t.v[q] = c ? x : t.v[q];
    t.id[q] = c ? xi : t.id[q];
    x = lo;
    xi = loi;
  }
  t.v[K - 1] = fmaxf(t.v[K - 1], x);
}

// After pass A over a row: the threshold, x and the deposits (modes below);
// col0/ca0 are the slice's element streams.
template <class P, bool STATS, bool REG3, int K>
__device__ __forceinline__ void finish_slice(const InstDesc& D, const Seg& S, const float* __restrict__ ys,
                                             unsigned long long* accG, unsigned long long* accC,
                                             unsigned long long* accQ, int64_t s, int w,
                                             const typename P::IX* __restrict__ col0,
                                             const typename P::T* __restrict__ ca0, const TopK<K>& tk, int coop_max,
                                             double& wobj, unsigned long long& cn, unsigned long long& oq) {
  const int lane = threadIdx.x & 31;
  const int w4 = w >> 2;
  const bool box = S.kind == DLM_BOX;
  const bool eq = S.kind == DLM_SIMPLEX_EQ;
  const float v0 = tk.v[0];
  const int i0 = tk.id[0];

  // The equality threshold solves sum_k max(u_k - tau, 0) = gamma z.  With
  // the values sorted, tau_r = (v_0 + ... + v_{r-1} - gamma z) / r and the
  // active count is the first r with v_r <= tau_r; scanning the K largest
  // either finds it (the active set lies among them) or shows that at least
  // K edges are active, and then tau_K is a lower bound for the iteration.
  // mode 0: no edge active; 1: the maximum alone, x = z; 2: threshold of the
  // final active set known (tau); 3: iterate from tau.
  int mode;
  float tau = 0.f, taul = 0.f;
  bool zero = box;
  int r = 0;
  if (box) {
    mode = (v0 > (P::kCount ? S.mu : 0.f)) ? 3 : 0;
  } else if (v0 == -INFINITY || (!eq && v0 <= (P::kCount ? S.mu : 0.f))) {
    mode = 0;
  } else {
    float sm = v0;
    r = 1;
    tau = v0 - S.gz;
#pragma unroll
    for (int q = 1; q < K; ++q) {
      if (r == q && tk.v[q] > tau) {
        sm += tk.v[q];
        r = q + 1;
        tau = __fdiv_rn(sm - S.gz, static_cast<float>(q + 1));
      }
    }
    mode = (r == 1 && (eq || tau >= (P::kCount ? S.mu : 0.f))) ? 1 : (r < K ? 2 : 3);
  }

  float ob = 0.f;
  if (mode == 2 && REG3) {
    const float4 res = rows_upto<P, STATS, K>(S, ys, accG, accC, accQ, col0, ca0, w4, r, tk.id, tau, eq, cn);
    tau = res.x;
    taul = res.y;
    zero = res.z != 0.f;
    ob += res.w;
  } else if (mode == 2) {
    // The active set is the r < K recorded edges (on the inequality simplex
    // with tau <= 0: those of them with u > 0).  Threshold over them in pair
    // arithmetic, then x on each (the edges are re-read from L1).
    zero = !eq && tau <= (P::kCount ? S.mu : 0.f);
    if (!zero) {
      F2 sum{0.f, 0.f};
#pragma unroll
      for (int i = 0; i < K - 1; ++i) {
        if (i >= r) break;
        const int el = sell_el(tk.id[i], lane, w4);
        const int j = static_cast<int>(__ldg(col0 + el));
        float c, a;
        P::get(__ldg(ca0 + el), c, a);
        sum = f2_add(sum, u_pair(c, a, ys[j]));
      }
      const F2 t2 = f2_threshold(sum, S.gz, S.gzl, r);
      if (!eq && t2.h + t2.l <= (P::kCount ? S.mu : 0.f)) {
        zero = true;
      } else {
        tau = t2.h;
        taul = t2.l;
      }
    }
    if (zero) {
    tau = (P::kCount ? S.mu : 0.f);
    taul = 0.f;
  }
#pragma unroll
    for (int i = 0; i < K - 1; ++i) {
      if (i >= r) break;
      const int el = sell_el(tk.id[i], lane, w4);
      const int j = static_cast<int>(__ldg(col0 + el));
      float c, a;
      P::get(__ldg(ca0 + el), c, a);
      const float x = x_general(S, false, tau, taul, c, a, ys[j]);
      if (x > 0.f) deposit<P, STATS>(S, j, c, a, x, accG, accC, accQ, ob, cn);
    }
  } else if (mode == 1) {
    const int el = sell_el(i0, lane, w4);
    const int j = static_cast<int>(__ldg(col0 + el));
    float c, a;
    P::get(__ldg(ca0 + el), c, a);
    deposit<P, STATS>(S, j, c, a, S.z, accG, accC, accQ, ob, cn);
  }

  // Mode 3 (K or more active edges, or the box): the whole warp per user
  // while few lanes need it, else each lane over its own row.
  const unsigned mask3 = __ballot_sync(kFull, mode == 3);
  const bool coop = mask3 != 0u && __popc(mask3) < coop_max;  // warp-uniform
  if (coop) {
    unsigned m = mask3;
    while (m) {
      const int t = __ffs(m) - 1;
      m &= m - 1;
      const float tt = __shfl_sync(kFull, tau, t);
      float ta, tl;
      bool zr;
      // every lane adds the objective of its edges of user t: that piece
      // goes to fixed point on its own, so the total does not depend on
      // which users share the warp
      float obu = 0.f;
      coop_user<P, STATS>(S, ys, accG, accC, accQ, col0, ca0, w, w4, t, tt, false, ta, tl, zr, obu, cn);
      if (STATS)
        ob += obu;
      else
        oq += fixp(obu, S.scaleO);
      if (lane == t) {
        tau = ta;
        taul = tl;
        zero = zr;
      }
    }
  } else if (mode == 3) {
    // Each lane over its own row, in groups of four edges (128-bit loads, as
    // in pass A) and then the tail, so every pass visits edges 0 .. w-1 in
    // order.
    auto row_pass = [&](auto&& visit) {
      for (int g = 0; g < w4; ++g) {
        const int q = 32 * g + lane;
        int jj[4];
        P::idx4(col0, q, jj);
        float c[4], a[4];
        P::get4(ca0, q, c, a);
        visit(jj[0], c[0], a[0]);
        visit(jj[1], c[1], a[1]);
        visit(jj[2], c[2], a[2]);
        visit(jj[3], c[3], a[3]);
      }
      for (int k = 4 * w4; k < w; ++k) {
        const int el = 128 * w4 + 32 * (k - 4 * w4) + lane;
        float c, a;
        P::get(__ldg(ca0 + el), c, a);
        visit(static_cast<int>(__ldg(col0 + el)), c, a);
      }
    };
    if (!box) {
      // Michelot iteration from tau_K, a lower bound of the threshold: the
      // active sets {u > tau} shrink until two passes agree.  Each pass also
      // sums its active set in pair arithmetic, so the pass that finds the
      // set unchanged already holds the sum the threshold is refined from.
      F2 psum{0.f, 0.f};
      int n = 0;
      bool settled = false;
      int prevn = -1;
      for (int it = 0; it < 256; ++it) {
        float sm = 0.f;
        int cnt = 0;
        F2 ps{0.f, 0.f};
        row_pass([&](int j, float c, float a) {
          const float y = ys[j];
          const float u = -fmaf(a, y, c);
          if (u > tau) {
            sm += u;
            ++cnt;
            ps = f2_add(ps, u_pair(c, a, y));
          }
        });
        psum = ps;
        n = cnt;
        if (cnt == prevn || cnt == 0) {
          settled = true;
          break;
        }
        prevn = cnt;
        const float tn = __fdiv_rn(sm - S.gz, static_cast<float>(cnt));
        if (tn == tau) {
          settled = true;
          break;
        }
        tau = tn;
      }
      zero = !eq && tau <= (P::kCount ? S.mu : 0.f);
      if (!zero) {
        if (!settled) {  // iteration cap: the sum over the current set
          psum = F2{0.f, 0.f};
          n = 0;
          row_pass([&](int j, float c, float a) {
            if (-fmaf(a, ys[j], c) > tau) {
              psum = f2_add(psum, u_pair(c, a, ys[j]));
              ++n;
            }
          });
        }
        const F2 t2 = f2_threshold(psum, S.gz, S.gzl, n > 0 ? n : 1);
        if (!eq && t2.h + t2.l <= (P::kCount ? S.mu : 0.f)) {
          zero = true;
        } else {
          tau = t2.h;
          taul = t2.l;
        }
      }
    }
    if (zero) {
      tau = (P::kCount ? S.mu : 0.f);
      taul = 0.f;
    }
    // x on the active edges (u > tau; for the box and tau = 0, u > 0)
    row_pass([&](int j, float c, float a) {
      const float y = ys[j];
      if (-fmaf(a, y, c) > tau) {
        const float x = x_general(S, box, tau, taul, c, a, y);
        if (x > 0.f) deposit<P, STATS>(S, j, c, a, x, accG, accC, accQ, ob, cn);
      }
    });
  }

  if (STATS) {
    const int64_t u = 32 * s + lane;
    if (D.xout != nullptr && u < D.nusers) {
      // x in the caller's order, every edge of the user
      const int64_t o = __ldg(D.orig_off + u);
      const int d = __ldg(D.udeg + u);
      const uint64_t ld = __ldg(D.lead + u);  // slice position k is caller edge lead_caller_pos(ld, k, d)
      for (int k = 0; k < d; ++k) {
        float x = 0.f;
        if (mode == 1) {
          x = (k == i0) ? S.z : 0.f;
        } else if (mode >= 2) {
          const int el = sell_el(k, lane, w4);
          const int j = static_cast<int>(__ldg(col0 + el));
          float c, a;
          P::get(__ldg(ca0 + el), c, a);
          if (-fmaf(a, ys[j], c) > tau) x = x_general(S, box, tau, taul, c, a, ys[j]);
        }
        D.xout[o + lead_caller_pos(ld, k, d)] = x;
      }
    }
    wobj += static_cast<double>(ob);
  } else {
    // the user's objective part, added exactly (64-bit fixed point)
    oq += fixp(ob, S.scaleO);
  }
}

// One slice: lane t = user t; edge k of lane t is element sell_el(k, t, w/4)
// of the slice.  Pass A streams the row in groups of four edges and keeps
// its four largest u with the positions of the first three.
template <class P, bool STATS, bool REG3, int K>
__device__ __forceinline__ void do_slice(const InstDesc& D, const Seg& S, const float* __restrict__ ys,
                                         unsigned long long* accG, unsigned long long* accC,
                                         unsigned long long* accQ, int64_t s, int coop_max, double& wobj,
                                         unsigned long long& cn, unsigned long long& oq) {
  const int lane = threadIdx.x & 31;
  const int64_t off = __ldg(D.slice_off + s);
  const int w = __ldg(D.slice_w + s);
  const int w4 = w >> 2;
  const typename P::IX* __restrict__ col0 = P::idx(D) + off;
  const typename P::T* __restrict__ ca0 = static_cast<const typename P::T*>(D.ca) + off;
  TopK<K> tk = topk_empty<K>();
  // groups of four edges in chunks of CH groups: the chunk's loads are issued
  // together, then each group is inserted unless no lane's group maximum tops
  // its K-th largest value (then the insertions change no record: strict
  // comparisons); the rows' lowest-cost edges come first (lead order,
  // layout.cu), so most groups after the first are skipped by the warp
  constexpr int CH = sizeof(typename P::T) == 4 ? 4 : 2;
  auto insert_group = [&](int g, const int (&jj)[4], const float (&c)[4], const float (&a)[4]) {
    float u[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) u[e] = -fmaf(a[e], ys[jj[e]], c[e]);
    const float m4 = fmaxf(fmaxf(u[0], u[1]), fmaxf(u[2], u[3]));
    if (__any_sync(kFull, m4 > tk.v[K - 1])) {
#pragma unroll
      for (int e = 0; e < 4; ++e) topk_insert<K>(u[e], 4 * g + e, tk);
    }
  };
  int g = 0;
  for (; g + CH <= w4; g += CH) {
    int jj[CH][4];
    float c[CH][4], a[CH][4];
#pragma unroll
    for (int h = 0; h < CH; ++h) {
      P::idx4(col0, 32 * (g + h) + lane, jj[h]);
      P::get4(ca0, 32 * (g + h) + lane, c[h], a[h]);
    }
#pragma unroll
    for (int h = 0; h < CH; ++h) insert_group(g + h, jj[h], c[h], a[h]);
  }
  for (; g < w4; ++g) {
    int jj[4];
    float c[4], a[4];
    P::idx4(col0, 32 * g + lane, jj);
    P::get4(ca0, 32 * g + lane, c, a);
    insert_group(g, jj, c, a);
  }
  for (int k = 4 * w4; k < w; ++k) {
    const int el = 128 * w4 + 32 * (k - 4 * w4) + lane;
    const int j = static_cast<int>(__ldg(col0 + el));
    float c, a;
    P::get(__ldg(ca0 + el), c, a);
    const float u = -fmaf(a, ys[j], c);
    topk_insert<K>(u, k, tk);
  }
  finish_slice<P, STATS, REG3, K>(D, S, ys, accG, accC, accQ, s, w, col0, ca0, tk, coop_max, wobj, cn, oq);
}

// Certificate sweeps (STATS) keep the item sums of the window of items
// jlo .. jlo + jw - 1 only, so that instances whose three item arrays do not
// fit in shared memory take one launch per window; every launch recomputes
// the same x and writes the same objective partials, and the count sum is
// flushed by the launch with jlo = 0.
template <class P, bool STATS, int K>
__global__ void __launch_bounds__(kSweepThreads, 1)
    sweep_kernel(const InstDesc* __restrict__ insts, const Task* __restrict__ tasks,
                 const int32_t* __restrict__ cta_task, int smemJ, int coop_max, int jlo, int jw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int accN = STATS ? jw : smemJ;
  unsigned long long* accG = reinterpret_cast<unsigned long long*>(smem_raw);
  unsigned long long* accC = accG + accN;
  unsigned long long* accQ = accC + accN;
  float* ys = reinterpret_cast<float*>(accG + (STATS ? 3 : 1) * static_cast<size_t>(accN));
  double* wsum = reinterpret_cast<double*>(ys + ((smemJ + 1) & ~1));

  __shared__ InstDesc sD;
  __shared__ unsigned long long s_next;
  __shared__ unsigned long long s_red[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const int t_last = cta_task[blockIdx.x + 1];
  int t = cta_task[blockIdx.x];
  while (t < t_last) {
    const int inst = tasks[t].inst;
    int te = t + 1;
    while (te < t_last && tasks[te].inst == inst) ++te;
    if (threadIdx.x == 0) sD = insts[inst];
    __syncthreads();
    const int J = sD.J;
    // items with sums in this launch (STATS: the window, clipped to J)
    const int nacc = STATS ? max(0, min(J - jlo, jw)) : J;
    for (int j = threadIdx.x; j < J; j += blockDim.x) ys[j] = sD.y[j];
    for (int j = threadIdx.x; j < nacc; j += blockDim.x) {
      accG[j] = 0ull;
      if (STATS) {
        accC[j] = 0ull;
        accQ[j] = 0ull;
      }
    }
    Seg S;
    {
      const double g = *sD.gamma;
      S.gamma = static_cast<float>(g);
      S.invg = static_cast<float>(1.0 / g);
      const double gz = g * static_cast<double>(sD.z);
      S.gz = static_cast<float>(gz);
      S.gzl = static_cast<float>(gz - static_cast<double>(S.gz));
      S.z = sD.z;
      S.scaleG = sD.scaleG;
      S.scaleC = sD.scaleC;
      S.scaleQ = sD.scaleQ;
      S.scaleN = sD.scaleN;
      S.scaleO = sD.scaleO;
      S.kind = sD.kind;
      S.count = sD.count_on;
      S.mu = sD.count_on ? sD.y[J] : 0.f;
      S.jlo = STATS ? jlo : 0;
      S.jw = nacc;
    }
    unsigned long long cn = 0ull, oq = 0ull;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    double wobj = 0.0;
    for (int k = t; k < te; ++k) {
      const Task T = tasks[k];
      if (STATS) {
        // static order: the FP64 objective partials are summed in a fixed order
        const int64_t step = static_cast<int64_t>(T.stride) * nw;
        for (int64_t s = T.first + static_cast<int64_t>(T.stride) * warp; s < T.end; s += step)
          do_slice<P, STATS, false, K>(sD, S, ys, accG, accC, accQ, s, coop_max, wobj, cn, oq);
      } else {
        // dynamic order within the CTA (item sums are exact, so the order of
        // slices does not change any result)
        const int64_t nsl = (T.end - T.first + T.stride - 1) / T.stride;
        for (;;) {
          int64_t i = 0;
          if (lane == 0) i = atomicAdd(&s_next, 1ull);
          i = __shfl_sync(kFull, i, 0);
          if (i >= nsl) break;
          do_slice<P, STATS, !STATS, K>(sD, S, ys, accG, accC, accQ, T.first + i * T.stride, coop_max, wobj, cn,
                                        oq);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
      }
    }
    if (STATS) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wobj += __shfl_xor_sync(kFull, wobj, o);
      if (lane == 0) wsum[warp] = wobj;
    } else {
      cta_add_u64(oq, s_red, sD.objq);
    }
    if (P::kCount && sD.count_on && (!STATS || jlo == 0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cn += __shfl_xor_sync(kFull, cn, o);
      if (lane == 0 && cn) atomicAdd(sD.cnt, cn);
    }
    __syncthreads();
    {
      const int j0 = STATS ? jlo : 0;
      for (int j = threadIdx.x; j < nacc; j += blockDim.x) {
        const unsigned long long v = accG[j];
        if (v) atomicAdd(sD.acc + j0 + j, v);
        if (STATS) {
          const unsigned long long vc = accC[j], vq = accQ[j];
          if (vc) atomicAdd(sD.accC + j0 + j, vc);
          if (vq) atomicAdd(sD.accQ + j0 + j, vq);
        }
      }
    }
    if (STATS && threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < nw; ++w) sum += wsum[w];
      sD.seg_obj[t] = sum;
    }
    __syncthreads();
    t = te;
  }
}

// Sweep with dynamic work distribution (iteration sweeps only): CTAs take
// work units -- a range of slices of one instance -- from a global counter in
// table order.  A CTA keeps an instance's y and item sums in shared memory
// across consecutive units of that instance and flushes the sums when it
// moves to another instance.  The last CTA to finish resets the counters for
// the next launch.  The units are ordered by instance and shrink toward the
// end of the table, so the CTAs finish together.
template <class P, int K>
__global__ void __launch_bounds__(kSweepThreads, 1)
    sweep_dyn_kernel(const InstDesc* __restrict__ insts, const Task* __restrict__ units, int nunits,
                     unsigned* __restrict__ ctr, int smemJ, int coop_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* accG = reinterpret_cast<unsigned long long*>(smem_raw);
  float* ys = reinterpret_cast<float*>(accG + smemJ);

  __shared__ InstDesc sD;
  __shared__ unsigned s_unit;
  __shared__ unsigned long long s_next;
  __shared__ unsigned long long s_red[32];
  const int lane = threadIdx.x & 31;
  int cur = -1;
  Seg S{};
  double wobj = 0.0;
  unsigned long long cn = 0ull, oq = 0ull;
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = atomicAdd(ctr, 1u);
      s_next = 0;
    }
    __syncthreads();
    const unsigned u = s_unit;
    const bool out_of_work = u >= static_cast<unsigned>(nunits);
    const int inst = out_of_work ? -1 : units[u].inst;
    if (out_of_work || inst != cur) {
      if (cur >= 0) {
        if (P::kCount && sD.count_on) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) cn += __shfl_xor_sync(kFull, cn, o);
          if (lane == 0 && cn) atomicAdd(sD.cnt, cn);
        }
        cn = 0ull;
        for (int j = threadIdx.x; j < sD.J; j += blockDim.x) {
          const unsigned long long v = accG[j];
          if (v) atomicAdd(sD.acc + j, v);
        }
        cta_add_u64(oq, s_red, sD.objq);
        oq = 0ull;
      }
      __syncthreads();
      if (out_of_work) break;
      if (threadIdx.x == 0) sD = insts[inst];
      __syncthreads();
      for (int j = threadIdx.x; j < sD.J; j += blockDim.x) {
        ys[j] = sD.y[j];
        accG[j] = 0ull;
      }
      const double g = *sD.gamma;
      S.gamma = static_cast<float>(g);
      S.invg = static_cast<float>(1.0 / g);
      const double gz = g * static_cast<double>(sD.z);
      S.gz = static_cast<float>(gz);
      S.gzl = static_cast<float>(gz - static_cast<double>(S.gz));
      S.z = sD.z;
      S.scaleG = sD.scaleG;
      S.scaleC = sD.scaleC;
      S.scaleQ = sD.scaleQ;
      S.scaleN = sD.scaleN;
      S.scaleO = sD.scaleO;
      S.kind = sD.kind;
      S.count = sD.count_on;
      S.mu = sD.count_on ? sD.y[sD.J] : 0.f;
      cur = inst;
      __syncthreads();
    }
    const Task T = units[u];
    const int64_t nsl = T.end - T.first;
    for (;;) {
      int64_t i = 0;
      if (lane == 0) i = static_cast<int64_t>(atomicAdd(&s_next, 1ull));
      i = __shfl_sync(kFull, i, 0);
      if (i >= nsl) break;
      do_slice<P, false, true, K>(sD, S, ys, accG, nullptr, nullptr, T.first + i, coop_max, wobj, cn, oq);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(ctr + 1, 1u);
    if (prev == gridDim.x - 1) {
      ctr[0] = 0u;
      ctr[1] = 0u;
    }
  }
}

template <class P, bool STATS, int K>
constexpr auto kernel_of() {
  return &sweep_kernel<P, STATS, K>;
}

}  // namespace

size_t sweep_smem_bytes(int smemJ, bool stats) { return sweep_stats_smem_bytes(smemJ, stats ? smemJ : 0); }

size_t sweep_stats_smem_bytes(int smemJ, int win) {
  const size_t J = static_cast<size_t>(smemJ);
  const size_t acc = win > 0 ? 3 * static_cast<size_t>(win) : J;
  return acc * 8 + ((J + 1) & ~static_cast<size_t>(1)) * 4 + 32 * 8;
}

int sweep_stats_window(int smemJ) {
  const size_t lim = sweep_smem_limit();
  if (sweep_stats_smem_bytes(smemJ, smemJ) <= lim) return smemJ;
  const size_t fixed = sweep_stats_smem_bytes(smemJ, 0) - static_cast<size_t>(smemJ) * 8;
  if (fixed >= lim) return 0;
  return static_cast<int>(std::min<size_t>((lim - fixed) / 24, static_cast<size_t>(smemJ)));
}

size_t sweep_smem_limit() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return optin > 1024 ? static_cast<size_t>(optin - 1024) : 0;  // room for static shared memory
}

template <class P, int K>
cudaError_t prepare_width(int lim) {
  cudaError_t e = cudaFuncSetAttribute(&sweep_dyn_kernel<P, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel_of<P, false, K>(), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel_of<P, true, K>(), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <class P>
cudaError_t prepare_policy(int lim) {
  const cudaError_t e = prepare_width<P, 4>(lim);
  return e != cudaSuccess ? e : prepare_width<P, 8>(lim);
}

template <class P, int K>
cudaError_t launch_width(const SweepLaunch& L, bool stats) {
  const int th = L.threads > 0 ? L.threads : kSweepThreads;
  const int cm = L.coop_max;
  if (stats) {
    const int w = L.win > 0 ? std::min(L.win, L.smemJ) : L.smemJ;
    if (w < 1) return cudaErrorInvalidValue;
    const size_t sm = sweep_stats_smem_bytes(L.smemJ, w);
    for (int jlo = 0; jlo < L.smemJ || jlo == 0; jlo += w) {
      sweep_kernel<P, true, K><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, cm, jlo, w);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const size_t sm = sweep_smem_bytes(L.smemJ, false);
  if (L.units != nullptr)
    sweep_dyn_kernel<P, K><<<L.grid, th, sm, L.stream>>>(L.inst, L.units, L.nunits, L.ctr, L.smemJ, cm);
  else
    sweep_kernel<P, false, K><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, cm, 0, L.smemJ);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_policy(const SweepLaunch& L, bool stats) {
  return L.topk == 8 ? launch_width<P, 8>(L, stats) : launch_width<P, 4>(L, stats);
}

template <class V>
cudaError_t prepare_values(int lim) {
  cudaError_t e = prepare_policy<Narrow<V>>(lim);
  if (e == cudaSuccess) e = prepare_policy<Counted<Narrow<V>>>(lim);
  return e;
}

template <class V>
cudaError_t launch_values(const SweepLaunch& L, bool stats) {
  return L.count ? launch_policy<Counted<Narrow<V>>>(L, stats) : launch_policy<Narrow<V>>(L, stats);
}

cudaError_t sweep_prepare(bool bf16) {
  const int lim = static_cast<int>(sweep_smem_limit());
  const cudaError_t e = bf16 ? prepare_values<BF16Pair>(lim) : prepare_values<F32Pair>(lim);
  return e != cudaSuccess ? e : sweep_short_prepare(bf16);
}

cudaError_t launch_sweep(const SweepLaunch& L, bool stats, bool bf16) {
  // iteration sweeps of a handle with the short-row sweep on take it alone
  if (!stats && L.short_rows) return launch_sweep_short(L, bf16);
  return bf16 ? launch_values<BF16Pair>(L, stats) : launch_values<F32Pair>(L, stats);
}

}  // namespace dlm
