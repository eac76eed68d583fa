// sweep_short.cu -- the iteration sweep for instances of short rows.
//
// Rows of at most kShortRowW (32) edges are projected from registers: one
// pass streams the row and keeps its values u = -(c + a y) (with, for short
// enough rows, each edge's value as a float pair or its dual); a sorting
// network orders the values and the sort-based threshold rule finds the
// active set in one scan; the threshold's refinement and the deposits read
// the row's c, a and items again (from L1).  The general sweep (sweep.cu)
// tracks the four (or eight) largest values and, for rows with more active
// edges, iterates over the row, streaming it again for every pass -- the
// usual case near the optimum on instances whose rows are short and mostly
// active (App. A's construction: about ten edges per request, many within
// gamma z of the row's maximum).  With this sweep switched on
// (dlm_options.short_rows) it takes every slice of the iteration sweep; the
// rare wider rows take a plain re-reading threshold iteration.  Certificate
// sweeps always take the general sweep.
//
// Arithmetic per row (Sec. 3.2 Eq. primal-recovery; Sec. 4.3 sorts the row to
// find the simplex threshold, as here): with the values sorted,
// v_0 >= v_1 >= ..., the active count is the largest r with
// r v_{r-1} > v_0 + ... + v_{r-1} - gamma z (FP32), and tau is then recomputed
// over the r active edges as v_0 plus an offset: the edges' values are float
// pairs (c + a y evaluated exactly), and their differences from v_0, all within
// gamma z of 0, are summed in FP32, so that x = (u - tau) / gamma is accurate
// to FP32 relative to z whatever the size of u; one active edge with tau >= 0
// gets x = z exactly.  The inequality simplex takes max(tau, 0) (the
// early exit of Sec. 4.3); the box clips u / gamma to [0, z].  A row's
// arithmetic involves no other row, so its result does not depend on the
// mapping or on the other rows of its slice.
#include "dlm_impl.cuh"
#include "sortnet.h"
#include "sweep_common.cuh"

namespace dlm {
namespace {

// Sorts v into descending order with the comparators of sortnet.h, one max
// and one min each (the loop unrolls; every index is a compile-time constant).
template <int N>
__device__ __forceinline__ void sort_desc(float (&v)[N]) {
  constexpr typename Batcher<N>::Pairs P = Batcher<N>::pairs();
#pragma unroll
  for (int t = 0; t < Batcher<N>::kCount; ++t) {
    const float x = v[P.lo[t]], y = v[P.hi[t]];
    v[P.lo[t]] = fmaxf(x, y);
    v[P.hi[t]] = fminf(x, y);
  }
}

// One slice of width w <= WC (the width class: 4, 6, 8, 10, 12, 16, 24 or
// 32; the classes below 12 are two apart because the sort and every per-slot
// pass cost in proportion to WC, and App. A's rows have about ten edges):
// the lane's edges 0 .. 4 w4 - 1 are w4 = w / 4 groups of four, the rest the
// slice's tail of w - 4 w4 edges, stored edge-major (layout.cu); positions
// past w are padding.
//
// What the first pass keeps besides the sorted values depends on the width
// (registers): up to 12 edges every edge's u as a float pair (uh, ul), so the
// refinement is a register pass and the deposits read only the edges' c, a
// and item again; 13 to 16 edges each edge's dual y_j, the later passes
// recomputing the pair from c, a read again; wider rows nothing more, the
// later passes also gathering y_j again.
template <class P, int WC>
__device__ __forceinline__ void short_slice(const InstDesc& D, const Seg& S, const float* __restrict__ ys,
                                            unsigned long long* accG, int64_t off, int w,
                                            unsigned long long& oq) {
  constexpr int G = (WC + 3) / 4;  // groups of four; slots past WC are never read
  constexpr bool KEEP = WC <= 12;
  constexpr bool YK = WC > 12 && WC <= 16;
  const int lane = threadIdx.x & 31;
  const int w4 = w >> 2;
  const uint16_t* __restrict__ col0 = D.col16 + off;
  const typename P::T* __restrict__ ca0 = static_cast<const typename P::T*>(D.ca) + off;
  const bool box = S.kind == DLM_BOX;
  const bool eq = S.kind == DLM_SIMPLEX_EQ;

  // Edges 4 g .. 4 g + 3 of the lane (padding and edges past w: c = +inf,
  // a = 0, j = 0, so that u = -inf).
  struct Grp {
    int j[4];
    float c[4], a[4];
  };
  auto group = [&](int g) {
    Grp r;
    if (g < w4) {
      const int q = 32 * g + lane;
      P::idx4(col0, q, r.j);
      P::get4(ca0, q, r.c, r.a);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        r.j[e] = 0;
        r.c[e] = INFINITY;
        r.a[e] = 0.f;
        if (g == w4 && 4 * g + e < w) {
          const int el = 128 * g + 32 * e + lane;
          P::get(__ldg(ca0 + el), r.c[e], r.a[e]);
          r.j[e] = static_cast<int>(__ldg(col0 + el));
        }
      }
    }
    return r;
  };

  // First pass: the values sorted descending into v; per edge (edge order)
  // the pair (uh, ul) with KEEP, else the dual y.  The value an edge is
  // ranked and tested by is uh with KEEP (the pair's high part; -inf for
  // padding) and -fma(a, y, c) otherwise.
  float v[WC], uh[KEEP ? WC : 1], ul[KEEP ? WC : 1], yk[YK ? WC : 1];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const Grp r = group(g);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 4 * g + e;
      if (k >= WC) break;
      const float y = ys[r.j[e]];
      if constexpr (KEEP) {
        // padding: uh = -inf (c = +inf, a = 0); its ul (NaN) is never read,
        // every later use being guarded by uh > tau
        const F2 u = u_pair(r.c[e], r.a[e], y);
        uh[k] = u.h;
        ul[k] = u.l;
        v[k] = u.h;
      } else {
        if constexpr (YK) yk[k] = y;
        v[k] = -fmaf(r.a[e], y, r.c[e]);
      }
    }
  }
  sort_desc<WC>(v);
  // no edge with x > 0: an empty row (all padding), or every u <= 0 on the
  // inequality simplex or the box
  const bool none = v[0] == -INFINITY || (!eq && !(v[0] > 0.f));
  if (__all_sync(kFull, none)) return;

  float tau = 0.f, taul = 0.f;
  bool single = false;
  if (!box && !none) {
    // sort-based rule: r = the largest q + 1 with (q + 1) v_q - S_{q+1} > -gamma z
    float sm = 0.f, sr = v[0];
    int r = 1;
#pragma unroll
    for (int q = 0; q < WC; ++q) {
      sm += v[q];
      if (q > 0 && fmaf(static_cast<float>(q + 1), v[q], -sm) > -S.gz) {
        r = q + 1;
        sr = sm;
      }
    }
    tau = r == 1 ? v[0] - S.gz : __fdiv_rn(sr - S.gz, static_cast<float>(r));
    bool zero = !eq && tau <= 0.f;
    single = !zero && r == 1;
    if (!zero && !single) {
      // the threshold over the active set (edge order) as an offset from
      // v_0: the active values lie within gamma z of v_0, so the FP32 sum of
      // the differences u - v_0 (each u a float pair) is accurate to FP32
      // relative to gamma z, as x = (u - tau) / gamma needs
      const float v0 = v[0];
      float sd = 0.f;
      int cnt = 0;
      if constexpr (KEEP) {
#pragma unroll
        for (int k = 0; k < WC; ++k) {
          if (uh[k] > tau) {
            sd += (uh[k] - v0) + ul[k];
            ++cnt;
          }
        }
      } else {
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const Grp rg = group(g);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (4 * g + e >= WC) break;
            const float y = YK ? yk[YK ? 4 * g + e : 0] : ys[rg.j[e]];
            if (-fmaf(rg.a[e], y, rg.c[e]) > tau) {
              const F2 u = u_pair(rg.c[e], rg.a[e], y);
              sd += (u.h - v0) + u.l;
              ++cnt;
            }
          }
        }
      }
      const float t = __fdiv_rn((sd - S.gz) - S.gzl, static_cast<float>(cnt > 0 ? cnt : 1));
      if (!eq && v0 + t <= 0.f) {
        zero = true;
      } else {
        tau = v0;
        taul = t;
      }
    }
    if (zero) {
      tau = 0.f;
      taul = 0.f;
    }
  }
  // x on the active edges, their item sums and the row's objective:
  // x = (((u_h - tau) + u_l) - taul) / gamma on the edges with u above
  // tau + taul, (tau, taul) being (v_0, the offset) after the refinement and
  // (0, 0) at the inequality simplex's early exit and for the box
  float ob = 0.f;
  const float hg = 0.5f * S.gamma;
  const float tt = tau + taul;
  const float zc = box ? S.z : INFINITY;  // the box's upper bound
  if (!none) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const Grp rg = group(g);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 4 * g + e;
        if (k >= WC) break;
        float x = 0.f;
        if constexpr (KEEP) {
          if (uh[k] > tt) {
            const float d = ((uh[k] - tau) + ul[k]) - taul;
            x = single ? S.z : fminf(fmaxf(d * S.invg, 0.f), zc);
          }
        } else {
          const float y = YK ? yk[YK ? k : 0] : ys[rg.j[e]];
          if (-fmaf(rg.a[e], y, rg.c[e]) > tt) {
            const F2 u = u_pair(rg.c[e], rg.a[e], y);
            const float d = ((u.h - tau) + u.l) - taul;
            x = single ? S.z : fminf(fmaxf(d * S.invg, 0.f), zc);
          }
        }
        if (x > 0.f) {
          // the item sum a x in 64-bit fixed point; the objective c x + gamma/2 x^2
          atomicAdd(&accG[rg.j[e]], fixp(rg.a[e] * x, S.scaleG));
          ob = fmaf(fmaf(hg, x, rg.c[e]), x, ob);
        }
      }
    }
  }
  oq += fixp(ob, S.scaleO);
}

// A slice of rows wider than kShortRowW (few, on the instances this sweep is
// for): each pass reads the lane's row again -- its maximum, then the
// Michelot iteration tau <- (sum_{u > tau} u - gamma z) / #{u > tau} from the
// lower bound max u - gamma z (the active sets shrink until two passes
// agree), the pair-arithmetic refinement over the final set and the deposits.
template <class P>
__device__ __forceinline__ void wide_slice(const InstDesc& D, const Seg& S, const float* __restrict__ ys,
                                        unsigned long long* accG, int64_t off, int w, unsigned long long& oq) {
  const int lane = threadIdx.x & 31;
  const int w4 = w >> 2;
  const uint16_t* __restrict__ col0 = D.col16 + off;
  const typename P::T* __restrict__ ca0 = static_cast<const typename P::T*>(D.ca) + off;
  const bool box = S.kind == DLM_BOX;
  const bool eq = S.kind == DLM_SIMPLEX_EQ;
  auto edge = [&](int k, int& j, float& c, float& a) {
    const int el = sell_el(k, lane, w4);
    j = static_cast<int>(__ldg(col0 + el));
    P::get(__ldg(ca0 + el), c, a);
  };
  float m = -INFINITY;
#pragma unroll 1
  for (int k = 0; k < w; ++k) {
    int j;
    float c, a;
    edge(k, j, c, a);
    m = fmaxf(m, -fmaf(a, ys[j], c));
  }
  const bool none = m == -INFINITY || (!eq && !(m > 0.f));
  float tau = 0.f, taul = 0.f;
  bool single = false;
  if (!box && !none) {
    tau = m - S.gz;
    int n = 0, prevn = -1;
#pragma unroll 1
    for (int it = 0; it <= w; ++it) {  // every pass shrinks the set or stops
      float sm = 0.f;
      int cnt = 0;
#pragma unroll 1
      for (int k = 0; k < w; ++k) {
        int j;
        float c, a;
        edge(k, j, c, a);
        const float u = -fmaf(a, ys[j], c);
        if (u > tau) {
          sm += u;
          ++cnt;
        }
      }
      n = cnt;
      if (cnt == prevn || cnt == 0) break;
      prevn = cnt;
      const float tn = __fdiv_rn(sm - S.gz, static_cast<float>(cnt));
      if (tn == tau) break;
      tau = tn;
    }
    bool zero = !eq && tau <= 0.f;
    single = !zero && n == 1;
    if (!zero && !single) {
      F2 ps{0.f, 0.f};
      int cnt = 0;
#pragma unroll 1
      for (int k = 0; k < w; ++k) {
        int j;
        float c, a;
        edge(k, j, c, a);
        const float y = ys[j];
        if (-fmaf(a, y, c) > tau) {
          ps = f2_add(ps, u_pair(c, a, y));
          ++cnt;
        }
      }
      const F2 t2 = f2_threshold(ps, S.gz, S.gzl, cnt > 0 ? cnt : 1);
      if (!eq && t2.h + t2.l <= 0.f) {
        zero = true;
      } else {
        tau = t2.h;
        taul = t2.l;
      }
    }
    if (zero) {
      tau = 0.f;
      taul = 0.f;
    }
  }
  float ob = 0.f;
  unsigned long long cn = 0ull;
  if (!none) {
#pragma unroll 1
    for (int k = 0; k < w; ++k) {
      int j;
      float c, a;
      edge(k, j, c, a);
      const float y = ys[j];
      if (-fmaf(a, y, c) > tau) {
        const float x = single ? S.z : x_general(S, box, tau, taul, c, a, y);
        if (x > 0.f) deposit<P, false>(S, j, c, a, x, accG, nullptr, nullptr, ob, cn);
      }
    }
  }
  oq += fixp(ob, S.scaleO);
}

// Every slice of instance 0, dealt to the warps in turn (every warp gets the
// same mix of widths); item sums in shared memory, flushed once per CTA.
template <class P>
__global__ void __launch_bounds__(kSweepThreads, 1)
    sweep_short_kernel(const InstDesc* __restrict__ insts, int64_t nslices) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDesc sD;
  __shared__ unsigned long long s_red[32];
  if (threadIdx.x == 0) sD = insts[0];
  __syncthreads();
  const int J = sD.J;
  unsigned long long* accG = reinterpret_cast<unsigned long long*>(smem_raw);
  float* ys = reinterpret_cast<float*>(accG + J);
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    ys[j] = sD.y[j];
    accG[j] = 0ull;
  }
  Seg S{};
  {
    const double g = *sD.gamma;
    S.gamma = static_cast<float>(g);
    S.invg = static_cast<float>(1.0 / g);
    const double gz = g * static_cast<double>(sD.z);
    S.gz = static_cast<float>(gz);
    S.gzl = static_cast<float>(gz - static_cast<double>(S.gz));
    S.z = sD.z;
    S.scaleG = sD.scaleG;
    S.scaleO = sD.scaleO;
    S.kind = sD.kind;
  }
  __syncthreads();
  unsigned long long oq = 0ull;
  const int nw = blockDim.x >> 5;
  const int64_t step = static_cast<int64_t>(gridDim.x) * nw;
  for (int64_t s = static_cast<int64_t>(blockIdx.x) * nw + (threadIdx.x >> 5); s < nslices; s += step) {
    const int64_t off = __ldg(sD.slice_off + s);
    const int w = __ldg(sD.slice_w + s);
    // width classes (warp-uniform branch)
    if (w > kShortRowW)
      wide_slice<P>(sD, S, ys, accG, off, w, oq);
    else if (w > 24)
      short_slice<P, 32>(sD, S, ys, accG, off, w, oq);
    else if (w > 16)
      short_slice<P, 24>(sD, S, ys, accG, off, w, oq);
    else if (w > 12)
      short_slice<P, 16>(sD, S, ys, accG, off, w, oq);
    else if (w > 10)
      short_slice<P, 12>(sD, S, ys, accG, off, w, oq);
    else if (w > 8)
      short_slice<P, 10>(sD, S, ys, accG, off, w, oq);
    else if (w > 6)
      short_slice<P, 8>(sD, S, ys, accG, off, w, oq);
    else if (w > 4)
      short_slice<P, 6>(sD, S, ys, accG, off, w, oq);
    else
      short_slice<P, 4>(sD, S, ys, accG, off, w, oq);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    const unsigned long long v = accG[j];
    if (v) atomicAdd(sD.acc + j, v);
  }
  cta_add_u64(oq, s_red, sD.objq);
}

template <class V>
cudaError_t launch_short_values(const SweepLaunch& L) {
  const int th = L.threads > 0 ? L.threads : kSweepThreads;
  const size_t sm = sweep_smem_bytes(L.smemJ, false);
  sweep_short_kernel<Narrow<V>><<<L.grid, th, sm, L.stream>>>(L.inst, L.nslices0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t sweep_short_prepare(bool bf16) {
  const int lim = static_cast<int>(sweep_smem_limit());
  return bf16 ? cudaFuncSetAttribute(&sweep_short_kernel<Narrow<BF16Pair>>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
              : cudaFuncSetAttribute(&sweep_short_kernel<Narrow<F32Pair>>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t launch_sweep_short(const SweepLaunch& L, bool bf16) {
  return bf16 ? launch_short_values<BF16Pair>(L) : launch_short_values<F32Pair>(L);
}

}  // namespace dlm
