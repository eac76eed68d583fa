// sweep_short.cu -- the iteration sweep over slices of short rows.
//
// Rows of at most kShortRowW edges (the tail of the degree-sorted slice
// order) are projected from registers: one pass streams the row and keeps its
// values u = -(c + a y); a sorting network orders them and the sort-based
// threshold rule finds the active set in one scan; the pair-arithmetic
// refinement and the deposits read the row's edges again (from L1).  The
// general sweep (sweep.cu) tracks the four (or eight) largest values and, for
// rows with more active edges, iterates over the row, streaming it again for
// every pass -- the usual case near the optimum on instances whose short rows
// are mostly active (App. A's construction: about ten edges per request, many
// within gamma z of the row's maximum).  With this sweep switched on
// (dlm_options.short_rows) an iteration takes two launches, the general sweep
// over the wider slices and this one over the rest, both adding into the same
// exact fixed-point sums; certificate sweeps always take the general sweep.
//
// Arithmetic per row (Sec. 3.2 Eq. primal-recovery; Sec. 4.3 sorts the row to
// find the simplex threshold, as here): with the values sorted,
// v_0 >= v_1 >= ..., the active count is the largest r with
// r v_{r-1} > v_0 + ... + v_{r-1} - gamma z (FP32), and tau is then recomputed
// over the r active edges in float-pair arithmetic, so that
// x = (u - tau) / gamma keeps FP32 relative accuracy; one active edge with
// tau >= 0 gets x = z exactly.  The inequality simplex takes max(tau, 0) (the
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

// One slice whose width w lies in (WC - 4, WC]: groups 0 .. G - 2 of the
// lane's edges are full groups of four, group G - 1 is a full group when
// w = WC and otherwise the slice's tail of w - 4 (G - 1) edges, stored
// edge-major (layout.cu).
template <class P, int WC>
__device__ __forceinline__ void short_slice(const InstDesc& D, const Seg& S, const float* __restrict__ ys,
                                            unsigned long long* accG, int64_t off, int w,
                                            unsigned long long& oq) {
  constexpr int G = WC / 4;
  const int lane = threadIdx.x & 31;
  const bool full = w == WC;
  const uint16_t* __restrict__ col0 = D.col16 + off;
  const typename P::T* __restrict__ ca0 = static_cast<const typename P::T*>(D.ca) + off;
  const bool box = S.kind == DLM_BOX;
  const bool eq = S.kind == DLM_SIMPLEX_EQ;

  // Loads edges 4 g .. 4 g + 3 of the lane (padding and edges past w:
  // c = +inf, a = 0, j = 0, so that u = -inf).
  struct Grp {
    int j[4];
    float c[4], a[4];
  };
  auto group = [&](int g) {
    Grp r;
    if (g < G - 1 || full) {
      const int q = 32 * g + lane;
      P::idx4(col0, q, r.j);
      P::get4(ca0, q, r.c, r.a);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        r.j[e] = 0;
        r.c[e] = INFINITY;
        r.a[e] = 0.f;
        if (4 * g + e < w) {
          const int el = 128 * g + 32 * e + lane;
          P::get(__ldg(ca0 + el), r.c[e], r.a[e]);
          r.j[e] = static_cast<int>(__ldg(col0 + el));
        }
      }
    }
    return r;
  };

  // The row's u, sorted descending (the edge order is not kept: the passes
  // below read the edges again).
  float v[WC];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const Grp r = group(g);
#pragma unroll
    for (int e = 0; e < 4; ++e) v[4 * g + e] = -fmaf(r.a[e], ys[r.j[e]], r.c[e]);
  }
  sort_desc<WC>(v);
  // no edge with x > 0: an empty row (all padding), or every u <= 0 on the
  // inequality simplex or the box
  const bool none = v[0] == -INFINITY || (!eq && !(v[0] > 0.f));
  if (__all_sync(kFull, none)) return;

  float tau = 0.f, taul = 0.f;
  bool single = false;
  if (!box && !none) {
    // sort-based rule: r = the largest q + 1 with (q + 1) v_q > S_{q+1} - gamma z
    float sm = 0.f, sr = v[0];
    int r = 1;
#pragma unroll
    for (int q = 0; q < WC; ++q) {
      sm += v[q];
      if (q > 0 && static_cast<float>(q + 1) * v[q] > sm - S.gz) {
        r = q + 1;
        sr = sm;
      }
    }
    tau = r == 1 ? v[0] - S.gz : __fdiv_rn(sr - S.gz, static_cast<float>(r));
    bool zero = !eq && tau <= 0.f;
    single = !zero && r == 1;
    if (!zero && !single) {
      // the threshold over the active set in pair arithmetic (edge order)
      F2 ps{0.f, 0.f};
      int cnt = 0;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const Grp r = group(g);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float y = ys[r.j[e]];
          if (-fmaf(r.a[e], y, r.c[e]) > tau) {
            ps = f2_add(ps, u_pair(r.c[e], r.a[e], y));
            ++cnt;
          }
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
  // x on the active edges, their item sums and the row's objective
  float ob = 0.f;
  unsigned long long cn = 0ull;
  if (!none) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const Grp r = group(g);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float y = ys[r.j[e]];
        if (-fmaf(r.a[e], y, r.c[e]) > tau) {
          const float x = single ? S.z : x_general(S, box, tau, taul, r.c[e], r.a[e], y);
          if (x > 0.f) deposit<P, false>(S, r.j[e], r.c[e], r.a[e], x, accG, nullptr, nullptr, ob, cn);
        }
      }
    }
  }
  oq += fixp(ob, S.scaleO);
}

// Slices s_begin .. s_end - 1 of instance 0, dealt to the warps in turn
// (every warp gets the same mix of widths); item sums in shared memory,
// flushed once per CTA.
template <class P>
__global__ void __launch_bounds__(kSweepThreads, 1)
    sweep_short_kernel(const InstDesc* __restrict__ insts, int64_t s_begin, int64_t s_end) {
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
  for (int64_t s = s_begin + static_cast<int64_t>(blockIdx.x) * nw + (threadIdx.x >> 5); s < s_end; s += step) {
    const int64_t off = __ldg(sD.slice_off + s);
    const int w = __ldg(sD.slice_w + s);
    // width classes of four (warp-uniform branch)
    if (w > 12)
      short_slice<P, 16>(sD, S, ys, accG, off, w, oq);
    else if (w > 8)
      short_slice<P, 12>(sD, S, ys, accG, off, w, oq);
    else if (w > 4)
      short_slice<P, 8>(sD, S, ys, accG, off, w, oq);
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
  sweep_short_kernel<Narrow<V>><<<L.grid, th, sm, L.stream>>>(L.inst, L.short_first, L.short_end);
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
  if (L.short_first < 0 || L.short_end <= L.short_first) return cudaSuccess;
  return bf16 ? launch_short_values<BF16Pair>(L) : launch_short_values<F32Pair>(L);
}

}  // namespace dlm
