// sweep_boxcut.cu -- the dual sweep for the box cut by one budget,
// C_i = {0 <= x_ij <= z, sum_j x_ij <= cut}.
//
// In u-space (u = -(c + a y), x = clip((u - tau) / gamma, 0, z)) the threshold
// is tau = 0 when the clipped row meets the budget, else the root of
//     phi(tau) = sum_k clip((u_k - tau) / gamma, 0, z) - cut,
// which is continuous, nonincreasing and piecewise linear: on a piece the set
// F of free edges (0 < u - tau < gamma z) and the set U of capped ones
// (u - tau >= gamma z) are fixed and phi(tau) = (sum_F u - |F| tau) / gamma
// + z |U| - cut.  Each lane brackets the root of its own row, tries the root
// of the piece at the bracket's left end (a Newton step from the left), keeps
// it when the sets at the trial point are those of the piece (then it is the
// root), and otherwise narrows the bracket (bisecting when the trial point
// falls outside).  Every trial is one pass over the row, re-read from L1/L2.
// The final threshold is recomputed over F in float-pair arithmetic, as the
// simplex sweep does, so x keeps FP32 relative accuracy at small gamma.
//
// Layout, item sums (64-bit fixed point in shared memory, flushed once per
// CTA), static slice order and the FP64 objective partials are those of the
// one-family sweep (sweep.cu).
#include <algorithm>

#include "boxcut.cuh"
#include "sweep_common.cuh"

namespace dlm {
namespace {

struct BSeg {
  float gamma, invg, z, gzh, gzl, gch, gcl, cut;
  float scaleG, scaleC, scaleQ, scaleO;
  int jlo, jw;
};

template <class V, bool STATS>
__device__ __forceinline__ void deposit_b(const BSeg& S, int j, float c, float a, float x, unsigned long long* accG,
                                          unsigned long long* accC, unsigned long long* accQ, float& ob) {
  if (STATS) {
    const unsigned jj = static_cast<unsigned>(j - S.jlo);
    if (jj < static_cast<unsigned>(S.jw)) {
      atomicAdd(&accG[jj], fixp(a * x, S.scaleG));
      atomicAdd(&accC[jj], fixp(c * x, S.scaleC));
      atomicAdd(&accQ[jj], fixp(x * x, S.scaleQ));
    }
  } else {
    atomicAdd(&accG[j], fixp(a * x, S.scaleG));
  }
  ob += fmaf(0.5f * S.gamma * x, x, c * x);
}

// gamma (cut - z n) as a float pair: gamma cut minus n times gamma z, with the
// product's rounding error kept by FMA.
__device__ __forceinline__ F2 budget_pair(const BSeg& S, int n) {
  const float fn = static_cast<float>(n);
  const float p = fn * S.gzh;
  const float pe = fmaf(fn, S.gzh, -p);
  const F2 d = two_sum(S.gch, -p);
  return {d.h, d.l + (S.gcl - (pe + fn * S.gzl))};
}

template <class V, bool STATS>
__device__ __forceinline__ void boxcut_slice(const InstDesc& D, const BSeg& S, const float* __restrict__ ys,
                                             unsigned long long* accG, unsigned long long* accC,
                                             unsigned long long* accQ, int64_t s, double& wobj,
                                             unsigned long long& oq) {
  const int lane = threadIdx.x & 31;
  const int64_t off = __ldg(D.slice_off + s);
  const int w = __ldg(D.slice_w + s);
  const int w4 = w >> 2;
  const uint16_t* __restrict__ col0 = D.col16 + off;
  const typename V::T* __restrict__ ca0 = static_cast<const typename V::T*>(D.ca) + off;
  // the row in groups of four (one 64-bit index load, value loads as in the
  // simplex sweep), then the tail: edges 0 .. w-1 in order
  auto row_pass = [&](auto&& visit) {
    for (int g = 0; g < w4; ++g) {
      const int q = 32 * g + lane;
      const uint2 jv = __ldg(reinterpret_cast<const uint2*>(col0) + q);
      float c[4], a[4];
      V::get4(ca0, q, c, a);
      visit(static_cast<int>(jv.x & 0xffffu), c[0], a[0]);
      visit(static_cast<int>(jv.x >> 16), c[1], a[1]);
      visit(static_cast<int>(jv.y & 0xffffu), c[2], a[2]);
      visit(static_cast<int>(jv.y >> 16), c[3], a[3]);
    }
    for (int k = 4 * w4; k < w; ++k) {
      const int el = 128 * w4 + 32 * (k - 4 * w4) + lane;
      float c, a;
      V::get(__ldg(ca0 + el), c, a);
      visit(static_cast<int>(__ldg(col0 + el)), c, a);
    }
  };
  const float gz = S.gzh;
  // sets at a trial threshold t: free count and sum, capped count
  auto sets_at = [&](float t, int& nf, int& nu, float& sf) {
    nf = 0;
    nu = 0;
    sf = 0.f;
    row_pass([&](int j, float c, float a) {
      const float u = -fmaf(a, ys[j], c);
      const float y = u - t;
      if (y >= gz) {
        ++nu;
      } else if (y > 0.f) {
        ++nf;
        sf += u;
      }
    });
  };
  // phi(t) * gamma = sum_F (u - t) + gamma (z |U| - cut)
  auto phi_g = [&](float t, int nf, int nu, float sf) {
    return (sf - static_cast<float>(nf) * t) + (static_cast<float>(nu) * gz - S.gch);
  };

  // Pass A: the four largest u (v0 >= v1 >= v2 >= v3) and the sets at tau = 0.
  float v[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
  int nf = 0, nu = 0;
  float sf = 0.f;
  int i0 = 0, i1 = 0, i2 = 0;
  {
    // Groups of four edges, two groups' loads issued together (more spill);
    // every edge updates the sets at tau = 0, and a group
    // enters the record only if some lane's largest value of the group tops
    // its fourth largest (otherwise the insertions change no record: strict
    // comparisons) -- most groups after the first, the rows' lowest-cost edges
    // coming first (lead order, layout.cu).  Edges are visited in order, so
    // the sums are those of row_pass.
    auto count = [&](float u) {
      if (u >= gz) {
        ++nu;
      } else if (u > 0.f) {
        ++nf;
        sf += u;
      }
    };
    auto group_in = [&](int g, uint2 jv, const float (&c)[4], const float (&a)[4]) {
      const int jj[4] = {static_cast<int>(jv.x & 0xffffu), static_cast<int>(jv.x >> 16),
                         static_cast<int>(jv.y & 0xffffu), static_cast<int>(jv.y >> 16)};
      float u[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        u[e] = -fmaf(a[e], ys[jj[e]], c[e]);
        count(u[e]);
      }
      const float m4 = fmaxf(fmaxf(u[0], u[1]), fmaxf(u[2], u[3]));
      if (__any_sync(kFull, m4 > v[3])) {
#pragma unroll
        for (int e = 0; e < 4; ++e) top4_insert(u[e], 4 * g + e, v[0], v[1], v[2], v[3], i0, i1, i2);
      }
    };
    constexpr int CH = 2;
    int g = 0;
    for (; g + CH <= w4; g += CH) {
      uint2 jv[CH];
      float c[CH][4], a[CH][4];
#pragma unroll
      for (int h = 0; h < CH; ++h) {
        const int q = 32 * (g + h) + lane;
        jv[h] = __ldg(reinterpret_cast<const uint2*>(col0) + q);
        V::get4(ca0, q, c[h], a[h]);
      }
#pragma unroll
      for (int h = 0; h < CH; ++h) group_in(g + h, jv[h], c[h], a[h]);
    }
    for (; g < w4; ++g) {
      const int q = 32 * g + lane;
      const uint2 jv = __ldg(reinterpret_cast<const uint2*>(col0) + q);
      float c[4], a[4];
      V::get4(ca0, q, c, a);
      group_in(g, jv, c, a);
    }
    for (int k = 4 * w4; k < w; ++k) {
      const int el = 128 * w4 + 32 * (k - 4 * w4) + lane;
      float c, a;
      V::get(__ldg(ca0 + el), c, a);
      const float u = -fmaf(a, ys[__ldg(col0 + el)], c);
      count(u);
      top4_insert(u, k, v[0], v[1], v[2], v[3], i0, i1, i2);
    }
  }
  const float umax = v[0];
  float tau = 0.f, taul = 0.f;
  float ob = 0.f;
  bool deposited = false;
  if (umax > 0.f) {  // padding lanes and rows without a positive u deposit nothing
    if (phi_g(0.f, nf, nu, sf) > 0.f) {
      // The budget binds.  First try the pieces spanned by the four largest
      // values: a capped, f free (a + f <= 3), the rest at most v[a + f]; the
      // consistent one is the root's piece (phi is monotone).  A flat piece
      // (no free edge, a z = cut) has every point of it as a root.
      float lo = 0.f, hi = umax;
      int nfl = nf, nul = nu;
      float sfl = sf;
      bool found = false;
      const float ka = rintf(S.cut / S.z);
      const bool flat_ok = fabsf(S.cut / S.z - ka) <= 1e-6f * fmaxf(ka, 1.f);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int f = 0; f + a < 4; ++f) {
          if (found) continue;
          const float next = v[a + f];  // the largest value not in the capped or free part
          float t;
          if (f == 0) {
            if (!(flat_ok && static_cast<float>(a) == ka && a > 0)) continue;
            t = fmaxf(next, 0.f);
          } else {
            float sfree = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (i >= a && i < a + f) sfree += v[i];
            t = __fdiv_rn(sfree - (S.gch - static_cast<float>(a) * gz), static_cast<float>(f));
            if (!(v[a] - t < gz && v[a + f - 1] - t > 0.f)) continue;
          }
          if (!(t > 0.f) && f > 0) continue;
          if (a > 0 && !(v[a - 1] - t >= gz)) continue;
          if (!(next <= t)) continue;
          found = true;
          lo = t;
          if (a + f > 0) {
            // the nonzero edges are the a + f <= 3 largest, at the recorded
            // positions: load them once, refine the threshold over the free
            // ones in pair arithmetic and deposit (no further pass)
            int jr[3];
            float cr[3], ar[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              jr[i] = 0;
              cr[i] = ar[i] = 0.f;
              if (i < a + f) {
                const int el = sell_el(i == 0 ? i0 : (i == 1 ? i1 : i2), lane, w4);
                jr[i] = static_cast<int>(__ldg(col0 + el));
                V::get(__ldg(ca0 + el), cr[i], ar[i]);
              }
            }
            tau = t;
            taul = 0.f;
            if (f > 0) {
              F2 ps{0.f, 0.f};
#pragma unroll
              for (int i = 0; i < 3; ++i)
                if (i >= a && i < a + f) ps = f2_add(ps, u_pair(cr[i], ar[i], ys[jr[i]]));
              const F2 b = budget_pair(S, a);
              const F2 t2 = f2_threshold(ps, b.h, b.l, f);
              tau = t2.h;
              taul = t2.l;
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              if (i < a + f) {
                const F2 up = u_pair(cr[i], ar[i], ys[jr[i]]);
                const float x = fminf(fmaxf(((up.h - tau) + (up.l - taul)) * S.invg, 0.f), S.z);
                if (x > 0.f) deposit_b<V, STATS>(S, jr[i], cr[i], ar[i], x, accG, accC, accQ, ob);
              }
            }
            deposited = true;
          }
        }
      }
      for (int it = 0; it < 96 && !found; ++it) {
        bool newton = nfl > 0;
        float cand = newton ? __fdiv_rn(sfl + (static_cast<float>(nul) * gz - S.gch), static_cast<float>(nfl))
                            : 0.f;
        if (!(cand > lo && cand < hi)) {
          cand = 0.5f * (lo + hi);
          newton = false;
        }
        if (!(cand > lo && cand < hi)) break;  // the bracket is at float resolution
        int nf2, nu2;
        float sf2;
        sets_at(cand, nf2, nu2, sf2);
        if (newton && nf2 == nfl && nu2 == nul) {  // same piece: cand is its root
          lo = cand;
          break;
        }
        if (phi_g(cand, nf2, nu2, sf2) > 0.f) {
          lo = cand;
          nfl = nf2;
          nul = nu2;
          sfl = sf2;
        } else {
          hi = cand;
        }
      }
      // the threshold over the final free set in pair arithmetic
      F2 ps{0.f, 0.f};
      int n_f = 0, n_u = 0;
      if (!deposited) row_pass([&](int j, float c, float a) {
        const float y = ys[j];
        const float u = -fmaf(a, y, c);
        const float d = u - lo;
        if (d >= gz) {
          ++n_u;
        } else if (d > 0.f) {
          ++n_f;
          ps = f2_add(ps, u_pair(c, a, y));
        }
      });
      if (deposited) {
        // tau, taul set on the fast path
      } else if (n_f > 0) {
        const F2 b = budget_pair(S, n_u);
        const F2 t2 = f2_threshold(ps, b.h, b.l, n_f);
        tau = t2.h;
        taul = t2.l;
      } else {
        tau = lo;  // a flat piece: every x is 0 or z there
      }
    }
    // x = clip((u - tau) / gamma, 0, z) on the edges with u > tau
    if (!deposited) row_pass([&](int j, float c, float a) {
      const float y = ys[j];
      if (-fmaf(a, y, c) > tau) {
        const F2 up = u_pair(c, a, y);
        const float x = fminf(fmaxf(((up.h - tau) + (up.l - taul)) * S.invg, 0.f), S.z);
        if (x > 0.f) deposit_b<V, STATS>(S, j, c, a, x, accG, accC, accQ, ob);
      }
    });
  } else {
    tau = INFINITY;
  }
  if (STATS) {
    const int64_t u = 32 * s + lane;
    if (D.xout != nullptr && u < D.nusers) {
      // x in the caller's order, every edge of the user
      const int64_t o = __ldg(D.orig_off + u);
      const int d = __ldg(D.udeg + u);
      const uint64_t ld = __ldg(D.lead + u);  // slice position k is caller edge lead_caller_pos(ld, k, d)
      for (int k = 0; k < d; ++k) {
        const int el = sell_el(k, lane, w4);
        const int j = static_cast<int>(__ldg(col0 + el));
        float c, a;
        V::get(__ldg(ca0 + el), c, a);
        float x = 0.f;
        if (-fmaf(a, ys[j], c) > tau) {
          const F2 up = u_pair(c, a, ys[j]);
          x = fminf(fmaxf(((up.h - tau) + (up.l - taul)) * S.invg, 0.f), S.z);
        }
        D.xout[o + lead_caller_pos(ld, k, d)] = x;
      }
    }
    wobj += static_cast<double>(ob);
  } else {
    oq += fixp(ob, S.scaleO);  // the user's objective part, added exactly
  }
}

// Per CTA its tasks; certificate sweeps deal a task's slices to warps in a
// static order (first + stride (warp + k nw)), iteration sweeps from a
// per-CTA ticket counter.
template <class V, bool STATS>
__global__ void __launch_bounds__(kSweepThreads, 1)
    sweep_boxcut_kernel(const InstDesc* __restrict__ insts, const Task* __restrict__ tasks,
                        const int32_t* __restrict__ cta_task, int smemJ, int jlo, int jw,
                        const double* __restrict__ cuts) {
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
    const int nacc = STATS ? max(0, min(J - jlo, jw)) : J;
    for (int j = threadIdx.x; j < J; j += blockDim.x) ys[j] = sD.y[j];
    for (int j = threadIdx.x; j < nacc; j += blockDim.x) {
      accG[j] = 0ull;
      if (STATS) {
        accC[j] = 0ull;
        accQ[j] = 0ull;
      }
    }
    BSeg S;
    {
      const double g = *sD.gamma;
      S.gamma = static_cast<float>(g);
      S.invg = static_cast<float>(1.0 / g);
      S.z = sD.z;
      const double gz = g * static_cast<double>(sD.z);
      S.gzh = static_cast<float>(gz);
      S.gzl = static_cast<float>(gz - static_cast<double>(S.gzh));
      const double cut = cuts[inst];
      const double gc = g * cut;
      S.gch = static_cast<float>(gc);
      S.gcl = static_cast<float>(gc - static_cast<double>(S.gch));
      S.cut = static_cast<float>(cut);
      S.scaleG = sD.scaleG;
      S.scaleC = sD.scaleC;
      S.scaleQ = sD.scaleQ;
      S.scaleO = sD.scaleO;
      S.jlo = STATS ? jlo : 0;
      S.jw = nacc;
    }
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    double wobj = 0.0;
    unsigned long long oq = 0ull;
    for (int k = t; k < te; ++k) {
      const Task T = tasks[k];
      if (STATS) {
        // static order: the FP64 objective partials are summed in a fixed order
        const int64_t step = static_cast<int64_t>(T.stride) * nw;
        for (int64_t s = T.first + static_cast<int64_t>(T.stride) * warp; s < T.end; s += step)
          boxcut_slice<V, STATS>(sD, S, ys, accG, accC, accQ, s, wobj, oq);
      } else {
        // dynamic order within the CTA: rows whose threshold needs the
        // bracketed search take many passes, and the item sums are exact in
        // any order
        const int64_t nsl = (T.end - T.first + T.stride - 1) / T.stride;
        for (;;) {
          int64_t i = 0;
          if (lane == 0) i = static_cast<int64_t>(atomicAdd(&s_next, 1ull));
          i = __shfl_sync(kFull, i, 0);
          if (i >= nsl) break;
          boxcut_slice<V, STATS>(sD, S, ys, accG, accC, accQ, T.first + i * T.stride, wobj, oq);
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

template <class V>
cudaError_t prepare_values(int lim) {
  cudaError_t e = cudaFuncSetAttribute(&sweep_boxcut_kernel<V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       lim);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(&sweep_boxcut_kernel<V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <class V>
cudaError_t launch_values(const SweepLaunch& L, bool stats, const double* cuts) {
  const int th = L.threads > 0 ? L.threads : kSweepThreads;
  if (stats) {
    const int w = L.win > 0 ? std::min(L.win, L.smemJ) : L.smemJ;
    if (w < 1) return cudaErrorInvalidValue;
    const size_t sm = sweep_stats_smem_bytes(L.smemJ, w);
    for (int jlo = 0; jlo < L.smemJ || jlo == 0; jlo += w) {
      sweep_boxcut_kernel<V, true><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, jlo, w, cuts);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  sweep_boxcut_kernel<V, false><<<L.grid, th, sweep_smem_bytes(L.smemJ, false), L.stream>>>(
      L.inst, L.tasks, L.cta_task, L.smemJ, 0, L.smemJ, cuts);
  return cudaGetLastError();
}

}  // namespace

cudaError_t sweep_boxcut_prepare(bool bf16) {
  const int lim = static_cast<int>(sweep_smem_limit());
  return bf16 ? prepare_values<BF16Pair>(lim) : prepare_values<F32Pair>(lim);
}

cudaError_t launch_sweep_boxcut(const SweepLaunch& L, bool stats, bool bf16, const double* cuts) {
  if (cuts == nullptr) return cudaErrorInvalidValue;
  return bf16 ? launch_values<BF16Pair>(L, stats, cuts) : launch_values<F32Pair>(L, stats, cuts);
}

}  // namespace dlm
