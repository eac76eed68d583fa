// sweep_multi.cu -- the dual sweep for instances with m > 1 capacity families
// (Def. 1: every family has one diagonal block per user, so edge (i, j)
// carries one coefficient a_kij per family k).  For every user i and dual
// point y (m item vectors):
//     u_ij = -(c_ij + sum_k a_kij y_kj),   x_i = Proj_C_i(u_i / gamma),
// and per family and item (A_k x)_j = sum_i a_kij x_ij.
//
// Layout: the slices of sweep.cu (users sorted by degree, 32 per slice) with
// the (c, a_0) stream and, for k >= 1, one more stream of a_k in the same
// element order (a_ext + (k - 1) * ext_stride).  One lane per user, slices
// dealt to warps in a static order.  The projection follows sweep.cu: a
// streaming pass keeps the four largest u with the positions of the first
// three, rows with at most three active edges are finished from those
// positions, larger active sets take the Michelot iteration from tau_4; the
// threshold is recomputed over the active set in float-pair arithmetic
// (TwoSum / TwoProduct over the m products).
// Item sums are 64-bit fixed point in shared memory (one array per family),
// flushed once per CTA: exact and order independent.  This is the general
// path, kept apart from the one-family sweep so that the latter's code is
// unchanged.
#include <cuda_bf16.h>

#include "dlm_impl.cuh"
#include "sweep_common.cuh"

namespace dlm {
namespace {

constexpr int kMaxFam = kMaxFamilies;

__device__ __forceinline__ float ext_val(const void* base, int64_t el, bool bf16) {
  if (bf16) return __uint_as_float(static_cast<uint32_t>(__ldg(static_cast<const uint16_t*>(base) + el)) << 16);
  return __ldg(static_cast<const float*>(base) + el);
}

struct MSeg {
  float gamma, invg, gz, gzl, z;
  float scaleG, scaleC, scaleQ, scaleO;
  int kind, m, J;
};

// Whether family f (< M) is present: the two-family instantiation is used for
// m = 2 only, so there it is known at compile time.
template <int M>
__device__ __forceinline__ bool fam_on(const MSeg& S, int f) {
  return M == 2 ? true : f < S.m;
}

// Edge k of lane `lane` in the slice: item j, cost c, coefficients a[0..m).
// M is the compiled number of families (m <= M; the extra ones are 0).
template <class P, int M>
__device__ __forceinline__ void load_edge(const InstDesc& D, const MSeg& S, int64_t off, int k, int lane, int w4,
                                          bool bf16, int& j, float& c, float a[M]) {
  const int64_t el = off + sell_el(k, lane, w4);
  j = static_cast<int>(__ldg(D.col16 + el));
  P::get(__ldg(static_cast<const typename P::T*>(D.ca) + el), c, a[0]);
#pragma unroll
  for (int f = 1; f < M; ++f)
    a[f] = fam_on<M>(S, f) ? ext_val(D.a_ext, (f - 1) * D.ext_stride + el, bf16) : 0.f;
}

template <int M>
__device__ __forceinline__ float u_of(const MSeg& S, const float* ys, int j, float c, const float a[M]) {
  float t = c;
#pragma unroll
  for (int f = 0; f < M; ++f)
    if (fam_on<M>(S, f)) t = fmaf(a[f], ys[f * S.J + j], t);
  return -t;
}

// u = -(c + sum_f a_f y_f) as a float pair: every product is split exactly by
// FMA and the terms are added by TwoSum.
template <int M>
__device__ __forceinline__ F2 u_pair_m(const MSeg& S, const float* ys, int j, float c, const float a[M]) {
  F2 s{-c, 0.f};
#pragma unroll
  for (int f = 0; f < M; ++f) {
    if (fam_on<M>(S, f)) {
      const float y = ys[f * S.J + j];
      const float p = a[f] * y;
      const float pe = fmaf(a[f], y, -p);
      s = f2_add(s, F2{-p, -pe});
    }
  }
  return s;
}

// Four consecutive coefficients of an extra family's stream (element index
// 4 q .. 4 q + 3 from the slice start; 8- or 16-byte aligned).
__device__ __forceinline__ void ext_get4(const void* base, int q, bool bf16, float v[4]) {
  if (bf16) {
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(base) + q);
    v[0] = __uint_as_float(w.x << 16);
    v[1] = __uint_as_float(w.x & 0xffff0000u);
    v[2] = __uint_as_float(w.y << 16);
    v[3] = __uint_as_float(w.y & 0xffff0000u);
  } else {
    const float4 w = __ldg(reinterpret_cast<const float4*>(base) + q);
    v[0] = w.x, v[1] = w.y, v[2] = w.z, v[3] = w.w;
  }
}

template <bool STATS, int M>
__device__ __forceinline__ void deposit_m(const MSeg& S, int j, float c, const float a[M], float x,
                                          unsigned long long* accG, unsigned long long* accC,
                                          unsigned long long* accQ, float& ob) {
#pragma unroll
  for (int f = 0; f < M; ++f)
    if (fam_on<M>(S, f)) atomicAdd(&accG[f * S.J + j], fixp(a[f] * x, S.scaleG));
  if (STATS) {
    atomicAdd(&accC[j], fixp(c * x, S.scaleC));
    atomicAdd(&accQ[j], fixp(x * x, S.scaleQ));
  }
  ob += fmaf(0.5f * S.gamma * x, x, c * x);
}

__device__ __forceinline__ float x_of(const MSeg& S, bool box, float tau, float taul, F2 up) {
  if (box) return fminf(fmaxf(((up.h - tau) + (up.l - taul)) * S.invg, 0.f), S.z);
  return fmaxf((up.h - tau) + (up.l - taul), 0.f) * S.invg;
}

// One slice.  The first pass streams the row in groups of four edges (128-
// and 64-bit loads) and keeps its four largest u with the positions of the
// first three, as in sweep.cu: at most three active edges (mode 1, 2) are
// then handled from those positions; four or more (mode 3), and the box, take
// the Michelot iteration and full passes.
template <class P, bool STATS, int M>
__device__ __forceinline__ void multi_slice(const InstDesc& D, const MSeg& S, const float* __restrict__ ys,
                                            unsigned long long* accG, unsigned long long* accC,
                                            unsigned long long* accQ, int64_t s, bool bf16, double& wobj,
                                            unsigned long long& oq) {
  const int lane = threadIdx.x & 31;
  const int64_t off = __ldg(D.slice_off + s);
  const int w = __ldg(D.slice_w + s);
  const int w4 = w >> 2;
  const bool box = S.kind == DLM_BOX;
  const bool eq = S.kind == DLM_SIMPLEX_EQ;
  const uint16_t* __restrict__ col0 = D.col16 + off;
  const typename P::T* __restrict__ ca0 = static_cast<const typename P::T*>(D.ca) + off;
  const size_t vs = bf16 ? 2 : 4;
  auto ext0 = [&](int f) {
    return static_cast<const char*>(D.a_ext) + vs * ((f - 1) * D.ext_stride + off);
  };

  float v0 = -INFINITY, v1 = -INFINITY, v2 = -INFINITY, v3 = -INFINITY;
  int i0 = 0, i1 = 0, i2 = 0;
  // Groups of four edges.  With two families, two groups' loads are issued
  // together and a group is inserted only if some lane's largest value of the
  // group tops its fourth largest (otherwise the insertions change no record:
  // strict comparisons) -- most groups after the first, the rows'
  // lowest-cost edges coming first (lead order, layout.cu).  With more
  // families the chunk's registers would spill: one group at a time, all
  // inserted.
  struct Grp {
    uint2 jv;  // four 16-bit item indices
    float c[4], a[M][4];
  };
  auto load = [&](int g) {
    Grp r;
    const int q = 32 * g + lane;
    r.jv = __ldg(reinterpret_cast<const uint2*>(col0) + q);
    P::get4(ca0, q, r.c, r.a[0]);
#pragma unroll
    for (int f = 1; f < M; ++f)
      if (fam_on<M>(S, f)) ext_get4(ext0(f), q, bf16, r.a[f]);
    return r;
  };
  auto insert = [&](int g, const Grp& r) {
    const int jj[4] = {static_cast<int>(r.jv.x & 0xffffu), static_cast<int>(r.jv.x >> 16),
                       static_cast<int>(r.jv.y & 0xffffu), static_cast<int>(r.jv.y >> 16)};
    float u[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float t = r.c[e];
#pragma unroll
      for (int f = 0; f < M; ++f)
        if (fam_on<M>(S, f)) t = fmaf(r.a[f][e], ys[f * S.J + jj[e]], t);
      u[e] = -t;
    }
    const float m4 = fmaxf(fmaxf(u[0], u[1]), fmaxf(u[2], u[3]));
    if (M > 2 || __any_sync(kFull, m4 > v3)) {
#pragma unroll
      for (int e = 0; e < 4; ++e) top4_insert(u[e], 4 * g + e, v0, v1, v2, v3, i0, i1, i2);
    }
  };
  int g = 0;
  if (M <= 2) {
    for (; g + 2 <= w4; g += 2) {
      const Grp r0 = load(g), r1 = load(g + 1);
      insert(g, r0);
      insert(g + 1, r1);
    }
  }
  for (; g < w4; ++g) insert(g, load(g));
  int j;
  float c, a[M];
  for (int k = 4 * w4; k < w; ++k) {
    load_edge<P, M>(D, S, off, k, lane, w4, bf16, j, c, a);
    top4_insert(u_of<M>(S, ys, j, c, a), k, v0, v1, v2, v3, i0, i1, i2);
  }

  // mode 0: nothing active; 1: the maximum alone, x = z; 2: r <= 3 active
  // edges at the recorded positions; 3: iterate (and the box)
  int mode;
  int r = 0;
  float tau = 0.f, taul = 0.f;
  if (box) {
    mode = v0 > 0.f ? 3 : 0;
  } else if (v0 == -INFINITY || (!eq && v0 <= 0.f)) {
    mode = 0;
  } else {
    float sm = v0;
    r = 1;
    tau = v0 - S.gz;
    if (v1 > tau) {
      sm += v1;
      r = 2;
      tau = __fdiv_rn(sm - S.gz, 2.f);
      if (v2 > tau) {
        sm += v2;
        r = 3;
        tau = __fdiv_rn(sm - S.gz, 3.f);
        if (v3 > tau) {
          sm += v3;
          r = 4;
          tau = __fdiv_rn(sm - S.gz, 4.f);
        }
      }
    }
    mode = (r == 1 && (eq || tau >= 0.f)) ? 1 : (r < 4 ? 2 : 3);
  }
  float ob = 0.f;
  bool zero = box;
  if (mode == 1) {
    load_edge<P, M>(D, S, off, i0, lane, w4, bf16, j, c, a);
    deposit_m<STATS, M>(S, j, c, a, S.z, accG, accC, accQ, ob);
  } else if (mode == 2) {
    zero = !eq && tau <= 0.f;
    if (!zero) {
      F2 sum{0.f, 0.f};
      for (int i = 0; i < r; ++i) {
        load_edge<P, M>(D, S, off, i == 0 ? i0 : (i == 1 ? i1 : i2), lane, w4, bf16, j, c, a);
        sum = f2_add(sum, u_pair_m<M>(S, ys, j, c, a));
      }
      const F2 t2 = f2_threshold(sum, S.gz, S.gzl, r);
      if (!eq && t2.h + t2.l <= 0.f) {
        zero = true;
      } else {
        tau = t2.h;
        taul = t2.l;
      }
    }
    if (zero) tau = taul = 0.f;
    for (int i = 0; i < r; ++i) {
      load_edge<P, M>(D, S, off, i == 0 ? i0 : (i == 1 ? i1 : i2), lane, w4, bf16, j, c, a);
      const float x = x_of(S, false, tau, taul, u_pair_m<M>(S, ys, j, c, a));
      if (x > 0.f) deposit_m<STATS, M>(S, j, c, a, x, accG, accC, accQ, ob);
    }
  } else if (mode == 3) {
    if (!box) {
      // Michelot iteration from tau_4, a lower bound of the threshold
      int prevn = -1;
      for (int it = 0; it < 256; ++it) {
        float sm = 0.f;
        int n = 0;
        for (int k = 0; k < w; ++k) {
          load_edge<P, M>(D, S, off, k, lane, w4, bf16, j, c, a);
          const float u = u_of<M>(S, ys, j, c, a);
          if (u > tau) {
            sm += u;
            ++n;
          }
        }
        if (n == prevn || n == 0) break;
        prevn = n;
        const float tn = __fdiv_rn(sm - S.gz, static_cast<float>(n));
        if (tn == tau) break;
        tau = tn;
      }
      zero = !eq && tau <= 0.f;
      if (!zero) {
        F2 sum{0.f, 0.f};
        int n = 0;
        for (int k = 0; k < w; ++k) {
          load_edge<P, M>(D, S, off, k, lane, w4, bf16, j, c, a);
          if (u_of<M>(S, ys, j, c, a) > tau) {
            sum = f2_add(sum, u_pair_m<M>(S, ys, j, c, a));
            ++n;
          }
        }
        const F2 t2 = f2_threshold(sum, S.gz, S.gzl, n > 0 ? n : 1);
        if (!eq && t2.h + t2.l <= 0.f) {
          zero = true;
        } else {
          tau = t2.h;
          taul = t2.l;
        }
      }
    }
    if (zero) tau = taul = 0.f;
    for (int k = 0; k < w; ++k) {
      load_edge<P, M>(D, S, off, k, lane, w4, bf16, j, c, a);
      if (u_of<M>(S, ys, j, c, a) > tau) {
        const float x = x_of(S, box, tau, taul, u_pair_m<M>(S, ys, j, c, a));
        if (x > 0.f) deposit_m<STATS, M>(S, j, c, a, x, accG, accC, accQ, ob);
      }
    }
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
          x = k == i0 ? S.z : 0.f;
        } else if (mode >= 2) {
          load_edge<P, M>(D, S, off, k, lane, w4, bf16, j, c, a);
          if (u_of<M>(S, ys, j, c, a) > tau) x = x_of(S, box, tau, taul, u_pair_m<M>(S, ys, j, c, a));
        }
        D.xout[o + lead_caller_pos(ld, k, d)] = x;
      }
    }
    wobj += static_cast<double>(ob);
  } else {
    oq += fixp(ob, S.scaleO);  // the users' objective parts, added exactly
  }
}

// Shared memory: accG [m smemJ], then (STATS) accC, accQ [smemJ each], then
// ys [m smemJ] floats, then 32 doubles of warp partials.
template <class P, bool STATS, int M>
__global__ void __launch_bounds__(kSweepThreads, 1)
    sweep_multi_kernel(const InstDesc* __restrict__ insts, const Task* __restrict__ tasks,
                       const int32_t* __restrict__ cta_task, int smemJ, int m, bool bf16) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* accG = reinterpret_cast<unsigned long long*>(smem_raw);
  unsigned long long* accC = accG + static_cast<size_t>(m) * smemJ;
  unsigned long long* accQ = accC + smemJ;
  float* ys = reinterpret_cast<float*>(accG + static_cast<size_t>(m + (STATS ? 2 : 0)) * smemJ);
  double* wsum = reinterpret_cast<double*>(ys + ((static_cast<size_t>(m) * smemJ + 1) & ~static_cast<size_t>(1)));

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
    const int mJ = sD.m * J;
    for (int q = threadIdx.x; q < mJ; q += blockDim.x) {
      ys[q] = sD.y[q];  // family-major, as the dual vector
      accG[q] = 0ull;
    }
    if (STATS)
      for (int j = threadIdx.x; j < J; j += blockDim.x) accC[j] = accQ[j] = 0ull;
    MSeg S;
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
      S.scaleO = sD.scaleO;
      S.kind = sD.kind;
      S.m = sD.m;
      S.J = J;
    }
    __syncthreads();
    double wobj = 0.0;
    unsigned long long oq = 0ull;
    for (int k = t; k < te; ++k) {
      const Task T = tasks[k];
      if (STATS) {
        // static order: the FP64 objective partials are summed in a fixed order
        const int64_t step = static_cast<int64_t>(T.stride) * nw;
        for (int64_t s = T.first + static_cast<int64_t>(T.stride) * warp; s < T.end; s += step)
          multi_slice<P, STATS, M>(sD, S, ys, accG, accC, accQ, s, bf16, wobj, oq);
      } else {
        // dynamic order within the CTA (the item sums are exact)
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
        const int64_t nsl = (T.end - T.first + T.stride - 1) / T.stride;
        for (;;) {
          int64_t i = 0;
          if (lane == 0) i = static_cast<int64_t>(atomicAdd(&s_next, 1ull));
          i = __shfl_sync(kFull, i, 0);
          if (i >= nsl) break;
          multi_slice<P, STATS, M>(sD, S, ys, accG, accC, accQ, T.first + i * T.stride, bf16, wobj, oq);
        }
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
    for (int q = threadIdx.x; q < mJ; q += blockDim.x) {
      const unsigned long long v = accG[q];
      if (v) atomicAdd(sD.acc + q, v);
    }
    if (STATS) {
      for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const unsigned long long vc = accC[j], vq = accQ[j];
        if (vc) atomicAdd(sD.accC + j, vc);
        if (vq) atomicAdd(sD.accQ + j, vq);
      }
      if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < nw; ++w) sum += wsum[w];
        sD.seg_obj[t] = sum;
      }
    }
    __syncthreads();
    t = te;
  }
}

}  // namespace

size_t sweep_multi_smem_bytes(int smemJ, int m, bool stats) {
  const size_t J = static_cast<size_t>(smemJ), M = static_cast<size_t>(m);
  return (M + (stats ? 2 : 0)) * J * 8 + ((M * J + 1) & ~static_cast<size_t>(1)) * 4 + 32 * 8;
}

namespace {

template <class P, int M>
cudaError_t prepare_m(int lim) {
  cudaError_t e =
      cudaFuncSetAttribute(&sweep_multi_kernel<P, false, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(&sweep_multi_kernel<P, true, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <class P, int M>
cudaError_t launch_m(const SweepLaunch& L, bool stats, bool bf16) {
  const size_t sm = sweep_multi_smem_bytes(L.smemJ, L.fam, stats);
  const int th = L.threads > 0 ? L.threads : kSweepThreads;
  if (stats)
    sweep_multi_kernel<P, true, M><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, L.fam, bf16);
  else
    sweep_multi_kernel<P, false, M><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, L.fam, bf16);
  return cudaGetLastError();
}

}  // namespace

// Two families have their own instantiation; three and four share one.
cudaError_t sweep_multi_prepare(bool bf16) {
  const int lim = static_cast<int>(sweep_smem_limit());
  cudaError_t e = bf16 ? prepare_m<BF16Pair, 2>(lim) : prepare_m<F32Pair, 2>(lim);
  if (e != cudaSuccess) return e;
  return bf16 ? prepare_m<BF16Pair, kMaxFam>(lim) : prepare_m<F32Pair, kMaxFam>(lim);
}

cudaError_t launch_sweep_multi(const SweepLaunch& L, bool stats, bool bf16) {
  if (L.fam <= 2) return bf16 ? launch_m<BF16Pair, 2>(L, stats, bf16) : launch_m<F32Pair, 2>(L, stats, bf16);
  return bf16 ? launch_m<BF16Pair, kMaxFam>(L, stats, bf16) : launch_m<F32Pair, kMaxFam>(L, stats, bf16);
}

}  // namespace dlm
