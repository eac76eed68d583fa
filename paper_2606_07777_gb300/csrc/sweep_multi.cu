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
// dealt to warps in a static order.  The projection takes the exact threshold
// by the Michelot iteration from max(u) - gamma z (monotone from below), then
// recomputes it over the active set in float-pair arithmetic (TwoSum /
// TwoProduct over the m products), as sweep.cu does for large active sets.
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
  float scaleG, scaleC, scaleQ;
  int kind, m, J;
};

// Edge k of lane `lane` in the slice: item j, cost c, coefficients a[0..m).
template <class P>
__device__ __forceinline__ void load_edge(const InstDesc& D, const MSeg& S, int64_t off, int k, int lane, int w4,
                                          bool bf16, int& j, float& c, float a[kMaxFam]) {
  const int64_t el = off + sell_el(k, lane, w4);
  j = __ldg(D.col + el);
  P::get(__ldg(static_cast<const typename P::T*>(D.ca) + el), c, a[0]);
#pragma unroll
  for (int f = 1; f < kMaxFam; ++f)
    a[f] = f < S.m ? ext_val(D.a_ext, (f - 1) * D.ext_stride + el, bf16) : 0.f;
}

__device__ __forceinline__ float u_of(const MSeg& S, const float* ys, int j, float c, const float a[kMaxFam]) {
  float t = c;
#pragma unroll
  for (int f = 0; f < kMaxFam; ++f)
    if (f < S.m) t = fmaf(a[f], ys[f * S.J + j], t);
  return -t;
}

// u = -(c + sum_f a_f y_f) as a float pair: every product is split exactly by
// FMA and the terms are added by TwoSum.
__device__ __forceinline__ F2 u_pair_m(const MSeg& S, const float* ys, int j, float c, const float a[kMaxFam]) {
  F2 s{-c, 0.f};
#pragma unroll
  for (int f = 0; f < kMaxFam; ++f) {
    if (f < S.m) {
      const float y = ys[f * S.J + j];
      const float p = a[f] * y;
      const float pe = fmaf(a[f], y, -p);
      s = f2_add(s, F2{-p, -pe});
    }
  }
  return s;
}

template <class P, bool STATS>
__device__ __forceinline__ void multi_slice(const InstDesc& D, const MSeg& S, const float* __restrict__ ys,
                                            unsigned long long* accG, unsigned long long* accC,
                                            unsigned long long* accQ, int64_t s, bool bf16, double& wobj) {
  const int lane = threadIdx.x & 31;
  const int64_t off = __ldg(D.slice_off + s);
  const int w = __ldg(D.slice_w + s);
  const int w4 = w >> 2;
  const bool box = S.kind == DLM_BOX;
  const bool eq = S.kind == DLM_SIMPLEX_EQ;
  int j;
  float c, a[kMaxFam];
  float m1 = -INFINITY;
  for (int k = 0; k < w; ++k) {
    load_edge<P>(D, S, off, k, lane, w4, bf16, j, c, a);
    m1 = fmaxf(m1, u_of(S, ys, j, c, a));
  }
  float tau = 0.f, taul = 0.f;
  bool active = m1 != -INFINITY && (box || eq || m1 > 0.f);
  if (active && !box) {
    // Michelot iteration from m1 - gamma z
    tau = m1 - S.gz;
    int prevn = -1;
    for (int it = 0; it < 256; ++it) {
      float sm = 0.f;
      int n = 0;
      for (int k = 0; k < w; ++k) {
        load_edge<P>(D, S, off, k, lane, w4, bf16, j, c, a);
        const float u = u_of(S, ys, j, c, a);
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
    bool zero = !eq && tau <= 0.f;
    if (!zero) {
      F2 sum{0.f, 0.f};
      int n = 0;
      for (int k = 0; k < w; ++k) {
        load_edge<P>(D, S, off, k, lane, w4, bf16, j, c, a);
        if (u_of(S, ys, j, c, a) > tau) {
          sum = f2_add(sum, u_pair_m(S, ys, j, c, a));
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
    if (zero) tau = taul = 0.f;
  }
  float ob = 0.f;
  const int64_t u = 32 * s + lane;
  const bool write_x = STATS && D.xout != nullptr && u < D.nusers;
  const int64_t o = write_x ? __ldg(D.orig_off + u) : 0;
  const int d = write_x ? __ldg(D.udeg + u) : 0;
  for (int k = 0; k < w; ++k) {
    load_edge<P>(D, S, off, k, lane, w4, bf16, j, c, a);
    float x = 0.f;
    if (active && u_of(S, ys, j, c, a) > tau) {
      const F2 up = u_pair_m(S, ys, j, c, a);
      x = box ? fminf(fmaxf(((up.h - tau) + (up.l - taul)) * S.invg, 0.f), S.z)
              : fmaxf((up.h - tau) + (up.l - taul), 0.f) * S.invg;
    }
    if (x > 0.f) {
#pragma unroll
      for (int f = 0; f < kMaxFam; ++f)
        if (f < S.m) atomicAdd(&accG[f * S.J + j], fixp(a[f] * x, S.scaleG));
      if (STATS) {
        atomicAdd(&accC[j], fixp(c * x, S.scaleC));
        atomicAdd(&accQ[j], fixp(x * x, S.scaleQ));
        ob += fmaf(0.5f * S.gamma * x, x, c * x);
      }
    }
    if (write_x && k < d) D.xout[o + k] = x;
  }
  if (STATS) wobj += static_cast<double>(ob);
}

// Shared memory: accG [m smemJ], then (STATS) accC, accQ [smemJ each], then
// ys [m smemJ] floats, then 32 doubles of warp partials.
template <class P, bool STATS>
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
      S.kind = sD.kind;
      S.m = sD.m;
      S.J = J;
    }
    __syncthreads();
    double wobj = 0.0;
    for (int k = t; k < te; ++k) {
      const Task T = tasks[k];
      const int64_t step = static_cast<int64_t>(T.stride) * nw;
      for (int64_t s = T.first + static_cast<int64_t>(T.stride) * warp; s < T.end; s += step)
        multi_slice<P, STATS>(sD, S, ys, accG, accC, accQ, s, bf16, wobj);
    }
    if (STATS) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wobj += __shfl_xor_sync(kFull, wobj, o);
      if (lane == 0) wsum[warp] = wobj;
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

cudaError_t sweep_multi_prepare(bool bf16) {
  const int lim = static_cast<int>(sweep_smem_limit());
  cudaError_t e;
  if (bf16) {
    e = cudaFuncSetAttribute(&sweep_multi_kernel<BF16Pair, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(&sweep_multi_kernel<BF16Pair, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               lim);
  } else {
    e = cudaFuncSetAttribute(&sweep_multi_kernel<F32Pair, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(&sweep_multi_kernel<F32Pair, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  }
  return e;
}

cudaError_t launch_sweep_multi(const SweepLaunch& L, bool stats, bool bf16) {
  const size_t sm = sweep_multi_smem_bytes(L.smemJ, L.fam, stats);
  const int th = L.threads > 0 ? L.threads : kSweepThreads;
  if (bf16) {
    if (stats)
      sweep_multi_kernel<BF16Pair, true><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, L.fam,
                                                                        true);
    else
      sweep_multi_kernel<BF16Pair, false><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, L.fam,
                                                                         true);
  } else {
    if (stats)
      sweep_multi_kernel<F32Pair, true><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, L.fam,
                                                                       false);
    else
      sweep_multi_kernel<F32Pair, false><<<L.grid, th, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ, L.fam,
                                                                        false);
  }
  return cudaGetLastError();
}

}  // namespace dlm
