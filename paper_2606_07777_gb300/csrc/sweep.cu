// sweep.cu -- the fused dual sweep (the per-iteration hot path).
//
// For every user i and dual point y (Sec. 3.2, Eq. primal-recovery):
//     u_ik  = -(c_ik + a_ik * y_j(k))                      (gamma-scaled v)
//     x_i   = Proj_C_i(u_i / gamma)
// and per item j (Eq. dual-gradient):  (A x)_j = sum_i a_ij x_ij.
// With `STATS` it also accumulates per item sum c x and sum x^2 and the
// objective sum (c x + gamma/2 x^2) for the dual value and the certified gap,
// and optionally writes x in the caller's edge order.
//
// Simplex projection (Sec. 4.3 computes the same threshold with a sort; here
// no sort): in u-space the threshold tau solves sum max(u - tau, 0) = gamma z.
// Start from tau_1 = max(u) - gamma z, a lower bound on tau, and iterate
// tau <- (sum_{u > tau} u - gamma z) / #{u > tau} (Michelot 1986; the
// iteration is monotone from below and stops when the active set stops
// changing).  The inequality simplex then takes max(tau, 0), which equals the
// early exit of Sec. 4.3 (sum max(u, 0) <= gamma z gives tau = 0).
// x = max(u - tau, 0) / gamma.  Box: x = clip(u / gamma, 0, z).
//
// Work layout: users are grouped by degree class; a task is one class's
// slice of one CTA; a warp pass covers 32/L users of a class with L lanes per
// user and K edges per lane (register resident), or one user per warp with a
// streamed row for long rows.  Passes of a CTA are dealt to its warps
// round-robin, so every accumulation below has a fixed order.
//
// Determinism: item sums are accumulated in 64-bit fixed point (value *
// 2^s rounded to an integer, s chosen at set-up so no item sum can overflow),
// so the sum is exact and independent of the order in which atomics land.
// The objective is summed per warp in FP64 in pass order, per CTA in warp
// order, and across CTAs in task order by the statistics kernel.
#include <cuda_bf16.h>

#include "dlm_impl.cuh"

namespace dlm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxSegTasks = kNumClasses;

__device__ __forceinline__ float ld_val(const float* p, int64_t e) { return __ldg(p + e); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16* p, int64_t e) {
  const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + e);
  return __uint_as_float(static_cast<unsigned>(b) << 16);
}

template <int L>
__device__ __forceinline__ float sub_max(float v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
template <int L>
__device__ __forceinline__ float sub_sum(float v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
template <int L>
__device__ __forceinline__ int sub_sumi(int v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long fixp(float v, float scale) {
  return static_cast<unsigned long long>(__float2ll_rn(v * scale));
}

// Unevaluated float pairs (hi + lo) for the few active edges of a user: the
// error-free transformations TwoSum (Knuth) and TwoProduct by FMA make
// u = -(c + a y) and the threshold tau exact to ~2^-48 relative, so
// x = (u - tau) / gamma keeps full FP32 relative accuracy even when u and tau
// nearly cancel (small gamma).
struct F2 {
  float h, l;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return {s, (a - (s - bp)) + (b - bp)};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const F2 s = two_sum(a.h, b.h);
  return {s.h, s.l + (a.l + b.l)};
}
// u = -(c + a*y) as a pair: a*y = p + pe exactly (FMA), then -c - p by TwoSum.
__device__ __forceinline__ F2 u_pair(float c, float a, float y) {
  const float p = a * y;
  const float pe = fmaf(a, y, -p);
  const F2 s = two_sum(-c, -p);
  return {s.h, s.l - pe};
}
// (sum - gz) / n for a pair sum; the FP32 quotient's remainder is exact by FMA.
__device__ __forceinline__ F2 f2_threshold(F2 sum, float gzh, float gzl, int n) {
  const F2 num = f2_add(sum, F2{-gzh, -gzl});
  const float fn = static_cast<float>(n);
  const float th = __fdiv_rn(num.h, fn);
  const float r = fmaf(-th, fn, num.h);
  return {th, __fdiv_rn(r + num.l, fn)};
}

struct Seg {
  float gamma, invg, gz, gzl, z;
  float scaleG, scaleC, scaleQ;
  int kind;
};

// One warp pass of a register mapping: users [uf, uf + 32/L) (clipped at ue),
// L lanes per user, K edges per lane (edge sl + k*L of the row).
template <int L, int K, typename VT, bool STATS>
__device__ __forceinline__ void pass_reg(const InstDesc& D, const Seg& S, const float* __restrict__ ys,
                                         unsigned long long* accG, unsigned long long* accC,
                                         unsigned long long* accQ, int64_t uf, int64_t ue, double& wobj) {
  const int lane = threadIdx.x & 31;
  const int sl = lane & (L - 1);
  const int64_t u = uf + lane / L;
  int64_t s = 0;
  int d = 0;
  if (u < ue) {
    s = __ldg(D.rp + u);
    d = static_cast<int>(__ldg(D.rp + u + 1) - s);
  }
  const VT* __restrict__ cp = static_cast<const VT*>(D.c);
  const VT* __restrict__ ap = static_cast<const VT*>(D.a);
  int cj[K];
  float cv[K], av[K], uu[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int idx = sl + k * L;
    if (idx < d) {
      const int64_t e = s + idx;
      cj[k] = __ldg(D.col + e);
      cv[k] = ld_val(cp, e);
      av[k] = ld_val(ap, e);
    } else {
      cj[k] = -1;
      cv[k] = 0.f;
      av[k] = 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) uu[k] = (cj[k] >= 0) ? -fmaf(av[k], ys[cj[k]], cv[k]) : -INFINITY;

  float tau = 0.f, taul = 0.f;
  if (S.kind != DLM_BOX) {
    const bool eq = S.kind == DLM_SIMPLEX_EQ;
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < K; ++k) m = fmaxf(m, uu[k]);
    m = sub_max<L>(m);
    const bool trivial = (d == 0) || (!eq && m <= 0.f);
    bool done = trivial;
    tau = m - S.gz;
    int prevn = -1;
    for (int it = 0; it < L * K + 2; ++it) {
      if (!__any_sync(kFull, !done)) break;
      float sm = 0.f;
      int n = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (uu[k] > tau) {
          sm += uu[k];
          ++n;
        }
      }
      sm = sub_sum<L>(sm);
      n = sub_sumi<L>(n);
      if (!done) {
        if (n == prevn || n == 0) {
          done = true;
        } else {
          prevn = n;
          const float tn = __fdiv_rn(sm - S.gz, static_cast<float>(n));
          done = (tn == tau);
          tau = tn;
        }
      }
    }
    // Refine tau over the active set {u > tau} in pair arithmetic.  The
    // shuffles run on every lane (warp-uniform); `zero` is uniform per user.
    const bool zero = trivial || (!eq && tau <= 0.f);
    F2 sum{0.f, 0.f};
    int n = 0;
    if (!zero) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (uu[k] > tau) {
          sum = f2_add(sum, u_pair(cv[k], av[k], ys[cj[k]]));
          ++n;
        }
      }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
      const F2 other{__shfl_xor_sync(kFull, sum.h, o), __shfl_xor_sync(kFull, sum.l, o)};
      sum = f2_add(sum, other);
      n += __shfl_xor_sync(kFull, n, o);
    }
    const F2 t2 = f2_threshold(sum, S.gz, S.gzl, n > 0 ? n : 1);
    if (zero || (!eq && t2.h + t2.l <= 0.f)) {
      tau = 0.f;
    } else {
      tau = t2.h;
      taul = t2.l;
    }
  }

  float ob = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float x = 0.f;
    if (cj[k] >= 0) {
      if (S.kind == DLM_BOX) {
        if (uu[k] > 0.f) {
          const F2 up = u_pair(cv[k], av[k], ys[cj[k]]);
          x = fminf((up.h + up.l) * S.invg, S.z);
        }
      } else if (uu[k] > tau) {
        const F2 up = u_pair(cv[k], av[k], ys[cj[k]]);
        x = fmaxf((up.h - tau) + (up.l - taul), 0.f) * S.invg;
      }
    }
    if (x > 0.f) {
      atomicAdd(&accG[cj[k]], fixp(av[k] * x, S.scaleG));
      if (STATS) {
        atomicAdd(&accC[cj[k]], fixp(cv[k] * x, S.scaleC));
        atomicAdd(&accQ[cj[k]], fixp(x * x, S.scaleQ));
        ob += fmaf(0.5f * S.gamma * x, x, cv[k] * x);
      }
    }
    if (STATS && D.xout != nullptr) {
      const int idx = sl + k * L;
      if (idx < d) D.xout[__ldg(D.orig_off + u) + idx] = x;
    }
  }
  if (STATS) {
    ob = sub_sum<L>(ob);
    if (sl == 0 && d > 0) wobj += static_cast<double>(ob);
  }
}

__device__ __forceinline__ float warp_max(float v) { return sub_max<32>(v); }
__device__ __forceinline__ float warp_sum(float v) { return sub_sum<32>(v); }
__device__ __forceinline__ int warp_sumi(int v) { return sub_sumi<32>(v); }

// One user of any degree, one warp, the row streamed from memory in every
// pass of the threshold iteration (rows here are long and rare).
template <typename VT, bool STATS>
__device__ __forceinline__ void pass_stream(const InstDesc& D, const Seg& S, const float* __restrict__ ys,
                                            unsigned long long* accG, unsigned long long* accC,
                                            unsigned long long* accQ, int64_t u, double& wobj) {
  const int lane = threadIdx.x & 31;
  const int64_t s = __ldg(D.rp + u);
  const int64_t d = __ldg(D.rp + u + 1) - s;
  const VT* __restrict__ cp = static_cast<const VT*>(D.c);
  const VT* __restrict__ ap = static_cast<const VT*>(D.a);
  float tau = 0.f, taul = 0.f;
  if (S.kind != DLM_BOX && d > 0) {
    const bool eq = S.kind == DLM_SIMPLEX_EQ;
    float m = -INFINITY;
    for (int64_t i = lane; i < d; i += 32) {
      const int64_t e = s + i;
      m = fmaxf(m, -fmaf(ld_val(ap, e), ys[__ldg(D.col + e)], ld_val(cp, e)));
    }
    m = warp_max(m);
    if (eq || m > 0.f) {
      tau = m - S.gz;
      int prevn = -1;
      for (int it = 0; it < 256; ++it) {
        float sm = 0.f;
        int n = 0;
        for (int64_t i = lane; i < d; i += 32) {
          const int64_t e = s + i;
          const float uv = -fmaf(ld_val(ap, e), ys[__ldg(D.col + e)], ld_val(cp, e));
          if (uv > tau) {
            sm += uv;
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
      if (!eq && tau <= 0.f) {
        tau = 0.f;
      } else {
        F2 sum{0.f, 0.f};
        int n = 0;
        for (int64_t i = lane; i < d; i += 32) {
          const int64_t e = s + i;
          const int j = __ldg(D.col + e);
          const float cv = ld_val(cp, e), av = ld_val(ap, e);
          if (-fmaf(av, ys[j], cv) > tau) {
            sum = f2_add(sum, u_pair(cv, av, ys[j]));
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
        if (!eq && t2.h + t2.l <= 0.f) {
          tau = 0.f;
        } else {
          tau = t2.h;
          taul = t2.l;
        }
      }
    } else {
      tau = 0.f;
    }
  }
  float ob = 0.f;
  const int64_t off = (STATS && D.xout != nullptr) ? __ldg(D.orig_off + u) : 0;
  for (int64_t i = lane; i < d; i += 32) {
    const int64_t e = s + i;
    const int j = __ldg(D.col + e);
    const float cv = ld_val(cp, e), av = ld_val(ap, e);
    const float uv = -fmaf(av, ys[j], cv);
    float x = 0.f;
    if (S.kind == DLM_BOX) {
      if (uv > 0.f) {
        const F2 up = u_pair(cv, av, ys[j]);
        x = fminf((up.h + up.l) * S.invg, S.z);
      }
    } else if (uv > tau) {
      const F2 up = u_pair(cv, av, ys[j]);
      x = fmaxf((up.h - tau) + (up.l - taul), 0.f) * S.invg;
    }
    if (x > 0.f) {
      atomicAdd(&accG[j], fixp(av * x, S.scaleG));
      if (STATS) {
        atomicAdd(&accC[j], fixp(cv * x, S.scaleC));
        atomicAdd(&accQ[j], fixp(x * x, S.scaleQ));
        ob += fmaf(0.5f * S.gamma * x, x, cv * x);
      }
    }
    if (STATS && D.xout != nullptr) D.xout[off + i] = x;
  }
  if (STATS) {
    ob = warp_sum(ob);
    if (lane == 0 && d > 0) wobj += static_cast<double>(ob);
  }
}

template <typename VT, bool STATS>
__global__ void __launch_bounds__(kSweepThreads, 2)
    sweep_kernel(const InstDesc* __restrict__ insts, const Task* __restrict__ tasks,
                 const int32_t* __restrict__ cta_task, int smemJ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* accG = reinterpret_cast<unsigned long long*>(smem_raw);
  unsigned long long* accC = accG + smemJ;
  unsigned long long* accQ = accC + smemJ;
  float* ys = reinterpret_cast<float*>(accG + (STATS ? 3 : 1) * static_cast<size_t>(smemJ));
  double* wsum = reinterpret_cast<double*>(ys + ((smemJ + 1) & ~1));

  __shared__ InstDesc sD;
  __shared__ Task sT[kMaxSegTasks];
  __shared__ int sPre[kMaxSegTasks + 1];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const int t_last = cta_task[blockIdx.x + 1];
  int t = cta_task[blockIdx.x];
  while (t < t_last) {
    const int inst = tasks[t].inst;
    int te = t + 1;
    while (te < t_last && tasks[te].inst == inst && te - t < kMaxSegTasks) ++te;
    if (threadIdx.x == 0) {
      sD = insts[inst];
      sPre[0] = 0;
      for (int k = 0; k < te - t; ++k) {
        const Task T = tasks[t + k];
        sT[k] = T;
        const int up = map_users_per_pass(T.map);
        sPre[k + 1] = sPre[k] + (T.u1 - T.u0 + up - 1) / up;
      }
    }
    __syncthreads();
    const int J = sD.J;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
      ys[j] = sD.y[j];
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
      S.kind = sD.kind;
    }
    __syncthreads();
    double wobj = 0.0;
    const int ntask = te - t;
    const int total = sPre[ntask];
    for (int p = warp; p < total; p += nw) {
      int k = 0;
      while (p >= sPre[k + 1]) ++k;
      const Task T = sT[k];
      const int64_t uf = T.u0 + static_cast<int64_t>(p - sPre[k]) * map_users_per_pass(T.map);
      const int64_t ue = T.u1;
      switch (T.map) {
        case kMapStream: pass_stream<VT, STATS>(sD, S, ys, accG, accC, accQ, uf, wobj); break;
        case kMapL1K4: pass_reg<1, 4, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL1K8: pass_reg<1, 8, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL2K8: pass_reg<2, 8, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL4K8: pass_reg<4, 8, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL8K8: pass_reg<8, 8, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL16K8: pass_reg<16, 8, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL32K8: pass_reg<32, 8, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL2K4: pass_reg<2, 4, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL4K4: pass_reg<4, 4, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL8K4: pass_reg<8, 4, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL16K4: pass_reg<16, 4, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        case kMapL32K4: pass_reg<32, 4, VT, STATS>(sD, S, ys, accG, accC, accQ, uf, ue, wobj); break;
        default: break;
      }
    }
    if (STATS) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wobj += __shfl_xor_sync(kFull, wobj, o);
      if (lane == 0) wsum[warp] = wobj;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
      const unsigned long long v = accG[j];
      if (v) atomicAdd(sD.acc + j, v);
      if (STATS) {
        const unsigned long long vc = accC[j], vq = accQ[j];
        if (vc) atomicAdd(sD.accC + j, vc);
        if (vq) atomicAdd(sD.accQ + j, vq);
      }
    }
    if (STATS && threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += wsum[w];
      sD.seg_obj[t] = s;
    }
    __syncthreads();
    t = te;
  }
}

template <typename VT, bool STATS>
constexpr auto kernel_of() {
  return &sweep_kernel<VT, STATS>;
}

}  // namespace

size_t sweep_smem_bytes(int smemJ, bool stats, bool /*bf16*/) {
  const size_t J = static_cast<size_t>(smemJ);
  return (stats ? 3 : 1) * J * 8 + ((J + 1) & ~static_cast<size_t>(1)) * 4 + (kSweepThreads / 32) * 8;
}

size_t sweep_smem_limit() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  // room for the kernel's static shared memory
  return optin > 4096 ? static_cast<size_t>(optin - 4096) : 0;
}

cudaError_t sweep_prepare(bool bf16) {
  const int lim = static_cast<int>(sweep_smem_limit());
  cudaError_t e;
  if (bf16) {
    e = cudaFuncSetAttribute(kernel_of<__nv_bfloat16, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel_of<__nv_bfloat16, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  } else {
    e = cudaFuncSetAttribute(kernel_of<float, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel_of<float, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  }
  return e;
}

int sweep_occupancy(int smemJ, bool stats, bool bf16) {
  int n = 0;
  const size_t sm = sweep_smem_bytes(smemJ, stats, bf16);
  cudaError_t e;
  if (bf16)
    e = stats ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_of<__nv_bfloat16, true>(), kSweepThreads, sm)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_of<__nv_bfloat16, false>(), kSweepThreads, sm);
  else
    e = stats ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_of<float, true>(), kSweepThreads, sm)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_of<float, false>(), kSweepThreads, sm);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_sweep(const SweepLaunch& L, bool stats, bool bf16) {
  const size_t sm = sweep_smem_bytes(L.smemJ, stats, bf16);
  if (bf16) {
    if (stats)
      sweep_kernel<__nv_bfloat16, true><<<L.grid, kSweepThreads, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ);
    else
      sweep_kernel<__nv_bfloat16, false><<<L.grid, kSweepThreads, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ);
  } else {
    if (stats)
      sweep_kernel<float, true><<<L.grid, kSweepThreads, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ);
    else
      sweep_kernel<float, false><<<L.grid, kSweepThreads, sm, L.stream>>>(L.inst, L.tasks, L.cta_task, L.smemJ);
  }
  return cudaGetLastError();
}

}  // namespace dlm
