// sweep_common.cuh -- device helpers shared by the sweep kernels (sweep.cu,
// sweep_short.cu, sweep_multi.cu, sweep_boxcut.cu): the value layouts of the
// interleaved (c, a) stream, the slice element order, 64-bit fixed point,
// float-pair arithmetic, and the per-edge deposit of the one-family sweeps.
#pragma once

#include <cuda_bf16.h>

#include "dlm_impl.cuh"

namespace dlm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// One interleaved (c, a) element, and a group of four consecutive edges of a
// lane (element index 4 q .. 4 q + 3 of the stream, 16-byte aligned).
struct F32Pair {
  using T = float2;
  static constexpr bool kCount = false;
  __device__ __forceinline__ static void get(const T& w, float& c, float& a) {
    c = w.x;
    a = w.y;
  }
  __device__ __forceinline__ static void get4(const T* base, int q, float c[4], float a[4]) {
    const float4* p = reinterpret_cast<const float4*>(base) + 2 * q;
    const float4 v0 = __ldg(p), v1 = __ldg(p + 1);
    c[0] = v0.x, a[0] = v0.y, c[1] = v0.z, a[1] = v0.w;
    c[2] = v1.x, a[2] = v1.y, c[3] = v1.z, a[3] = v1.w;
  }
};
struct BF16Pair {
  using T = uint32_t;
  static constexpr bool kCount = false;
  __device__ __forceinline__ static void get(const T& w, float& c, float& a) {
    c = __uint_as_float(w << 16);
    a = __uint_as_float(w & 0xffff0000u);
  }
  __device__ __forceinline__ static void get4(const T* base, int q, float c[4], float a[4]) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(base) + q);
    get(v.x, c[0], a[0]);
    get(v.y, c[1], a[1]);
    get(v.z, c[2], a[2]);
    get(v.w, c[3], a[3]);
  }
};

// Position of edge k of lane t inside a slice of width w (w4 = w / 4 groups
// of four edges per lane, then w % 4 edges edge-major; see layout.cu).
__device__ __forceinline__ int sell_el(int k, int t, int w4) {
  return k < 4 * w4 ? 4 * (32 * (k >> 2) + t) + (k & 3) : 128 * w4 + 32 * (k - 4 * w4) + t;
}

__device__ __forceinline__ unsigned long long fixp(float v, float scale) {
  return static_cast<unsigned long long>(__float2ll_rn(v * scale));
}

// Unevaluated float pairs hi + lo (error-free transformations: Knuth's
// TwoSum, and TwoProduct by FMA).
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
// u = -(c + a*y) as a pair: a*y = p + pe exactly, then -c - p by TwoSum.
__device__ __forceinline__ F2 u_pair(float c, float a, float y) {
  const float p = a * y;
  const float pe = fmaf(a, y, -p);
  const F2 s = two_sum(-c, -p);
  return {s.h, s.l - pe};
}
// (sum - gz) / n for a pair sum; the quotient's remainder is exact by FMA.
__device__ __forceinline__ F2 f2_threshold(F2 sum, float gzh, float gzl, int n) {
  const F2 num = f2_add(sum, F2{-gzh, -gzl});
  const float fn = static_cast<float>(n);
  const float th = __fdiv_rn(num.h, fn);
  const float r = fmaf(-th, fn, num.h);
  return {th, __fdiv_rn(r + num.l, fn)};
}

// Item indices as uint16: the shared-memory item arrays bound a handle to
// fewer than 65,536 items, so the layout keeps the index stream in 16 bits
// (2 bytes per edge less to stream than int32).  A group of four edges of a
// lane is one 64-bit load.
template <class V>
struct Narrow : V {
  using IX = uint16_t;
  __device__ __forceinline__ static const IX* idx(const InstDesc& D) { return D.col16; }
  __device__ __forceinline__ static void idx4(const IX* p, int q, int j[4]) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p) + q);
    j[0] = static_cast<int>(v.x & 0xffffu), j[1] = static_cast<int>(v.x >> 16);
    j[2] = static_cast<int>(v.y & 0xffffu), j[3] = static_cast<int>(v.y >> 16);
  }
};

struct Seg {
  float gamma, invg, gz, gzl, z;
  float scaleG, scaleC, scaleQ, scaleN, scaleO;
  float mu;  // count dual (0 without a count constraint): the floor of the threshold
  int kind;
  int count;
  int jlo, jw;  // certificate sweeps: item sums kept for items jlo .. jlo + jw - 1
};

// Contributions of one edge with x > 0.
template <class P, bool STATS>
__device__ __forceinline__ void deposit(const Seg& S, int j, float c, float a, float x, unsigned long long* accG,
                                        unsigned long long* accC, unsigned long long* accQ, float& ob,
                                        unsigned long long& cn) {
  if (P::kCount) cn += fixp(x, S.scaleN);
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

// x of one edge given the user's threshold (tau, taul): (u - tau) / gamma
// clipped at 0 (and at z for the box).  On the inequality simplex with the
// threshold at its floor, and for the box, the caller passes tau = mu (the
// count dual; 0 without a count constraint), taul = 0.
__device__ __forceinline__ float x_general(const Seg& S, bool box, float tau, float taul, float c, float a,
                                           float y) {
  const F2 up = u_pair(c, a, y);
  if (box) return fminf(fmaxf(((up.h - tau) + (up.l - taul)) * S.invg, 0.f), S.z);
  return fmaxf((up.h - tau) + (up.l - taul), 0.f) * S.invg;
}

// Adds one value per thread into *dst exactly: warp sums, then thread 0 adds
// the warps' partials and makes one global atomic (64-bit fixed point: the
// result does not depend on the order).  Every thread of the block calls it.
__device__ __forceinline__ void cta_add_u64(unsigned long long v, unsigned long long* sh32, unsigned long long* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0) sh32[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0ull;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += sh32[w];
    if (t && dst) atomicAdd(dst, t);
  }
  __syncthreads();
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ int warp_sumi(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Sorted insertion of edge k with value u into the four largest values seen
// (v0 >= ... >= v3), keeping the edge positions of the first three (i0..i2).
// Strict comparisons: among equal values the earlier edge ranks first.
__device__ __forceinline__ void top4_insert(float u, int k, float& v0, float& v1, float& v2, float& v3, int& i0,
                                            int& i1, int& i2) {
  const bool c0 = u > v0;
  const float t1 = c0 ? v0 : u;
  const int k1 = c0 ? i0 : k;
  v0 = c0 ? u : v0;
  i0 = c0 ? k : i0;
  const bool c1 = t1 > v1;
  const float t2 = c1 ? v1 : t1;
  const int k2 = c1 ? i1 : k1;
  v1 = c1 ? t1 : v1;
  i1 = c1 ? k1 : i1;
  const bool c2 = t2 > v2;
  const float t3 = c2 ? v2 : t2;
  v2 = c2 ? t2 : v2;
  i2 = c2 ? k2 : i2;
  v3 = fmaxf(v3, t3);
}

}  // namespace
}  // namespace dlm
