// warmstart.cu -- the learned warm start: per-item features of an instance, a
// three-layer perceptron whose products run on the tensor cores
// (tcgen05.mma with TMEM accumulators, BF16 operands, FP32 accumulation), trained with Adam on
// solved days, and its prediction of the item duals.
//
// Network (width H, F = 7 features):
//   xn = bf16((x - mu) / sd)
//   z1 = xn W1 + b1,  h1 = bf16(relu(z1))
//   z2 = h1 W2 + b2,  h2 = bf16(relu(z2))
//   z3 = h2 . w3 + b3 (FP32 dot product)
//   out = softplus(z3 + softplus^-1(max(lam_prev, 1e-6)))
// with bf16 copies of W1, W2, w3 and FP32 master weights.  The last line is a
// residual form: the network predicts a correction to the previous day's dual
// (feature 4) in softplus pre-activation space, so out >= 0 and an untrained
// last layer (w3 = 0, b3 = 0) returns lam_prev.  Loss: mean squared error
// against the solved duals.  Every reduction (split-K partial sums, column
// sums, the loss) adds in a fixed order, so training is deterministic.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dlm_impl.cuh"

namespace dlm {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kF = DLM_WS_FEATURES;
constexpr float kLamFloor = 1e-6f;
constexpr float kSdFloor = 1e-6f;

// ---------------------------------------------------------------------------
// Features
// ---------------------------------------------------------------------------

// Signed-integer keys that order like the floats they encode.
__device__ __forceinline__ int float_key(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

constexpr int kFeatSmemItems = 8192;

// Per item: degree, max(-c) and sum(-c) (64-bit fixed point, exact) over the
// laid-out edges; padding (c = +inf) is skipped.
__global__ void k_feat_accum(const uint16_t* __restrict__ col, const void* __restrict__ ca, bool bf, int64_t n,
                             int J, float scale, unsigned* __restrict__ gdeg, int* __restrict__ gmax,
                             unsigned long long* __restrict__ gsum) {
  extern __shared__ __align__(16) unsigned char smem[];
  const bool sm = J <= kFeatSmemItems;
  unsigned long long* ssum = reinterpret_cast<unsigned long long*>(smem);
  unsigned* sdeg = reinterpret_cast<unsigned*>(ssum + (sm ? J : 0));
  int* smax = reinterpret_cast<int*>(sdeg + (sm ? J : 0));
  unsigned long long* dsum = sm ? ssum : gsum;
  unsigned* ddeg = sm ? sdeg : gdeg;
  int* dmax = sm ? smax : gmax;
  if (sm) {
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
      ssum[j] = 0ull;
      sdeg[j] = 0u;
      smax[j] = INT_MIN;
    }
    __syncthreads();
  }
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * per;
  const int64_t e1 = e0 + per < n ? e0 + per : n;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    float c;
    if (bf) {
      const uint32_t w = static_cast<const uint32_t*>(ca)[e];
      if ((w & 0xffffu) == 0x7f80u) continue;  // padding
      c = __uint_as_float(w << 16);
    } else {
      c = static_cast<const float2*>(ca)[e].x;
      if (c == INFINITY) continue;  // padding
    }
    const int j = static_cast<int>(col[e]);
    const float nc = -c;
    atomicAdd(&ddeg[j], 1u);
    atomicMax(&dmax[j], float_key(nc));
    atomicAdd(&dsum[j], static_cast<unsigned long long>(__float2ll_rn(nc * scale)));
  }
  if (sm) {
    __syncthreads();
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
      if (sdeg[j]) {
        atomicAdd(&gdeg[j], sdeg[j]);
        atomicMax(&gmax[j], smax[j]);
        atomicAdd(&gsum[j], ssum[j]);
      }
    }
  }
}

__global__ void k_feat_init(int J, unsigned* deg, int* mx, unsigned long long* sum) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
    deg[j] = 0u;
    mx[j] = INT_MIN;
    sum[j] = 0ull;
  }
}

__global__ void k_feat_final(int J, const unsigned* __restrict__ deg, const int* __restrict__ mx,
                             const unsigned long long* __restrict__ sum, double inv_scale,
                             const double* __restrict__ b, const float* __restrict__ lam_prev, double loggamma,
                             const float* __restrict__ grad, float* __restrict__ X) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
    const unsigned d = deg[j];
    const double bj = b[j];
    float* x = X + static_cast<int64_t>(j) * kF;
    x[0] = static_cast<float>(log1p(bj));
    x[1] = static_cast<float>(log1p(static_cast<double>(d)));
    x[2] = d ? static_cast<float>(static_cast<double>(static_cast<long long>(sum[j])) * inv_scale / d) : 0.f;
    x[3] = d ? key_float(mx[j]) : 0.f;
    x[4] = lam_prev[j];
    x[5] = static_cast<float>(loggamma);
    x[6] = static_cast<float>(static_cast<double>(grad[j]) / (1.0 + bj));
  }
}

// ---------------------------------------------------------------------------
// Tensor-core GEMM (tcgen05, TMEM accumulator): part[z] = sum over the z-th K
// range of A(m, k) B(k, n), A and B bf16 with arbitrary element strides,
// FP32 accumulation.  One CTA of 128 threads per 128 x 128 output tile and K
// range: the threads stage 64-wide K slices of A and of B^T into shared
// memory in the no-swizzle K-major layout (8-row x 16-byte core matrices:
// K-adjacent ones 128 bytes apart, the next 8 rows 256 bytes on; a 16-wide K
// step of a 128-row operand is 4 KB); one thread issues the four
// tcgen05.mma.kind::f16 steps (M = N = 128, K = 16) into the CTA's 128 TMEM
// columns and commits them to an mbarrier; after the last slice each warp
// reads its 32 accumulator rows (TMEM lanes) back with tcgen05.ld.
// ---------------------------------------------------------------------------

struct GemmArgs {
  const bf16* A;
  long long sam, sak;
  const bf16* B;
  long long sbk, sbn;
  float* part;  // [splits][M][N]
  int M, N, K, kchunk;
  int* err;     // set when a completion wait runs out
};

constexpr int kTM = 128, kTN = 128, kTK = 64;        // CTA tile; K per staged slice
constexpr int kStepBytes = 128 * 16 * 2;              // one K = 16 step of a 128-row operand
constexpr int kOpBytes = (kTK / 16) * kStepBytes;     // one staged operand slice (16 KB)
// Dynamic shared memory per CTA: both operands plus room that caps an SM at
// four CTAs, so that their TMEM allocations (128 of the 512 columns each)
// never wait for one another.
constexpr int kGemmSmem = 3 * kOpBytes;
constexpr uint32_t kTmemCols = 128;
// kind::f16 instruction descriptor: F32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16 at
// bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kTN >> 3) << 17) | ((kTM >> 4) << 24);
constexpr long long kWaitCycles = 2000000000LL;  // about a second at the SM clock

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (row-direction) byte offsets, each in 16-byte units; bits 46-48 hold
// the fixed value 1; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (static_cast<uint64_t>(1) << 46);
}
// Byte offset of element (row, k) of a staged slice (k < kTK).
__device__ __forceinline__ uint32_t slice_off(int row, int k) {
  return (k >> 4) * kStepBytes + (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
// Waits for completion phase `parity` of the mbarrier, at most kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
  extern __shared__ __align__(128) unsigned char gsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  unsigned char* sA = gsm;
  unsigned char* sB = gsm + kOpBytes;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long m0 = static_cast<long long>(blockIdx.x) * kTM;
  const int n0 = blockIdx.y * kTN;
  const int kb0 = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kb0 + g.kchunk);
  const bf16 zero = __float2bfloat16(0.f);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tslot;

  bool ok = true;
  uint32_t phase = 0;
  int issued = 0;
  for (int kb = kb0; kb < kend; kb += kTK) {
    // stage A(m0.., kb..) and B(kb.., n0..)^T, zeros outside the ranges;
    // consecutive threads take the unit-stride direction
#pragma unroll 8
    for (int i = tid; i < kTM * kTK; i += 128) {
      const int r = g.sam == 1 ? (i % kTM) : (i / kTK);
      const int kk = g.sam == 1 ? (i / kTM) : (i % kTK);
      const long long m = m0 + r;
      const int k = kb + kk;
      *reinterpret_cast<bf16*>(sA + slice_off(r, kk)) = (m < g.M && k < kend) ? g.A[m * g.sam + k * g.sak] : zero;
    }
#pragma unroll 8
    for (int i = tid; i < kTN * kTK; i += 128) {
      const int r = g.sbn == 1 ? (i % kTN) : (i / kTK);
      const int kk = g.sbn == 1 ? (i / kTN) : (i % kTK);
      const int nn = n0 + r;
      const int k = kb + kk;
      *reinterpret_cast<bf16*>(sB + slice_off(r, kk)) =
          (nn < g.N && k < kend) ? g.B[static_cast<long long>(k) * g.sbk + static_cast<long long>(nn) * g.sbn]
                                 : zero;
    }
    // the tensor cores read shared memory through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int st = 0; st < kTK / 16; ++st) {
        const uint64_t ad = smem_desc(smem_addr(sA + st * kStepBytes), 128, 256);
        const uint64_t bd = smem_desc(smem_addr(sB + st * kStepBytes), 128, 256);
        const uint32_t acc = (issued > 0 || st > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&mbar))
                   : "memory");
    }
    ++issued;
    // the slice's products must finish before the next slice overwrites it
    // (the outcome is made uniform across the CTA before anyone leaves)
    ok = __syncthreads_and(mbar_wait(smem_addr(&mbar), phase)) != 0;
    phase ^= 1u;
    if (!ok) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");

  // accumulator rows m0 + 32 warp + lane, 8 columns per load
  float* out = g.part + static_cast<long long>(blockIdx.z) * g.M * g.N;
  const long long row = m0 + warp * 32 + lane;
  for (int c = 0; c < kTN; c += 8) {
    float v[8];
    if (issued > 0 && ok) {
      uint32_t r[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                   : "r"(taddr + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = ok ? 0.f : __int_as_float(0x7fc00000);  // empty K range: 0; timeout: NaN
    }
    if (row < g.M) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (n0 + c + q < g.N) out[row * g.N + n0 + c + q] = v[q];
    }
  }
  if (!ok && tid == 0) {
    atomicOr(g.err, 1);
    mbar_wait(smem_addr(&mbar), phase ^ 1u);  // a last bounded wait for the products in flight
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// Elementwise and reduction kernels
// ---------------------------------------------------------------------------

__device__ __forceinline__ float softplus_f(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ float sigmoid_f(float z) { return 0.5f * (1.f + tanhf(0.5f * z)); }
__device__ __forceinline__ float softplus_inv_f(float y) { return y + logf(-expm1f(-y)); }

__global__ void k_norm_apply(const float* __restrict__ X, int64_t n, const float* __restrict__ mu,
                             const float* __restrict__ sd, bf16* __restrict__ Xn) {
  const int64_t tot = n * kF;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < tot;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int f = static_cast<int>(i % kF);
    Xn[i] = __float2bfloat16_rn((X[i] - mu[f]) / sd[f]);
  }
}

// v = sum_z part[z] + bias; Z = v (if Z); H = bf16(relu(v)).
__global__ void k_bias_relu(const float* __restrict__ part, int S, int64_t MN, int N, const float* __restrict__ bias,
                            float* __restrict__ Z, bf16* __restrict__ H) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < MN;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float v = part[i];
    for (int z = 1; z < S; ++z) v += part[z * MN + i];
    v += bias[i % N];
    if (Z) Z[i] = v;
    H[i] = __float2bfloat16_rn(fmaxf(v, 0.f));
  }
}

// Layer 3 and the output, one warp per row.
__global__ void k_layer3(const bf16* __restrict__ H2, const bf16* __restrict__ w3, const float* __restrict__ b3,
                         const float* __restrict__ X, int64_t n, int Hd, float* __restrict__ s_out,
                         float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = w0; r < n; r += nw) {
    float acc = 0.f;
    for (int h = lane; h < Hd; h += 32)
      acc = fmaf(__bfloat162float(H2[r * Hd + h]), __bfloat162float(w3[h]), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const float s = acc + b3[0] + softplus_inv_f(fmaxf(X[r * kF + 4], kLamFloor));
      if (s_out) s_out[r] = s;
      out[r] = softplus_f(s);
    }
  }
}

// dz3 = (2/n)(out - y) sigmoid(s); the loss (mean of squared errors) in FP64
// by one CTA in a fixed order.
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ s, const float* __restrict__ y,
                       int64_t n, float* __restrict__ dz3, double* __restrict__ loss) {
  __shared__ double red[1024];
  double acc = 0.0;
  const float two_n = static_cast<float>(2.0 / static_cast<double>(n));
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const float e = out[r] - y[r];
    dz3[r] = two_n * e * sigmoid_f(s[r]);
    acc += static_cast<double>(e) * e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / static_cast<double>(n);
}

__global__ void k_dz2(const float* __restrict__ dz3, const bf16* __restrict__ w3, const float* __restrict__ Z2,
                      int64_t n, int Hd, bf16* __restrict__ dZ2) {
  const int64_t tot = n * Hd;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < tot;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = i / Hd;
    const int h = static_cast<int>(i % Hd);
    const float v = Z2[i] > 0.f ? dz3[r] * __bfloat162float(w3[h]) : 0.f;
    dZ2[i] = __float2bfloat16_rn(v);
  }
}

__global__ void k_dz1(const float* __restrict__ part, const float* __restrict__ Z1, int64_t tot,
                      bf16* __restrict__ dZ1) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < tot;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dZ1[i] = __float2bfloat16_rn(Z1[i] > 0.f ? part[i] : 0.f);
}

// dst[i] = sum_z part[z][i], i < MN.
__global__ void k_sum_parts(const float* __restrict__ part, int S, int64_t MN, float* __restrict__ dst) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < MN;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float v = part[i];
    for (int z = 1; z < S; ++z) v += part[z * MN + i];
    dst[i] = v;
  }
}

// Column c of an [n x C] bf16 matrix (times an optional row weight), summed in
// a fixed order by one CTA per column.
__global__ void k_colsum(const bf16* __restrict__ M, const float* __restrict__ wrow, int64_t n, int C,
                         float* __restrict__ dst) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    double v = __bfloat162float(M[r * C + c]);
    if (wrow) v *= wrow[r];
    acc += v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) dst[c] = static_cast<float>(red[0]);
}

__global__ void k_vecsum(const float* __restrict__ v, int64_t n, float* __restrict__ dst) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) acc += v[r];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *dst = static_cast<float>(red[0]);
}

// Column means and (population) standard deviations of X [n x F], one CTA per
// column, FP64 in a fixed order.
__global__ void k_normalizer(const float* __restrict__ X, int64_t n, float* __restrict__ mu, float* __restrict__ sd) {
  __shared__ double red[256];
  const int f = blockIdx.x;
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) acc += X[r * kF + f];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double m = red[0] / static_cast<double>(n);
  __syncthreads();
  acc = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double d = X[r * kF + f] - m;
    acc += d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double s = sqrt(red[0] / static_cast<double>(n));
    mu[f] = static_cast<float>(m);
    sd[f] = s < kSdFloor ? 1.f : static_cast<float>(s);
  }
}

// Adam (bias-corrected) on the FP32 master weights, then their bf16 copies.
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t P, float lr, float c1, float c2) {
  constexpr float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < P;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_to_bf16(const float* __restrict__ src, int64_t n, bf16* __restrict__ dst) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, 4096)));
}

}  // namespace

cudaError_t launch_item_features(const uint16_t* col, const void* ca, bool bf, int64_t padded, int J, double scale,
                                 const double* b, const float* lam_prev, double gamma, const float* grad, float* X,
                                 unsigned* deg, int* mx, unsigned long long* sum, cudaStream_t s) {
  k_feat_init<<<grid_for(J), 256, 0, s>>>(J, deg, mx, sum);
  if (padded > 0) {
    const size_t sm = J <= kFeatSmemItems ? static_cast<size_t>(J) * 16 : 0;
    cudaError_t e = cudaFuncSetAttribute(k_feat_accum, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kFeatSmemItems * 16));
    if (e != cudaSuccess) return e;
    const int g = static_cast<int>(std::min<int64_t>(padded / 16384 + 1, 1216));
    k_feat_accum<<<g, 1024, sm, s>>>(col, ca, bf, padded, J, static_cast<float>(scale), deg, mx, sum);
  }
  k_feat_final<<<grid_for(J), 256, 0, s>>>(J, deg, mx, sum, 1.0 / scale, b, lam_prev, std::log(gamma), grad, X);
  return cudaGetLastError();
}

}  // namespace dlm

// ---------------------------------------------------------------------------
// The predictor object (C-ABI)
// ---------------------------------------------------------------------------

using namespace dlm;

struct dlm_ws {
  int H = 128;
  int64_t P = 0;  // parameter count
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, ow3 = 0, ob3 = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  bf16 *W1b = nullptr, *W2b = nullptr, *w3b = nullptr;
  float *mu = nullptr, *sd = nullptr;
  bool have_norm = false;
  int64_t t = 0;  // Adam steps taken
  // workspace for up to cap rows
  int64_t cap = 0;
  bf16 *Xn = nullptr, *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *s = nullptr, *out = nullptr, *dz3 = nullptr, *part = nullptr;
  int64_t part_cap = 0;
  double* loss = nullptr;  // [loss_cap]
  int64_t loss_cap = 0;
  int* gemm_err = nullptr;  // set by a tensor-core product whose completion wait ran out (device)
};

namespace {

dlm_status wfail(dlm_status s, const std::string& m) {
  dlm::set_last_error(m);
  return s;
}

#define WCK(x)                                                                                          \
  do {                                                                                                  \
    cudaError_t e_ = (x);                                                                               \
    if (e_ != cudaSuccess) return wfail(DLM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
cudaError_t walloc(T** p, int64_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * static_cast<size_t>(n > 0 ? n : 1));
}

void free_work(dlm_ws* w) {
  void* ptrs[] = {w->Xn, w->H1, w->H2, w->dZ2, w->dZ1, w->Z1, w->Z2, w->s, w->out, w->dz3};
  for (void* q : ptrs) cudaFree(q);
  w->Xn = w->H1 = w->H2 = w->dZ2 = w->dZ1 = nullptr;
  w->Z1 = w->Z2 = w->s = w->out = w->dz3 = nullptr;
  w->cap = 0;
}

int last_splits(int64_t K, int splits);

// Split-K ranges of about two staged slices each, so that the long products
// (K = rows) spread over the SMs.
int splits_for(int64_t K) {
  const int64_t s = K / (2 * kTK);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(s, 512)));
}

dlm_status ensure_part(dlm_ws* w, int64_t need) {
  if (need <= w->part_cap) return DLM_OK;
  WCK(cudaStreamSynchronize(w->stream));  // queued kernels may still read the old buffer
  cudaFree(w->part);
  w->part = nullptr;
  w->part_cap = 0;
  WCK(walloc(&w->part, need));
  w->part_cap = need;
  return DLM_OK;
}

dlm_status ensure_work(dlm_ws* w, int64_t n) {
  if (n <= w->cap) return DLM_OK;
  WCK(cudaStreamSynchronize(w->stream));
  free_work(w);
  const int64_t nh = n * w->H;
  WCK(walloc(&w->Xn, n * kF));
  WCK(walloc(&w->H1, nh));
  WCK(walloc(&w->H2, nh));
  WCK(walloc(&w->dZ2, nh));
  WCK(walloc(&w->dZ1, nh));
  WCK(walloc(&w->Z1, nh));
  WCK(walloc(&w->Z2, nh));
  WCK(walloc(&w->s, n));
  WCK(walloc(&w->out, n));
  WCK(walloc(&w->dz3, n));
  w->cap = n;
  const int64_t S = last_splits(n, splits_for(n));
  return ensure_part(w, std::max<int64_t>(nh, S * std::max<int64_t>(w->H, kF) * w->H));
}

dlm_status gemm(dlm_ws* w, const bf16* A, long long sam, long long sak, const bf16* B, long long sbk, long long sbn,
                int64_t M, int N, int64_t K, int splits) {
  if (M <= 0 || N <= 0) return DLM_OK;
  int kchunk = static_cast<int>((K + splits - 1) / splits);
  kchunk = (kchunk + kTK - 1) / kTK * kTK;
  if (kchunk < kTK) kchunk = kTK;
  splits = static_cast<int>((K + kchunk - 1) / kchunk);
  if (splits < 1) splits = 1;
  dlm_status st = ensure_part(w, static_cast<int64_t>(splits) * M * N);
  if (st != DLM_OK) return st;
  GemmArgs g;
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.B = B;
  g.sbk = sbk;
  g.sbn = sbn;
  g.part = w->part;
  g.M = static_cast<int>(M);
  g.N = N;
  g.K = static_cast<int>(K);
  g.kchunk = kchunk;
  if (K <= 0) {
    WCK(cudaMemsetAsync(w->part, 0, sizeof(float) * M * N, w->stream));
    return DLM_OK;
  }
  dim3 grid(static_cast<unsigned>((M + kTM - 1) / kTM), static_cast<unsigned>((N + kTN - 1) / kTN), splits);
  g.err = w->gemm_err;
  k_gemm<<<grid, 128, kGemmSmem, w->stream>>>(g);
  WCK(cudaGetLastError());
  return DLM_OK;
}

int last_splits(int64_t K, int splits) {
  int kchunk = static_cast<int>((K + splits - 1) / splits);
  kchunk = (kchunk + kTK - 1) / kTK * kTK;
  if (kchunk < kTK) kchunk = kTK;
  return static_cast<int>(std::max<int64_t>(1, (K + kchunk - 1) / kchunk));
}

// DLM_ERR_TIMEOUT when a tensor-core product's completion wait ran out
// (the word is cleared for the next call).
dlm_status check_gemm(dlm_ws* w) {
  int h = 0;
  WCK(cudaMemcpyAsync(&h, w->gemm_err, sizeof(int), cudaMemcpyDeviceToHost, w->stream));
  WCK(cudaStreamSynchronize(w->stream));
  if (h) {
    WCK(cudaMemsetAsync(w->gemm_err, 0, sizeof(int), w->stream));
    return wfail(DLM_ERR_TIMEOUT, "a tensor-core product did not complete in time");
  }
  return DLM_OK;
}

dlm_status refresh_bf16(dlm_ws* w) {
  k_to_bf16<<<grid_for(kF * w->H), 256, 0, w->stream>>>(w->theta + w->oW1, kF * w->H, w->W1b);
  k_to_bf16<<<grid_for(static_cast<int64_t>(w->H) * w->H), 256, 0, w->stream>>>(
      w->theta + w->oW2, static_cast<int64_t>(w->H) * w->H, w->W2b);
  k_to_bf16<<<grid_for(w->H), 256, 0, w->stream>>>(w->theta + w->ow3, w->H, w->w3b);
  WCK(cudaGetLastError());
  return DLM_OK;
}

// Forward pass over n rows of X (device, n x F); leaves out/s/Z/H in the workspace.
dlm_status forward(dlm_ws* w, const float* X, int64_t n) {
  const int H = w->H;
  const int64_t nh = n * H;
  k_norm_apply<<<grid_for(n * kF), 256, 0, w->stream>>>(X, n, w->mu, w->sd, w->Xn);
  WCK(cudaGetLastError());
  dlm_status st = gemm(w, w->Xn, kF, 1, w->W1b, H, 1, n, H, kF, 1);
  if (st != DLM_OK) return st;
  k_bias_relu<<<grid_for(nh), 256, 0, w->stream>>>(w->part, 1, nh, H, w->theta + w->ob1, w->Z1, w->H1);
  st = gemm(w, w->H1, H, 1, w->W2b, H, 1, n, H, H, 1);
  if (st != DLM_OK) return st;
  k_bias_relu<<<grid_for(nh), 256, 0, w->stream>>>(w->part, 1, nh, H, w->theta + w->ob2, w->Z2, w->H2);
  k_layer3<<<grid_for(n * 32), 256, 0, w->stream>>>(w->H2, w->w3b, w->theta + w->ob3, X, n, H, w->s, w->out);
  WCK(cudaGetLastError());
  return DLM_OK;
}

// Loss (into w->loss[slot]) and gradient (into w->grad) at the current weights.
dlm_status loss_grad(dlm_ws* w, const float* X, const float* y, int64_t n, int64_t slot) {
  dlm_status st = forward(w, X, n);
  if (st != DLM_OK) return st;
  const int H = w->H;
  const int64_t nh = n * H;
  k_loss<<<1, 1024, 0, w->stream>>>(w->out, w->s, y, n, w->dz3, w->loss + slot);
  k_dz2<<<grid_for(nh), 256, 0, w->stream>>>(w->dz3, w->w3b, w->Z2, n, H, w->dZ2);
  WCK(cudaGetLastError());
  // dW2 = H1^T dZ2 (split over rows)
  int S = splits_for(n);
  st = gemm(w, w->H1, 1, H, w->dZ2, H, 1, H, H, n, S);
  if (st != DLM_OK) return st;
  S = last_splits(n, S);
  k_sum_parts<<<grid_for(static_cast<int64_t>(H) * H), 256, 0, w->stream>>>(w->part, S, static_cast<int64_t>(H) * H,
                                                                             w->grad + w->oW2);
  // dH1 = dZ2 W2^T, dZ1 = bf16(dH1 * [z1 > 0])
  st = gemm(w, w->dZ2, H, 1, w->W2b, 1, H, n, H, H, 1);
  if (st != DLM_OK) return st;
  k_dz1<<<grid_for(nh), 256, 0, w->stream>>>(w->part, w->Z1, nh, w->dZ1);
  // dW1 = Xn^T dZ1
  S = splits_for(n);
  st = gemm(w, w->Xn, 1, kF, w->dZ1, H, 1, kF, H, n, S);
  if (st != DLM_OK) return st;
  S = last_splits(n, S);
  k_sum_parts<<<grid_for(kF * H), 256, 0, w->stream>>>(w->part, S, kF * H, w->grad + w->oW1);
  k_colsum<<<H, 256, 0, w->stream>>>(w->dZ1, nullptr, n, H, w->grad + w->ob1);
  k_colsum<<<H, 256, 0, w->stream>>>(w->dZ2, nullptr, n, H, w->grad + w->ob2);
  k_colsum<<<H, 256, 0, w->stream>>>(w->H2, w->dz3, n, H, w->grad + w->ow3);
  k_vecsum<<<1, 256, 0, w->stream>>>(w->dz3, n, w->grad + w->ob3);
  WCK(cudaGetLastError());
  return DLM_OK;
}

dlm_status ensure_loss(dlm_ws* w, int64_t k) {
  if (k <= w->loss_cap) return DLM_OK;
  WCK(cudaStreamSynchronize(w->stream));
  cudaFree(w->loss);
  w->loss = nullptr;
  w->loss_cap = 0;
  WCK(walloc(&w->loss, k));
  w->loss_cap = k;
  return DLM_OK;
}

dlm_status check_rows(const void* X, int64_t n) {
  if (!X) return wfail(DLM_ERR_INVALID_ARG, "null array");
  if (n <= 0 || n > (int64_t(1) << 26)) return wfail(DLM_ERR_INVALID_ARG, "need 0 < n <= 2^26 rows");
  return DLM_OK;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

dlm_status dlm_ws_create(int32_t width, uint64_t seed, void* stream, dlm_ws** out) {
  if (!out) return wfail(DLM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (width < 8 || width > 1024 || width % 8 != 0) return wfail(DLM_ERR_INVALID_ARG, "width must be 8..1024, a multiple of 8");
  dlm_ws* w = new dlm_ws();
  w->H = width;
  const int64_t H = width;
  w->oW1 = 0;
  w->ob1 = w->oW1 + kF * H;
  w->oW2 = w->ob1 + H;
  w->ob2 = w->oW2 + H * H;
  w->ow3 = w->ob2 + H;
  w->ob3 = w->ow3 + H;
  w->P = w->ob3 + 1;
  if (stream) {
    w->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamDefault) != cudaSuccess) {
      delete w;
      return wfail(DLM_ERR_CUDA, "stream creation failed");
    }
    w->own_stream = true;
  }
  // He-uniform first two layers, zero last layer and biases (the untrained
  // predictor returns the previous dual).
  std::vector<float> th(w->P, 0.f);
  uint64_t st = seed;
  auto uni = [&]() { return static_cast<double>(splitmix(st) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; };
  for (int64_t i = 0; i < kF * H; ++i) th[w->oW1 + i] = static_cast<float>(uni() * std::sqrt(6.0 / kF));
  for (int64_t i = 0; i < H * H; ++i) th[w->oW2 + i] = static_cast<float>(uni() * std::sqrt(6.0 / H));
  std::vector<float> one(kF, 1.f), zero(kF, 0.f);
  dlm_status s = DLM_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && s == DLM_OK) s = wfail(DLM_ERR_CUDA, cudaGetErrorString(e));
  };
  ck(walloc(&w->theta, w->P));
  ck(walloc(&w->grad, w->P));
  ck(walloc(&w->m, w->P));
  ck(walloc(&w->v, w->P));
  ck(walloc(&w->W1b, kF * H));
  ck(walloc(&w->W2b, H * H));
  ck(walloc(&w->w3b, H));
  ck(walloc(&w->mu, kF));
  ck(walloc(&w->sd, kF));
  ck(walloc(&w->gemm_err, 1));
  if (s == DLM_OK) ck(cudaMemset(w->gemm_err, 0, sizeof(int)));
  if (s == DLM_OK) {
    ck(cudaMemcpy(w->theta, th.data(), sizeof(float) * w->P, cudaMemcpyHostToDevice));
    ck(cudaMemset(w->m, 0, sizeof(float) * w->P));
    ck(cudaMemset(w->v, 0, sizeof(float) * w->P));
    ck(cudaMemset(w->grad, 0, sizeof(float) * w->P));
    ck(cudaMemcpy(w->mu, zero.data(), sizeof(float) * kF, cudaMemcpyHostToDevice));
    ck(cudaMemcpy(w->sd, one.data(), sizeof(float) * kF, cudaMemcpyHostToDevice));
  }
  if (s == DLM_OK) ck(cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem));
  if (s == DLM_OK) s = refresh_bf16(w);
  if (s == DLM_OK) s = ensure_loss(w, 1);
  if (s == DLM_OK) {
    cudaError_t e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) s = wfail(DLM_ERR_CUDA, cudaGetErrorString(e));
  }
  if (s != DLM_OK) {
    dlm_ws_destroy(w);
    return s;
  }
  *out = w;
  return DLM_OK;
}

dlm_status dlm_ws_num_params(dlm_ws* w, int64_t* n) {
  if (!w || !n) return wfail(DLM_ERR_INVALID_ARG, "null argument");
  *n = w->P;
  return DLM_OK;
}

dlm_status dlm_ws_get_params(dlm_ws* w, float* theta, float* mu, float* sd) {
  if (!w) return wfail(DLM_ERR_INVALID_ARG, "null handle");
  WCK(cudaStreamSynchronize(w->stream));
  if (theta) WCK(cudaMemcpy(theta, w->theta, sizeof(float) * w->P, cudaMemcpyDeviceToHost));
  if (mu) WCK(cudaMemcpy(mu, w->mu, sizeof(float) * kF, cudaMemcpyDeviceToHost));
  if (sd) WCK(cudaMemcpy(sd, w->sd, sizeof(float) * kF, cudaMemcpyDeviceToHost));
  return DLM_OK;
}

dlm_status dlm_ws_set_params(dlm_ws* w, const float* theta, const float* mu, const float* sd) {
  if (!w) return wfail(DLM_ERR_INVALID_ARG, "null handle");
  if ((mu == nullptr) != (sd == nullptr)) return wfail(DLM_ERR_INVALID_ARG, "give both mu and sd, or neither");
  if (sd)
    for (int f = 0; f < kF; ++f)
      if (!(sd[f] > 0) || !std::isfinite(sd[f]) || !std::isfinite(mu[f]))
        return wfail(DLM_ERR_INVALID_ARG, "sd must be finite and > 0, mu finite");
  WCK(cudaStreamSynchronize(w->stream));
  if (theta) {
    WCK(cudaMemcpy(w->theta, theta, sizeof(float) * w->P, cudaMemcpyHostToDevice));
    WCK(cudaMemset(w->m, 0, sizeof(float) * w->P));
    WCK(cudaMemset(w->v, 0, sizeof(float) * w->P));
    w->t = 0;
  }
  if (mu) {
    WCK(cudaMemcpy(w->mu, mu, sizeof(float) * kF, cudaMemcpyHostToDevice));
    WCK(cudaMemcpy(w->sd, sd, sizeof(float) * kF, cudaMemcpyHostToDevice));
    w->have_norm = true;
  }
  dlm_status s = refresh_bf16(w);
  if (s != DLM_OK) return s;
  WCK(cudaStreamSynchronize(w->stream));
  return DLM_OK;
}

dlm_status dlm_ws_fit_normalizer(dlm_ws* w, const float* X, int64_t n) {
  if (!w) return wfail(DLM_ERR_INVALID_ARG, "null handle");
  dlm_status s = check_rows(X, n);
  if (s != DLM_OK) return s;
  k_normalizer<<<kF, 256, 0, w->stream>>>(X, n, w->mu, w->sd);
  WCK(cudaGetLastError());
  WCK(cudaStreamSynchronize(w->stream));
  w->have_norm = true;
  return DLM_OK;
}

dlm_status dlm_ws_loss_grad(dlm_ws* w, const float* X, const float* y, int64_t n, double* loss, float* grad) {
  if (!w || !y) return wfail(DLM_ERR_INVALID_ARG, "null argument");
  dlm_status s = check_rows(X, n);
  if (s == DLM_OK) s = ensure_work(w, n);
  if (s == DLM_OK) s = loss_grad(w, X, y, n, 0);
  if (s != DLM_OK) return s;
  if (loss) WCK(cudaMemcpyAsync(loss, w->loss, sizeof(double), cudaMemcpyDeviceToHost, w->stream));
  if (grad) WCK(cudaMemcpyAsync(grad, w->grad, sizeof(float) * w->P, cudaMemcpyDeviceToHost, w->stream));
  WCK(cudaStreamSynchronize(w->stream));
  return check_gemm(w);
}

dlm_status dlm_ws_train(dlm_ws* w, const float* X, const float* y, int64_t n, int32_t steps, float lr,
                        float* losses) {
  if (!w || !y) return wfail(DLM_ERR_INVALID_ARG, "null argument");
  if (steps < 0 || !(lr > 0) || !std::isfinite(lr)) return wfail(DLM_ERR_INVALID_ARG, "need steps >= 0, lr > 0");
  dlm_status s = check_rows(X, n);
  if (s == DLM_OK && !w->have_norm) s = dlm_ws_fit_normalizer(w, X, n);
  if (s == DLM_OK) s = ensure_work(w, n);
  if (s == DLM_OK) s = ensure_loss(w, steps > 0 ? steps : 1);
  if (s != DLM_OK) return s;
  for (int32_t k = 0; k < steps; ++k) {
    s = loss_grad(w, X, y, n, k);
    if (s != DLM_OK) return s;
    ++w->t;
    const float c1 = static_cast<float>(1.0 - std::pow(0.9, static_cast<double>(w->t)));
    const float c2 = static_cast<float>(1.0 - std::pow(0.999, static_cast<double>(w->t)));
    k_adam<<<grid_for(w->P), 256, 0, w->stream>>>(w->theta, w->grad, w->m, w->v, w->P, lr, c1, c2);
    WCK(cudaGetLastError());
    s = refresh_bf16(w);
    if (s != DLM_OK) return s;
  }
  if (losses && steps > 0) {
    std::vector<double> h(steps);
    WCK(cudaMemcpyAsync(h.data(), w->loss, sizeof(double) * steps, cudaMemcpyDeviceToHost, w->stream));
    WCK(cudaStreamSynchronize(w->stream));
    for (int32_t k = 0; k < steps; ++k) losses[k] = static_cast<float>(h[k]);
  }
  WCK(cudaStreamSynchronize(w->stream));
  return check_gemm(w);
}

dlm_status dlm_ws_predict(dlm_ws* w, const float* X, int64_t n, float* out) {
  if (!w || !out) return wfail(DLM_ERR_INVALID_ARG, "null argument");
  dlm_status s = check_rows(X, n);
  if (s == DLM_OK) s = ensure_work(w, n);
  if (s == DLM_OK) s = forward(w, X, n);
  if (s != DLM_OK) return s;
  WCK(cudaMemcpyAsync(out, w->out, sizeof(float) * n, cudaMemcpyDeviceToDevice, w->stream));
  WCK(cudaStreamSynchronize(w->stream));
  return check_gemm(w);
}

void dlm_ws_destroy(dlm_ws* w) {
  if (!w) return;
  if (w->stream) cudaStreamSynchronize(w->stream);
  free_work(w);
  void* ptrs[] = {w->theta, w->grad, w->m, w->v, w->W1b, w->W2b, w->w3b, w->mu, w->sd, w->part, w->loss, w->gemm_err};
  for (void* q : ptrs) cudaFree(q);
  if (w->own_stream && w->stream) cudaStreamDestroy(w->stream);
  delete w;
}

}  // extern "C"
