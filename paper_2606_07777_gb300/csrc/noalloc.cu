// noalloc.cu -- one dual evaluation that allocates no device memory.
//
// For callers that cannot allocate device memory (code running under a
// memory budget that forbids cudaMalloc, inside an allocator of its own, or
// in a process whose memory is owned by another framework), this file gives
// a variant of the dual evaluation that reads the caller's CSR arrays
// directly and keeps all of its scratch (fixed-point item sums, per-block
// objective partials, value bounds, an error word) in one file-scope
// __device__ array of fixed size.  Every GPU that loads the library holds that
// array until the process exits.  Calls that overlap on the GPU share it and
// race; run them one after another on one stream.
#include <cmath>
#include <mutex>

#include "dlm_impl.cuh"

namespace {

constexpr int64_t kStaticMaxItems = 65536;  // largest num_items accepted
constexpr int kStaticBlocks = 512;          // fixed grid of the sweep kernel
constexpr int kStaticThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

struct StaticScratch {
  unsigned long long acc[kStaticMaxItems];  // fixed-point sum a x per item
  double obj[kStaticBlocks];                // objective partial per block
  unsigned int bits[4];                     // max |a|, max |c| (float bits), error word, unused
};

static __device__ __align__(256) StaticScratch g_scratch;

// Device address of g_scratch, looked up once per device (host code may not
// use the symbol itself as a device address).  The address belongs to the
// device's primary context: it is not valid after cudaDeviceReset.
std::mutex g_sym_mu;
void* g_sym_addr[64] = {nullptr};

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
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

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
__device__ __forceinline__ F2 u_pair(float c, float a, float y) {
  const float p = a * y;
  const float pe = fmaf(a, y, -p);
  const F2 s = two_sum(-c, -p);
  return {s.h, s.l - pe};
}

__device__ __forceinline__ int shift_for(double bound) {
  if (!(bound > 0)) return 60;
  int s = static_cast<int>(floor(61.0 - log2(bound)));
  return s > 100 ? 100 : (s < 0 ? 0 : s);
}

// Clears the scratch that must start at zero.
__global__ void k_clear(StaticScratch* S, int64_t J) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < J;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    S->acc[i] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x < 4) S->bits[threadIdx.x] = 0u;
}

// Bounds of |a| and |c| (for the fixed-point scales).
__global__ void k_bounds(const float* c, const float* a, int64_t nnz, StaticScratch* S) {
  unsigned ma = 0, mc = 0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    ma = max(ma, __float_as_uint(fabsf(a[e])));
    mc = max(mc, __float_as_uint(fabsf(c[e])));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ma = max(ma, __shfl_xor_sync(kFull, ma, o));
    mc = max(mc, __shfl_xor_sync(kFull, mc, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&S->bits[0], ma);
    atomicMax(&S->bits[1], mc);
  }
}

// One warp per user (users dealt to warps statically): the simplex threshold
// by the Michelot iteration from max(u) - gamma z with warp sums, refined in
// float-pair arithmetic, then x and the item sums (global 64-bit fixed-point
// atomics into the scratch) and the objective (per block, FP64).
__global__ void __launch_bounds__(kStaticThreads) k_static_sweep(const int64_t* rp, const int32_t* col,
                                                                 const float* c, const float* a, int64_t I,
                                                                 int64_t J, int64_t nnz, int kind, double z,
                                                                 const float* lam, double gamma, float* xout,
                                                                 StaticScratch* S) {
  __shared__ double wsum[kStaticThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float amax = __uint_as_float(S->bits[0]), cmax = __uint_as_float(S->bits[1]);
  const double n = static_cast<double>(nnz > 0 ? nnz : 1);
  (void)cmax;
  const float scG = ldexpf(1.f, shift_for(n * amax * z));
  const float gf = static_cast<float>(gamma), invg = static_cast<float>(1.0 / gamma);
  const double gzd = gamma * z;
  const float gz = static_cast<float>(gzd), gzl = static_cast<float>(gzd - static_cast<double>(gz));
  const float zf = static_cast<float>(z);
  const bool eq = kind == DLM_SIMPLEX_EQ, box = kind == DLM_BOX;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  double wobj = 0.0;
  for (int64_t u = gw; u < I; u += nwarps) {
    const int64_t s = rp[u], d = rp[u + 1] - s;
    if (s < 0 || d < 0 || s + d > nnz) {  // invalid row pointer: no access, flagged
      if (lane == 0) atomicOr(&S->bits[2], 1u);
      continue;
    }
    auto uval = [&](int64_t i, int& j, float& cv, float& av) {
      j = col[s + i];
      cv = c[s + i];
      av = a[s + i];
      if (j < 0 || j >= J) {  // invalid item: no access, flagged
        j = -1;
        return -INFINITY;
      }
      return -fmaf(av, lam[j], cv);
    };
    float tau = 0.f, taul = 0.f;
    bool zero = box;
    if (!box && d > 0) {
      float m = -INFINITY;
      for (int64_t i = lane; i < d; i += 32) {
        int j;
        float cv, av;
        m = fmaxf(m, uval(i, j, cv, av));
      }
      m = warp_max(m);
      if (eq || m > 0.f) {
        tau = m - gz;
        // the iteration stops once the threshold no longer rises (from the
        // lower bound m - gamma z it cannot in exact arithmetic; in FP32 two
        // sets whose thresholds round past each other would otherwise
        // alternate), so every further pass strictly shrinks the active set
        // and d + 1 passes always reach the stop
        int prevn = -1;
        for (int64_t it = 0; it <= d; ++it) {
          float sm = 0.f;
          int cnt = 0;
          for (int64_t i = lane; i < d; i += 32) {
            int j;
            float cv, av;
            const float uv = uval(i, j, cv, av);
            if (uv > tau) {
              sm += uv;
              ++cnt;
            }
          }
          sm = warp_sum(sm);
          cnt = warp_sumi(cnt);
          if (cnt == prevn || cnt == 0) break;
          prevn = cnt;
          const float tn = __fdiv_rn(sm - gz, static_cast<float>(cnt));
          if (!(tn > tau)) break;
          tau = tn;
        }
        zero = !eq && tau <= 0.f;
        if (!zero) {
          F2 sum{0.f, 0.f};
          int cnt = 0;
          for (int64_t i = lane; i < d; i += 32) {
            int j;
            float cv, av;
            if (uval(i, j, cv, av) > tau) {
              sum = f2_add(sum, u_pair(cv, av, lam[j]));
              ++cnt;
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const F2 other{__shfl_xor_sync(kFull, sum.h, o), __shfl_xor_sync(kFull, sum.l, o)};
            sum = f2_add(sum, other);
            cnt += __shfl_xor_sync(kFull, cnt, o);
          }
          const F2 num = f2_add(sum, F2{-gz, -gzl});
          const float fn = static_cast<float>(cnt > 0 ? cnt : 1);
          const float th = __fdiv_rn(num.h, fn);
          const float tl = __fdiv_rn(fmaf(-th, fn, num.h) + num.l, fn);
          if (!eq && th + tl <= 0.f) {
            zero = true;
          } else {
            tau = th;
            taul = tl;
          }
        }
      } else {
        zero = true;
      }
    }
    if (zero) tau = taul = 0.f;
    float ob = 0.f;
    for (int64_t i = lane; i < d; i += 32) {
      int j;
      float cv, av;
      const float uv = uval(i, j, cv, av);
      float x = 0.f;
      if (j < 0) {
        atomicOr(&S->bits[2], 1u);
      } else if (uv > tau) {
        const F2 up = u_pair(cv, av, lam[j]);
        x = box ? fminf(fmaxf((up.h + up.l) * invg, 0.f), zf)
                : (zero ? fmaxf(up.h + up.l, 0.f) * invg : fmaxf((up.h - tau) + (up.l - taul), 0.f) * invg);
        if (x > 0.f) {
          atomicAdd(&S->acc[j], static_cast<unsigned long long>(__float2ll_rn(av * x * scG)));
          ob += fmaf(0.5f * gf * x, x, cv * x);
        }
      }
      if (xout) xout[s + i] = x;
    }
    wobj += static_cast<double>(warp_sum(ob));
  }
  if (lane == 0) wsum[warp] = wobj;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += wsum[w];
    S->obj[blockIdx.x] = t;
  }
}

// g = sum_i (c x + gamma/2 x^2) + lam^T (A x - b), grad = A x - b; then the
// scratch is cleared for the next call.  A flagged invalid item gives NaN.
__global__ void k_static_finish(const double* b, int64_t J, int64_t nnz, double z, const float* lam, double* g_out,
                                float* grad_out, StaticScratch* S) {
  __shared__ double sh[32];
  const double amax = __uint_as_float(S->bits[0]);
  const double n = static_cast<double>(nnz > 0 ? nnz : 1);
  const double invG = ldexp(1.0, -shift_for(n * amax * z));
  const bool bad = S->bits[2] != 0u;
  double lg = 0.0, obj = 0.0;
  for (int k = threadIdx.x; k < kStaticBlocks; k += blockDim.x) obj += S->obj[k];
  for (int64_t j = threadIdx.x; j < J; j += blockDim.x) {
    const double G = static_cast<double>(static_cast<long long>(S->acc[j])) * invG - b[j];
    lg += static_cast<double>(lam[j]) * G;
    if (grad_out) grad_out[j] = bad ? NAN : static_cast<float>(G);
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < J; i += blockDim.x) S->acc[i] = 0ull;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double v[2] = {lg, obj};
  for (int q = 0; q < 2; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(kFull, v[q], o);
    __syncthreads();
    if (lane == 0) sh[w] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) t += sh[k];
      v[q] = t;
    }
  }
  if (threadIdx.x == 0) {
    *g_out = bad ? NAN : v[1] + v[0];
    for (int k = 0; k < 4; ++k) S->bits[k] = 0u;
    for (int k = 0; k < kStaticBlocks; ++k) S->obj[k] = 0.0;
  }
}

dlm_status sfail(dlm_status s, const char* m) {
  dlm::set_last_error(m);
  return s;
}

}  // namespace

extern "C" {

dlm_status dlm_calculate_static(int64_t num_users, int64_t num_items, int64_t nnz, const int64_t* row_ptr,
                                const int32_t* item_idx, const float* c, const float* a, const double* b,
                                int32_t kind, double z, const float* lambda, double gamma, double* g, float* grad,
                                float* x, void* stream) {
  dlm::set_last_error("");
  if (num_users < 0 || num_items <= 0 || nnz < 0) return sfail(DLM_ERR_INVALID_ARG, "bad sizes");
  if (num_items > kStaticMaxItems)
    return sfail(DLM_ERR_UNSUPPORTED, "num_items exceeds the static scratch limit of 65536 items");
  if (!row_ptr || (nnz > 0 && (!item_idx || !c || !a)) || !b || !lambda || !g)
    return sfail(DLM_ERR_INVALID_ARG, "null pointer");
  if (kind == DLM_BOX_CUT) return sfail(DLM_ERR_UNSUPPORTED, "DLM_BOX_CUT needs a handle (dlm_create)");
  if (kind != DLM_SIMPLEX_LE && kind != DLM_SIMPLEX_EQ && kind != DLM_BOX)
    return sfail(DLM_ERR_INVALID_ARG, "bad simple-set kind");
  if (!(z > 0) || !std::isfinite(z) || !(gamma > 0) || !std::isfinite(gamma))
    return sfail(DLM_ERR_INVALID_ARG, "z and gamma must be finite and > 0");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return sfail(DLM_ERR_CUDA, "no current CUDA device");
  void* sym = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_sym_mu);
    if (!g_sym_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) return sfail(DLM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      g_sym_addr[dev] = p;
    }
    sym = g_sym_addr[dev];
  }
  StaticScratch* S = static_cast<StaticScratch*>(sym);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_clear<<<64, 256, 0, st>>>(S, num_items);
  if (nnz > 0) k_bounds<<<256, 256, 0, st>>>(c, a, nnz, S);
  k_static_sweep<<<kStaticBlocks, kStaticThreads, 0, st>>>(row_ptr, item_idx, c, a, num_users, num_items, nnz, kind,
                                                           z, lambda, gamma, x, S);
  k_static_finish<<<1, 1024, 0, st>>>(b, num_items, nnz, z, lambda, g, grad, S);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sfail(DLM_ERR_CUDA, cudaGetErrorString(e));
  return DLM_OK;
}

}  // extern "C"
