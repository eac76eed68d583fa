// families.cu -- set-up of instances with m > 1 capacity families (Def. 1):
// splitting the caller's edge-major coefficients [nnz x m] into one array per
// family, validating the extra families, laying them out in the slice order
// of layout.cu, and the per-item Gram sums sum_i a_kij a_lij that bound the
// curvature of the dual (A A^T is block diagonal with one m x m block per
// item).  All sums are 64-bit fixed point: exact and order independent.
#include <cmath>

#include "dlm_impl.cuh"

namespace dlm {
namespace {

__device__ __forceinline__ float val(const void* p, int64_t e, bool bf16) {
  if (bf16) return __uint_as_float(static_cast<uint32_t>(static_cast<const uint16_t*>(p)[e]) << 16);
  return static_cast<const float*>(p)[e];
}

// out_f[e] = a[e m + f] (value bytes copied as they are).
__global__ void k_split(const void* a, int64_t nnz, int m, bool bf16, void* out, int64_t stride) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int f = 0; f < m; ++f) {
      if (bf16)
        static_cast<uint16_t*>(out)[f * stride + e] = static_cast<const uint16_t*>(a)[e * m + f];
      else
        static_cast<float*>(out)[f * stride + e] = static_cast<const float*>(a)[e * m + f];
    }
  }
}

// Flags: 1 a non-finite value, 2 a negative value; max |a| as ordered bits.
__global__ void k_check(const void* a, int64_t n, bool bf16, int* flags, unsigned* max_abs) {
  int fl = 0;
  unsigned mx = 0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float v = val(a, e, bf16);
    if (!isfinite(v)) fl |= 1;
    if (v < 0.f) fl |= 2;
    mx = max(mx, __float_as_uint(fabsf(v)));
  }
  if (fl) atomicOr(flags, fl);
  if (mx) atomicMax(max_abs, mx);
}

// dst in slice order (layout.cu): edge k of sorted user u = 32 s + t sits at
// slice_off[s] + sell_el(k, t, width[s] / 4) and is the row's caller edge
// lead_caller_pos(lead[u], k, d); padding gets 0.
__global__ void k_gather_ext(const int64_t* orig_off, const int32_t* udeg, const uint64_t* lead, const int64_t* slice_off,
                             const int32_t* width, int64_t nusers, int64_t nslices, const void* src, bool bf16,
                             void* dst) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = w0; s < nslices; s += nwarps) {
    const int64_t u = 32 * s + lane;
    const int64_t r = u < nusers ? orig_off[u] : 0;
    const int d = u < nusers ? udeg[u] : 0;
    const uint64_t ld = u < nusers ? lead[u] : 0ull;
    const int w = width[s];
    const int w4 = w >> 2;
    const int64_t base = slice_off[s];
    for (int k = 0; k < w; ++k) {
      const int64_t e = k < 4 * w4 ? base + 4 * (32 * static_cast<int64_t>(k >> 2) + lane) + (k & 3)
                                   : base + 128 * static_cast<int64_t>(w4) + 32 * static_cast<int64_t>(k - 4 * w4) + lane;
      const int64_t q = k < d ? r + lead_caller_pos(ld, k, d) : 0;
      if (bf16)
        static_cast<uint16_t*>(dst)[e] = k < d ? static_cast<const uint16_t*>(src)[q] : static_cast<uint16_t>(0);
      else
        static_cast<float*>(dst)[e] = k < d ? static_cast<const float*>(src)[q] : 0.f;
    }
  }
}

// acc[j] += sum over edges of item j of a_f a_l (fixed point, signed).
__global__ void k_gram(const int32_t* col, const void* af, const void* al, int64_t nnz, bool bf16, float scale,
                       unsigned long long* acc) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float p = val(af, e, bf16) * val(al, e, bf16);
    if (p != 0.f) atomicAdd(&acc[col[e]], static_cast<unsigned long long>(__float2ll_rn(p * scale)));
  }
}

int blocks(int64_t n) {
  int64_t g = (n + 255) / 256;
  return static_cast<int>(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

cudaError_t families_split(const void* a, int64_t nnz, int m, bool bf16, void* out, int64_t stride, cudaStream_t s) {
  k_split<<<blocks(nnz), 256, 0, s>>>(a, nnz, m, bf16, out, stride);
  return cudaGetLastError();
}

cudaError_t families_check(const void* a, int64_t n, bool bf16, int* flags, unsigned* max_abs, cudaStream_t s) {
  k_check<<<blocks(n), 256, 0, s>>>(a, n, bf16, flags, max_abs);
  return cudaGetLastError();
}

cudaError_t families_gather(const LayoutOut& lay, const void* src, bool bf16, void* dst, cudaStream_t s) {
  if (lay.nslices == 0) return cudaSuccess;
  const int64_t g = (lay.nslices * 32 + 255) / 256;
  k_gather_ext<<<static_cast<int>(g < 4096 ? g : 4096), 256, 0, s>>>(lay.orig_off, lay.udeg, lay.lead, lay.slice_off,
                                                                    lay.slice_w, lay.num_active_users, lay.nslices,
                                                                    src, bf16, dst);
  return cudaGetLastError();
}

cudaError_t families_gram(const int32_t* col, const void* af, const void* al, int64_t nnz, bool bf16, float scale,
                          unsigned long long* acc, cudaStream_t s) {
  if (nnz > 0) k_gram<<<blocks(nnz), 256, 0, s>>>(col, af, al, nnz, bf16, scale, acc);
  return cudaGetLastError();
}

}  // namespace dlm
