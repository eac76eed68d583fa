// layout.cu -- one-time set-up of an instance: input validation, degree
// classes, the degree-bucketed edge layout the sweep reads, and per-item
// constants (sum_i a_ij^2 for the step size and row normalization, App. B.2;
// item degrees and value bounds for the fixed-point scales).
//
// The caller's CSR is user-major (one row per user, Sec. 4.1's one column per
// source).  Users are stably sorted by degree class (the log-bucketing idea
// of Sec. 4.2: classes [2^(t-1), 2^t)), and their rows are copied into that
// order, so the rows of one class are contiguous and a sweep task streams a
// contiguous byte range.
#include <cub/cub.cuh>

#include <cmath>
#include <string>
#include <vector>

#include "dlm_impl.cuh"

namespace dlm {
namespace {

constexpr int kT = 256;

enum : int { kBadRowPtr = 1, kBadItem = 2, kBadValue = 4, kBadB = 8, kNegA = 16 };

__device__ __forceinline__ float load_val(const void* p, int64_t e, bool bf16) {
  if (bf16) {
    const unsigned short b = reinterpret_cast<const unsigned short*>(p)[e];
    return __uint_as_float(static_cast<unsigned>(b) << 16);
  }
  return reinterpret_cast<const float*>(p)[e];
}

// Row pointer checks, degree classes and class histogram.
__global__ void k_rows(const int64_t* rp, int64_t I, int64_t nnz, int32_t* cls, unsigned long long* class_cnt,
                       int* bad) {
  __shared__ unsigned long long h[kNumClasses];
  if (threadIdx.x < kNumClasses) h[threadIdx.x] = 0;
  __syncthreads();
  int flag = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < I;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r0 = rp[i], r1 = rp[i + 1];
    const int64_t d = r1 - r0;
    if (d < 0 || r0 < 0 || r1 > nnz) flag |= kBadRowPtr;
    const int c = degree_class(d < 0 ? 0 : d);
    cls[i] = c;
    atomicAdd(&h[c], 1ull);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (rp[0] != 0 || rp[I] != nnz) flag |= kBadRowPtr;
  }
  if (flag) atomicOr(bad, flag);
  __syncthreads();
  if (threadIdx.x < kNumClasses && h[threadIdx.x]) atomicAdd(&class_cnt[threadIdx.x], h[threadIdx.x]);
}

// Edge checks, item degrees, max |a|, max |c|.
__global__ void k_edges(const int32_t* col, const void* c, const void* a, bool bf16, int64_t nnz, int64_t J,
                        unsigned long long* item_deg, unsigned* max_a, unsigned* max_c, int* bad) {
  __shared__ unsigned s_ma, s_mc;
  if (threadIdx.x == 0) s_ma = s_mc = 0;
  __syncthreads();
  int flag = 0;
  unsigned ma = 0, mc = 0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t j = col[e];
    if (j < 0 || j >= J)
      flag |= kBadItem;
    else
      atomicAdd(&item_deg[j], 1ull);
    const float cv = load_val(c, e, bf16), av = load_val(a, e, bf16);
    if (!isfinite(cv) || !isfinite(av)) flag |= kBadValue;
    if (av < 0.f) flag |= kNegA;
    ma = max(ma, __float_as_uint(fabsf(av)));
    mc = max(mc, __float_as_uint(fabsf(cv)));
  }
  if (flag) atomicOr(bad, flag);
  atomicMax(&s_ma, ma);
  atomicMax(&s_mc, mc);
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(max_a, s_ma);
    atomicMax(max_c, s_mc);
  }
}

__global__ void k_b(const double* b, int64_t J, int* bad) {
  int flag = 0;
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < J;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x)
    if (!isfinite(b[j]) || b[j] < 0.0) flag |= kBadB;
  if (flag) atomicOr(bad, flag);
}

__global__ void k_iota(int32_t* v, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    v[i] = static_cast<int32_t>(i);
}

__global__ void k_perm_deg(const int64_t* rp, const int32_t* perm, int64_t I, int64_t* deg_p, int64_t* orig_off) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < I;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = perm[i];
    deg_p[i] = rp[o + 1] - rp[o];
    orig_off[i] = rp[o];
  }
}

// Copy each user's row into the bucketed order: one warp per user.
template <typename VT>
__global__ void k_gather(const int32_t* col, const VT* c, const VT* a, const int64_t* orig_off,
                         const int64_t* rp_new, int64_t I, int32_t* col_o, VT* c_o, VT* a_o) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t u = w0; u < I; u += nwarps) {
    const int64_t s = orig_off[u], t = rp_new[u], d = rp_new[u + 1] - t;
    for (int64_t k = lane; k < d; k += 32) {
      col_o[t + k] = col[s + k];
      c_o[t + k] = c[s + k];
      a_o[t + k] = a[s + k];
    }
  }
}

// sum_i a_ij^2 per item in 64-bit fixed point (exact, order independent).
__global__ void k_item_sq(const int32_t* col, const void* a, bool bf16, int64_t nnz, float scale,
                          unsigned long long* acc) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float av = load_val(a, e, bf16);
    atomicAdd(&acc[col[e]], static_cast<unsigned long long>(__float2ll_rn(av * av * scale)));
  }
}

__global__ void k_fix_to_double(const unsigned long long* acc, int64_t J, double inv_scale, double* out) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < J;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[j] = static_cast<double>(static_cast<long long>(acc[j])) * inv_scale;
}

int grid_for(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

}  // namespace

// Fixed-point exponent for sums bounded by `bound`: the largest s with
// bound * 2^s <= 2^61 (two bits of headroom), clamped to [0, 100].
int fixed_point_shift(double bound) {
  if (!(bound > 0)) return 60;
  int s = static_cast<int>(std::floor(61.0 - std::log2(bound)));
  if (s > 100) s = 100;
  return s;
}

#define DLM_CK(x)                                                   \
  do {                                                              \
    cudaError_t e_ = (x);                                           \
    if (e_ != cudaSuccess) {                                        \
      *msg = std::string("CUDA error in layout: ") + cudaGetErrorString(e_); \
      goto fail;                                                    \
    }                                                               \
  } while (0)

dlm_status build_layout(int64_t I, int64_t J, int64_t nnz, const int64_t* rp, const int32_t* col, const void* c,
                        const void* a, const double* b, bool bf16, cudaStream_t s, LayoutOut* out,
                        std::string* msg) {
  const size_t vs = bf16 ? 2 : 4;
  dlm_status st = DLM_OK;
  int32_t *cls = nullptr, *cls_sorted = nullptr, *idx = nullptr, *perm = nullptr;
  int64_t* deg_p = nullptr;
  unsigned long long *class_cnt = nullptr, *item_deg = nullptr, *sq = nullptr;
  unsigned* mx = nullptr;
  int* bad = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  int h_bad = 0;
  unsigned h_mx[2] = {0, 0};
  unsigned long long h_cnt[kNumClasses];
  std::vector<unsigned long long> h_deg;
  double bound_sq = 0;
  int ssq = 0;

  DLM_CK(cudaMalloc(&cls, sizeof(int32_t) * (I > 0 ? I : 1)));
  DLM_CK(cudaMalloc(&class_cnt, sizeof(unsigned long long) * kNumClasses));
  DLM_CK(cudaMalloc(&item_deg, sizeof(unsigned long long) * (J > 0 ? J : 1)));
  DLM_CK(cudaMalloc(&mx, sizeof(unsigned) * 2));
  DLM_CK(cudaMalloc(&bad, sizeof(int)));
  DLM_CK(cudaMemsetAsync(class_cnt, 0, sizeof(unsigned long long) * kNumClasses, s));
  DLM_CK(cudaMemsetAsync(item_deg, 0, sizeof(unsigned long long) * (J > 0 ? J : 1), s));
  DLM_CK(cudaMemsetAsync(mx, 0, sizeof(unsigned) * 2, s));
  DLM_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (I > 0) k_rows<<<grid_for(I), kT, 0, s>>>(rp, I, nnz, cls, class_cnt, bad);
  DLM_CK(cudaGetLastError());
  if (J > 0) k_b<<<grid_for(J), kT, 0, s>>>(b, J, bad);
  DLM_CK(cudaGetLastError());
  DLM_CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  DLM_CK(cudaStreamSynchronize(s));
  if (h_bad & kBadRowPtr) {
    *msg = "row_ptr must start at 0, be non-decreasing and end at nnz";
    st = DLM_ERR_INVALID_ARG;
    goto done;
  }
  if (h_bad & kBadB) {
    *msg = "b must be finite and >= 0";
    st = DLM_ERR_INVALID_ARG;
    goto done;
  }
  if (nnz > 0) k_edges<<<grid_for(nnz), kT, 0, s>>>(col, c, a, bf16, nnz, J, item_deg, mx, mx + 1, bad);
  DLM_CK(cudaGetLastError());
  DLM_CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  DLM_CK(cudaMemcpyAsync(h_mx, mx, sizeof(unsigned) * 2, cudaMemcpyDeviceToHost, s));
  DLM_CK(cudaMemcpyAsync(h_cnt, class_cnt, sizeof(h_cnt), cudaMemcpyDeviceToHost, s));
  h_deg.resize(J > 0 ? J : 1);
  DLM_CK(cudaMemcpyAsync(h_deg.data(), item_deg, sizeof(unsigned long long) * h_deg.size(), cudaMemcpyDeviceToHost,
                         s));
  DLM_CK(cudaStreamSynchronize(s));
  if (h_bad & kBadItem) {
    *msg = "item_idx out of range [0, num_items)";
    st = DLM_ERR_INVALID_ARG;
    goto done;
  }
  if (h_bad & kBadValue) {
    *msg = "c and a must be finite";
    st = DLM_ERR_INVALID_ARG;
    goto done;
  }
  out->a_nonneg = !(h_bad & kNegA);
  {
    float fa, fc;
    memcpy(&fa, &h_mx[0], 4);
    memcpy(&fc, &h_mx[1], 4);
    out->max_abs_a = fa;
    out->max_abs_c = fc;
  }
  out->max_item_deg = 0;
  for (int64_t j = 0; j < J; ++j)
    if (static_cast<int64_t>(h_deg[j]) > out->max_item_deg) out->max_item_deg = static_cast<int64_t>(h_deg[j]);
  {
    int64_t acc = 0;
    for (int k = 0; k < kNumClasses; ++k) {
      out->class_count[k] = static_cast<int64_t>(h_cnt[k]);
      out->class_begin[k] = acc;
      acc += static_cast<int64_t>(h_cnt[k]);
    }
    out->class_begin[kNumClasses] = acc;
  }

  // ---- stable sort of users by degree class ----
  DLM_CK(cudaMalloc(&cls_sorted, sizeof(int32_t) * (I > 0 ? I : 1)));
  DLM_CK(cudaMalloc(&idx, sizeof(int32_t) * (I > 0 ? I : 1)));
  DLM_CK(cudaMalloc(&perm, sizeof(int32_t) * (I > 0 ? I : 1)));
  if (I > 0) {
    k_iota<<<grid_for(I), kT, 0, s>>>(idx, I);
    DLM_CK(cudaGetLastError());
    DLM_CK(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, cls, cls_sorted, idx, perm, I, 0, 4, s));
    DLM_CK(cudaMalloc(&tmp, tmp_bytes > 0 ? tmp_bytes : 16));
    DLM_CK(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, cls, cls_sorted, idx, perm, I, 0, 4, s));
    DLM_CK(cudaFree(tmp));
    tmp = nullptr;
  }

  // ---- bucketed row pointer and caller offsets ----
  DLM_CK(cudaMalloc(&deg_p, sizeof(int64_t) * (I > 0 ? I : 1)));
  DLM_CK(cudaMalloc(&out->rp, sizeof(int64_t) * (I + 1)));
  DLM_CK(cudaMalloc(&out->orig_off, sizeof(int64_t) * (I > 0 ? I : 1)));
  if (I > 0) k_perm_deg<<<grid_for(I), kT, 0, s>>>(rp, perm, I, deg_p, out->orig_off);
  DLM_CK(cudaGetLastError());
  DLM_CK(cudaMemsetAsync(out->rp, 0, sizeof(int64_t), s));
  if (I > 0) {
    tmp_bytes = 0;
    DLM_CK(cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, deg_p, out->rp + 1, I, s));
    DLM_CK(cudaMalloc(&tmp, tmp_bytes > 0 ? tmp_bytes : 16));
    DLM_CK(cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, deg_p, out->rp + 1, I, s));
    DLM_CK(cudaFree(tmp));
    tmp = nullptr;
  }

  // ---- edge arrays in bucketed order ----
  DLM_CK(cudaMalloc(&out->col, sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
  DLM_CK(cudaMalloc(&out->c, vs * (nnz > 0 ? nnz : 1)));
  DLM_CK(cudaMalloc(&out->a, vs * (nnz > 0 ? nnz : 1)));
  if (I > 0) {
    const int g = grid_for(I * 32);
    if (bf16)
      k_gather<unsigned short><<<g, kT, 0, s>>>(col, static_cast<const unsigned short*>(c),
                                                 static_cast<const unsigned short*>(a), out->orig_off, out->rp, I,
                                                 out->col, static_cast<unsigned short*>(out->c),
                                                 static_cast<unsigned short*>(out->a));
    else
      k_gather<float><<<g, kT, 0, s>>>(col, static_cast<const float*>(c), static_cast<const float*>(a),
                                        out->orig_off, out->rp, I, out->col, static_cast<float*>(out->c),
                                        static_cast<float*>(out->a));
    DLM_CK(cudaGetLastError());
  }

  // ---- n_j = sum_i a_ij^2 (exact fixed point) ----
  bound_sq = static_cast<double>(out->max_item_deg) * out->max_abs_a * out->max_abs_a;
  ssq = fixed_point_shift(bound_sq);
  DLM_CK(cudaMalloc(&sq, sizeof(unsigned long long) * (J > 0 ? J : 1)));
  DLM_CK(cudaMalloc(&out->n2, sizeof(double) * (J > 0 ? J : 1)));
  DLM_CK(cudaMemsetAsync(sq, 0, sizeof(unsigned long long) * (J > 0 ? J : 1), s));
  if (nnz > 0) k_item_sq<<<grid_for(nnz), kT, 0, s>>>(col, a, bf16, nnz, std::ldexp(1.0f, ssq), sq);
  DLM_CK(cudaGetLastError());
  if (J > 0) k_fix_to_double<<<grid_for(J), kT, 0, s>>>(sq, J, std::ldexp(1.0, -ssq), out->n2);
  DLM_CK(cudaGetLastError());
  {
    std::vector<double> n2(J > 0 ? J : 1);
    DLM_CK(cudaMemcpyAsync(n2.data(), out->n2, sizeof(double) * n2.size(), cudaMemcpyDeviceToHost, s));
    DLM_CK(cudaStreamSynchronize(s));
    out->n2max = 0;
    for (int64_t j = 0; j < J; ++j) out->n2max = n2[j] > out->n2max ? n2[j] : out->n2max;
  }
  goto done;

fail:
  st = DLM_ERR_CUDA;
done:
  cudaStreamSynchronize(s);
  cudaFree(cls);
  cudaFree(cls_sorted);
  cudaFree(idx);
  cudaFree(perm);
  cudaFree(deg_p);
  cudaFree(class_cnt);
  cudaFree(item_deg);
  cudaFree(sq);
  cudaFree(mx);
  cudaFree(bad);
  if (tmp) cudaFree(tmp);
  if (st != DLM_OK) {
    cudaFree(out->rp);
    cudaFree(out->col);
    cudaFree(out->c);
    cudaFree(out->a);
    cudaFree(out->orig_off);
    cudaFree(out->n2);
    out->rp = nullptr;
    out->col = nullptr;
    out->c = out->a = nullptr;
    out->orig_off = nullptr;
    out->n2 = nullptr;
  }
  return st;
}

}  // namespace dlm
