// layout.cu -- one-time set-up of an instance: input validation, the
// degree-sorted sliced layout the sweep reads, and per-item constants
// (sum_i a_ij^2 for the step size and row normalization, App. B.2; item
// degrees and value bounds for the fixed-point scales).
//
// The caller's CSR is user-major (one row per user; the paper's CSC with one
// column per source, Sec. 4.1).  Users are stably sorted by degree, largest
// first (the paper buckets by degree to limit padding, Sec. 4.2; sorting by
// the exact degree takes that to its limit), and cut into slices of 32
// consecutive users.  A slice of width w (its largest degree) holds 32 w
// elements per stream (item index; interleaved (c, a)).  Its first 4 (w / 4)
// edges of every user are stored in groups of four: edge k < 4 (w / 4) of
// user t at slice_off + 4 (32 (k / 4) + t) + k % 4, so that lane t reads four
// consecutive edges of its user with one 128-bit value load (one float2 pair
// per edge in FP32: two 128-bit loads) and a warp load covers 512 contiguous
// bytes.  The remaining w % 4 edges follow edge-major: edge k at
// slice_off + 128 (w / 4) + 32 (k - 4 (w / 4)) + t.  Edges past a user's
// degree are padding with c = +inf, a = 0 (they give u = -inf and are never
// active).  Users with no edges are dropped from the slices.  The item index
// stream is written as uint16 (every handle has fewer than 65,536 items), so
// four indices are one 64-bit load.
//
// Device memory comes from a stream-ordered pool per device that keeps what
// handles free (dev_alloc / dev_free): a daily re-creation of an instance of
// the same size then maps no new memory.
#include <cub/cub.cuh>

#include <chrono>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "dlm_impl.cuh"

namespace dlm {
namespace {

constexpr int kT = 256;

enum : int { kBadRowPtr = 1, kBadItem = 2, kBadValue = 4, kBadB = 8, kNegA = 16, kDupItem = 32 };
constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kDupThreads = 256;

__device__ __forceinline__ float load_val(const void* p, int64_t e, bool bf16) {
  if (bf16) {
    const unsigned short b = reinterpret_cast<const unsigned short*>(p)[e];
    return __uint_as_float(static_cast<unsigned>(b) << 16);
  }
  return reinterpret_cast<const float*>(p)[e];
}

// Row pointer checks; degree of every user; users with no edges.
__global__ void k_rows(const int64_t* rp, int64_t I, int64_t nnz, int32_t* deg, unsigned long long* zero_cnt,
                       int* bad) {
  int flag = 0;
  unsigned long long z = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < I;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r0 = rp[i], r1 = rp[i + 1];
    const int64_t d = r1 - r0;
    if (d < 0 || r0 < 0 || r1 > nnz || d > 0x7fffffff) flag |= kBadRowPtr;
    deg[i] = d < 0 ? 0 : static_cast<int32_t>(d);
    z += (d == 0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (rp[0] != 0 || rp[I] != nnz) flag |= kBadRowPtr;
  }
  if (flag) atomicOr(bad, flag);
  if (z) atomicAdd(zero_cnt, z);
}

// Edge checks, item degrees, max |a|, max |c|.  With J <= 16384 each block
// counts its contiguous edge range in shared memory and flushes once per item.
__global__ void k_edges(const int32_t* col, const void* c, const void* a, bool bf16, int64_t nnz, int64_t J,
                        unsigned long long* item_deg, unsigned* max_a, unsigned* max_c, int* bad) {
  extern __shared__ unsigned scnt[];
  __shared__ unsigned s_ma, s_mc;
  const bool sm = J <= 16384;
  if (threadIdx.x == 0) s_ma = s_mc = 0;
  if (sm)
    for (int64_t j = threadIdx.x; j < J; j += blockDim.x) scnt[j] = 0u;
  __syncthreads();
  int flag = 0;
  unsigned ma = 0, mc = 0;
  const int64_t per = (nnz + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * per, e1 = e0 + per < nnz ? e0 + per : nnz;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int32_t j = col[e];
    if (j < 0 || j >= J)
      flag |= kBadItem;
    else if (sm)
      atomicAdd(&scnt[j], 1u);
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
  if (sm)
    for (int64_t j = threadIdx.x; j < J; j += blockDim.x)
      if (scnt[j]) atomicAdd(&item_deg[j], static_cast<unsigned long long>(scnt[j]));
}

// Items distinct within each row (the eligible set of Sec. 3.3 is a set of
// (user, item) pairs).  A warp takes 32 consecutive rows, whose edges are
// contiguous: it touches them once (prefetch to L1), then checks one row at a
// time -- a row of at most 32 edges by __match_any_sync over the lanes'
// items, a longer one by marking its items in a per-warp bitmap of J bits in
// shared memory, cleared again after the row.  Runs after the row pointers
// are checked; items outside [0, J) are skipped here (k_edges flags them).
__global__ void k_dups(const int64_t* rp, const int32_t* col, int64_t I, int64_t J, int* bad) {
  extern __shared__ unsigned bm[];
  const int lane = threadIdx.x & 31;
  const int words = static_cast<int>((J + 31) >> 5);
  unsigned* my = bm + static_cast<size_t>(threadIdx.x >> 5) * words;
  for (int k = lane; k < words; k += 32) my[k] = 0u;
  __syncwarp();
  const int64_t gw = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  int flag = 0;
  for (int64_t i0 = 32 * gw; i0 < I; i0 += 32 * nw) {
    const int nrow = static_cast<int>(I - i0 < 32 ? I - i0 : 32);
    const int64_t rk = lane < nrow ? rp[i0 + lane] : 0;
    const int64_t rend = rp[i0 + nrow];
    const int64_t e0 = __shfl_sync(kFullMask, rk, 0);
    for (int64_t e = e0 + 32 * static_cast<int64_t>(lane); e < rend; e += 32 * 32)
      asm volatile("prefetch.global.L1 [%0];" ::"l"(col + e));
    for (int r = 0; r < nrow; ++r) {
      const int64_t s = __shfl_sync(kFullMask, rk, r);
      const int64_t t = __shfl_sync(kFullMask, rk, r + 1 < nrow ? r + 1 : 0);
      const int64_t e = r + 1 < nrow ? t : rend;
      const int64_t d = e - s;
      if (d <= 1) continue;  // warp-uniform
      if (d > J) {           // more edges than items: some item repeats
        flag = 1;
        continue;
      }
      if (d <= 32) {
        const int j = lane < d ? col[s + lane] : -1 - lane;  // idle lanes: distinct negative keys
        if (__popc(__match_any_sync(kFullMask, j)) > 1) flag = 1;
      } else {
        for (int64_t q = s + lane; q < e; q += 32) {
          const int j = col[q];
          if (static_cast<unsigned>(j) >= static_cast<unsigned>(J)) continue;
          const unsigned bit = 1u << (j & 31);
          if (atomicOr(&my[j >> 5], bit) & bit) flag = 1;
        }
        __syncwarp();
        for (int64_t q = s + lane; q < e; q += 32) {
          const int j = col[q];
          if (static_cast<unsigned>(j) < static_cast<unsigned>(J)) my[j >> 5] = 0u;
        }
        __syncwarp();
      }
    }
  }
  if (__any_sync(kFullMask, flag) && lane == 0) atomicOr(bad, kDupItem);
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

// Slice widths (edges per lane) and slice sizes in elements (32 w).
__global__ void k_slices(const int32_t* sdeg, int64_t nslices, int32_t* width, int64_t* size) {
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < nslices;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t w = sdeg[32 * s];  // largest degree of the slice (sorted descending)
    width[s] = w;
    size[s] = 32 * static_cast<int64_t>(w);
  }
}

// The cost c of edge e as a float (bf16 bits widened exactly, or FP32).
template <typename CA>
__device__ __forceinline__ float cost_of(const void* c, int64_t e);
template <>
__device__ __forceinline__ float cost_of<float2>(const void* c, int64_t e) {
  return static_cast<const float*>(c)[e];
}
template <>
__device__ __forceinline__ float cost_of<uint32_t>(const void* c, int64_t e) {
  return __uint_as_float(static_cast<uint32_t>(static_cast<const unsigned short*>(c)[e]) << 16);
}

// One warp per slice: lane t copies user t's row into column t of the slice,
// in lead order (dlm_impl.cuh: the row's four lowest-cost edges first).
// CA = float2 {c, a} (FP32) or uint32 (bf16 c low, bf16 a high).
template <typename CA>
__device__ __forceinline__ CA pack_ca(const void* c, const void* a, int64_t e);
template <>
__device__ __forceinline__ float2 pack_ca<float2>(const void* c, const void* a, int64_t e) {
  return make_float2(static_cast<const float*>(c)[e], static_cast<const float*>(a)[e]);
}
template <>
__device__ __forceinline__ uint32_t pack_ca<uint32_t>(const void* c, const void* a, int64_t e) {
  return static_cast<uint32_t>(static_cast<const unsigned short*>(c)[e]) |
         (static_cast<uint32_t>(static_cast<const unsigned short*>(a)[e]) << 16);
}
template <typename CA>
__device__ __forceinline__ CA pad_ca();
template <>
__device__ __forceinline__ float2 pad_ca<float2>() {
  return make_float2(INFINITY, 0.f);
}
template <>
__device__ __forceinline__ uint32_t pad_ca<uint32_t>() {
  return 0x00007F80u;  // c = bf16 +inf, a = 0
}

template <typename CA>
__global__ void k_gather(const int64_t* rp, const int32_t* col, const void* c, const void* a, const int32_t* perm,
                         const int32_t* sdeg, int64_t In, int64_t nslices, const int64_t* slice_off,
                         const int32_t* width, uint16_t* col_o, CA* ca_o, int64_t* orig_off, int32_t* udeg,
                         uint64_t* lead_o) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = w0; s < nslices; s += nwarps) {
    const int64_t u = 32 * s + lane;
    int64_t r = 0;
    int d = 0;
    if (u < In) {
      const int32_t o = perm[u];
      r = rp[o];
      d = sdeg[u];
      orig_off[u] = r;
      udeg[u] = d;
    }
    // lead edges: min(4, d) edges of the row's lowest costs, ascending, by a
    // sorted insertion with strict comparisons (a deterministic choice among
    // edges of equal cost)
    float lv[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
    int lp[4] = {0, 0, 0, 0};
    for (int k = 0; k < d && k < 0xFFFF; ++k) {  // positions fit 16 bits
      float x = cost_of<CA>(c, r + k);
      int xi = k;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool lt = x < lv[q];
        const float hv = lt ? lv[q] : x;
        const int hi = lt ? lp[q] : xi;
        lv[q] = lt ? x : lv[q];
        lp[q] = lt ? xi : lp[q];
        x = hv;
        xi = hi;
      }
    }
    uint64_t lead = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) lead |= static_cast<uint64_t>(q < d ? lp[q] : 0xFFFF) << (16 * q);
    if (u < In) lead_o[u] = lead;
    const int w = width[s];
    const int w4 = w >> 2;
    const int64_t base = slice_off[s];
    for (int k = 0; k < w; ++k) {
      const bool v = k < d;
      const int64_t e = k < 4 * w4 ? base + 4 * (32 * static_cast<int64_t>(k >> 2) + lane) + (k & 3)
                                   : base + 128 * static_cast<int64_t>(w4) + 32 * static_cast<int64_t>(k - 4 * w4) + lane;
      const int64_t src = v ? r + lead_caller_pos(lead, k, d) : 0;
      col_o[e] = v ? static_cast<uint16_t>(col[src]) : uint16_t(0);
      ca_o[e] = v ? pack_ca<CA>(c, a, src) : pad_ca<CA>();
    }
  }
}


// sum_i a_ij^2 (or sum_i a_ij) per item in 64-bit fixed point (exact, order
// independent).
// With J <= kSmemItems each block sums its contiguous edge range in shared
// memory and flushes once per item.
constexpr int kSmemItems = 16384;
__global__ void k_item_sq(const int32_t* col, const void* a, bool bf16, int64_t nnz, int64_t J, float scale,
                          bool square, unsigned long long* acc) {
  extern __shared__ unsigned long long sacc[];
  const bool sm = J <= kSmemItems;
  if (sm) {
    for (int64_t j = threadIdx.x; j < J; j += blockDim.x) sacc[j] = 0ull;
    __syncthreads();
  }
  const int64_t per = (nnz + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * per, e1 = e0 + per < nnz ? e0 + per : nnz;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const float av = load_val(a, e, bf16);
    const unsigned long long q = static_cast<unsigned long long>(__float2ll_rn((square ? av * av : av) * scale));
    if (sm)
      atomicAdd(&sacc[col[e]], q);
    else
      atomicAdd(&acc[col[e]], q);
  }
  if (sm) {
    __syncthreads();
    for (int64_t j = threadIdx.x; j < J; j += blockDim.x)
      if (sacc[j]) atomicAdd(&acc[j], sacc[j]);
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

std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&g_pool[dev], &props);
      if (e != cudaSuccess) {
        g_pool[dev] = nullptr;
        return e;
      }
      uint64_t keep = UINT64_MAX;  // freed memory stays with the pool until dlm_release_cached_memory
      e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 16, pool, s);
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

cudaError_t release_cached_memory() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  cudaError_t first = cudaSuccess;
  for (cudaMemPool_t& q : g_pool) {
    if (!q) continue;
    const cudaError_t e = cudaMemPoolTrimTo(q, 0);
    if (e != cudaSuccess && first == cudaSuccess) first = e;
  }
  return first;
}

// Fixed-point exponent for sums bounded by `bound`: the largest s with
// bound * 2^s <= 2^61 (two bits of headroom), clamped to [0, 100].
int fixed_point_shift(double bound) {
  if (!(bound > 0)) return 60;
  int s = static_cast<int>(std::floor(61.0 - std::log2(bound)));
  if (s > 100) s = 100;
  return s;
}

#define DLM_CK(x)                                                            \
  do {                                                                       \
    cudaError_t e_ = (x);                                                    \
    if (e_ != cudaSuccess) {                                                 \
      *msg = std::string("CUDA error in layout: ") + cudaGetErrorString(e_); \
      goto fail;                                                             \
    }                                                                        \
  } while (0)

void item_sum_shifts(int64_t max_item_deg, double max_abs_a, int* ssq, int* ss1) {
  *ssq = fixed_point_shift(static_cast<double>(max_item_deg) * max_abs_a * max_abs_a);
  *ss1 = fixed_point_shift(static_cast<double>(max_item_deg) * max_abs_a);
}

dlm_status item_sums(int64_t J, int64_t nnz, const int32_t* col, const void* a, bool bf16, int ssq, int ss1,
                     cudaStream_t s, int64_t* sq, int64_t* s1, std::string* msg) {
  cudaFuncSetAttribute(k_item_sq, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kSmemItems);
  unsigned long long* acc = nullptr;
  dlm_status st = DLM_OK;
  const int g = static_cast<int>(nnz / 8192 + 1 < 608 ? nnz / 8192 + 1 : 608);
  const size_t smem = J <= kSmemItems ? sizeof(unsigned long long) * J : 0;
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&acc), sizeof(unsigned long long) * 2 * (J > 0 ? J : 1), s));
  DLM_CK(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 2 * (J > 0 ? J : 1), s));
  if (nnz > 0) {
    k_item_sq<<<g, 1024, smem, s>>>(col, a, bf16, nnz, J, std::ldexp(1.0f, ssq), true, acc);
    DLM_CK(cudaGetLastError());
    k_item_sq<<<g, 1024, smem, s>>>(col, a, bf16, nnz, J, std::ldexp(1.0f, ss1), false, acc + J);
    DLM_CK(cudaGetLastError());
  }
  DLM_CK(cudaMemcpyAsync(sq, acc, sizeof(int64_t) * J, cudaMemcpyDeviceToHost, s));
  DLM_CK(cudaMemcpyAsync(s1, acc + J, sizeof(int64_t) * J, cudaMemcpyDeviceToHost, s));
  DLM_CK(cudaStreamSynchronize(s));
  goto done;
fail:
  st = DLM_ERR_CUDA;
done:
  dev_free(acc, s);
  cudaStreamSynchronize(s);
  return st;
}

dlm_status build_layout(int64_t I, int64_t J, int64_t nnz, const int64_t* rp, const int32_t* col, const void* c,
                        const void* a, const double* b, bool bf16, cudaStream_t s, LayoutOut* out,
                        std::string* msg, RowStats* measure, const ShardGlobal* shard) {
  const auto t_start = std::chrono::steady_clock::now();
  auto lap = [&](int k) {
    out->phase_s[k] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() -
                      (k > 0 ? out->phase_s[0] : 0.0) - (k > 1 ? out->phase_s[1] : 0.0);
  };
  const size_t vs = bf16 ? 2 : 4;
  cudaFuncSetAttribute(k_item_sq, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kSmemItems);
  cudaFuncSetAttribute(k_edges, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 16384);
  dlm_status st = DLM_OK;
  int32_t *deg = nullptr, *sdeg = nullptr, *idx = nullptr, *perm = nullptr;
  int64_t* ssize = nullptr;
  unsigned long long *zero_cnt = nullptr, *item_deg = nullptr, *sq = nullptr;
  unsigned* mx = nullptr;
  int* bad = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  int h_bad = 0;
  unsigned h_mx[2] = {0, 0};
  unsigned long long h_zero = 0;
  std::vector<unsigned long long> h_deg;
  double bound_sq = 0;
  int ssq = 0;
  int64_t In = 0, ns = 0;

  DLM_CK(dev_alloc(reinterpret_cast<void**>(&deg), sizeof(int32_t) * (I > 0 ? I : 1), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&zero_cnt), sizeof(unsigned long long), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&item_deg), sizeof(unsigned long long) * (J > 0 ? J : 1), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&mx), sizeof(unsigned) * 2, s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&bad), sizeof(int), s));
  DLM_CK(cudaMemsetAsync(zero_cnt, 0, sizeof(unsigned long long), s));
  DLM_CK(cudaMemsetAsync(item_deg, 0, sizeof(unsigned long long) * (J > 0 ? J : 1), s));
  DLM_CK(cudaMemsetAsync(mx, 0, sizeof(unsigned) * 2, s));
  DLM_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (I > 0) k_rows<<<grid_for(I), kT, 0, s>>>(rp, I, nnz, deg, zero_cnt, bad);
  DLM_CK(cudaGetLastError());
  if (J > 0) k_b<<<grid_for(J), kT, 0, s>>>(b, J, bad);
  DLM_CK(cudaGetLastError());
  DLM_CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  DLM_CK(cudaMemcpyAsync(&h_zero, zero_cnt, sizeof(h_zero), cudaMemcpyDeviceToHost, s));
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
  if (nnz > 0) {
    const int g = static_cast<int>(nnz / 8192 + 1 < 608 ? nnz / 8192 + 1 : 608);
    const size_t smem = J <= 16384 ? sizeof(unsigned) * J : 0;
    k_edges<<<g, 1024, smem, s>>>(col, c, a, bf16, nnz, J, item_deg, mx, mx + 1, bad);
    DLM_CK(cudaGetLastError());
    const size_t dsm = sizeof(unsigned) * static_cast<size_t>((J + 31) / 32) * (kDupThreads / 32);
    if (dsm > 48 * 1024) DLM_CK(cudaFuncSetAttribute(k_dups, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(dsm)));
    int dev = 0, sms = 0;
    DLM_CK(cudaGetDevice(&dev));
    DLM_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = (I + kDupThreads - 1) / kDupThreads;
    const int gd = static_cast<int>(want < 8LL * sms ? (want > 0 ? want : 1) : 8LL * sms);
    k_dups<<<gd, kDupThreads, dsm, s>>>(rp, col, I, J, bad);
  }
  DLM_CK(cudaGetLastError());
  DLM_CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  DLM_CK(cudaMemcpyAsync(h_mx, mx, sizeof(unsigned) * 2, cudaMemcpyDeviceToHost, s));
  h_deg.resize(J > 0 ? J : 1);
  DLM_CK(cudaMemcpyAsync(h_deg.data(), item_deg, sizeof(unsigned long long) * h_deg.size(), cudaMemcpyDeviceToHost,
                         s));
  DLM_CK(cudaStreamSynchronize(s));
  lap(0);
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
  if (h_bad & kDupItem) {
    *msg = "an item appears twice in one row (the eligible items of a user must be distinct)";
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
  if (measure) {
    measure->nnz = nnz;
    measure->active_users = I - static_cast<int64_t>(h_zero);
    measure->max_item_deg = out->max_item_deg;
    measure->max_abs_a = out->max_abs_a;
    measure->max_abs_c = out->max_abs_c;
    measure->a_nonneg = out->a_nonneg;
    measure->item_deg.assign(h_deg.begin(), h_deg.begin() + J);
    goto done;
  }
  if (shard) {  // bounds of the whole instance: the fixed-point exponents must agree on every shard
    out->max_item_deg = shard->max_item_deg;
    out->max_abs_a = shard->max_abs_a;
    out->max_abs_c = shard->max_abs_c;
    out->a_nonneg = shard->a_nonneg;
  }

  // ---- stable sort of users by degree, largest first ----
  In = I - static_cast<int64_t>(h_zero);
  ns = (In + 31) / 32;
  out->num_active_users = In;
  out->nslices = ns;
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&sdeg), sizeof(int32_t) * (I + 32), s));
  DLM_CK(cudaMemsetAsync(sdeg, 0, sizeof(int32_t) * (I + 32), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&idx), sizeof(int32_t) * (I > 0 ? I : 1), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&perm), sizeof(int32_t) * (I > 0 ? I : 1), s));
  if (I > 0) {
    k_iota<<<grid_for(I), kT, 0, s>>>(idx, I);
    DLM_CK(cudaGetLastError());
    DLM_CK(cub::DeviceRadixSort::SortPairsDescending(nullptr, tmp_bytes, deg, sdeg, idx, perm, I, 0, 32, s));
    DLM_CK(dev_alloc(reinterpret_cast<void**>(&tmp), tmp_bytes > 0 ? tmp_bytes : 16, s));
    DLM_CK(cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, deg, sdeg, idx, perm, I, 0, 32, s));
    dev_free(tmp, s);
    tmp = nullptr;
  }

  // ---- slices ----
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->slice_w), sizeof(int32_t) * (ns + 1), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->slice_off), sizeof(int64_t) * (ns + 1), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&ssize), sizeof(int64_t) * (ns + 1), s));
  DLM_CK(cudaMemsetAsync(out->slice_off, 0, sizeof(int64_t), s));
  if (ns > 0) {
    k_slices<<<grid_for(ns), kT, 0, s>>>(sdeg, ns, out->slice_w, ssize);
    DLM_CK(cudaGetLastError());
    tmp_bytes = 0;
    DLM_CK(cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, ssize, out->slice_off + 1, ns, s));
    DLM_CK(dev_alloc(reinterpret_cast<void**>(&tmp), tmp_bytes > 0 ? tmp_bytes : 16, s));
    DLM_CK(cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, ssize, out->slice_off + 1, ns, s));
    dev_free(tmp, s);
    tmp = nullptr;
  }
  DLM_CK(cudaMemcpyAsync(&out->padded_nnz, out->slice_off + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DLM_CK(cudaStreamSynchronize(s));
  lap(1);

  // ---- edge streams in slice order (16-bit item indices: every handle has
  // fewer than 65,536 items) ----
  if (J > 65536) {
    *msg = "num_items above 65,536";
    st = DLM_ERR_UNSUPPORTED;
    goto done;
  }
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->col16), sizeof(uint16_t) * (out->padded_nnz + 64), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->ca), 2 * vs * (out->padded_nnz + 32), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->orig_off), sizeof(int64_t) * (In + 32), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->udeg), sizeof(int32_t) * (In + 32), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->lead), sizeof(uint64_t) * (In + 32), s));
  DLM_CK(cudaMemsetAsync(out->col16 + out->padded_nnz, 0, sizeof(uint16_t) * 64, s));
  if (ns > 0) {
    const int g = grid_for(ns * 32);
    if (bf16)
      k_gather<uint32_t><<<g, kT, 0, s>>>(rp, col, c, a, perm, sdeg, In, ns, out->slice_off, out->slice_w, out->col16,
                                          static_cast<uint32_t*>(out->ca), out->orig_off, out->udeg, out->lead);
    else
      k_gather<float2><<<g, kT, 0, s>>>(rp, col, c, a, perm, sdeg, In, ns, out->slice_off, out->slice_w, out->col16,
                                        static_cast<float2*>(out->ca), out->orig_off, out->udeg, out->lead);
    DLM_CK(cudaGetLastError());
  }

  // ---- n_j = sum_i a_ij^2 and s_j = sum_i a_ij (exact fixed point; the
  // whole instance's sums for a shard) ----
  if (shard) {
    int sq_shift = 0, s1_shift = 0;
    item_sum_shifts(out->max_item_deg, out->max_abs_a, &sq_shift, &s1_shift);
    out->h_n2.assign(J > 0 ? J : 1, 0.0);
    out->h_s1.assign(J > 0 ? J : 1, 0.0);
    out->n2max = 0;
    for (int64_t j = 0; j < J; ++j) {
      out->h_n2[j] = static_cast<double>(shard->item_sq[j]) * std::ldexp(1.0, -sq_shift);
      out->h_s1[j] = static_cast<double>(shard->item_sum[j]) * std::ldexp(1.0, -s1_shift);
      out->n2max = out->h_n2[j] > out->n2max ? out->h_n2[j] : out->n2max;
    }
    DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->n2), sizeof(double) * (J > 0 ? J : 1), s));
    DLM_CK(cudaMemcpyAsync(out->n2, out->h_n2.data(), sizeof(double) * out->h_n2.size(), cudaMemcpyHostToDevice, s));
    DLM_CK(cudaStreamSynchronize(s));
    lap(2);
    goto done;
  }
  bound_sq = static_cast<double>(out->max_item_deg) * out->max_abs_a * out->max_abs_a;
  ssq = fixed_point_shift(bound_sq);
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&sq), sizeof(unsigned long long) * (J > 0 ? J : 1), s));
  DLM_CK(dev_alloc(reinterpret_cast<void**>(&out->n2), sizeof(double) * (J > 0 ? J : 1), s));
  DLM_CK(cudaMemsetAsync(sq, 0, sizeof(unsigned long long) * (J > 0 ? J : 1), s));
  if (nnz > 0) {
    const int g = static_cast<int>(nnz / 8192 + 1 < 608 ? nnz / 8192 + 1 : 608);
    const size_t smem = J <= kSmemItems ? sizeof(unsigned long long) * J : 0;
    k_item_sq<<<g, 1024, smem, s>>>(col, a, bf16, nnz, J, std::ldexp(1.0f, ssq), true, sq);
  }
  DLM_CK(cudaGetLastError());
  if (J > 0) k_fix_to_double<<<grid_for(J), kT, 0, s>>>(sq, J, std::ldexp(1.0, -ssq), out->n2);
  DLM_CK(cudaGetLastError());
  out->h_n2.assign(J > 0 ? J : 1, 0.0);
  DLM_CK(cudaMemcpyAsync(out->h_n2.data(), out->n2, sizeof(double) * out->h_n2.size(), cudaMemcpyDeviceToHost, s));
  // ---- s_j = sum_i a_ij (the coupling of item rows with a count row) ----
  ssq = fixed_point_shift(static_cast<double>(out->max_item_deg) * out->max_abs_a);
  DLM_CK(cudaMemsetAsync(sq, 0, sizeof(unsigned long long) * (J > 0 ? J : 1), s));
  if (nnz > 0) {
    const int g = static_cast<int>(nnz / 8192 + 1 < 608 ? nnz / 8192 + 1 : 608);
    const size_t smem = J <= kSmemItems ? sizeof(unsigned long long) * J : 0;
    k_item_sq<<<g, 1024, smem, s>>>(col, a, bf16, nnz, J, std::ldexp(1.0f, ssq), false, sq);
  }
  DLM_CK(cudaGetLastError());
  {
    std::vector<unsigned long long> q(J > 0 ? J : 1);
    DLM_CK(cudaMemcpyAsync(q.data(), sq, sizeof(unsigned long long) * q.size(), cudaMemcpyDeviceToHost, s));
    DLM_CK(cudaStreamSynchronize(s));
    out->h_s1.assign(J > 0 ? J : 1, 0.0);
    for (int64_t j = 0; j < J; ++j)
      out->h_s1[j] = static_cast<double>(static_cast<long long>(q[j])) * std::ldexp(1.0, -ssq);
    out->n2max = 0;
    for (int64_t j = 0; j < J; ++j) out->n2max = out->h_n2[j] > out->n2max ? out->h_n2[j] : out->n2max;
  }
  lap(2);
  goto done;

fail:
  st = DLM_ERR_CUDA;
done:
  dev_free(deg, s);
  dev_free(sdeg, s);
  dev_free(idx, s);
  dev_free(perm, s);
  dev_free(ssize, s);
  dev_free(zero_cnt, s);
  dev_free(item_deg, s);
  dev_free(sq, s);
  dev_free(mx, s);
  dev_free(bad, s);
  dev_free(tmp, s);
  if (st != DLM_OK) {
    dev_free(out->slice_w, s);
    dev_free(out->slice_off, s);
    dev_free(out->col16, s);
    dev_free(out->ca, s);
    dev_free(out->orig_off, s);
    dev_free(out->udeg, s);
    dev_free(out->lead, s);
    dev_free(out->n2, s);
    out->slice_w = nullptr;
    out->slice_off = nullptr;
    out->col16 = nullptr;
    out->ca = nullptr;
    out->orig_off = nullptr;
    out->udeg = nullptr;
    out->lead = nullptr;
    out->n2 = nullptr;
  }
  return st;
}

}  // namespace dlm
