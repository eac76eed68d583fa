// update.cu -- the O(J) kernels that follow a sweep: the accelerated
// projected dual step with gamma continuation, and the dual objective /
// certified-gap statistics.  One CTA per instance; every reduction runs in a
// fixed order (thread-strided, then a fixed shuffle tree, then warps in
// order), so results are bit-identical from run to run.
#include <math.h>

#include "dlm_impl.cuh"

namespace dlm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double to_real(unsigned long long v, double inv_scale) {
  return static_cast<double>(static_cast<long long>(v)) * inv_scale;
}

// Sum over the block in a fixed order; result valid in thread 0.
__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) s += sh[k];
  __syncthreads();
  return s;
}
__device__ double block_max(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(kFull, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = -INFINITY;
  if (threadIdx.x == 0)
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) s = fmax(s, sh[k]);
  __syncthreads();
  return s;
}

// Accelerated projected step (Sec. 4.4; App. B.2), for iteration t at y:
//   G_j    = (A x(y))_j - b_j
//   lam+_j = max(0, y_j + step_j G_j),  step_j = gamma / max_k n_k  (1/L)
//                                         or gamma / n_j (row normalization)
//   theta+ = (1 + sqrt(1 + 4 theta^2)) / 2,  y+ = lam+ + (theta - 1)/theta+ (lam+ - lam)
// and, when iteration t+1 starts a stage with a different gamma, a momentum
// restart (theta = 1, y+ = lam+).  With adaptive restart on, the momentum also
// restarts when the step just taken points against the momentum in the
// step metric: sum_j (lam+_j - y_j) (lam+_j - lam_j) / step_j < 0 (the
// gradient-mapping test of O'Donoghue & Candes 2015, for ascent).  lam and y
// are FP32; G is formed from the exact fixed-point sum minus b and rounded
// once to FP32; the restart test sums in FP64 in a fixed order.
__global__ void __launch_bounds__(kUpdThreads) fista_update_kernel(const UpdInst* __restrict__ tab) {
  __shared__ double sh[32];
  __shared__ int s_restart;
  const UpdInst U = tab[blockIdx.x];
  const DevState st = *U.state;
  const double gamma = st.gamma;
  const int64_t t1 = st.iter + 1;
  const int64_t s1 = t1 / U.iters_per_stage;
  const double gamma1 = U.gamma_tab[s1 < kMaxStages ? s1 : kMaxStages - 1];
  const bool stage_restart = gamma1 != gamma;
  const double th1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * st.theta * st.theta));
  const float beta = static_cast<float>((st.theta - 1.0) / th1);
  const float step0 = static_cast<float>(gamma * U.inv_nmax);
  // coordinates 0..ncap-1 are (family, item) pairs; ncap is the count dual
  // when present
  const int NC = U.ncap;
  const int D = NC + (U.count_on ? 1 : 0);
  auto grad_of = [&](int j) {
    return j < NC ? static_cast<float>(to_real(U.acc[j], U.inv_scaleG) - U.b[j])
                  : static_cast<float>(to_real(*U.cnt, U.inv_scaleN) - U.count_M);
  };
  auto lam_next = [&](int j, float& step, float& yj) {
    const float G = grad_of(j);
    step = U.precondition ? static_cast<float>(gamma * (j < NC ? U.inv_n2[j] : U.inv_h_count)) : step0;
    yj = U.y[j];
    return fmaxf(0.f, fmaf(step, G, yj));
  };
  bool restart = stage_restart;
  if (U.adaptive_restart && !stage_restart) {
    double dot = 0.0;
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
      float step, yj;
      const float ln = lam_next(j, step, yj);
      if (step > 0.f)
        dot += (static_cast<double>(ln) - yj) * (static_cast<double>(ln) - U.lam[j]) / static_cast<double>(step);
    }
    dot = block_sum(dot, sh);
    if (threadIdx.x == 0) s_restart = dot < 0.0;
    __syncthreads();
    restart = s_restart != 0;
  }
  double bad = 0.0;
  __syncthreads();  // every thread has read the count sum before it is reset
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    const float G = grad_of(j);
    float step, yj;
    const float ln = lam_next(j, step, yj);
    const float yn = restart ? ln : fmaf(beta, ln - U.lam[j], ln);
    U.lam[j] = ln;
    U.y[j] = yn;
    if (j < NC)
      U.acc[j] = 0ull;
    else
      *U.cnt_rw = 0ull;
    if (!isfinite(G) || !isfinite(yj) || !isfinite(yn)) bad = 1.0;
  }
  bad = block_max(bad, sh);
  if (threadIdx.x == 0) {
    DevState n = st;
    n.iter = t1;
    n.theta = restart ? 1.0 : th1;
    n.gamma = gamma1;
    n.stage = static_cast<int32_t>(s1 < 0x7fffffff ? s1 : 0x7fffffff);
    if (bad > 0.0) n.status |= kStatNumeric;
    *U.state = n;
  }
}

// Dual value and certified gap at the dual point of the certificate sweep
// (Sec. 3.2 Eq. dual; scaled-point gap as defined in the header):
//   G_j = (A x)_j - b_j,  g = sum_i (c x + gamma/2 x^2) + lam^T G,
//   s_j = min(1, b_j / (A x)_j),  P = sum_j s_j (c x)_j + gamma/2 s_j^2 (x^2)_j.
// With a count constraint sum x <= M (dual mu = lam[J]): g gains mu (sum x - M)
// and every s_j is multiplied by t = min(1, M / sum x), which keeps the scaled
// point within the count (sum_j s_j (sum_i x_ij) <= sum x).  With m capacity
// families, s_j = min over the families of min(1, b_kj / (A_k x)_j).
__global__ void __launch_bounds__(kUpdThreads) stats_kernel(const StatsInst* __restrict__ tab) {
  __shared__ double sh[32];
  const StatsInst S = tab[blockIdx.x];
  const double gamma = *S.gamma;
  double obj = 0.0;
  for (int k = threadIdx.x; k < S.nseg; k += blockDim.x) obj += S.seg_obj[S.seg_list[k]];
  // count constraint: sum x and the common scaling t = min(1, M / sum x)
  const double total = S.count_on ? to_real(*S.cnt, S.inv_sN) : 0.0;
  const double t = (S.count_on && total > S.count_M) ? S.count_M / total : 1.0;
  __syncthreads();  // every thread has read the count sum before it is reset below
  double lg = 0.0, P = 0.0, viol = 0.0;
  const int m = S.m > 0 ? S.m : 1;
  for (int j = threadIdx.x; j < S.J; j += blockDim.x) {
    double s = t;
    for (int f = 0; f < m; ++f) {
      const int q = f * S.J + j;
      const double Ax = to_real(S.acc[q], S.inv_sG);
      const double G = Ax - S.b[q];
      lg += static_cast<double>(S.lam[q]) * G;
      if (Ax > S.b[q]) s = fmin(s, t * (S.b[q] / Ax));
      viol = fmax(viol, G);
      if (S.grad_out) S.grad_out[q] = static_cast<float>(G);
      S.acc[q] = 0ull;
    }
    const double Cx = to_real(S.accC[j], S.inv_sC);
    const double Qx = to_real(S.accQ[j], S.inv_sQ);
    P += s * Cx + 0.5 * gamma * s * s * Qx;
    S.accC[j] = 0ull;
    S.accQ[j] = 0ull;
  }
  if (S.count_on && threadIdx.x == 0) {
    const double G = total - S.count_M;
    lg += static_cast<double>(S.lam[m * S.J]) * G;
    viol = fmax(viol, G);
    if (S.grad_out) S.grad_out[m * S.J] = static_cast<float>(G);
    *S.cnt = 0ull;
  }
  obj = block_sum(obj, sh);
  lg = block_sum(lg, sh);
  P = block_sum(P, sh);
  viol = block_max(viol, sh);
  if (threadIdx.x == 0) {
    const double g = obj + lg;
    const double den = fabs(g) > 1e-30 ? fabs(g) : 1e-30;
    S.out[0] = g;
    S.out[1] = P;
    S.out[2] = S.certified ? (P - g) / den : NAN;
    S.out[3] = -lg / den;
    S.out[4] = viol;
    S.out[5] = obj;
    S.out[6] = S.state ? static_cast<double>(S.state->iter) : 0.0;
    S.out[7] = S.state ? static_cast<double>(S.state->status) : 0.0;
  }
}

}  // namespace

cudaError_t launch_update(const UpdInst* dev_tab, int ninst, cudaStream_t s) {
  fista_update_kernel<<<ninst, kUpdThreads, 0, s>>>(dev_tab);
  return cudaGetLastError();
}

cudaError_t launch_stats(const StatsInst* dev_tab, int ninst, cudaStream_t s) {
  stats_kernel<<<ninst, kUpdThreads, 0, s>>>(dev_tab);
  return cudaGetLastError();
}

}  // namespace dlm
