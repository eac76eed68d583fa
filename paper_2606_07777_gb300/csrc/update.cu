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
//   lam+_j = max(0, y_j + step_j G_j),  step_j = gamma / max_k h_k  (1/L)
//                                         or gamma / h_j (row normalization)
//   theta+ = (1 + sqrt(1 + 4 theta^2)) / 2,  y+ = lam+ + (theta - 1)/theta+ (lam+ - lam)
// and, when iteration t+1 starts a stage with a different gamma, a momentum
// restart (theta = 1, y+ = lam+).  With adaptive restart on, the momentum also
// restarts when the step just taken points against the momentum in the
// step metric: sum_j (lam+_j - y_j) (lam+_j - lam_j) / step_j < 0 (the
// gradient-mapping test of O'Donoghue & Candes 2015, for ascent).
// The iterate lam, y is FP64 (G from the exact fixed-point sum minus b in
// FP64; products and sums rounded separately, no fused multiply-add, as the
// FP64 reference arithmetic of the method takes them); the sweeps read FP32
// copies written here.  The kernel also records the dual objective at the
// sweep point (Sec. 3.2, Eq. dual):
//   g(y) = sum_i (c x + gamma/2 x^2) + y^T G,
// from the sweep's exact fixed-point objective sum and an FP64 dot product in
// a fixed order, into the trajectory slot t mod kTrajCap.
constexpr int kUpdPer = 4;          // coordinates per thread whose loads are issued together
constexpr int kFistaThreads = 512;  // threads of the update CTA (registers for kUpdPer coordinates)

// Sums of two values over the block in a fixed order; results valid in thread 0.
__device__ void block_sum2(double& a, double& b, double (*sh)[32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(kFull, a, o);
    b += __shfl_down_sync(kFull, b, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    sh[0][w] = a;
    sh[1][w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = 0.0;
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) {
      a += sh[0][k];
      b += sh[1][k];
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kFistaThreads) fista_update_kernel(const UpdInst* __restrict__ tab) {
  __shared__ double sh[2][32];
  __shared__ int s_restart;
  const UpdInst U = tab[blockIdx.x];
  const DevState st = *U.state;
  const double gamma = st.gamma;
  const int64_t t1 = st.iter + 1;
  const int64_t s1 = t1 / U.iters_per_stage;
  const double gamma1 = U.gamma_tab[s1 < U.nstages ? s1 : U.nstages - 1];
  const bool stage_restart = gamma1 != gamma;
  const double th1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * st.theta * st.theta));
  const double beta = (st.theta - 1.0) / th1;
  const double step0 = U.curv_max > 0.0 ? gamma / U.curv_max : 0.0;
  // coordinates 0..ncap-1 are (family, item) pairs; ncap is the count dual
  // when present
  const int NC = U.ncap;
  const int D = NC + (U.count_on ? 1 : 0);
  unsigned long long* __restrict__ acc = U.acc;
  const double* __restrict__ b = U.b;
  const double* __restrict__ curv = U.curv;
  double* __restrict__ lam64 = U.lam64;
  double* __restrict__ y64 = U.y64;
  float* __restrict__ lam32 = U.lam;
  float* __restrict__ y32 = U.y;
  const bool pre = U.precondition != 0;
  const bool test = U.adaptive_restart && !stage_restart;  // the restart test decides before any write
  const double count_G = U.count_on ? to_real(*U.cnt, U.inv_scaleN) - U.count_M : 0.0;
  auto step_of = [&](double h) { return pre ? (h > 0.0 ? gamma / h : 0.0) : step0; };
  auto lam_next = [&](double G, double step, double yj) {
    const double v = __dadd_rn(yj, __dmul_rn(step, G));
    return v > 0.0 ? v : 0.0;
  };
  const int stride = static_cast<int>(blockDim.x);
  double lg = 0.0, dot = 0.0, bad = 0.0;
  bool restart = stage_restart;
  // One pass loads kUpdPer coordinates per thread at once (their loads are
  // independent); pass 0 runs only for the restart test, pass 1 writes.
  for (int pass = test ? 0 : 1; pass < 2; ++pass) {
    for (int j0 = threadIdx.x; j0 < D; j0 += stride * kUpdPer) {
      double G[kUpdPer], yv[kUpdPer], lv[kUpdPer], hv[kUpdPer];
      float yf[kUpdPer];
#pragma unroll
      for (int q = 0; q < kUpdPer; ++q) {
        const int j = j0 + q * stride;
        G[q] = yv[q] = lv[q] = hv[q] = 0.0;
        yf[q] = 0.f;
        if (j < D) {
          G[q] = j < NC ? to_real(acc[j], U.inv_scaleG) - __ldg(b + j) : count_G;
          yf[q] = y32[j];
          yv[q] = y64[j];
          lv[q] = lam64[j];
          if (pre) hv[q] = __ldg(curv + j);
        }
      }
#pragma unroll
      for (int q = 0; q < kUpdPer; ++q) {
        const int j = j0 + q * stride;
        if (j >= D) continue;
        const double step = step_of(hv[q]);
        const double ln = lam_next(G[q], step, yv[q]);
        if (pass == 0) {
          // dual objective at the point the sweep read (the FP32 copy of y)
          lg += static_cast<double>(yf[q]) * G[q];
          if (step > 0.0) dot += __ddiv_rn(__dmul_rn(ln - yv[q], ln - lv[q]), step);
        } else {
          if (!test) lg += static_cast<double>(yf[q]) * G[q];
          const double yn = restart ? ln : __dadd_rn(ln, __dmul_rn(beta, ln - lv[q]));
          lam64[j] = ln;
          y64[j] = yn;
          lam32[j] = static_cast<float>(ln);
          y32[j] = static_cast<float>(yn);
          if (j < NC) acc[j] = 0ull;
          if (!isfinite(G[q]) || !isfinite(yv[q]) || !isfinite(yn)) bad = 1.0;
        }
      }
    }
    if (pass == 0) {
      block_sum2(lg, dot, sh);
      if (threadIdx.x == 0) s_restart = dot < 0.0;
      __syncthreads();
      restart = s_restart != 0;
    }
  }
  double lg2 = test ? 0.0 : lg;
  block_sum2(lg2, bad, sh);
  if (threadIdx.x == 0) {
    if (!test) lg = lg2;
    const double g = to_real(*U.objq, U.inv_scaleO) + lg;
    *U.objq = 0ull;
    if (U.count_on) *U.cnt_rw = 0ull;
    U.traj[st.iter % kTrajCap] = g;
    DevState n = st;
    n.iter = t1;
    n.theta = restart ? 1.0 : th1;
    n.gamma = gamma1;
    n.stage = static_cast<int32_t>(s1 < 0x7fffffff ? s1 : 0x7fffffff);
    if (bad > 0.0 || !isfinite(g)) n.status |= kStatNumeric;
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
  fista_update_kernel<<<ninst, kFistaThreads, 0, s>>>(dev_tab);
  return cudaGetLastError();
}

cudaError_t launch_stats(const StatsInst* dev_tab, int ninst, cudaStream_t s) {
  stats_kernel<<<ninst, kUpdThreads, 0, s>>>(dev_tab);
  return cudaGetLastError();
}

}  // namespace dlm
