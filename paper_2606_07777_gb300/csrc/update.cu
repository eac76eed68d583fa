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
// copies written here.  The update also records the dual objective at the
// sweep point (Sec. 3.2, Eq. dual):
//   g(y) = sum_i (c x + gamma/2 x^2) + y^T G,
// from the sweep's exact fixed-point objective sum and an FP64 dot product,
// into the trajectory slot t mod kTrajCap.
//
// Grid: CTA x of row y takes coordinates x kUpdChunk .. of instance y (one
// coordinate per thread: the FP64 work is spread over the SMs).  Scalars
// that need every coordinate -- the dot product of g, the restart test, the
// finiteness flag -- are summed per CTA in a fixed order, written as
// partials, and added in CTA order by the last CTA of the instance to finish
// (an integer ticket; no CTA waits for another), which also writes the new
// iteration state.  With the adaptive restart a first kernel computes the
// test the same way and leaves its decision for the second.
constexpr int kUpdChunk = 256;  // coordinates per update CTA (one per thread)

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

// The step's scalars for iteration t of instance U.
struct StepScalars {
  DevState st;
  int64_t s1;
  double gamma1, th1, beta, step0;
  bool stage_restart, test;
  int NC, D;
};
__device__ __forceinline__ StepScalars step_scalars(const UpdInst& U) {
  StepScalars c;
  c.st = *U.state;
  const int64_t t1 = c.st.iter + 1;
  c.s1 = t1 / U.iters_per_stage;
  c.gamma1 = U.gamma_tab[c.s1 < U.nstages ? c.s1 : U.nstages - 1];
  c.stage_restart = c.gamma1 != c.st.gamma;
  c.th1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * c.st.theta * c.st.theta));
  c.beta = (c.st.theta - 1.0) / c.th1;
  c.step0 = U.curv_max > 0.0 ? c.st.gamma / U.curv_max : 0.0;
  c.test = U.adaptive_restart && !c.stage_restart;  // the restart test decides before any write
  c.NC = U.ncap;
  c.D = c.NC + (U.count_on ? 1 : 0);
  return c;
}

// Coordinate j's gradient, step and candidate lam+ (j < D).
__device__ __forceinline__ void coord(const UpdInst& U, const StepScalars& c, int j, double& G, double& step,
                                      double& yj, double& ln) {
  G = j < c.NC ? to_real(U.acc[j], U.inv_scaleG) - __ldg(U.b + j) : to_real(*U.cnt, U.inv_scaleN) - U.count_M;
  if (U.precondition) {
    const double h = __ldg(U.curv + j);
    step = h > 0.0 ? c.st.gamma / h : 0.0;
  } else {
    step = c.step0;
  }
  yj = U.y64[j];
  const double v = __dadd_rn(yj, __dmul_rn(step, G));
  ln = v > 0.0 ? v : 0.0;
}

// Adds this CTA's two partials and, in the last CTA of the instance to
// arrive, returns true with all of them visible (the ticket is reset).
__device__ __forceinline__ bool arrive(const UpdInst& U, int slot, double a, double b, int* s_last) {
  if (threadIdx.x == 0) {
    U.part[2 * blockIdx.x] = a;
    U.part[2 * blockIdx.x + 1] = b;
    __threadfence();
    const unsigned prev = atomicAdd(&U.ticket[slot], 1u);
    *s_last = prev == static_cast<unsigned>(U.nct) - 1u;
    if (*s_last) {
      __threadfence();
      U.ticket[slot] = 0u;
    }
  }
  __syncthreads();
  return *s_last != 0;
}

// Kernel A (instances with the adaptive restart test due): the test's dot
// product and g's dot product; the last CTA decides and keeps g's part.
__global__ void __launch_bounds__(kUpdChunk) restart_test_kernel(const UpdInst* __restrict__ tab) {
  __shared__ double sh[2][32];
  __shared__ int s_last;
  const UpdInst U = tab[blockIdx.y];
  if (static_cast<int>(blockIdx.x) >= U.nct) return;
  const StepScalars c = step_scalars(U);
  if (!c.test) return;
  const int j = blockIdx.x * kUpdChunk + threadIdx.x;
  double lg = 0.0, dot = 0.0;
  if (j < c.D) {
    double G, step, yj, ln;
    coord(U, c, j, G, step, yj, ln);
    lg = static_cast<double>(U.y[j]) * G;
    if (step > 0.0) dot = __ddiv_rn(__dmul_rn(ln - yj, ln - U.lam64[j]), step);
  }
  block_sum2(lg, dot, sh);
  if (arrive(U, 0, lg, dot, &s_last) && threadIdx.x == 0) {
    double L = 0.0, Dt = 0.0;
    for (int k = 0; k < U.nct; ++k) {
      L += __ldcg(U.part + 2 * k);
      Dt += __ldcg(U.part + 2 * k + 1);
    }
    U.part[2 * U.nct] = L;
    *U.flag = Dt < 0.0 ? 1 : 0;
  }
}

// Kernel B: the step on every coordinate; the last CTA writes the state and
// the trajectory.
__global__ void __launch_bounds__(kUpdChunk) fista_update_kernel(const UpdInst* __restrict__ tab) {
  __shared__ double sh[2][32];
  __shared__ int s_last;
  const UpdInst U = tab[blockIdx.y];
  if (static_cast<int>(blockIdx.x) >= U.nct) return;
  const StepScalars c = step_scalars(U);
  const bool restart = c.stage_restart || (c.test && *U.flag != 0);
  const int j = blockIdx.x * kUpdChunk + threadIdx.x;
  double lg = 0.0, bad = 0.0;
  if (j < c.D) {
    double G, step, yj, ln;
    coord(U, c, j, G, step, yj, ln);
    if (!c.test) lg = static_cast<double>(U.y[j]) * G;  // (with the test, kernel A summed it)
    const double yn = restart ? ln : __dadd_rn(ln, __dmul_rn(c.beta, ln - U.lam64[j]));
    U.lam64[j] = ln;
    U.y64[j] = yn;
    U.lam[j] = static_cast<float>(ln);
    U.y[j] = static_cast<float>(yn);
    if (j < c.NC) U.acc[j] = 0ull;
    if (!isfinite(G) || !isfinite(yj) || !isfinite(yn)) bad = 1.0;
  }
  block_sum2(lg, bad, sh);
  if (arrive(U, 1, lg, bad, &s_last) && threadIdx.x == 0) {
    double L = 0.0, B = 0.0;
    for (int k = 0; k < U.nct; ++k) {
      L += __ldcg(U.part + 2 * k);
      B += __ldcg(U.part + 2 * k + 1);
    }
    if (c.test) L = __ldcg(U.part + 2 * U.nct);
    const double g = to_real(*U.objq, U.inv_scaleO) + L;
    *U.objq = 0ull;
    if (U.count_on) *U.cnt_rw = 0ull;
    U.traj[c.st.iter % kTrajCap] = g;
    DevState n = c.st;
    n.iter = c.st.iter + 1;
    n.theta = restart ? 1.0 : c.th1;
    n.gamma = c.gamma1;
    n.stage = static_cast<int32_t>(c.s1 < 0x7fffffff ? c.s1 : 0x7fffffff);
    if (B > 0.0 || !isfinite(g)) n.status |= kStatNumeric;
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
  if (S.obj_in) {
    if (threadIdx.x == 0) obj = *S.obj_in;
  } else {
    for (int k = threadIdx.x; k < S.nseg; k += blockDim.x) obj += S.seg_obj[S.seg_list[k]];
  }
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

// The objective partials of instance 0's certificate-sweep segments, summed
// in a fixed order (a shard's share of the certificate objective).
__global__ void __launch_bounds__(kUpdThreads) seg_sum_kernel(const StatsInst* __restrict__ tab, double* out) {
  __shared__ double sh[32];
  const StatsInst S = tab[0];
  double obj = 0.0;
  for (int k = threadIdx.x; k < S.nseg; k += blockDim.x) obj += S.seg_obj[S.seg_list[k]];
  obj = block_sum(obj, sh);
  if (threadIdx.x == 0) *out = obj;
}

}  // namespace

cudaError_t launch_update(const UpdInst* dev_tab, int ninst, int max_cta, bool any_test, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>(max_cta > 0 ? max_cta : 1), static_cast<unsigned>(ninst));
  if (any_test) {
    restart_test_kernel<<<grid, kUpdChunk, 0, s>>>(dev_tab);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  fista_update_kernel<<<grid, kUpdChunk, 0, s>>>(dev_tab);
  return cudaGetLastError();
}

int update_ctas(int64_t D) { return static_cast<int>((D + kUpdChunk - 1) / kUpdChunk); }

cudaError_t launch_stats(const StatsInst* dev_tab, int ninst, cudaStream_t s) {
  stats_kernel<<<ninst, kUpdThreads, 0, s>>>(dev_tab);
  return cudaGetLastError();
}

cudaError_t launch_seg_sum(const StatsInst* dev_tab, double* out, cudaStream_t s) {
  seg_sum_kernel<<<1, kUpdThreads, 0, s>>>(dev_tab, out);
  return cudaGetLastError();
}

}  // namespace dlm
