// dlm_impl.cuh -- internal structures of the dual-sweep solver (not part of
// the C-ABI).  Shared by the sweep, update, layout and API translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dlm.h"

namespace dlm {

constexpr int kWarp = 32;
constexpr int kSweepThreads = 1024;  // 32 warps per sweep CTA, one CTA per SM
constexpr int kUpdThreads = 1024;    // one CTA per instance for the O(J) kernels
constexpr int64_t kMaxStageTable = int64_t(1) << 20;  // continuation stages a schedule may take to reach gamma_end
constexpr int kTrajCap = 4096;       // dual objective values kept per handle (ring, one per iteration)
constexpr int kMaxSegTasks = 16;     // tasks of one instance in one CTA
constexpr int kMaxFamilies = 4;      // capacity families per instance (Def. 1)
constexpr int kShortRowW = 32;       // widest rows the short-row sweep holds in registers (sweep_short.cu)

// Error bits of the device status word.
enum : int32_t { kStatNumeric = 1, kStatTimeout = 2 };

// Per-instance iteration state (device memory).
struct DevState {
  int64_t iter;   // next iteration index t
  double theta;   // momentum scalar
  double gamma;   // gamma of iteration t's stage
  int32_t stage;  // stage index of iteration t
  int32_t status; // error bits
};

// Per-instance constants of the update step (device memory).  The iterate
// (lam, y) is kept in FP64; the sweeps read FP32 copies of it.
struct UpdInst {
  DevState* state;
  const double* gamma_tab;  // [nstages]: gamma of stage s (the last entry is gamma_end)
  int64_t nstages;
  const double* b;          // [J]
  const double* curv;       // [D] per-coordinate curvature bound h (0 for an empty item); step = gamma / h
  double* lam64;            // [D] the iterate
  double* y64;              // [D] the momentum point
  float* lam;               // [D] FP32 copies read by the sweeps
  float* y;                 // [D]
  unsigned long long* acc;  // [J] fixed-point A x at y
  unsigned long long* objq; // fixed-point sum of (c x + gamma/2 x^2) at y (reset here)
  double* traj;             // [kTrajCap] g(y_t) at slot t mod kTrajCap
  double* part;             // [2 nct + 1] per-CTA partials of the update's sums
  unsigned* ticket;         // [2] CTAs of the instance done (reset by the last)
  int32_t* flag;            // the adaptive restart decision of the iteration
  int32_t nct;              // update CTAs of the instance (update_ctas(D))
  int64_t iters_per_stage;
  double curv_max;          // the largest curvature bound (plain step gamma / curv_max)
  double inv_scaleG;        // 2^-sG
  double inv_scaleO;        // 2^-sO
  int32_t J;
  int32_t precondition;
  int32_t adaptive_restart;
  // global count constraint sum x <= M (dual entry J)
  int32_t count_on;
  const unsigned long long* cnt;  // fixed-point sum of all x at y
  unsigned long long* cnt_rw;     // the same, reset here
  double inv_scaleN;
  double count_M;
  int32_t ncap;                   // capacity coordinates m J (the count dual is coordinate ncap)
};

// Per-instance view for the sweep kernels (device memory; one table for the
// iteration sweep at y, one for the certificate sweep at lam).  Edges are in
// slices of 32 users (see layout.cu): edge k of user t of slice s is at
// slice_off[s] + 32 k + t.
struct InstDesc {
  const int64_t* slice_off; // [nslices + 1]
  const int32_t* slice_w;   // [nslices] edges per lane (the slice's largest degree)
  const uint16_t* col16;    // [padded nnz] item index as uint16 (every handle: J < 65,536)
  const void* ca;           // [padded nnz] interleaved (c, a): float2, or bf16 pair in a uint32
  const int64_t* orig_off;  // [users with edges] caller row start of each sorted user
  const int32_t* udeg;      // [users with edges] degree of each sorted user
  const uint64_t* lead;     // [users with edges] caller positions of the row's lead edges (lead_caller_pos)
  int64_t nusers;           // users with edges (sorted users 0 .. nusers-1)
  int32_t* status;          // device error word (kStat* bits)
  const float* y;           // sweep point [J]
  const double* gamma;      // ridge used by this sweep
  unsigned long long* acc;  // [J] fixed-point sum a x
  unsigned long long* accC; // [J] fixed-point sum c x (stats)
  unsigned long long* accQ; // [J] fixed-point sum x^2 (stats)
  double* seg_obj;          // [tasks] FP64 objective partial per (CTA, instance) segment (stats)
  float* xout;              // caller-order x or nullptr (stats)
  unsigned long long* cnt;  // fixed-point sum of all x (global count constraint) or nullptr
  unsigned long long* objq; // iteration sweeps: fixed-point sum of (c x + gamma/2 x^2) over all users
  float scaleG, scaleC, scaleQ, scaleN, scaleO;
  float z;
  int32_t J;
  int32_t kind;
  int32_t count_on;         // 1: the dual vector has J + 1 entries, y[J] is the count dual mu
  // m capacity families (sweep_multi.cu): y, acc are [m J] family-major, and
  // family k >= 1's coefficients are a stream at a_ext + (k - 1) * ext_stride
  int32_t m;
  const void* a_ext;
  int64_t ext_stride;
};

// Lead order of a row in the slice layout (layout.cu): min(4, d) edges of
// the row's lowest costs c, in ascending order of c, come first (among edges
// of equal cost at the boundary, the one the layout's sorted insertion keeps);
// the others follow in caller order.  A row's largest values u = -(c + a y) then tend
// to come first, so the sweeps' first pass rarely has to insert later edges
// into its record of the largest values.  `lead` packs the lead edges' caller
// positions, 16 bits each (slot i at bits 16 i).  Returns the caller position
// (0 .. d - 1) of slice position k of a row of d edges.
__device__ __forceinline__ int lead_caller_pos(uint64_t lead, int k, int d) {
  const int nl = d < 4 ? d : 4;
  if (k < nl) return static_cast<int>((lead >> (16 * k)) & 0xFFFFu);
  int p[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) p[i] = i < nl ? static_cast<int>((lead >> (16 * i)) & 0xFFFFu) : 0x7FFFFFFF;
  // ascending (a four-input network)
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int i = q == 0 ? 0 : q == 1 ? 2 : q == 2 ? 0 : q == 3 ? 1 : 1;
    const int j = q == 0 ? 1 : q == 1 ? 3 : q == 2 ? 2 : q == 3 ? 3 : 2;
    const int lo = min(p[i], p[j]), hi = max(p[i], p[j]);
    p[i] = lo;
    p[j] = hi;
  }
  // the (k - nl)-th position outside the lead set: step past every lead
  // position at or below the candidate, in ascending order
  int c = k - nl;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (p[i] <= c) ++c;
  return c;
}

// A task: slices first, first + stride, ... (< end) of instance `inst`.  The
// tasks of one CTA are contiguous and grouped by instance.
struct Task {
  int32_t inst;
  int32_t stride;
  int64_t first;
  int64_t end;
};

struct SweepLaunch {
  const InstDesc* inst;     // device table
  const Task* tasks;        // device
  const int32_t* cta_task;  // device [grid + 1]
  int32_t grid;
  int32_t smemJ;            // item capacity of the shared arrays
  int32_t win;              // certificate sweeps: item window per launch (0: all smemJ items)
  int32_t threads;          // threads per sweep CTA (0: kSweepThreads)
  int32_t coop_max;         // warp-cooperative threshold path below this many users per warp
  cudaStream_t stream;
  // Dynamic distribution of iteration sweeps (null: the static tasks above).
  const Task* units;        // device [nunits] work units (stride 1), ordered by instance
  int32_t nunits;
  unsigned* ctr;            // device [2]: next unit, finished CTAs (zero between launches)
  bool count;               // some instance has a global count constraint (its own instantiation)
  int32_t fam;              // capacity families (> 1: the general sweep of sweep_multi.cu)
  int32_t topk = 4;         // one-family sweep: largest values tracked per row in the first pass (4 or 8)
  // Short-row sweep (iteration sweeps of a single one-family handle without a
  // count constraint, sweep_short.cu): slices 0 .. nslices0 - 1 of instance 0.
  bool short_rows = false;
  int64_t nslices0 = 0;
};
constexpr int kDefaultCoopMax = 12;

struct StatsInst {
  const double* b;
  const float* lam;           // dual point the certificate sweep used
  const double* gamma;
  unsigned long long *acc, *accC, *accQ;
  const double* seg_obj;
  const int32_t* seg_list;    // task indices that start a segment of this instance, ascending
  int32_t nseg;
  int32_t J;
  double inv_sG, inv_sC, inv_sQ;
  float* grad_out;            // optional [J] (+1 with the count constraint)
  double* out;                // [8]: g, P, rel_gap, uncert_gap, max_viol, obj, iter, status
  const DevState* state;
  int32_t certified;          // 0: scaled point not certified (EQ simplex or a < 0)
  int32_t count_on;
  unsigned long long* cnt;    // fixed-point sum of all x at lam (reset here)
  double inv_sN;
  double count_M;
  int32_t m;                  // capacity families: acc, b, lam, grad_out are [m J] family-major
  const double* obj_in;       // non-null: the objective sum (a shard's, added over the ranks) instead of seg_obj
};

// Sets the thread-local message returned by dlm_last_error (api.cu).
void set_last_error(const std::string& m);

// layout.cu: stream-ordered device memory from one pool per device that keeps
// freed memory for later handles (trimmed by release_cached_memory).
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);
cudaError_t release_cached_memory();

// ---- launchers (defined in the .cu files) ----
size_t sweep_smem_bytes(int smemJ, bool stats);
// Certificate sweep with item sums for a window of win items (0: none).
size_t sweep_stats_smem_bytes(int smemJ, int win);
// Widest item window whose certificate sweep fits (smemJ: no windows; 0: none fits).
int sweep_stats_window(int smemJ);
size_t sweep_smem_limit();             // usable dynamic shared memory per sweep CTA on this device
cudaError_t sweep_prepare(bool bf16);  // raises the dynamic shared-memory limit
cudaError_t launch_sweep(const SweepLaunch& L, bool stats, bool bf16);
// sweep_short.cu: the iteration sweep with rows of at most kShortRowW edges
// held in registers (L.short_rows).
cudaError_t sweep_short_prepare(bool bf16);
cudaError_t launch_sweep_short(const SweepLaunch& L, bool bf16);
// The update of ninst instances: a grid of max_cta x ninst CTAs (instance i
// uses its first update_ctas(D_i)); any_test: some instance has the adaptive
// restart on (a first kernel takes the test).
cudaError_t launch_update(const UpdInst* dev_tab, int ninst, int max_cta, bool any_test, cudaStream_t s);
int update_ctas(int64_t D);
cudaError_t launch_stats(const StatsInst* dev_tab, int ninst, cudaStream_t s);
// The certificate sweep's objective partials of instance 0 summed into *out.
cudaError_t launch_seg_sum(const StatsInst* dev_tab, double* out, cudaStream_t s);
// sweep_multi.cu (m > 1 families; static tasks only)
size_t sweep_multi_smem_bytes(int smemJ, int m, bool stats);
cudaError_t sweep_multi_prepare(bool bf16);
cudaError_t launch_sweep_multi(const SweepLaunch& L, bool stats, bool bf16);

// warmstart.cu: per-item features from the laid-out edges (scratch: J each).
cudaError_t launch_item_features(const uint16_t* col, const void* ca, bool bf, int64_t padded, int J, double scale,
                                 const double* b, const float* lam_prev, double gamma, const float* grad, float* X,
                                 unsigned* deg, int* mx, unsigned long long* sum, cudaStream_t s);

// layout.cu
struct LayoutOut {
  double phase_s[3] = {0, 0, 0};  // wall seconds: validation, degree sort, slice layout + item sums
  int64_t* slice_off = nullptr;  // [nslices + 1]
  int32_t* slice_w = nullptr;    // [nslices]
  uint16_t* col16 = nullptr;     // [padded_nnz + 64] item index (uint16: J <= 65,536)
  void* ca = nullptr;            // [padded_nnz + 32]
  int64_t* orig_off = nullptr;   // [num_active_users + 32]
  int32_t* udeg = nullptr;       // [num_active_users + 32]
  uint64_t* lead = nullptr;      // [num_active_users + 32] lead edges of each sorted row (lead_caller_pos)
  int64_t num_active_users = 0, nslices = 0, padded_nnz = 0;
  double* n2 = nullptr;          // [J] sum_i a_ij^2
  double n2max = 0;
  std::vector<double> h_n2, h_s1;  // host copies: sum_i a_ij^2, sum_i a_ij
  int64_t max_item_deg = 0;
  double max_abs_a = 0, max_abs_c = 0;
  bool a_nonneg = true;
};
// families.cu: set-up of instances with m > 1 capacity families.
struct LayoutOut;
cudaError_t families_split(const void* a, int64_t nnz, int m, bool bf16, void* out, int64_t stride, cudaStream_t s);
cudaError_t families_check(const void* a, int64_t n, bool bf16, int* flags, unsigned* max_abs, cudaStream_t s);
cudaError_t families_gather(const LayoutOut& lay, const void* src, bool bf16, void* dst, cudaStream_t s);
cudaError_t families_gram(const int32_t* col, const void* af, const void* al, int64_t nnz, bool bf16, float scale,
                          unsigned long long* acc, cudaStream_t s);

// Statistics of an instance's rows (one shard's, or all of them).
struct RowStats {
  int64_t nnz = 0, active_users = 0, max_item_deg = 0;
  double max_abs_a = 0, max_abs_c = 0;
  bool a_nonneg = true;
  std::vector<unsigned long long> item_deg;  // [J]
};
// The statistics of all shards of a user-sharded instance, and its exact
// fixed-point item sums (sum_i a_ij^2 and sum_i a_ij at the exponents
// item_sum_shifts gives for max_item_deg and max_abs_a), host memory.
struct ShardGlobal {
  int64_t nnz, active_users, max_item_deg;
  double max_abs_a, max_abs_c;
  bool a_nonneg;
  const int64_t* item_sq;
  const int64_t* item_sum;
};
void item_sum_shifts(int64_t max_item_deg, double max_abs_a, int* ssq, int* ss1);

// Validates and lays out one instance; all pointers are device pointers.
// With `measure`, validates and fills the row statistics only (no layout);
// with `shard`, the instance is one shard of a larger one and the item sums
// and bounds are the global ones given.  Returns DLM_OK or an error with
// `msg` set.
dlm_status build_layout(int64_t I, int64_t J, int64_t nnz, const int64_t* rp, const int32_t* col, const void* c,
                        const void* a, const double* b, bool bf16, cudaStream_t s, LayoutOut* out, std::string* msg,
                        RowStats* measure = nullptr, const ShardGlobal* shard = nullptr);
// Fixed-point sums over the given rows: sum_i a_ij^2 at 2^ssq and sum_i a_ij
// at 2^ss1 into the host arrays sq, s1 [J].
dlm_status item_sums(int64_t J, int64_t nnz, const int32_t* col, const void* a, bool bf16, int ssq, int ss1,
                     cudaStream_t s, int64_t* sq, int64_t* s1, std::string* msg);

}  // namespace dlm
