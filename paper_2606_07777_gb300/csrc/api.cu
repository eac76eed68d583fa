// api.cu -- the C-ABI (include/dlm.h): handle life cycle, schedule and
// options, the runner that sweeps one instance or a batch (device tables,
// slice-to-CTA tasks, CUDA-graph replay, timed stepping), certified-gap checks,
// the solve loop, and the mapping tuner.  All device work of a handle or a
// batch runs on its stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "boxcut.cuh"
#include "dlm_impl.cuh"

namespace dlm {
int fixed_point_shift(double bound);
}

namespace {
thread_local std::string g_err;
}

void dlm::set_last_error(const std::string& m) { g_err = m; }

using namespace dlm;

namespace {

dlm_status fail(dlm_status s, const std::string& m) {
  g_err = m;
  return s;
}

#define CK(x)                                                                                          \
  do {                                                                                                 \
    cudaError_t e_ = (x);                                                                              \
    if (e_ != cudaSuccess) return fail(DLM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

__global__ void k_set_double(double* p, double v) { *p = v; }

// lam <- max(src, 0), y <- lam, theta <- 1 (warm start); the FP64 iterate
// and its FP32 copies.
__global__ void k_warm(const float* src, double* lam64, double* y64, float* lam, float* y, int64_t J,
                       DevState* st) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < J;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float v = fmaxf(src[j], 0.f);
    lam64[j] = v;
    y64[j] = v;
    lam[j] = v;
    y[j] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->theta = 1.0;
}

// y <- lam (the momentum restart of a new schedule), theta <- 1; FP32 copies.
__global__ void k_momentum_reset(const double* lam64, double* y64, float* lam, float* y, int64_t n, DevState* st) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double v = lam64[j];
    y64[j] = v;
    lam[j] = static_cast<float>(v);
    y[j] = static_cast<float>(v);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->theta = 1.0;
}

// FP32 copies of the FP64 iterate (after a restore).
__global__ void k_shadow(const double* lam64, const double* y64, float* lam, float* y, int64_t n) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    lam[j] = static_cast<float>(lam64[j]);
    y[j] = static_cast<float>(y64[j]);
  }
}

__global__ void k_state_reset(DevState* st, double gamma0) {
  DevState n;
  n.iter = 0;
  n.theta = 1.0;
  n.gamma = gamma0;
  n.stage = 0;
  n.status = 0;
  *st = n;
}

int blocks_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return static_cast<int>(g);
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n > 0 ? n : 1));
}

// Slice-to-CTA assignment orders.
enum : int { kAssignInterleaved = 0, kAssignContiguous = 1, kAssignDynamic = 2 };

// The launch state of a set of instances swept together: one instance for a
// handle, several for a batch.  Instance data (layout, duals, accumulators,
// state) stay in the dlm_problem objects; the runner owns the device tables
// that point at them, the slice-to-CTA tasks and the captured graph.
struct Runner {
  std::vector<dlm_problem*> probs;
  cudaStream_t stream = nullptr;
  bool bf16 = false;
  int device = 0;
  int sms = 0;
  int grid = 0;
  int threads = kSweepThreads;
  int coop_max = kDefaultCoopMax;
  int assign = kAssignInterleaved;
  int smemJ = 0;
  int win = 0;  // item window of certificate sweeps (smemJ when their arrays fit at once)
  int graph_iters = 10;
  int topk = 4;  // one-family sweeps: values tracked per row in the first pass
  bool short_rows = false;   // iteration sweeps take the short-row sweep (sweep_short.cu)
  int upd_ctas = 1;      // update grid width (the largest member's)
  bool upd_test = false; // some member has the adaptive restart (a test kernel runs first)
  InstDesc *inst_iter = nullptr, *inst_stats = nullptr;
  double* cuts = nullptr;  // per-instance DLM_BOX_CUT budgets (box-cut runners only)
  UpdInst* upd = nullptr;
  StatsInst* st_stats = nullptr;
  Task* tasks = nullptr;
  int32_t *cta_task = nullptr, *seg_lists = nullptr;
  double* seg_obj = nullptr;
  std::vector<Task> h_tasks;
  std::vector<int32_t> h_cta;
  std::vector<std::vector<int32_t>> h_seg;
  std::vector<int32_t> seg_off;
  Task* units = nullptr;      // dynamic assignment: work units of the iteration sweeps
  unsigned* ctr = nullptr;    // their counters [2]
  std::vector<Task> h_units;
  cudaGraphExec_t gexec = nullptr;
  int gexec_iters = 0;
  std::vector<cudaEvent_t> events;
  cudaEvent_t done = nullptr;  // batches: end of the last enqueued batch work
};

}  // namespace

struct dlm_problem {
  int64_t I = 0, J = 0, nnz = 0;
  bool bf16 = false;
  int kind = DLM_SIMPLEX_LE;
  double z = 1.0;
  double cut = 0.0;  // DLM_BOX_CUT budget
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev = nullptr;  // orders the handle's stream before batch work
  int device = 0;
  LayoutOut lay;
  std::vector<int64_t> h_slice_off;  // host copy of the slice offsets (task balancing)
  int sG = 0, sC = 0, sQ = 0;
  bool certified = true;

  double *b = nullptr, *curv = nullptr;  // curv: per-coordinate curvature bounds h (steps gamma / h)
  double curv_max = 0;                    // the largest bound (plain step gamma / curv_max)
  // global count constraint sum x <= M: dual entry J of lam and y
  bool count_on = false;
  double count_M = INFINITY;
  int sN = 0;
  unsigned long long *cnt = nullptr, *cnt2 = nullptr;  // fixed-point sum x at y / at lam
  // m capacity families (Def. 1): duals and item sums are [m J] family-major;
  // family k >= 1's coefficients are a stream in slice order at a_ext
  int m = 1;
  void* a_ext = nullptr;
  int64_t ext_stride = 0;
  std::vector<double> h_gram;  // [m m J]: sum_i a_kij a_lij
  int64_t MJ() const { return static_cast<int64_t>(m) * J; }
  int64_t D() const { return MJ() + (count_on ? 1 : 0); }  // dual dimension
  // Partial sums: xsum = [A x (m J) | count | objective] of the iteration
  // sweep, csum = [A x (m J) | C x (J) | Q x (J) | count] of the certificate
  // sweep (the views below point into them).  A shard of a user-sharded
  // instance uses the caller's buffers, which the ranks add up in place.
  unsigned long long *xsum = nullptr, *csum = nullptr;
  double* cobj = nullptr;    // shard: the certificate's objective partial
  bool own_sums = true;
  bool sharded = false;
  int64_t glob_nnz = 0, glob_users = 0;  // the whole instance's edges and users with edges
  double *lam64 = nullptr, *y64 = nullptr;  // the iterate (FP64)
  float *lam = nullptr, *y = nullptr;       // its FP32 copies, read by the sweeps
  unsigned long long *acc = nullptr, *acc2 = nullptr, *accC = nullptr, *accQ = nullptr;
  unsigned long long* objq = nullptr;       // fixed-point objective sum of the iteration sweep
  int sO = 0;                               // its exponent
  double* traj = nullptr;                   // [kTrajCap] g(y_t) per iteration (ring)
  double* upd_part = nullptr;               // update partials [2 update_ctas(m J + 1) + 1]
  unsigned* upd_ticket = nullptr;           // [2]
  int32_t* upd_flag = nullptr;
  int64_t traj_from = 0;                    // first iteration whose trajectory entry is valid
  double *gamma_tab = nullptr, *calc_gamma = nullptr, *stats_out = nullptr;
  int64_t nstages = 1, gamma_tab_cap = 0;
  DevState* state = nullptr;
  InstDesc* inst_calc = nullptr;
  StatsInst* st_calc = nullptr;

  // pinned host staging
  double* h_out = nullptr;  // 8 doubles
  InstDesc* h_inst = nullptr;
  StatsInst* h_stinst = nullptr;

  double gamma0 = 1e-2, gamma_end = 1e-2, factor = 0.5;
  int64_t ips = 1 << 30;
  dlm_options opt{};
  std::vector<double> h_gamma_tab;
  double last_solve_seconds = 0;
  double setup_s[6] = {0, 0, 0, 0, 0, 0};  // see dlm_get_setup_seconds

  Runner run;
};

struct dlm_batch {
  Runner run;
  dlm_options opt{};  // mapping and loop options of the batch
  bool own_stream = false;
  double last_solve_seconds = 0;
};

namespace {

InstDesc base_desc(const dlm_problem* p) {
  InstDesc d{};
  d.slice_off = p->lay.slice_off;
  d.slice_w = p->lay.slice_w;
  d.col16 = p->lay.col16;
  d.ca = p->lay.ca;
  d.orig_off = p->lay.orig_off;
  d.udeg = p->lay.udeg;
  d.lead = p->lay.lead;
  d.nusers = p->lay.num_active_users;
  d.status = &p->state->status;
  d.scaleG = std::ldexp(1.0f, p->sG);
  d.scaleC = std::ldexp(1.0f, p->sC);
  d.scaleQ = std::ldexp(1.0f, p->sQ);
  d.z = static_cast<float>(p->z);
  d.J = static_cast<int32_t>(p->J);
  d.kind = p->kind;
  d.count_on = p->count_on ? 1 : 0;
  d.cnt = p->cnt2;
  d.scaleN = std::ldexp(1.0f, p->sN);
  d.m = p->m;
  d.a_ext = p->a_ext;
  d.ext_stride = p->ext_stride;
  return d;
}

StatsInst base_stats(const dlm_problem* p, const Runner& R, int i) {
  StatsInst s{};
  s.b = p->b;
  s.acc = p->acc2;
  s.accC = p->accC;
  s.accQ = p->accQ;
  s.seg_obj = R.seg_obj;
  s.seg_list = R.seg_lists + (R.seg_off.empty() ? 0 : R.seg_off[i]);
  s.nseg = R.h_seg.empty() ? 0 : static_cast<int32_t>(R.h_seg[i].size());
  s.J = static_cast<int32_t>(p->J);
  s.inv_sG = std::ldexp(1.0, -p->sG);
  s.inv_sC = std::ldexp(1.0, -p->sC);
  s.inv_sQ = std::ldexp(1.0, -p->sQ);
  s.out = p->stats_out;
  s.certified = p->certified ? 1 : 0;
  s.count_on = p->count_on ? 1 : 0;
  s.cnt = p->cnt2;
  s.inv_sN = std::ldexp(1.0, -p->sN);
  s.count_M = p->count_M;
  s.m = p->m;
  s.obj_in = nullptr;
  return s;
}

void invalidate_graph(Runner& R) {
  if (R.gexec) cudaGraphExecDestroy(R.gexec);
  R.gexec = nullptr;
  R.gexec_iters = 0;
}

void runner_free(Runner& R) {
  invalidate_graph(R);
  void* ptrs[] = {R.inst_iter, R.inst_stats, R.upd,   R.st_stats, R.tasks, R.cta_task,
                  R.seg_lists, R.seg_obj,    R.units, R.ctr,      R.cuts};
  for (void* q : ptrs) cudaFree(q);
  for (cudaEvent_t e : R.events) cudaEventDestroy(e);
  R.events.clear();
  if (R.done) cudaEventDestroy(R.done);
  R.done = nullptr;
  R.inst_iter = R.inst_stats = nullptr;
  R.cuts = nullptr;
  R.upd = nullptr;
  R.st_stats = nullptr;
  R.tasks = nullptr;
  R.cta_task = R.seg_lists = nullptr;
  R.seg_obj = nullptr;
  R.units = nullptr;
  R.ctr = nullptr;
}

// Slice-to-CTA tasks.  Interleaved: CTA k sweeps slices k, k + V, ... of
// every instance; slices are sorted by width, so every CTA gets the same mix.
// Contiguous: the slices of all instances, in order, are cut into V ranges of
// equal weight (edges plus a per-slice cost), so a CTA touches few instances.
void build_task_list(Runner& R) {
  const int V = R.grid;
  const int n = static_cast<int>(R.probs.size());
  R.h_tasks.clear();
  R.h_cta.assign(V + 1, 0);
  // certificate sweeps of a dynamic mapping use a static order
  const int assign =
      R.assign != kAssignDynamic ? R.assign : (n > 1 ? kAssignContiguous : kAssignInterleaved);
  if (assign == kAssignInterleaved) {
    for (int k = 0; k < V; ++k) {
      R.h_cta[k] = static_cast<int32_t>(R.h_tasks.size());
      for (int i = 0; i < n; ++i) {
        const int64_t ns = R.probs[i]->lay.nslices;
        if (k < ns) {
          Task t;
          t.inst = i;
          t.stride = V;
          t.first = k;
          t.end = ns;
          R.h_tasks.push_back(t);
        }
      }
    }
  } else {
    constexpr int64_t kSliceCost = 128;  // fixed work of a slice, in edge units
    std::vector<int64_t> base(n + 1, 0);
    auto weight = [&](int i, int64_t s) { return R.probs[i]->h_slice_off[s] + kSliceCost * s; };
    for (int i = 0; i < n; ++i) base[i + 1] = base[i] + weight(i, R.probs[i]->lay.nslices);
    const int64_t W = base[n];
    for (int k = 0; k < V; ++k) {
      R.h_cta[k] = static_cast<int32_t>(R.h_tasks.size());
      const int64_t lo = W * k / V, hi = W * (k + 1) / V;
      for (int i = 0; i < n; ++i) {
        const int64_t ns = R.probs[i]->lay.nslices;
        if (ns == 0 || base[i + 1] <= lo || base[i] >= hi) continue;
        // first slice whose start is at or after x
        auto first_at = [&](int64_t x) {
          int64_t a = 0, b = ns;
          while (a < b) {
            const int64_t m = (a + b) / 2;
            if (base[i] + weight(i, m) < x)
              a = m + 1;
            else
              b = m;
          }
          return a;
        };
        const int64_t f = first_at(lo), e = first_at(hi);
        if (e > f) {
          Task t;
          t.inst = i;
          t.stride = 1;
          t.first = f;
          t.end = e;
          R.h_tasks.push_back(t);
        }
      }
    }
  }
  R.h_cta[V] = static_cast<int32_t>(R.h_tasks.size());
  R.h_units.clear();
  if (R.assign == kAssignDynamic) {
    // Work units in instance order, each about max(Wmin, R / (2 V)) of the
    // remaining weight R (guided self-scheduling: large units first, small
    // ones last, so the CTAs run out of work together).
    constexpr int64_t kSliceCost = 128;
    std::vector<int64_t> tot(n, 0);
    int64_t W = 0;
    for (int i = 0; i < n; ++i) {
      const int64_t ns = R.probs[i]->lay.nslices;
      tot[i] = R.probs[i]->h_slice_off[ns] + kSliceCost * ns;
      W += tot[i];
    }
    const int64_t wmin = std::max<int64_t>(8192, W / (64 * static_cast<int64_t>(V)));
    int64_t rem = W;
    for (int i = 0; i < n; ++i) {
      const int64_t ns = R.probs[i]->lay.nslices;
      const std::vector<int64_t>& so = R.probs[i]->h_slice_off;
      auto weight = [&](int64_t s) { return so[s] + kSliceCost * s; };
      int64_t s = 0;
      while (s < ns) {
        const int64_t size = std::max(wmin, rem / (2 * static_cast<int64_t>(V)));
        // first slice e > s with weight(e) - weight(s) >= size (or ns)
        int64_t a = s + 1, b = ns;
        while (a < b) {
          const int64_t m = (a + b) / 2;
          if (weight(m) - weight(s) < size)
            a = m + 1;
          else
            b = m;
        }
        Task t;
        t.inst = i;
        t.stride = 1;
        t.first = s;
        t.end = a;
        R.h_units.push_back(t);
        rem -= weight(a) - weight(s);
        s = a;
      }
    }
  }
  R.h_seg.assign(n, {});
  for (size_t t = 0; t < R.h_tasks.size(); ++t) R.h_seg[R.h_tasks[t].inst].push_back(static_cast<int32_t>(t));
  R.seg_off.assign(n, 0);
  for (int i = 1; i < n; ++i) R.seg_off[i] = R.seg_off[i - 1] + static_cast<int32_t>(R.h_seg[i - 1].size());
}

// Device tables of the runner from the members' current state and options.
dlm_status write_tables(Runner& R) {
  const int n = static_cast<int>(R.probs.size());
  std::vector<InstDesc> it(n), ss(n);
  std::vector<UpdInst> up(n);
  std::vector<StatsInst> st(n);
  for (int i = 0; i < n; ++i) {
    const dlm_problem* p = R.probs[i];
    it[i] = base_desc(p);
    it[i].y = p->y;
    it[i].gamma = &p->state->gamma;
    it[i].acc = p->acc;
    it[i].accC = p->accC;
    it[i].accQ = p->accQ;
    it[i].seg_obj = R.seg_obj;
    it[i].xout = nullptr;
    it[i].cnt = p->cnt;
    it[i].objq = p->objq;
    it[i].scaleO = std::ldexp(1.0f, p->sO);
    ss[i] = base_desc(p);
    ss[i].y = p->lam;
    ss[i].gamma = &p->state->gamma;
    ss[i].acc = p->acc2;
    ss[i].accC = p->accC;
    ss[i].accQ = p->accQ;
    ss[i].seg_obj = R.seg_obj;
    ss[i].xout = nullptr;
    UpdInst u{};
    u.state = p->state;
    u.gamma_tab = p->gamma_tab;
    u.nstages = p->nstages;
    u.b = p->b;
    u.curv = p->curv;
    u.lam64 = p->lam64;
    u.y64 = p->y64;
    u.lam = p->lam;
    u.y = p->y;
    u.acc = p->acc;
    u.objq = p->objq;
    u.traj = p->traj;
    u.part = p->upd_part;
    u.ticket = p->upd_ticket;
    u.flag = p->upd_flag;
    u.nct = update_ctas(p->D());
    u.iters_per_stage = p->ips;
    u.curv_max = p->curv_max;
    u.inv_scaleG = std::ldexp(1.0, -p->sG);
    u.inv_scaleO = std::ldexp(1.0, -p->sO);
    u.J = static_cast<int32_t>(p->J);
    u.precondition = p->opt.precondition ? 1 : 0;
    u.adaptive_restart = p->opt.restart ? 1 : 0;
    u.count_on = p->count_on ? 1 : 0;
    u.cnt = p->cnt;
    u.cnt_rw = p->cnt;
    u.inv_scaleN = std::ldexp(1.0, -p->sN);
    u.count_M = p->count_M;
    u.ncap = static_cast<int32_t>(p->MJ());
    up[i] = u;
    st[i] = base_stats(p, R, i);
    st[i].obj_in = p->sharded ? p->cobj : nullptr;
    st[i].lam = p->lam;
    st[i].gamma = &p->state->gamma;
    st[i].grad_out = nullptr;
    st[i].state = p->state;
  }
  CK(cudaMemcpy(R.inst_iter, it.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(R.inst_stats, ss.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(R.upd, up.data(), sizeof(UpdInst) * n, cudaMemcpyHostToDevice));
  R.upd_ctas = 1;
  R.upd_test = false;
  for (const UpdInst& u : up) {
    R.upd_ctas = std::max(R.upd_ctas, u.nct);
    R.upd_test = R.upd_test || u.adaptive_restart;
  }
  CK(cudaMemcpy(R.st_stats, st.data(), sizeof(StatsInst) * n, cudaMemcpyHostToDevice));
  return DLM_OK;
}

// (Re)builds tasks and tables for the runner's current grid/assignment.
dlm_status runner_build(Runner& R) {
  CK(cudaStreamSynchronize(R.stream));
  invalidate_graph(R);
  const int n = static_cast<int>(R.probs.size());
  if (!R.inst_iter) {
    CK(dalloc(&R.inst_iter, n));
    CK(dalloc(&R.inst_stats, n));
    CK(dalloc(&R.upd, n));
    CK(dalloc(&R.st_stats, n));
  }
  if (R.probs[0]->kind == DLM_BOX_CUT && !R.cuts) {
    std::vector<double> h(n);
    for (int i = 0; i < n; ++i) h[i] = R.probs[i]->cut;
    CK(dalloc(&R.cuts, n));
    CK(cudaMemcpy(R.cuts, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  }
  build_task_list(R);
  cudaFree(R.tasks);
  cudaFree(R.cta_task);
  cudaFree(R.seg_lists);
  cudaFree(R.seg_obj);
  R.tasks = nullptr;
  R.cta_task = R.seg_lists = nullptr;
  R.seg_obj = nullptr;
  CK(dalloc(&R.tasks, R.h_tasks.size()));
  CK(dalloc(&R.cta_task, R.h_cta.size()));
  CK(dalloc(&R.seg_lists, R.h_tasks.size()));
  CK(dalloc(&R.seg_obj, R.h_tasks.size()));
  if (!R.h_tasks.empty())
    CK(cudaMemcpy(R.tasks, R.h_tasks.data(), sizeof(Task) * R.h_tasks.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(R.cta_task, R.h_cta.data(), sizeof(int32_t) * R.h_cta.size(), cudaMemcpyHostToDevice));
  std::vector<int32_t> flat;
  for (const auto& v : R.h_seg) flat.insert(flat.end(), v.begin(), v.end());
  if (!flat.empty()) CK(cudaMemcpy(R.seg_lists, flat.data(), sizeof(int32_t) * flat.size(), cudaMemcpyHostToDevice));
  cudaFree(R.units);
  R.units = nullptr;
  if (!R.h_units.empty()) {
    CK(dalloc(&R.units, R.h_units.size()));
    CK(cudaMemcpy(R.units, R.h_units.data(), sizeof(Task) * R.h_units.size(), cudaMemcpyHostToDevice));
  }
  if (!R.ctr) CK(dalloc(&R.ctr, 2));
  CK(cudaMemset(R.ctr, 0, 2 * sizeof(unsigned)));
  return write_tables(R);
}

// Whether the runner's iteration sweeps can take the short-row sweep: a
// single one-family handle, not box-cut (a count constraint, set later, is
// checked at launch).
bool short_capable(const Runner& R) {
  if (R.probs.size() != 1) return false;
  const dlm_problem* p = R.probs[0];
  return p->m == 1 && p->kind != DLM_BOX_CUT;
}

// Whether some slice's rows have at most kShortRowW edges (slices are sorted
// by width, widest first: the last one is the narrowest).
bool has_short_slices(const Runner& R) {
  const dlm_problem* p = R.probs[0];
  const int64_t ns = p->lay.nslices;
  return ns > 0 && p->h_slice_off[ns] - p->h_slice_off[ns - 1] <= 32 * static_cast<int64_t>(kShortRowW);
}

SweepLaunch launch_of(const Runner& R, const InstDesc* tab) {
  SweepLaunch L;
  L.inst = tab;
  L.tasks = R.tasks;
  L.cta_task = R.cta_task;
  L.grid = R.grid;
  L.smemJ = R.smemJ;
  L.win = R.win;
  L.threads = R.threads;
  L.coop_max = R.coop_max;
  L.stream = R.stream;
  L.count = false;
  L.fam = 1;
  for (const dlm_problem* p : R.probs) {
    L.count = L.count || p->count_on;
    L.fam = std::max(L.fam, p->m);
  }
  L.units = R.h_units.empty() ? nullptr : R.units;
  L.nunits = static_cast<int32_t>(R.h_units.size());
  L.ctr = R.ctr;
  L.topk = R.topk;
  if (R.short_rows && short_capable(R) && !L.count) {
    L.short_rows = true;
    L.nslices0 = R.probs[0]->lay.nslices;
  }
  return L;
}

// One-family instances take the sweep of sweep.cu, several families the
// general sweep of sweep_multi.cu (static tasks only).
cudaError_t dispatch_sweep(const SweepLaunch& L, bool stats, bool bf16) {
  return L.fam > 1 ? launch_sweep_multi(L, stats, bf16) : launch_sweep(L, stats, bf16);
}

// Handles on the box cut by a budget sweep with their own kernel (a runner's
// members are all box-cut or none).
cudaError_t dispatch_sweep(const Runner& R, const SweepLaunch& L, bool stats, bool bf16) {
  if (R.probs[0]->kind == DLM_BOX_CUT) return launch_sweep_boxcut(L, stats, bf16, R.cuts);
  return dispatch_sweep(L, stats, bf16);
}

dlm_status enqueue_iteration(Runner& R) {
  CK(dispatch_sweep(R, launch_of(R, R.inst_iter), false, R.bf16));
  CK(launch_update(R.upd, static_cast<int>(R.probs.size()), R.upd_ctas, R.upd_test, R.stream));
  return DLM_OK;
}

dlm_status enqueue_certificate(Runner& R, const InstDesc* inst_tab, const StatsInst* st_tab) {
  CK(dispatch_sweep(R, launch_of(R, inst_tab), true, R.bf16));
  CK(launch_stats(st_tab, static_cast<int>(R.probs.size()), R.stream));
  return DLM_OK;
}

dlm_status capture_graph(Runner& R, int iters) {
  invalidate_graph(R);
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(R.stream, cudaStreamCaptureModeThreadLocal));
  dlm_status st = DLM_OK;
  for (int i = 0; i < iters && st == DLM_OK; ++i) st = enqueue_iteration(R);
  cudaError_t e = cudaStreamEndCapture(R.stream, &g);
  if (st != DLM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(DLM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&R.gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(DLM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  R.gexec_iters = iters;
  return DLM_OK;
}

dlm_status runner_step(Runner& R, int64_t n_iters) {
  const int gi = R.graph_iters > 0 ? R.graph_iters : 10;
  if (n_iters >= gi && (!R.gexec || R.gexec_iters != gi)) {
    dlm_status st = capture_graph(R, gi);
    if (st != DLM_OK) return st;
  }
  int64_t done = 0;
  for (; done + gi <= n_iters; done += gi) CK(cudaGraphLaunch(R.gexec, R.stream));
  for (; done < n_iters; ++done) {
    dlm_status st = enqueue_iteration(R);
    if (st != DLM_OK) return st;
  }
  return DLM_OK;
}

dlm_status runner_step_timed(Runner& R, int64_t n_iters, double* sweep_ms, double* update_ms, double* total_ms) {
  const size_t need = static_cast<size_t>(2 * n_iters + 1);
  while (R.events.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    R.events.push_back(e);
  }
  const SweepLaunch L = launch_of(R, R.inst_iter);
  const int n = static_cast<int>(R.probs.size());
  CK(cudaEventRecord(R.events[0], R.stream));
  for (int64_t i = 0; i < n_iters; ++i) {
    CK(dispatch_sweep(R, L, false, R.bf16));
    CK(cudaEventRecord(R.events[2 * i + 1], R.stream));
    CK(launch_update(R.upd, n, R.upd_ctas, R.upd_test, R.stream));
    CK(cudaEventRecord(R.events[2 * i + 2], R.stream));
  }
  CK(cudaStreamSynchronize(R.stream));
  double ss = 0, su = 0;
  for (int64_t i = 0; i < n_iters; ++i) {
    float a = 0, b = 0;
    CK(cudaEventElapsedTime(&a, R.events[2 * i], R.events[2 * i + 1]));
    CK(cudaEventElapsedTime(&b, R.events[2 * i + 1], R.events[2 * i + 2]));
    ss += a;
    su += b;
  }
  float tot = 0;
  if (n_iters > 0) CK(cudaEventElapsedTime(&tot, R.events[0], R.events[2 * n_iters]));
  if (sweep_ms) *sweep_ms = ss;
  if (update_ms) *update_ms = su;
  if (total_ms) *total_ms = tot;
  return DLM_OK;
}

// Applies mapping options to a runner: grid, threads, cooperative threshold,
// assignment.  Rebuilds the tasks when the launch shape changes.
dlm_status runner_configure(Runner& R, const dlm_options& o, bool force) {
  const int threads = o.block_threads > 0 ? o.block_threads : kSweepThreads;
  const int per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : (threads <= 512 ? 2 : 1);
  const int grid = R.sms * per_sm;
  const int assign = o.mapping == 1   ? kAssignInterleaved
                     : o.mapping == 2 ? kAssignContiguous
                     : o.mapping == 3 ? kAssignDynamic
                                      : (R.probs.size() > 1 ? kAssignDynamic : kAssignInterleaved);
  int assign2 = assign;
  for (const dlm_problem* p : R.probs)
    if ((p->m > 1 || p->kind == DLM_BOX_CUT) && assign2 == kAssignDynamic)
      assign2 = R.probs.size() > 1 ? kAssignContiguous : kAssignInterleaved;
  R.coop_max = o.coop_max > 0 ? o.coop_max : kDefaultCoopMax;
  R.graph_iters = o.graph_iters > 0 ? o.graph_iters : 10;
  const int topk = o.topk == 8 ? 8 : 4;
  if (topk != R.topk) invalidate_graph(R);
  R.topk = topk;
  if ((o.short_rows != 0) != R.short_rows) invalidate_graph(R);
  R.short_rows = o.short_rows != 0;
  if (force || grid != R.grid || threads != R.threads || assign2 != R.assign) {
    R.grid = grid;
    R.threads = threads;
    R.assign = assign2;
    return runner_build(R);
  }
  invalidate_graph(R);
  return write_tables(R);
}

dlm_status read_stats(dlm_problem* p, dlm_stats* out) {
  CK(cudaMemcpyAsync(p->h_out, p->stats_out, sizeof(double) * 8, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  DevState hs;
  CK(cudaMemcpy(&hs, p->state, sizeof(DevState), cudaMemcpyDeviceToHost));
  if (out) {
    out->iter = hs.iter;
    out->gamma = hs.gamma;
    out->dual_obj = p->h_out[0];
    out->primal_obj = p->h_out[1];
    out->rel_gap = p->h_out[2];
    out->uncert_gap = p->h_out[3];
    out->max_viol = p->h_out[4];
    out->seconds = p->last_solve_seconds;
    out->status =
        (hs.status & kStatNumeric) ? DLM_ERR_NUMERIC : (hs.status & kStatTimeout) ? DLM_ERR_TIMEOUT : DLM_OK;
    out->converged = 0;
  }
  return DLM_OK;
}

void free_problem(dlm_problem* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  runner_free(p->run);
  cudaStream_t s = p->stream;
  void* pooled[] = {p->lay.slice_off, p->lay.slice_w, p->lay.col16, p->lay.ca, p->lay.orig_off,
                    p->lay.udeg,      p->lay.lead,    p->lay.n2,  p->a_ext};
  for (void* q : pooled) dev_free(q, s);
  if (s) cudaStreamSynchronize(s);
  if (p->own_sums) {
    cudaFree(p->xsum);
    cudaFree(p->csum);
  }
  void* ptrs[] = {p->b,         p->curv,      p->lam,      p->y,      p->gamma_tab, p->calc_gamma, p->stats_out,
                  p->state,     p->inst_calc, p->st_calc,  p->lam64,  p->y64,       p->traj,       p->upd_part,
                  p->upd_ticket, p->upd_flag};
  for (void* q : ptrs) cudaFree(q);
  cudaFreeHost(p->h_out);
  cudaFreeHost(p->h_inst);
  cudaFreeHost(p->h_stinst);
  if (p->ev) cudaEventDestroy(p->ev);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

// Per-coordinate curvature bounds and the steps built from them.  One
// capacity family: A A^T = diag(n), n_j = sum_i a_ij^2 (Def. 1), so the step
// of item j is gamma / n_j with row normalization and gamma / max_j n_j
// otherwise (App. B.2).  A count row of ones adds the row and column
// s_j = sum_i a_ij and the corner nnz; Gershgorin row sums n_j + |s_j| and
// nnz + sum_j |s_j| then bound the curvature (the diagonal scaling by their
// inverses is a valid preconditioner and their maximum bounds ||A||^2).
dlm_status upload_steps(dlm_problem* p) {
  const int64_t J = p->J, MJ = p->MJ();
  const int m = p->m;
  std::vector<double> h(MJ + 1, 0.0);
  double hmax = 0.0, tot = 0.0;
  for (int64_t q = 0; q < MJ; ++q) {
    double hq;
    if (m == 1) {
      hq = p->lay.h_n2[q];
    } else {  // Gershgorin row sum of item j's m x m block
      const int64_t f = q / J, j = q % J;
      hq = 0.0;
      for (int l = 0; l < m; ++l) hq += std::fabs(p->h_gram[(static_cast<size_t>(f) * m + l) * J + j]);
    }
    if (p->count_on) {
      hq += std::fabs(p->lay.h_s1[q]);
      tot += std::fabs(p->lay.h_s1[q]);
    }
    h[q] = hq;
    hmax = hq > hmax ? hq : hmax;
  }
  if (p->count_on) {
    const double hc = static_cast<double>(p->glob_nnz) + tot;
    h[MJ] = hc;
    hmax = hc > hmax ? hc : hmax;
  }
  p->curv_max = hmax;
  CK(cudaMemcpyAsync(p->curv, h.data(), sizeof(double) * (MJ + 1), cudaMemcpyHostToDevice, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return DLM_OK;
}

// Exponent of the iteration sweep's fixed-point objective sum: a bound on
// |sum_i (c x_i + gamma/2 ||x_i||^2)| for the largest gamma of the schedule
// (every x_ij <= z; on the simplex sum_j x_ij <= z per user).
int objective_shift(const dlm_problem* p) {
  const bool simplex = p->kind == DLM_SIMPLEX_LE || p->kind == DLM_SIMPLEX_EQ;
  const double units = static_cast<double>(simplex ? p->glob_users : p->glob_nnz);
  const double per = p->z * (p->lay.max_abs_c + 0.5 * p->gamma0 * p->z);
  const double bound = (units > 0 ? units : 1.0) * (per > 0 ? per : 1.0);
  return std::max(fixed_point_shift(bound), 0);
}

// The stage table of the continuation schedule (Sec. 6, App. B.2):
// gamma_0 = gamma0, gamma_{s+1} = max(gamma_end, gamma_s * factor), up to the
// first stage at gamma_end (every later stage has the same gamma).
dlm_status upload_schedule(dlm_problem* p) {
  std::vector<double> tab(1, p->gamma0);
  while (tab.back() != p->gamma_end) {
    if (static_cast<int64_t>(tab.size()) >= kMaxStageTable)
      return fail(DLM_ERR_UNSUPPORTED, "the schedule takes more than 2^20 stages to reach gamma_end");
    const double n = tab.back() * p->factor;
    tab.push_back(n > p->gamma_end ? n : p->gamma_end);
  }
  CK(cudaStreamSynchronize(p->stream));
  if (static_cast<int64_t>(tab.size()) > p->gamma_tab_cap) {
    cudaFree(p->gamma_tab);
    p->gamma_tab = nullptr;
    p->gamma_tab_cap = 0;
    CK(dalloc(&p->gamma_tab, tab.size()));
    p->gamma_tab_cap = static_cast<int64_t>(tab.size());
  }
  p->h_gamma_tab = tab;
  p->nstages = static_cast<int64_t>(tab.size());
  p->sO = objective_shift(p);
  CK(cudaMemcpyAsync(p->gamma_tab, p->h_gamma_tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice,
                     p->stream));
  k_state_reset<<<1, 1, 0, p->stream>>>(p->state, p->gamma0);
  CK(cudaGetLastError());
  k_momentum_reset<<<blocks_for(p->D()), 256, 0, p->stream>>>(p->lam64, p->y64, p->lam, p->y, p->D(), p->state);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(p->objq, 0, sizeof(unsigned long long), p->stream));
  CK(cudaStreamSynchronize(p->stream));
  p->traj_from = 0;
  invalidate_graph(p->run);
  return write_tables(p->run);
}

// Saved iterates and state of the members (tuning trials must not advance them).
struct Saved {
  std::vector<double*> lam, y;
  std::vector<DevState> st;
};
dlm_status save_state(Runner& R, Saved* S) {
  CK(cudaStreamSynchronize(R.stream));
  for (dlm_problem* p : R.probs) {
    double *l = nullptr, *y = nullptr;
    CK(dalloc(&l, p->D()));
    CK(dalloc(&y, p->D()));
    CK(cudaMemcpy(l, p->lam64, sizeof(double) * p->D(), cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(y, p->y64, sizeof(double) * p->D(), cudaMemcpyDeviceToDevice));
    DevState hs;
    CK(cudaMemcpy(&hs, p->state, sizeof(DevState), cudaMemcpyDeviceToHost));
    S->lam.push_back(l);
    S->y.push_back(y);
    S->st.push_back(hs);
  }
  return DLM_OK;
}
dlm_status restore_state(Runner& R, const Saved& S) {
  CK(cudaStreamSynchronize(R.stream));
  for (size_t i = 0; i < R.probs.size(); ++i) {
    dlm_problem* p = R.probs[i];
    CK(cudaMemcpy(p->lam64, S.lam[i], sizeof(double) * p->D(), cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(p->y64, S.y[i], sizeof(double) * p->D(), cudaMemcpyDeviceToDevice));
    k_shadow<<<blocks_for(p->D()), 256, 0, R.stream>>>(p->lam64, p->y64, p->lam, p->y, p->D());
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(R.stream));
    CK(cudaMemset(p->cnt, 0, sizeof(unsigned long long)));
    CK(cudaMemset(p->objq, 0, sizeof(unsigned long long)));
    CK(cudaMemcpy(p->state, &S.st[i], sizeof(DevState), cudaMemcpyHostToDevice));
    CK(cudaMemset(p->acc, 0, sizeof(unsigned long long) * p->MJ()));
    p->traj_from = S.st[i].iter;
  }
  return DLM_OK;
}
void free_saved(Saved& S) {
  for (double* q : S.lam) cudaFree(q);
  for (double* q : S.y) cudaFree(q);
  S.lam.clear();
  S.y.clear();
}

// Times candidate mappings for `iters` iterations each (after one warm-up
// iteration) from the same state, keeps the fastest sweep, restores the state.
dlm_status tune(Runner& R, dlm_options base, int iters, dlm_options* chosen, double* best_ms_out) {
  if (iters < 1) iters = 3;
  Saved S;
  dlm_status st = save_state(R, &S);
  if (st != DLM_OK) return st;
  const int threads_c[] = {1024, 512};
  const int coop_c[] = {1, 6, 12, 20, 33};
  const int assign_c[] = {kAssignInterleaved, kAssignContiguous, kAssignDynamic};
  const size_t smem = sweep_smem_bytes(R.smemJ, false);
  int sm_bytes = 0;
  cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, R.device);
  dlm_options best = base;
  double best_ms = 1e300;
  for (int th : threads_c) {
    if (th == 512 && 2 * (smem + 2048) > static_cast<size_t>(sm_bytes)) continue;  // two CTAs per SM must fit
    for (int as : assign_c) {
      if (as == kAssignInterleaved && R.probs.size() > 8) continue;  // too many segments per CTA
      for (int cm : coop_c) {
        dlm_options o = base;
        o.block_threads = th;
        o.ctas_per_sm = 0;
        o.mapping = as + 1;
        o.coop_max = cm;
        st = runner_configure(R, o, false);
        if (st == DLM_OK) st = restore_state(R, S);
        double sw = 0;
        if (st == DLM_OK) st = runner_step_timed(R, 1, nullptr, nullptr, nullptr);
        if (st == DLM_OK) st = restore_state(R, S);
        if (st == DLM_OK) st = runner_step_timed(R, iters, &sw, nullptr, nullptr);
        if (st != DLM_OK) {
          free_saved(S);
          return st;
        }
        if (sw < best_ms) {
          best_ms = sw;
          best = o;
        }
      }
    }
  }
  // the first-pass scan width, with the mapping chosen above (one-family
  // sweeps; rows with many active edges resolve without the threshold
  // iteration when eight values are tracked)
  bool one_family = true;
  for (const dlm_problem* p : R.probs) one_family = one_family && p->m == 1 && p->kind != DLM_BOX_CUT;
  if (one_family) {
    dlm_options o = best;
    o.topk = best.topk == 8 ? 4 : 8;
    double sw = 0;
    st = runner_configure(R, o, false);
    if (st == DLM_OK) st = restore_state(R, S);
    if (st == DLM_OK) st = runner_step_timed(R, 1, nullptr, nullptr, nullptr);
    if (st == DLM_OK) st = restore_state(R, S);
    if (st == DLM_OK) st = runner_step_timed(R, iters, &sw, nullptr, nullptr);
    if (st != DLM_OK) {
      free_saved(S);
      return st;
    }
    if (sw < best_ms) {
      best_ms = sw;
      best = o;
    }
  }
  // the short-row sweep, with the choices above (single one-family handles
  // with rows of at most kShortRowW edges)
  if (short_capable(R) && has_short_slices(R)) {
    dlm_options o = best;
    o.short_rows = best.short_rows ? 0 : 1;
    double sw = 0;
    st = runner_configure(R, o, false);
    if (st == DLM_OK) st = restore_state(R, S);
    if (st == DLM_OK) st = runner_step_timed(R, 1, nullptr, nullptr, nullptr);
    if (st == DLM_OK) st = restore_state(R, S);
    if (st == DLM_OK) st = runner_step_timed(R, iters, &sw, nullptr, nullptr);
    if (st != DLM_OK) {
      free_saved(S);
      return st;
    }
    if (sw < best_ms) {
      best_ms = sw;
      best = o;
    }
  }
  st = runner_configure(R, best, false);
  if (st == DLM_OK) st = restore_state(R, S);
  free_saved(S);
  if (chosen) *chosen = best;
  if (best_ms_out) *best_ms_out = best_ms / iters;
  return st;
}

// A batch's stream and its members' streams may differ: batch work waits for
// the work already enqueued on each member's stream, and later member work
// waits for the batch work (stream-ordered, no host synchronization).
dlm_status batch_enter(Runner& R) {
  for (dlm_problem* p : R.probs) {
    if (p->stream == R.stream) continue;
    CK(cudaEventRecord(p->ev, p->stream));
    CK(cudaStreamWaitEvent(R.stream, p->ev, 0));
  }
  return DLM_OK;
}
dlm_status batch_leave(Runner& R) {
  CK(cudaEventRecord(R.done, R.stream));
  for (dlm_problem* p : R.probs)
    if (p->stream != R.stream) CK(cudaStreamWaitEvent(p->stream, R.done, 0));
  return DLM_OK;
}

dlm_status check_options(const dlm_options* opt) {
  if (!opt) return fail(DLM_ERR_INVALID_ARG, "null options");
  if (opt->gap_every < 0 || opt->graph_iters < 0 || opt->mapping < 0 || opt->mapping > 3 || opt->ctas_per_sm < 0 ||
      opt->ctas_per_sm > 4 || opt->coop_max < 0 || opt->coop_max > 33 ||
      (opt->block_threads != 0 && opt->block_threads != 512 && opt->block_threads != 1024) || opt->restart < 0 ||
      opt->restart > 1 || (opt->topk != 0 && opt->topk != 4 && opt->topk != 8) || opt->short_rows < 0 ||
      opt->short_rows > 1)
    return fail(DLM_ERR_INVALID_ARG, "bad option value");
  return DLM_OK;
}

dlm_status shard_only_error() {
  return fail(DLM_ERR_UNSUPPORTED, "a shard handle iterates through dlm_shard_sweep / dlm_shard_update");
}


// A shard's rows on the device (copied from host memory when they live
// there); the copies are freed with the object.
struct ShardRows {
  const int64_t* rp = nullptr;
  const int32_t* col = nullptr;
  const void *c = nullptr, *a = nullptr;
  const double* b = nullptr;
  void* tmp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaStream_t s = nullptr;
  ~ShardRows() {
    for (void* q : tmp) dev_free(q, s);
    if (s) cudaStreamSynchronize(s);
  }
};

dlm_status shard_rows(const dlm_problem_desc* d, cudaStream_t s, ShardRows* r) {
  if (!d) return fail(DLM_ERR_INVALID_ARG, "null argument");
  if (d->num_users < 0 || d->num_items <= 0 || d->nnz < 0 || d->num_users >= (int64_t(1) << 31) ||
      d->num_items > 65536)
    return fail(DLM_ERR_INVALID_ARG, "bad sizes");
  if (!d->row_ptr || (d->nnz > 0 && (!d->item_idx || !d->c || !d->a)) || !d->b)
    return fail(DLM_ERR_INVALID_ARG, "null array pointer");
  if (d->val_dtype != DLM_F32 && d->val_dtype != DLM_BF16) return fail(DLM_ERR_INVALID_ARG, "bad val_dtype");
  if (d->num_families > 1) return fail(DLM_ERR_UNSUPPORTED, "a user-sharded instance with several capacity families");
  if (d->memspace != DLM_MEM_DEVICE && d->memspace != DLM_MEM_HOST) return fail(DLM_ERR_INVALID_ARG, "bad memspace");
  r->s = s;
  r->rp = d->row_ptr;
  r->col = d->item_idx;
  r->c = d->c;
  r->a = d->a;
  r->b = d->b;
  if (d->memspace == DLM_MEM_HOST) {
    const size_t vs = d->val_dtype == DLM_BF16 ? 2 : 4;
    const size_t sz[5] = {sizeof(int64_t) * (d->num_users + 1), sizeof(int32_t) * d->nnz, vs * d->nnz, vs * d->nnz,
                          sizeof(double) * d->num_items};
    const void* src[5] = {d->row_ptr, d->item_idx, d->c, d->a, d->b};
    for (int k = 0; k < 5; ++k) {
      if (dev_alloc(&r->tmp[k], sz[k], s) != cudaSuccess) return fail(DLM_ERR_OOM, "device allocation failed");
      if (sz[k] > 0) CK(cudaMemcpyAsync(r->tmp[k], src[k], sz[k], cudaMemcpyHostToDevice, s));
    }
    r->rp = static_cast<const int64_t*>(r->tmp[0]);
    r->col = static_cast<const int32_t*>(r->tmp[1]);
    r->c = r->tmp[2];
    r->a = r->tmp[3];
    r->b = static_cast<const double*>(r->tmp[4]);
  }
  return DLM_OK;
}

dlm_status shard_handle(dlm_problem* p) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  if (!p->sharded) return fail(DLM_ERR_INVALID_ARG, "not a shard handle (dlm_problem_desc.shard was NULL)");
  return DLM_OK;
}

}  // namespace

extern "C" {

const char* dlm_last_error(void) { return g_err.c_str(); }

dlm_status dlm_create(const dlm_problem_desc* desc, void* stream, dlm_problem** out) {
  g_err.clear();
  const auto t_create = std::chrono::steady_clock::now();
  auto since = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_create).count(); };
  if (!desc || !out) return fail(DLM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (desc->num_users < 0 || desc->num_items <= 0 || desc->nnz < 0)
    return fail(DLM_ERR_INVALID_ARG, "num_users >= 0, num_items > 0, nnz >= 0 required");
  if (desc->num_users >= (int64_t(1) << 31) || desc->num_items >= (int64_t(1) << 31))
    return fail(DLM_ERR_UNSUPPORTED, "num_users and num_items must be < 2^31");
  if (!desc->row_ptr || (desc->nnz > 0 && (!desc->item_idx || !desc->c || !desc->a)) || !desc->b)
    return fail(DLM_ERR_INVALID_ARG, "null array pointer");
  if (desc->val_dtype != DLM_F32 && desc->val_dtype != DLM_BF16) return fail(DLM_ERR_INVALID_ARG, "bad val_dtype");
  if (desc->kind != DLM_SIMPLEX_LE && desc->kind != DLM_SIMPLEX_EQ && desc->kind != DLM_BOX &&
      desc->kind != DLM_BOX_CUT)
    return fail(DLM_ERR_INVALID_ARG, "bad simple-set kind");
  if (desc->kind == DLM_BOX_CUT && !(desc->cut > 0 && std::isfinite(desc->cut)))
    return fail(DLM_ERR_INVALID_ARG, "DLM_BOX_CUT needs a finite cut > 0");
  if (desc->kind == DLM_BOX_CUT && desc->num_families > 1)
    return fail(DLM_ERR_UNSUPPORTED, "DLM_BOX_CUT with several capacity families");
  if (!(desc->z > 0) || !std::isfinite(desc->z)) return fail(DLM_ERR_INVALID_ARG, "z must be finite and > 0");
  if (desc->memspace != DLM_MEM_DEVICE && desc->memspace != DLM_MEM_HOST)
    return fail(DLM_ERR_INVALID_ARG, "bad memspace");
  const int m = desc->num_families > 0 ? desc->num_families : 1;
  if (m > kMaxFamilies) return fail(DLM_ERR_UNSUPPORTED, "at most 4 capacity families");
  const dlm_shard* shard = desc->shard;
  if (shard) {
    if (m > 1) return fail(DLM_ERR_UNSUPPORTED, "a user-sharded instance with several capacity families");
    if (!shard->item_sq || !shard->item_sum || !shard->exchange || !shard->cert_exchange || !shard->cert_obj)
      return fail(DLM_ERR_INVALID_ARG, "dlm_shard: null item sums or exchange buffer");
    if (shard->nnz < desc->nnz || shard->active_users < 0 || shard->max_item_degree < 0 ||
        !(shard->max_abs_a >= 0) || !(shard->max_abs_c >= 0))
      return fail(DLM_ERR_INVALID_ARG, "dlm_shard: statistics smaller than this shard's");
  }

  dlm_problem* p = new dlm_problem();
  p->I = desc->num_users;
  p->J = desc->num_items;
  p->nnz = desc->nnz;
  p->bf16 = desc->val_dtype == DLM_BF16;
  p->kind = desc->kind;
  p->cut = desc->kind == DLM_BOX_CUT ? desc->cut : 0.0;
  p->z = desc->z;
  p->m = m;
  p->opt.gap_every = 50;
  p->opt.graph_iters = 10;
  cudaGetDevice(&p->device);
  if (stream) {
    p->stream = static_cast<cudaStream_t>(stream);
  } else {
    // A blocking stream: ordered with the legacy default stream both ways, so
    // callers that produce inputs or read outputs on the default stream see
    // the handle's work in program order.
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamDefault) != cudaSuccess) {
      delete p;
      return fail(DLM_ERR_CUDA, "stream creation failed");
    }
    p->own_stream = true;
  }
  const size_t vs = p->bf16 ? 2 : 4;
  const int64_t I = p->I, J = p->J, nnz = p->nnz;
  // One family: the iteration sweep holds y and G for all items; certificate
  // sweeps take item windows when their three item arrays do not fit.
  if (m > 1 ? sweep_multi_smem_bytes(static_cast<int>(J), m, true) > sweep_smem_limit()
            : (sweep_smem_bytes(static_cast<int>(J), false) > sweep_smem_limit() ||
               sweep_stats_window(static_cast<int>(J)) < 1)) {
    free_problem(p);
    return fail(DLM_ERR_UNSUPPORTED, "num_items too large for the shared-memory item arrays of this build");
  }

  // Bring host inputs to the device (stream ordered).
  const int64_t* rp = desc->row_ptr;
  const int32_t* col = desc->item_idx;
  const void* c = desc->c;
  const void* a = desc->a;
  const double* b = desc->b;
  void* tmp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  dlm_status st = DLM_OK;
  auto cleanup_tmp = [&]() {
    for (void*& q : tmp) {
      dev_free(q, p->stream);
      q = nullptr;
    }
  };
  if (desc->memspace == DLM_MEM_HOST) {
    size_t sz[5] = {sizeof(int64_t) * (I + 1), sizeof(int32_t) * nnz, vs * nnz, vs * nnz * m, sizeof(double) * J * m};
    const void* src[5] = {rp, col, c, a, b};
    for (int k = 0; k < 5; ++k) {
      if (dev_alloc(&tmp[k], sz[k], p->stream) != cudaSuccess) {
        cleanup_tmp();
        free_problem(p);
        return fail(DLM_ERR_OOM, "device allocation for host inputs failed");
      }
      if (sz[k] > 0 && cudaMemcpyAsync(tmp[k], src[k], sz[k], cudaMemcpyHostToDevice, p->stream) != cudaSuccess) {
        cleanup_tmp();
        free_problem(p);
        return fail(DLM_ERR_CUDA, "host-to-device copy failed");
      }
    }
    rp = static_cast<const int64_t*>(tmp[0]);
    col = static_cast<const int32_t*>(tmp[1]);
    c = tmp[2];
    a = tmp[3];
    b = static_cast<const double*>(tmp[4]);
    cudaStreamSynchronize(p->stream);
  }
  p->setup_s[0] = since();

  // Several families: one contiguous array per family (family 0 goes through
  // the one-family layout and validation, the others are checked here).
  void* split = nullptr;
  auto cleanup_all = [&]() {
    cleanup_tmp();
    dev_free(split, p->stream);
    split = nullptr;
  };
  if (m > 1) {
    if (dev_alloc(&split, vs * (nnz > 0 ? nnz : 1) * m, p->stream) != cudaSuccess) {
      cleanup_all();
      free_problem(p);
      return fail(DLM_ERR_OOM, "device allocation for the family split failed");
    }
    if (families_split(a, nnz, m, p->bf16, split, nnz, p->stream) != cudaSuccess) {
      cleanup_all();
      free_problem(p);
      return fail(DLM_ERR_CUDA, "family split failed");
    }
  }
  const void* a0 = m > 1 ? split : a;
  auto fam_ptr = [&](int f) { return static_cast<const char*>(split) + vs * nnz * f; };

  std::string msg;
  ShardGlobal sg{};
  if (shard) {
    sg.nnz = shard->nnz;
    sg.active_users = shard->active_users;
    sg.max_item_deg = shard->max_item_degree;
    sg.max_abs_a = shard->max_abs_a;
    sg.max_abs_c = shard->max_abs_c;
    sg.a_nonneg = shard->a_nonneg != 0;
    sg.item_sq = shard->item_sq;
    sg.item_sum = shard->item_sum;
  }
  st = build_layout(I, J, nnz, rp, col, c, a0, b, p->bf16, p->stream, &p->lay, &msg, nullptr, shard ? &sg : nullptr);
  if (st != DLM_OK) {
    cleanup_all();
    free_problem(p);
    return fail(st, msg);
  }
  for (int k = 0; k < 3; ++k) p->setup_s[1 + k] = p->lay.phase_s[k];
  const double t_layout_end = since();
  p->sharded = shard != nullptr;
  p->glob_nnz = shard ? shard->nnz : nnz;
  p->glob_users = shard ? shard->active_users : p->lay.num_active_users;
  if (m > 1) {
    // the other families: finite values, b >= 0, max |a|, sign
    int* flags = nullptr;
    unsigned* mx = nullptr;
    int h_flags = 0;
    unsigned h_mx = 0;
    std::vector<double> hb(static_cast<size_t>(J) * m);
    cudaError_t e = cudaMalloc(&flags, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&mx, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0, sizeof(unsigned), p->stream);
    for (int f = 1; f < m && e == cudaSuccess; ++f) e = families_check(fam_ptr(f), nnz, p->bf16, flags, mx, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_flags, flags, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_mx, mx, sizeof(unsigned), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hb.data(), b, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cudaFree(flags);
    cudaFree(mx);
    if (e != cudaSuccess) {
      cleanup_all();
      free_problem(p);
      return fail(DLM_ERR_CUDA, std::string("family checks: ") + cudaGetErrorString(e));
    }
    bool bad_b = false;
    for (double v : hb) bad_b = bad_b || !std::isfinite(v) || v < 0;
    if ((h_flags & 1) || bad_b) {
      cleanup_all();
      free_problem(p);
      return fail(DLM_ERR_INVALID_ARG, "non-finite coefficient, or b not finite and >= 0, in a capacity family");
    }
    if (h_flags & 2) p->lay.a_nonneg = false;
    float fm;
    std::memcpy(&fm, &h_mx, sizeof(float));
    p->lay.max_abs_a = std::max(p->lay.max_abs_a, static_cast<double>(fm));
  }
  p->certified = p->lay.a_nonneg && p->kind != DLM_SIMPLEX_EQ;

  // Fixed-point exponents from bounds on any item sum: deg_j * max|v| * xmax.
  const double xmax = p->z;
  const double degm = static_cast<double>(p->lay.max_item_deg > 0 ? p->lay.max_item_deg : 1);
  p->sG = fixed_point_shift(degm * (p->lay.max_abs_a > 0 ? p->lay.max_abs_a : 1.0) * xmax);
  p->sC = fixed_point_shift(degm * (p->lay.max_abs_c > 0 ? p->lay.max_abs_c : 1.0) * xmax);
  p->sQ = fixed_point_shift(degm * xmax * xmax);
  // sum x <= z per user on the simplex, z per edge on the box
  const double nmaxx = static_cast<double>(p->kind == DLM_BOX ? p->glob_nnz : p->glob_users);
  p->sN = fixed_point_shift((nmaxx > 0 ? nmaxx : 1.0) * xmax);
  if (p->sG < 0 || p->sC < 0 || p->sQ < 0 || p->sN < 0) {
    cleanup_all();
    free_problem(p);
    return fail(DLM_ERR_UNSUPPORTED, "item sums too large for 64-bit fixed point");
  }

#define CKC(x)                                                                     \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      cleanup_all();                                                               \
      free_problem(p);                                                             \
      return fail(DLM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    }                                                                              \
  } while (0)

  const int64_t MJ = p->MJ();
  if (m > 1) {
    // extra family streams in slice order, and the per-item Gram sums
    p->ext_stride = p->lay.padded_nnz + 32;
    CKC(dev_alloc(&p->a_ext, vs * p->ext_stride * (m - 1), p->stream));
    for (int f = 1; f < m; ++f)
      CKC(families_gather(p->lay, fam_ptr(f), p->bf16,
                          static_cast<char*>(p->a_ext) + vs * p->ext_stride * (f - 1), p->stream));
    const double degm2 = static_cast<double>(p->lay.max_item_deg > 0 ? p->lay.max_item_deg : 1);
    const int sgr = fixed_point_shift(degm2 * std::max(p->lay.max_abs_a * p->lay.max_abs_a, 1e-300));
    unsigned long long* gacc = nullptr;
    CKC(dalloc(&gacc, J));
    p->h_gram.assign(static_cast<size_t>(m) * m * J, 0.0);
    std::vector<unsigned long long> hq(J);
    for (int f = 0; f < m; ++f)
      for (int l = f; l < m; ++l) {
        CKC(cudaMemsetAsync(gacc, 0, sizeof(unsigned long long) * J, p->stream));
        CKC(families_gram(col, fam_ptr(f), fam_ptr(l), nnz, p->bf16, std::ldexp(1.0f, sgr), gacc, p->stream));
        CKC(cudaMemcpyAsync(hq.data(), gacc, sizeof(unsigned long long) * J, cudaMemcpyDeviceToHost, p->stream));
        CKC(cudaStreamSynchronize(p->stream));
        for (int64_t j = 0; j < J; ++j) {
          const double v = static_cast<double>(static_cast<long long>(hq[j])) * std::ldexp(1.0, -sgr);
          p->h_gram[(static_cast<size_t>(f) * m + l) * J + j] = v;
          p->h_gram[(static_cast<size_t>(l) * m + f) * J + j] = v;
        }
      }
    cudaFree(gacc);
    CKC(sweep_multi_prepare(p->bf16));
  }
  CKC(dalloc(&p->b, MJ));
  CKC(cudaMemcpyAsync(p->b, b, sizeof(double) * MJ, cudaMemcpyDeviceToDevice, p->stream));
  CKC(dalloc(&p->curv, MJ + 1));
  CKC(dalloc(&p->lam, MJ + 1));
  CKC(dalloc(&p->y, MJ + 1));
  CKC(dalloc(&p->lam64, MJ + 1));
  CKC(dalloc(&p->y64, MJ + 1));
  CKC(dalloc(&p->traj, kTrajCap));
  CKC(dalloc(&p->upd_part, 2 * static_cast<size_t>(update_ctas(MJ + 1)) + 1));
  CKC(dalloc(&p->upd_ticket, 2));
  CKC(dalloc(&p->upd_flag, 1));
  CKC(cudaMemsetAsync(p->upd_ticket, 0, sizeof(unsigned) * 2, p->stream));
  CKC(cudaMemsetAsync(p->upd_flag, 0, sizeof(int32_t), p->stream));
  CKC(cudaMemsetAsync(p->lam64, 0, sizeof(double) * (MJ + 1), p->stream));
  CKC(cudaMemsetAsync(p->y64, 0, sizeof(double) * (MJ + 1), p->stream));
  CKC(cudaMemsetAsync(p->traj, 0, sizeof(double) * kTrajCap, p->stream));
  if (shard) {
    p->xsum = reinterpret_cast<unsigned long long*>(shard->exchange);
    p->csum = reinterpret_cast<unsigned long long*>(shard->cert_exchange);
    p->cobj = shard->cert_obj;
    p->own_sums = false;
  } else {
    CKC(dalloc(&p->xsum, MJ + 2));
    CKC(dalloc(&p->csum, MJ + 2 * J + 1));
  }
  CKC(cudaMemsetAsync(p->xsum, 0, sizeof(unsigned long long) * (MJ + 2), p->stream));
  CKC(cudaMemsetAsync(p->csum, 0, sizeof(unsigned long long) * (MJ + 2 * J + 1), p->stream));
  p->acc = p->xsum;
  p->cnt = p->xsum + MJ;
  p->objq = p->xsum + MJ + 1;
  p->acc2 = p->csum;
  p->accC = p->csum + MJ;
  p->accQ = p->csum + MJ + J;
  p->cnt2 = p->csum + MJ + 2 * J;
  CKC(cudaMemsetAsync(p->lam, 0, sizeof(float) * (MJ + 1), p->stream));
  CKC(cudaMemsetAsync(p->y, 0, sizeof(float) * (MJ + 1), p->stream));
  CKC(dalloc(&p->calc_gamma, 1));
  CKC(dalloc(&p->stats_out, 8));
  CKC(dalloc(&p->state, 1));
  CKC(dalloc(&p->inst_calc, 1));
  CKC(dalloc(&p->st_calc, 1));
  CKC(cudaMallocHost(reinterpret_cast<void**>(&p->h_out), sizeof(double) * 8));
  CKC(cudaMallocHost(reinterpret_cast<void**>(&p->h_inst), sizeof(InstDesc)));
  CKC(cudaMallocHost(reinterpret_cast<void**>(&p->h_stinst), sizeof(StatsInst)));
  CKC(sweep_prepare(p->bf16));
  if (p->kind == DLM_BOX_CUT) CKC(sweep_boxcut_prepare(p->bf16));
  CKC(cudaEventCreateWithFlags(&p->ev, cudaEventDisableTiming));
  p->h_slice_off.resize(p->lay.nslices + 1);
  CKC(cudaMemcpyAsync(p->h_slice_off.data(), p->lay.slice_off, sizeof(int64_t) * (p->lay.nslices + 1),
                      cudaMemcpyDeviceToHost, p->stream));
  CKC(cudaStreamSynchronize(p->stream));
  cleanup_all();
  for (void*& q : tmp) q = nullptr;
#undef CKC
  // The handle's own runner: this one instance.
  Runner& R = p->run;
  R.probs = {p};
  R.stream = p->stream;
  R.bf16 = p->bf16;
  R.device = p->device;
  R.smemJ = static_cast<int>(J);
  R.win = m > 1 ? R.smemJ : sweep_stats_window(R.smemJ);
  cudaDeviceGetAttribute(&R.sms, cudaDevAttrMultiProcessorCount, p->device);
  p->h_gamma_tab.assign(1, p->gamma0);
  st = upload_steps(p);
  if (st == DLM_OK) st = runner_configure(R, p->opt, true);
  if (st == DLM_OK) st = upload_schedule(p);
  if (st != DLM_OK) {
    free_problem(p);
    return st;
  }
  p->setup_s[5] = since();
  p->setup_s[4] = p->setup_s[5] - t_layout_end;
  *out = p;
  return DLM_OK;
}

dlm_status dlm_set_schedule(dlm_problem* p, double gamma0, double gamma_end, double factor, int64_t iters_per_stage) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  if (!(gamma_end > 0) || !(gamma0 >= gamma_end) || !std::isfinite(gamma0) || !(factor > 0) || factor > 1 ||
      iters_per_stage < 1 || (factor == 1 && gamma0 != gamma_end))
    return fail(DLM_ERR_INVALID_ARG,
                "need gamma0 >= gamma_end > 0, 0 < factor <= 1 (1 only with gamma0 == gamma_end), "
                "iters_per_stage >= 1");
  const double g0 = p->gamma0, ge = p->gamma_end, f = p->factor;
  const int64_t ips = p->ips;
  p->gamma0 = gamma0;
  p->gamma_end = gamma_end;
  p->factor = factor;
  p->ips = iters_per_stage;
  const dlm_status st = upload_schedule(p);
  if (st == DLM_ERR_UNSUPPORTED) {  // keep the previous schedule
    p->gamma0 = g0;
    p->gamma_end = ge;
    p->factor = f;
    p->ips = ips;
  }
  return st;
}

dlm_status dlm_set_count_limit(dlm_problem* p, double M) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  if (p->m > 1) return fail(DLM_ERR_UNSUPPORTED, "a count constraint with several capacity families");
  if (p->kind == DLM_BOX_CUT) return fail(DLM_ERR_UNSUPPORTED, "a count constraint with DLM_BOX_CUT");
  if (std::isnan(M) || M < 0) return fail(DLM_ERR_INVALID_ARG, "M must be >= 0 (INFINITY removes the constraint)");
  CK(cudaStreamSynchronize(p->stream));
  p->count_on = std::isfinite(M);
  p->count_M = M;
  // the count dual starts at 0; its accumulators are clear
  CK(cudaMemset(p->lam + p->J, 0, sizeof(float)));
  CK(cudaMemset(p->y + p->J, 0, sizeof(float)));
  CK(cudaMemset(p->lam64 + p->J, 0, sizeof(double)));
  CK(cudaMemset(p->y64 + p->J, 0, sizeof(double)));
  CK(cudaMemset(p->cnt, 0, sizeof(unsigned long long)));
  CK(cudaMemset(p->cnt2, 0, sizeof(unsigned long long)));
  dlm_status st = upload_steps(p);
  if (st != DLM_OK) return st;
  invalidate_graph(p->run);
  return write_tables(p->run);
}

dlm_status dlm_set_options(dlm_problem* p, const dlm_options* opt) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  dlm_status st = check_options(opt);
  if (st != DLM_OK) return st;
  dlm_options o = *opt;
  if (o.gap_every == 0) o.gap_every = 50;
  if (o.graph_iters == 0) o.graph_iters = 10;
  p->opt = o;
  return runner_configure(p->run, o, false);
}

dlm_status dlm_get_options(dlm_problem* p, dlm_options* opt) {
  if (!p || !opt) return fail(DLM_ERR_INVALID_ARG, "null argument");
  *opt = p->opt;
  return DLM_OK;
}

dlm_status dlm_autotune(dlm_problem* p, int32_t iters, dlm_options* chosen, double* sweep_ms) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  dlm_options best{};
  dlm_status st = tune(p->run, p->opt, iters, &best, sweep_ms);
  if (st != DLM_OK) return st;
  p->opt = best;
  if (chosen) *chosen = best;
  return DLM_OK;
}

dlm_status dlm_set_lambda(dlm_problem* p, const float* lambda0, int32_t memspace) {
  if (!p || !lambda0) return fail(DLM_ERR_INVALID_ARG, "null argument");
  const float* src = lambda0;
  float* tmp = nullptr;
  if (memspace == DLM_MEM_HOST) {
    CK(dalloc(&tmp, p->D()));
    CK(cudaMemcpyAsync(tmp, lambda0, sizeof(float) * p->D(), cudaMemcpyHostToDevice, p->stream));
    src = tmp;
  }
  k_warm<<<blocks_for(p->D()), 256, 0, p->stream>>>(src, p->lam64, p->y64, p->lam, p->y, p->D(), p->state);
  cudaError_t e = cudaGetLastError();
  if (tmp) {
    cudaStreamSynchronize(p->stream);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) return fail(DLM_ERR_CUDA, cudaGetErrorString(e));
  return DLM_OK;
}

dlm_status dlm_step(dlm_problem* p, int64_t n_iters) {
  if (!p || n_iters < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  if (p->sharded) return shard_only_error();
  return runner_step(p->run, n_iters);
}

dlm_status dlm_step_timed(dlm_problem* p, int64_t n_iters, double* sweep_ms, double* update_ms, double* total_ms) {
  if (!p || n_iters < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  if (p->sharded) return shard_only_error();
  return runner_step_timed(p->run, n_iters, sweep_ms, update_ms, total_ms);
}

dlm_status dlm_get_stats(dlm_problem* p, dlm_stats* out) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  if (p->sharded) return shard_only_error();
  dlm_status st = enqueue_certificate(p->run, p->run.inst_stats, p->run.st_stats);
  if (st != DLM_OK) return st;
  return read_stats(p, out);
}

dlm_status dlm_solve(dlm_problem* p, double target_rel_gap, int64_t max_iters, dlm_stats* out) {
  if (!p || max_iters < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  if (p->sharded) return shard_only_error();
  const auto t0 = std::chrono::steady_clock::now();
  dlm_stats s{};
  int64_t start_iter = 0;
  {
    DevState hs;
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaMemcpy(&hs, p->state, sizeof(DevState), cudaMemcpyDeviceToHost));
    start_iter = hs.iter;
  }
  dlm_status result = DLM_ERR_TIMEOUT;
  for (;;) {
    dlm_status st = dlm_get_stats(p, &s);
    if (st != DLM_OK) return st;
    if (s.status != DLM_OK) {
      result = static_cast<dlm_status>(s.status);
      g_err = s.status == DLM_ERR_NUMERIC ? "non-finite value in the iteration" : "a device-side check failed";
      break;
    }
    if (s.gamma == p->gamma_end && s.rel_gap <= target_rel_gap) {
      result = DLM_OK;
      s.converged = 1;
      break;
    }
    const int64_t done = s.iter - start_iter;
    if (done >= max_iters) break;
    int64_t n = p->opt.gap_every > 0 ? p->opt.gap_every : 50;
    if (n > max_iters - done) n = max_iters - done;
    st = runner_step(p->run, n);
    if (st != DLM_OK) return st;
  }
  const auto t1 = std::chrono::steady_clock::now();
  p->last_solve_seconds = std::chrono::duration<double>(t1 - t0).count();
  s.seconds = p->last_solve_seconds;
  if (out) *out = s;
  if (result == DLM_ERR_TIMEOUT && s.status == DLM_OK) g_err = "max_iters reached before the target gap";
  return result;
}

dlm_status dlm_calculate(dlm_problem* p, const float* lambda, double gamma, double* g, float* grad, float* x) {
  if (!p || !lambda) return fail(DLM_ERR_INVALID_ARG, "null argument");
  if (p->sharded) return shard_only_error();
  if (!(gamma > 0) || !std::isfinite(gamma)) return fail(DLM_ERR_INVALID_ARG, "gamma must be > 0");
  CK(cudaStreamSynchronize(p->stream));
  k_set_double<<<1, 1, 0, p->stream>>>(p->calc_gamma, gamma);
  CK(cudaGetLastError());
  InstDesc d = base_desc(p);
  d.y = lambda;
  d.gamma = p->calc_gamma;
  d.acc = p->acc2;
  d.accC = p->accC;
  d.accQ = p->accQ;
  d.seg_obj = p->run.seg_obj;
  d.xout = x;
  *p->h_inst = d;
  CK(cudaMemcpyAsync(p->inst_calc, p->h_inst, sizeof(InstDesc), cudaMemcpyHostToDevice, p->stream));
  StatsInst s = base_stats(p, p->run, 0);
  s.lam = lambda;
  s.gamma = p->calc_gamma;
  s.grad_out = grad;
  s.state = nullptr;
  *p->h_stinst = s;
  CK(cudaMemcpyAsync(p->st_calc, p->h_stinst, sizeof(StatsInst), cudaMemcpyHostToDevice, p->stream));
  dlm_status st = enqueue_certificate(p->run, p->inst_calc, p->st_calc);
  if (st != DLM_OK) return st;
  CK(cudaMemcpyAsync(p->h_out, p->stats_out, sizeof(double) * 8, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (g) *g = p->h_out[0];
  return DLM_OK;
}

dlm_status dlm_get_lambda(dlm_problem* p, float* out, int32_t memspace) {
  if (!p || !out) return fail(DLM_ERR_INVALID_ARG, "null argument");
  CK(cudaMemcpyAsync(out, p->lam, sizeof(float) * p->D(),
                     memspace == DLM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, p->stream));
  if (memspace == DLM_MEM_HOST) CK(cudaStreamSynchronize(p->stream));
  return DLM_OK;
}

dlm_status dlm_get_x(dlm_problem* p, float* out, int32_t memspace) {
  if (!p || !out) return fail(DLM_ERR_INVALID_ARG, "null argument");
  float* dst = out;
  float* tmp = nullptr;
  if (memspace == DLM_MEM_HOST) {
    CK(dalloc(&tmp, p->nnz));
    dst = tmp;
  }
  CK(cudaStreamSynchronize(p->stream));
  InstDesc d = base_desc(p);
  d.y = p->lam;
  d.gamma = &p->state->gamma;
  d.acc = p->acc2;
  d.accC = p->accC;
  d.accQ = p->accQ;
  d.seg_obj = p->run.seg_obj;
  d.xout = dst;
  *p->h_inst = d;
  CK(cudaMemcpyAsync(p->inst_calc, p->h_inst, sizeof(InstDesc), cudaMemcpyHostToDevice, p->stream));
  StatsInst s = base_stats(p, p->run, 0);
  s.lam = p->lam;
  s.gamma = &p->state->gamma;
  s.state = p->state;
  *p->h_stinst = s;
  CK(cudaMemcpyAsync(p->st_calc, p->h_stinst, sizeof(StatsInst), cudaMemcpyHostToDevice, p->stream));
  dlm_status st = enqueue_certificate(p->run, p->inst_calc, p->st_calc);
  if (st == DLM_OK && tmp) {
    CK(cudaMemcpyAsync(out, tmp, sizeof(float) * p->nnz, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
  }
  if (tmp) {
    cudaStreamSynchronize(p->stream);
    cudaFree(tmp);
  }
  return st;
}

dlm_status dlm_get_state(dlm_problem* p, double* lam, double* y, dlm_state* s, int32_t memspace) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  const cudaMemcpyKind k = memspace == DLM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (lam) CK(cudaMemcpyAsync(lam, p->lam64, sizeof(double) * p->D(), k, p->stream));
  if (y) CK(cudaMemcpyAsync(y, p->y64, sizeof(double) * p->D(), k, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (s) {
    DevState hs;
    CK(cudaMemcpy(&hs, p->state, sizeof(DevState), cudaMemcpyDeviceToHost));
    s->iter = hs.iter;
    s->theta = hs.theta;
    s->stage = hs.stage;
    s->reserved = 0;
  }
  return DLM_OK;
}

dlm_status dlm_set_state(dlm_problem* p, const double* lam, const double* y, const dlm_state* s, int32_t memspace) {
  if (!p || !lam || !y || !s) return fail(DLM_ERR_INVALID_ARG, "null argument");
  if (s->iter < 0 || s->stage < 0) return fail(DLM_ERR_INVALID_ARG, "bad state");
  const cudaMemcpyKind k = memspace == DLM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaStreamSynchronize(p->stream));
  CK(cudaMemcpy(p->lam64, lam, sizeof(double) * p->D(), k));
  CK(cudaMemcpy(p->y64, y, sizeof(double) * p->D(), k));
  k_shadow<<<blocks_for(p->D()), 256, 0, p->stream>>>(p->lam64, p->y64, p->lam, p->y, p->D());
  CK(cudaGetLastError());
  DevState hs{};
  hs.iter = s->iter;
  hs.theta = s->theta;
  hs.stage = s->stage;
  hs.gamma = p->h_gamma_tab[s->stage < p->nstages ? s->stage : p->nstages - 1];
  hs.status = 0;
  CK(cudaStreamSynchronize(p->stream));
  CK(cudaMemcpy(p->state, &hs, sizeof(DevState), cudaMemcpyHostToDevice));
  p->traj_from = s->iter;
  return DLM_OK;
}

dlm_status dlm_get_trajectory(dlm_problem* p, int64_t first_iter, int64_t n, double* g_out) {
  if (!p || (n > 0 && !g_out) || n < 0 || first_iter < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  DevState hs;
  CK(cudaStreamSynchronize(p->stream));
  CK(cudaMemcpy(&hs, p->state, sizeof(DevState), cudaMemcpyDeviceToHost));
  const int64_t lo = std::max<int64_t>(p->traj_from, hs.iter - kTrajCap);
  if (first_iter < lo || first_iter + n > hs.iter)
    return fail(DLM_ERR_INVALID_ARG, "requested iterations [" + std::to_string(first_iter) + ", " +
                                         std::to_string(first_iter + n) + ") outside the recorded range [" +
                                         std::to_string(lo) + ", " + std::to_string(hs.iter) + ")");
  std::vector<double> ring(kTrajCap);
  CK(cudaMemcpy(ring.data(), p->traj, sizeof(double) * kTrajCap, cudaMemcpyDeviceToHost));
  for (int64_t k = 0; k < n; ++k) g_out[k] = ring[(first_iter + k) % kTrajCap];
  return DLM_OK;
}

dlm_status dlm_get_info(dlm_problem* p, int64_t* num_users, int64_t* num_items, int64_t* nnz,
                        int64_t* bytes_per_iter) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  if (num_users) *num_users = p->I;
  if (num_items) *num_items = p->J;
  if (nnz) *nnz = p->nnz;
  if (bytes_per_iter) *bytes_per_iter = p->nnz * (4 + (1 + p->m) * (p->bf16 ? 2 : 4)) + (p->I + 1) * 8;
  return DLM_OK;
}

void dlm_destroy(dlm_problem* p) { free_problem(p); }

dlm_status dlm_get_setup_seconds(dlm_problem* p, double* out, int32_t n) {
  if (!p || (n > 0 && !out) || n < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  for (int k = 0; k < n && k < 6; ++k) out[k] = p->setup_s[k];
  return DLM_OK;
}

// ---------------------------------------------------------------------------
// User-sharded instances
// ---------------------------------------------------------------------------

dlm_status dlm_shard_local(const dlm_problem_desc* desc, void* stream, dlm_shard* local, int64_t* item_degree) {
  g_err.clear();
  if (!local || !item_degree) return fail(DLM_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ShardRows r;
  dlm_status st = shard_rows(desc, s, &r);
  if (st != DLM_OK) return st;
  LayoutOut lay;
  RowStats rs;
  std::string msg;
  st = build_layout(desc->num_users, desc->num_items, desc->nnz, r.rp, r.col, r.c, r.a, r.b,
                    desc->val_dtype == DLM_BF16, s, &lay, &msg, &rs, nullptr);
  if (st != DLM_OK) return fail(st, msg);
  *local = dlm_shard{};
  local->nnz = rs.nnz;
  local->active_users = rs.active_users;
  local->max_item_degree = rs.max_item_deg;
  local->max_abs_a = rs.max_abs_a;
  local->max_abs_c = rs.max_abs_c;
  local->a_nonneg = rs.a_nonneg ? 1 : 0;
  for (int64_t j = 0; j < desc->num_items; ++j) item_degree[j] = static_cast<int64_t>(rs.item_deg[j]);
  return DLM_OK;
}

dlm_status dlm_shard_item_sums(const dlm_problem_desc* desc, const dlm_shard* global, void* stream, int64_t* item_sq,
                               int64_t* item_sum) {
  g_err.clear();
  if (!global || !item_sq || !item_sum) return fail(DLM_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ShardRows r;
  dlm_status st = shard_rows(desc, s, &r);
  if (st != DLM_OK) return st;
  int ssq = 0, ss1 = 0;
  item_sum_shifts(global->max_item_degree, global->max_abs_a, &ssq, &ss1);
  std::string msg;
  st = item_sums(desc->num_items, desc->nnz, r.col, r.a, desc->val_dtype == DLM_BF16, ssq, ss1, s, item_sq, item_sum,
                 &msg);
  if (st != DLM_OK) return fail(st, msg);
  return DLM_OK;
}

dlm_status dlm_shard_sweep(dlm_problem* p) {
  dlm_status st = shard_handle(p);
  if (st != DLM_OK) return st;
  CK(dispatch_sweep(p->run, launch_of(p->run, p->run.inst_iter), false, p->bf16));
  return DLM_OK;
}

dlm_status dlm_shard_update(dlm_problem* p) {
  dlm_status st = shard_handle(p);
  if (st != DLM_OK) return st;
  CK(launch_update(p->run.upd, 1, p->run.upd_ctas, p->run.upd_test, p->stream));
  return DLM_OK;
}

dlm_status dlm_shard_cert_sweep(dlm_problem* p) {
  dlm_status st = shard_handle(p);
  if (st != DLM_OK) return st;
  CK(dispatch_sweep(p->run, launch_of(p->run, p->run.inst_stats), true, p->bf16));
  CK(launch_seg_sum(p->run.st_stats, p->cobj, p->stream));
  return DLM_OK;
}

dlm_status dlm_shard_cert_finish(dlm_problem* p, dlm_stats* out) {
  dlm_status st = shard_handle(p);
  if (st != DLM_OK) return st;
  CK(launch_stats(p->run.st_stats, 1, p->stream));
  return read_stats(p, out);
}

dlm_status dlm_release_cached_memory(void) {
  const cudaError_t e = release_cached_memory();
  if (e != cudaSuccess) return fail(DLM_ERR_CUDA, std::string("memory pool trim: ") + cudaGetErrorString(e));
  return DLM_OK;
}

dlm_status dlm_ws_features(dlm_problem* p, const float* lam_prev, double gamma, float* X) {
  if (!p || !lam_prev || !X) return fail(DLM_ERR_INVALID_ARG, "null argument");
  if (p->m > 1) return fail(DLM_ERR_UNSUPPORTED, "warm-start features with several capacity families");
  if (!(gamma > 0) || !std::isfinite(gamma)) return fail(DLM_ERR_INVALID_ARG, "gamma must be > 0");
  float* grad = nullptr;
  unsigned* deg = nullptr;
  int* mx = nullptr;
  unsigned long long* sum = nullptr;
  auto release = [&]() {
    cudaFree(grad);
    cudaFree(deg);
    cudaFree(mx);
    cudaFree(sum);
  };
  if (dalloc(&grad, p->D()) != cudaSuccess || dalloc(&deg, p->J) != cudaSuccess || dalloc(&mx, p->J) != cudaSuccess ||
      dalloc(&sum, p->J) != cudaSuccess) {
    release();
    return fail(DLM_ERR_OOM, "device allocation failed");
  }
  double g = 0;
  dlm_status st = dlm_calculate(p, lam_prev, gamma, &g, grad, nullptr);
  if (st == DLM_OK) {
    const double bound = static_cast<double>(p->lay.max_item_deg > 0 ? p->lay.max_item_deg : 1) *
                         (p->lay.max_abs_c > 0 ? p->lay.max_abs_c : 1.0);
    const double scale = std::ldexp(1.0, fixed_point_shift(bound));
    cudaError_t e = launch_item_features(p->lay.col16, p->lay.ca, p->bf16, p->lay.padded_nnz, static_cast<int>(p->J),
                                         scale, p->b, lam_prev, gamma, grad, X, deg, mx, sum, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) st = fail(DLM_ERR_CUDA, std::string("item features: ") + cudaGetErrorString(e));
  }
  release();
  return st;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------

dlm_status dlm_batch_create(dlm_problem* const* probs, int32_t n, void* stream, dlm_batch** out) {
  if (!probs || n <= 0 || !out) return fail(DLM_ERR_INVALID_ARG, "need n > 0 problems");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!probs[i]) return fail(DLM_ERR_INVALID_ARG, "null problem in batch");
    if (probs[i]->bf16 != probs[0]->bf16) return fail(DLM_ERR_INVALID_ARG, "batch members must share val_dtype");
    if (probs[i]->device != probs[0]->device) return fail(DLM_ERR_INVALID_ARG, "batch members must share a device");
    if (probs[i]->m != probs[0]->m)
      return fail(DLM_ERR_UNSUPPORTED, "batch members with different numbers of capacity families");
    if (probs[i]->m > 1 && probs[i]->count_on)
      return fail(DLM_ERR_UNSUPPORTED, "a count constraint with several capacity families");
    if ((probs[i]->kind == DLM_BOX_CUT) != (probs[0]->kind == DLM_BOX_CUT))
      return fail(DLM_ERR_UNSUPPORTED, "DLM_BOX_CUT members batch only with each other");
    if (probs[i]->sharded) return fail(DLM_ERR_UNSUPPORTED, "a shard handle in a batch");
    for (int k = 0; k < i; ++k)
      if (probs[k] == probs[i]) return fail(DLM_ERR_INVALID_ARG, "a problem appears twice in the batch");
  }
  dlm_batch* bt = new dlm_batch();
  Runner& R = bt->run;
  R.probs.assign(probs, probs + n);
  R.bf16 = probs[0]->bf16;
  R.device = probs[0]->device;
  cudaDeviceGetAttribute(&R.sms, cudaDevAttrMultiProcessorCount, R.device);
  if (stream) {
    R.stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&R.stream, cudaStreamDefault) != cudaSuccess) {
      delete bt;
      return fail(DLM_ERR_CUDA, "stream creation failed");
    }
    bt->own_stream = true;
  }
  for (int i = 0; i < n; ++i) {
    cudaStreamSynchronize(probs[i]->stream);
    R.smemJ = std::max(R.smemJ, static_cast<int>(probs[i]->J));
  }
  const int m = probs[0]->m;
  R.win = m > 1 ? R.smemJ : sweep_stats_window(R.smemJ);
  if (m > 1 ? sweep_multi_smem_bytes(R.smemJ, m, true) > sweep_smem_limit()
            : (sweep_smem_bytes(R.smemJ, false) > sweep_smem_limit() || R.win < 1)) {
    if (bt->own_stream) cudaStreamDestroy(R.stream);
    delete bt;
    return fail(DLM_ERR_UNSUPPORTED, "largest num_items of the batch too large for the shared-memory item arrays");
  }
  if (cudaEventCreateWithFlags(&R.done, cudaEventDisableTiming) != cudaSuccess) {
    if (bt->own_stream) cudaStreamDestroy(R.stream);
    delete bt;
    return fail(DLM_ERR_CUDA, "event creation failed");
  }
  dlm_options o = probs[0]->opt;
  o.mapping = 0;
  o.precondition = 0;  // per member, not a batch option
  o.restart = 0;
  bt->opt = o;
  dlm_status st = runner_configure(R, o, true);
  if (st != DLM_OK) {
    runner_free(R);
    if (bt->own_stream) cudaStreamDestroy(R.stream);
    delete bt;
    return st;
  }
  *out = bt;
  return DLM_OK;
}

dlm_status dlm_batch_set_options(dlm_batch* bt, const dlm_options* opt) {
  if (!bt) return fail(DLM_ERR_INVALID_ARG, "null batch");
  dlm_status st = check_options(opt);
  if (st != DLM_OK) return st;
  dlm_options o = *opt;
  if (o.gap_every == 0) o.gap_every = 50;
  if (o.graph_iters == 0) o.graph_iters = 10;
  bt->opt = o;
  return runner_configure(bt->run, o, false);
}

dlm_status dlm_batch_autotune(dlm_batch* bt, int32_t iters, dlm_options* chosen, double* sweep_ms) {
  if (!bt) return fail(DLM_ERR_INVALID_ARG, "null batch");
  dlm_options best{};
  dlm_status st = batch_enter(bt->run);
  if (st == DLM_OK) st = tune(bt->run, bt->opt, iters, &best, sweep_ms);
  if (st != DLM_OK) return st;
  bt->opt = best;
  if (chosen) *chosen = best;
  return DLM_OK;
}

dlm_status dlm_batch_step(dlm_batch* bt, int64_t n_iters) {
  if (!bt || n_iters < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  dlm_status st = batch_enter(bt->run);
  if (st == DLM_OK) st = runner_step(bt->run, n_iters);
  if (st == DLM_OK) st = batch_leave(bt->run);
  return st;
}

dlm_status dlm_batch_step_timed(dlm_batch* bt, int64_t n_iters, double* sweep_ms, double* update_ms,
                                double* total_ms) {
  if (!bt || n_iters < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  dlm_status st = batch_enter(bt->run);
  if (st == DLM_OK) st = runner_step_timed(bt->run, n_iters, sweep_ms, update_ms, total_ms);
  if (st == DLM_OK) st = batch_leave(bt->run);
  return st;
}

dlm_status dlm_batch_get_stats(dlm_batch* bt, dlm_stats* out) {
  if (!bt) return fail(DLM_ERR_INVALID_ARG, "null batch");
  Runner& R = bt->run;
  dlm_status st = batch_enter(R);
  if (st == DLM_OK) st = enqueue_certificate(R, R.inst_stats, R.st_stats);
  if (st != DLM_OK) return st;
  CK(cudaStreamSynchronize(R.stream));
  for (size_t i = 0; i < R.probs.size(); ++i) {
    st = read_stats(R.probs[i], out ? out + i : nullptr);
    if (st != DLM_OK) return st;
  }
  return DLM_OK;
}

dlm_status dlm_batch_solve(dlm_batch* bt, double target_rel_gap, int64_t max_iters, dlm_stats* out) {
  if (!bt || max_iters < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  Runner& R = bt->run;
  const size_t n = R.probs.size();
  std::vector<dlm_stats> s(n);
  const auto t0 = std::chrono::steady_clock::now();
  int64_t done = 0;
  const int64_t every = bt->opt.gap_every > 0 ? bt->opt.gap_every : 50;
  dlm_status result = DLM_ERR_TIMEOUT;
  for (;;) {
    dlm_status st = dlm_batch_get_stats(bt, s.data());
    if (st != DLM_OK) return st;
    bool all = true, bad = false;
    for (size_t i = 0; i < n; ++i) {
      if (s[i].status != DLM_OK) bad = true;
      s[i].converged = (s[i].gamma == R.probs[i]->gamma_end && s[i].rel_gap <= target_rel_gap) ? 1 : 0;
      all = all && s[i].converged;
    }
    if (bad) {
      result = DLM_ERR_NUMERIC;
      g_err = "a batch member reported a device-side error";
      break;
    }
    if (all) {
      result = DLM_OK;
      break;
    }
    if (done >= max_iters) break;
    const int64_t k = std::min(every, max_iters - done);
    st = runner_step(R, k);
    if (st == DLM_OK) st = batch_leave(R);
    if (st != DLM_OK) return st;
    done += k;
  }
  bt->last_solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (size_t i = 0; i < n; ++i) s[i].seconds = bt->last_solve_seconds;
  if (out) std::copy(s.begin(), s.end(), out);
  if (result == DLM_ERR_TIMEOUT) g_err = "max_iters reached before every member met the target gap";
  return result;
}

void dlm_batch_destroy(dlm_batch* bt) {
  if (!bt) return;
  cudaStreamSynchronize(bt->run.stream);
  runner_free(bt->run);
  if (bt->own_stream) cudaStreamDestroy(bt->run.stream);
  delete bt;
}

}  // extern "C"
