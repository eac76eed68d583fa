// api.cu -- the C-ABI (include/dlm.h): handle life cycle, schedule and
// options, CUDA-graph replay of the iteration, certified-gap checks and the
// solve loop.  All device work of a handle runs on its stream.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

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

#define CK(x)                                                                                      \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ != cudaSuccess) return fail(DLM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kNumTables = 1;  // slice assignment orders (reserved for the tuner)

__global__ void k_set_double(double* p, double v) { *p = v; }

// lam <- max(src, 0), y <- lam, theta <- 1 (warm start).
__global__ void k_warm(const float* src, float* lam, float* y, int64_t J, DevState* st) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < J;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float v = fmaxf(src[j], 0.f);
    lam[j] = v;
    y[j] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->theta = 1.0;
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

__global__ void k_inv(const double* n2, double* inv, int64_t J) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < J;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x)
    inv[j] = n2[j] > 0.0 ? 1.0 / n2[j] : 0.0;
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

}  // namespace

struct dlm_problem {
  int64_t I = 0, J = 0, nnz = 0;
  bool bf16 = false;
  int kind = DLM_SIMPLEX_LE;
  double z = 1.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  LayoutOut lay;
  int sG = 0, sC = 0, sQ = 0;
  bool certified = true;

  double *b = nullptr, *inv_n2 = nullptr;
  float *lam = nullptr, *y = nullptr;
  unsigned long long *acc = nullptr, *acc2 = nullptr, *accC = nullptr, *accQ = nullptr;
  double *gamma_tab = nullptr, *calc_gamma = nullptr, *seg_obj = nullptr, *stats_out = nullptr;
  DevState* state = nullptr;
  InstDesc *inst_iter = nullptr, *inst_stats = nullptr, *inst_calc = nullptr;
  UpdInst* upd = nullptr;
  StatsInst *st_stats = nullptr, *st_calc = nullptr;
  Task* tasks = nullptr;
  int32_t *cta_task = nullptr, *seg_list = nullptr;
  int ntasks = 0, nseg = 0, grid = 0, smemJ = 0, table = 0;
  std::vector<Task> h_tasks;
  std::vector<int32_t> h_cta, h_seg;

  // pinned host staging
  double* h_out = nullptr;  // 8 doubles
  InstDesc* h_inst = nullptr;
  StatsInst* h_stinst = nullptr;
  UpdInst* h_upd = nullptr;

  double gamma0 = 1e-2, gamma_end = 1e-2, factor = 0.5;
  int64_t ips = 1 << 30;
  dlm_options opt{};
  std::vector<double> h_gamma_tab;

  cudaGraphExec_t gexec = nullptr;
  int gexec_iters = 0;
  std::vector<cudaEvent_t> events;
  double last_solve_seconds = 0;
};

namespace {

InstDesc base_desc(const dlm_problem* p) {
  InstDesc d{};
  d.slice_off = p->lay.slice_off;
  d.slice_w = p->lay.slice_w;
  d.col = p->lay.col;
  d.ca = p->lay.ca;
  d.orig_off = p->lay.orig_off;
  d.udeg = p->lay.udeg;
  d.nusers = p->lay.num_active_users;
  d.status = &p->state->status;
  d.scaleG = std::ldexp(1.0f, p->sG);
  d.scaleC = std::ldexp(1.0f, p->sC);
  d.scaleQ = std::ldexp(1.0f, p->sQ);
  d.z = static_cast<float>(p->z);
  d.J = static_cast<int32_t>(p->J);
  d.kind = p->kind;
  return d;
}

StatsInst base_stats(const dlm_problem* p) {
  StatsInst s{};
  s.b = p->b;
  s.acc = p->acc2;
  s.accC = p->accC;
  s.accQ = p->accQ;
  s.seg_obj = p->seg_obj;
  s.seg_list = p->seg_list;
  s.nseg = p->nseg;
  s.J = static_cast<int32_t>(p->J);
  s.inv_sG = std::ldexp(1.0, -p->sG);
  s.inv_sC = std::ldexp(1.0, -p->sC);
  s.inv_sQ = std::ldexp(1.0, -p->sQ);
  s.out = p->stats_out;
  s.certified = p->certified ? 1 : 0;
  return s;
}

void invalidate_graph(dlm_problem* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  p->gexec = nullptr;
  p->gexec_iters = 0;
}

// Per-CTA task lists: CTA k sweeps slices k, k + V, k + 2V, ...; slices are
// sorted by width, so every CTA (and every warp) gets the same mix of widths.
dlm_status build_tasks(dlm_problem* p) {
  const int V = p->grid;
  p->h_tasks.clear();
  p->h_cta.assign(V + 1, 0);
  p->h_seg.clear();
  for (int k = 0; k < V; ++k) {
    p->h_cta[k] = static_cast<int32_t>(p->h_tasks.size());
    if (k < p->lay.nslices) {
      Task t;
      t.inst = 0;
      t.stride = V;
      t.first = k;
      t.end = p->lay.nslices;
      p->h_tasks.push_back(t);
      p->h_seg.push_back(p->h_cta[k]);
    }
  }
  p->h_cta[V] = static_cast<int32_t>(p->h_tasks.size());
  p->ntasks = static_cast<int>(p->h_tasks.size());
  p->nseg = static_cast<int>(p->h_seg.size());
  cudaFree(p->tasks);
  cudaFree(p->cta_task);
  cudaFree(p->seg_list);
  cudaFree(p->seg_obj);
  p->tasks = nullptr;
  p->cta_task = nullptr;
  p->seg_list = nullptr;
  p->seg_obj = nullptr;
  CK(dalloc(&p->tasks, p->h_tasks.size()));
  CK(dalloc(&p->cta_task, p->h_cta.size()));
  CK(dalloc(&p->seg_list, p->h_seg.size()));
  CK(dalloc(&p->seg_obj, p->h_tasks.size()));
  if (!p->h_tasks.empty())
    CK(cudaMemcpy(p->tasks, p->h_tasks.data(), sizeof(Task) * p->h_tasks.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->cta_task, p->h_cta.data(), sizeof(int32_t) * p->h_cta.size(), cudaMemcpyHostToDevice));
  if (!p->h_seg.empty())
    CK(cudaMemcpy(p->seg_list, p->h_seg.data(), sizeof(int32_t) * p->h_seg.size(), cudaMemcpyHostToDevice));
  invalidate_graph(p);
  return DLM_OK;
}

// Device tables derived from the handle (re-written after option changes).
dlm_status write_tables(dlm_problem* p) {
  InstDesc it = base_desc(p);
  it.y = p->y;
  it.gamma = &p->state->gamma;
  it.acc = p->acc;
  it.accC = p->accC;
  it.accQ = p->accQ;
  it.seg_obj = p->seg_obj;
  it.xout = nullptr;
  InstDesc ss = base_desc(p);
  ss.y = p->lam;
  ss.gamma = &p->state->gamma;
  ss.acc = p->acc2;
  ss.accC = p->accC;
  ss.accQ = p->accQ;
  ss.seg_obj = p->seg_obj;
  ss.xout = nullptr;
  CK(cudaMemcpy(p->inst_iter, &it, sizeof(InstDesc), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->inst_stats, &ss, sizeof(InstDesc), cudaMemcpyHostToDevice));

  UpdInst u{};
  u.state = p->state;
  u.gamma_tab = p->gamma_tab;
  u.b = p->b;
  u.inv_n2 = p->inv_n2;
  u.lam = p->lam;
  u.y = p->y;
  u.acc = p->acc;
  u.iters_per_stage = p->ips;
  u.inv_nmax = p->lay.n2max > 0 ? 1.0 / p->lay.n2max : 0.0;
  u.inv_scaleG = std::ldexp(1.0, -p->sG);
  u.J = static_cast<int32_t>(p->J);
  u.precondition = p->opt.precondition ? 1 : 0;
  CK(cudaMemcpy(p->upd, &u, sizeof(UpdInst), cudaMemcpyHostToDevice));

  StatsInst st = base_stats(p);
  st.lam = p->lam;
  st.gamma = &p->state->gamma;
  st.grad_out = nullptr;
  st.state = p->state;
  CK(cudaMemcpy(p->st_stats, &st, sizeof(StatsInst), cudaMemcpyHostToDevice));
  invalidate_graph(p);
  return DLM_OK;
}

dlm_status enqueue_iteration(dlm_problem* p) {
  SweepLaunch L;
  L.inst = p->inst_iter;
  L.tasks = p->tasks;
  L.cta_task = p->cta_task;
  L.grid = p->grid;
  L.smemJ = p->smemJ;
  L.stream = p->stream;
  CK(launch_sweep(L, false, p->bf16));
  CK(launch_update(p->upd, 1, p->stream));
  return DLM_OK;
}

dlm_status enqueue_certificate(dlm_problem* p, const InstDesc* inst_tab, const StatsInst* st_tab) {
  SweepLaunch L;
  L.inst = inst_tab;
  L.tasks = p->tasks;
  L.cta_task = p->cta_task;
  L.grid = p->grid;
  L.smemJ = p->smemJ;
  L.stream = p->stream;
  CK(launch_sweep(L, true, p->bf16));
  CK(launch_stats(st_tab, 1, p->stream));
  return DLM_OK;
}

dlm_status capture_graph(dlm_problem* p, int iters) {
  invalidate_graph(p);
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  dlm_status st = DLM_OK;
  for (int i = 0; i < iters && st == DLM_OK; ++i) st = enqueue_iteration(p);
  cudaError_t e = cudaStreamEndCapture(p->stream, &g);
  if (st != DLM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(DLM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&p->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(DLM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  p->gexec_iters = iters;
  return DLM_OK;
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
    out->status = (hs.status & kStatNumeric) ? DLM_ERR_NUMERIC
                  : (hs.status & kStatTimeout) ? DLM_ERR_TIMEOUT
                                               : DLM_OK;
    out->converged = 0;
  }
  return DLM_OK;
}

void free_problem(dlm_problem* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  invalidate_graph(p);
  cudaFree(p->lay.slice_off);
  cudaFree(p->lay.slice_w);
  cudaFree(p->lay.col);
  cudaFree(p->lay.ca);
  cudaFree(p->lay.orig_off);
  cudaFree(p->lay.udeg);
  cudaFree(p->lay.n2);
  void* ptrs[] = {p->b,        p->inv_n2,    p->lam,      p->y,        p->acc,      p->acc2,     p->accC,
                  p->accQ,     p->gamma_tab, p->calc_gamma, p->seg_obj, p->stats_out, p->state,    p->inst_iter,
                  p->inst_stats, p->inst_calc, p->upd,     p->st_stats, p->st_calc,  p->tasks,    p->cta_task,
                  p->seg_list};
  for (void* q : ptrs) cudaFree(q);
  cudaFreeHost(p->h_out);
  cudaFreeHost(p->h_inst);
  cudaFreeHost(p->h_stinst);
  cudaFreeHost(p->h_upd);
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

dlm_status upload_schedule(dlm_problem* p) {
  p->h_gamma_tab.assign(kMaxStages, 0.0);
  double g = p->gamma0;
  for (int s = 0; s < kMaxStages; ++s) {
    p->h_gamma_tab[s] = g;
    const double n = g * p->factor;
    g = n > p->gamma_end ? n : p->gamma_end;
  }
  CK(cudaMemcpyAsync(p->gamma_tab, p->h_gamma_tab.data(), sizeof(double) * kMaxStages, cudaMemcpyHostToDevice,
                     p->stream));
  k_state_reset<<<1, 1, 0, p->stream>>>(p->state, p->gamma0);
  CK(cudaGetLastError());
  k_warm<<<blocks_for(p->J), 256, 0, p->stream>>>(p->lam, p->lam, p->y, p->J, p->state);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  return write_tables(p);
}

}  // namespace

extern "C" {

const char* dlm_last_error(void) { return g_err.c_str(); }

dlm_status dlm_create(const dlm_problem_desc* desc, void* stream, dlm_problem** out) {
  g_err.clear();
  if (!desc || !out) return fail(DLM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (desc->num_users < 0 || desc->num_items <= 0 || desc->nnz < 0)
    return fail(DLM_ERR_INVALID_ARG, "num_users >= 0, num_items > 0, nnz >= 0 required");
  if (desc->num_users >= (int64_t(1) << 31) || desc->num_items >= (int64_t(1) << 31))
    return fail(DLM_ERR_UNSUPPORTED, "num_users and num_items must be < 2^31");
  if (!desc->row_ptr || (desc->nnz > 0 && (!desc->item_idx || !desc->c || !desc->a)) || !desc->b)
    return fail(DLM_ERR_INVALID_ARG, "null array pointer");
  if (desc->val_dtype != DLM_F32 && desc->val_dtype != DLM_BF16) return fail(DLM_ERR_INVALID_ARG, "bad val_dtype");
  if (desc->kind != DLM_SIMPLEX_LE && desc->kind != DLM_SIMPLEX_EQ && desc->kind != DLM_BOX)
    return fail(DLM_ERR_INVALID_ARG, "bad simple-set kind");
  if (!(desc->z > 0) || !std::isfinite(desc->z)) return fail(DLM_ERR_INVALID_ARG, "z must be finite and > 0");
  if (desc->memspace != DLM_MEM_DEVICE && desc->memspace != DLM_MEM_HOST)
    return fail(DLM_ERR_INVALID_ARG, "bad memspace");

  dlm_problem* p = new dlm_problem();
  p->I = desc->num_users;
  p->J = desc->num_items;
  p->nnz = desc->nnz;
  p->bf16 = desc->val_dtype == DLM_BF16;
  p->kind = desc->kind;
  p->z = desc->z;
  p->opt.gap_every = 50;
  p->opt.mapping = -1;
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

  // Bring host inputs to the device (stream ordered).
  const int64_t* rp = desc->row_ptr;
  const int32_t* col = desc->item_idx;
  const void* c = desc->c;
  const void* a = desc->a;
  const double* b = desc->b;
  void* tmp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  dlm_status st = DLM_OK;
  auto cleanup_tmp = [&]() {
    for (void* q : tmp) cudaFree(q);
  };
  if (desc->memspace == DLM_MEM_HOST) {
    size_t sz[5] = {sizeof(int64_t) * (I + 1), sizeof(int32_t) * nnz, vs * nnz, vs * nnz, sizeof(double) * J};
    const void* src[5] = {rp, col, c, a, b};
    for (int k = 0; k < 5; ++k) {
      if (cudaMalloc(&tmp[k], sz[k] > 0 ? sz[k] : 16) != cudaSuccess) {
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
  }

  std::string msg;
  st = build_layout(I, J, nnz, rp, col, c, a, b, p->bf16, p->stream, &p->lay, &msg);
  if (st != DLM_OK) {
    cleanup_tmp();
    free_problem(p);
    return fail(st, msg);
  }
  p->certified = p->lay.a_nonneg && p->kind != DLM_SIMPLEX_EQ;

  // Fixed-point exponents from bounds on any item sum: deg_j * max|v| * xmax.
  const double xmax = p->z;
  const double degm = static_cast<double>(p->lay.max_item_deg > 0 ? p->lay.max_item_deg : 1);
  p->sG = fixed_point_shift(degm * (p->lay.max_abs_a > 0 ? p->lay.max_abs_a : 1.0) * xmax);
  p->sC = fixed_point_shift(degm * (p->lay.max_abs_c > 0 ? p->lay.max_abs_c : 1.0) * xmax);
  p->sQ = fixed_point_shift(degm * xmax * xmax);
  if (p->sG < 0 || p->sC < 0 || p->sQ < 0) {
    cleanup_tmp();
    free_problem(p);
    return fail(DLM_ERR_UNSUPPORTED, "item sums too large for 64-bit fixed point");
  }

  p->smemJ = static_cast<int>(J);
  if (sweep_smem_bytes(p->smemJ, true) > sweep_smem_limit()) {
    cleanup_tmp();
    free_problem(p);
    return fail(DLM_ERR_UNSUPPORTED, "num_items too large for the shared-memory item arrays of this build");
  }

#define CKC(x)                                                                 \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      cleanup_tmp();                                                           \
      free_problem(p);                                                         \
      return fail(DLM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    }                                                                          \
  } while (0)

  CKC(dalloc(&p->b, J));
  CKC(cudaMemcpyAsync(p->b, b, sizeof(double) * J, cudaMemcpyDeviceToDevice, p->stream));
  CKC(dalloc(&p->inv_n2, J));
  k_inv<<<blocks_for(J), 256, 0, p->stream>>>(p->lay.n2, p->inv_n2, J);
  CKC(cudaGetLastError());
  CKC(dalloc(&p->lam, J));
  CKC(dalloc(&p->y, J));
  CKC(dalloc(&p->acc, J));
  CKC(dalloc(&p->acc2, J));
  CKC(dalloc(&p->accC, J));
  CKC(dalloc(&p->accQ, J));
  for (unsigned long long* q : {p->acc, p->acc2, p->accC, p->accQ})
    CKC(cudaMemsetAsync(q, 0, sizeof(unsigned long long) * J, p->stream));
  CKC(cudaMemsetAsync(p->lam, 0, sizeof(float) * J, p->stream));
  CKC(cudaMemsetAsync(p->y, 0, sizeof(float) * J, p->stream));
  CKC(dalloc(&p->gamma_tab, kMaxStages));
  CKC(dalloc(&p->calc_gamma, 1));
  CKC(dalloc(&p->stats_out, 8));
  CKC(dalloc(&p->state, 1));
  CKC(dalloc(&p->inst_iter, 1));
  CKC(dalloc(&p->inst_stats, 1));
  CKC(dalloc(&p->inst_calc, 1));
  CKC(dalloc(&p->upd, 1));
  CKC(dalloc(&p->st_stats, 1));
  CKC(dalloc(&p->st_calc, 1));
  CKC(cudaMallocHost(reinterpret_cast<void**>(&p->h_out), sizeof(double) * 8));
  CKC(cudaMallocHost(reinterpret_cast<void**>(&p->h_inst), sizeof(InstDesc)));
  CKC(cudaMallocHost(reinterpret_cast<void**>(&p->h_stinst), sizeof(StatsInst)));
  CKC(cudaMallocHost(reinterpret_cast<void**>(&p->h_upd), sizeof(UpdInst)));
  CKC(sweep_prepare(p->bf16));
  {
    int sms = 0;
    CKC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    p->grid = sms;  // persistent: one sweep CTA per SM
  }
  CKC(cudaStreamSynchronize(p->stream));
  cleanup_tmp();
  for (void*& q : tmp) q = nullptr;
#undef CKC
  p->table = 0;
  st = build_tasks(p);
  if (st == DLM_OK) st = upload_schedule(p);
  if (st != DLM_OK) {
    free_problem(p);
    return st;
  }
  *out = p;
  return DLM_OK;
}

dlm_status dlm_set_schedule(dlm_problem* p, double gamma0, double gamma_end, double factor, int64_t iters_per_stage) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  if (!(gamma_end > 0) || !(gamma0 >= gamma_end) || !std::isfinite(gamma0) || !(factor > 0) || factor > 1 ||
      iters_per_stage < 1)
    return fail(DLM_ERR_INVALID_ARG, "need gamma0 >= gamma_end > 0, 0 < factor <= 1, iters_per_stage >= 1");
  p->gamma0 = gamma0;
  p->gamma_end = gamma_end;
  p->factor = factor;
  p->ips = iters_per_stage;
  return upload_schedule(p);
}

dlm_status dlm_set_options(dlm_problem* p, const dlm_options* opt) {
  if (!p || !opt) return fail(DLM_ERR_INVALID_ARG, "null argument");
  if (opt->gap_every < 0 || opt->graph_iters < 0 || opt->mapping >= kNumTables || opt->ctas_per_sm < 0)
    return fail(DLM_ERR_INVALID_ARG, "bad option value");
  dlm_options o = *opt;
  if (o.gap_every == 0) o.gap_every = 50;
  if (o.graph_iters == 0) o.graph_iters = 10;
  const int table = o.mapping < 0 ? 0 : o.mapping;
  int grid = p->grid;
  if (o.ctas_per_sm > 0) {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    grid = sms * o.ctas_per_sm;
  }
  p->opt = o;
  CK(cudaStreamSynchronize(p->stream));
  if (table != p->table || grid != p->grid) {
    p->table = table;
    p->grid = grid;
    dlm_status st = build_tasks(p);
    if (st != DLM_OK) return st;
  }
  return write_tables(p);
}

dlm_status dlm_set_lambda(dlm_problem* p, const float* lambda0, int32_t memspace) {
  if (!p || !lambda0) return fail(DLM_ERR_INVALID_ARG, "null argument");
  const float* src = lambda0;
  float* tmp = nullptr;
  if (memspace == DLM_MEM_HOST) {
    CK(dalloc(&tmp, p->J));
    CK(cudaMemcpyAsync(tmp, lambda0, sizeof(float) * p->J, cudaMemcpyHostToDevice, p->stream));
    src = tmp;
  }
  k_warm<<<blocks_for(p->J), 256, 0, p->stream>>>(src, p->lam, p->y, p->J, p->state);
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
  const int gi = p->opt.graph_iters > 0 ? p->opt.graph_iters : 10;
  if (n_iters >= gi && (!p->gexec || p->gexec_iters != gi)) {
    dlm_status st = capture_graph(p, gi);
    if (st != DLM_OK) return st;
  }
  int64_t done = 0;
  for (; done + gi <= n_iters; done += gi) CK(cudaGraphLaunch(p->gexec, p->stream));
  for (; done < n_iters; ++done) {
    dlm_status st = enqueue_iteration(p);
    if (st != DLM_OK) return st;
  }
  return DLM_OK;
}

dlm_status dlm_step_timed(dlm_problem* p, int64_t n_iters, double* sweep_ms, double* update_ms, double* total_ms) {
  if (!p || n_iters < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
  const size_t need = static_cast<size_t>(2 * n_iters + 1);
  while (p->events.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    p->events.push_back(e);
  }
  SweepLaunch L;
  L.inst = p->inst_iter;
  L.tasks = p->tasks;
  L.cta_task = p->cta_task;
  L.grid = p->grid;
  L.smemJ = p->smemJ;
  L.stream = p->stream;
  CK(cudaEventRecord(p->events[0], p->stream));
  for (int64_t i = 0; i < n_iters; ++i) {
    CK(launch_sweep(L, false, p->bf16));
    CK(cudaEventRecord(p->events[2 * i + 1], p->stream));
    CK(launch_update(p->upd, 1, p->stream));
    CK(cudaEventRecord(p->events[2 * i + 2], p->stream));
  }
  CK(cudaStreamSynchronize(p->stream));
  double ss = 0, su = 0;
  for (int64_t i = 0; i < n_iters; ++i) {
    float a = 0, b = 0;
    CK(cudaEventElapsedTime(&a, p->events[2 * i], p->events[2 * i + 1]));
    CK(cudaEventElapsedTime(&b, p->events[2 * i + 1], p->events[2 * i + 2]));
    ss += a;
    su += b;
  }
  float tot = 0;
  if (n_iters > 0) CK(cudaEventElapsedTime(&tot, p->events[0], p->events[2 * n_iters]));
  if (sweep_ms) *sweep_ms = ss;
  if (update_ms) *update_ms = su;
  if (total_ms) *total_ms = tot;
  return DLM_OK;
}

dlm_status dlm_get_stats(dlm_problem* p, dlm_stats* out) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  dlm_status st = enqueue_certificate(p, p->inst_stats, p->st_stats);
  if (st != DLM_OK) return st;
  return read_stats(p, out);
}

dlm_status dlm_solve(dlm_problem* p, double target_rel_gap, int64_t max_iters, dlm_stats* out) {
  if (!p || max_iters < 0) return fail(DLM_ERR_INVALID_ARG, "bad argument");
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
  int64_t done = 0;
  for (;;) {
    dlm_status st = dlm_get_stats(p, &s);
    if (st != DLM_OK) return st;
    if (s.status != DLM_OK) {
      result = static_cast<dlm_status>(s.status);
      g_err = s.status == DLM_ERR_NUMERIC ? "non-finite value in the iteration"
                                          : "a device-side wait ran out of its limit";
      break;
    }
    if (s.gamma == p->gamma_end && s.rel_gap <= target_rel_gap) {
      result = DLM_OK;
      s.converged = 1;
      break;
    }
    done = s.iter - start_iter;
    if (done >= max_iters) break;
    int64_t n = p->opt.gap_every;
    if (n > max_iters - done) n = max_iters - done;
    st = dlm_step(p, n);
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
  d.seg_obj = p->seg_obj;
  d.xout = x;
  *p->h_inst = d;
  CK(cudaMemcpyAsync(p->inst_calc, p->h_inst, sizeof(InstDesc), cudaMemcpyHostToDevice, p->stream));
  StatsInst s = base_stats(p);
  s.lam = lambda;
  s.gamma = p->calc_gamma;
  s.grad_out = grad;
  s.state = nullptr;
  *p->h_stinst = s;
  CK(cudaMemcpyAsync(p->st_calc, p->h_stinst, sizeof(StatsInst), cudaMemcpyHostToDevice, p->stream));
  dlm_status st = enqueue_certificate(p, p->inst_calc, p->st_calc);
  if (st != DLM_OK) return st;
  CK(cudaMemcpyAsync(p->h_out, p->stats_out, sizeof(double) * 8, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (g) *g = p->h_out[0];
  return DLM_OK;
}

dlm_status dlm_get_lambda(dlm_problem* p, float* out, int32_t memspace) {
  if (!p || !out) return fail(DLM_ERR_INVALID_ARG, "null argument");
  CK(cudaMemcpyAsync(out, p->lam, sizeof(float) * p->J,
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
  d.seg_obj = p->seg_obj;
  d.xout = dst;
  *p->h_inst = d;
  CK(cudaMemcpyAsync(p->inst_calc, p->h_inst, sizeof(InstDesc), cudaMemcpyHostToDevice, p->stream));
  StatsInst s = base_stats(p);
  s.lam = p->lam;
  s.gamma = &p->state->gamma;
  s.state = p->state;
  *p->h_stinst = s;
  CK(cudaMemcpyAsync(p->st_calc, p->h_stinst, sizeof(StatsInst), cudaMemcpyHostToDevice, p->stream));
  dlm_status st = enqueue_certificate(p, p->inst_calc, p->st_calc);
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

dlm_status dlm_get_state(dlm_problem* p, float* lam, float* y, dlm_state* s, int32_t memspace) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  const cudaMemcpyKind k = memspace == DLM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (lam) CK(cudaMemcpyAsync(lam, p->lam, sizeof(float) * p->J, k, p->stream));
  if (y) CK(cudaMemcpyAsync(y, p->y, sizeof(float) * p->J, k, p->stream));
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

dlm_status dlm_set_state(dlm_problem* p, const float* lam, const float* y, const dlm_state* s, int32_t memspace) {
  if (!p || !lam || !y || !s) return fail(DLM_ERR_INVALID_ARG, "null argument");
  if (s->iter < 0 || s->stage < 0) return fail(DLM_ERR_INVALID_ARG, "bad state");
  const cudaMemcpyKind k = memspace == DLM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaStreamSynchronize(p->stream));
  CK(cudaMemcpy(p->lam, lam, sizeof(float) * p->J, k));
  CK(cudaMemcpy(p->y, y, sizeof(float) * p->J, k));
  DevState hs{};
  hs.iter = s->iter;
  hs.theta = s->theta;
  hs.stage = s->stage;
  hs.gamma = p->h_gamma_tab[s->stage < kMaxStages ? s->stage : kMaxStages - 1];
  hs.status = 0;
  CK(cudaMemcpy(p->state, &hs, sizeof(DevState), cudaMemcpyHostToDevice));
  return DLM_OK;
}

dlm_status dlm_get_info(dlm_problem* p, int64_t* num_users, int64_t* num_items, int64_t* nnz,
                        int64_t* bytes_per_iter) {
  if (!p) return fail(DLM_ERR_INVALID_ARG, "null handle");
  if (num_users) *num_users = p->I;
  if (num_items) *num_items = p->J;
  if (nnz) *nnz = p->nnz;
  if (bytes_per_iter) *bytes_per_iter = p->nnz * (4 + 2 * (p->bf16 ? 2 : 4)) + (p->I + 1) * 8;
  return DLM_OK;
}

void dlm_destroy(dlm_problem* p) { free_problem(p); }

}  // extern "C"
