// dlm_impl.cuh -- internal structures of the dual-sweep solver (not part of
// the C-ABI).  Shared by the sweep, update, layout and API translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dlm.h"

namespace dlm {

constexpr int kWarp = 32;
constexpr int kSweepThreads = 512;  // 16 warps per sweep CTA
constexpr int kUpdThreads = 1024;   // one CTA per instance for the O(J) kernels
constexpr int kMaxStages = 64;      // continuation stages tabulated (gamma is flat after)
constexpr int kNumClasses = 12;     // degree classes: 0, 1, 2, 3-4, 5-8, ..., 257-512, 513+

// Error bits of the device status word.
enum : int32_t { kStatNumeric = 1, kStatTimeout = 2, kStatBadMap = 4 };

// Degree class of a user: 0 for d = 0, otherwise 1 + ceil(log2 d) capped.
__host__ __device__ inline int degree_class(int64_t d) {
  if (d <= 0) return 0;
  int c = 1;
  int64_t cap = 1;
  while (cap < d && c < kNumClasses - 1) {
    cap <<= 1;
    ++c;
  }
  return c;
}

// Mapping ids (how a degree class is laid on lanes).  Register mappings
// process users of degree <= L*K with L lanes per user and K edges per lane;
// kMapStream runs one warp per user over an arbitrarily long row.
enum : int32_t {
  kMapStream = 0,
  kMapL1K4 = 1,
  kMapL1K8 = 2,
  kMapL2K8 = 3,
  kMapL4K8 = 4,
  kMapL8K8 = 5,
  kMapL16K8 = 6,
  kMapL32K8 = 7,
  kMapL2K4 = 8,
  kMapL4K4 = 9,
  kMapL8K4 = 10,
  kMapL16K4 = 11,
  kMapL32K4 = 12,
  kNumMaps = 13
};
__host__ __device__ inline int map_lanes(int m) {
  switch (m) {
    case kMapL1K4: case kMapL1K8: return 1;
    case kMapL2K8: case kMapL2K4: return 2;
    case kMapL4K8: case kMapL4K4: return 4;
    case kMapL8K8: case kMapL8K4: return 8;
    case kMapL16K8: case kMapL16K4: return 16;
    default: return 32;
  }
}
__host__ __device__ inline int map_k(int m) {
  switch (m) {
    case kMapL1K4: case kMapL2K4: case kMapL4K4: case kMapL8K4: case kMapL16K4: case kMapL32K4: return 4;
    case kMapStream: return 0;
    default: return 8;
  }
}
// Users handled by one warp pass.
__host__ __device__ inline int map_users_per_pass(int m) { return m == kMapStream ? 1 : kWarp / map_lanes(m); }

// Per-instance iteration state (device memory).
struct DevState {
  int64_t iter;   // next iteration index t
  double theta;   // momentum scalar
  double gamma;   // gamma of iteration t's stage
  int32_t stage;  // stage index of iteration t
  int32_t status; // error bits
};

// Per-instance constants of the update step (device memory).
struct UpdInst {
  DevState* state;
  const double* gamma_tab;  // [kMaxStages]
  const double* b;          // [J]
  const double* inv_n2;     // [J] 1 / sum_i a_ij^2 (0 for empty items)
  float* lam;               // [J]
  float* y;                 // [J]
  unsigned long long* acc;  // [J] fixed-point A x at y
  int64_t iters_per_stage;
  double inv_nmax;          // 1 / max_j sum_i a_ij^2
  double inv_scaleG;        // 2^-sG
  int32_t J;
  int32_t precondition;
};

// Per-instance view for the sweep kernels (device memory; one table for the
// iteration sweep at y, one for the certificate sweep at lam).
struct InstDesc {
  const int64_t* rp;        // bucketed row pointer [I+1]
  const int32_t* col;       // [nnz]
  const void* c;            // [nnz] float or bf16
  const void* a;            // [nnz]
  const int64_t* orig_off;  // [I] caller row start of each bucketed user
  const float* y;           // sweep point [J]
  const double* gamma;      // ridge used by this sweep
  unsigned long long* acc;  // [J] fixed-point sum a x
  unsigned long long* accC; // [J] fixed-point sum c x (stats)
  unsigned long long* accQ; // [J] fixed-point sum x^2 (stats)
  double* seg_obj;          // [tasks] FP64 objective partial per (CTA, instance) segment (stats)
  float* xout;              // caller-order x or nullptr (stats)
  float scaleG, scaleC, scaleQ;
  float z;
  int32_t J;
  int32_t kind;
};

// A task: users [u0, u1) of instance `inst`, all of one degree class, laid
// on lanes by mapping `map`.  The tasks of one CTA are contiguous and sorted
// by instance.
struct Task {
  int32_t inst;
  int32_t map;
  int32_t u0;
  int32_t u1;
};

struct SweepLaunch {
  const InstDesc* inst;     // device table
  const Task* tasks;        // device
  const int32_t* cta_task;  // device [grid + 1]
  int32_t grid;
  int32_t smemJ;            // item capacity of the shared arrays
  cudaStream_t stream;
};

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
  float* grad_out;            // optional [J]
  double* out;                // [8]: g, P, rel_gap, uncert_gap, max_viol, obj, iter, status
  const DevState* state;
  int32_t certified;          // 0: scaled point not certified (EQ simplex or a < 0)
};

// ---- launchers (defined in the .cu files) ----
size_t sweep_smem_bytes(int smemJ, bool stats, bool bf16);
size_t sweep_smem_limit();  // usable dynamic shared memory per sweep CTA on this device
cudaError_t sweep_prepare(bool bf16);  // raises the dynamic shared-memory limit
int sweep_occupancy(int smemJ, bool stats, bool bf16);
cudaError_t launch_sweep(const SweepLaunch& L, bool stats, bool bf16);
cudaError_t launch_update(const UpdInst* dev_tab, int ninst, cudaStream_t s);
cudaError_t launch_stats(const StatsInst* dev_tab, int ninst, cudaStream_t s);

// layout.cu
struct LayoutOut {
  int64_t* rp = nullptr;        // [I+1]
  int32_t* col = nullptr;       // [nnz]
  void* c = nullptr;            // [nnz]
  void* a = nullptr;            // [nnz]
  int64_t* orig_off = nullptr;  // [I]
  int64_t class_count[kNumClasses] = {0};
  int64_t class_begin[kNumClasses + 1] = {0};
  double* n2 = nullptr;         // [J] sum_i a_ij^2
  double n2max = 0;
  int64_t max_item_deg = 0;
  double max_abs_a = 0, max_abs_c = 0;
  bool a_nonneg = true;
};
// Validates and lays out one instance; all pointers are device pointers.
// Returns DLM_OK or an error with `msg` set.
dlm_status build_layout(int64_t I, int64_t J, int64_t nnz, const int64_t* rp, const int32_t* col, const void* c,
                        const void* a, const double* b, bool bf16, cudaStream_t s, LayoutOut* out, std::string* msg);

}  // namespace dlm
