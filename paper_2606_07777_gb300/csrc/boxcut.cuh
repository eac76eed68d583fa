// boxcut.cuh -- the sweep for handles whose simple set is the box cut by one
// budget, C_i = {0 <= x_ij <= z, sum_j x_ij <= cut} (sweep_boxcut.cu).
#pragma once

#include "dlm_impl.cuh"

namespace dlm {

// One sweep (iteration or certificate) over the box-cut instances of L's
// task table; certificate sweeps take item windows like the one-family
// sweep.  cuts (device, one per instance of the table) are the per-user
// budgets, each > 0.
cudaError_t launch_sweep_boxcut(const SweepLaunch& L, bool stats, bool bf16, const double* cuts);
cudaError_t sweep_boxcut_prepare(bool bf16);

}  // namespace dlm
