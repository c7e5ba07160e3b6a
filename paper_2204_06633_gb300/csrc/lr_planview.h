// Read-only view of a plan for entry points implemented outside the plan's own file.
#pragma once
#include <cuda_runtime.h>

#include "lr_internal.h"

namespace lr {

struct PlanView {
    FwdParams base;  // launch parameters prepared at plan creation
    int precision, order, threads, sms, device;
};

int plan_view(const lr_plan *plan, PlanView *v);
// sets the plan's tile (output samples per CTA) and the window capacities derived from it
int plan_set_tile(lr_plan *plan, int tile);
// makes sure the plan's batch tables hold S sources (may allocate): the tile table (S+1
// entries) and the sources' sky frames
int plan_reserve_batch(lr_plan *plan, int64_t S);
// the plan's batch sky-frame table (valid after plan_reserve_batch)
SkyConst *plan_sky_table(lr_plan *plan);
// every device allocation of the library (honours lr_debug_fail_allocations)
cudaError_t dev_malloc(void **p, size_t bytes);
// records a failing cudaError_t in the plan's context and returns LR_ERR_CUDA
int plan_cuda_fail(lr_plan *plan, int cuda_error);
// looks up the allocation-free entry point's fixed device arrays on `device` (current); returns a
// cudaError_t value
int noalloc_setup(int device);

}  // namespace lr
