// Read-only view of a plan for entry points implemented outside the plan's own file.
#pragma once
#include "lr_internal.h"

namespace lr {

struct PlanView {
    FwdParams base;  // launch parameters prepared at plan creation
    int precision, order, threads, sms, device;
};

int plan_view(const lr_plan *plan, PlanView *v);
// records a failing cudaError_t in the plan's context and returns LR_ERR_CUDA
int plan_cuda_fail(lr_plan *plan, int cuda_error);

}  // namespace lr
