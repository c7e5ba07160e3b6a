// Host-buffer pipeline of lr_response_batched_host: its per-plan workspace (device slots, pinned
// staging, streams, events), created on first use and freed with the plan.
#pragma once
#include "lr_internal.h"

namespace lr {
struct PipeWork;
void pipe_free(PipeWork *w);
// the plan's pipeline workspace (null until the first call)
PipeWork *&plan_pipe(lr_plan *plan);
}  // namespace lr
