// What the batched march (batch.cu) needs of a single plan (api.cu) to run that plan's ordinary
// steps as one branch of the batch's step graph: the large instances of a batch are single plans
// without pair lists (opts.local_weights = 1), stepped concurrently with one another.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/wave1d.h"

namespace wave1d {

struct PlanHooks {
    int64_t M, R, Nt;
    int chunk;            // rows of the receiver and density rings (row = step mod chunk)
    double* rec_hist;     // device, chunk x R receiver values, caller order
    int* status;          // device status word (0, WAVE1D_ENONFINITE, WAVE1D_ENOTCONV)
};
int plan_hooks(wave1d_plan_t p, PlanHooks& out);

// Queue plan p's next ordinary step on its private stream as a branch: the stream waits on event
// fork (recorded on the stream the branches leave), then the step.  plan_branch_join makes stream
// s wait for that step.  Valid inside a capture on the forking stream; fork all branches before
// joining any, so that they run concurrently.  sig_hist: NULL, or the plan's density ring
// (plan_sigma_ring).
int plan_branch_step(wave1d_plan_t p, cudaEvent_t fork, double* sig_hist);
int plan_branch_join(wave1d_plan_t p, cudaStream_t s);

// The plan's chunk x M density ring (caller order), allocated on first use.
int plan_sigma_ring(wave1d_plan_t p, double** out);

// Count k steps taken through plan_branch_step (the host mirror of the device step counter).
void plan_count_steps(wave1d_plan_t p, int64_t k);

}  // namespace wave1d
