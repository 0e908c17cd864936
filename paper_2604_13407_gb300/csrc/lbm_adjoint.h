// Adjoint driver interface (checkpointed backward pass of the step).
#pragma once

#include <string>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm {

struct AdjointState;  // device buffers owned by the adjoint driver

// What the adjoint driver may see of a context.
struct ContextView {
    const lbm_params *p;
    KParams *kp;
    cudaStream_t stream;
    void **pops;
    float **refp;
    int *cur;
    int64_t *steps;
    size_t elem;
    int64_t plane;
    AdjointState **adj;
    lbm_status (*run_steps)(lbm_ctx *, int64_t);
    uint32_t (*sr_seed)(int64_t step);  // seed of the storage's stochastic rounding at a step
    void (*bind)(lbm_ctx *, int);
    cudaError_t (*psi_pass)(const KParams &, cudaStream_t);
    cudaError_t (*collide_pass)(const KParams &, cudaStream_t);
    // the one-pass step when the context steps with it and it can write the psi field of the
    // state it reads (FP32 arithmetic); null otherwise
    cudaError_t (*fused_pass)(const KParams &, cudaStream_t);
    const Launchers *L;
    lbm_status (*check_error)(lbm_ctx *, std::string &msg);  // device error word of the steps
    int64_t n_fluid;
    lbm_ctx *ctx;
};

ContextView view_of(lbm_ctx *c);
void adjoint_free(AdjointState *a);
lbm_status adjoint_run(lbm_ctx *c, int64_t nsteps, int32_t checkpoint_every, int32_t objective, double *J,
                       double grad[4], double *lambda0, std::string &msg);

}  // namespace lbm
