// Checkpointed adjoint of the step (placeholder until the transposed kernels land).
#include "lbm_adjoint.h"

namespace lbm {

struct AdjointState {
};

void adjoint_free(AdjointState *a) { delete a; }

lbm_status adjoint_run(lbm_ctx *, int64_t, int32_t, int32_t, double *, double *, double *, std::string &msg)
{
    msg = "adjoint not available in this build";
    return LBM_ENOTSUP;
}

}  // namespace lbm
