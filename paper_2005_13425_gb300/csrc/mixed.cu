// Mixed-precision defect correction (placeholder).
#include "internal.cuh"

namespace nekgb {

nb_status prepare_fp32(nb_ctx *) { return NB_OK; }

nb_status cg_solve_mixed(nb_ctx *, const double *, double *, double, int, int *, double *) {
    return fail(NB_ERR_STATE, "mixed precision solve is not available yet");
}

}  // namespace nekgb
