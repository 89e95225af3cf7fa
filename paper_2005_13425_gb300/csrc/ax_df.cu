// Double-float (FP32-pair) ax_e: placeholder until the kernel lands; the
// dispatcher falls back to the native FP64 kernel while df_supported() is
// false.
#include "internal.cuh"

namespace nekgb {

bool df_supported(int) { return false; }

nb_status launch_ax_df(nb_ctx *c, const double *, double *, int) {
    return fail(NB_ERR_STATE, "double-float ax_e is not available");
}

nb_status prepare_df(nb_ctx *) { return NB_OK; }

}  // namespace nekgb
