// ORAS preconditioner (Eq. oras, Eq. 2lvl): placeholder entry points until the
// local factorisation kernels land.
#include "internal.h"

extern "C" helm_status oras_factor(helm_grid g, const helm_oras_desc*, helm_oras* out) {
    if (out) *out = nullptr;
    return set_error(g ? g->ctx : nullptr, HELM_EINVAL, "oras_factor: not built yet");
}
extern "C" void oras_destroy(helm_oras) {}
extern "C" helm_status oras_apply(helm_oras, const void*, void*, int) { return HELM_EINVAL; }
extern "C" helm_status oras_box_info(helm_oras, int, int*, int*, int*) { return HELM_EINVAL; }
extern "C" helm_status oras_plane_inverse(helm_oras, int, int, void*) { return HELM_EINVAL; }
extern "C" double oras_setup_seconds(helm_oras) { return 0.0; }
extern "C" helm_status gmres_solve(helm_oras, const void*, void*, int, const helm_gmres_desc*, helm_rhs_stats*) {
    return HELM_EINVAL;
}
