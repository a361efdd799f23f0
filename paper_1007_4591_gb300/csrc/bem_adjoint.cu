// Transposed operator and adjoint gradients (spec differentiation).
#include "bem_internal.cuh"

namespace bem {

void matvec_t_sorted(Mesh &m, const double *xs, double *ys) {
    (void)m; (void)xs; (void)ys;
    throw Error(BEM_EUNSUPPORTED, "transposed operator not built yet");
}

void adjoint_gradients(Mesh &m, double grad_out, double *dq_s, double *dx_s) {
    (void)m; (void)grad_out; (void)dq_s; (void)dx_s;
    throw Error(BEM_EUNSUPPORTED, "adjoint gradients not built yet");
}

}  // namespace bem
