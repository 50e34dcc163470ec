// backward.cu -- adjoint of the tree walk (placeholder until implemented).
#include "tree.cuh"

namespace lens {

lens_status shoot_backward(lens_tree* t, double ox, double oy, const void* dx, const void* dy, int dtype,
                           int64_t n, const void* const g[5], void* const* g_species, void* g_halos,
                           int flags, cudaStream_t s)
{
    (void)t; (void)ox; (void)oy; (void)dx; (void)dy; (void)dtype; (void)n; (void)g; (void)g_species;
    (void)g_halos; (void)flags; (void)s;
    return lens_set_error(LENS_ERR_UNSUPPORTED, "backward walk not built yet");
}

}  // namespace lens
