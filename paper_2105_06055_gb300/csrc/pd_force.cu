// pd_force entry point; the pipelines are instantiated in pd_force_f32.cu / pd_force_f64.cu.
#include "pd_ops.cuh"

namespace pd {
template <typename T>
pd_status force_public(pd_plan *p, const T *u, const T *s, T *L, T *W, cudaStream_t st);
template <typename T>
pd_status force_nl(pd_plan *p, const T *u, T *L, cudaStream_t st);
}  // namespace pd

using namespace pd;

extern "C" pd_status pd_force(pd_plan *p, const void *u, const void *s, void *L, void *W, void *stream)
{
    if (!p || !u || !L) {
        set_error("pd_force: null plan, u or L");
        return PD_ERR_ARG;
    }
    if (u == L) {
        set_error("pd_force: u and L must not overlap");
        return PD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (p->nonlinear) {
        if (s || W) {
            set_error("pd_force: the nonlinear bond model takes no node weight and no energy output");
            return PD_ERR_ARG;
        }
        if (p->prob.fp64) return force_nl<double>(p, (const double *)u, (double *)L, st);
        return force_nl<float>(p, (const float *)u, (float *)L, st);
    }
    if (p->prob.fp64)
        return force_public<double>(p, (const double *)u, (const double *)s, (double *)L, (double *)W, st);
    return force_public<float>(p, (const float *)u, (const float *)s, (float *)L, (float *)W, st);
}
