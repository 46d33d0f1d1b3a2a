// Instantiation of the force pipelines for double (separate unit for build parallelism).
#include "pd_force_impl.cuh"

namespace pd {
template pd_status weight_gfield<double>(pd_plan *, const double *, const uint8_t *, double *, cudaStream_t);
template pd_status force_any<double>(pd_plan *, const double *, const double *, const uint8_t *, const double *, double *, double *,
                                   cudaStream_t);
template pd_status force_plain<double>(pd_plan *, const double *, const double *, double *, double *, cudaStream_t);
template pd_status force_public<double>(pd_plan *, const double *, const double *, double *, double *, cudaStream_t);
}  // namespace pd
