// Instantiation of the force pipelines for float (separate unit for build parallelism).
#include "pd_force_impl.cuh"

namespace pd {
template pd_status weight_gfield<float>(pd_plan *, const float *, const uint8_t *, float *, cudaStream_t);
template pd_status force_any<float>(pd_plan *, const float *, const float *, const uint8_t *, const float *, float *, float *,
                                   cudaStream_t);
template pd_status force_plain<float>(pd_plan *, const float *, const float *, float *, float *, cudaStream_t);
template pd_status force_public<float>(pd_plan *, const float *, const float *, float *, float *, cudaStream_t);
}  // namespace pd
