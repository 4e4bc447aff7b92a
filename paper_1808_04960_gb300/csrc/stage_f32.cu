// FP32 instantiations of the stage kernels (bulk arithmetic in FP32; tables
// rounded from double-double).
#include <cstring>

#include "dispatch.cuh"

namespace gpweno {

gpweno_status launch_stage_f32(gpweno_plan p, const void *U, const void *U0, void *out, double a0, double b, int mode,
                               double dt, const double *dt_dev, bool want_rate, cudaStream_t st)
{
    return launch_stage_T<float>(p, U, U0, out, a0, b, mode, dt, dt_dev, want_rate, st);
}

gpweno_status launch_max_rate_f32(gpweno_plan p, const void *U, cudaStream_t st)
{
    return launch_max_rate_T<float>(p, U, st);
}

}  // namespace gpweno
