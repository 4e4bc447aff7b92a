// FP32 instantiations of the stage kernels (bulk arithmetic in FP32; tables
// rounded from double-double).
#include <cstring>

#include "dispatch.cuh"

namespace gpweno {

gpweno_status launch_stage_f32(gpweno_plan p, const StageIO &io, cudaStream_t st)
{
    if (p->opts.beta_mean) return launch_stage_f32_mean(p, io, st);
    return launch_stage_T<float, false>(p, io, st);
}

gpweno_status launch_max_rate_f32(gpweno_plan p, const void *U, cudaStream_t st)
{
    return launch_max_rate_T<float>(p, U, st);
}

}  // namespace gpweno
