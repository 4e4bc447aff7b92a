// FP64 instantiations of the stage kernels (all arithmetic in FP64; tables
// rounded from double-double).
#include <cstring>

#include "dispatch.cuh"

namespace gpweno {

gpweno_status launch_stage_f64(gpweno_plan p, const StageIO &io, cudaStream_t st)
{
    if (p->opts.beta_mean) return launch_stage_f64_mean(p, io, st);
    return launch_stage_T<double, false>(p, io, st);
}

gpweno_status launch_max_rate_f64(gpweno_plan p, const void *U, cudaStream_t st)
{
    return launch_max_rate_T<double>(p, U, st);
}

}  // namespace gpweno
