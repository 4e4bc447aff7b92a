// FP32 instantiations of the stage kernels with the non-zero-mean smoothness
// indicators (beta on f - f_centre); a translation unit of their own so that
// they compile in parallel with the default kernels.
#include <cstring>

#include "dispatch.cuh"

namespace gpweno {

gpweno_status launch_stage_f32_mean(gpweno_plan p, const StageIO &io, cudaStream_t st)
{
    return launch_stage_T<float, true>(p, io, st);
}

}  // namespace gpweno
