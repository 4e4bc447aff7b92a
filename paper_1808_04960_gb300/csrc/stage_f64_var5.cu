// FP64 instantiations of the stage kernels for GP-AO with the non-zero-mean smoothness indicators;
// a translation unit of its own so that it compiles in parallel with the others.
#include <cstring>

#include "dispatch.cuh"

namespace gpweno {

gpweno_status launch_stage_f64_var5(gpweno_plan p, const StageIO &io, cudaStream_t st)
{
    return launch_stage_T<double, 5>(p, io, st);
}

}  // namespace gpweno
