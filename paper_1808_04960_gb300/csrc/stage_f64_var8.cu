// FP64 instantiations of the stage kernels for grids with an external (halo) side,
// the slabs of a decomposed grid; a translation unit of its own so that it
// compiles in parallel with the others.
#include <cstring>

#include "dispatch.cuh"

namespace gpweno {

gpweno_status launch_stage_f64_var8(gpweno_plan p, const StageIO &io, cudaStream_t st)
{
    return launch_stage_T<double, kVarSlab>(p, io, st);
}

}  // namespace gpweno
