// FP32 instantiations of the batched persistent stage kernel.
#include "batch_host.cuh"

namespace gpweno {

gpweno_status build_batch_f32(gpweno_plan batch) { return build_batch_T<float>(batch); }

gpweno_status launch_batch_stage_f32(gpweno_plan batch, int stage, void *const *U, void *const *scratch,
                                     const double *dt_dev, cudaStream_t st)
{
    return launch_batch_stage_T<float>(batch, stage, U, scratch, dt_dev, st);
}

}  // namespace gpweno
