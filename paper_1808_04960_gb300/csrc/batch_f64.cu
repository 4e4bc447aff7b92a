// FP64 instantiations of the batched persistent stage kernel.
#include "batch_host.cuh"

namespace gpweno {

gpweno_status build_batch_f64(gpweno_plan batch) { return build_batch_T<double>(batch); }

gpweno_status launch_batch_stage_f64(gpweno_plan batch, int stage, void *const *U, void *const *scratch,
                                     const double *dt_dev, cudaStream_t st)
{
    return launch_batch_stage_T<double>(batch, stage, U, scratch, dt_dev, st);
}

}  // namespace gpweno
