// FP32 instantiations of the stage kernels (bulk arithmetic in FP32; tables
// rounded from double-double).
#include <cstring>

#include "dispatch.cuh"

namespace gpweno {

gpweno_status launch_stage_f32(gpweno_plan p, const StageIO &io, cudaStream_t st)
{
    const int var = (p->opts.beta_mean ? kVarMean : 0) | (p->opts.scheme ? kVarFdFlux : 0) | (p->opts.ao ? kVarAo : 0) |
                    (has_external_side(p) ? kVarSlab : 0);
    switch (var) {
    case kVarSlab: return launch_stage_f32_var8(p, io, st);
    case kVarMean: return launch_stage_f32_var1(p, io, st);
    case kVarFdFlux: return launch_stage_f32_var2(p, io, st);
    case kVarFdFlux | kVarMean: return launch_stage_f32_var3(p, io, st);
    case kVarAo: return launch_stage_f32_var4(p, io, st);
    case kVarAo | kVarMean: return launch_stage_f32_var5(p, io, st);
    default: return launch_stage_T<float, 0>(p, io, st);
    }
}

gpweno_status launch_max_rate_f32(gpweno_plan p, const void *U, cudaStream_t st)
{
    return launch_max_rate_T<float>(p, U, st);
}

}  // namespace gpweno
