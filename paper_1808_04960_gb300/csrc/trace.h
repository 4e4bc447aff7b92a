// NVTX ranges of the library's calls, in the domain "gpweno" (NVTX v3, header
// only: without a profiler attached a range costs one call into a stub).  The
// step functions push one range for the call and one per RK stage, so a
// profiler can select a stage's launches by range, e.g.
//   ncu --nvtx --nvtx-include "gpweno@gpweno_rk3_step/rk3 stage 2/" ...
#pragma once
#include <cstring>

#include <nvtx3/nvToolsExt.h>

namespace gpweno {

inline nvtxDomainHandle_t trace_domain()
{
    static nvtxDomainHandle_t d = nvtxDomainCreateA("gpweno");
    return d;
}

// One range for the lifetime of the object; `name` must outlive it (a literal).
struct TraceRange {
    explicit TraceRange(const char *name)
    {
        nvtxEventAttributes_t e;
        std::memset(&e, 0, sizeof(e));
        e.version = NVTX_VERSION;
        e.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        e.messageType = NVTX_MESSAGE_TYPE_ASCII;
        e.message.ascii = name;
        nvtxDomainRangePushEx(trace_domain(), &e);
    }
    ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

inline const char *stage_range_name(int k)
{
    static const char *const names[3] = {"rk3 stage 1", "rk3 stage 2", "rk3 stage 3"};
    return names[k < 0 ? 0 : (k > 2 ? 2 : k)];
}

}  // namespace gpweno
