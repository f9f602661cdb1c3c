// lbm_trace.hpp -- NVTX ranges around the calls of the C ABI that put work on the GPU
// (lbm_step, lbm_set_fields / lbm_get_fields, lbm_get_diagnostics, the batch, slab and
// adjoint calls), in the NVTX domain "lbm", so that a profiler shows each call's kernels
// under the call's name.  NVTX v3 is header-only: without a profiler attached a range
// costs a test of one function pointer, and nothing is linked.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbm {

inline nvtxDomainHandle_t trace_domain()
{
    static nvtxDomainHandle_t d = nvtxDomainCreateA("lbm");
    return d;
}

// A range from construction to destruction (the scope of one C ABI call).
class TraceRange {
public:
    explicit TraceRange(const char* name)
    {
        nvtxEventAttributes_t a{};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace lbm
