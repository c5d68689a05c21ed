// trace.h -- NVTX ranges around the C ABI's entry points, so that profilers
// (nsys, ncu --nvtx) can attribute kernels to the call that launched them.
// Without an attached tool NVTX calls are cheap no-ops; without the NVTX
// headers the ranges compile away.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define MRNMF_HAVE_NVTX 1
#endif
#endif

namespace mrnmf {

struct TraceRange {
    explicit TraceRange(const char* name)
    {
#ifdef MRNMF_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~TraceRange()
    {
#ifdef MRNMF_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace mrnmf

#define MRNMF_TRACE(name) ::mrnmf::TraceRange mrnmf_trace_range_(name)
