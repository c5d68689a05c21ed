// tsqr_group_wide.cu -- the lane-group leaf (group_leaf.cuh, described in
// tsqr_group.cu) for 17 <= n <= 28: one 32-lane group per warp, two rows a
// lane, the group sums through shared memory.  A translation unit of its own
// so that the widths compile in parallel.  (At n = 32 the warp leaf is faster:
// the unrolled 32-step body and its spills cost more than the layout saves.)
#include "group_leaf.cuh"

namespace mrnmf {

// One case per width n = 17 .. 28: CALL<n>(ARGS).
#define MRNMF_BY_WIDTH(n, CALL, ...)                 \
    switch (n) {                                     \
    case 17: return CALL<17>(__VA_ARGS__);       \
    case 18: return CALL<18>(__VA_ARGS__);       \
    case 19: return CALL<19>(__VA_ARGS__);       \
    case 20: return CALL<20>(__VA_ARGS__);       \
    case 21: return CALL<21>(__VA_ARGS__);       \
    case 22: return CALL<22>(__VA_ARGS__);       \
    case 23: return CALL<23>(__VA_ARGS__);       \
    case 24: return CALL<24>(__VA_ARGS__);       \
    case 25: return CALL<25>(__VA_ARGS__);       \
    case 26: return CALL<26>(__VA_ARGS__);       \
    case 27: return CALL<27>(__VA_ARGS__);       \
    default: return CALL<28>(__VA_ARGS__);       \
    }


cudaError_t group_launch_wide(const LeafArgs& a, int streams, cudaStream_t s)
{
    MRNMF_BY_WIDTH(a.n, launch_group, a, streams, s)
}

int group_ctas_wide(int n) { MRNMF_BY_WIDTH(n, group_ctas, ) }

#undef MRNMF_BY_WIDTH

}  // namespace mrnmf
