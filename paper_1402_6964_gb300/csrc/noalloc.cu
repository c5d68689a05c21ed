// noalloc.cu -- mrnmf_tsqr_r_noalloc: the R / column-sum pass for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// host callback or a custom allocator hook, under a memory pool that the
// embedding application owns outright, or in a process that must not grow its
// device footprint after start-up.  Such callers can still pass their own
// input and output buffers; what they cannot provide is the pass's scratch
// (one n-by-n triangle per row stream, the tree's ping-pong buffer, the
// partial column sums and a status word).  Here that scratch is a file-scope
// __device__ array of fixed size, so no call allocates anything: no
// cudaMalloc, no cudaFree, no allocating library routine.
//
// Costs and rules (also stated in include/mrnmf.h):
//  - every GPU that loads this library holds kNoAllocScratchBytes (32 MiB)
//    for the array until the process exits;
//  - all calls share the one array per device, so calls that overlap on the
//    GPU (different streams, or different host threads) race on it and give
//    wrong results: serialise them;
//  - the array keeps the last call's contents; each call clears the parts
//    that must start at zero before its kernels read them;
//  - the first call on each device resolves the array's device address with
//    cudaGetSymbolAddress (the host-side name is only a stand-in for it), so
//    make that first call before any stream capture; the address is cached
//    per device for the life of the process, so after a cudaDeviceReset the
//    entry point must not be called again in that process;
//  - the caller must pass a status word: device-side errors (a negative or
//    NaN entry of X) are reported there and nowhere else.

#include <mutex>

#include "../../include/mrnmf.h"
#include "internal.h"
#include "leaf.h"
#include "trace.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr size_t kStatePad = 256;  // the pass state starts 256 bytes into the array
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (resolved once per device).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" mrnmf_status mrnmf_tsqr_r_noalloc(const float* X, int64_t m, int32_t n, int64_t ldx, double* R,
                                             double* colsum, int32_t* status, void* stream)
{
    MRNMF_TRACE("mrnmf_tsqr_r_noalloc");
    if (!X || !R || !status) return MRNMF_ERR_INVALID_ARG;
    if (n < 1 || n > MRNMF_NMAX || m < n || ldx < n) return MRNMF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return MRNMF_ERR_CUDA;

    mrnmf::PassState st;
    st.n = n;
    st.k = 0;
    st.fp64 = 0;
    st.tc = 0;
    // The usual stream count, or the largest one whose state fits the array
    // (the state grows with P), kept a multiple of the warp leaf's streams per
    // CTA where that leaf serves n so that the pass does not change kernels.
    const int P0 = mrnmf::choose_streams(n, 0, 0, 0, m);
    const size_t avail = kNoAllocScratchBytes - kStatePad;
    int lo = 1, hi = P0;
    if (mrnmf::pass_state_bytes(n, 0, 1, 0) > avail) return MRNMF_ERR_INVALID_ARG;
    while (lo < hi) {  // largest P in [1, P0] with pass_state_bytes(P) <= avail
        const int mid = lo + (hi - lo + 1) / 2;
        if (mrnmf::pass_state_bytes(n, 0, mid, 0) <= avail) lo = mid;
        else hi = mid - 1;
    }
    st.P = lo;
    const int w = mrnmf::warp_leaf_warps_per_cta();
    if (st.P < P0 && mrnmf::warp_leaf_supported(n, 0) && st.P >= w) st.P -= st.P % w;
    mrnmf::pass_state_carve(st, static_cast<unsigned char*>(base) + kStatePad);

    int* word = reinterpret_cast<int*>(status);
    if (cudaMemsetAsync(word, 0, sizeof(int), s) != cudaSuccess) return MRNMF_ERR_CUDA;
    if (mrnmf::pass_reset(st, s) != cudaSuccess) return MRNMF_ERR_CUDA;
    if (mrnmf::pass_push(st, X, m, ldx, 0, 1, word, s) != cudaSuccess) return MRNMF_ERR_CUDA;
    if (mrnmf::pass_finish(st, 1, R, colsum, nullptr, word, s) != cudaSuccess) return MRNMF_ERR_CUDA;
    return MRNMF_OK;
}
