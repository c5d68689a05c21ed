// handle.h -- the mrnmf_handle object and the helpers the ABI translation
// units share (api.cu, batched.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/mrnmf.h"
#include "internal.h"

struct mrnmf_handle {
    int device = -1;
    int* d_status = nullptr;
    void* ws = nullptr;  // pass state
    size_t ws_bytes = 0;
    void* sws = nullptr;  // small-step workspace
    size_t sws_bytes = 0;
    std::string err = "no error";
    // streaming
    bool open = false;
    int xdtype = MRNMF_F32;
    mrnmf::PassState st;
    // host end-to-end path
    void* xbuf = nullptr;
    size_t xbuf_bytes = 0;
    double* dout = nullptr;
    size_t dout_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
    // instrumentation
    cudaEvent_t prof_start = nullptr, prof_stop = nullptr;
    // rank sweep scratch (r_max * n coefficients)
    void* sweep = nullptr;
    size_t sweep_bytes = 0;
    // batched pass: device descriptors + state, pinned host staging of the descriptors
    void* bws = nullptr;
    size_t bws_bytes = 0;
    void* bstage = nullptr;
    size_t bstage_bytes = 0;
    cudaEvent_t ev_bstage = nullptr;
    // follow-ups (second read of X): per-block partial sums of the full-space residual
    void* fws = nullptr;
    size_t fws_bytes = 0;
    // R-SVD scratch
    void* svd = nullptr;
    size_t svd_bytes = 0;
};

namespace mrnmf {
namespace api {

mrnmf_status fail(mrnmf_handle* h, mrnmf_status s, const std::string& msg);
mrnmf_status cuda_fail(mrnmf_handle* h, cudaError_t e, const char* where);
mrnmf_status bind_device(mrnmf_handle* h);
mrnmf_status grow(mrnmf_handle* h, void** buf, size_t* have, size_t need, const char* what);
mrnmf_status run_pass(mrnmf_handle* h, const void* X, int64_t m, int32_t n, int64_t ldx, int32_t dtype, int32_t prec,
                      int qr, double* R, double* colsum, int32_t k, uint64_t seed, int64_t row_offset, double* GX,
                      cudaStream_t s, int gp_form = 0);

}  // namespace api
}  // namespace mrnmf
