// api.cu -- the extern "C" entry points of include/mrnmf.h.
//
// Argument checking, the handle's device workspace, stream ordering, and the
// composition of the pass kernels (tsqr_simt.cu, tsqr_warp.cu, tsqr_pipe.cu, tsqr_wy.cu) and the n-by-n
// step kernels (small_step.cu).  No entry point computes on the host.

#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/mrnmf.h"
#include "internal.h"
#include "trace.h"
#include "handle.h"
#include "leaf.h"




namespace mrnmf {
namespace api {

mrnmf_status fail(mrnmf_handle* h, mrnmf_status s, const std::string& msg)
{
    if (h) h->err = msg;
    return s;
}

mrnmf_status cuda_fail(mrnmf_handle* h, cudaError_t e, const char* where)
{
    // consume the runtime's record of a non-sticky error, so that it is not
    // reported again by the next cudaGetLastError of a later, unrelated call
    (void)cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? MRNMF_ERR_NO_MEMORY : MRNMF_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

mrnmf_status bind_device(mrnmf_handle* h)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
    if (h->device < 0) {
        h->device = dev;
        e = cudaMalloc(&h->d_status, 256);
        if (e != cudaSuccess) return cuda_fail(h, e, "status word");
        e = cudaMemset(h->d_status, 0, 256);
        if (e != cudaSuccess) return cuda_fail(h, e, "status word");
    } else if (h->device != dev) {
        return fail(h, MRNMF_ERR_INVALID_ARG, "handle is bound to device " + std::to_string(h->device) +
                                                  " but device " + std::to_string(dev) + " is current");
    }
    return MRNMF_OK;
}

mrnmf_status grow(mrnmf_handle* h, void** buf, size_t* have, size_t need, const char* what)
{
    if (need <= *have) return MRNMF_OK;
    if (*buf) {
        cudaError_t e = cudaFree(*buf);  // synchronises with work that may still use it
        *buf = nullptr;
        *have = 0;
        if (e != cudaSuccess) return cuda_fail(h, e, what);
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    *have = need;
    return MRNMF_OK;
}

int resolve_prec(int prec, int dtype, int n, int k)
{
    if (prec == MRNMF_PREC_AUTO) {
        if (dtype == MRNMF_F64) return MRNMF_PREC_FP64;
        return mrnmf::tc_preferred(n, k) ? MRNMF_PREC_TF32X3 : MRNMF_PREC_FP32;
    }
    return prec;
}

mrnmf_status check_pass_args(mrnmf_handle* h, const void* X, int64_t m, int32_t n, int64_t ldx, int32_t dtype,
                             int32_t prec, int32_t k)
{
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!X) return fail(h, MRNMF_ERR_INVALID_ARG, "X is NULL");
    if (n < 1 || n > MRNMF_NMAX) return fail(h, MRNMF_ERR_INVALID_ARG, "n must be in [1, 256]");
    if (m < n) return fail(h, MRNMF_ERR_INVALID_ARG, "need m >= n (tall-and-skinny X)");
    if (ldx < n) return fail(h, MRNMF_ERR_INVALID_ARG, "ldx < n");
    if (dtype != MRNMF_F32 && dtype != MRNMF_F64) return fail(h, MRNMF_ERR_INVALID_ARG, "dtype must be F32 or F64");
    if (prec < MRNMF_PREC_AUTO || prec > MRNMF_PREC_TF32 || prec == MRNMF_PREC_BF16)
        return fail(h, MRNMF_ERR_INVALID_ARG, "bad prec");
    if (k < 0 || k > MRNMF_KMAX) return fail(h, MRNMF_ERR_INVALID_ARG, "k must be in [0, 64]");
    return MRNMF_OK;
}

// Set up h->st for a pass: precision, stream count, workspace.
// qr = 0 is a projection-only pass; gp_form names its tensor-core form (0: SIMT).
mrnmf_status setup_pass(mrnmf_handle* h, int n, int dtype, int prec, int k, uint64_t seed, int64_t m_hint, int qr = 1,
                        int gp_form = 0)
{
    prec = resolve_prec(prec, dtype, n, k);
    if (prec == MRNMF_PREC_FP32 && dtype == MRNMF_F64)
        return fail(h, MRNMF_ERR_INVALID_ARG, "FP32 pass needs F32 input (the library never narrows X)");
    if ((prec == MRNMF_PREC_TF32X3 || prec == MRNMF_PREC_TF32) && (dtype != MRNMF_F32 || !mrnmf::tc_supported(n, k)))
        return fail(h, MRNMF_ERR_INVALID_ARG, "TF32X3 / TF32 pass needs F32 input and a supported n");
    mrnmf::PassState st;
    st.n = n;
    st.k = k;
    st.fp64 = prec == MRNMF_PREC_FP64;
    st.tc = prec == MRNMF_PREC_TF32X3 ? 1 : (prec == MRNMF_PREC_TF32 ? 2 : 0);
    st.tree64 = !st.fp64 && mrnmf::tree64_requested() && mrnmf::tree64_supported(n);
    st.seed = seed;
    st.rows_seen = 0;
    const bool gp_warp = !qr && !st.fp64 && dtype == MRNMF_F32 && k > 0 && mrnmf::gp_pass_form(gp_form) == 0 &&
                         mrnmf::gp_warp_supported(n, k);
    st.P = gp_warp ? mrnmf::gp_warp_streams(n, k, m_hint) : mrnmf::choose_streams(n, k, st.fp64, st.tc, m_hint);
    mrnmf_status s = grow(h, &h->ws, &h->ws_bytes, mrnmf::pass_state_bytes(n, k, st.P, st.fp64), "pass workspace");
    if (s != MRNMF_OK) return s;
    mrnmf::pass_state_carve(st, h->ws);
    st.ev_leaf_start = h->prof_start;
    st.ev_leaf_stop = h->prof_stop;
    h->st = st;
    return MRNMF_OK;
}

mrnmf_status run_pass(mrnmf_handle* h, const void* X, int64_t m, int32_t n, int64_t ldx, int32_t dtype, int32_t prec,
                      int qr, double* R, double* colsum, int32_t k, uint64_t seed, int64_t row_offset, double* GX,
                      cudaStream_t s, int gp_form)
{
    mrnmf_status st = setup_pass(h, n, dtype, prec, k, seed, m, qr, gp_form);
    if (st != MRNMF_OK) return st;
    h->st.rows_seen = row_offset;
    h->st.gp_form = gp_form;
    cudaError_t e = mrnmf::pass_reset(h->st, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "pass reset");
    e = mrnmf::pass_push(h->st, X, m, ldx, dtype == MRNMF_F64, qr, h->d_status, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "pass");
    e = mrnmf::pass_finish(h->st, qr, R, colsum, GX, h->d_status, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "tree / finalize");
    return MRNMF_OK;
}

}  // namespace api
}  // namespace mrnmf

using namespace mrnmf::api;

extern "C" {

mrnmf_status mrnmf_create(mrnmf_handle** handle)
{
    if (!handle) return MRNMF_ERR_INVALID_ARG;
    *handle = new (std::nothrow) mrnmf_handle();
    return *handle ? MRNMF_OK : MRNMF_ERR_NO_MEMORY;
}

void mrnmf_destroy(mrnmf_handle* h)
{
    if (!h) return;
    if (h->device >= 0) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(h->device);
        cudaDeviceSynchronize();
        cudaFree(h->d_status);
        cudaFree(h->ws);
        cudaFree(h->sws);
        cudaFree(h->xbuf);
        cudaFree(h->dout);
        cudaFree(h->sweep);
        cudaFree(h->bws);
        cudaFree(h->fws);
        cudaFree(h->svd);
        if (h->bstage) cudaFreeHost(h->bstage);
        if (h->ev_bstage) cudaEventDestroy(h->ev_bstage);
        for (int i = 0; i < 2; ++i) {
            if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
            if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
        }
        if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
        cudaSetDevice(cur);
    }
    delete h;
}

const char* mrnmf_last_error_string(const mrnmf_handle* h)
{
    return h ? h->err.c_str() : "NULL handle";
}

mrnmf_status mrnmf_sync_status(mrnmf_handle* h, void* stream)
{
    MRNMF_TRACE("mrnmf_sync_status");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (h->device < 0) return MRNMF_OK;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "stream");
    int code = 0;
    e = cudaMemcpy(&code, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (code != 0) {
        e = cudaMemset(h->d_status, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(h, e, "status reset");
        const char* what = code == MRNMF_ERR_BAD_INPUT        ? "input has a negative or NaN entry, or a zero column"
                           : code == MRNMF_ERR_NOT_CONVERGED  ? "NNLS did not converge"
                           : code == MRNMF_ERR_RANK_DEFICIENT ? "R(:,K) is singular or too few GP candidates"
                           : code == MRNMF_ERR_TIMEOUT        ? "a bounded device wait timed out"
                                                              : "device error";
        return fail(h, (mrnmf_status)code, what);
    }
    return MRNMF_OK;
}

mrnmf_status mrnmf_tsqr_r(mrnmf_handle* h, const void* X, int64_t m, int32_t n, int64_t ldx, int32_t dtype,
                          int32_t prec, double* R, double* colsum, void* stream)
{
    MRNMF_TRACE("mrnmf_tsqr_r");
    mrnmf_status s = check_pass_args(h, X, m, n, ldx, dtype, prec, 0);
    if (s != MRNMF_OK) return s;
    if (!R) return fail(h, MRNMF_ERR_INVALID_ARG, "R is NULL");
    if ((s = bind_device(h)) != MRNMF_OK) return s;
    return run_pass(h, X, m, n, ldx, dtype, prec, 1, R, colsum, 0, 0, 0, nullptr, static_cast<cudaStream_t>(stream));
}

mrnmf_status mrnmf_gauss_project(mrnmf_handle* h, const void* X, int64_t m, int32_t n, int64_t ldx, int32_t dtype,
                                 int32_t k, uint64_t seed, int64_t row_offset, double* GX, double* colsum,
                                 void* stream)
{
    MRNMF_TRACE("mrnmf_gauss_project");
    mrnmf_status s = check_pass_args(h, X, m, n, ldx, dtype, MRNMF_PREC_AUTO, k);
    if (s != MRNMF_OK) return s;
    if (k < 1 || !GX) return fail(h, MRNMF_ERR_INVALID_ARG, "need k >= 1 and GX");
    if (row_offset < 0) return fail(h, MRNMF_ERR_INVALID_ARG, "row_offset < 0");
    if ((s = bind_device(h)) != MRNMF_OK) return s;
    const int prec = dtype == MRNMF_F64 ? MRNMF_PREC_FP64 : MRNMF_PREC_FP32;
    return run_pass(h, X, m, n, ldx, dtype, prec, 0, nullptr, colsum, k, seed, row_offset, GX,
                    static_cast<cudaStream_t>(stream));
}

mrnmf_status mrnmf_gauss_project_tc(mrnmf_handle* h, const float* X, int64_t m, int32_t n, int64_t ldx, int32_t k,
                                    uint64_t seed, int64_t row_offset, int32_t form, double* GX, double* colsum,
                                    void* stream)
{
    MRNMF_TRACE("mrnmf_gauss_project_tc");
    mrnmf_status s = check_pass_args(h, X, m, n, ldx, MRNMF_F32, MRNMF_PREC_AUTO, k);
    if (s != MRNMF_OK) return s;
    if (k < 1 || !GX) return fail(h, MRNMF_ERR_INVALID_ARG, "need k >= 1 and GX");
    if (row_offset < 0) return fail(h, MRNMF_ERR_INVALID_ARG, "row_offset < 0");
    if (form != MRNMF_PREC_TF32X3 && form != MRNMF_PREC_BF16)
        return fail(h, MRNMF_ERR_INVALID_ARG, "form must be MRNMF_PREC_TF32X3 or MRNMF_PREC_BF16");
    if (!mrnmf::gp_tc_supported(n, k)) return fail(h, MRNMF_ERR_INVALID_ARG, "tensor-core projection needs n <= 128");
    if ((s = bind_device(h)) != MRNMF_OK) return s;
    return run_pass(h, X, m, n, ldx, MRNMF_F32, MRNMF_PREC_FP32, 0, nullptr, colsum, k, seed, row_offset, GX,
                    static_cast<cudaStream_t>(stream), form);
}

mrnmf_status mrnmf_tsqr_gp(mrnmf_handle* h, const void* X, int64_t m, int32_t n, int64_t ldx, int32_t dtype,
                           int32_t prec, double* R, double* colsum, int32_t k, uint64_t seed, double* GX,
                           void* stream)
{
    MRNMF_TRACE("mrnmf_tsqr_gp");
    mrnmf_status s = check_pass_args(h, X, m, n, ldx, dtype, prec, k);
    if (s != MRNMF_OK) return s;
    if (!R) return fail(h, MRNMF_ERR_INVALID_ARG, "R is NULL");
    if (k > 0 && !GX) return fail(h, MRNMF_ERR_INVALID_ARG, "k > 0 needs GX");
    if ((s = bind_device(h)) != MRNMF_OK) return s;
    return run_pass(h, X, m, n, ldx, dtype, prec, 1, R, colsum, k, seed, 0, k > 0 ? GX : nullptr,
                    static_cast<cudaStream_t>(stream));
}

mrnmf_status mrnmf_select_extreme(mrnmf_handle* h, int32_t method, const double* R, int32_t n, const double* colsum,
                                  const double* GX, int32_t k, int32_t r, int32_t* K, double* gap, void* stream)
{
    MRNMF_TRACE("mrnmf_select_extreme");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (n < 1 || n > MRNMF_NMAX) return fail(h, MRNMF_ERR_INVALID_ARG, "n must be in [1, 256]");
    if (r < 1 || r > n) return fail(h, MRNMF_ERR_INVALID_ARG, "need 1 <= r <= n");
    if (!K) return fail(h, MRNMF_ERR_INVALID_ARG, "K is NULL");
    if (method == MRNMF_SPA) {
        if (!R || !colsum) return fail(h, MRNMF_ERR_INVALID_ARG, "SPA needs R and colsum");
    } else if (method == MRNMF_XRAY) {
        if (!R) return fail(h, MRNMF_ERR_INVALID_ARG, "XRAY needs R");
        if (r > 64) return fail(h, MRNMF_ERR_INVALID_ARG, "XRAY supports r <= 64");
    } else if (method == MRNMF_GP) {
        if (!GX || !colsum || k < 1 || k > MRNMF_KMAX)
            return fail(h, MRNMF_ERR_INVALID_ARG, "GP needs GX, colsum and 1 <= k <= 64");
    } else {
        return fail(h, MRNMF_ERR_INVALID_ARG, "unknown method");
    }
    mrnmf_status s = bind_device(h);
    if (s != MRNMF_OK) return s;
    if ((s = grow(h, &h->sws, &h->sws_bytes, mrnmf::small_ws_bytes(n, k, r), "small-step workspace")) != MRNMF_OK)
        return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (method == MRNMF_SPA) e = mrnmf::select_spa(R, n, colsum, r, K, gap, h->sws, h->d_status, st);
    else if (method == MRNMF_XRAY) e = mrnmf::select_xray(R, n, r, K, gap, h->sws, h->d_status, st);
    else e = mrnmf::select_gp(GX, k, n, colsum, r, K, gap, h->sws, h->d_status, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "select");
    return MRNMF_OK;
}

mrnmf_status mrnmf_nnls_h(mrnmf_handle* h, const double* R, int32_t n, const int32_t* K, int32_t r, double* H,
                          void* stream)
{
    MRNMF_TRACE("mrnmf_nnls_h");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!R || !K || !H) return fail(h, MRNMF_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > MRNMF_NMAX || r < 1 || r > n || r > 64)
        return fail(h, MRNMF_ERR_INVALID_ARG, "need 1 <= r <= min(n, 64), n <= 256");
    mrnmf_status s = bind_device(h);
    if (s != MRNMF_OK) return s;
    if ((s = grow(h, &h->sws, &h->sws_bytes, mrnmf::small_ws_bytes(n, 0, r), "small-step workspace")) != MRNMF_OK)
        return s;
    cudaError_t e = mrnmf::nnls_h(R, n, K, r, H, h->sws, h->d_status, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "nnls");
    return MRNMF_OK;
}

mrnmf_status mrnmf_residual(mrnmf_handle* h, const double* R, int32_t n, const int32_t* K, int32_t r, const double* H,
                            double* out, void* stream)
{
    MRNMF_TRACE("mrnmf_residual");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!R || !K || !H || !out) return fail(h, MRNMF_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > MRNMF_NMAX || r < 1 || r > n) return fail(h, MRNMF_ERR_INVALID_ARG, "need 1 <= r <= n <= 256");
    mrnmf_status s = bind_device(h);
    if (s != MRNMF_OK) return s;
    if ((s = grow(h, &h->sws, &h->sws_bytes, mrnmf::small_ws_bytes(n, 0, r), "small-step workspace")) != MRNMF_OK)
        return s;
    cudaError_t e = mrnmf::residual(R, n, K, r, H, out, h->sws, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "residual");
    return MRNMF_OK;
}

mrnmf_status mrnmf_rank_sweep(mrnmf_handle* h, int32_t method, const double* R, int32_t n, const double* colsum,
                              const double* GX, int32_t k, int32_t r_max, int32_t* K, double* curve, void* stream)
{
    MRNMF_TRACE("mrnmf_rank_sweep");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!R || !K || !curve) return fail(h, MRNMF_ERR_INVALID_ARG, "R, K and curve are required");
    if (n < 1 || n > MRNMF_NMAX || r_max < 1 || r_max > n || r_max > 64)
        return fail(h, MRNMF_ERR_INVALID_ARG, "need 1 <= r_max <= min(n, 64), n <= 256");
    mrnmf_status s = mrnmf_select_extreme(h, method, R, n, colsum, GX, k, r_max, K, nullptr, stream);
    if (s != MRNMF_OK) return s;
    if ((s = grow(h, &h->sweep, &h->sweep_bytes, 8ull * r_max * n, "rank sweep scratch")) != MRNMF_OK) return s;
    double* H = static_cast<double*>(h->sweep);
    for (int r = 1; r <= r_max; ++r) {
        if ((s = mrnmf_nnls_h(h, R, n, K, r, H, stream)) != MRNMF_OK) return s;
        if ((s = mrnmf_residual(h, R, n, K, r, H, curve + 2 * (r - 1), stream)) != MRNMF_OK) return s;
    }
    return MRNMF_OK;
}

mrnmf_status mrnmf_stream_begin(mrnmf_handle* h, int32_t n, int32_t dtype, int32_t prec, int32_t k, uint64_t seed,
                                void* stream)
{
    MRNMF_TRACE("mrnmf_stream_begin");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (n < 1 || n > MRNMF_NMAX) return fail(h, MRNMF_ERR_INVALID_ARG, "n must be in [1, 256]");
    if (dtype != MRNMF_F32 && dtype != MRNMF_F64) return fail(h, MRNMF_ERR_INVALID_ARG, "bad dtype");
    if (prec < MRNMF_PREC_AUTO || prec > MRNMF_PREC_TF32 || prec == MRNMF_PREC_BF16)
        return fail(h, MRNMF_ERR_INVALID_ARG, "bad prec");
    if (k < 0 || k > MRNMF_KMAX) return fail(h, MRNMF_ERR_INVALID_ARG, "k must be in [0, 64]");
    mrnmf_status s = bind_device(h);
    if (s != MRNMF_OK) return s;
    if ((s = setup_pass(h, n, dtype, prec, k, seed, 0)) != MRNMF_OK) return s;
    h->xdtype = dtype;
    cudaError_t e = mrnmf::pass_reset(h->st, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "stream begin");
    h->open = true;
    return MRNMF_OK;
}

mrnmf_status mrnmf_stream_push(mrnmf_handle* h, const void* X_chunk, int64_t rows, int64_t ldx, void* stream)
{
    MRNMF_TRACE("mrnmf_stream_push");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!h->open) return fail(h, MRNMF_ERR_INVALID_ARG, "no open stream (call mrnmf_stream_begin)");
    if (rows < 0 || (rows > 0 && !X_chunk) || ldx < h->st.n) return fail(h, MRNMF_ERR_INVALID_ARG, "bad chunk");
    mrnmf_status s = bind_device(h);
    if (s != MRNMF_OK) return s;
    cudaError_t e = mrnmf::pass_push(h->st, X_chunk, rows, ldx, h->xdtype == MRNMF_F64, 1, h->d_status,
                                     static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "stream push");
    return MRNMF_OK;
}

namespace {

// Serialised streaming state: a header, then the running triangles, the
// partial column sums and the partial projections, as they sit on the device.
struct StreamStateHeader {
    uint64_t magic;
    int32_t n, k, P, fp64, tc, tri, xdtype, reserved;
    uint64_t seed;
    int64_t rows_seen;
    uint64_t r_bytes, cs_bytes, gx_bytes;
};
constexpr uint64_t kStateMagic = 0x3154534D4E524D4Dull;  // "MMRNMST1"

void state_parts(const mrnmf::PassState& st, uint64_t* rb, uint64_t* cb, uint64_t* gb)
{
    *rb = (uint64_t)(st.fp64 ? 8 : 4) * st.P * st.n * st.n;
    *cb = 8ull * st.P * st.n;
    *gb = st.k > 0 ? 8ull * st.P * st.k * st.n : 0;
}

}  // namespace

mrnmf_status mrnmf_stream_state_size(mrnmf_handle* h, size_t* bytes)
{
    if (!h || !bytes) return MRNMF_ERR_INVALID_ARG;
    if (!h->open) return fail(h, MRNMF_ERR_INVALID_ARG, "no open stream");
    uint64_t rb, cb, gb;
    state_parts(h->st, &rb, &cb, &gb);
    *bytes = sizeof(StreamStateHeader) + rb + cb + gb;
    return MRNMF_OK;
}

mrnmf_status mrnmf_stream_state_save(mrnmf_handle* h, void* host, size_t bytes, void* stream)
{
    MRNMF_TRACE("mrnmf_stream_state_save");
    if (!h || !host) return MRNMF_ERR_INVALID_ARG;
    if (!h->open) return fail(h, MRNMF_ERR_INVALID_ARG, "no open stream");
    size_t need = 0;
    mrnmf_status s = mrnmf_stream_state_size(h, &need);
    if (s != MRNMF_OK) return s;
    if (bytes < need) return fail(h, MRNMF_ERR_INVALID_ARG, "state buffer too small");
    if ((s = bind_device(h)) != MRNMF_OK) return s;
    const mrnmf::PassState& st = h->st;
    StreamStateHeader hd{};
    hd.magic = kStateMagic;
    hd.n = st.n;
    hd.k = st.k;
    hd.P = st.P;
    hd.fp64 = st.fp64;
    hd.tc = st.tc;
    hd.tri = st.tri;
    hd.xdtype = h->xdtype;
    hd.seed = st.seed;
    hd.rows_seen = st.rows_seen;
    state_parts(st, &hd.r_bytes, &hd.cs_bytes, &hd.gx_bytes);
    std::memcpy(host, &hd, sizeof(hd));
    char* p = static_cast<char*>(host) + sizeof(hd);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(p, st.R, hd.r_bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + hd.r_bytes, st.cs, hd.cs_bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && hd.gx_bytes)
        e = cudaMemcpyAsync(p + hd.r_bytes + hd.cs_bytes, st.gx, hd.gx_bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    return e == cudaSuccess ? MRNMF_OK : cuda_fail(h, e, "state save");
}

mrnmf_status mrnmf_stream_state_load(mrnmf_handle* h, const void* host, size_t bytes, void* stream)
{
    MRNMF_TRACE("mrnmf_stream_state_load");
    if (!h || !host) return MRNMF_ERR_INVALID_ARG;
    if (!h->open) return fail(h, MRNMF_ERR_INVALID_ARG, "no open stream (begin one with the saved parameters)");
    if (bytes < sizeof(StreamStateHeader)) return fail(h, MRNMF_ERR_INVALID_ARG, "state buffer too small");
    StreamStateHeader hd;
    std::memcpy(&hd, host, sizeof(hd));
    mrnmf::PassState& st = h->st;
    uint64_t rb, cb, gb;
    state_parts(st, &rb, &cb, &gb);
    if (hd.magic != kStateMagic || hd.n != st.n || hd.k != st.k || hd.P != st.P || hd.fp64 != st.fp64 ||
        hd.tc != st.tc || hd.xdtype != h->xdtype || hd.seed != st.seed || hd.r_bytes != rb || hd.cs_bytes != cb ||
        hd.gx_bytes != gb)
        return fail(h, MRNMF_ERR_INVALID_ARG, "saved state does not match the open stream's parameters");
    if (bytes < sizeof(hd) + rb + cb + gb) return fail(h, MRNMF_ERR_INVALID_ARG, "state buffer too small");
    mrnmf_status s = bind_device(h);
    if (s != MRNMF_OK) return s;
    const char* p = static_cast<const char*>(host) + sizeof(hd);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(st.R, p, rb, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st.cs, p + rb, cb, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && gb) e = cudaMemcpyAsync(st.gx, p + rb + cb, gb, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(h, e, "state load");
    st.tri = hd.tri;
    st.rows_seen = hd.rows_seen;
    return MRNMF_OK;
}

mrnmf_status mrnmf_stream_end(mrnmf_handle* h, double* R, double* colsum, double* GX, void* stream)
{
    MRNMF_TRACE("mrnmf_stream_end");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!h->open) return fail(h, MRNMF_ERR_INVALID_ARG, "no open stream");
    if (!R) return fail(h, MRNMF_ERR_INVALID_ARG, "R is NULL");
    if (h->st.rows_seen < h->st.n) return fail(h, MRNMF_ERR_INVALID_ARG, "fewer rows than columns were pushed");
    mrnmf_status s = bind_device(h);
    if (s != MRNMF_OK) return s;
    h->open = false;
    cudaError_t e = mrnmf::pass_finish(h->st, 1, R, colsum, h->st.k > 0 ? GX : nullptr, h->d_status,
                                       static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "stream end");
    return MRNMF_OK;
}

mrnmf_status mrnmf_factorize_host(mrnmf_handle* h, const float* X, int64_t m, int32_t n, int64_t ldx, int32_t prec,
                                  int32_t method, int32_t r, int32_t k, uint64_t seed, int32_t* K, double* H,
                                  double* resid, double* R, void* stream)
{
    MRNMF_TRACE("mrnmf_factorize_host");
    mrnmf_status s = check_pass_args(h, X, m, n, ldx, MRNMF_F32, prec, method == MRNMF_GP ? k : 0);
    if (s != MRNMF_OK) return s;
    if (!K || !H || !resid) return fail(h, MRNMF_ERR_INVALID_ARG, "K, H and resid are required");
    if (r < 1 || r > n || r > 64) return fail(h, MRNMF_ERR_INVALID_ARG, "need 1 <= r <= min(n, 64)");
    if (method < MRNMF_SPA || method > MRNMF_GP) return fail(h, MRNMF_ERR_INVALID_ARG, "unknown method");
    if (method == MRNMF_GP && k < 1) return fail(h, MRNMF_ERR_INVALID_ARG, "GP needs k >= 1");
    if ((s = bind_device(h)) != MRNMF_OK) return s;
    const int kk = method == MRNMF_GP ? k : 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!h->copy_stream) {
        if ((e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(h, e, "copy stream");
        for (int i = 0; i < 2; ++i) {
            if ((e = cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(h, e, "events");
        }
    }
    // two staging buffers of up to MRNMF_STAGE_MB MiB each (default 64)
    static const int64_t stage_mb = [] {
        const char* v = getenv("MRNMF_STAGE_MB");
        const long x = v ? atol(v) : 64;
        return (int64_t)(x >= 1 && x <= 4096 ? x : 64);
    }();
    const int64_t row_bytes = (int64_t)n * 4;
    int64_t chunk = std::max<int64_t>(1, (stage_mb << 20) / row_bytes);
    if (chunk > m) chunk = m;
    if ((s = grow(h, &h->xbuf, &h->xbuf_bytes, 2 * (size_t)chunk * row_bytes, "staging buffers")) != MRNMF_OK)
        return s;
    const size_t nd = (size_t)n * n + n + (size_t)kk * n + (size_t)r * n + 2 + r;
    if ((s = grow(h, (void**)&h->dout, &h->dout_bytes, 8 * nd + 64, "device outputs")) != MRNMF_OK) return s;
    double* dR = h->dout;
    double* dcs = dR + (size_t)n * n;
    double* dGX = dcs + n;
    double* dH = dGX + (size_t)kk * n;
    double* dres = dH + (size_t)r * n;
    int32_t* dK = reinterpret_cast<int32_t*>(dres + 2);

    if ((s = mrnmf_stream_begin(h, n, MRNMF_F32, prec, kk, seed, stream)) != MRNMF_OK) return s;
    // the staging buffers start free: mark them done on the compute stream
    for (int i = 0; i < 2; ++i)
        if ((e = cudaEventRecord(h->ev_done[i], st)) != cudaSuccess) return cuda_fail(h, e, "event");
    char* xb = static_cast<char*>(h->xbuf);
    int q = 0;
    for (int64_t r0 = 0; r0 < m; r0 += chunk, q ^= 1) {
        const int64_t rows = std::min(chunk, m - r0);
        char* dst = xb + (size_t)q * chunk * row_bytes;
        if ((e = cudaStreamWaitEvent(h->copy_stream, h->ev_done[q], 0)) != cudaSuccess) return cuda_fail(h, e, "wait");
        if (ldx == n)
            e = cudaMemcpyAsync(dst, X + r0 * ldx, (size_t)rows * row_bytes, cudaMemcpyHostToDevice, h->copy_stream);
        else
            e = cudaMemcpy2DAsync(dst, row_bytes, X + r0 * ldx, ldx * 4, row_bytes, rows, cudaMemcpyHostToDevice,
                                  h->copy_stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "H2D copy");
        if ((e = cudaEventRecord(h->ev_copied[q], h->copy_stream)) != cudaSuccess) return cuda_fail(h, e, "event");
        if ((e = cudaStreamWaitEvent(st, h->ev_copied[q], 0)) != cudaSuccess) return cuda_fail(h, e, "wait");
        if ((s = mrnmf_stream_push(h, dst, rows, n, stream)) != MRNMF_OK) return s;
        if ((e = cudaEventRecord(h->ev_done[q], st)) != cudaSuccess) return cuda_fail(h, e, "event");
    }
    if ((s = mrnmf_stream_end(h, dR, dcs, kk ? dGX : nullptr, stream)) != MRNMF_OK) return s;
    if ((s = mrnmf_select_extreme(h, method, dR, n, dcs, kk ? dGX : nullptr, kk, r, dK, nullptr, stream)) != MRNMF_OK)
        return s;
    if ((s = mrnmf_nnls_h(h, dR, n, dK, r, dH, stream)) != MRNMF_OK) return s;
    if ((s = mrnmf_residual(h, dR, n, dK, r, dH, dres, stream)) != MRNMF_OK) return s;
    if ((e = cudaMemcpyAsync(K, dK, 4 * (size_t)r, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(H, dH, 8 * (size_t)r * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(resid, dres, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(h, e, "D2H copy");
    if (R && (e = cudaMemcpyAsync(R, dR, 8 * (size_t)n * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(h, e, "D2H copy");
    return mrnmf_sync_status(h, stream);
}

mrnmf_status mrnmf_profile_events(mrnmf_handle* h, void* ev_start, void* ev_stop)
{
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if ((ev_start == nullptr) != (ev_stop == nullptr))
        return fail(h, MRNMF_ERR_INVALID_ARG, "give both events or neither");
    h->prof_start = static_cast<cudaEvent_t>(ev_start);
    h->prof_stop = static_cast<cudaEvent_t>(ev_stop);
    h->st.ev_leaf_start = h->prof_start;
    h->st.ev_leaf_stop = h->prof_stop;
    return MRNMF_OK;
}

uint64_t mrnmf_kernel_launches(void)
{
    return mrnmf::g_launches.load();
}

}  // extern "C"
