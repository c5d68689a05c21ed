// followup.cu -- the two optional follow-ups of the method that read X a
// second time (the method itself needs only the one pass of Sec. 3.5):
//  * W = X(:,K), the left factor of the factorization X ~ X(:,K) H (Sec. 2);
//  * the full-space residual ||X - X(:,K) H||_F and ||.||_F^2 / ||X||_F^2,
//    equal to the reduced residual ||R - R(:,K) H||_F in exact arithmetic
//    (Sec. 2.4), so a check of the reduced computation.
#include <string>

#include "../../include/mrnmf.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"
#include "trace.h"

namespace mrnmf {
namespace {

constexpr int kThreads = 256;
constexpr int kRowsFlush = 32;  // rows between binary64 flushes of a lane's sums

// W(i, a) = X(i, K[a]); an index outside [0, n) is reported and read as column 0.
template <typename T>
__global__ void gather_kernel(const T* __restrict__ X, int64_t m, int n, int64_t ldx, const int32_t* __restrict__ K,
                              int r, T* __restrict__ W, int64_t ldw, int* status)
{
    const int64_t total = m * r;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r;
        const int a = (int)(e - i * r);
        int kc = K[a];
        if (kc < 0 || kc >= n) {
            set_status(status, MRNMF_ERR_INVALID_ARG);
            kc = 0;
        }
        W[i * ldw + a] = X[i * ldx + kc];
    }
}

// One warp per group of kRowsW consecutive rows (grid-stride): lane l holds
// X(i, l + 32 s), s < NS, and forms E(i, c) = X(i, c) - sum_a X(i, K[a]) H(a, c)
// in the input's precision (each H(a, c) read once per group); squares are
// summed per lane, flushed to binary64 every kRowsFlush rows, and reduced per
// block in a fixed order.
constexpr int kRowsW = 4;

template <typename T, int NS>
__global__ void __launch_bounds__(kThreads) full_residual_kernel(const T* __restrict__ X, int64_t m, int n,
                                                                 int64_t ldx, const int32_t* __restrict__ K, int r,
                                                                 const double* __restrict__ H,
                                                                 double* __restrict__ part, int* status)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Hs = reinterpret_cast<T*>(smraw);
    int* Ks = reinterpret_cast<int*>(Hs + (size_t)r * n);
    __shared__ double red[2][kThreads / 32];
    for (int e = threadIdx.x; e < r * n; e += blockDim.x) Hs[e] = (T)H[e];
    for (int a = threadIdx.x; a < r; a += blockDim.x) {
        int kc = K[a];
        if (kc < 0 || kc >= n) {
            set_status(status, MRNMF_ERR_INVALID_ARG);
            kc = 0;
        }
        Ks[a] = kc;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t groups = (m + kRowsW - 1) / kRowsW;
    const int64_t w0 = (int64_t)blockIdx.x * (kThreads / 32) + warp, nw = (int64_t)gridDim.x * (kThreads / 32);
    double e2 = 0.0, x2 = 0.0;
    T ea = 0, xa = 0;
    int cnt = 0;
    for (int64_t gidx = w0; gidx < groups; gidx += nw) {
        const int64_t i0 = gidx * kRowsW;
        T e[kRowsW][NS];
        const T* xr[kRowsW];
#pragma unroll
        for (int q = 0; q < kRowsW; ++q) {
            const bool ok = i0 + q < m;
            xr[q] = X + (ok ? i0 + q : i0) * ldx;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int c = lane + 32 * s;
                e[q][s] = (ok && c < n) ? xr[q][c] : (T)0;
            }
        }
#pragma unroll
        for (int q = 0; q < kRowsW; ++q)
#pragma unroll
            for (int s = 0; s < NS; ++s) xa = fma(e[q][s], e[q][s], xa);
        for (int a = 0; a < r; ++a) {
            const int kc = Ks[a];
            T xk[kRowsW];
#pragma unroll
            for (int q = 0; q < kRowsW; ++q) xk[q] = (i0 + q < m) ? xr[q][kc] : (T)0;
            const T* ha = Hs + (size_t)a * n;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int c = lane + 32 * s;
                const T hv = c < n ? ha[c] : (T)0;
#pragma unroll
                for (int q = 0; q < kRowsW; ++q) e[q][s] = fma(-xk[q], hv, e[q][s]);
            }
        }
#pragma unroll
        for (int q = 0; q < kRowsW; ++q)
#pragma unroll
            for (int s = 0; s < NS; ++s) ea = fma(e[q][s], e[q][s], ea);
        if (++cnt == kRowsFlush / kRowsW) {
            e2 += (double)ea;
            x2 += (double)xa;
            ea = xa = (T)0;
            cnt = 0;
        }
    }
    e2 += (double)ea;
    x2 += (double)xa;
    e2 = warp_sum(e2);
    x2 = warp_sum(x2);
    if (lane == 0) {
        red[0][warp] = e2;
        red[1][warp] = x2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double se = 0.0, sx = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            se += red[0][w];
            sx += red[1][w];
        }
        part[2 * blockIdx.x] = se;
        part[2 * blockIdx.x + 1] = sx;
    }
}

__global__ void residual_finish_kernel(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    double se = 0.0, sx = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) {
        se += part[2 * b];
        sx += part[2 * b + 1];
    }
    se = warp_sum(se);
    sx = warp_sum(sx);
    if (threadIdx.x == 0) {
        out[0] = sqrt(se);
        out[1] = sx > 0.0 ? se / sx : 0.0;
    }
}

int residual_blocks()
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 4 * (sms > 0 ? sms : 1);
}

template <typename T, int NS>
cudaError_t launch_res(const T* X, int64_t m, int n, int64_t ldx, const int32_t* K, int r, const double* H,
                       double* part, int nb, double* out, int* status, cudaStream_t s)
{
    const size_t smem = sizeof(T) * (size_t)r * n + sizeof(int) * (size_t)r;
    auto kern = full_residual_kernel<T, NS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<nb, kThreads, smem, s>>>(X, m, n, ldx, K, r, H, part, status);
    residual_finish_kernel<<<1, 32, 0, s>>>(part, nb, out);
    count_launch(2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t full_residual(const T* X, int64_t m, int n, int64_t ldx, const int32_t* K, int r, const double* H,
                          double* part, int nb, double* out, int* status, cudaStream_t s)
{
    if (n <= 32) return launch_res<T, 1>(X, m, n, ldx, K, r, H, part, nb, out, status, s);
    if (n <= 64) return launch_res<T, 2>(X, m, n, ldx, K, r, H, part, nb, out, status, s);
    if (n <= 128) return launch_res<T, 4>(X, m, n, ldx, K, r, H, part, nb, out, status, s);
    return launch_res<T, 8>(X, m, n, ldx, K, r, H, part, nb, out, status, s);
}

}  // namespace
}  // namespace mrnmf

using mrnmf::api::bind_device;
using mrnmf::api::cuda_fail;
using mrnmf::api::fail;
using mrnmf::api::grow;

extern "C" mrnmf_status mrnmf_gather_columns(mrnmf_handle* h, const void* X, int64_t m, int32_t n, int64_t ldx,
                                             int32_t dtype, const int32_t* K, int32_t r, void* W, int64_t ldw,
                                             void* stream)
{
    MRNMF_TRACE("mrnmf_gather_columns");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!X || !K || !W) return fail(h, MRNMF_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || m < 1 || ldx < n || r < 1 || r > n || ldw < r)
        return fail(h, MRNMF_ERR_INVALID_ARG, "need m >= 1, 1 <= r <= n, ldx >= n, ldw >= r");
    if (dtype != MRNMF_F32 && dtype != MRNMF_F64) return fail(h, MRNMF_ERR_INVALID_ARG, "dtype must be F32 or F64");
    mrnmf_status st = bind_device(h);
    if (st != MRNMF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = 8 * mrnmf::residual_blocks();
    if (dtype == MRNMF_F32)
        mrnmf::gather_kernel<float><<<blocks, mrnmf::kThreads, 0, s>>>(static_cast<const float*>(X), m, n, ldx, K, r,
                                                                      static_cast<float*>(W), ldw, h->d_status);
    else
        mrnmf::gather_kernel<double><<<blocks, mrnmf::kThreads, 0, s>>>(static_cast<const double*>(X), m, n, ldx, K,
                                                                       r, static_cast<double*>(W), ldw, h->d_status);
    mrnmf::count_launch();
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MRNMF_OK : cuda_fail(h, e, "gather");
}

extern "C" mrnmf_status mrnmf_full_residual(mrnmf_handle* h, const void* X, int64_t m, int32_t n, int64_t ldx,
                                            int32_t dtype, const int32_t* K, int32_t r, const double* H, double* out,
                                            void* stream)
{
    MRNMF_TRACE("mrnmf_full_residual");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!X || !K || !H || !out) return fail(h, MRNMF_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > MRNMF_NMAX || m < 1 || ldx < n || r < 1 || r > n)
        return fail(h, MRNMF_ERR_INVALID_ARG, "need m >= 1, 1 <= r <= n <= 256, ldx >= n");
    if (dtype != MRNMF_F32 && dtype != MRNMF_F64) return fail(h, MRNMF_ERR_INVALID_ARG, "dtype must be F32 or F64");
    mrnmf_status st = bind_device(h);
    if (st != MRNMF_OK) return st;
    const int nb = mrnmf::residual_blocks();
    if ((st = grow(h, &h->fws, &h->fws_bytes, 16ull * nb, "residual partial sums")) != MRNMF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* part = static_cast<double*>(h->fws);
    const cudaError_t e =
        dtype == MRNMF_F32
            ? mrnmf::full_residual(static_cast<const float*>(X), m, n, ldx, K, r, H, part, nb, out, h->d_status, s)
            : mrnmf::full_residual(static_cast<const double*>(X), m, n, ldx, K, r, H, part, nb, out, h->d_status, s);
    return e == cudaSuccess ? MRNMF_OK : cuda_fail(h, e, "full residual");
}
