// tc_selftest.cu -- a one-CTA tcgen05 GEMM, D = A B^T (A 128-by-K, B N-by-K,
// both K-major in shared memory without swizzle, D accumulated in TMEM), used
// to check the operand-descriptor and instruction-descriptor encodings of the
// tensor-core kernels against a host GEMM.
#include "../../include/mrnmf.h"
#include "common.cuh"
#include "internal.h"
#include <cuda_bf16.h>

#include "tc_common.cuh"

namespace mrnmf {
namespace {

__global__ void __launch_bounds__(128) tc_selftest_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                          float* __restrict__ D, int N, int K, int kind, int* status)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int eb = kind == 2 ? 2 : 4;  // element bytes: bf16 or tf32
    const uint32_t lbo = 128;
    const uint32_t sboA = (uint32_t)K * eb * 8, sboB = sboA;
    const size_t aBytes = (size_t)128 * K * eb, bBytes = (size_t)N * K * eb;
    unsigned char* Ahi = sm;
    unsigned char* Alo = Ahi + aBytes;
    unsigned char* Bhi = Alo + aBytes;
    unsigned char* Blo = Bhi + bBytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Blo + bBytes);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    auto put = [&](unsigned char* hi, unsigned char* lo, int row, int k, float v, uint32_t sbo) {
        const uint32_t off = tc::kmajor_off(row, k, eb, lbo, sbo);
        if (kind == 2) {
            *reinterpret_cast<__nv_bfloat16*>(hi + off) = __float2bfloat16_rn(v);
        } else {
            float h, l;
            tc::split_tf32(v, h, l);
            *reinterpret_cast<float*>(hi + off) = kind == 1 ? h : v;
            *reinterpret_cast<float*>(lo + off) = l;
        }
    };
    for (int e = t; e < 128 * K; e += 128) put(Ahi, Alo, e / K, e % K, A[e], sboA);
    for (int e = t; e < N * K; e += 128) put(Bhi, Blo, e / K, e % K, B[e], sboB);
    if (t == 0) tc::mbar_init(bar, 1);
    int ncols = 32;
    while (ncols < N) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(slot, (uint32_t)ncols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;

    if (t == 0) {
        const uint32_t idesc = tc::instr_desc(kind == 2 ? 1u : 2u, 128, N);
        const int kstep = kind == 2 ? 16 : 8;  // K per MMA: 32 bytes of each operand row
        for (int ks = 0; ks < K / kstep; ++ks) {
            const uint32_t koff = (uint32_t)ks * 2 * lbo;  // two 16-byte chunks along K per MMA
            const uint64_t ah = tc::smem_desc(tc::smem_addr(Ahi) + koff, lbo, sboA);
            const uint64_t al = tc::smem_desc(tc::smem_addr(Alo) + koff, lbo, sboA);
            const uint64_t bh = tc::smem_desc(tc::smem_addr(Bhi) + koff, lbo, sboB);
            const uint64_t bl = tc::smem_desc(tc::smem_addr(Blo) + koff, lbo, sboB);
            if (kind == 2) {
                tc::mma_f16(tmem, ah, bh, idesc, ks > 0);
            } else {
                tc::mma_tf32(tmem, ah, bh, idesc, ks > 0);
                if (kind == 1) {
                    tc::mma_tf32(tmem, ah, bl, idesc, true);
                    tc::mma_tf32(tmem, al, bh, idesc, true);
                }
            }
        }
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, 0);
    tc::fence_after_sync();
    if (!ok) {
        if (t == 0) set_status(status, MRNMF_ERR_TIMEOUT);
    } else {
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(size_t)(32 * warp + lane) * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)ncols);
}

}  // namespace
}  // namespace mrnmf

extern "C" mrnmf_status mrnmf_tc_selftest(const float* A, const float* B, float* D, int32_t N, int32_t K,
                                          int32_t kind, int32_t* status, void* stream)
{
    if (!A || !B || !D) return MRNMF_ERR_INVALID_ARG;
    if (N < 16 || N > 256 || N % 16 || K < 32 || K > 64 || K % 32 || kind < 0 || kind > 2)
        return MRNMF_ERR_INVALID_ARG;
    // Always 200 KiB: the operands use the first 2 (128 + N) K 4 <= 96 KiB, so
    // every read of the descriptors stays inside the CTA's allocation.
    const size_t smem = 200 * 1024;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (status && cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) return MRNMF_ERR_CUDA;
    if (cudaFuncSetAttribute(mrnmf::tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return MRNMF_ERR_CUDA;
    mrnmf::tc_selftest_kernel<<<1, 128, smem, s>>>(A, B, D, N, K, kind, reinterpret_cast<int*>(status));
    mrnmf::count_launch();
    return cudaGetLastError() == cudaSuccess ? MRNMF_OK : MRNMF_ERR_CUDA;
}
