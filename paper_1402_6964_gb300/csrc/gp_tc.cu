// gp_tc.cu -- the Gaussian projection pass (Sec. 2.3; Algorithm 1 with the
// combiner of Sec. 3.2) on the tcgen05 tensor cores: GX^T = X^T G accumulated
// in tensor memory, binary64 across CTAs.  Two forms:
//   TF32X3: 3-pass split TF32 (hi*hi + hi*lo + lo*hi), binary32 accumulation;
//   BF16:   G and X rounded to bfloat16 (round to nearest even), one pass of
//           kind::f16 MMAs: each product is exact in binary32, and the sums
//           are binary32 accumulations of those products.
// Column sums (of X as read, in binary32) and the input check ride along.
// n <= 128, k <= 64.
//
// Per CTA: a contiguous range of rows, consumed in 32-row slices.  A slice is
// staged into shared memory by a TMA bulk copy (two slices in flight), then
// the CTA's threads write the MMA operands: X^T as a K-major 128 x 32 matrix
// (row = column of X, padded to 128; K = the slice's rows) and G as a
// K-major kpad x 32 matrix (row = Gaussian coordinate): a TF32 high part and
// the remainder, or one bfloat16 part.  One thread issues the slice's MMAs
// (M = 128, N = kpad; 3 x 4 with K = 8, or 2 with K = 16) and commits them to
// the buffer's mbarrier; operand buffers are double-buffered so the
// conversion of slice s+1 overlaps the MMAs of slice s.  All waits are
// bounded (1 s).
#include <algorithm>

#include <cuda_bf16.h>

#include "../../include/mrnmf.h"
#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace mrnmf {

namespace {

constexpr int kThreads = 256;  // 8 warps: conversion and Philox spread wide; warps 0-3 read TMEM
constexpr int kSlice = 32;                     // rows per slice = K of one MMA group
constexpr uint32_t kLbo = 128;                 // K-adjacent core matrices
// 8-row groups: kSlice * elem_bytes / 16 chunks of 16 B along K
__host__ __device__ constexpr uint32_t sbo_for(int eb) { return (uint32_t)(kSlice * eb / 16) * 128; }

struct GpArgs {
    const float* X;
    int64_t rows;
    int64_t ldx;
    int n;
    int k;
    int64_t rows_per_cta;  // multiple of kSlice
    int64_t row_base;
    uint64_t seed;
    double* cs;  // P * n (+=)
    double* gx;  // P * k * n (+=)
    int* status;
    int bf16;  // 1: bfloat16 operands, one pass; 0: split TF32, three passes
};

__host__ __device__ inline size_t a128(size_t b) { return (b + 127) & ~size_t(127); }

// Shared memory: two staging buffers, then per buffer `parts` X^T operand
// parts and `parts` G parts (TF32X3: hi and lo, 4-byte elements; BF16: one,
// 2-byte elements), then the mbarriers.
struct GpLayout {
    size_t stage, xop, gop, bars, total;
    int eb, parts;
    __host__ __device__ GpLayout(int n, int kpad, bool bf16)
    {
        eb = bf16 ? 2 : 4;
        parts = bf16 ? 1 : 2;
        stage = a128((size_t)kSlice * n * 4);     // one staging buffer (binary32 rows of X)
        xop = (size_t)128 * kSlice * eb;          // one X^T operand part
        gop = (size_t)kpad * kSlice * eb;         // one G operand part
        bars = 128;
        total = 2 * stage + 2 * (parts * xop) + 2 * (parts * gop) + bars;
    }
};

__device__ __forceinline__ void put4(unsigned char* hi, unsigned char* lo, uint32_t off, float a, float b, float c,
                                     float d)
{
    float ha, la, hb, lb, hc, lc, hd, ld;
    tc::split_tf32(a, ha, la);
    tc::split_tf32(b, hb, lb);
    tc::split_tf32(c, hc, lc);
    tc::split_tf32(d, hd, ld);
    *reinterpret_cast<float4*>(hi + off) = make_float4(ha, hb, hc, hd);
    *reinterpret_cast<float4*>(lo + off) = make_float4(la, lb, lc, ld);
}

// Four consecutive K elements of one operand row, rounded to bfloat16 (8 bytes).
__device__ __forceinline__ void put4_bf16(unsigned char* p, uint32_t off, float a, float b, float c, float d)
{
    const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    *reinterpret_cast<uint2*>(p + off) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

// One operand chunk of four K elements in the pass's form.
__device__ __forceinline__ void put_op(bool bf, unsigned char* hi, unsigned char* lo, int row, int k0, float a, float b,
                                       float c, float d)
{
    if (bf) put4_bf16(hi, tc::kmajor_off(row, k0, 2, kLbo, sbo_for(2)), a, b, c, d);
    else put4(hi, lo, tc::kmajor_off(row, k0, 4, kLbo, sbo_for(4)), a, b, c, d);
}

__global__ void __launch_bounds__(kThreads) gp_tc_kernel(const GpArgs a)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int n = a.n, k = a.k;
    const int kpad = k <= 16 ? 16 : (k <= 32 ? 32 : 64);
    const bool bf = a.bf16 != 0;
    const GpLayout lay(n, kpad, bf);
    const size_t xpb = lay.parts * lay.xop, gpb = lay.parts * lay.gop;  // operand bytes per buffer
    unsigned char* stage[2] = {sm, sm + lay.stage};
    unsigned char* xhi[2] = {sm + 2 * lay.stage, sm + 2 * lay.stage + xpb};
    unsigned char* xlo[2] = {xhi[0] + lay.xop, xhi[1] + lay.xop};  // TF32X3 only
    unsigned char* gbase = sm + 2 * lay.stage + 2 * xpb;
    unsigned char* ghi[2] = {gbase, gbase + gpb};
    unsigned char* glo[2] = {ghi[0] + lay.gop, ghi[1] + lay.gop};  // TF32X3 only
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + 2 * gpb);  // tma[2], mma[2]
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 4);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_cta;
    const int64_t r1 = min(a.rows, r0 + a.rows_per_cta);
    const int64_t nslices = r1 > r0 ? (r1 - r0 + kSlice - 1) / kSlice : 0;
    const bool tma_ok = a.ldx == n && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);

    // operand rows past n (X^T) and past k (G) stay zero for the whole kernel
    for (int e = t; e < (int)(2 * xpb / 16); e += kThreads)
        reinterpret_cast<float4*>(xhi[0])[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = t; e < (int)(2 * gpb / 16); e += kThreads)
        reinterpret_cast<float4*>(gbase)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t == 0)
        for (int i = 0; i < 4; ++i) tc::mbar_init(&bars[i], 1);
    if (warp == 0) tc::tmem_alloc(slot, (uint32_t)(kpad < 32 ? 32 : kpad));
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;

    // slice s -> staging buffer s & 1, by TMA when the bytes allow it
    auto issue = [&](int64_t s) -> bool {
        const int64_t row0 = r0 + s * kSlice;
        const int rows_v = (int)min((int64_t)kSlice, r1 - row0);
        const uint32_t bytes = (uint32_t)rows_v * (uint32_t)n * 4u;
        if (!tma_ok || (bytes & 15u)) return false;
        if (t == 0) {
            const uint32_t bar = tc::smem_addr(&bars[s & 1]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_addr(stage[s & 1])),
                "l"(a.X + row0 * n), "r"(bytes), "r"(bar)
                : "memory");
        }
        return true;
    };
    bool via_tma[2] = {false, false};
    if (nslices > 0) via_tma[0] = issue(0);
    if (nslices > 1) via_tma[1] = issue(1);
    uint32_t tma_phase[2] = {0u, 0u}, mma_phase[2] = {0u, 0u};
    int mma_pending[2] = {0, 0};
    bool ok = true, bad = false;
    float csum = 0.f;
    double csum_d = 0.0;
    const uint32_t idesc = tc::instr_desc(bf ? 1u : 2u, 128, kpad);

    for (int64_t s = 0; s < nslices && ok; ++s) {
        const int b = (int)(s & 1);
        const int64_t row0 = r0 + s * kSlice;
        const int rows_v = (int)min((int64_t)kSlice, r1 - row0);
        const float* tile;
        if (via_tma[b]) {
            ok = __syncthreads_and(tc::mbar_wait(&bars[b], tma_phase[b]));
            tma_phase[b] ^= 1u;
            tile = reinterpret_cast<const float*>(stage[b]);
        } else {
            // direct loads into the staging buffer (ragged slice or unaligned X)
            float* st = reinterpret_cast<float*>(stage[b]);
            for (int e = t; e < rows_v * n; e += kThreads) {
                const int r = e / n, c = e - r * n;
                st[e] = a.X[(row0 + r) * a.ldx + c];
            }
            __syncthreads();
            tile = st;
        }
        if (!ok) break;
        // operand buffers b are free once the MMAs of slice s-2 completed
        if (mma_pending[b]) {
            ok = __syncthreads_and(tc::mbar_wait(&bars[2 + b], mma_phase[b]));
            mma_phase[b] ^= 1u;
            mma_pending[b] = 0;
            if (!ok) break;
        }
        // X^T: task (column c, 4-row chunk q) -> one 16-byte chunk per part,
        // spread over all threads; thread t keeps the column sums of the
        // columns c = t (mod 128) it visits (c < n <= 128: exactly column t)
        for (int task = t; task < n * (kSlice / 4); task += kThreads) {
            const int c = task % n, q = task / n;
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = 4 * q + u;
                v[u] = r < rows_v ? tile[r * n + c] : 0.f;
                bad |= !(v[u] >= 0.f);
            }
            put_op(bf, xhi[b], xlo[b], c, 4 * q, v[0], v[1], v[2], v[3]);
        }
        if (t < n) {
            float part = 0.f;
            for (int r = 0; r < rows_v; ++r) part += tile[r * n + t];
            csum += part;
        }
        // G: task (4-row chunk q4, coordinate quad g4) -> 4 Philox blocks -> one
        // 16-byte chunk per coordinate and part (no bank conflicts);
        // coordinates past k stay zero
        {
            const int kq = kpad >> 2;
            for (int task = t; task < (kSlice / 4) * kq; task += kThreads) {
                const int g4 = task % kq, q4 = task / kq;
                const int l0 = 4 * g4;
                float4 g[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = 4 * q4 + u;
                    g[u] = (r < rows_v && l0 < k) ? gauss4(a.seed, a.row_base + row0 + r, (uint32_t)g4)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                const float m1 = l0 + 1 < k ? 1.f : 0.f, m2 = l0 + 2 < k ? 1.f : 0.f, m3 = l0 + 3 < k ? 1.f : 0.f;
                put_op(bf, ghi[b], glo[b], l0, 4 * q4, g[0].x, g[1].x, g[2].x, g[3].x);
                put_op(bf, ghi[b], glo[b], l0 + 1, 4 * q4, m1 * g[0].y, m1 * g[1].y, m1 * g[2].y, m1 * g[3].y);
                put_op(bf, ghi[b], glo[b], l0 + 2, 4 * q4, m2 * g[0].z, m2 * g[1].z, m2 * g[2].z, m2 * g[3].z);
                put_op(bf, ghi[b], glo[b], l0 + 3, 4 * q4, m3 * g[0].w, m3 * g[1].w, m3 * g[2].w, m3 * g[3].w);
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
            // the staging buffer is free again: fetch slice s+2 into it
            if (s + 2 < nslices) via_tma[b] = issue(s + 2);
            if (bf) {
                // K = 16 per MMA: two 16-byte chunks of each operand row
                for (int ks = 0; ks < kSlice / 16; ++ks) {
                    const uint32_t koff = (uint32_t)ks * 2 * kLbo;
                    const uint64_t ah = tc::smem_desc(tc::smem_addr(xhi[b]) + koff, kLbo, sbo_for(2));
                    const uint64_t bh = tc::smem_desc(tc::smem_addr(ghi[b]) + koff, kLbo, sbo_for(2));
                    tc::mma_f16(tmem, ah, bh, idesc, s > 0 || ks > 0);
                }
            } else {
                for (int ks = 0; ks < kSlice / 8; ++ks) {
                    const uint32_t koff = (uint32_t)ks * 2 * kLbo;
                    const uint64_t ah = tc::smem_desc(tc::smem_addr(xhi[b]) + koff, kLbo, sbo_for(4));
                    const uint64_t al = tc::smem_desc(tc::smem_addr(xlo[b]) + koff, kLbo, sbo_for(4));
                    const uint64_t bh = tc::smem_desc(tc::smem_addr(ghi[b]) + koff, kLbo, sbo_for(4));
                    const uint64_t bl = tc::smem_desc(tc::smem_addr(glo[b]) + koff, kLbo, sbo_for(4));
                    tc::mma_tf32(tmem, ah, bh, idesc, s > 0 || ks > 0);
                    tc::mma_tf32(tmem, ah, bl, idesc, true);
                    tc::mma_tf32(tmem, al, bh, idesc, true);
                }
            }
            tc::mma_commit(&bars[2 + b]);
        } else if (s + 2 < nslices) {
            via_tma[b] = tma_ok && (((uint32_t)min((int64_t)kSlice, r1 - (r0 + (s + 2) * kSlice)) * (uint32_t)n * 4u) & 15u) == 0;
        }
        mma_pending[b] = 1;
        if (((s + 1) & 31) == 0) {
            csum_d += (double)csum;
            csum = 0.f;
        }
    }
    // drain the MMAs still in flight
    for (int b = 0; b < 2; ++b)
        if (mma_pending[b]) {
            const bool w = tc::mbar_wait(&bars[2 + b], mma_phase[b]);
            ok = ok && w;
        }
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    if (!ok && t == 0) set_status(a.status, MRNMF_ERR_TIMEOUT);
    if (ok && nslices > 0 && warp < 4) {
        // D (lane = column of X, TMEM column = coordinate) -> this CTA's partial GX
        const int c = 32 * warp + lane;
        for (int l0 = 0; l0 < kpad; l0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)l0, v);
            if (c < n)
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (l0 + i < k) a.gx[((size_t)blockIdx.x * k + l0 + i) * n + c] += (double)v[i];
        }
    }
    if (t < n && a.cs) a.cs[(size_t)blockIdx.x * n + t] += csum_d + (double)csum;
    if (__syncthreads_or(bad) && t == 0) set_status(a.status, MRNMF_ERR_BAD_INPUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)(kpad < 32 ? 32 : kpad));
}

}  // namespace

bool gp_tc_supported(int n, int k) { return n >= 1 && n <= 128 && k >= 1 && k <= 64; }

cudaError_t launch_gp_tc(const float* X, int64_t rows, int64_t ldx, int n, int k, int64_t row_base, uint64_t seed,
                         int max_ctas, double* cs, double* gx, int* status, int bf16, cudaStream_t s)
{
    const int kpad = k <= 16 ? 16 : (k <= 32 ? 32 : 64);
    const GpLayout lay(n, kpad, bf16 != 0);
    const size_t smem = lay.total + 16;
    cudaError_t e = cudaFuncSetAttribute(gp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 1, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int per_sm = smem_sm > 0 ? (int)(smem_sm / (smem + 1024)) : 1;  // resident CTAs by shared memory
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;
    int grid = sms * per_sm;
    if (grid > max_ctas) grid = max_ctas;
    const int64_t min_rows = 4 * kSlice;
    if ((int64_t)grid * min_rows > rows) grid = (int)std::max<int64_t>(1, (rows + min_rows - 1) / min_rows);
    GpArgs a;
    a.X = X;
    a.rows = rows;
    a.ldx = ldx;
    a.n = n;
    a.k = k;
    int64_t per = (rows + grid - 1) / grid;
    a.rows_per_cta = (per + kSlice - 1) / kSlice * kSlice;
    a.row_base = row_base;
    a.seed = seed;
    a.cs = cs;
    a.gx = gx;
    a.status = status;
    a.bf16 = bf16;
    gp_tc_kernel<<<grid, kThreads, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mrnmf
