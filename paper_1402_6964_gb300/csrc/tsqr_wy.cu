// tsqr_wy.cu -- the pass over X with the trailing updates of the leaf QR on
// the tensor cores: tcgen05 MMAs in TF32 with FP32 accumulation, three
// products per product of values (TF32X3) or one (TF32), for 16 < n <= 256.
//
// One CTA of 128 threads per row stream.  Each 128-row tile A of X is folded
// into the stream's running triangle R (binary32; it stays in the stream's
// state slot, L2-resident, with the current panel's 16 rows staged in shared
// memory) by the
// blocked Householder QR of the stacked [R; A] (the local QR of Sec. 3.1) in
// compact-WY form (Schreiber and Van Loan, SIAM J. Sci. Stat. Comput. 10,
// 1989), one 16-column panel P = j0 .. j0+15 at a time:
//
//   1. the panel of [R; A] is factored on the SIMT cores by all four warps,
//      lane (c, h) of warp w holding column j0+c of 16 tile rows, the warps'
//      partial dot products summed through shared memory: reflectors
//      v_q = [e_(j0+q); y_q] with the same column step as the SIMT leaves
//      (beta = -sign(alpha) sqrt(alpha^2 + sigma), y = A(:,j) / (alpha -
//      beta), tau = (beta - alpha) / beta); the lanes of finished columns
//      form the Gram Y'Y from the published pivot at no extra cost, and T
//      (Q_P = I - V T V') follows from the forward recurrence;
//   2. Z = Y' A(:, trail) on the tensor cores (GEMM1).  The contraction runs
//      over the tile's rows, so the trailing block is transposed in chunks of
//      16 rows into tensor memory (lane = column of A, TMEM column = tile
//      row; columns 128.. in a second lane block for n > 128) and serves as
//      the MMA's A operand, with Y' from shared memory as the B operand; two
//      chunk buffers let the transpose of one chunk overlap the MMAs of the
//      previous one (one buffer for n > 128, where tensor memory is full);
//   3. W = T' (R(P, trail) + Z), R(P, trail) -= W on the SIMT cores, one
//      thread per trailing column;
//   4. A(:, trail) -= Y W on the tensor cores (GEMM2): the tile itself lives
//      in tensor memory (lane = tile row) as the accumulator, Y is the A
//      operand (tensor memory, lane = tile row) and -W the B operand.
//
// The Gaussian projection of the same tile (Algorithm 1 with the combiner of
// Sec. 3.2), X' G, rides on the first panel's transposed chunks, which hold
// all of X's columns: one more MMA per chunk into an accumulator that stays
// in tensor memory across tiles and is flushed to the binary64 partial sums
// every kFlushTiles tiles.  The column sums (the scaling D of Sec. 2.3) are
// summed from the same chunks, pairwise in binary32 over 16 rows and in
// binary64 across chunks.
//
// Precision: in the TF32X3 form every product is formed as hi*hi + hi*lo +
// lo*hi with hi = the value as the tensor core reads it (kind::tf32 keeps the
// top 19 bits of a binary32 operand and drops the rest) and lo = x - hi,
// exact in binary32; the TF32 form (LeafArgs::tc_split = 0) takes hi*hi
// alone, skipping the low parts and the correction MMAs.
// The MMA instructions are issued by one elected lane of warp 0, unrolled,
// with their operands in tensor memory wherever the operand spans the 128
// lanes: on GB300 such MMAs cost a fraction of those that read a 128-row
// operand from shared memory.
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "leaf.h"
#include "tc_common.cuh"

namespace mrnmf {

namespace {

constexpr int kRows = 128;       // tile height = TMEM lanes = threads
constexpr int kNB = 16;          // panel width
constexpr int kCH = 16;          // tile rows per transposed chunk
constexpr int kFlushTiles = 32;  // tiles between binary64 flushes of the projection
constexpr int kTld = kNB + 1;    // row stride (floats) of T, Y'Y and the panel buffer

__host__ __device__ constexpr uint32_t up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Tensor-memory columns and shared-memory offsets of one instance.  NP is the
// padded column count (64, 128 or 256), KP the padded projection width.
template <int NP, int KP>
struct WyMap {
    static constexpr int LB = NP > 128 ? 2 : 1;       // lane blocks of column-indexed data
    static constexpr int NBUF = NP > 128 ? 1 : 2;     // transposed-chunk buffers
    static constexpr int XR = NP > 128 ? 64 : 128;    // tile rows held by the transpose buffer
    // TMEM (columns)
    static constexpr uint32_t cTile = 0;              // the tile, lane = row, NP columns
    static constexpr uint32_t cYH = NP;               // Y (hi, lo), lane = row, 16 columns each
    static constexpr uint32_t cYL = cYH + kNB;
    static constexpr uint32_t cAT0 = cYL + kNB;       // chunks of A(:, trail)': [buf][lane block][hi, lo][16]
    static constexpr uint32_t cZ0 = cAT0 + NBUF * LB * 2 * kCH;  // GEMM1 result: [hi*hi, corrections][lane block][16]
    static constexpr uint32_t cGX0 = cZ0 + 2 * LB * kNB;  // X' G accumulator: [lane block][KP]
    static constexpr uint32_t used = cGX0 + LB * KP;
    static constexpr uint32_t cols = used <= 128 ? 128u : used <= 256 ? 256u : 512u;
    static_assert(used <= 512, "tensor memory");
    __host__ __device__ static constexpr uint32_t cAT(int buf, int lb, int part)
    {
        return cAT0 + (uint32_t)(((buf * LB + lb) * 2 + part) * kCH);
    }
    __host__ __device__ static constexpr uint32_t cZ(int part, int lb) { return cZ0 + (uint32_t)((part * LB + lb) * kNB); }
    __host__ __device__ static constexpr uint32_t cGX(int lb) { return cGX0 + (uint32_t)(lb * KP); }

    // shared memory (bytes from a 1024-byte aligned base)
    static constexpr int xld = NP + 1;                   // row stride (floats) of the transpose buffer
    static constexpr uint32_t oYsH = 0;                  // Y' as GEMM1's B operand: N = 16, K = 128, SW128
    static constexpr uint32_t ysBytes = kNB * kRows * 4;
    static constexpr uint32_t oYsL = oYsH + ysBytes;
    static constexpr uint32_t gsBytes = KP * kRows * 4;  // G' as the projection's B operand, SW128
    static constexpr uint32_t oGsH = oYsL + ysBytes;
    static constexpr uint32_t oGsL = oGsH + gsBytes;
    static constexpr uint32_t wsBytes = NP * kNB * 4;    // -W as GEMM2's B operand: N = trail, K = 16
    static constexpr uint32_t oWsH = oGsL + gsBytes;
    static constexpr uint32_t oWsL = oWsH + wsBytes;
    static constexpr uint32_t oXS = oWsL + wsBytes;      // transpose buffer, XR rows x xld
    static constexpr uint32_t oXP = up(oXS + XR * xld * 4, 16);  // panel columns / Y, 128 x kTld
    static constexpr uint32_t oRR = up(oXP + kRows * kTld * 4, 16);  // R rows j0 .. j0+15, 16 x NP
    static constexpr uint32_t oPub = oRR + kNB * NP * 4;  // published pivot column, 128 floats
    static constexpr uint32_t oRed = oPub + kRows * 4;    // per-warp partial dots: [step parity][4 warps][16]
    static constexpr uint32_t oT = oRed + 2 * 4 * kNB * 4;  // T, 16 x 17
    static constexpr uint32_t oGy = oT + kNB * kTld * 4;  // Y'Y, 16 x 17
    static constexpr uint32_t oTau = oGy + kNB * kTld * 4;
    static constexpr uint32_t oBar = up(oTau + kNB * 4, 16);
    static constexpr uint32_t oSlot = oBar + 32;
    static constexpr uint32_t bytes = oSlot + 16;
    static constexpr uint32_t alloc = bytes + 1024;       // slack for the 1024-byte alignment
    static_assert(oYsL % 1024 == 0 && oGsH % 1024 == 0 && oGsL % 1024 == 0, "SW128 operands need 1 KB alignment");
    static_assert(alloc <= 227 * 1024, "shared memory");
};

// Byte offset of element (row n, K index k) of a K-major operand with 128-byte
// swizzle and K = 128 (the tile rows): atoms of 8 rows x 32 K-elements,
// `ng` 8-row groups per 32-element K block.
__device__ __forceinline__ uint32_t sw128_off(int n, int k, int ng)
{
    return (uint32_t)(k >> 5) * (uint32_t)ng * 1024u + (uint32_t)(n >> 3) * 1024u + (uint32_t)(n & 7) * 128u +
           ((uint32_t)(((k & 31) >> 2) ^ (n & 7)) << 4) + (uint32_t)(k & 3) * 4u;
}
// Descriptor of the 8-element K step starting at K index k0 (a multiple of 8).
__device__ __forceinline__ uint64_t sw128_step(uint32_t base, int k0, int ng)
{
    return tc::smem_desc_sw128(base + (uint32_t)(k0 >> 5) * (uint32_t)ng * 1024u + (uint32_t)(k0 & 31) * 4u, 1024u);
}
// Element (row n, K index q < 16) of the no-swizzle K-major operand -W:
// core matrices of 8 rows x 16 bytes, LBO 128 (along K), SBO 512 (along N).
__device__ __forceinline__ uint32_t wq_off(int n, int q)
{
    return (uint32_t)(n >> 3) * 512u + (uint32_t)(q >> 2) * 128u + (uint32_t)(n & 7) * 16u + (uint32_t)(q & 3) * 4u;
}

__device__ __forceinline__ float sum16(const float* v)
{
    const float a = (v[0] + v[1]) + (v[2] + v[3]), b = (v[4] + v[5]) + (v[6] + v[7]);
    const float c = (v[8] + v[9]) + (v[10] + v[11]), d = (v[12] + v[13]) + (v[14] + v[15]);
    return (a + b) + (c + d);
}

template <int NP, int KP>
__global__ void __launch_bounds__(kRows, NP <= 64 ? 2 : 1) tsqr_wy_kernel(const LeafArgs a)
{
    using M = WyMap<NP, KP>;
    constexpr int LB = M::LB, NBUF = M::NBUF, XR = M::XR;
    extern __shared__ unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((1024u - (tc::smem_addr(sm_raw) & 1023u)) & 1023u);
    const uint32_t sb = tc::smem_addr(sm);
    const unsigned FULL = 0xffffffffu;
    const int n = a.n, nt = (n + 15) & ~15;
    const int k = (KP > 0 && a.gx) ? a.k : 0;
    const bool split = a.tc_split != 0;  // three products (TF32X3), or one (TF32)
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int cta = blockIdx.x;
    float* XS = reinterpret_cast<float*>(sm + M::oXS);
    float* XP = reinterpret_cast<float*>(sm + M::oXP);
    float* RR = reinterpret_cast<float*>(sm + M::oRR);
    float* PUB = reinterpret_cast<float*>(sm + M::oPub);
    float* Ts = reinterpret_cast<float*>(sm + M::oT);
    float* Gy = reinterpret_cast<float*>(sm + M::oGy);
    float* tau = reinterpret_cast<float*>(sm + M::oTau);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + M::oBar);  // [0], [1]: chunk buffers; [2]: GEMM2
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + M::oSlot);
    // The stream's running triangle R (binary32, n x n row-major) lives in its
    // state slot in global memory (it stays in L2); the rows of the current
    // panel are staged in shared memory.
    float* Rg = static_cast<float*>(a.R_out) + (size_t)cta * n * n;
    {
        const float* Rin = static_cast<const float*>(a.R_in);
        if (Rin != a.R_out) {
            for (int e = t; e < n * n; e += kRows) Rg[e] = Rin ? Rin[(size_t)cta * n * n + e] : 0.f;
        }
    }
    if (t == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::mbar_init(&bar[2], 1);
    }
    if (warp == 0) tc::tmem_alloc(slot, M::cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t tq = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's lane quadrant

    const int64_t r0 = (int64_t)cta * a.rows_per_cta;
    const int64_t r1 = min(a.rows, r0 + a.rows_per_cta);
    const int64_t ntiles = r1 > r0 ? (r1 - r0 + kRows - 1) / kRows : 0;
    const float* X = static_cast<const float*>(a.X);
    const int npan = (n + kNB - 1) / kNB;
    uint32_t ph[3] = {0u, 0u, 0u};
    bool bad = false, dead = false, gx_fresh = true;
    int since_flush = 0;
    double cs_acc[LB];  // column t + 128 lb's sum
#pragma unroll
    for (int lb = 0; lb < LB; ++lb) cs_acc[lb] = 0.0;

    // Bounded wait for the commit on mbarrier b; block-uniform outcome.
    auto wait_bar = [&](int b) -> bool {
        bool ok = tc::mbar_wait(&bar[b], ph[b]);
        if (!ok) tc::mbar_wait(&bar[b], ph[b]);  // a second bounded wait for the MMAs in flight
        ph[b] ^= 1u;
        tc::fence_after_sync();
        if (__syncthreads_or(!ok)) {
            if (t == 0) set_status(a.status, MRNMF_ERR_TIMEOUT);
            return false;
        }
        return true;
    };
    auto block_sync = [&]() {
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    // Rows [XR h, XR h + XR) of tile columns [c0, nt) from tensor memory into the transpose buffer.
    auto refresh_xs = [&](int c0, int h) {
        if (warp * 32 >= XR * h && warp * 32 < XR * (h + 1)) {
            const int rr = t - XR * h;
            for (int c = c0 & ~15; c < nt; c += 16) {
                float v[16];
                tc::tmem_ld16(tq + M::cTile + (uint32_t)c, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) XS[rr * M::xld + c + i] = v[i];
            }
        }
    };

    for (int64_t tile = 0; tile < ntiles && !dead; ++tile) {
        // ---- the tile into tensor memory (lane t = row t), 16 columns at a time
        {
            const int64_t row = r0 + tile * kRows + t;
            const bool valid = row < r1;
            const float* src = X + (valid ? row : r0) * a.ldx;
            for (int c0 = 0; c0 < nt; c0 += 16) {
                float x[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = c0 + i;
                    x[i] = (valid && c < n) ? __ldg(src + c) : 0.f;
                    bad |= !(x[i] >= 0.f);
                }
                tc::tmem_st16_nowait(tq + M::cTile + (uint32_t)c0, x);
            }
            tc::tmem_wait_st();
            if (KP > 0 && k > 0) {
                // G' (Algorithm 1: g_i ~ N(0, I_k) keyed by the global row), K index = tile row t
                const int64_t grow = a.row_base + row;
#pragma unroll
                for (int q4 = 0; q4 < (KP > 0 ? KP : 4) / 4; ++q4) {
                    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (valid && 4 * q4 < k) g = gauss4(a.seed, grow, (uint32_t)q4);
                    const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int q = 4 * q4 + i;
                        const float v = q < k ? gv[i] : 0.f;
                        const uint32_t off = sw128_off(q, t, KP / 8);
                        *reinterpret_cast<float*>(sm + M::oGsH + off) = v;
                        if (split) *reinterpret_cast<float*>(sm + M::oGsL + off) = tc::tf32_lo(v);
                    }
                }
                tc::fence_async_smem();
            }
        }
        block_sync();

        for (int p = 0; p < npan && !dead; ++p) {
            const int j0 = kNB * p;
            const int pw = min(kNB, n - j0);
            const int trail0 = j0 + kNB;
            const int ntr = nt > trail0 ? nt - trail0 : 0;  // trailing columns, padded to 16
            // ---- the panel columns (lane t = row t) and the panel's rows of R
            {
                float v[16];
                tc::tmem_ld16(tq + M::cTile + (uint32_t)j0, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) XP[t * kTld + i] = v[i];
                for (int e = t; e < kNB * NP; e += kRows) {
                    const int q = e / NP, c = e - q * NP;
                    RR[e] = (j0 + q < n && c >= j0 && c < n) ? Rg[(size_t)(j0 + q) * n + c] : 0.f;
                }
            }
            __syncthreads();

            // ---- 1. panel factorization, all four warps: lane (c, h) of warp w holds
            // column j0+c of tile rows 32w + 16h .. 32w + 16h + 15.  Each column step
            // forms the warp's partial dot products with the published pivot, sums
            // the two row halves with one xor shuffle and the four warps' partials
            // through shared memory (one barrier per step, buffers alternating by
            // step parity); every lane then applies the step to its own rows.
            {
                const int c = lane & 15, h = lane >> 4;
                const int rb = 32 * warp + 16 * h;  // first tile row of this lane
                float* red = reinterpret_cast<float*>(sm + M::oRed);
                float av[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) av[i] = XP[(rb + i) * kTld + c];
                for (int j = 0; j < pw; ++j) {
                    if (c == j) {
#pragma unroll
                        for (int i4 = 0; i4 < 4; ++i4)
                            reinterpret_cast<float4*>(PUB)[rb / 4 + i4] =
                                make_float4(av[4 * i4], av[4 * i4 + 1], av[4 * i4 + 2], av[4 * i4 + 3]);
                    }
                    const int jg = j0 + j;
                    const float alpha = RR[j * NP + jg];
                    const float rjc = RR[j * NP + j0 + c];
                    __syncwarp();
                    float pv[16];
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4) {
                        const float4 v = reinterpret_cast<const float4*>(PUB)[rb / 4 + i4];
                        pv[4 * i4] = v.x;
                        pv[4 * i4 + 1] = v.y;
                        pv[4 * i4 + 2] = v.z;
                        pv[4 * i4 + 3] = v.w;
                    }
                    float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        g0 = fmaf(pv[i], av[i], g0);
                        g1 = fmaf(pv[i + 1], av[i + 1], g1);
                        g2 = fmaf(pv[i + 2], av[i + 2], g2);
                        g3 = fmaf(pv[i + 3], av[i + 3], g3);
                    }
                    float g = (g0 + g1) + (g2 + g3);
                    g += __shfl_xor_sync(FULL, g, 16);
                    float* rj = red + (j & 1) * 4 * kNB;
                    if (h == 0) rj[warp * kNB + c] = g;
                    __syncthreads();
                    g = (rj[c] + rj[kNB + c]) + (rj[2 * kNB + c] + rj[3 * kNB + c]);
                    const float sig = __shfl_sync(FULL, g, j);
                    if (sig > 0.f) {
                        const HhScalars hs = hh_scalars(alpha, sig);
                        if (c > j && c < pw) {
                            const float wp = fmaf(hs.d, rjc, g);  // d (R_jc + g_c / d)
                            const float f = (wp * hs.rd) * hs.rb;
#pragma unroll
                            for (int i = 0; i < 16; ++i) av[i] = fmaf(f, pv[i], av[i]);
                            if (warp == 0 && h == 0) RR[j * NP + j0 + c] = fmaf(wp, hs.rb, rjc);
                        } else if (c == j) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) av[i] *= hs.rd;  // y_j = A(:,j) / (alpha - beta)
                            if (warp == 0 && h == 0) {
                                RR[j * NP + jg] = hs.beta;
                                tau[j] = -hs.d * hs.rb;
                            }
                        } else if (c < j && warp == 0 && h == 0) {
                            Gy[c * kTld + j] = g * hs.rd;  // y_c' y_j
                        }
                    } else if (warp == 0 && h == 0) {
                        // nothing below R_jj: the identity (tau = 0, y_j = 0)
                        if (c == j) tau[j] = 0.f;
                        if (c < j) Gy[c * kTld + j] = 0.f;
                    }
                    __syncwarp();
                }
                // Y into the panel buffer (rows of Y for the tensor-memory copy)
#pragma unroll
                for (int i = 0; i < 16; ++i) XP[(rb + i) * kTld + c] = av[i];
                if (ntr > 0) {
                    // Y' as GEMM1's B operand (row c, K = tile row), hi and lo
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4) {
                        const uint32_t off = sw128_off(c, rb + 4 * i4, kNB / 8);
                        const float4 v = make_float4(av[4 * i4], av[4 * i4 + 1], av[4 * i4 + 2], av[4 * i4 + 3]);
                        *reinterpret_cast<float4*>(sm + M::oYsH + off) = v;
                        if (split)
                            *reinterpret_cast<float4*>(sm + M::oYsL + off) =
                                make_float4(tc::tf32_lo(v.x), tc::tf32_lo(v.y), tc::tf32_lo(v.z), tc::tf32_lo(v.w));
                    }
                    tc::fence_async_smem();
                }
            }
            __syncthreads();
            if (ntr > 0 && warp == 0 && lane < kNB) {
                // row i of T: T(i,i) = tau_i, T(i,q) = -tau_q sum_{i<=m<q} T(i,m) (Y'Y)(m,q)
                const int i = lane;
                float Ti[kNB];
#pragma unroll
                for (int q = 0; q < kNB; ++q) {
                    float v = 0.f;
                    if (q == i) {
                        v = tau[i];
                    } else if (q > i) {
                        float s = 0.f;
#pragma unroll
                        for (int m = 0; m < q; ++m)
                            if (m >= i) s = fmaf(Ti[m], Gy[m * kTld + q], s);
                        v = -tau[q] * s;
                    }
                    Ti[q] = v;
                }
#pragma unroll
                for (int q = 0; q < kNB; ++q) Ts[i * kTld + q] = Ti[q];
            }
            __syncthreads();

            if (ntr > 0) {
                // ---- Y (hi, lo) into tensor memory, lane = tile row
                {
                    float y[16], lo[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        y[q] = XP[t * kTld + q];
                        lo[q] = tc::tf32_lo(y[q]);
                    }
                    tc::tmem_st16_nowait(tq + M::cYH, y);
                    if (split) tc::tmem_st16_nowait(tq + M::cYL, lo);
                    tc::tmem_wait_st();
                }

                // ---- 2. GEMM1 (and the projection on the first panel), 16 tile rows per chunk
                const bool gp = p == 0 && k > 0;
                const int cA = p == 0 ? 0 : trail0;  // first column that is transposed
                const uint32_t idZ = tc::instr_desc(2, 128, kNB);
                for (int hx = 0; hx < kRows / XR && !dead; ++hx) {
                    refresh_xs(cA, hx);
                    __syncthreads();
                    for (int qq = 0; qq < XR / kCH; ++qq) {
                        const int q = hx * (XR / kCH) + qq;
                        const int buf = q % NBUF;
                        if (q >= NBUF && !wait_bar(buf)) {
                            dead = true;
                            break;
                        }
#pragma unroll
                        for (int lb = 0; lb < LB; ++lb) {
                            const int cw = 128 * lb + 32 * warp;  // this warp's first column in block lb
                            if (cw < nt && cw + 32 > cA) {
                                const int c = 128 * lb + t;
                                float v[16], lo[16];
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    v[i] = c < nt ? XS[(qq * kCH + i) * M::xld + c] : 0.f;
                                    lo[i] = tc::tf32_lo(v[i]);
                                }
                                if (p == 0 && c < n) cs_acc[lb] += (double)sum16(v);
                                tc::tmem_st16_nowait(tq + M::cAT(buf, lb, 0), v);
                                if (split) tc::tmem_st16_nowait(tq + M::cAT(buf, lb, 1), lo);
                                tc::tmem_wait_st();
                            }
                        }
                        block_sync();
                        // the MMAs are issued from warp 3: for n <= 96 it has no columns to
                        // transpose, so the issue overlaps the other warps' next chunk
                        if (warp == 3) {
                            if (tc::elect_one()) {
#pragma unroll
                                for (int ks = 0; ks < kCH / 8; ++ks) {
                                    const int k0 = q * kCH + ks * 8;
                                    const uint64_t bh = sw128_step(sb + M::oYsH, k0, kNB / 8);
                                    const uint64_t bl = sw128_step(sb + M::oYsL, k0, kNB / 8);
#pragma unroll
                                    for (int lb = 0; lb < LB; ++lb) {
                                        if (128 * lb >= nt || 128 * lb + 128 <= cA) continue;  // no live column
                                        const uint32_t ah = tmem + M::cAT(buf, lb, 0) + 8 * ks;
                                        const uint32_t al = tmem + M::cAT(buf, lb, 1) + 8 * ks;
                                        // hi*hi and the two correction products in separate
                                        // accumulators: each MMA truncates its binary32 sum,
                                        // and the corrections are 2^-11 of the main term
                                        const uint32_t za = tmem + M::cZ(0, lb), zb = tmem + M::cZ(1, lb);
                                        tc::mma_tf32_ts(za, ah, bh, idZ, (q | ks) != 0);
                                        if (split) {
                                            tc::mma_tf32_ts(zb, ah, bl, idZ, (q | ks) != 0);
                                            tc::mma_tf32_ts(zb, al, bh, idZ, true);
                                        }
                                        if (KP > 0 && gp) {
                                            const uint32_t idG = tc::instr_desc(2, 128, KP > 0 ? KP : 16);
                                            const uint64_t gh = sw128_step(sb + M::oGsH, k0, KP / 8);
                                            const uint64_t gl = sw128_step(sb + M::oGsL, k0, KP / 8);
                                            const uint32_t gxa = tmem + M::cGX(lb);
                                            tc::mma_tf32_ts(gxa, ah, gh, idG, !(gx_fresh && q == 0 && ks == 0));
                                            if (split) {
                                                tc::mma_tf32_ts(gxa, ah, gl, idG, true);
                                                tc::mma_tf32_ts(gxa, al, gh, idG, true);
                                            }
                                        }
                                    }
                                }
                                tc::mma_commit(&bar[buf]);
                            }
                            __syncwarp();
                        }
                    }
                }
                // the outstanding chunk commits, oldest first
                for (int b = 0; b < NBUF && !dead; ++b) {
                    const int q = kRows / kCH - NBUF + b;
                    if (!wait_bar(q % NBUF)) dead = true;
                }
                if (dead) break;
                if (gp) gx_fresh = false;

                // ---- 3. W = T' (R(P, trail) + Z); R(P, trail) -= W; -W staged as GEMM2's B operand
#pragma unroll
                for (int lb = 0; lb < LB; ++lb) {
                    const int cw = 128 * lb + 32 * warp;
                    if (cw < nt && cw + 32 > trail0) {
                        float z[16];
                        tc::tmem_ld16(tq + M::cZ(0, lb), z);
                        if (split) {  // the corrections' accumulator is written by the three-product form only
                            float zb[16];
                            tc::tmem_ld16(tq + M::cZ(1, lb), zb);
#pragma unroll
                            for (int q = 0; q < 16; ++q) z[q] += zb[q];
                        }
                        const int c = 128 * lb + t;
                        if (c >= trail0 && c < nt) {
                            float w[16];
                            if (c < n) {
                                float u[16];
#pragma unroll
                                for (int q = 0; q < 16; ++q) u[q] = RR[q * NP + c] + z[q];
#pragma unroll
                                for (int q = 0; q < 16; ++q) {
                                    float s = 0.f;
#pragma unroll
                                    for (int m = 0; m <= q; ++m) s = fmaf(Ts[m * kTld + q], u[m], s);
                                    w[q] = s;
                                }
#pragma unroll
                                for (int q = 0; q < 16; ++q) RR[q * NP + c] -= w[q];
                            } else {
#pragma unroll
                                for (int q = 0; q < 16; ++q) w[q] = 0.f;
                            }
                            const int nrow = c - trail0;
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4) {
                                const float4 v =
                                    make_float4(-w[4 * q4], -w[4 * q4 + 1], -w[4 * q4 + 2], -w[4 * q4 + 3]);
                                const uint32_t off = wq_off(nrow, 4 * q4);
                                *reinterpret_cast<float4*>(sm + M::oWsH + off) = v;
                                if (split)
                                    *reinterpret_cast<float4*>(sm + M::oWsL + off) = make_float4(
                                        tc::tf32_lo(v.x), tc::tf32_lo(v.y), tc::tf32_lo(v.z), tc::tf32_lo(v.w));
                            }
                        }
                    }
                }
                tc::fence_async_smem();
                block_sync();

                // ---- 4. GEMM2: A(:, trail) += Y (-W), the tile in tensor memory as accumulator
                if (warp == 0) {
                    if (tc::elect_one()) {
                        const uint32_t idW = tc::instr_desc(2, 128, ntr);
                        const uint32_t d = tmem + M::cTile + (uint32_t)trail0;
#pragma unroll
                        for (int ks = 0; ks < kNB / 8; ++ks) {
                            const uint64_t wh = tc::smem_desc(sb + M::oWsH + 256u * ks, 128u, 512u);
                            const uint64_t wl = tc::smem_desc(sb + M::oWsL + 256u * ks, 128u, 512u);
                            const uint32_t yh = tmem + M::cYH + 8 * ks, yl = tmem + M::cYL + 8 * ks;
                            tc::mma_tf32_ts(d, yh, wh, idW, true);
                            if (split) {
                                tc::mma_tf32_ts(d, yh, wl, idW, true);
                                tc::mma_tf32_ts(d, yl, wh, idW, true);
                            }
                        }
                        tc::mma_commit(&bar[2]);
                    }
                    __syncwarp();
                }
            }
            // ---- the panel's rows of R back to the stream's slot
            for (int e = t; e < kNB * NP; e += kRows) {
                const int q = e / NP, c = e - q * NP;
                if (j0 + q < n && c >= j0 && c < n) Rg[(size_t)(j0 + q) * n + c] = RR[e];
            }
            if (ntr > 0 && !wait_bar(2)) {
                dead = true;
                break;
            }
            __syncthreads();
        }
        if (dead) break;

        // ---- projection partials -> binary64
        if (KP > 0 && k > 0 && (++since_flush == kFlushTiles || tile + 1 == ntiles)) {
#pragma unroll
            for (int lb = 0; lb < LB; ++lb) {
                if (128 * lb + 32 * warp < n) {
#pragma unroll
                    for (int q0 = 0; q0 < (KP > 0 ? KP : 16); q0 += 16) {
                        float v[16];
                        tc::tmem_ld16(tq + M::cGX(lb) + q0, v);
                        const int c = 128 * lb + t;
                        if (c < n) {
                            double* gx = a.gx + (size_t)cta * k * n;
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (q0 + i < k) gx[(size_t)(q0 + i) * n + c] += (double)v[i];
                        }
                    }
                }
            }
            gx_fresh = true;
            since_flush = 0;
            block_sync();
        }
    }

    if (a.check && __any_sync(FULL, bad) && lane == 0) set_status(a.status, MRNMF_ERR_BAD_INPUT);
    if (a.cs) {
#pragma unroll
        for (int lb = 0; lb < LB; ++lb)
            if (128 * lb + t < n) a.cs[(size_t)cta * n + 128 * lb + t] += cs_acc[lb];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, M::cols);
}

template <int NP, int KP>
cudaError_t launch_np_kp(const LeafArgs& a, int grid, cudaStream_t s)
{
    auto kern = tsqr_wy_kernel<NP, KP>;
    const int bytes = (int)WyMap<NP, KP>::alloc;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, kRows, bytes, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_np(const LeafArgs& a, int kp, int grid, cudaStream_t s)
{
    switch (kp) {
    case 0: return launch_np_kp<NP, 0>(a, grid, s);
    case 16: return launch_np_kp<NP, 16>(a, grid, s);
    case 32: return launch_np_kp<NP, 32>(a, grid, s);
    default: return launch_np_kp<NP, 48>(a, grid, s);
    }
}

int kp_for(int k) { return k == 0 ? 0 : k <= 16 ? 16 : k <= 32 ? 32 : 48; }

}  // namespace

bool tc_supported(int n, int k) { return n > kNB && n <= 256 && k >= 0 && k <= (n <= 64 ? 32 : 48); }

bool tc_preferred(int n, int k)
{
    (void)n;
    (void)k;
    return false;
}

int tc_leaf_rows_per_tile() { return kRows; }

int tc_leaf_ctas_per_sm(int n) { return n <= 64 ? 2 : 1; }

cudaError_t launch_tc_leaf(const LeafArgs& a, int grid, cudaStream_t s)
{
    const int k = a.gx ? a.k : 0;
    if (!tc_supported(a.n, k)) return cudaErrorInvalidValue;
    const int kp = kp_for(k);
    if (a.n <= 64) return kp <= 16 ? (kp == 0 ? launch_np_kp<64, 0>(a, grid, s) : launch_np_kp<64, 16>(a, grid, s))
                                   : launch_np_kp<64, 32>(a, grid, s);
    if (a.n <= 128) return launch_np<128>(a, kp, grid, s);
    return launch_np<256>(a, kp, grid, s);
}

}  // namespace mrnmf
