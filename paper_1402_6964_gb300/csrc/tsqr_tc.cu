// tsqr_tc.cu -- the pass over X with the trailing updates of the leaf QR on
// the tensor cores (tcgen05, three-pass TF32 products with FP32 accumulation),
// for 16 < n <= 64.
//
// One CTA of 128 threads per row stream.  The stream's running triangle R
// (binary32, 64 x 64 padded) stays in shared memory; each 128-row tile A of X
// sits in tensor memory, lane t = tile row t.  The tile is folded into R by
// the blocked Householder QR of the stacked [R; A] (the local QR of Sec. 3.1)
// in compact-WY form (Schreiber and Van Loan, SIAM J. Sci. Stat. Comput. 10,
// 1989), one 16-column panel P = j0 .. j0+15 at a time:
//
//   1. the panel of [R; A] is factored on the SIMT cores with reflectors
//      v_q = [e_(j0+q); y_q] (y_q has 128 entries, one per tile row): the
//      same column step as the SIMT leaves (beta = -sign(alpha) sqrt(alpha^2 +
//      sigma), y = A(:,j) / (alpha - beta), tau = (beta - alpha) / beta); the
//      dot products that finished columns compute anyway are the Gram Y'Y;
//   2. T (16 x 16, upper triangular, Q_P = I - V T V') by the forward
//      recurrence T(0:q, q) = -tau_q T(0:q, 0:q) Y(:, 0:q)' y_q;
//   3. Z = Y' A(:, trail)                          tcgen05 GEMM1 (K = 128)
//   4. W = T' (R(P, trail) + Z), R(P, trail) -= W  SIMT, one thread per column
//   5. A(:, trail) -= Y W                          tcgen05 GEMM2, into TMEM
//
// The Gaussian projection of the same tile (Algorithm 1 with the combiner of
// Sec. 3.2) is one more tcgen05 GEMM per tile, X' G; the column sums (the
// scaling D of Sec. 2.3) are summed on the SIMT cores from the staged X'
// (exactly, hi + lo).  Both are kept in binary32 registers across tiles and
// flushed to the binary64 partial sums every kFlushTiles tiles.
//
// Every product is split as x = hi + lo (hi exact in TF32) and formed as
// hi*hi + hi*lo + lo*hi.  The tensor core's binary32 accumulation truncates
// the aligned addends, so the GEMMs carry about 20 bits, not 24: enough for
// the updates of the QR and for GX, not for the column sums.
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "leaf.h"
#include "tc_common.cuh"

namespace mrnmf {

namespace {

constexpr int kRows = 128;       // tile height = TMEM lanes = threads
constexpr int kNB = 16;          // panel width
constexpr int kNP = 64;          // padded column count of this kernel
constexpr int kFlushTiles = 32;  // tiles between binary64 flushes of the projection
constexpr int kPld = 17;         // row stride (floats) of the panel buffer

// Operands with K = tile row (X', Y', G'): 16-byte chunks of 4 tile rows; a
// 16-byte pad after every 128 bytes (LBO = 144) puts the 32 tile rows of a
// warp in 32 distinct banks when each thread writes its own row's element.
constexpr uint32_t kLboT = 144, kSboT = 32 * kLboT;  // 8-row group: 4608 B
// Operands with K = reflector index (Y, W): 16 deep, LBO 128, SBO 512.
constexpr uint32_t kLboQ = 128, kSboQ = 512;

// Shared-memory map (bytes).
constexpr uint32_t kOpT64 = (kNP / 8) * kSboT;           // 64 rows of a K = 128 operand
constexpr uint32_t kOffAhi = 0;                          // X' / A(:, trail)'
constexpr uint32_t kOffAlo = kOffAhi + kOpT64;
constexpr uint32_t kOffGY = kOffAlo + kOpT64;            // G' (hi, lo), later Y' (hi, lo) and W
constexpr uint32_t kGYBytes = 2 * (32 / 8) * kSboT;
constexpr uint32_t kOffYcHi = kOffGY;
constexpr uint32_t kOffYcLo = kOffGY + 2 * kSboT;
constexpr uint32_t kWBytes = ((kNP - kNB) / 8) * kSboQ;
constexpr uint32_t kOffWhi = kOffGY + 4 * kSboT;
constexpr uint32_t kOffWlo = kOffWhi + kWBytes;
constexpr uint32_t kYrBytes = (kRows / 8) * kSboQ;
constexpr uint32_t kOffYrHi = kOffGY + kGYBytes;         // Y (hi, lo), rows = tile rows
constexpr uint32_t kOffYrLo = kOffYrHi + kYrBytes;
constexpr uint32_t kOffR = kOffYrLo + kYrBytes;          // R, 64 x 64 row-major
constexpr uint32_t kOffP = kOffR + 4 * kNP * kNP;        // panel, 128 x 17
constexpr uint32_t kOffT = kOffP + 4 * kRows * kPld;     // T, 16 x 17
constexpr uint32_t kOffGy = kOffT + 4 * kNB * kPld;      // Y'Y, 16 x 17
constexpr uint32_t kOffTau = kOffGy + 4 * kNB * kPld;
constexpr uint32_t kOffRed = kOffTau + 4 * kNB;          // [2][4 warps][16]
constexpr uint32_t kOffPub = kOffRed + 4 * 2 * 4 * kNB;  // [4 warps][2 halves][16]
constexpr uint32_t kOffBar = kOffPub + 4 * 4 * 2 * kNB;  // two mbarriers
constexpr uint32_t kOffSlot = kOffBar + 16;
constexpr uint32_t kSmemBytes = kOffSlot + 16;
static_assert(kOffWlo + kWBytes <= kOffGY + kGYBytes, "W must fit in the G region");
static_assert(kOffBar % 16 == 0 && kOffPub % 16 == 0, "alignment");
// An M = 128 MMA reads 128 operand rows although only npad <= 64 hold data;
// the extra rows are read from the buffers that follow (their D lanes are
// never used), so 16 groups from the highest operand base must stay inside
// the allocation: A(lo) + 2 groups (first panel) + 16 groups.
static_assert(kOffAlo + 2 * kSboT + 16 * kSboT <= kSmemBytes, "operand over-read leaves the allocation");

// TMEM columns.
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kColZ = 64;   // GEMM1 result (lane = trailing column), 16 columns
constexpr uint32_t kColGX = 96;  // X' G of one tile (lane = column of X), up to 32 columns

__device__ __forceinline__ uint32_t offT(int row, int t)  // element (row, K = tile row t)
{
    return (uint32_t)(row >> 3) * kSboT + (uint32_t)(t >> 2) * kLboT + (uint32_t)(row & 7) * 16u + (uint32_t)(t & 3) * 4u;
}
__device__ __forceinline__ uint32_t offQ(int row, int q4)  // 16-byte chunk (row, K = 4 q4 .. 4 q4 + 3)
{
    return (uint32_t)(row >> 3) * kSboQ + (uint32_t)q4 * kLboQ + (uint32_t)(row & 7) * 16u;
}

__device__ __forceinline__ void put_split(unsigned char* sm, uint32_t hi_off, uint32_t lo_off, uint32_t off, float v)
{
    float h, l;
    tc::split_tf32(v, h, l);
    *reinterpret_cast<float*>(sm + hi_off + off) = h;
    *reinterpret_cast<float*>(sm + lo_off + off) = l;
}
__device__ __forceinline__ void put_split4(unsigned char* sm, uint32_t hi_off, uint32_t lo_off, uint32_t off, float a,
                                           float b, float c, float d)
{
    float ha, la, hb, lb, hc, lc, hd, ld;
    tc::split_tf32(a, ha, la);
    tc::split_tf32(b, hb, lb);
    tc::split_tf32(c, hc, lc);
    tc::split_tf32(d, hd, ld);
    *reinterpret_cast<float4*>(sm + hi_off + off) = make_float4(ha, hb, hc, hd);
    *reinterpret_cast<float4*>(sm + lo_off + off) = make_float4(la, lb, lc, ld);
}

// D += A B' in three TF32 passes, K = 8 * ksteps, both operands K-major.
__device__ __forceinline__ void mma3(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                     uint32_t lbo_a, uint32_t sbo_a, uint32_t lbo_b, uint32_t sbo_b, int ksteps,
                                     uint32_t idesc, bool accumulate)
{
    for (int ks = 0; ks < ksteps; ++ks) {
        const uint32_t ka = (uint32_t)ks * 2u * lbo_a, kb = (uint32_t)ks * 2u * lbo_b;
        const uint64_t ah = tc::smem_desc(a_hi + ka, lbo_a, sbo_a), al = tc::smem_desc(a_lo + ka, lbo_a, sbo_a);
        const uint64_t bh = tc::smem_desc(b_hi + kb, lbo_b, sbo_b), bl = tc::smem_desc(b_lo + kb, lbo_b, sbo_b);
        tc::mma_tf32(d, ah, bh, idesc, accumulate || ks > 0);
        tc::mma_tf32(d, ah, bl, idesc, true);
        tc::mma_tf32(d, al, bh, idesc, true);
    }
}

// Householder steps of one 16-column panel of [R; A] (R rows/columns j0..,
// A = the panel buffer, 128 x 16), all four warps: lane (c, h) of warp w holds
// column c of tile rows 32w + 16h .. +15.  On return the panel buffer holds
// Y, R(P, P) is updated, tau and the strict upper triangle of Y'Y are set.
// One block barrier per column.
__device__ __forceinline__ void panel_steps(float* Pb, float* R, int j0, float* red, float* pub, float* Gy, float* tau,
                                            int warp, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const int c = lane & 15, h = lane >> 4;
    const int tb = 32 * warp + 16 * h;
    const bool writer = warp == 0 && h == 0;
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = Pb[(tb + i) * kPld + c];
    float4* mypub = reinterpret_cast<float4*>(pub + (warp * 2 + h) * kNB);
    for (int j = 0; j < kNB; ++j) {
        if (c == j) {
#pragma unroll
            for (int i4 = 0; i4 < 4; ++i4) mypub[i4] = make_float4(a[4 * i4], a[4 * i4 + 1], a[4 * i4 + 2], a[4 * i4 + 3]);
        }
        const float alpha = R[(j0 + j) * kNP + j0 + j];
        const float rjc = R[(j0 + j) * kNP + j0 + c];
        __syncwarp();
        float pv[16];
#pragma unroll
        for (int i4 = 0; i4 < 4; ++i4) {
            const float4 v = mypub[i4];
            pv[4 * i4] = v.x;
            pv[4 * i4 + 1] = v.y;
            pv[4 * i4 + 2] = v.z;
            pv[4 * i4 + 3] = v.w;
        }
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
            g0 = fmaf(pv[i], a[i], g0);
            g1 = fmaf(pv[i + 1], a[i + 1], g1);
            g2 = fmaf(pv[i + 2], a[i + 2], g2);
            g3 = fmaf(pv[i + 3], a[i + 3], g3);
        }
        float g = (g0 + g1) + (g2 + g3);
        g += __shfl_xor_sync(FULL, g, 16);
        float* rj = red + (j & 1) * 4 * kNB;
        if (h == 0) rj[warp * kNB + c] = g;
        __syncthreads();
        const float gs = (rj[c] + rj[kNB + c]) + (rj[2 * kNB + c] + rj[3 * kNB + c]);
        const float sig = __shfl_sync(FULL, gs, j);
        if (sig > 0.f) {
            const HhScalars hs = hh_scalars(alpha, sig);
            const float beta = hs.beta, d = hs.d, rb = hs.rb, rd = hs.rd;
            if (c > j) {
                const float wp = fmaf(d, rjc, gs);  // d (R_jc + g_c / d)
                const float f = (wp * rd) * rb;
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] = fmaf(f, pv[i], a[i]);
                if (writer) R[(j0 + j) * kNP + j0 + c] = fmaf(wp, rb, rjc);
            } else if (c == j) {
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] *= rd;  // y_j = A(:,j) / (alpha - beta)
                if (writer) {
                    R[(j0 + j) * kNP + j0 + j] = beta;
                    tau[j] = -d * rb;
                }
            } else if (writer) {
                Gy[c * kPld + j] = gs * rd;  // y_c' y_j
            }
        } else if (writer) {
            // nothing below R_jj: the identity (tau = 0)
            if (c == j) tau[j] = 0.f;
            if (c < j) Gy[c * kPld + j] = 0.f;
        }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) Pb[(tb + i) * kPld + c] = a[i];
}

template <int KP>
__global__ void __launch_bounds__(kRows, 1) tsqr_tc_kernel(const LeafArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const unsigned FULL = 0xffffffffu;
    const int n = a.n, npad = (n + 15) & ~15;
    const int k = (KP > 0 && a.gx) ? a.k : 0;  // Gaussian columns
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int cta = blockIdx.x;
    float* R = reinterpret_cast<float*>(sm + kOffR);
    float* Pb = reinterpret_cast<float*>(sm + kOffP);
    float* Ts = reinterpret_cast<float*>(sm + kOffT);
    float* Gy = reinterpret_cast<float*>(sm + kOffGy);
    float* tau = reinterpret_cast<float*>(sm + kOffTau);
    float* red = reinterpret_cast<float*>(sm + kOffRed);
    float* pub = reinterpret_cast<float*>(sm + kOffPub);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);  // [0]: projection GEMM, [1]: GEMM1 / GEMM2
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kOffSlot);
    const uint32_t sbase = tc::smem_addr(sm);

    {
        const float* Rin = static_cast<const float*>(a.R_in);
        for (int e = t; e < kNP * kNP; e += kRows) {
            const int j = e / kNP, c = e - j * kNP;
            R[e] = (Rin && j < n && c < n && c >= j) ? Rin[(size_t)cta * n * n + j * n + c] : 0.f;
        }
    }
    if (t == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(slot, kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's lane quadrant

    const int64_t r0 = (int64_t)cta * a.rows_per_cta;
    const int64_t r1 = min(a.rows, r0 + a.rows_per_cta);
    const int64_t ntiles = r1 > r0 ? (r1 - r0 + kRows - 1) / kRows : 0;
    const float* X = static_cast<const float*>(a.X);
    uint32_t ph_gx = 0, ph_mma = 0;
    bool bad = false, dead = false;
    int since_flush = 0;
    float cs_acc = 0.f, gx_acc[KP > 0 ? KP : 1];
#pragma unroll
    for (int q = 0; q < (KP > 0 ? KP : 1); ++q) gx_acc[q] = 0.f;

    // Bounded wait on an MMA commit, block-uniform outcome.
    auto wait_mma = [&](int b, uint32_t& ph) -> bool {
        bool ok = tc::mbar_wait(&bar[b], ph);
        if (!ok) tc::mbar_wait(&bar[b], ph);  // a second bounded wait for the MMAs in flight
        ph ^= 1u;
        tc::fence_after_sync();
        if (__syncthreads_or(!ok)) {
            if (t == 0) set_status(a.status, MRNMF_ERR_TIMEOUT);
            return false;
        }
        return true;
    };

    for (int64_t tile = 0; tile < ntiles && !dead; ++tile) {
        const int64_t row = r0 + tile * kRows + t;
        const bool valid = row < r1;
        float x[kNP];
        {
            const float* src = X + (valid ? row : r0) * a.ldx;
#pragma unroll
            for (int c = 0; c < kNP; ++c) x[c] = (valid && c < n) ? __ldg(src + c) : 0.f;
        }
#pragma unroll
        for (int c = 0; c < kNP; ++c) bad |= !(x[c] >= 0.f);
        // the tile into TMEM (lane t = row t), X' into the K = tile-row operand
#pragma unroll
        for (int c0 = 0; c0 < kNP; c0 += 16) tc::tmem_st16(tl + c0, &x[c0]);
        tc::tmem_wait_st();
#pragma unroll
        for (int c = 0; c < kNP; ++c)
            if (c < npad) put_split(sm, kOffAhi, kOffAlo, offT(c, t), x[c]);
        // G' rows (Algorithm 1: g_i ~ N(0, I_k) keyed by the global row)
        if (KP > 0) {
            const int64_t grow = a.row_base + row;
#pragma unroll
            for (int q4 = 0; q4 < KP / 4; ++q4) {
                float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid && 4 * q4 < k) g = gauss4(a.seed, grow, (uint32_t)q4);
                const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int q = 4 * q4 + i;
                    put_split(sm, kOffGY, kOffGY + (KP / 8) * kSboT, offT(q, t), q < k ? gv[i] : 0.f);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kNB; ++q) Pb[t * kPld + q] = x[q];
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (KP > 0 && t == 0) {
            // this tile's GX': D[c][q] = sum_t X[t][c] G[t][q]
            mma3(tmem + kColGX, sbase + kOffAhi, sbase + kOffAlo, sbase + kOffGY,
                 sbase + kOffGY + (KP / 8) * kSboT, kLboT, kSboT, kLboT, kSboT, kRows / 8,
                 tc::instr_desc(2, 128, KP), false);
            tc::mma_commit(&bar[0]);
        }
        // column sums of the tile from the staged X' (thread c sums column c: hi + lo = x exactly)
        if (t < n) {
            float s0 = 0.f, s1 = 0.f;
            const unsigned char* ch = sm + kOffAhi + (uint32_t)(t >> 3) * kSboT + (uint32_t)(t & 7) * 16u;
#pragma unroll 8
            for (int r4 = 0; r4 < kRows / 4; ++r4) {
                const float4 h4 = *reinterpret_cast<const float4*>(ch + r4 * kLboT);
                const float4 l4 = *reinterpret_cast<const float4*>(ch + (kOffAlo - kOffAhi) + r4 * kLboT);
                s0 += (h4.x + l4.x) + (h4.y + l4.y);
                s1 += (h4.z + l4.z) + (h4.w + l4.w);
            }
            cs_acc += s0 + s1;
        }

        for (int p = 0; p < npad / kNB; ++p) {
            const int j0 = kNB * p;
            const int ntrail = npad - j0 - kNB;
            __syncthreads();
            panel_steps(Pb, R, j0, red, pub, Gy, tau, warp, lane);
            __syncthreads();
            float y[kNB];
#pragma unroll
            for (int q = 0; q < kNB; ++q) y[q] = Pb[t * kPld + q];
            if (KP > 0 && p == 0) {  // Y' overwrites G'; the tile's GX' is read out now
                if (!wait_mma(0, ph_gx)) {
                    dead = true;
                    break;
                }
                if (warp * 32 < n) {
                    float v[16];
                    tc::tmem_ld16(tl + kColGX, v);
#pragma unroll
                    for (int q = 0; q < 16; ++q) gx_acc[q] += v[q];
                    if (KP > 16) {
                        tc::tmem_ld16(tl + kColGX + 16, v);
#pragma unroll
                        for (int q = 0; q < 16; ++q) gx_acc[(KP > 16 ? 16 : 0) + q] += v[q];
                    }
                }
            }
            if (ntrail > 0) {
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4)
                    put_split4(sm, kOffYrHi, kOffYrLo, offQ(t, q4), y[4 * q4], y[4 * q4 + 1], y[4 * q4 + 2],
                               y[4 * q4 + 3]);
#pragma unroll
                for (int q = 0; q < kNB; ++q) put_split(sm, kOffYcHi, kOffYcLo, offT(q, t), y[q]);
                if (warp == 0 && lane < kNB) {
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
                                if (m >= i) s = fmaf(Ti[m], Gy[m * kPld + q], s);
                            v = -tau[q] * s;
                        }
                        Ti[q] = v;
                    }
#pragma unroll
                    for (int q = 0; q < kNB; ++q) Ts[i * kPld + q] = Ti[q];
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                if (t == 0) {
                    // GEMM1: Z[c'][q] = sum_t A[t][j0+16+c'] y_q[t]; on the first
                    // panel the trailing columns are rows 16.. of X'
                    const uint32_t aoff = p == 0 ? 2 * kSboT : 0;
                    mma3(tmem + kColZ, sbase + kOffAhi + aoff, sbase + kOffAlo + aoff, sbase + kOffYcHi,
                         sbase + kOffYcLo, kLboT, kSboT, kLboT, kSboT, kRows / 8, tc::instr_desc(2, 128, kNB), false);
                    tc::mma_commit(&bar[1]);
                }
                if (!wait_mma(1, ph_mma)) {
                    dead = true;
                    break;
                }
                // W = T' (R(P, trail) + Z); R(P, trail) -= W; stage -W (row c', K = q)
                if (warp * 32 < ntrail) {
                    float z[kNB];
                    tc::tmem_ld16(tl + kColZ, z);
                    if (t < ntrail) {
                        const int c = j0 + kNB + t;
                        float u[kNB], w[kNB];
#pragma unroll
                        for (int q = 0; q < kNB; ++q) u[q] = R[(j0 + q) * kNP + c] + z[q];
#pragma unroll
                        for (int q = 0; q < kNB; ++q) {
                            float s = 0.f;
#pragma unroll
                            for (int m = 0; m <= q; ++m) s = fmaf(Ts[m * kPld + q], u[m], s);
                            w[q] = s;
                        }
#pragma unroll
                        for (int q = 0; q < kNB; ++q) R[(j0 + q) * kNP + c] -= w[q];
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4)
                            put_split4(sm, kOffWhi, kOffWlo, offQ(t, q4), -w[4 * q4], -w[4 * q4 + 1], -w[4 * q4 + 2],
                                       -w[4 * q4 + 3]);
                    }
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                if (t == 0) {
                    // GEMM2: A[t][j0+16+c'] += sum_q y_q[t] (-W)[q][c']
                    mma3(tmem + (uint32_t)(j0 + kNB), sbase + kOffYrHi, sbase + kOffYrLo, sbase + kOffWhi,
                         sbase + kOffWlo, kLboQ, kSboQ, kLboQ, kSboQ, kNB / 8, tc::instr_desc(2, 128, ntrail), true);
                    tc::mma_commit(&bar[1]);
                }
                if (!wait_mma(1, ph_mma)) {
                    dead = true;
                    break;
                }
                // next panel -> panel buffer; the columns after it -> rows 0.. of the A' operand
                for (int c0 = j0 + kNB; c0 < npad; c0 += kNB) {
                    float v[kNB];
                    tc::tmem_ld16(tl + (uint32_t)c0, v);
                    if (c0 == j0 + kNB) {
#pragma unroll
                        for (int q = 0; q < kNB; ++q) Pb[t * kPld + q] = v[q];
                    } else {
                        const int rb = c0 - (j0 + 2 * kNB);
#pragma unroll
                        for (int q = 0; q < kNB; ++q) put_split(sm, kOffAhi, kOffAlo, offT(rb + q, t), v[q]);
                    }
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
            }
        }
        if (dead) break;

        // projection / column-sum partials -> binary64
        if (++since_flush == kFlushTiles || tile + 1 == ntiles) {
            if (t < n) {
                if (a.cs) a.cs[(size_t)cta * n + t] += (double)cs_acc;
                if (k > 0) {
                    double* gx = a.gx + (size_t)cta * k * n;
#pragma unroll
                    for (int q = 0; q < (KP > 0 ? KP : 1); ++q) {
                        if (q < k) gx[(size_t)q * n + t] += (double)gx_acc[q];
                        gx_acc[q] = 0.f;
                    }
                }
            }
            cs_acc = 0.f;
            since_flush = 0;
        }
    }

    if (a.check && __any_sync(FULL, bad) && lane == 0) set_status(a.status, MRNMF_ERR_BAD_INPUT);
    __syncthreads();
    {
        float* Rout = static_cast<float*>(a.R_out) + (size_t)cta * n * n;
        for (int e = t; e < n * n; e += kRows) {
            const int j = e / n, c = e - j * n;
            Rout[e] = c >= j ? R[j * kNP + c] : 0.f;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int KP>
cudaError_t launch_kp(const LeafArgs& a, int grid, cudaStream_t s)
{
    auto kern = tsqr_tc_kernel<KP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, kRows, kSmemBytes, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

bool tc_supported(int n, int k) { return n > kNB && n <= kNP && k >= 0 && k <= 32; }

bool tc_preferred(int n, int k)
{
    (void)n;
    (void)k;
    return false;
}

int tc_leaf_rows_per_tile() { return kRows; }

int tc_leaf_ctas_per_sm() { return 1; }

cudaError_t launch_tc_leaf(const LeafArgs& a, int grid, cudaStream_t s)
{
    const int k = a.gx ? a.k : 0;
    if (!tc_supported(a.n, k)) return cudaErrorInvalidValue;
    if (k == 0) return launch_kp<0>(a, grid, s);
    return k <= 16 ? launch_kp<16>(a, grid, s) : launch_kp<32>(a, grid, s);
}

}  // namespace mrnmf
