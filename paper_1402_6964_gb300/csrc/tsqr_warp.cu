// tsqr_warp.cu -- the pass over X for n <= 64 in binary32: one warp per row
// stream (Sec. 3.5's map task), no block-wide barriers.
//
// Layout.  Lane l owns columns l and l+32 of the stream's tiles: the L rows of
// those columns sit in its registers, so every reflector dot product is a
// lane-local sum.  The stream's running triangle R (packed upper, binary32)
// lives in the warp's slice of shared memory.  Tiles of L consecutive rows are
// staged into shared memory by the TMA bulk-copy engine (cp.async.bulk with an
// mbarrier) one tile ahead of the arithmetic, then moved to registers.
//
// Column step j on the stacked [R; A] (A = tile): the owner of column j
// publishes the column's raw values in shared memory; every lane forms
// g_c = A(:,j)' A(:,c) for its columns c >= j in one loop (g_j is the squared
// norm sigma); then, with alpha = R_jj, beta = -sign(alpha) sqrt(alpha^2 +
// sigma), s = 1/(alpha - beta), tau = (beta - alpha)/beta (the reflector
// v = [e_j; s A(:,j)]), each column c > j gets w = R_jc + s g_c,
// R_jc -= tau w, A(:,c) -= (tau w s) A(:,j) (evaluated with reciprocals of
// beta and alpha - beta, since tau s = -1/beta).  The owner of column j+1 then
// publishes its updated column.  One warp barrier per column, no block
// barriers, no cross-lane reductions except the broadcast of sigma.
// Once at most 16 (8) columns of a tile remain, two (four) lanes share each
// column by rows, and xor shuffles sum the parts of its dot products.
//
// Column sums and the Gaussian projection (Algorithm 1, with the combiner of
// Sec. 3.2) are folded into the same pass: binary32 per tile, binary64 across
// tiles.
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "leaf.h"

namespace mrnmf {

namespace {

constexpr int kWarps = 4;  // streams per CTA
constexpr int kFlush = 32;  // tiles between binary64 flushes of the partial sums

// Tile heights: by default 64 rows when a lane owns one column (n <= 32), 32
// rows when it owns two (n <= 64); leaf_rows() below says what can change that.

__host__ __device__ inline int pk_row(int j, int n) { return j * n - (j * (j + 1)) / 2; }
__host__ __device__ inline size_t up(size_t b, size_t a) { return (b + a - 1) / a * a; }

// Per-warp shared-memory slice: [mbarrier | tile L*n | R packed | pub 2L | gbuf kp*L | gxs kp*n]
template <int L>
__host__ __device__ inline size_t warp_slice_bytes(int n, int k)
{
    const int kp = (k + 3) & ~3;
    size_t b = 128;                                   // mbarrier (own 128 B so the tile is 128-aligned)
    b += up(sizeof(float) * (size_t)L * n, 128);      // tile
    b += up(sizeof(float) * (size_t)(n * (n + 1) / 2), 16);
    b += sizeof(float) * 2 * L;                       // published column, double buffer
    b += sizeof(float) * (size_t)kp * L;              // Gaussian tile, coordinate-major
    b += sizeof(float) * (size_t)kp * n;              // projection accumulators
    return up(b, 128);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase `parity` to complete; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

// Column steps j .. jend-1 in a split form: the 32 / G columns jbase + q are
// each held by G lanes q + (32 / G) g, lane g owning rows [g L/G, (g+1) L/G)
// of the tile in a0[0 .. L/G).  Same arithmetic as the one-column steps;
// the G parts of each dot product are summed by xor shuffles.
template <int L, int G>
__device__ __forceinline__ void split_steps(float (&a0)[L], float* Rw, float* pub, int n, int lane, int& j, int jend,
                                            int jbase)
{
    const unsigned FULL = 0xffffffffu;
    constexpr int QN = 32 / G, LG = L / G;
    const int g = lane / QN, q = lane % QN;
    const int cq = jbase + q;
    const bool oq = cq < n;
    for (; j < jend; ++j) {
        const float4* pj = reinterpret_cast<const float4*>(pub + (j & 1) * L + g * LG);
        const int pr = pk_row(j, n);
        const float alpha = Rw[pr + j];
        const float rq = oq ? Rw[pr + cq] : 0.f;
        constexpr bool kPivReg = LG <= 32;
        float4 pv[kPivReg ? LG / 4 : 1];
        float g0a = 0.f, g0b = 0.f, g0c = 0.f, g0d = 0.f;
#pragma unroll
        for (int l4 = 0; l4 < LG / 4; ++l4) {
            const float4 v = pj[l4];
            if (kPivReg) pv[kPivReg ? l4 : 0] = v;
            g0a = fmaf(v.x, a0[4 * l4], g0a);
            g0b = fmaf(v.y, a0[4 * l4 + 1], g0b);
            g0c = fmaf(v.z, a0[4 * l4 + 2], g0c);
            g0d = fmaf(v.w, a0[4 * l4 + 3], g0d);
        }
        float g0 = (g0a + g0b) + (g0c + g0d);
#pragma unroll
        for (int o = QN; o < 32; o <<= 1) g0 += __shfl_xor_sync(FULL, g0, o);
        const float sig = __shfl_sync(FULL, g0, j - jbase);
        __syncwarp();
        float beta = alpha;
        if (sig > 0.f) {
            const HhScalars hs = hh_scalars(alpha, sig);
            beta = hs.beta;
            const float d = hs.d, rb = hs.rb, rd = hs.rd;
            float f0 = 0.f;
            if (oq && cq > j) {
                const float wp = fmaf(d, rq, g0);
                f0 = (wp * rd) * rb;
                if (g == 0) Rw[pr + cq] = fmaf(wp, rb, rq);
            }
#pragma unroll
            for (int l4 = 0; l4 < LG / 4; ++l4) {
                const float4 v = kPivReg ? pv[kPivReg ? l4 : 0] : pj[l4];
                a0[4 * l4] = fmaf(f0, v.x, a0[4 * l4]);
                a0[4 * l4 + 1] = fmaf(f0, v.y, a0[4 * l4 + 1]);
                a0[4 * l4 + 2] = fmaf(f0, v.z, a0[4 * l4 + 2]);
                a0[4 * l4 + 3] = fmaf(f0, v.w, a0[4 * l4 + 3]);
            }
        }
        if (lane == j - jbase) Rw[pr + j] = beta;
        const int jn = j + 1;
        if (jn < n && q == jn - jbase) {  // every part of the next pivot publishes
            float4* dst = reinterpret_cast<float4*>(pub + (jn & 1) * L + g * LG);
#pragma unroll
            for (int l4 = 0; l4 < LG / 4; ++l4)
                dst[l4] = make_float4(a0[4 * l4], a0[4 * l4 + 1], a0[4 * l4 + 2], a0[4 * l4 + 3]);
        }
        __syncwarp();
    }
}

// Householder column steps of the stacked [R; A] for one L-row tile A held in
// registers (a0: column lane, a1: column lane + 32): R (packed, the warp's
// shared memory) absorbs A; A is destroyed.  pub is the warp's 2L-float
// publication buffer.
template <int NC, int L>
__device__ __forceinline__ void column_steps(float (&a0)[L], float (&a1)[NC == 2 ? L : 1], float* Rw, float* pub,
                                             int n, int lane, bool own0, bool own1)
{
    const unsigned FULL = 0xffffffffu;
    const int c0 = lane, c1 = lane + 32;
    if (lane == 0) {
#pragma unroll
        for (int l4 = 0; l4 < L / 4; ++l4)
            reinterpret_cast<float4*>(pub)[l4] =
                make_float4(a0[4 * l4], a0[4 * l4 + 1], a0[4 * l4 + 2], a0[4 * l4 + 3]);
    }
    __syncwarp();
    // beta = -sign(alpha) sqrt(alpha^2 + sigma), d = alpha - beta.  With
    // w' = d R_jc + g_c (= d w), the reflector's action is
    // R_jc -= tau w  =  R_jc + w'/beta  and
    // A(:,c) -= tau s w A(:,j)  =  A(:,c) + (w'/d)(1/beta) A(:,j).
    // beta, d and the reciprocals come from hh_scalars, accurate to the last
    // bit (measured: R error 13x larger with the raw SFU approximations at
    // 1e7 x 50).
    int j = 0;
    if (NC == 2) {
        // two live columns per lane while more than 32 columns remain (j < n - 32 <= 32)
        const int jm = n - 32;
        for (; j < jm; ++j) {
            const float4* pj = reinterpret_cast<const float4*>(pub + (j & 1) * L);
            // row j of R: only this step writes it, so it is read before the dot
            // (off the step's critical path)
            const int pr = pk_row(j, n);
            const float alpha = Rw[pr + j];
            const float r0v = own0 ? Rw[pr + c0] : 0.f, r1v = own1 ? Rw[pr + c1] : 0.f;
            float g0a = 0.f, g0b = 0.f, g0c = 0.f, g0d = 0.f, g1a = 0.f, g1b = 0.f, g1c = 0.f, g1d = 0.f;
#pragma unroll
            for (int l4 = 0; l4 < L / 4; ++l4) {
                const float4 v = pj[l4];
                g0a = fmaf(v.x, a0[4 * l4], g0a);
                g0b = fmaf(v.y, a0[4 * l4 + 1], g0b);
                g0c = fmaf(v.z, a0[4 * l4 + 2], g0c);
                g0d = fmaf(v.w, a0[4 * l4 + 3], g0d);
                g1a = fmaf(v.x, a1[4 * l4], g1a);
                g1b = fmaf(v.y, a1[4 * l4 + 1], g1b);
                g1c = fmaf(v.z, a1[4 * l4 + 2], g1c);
                g1d = fmaf(v.w, a1[4 * l4 + 3], g1d);
            }
            const float g0 = (g0a + g0b) + (g0c + g0d), g1 = (g1a + g1b) + (g1c + g1d);
            const float sig = __shfl_sync(FULL, g0, j);
            __syncwarp();
            float beta = alpha;
            if (sig > 0.f) {
                const HhScalars hs = hh_scalars(alpha, sig);
                beta = hs.beta;
                const float d = hs.d, rb = hs.rb, rd = hs.rd;
                float f0 = 0.f, f1 = 0.f;
                if (own0 && c0 > j) {
                    const float wp = fmaf(d, r0v, g0);
                    f0 = (wp * rd) * rb;
                    Rw[pr + c0] = fmaf(wp, rb, r0v);
                }
                if (own1) {
                    const float wp = fmaf(d, r1v, g1);
                    f1 = (wp * rd) * rb;
                    Rw[pr + c1] = fmaf(wp, rb, r1v);
                }
#pragma unroll
                for (int l4 = 0; l4 < L / 4; ++l4) {
                    const float4 v = pj[l4];
                    a0[4 * l4] = fmaf(f0, v.x, a0[4 * l4]);
                    a0[4 * l4 + 1] = fmaf(f0, v.y, a0[4 * l4 + 1]);
                    a0[4 * l4 + 2] = fmaf(f0, v.z, a0[4 * l4 + 2]);
                    a0[4 * l4 + 3] = fmaf(f0, v.w, a0[4 * l4 + 3]);
                    a1[4 * l4] = fmaf(f1, v.x, a1[4 * l4]);
                    a1[4 * l4 + 1] = fmaf(f1, v.y, a1[4 * l4 + 1]);
                    a1[4 * l4 + 2] = fmaf(f1, v.z, a1[4 * l4 + 2]);
                    a1[4 * l4 + 3] = fmaf(f1, v.w, a1[4 * l4 + 3]);
                }
            }
            if (lane == j) Rw[pr + j] = beta;
            // the owner of column j+1 publishes its updated values
            const int jn = j + 1;
            if (lane == (jn & 31)) {
                float4* dst = reinterpret_cast<float4*>(pub + (jn & 1) * L);
                if (jn < 32) {
#pragma unroll
                    for (int l4 = 0; l4 < L / 4; ++l4)
                        dst[l4] = make_float4(a0[4 * l4], a0[4 * l4 + 1], a0[4 * l4 + 2], a0[4 * l4 + 3]);
                } else {
#pragma unroll
                    for (int l4 = 0; l4 < L / 4; ++l4)
                        dst[l4] = make_float4(a1[4 * l4], a1[4 * l4 + 1], a1[4 * l4 + 2], a1[4 * l4 + 3]);
                }
            }
            __syncwarp();
        }
        // from here on the live columns are jm .. jm+31, one per lane: the
        // lanes whose first column is finished move their second into slot 0
        if (lane < jm) {
#pragma unroll
            for (int l = 0; l < L; ++l) a0[l] = a1[l];
        }
    }
    const int cm = (NC == 2 && lane < n - 32) ? lane + 32 : lane;  // the lane's live column
    const bool om = NC == 2 ? true : own0;
    // one column per lane until at most 16 columns remain (the split form below)
    const int jsplit = n - 16 > j ? n - 16 : j;
    for (; j < jsplit; ++j) {
        const float4* pj = reinterpret_cast<const float4*>(pub + (j & 1) * L);
        const int pr = pk_row(j, n);
        const float alpha = Rw[pr + j];
        const float rmv = om ? Rw[pr + cm] : 0.f;
        // short tiles keep the pivot in registers for the update (one read of
        // the publication buffer per step instead of two)
        constexpr bool kPivReg = L <= 64;
        float4 pv[kPivReg ? L / 4 : 1];
        float g0a = 0.f, g0b = 0.f, g0c = 0.f, g0d = 0.f;
#pragma unroll
        for (int l4 = 0; l4 < L / 4; ++l4) {
            const float4 v = pj[l4];
            if (kPivReg) pv[kPivReg ? l4 : 0] = v;
            g0a = fmaf(v.x, a0[4 * l4], g0a);
            g0b = fmaf(v.y, a0[4 * l4 + 1], g0b);
            g0c = fmaf(v.z, a0[4 * l4 + 2], g0c);
            g0d = fmaf(v.w, a0[4 * l4 + 3], g0d);
        }
        const float g0 = (g0a + g0b) + (g0c + g0d);
        const float sig = __shfl_sync(FULL, g0, j & 31);
        __syncwarp();
        float beta = alpha;
        if (sig > 0.f) {
            const HhScalars hs = hh_scalars(alpha, sig);
            beta = hs.beta;
            const float d = hs.d, rb = hs.rb, rd = hs.rd;
            float f0 = 0.f;
            if (om && cm > j) {
                const float wp = fmaf(d, rmv, g0);
                f0 = (wp * rd) * rb;
                Rw[pr + cm] = fmaf(wp, rb, rmv);
            }
#pragma unroll
            for (int l4 = 0; l4 < L / 4; ++l4) {
                const float4 v = kPivReg ? pv[kPivReg ? l4 : 0] : pj[l4];
                a0[4 * l4] = fmaf(f0, v.x, a0[4 * l4]);
                a0[4 * l4 + 1] = fmaf(f0, v.y, a0[4 * l4 + 1]);
                a0[4 * l4 + 2] = fmaf(f0, v.z, a0[4 * l4 + 2]);
                a0[4 * l4 + 3] = fmaf(f0, v.w, a0[4 * l4 + 3]);
            }
        }
        if (lane == (j & 31)) Rw[pr + j] = beta;
        const int jn = j + 1;
        if (jn < n && lane == (jn & 31)) {
            float4* dst = reinterpret_cast<float4*>(pub + (jn & 1) * L);
#pragma unroll
            for (int l4 = 0; l4 < L / 4; ++l4)
                dst[l4] = make_float4(a0[4 * l4], a0[4 * l4 + 1], a0[4 * l4 + 2], a0[4 * l4 + 3]);
        }
        __syncwarp();
    }
    if (j >= n) return;
    // Split forms for the last columns: with at most 16 left, column
    // jsplit + q is held by lanes q and q + 16, each with half of the rows;
    // with at most 8 left, by lanes q + 8g (g = 0..3), each with a quarter.
    // A step then costs 1/2 (1/4) of the FMAs and pivot loads, and the parts
    // of each dot product are summed by xor shuffles.
    {
        // one column per lane -> halves: column c comes from lane (c & 31)
        const int hf = lane >> 4, cq = jsplit + (lane & 15);
        const int src = cq & 31;
#pragma unroll
        for (int i = 0; i < L / 2; ++i) {
            const float lo = __shfl_sync(FULL, a0[i], src);
            const float hi = __shfl_sync(FULL, a0[L / 2 + i], src);
            a0[i] = hf ? hi : lo;
        }
    }
    // quarters only pay with at least 16 rows per lane (measured: 2-13% faster
    // for the 64-row one-column form, 0.5-2% slower for 32-row tiles)
    const int jq = L < 64 ? n : (n - 8 > jsplit ? n - 8 : jsplit);
    split_steps<L, 2>(a0, Rw, pub, n, lane, j, jq, jsplit);
    if (L < 64 || j >= n) return;
    {
        // halves -> quarters: rows [gL/4, (g+1)L/4) of column jq + q sit in
        // half g/2 of that column, at offset (g & 1) L/4
        const int g = lane >> 3, cq = jq + (lane & 7);
        const int src = ((cq - jsplit) + 16 * (g >> 1)) & 31;
#pragma unroll
        for (int i = 0; i < L / 4; ++i) {
            const float v0 = __shfl_sync(FULL, a0[i], src);
            const float v1 = __shfl_sync(FULL, a0[L / 4 + i], src);
            a0[i] = (g & 1) ? v1 : v0;
        }
    }
    split_steps<L, 4>(a0, Rw, pub, n, lane, j, n, jq);
}

template <int NC, int L, bool GP>
__device__ __forceinline__ void warp_stream_body(const LeafArgs& a, const int cta)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int n = a.n;
    const int k = GP ? a.k : 0;
    const int kp = (k + 3) & ~3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ws = cta * kWarps + warp;  // stream id within the problem = partial-sum slot
    const unsigned FULL = 0xffffffffu;

    unsigned char* base = smem + (size_t)warp * warp_slice_bytes<L>(n, k);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base);
    float* tile = reinterpret_cast<float*>(base + 128);
    float* Rw = reinterpret_cast<float*>(base + 128 + up(sizeof(float) * (size_t)L * n, 128));
    float* pub = Rw + up((size_t)(n * (n + 1) / 2), 4);
    float* gbuf = pub + 2 * L;
    float* gxs = gbuf + (size_t)kp * L;

    const int c0 = lane, c1 = lane + 32;
    const bool own0 = c0 < n, own1 = NC == 2 && c1 < n;
    const uint32_t bar_s = smem_u32(bar);

    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // running triangle: warp 0 continues from the CTA's state slot (zeros on a
    // fresh pass), the other warps start from zero -- the CTA's streams are
    // folded into one triangle at the end of every launch
    {
        const float* Rin = static_cast<const float*>(a.R_in);
        const int nn = n * n;
        for (int e = lane; e < nn; e += 32) {
            const int j = e / n, c = e - j * n;
            if (c >= j) Rw[pk_row(j, n) + c] = (Rin && warp == 0) ? Rin[(size_t)cta * nn + e] : 0.f;
        }
        for (int e = lane; e < kp * n; e += 32) gxs[e] = 0.f;
    }
    __syncwarp();

    const int64_t r0 = (int64_t)ws * a.rows_per_cta;
    const int64_t r1 = min(a.rows, r0 + a.rows_per_cta);
    const int64_t ntiles = r1 > r0 ? (r1 - r0 + L - 1) / L : 0;
    const float* X = static_cast<const float*>(a.X);
    const bool tma_ok = a.ldx == n && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);

    // Issue the TMA copy of tile t into `tile`; false if it must be loaded directly.
    auto issue = [&](int64_t t) -> bool {
        const int64_t row0 = r0 + t * L;
        const int rows_v = (int)min((int64_t)L, r1 - row0);
        const uint32_t bytes = (uint32_t)rows_v * (uint32_t)n * 4u;
        if (!tma_ok || (bytes & 15u)) return false;
        if (lane == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(tile)),
                "l"(X + row0 * n), "r"(bytes), "r"(bar_s)
                : "memory");
        }
        return true;
    };

    float a0[L], a1[NC == 2 ? L : 1];
    float cs0 = 0.f, cs1 = 0.f;
    bool bad = false;
    uint32_t phase = 0;
    bool inflight = ntiles > 0 ? issue(0) : false;

    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t row0 = r0 + t * L;
        const int rows_v = (int)min((int64_t)L, r1 - row0);
        if (inflight) {
            // the decision is warp-uniform, so no lane leaves while others still shuffle
            if (!__all_sync(FULL, mbar_wait(bar_s, phase))) {
                if (lane == 0) set_status(a.status, MRNMF_ERR_TIMEOUT);
                mbar_wait(bar_s, phase);  // bounded second wait for the copy in flight
                break;                    // leave the tile loop; the CTA still meets at its barriers
            }
            phase ^= 1u;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                a0[l] = (own0 && l < rows_v) ? tile[l * n + c0] : 0.f;
                if (NC == 2) a1[l] = (own1 && l < rows_v) ? tile[l * n + c1] : 0.f;
            }
        } else {
            const float* src = X + row0 * a.ldx;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                a0[l] = (own0 && l < rows_v) ? src[(int64_t)l * a.ldx + c0] : 0.f;
                if (NC == 2) a1[l] = (own1 && l < rows_v) ? src[(int64_t)l * a.ldx + c1] : 0.f;
            }
        }
        __syncwarp();
        if (t + 1 < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            inflight = issue(t + 1);
        } else {
            inflight = false;
        }

        // input check, column sums (Sec. 3.3)
        {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                bad |= !(a0[l] >= 0.f);
                s0 += a0[l];
                if (NC == 2) {
                    bad |= !(a1[l] >= 0.f);
                    s1 += a1[l];
                }
            }
            cs0 += s0;
            cs1 += s1;
        }

        if (GP) {
            // G rows of this tile (coordinate-major), then GX(:, c) += G' A(:, c)
            const int kq = kp >> 2 > 0 ? kp >> 2 : 1;
            for (int idx = lane; idx < L * (kp >> 2); idx += 32) {
                const int l = idx / kq, q = idx - l * kq;
                float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                if (l < rows_v) g = gauss4(a.seed, a.row_base + row0 + l, (uint32_t)q);
                gbuf[(4 * q + 0) * L + l] = g.x;
                gbuf[(4 * q + 1) * L + l] = g.y;
                gbuf[(4 * q + 2) * L + l] = g.z;
                gbuf[(4 * q + 3) * L + l] = g.w;
            }
            __syncwarp();
            // packed FMAs: .x sums the even rows, .y the odd ones (the same
            // two binary32 chains as one FMA a row would give)
            for (int q = 0; q < k; ++q) {
                const float4* gq = reinterpret_cast<const float4*>(gbuf + q * L);
                float2 p0 = make_float2(0.f, 0.f), p1 = p0;
#pragma unroll
                for (int l4 = 0; l4 < L / 4; ++l4) {
                    const float4 g = gq[l4];
                    const float2 g01 = make_float2(g.x, g.y), g23 = make_float2(g.z, g.w);
                    p0 = __ffma2_rn(g01, make_float2(a0[4 * l4], a0[4 * l4 + 1]), p0);
                    p0 = __ffma2_rn(g23, make_float2(a0[4 * l4 + 2], a0[4 * l4 + 3]), p0);
                    if (NC == 2) {
                        p1 = __ffma2_rn(g01, make_float2(a1[4 * l4], a1[4 * l4 + 1]), p1);
                        p1 = __ffma2_rn(g23, make_float2(a1[4 * l4 + 2], a1[4 * l4 + 3]), p1);
                    }
                }
                if (own0) gxs[q * n + c0] += p0.x + p0.y;
                if (NC == 2 && own1) gxs[q * n + c1] += p1.x + p1.y;
            }
        }

        column_steps<NC, L>(a0, a1, Rw, pub, n, lane, own0, own1);

        if ((t + 1) % kFlush == 0 || t + 1 == ntiles) {
            if (a.cs) {
                if (own0) a.cs[(size_t)ws * n + c0] += (double)cs0;
                if (own1) a.cs[(size_t)ws * n + c1] += (double)cs1;
            }
            cs0 = cs1 = 0.f;
            if (GP && a.gx) {
                for (int e = lane; e < k * n; e += 32) {
                    a.gx[(size_t)ws * k * n + e] += (double)gxs[e];
                    gxs[e] = 0.f;
                }
            }
            __syncwarp();
        }
    }

    if (a.check && __any_sync(FULL, bad)) {
        if (lane == 0) set_status(a.status, MRNMF_ERR_BAD_INPUT);
    }
    // fold the CTA's four triangles into warp 0's: R([R0;R1;R2;R3]) by the
    // same column steps, each absorbed triangle loaded as an L-row tile (L >= n)
    for (int span = 1; span < kWarps; span <<= 1) {
        __syncthreads();
        if ((warp & (2 * span - 1)) == 0) {
            const float* Rb = reinterpret_cast<const float*>(
                smem + (size_t)(warp + span) * warp_slice_bytes<L>(n, k) + 128 + up(sizeof(float) * (size_t)L * n, 128));
            for (int rb = 0; rb < n; rb += L) {  // the triangle's rows, L at a time
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    const int row = rb + l;
                    a0[l] = (own0 && row < n && c0 >= row) ? Rb[pk_row(row, n) + c0] : 0.f;
                    if (NC == 2) a1[l] = (own1 && row < n && c1 >= row) ? Rb[pk_row(row, n) + c1] : 0.f;
                }
                __syncwarp();
                column_steps<NC, L>(a0, a1, Rw, pub, n, lane, own0, own1);
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        float* Rout = static_cast<float*>(a.R_out) + (size_t)cta * n * n;
        const int nn = n * n;
        for (int e = lane; e < nn; e += 32) {
            const int j = e / n, c = e - j * n;
            Rout[e] = (c >= j) ? Rw[pk_row(j, n) + c] : 0.f;
        }
    }
}


// Residency targets (measured): the 32-row forms run three CTAs per SM with
// the projection (shared memory allows no more) and four without it (n up to
// about 56 fits four in shared memory); the one-column 64-row form three.
template <int NC, int L, bool GP>
__global__ void __launch_bounds__(kWarps * 32, (L == 32 && !GP) ? 4 : (L == 32 || (NC == 1 && L == 64)) ? 3 : 1)
    tsqr_warp_kernel(const LeafArgs a)
{
    warp_stream_body<NC, L, GP>(a, blockIdx.x);
}

// Batched form: CTA b works on problem desc[b].p, as that problem's CTA desc[b].cta.
template <int NC, int L>
__global__ void __launch_bounds__(kWarps * 32) tsqr_warp_batched_kernel(const BatchCta* __restrict__ desc,
                                                                        const BatchProblem* __restrict__ probs,
                                                                        int* status)
{
    const BatchCta d = desc[blockIdx.x];
    const BatchProblem pb = probs[d.p];
    LeafArgs a{};
    a.X = pb.X;
    a.rows = pb.m;
    a.ldx = pb.ldx;
    a.n = pb.n;
    a.rows_per_cta = pb.rows_per_stream;
    a.R_in = nullptr;
    a.R_out = pb.tri;
    a.cs = pb.cs;
    a.check = 1;
    a.status = status;
    warp_stream_body<NC, L, false>(a, d.cta);
}

// ---------------------------------------------------------------------------
// Wide tree level for n <= 64: CTA q merges triangles [q*(S+1), (q+1)*(S+1)).
// The first one seeds the running triangle (shared memory); thread (c, s)
// holds column c of the s-th remaining triangle in registers (rows 0..c are
// its only nonzeros, and reflectors 0..j-1 keep it that way).  Column step j:
// sigma = sum over s of ||T_s(0..j, j)||^2 (two barriers per column: one after
// the pivot columns and partial norms are published, one after the partial
// dot products are), then every column c > j of every triangle is updated.
template <int NP, int S>
__device__ __forceinline__ void tree_wide_body(const float* __restrict__ Rin, int first, int P_in, int n,
                                               float* __restrict__ dst)
{
    __shared__ float Rs[NP * (NP + 1) / 2];
    __shared__ __align__(16) float piv[2][S][NP];
    __shared__ float sig[2][S];
    __shared__ float dpart[2][S][NP];
    const int c = threadIdx.x % NP, sgm = threadIdx.x / NP;
    const int tri = first + 1 + sgm;
    const bool have = tri < P_in && c < n;
    const int nn = n * n;
    for (int e = threadIdx.x; e < nn; e += NP * S) {
        const int j = e / n, cc = e - j * n;
        if (cc >= j) Rs[pk_row(j, n) + cc] = first < P_in ? Rin[(size_t)first * nn + e] : 0.f;
    }
    float col[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) col[i] = (have && i <= c) ? Rin[(size_t)tri * nn + (size_t)i * n + c] : 0.f;
    __syncthreads();

    // Column c of every triangle is zero below row c, so the pivot column j has
    // no entries past row j: every loop below stops at the first 4-row chunk
    // past j and needs no masking.
    for (int j = 0; j < n; ++j) {
        const int b = j & 1;
        float4* pv = reinterpret_cast<float4*>(&piv[b][sgm][0]);
        if (c == j) {
            // four partial sums: the pivot's squared norm is on the step's critical path
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                if (4 * q > j) break;
                const float4 v = make_float4(col[4 * q], col[4 * q + 1], col[4 * q + 2], col[4 * q + 3]);
                s0 = fmaf(v.x, v.x, s0);
                s1 = fmaf(v.y, v.y, s1);
                s2 = fmaf(v.z, v.z, s2);
                s3 = fmaf(v.w, v.w, s3);
                pv[q] = v;
            }
            sig[b][sgm] = (s0 + s1) + (s2 + s3);
        }
        __syncthreads();
        float sigma = 0.f;
#pragma unroll
        for (int q = 0; q < S; ++q) sigma += sig[b][q];
        const int pr = pk_row(j, n);
        const float alpha = Rs[pr + j];
        // the leaves' column step: with w' = d R_jc + g_c, R_jc += w'/beta and
        // column c += (w'/d)(1/beta) times the raw pivot column
        float beta = alpha, d = 0.f, rb = 0.f, rd = 0.f;
        if (sigma > 0.f) {
            const HhScalars hs = hh_scalars(alpha, sigma);
            beta = hs.beta;
            d = hs.d;
            rb = hs.rb;
            rd = hs.rd;
        }
        const bool upd = sigma > 0.f && c > j && c < n;
        const float r = upd ? Rs[pr + c] : 0.f;  // read before the barrier: segment 0 rewrites it after
        if (upd) {
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                if (4 * q > j) break;
                const float4 v = pv[q];
                d0 = fmaf(v.x, col[4 * q], d0);
                d1 = fmaf(v.y, col[4 * q + 1], d1);
                d0 = fmaf(v.z, col[4 * q + 2], d0);
                d1 = fmaf(v.w, col[4 * q + 3], d1);
            }
            dpart[b][sgm][c] = d0 + d1;
        }
        __syncthreads();
        if (upd) {
            float dsum = 0.f;
#pragma unroll
            for (int q = 0; q < S; ++q) dsum += dpart[b][q][c];
            const float wp = fmaf(d, r, dsum);
            const float f = (wp * rd) * rb;
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                if (4 * q > j) break;
                const float4 v = pv[q];
                col[4 * q] = fmaf(f, v.x, col[4 * q]);
                col[4 * q + 1] = fmaf(f, v.y, col[4 * q + 1]);
                col[4 * q + 2] = fmaf(f, v.z, col[4 * q + 2]);
                col[4 * q + 3] = fmaf(f, v.w, col[4 * q + 3]);
            }
            if (sgm == 0) Rs[pr + c] = fmaf(wp, rb, r);
        }
        if (c == j && sgm == 0) Rs[pr + j] = beta;
        // the next step writes the other buffers; this step's readers are past the barrier above
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += NP * S) {
        const int j = e / n, cc = e - j * n;
        dst[e] = cc >= j ? Rs[pk_row(j, n) + cc] : 0.f;
    }
}

template <int NP, int S>
__global__ void __launch_bounds__(NP * S) tsqr_tree_wide_kernel(const float* __restrict__ Rin, int P_in, int n,
                                                                float* __restrict__ Rout)
{
    tree_wide_body<NP, S>(Rin, blockIdx.x * (S + 1), P_in, n, Rout + (size_t)blockIdx.x * n * n);
}

// Batched tree level: CTA b folds desc[b].count triangles at desc[b].in into desc[b].out.
template <int NP, int S>
__global__ void __launch_bounds__(NP * S) tsqr_tree_wide_batched_kernel(const TreeCta* __restrict__ desc)
{
    const TreeCta d = desc[blockIdx.x];
    tree_wide_body<NP, S>(d.in, 0, d.count, d.n, d.out);
}

template <int NP, int S>
cudaError_t launch_tree_wide(const float* Rin, int P_in, int n, float* Rout, cudaStream_t s, int* P_out)
{
    const int grid = (P_in + S) / (S + 1);
    tsqr_tree_wide_kernel<NP, S><<<grid, NP * S, 0, s>>>(Rin, P_in, n, Rout);
    count_launch();
    *P_out = grid;
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// CTA-per-stream leaf for 64 < n <= 256 in binary32.  Thread c owns column c:
// the 32 rows of each tile for that column sit in its registers, so all dot
// products are thread-local; the running triangle (packed) is in shared
// memory.  One barrier per column step: the owner of column j+1 publishes the
// column's raw values, its squared norm and R(j+1, j+1) right after its own
// update in step j, so step j+1 can start with everything it needs.
// Tile height: 64 rows without the projection while two CTAs still fit per
// SM (n <= 184; halves the barriers and the per-column scalar work per row),
// else 32 (the projection accumulators need the registers).
__host__ __device__ constexpr int cta_rows(int k, int n) { return (k > 0 || n > 184) ? 32 : 64; }

__host__ __device__ inline size_t cta_smem_bytes(int n, int k)
{
    const int kp = (k + 3) & ~3;
    const int L = cta_rows(k, n);
    size_t b = 128;                                          // mbarrier
    b += up(sizeof(float) * (size_t)L * n, 128);             // TMA staging tile
    b += up(sizeof(float) * (size_t)(n * (n + 1) / 2), 16);  // packed R
    b += sizeof(float) * 2 * (L + 4);                        // published column (+ sigma, alpha)
    b += sizeof(float) * (size_t)kp * L;                     // Gaussian tile
    return up(b, 128);
}

// KMAX: 0 (no projection) or a bound on k; thread c keeps GX(:, c) in registers.
template <int KMAX, int L>
__global__ void __launch_bounds__(256, KMAX <= 48 ? 2 : 1) tsqr_cta_kernel(const LeafArgs a)
{
    constexpr bool GP = KMAX > 0;
    extern __shared__ __align__(128) unsigned char smem[];
    const int n = a.n;
    const int k = GP ? a.k : 0;
    const int kp = (k + 3) & ~3;
    const int c = threadIdx.x, nt = blockDim.x;
    const bool own = c < n;
    const int last_col = (c | 31);  // highest column of this warp
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float* tile = reinterpret_cast<float*>(smem + 128);
    float* Rs = reinterpret_cast<float*>(smem + 128 + up(sizeof(float) * (size_t)L * n, 128));
    float* pub = Rs + up((size_t)(n * (n + 1) / 2), 4);  // [2][L + 4]: values, then sigma, alpha
    float* gbuf = pub + 2 * (L + 4);
    const uint32_t bar_s = smem_u32(bar);
    const int cta = blockIdx.x;
    float gacc[KMAX > 0 ? KMAX : 1];
#pragma unroll
    for (int q = 0; q < (KMAX > 0 ? KMAX : 1); ++q) gacc[q] = 0.f;

    if (c == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const float* Rin = static_cast<const float*>(a.R_in);
        const int nn = n * n;
        for (int e = c; e < nn; e += nt) {
            const int j = e / n, cc = e - j * n;
            if (cc >= j) Rs[pk_row(j, n) + cc] = Rin ? Rin[(size_t)cta * nn + e] : 0.f;
        }
    }
    __syncthreads();

    const int64_t r0 = (int64_t)cta * a.rows_per_cta;
    const int64_t r1 = min(a.rows, r0 + a.rows_per_cta);
    const int64_t ntiles = r1 > r0 ? (r1 - r0 + L - 1) / L : 0;
    const float* X = static_cast<const float*>(a.X);
    const bool tma_ok = a.ldx == n && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    auto issue = [&](int64_t t) -> bool {
        const int64_t row0 = r0 + t * L;
        const int rows_v = (int)min((int64_t)L, r1 - row0);
        const uint32_t bytes = (uint32_t)rows_v * (uint32_t)n * 4u;
        if (!tma_ok || (bytes & 15u)) return false;
        if (c == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(bytes) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(tile)),
                "l"(X + row0 * n), "r"(bytes), "r"(bar_s)
                : "memory");
        }
        return true;
    };

    float av[L];
    float cs_acc = 0.f;
    bool bad = false, timed_out = false;
    uint32_t phase = 0;
    bool inflight = ntiles > 0 ? issue(0) : false;

    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t row0 = r0 + t * L;
        const int rows_v = (int)min((int64_t)L, r1 - row0);
        if (inflight) {
            if (!__syncthreads_and(mbar_wait(bar_s, phase))) {
                timed_out = true;
                mbar_wait(bar_s, phase);
                break;
            }
            phase ^= 1u;
#pragma unroll
            for (int l = 0; l < L; ++l) av[l] = (own && l < rows_v) ? tile[l * n + c] : 0.f;
        } else {
            const float* src = X + row0 * a.ldx;
#pragma unroll
            for (int l = 0; l < L; ++l) av[l] = (own && l < rows_v) ? src[(int64_t)l * a.ldx + c] : 0.f;
        }
        __syncthreads();
        if (t + 1 < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            inflight = issue(t + 1);
        } else {
            inflight = false;
        }
        {
            float s0 = 0.f;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                bad |= !(av[l] >= 0.f);
                s0 += av[l];
            }
            cs_acc += s0;
        }
        if (GP) {
            const int kq = kp >> 2 > 0 ? kp >> 2 : 1;
            for (int idx = c; idx < L * (kp >> 2); idx += nt) {
                const int l = idx / kq, q = idx - l * kq;
                float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                if (l < rows_v) g = gauss4(a.seed, a.row_base + row0 + l, (uint32_t)q);
                gbuf[(4 * q + 0) * L + l] = g.x;
                gbuf[(4 * q + 1) * L + l] = g.y;
                gbuf[(4 * q + 2) * L + l] = g.z;
                gbuf[(4 * q + 3) * L + l] = g.w;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < (KMAX > 0 ? KMAX : 1); ++q) {
                if (q < k) {
                    const float4* gq = reinterpret_cast<const float4*>(gbuf + q * L);
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int l4 = 0; l4 < L / 4; ++l4) {
                        const float4 g = gq[l4];
                        s0 = fmaf(g.x, av[4 * l4], s0);
                        s1 = fmaf(g.y, av[4 * l4 + 1], s1);
                        s0 = fmaf(g.z, av[4 * l4 + 2], s0);
                        s1 = fmaf(g.w, av[4 * l4 + 3], s1);
                    }
                    gacc[q] += s0 + s1;
                }
            }
        }
        // The owner of a column publishes its values, squared norm and
        // diagonal entry of R (column 0's owner before the first step).
        auto publish = [&](float* pn, float rjj) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
            for (int l4 = 0; l4 < L / 4; ++l4) {
                reinterpret_cast<float4*>(pn)[l4] = make_float4(av[4 * l4], av[4 * l4 + 1], av[4 * l4 + 2], av[4 * l4 + 3]);
                s0 = fmaf(av[4 * l4], av[4 * l4], s0);
                s1 = fmaf(av[4 * l4 + 1], av[4 * l4 + 1], s1);
                s2 = fmaf(av[4 * l4 + 2], av[4 * l4 + 2], s2);
                s3 = fmaf(av[4 * l4 + 3], av[4 * l4 + 3], s3);
            }
            pn[L] = (s0 + s1) + (s2 + s3);
            pn[L + 1] = rjj;
        };
        if (c == 0) publish(pub, Rs[0]);
        for (int j = 0; j < n; ++j) {
            __syncthreads();
            if (last_col < j) continue;  // every column of this warp is finished
            const float* pj = pub + (j & 1) * (L + 4);
            const float sig = pj[L], alpha = pj[L + 1];
            const int pr = pk_row(j, n);
            float beta = alpha;
            if (sig > 0.f) {
                const HhScalars hs = hh_scalars(alpha, sig);
                beta = hs.beta;
                if (own && c > j) {
                    const float d = hs.d, rb = hs.rb, rd = hs.rd;
                    const float4* p4 = reinterpret_cast<const float4*>(pj);
                    float ga = 0.f, gb = 0.f, gc = 0.f, gd = 0.f;
#pragma unroll
                    for (int l4 = 0; l4 < L / 4; ++l4) {
                        const float4 v = p4[l4];
                        ga = fmaf(v.x, av[4 * l4], ga);
                        gb = fmaf(v.y, av[4 * l4 + 1], gb);
                        gc = fmaf(v.z, av[4 * l4 + 2], gc);
                        gd = fmaf(v.w, av[4 * l4 + 3], gd);
                    }
                    const float g = (ga + gb) + (gc + gd);
                    const float r = Rs[pr + c];
                    const float wp = fmaf(d, r, g);
                    const float f = (wp * rd) * rb;
                    Rs[pr + c] = fmaf(wp, rb, r);
#pragma unroll
                    for (int l4 = 0; l4 < L / 4; ++l4) {
                        const float4 v = p4[l4];
                        av[4 * l4] = fmaf(f, v.x, av[4 * l4]);
                        av[4 * l4 + 1] = fmaf(f, v.y, av[4 * l4 + 1]);
                        av[4 * l4 + 2] = fmaf(f, v.z, av[4 * l4 + 2]);
                        av[4 * l4 + 3] = fmaf(f, v.w, av[4 * l4 + 3]);
                    }
                }
            }
            if (c == j) Rs[pr + j] = beta;
            // the owner of column j+1 publishes its updated column, norm and diagonal
            if (c == j + 1 && j + 1 < n) publish(pub + ((j + 1) & 1) * (L + 4), Rs[pk_row(j + 1, n) + j + 1]);
        }
        if ((t + 1) % kFlush == 0 || t + 1 == ntiles) {
            if (own && a.cs) a.cs[(size_t)cta * n + c] += (double)cs_acc;
            cs_acc = 0.f;
            if (GP && a.gx && own) {
#pragma unroll
                for (int q = 0; q < (KMAX > 0 ? KMAX : 1); ++q)
                    if (q < k) {
                        a.gx[((size_t)cta * k + q) * n + c] += (double)gacc[q];
                        gacc[q] = 0.f;
                    }
            }
        }
        __syncthreads();
    }
    if (timed_out && c == 0) set_status(a.status, MRNMF_ERR_TIMEOUT);
    if (a.check && __syncthreads_or(bad) && c == 0) set_status(a.status, MRNMF_ERR_BAD_INPUT);
    __syncthreads();
    float* Rout = static_cast<float*>(a.R_out) + (size_t)cta * n * n;
    const int nn = n * n;
    for (int e = c; e < nn; e += nt) {
        const int j = e / n, cc = e - j * n;
        Rout[e] = (cc >= j) ? Rs[pk_row(j, n) + cc] : 0.f;
    }
}

template <int KMAX, int L>
int cta_ctas_per_sm_k(int n, int k)
{
    const size_t smem = cta_smem_bytes(n, KMAX > 0 ? k : 0);
    auto kern = tsqr_cta_kernel<KMAX, L>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    int blocks = 0;
    const int block = ((n + 31) / 32) * 32;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, block, smem) != cudaSuccess) return 1;
    return blocks < 1 ? 1 : blocks;
}

template <int KMAX, int L>
cudaError_t launch_cta_k(const LeafArgs& a, int grid, cudaStream_t s)
{
    const size_t smem = cta_smem_bytes(a.n, KMAX > 0 ? a.k : 0);
    auto kern = tsqr_cta_kernel<KMAX, L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    kern<<<grid, ((a.n + 31) / 32) * 32, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int NC, int L, bool GP>
cudaError_t launch_nc(const LeafArgs& a, int streams, cudaStream_t s)
{
    const size_t smem = (size_t)kWarps * warp_slice_bytes<L>(a.n, GP ? a.k : 0);
    auto kern = tsqr_warp_kernel<NC, L, GP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (streams + kWarps - 1) / kWarps;
    kern<<<grid, kWarps * 32, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int NC, int L, bool GP>
int ctas_per_sm_nc(int n, int k)
{
    const size_t smem = (size_t)kWarps * warp_slice_bytes<L>(n, GP ? k : 0);
    auto kern = tsqr_warp_kernel<NC, L, GP>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kWarps * 32, smem) != cudaSuccess) return 1;
    return blocks < 1 ? 1 : blocks;
}

// Shared memory of one CTA of the warp leaf at tile height L; 0 where the form
// serving n has no such height (one column per lane, n <= 32: 64 or 128 rows;
// two columns per lane, 33..64: 32 or 64 rows).
size_t warp_cta_smem(int n, int k, int L)
{
    if (n <= 32) return L == 64 ? kWarps * warp_slice_bytes<64>(n, k) : L == 128 ? kWarps * warp_slice_bytes<128>(n, k) : 0;
    return L == 32 ? kWarps * warp_slice_bytes<32>(n, k) : L == 64 ? kWarps * warp_slice_bytes<64>(n, k) : 0;
}

constexpr size_t kWarpSmemCap = 220 * 1024;

int env_rows(const char* name, int a, int b)
{
    const char* e = getenv(name);
    const int v = e ? atoi(e) : 0;
    return (v == a || v == b) ? v : 0;
}

// Tile height of the warp leaf for n columns and k projection rows (k = 0
// without the projection).  In order: MRNMF_WARP_ROWS1=64|128 (n <= 32) or
// MRNMF_WARP_ROWS=32|64 (33..64); the tuning table's `rows` line for (n, k);
// the default.  Defaults, measured on GB300: the one-column form at 64 rows
// ran 3-7% faster than at 128 with the projection (n = 16..28, 1.6e7 rows) and
// up to 8% without it; the two-column form at 32 rows holds three or four CTAs
// per SM.  A height whose CTA does not fit in shared memory gives the default.
int leaf_rows(int n, int k)
{
    static const int f1 = env_rows("MRNMF_WARP_ROWS1", 64, 128);
    static const int f2 = env_rows("MRNMF_WARP_ROWS", 32, 64);
    const int dflt = n <= 32 ? 64 : 32;
    int L = n <= 32 ? f1 : f2;
    if (!L) L = tune_leaf_rows(n, k);
    const size_t smem = L ? warp_cta_smem(n, k, L) : 0;
    return (smem == 0 || smem > kWarpSmemCap) ? dflt : L;
}

}  // namespace

bool wide_tree_supported(int n) { return n >= 1 && n <= 128; }

cudaError_t tree_wide_level(const float* Rin, int P_in, int n, float* Rout, cudaStream_t s, int* P_out)
{
    if (n <= 32) return launch_tree_wide<32, 16>(Rin, P_in, n, Rout, s, P_out);
    if (n <= 64) return launch_tree_wide<64, 8>(Rin, P_in, n, Rout, s, P_out);
    return launch_tree_wide<128, 3>(Rin, P_in, n, Rout, s, P_out);
}

bool warp_leaf_supported(int n, int k)
{
    if (n < 1 || n > 64 || k > 64) return false;
    const size_t smem = warp_cta_smem(n, k, leaf_rows(n, k));
    return smem > 0 && smem <= kWarpSmemCap;
}

int warp_leaf_rows_per_tile(int n, int k) { return group_leaf_supported(n, k) ? group_leaf_rows_per_tile(n) : leaf_rows(n, k); }

int warp_leaf_warps_per_cta() { return kWarps; }

int warp_leaf_ctas_per_sm(int n, int k)
{
    if (group_leaf_supported(n, k)) return group_leaf_ctas_per_sm(n);
    const int L = leaf_rows(n, k);
    if (n <= 32 && L == 64) return k > 0 ? ctas_per_sm_nc<1, 64, true>(n, k) : ctas_per_sm_nc<1, 64, false>(n, k);
    if (n <= 32) return k > 0 ? ctas_per_sm_nc<1, 128, true>(n, k) : ctas_per_sm_nc<1, 128, false>(n, k);
    if (L == 32) return k > 0 ? ctas_per_sm_nc<2, 32, true>(n, k) : ctas_per_sm_nc<2, 32, false>(n, k);
    return k > 0 ? ctas_per_sm_nc<2, 64, true>(n, k) : ctas_per_sm_nc<2, 64, false>(n, k);
}

cudaError_t launch_warp_batched(const BatchCta* desc, int nctas, const BatchProblem* probs, int family, int max_n,
                                int* status, cudaStream_t s)
{
    if (nctas <= 0) return cudaSuccess;
    cudaError_t e;
    size_t smem;
    if (family == 1) {
        smem = (size_t)kWarps * warp_slice_bytes<64>(max_n, 0);
        e = cudaFuncSetAttribute(tsqr_warp_batched_kernel<1, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        tsqr_warp_batched_kernel<1, 64><<<nctas, kWarps * 32, smem, s>>>(desc, probs, status);
    } else {
        smem = (size_t)kWarps * warp_slice_bytes<32>(max_n, 0);
        e = cudaFuncSetAttribute(tsqr_warp_batched_kernel<2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        tsqr_warp_batched_kernel<2, 32><<<nctas, kWarps * 32, smem, s>>>(desc, probs, status);
    }
    count_launch();
    return cudaGetLastError();
}

int warp_batched_rows_per_tile(int family) { return family == 1 ? 64 : 32; }

bool cta_leaf_supported(int n, int k)
{
    return n > 64 && n <= 256 && k <= 64 && cta_smem_bytes(n, k) <= 220 * 1024;
}

int cta_leaf_rows_per_tile(int k, int n) { return cta_rows(k, n); }

int cta_leaf_ctas_per_sm(int n, int k)
{
    if (k <= 0) return cta_rows(0, n) == 64 ? cta_ctas_per_sm_k<0, 64>(n, 0) : cta_ctas_per_sm_k<0, 32>(n, 0);
    if (k <= 16) return cta_ctas_per_sm_k<16, 32>(n, k);
    if (k <= 32) return cta_ctas_per_sm_k<32, 32>(n, k);
    if (k <= 48) return cta_ctas_per_sm_k<48, 32>(n, k);
    return cta_ctas_per_sm_k<64, 32>(n, k);
}

cudaError_t launch_cta_leaf(const LeafArgs& a, int grid, cudaStream_t s)
{
    const int k = (a.gx != nullptr && a.k > 0) ? a.k : 0;
    if (k == 0) return cta_rows(0, a.n) == 64 ? launch_cta_k<0, 64>(a, grid, s) : launch_cta_k<0, 32>(a, grid, s);
    if (k <= 16) return launch_cta_k<16, 32>(a, grid, s);
    if (k <= 32) return launch_cta_k<32, 32>(a, grid, s);
    if (k <= 48) return launch_cta_k<48, 32>(a, grid, s);
    return launch_cta_k<64, 32>(a, grid, s);
}

int tree_fan_in(int family) { return family == 1 ? 17 : (family == 2 ? 9 : 4); }

cudaError_t launch_tree_batched(const TreeCta* desc, int nctas, int family, cudaStream_t s)
{
    if (nctas <= 0) return cudaSuccess;
    if (family == 1) tsqr_tree_wide_batched_kernel<32, 16><<<nctas, 32 * 16, 0, s>>>(desc);
    else if (family == 2) tsqr_tree_wide_batched_kernel<64, 8><<<nctas, 64 * 8, 0, s>>>(desc);
    else tsqr_tree_wide_batched_kernel<128, 3><<<nctas, 128 * 3, 0, s>>>(desc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_warp_leaf(const LeafArgs& a, int streams, cudaStream_t s)
{
    const bool gp = a.gx != nullptr && a.k > 0;
    if (group_leaf_supported(a.n, gp ? a.k : 0)) return launch_group_leaf(a, streams, s);
    // the height rows_per_cta was rounded to, so that a table reloaded in between changes nothing
    const int L = a.tile_rows ? a.tile_rows : leaf_rows(a.n, gp ? a.k : 0);
    if (warp_cta_smem(a.n, gp ? a.k : 0, L) == 0 || a.rows_per_cta % L != 0) return cudaErrorInvalidValue;
    if (a.n <= 32 && L == 64) return gp ? launch_nc<1, 64, true>(a, streams, s) : launch_nc<1, 64, false>(a, streams, s);
    if (a.n <= 32) return gp ? launch_nc<1, 128, true>(a, streams, s) : launch_nc<1, 128, false>(a, streams, s);
    if (L == 32) return gp ? launch_nc<2, 32, true>(a, streams, s) : launch_nc<2, 32, false>(a, streams, s);
    return gp ? launch_nc<2, 64, true>(a, streams, s) : launch_nc<2, 64, false>(a, streams, s);
}

}  // namespace mrnmf
