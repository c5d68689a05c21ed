// tsqr_pipe.cu -- the pass over X for 64 < n <= 256 in binary32 as a warp
// pipeline: one CTA per row stream, warp w owns the 32-column block
// [32w, 32w+32) of every tile, and no block-wide barrier runs per column.
//
// Reflector j of a tile (the column step of the local QR of Sec. 3.1 on the
// stacked [R; A], as in the SIMT leaves) is produced by the warp that owns
// column j: it publishes the column's values and three scalars (d = alpha -
// beta, 1/beta, 1/d) in a shared-memory ring of tile slots.  Warp w applies,
// in order, the reflectors of blocks 0 .. w-1 (waiting on each producer's
// mbarrier), then performs its own 32 column steps inside the warp (only
// __syncwarp), then signals its block.  Every thread applies the reflectors
// to its own column in the global order (tile by tile, column by column), so
// the arithmetic is that of the one-barrier-per-column leaf; what changes is
// that different warps work on different tiles at the same time.
//
// Each column's R entries (packed triangle in shared memory) belong to the
// column's thread.  Ring slots are reused after every consumer warp has
// signalled the slot's "free" mbarrier.  Every wait is bounded (1 s); the
// first warp that gives up raises a CTA-wide abort flag that ends every
// other wait at once, and MRNMF_ERR_TIMEOUT is reported.
//
// Column sums and the Gaussian projection (Algorithm 1, Sec. 3.2) are folded
// in: warp 0 draws each tile's G into the slot, every thread accumulates
// G' A(:, c) for its column in binary32 (in shared memory), flushed to
// binary64 every kFlush tiles.
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "leaf.h"

namespace mrnmf {

namespace {

constexpr int kL = 32;          // tile height
// ring slots (tiles in flight): 2, or 4 where the SM holds one CTA anyway (pipe_cfg)
constexpr int kRS = kL + 4;     // ring entry: L values, then d, 1/beta, 1/d, v_j' v_(j+1)
constexpr int kMaxW = 8;        // warps (n <= 256)
constexpr int kFlushT = 32;     // tiles between binary64 flushes

__host__ __device__ inline int pk(int j, int n) { return j * n - (j * (j + 1)) / 2; }
__host__ __device__ inline size_t up16(size_t b) { return (b + 15) / 16 * 16; }

struct PipeLayout {
    size_t ring, gbuf, gx, bars, flag, total;
};

// gxs: the projection's binary32 partials in shared memory ([coordinate][column])
// instead of registers
__host__ __device__ inline PipeLayout pipe_layout(int n, int k, bool gxs = false, int kD = 2)
{
    const int kp = (k + 3) & ~3;
    PipeLayout p;
    size_t off = up16(sizeof(float) * (size_t)(n * (n + 1) / 2));  // packed R
    p.ring = off;
    off += up16(sizeof(float) * (size_t)kD * n * kRS);
    p.gbuf = off;
    off += up16(sizeof(float) * (size_t)kD * kp * kL);
    p.gx = off;
    if (gxs) off += up16(sizeof(float) * (size_t)k * n);
    p.bars = off;
    off += sizeof(uint64_t) * 2 * kD * kMaxW;  // pub[kD][kMaxW], fre[kD][kMaxW]
    p.flag = off;
    off += 16;
    p.total = off;
    return p;
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

// Lane 0 waits for the phase of parity `par` to complete (bounded by
// `limit_ns`, and abandoned at once when another warp has aborted); the
// outcome is broadcast to the warp and ordered before the warp's later reads.
// Returns 0 when the phase completed, 1 when this wait ran out (it then sets
// the abort flag and MRNMF_ERR_TIMEOUT), 2 when it was abandoned.
__device__ __forceinline__ int warp_wait_code(uint64_t* b, uint32_t par, volatile int* abort_flag, int* status,
                                              uint64_t limit_ns)
{
    int code = 0;
    if ((threadIdx.x & 31) == 0) {
        const uint32_t a = saddr(b);
        const uint64_t t0 = gtime();
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
                " selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(a), "r"(par)
                : "memory");
            if (done) break;
            if (*abort_flag) {
                code = 2;
                break;
            }
            if (gtime() - t0 > limit_ns) {
                *abort_flag = 1;
                set_status(status, MRNMF_ERR_TIMEOUT);
                code = 1;
                break;
            }
        }
    }
    code = __shfl_sync(0xffffffffu, code, 0);
    __syncwarp();
    return code;
}

__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t par, volatile int* abort_flag, int* status)
{
    return warp_wait_code(b, par, abort_flag, status, 1000000000ull) == 0;
}

// Failure injection for the hand-over above: four warps in a chain, warp v
// (v >= 1) waiting on barrier v, which warp v - 1 arrives on once its own
// wait has completed (warp 0 waits on nothing), with a limit of
// v * limit_ns so that the order in which the waits give up is fixed.
// Barrier `missing` (1..3; 0 = none) never gets its arrival: its wait runs
// out, and the waits after it in the chain are abandoned through the abort
// flag instead of running out in turn.  out[w]: 0 completed, 1 ran out,
// 2 abandoned (warp 0 writes 0).
__global__ void __launch_bounds__(128) wait_selftest_kernel(int missing, uint64_t limit_ns, int* out, int* status)
{
    __shared__ __align__(8) uint64_t bars[4];
    __shared__ int abort_flag;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) bar_init(&bars[i], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int code = 0;
    if (w > 0) code = warp_wait_code(&bars[w], 0, &abort_flag, status, limit_ns * (uint64_t)w);
    if (lane == 0) {
        if (code == 0 && w + 1 < 4 && w + 1 != missing) bar_arrive(&bars[w + 1]);
        out[w] = code;
    }
    // every barrier is either completed or abandoned before the CTA ends
    __syncthreads();
}

// One stream (row range cta * rows_per_cta ..) of the problem in `a`; the
// block may have more warps than the problem's column blocks (batched
// launches size the block for the widest problem): those warps only meet the
// CTA-wide barriers.
// GXS: the projection's partials in shared memory (fewer registers; used where
// the larger layout fits), else in registers.
template <int KMAX, bool GXS = false>
__device__ __forceinline__ void pipe_body(const LeafArgs& a, const int cta)
{
    constexpr bool GP = KMAX > 0;
    extern __shared__ __align__(128) unsigned char smem[];
    const unsigned FULL = 0xffffffffu;
    const int n = a.n;
    const int k = GP ? a.k : 0;
    const int kp = (k + 3) & ~3;
    const int W = (n + 31) / 32;
    // Column blocks: the partial block (rem = n - 32 (W - 1) columns) first,
    // then full 32-column blocks, so the warps that apply the most reflectors
    // have every lane busy.  Block b = [bstart(b), bstart(b + 1)).
    const int rem = n - 32 * (W - 1);
    auto bstart = [&](int b) { return b == 0 ? 0 : rem + 32 * (b - 1); };
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int jb0 = w < W ? bstart(w) : n, jb1 = w < W ? bstart(w + 1) : n;  // this warp's block
    const int c = jb0 + lane;                                                  // this thread's column
    const bool own = c < jb1;
    const int kD = a.ring_depth == 4 ? 4 : 2;  // tiles in flight
    const int lgD = kD == 4 ? 2 : 1;
    const PipeLayout lay = pipe_layout(n, k, GXS, kD);
    float* Rs = reinterpret_cast<float*>(smem);
    float* ring = reinterpret_cast<float*>(smem + lay.ring);
    float* gbuf = reinterpret_cast<float*>(smem + lay.gbuf);
    float* gxs = reinterpret_cast<float*>(smem + lay.gx);
    uint64_t* pub = reinterpret_cast<uint64_t*>(smem + lay.bars);  // [kD][kMaxW]
    uint64_t* fre = pub + kD * kMaxW;                               // [kD][kMaxW]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + lay.flag);

    {
        const float* Rin = static_cast<const float*>(a.R_in);
        const int nn = n * n;
        for (int e = (int)threadIdx.x; e < nn; e += blockDim.x) {
            const int j = e / n, cc = e - j * n;
            if (cc >= j) Rs[pk(j, n) + cc] = Rin ? Rin[(size_t)cta * nn + e] : 0.f;
        }
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kD; ++s)
            for (int b = 0; b < kMaxW; ++b) {
                bar_init(&pub[s * kMaxW + b], 1);
                bar_init(&fre[s * kMaxW + b], (uint32_t)max(W - 1 - b, 1));
            }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int64_t r0 = (int64_t)cta * a.rows_per_cta;
    const int64_t r1 = min(a.rows, r0 + a.rows_per_cta);
    const int64_t ntiles = (r1 > r0 && w < W) ? (r1 - r0 + kL - 1) / kL : 0;
    const float* X = static_cast<const float*>(a.X);

    float av[kL];
    float gacc[(!GXS && KMAX > 0) ? KMAX : 1];
#pragma unroll
    for (int q = 0; q < ((!GXS && KMAX > 0) ? KMAX : 1); ++q) gacc[q] = 0.f;
    if (GXS && GP)
        for (int e = (int)threadIdx.x; e < k * n; e += blockDim.x) gxs[e] = 0.f;
    float cs_acc = 0.f;
    bool bad = false;

    // G' A(:, c) for this tile (original values of the column), added to the
    // column's binary32 partials; packed FMAs, .x over the even rows and .y over
    // the odd ones
    auto proj1 = [&](const float* gq) {
        float2 p2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int l4 = 0; l4 < kL / 4; ++l4) {
            const float4 g = reinterpret_cast<const float4*>(gq)[l4];
            p2 = __ffma2_rn(make_float2(g.x, g.y), make_float2(av[4 * l4], av[4 * l4 + 1]), p2);
            p2 = __ffma2_rn(make_float2(g.z, g.w), make_float2(av[4 * l4 + 2], av[4 * l4 + 3]), p2);
        }
        return p2.x + p2.y;
    };
    auto project = [&](const float* gs) {
        if constexpr (GXS) {
            if (!own) return;
            for (int q = 0; q < k; ++q) gxs[q * n + c] += proj1(gs + q * kL);
        } else {
#pragma unroll
            for (int q = 0; q < (KMAX > 0 ? KMAX : 1); ++q)
                if (q < k) gacc[q] += proj1(gs + q * kL);
        }
    };

    int64_t t = 0;
    for (; t < ntiles; ++t) {
        const int s = (int)(t & (kD - 1));
        const uint32_t par = (uint32_t)((t >> lgD) & 1);
        const uint32_t par_prev = par ^ 1u;  // the slot's previous use (tile t - kD)
        const int64_t row0 = r0 + t * kL;
        const int rows_v = (int)min((int64_t)kL, r1 - row0);
        float* rs = ring + (size_t)s * n * kRS;
        float* gs = gbuf + (size_t)s * kp * kL;
        {
            const float* src = X + row0 * a.ldx + (own ? c : 0);
#pragma unroll
            for (int l = 0; l < kL; ++l) av[l] = (own && l < rows_v) ? __ldg(src + (int64_t)l * a.ldx) : 0.f;
            float s0 = 0.f;
#pragma unroll
            for (int l = 0; l < kL; ++l) {
                bad |= !(av[l] >= 0.f);
                s0 += av[l];
            }
            cs_acc += s0;
        }
        bool ok = true;
        if (w == 0) {
            // the slot's G and block-0 reflectors of tile t - kD must be consumed
            if (t >= kD && W > 1) ok = warp_wait(&fre[s * kMaxW + 0], par_prev, abort_flag, a.status);
            if (!ok) break;
            if (GP) {
                const int kq = kp >> 2;
                for (int idx = lane; idx < kL * kq; idx += 32) {
                    const int l = idx / kq, q = idx - l * kq;
                    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (l < rows_v) g = gauss4(a.seed, a.row_base + row0 + l, (uint32_t)q);
                    gs[(4 * q + 0) * kL + l] = g.x;
                    gs[(4 * q + 1) * kL + l] = g.y;
                    gs[(4 * q + 2) * kL + l] = g.z;
                    gs[(4 * q + 3) * kL + l] = g.w;
                }
                __syncwarp();
                project(gs);
            }
        }
        // the reflectors of the earlier blocks, in order
        for (int b = 0; b < w && ok; ++b) {
            ok = warp_wait(&pub[s * kMaxW + b], par, abort_flag, a.status);
            if (!ok) break;
            if (GP && b == 0) project(gs);
            const int j1 = bstart(b + 1);
            int j = bstart(b);
            // two reflectors per dependent chain: both dot products from the same
            // column, the second corrected by the pair coefficient
            // c = v_j' v_(j+1) that the producer published (g_(j+1) of the column
            // after reflector j is g_(j+1) + f_j c); the update is the same two
            // FMAs per element as applying them one after the other
            for (; j + 1 < j1; j += 2) {
                const float* rv0 = rs + (size_t)j * kRS;
                const float* rv1 = rv0 + kRS;
                const float4* p0 = reinterpret_cast<const float4*>(rv0);
                const float4* p1 = reinterpret_cast<const float4*>(rv1);
                float ga = 0.f, gb = 0.f, gc = 0.f, gd = 0.f, ha = 0.f, hb = 0.f, hc = 0.f, hd = 0.f;
#pragma unroll
                for (int l4 = 0; l4 < kL / 4; ++l4) {
                    const float4 v = p0[l4], u = p1[l4];
                    ga = fmaf(v.x, av[4 * l4], ga);
                    gb = fmaf(v.y, av[4 * l4 + 1], gb);
                    gc = fmaf(v.z, av[4 * l4 + 2], gc);
                    gd = fmaf(v.w, av[4 * l4 + 3], gd);
                    ha = fmaf(u.x, av[4 * l4], ha);
                    hb = fmaf(u.y, av[4 * l4 + 1], hb);
                    hc = fmaf(u.z, av[4 * l4 + 2], hc);
                    hd = fmaf(u.w, av[4 * l4 + 3], hd);
                }
                const float g0 = (ga + gb) + (gc + gd);
                float g1 = (ha + hb) + (hc + hd);
                const float d0 = rv0[kL], rb0 = rv0[kL + 1], rd0 = rv0[kL + 2], c01 = rv0[kL + 3];
                const float d1 = rv1[kL], rb1 = rv1[kL + 1], rd1 = rv1[kL + 2];
                {  // a consumer (w >= 1) holds a full block: every lane owns its column
                    const int e0 = pk(j, n) + c, e1 = pk(j + 1, n) + c;
                    const float r0 = Rs[e0], r1 = Rs[e1];
                    const float wp0 = fmaf(d0, r0, g0);
                    const float f0 = (wp0 * rd0) * rb0;
                    Rs[e0] = fmaf(wp0, rb0, r0);
                    g1 = fmaf(f0, c01, g1);
                    const float wp1 = fmaf(d1, r1, g1);
                    const float f1 = (wp1 * rd1) * rb1;
                    Rs[e1] = fmaf(wp1, rb1, r1);
#pragma unroll
                    for (int l4 = 0; l4 < kL / 4; ++l4) {
                        const float4 v = p0[l4], u = p1[l4];
                        av[4 * l4] = fmaf(f1, u.x, fmaf(f0, v.x, av[4 * l4]));
                        av[4 * l4 + 1] = fmaf(f1, u.y, fmaf(f0, v.y, av[4 * l4 + 1]));
                        av[4 * l4 + 2] = fmaf(f1, u.z, fmaf(f0, v.z, av[4 * l4 + 2]));
                        av[4 * l4 + 3] = fmaf(f1, u.w, fmaf(f0, v.w, av[4 * l4 + 3]));
                    }
                }
            }
            for (; j < j1; ++j) {
                const float* rv = rs + (size_t)j * kRS;
                const float4* p4 = reinterpret_cast<const float4*>(rv);
                float ga = 0.f, gb = 0.f, gc = 0.f, gd = 0.f;
#pragma unroll
                for (int l4 = 0; l4 < kL / 4; ++l4) {
                    const float4 v = p4[l4];
                    ga = fmaf(v.x, av[4 * l4], ga);
                    gb = fmaf(v.y, av[4 * l4 + 1], gb);
                    gc = fmaf(v.z, av[4 * l4 + 2], gc);
                    gd = fmaf(v.w, av[4 * l4 + 3], gd);
                }
                const float g = (ga + gb) + (gc + gd);
                const float d = rv[kL], rb = rv[kL + 1], rd = rv[kL + 2];
                {
                    const int e = pk(j, n) + c;
                    const float r = Rs[e];
                    const float wp = fmaf(d, r, g);
                    const float f = (wp * rd) * rb;
                    Rs[e] = fmaf(wp, rb, r);
#pragma unroll
                    for (int l4 = 0; l4 < kL / 4; ++l4) {
                        const float4 v = p4[l4];
                        av[4 * l4] = fmaf(f, v.x, av[4 * l4]);
                        av[4 * l4 + 1] = fmaf(f, v.y, av[4 * l4 + 1]);
                        av[4 * l4 + 2] = fmaf(f, v.z, av[4 * l4 + 2]);
                        av[4 * l4 + 3] = fmaf(f, v.w, av[4 * l4 + 3]);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) bar_arrive(&fre[s * kMaxW + b]);
        }
        if (!ok) break;
        // this warp's own column steps; its ring entries of tile t - kD must be consumed
        if (w > 0 && t >= kD && w < W - 1) ok = warp_wait(&fre[s * kMaxW + w], par_prev, abort_flag, a.status);
        if (!ok) break;
        for (int j = jb0; j < jb1; ++j) {
            float* rv = rs + (size_t)j * kRS;
            if (c == j) {
#pragma unroll
                for (int l4 = 0; l4 < kL / 4; ++l4)
                    reinterpret_cast<float4*>(rv)[l4] =
                        make_float4(av[4 * l4], av[4 * l4 + 1], av[4 * l4 + 2], av[4 * l4 + 3]);
            }
            __syncwarp();
            const float4* p4 = reinterpret_cast<const float4*>(rv);
            float ga = 0.f, gb = 0.f, gc = 0.f, gd = 0.f;
#pragma unroll
            for (int l4 = 0; l4 < kL / 4; ++l4) {
                const float4 v = p4[l4];
                ga = fmaf(v.x, av[4 * l4], ga);
                gb = fmaf(v.y, av[4 * l4 + 1], gb);
                gc = fmaf(v.z, av[4 * l4 + 2], gc);
                gd = fmaf(v.w, av[4 * l4 + 3], gd);
            }
            const float g = (ga + gb) + (gc + gd);
            const float sig = __shfl_sync(FULL, g, j - jb0);
            const int pr = pk(j, n);
            const float alpha = Rs[pr + j];
            __syncwarp();
            float beta = alpha, d = 0.f, rb = 0.f, rd = 0.f;
            if (sig > 0.f) {
                const HhScalars hs = hh_scalars(alpha, sig);
                beta = hs.beta;
                d = hs.d;
                rb = hs.rb;
                rd = hs.rd;
                if (own && c > j) {
                    const float r = Rs[pr + c];
                    const float wp = fmaf(d, r, g);
                    const float f = (wp * rd) * rb;
                    Rs[pr + c] = fmaf(wp, rb, r);
#pragma unroll
                    for (int l4 = 0; l4 < kL / 4; ++l4) {
                        const float4 v = p4[l4];
                        av[4 * l4] = fmaf(f, v.x, av[4 * l4]);
                        av[4 * l4 + 1] = fmaf(f, v.y, av[4 * l4 + 1]);
                        av[4 * l4 + 2] = fmaf(f, v.z, av[4 * l4 + 2]);
                        av[4 * l4 + 3] = fmaf(f, v.w, av[4 * l4 + 3]);
                    }
                }
            }
            if (c == j) {
                Rs[pr + j] = beta;
                rv[kL] = d;  // d = rb = rd = 0 marks the identity (nothing below R_jj)
                rv[kL + 1] = rb;
                rv[kL + 2] = rd;
            }
            // the pair coefficient v_(j-1)' v_j for the consumers: lane j-1 still holds
            // v_(j-1) (a reflector leaves its own column alone), so its dot product
            // with this step's pivot is that coefficient
            if (c == j - 1 && j > jb0) rs[(size_t)(j - 1) * kRS + kL + 3] = g;
            __syncwarp();
        }
        if (lane == 0 && w < W - 1) bar_arrive(&pub[s * kMaxW + w]);

        if ((t + 1) % kFlushT == 0 || t + 1 == ntiles) {
            if (own && a.cs) a.cs[(size_t)cta * n + c] += (double)cs_acc;
            cs_acc = 0.f;
            if (GP && a.gx && own) {
                if constexpr (GXS) {
                    for (int q = 0; q < k; ++q) {
                        a.gx[((size_t)cta * k + q) * n + c] += (double)gxs[q * n + c];
                        gxs[q * n + c] = 0.f;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < (KMAX > 0 ? KMAX : 1); ++q)
                        if (q < k) {
                            a.gx[((size_t)cta * k + q) * n + c] += (double)gacc[q];
                            gacc[q] = 0.f;
                        }
                }
            }
        }
    }
    if (a.check && __any_sync(FULL, bad) && lane == 0) set_status(a.status, MRNMF_ERR_BAD_INPUT);
    __syncthreads();
    float* Rout = static_cast<float*>(a.R_out) + (size_t)cta * n * n;
    const int nn = n * n;
    for (int e = (int)threadIdx.x; e < nn; e += blockDim.x) {
        const int j = e / n, cc = e - j * n;
        Rout[e] = (cc >= j) ? Rs[pk(j, n) + cc] : 0.f;
    }
}

template <int KMAX, bool GXS>
__global__ void __launch_bounds__(kMaxW * 32, 1) tsqr_pipe_kernel(const LeafArgs a)
{
    pipe_body<KMAX, GXS>(a, blockIdx.x);
}

// Ring depth and the projection partials' place for n columns and k projection
// rows.  Four tiles in flight where the two-slot layout already leaves one CTA
// per SM (more than half of the SM's shared memory) and four fit: the
// wavefront of a tile through the warps then has room; measured on GB300 at
// n = 200: 106.7 -> 118.3 GB/s (k = 0), 181.7 -> 157.8 ms per 2e7 rows
// (k = 40).  Where several CTAs fit, two slots keep them (n = 100: 286 GB/s
// with two, 184 with four).  The projection's partials go to shared memory
// where that layout still fits, else to registers.
struct PipeCfg {
    int depth;
    bool gxs;
};

inline PipeCfg pipe_cfg(int n, int k)
{
    constexpr size_t cap = 220 * 1024;
    if (pipe_layout(n, k, false, 2).total > 113 * 1024) {
        if (k > 0 && pipe_layout(n, k, true, 4).total <= cap) return {4, true};
        if (pipe_layout(n, k, false, 4).total <= cap) return {4, false};
    }
    return {2, k > 0 && pipe_layout(n, k, true, 2).total <= cap};
}

// Batched form: CTA b runs stream desc[b].cta of problem desc[b].p (R from
// zero, no projection); triangles and partial column sums go to the
// problem's slots.
__global__ void __launch_bounds__(kMaxW * 32, 1) tsqr_pipe_batched_kernel(const BatchCta* __restrict__ desc,
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
    a.row_base = 0;
    a.R_in = nullptr;
    a.R_out = pb.tri;
    a.cs = pb.cs;
    a.gx = nullptr;
    a.k = 0;
    a.check = 1;
    a.status = status;
    pipe_body<0>(a, d.cta);
}

template <int KMAX, bool GXS>
cudaError_t launch_pipe_kg(const LeafArgs& a, int grid, cudaStream_t s)
{
    const size_t smem = pipe_layout(a.n, KMAX > 0 ? a.k : 0, GXS, a.ring_depth == 4 ? 4 : 2).total;
    auto kern = tsqr_pipe_kernel<KMAX, GXS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, ((a.n + 31) / 32) * 32, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t launch_pipe_k(const LeafArgs& a0, int grid, cudaStream_t s)
{
    const PipeCfg cfg = pipe_cfg(a0.n, KMAX > 0 ? a0.k : 0);
    LeafArgs a = a0;
    a.ring_depth = cfg.depth;
    if (KMAX > 0 && cfg.gxs) return launch_pipe_kg<KMAX, KMAX != 0>(a, grid, s);
    return launch_pipe_kg<KMAX, false>(a, grid, s);
}

template <int KMAX, bool GXS>
int pipe_ctas_per_sm_kg(int n, int k, int depth)
{
    const size_t smem = pipe_layout(n, KMAX > 0 ? k : 0, GXS, depth).total;
    auto kern = tsqr_pipe_kernel<KMAX, GXS>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, ((n + 31) / 32) * 32, smem) != cudaSuccess)
        return 1;
    return blocks < 1 ? 1 : blocks;
}

template <int KMAX>
int pipe_ctas_per_sm_k(int n, int k)
{
    const PipeCfg cfg = pipe_cfg(n, KMAX > 0 ? k : 0);
    if (KMAX > 0 && cfg.gxs) return pipe_ctas_per_sm_kg<KMAX, KMAX != 0>(n, k, cfg.depth);
    return pipe_ctas_per_sm_kg<KMAX, false>(n, k, cfg.depth);
}

}  // namespace

bool pipe_leaf_supported(int n, int k)
{
    static const bool off = [] {
        const char* v = getenv("MRNMF_PIPE_LEAF");
        return v && v[0] == '0';
    }();
    return !off && n > 64 && n <= 256 && k >= 0 && k <= 64 && pipe_layout(n, k).total <= 220 * 1024;
}

int pipe_leaf_rows_per_tile() { return kL; }

int pipe_leaf_ctas_per_sm(int n, int k)
{
    if (k <= 0) return pipe_ctas_per_sm_k<0>(n, 0);
    if (k <= 16) return pipe_ctas_per_sm_k<16>(n, k);
    if (k <= 32) return pipe_ctas_per_sm_k<32>(n, k);
    if (k <= 48) return pipe_ctas_per_sm_k<48>(n, k);
    return pipe_ctas_per_sm_k<64>(n, k);
}

cudaError_t launch_pipe_batched(const BatchCta* desc, int nctas, const BatchProblem* probs, int max_n, int* status,
                                cudaStream_t s)
{
    if (nctas <= 0) return cudaSuccess;
    const size_t smem = pipe_layout(max_n, 0).total;
    cudaError_t e =
        cudaFuncSetAttribute(tsqr_pipe_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tsqr_pipe_batched_kernel<<<nctas, ((max_n + 31) / 32) * 32, smem, s>>>(desc, probs, status);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pipe_leaf(const LeafArgs& a, int grid, cudaStream_t s)
{
    const int k = (a.gx != nullptr && a.k > 0) ? a.k : 0;
    if (k == 0) return launch_pipe_k<0>(a, grid, s);
    if (k <= 16) return launch_pipe_k<16>(a, grid, s);
    if (k <= 32) return launch_pipe_k<32>(a, grid, s);
    if (k <= 48) return launch_pipe_k<48>(a, grid, s);
    return launch_pipe_k<64>(a, grid, s);
}

}  // namespace mrnmf

extern "C" mrnmf_status mrnmf_wait_selftest(int32_t missing, int64_t limit_ns, int32_t* out, int32_t* status,
                                            void* stream)
{
    if (!out || !status || missing < 0 || missing > 3 || limit_ns < 1000 || limit_ns > 1000000000)
        return MRNMF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) return MRNMF_ERR_CUDA;
    mrnmf::wait_selftest_kernel<<<1, 128, 0, s>>>(missing, (uint64_t)limit_ns, reinterpret_cast<int*>(out),
                                                  reinterpret_cast<int*>(status));
    mrnmf::count_launch();
    return cudaGetLastError() == cudaSuccess ? MRNMF_OK : MRNMF_ERR_CUDA;
}
