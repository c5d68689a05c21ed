// group_leaf.cuh -- the lane-group leaf's kernel (tsqr_group.cu describes it),
// shared by the two translation units that instantiate it: tsqr_group.cu for
// n <= 16 and tsqr_group_wide.cu for 17 <= n <= 28.
#pragma once

#include <cstdint>
#include <cstdlib>
#include <utility>

#include "common.cuh"
#include "internal.h"
#include "leaf.h"
#include "tc_common.cuh"

namespace mrnmf {
namespace {


constexpr int kGW = 4;       // warps per CTA: one stream of the pass each
constexpr int kGFlush = 32;  // tiles between binary64 flushes of the column sums
__host__ __device__ constexpr int group_lanes(int n) { return n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32; }
// rows of a fold block (>= n)
__host__ __device__ constexpr int fold_rows(int n) { return n <= 16 ? 16 : 32; }

__host__ __device__ inline size_t gup(size_t b, size_t a) { return (b + a - 1) / a * a; }

// Partial dot products of the 16- and 32-lane groups (n > 8), transposed:
// group g, column c, lane s at g * part_group + c * part_col + s.  The strides keep both
// the stores (a column's S lanes; two 16-lane groups 16 banks apart) and lane
// c's 16-byte loads on distinct banks.
template <int S>
__host__ __device__ constexpr int part_col() { return S + 4; }  // floats per column
template <int S>
__host__ __device__ constexpr int part_group() { return S * part_col<S>() + 16; }  // floats per group

// Per-warp shared memory: [mbarrier | super-tile (32 * 64/S) x n | fold pivots
// 2 x (32/S) x (fold_rows + 4) | partial dots (32/S) x part_group, then update factors
// (32/S) x 32 (n > 8)].  After the tile loop the super-tile area holds the groups'
// triangles for the fold ((32/S) n^2 <= 32 (64/S) n floats).
template <int NC>
__host__ __device__ constexpr bool group_smem_sums() { return group_lanes(NC) >= 16; }

template <int NC>
__host__ __device__ inline size_t group_pub_floats() { return 2 * (32 / group_lanes(NC)) * (fold_rows(NC) + 4); }

template <int NC>
__host__ __device__ inline size_t group_slice_bytes()
{
    constexpr int S = group_lanes(NC), TR = 32 * (64 / S);
    const size_t red = group_smem_sums<NC>() ? sizeof(float) * (32 / S) * (part_group<S>() + 32) : 0;
    return gup(128 + gup(sizeof(float) * (size_t)TR * NC, 128) + sizeof(float) * group_pub_floats<NC>() + red, 128);
}

// Fold steps, column layout: lane s of group g holds column s of a LF-row
// block of the absorbed triangle in a and column s of its own triangle in r.
// Per step j, with p = A(:, j) (published through `pub`) and
// g_c = p . A(:, c), so that sigma = g_j:
//   beta = -sign(alpha) sqrt(alpha^2 + sigma), d = alpha - beta  (alpha = R(j,j)),
//   w'_c = d R(j,c) + g_c,  R(j,c) += w'_c / beta,  A(:,c) += (w'_c / d)(1 / beta) p,
// and R(j,j) = beta; sigma = 0 leaves column j as it is.
template <int NC>
__device__ __forceinline__ void fold_steps(float (&a)[fold_rows(NC)], float (&r)[NC], float* pub, int s, int g)
{
    constexpr int S = group_lanes(NC), NG = 32 / S, kLF = fold_rows(NC), LP = kLF + 4;
    const unsigned FULL = 0xffffffffu;
    const int lead = g * S;
    const bool own = s < NC;
    if (s == 0) {
#pragma unroll
        for (int i = 0; i < kLF; ++i) pub[g * LP + i] = a[i];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const float* pj = pub + ((j & 1) * NG + g) * LP;
        float gc = 0.f;
#pragma unroll
        for (int i = 0; i < kLF; ++i) gc = fmaf(pj[i], a[i], gc);
        const float sig = __shfl_sync(FULL, gc, lead + j);
        const float alpha = __shfl_sync(FULL, r[j], lead + j);
        float f = 0.f;
        if (sig > 0.f) {
            const HhScalars hs = hh_scalars(alpha, sig);
            if (own && s > j) {
                const float wp = fmaf(hs.d, r[j], gc);
                f = (wp * hs.rd) * hs.rb;
                r[j] = fmaf(wp, hs.rb, r[j]);
            } else if (s == j) {
                r[j] = hs.beta;
            }
        }
#pragma unroll
        for (int i = 0; i < kLF; ++i) a[i] = fmaf(f, pj[i], a[i]);
        if (s == j + 1 && j + 1 < NC) {
            float* dst = pub + (((j + 1) & 1) * NG + g) * LP;
#pragma unroll
            for (int i = 0; i < kLF; ++i) dst[i] = a[i];
        }
        __syncwarp();
    }
}

// Column step J of the stacked [R; A] in the row layout: lane s of group g
// holds rows of A in A2 (A2[p][c] = its rows 2p and 2p+1 of column c) and
// column s of R in r.  Same scalars as fold_steps; g_c is summed over the
// group's lanes, and lane c's update factor w'_c / (d beta) is broadcast.
// J is a template parameter so that every register index is static.
template <int NC, int J>
__device__ __forceinline__ void row_step(float2 (&A2)[64 / group_lanes(NC) / 2][NC], float (&r)[NC], int s, int g,
                                         float* red)
{
    constexpr int S = group_lanes(NC), RP = 64 / S / 2;
    const unsigned FULL = 0xffffffffu;
    const int lead = g * S;
    const bool own = s < NC;
    float sig, gs = 0.f;
    if constexpr (group_smem_sums<NC>()) {
        // 16-lane groups: the partials go to shared memory transposed, and lane c
        // sums the 16 of its own column (one fixed tree), so g_c arrives where it
        // is used; sigma = g_J is broadcast from lane J
        constexpr int kPC = part_col<S>();
        float* pg = red + g * part_group<S>();
#pragma unroll
        for (int c = J; c < NC; ++c) {
            float2 acc = __fmul2_rn(A2[0][J], A2[0][c]);
#pragma unroll
            for (int p = 1; p < RP; ++p) acc = __ffma2_rn(A2[p][J], A2[p][c], acc);
            pg[c * kPC + s] = acc.x + acc.y;
        }
        __syncwarp();
        if (s >= J && s < NC) {
            const float4* q = reinterpret_cast<const float4*>(pg + s * kPC);
            const float4 u0 = q[0], u1 = q[1], u2 = q[2], u3 = q[3];
            gs = (((u0.x + u0.y) + (u0.z + u0.w)) + ((u1.x + u1.y) + (u1.z + u1.w))) +
                 (((u2.x + u2.y) + (u2.z + u2.w)) + ((u3.x + u3.y) + (u3.z + u3.w)));
            if constexpr (S == 32) {
                const float4 u4 = q[4], u5 = q[5], u6 = q[6], u7 = q[7];
                gs += (((u4.x + u4.y) + (u4.z + u4.w)) + ((u5.x + u5.y) + (u5.z + u5.w))) +
                      (((u6.x + u6.y) + (u6.z + u6.w)) + ((u7.x + u7.y) + (u7.z + u7.w)));
            }
        }
        __syncwarp();  // every read of this step's partials is done before the next step writes
        sig = __shfl_sync(FULL, gs, lead + J);
    } else {
        float gv[NC];
#pragma unroll
        for (int c = J; c < NC; ++c) {
            float2 acc = __fmul2_rn(A2[0][J], A2[0][c]);
#pragma unroll
            for (int p = 1; p < RP; ++p) acc = __ffma2_rn(A2[p][J], A2[p][c], acc);
            gv[c] = acc.x + acc.y;
        }
        // group sums (a butterfly: every lane adds the same operands in the same tree)
#pragma unroll
        for (int o = 1; o < S; o <<= 1) {
#pragma unroll
            for (int c = J; c < NC; ++c) gv[c] += __shfl_xor_sync(FULL, gv[c], o);
        }
        sig = gv[J];
#pragma unroll
        for (int c = J + 1; c < NC; ++c) gs = (s == c) ? gv[c] : gs;
    }
    const float alpha = __shfl_sync(FULL, r[J], lead + J);
    float fs = 0.f;
    if (sig > 0.f) {
        const HhScalars hs = hh_scalars(alpha, sig);
        if (own && s > J) {
            const float wp = fmaf(hs.d, r[J], gs);
            fs = (wp * hs.rd) * hs.rb;
            r[J] = fmaf(wp, hs.rb, r[J]);
        } else if (s == J) {
            r[J] = hs.beta;
        }
    }
    if constexpr (group_smem_sums<NC>()) {
        // 16- and 32-lane groups: lane c publishes its factor, and every lane
        // reads the live ones as broadcast 16-byte loads (one load per four
        // columns instead of a shuffle per column).  The next step's factors
        // are written only after its partial sums, which every lane reaches
        // after these reads.
        float* fb = red + (32 / S) * part_group<S>() + g * 32;
        if (own && s > J) fb[s] = fs;
        __syncwarp();
#pragma unroll
        for (int c4 = (J + 1) & ~3; c4 < NC; c4 += 4) {
            const float4 f = *reinterpret_cast<const float4*>(fb + c4);
            const float fv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c4 + u;
                if (c > J && c < NC) {
                    const float2 f2 = make_float2(fv[u], fv[u]);
#pragma unroll
                    for (int p = 0; p < RP; ++p) A2[p][c] = __ffma2_rn(f2, A2[p][J], A2[p][c]);
                }
            }
        }
    } else {
#pragma unroll
        for (int c = J + 1; c < NC; ++c) {
            const float fc = __shfl_sync(FULL, fs, lead + c);
            const float2 f2 = make_float2(fc, fc);
#pragma unroll
            for (int p = 0; p < RP; ++p) A2[p][c] = __ffma2_rn(f2, A2[p][J], A2[p][c]);
        }
    }
}

template <int NC, int... J>
__device__ __forceinline__ void row_steps_seq(float2 (&A2)[64 / group_lanes(NC) / 2][NC], float (&r)[NC], int s, int g,
                                              float* red, std::integer_sequence<int, J...>)
{
    (row_step<NC, J>(A2, r, s, g, red), ...);
}

// Column steps 0 .. NC-1 of one block.
template <int NC>
__device__ __forceinline__ void row_steps(float2 (&A2)[64 / group_lanes(NC) / 2][NC], float (&r)[NC], int s, int g,
                                          float* red)
{
    row_steps_seq<NC>(A2, r, s, g, red, std::make_integer_sequence<int, NC>{});
}

template <int NC>
__device__ __forceinline__ void set_row(float2 (&A2)[64 / group_lanes(NC) / 2][NC], int p, int h, int c, float v)
{
    if (h) A2[p][c].y = v;
    else A2[p][c].x = v;
}

// Residency: 4 CTAs per SM for n <= 16 (at most 128 registers a thread; no
// width spills more than a few bytes there, several do at 5); 3 above, where
// the rows, the triangle's column and the column sums of 32 columns need
// more than 128.
__host__ __device__ constexpr int group_min_ctas(int n) { return n <= 16 ? 4 : 3; }

template <int NC>
__global__ void __launch_bounds__(kGW * 32, group_min_ctas(NC)) tsqr_group_kernel(const LeafArgs a)
{
    constexpr int S = group_lanes(NC), NG = 32 / S, RL = 64 / S, RP = RL / 2, TR = 32 * RL;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / S, s = lane % S;
    const int cta = blockIdx.x;
    const int ws = cta * kGW + warp;  // the pass's stream = partial-sum slot
    const unsigned FULL = 0xffffffffu;
    const bool own = s < NC;

    unsigned char* base = smem + (size_t)warp * group_slice_bytes<NC>();
    uint64_t* bar = reinterpret_cast<uint64_t*>(base);
    float* tile = reinterpret_cast<float*>(base + 128);
    float* pub = tile + gup((size_t)TR * NC, 32);
    float* red = pub + group_pub_floats<NC>();  // partial dots (16-lane groups)
    if (lane == 0) tc::mbar_init(bar, 1);
    __syncwarp();

    // running triangle: group 0 of warp 0 continues from the CTA's state slot
    // (zeros on a fresh pass), every other group starts from zero
    float r[NC];
    {
        const float* Rin = static_cast<const float*>(a.R_in);
        const bool cont = Rin != nullptr && warp == 0 && g == 0 && own;
#pragma unroll
        for (int i = 0; i < NC; ++i) r[i] = (cont && i <= s) ? Rin[(size_t)cta * NC * NC + (size_t)i * NC + s] : 0.f;
    }

    const int64_t r0 = (int64_t)ws * a.rows_per_cta;
    const int64_t r1 = min(a.rows, r0 + a.rows_per_cta);
    const int64_t ntiles = r1 > r0 ? (r1 - r0 + TR - 1) / TR : 0;
    const float* X = static_cast<const float*>(a.X);
    const bool tma_ok = a.ldx == NC && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const uint32_t bar_s = tc::smem_addr(bar);

    // Issue the bulk copy of super-tile t; false if it must be loaded directly.
    auto issue = [&](int64_t t) -> bool {
        const int64_t row0 = r0 + t * TR;
        const int rows_v = (int)min((int64_t)TR, r1 - row0);
        const uint32_t bytes = (uint32_t)rows_v * (uint32_t)NC * 4u;
        if (!tma_ok || (bytes & 15u)) return false;
        if (lane == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_addr(tile)),
                "l"(X + row0 * NC), "r"(bytes), "r"(bar_s)
                : "memory");
        }
        return true;
    };

    float2 A2[RP][NC];
    float cs[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) cs[c] = 0.f;
    bool bad = false;
    uint32_t phase = 0;
    bool inflight = ntiles > 0 ? issue(0) : false;

    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t row0 = r0 + t * TR;
        const int rows_v = (int)min((int64_t)TR, r1 - row0);
        if (inflight) {
            // warp-uniform decision, so no lane leaves while others still shuffle
            if (!__all_sync(FULL, tc::mbar_wait(bar, phase))) {
                if (lane == 0) set_status(a.status, MRNMF_ERR_TIMEOUT);
                tc::mbar_wait(bar, phase);  // bounded second wait for the copy in flight
                break;
            }
            phase ^= 1u;
            // row (2p + h) * 32 + lane of the super-tile -> A2[p][.].{x, y}
#pragma unroll
            for (int p = 0; p < RP; ++p) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int row = (2 * p + h) * 32 + lane;
                    const bool v = row < rows_v;
                    const float* src = tile + (size_t)row * NC;
                    if constexpr (NC % 4 == 0) {
#pragma unroll
                        for (int q = 0; q < NC / 4; ++q) {
                            const float4 w =
                                v ? reinterpret_cast<const float4*>(src)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                            set_row<NC>(A2, p, h, 4 * q, w.x);
                            set_row<NC>(A2, p, h, 4 * q + 1, w.y);
                            set_row<NC>(A2, p, h, 4 * q + 2, w.z);
                            set_row<NC>(A2, p, h, 4 * q + 3, w.w);
                        }
                    } else if constexpr (NC % 2 == 0) {
#pragma unroll
                        for (int q = 0; q < NC / 2; ++q) {
                            const float2 w = v ? reinterpret_cast<const float2*>(src)[q] : make_float2(0.f, 0.f);
                            set_row<NC>(A2, p, h, 2 * q, w.x);
                            set_row<NC>(A2, p, h, 2 * q + 1, w.y);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < NC; ++c) set_row<NC>(A2, p, h, c, v ? src[c] : 0.f);
                    }
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < RP; ++p) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int row = (2 * p + h) * 32 + lane;
                    const bool v = row < rows_v;
                    const float* src = X + (row0 + row) * a.ldx;
#pragma unroll
                    for (int c = 0; c < NC; ++c) set_row<NC>(A2, p, h, c, v ? src[c] : 0.f);
                }
            }
        }
        __syncwarp();
        if (t + 1 < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            inflight = issue(t + 1);
        } else {
            inflight = false;
        }

        // column sums (Sec. 3.3) and the input check: the OR of the raw words
        // has its sign bit set if any entry does, and a NaN makes a sum NaN;
        // only then are the entries tested one by one (-0 is accepted).
        {
            uint32_t ob = 0;
            float tot = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float2 t2 = A2[0][c];
                ob |= __float_as_uint(A2[0][c].x) | __float_as_uint(A2[0][c].y);
#pragma unroll
                for (int p = 1; p < RP; ++p) {
                    t2 = __fadd2_rn(t2, A2[p][c]);
                    ob |= __float_as_uint(A2[p][c].x) | __float_as_uint(A2[p][c].y);
                }
                const float ts = t2.x + t2.y;
                cs[c] += ts;
                tot += ts;
            }
            if ((ob >> 31) || !(tot >= 0.f)) {
#pragma unroll
                for (int p = 0; p < RP; ++p)
#pragma unroll
                    for (int c = 0; c < NC; ++c) bad |= !(A2[p][c].x >= 0.f) || !(A2[p][c].y >= 0.f);
            }
        }

        row_steps<NC>(A2, r, s, g, red);

        if ((t + 1) % kGFlush == 0 || t + 1 == ntiles) {
            float mine = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float v = cs[c];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) v += __shfl_xor_sync(FULL, v, o);
                mine = (lane == c) ? v : mine;
                cs[c] = 0.f;
            }
            if (a.cs && lane < NC) a.cs[(size_t)ws * NC + lane] += (double)mine;
        }
    }

    if (a.check && __any_sync(FULL, bad)) {
        if (lane == 0) set_status(a.status, MRNMF_ERR_BAD_INPUT);
    }

    // Fold the CTA's kGW * NG triangles into that of group 0 of warp 0: in
    // round h the triangle of id + h (id = warp * NG + g) is absorbed by that
    // of id, for id a multiple of 2h, loaded as an NC-row block.
    constexpr int T = kGW * NG;
    const int id = warp * NG + g;
    for (int h = 1; h < T; h <<= 1) {
        __syncthreads();
        if ((id & (2 * h - 1)) == h && own) {
            float* slot = tile + (size_t)g * NC * NC;
#pragma unroll
            for (int i = 0; i < NC; ++i) slot[i * NC + s] = (i <= s) ? r[i] : 0.f;
        }
        __syncthreads();
        const bool recv = (id & (2 * h - 1)) == 0;
        if (__any_sync(FULL, recv)) {
            const int src = min(id + h, T - 1);
            const float* slot =
                reinterpret_cast<const float*>(smem + (size_t)(src / NG) * group_slice_bytes<NC>() + 128) +
                (size_t)(src % NG) * NC * NC;
            float fa[fold_rows(NC)];
#pragma unroll
            for (int i = 0; i < fold_rows(NC); ++i) fa[i] = (recv && own && i < NC) ? slot[i * NC + s] : 0.f;
            __syncwarp();
            fold_steps<NC>(fa, r, pub, s, g);
        }
    }
    if (warp == 0 && g == 0 && own) {
        float* Rout = static_cast<float*>(a.R_out) + (size_t)cta * NC * NC;
#pragma unroll
        for (int i = 0; i < NC; ++i) Rout[(size_t)i * NC + s] = (i <= s) ? r[i] : 0.f;
    }
}

template <int NC>
cudaError_t launch_group(const LeafArgs& a, int streams, cudaStream_t s)
{
    const size_t smem = (size_t)kGW * group_slice_bytes<NC>();
    auto kern = tsqr_group_kernel<NC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (streams + kGW - 1) / kGW;
    kern<<<grid, kGW * 32, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int NC>
int group_ctas()
{
    const size_t smem = (size_t)kGW * group_slice_bytes<NC>();
    auto kern = tsqr_group_kernel<NC>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kGW * 32, smem) != cudaSuccess) return 1;
    return blocks < 1 ? 1 : blocks;
}

}  // namespace

// Launch and residency of the instantiations of one translation unit
// (narrow: n <= 16 in tsqr_group.cu; wide: 17 <= n <= 28 in tsqr_group_wide.cu).
cudaError_t group_launch_narrow(const LeafArgs& a, int streams, cudaStream_t s);
int group_ctas_narrow(int n);
cudaError_t group_launch_wide(const LeafArgs& a, int streams, cudaStream_t s);
int group_ctas_wide(int n);

}  // namespace mrnmf
