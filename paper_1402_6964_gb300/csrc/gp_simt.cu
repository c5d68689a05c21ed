// gp_simt.cu -- the Gaussian projection pass without the triangle (Sec. 2.3;
// Algorithm 1 with the combiner of Sec. 3.2) on the SIMT cores, for
// n <= 64 and k <= 32: GX = G'X and the column sums of X (Sec. 3.3).
//
// One warp per row stream, four streams per CTA, no block barriers.  Tiles of
// 32 consecutive rows are staged into the warp's shared memory by a bulk copy
// (cp.async.bulk on an mbarrier, every wait bounded), one tile ahead of the
// arithmetic.  Per tile:
//   - lane l draws row l of G (k Gaussians: Philox4x32-10 and Box-Muller,
//     keyed by the global row, the same generator as the fused leaves) into a
//     coordinate-major buffer, G(q, 0..31) contiguous;
//   - lane l holds column l of the tile (and l + 32 when n > 32) in registers;
//   - for each coordinate q, lane l forms G(q,:) . X(:, c) for its columns with
//     packed FMAs (even and odd rows in the two halves of a float2, rows 0-15
//     and 16-31 in separate chains), reading G(q,:) as broadcast 16-byte loads,
//     and adds it to its binary32 partial GX(q, c) in shared memory;
//   - every 32 tiles, and at the end, the partials are added to the stream's
//     binary64 slot (P x k x n), as are the column sums (P x n).
// Column c's partials belong to the lane that holds column c, so no lane reads
// another's accumulator.  The triangle is not formed: this is the pass for
// GP alone.
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "leaf.h"
#include "tc_common.cuh"

namespace mrnmf {

namespace {

constexpr int kPW = 4;       // warps (row streams) per CTA
constexpr int kPL = 32;      // rows per tile
constexpr int kPFlush = 32;  // tiles between binary64 flushes

__host__ __device__ inline size_t pup(size_t b, size_t a) { return (b + a - 1) / a * a; }

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Per-warp shared memory: [mbarrier (128 B) | tile 32 x n | G tile kp x 32 | partial GX kp x n].
__host__ __device__ inline size_t gp_slice_bytes(int n, int k)
{
    const size_t kp = (size_t)((k + 3) & ~3);
    return pup(128 + pup(sizeof(float) * kPL * (size_t)n, 128) + sizeof(float) * kp * kPL + sizeof(float) * kp * n,
               128);
}

// NC = 1: n <= 32 (one column a lane); NC = 2: 33 <= n <= 64 (two).
template <int NC>
__global__ void __launch_bounds__(kPW * 32, 4) gp_warp_kernel(const LeafArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int n = a.n, k = a.k;
    const int kp = (k + 3) & ~3, kq = kp >> 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ws = blockIdx.x * kPW + warp;  // stream = partial-sum slot
    const unsigned FULL = 0xffffffffu;

    unsigned char* base = smem + (size_t)warp * gp_slice_bytes(n, k);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base);
    float* tile = reinterpret_cast<float*>(base + 128);
    float* gbuf = tile + pup((size_t)kPL * n, 32);
    float* gxs = gbuf + (size_t)kp * kPL;

    const int c0 = lane, c1 = lane + 32;
    const bool own0 = c0 < n, own1 = NC == 2 && c1 < n;
    if (lane == 0) tc::mbar_init(bar, 1);
    for (int e = lane; e < kp * n; e += 32) gxs[e] = 0.f;
    __syncwarp();

    const int64_t r0 = (int64_t)ws * a.rows_per_cta;
    const int64_t r1 = min(a.rows, r0 + a.rows_per_cta);
    const int64_t ntiles = r1 > r0 ? (r1 - r0 + kPL - 1) / kPL : 0;
    const float* X = static_cast<const float*>(a.X);
    const bool tma_ok = a.ldx == n && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const uint32_t bar_s = tc::smem_addr(bar);

    // Issue the bulk copy of tile t; false if it must be loaded directly.
    auto issue = [&](int64_t t) -> bool {
        const int64_t row0 = r0 + t * kPL;
        const int rows_v = (int)min((int64_t)kPL, r1 - row0);
        const uint32_t bytes = (uint32_t)rows_v * (uint32_t)n * 4u;
        if (!tma_ok || (bytes & 15u)) return false;
        if (lane == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_addr(tile)),
                "l"(X + row0 * n), "r"(bytes), "r"(bar_s)
                : "memory");
        }
        return true;
    };
    // Row l of G for tile t (zeros past the stream's last row).
    auto draw = [&](int64_t t) {
        const int64_t row0 = r0 + t * kPL;
        const bool v = row0 + lane < r1;
        const int64_t grow = a.row_base + row0 + lane;
#pragma unroll 2
        for (int q4 = 0; q4 < kq; ++q4) {
            const float4 g = v ? gauss4(a.seed, grow, (uint32_t)q4) : make_float4(0.f, 0.f, 0.f, 0.f);
            gbuf[(4 * q4 + 0) * kPL + lane] = g.x;
            gbuf[(4 * q4 + 1) * kPL + lane] = g.y;
            gbuf[(4 * q4 + 2) * kPL + lane] = g.z;
            gbuf[(4 * q4 + 3) * kPL + lane] = g.w;
        }
    };

    float x0[kPL], x1[NC == 2 ? kPL : 1];
    float cs0 = 0.f, cs1 = 0.f;
    bool bad = false;
    uint32_t phase = 0;
    bool inflight = ntiles > 0 ? issue(0) : false;
    if (ntiles > 0) draw(0);

    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t row0 = r0 + t * kPL;
        const int rows_v = (int)min((int64_t)kPL, r1 - row0);
        if (inflight) {
            // warp-uniform decision, so no lane leaves while others still shuffle
            if (!__all_sync(FULL, tc::mbar_wait(bar, phase))) {
                if (lane == 0) set_status(a.status, MRNMF_ERR_TIMEOUT);
                tc::mbar_wait(bar, phase);  // bounded second wait for the copy in flight
                break;
            }
            phase ^= 1u;
#pragma unroll
            for (int l = 0; l < kPL; ++l) {
                x0[l] = (own0 && l < rows_v) ? tile[l * n + c0] : 0.f;
                if (NC == 2) x1[l] = (own1 && l < rows_v) ? tile[l * n + c1] : 0.f;
            }
        } else {
            const float* src = X + row0 * a.ldx;
#pragma unroll
            for (int l = 0; l < kPL; ++l) {
                x0[l] = (own0 && l < rows_v) ? src[(int64_t)l * a.ldx + c0] : 0.f;
                if (NC == 2) x1[l] = (own1 && l < rows_v) ? src[(int64_t)l * a.ldx + c1] : 0.f;
            }
        }
        __syncwarp();  // the tile is read and this tile's G is written
        if (t + 1 < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            inflight = issue(t + 1);
        } else {
            inflight = false;
        }

        // column sums and the input check (-0 passes, a negative entry or NaN does not)
        {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int l = 0; l < kPL; ++l) {
                bad |= !(x0[l] >= 0.f);
                s0 += x0[l];
                if (NC == 2) {
                    bad |= !(x1[l] >= 0.f);
                    s1 += x1[l];
                }
            }
            cs0 += s0;
            cs1 += s1;
        }

        // GX(q, c) += G(q, :) . X(:, c)
        for (int q = 0; q < k; ++q) {
            const float4* gq = reinterpret_cast<const float4*>(gbuf + q * kPL);
            float2 p0 = make_float2(0.f, 0.f), p2 = p0, p1 = p0, p3 = p0;
#pragma unroll
            for (int l4 = 0; l4 < kPL / 8; ++l4) {
                const float4 g = gq[l4], h = gq[l4 + kPL / 8];
                const int l = 4 * l4, m = kPL / 2 + 4 * l4;
                p0 = __ffma2_rn(make_float2(g.x, g.y), make_float2(x0[l], x0[l + 1]), p0);
                p0 = __ffma2_rn(make_float2(g.z, g.w), make_float2(x0[l + 2], x0[l + 3]), p0);
                p2 = __ffma2_rn(make_float2(h.x, h.y), make_float2(x0[m], x0[m + 1]), p2);
                p2 = __ffma2_rn(make_float2(h.z, h.w), make_float2(x0[m + 2], x0[m + 3]), p2);
                if (NC == 2) {
                    p1 = __ffma2_rn(make_float2(g.x, g.y), make_float2(x1[l], x1[l + 1]), p1);
                    p1 = __ffma2_rn(make_float2(g.z, g.w), make_float2(x1[l + 2], x1[l + 3]), p1);
                    p3 = __ffma2_rn(make_float2(h.x, h.y), make_float2(x1[m], x1[m + 1]), p3);
                    p3 = __ffma2_rn(make_float2(h.z, h.w), make_float2(x1[m + 2], x1[m + 3]), p3);
                }
            }
            if (own0) gxs[q * n + c0] += (p0.x + p0.y) + (p2.x + p2.y);
            if (NC == 2 && own1) gxs[q * n + c1] += (p1.x + p1.y) + (p3.x + p3.y);
        }
        __syncwarp();  // every read of this tile's G is done
        if (t + 1 < ntiles) draw(t + 1);

        if ((t + 1) % kPFlush == 0 || t + 1 == ntiles) {
            if (a.cs) {
                if (own0) a.cs[(size_t)ws * n + c0] += (double)cs0;
                if (own1) a.cs[(size_t)ws * n + c1] += (double)cs1;
            }
            cs0 = cs1 = 0.f;
            if (a.gx) {
                double* gxo = a.gx + (size_t)ws * k * n;
                for (int q = 0; q < k; ++q) {
                    if (own0) {
                        gxo[(size_t)q * n + c0] += (double)gxs[q * n + c0];
                        gxs[q * n + c0] = 0.f;
                    }
                    if (own1) {
                        gxo[(size_t)q * n + c1] += (double)gxs[q * n + c1];
                        gxs[q * n + c1] = 0.f;
                    }
                }
            }
        }
    }

    if (a.check && __any_sync(FULL, bad)) {
        if (lane == 0) set_status(a.status, MRNMF_ERR_BAD_INPUT);
    }
}

template <int NC>
cudaError_t launch_nc(const LeafArgs& a, int streams, cudaStream_t s)
{
    const size_t smem = (size_t)kPW * gp_slice_bytes(a.n, a.k);
    auto kern = gp_warp_kernel<NC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<streams / kPW, kPW * 32, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int NC>
int ctas_nc(int n, int k)
{
    const size_t smem = (size_t)kPW * gp_slice_bytes(n, k);
    auto kern = gp_warp_kernel<NC>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kPW * 32, smem) != cudaSuccess) return 1;
    return blocks < 1 ? 1 : blocks;
}

}  // namespace

bool gp_warp_supported(int n, int k)
{
    static const bool on = [] {
        const char* v = getenv("MRNMF_GP_WARP");
        return !(v && v[0] == '0');
    }();
    return on && n >= 1 && n <= 64 && k >= 1 && k <= 32;
}

int gp_warp_rows_per_tile() { return kPL; }
int gp_warp_streams_per_cta() { return kPW; }

int gp_warp_streams(int n, int k, int64_t m)
{
    const int per_sm = n <= 32 ? ctas_nc<1>(n, k) : ctas_nc<2>(n, k);
    int P = sm_count() * per_sm * kPW;
    if (m > 0) {
        const int64_t minrows = 2 * (int64_t)kPL;  // at least two tiles a stream
        const int64_t cap = (m + minrows - 1) / minrows;
        if (cap < P) P = (int)cap;
    }
    return P < kPW ? kPW : (P + kPW - 1) / kPW * kPW;
}

cudaError_t launch_gp_warp(const LeafArgs& a, int streams, cudaStream_t s)
{
    if (!gp_warp_supported(a.n, a.k) || streams % kPW != 0 || a.rows_per_cta % kPL != 0) return cudaErrorInvalidValue;
    return a.n <= 32 ? launch_nc<1>(a, streams, s) : launch_nc<2>(a, streams, s);
}

}  // namespace mrnmf
