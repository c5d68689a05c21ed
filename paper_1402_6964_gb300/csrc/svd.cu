// svd.cu -- the R-SVD form (Sec. 2.2: X = QR, R = U Sigma V', so
// X = (QU) Sigma V' and the separable step can run on Sigma V' in place of R;
// the experiments of Sec. 4 select on Sigma V').
//
// One-sided Jacobi (Hestenes 1958) on B = R': plane rotations from the right
// orthogonalise B's columns, B U = V Sigma with U orthogonal, so the final
// columns are sigma_i v_i and their transpose is Sigma V' -- U itself is never
// needed.  Rotation of columns (i, j) with a = |b_i|^2, b = |b_j|^2,
// g = b_i'b_j (Rutishauser's formulas): zeta = (b - a) / (2g),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t,
// b_i <- c b_i - s b_j, b_j <- s b_i + c b_j; skipped when
// |g| <= eps sqrt(a b).  Sweeps visit every pair once in round-robin order
// (n/2 disjoint pairs per round, one single-warp CTA per pair, a grid-wide
// barrier between rounds in a cooperative launch: binary64 runs at 1/64 of
// the binary32 rate on GB300, so the pairs go to separate SMs) until a sweep
// rotates nothing.  binary64 throughout, B in global memory (L2-resident).
#include <cooperative_groups.h>

#include <string>

#include "../../include/mrnmf.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"
#include "trace.h"

namespace mrnmf {
namespace {

constexpr int kMaxSweeps = 40;

// Players of the round-robin: N (even) columns, player N-1 fixed; in round k
// pair q (< N/2) is (k, N-1) for q = 0, else ((k + q) mod (N-1), (k - q) mod (N-1)).
__device__ __forceinline__ void rr_pair(int N, int k, int q, int& i, int& j)
{
    const int M = N - 1;
    if (q == 0) {
        i = k;
        j = M;
    } else {
        i = (k + q) % M;
        j = (k - q + M) % M;
    }
    if (i > j) {
        const int t = i;
        i = j;
        j = t;
    }
}

// B: n x n column-major (column c at B + c * n), N = n rounded up to even (a
// padding column, if any, is zero and never rotated).  Grid: N/2 CTAs of one
// warp; CTA q rotates pair q of every round.  flags[0] counts the rotations
// of the current sweep.
__global__ void __launch_bounds__(32) jacobi_svd_kernel(const double* __restrict__ R, int n, double* __restrict__ B,
                                                        unsigned int* __restrict__ flags,
                                                        double* __restrict__ sigma, double* __restrict__ SVt,
                                                        int* status)
{
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    __shared__ double norms[256];
    const int lane = threadIdx.x, q = blockIdx.x;
    const int N = (n + 1) & ~1;
    // B = R': column c of B is row c of R (the same bytes)
    for (int e = q * 32 + lane; e < n * n; e += gridDim.x * 32) B[e] = R[e];
    if (q == 0 && lane == 0) flags[0] = 0;
    grid.sync();
    const double eps = 1e-15;
    bool converged = false;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        for (int k = 0; k < N - 1; ++k) {
            int i, j;
            rr_pair(N, k, q, i, j);
            if (j < n) {
                double* bi = B + (size_t)i * n;
                double* bj = B + (size_t)j * n;
                double a = 0.0, b = 0.0, g = 0.0;
                // columns other CTAs rotated in earlier rounds: read through L2 (__ldcg)
                for (int e = lane; e < n; e += 32) {
                    const double x = __ldcg(bi + e), y = __ldcg(bj + e);
                    a = fma(x, x, a);
                    b = fma(y, y, b);
                    g = fma(x, y, g);
                }
                a = warp_sum(a);
                b = warp_sum(b);
                g = warp_sum(g);
                if (fabs(g) > eps * sqrt(a * b)) {
                    const double zeta = (b - a) / (2.0 * g);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    for (int e = lane; e < n; e += 32) {
                        const double x = __ldcg(bi + e), y = __ldcg(bj + e);
                        bi[e] = c * x - s * y;
                        bj[e] = s * x + c * y;
                    }
                    if (lane == 0) atomicAdd(&flags[0], 1u);
                }
            }
            grid.sync();
        }
        // every CTA reads the sweep's count, then CTA 0 resets it for the next sweep
        const unsigned int rot = *((volatile unsigned int*)&flags[0]);
        grid.sync();
        if (q == 0 && lane == 0) flags[0] = 0;
        grid.sync();
        if (rot == 0) {
            converged = true;
            break;
        }
    }
    if (q != 0) return;
    if (!converged && lane == 0) set_status(status, MRNMF_ERR_NOT_CONVERGED);
    // sigma_c = |B(:,c)|; rows of Sigma V' in descending sigma (ties: lower column first)
    for (int c = 0; c < n; ++c) {
        double s2 = 0.0;
        for (int e = lane; e < n; e += 32) {
            const double x = __ldcg(B + (size_t)c * n + e);
            s2 = fma(x, x, s2);
        }
        s2 = warp_sum(s2);
        if (lane == 0) norms[c] = sqrt(s2);
    }
    __syncwarp();
    for (int c = 0; c < n; ++c) {
        const double sc = norms[c];
        int rank = 0;
        for (int o = lane; o < n; o += 32) rank += (norms[o] > sc || (norms[o] == sc && o < c)) ? 1 : 0;
        for (int off = 16; off; off >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, off);
        if (lane == 0 && sigma) sigma[rank] = sc;
        for (int e = lane; e < n; e += 32) SVt[(size_t)rank * n + e] = __ldcg(B + (size_t)c * n + e);
    }
}

}  // namespace
}  // namespace mrnmf

using mrnmf::api::bind_device;
using mrnmf::api::cuda_fail;
using mrnmf::api::fail;
using mrnmf::api::grow;

extern "C" mrnmf_status mrnmf_r_svd(mrnmf_handle* h, const double* R, int32_t n, double* sigma, double* SVt,
                                    void* stream)
{
    MRNMF_TRACE("mrnmf_r_svd");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!R || !SVt) return fail(h, MRNMF_ERR_INVALID_ARG, "R and SVt are required");
    if (n < 1 || n > MRNMF_NMAX) return fail(h, MRNMF_ERR_INVALID_ARG, "n must be in [1, 256]");
    mrnmf_status st = bind_device(h);
    if (st != MRNMF_OK) return st;
    if ((st = grow(h, &h->svd, &h->svd_bytes, 8ull * n * n + 64, "R-SVD scratch")) != MRNMF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* B = static_cast<double*>(h->svd);
    unsigned int* flags = reinterpret_cast<unsigned int*>(B + (size_t)n * n);
    int nn = n;
    int* status = h->d_status;
    void* args[] = {(void*)&R, (void*)&nn, (void*)&B, (void*)&flags, (void*)&sigma, (void*)&SVt, (void*)&status};
    const int grid = ((n + 1) & ~1) / 2;
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)mrnmf::jacobi_svd_kernel, dim3(grid > 0 ? grid : 1),
                                                dim3(32), args, 0, s);
    mrnmf::count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? MRNMF_OK : cuda_fail(h, e, "R-SVD");
}
