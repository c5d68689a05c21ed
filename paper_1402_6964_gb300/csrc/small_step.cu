// small_step.cu -- the n-by-n separable step on the device, in binary64.
//
// Once the pass has produced R (n-by-n) and the column sums, X = X(:,K)H
// implies R = R(:,K)H (Sec. 2.2), so the extreme columns, the coefficients
// and the residual are all computed from R:
//   SPA       Sec. 2.1 (argmax of column 2-norms of R D^-1, then projection)
//   XRAY      Sec. 2.1 (greedy: argmax ||Res^T R(:,j)|| / ||R(:,j)||)
//   GP        Sec. 2.3 + Sec. 3.3 (argmax / argmin of the rows of GX D^-1)
//   NNLS      Sec. 2.4 (Lawson-Hanson active set on the normal equations)
//   residual  Sec. 2.4 / Sec. 4
// Ties go to the lowest index.  Work is O(n^2 r) to O(n^3 r): small next to
// the pass, and on GB300 binary64 runs on few units, so each kernel spreads
// its columns over threads and blocks.

#include <cfloat>
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace mrnmf {

namespace {

constexpr int kRMax = 64;  // largest r the NNLS scratch is laid out for

// ---------------------------------------------------------------- top-2 argmax
struct Top2 {
    double b1;
    int i1;
    double b2;
};

__device__ __forceinline__ Top2 top2_merge(Top2 a, Top2 b)
{
    // the better best (lowest index on ties); the second is the larger of the
    // loser's best and the winner's second
    const bool a_wins = (a.b1 > b.b1) || (a.b1 == b.b1 && a.i1 < b.i1);
    Top2 w = a_wins ? a : b, l = a_wins ? b : a;
    w.b2 = fmax(w.b2, l.b1);
    return w;
}

// Block-wide top-2 over one value per thread (score = -inf for excluded).
__device__ Top2 block_top2(double v, int idx, Top2* sh)
{
    Top2 t{v, idx, -INFINITY};
    for (int o = 16; o; o >>= 1) {
        Top2 u;
        u.b1 = __shfl_xor_sync(0xffffffffu, t.b1, o);
        u.i1 = __shfl_xor_sync(0xffffffffu, t.i1, o);
        u.b2 = __shfl_xor_sync(0xffffffffu, t.b2, o);
        t = top2_merge(t, u);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        Top2 acc = sh[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) acc = top2_merge(acc, sh[q]);
        sh[0] = acc;
    }
    __syncthreads();
    Top2 r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double pick_gap(const Top2& t)
{
    if (t.i1 < 0 || t.b1 == -INFINITY) return -1.0;
    if (t.b2 == -INFINITY) return 1.0;
    return t.b1 > 0.0 ? (t.b1 - t.b2) / t.b1 : 0.0;
}

// ------------------------------------------------------------------------ SPA
// One CTA.  Column j of Y = R D^-1 is held by a group of G consecutive
// threads (G divides 32), which split its rows: binary64 runs on few units
// per SM on GB300, so the column work is spread over all four sub-partitions.
// Y is kept column-major with an odd leading dimension, in shared memory when
// it fits (else in the global scratch).
template <int G>
__global__ void __launch_bounds__(256) spa_kernel(const double* __restrict__ R, int n, const double* __restrict__ colsum,
                                                  int r, int32_t* __restrict__ K, double* __restrict__ gap,
                                                  double* __restrict__ Yg, int y_in_smem)
{
    extern __shared__ double ydyn[];
    __shared__ Top2 sh[8];
    __shared__ double u[MRNMF_NMAX];
    __shared__ int chosen[MRNMF_NMAX];
    __shared__ double s_inv, s_f0;
    __shared__ int s_p;
    const unsigned FULL = 0xffffffffu;
    const int ld = n | 1;
    double* Y = y_in_smem ? ydyn : Yg;
    const int t = threadIdx.x, j = t / G, part = t - j * G;
    const bool own = j < n;
    for (int e = t; e < n * n; e += blockDim.x) {
        const int i = e / n, c = e - i * n;
        Y[(size_t)c * ld + i] = R[e] / colsum[c];
    }
    for (int c = t; c < n; c += blockDim.x) chosen[c] = 0;
    __syncthreads();
    for (int step = 0; step < r; ++step) {
        const bool cand = own && !chosen[j];
        const double* yj = Y + (size_t)(own ? j : 0) * ld;
        double f = 0.0;
        if (cand)
            for (int i = part; i < n; i += G) f = fma(yj[i], yj[i], f);
#pragma unroll
        for (int o = G / 2; o; o >>= 1) f += __shfl_xor_sync(FULL, f, o);
        const bool lead = cand && part == 0;
        const Top2 b = block_top2(lead ? f : -INFINITY, lead ? j : INT_MAX, sh);
        if (t == 0) {
            const int p = b.i1;
            if (step == 0) s_f0 = b.b1;
            double g = pick_gap(b);
            if (!(b.b1 > 1e-24 * s_f0)) g = -1.0;
            K[step] = p;
            if (gap) gap[step] = g;
            chosen[p] = 1;
            s_p = p;
            const double nrm = sqrt(b.b1);
            s_inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        }
        __syncthreads();
        const int p = s_p;
        const double inv = s_inv;
        if (!(inv > 0.0)) continue;
        for (int i = t; i < n; i += blockDim.x) u[i] = Y[(size_t)p * ld + i] * inv;
        __syncthreads();
        // project the chosen direction out of the remaining candidates
        const bool upd = own && !chosen[j];
        double c = 0.0;
        if (upd)
            for (int i = part; i < n; i += G) c = fma(u[i], yj[i], c);
#pragma unroll
        for (int o = G / 2; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        if (upd) {
            double* yw = Y + (size_t)j * ld;
            for (int i = part; i < n; i += G) yw[i] = fma(-c, u[i], yw[i]);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------- NNLS
// Normal equations: AtA (r x r), Atb (r x n), btb (n) from R and K.
__global__ void nnls_gram_kernel(const double* __restrict__ R, int n, const int32_t* __restrict__ K, int r,
                                 double* __restrict__ AtA, double* __restrict__ Atb, double* __restrict__ btb)
{
    const int total = r * r + r * n + n;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < total; o += gridDim.x * blockDim.x) {
        int ca, cb;
        double* dst;
        if (o < r * r) {
            ca = K[o / r];
            cb = K[o % r];
            dst = AtA + o;
        } else if (o < r * r + r * n) {
            const int q = o - r * r;
            ca = K[q / n];
            cb = q % n;
            dst = Atb + q;
        } else {
            ca = cb = o - r * r - r * n;
            dst = btb + ca;
        }
        double s = 0.0;
        #pragma unroll 8  // keep eight loads in flight: each is an L2 round trip
        for (int i = 0; i < n; ++i) s += R[(size_t)i * n + ca] * R[(size_t)i * n + cb];
        *dst = s;
    }
}

// Per-column Lawson-Hanson scratch, element e of array x at x[e * S] (S = the
// interleave stride: 32 columns share a bank-conflict-free shared block, or
// S = 1 for the global-memory fallback).
struct LhScratch {
    double* L;   // r*r Cholesky factor of the passive block
    double* y;   // r
    double* z;   // r
    double* zp;  // r
    double* w;   // r  (dual, then right-hand side)
    double* x;   // r  (iterate)
    int* passive;  // r
    int* idx;      // r
    int S;
};

// Solve AtA[idx,idx] z = rhs[idx] by Cholesky.  Returns false if the passive
// block is not positive definite.  The diagonal of L is stored inverted
// (L[i][i] holds 1/l_ii): one binary64 reciprocal per pivot instead of a
// division per entry -- binary64 division is a long sequence on GB300.
__device__ bool chol_solve(const double* AtA, int r, const double* rhs, int S, const int* idx, int p, double* L,
                           double* y, double* z)
{
    for (int i = 0; i < p; ++i) {
        for (int jj = 0; jj <= i; ++jj) {
            double s = AtA[idx[i * S] * r + idx[jj * S]];
            for (int q = 0; q < jj; ++q) s -= L[(i * p + q) * S] * L[(jj * p + q) * S];
            if (i == jj) {
                if (!(s > 0.0)) return false;
                L[(i * p + i) * S] = 1.0 / sqrt(s);
            } else {
                L[(i * p + jj) * S] = s * L[(jj * p + jj) * S];
            }
        }
    }
    for (int i = 0; i < p; ++i) {
        double s = rhs[idx[i * S] * S];
        for (int q = 0; q < i; ++q) s -= L[(i * p + q) * S] * y[q * S];
        y[i * S] = s * L[(i * p + i) * S];
    }
    for (int i = p - 1; i >= 0; --i) {
        double s = y[i * S];
        for (int q = i + 1; q < p; ++q) s -= L[(q * p + i) * S] * z[q * S];
        z[i * S] = s * L[(i * p + i) * S];
    }
    return true;
}

// Lawson-Hanson on the normal equations for column c (the oracle's steps:
// add the most positive dual, solve on the passive set, step back to the
// feasible boundary while any passive coefficient is not positive).
__device__ void lh_column(const double* AtA, const double* __restrict__ Atb, const double* __restrict__ btb, int r,
                          int n, int c, const LhScratch& sc, double* __restrict__ H, int* status)
{
    const int S = sc.S;
    double* x = sc.x;
    double* w = sc.w;
    double* z = sc.z;
    double* zp = sc.zp;
    int* passive = sc.passive;
    int* idx = sc.idx;
    double maxdiag = 0.0;
    for (int i = 0; i < r; ++i) {
        x[i * S] = 0.0;
        passive[i * S] = 0;
        maxdiag = fmax(maxdiag, AtA[i * r + i]);
    }
    const double bb = btb[c];
    const double tol = 1e-12 * sqrt(maxdiag * (bb > 0.0 ? bb : 0.0));
    int outer = 0;
    int st = 0;
    for (;;) {
        for (int i = 0; i < r; ++i) {
            double s = Atb[(size_t)i * n + c];
            for (int q = 0; q < r; ++q) s -= AtA[i * r + q] * x[q * S];
            w[i * S] = s;
        }
        int t = -1;
        double wmax = tol;
        for (int i = 0; i < r; ++i)
            if (!passive[i * S] && w[i * S] > wmax) {
                wmax = w[i * S];
                t = i;
            }
        if (t < 0) break;
        if (outer >= 3 * r) {
            st = MRNMF_ERR_NOT_CONVERGED;
            break;
        }
        ++outer;
        passive[t * S] = 1;
        for (int i = 0; i < r; ++i) w[i * S] = Atb[(size_t)i * n + c];  // right-hand side
        for (int inner = 0; inner <= r + 1; ++inner) {
            int p = 0;
            for (int i = 0; i < r; ++i)
                if (passive[i * S]) idx[(p++) * S] = i;
            if (!chol_solve(AtA, r, w, S, idx, p, sc.L, sc.y, zp)) {
                st = MRNMF_ERR_RANK_DEFICIENT;
                goto done;
            }
            for (int i = 0; i < r; ++i) z[i * S] = 0.0;
            bool allpos = true;
            for (int q = 0; q < p; ++q) {
                z[idx[q * S] * S] = zp[q * S];
                if (zp[q * S] <= 0.0) allpos = false;
            }
            if (allpos) {
                for (int i = 0; i < r; ++i) x[i * S] = z[i * S];
                break;
            }
            double alpha = 2.0;
            int blocking = -1;
            for (int q = 0; q < p; ++q) {
                const int i = idx[q * S];
                if (z[i * S] <= 0.0) {
                    const double den = x[i * S] - z[i * S];  // >= 0; 0 only if x_i = z_i = 0
                    const double a = den > 0.0 ? x[i * S] / den : 0.0;
                    if (a < alpha) {
                        alpha = a;
                        blocking = i;
                    }
                }
            }
            for (int i = 0; i < r; ++i) x[i * S] += alpha * (z[i * S] - x[i * S]);
            x[blocking * S] = 0.0;
            for (int q = 0; q < p; ++q) {
                const int i = idx[q * S];
                if (x[i * S] <= 0.0) {
                    passive[i * S] = 0;
                    x[i * S] = 0.0;
                }
            }
            if (inner == r + 1) {
                st = MRNMF_ERR_NOT_CONVERGED;
                goto done;
            }
        }
    }
done:
    if (st) set_status(status, st);
    for (int i = 0; i < r; ++i) H[(size_t)i * n + c] = x[i * S];
}

// Shared-memory form: C columns per block (one per thread of a warp, C <= 32),
// AtA staged in shared memory, each thread's scratch interleaved with stride C
// (thread t owns element e at [e * C + t]).  Few columns per block spread the
// solves over many SMs: on GB300 each SM has few binary64 units.
__global__ void __launch_bounds__(32) nnls_lh_smem_kernel(const double* __restrict__ AtA_g,
                                                          const double* __restrict__ Atb,
                                                          const double* __restrict__ btb, int r, int n, int C,
                                                          double* __restrict__ H, int* status)
{
    extern __shared__ __align__(16) double sm[];
    double* AtA = sm;
    double* base = sm + r * r;
    for (int i = threadIdx.x; i < r * r; i += 32) AtA[i] = AtA_g[i];
    __syncwarp();
    const int c = blockIdx.x * C + threadIdx.x;
    if (threadIdx.x >= C || c >= n) return;
    LhScratch sc;
    sc.S = C;
    double* mine = base + threadIdx.x;
    sc.L = mine;
    sc.y = sc.L + r * r * C;
    sc.z = sc.y + r * C;
    sc.zp = sc.z + r * C;
    sc.w = sc.zp + r * C;
    sc.x = sc.w + r * C;
    int* ibase = reinterpret_cast<int*>(base + C * (r * r + 5 * r)) + threadIdx.x;
    sc.passive = ibase;
    sc.idx = ibase + r * C;
    lh_column(AtA, Atb, btb, r, n, c, sc, H, status);
}


// ---------------------------------------------------------------------------
// Lawson-Hanson with one warp per column (r <= RM, RM = 16 or 32; the
// smaller instance halves the unrolled factor code): lane i holds coefficient i
// (x_i, the dual w_i, passive flag) and, during a solve, row i of the
// Cholesky factor of the passive block (Lrow) and its column (Lcol).  The
// steps are the oracle's; every O(p) inner product runs across lanes, so each
// Cholesky or triangular solve has O(p) latency instead of O(p^2).
__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// 1/sqrt(d) for d > 0 in binary64 without a binary64 square root or division
// (both are long sequences on GB300's reduced-rate binary64 pipe): a binary32
// seed, then two Newton steps y <- y + y (1 - d y^2) / 2, each of which about
// doubles the correct bits (2^-22 -> 2^-44 -> rounding level).  Outside the
// binary32 range of the seed the plain expression is used.
__device__ __forceinline__ double rsqrt_d(double d)
{
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    double y = (double)rsqrtf((float)d);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double e = fma(-d * y, y, 1.0);
        y = fma(0.5 * y, e, y);
    }
    return y;
}

// r0 > 0: warm start from H's first r0 rows (a feasible point, x >= 0, of the
// same problem with fewer columns -- greedy XRAY's previous pick).  The
// passive set starts as its support; feasibility is restored on it by the
// Lawson-Hanson inner loop before the usual outer iterations, so the result
// is the same minimiser (unique when R(:,K) has full column rank).  H is read
// and then overwritten, column by column (one warp per column).
// The normal equations are formed here: A'A = R(:,K)'R(:,K) in shared
// memory per block (the same sums, in the same order, as nnls_gram_kernel),
// and per column A'b = R(:,K)'R(:,c) and b'b = |R(:,c)|^2 (b'b only sets
// the dual tolerance).
template <int RM>
__global__ void __launch_bounds__(128) nnls_lh_warp_kernel(const double* __restrict__ R,
                                                           const int32_t* __restrict__ K, int r, int n,
                                                           double* __restrict__ H, int r0, int* status)
{
    __shared__ double AtA[32 * 32];
    __shared__ int Ks[32];
    for (int a = threadIdx.x; a < r; a += blockDim.x) Ks[a] = K[a];
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int ca = Ks[e / r], cb = Ks[e % r];
        double sum = 0.0;
        #pragma unroll 8  // keep eight loads in flight: each is an L2 round trip
        for (int i = 0; i < n; ++i) sum += R[(size_t)i * n + ca] * R[(size_t)i * n + cb];
        AtA[e] = sum;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= n) return;
    const unsigned FULL = 0xffffffffu;
    const bool act = lane < r;
    double rhs = 0.0;
    if (act) {
        const int ca = Ks[lane];
        #pragma unroll 8  // keep eight loads in flight: each is an L2 round trip
        for (int i = 0; i < n; ++i) rhs += R[(size_t)i * n + ca] * R[(size_t)i * n + c];
    }
    double maxdiag = act ? AtA[lane * r + lane] : 0.0;
    for (int o = 16; o; o >>= 1) maxdiag = fmax(maxdiag, __shfl_xor_sync(FULL, maxdiag, o));
    // b'b = |R(:,c)|^2, the rows split over the lanes (binary64 issues
    // slowly on GB300: seven instructions instead of n)
    double bb = 0.0;
    for (int i = lane; i < n; i += 32) bb = fma(R[(size_t)i * n + c], R[(size_t)i * n + c], bb);
    for (int o = 16; o; o >>= 1) bb += __shfl_xor_sync(FULL, bb, o);
    const double tol = 1e-12 * sqrt(maxdiag * (bb > 0.0 ? bb : 0.0));
    double x = 0.0;
    bool passive = false;
    int st = 0;
    // Cholesky factor of A^T A over the passive set, in factor order.  Lane k
    // (k < p) holds the k-th factor index idx, row k of L (Lrow[q] = L(k,q),
    // q < k), column k below the diagonal (Lcol[a] = L(a,k), a > k) and
    // 1/L(k,k); coefficient lane i holds its factor position `my` (or -1).
    // An entering index appends one row (forward substitution, O(p) dependent
    // steps); an index leaving the passive set triggers a full refactor.
    double Lrow[RM], Lcol[RM];
#pragma unroll
    for (int q = 0; q < RM; ++q) {
        Lrow[q] = 0.0;
        Lcol[q] = 0.0;
    }
    double invd = 0.0;
    int idx = 0, my = -1, p = 0;

    auto refactor = [&]() -> bool {
        const unsigned pm = __ballot_sync(FULL, act && passive);
        p = __popc(pm);
        my = act && passive ? __popc(pm & ((1u << lane) - 1u)) : -1;  // passive indices in increasing order
        {
            unsigned m = pm;
            for (int k = 0; k < lane && m; ++k) m &= m - 1;
            idx = m ? __ffs(m) - 1 : 0;
        }
        const bool in = lane < p;
#pragma unroll
        for (int q = 0; q < RM; ++q) {
            Lrow[q] = 0.0;
            Lcol[q] = 0.0;
        }
        invd = 0.0;
        bool ok = true;
        // right-looking Cholesky of AtA[idx, idx]
#pragma unroll
        for (int k = 0; k < RM; ++k) {
            if (k >= p) break;
            const int ik = __shfl_sync(FULL, idx, k);
            double d = 0.0;
            if (lane == k) {
                d = AtA[idx * r + idx];
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < k) d -= Lrow[q] * Lrow[q];
            }
            d = shfl_d(d, k);
            if (!(d > 0.0)) {
                ok = false;
                break;
            }
            const double ik_inv = rsqrt_d(d);
            if (lane == k) invd = ik_inv;
            // L(a,k) for a > k: (A(a,k) - sum_{q<k} L(a,q) L(k,q)) / L(k,k)
            double s = (in && lane > k) ? AtA[idx * r + ik] : 0.0;
#pragma unroll
            for (int q = 0; q < RM; ++q) {
                if (q < k) {
                    const double lkq = shfl_d(Lrow[q], k);
                    s -= Lrow[q] * lkq;
                }
            }
            const double lak = (in && lane > k) ? s * ik_inv : 0.0;
            if (in && lane > k) Lrow[k] = lak;
            // lane k collects its column: L(a,k) for a > k
#pragma unroll
            for (int a = 0; a < RM; ++a) {
                if (a > k && a < p) {
                    const double v = shfl_d(lak, a);
                    if (lane == k) Lcol[a] = v;
                }
            }
        }
        return ok;
    };

    // Append index bi to the factor: row p of L solves L l = AtA(idx, bi)
    // (same formula and summation order as the refactor's row p).
    auto add_index = [&](int bi) -> bool {
        double b = lane < p ? AtA[idx * r + bi] : 0.0;
        double l = 0.0;
#pragma unroll
        for (int q = 0; q < RM; ++q) {
            if (q >= p) break;
            if (lane == q) l = b * invd;
            const double lq = shfl_d(l, q);
            if (lane > q && lane < p) b -= Lrow[q] * lq;
            if (lane == p) Lrow[q] = lq;
        }
        double sq = lane < p ? l * l : 0.0;
        for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(FULL, sq, o);
        const double d = AtA[bi * r + bi] - sq;
        if (!(d > 0.0)) return false;
        const double ik_inv = rsqrt_d(d);
        if (lane == p) {
            invd = ik_inv;
            idx = bi;
#pragma unroll
            for (int q = 0; q < RM; ++q)
                if (q >= p) Lrow[q] = 0.0;
        }
        if (lane < p) {
#pragma unroll
            for (int a = 0; a < RM; ++a)
                if (a == p) Lcol[a] = l;
        }
        if (lane == bi) my = p;
        ++p;
        return true;
    };

    // Lawson-Hanson inner loop: solve on the passive set, step back to the
    // feasible boundary while a coefficient would be nonpositive
    auto inner = [&]() {
        for (int it = 0; it <= r + 1; ++it) {
            const bool in = lane < p;
            // forward solve L y = rhs[idx]
            const double bk = shfl_d(rhs, idx);  // lane k: rhs of its passive index (lanes >= p: junk, unused)
            double acc = 0.0, y = 0.0;
    #pragma unroll
            for (int k = 0; k < RM; ++k) {
                if (k >= p) break;
                double yk = 0.0;
                if (lane == k) {
                    y = (bk - acc) * invd;
                    yk = y;
                }
                yk = shfl_d(yk, k);
                if (in && lane > k) acc += Lrow[k] * yk;
            }
            // backward solve L^T z = y: z_k = (y_k - sum_{a>k} L(a,k) z_a) / L(k,k)
            double z = 0.0;
            double acc2 = 0.0;
    #pragma unroll
            for (int k = RM - 1; k >= 0; --k) {
                if (k >= p) continue;
                double zk = 0.0;
                if (lane == k) {
                    z = (y - acc2) * invd;
                    zk = z;
                }
                zk = shfl_d(zk, k);
                // every lane a < k adds L(k,a) z_k: lane a holds L(k,a) in Lcol[k]
                if (in && lane < k) acc2 += Lcol[k] * zk;
            }
            // scatter z back to coefficient lanes: coefficient i (passive, rank my) <- lane my's z
            double zi = shfl_d(z, my < 0 ? 0 : my);
            if (!(act && passive)) zi = 0.0;
            const bool allpos = __all_sync(FULL, !(act && passive) || zi > 0.0);
            if (allpos) {
                x = zi;
                break;
            }
            // step back to the feasible boundary
            double a = 2.0;
            int blk = 32;
            if (act && passive && zi <= 0.0) {
                const double den = x - zi;
                a = den > 0.0 ? x / den : 0.0;
                blk = lane;
            }
            for (int o = 16; o; o >>= 1) {
                const double oa = __shfl_xor_sync(FULL, a, o);
                const int ob = __shfl_xor_sync(FULL, blk, o);
                if (oa < a || (oa == a && ob < blk)) {
                    a = oa;
                    blk = ob;
                }
            }
            x += a * (zi - x);
            if (lane == blk) x = 0.0;
            if (act && passive && x <= 0.0) {
                passive = false;
                x = 0.0;
            }
            if (it == r + 1) {
                st = MRNMF_ERR_NOT_CONVERGED;
                break;
            }
            // some coefficients left the passive set
            if (!__all_sync(FULL, refactor())) {
                st = MRNMF_ERR_RANK_DEFICIENT;
                break;
            }
        }
    };

    if (r0 > 0) {
        if (act && lane < r0) {
            const double v = H[(size_t)lane * n + c];
            x = v > 0.0 ? v : 0.0;
        }
        passive = act && x > 0.0;
        if (__any_sync(FULL, passive)) {
            if (!__all_sync(FULL, refactor())) st = MRNMF_ERR_RANK_DEFICIENT;
            else inner();
        }
    }
    bool fact_ok = true;  // the factor covers exactly the passive set
    for (int outer = 0; !st; ++outer) {
        // dual w = A^T b - A^T A x
        double w = rhs;
        for (int q = 0; q < r; ++q) {
            const double xq = shfl_d(x, q);
            if (act) w -= AtA[lane * r + q] * xq;
        }
        // entering index: the largest dual above tol among non-passive (lowest index on ties)
        double best = (act && !passive && w > tol) ? w : -1.0;
        int bi = lane;
        for (int o = 16; o; o >>= 1) {
            const double ob = __shfl_xor_sync(FULL, best, o);
            const int oi = __shfl_xor_sync(FULL, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (best <= 0.0) break;  // KKT satisfied (no dual above tol)
        if (outer >= 3 * r) {
            st = MRNMF_ERR_NOT_CONVERGED;
            break;
        }
        if (lane == bi) passive = true;
        if (!__all_sync(FULL, fact_ok ? add_index(bi) : refactor())) {
            st = MRNMF_ERR_RANK_DEFICIENT;
            break;
        }
        fact_ok = true;
        inner();
        if (st) break;
    }
    if (st && lane == 0) set_status(status, st);
    if (act) H[(size_t)lane * n + c] = x;
}

// Global-memory fallback for large r (one thread per column).
__global__ void nnls_lh_kernel(const double* __restrict__ AtA, const double* __restrict__ Atb,
                               const double* __restrict__ btb, int r, int n, double* __restrict__ H,
                               double* __restrict__ scratch, int* __restrict__ iscratch, int* status)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    LhScratch sc;
    sc.S = 1;
    sc.L = scratch + (size_t)c * (r * r + 6 * r);
    sc.y = sc.L + r * r;
    sc.z = sc.y + r;
    sc.zp = sc.z + r;
    sc.w = sc.zp + r;
    sc.x = sc.w + r;
    sc.passive = iscratch + (size_t)c * 2 * r;
    sc.idx = sc.passive + r;
    lh_column(AtA, Atb, btb, r, n, c, sc, H, status);
}

size_t lh_smem_bytes(int r, int C) { return 8ull * r * r + (size_t)C * (8ull * (r * r + 5 * r) + 4ull * 2 * r); }

// ------------------------------------------------------------------- residual
// Per-block partial sums of ||R - R(:,K)H||^2 and ||R||^2.
__global__ void residual_partial_kernel(const double* __restrict__ R, int n, const int32_t* __restrict__ K, int r,
                                        const double* __restrict__ H, double* __restrict__ part)
{
    __shared__ double se[8], sr[8];
    double e2 = 0.0, r2 = 0.0;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < n * n) {
        const int i = o / n, c = o - i * n;
        const double v = R[o];
        double s = v;
        #pragma unroll 8  // keep eight loads in flight: each is an L2 round trip
        for (int a = 0; a < r; ++a) s -= R[(size_t)i * n + K[a]] * H[(size_t)a * n + c];
        e2 = s * s;
        r2 = v * v;
    }
    e2 = warp_sum(e2);
    r2 = warp_sum(r2);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        se[w] = e2;
        sr[w] = r2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += se[q];
            b += sr[q];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void residual_final_kernel(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nb; q += 32) {
        a += part[2 * q];
        b += part[2 * q + 1];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
        out[0] = sqrt(a);
        out[1] = b > 0.0 ? a / b : 0.0;
    }
}

// ----------------------------------------------------------------------- XRAY
// One launch per pick: block j scores candidate j,
//   score_j = ||Res^T R(:,j)|| / ||R(:,j)||  (unchosen j; -inf otherwise),
// and the last block to finish (a ticket counter) picks the argmax, so the
// pick needs no launch of its own.  The counter is zero on entry and left at
// zero.
__global__ void __launch_bounds__(128) xray_score_pick_kernel(const double* __restrict__ R,
                                                              const double* __restrict__ Res, int n,
                                                              int* __restrict__ chosen, double* __restrict__ score,
                                                              int t, int32_t* __restrict__ K,
                                                              double* __restrict__ gap, double* __restrict__ s0,
                                                              int* __restrict__ ticket)
{
    __shared__ double sh[8];
    __shared__ Top2 sht[8];
    __shared__ double rj[MRNMF_NMAX];
    __shared__ int last;
    const int j = blockIdx.x;
    if (!chosen[j]) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) rj[i] = R[(size_t)i * n + j];
        __syncthreads();
        double acc = 0.0, cn = 0.0;
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            // four partial sums: the binary64 chain is the latency of this kernel
            double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
            int i = 0;
            for (; i + 4 <= n; i += 4) {
                v0 = fma(Res[(size_t)i * n + q], rj[i], v0);
                v1 = fma(Res[(size_t)(i + 1) * n + q], rj[i + 1], v1);
                v2 = fma(Res[(size_t)(i + 2) * n + q], rj[i + 2], v2);
                v3 = fma(Res[(size_t)(i + 3) * n + q], rj[i + 3], v3);
            }
            for (; i < n; ++i) v0 = fma(Res[(size_t)i * n + q], rj[i], v0);
            const double v = (v0 + v1) + (v2 + v3);
            acc += v * v;
        }
        if (threadIdx.x < 32) {
            for (int i = threadIdx.x; i < n; i += 32) cn += rj[i] * rj[i];
            cn = warp_sum(cn);
        }
        acc = warp_sum(acc);
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) sh[w] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += sh[q];
            const double nrm = sqrt(cn);
            score[j] = nrm > 0.0 ? sqrt(sum) / nrm : 0.0;
        }
    } else if (threadIdx.x == 0) {
        score[j] = -INFINITY;
    }
    // the last block to finish picks
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == n - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = -INFINITY;
    int idx = INT_MAX;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        if (!chosen[c]) {
            const double sc = __ldcg(score + c);
            if (idx == INT_MAX || sc > v) {
                v = sc;
                idx = c;
            }
        }
    }
    Top2 b = block_top2(v, idx, sht);
    if (threadIdx.x == 0) {
        // with more candidates than threads the strided pre-pass may hide a
        // per-thread runner-up: recompute it (n <= blockDim: the merge is exact)
        if (n > (int)blockDim.x) {
            double second = -INFINITY;
            for (int c = 0; c < n; ++c)
                if (!chosen[c] && c != b.i1) second = fmax(second, __ldcg(score + c));
            b.b2 = second;
        }
        if (t == 0) *s0 = b.b1;
        double g = pick_gap(b);
        if (!(b.b1 > 1e-12 * (*s0))) g = -1.0;
        K[t] = b.i1;
        if (gap) gap[t] = g;
        chosen[b.i1] = 1;
        *ticket = 0;
    }
}

// Res = R - R(:,K) H (t = number of columns in K)
__global__ void xray_res_kernel(const double* __restrict__ R, int n, const int32_t* __restrict__ K, int t,
                                const double* __restrict__ H, double* __restrict__ Res)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * n) return;
    const int i = o / n, c = o - i * n;
    double s = R[o];
    #pragma unroll 8  // keep eight loads in flight: each is an L2 round trip
    for (int a = 0; a < t; ++a) s -= R[(size_t)i * n + K[a]] * H[(size_t)a * n + c];
    Res[o] = s;
}

__global__ void init_xray_kernel(const double* __restrict__ R, int n, double* __restrict__ Res, int* __restrict__ chosen,
                                 int* __restrict__ ticket)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < n * n) Res[o] = R[o];
    if (o < n) chosen[o] = 0;
    if (o == 0) *ticket = 0;
}

// ------------------------------------------------------------------------- GP
// One CTA.  Rows of Z = GX D^-1 are scanned by warps; thread 0 then walks the
// rows in order, appending argmax then argmin and skipping duplicates.
__global__ void __launch_bounds__(256) gp_select_kernel(const double* __restrict__ GX, int k, int n,
                                                        const double* __restrict__ colsum, int r,
                                                        int32_t* __restrict__ K, double* __restrict__ gap,
                                                        int* status)
{
    __shared__ int jmax_s[MRNMF_KMAX], jmin_s[MRNMF_KMAX];
    __shared__ double gmax_s[MRNMF_KMAX], gmin_s[MRNMF_KMAX];
    __shared__ int Ks[MRNMF_NMAX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kPer = MRNMF_NMAX / 32;  // row entries per lane
    for (int l = warp; l < k; l += blockDim.x >> 5) {
        double zmax = -INFINITY, zmin = INFINITY, scale = 0.0;
        int imax = INT_MAX, imin = INT_MAX;
        double zl[kPer];  // the lane's entries of row l of GX D^-1, formed once
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int j = lane + 32 * q;
            zl[q] = j < n ? GX[(size_t)l * n + j] / colsum[j] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int j = lane + 32 * q;
            if (j >= n) break;
            const double z = zl[q];
            if (z > zmax) {
                zmax = z;
                imax = j;
            }
            if (z < zmin) {
                zmin = z;
                imin = j;
            }
            scale = fmax(scale, fabs(z));
        }
        for (int o = 16; o; o >>= 1) {
            const double z2 = __shfl_xor_sync(0xffffffffu, zmax, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, imax, o);
            if (z2 > zmax || (z2 == zmax && i2 < imax)) {
                zmax = z2;
                imax = i2;
            }
            const double w2 = __shfl_xor_sync(0xffffffffu, zmin, o);
            const int k2 = __shfl_xor_sync(0xffffffffu, imin, o);
            if (w2 < zmin || (w2 == zmin && k2 < imin)) {
                zmin = w2;
                imin = k2;
            }
            scale = fmax(scale, __shfl_xor_sync(0xffffffffu, scale, o));
        }
        double s2max = -INFINITY, s2min = INFINITY;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int j = lane + 32 * q;
            if (j >= n) break;
            const double z = zl[q];
            if (j != imax) s2max = fmax(s2max, z);
            if (j != imin) s2min = fmin(s2min, z);
        }
        for (int o = 16; o; o >>= 1) {
            s2max = fmax(s2max, __shfl_xor_sync(0xffffffffu, s2max, o));
            s2min = fmin(s2min, __shfl_xor_sync(0xffffffffu, s2min, o));
        }
        if (lane == 0) {
            jmax_s[l] = imax;
            jmin_s[l] = imin;
            gmax_s[l] = (n > 1 && scale > 0.0) ? (zmax - s2max) / scale : 1.0;
            gmin_s[l] = (n > 1 && scale > 0.0) ? (s2min - zmin) / scale : 1.0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // the list is built in shared memory (every duplicate check reads it)
        int cnt = 0;
        for (int l = 0; l < k && cnt < r; ++l) {
            const int picks[2] = {jmax_s[l], jmin_s[l]};
            const double pg[2] = {gmax_s[l], gmin_s[l]};
            for (int q = 0; q < 2 && cnt < r; ++q) {
                bool dup = false;
                for (int c = 0; c < cnt; ++c)
                    if (Ks[c] == picks[q]) dup = true;
                if (!dup) {
                    if (gap) gap[cnt] = pg[q];
                    Ks[cnt++] = picks[q];
                }
            }
        }
        for (int t = cnt; t < r; ++t) {
            Ks[t] = -1;
            if (gap) gap[t] = -1.0;
        }
        if (cnt < r) set_status(status, MRNMF_ERR_RANK_DEFICIENT);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < r; t += blockDim.x) K[t] = Ks[t];
}

// Workspace layout of the small step.
struct SmallWs {
    double* Y;      // n*n (SPA)        / Res (XRAY)
    double* Hs;     // r*n (XRAY inner H)
    double* AtA;    // r*r
    double* Atb;    // r*n
    double* btb;    // n
    double* score;  // n
    double* part;   // 2*ceil(n*n/256)
    double* s0;     // 1
    double* nnls;   // n*(r*r + 6r)
    int* chosen;    // n
    int* inls;      // n*2r
};

size_t a16(size_t b) { return (b + 15) & ~size_t(15); }

SmallWs carve(void* ws, int n, int r)
{
    SmallWs w;
    char* p = static_cast<char*>(ws);
    auto take = [&](size_t bytes) {
        char* q = p;
        p += a16(bytes);
        return q;
    };
    w.Y = (double*)take(8ull * n * n);
    w.Hs = (double*)take(8ull * r * n);
    w.AtA = (double*)take(8ull * r * r);
    w.Atb = (double*)take(8ull * r * n);
    w.btb = (double*)take(8ull * n);
    w.score = (double*)take(8ull * n);
    w.part = (double*)take(8ull * 2 * ((n * n + 255) / 256));
    w.s0 = (double*)take(16);
    w.nnls = (double*)take(8ull * n * (r * r + 6 * r));
    w.chosen = (int*)take(4ull * n);
    w.inls = (int*)take(4ull * n * 2 * r);
    return w;
}

// r0 > 0 (r <= 32 only): H's first r0 rows hold a warm start (see nnls_lh_warp_kernel).
cudaError_t nnls_core(const double* R, int n, const int32_t* K, int r, double* H, const SmallWs& w, int* status,
                      cudaStream_t s, int r0 = 0)
{
    if (r <= 32) {
        if (r <= 16)
            nnls_lh_warp_kernel<16><<<(n + 3) / 4, 128, 0, s>>>(R, K, r, n, H, r0, status);
        else
            nnls_lh_warp_kernel<32><<<(n + 3) / 4, 128, 0, s>>>(R, K, r, n, H, r0, status);
        count_launch();
        return cudaGetLastError();
    }
    const int total = r * r + r * n + n;
    nnls_gram_kernel<<<(total + 127) / 128, 128, 0, s>>>(R, n, K, r, w.AtA, w.Atb, w.btb);
    count_launch();
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int C = (n + sms - 1) / sms;  // columns per block: one block per SM when n <= #SMs
    if (C > 32) C = 32;
    while (C > 1 && lh_smem_bytes(r, C) > 200 * 1024) --C;
    const size_t smem = lh_smem_bytes(r, C);
    if (smem <= 200 * 1024) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(nnls_lh_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        nnls_lh_smem_kernel<<<(n + C - 1) / C, 32, smem, s>>>(w.AtA, w.Atb, w.btb, r, n, C, H, status);
    } else {
        nnls_lh_kernel<<<(n + 31) / 32, 32, 0, s>>>(w.AtA, w.Atb, w.btb, r, n, H, w.nnls, w.inls, status);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace

size_t small_ws_bytes(int n, int k, int r)
{
    (void)k;
    if (r < 1) r = 1;
    size_t b = 0;
    b += a16(8ull * n * n) + a16(8ull * r * n) + a16(8ull * r * r) + a16(8ull * r * n);
    b += a16(8ull * n) * 2 + a16(8ull * 2 * ((n * n + 255) / 256)) + a16(16);
    b += a16(8ull * n * (r * r + 6 * r)) + a16(4ull * n) + a16(4ull * n * 2 * r);
    return b;
}

cudaError_t select_spa(const double* R, int n, const double* colsum, int r, int32_t* K, double* gap, void* ws,
                       int* status, cudaStream_t s)
{
    (void)status;
    SmallWs w = carve(ws, n, r);
    const int G = n <= 32 ? 8 : n <= 64 ? 4 : n <= 128 ? 2 : 1;
    const int threads = ((G * n + 31) / 32) * 32;
    const size_t ybytes = sizeof(double) * (size_t)n * (n | 1);
    const int in_smem = ybytes <= 160 * 1024;
    const size_t smem = in_smem ? ybytes : 0;
    auto launch = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<1, threads, smem, s>>>(R, n, colsum, r, K, gap, w.Y, in_smem);
        count_launch();
        return cudaGetLastError();
    };
    if (G == 8) return launch(spa_kernel<8>);
    if (G == 4) return launch(spa_kernel<4>);
    if (G == 2) return launch(spa_kernel<2>);
    return launch(spa_kernel<1>);
}

cudaError_t select_xray(const double* R, int n, int r, int32_t* K, double* gap, void* ws, int* status,
                        cudaStream_t s)
{
    if (r > kRMax) return cudaErrorInvalidValue;
    SmallWs w = carve(ws, n, r);
    int* ticket = reinterpret_cast<int*>(w.s0 + 1);  // the second half of the 16-byte s0 slot
    init_xray_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(R, n, w.Y, w.chosen, ticket);
    count_launch();
    for (int t = 0; t < r; ++t) {
        xray_score_pick_kernel<<<n, 128, 0, s>>>(R, w.Y, n, w.chosen, w.score, t, K, gap, w.s0, ticket);
        count_launch();
        if (t + 1 == r) break;  // the residual after the last pick scores nothing
        // warm start from the previous pick's coefficients (same K prefix)
        cudaError_t e = nnls_core(R, n, K, t + 1, w.Hs, w, status, s, t);
        if (e != cudaSuccess) return e;
        xray_res_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(R, n, K, t + 1, w.Hs, w.Y);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t select_gp(const double* GX, int k, int n, const double* colsum, int r, int32_t* K, double* gap,
                      void* ws, int* status, cudaStream_t s)
{
    (void)ws;
    gp_select_kernel<<<1, 256, 0, s>>>(GX, k, n, colsum, r, K, gap, status);
    count_launch();
    return cudaGetLastError();
}

cudaError_t nnls_h(const double* R, int n, const int32_t* K, int r, double* H, void* ws, int* status,
                   cudaStream_t s)
{
    if (r > kRMax) return cudaErrorInvalidValue;
    SmallWs w = carve(ws, n, r);
    return nnls_core(R, n, K, r, H, w, status, s);
}

cudaError_t residual(const double* R, int n, const int32_t* K, int r, const double* H, double* out, void* ws,
                     cudaStream_t s)
{
    SmallWs w = carve(ws, n, r);
    const int nb = (n * n + 255) / 256;
    residual_partial_kernel<<<nb, 256, 0, s>>>(R, n, K, r, H, w.part);
    count_launch();
    residual_final_kernel<<<1, 32, 0, s>>>(w.part, nb, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mrnmf
