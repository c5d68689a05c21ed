// tsqr_simt.cu -- the single pass over X (Sec. 3.1 TSQR, Sec. 3.3 column
// sums, Sec. 3.2 Gaussian projection) on SIMT cores, and the reduction tree
// over the stacked triangles.
//
// Layout.  One CTA is one row stream (one "map task" of Sec. 3.5).  Thread c
// owns column c of the tile: L consecutive rows of that column sit in its
// registers, so every reflector norm and every reflector-column dot product
// is a thread-local sum -- no cross-lane reduction at all.  The CTA's running
// triangle R (n-by-n, packed upper) lives in shared memory.  For a tile A
// (L-by-n) stacked under R, column j's Householder reflector is
// v = [e_j; y], y = A(:,j)/(alpha - beta), tau = (beta - alpha)/beta with
// alpha = R_jj and beta = -sign(alpha) sqrt(alpha^2 + ||A(:,j)||^2); applying
// it to column c > j is w = R_jc + y'A(:,c), R_jc -= tau w, A(:,c) -= tau w y.
// Thread j forms y and tau alone and publishes them through shared memory:
// one barrier per column.
//
// Tree.  The P triangles are themselves rows: a CTA of the next level takes
// two of them, starts from the first and streams the second through the same
// column loop, skipping the all-zero leading columns of each triangle tile.
// R([X1; X2]) = R([R1; R2]) (Sec. 3.1) makes the result the R of all rows.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "leaf.h"

namespace mrnmf {

namespace {

constexpr int kTileRows = 16;      // L: rows per tile and thread
constexpr int kTriRows = 32;       // tile height in the tree
constexpr int kFlushTiles = 64;    // binary32 partial sums flushed to binary64 every 64 tiles

__host__ __device__ inline int packed_row(int j, int n) { return j * n - (j * (j + 1)) / 2; }

template <typename T>
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T, int L, int KMAX>
__host__ __device__ inline size_t leaf_smem_bytes(int n)
{
    size_t b = align16<T>(sizeof(T) * (size_t)(n * (n + 1) / 2));  // packed R
    b += align16<T>(sizeof(T) * 2 * L);                               // y double buffer
    b += align16<T>(sizeof(T) * 4);                                   // tau double buffer
    b += sizeof(float) * (size_t)L * KMAX;                            // Gaussian tile
    return b;
}

template <typename TX, typename T, int L, int KMAX, bool QR, bool TRI>
__device__ __forceinline__ void leaf_body(const LeafArgs& a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n;
    const int c = threadIdx.x;
    const int nt = blockDim.x;
    const bool own = c < n;

    T* Rs = reinterpret_cast<T*>(smem_raw);
    size_t off = align16<T>(sizeof(T) * (size_t)(n * (n + 1) / 2));
    T* ybuf = reinterpret_cast<T*>(smem_raw + off);
    off += align16<T>(sizeof(T) * 2 * L);
    T* tbuf = reinterpret_cast<T*>(smem_raw + off);
    off += align16<T>(sizeof(T) * 4);
    float* gbuf = reinterpret_cast<float*>(smem_raw + off);

    const TX* X = static_cast<const TX*>(a.X);
    const int cta = blockIdx.x;

    // ---- running triangle: continue from the state, or start at zero ----
    // (the tree reads its input triangles in TX: binary32 leaf triangles can
    // enter a binary64 tree)
    const TX* Rin = static_cast<const TX*>(a.R_in);
    int64_t first_tri = 0, last_tri = 0;  // tree: triangles [first_tri+1, last_tri) are merged
    if (TRI) {
        first_tri = (int64_t)cta * a.rows_per_cta;
        last_tri = min((int64_t)a.P_in, first_tri + a.rows_per_cta);
    }
    const int64_t init_slot = TRI ? first_tri : cta;
    if (QR) {
        // independent loads over the whole triangle, unrolled so they overlap
        const bool have = Rin && (!TRI || init_slot < a.P_in);
        const int nn = n * n;
        if (TRI || is_same_t<TX, T>::value) {
            const TX* src = have ? Rin + (size_t)init_slot * n * n : nullptr;
#pragma unroll 8
            for (int e = threadIdx.x; e < nn; e += nt) {
                const int j = e / n, cc = e - j * n;
                if (cc >= j) Rs[packed_row(j, n) + cc] = have ? (T)src[e] : T(0);
            }
        } else {
            // a leaf continuing its state: the state is kept in T
            const T* src = have ? static_cast<const T*>(a.R_in) + (size_t)init_slot * n * n : nullptr;
#pragma unroll 8
            for (int e = threadIdx.x; e < nn; e += nt) {
                const int j = e / n, cc = e - j * n;
                if (cc >= j) Rs[packed_row(j, n) + cc] = have ? src[e] : T(0);
            }
        }
        __syncthreads();
    }

    // ---- tile schedule ----
    int64_t r0 = 0, r1 = 0, ntiles = 0;
    const int tpt = (n + L - 1) / L;  // tree: tiles per triangle
    if (TRI) {
        ntiles = (last_tri - first_tri - 1 > 0 ? last_tri - first_tri - 1 : 0) * tpt;
    } else {
        r0 = (int64_t)cta * a.rows_per_cta;
        r1 = min(a.rows, r0 + a.rows_per_cta);
        ntiles = r1 > r0 ? (r1 - r0 + L - 1) / L : 0;
    }

    auto load_tile = [&](int64_t t, T (&v)[L], int& j0) {
        if (TRI) {
            const int64_t tri = first_tri + 1 + t / tpt;
            const int i0 = (int)(t % tpt) * L;
            j0 = i0;
            const TX* src = Rin + ((size_t)tri * n + i0) * n + c;
#pragma unroll
            for (int l = 0; l < L; ++l) v[l] = (own && i0 + l < n) ? (T)src[(size_t)l * n] : T(0);
        } else {
            const int64_t row = r0 + t * L;
            j0 = 0;
            const TX* src = X + row * a.ldx + c;
#pragma unroll
            for (int l = 0; l < L; ++l) v[l] = (own && row + l < r1) ? (T)src[(int64_t)l * a.ldx] : T(0);
        }
    };

    T av[L], nv[L];
    int j0 = 0, nj0 = 0;
    if (ntiles > 0) load_tile(0, av, j0);

    float cs_acc = 0.f;   // binary32 partial column sum (binary64 for the FP64 form below)
    T cs_accT = T(0);
    T gacc[KMAX > 0 ? KMAX : 1];
#pragma unroll
    for (int q = 0; q < (KMAX > 0 ? KMAX : 1); ++q) gacc[q] = T(0);
    bool bad = false;
    unsigned it = 0;  // running column-step counter: parity of the shared buffers

    for (int64_t t = 0; t < ntiles; ++t) {
        if (t + 1 < ntiles) load_tile(t + 1, nv, nj0);

        if (!TRI) {
            // input check and column sums (Sec. 3.3: computed in the same pass)
            T ts = T(0);
#pragma unroll
            for (int l = 0; l < L; ++l) {
                bad |= !(av[l] >= T(0));
                ts += av[l];
            }
            if (is_f32<T>::value) cs_acc += (float)ts; else cs_accT += ts;

            if (KMAX > 0) {
                // Gaussian tile (Algorithm 1's map: g_i x_i^T, summed by the combiner)
                const int64_t row0 = r0 + t * L;
                const int kq = (a.k + 3) >> 2;
                for (int idx = c; idx < L * kq; idx += nt) {
                    const int l = idx / kq, q = idx - l * kq;
                    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (row0 + l < r1) g = gauss4(a.seed, a.row_base + row0 + l, (uint32_t)q);
                    *reinterpret_cast<float4*>(gbuf + l * KMAX + 4 * q) = g;
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < KMAX; ++q) {
                    if (q < a.k) {
                        T s = gacc[q];
#pragma unroll
                        for (int l = 0; l < L; ++l) s += (T)gbuf[l * KMAX + q] * av[l];
                        gacc[q] = s;
                    }
                }
            }
            if ((t + 1) % kFlushTiles == 0 || t + 1 == ntiles) {
                if (own && a.cs) a.cs[(size_t)cta * n + c] += is_f32<T>::value ? (double)cs_acc : (double)cs_accT;
                cs_acc = 0.f;
                cs_accT = T(0);
                if (KMAX > 0 && own && a.gx) {
#pragma unroll
                    for (int q = 0; q < KMAX; ++q)
                        if (q < a.k) {
                            a.gx[((size_t)cta * a.k + q) * n + c] += (double)gacc[q];
                            gacc[q] = T(0);
                        }
                }
            }
        }

        if (QR) {
            for (int j = j0; j < n; ++j, ++it) {
                T* yb = ybuf + (it & 1) * L;
                const int pj = packed_row(j, n);
                if (c == j) {
                    T sig = T(0);
#pragma unroll
                    for (int l = 0; l < L; ++l) sig += av[l] * av[l];
                    const T alpha = Rs[pj + j];
                    T beta = alpha, tau = T(0);
                    if (sig > T(0)) {
                        const T nrm = sqrt(alpha * alpha + sig);
                        beta = alpha >= T(0) ? -nrm : nrm;
                        const T scale = T(1) / (alpha - beta);
                        tau = (beta - alpha) / beta;
#pragma unroll
                        for (int l = 0; l < L; ++l) yb[l] = av[l] * scale;
                    }
                    Rs[pj + j] = beta;
                    tbuf[it & 1] = tau;
                }
                __syncthreads();
                const T tau = tbuf[it & 1];
                if (own && c > j && tau != T(0)) {
                    T w = Rs[pj + c];
#pragma unroll
                    for (int l = 0; l < L; ++l) w += yb[l] * av[l];
                    const T tw = tau * w;
                    Rs[pj + c] = Rs[pj + c] - tw;
#pragma unroll
                    for (int l = 0; l < L; ++l) av[l] -= tw * yb[l];
                }
            }
        }
        if (!QR || KMAX > 0) __syncthreads();  // gbuf / buffer reuse across tiles

#pragma unroll
        for (int l = 0; l < L; ++l) av[l] = nv[l];
        j0 = nj0;
    }

    if (!TRI && a.check && bad) set_status(a.status, MRNMF_ERR_BAD_INPUT);

    // ---- write the stream's triangle (dense, zeros below the diagonal) ----
    if (QR) {
        __syncthreads();
        T* Rout = static_cast<T*>(a.R_out) + (size_t)cta * n * n;
        const int nn = n * n;
#pragma unroll 8
        for (int e = threadIdx.x; e < nn; e += nt) {
            const int j = e / n, cc = e - j * n;
            Rout[e] = (cc >= j) ? Rs[packed_row(j, n) + cc] : T(0);
        }
    }
}

// The pass over X: one CTA per row stream.
template <typename TX, typename T, int L, int KMAX, bool QR>
__global__ void __launch_bounds__(256) tsqr_leaf_kernel(const LeafArgs a)
{
    leaf_body<TX, T, L, KMAX, QR, false>(a);
}

// One level of the reduction tree over the stacked triangles (input triangles
// in TX, arithmetic and output in T).
template <typename TX, typename T, int L>
__global__ void __launch_bounds__(256) tsqr_tree_kernel(const LeafArgs a)
{
    leaf_body<TX, T, L, 0, true, true>(a);
}

// R <- sign-normalised binary64 copy of the final triangle (diag >= 0).
template <typename T>
__global__ void finalize_r_kernel(const T* __restrict__ Rf, int n, double* __restrict__ R)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        double v = 0.0;
        if (j >= i) {
            v = (double)Rf[(size_t)i * n + j];
            if (Rf[(size_t)i * n + i] < T(0)) v = -v;
        }
        R[idx] = v;
    }
}

// One warp per output: colsum[c] = sum_p cs[p][c];  GX[l][c] = sum_p gx[p][l][c].
__global__ void reduce_partials_kernel(const double* __restrict__ cs, const double* __restrict__ gx, int P, int n,
                                       int k, double* __restrict__ colsum, double* __restrict__ GX, int* status)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nout = n + k * n;
    if (warp >= nout) return;
    double s = 0.0;
    if (warp < n) {
        for (int p = lane; p < P; p += 32) s += cs[(size_t)p * n + warp];
        s = warp_sum(s);
        if (lane == 0) {
            if (!(s > 0.0)) set_status(status, MRNMF_ERR_BAD_INPUT);
            if (colsum) colsum[warp] = s;
        }
    } else {
        const int o = warp - n;  // = l * n + c
        const int l = o / n, c = o - l * n;
        for (int p = lane; p < P; p += 32) s += gx[((size_t)p * k + l) * n + c];
        s = warp_sum(s);
        if (lane == 0 && GX) GX[o] = s;
    }
}

template <typename TX, typename T, int L, int KMAX, bool QR, bool TRI>
cudaError_t launch_leaf_on(const LeafArgs& a, int grid, cudaStream_t s)
{
    void (*kern)(const LeafArgs);
    if constexpr (TRI) kern = tsqr_tree_kernel<TX, T, L>;
    else kern = tsqr_leaf_kernel<TX, T, L, KMAX, QR>;
    const size_t smem = leaf_smem_bytes<T, L, KMAX>(a.n);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int block = ((a.n + 31) / 32) * 32;
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, block, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <typename TX, typename T>
cudaError_t dispatch_leaf(const LeafArgs& a, int grid, int qr, cudaStream_t s)
{
    const int k = a.gx ? a.k : 0;
    if (qr) {
        if (k == 0) return launch_leaf_on<TX, T, kTileRows, 0, true, false>(a, grid, s);
        if (k <= 16) return launch_leaf_on<TX, T, kTileRows, 16, true, false>(a, grid, s);
        if (k <= 32) return launch_leaf_on<TX, T, kTileRows, 32, true, false>(a, grid, s);
        return launch_leaf_on<TX, T, kTileRows, 64, true, false>(a, grid, s);
    }
    if (k == 0) return launch_leaf_on<TX, T, kTileRows, 0, false, false>(a, grid, s);
    if (k <= 16) return launch_leaf_on<TX, T, kTileRows, 16, false, false>(a, grid, s);
    if (k <= 32) return launch_leaf_on<TX, T, kTileRows, 32, false, false>(a, grid, s);
    return launch_leaf_on<TX, T, kTileRows, 64, false, false>(a, grid, s);
}

int num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

std::atomic<unsigned long long> g_launches{0};

size_t pass_state_bytes(int n, int k, int P, int fp64)
{
    const size_t ts = fp64 ? 8 : 4;
    size_t b = 0;
    b += align16<float>(ts * (size_t)P * n * n);              // R
    b += align16<float>(8 * (size_t)((P + 1) / 2) * n * n);   // Rtmp (binary64 also for the FP64 tree)
    b += align16<float>(8 * (size_t)P * n);                   // cs
    b += align16<float>(8 * (size_t)P * (k > 0 ? k : 1) * n); // gx
    return b;
}

void pass_state_carve(PassState& st, void* base)
{
    const size_t ts = st.fp64 ? 8 : 4;
    char* p = static_cast<char*>(base);
    st.R = p;
    p += align16<float>(ts * (size_t)st.P * st.n * st.n);
    st.Rtmp = p;
    p += align16<float>(8 * (size_t)((st.P + 1) / 2) * st.n * st.n);
    st.cs = reinterpret_cast<double*>(p);
    p += align16<float>(8 * (size_t)st.P * st.n);
    st.gx = reinterpret_cast<double*>(p);
}

static int choose_streams_default(int n, int k, int fp64, int tc, int64_t m);

// The default count, scaled by the tuning table's factor for (n, m): the
// warp leaf keeps a multiple of its streams per CTA.
int choose_streams(int n, int k, int fp64, int tc, int64_t m)
{
    const int P0 = choose_streams_default(n, k, fp64, tc, m);
    const double f = tune_stream_factor(n, m);
    if (f == 1.0) return P0;
    int P = std::max(1, (int)std::lround(P0 * f));
    if (!fp64 && !tc && warp_leaf_supported(n, k)) {
        const int w = warp_leaf_warps_per_cta();
        P = std::max(w, (P + w - 1) / w * w);
    }
    return P;
}

static int choose_streams_default(int n, int k, int fp64, int tc, int64_t m)
{
    if (tc && !fp64) {
        // one stream per CTA, as many CTAs as the SM holds at once
        int P = num_sms() * tc_leaf_ctas_per_sm(n);
        if (m > 0) {
            const int64_t minrows = 2 * (int64_t)tc_leaf_rows_per_tile();
            const int64_t cap = std::max<int64_t>(1, (m + minrows - 1) / minrows);
            P = (int)std::min<int64_t>(P, cap);
        }
        return std::max(P, 1);
    }
    if (!fp64 && warp_leaf_supported(n, k)) {
        // one stream per warp; as many warps as the SM holds at once
        const int w = warp_leaf_warps_per_cta();
        int P = num_sms() * warp_leaf_ctas_per_sm(n, k) * w;
        if (m > 0) {
            const int64_t minrows = 2 * (int64_t)warp_leaf_rows_per_tile(n, k);
            const int64_t cap = std::max<int64_t>(1, (m + minrows - 1) / minrows);
            P = (int)std::min<int64_t>(P, cap);
        }
        return std::max(w, (P + w - 1) / w * w);
    }
    if (!fp64 && pipe_leaf_supported(n, k)) {
        int P = num_sms() * pipe_leaf_ctas_per_sm(n, k);
        if (m > 0) {
            const int64_t minrows = 4 * (int64_t)pipe_leaf_rows_per_tile();
            const int64_t cap = std::max<int64_t>(1, (m + minrows - 1) / minrows);
            P = (int)std::min<int64_t>(P, cap);
        }
        return std::max(P, 1);
    }
    if (!fp64 && cta_leaf_supported(n, k)) {
        int P = num_sms() * std::min(8, cta_leaf_ctas_per_sm(n, k));
        if (m > 0) {
            const int64_t minrows = 4 * (int64_t)cta_leaf_rows_per_tile(k, n);
            const int64_t cap = std::max<int64_t>(1, (m + minrows - 1) / minrows);
            P = (int)std::min<int64_t>(P, cap);
        }
        return std::max(P, 1);
    }
    // CTA-per-stream kernel: enough resident CTAs to keep the SIMT pipes
    // issuing while each stream waits at its per-column barrier, but no more:
    // every extra stream adds a triangle to the tree.
    const int warps = (n + 31) / 32;
    int per_sm = fp64 ? 4 : std::max(2, std::min(8, 16 / warps));
    int P = num_sms() * per_sm;
    if (m > 0) {
        const int64_t minrows = 8 * kTileRows;
        const int64_t cap = std::max<int64_t>(1, (m + minrows - 1) / minrows);
        P = (int)std::min<int64_t>(P, cap);
    }
    return std::max(P, 1);
}

// The projection-only pass runs on the SIMT cores by default: G's generation
// (Philox + Box-Muller), not the k-by-n product, dominates it, and the tcgen05
// forms measured slower on GB300.  MRNMF_GP_TC=1 selects the tcgen05 (3-pass
// TF32) form; mrnmf_gauss_project_tc names a tcgen05 form explicitly.
int gp_pass_form(int gp_form)
{
    static const bool gp_tc = [] {
        const char* v = getenv("MRNMF_GP_TC");
        return v && v[0] == '1';
    }();
    return gp_form ? gp_form : (gp_tc ? MRNMF_PREC_TF32X3 : 0);
}

cudaError_t pass_reset(const PassState& st, cudaStream_t s)
{
    const size_t ts = st.fp64 ? 8 : 4;
    cudaError_t e = cudaMemsetAsync(st.R, 0, ts * (size_t)st.P * st.n * st.n, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(st.cs, 0, 8 * (size_t)st.P * st.n, s);
    if (e != cudaSuccess) return e;
    if (st.k > 0) e = cudaMemsetAsync(st.gx, 0, 8 * (size_t)st.P * st.k * st.n, s);
    return e;
}

cudaError_t pass_push(PassState& st, const void* X, int64_t rows, int64_t ldx, int xf64, int qr, int* status,
                      cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    LeafArgs a{};
    a.X = X;
    a.rows = rows;
    a.ldx = ldx;
    a.n = st.n;
    int64_t per = (rows + st.P - 1) / st.P;
    per = ((per + kTileRows - 1) / kTileRows) * kTileRows;
    a.rows_per_cta = per;
    a.row_base = st.rows_seen;
    a.R_in = st.R;
    a.R_out = st.R;
    a.cs = st.cs;
    a.gx = st.k > 0 ? st.gx : nullptr;
    a.k = st.k;
    a.seed = st.seed;
    a.check = 1;
    a.status = status;
    const int grid = st.P;  // every stream runs (possibly on zero rows) so its state slot is rewritten
    cudaError_t e;
    if (st.ev_leaf_start && (e = cudaEventRecord(st.ev_leaf_start, s)) != cudaSuccess) return e;
    const bool warp_path = !st.fp64 && !xf64 && qr && warp_leaf_supported(st.n, st.k) &&
                           st.P % warp_leaf_warps_per_cta() == 0;
    st.tri = st.P;
    const int gp_form = gp_pass_form(st.gp_form);
    if (!qr && !st.fp64 && !xf64 && st.k > 0 && gp_form && gp_tc_supported(st.n, st.k)) {
        // projection-only pass on the tensor cores
        e = launch_gp_tc(static_cast<const float*>(X), rows, ldx, st.n, st.k, st.rows_seen, st.seed, st.P, st.cs,
                         st.gx, status, gp_form == MRNMF_PREC_BF16, s);
    } else if (!qr && !st.fp64 && !xf64 && st.k > 0 && gp_warp_supported(st.n, st.k) &&
               st.P % gp_warp_streams_per_cta() == 0) {
        // projection-only pass, one warp per stream
        const int L = gp_warp_rows_per_tile();
        int64_t pw = (rows + st.P - 1) / st.P;
        a.rows_per_cta = ((pw + L - 1) / L) * L;
        e = launch_gp_warp(a, st.P, s);
    } else if (st.tc && !xf64 && qr) {
        a.tc_split = st.tc == 1;
        const int L = tc_leaf_rows_per_tile();
        int64_t pw = (rows + st.P - 1) / st.P;
        a.rows_per_cta = ((pw + L - 1) / L) * L;
        e = launch_tc_leaf(a, st.P, s);
    } else if (!st.fp64 && !xf64 && qr && pipe_leaf_supported(st.n, st.k)) {
        const int L = pipe_leaf_rows_per_tile();
        int64_t pw = (rows + st.P - 1) / st.P;
        a.rows_per_cta = ((pw + L - 1) / L) * L;
        e = launch_pipe_leaf(a, st.P, s);
    } else if (!st.fp64 && !xf64 && qr && cta_leaf_supported(st.n, st.k)) {
        const int L = cta_leaf_rows_per_tile(a.gx ? st.k : 0, st.n);
        int64_t pw = (rows + st.P - 1) / st.P;
        a.rows_per_cta = ((pw + L - 1) / L) * L;
        e = launch_cta_leaf(a, st.P, s);
    } else if (warp_path) {
        const int L = warp_leaf_rows_per_tile(st.n, a.gx ? st.k : 0);
        int64_t pw = (rows + st.P - 1) / st.P;
        a.rows_per_cta = ((pw + L - 1) / L) * L;
        a.tile_rows = L;
        e = launch_warp_leaf(a, st.P, s);
        st.tri = st.P / warp_leaf_warps_per_cta();
    } else if (st.fp64) {
        e = xf64 ? dispatch_leaf<double, double>(a, grid, qr, s) : dispatch_leaf<float, double>(a, grid, qr, s);
    } else {
        if (xf64) return cudaErrorInvalidValue;
        e = dispatch_leaf<float, float>(a, grid, qr, s);
    }
    if (e == cudaSuccess && st.ev_leaf_stop) e = cudaEventRecord(st.ev_leaf_stop, s);
    st.rows_seen += rows;
    return e;
}

template <typename T>
static cudaError_t tree_and_finalize(PassState& st, double* R, int* status, cudaStream_t s)
{
    const void* cur = st.R;
    void* bufs[2] = {st.Rtmp, st.R};
    int Pc = st.tri > 0 ? st.tri : st.P, which = 0;
    while (Pc > 1) {
        if constexpr (is_f32<T>::value) {
            if (wide_tree_supported(st.n)) {
                int Pn = 0;
                cudaError_t e = tree_wide_level(static_cast<const float*>(cur), Pc, st.n,
                                                static_cast<float*>(bufs[which]), s, &Pn);
                if (e != cudaSuccess) return e;
                cur = bufs[which];
                which ^= 1;
                Pc = Pn;
                continue;
            }
        }
        const int f = 2;
        const int Pn = (Pc + f - 1) / f;
        LeafArgs a{};
        a.n = st.n;
        a.rows_per_cta = f;
        a.R_in = cur;
        a.R_out = bufs[which];
        a.P_in = Pc;
        a.status = status;
        cudaError_t e = launch_leaf_on<T, T, kTriRows, 0, true, true>(a, Pn, s);
        if (e != cudaSuccess) return e;
        cur = bufs[which];
        which ^= 1;
        Pc = Pn;
    }
    if (R) {
        const int nn = st.n * st.n;
        finalize_r_kernel<T><<<(nn + 255) / 256, 256, 0, s>>>(static_cast<const T*>(cur), st.n, R);
        count_launch();
        return cudaGetLastError();
    }
    return cudaSuccess;
}

bool tree64_supported(int n) { return leaf_smem_bytes<double, kTriRows, 0>(n) <= 227 * 1024; }

bool tree64_requested()
{
    static const bool on = [] {
        const char* v = getenv("MRNMF_TREE64");
        return v && v[0] == '1';
    }();
    return on;
}

// The reduction of Sec. 3.1 over the stacked binary32 leaf triangles in
// binary64: the first level reads binary32 and folds in binary64, every later
// level is binary64 throughout (fan-in 2).  Level 1 writes Rtmp; later levels
// alternate with the leaf triangles' own region, which then holds at most
// ceil(P/4) binary64 triangles -- no more bytes than its P binary32 ones.
static cudaError_t tree64_and_finalize(PassState& st, double* R, int* status, cudaStream_t s)
{
    const void* cur = st.R;
    void* bufs[2] = {st.Rtmp, st.R};
    int Pc = st.tri > 0 ? st.tri : st.P, which = 0;
    bool cur64 = false;
    while (Pc > 1) {
        const int Pn = (Pc + 1) / 2;
        LeafArgs a{};
        a.n = st.n;
        a.rows_per_cta = 2;
        a.R_in = cur;
        a.R_out = bufs[which];
        a.P_in = Pc;
        a.status = status;
        cudaError_t e = cur64 ? launch_leaf_on<double, double, kTriRows, 0, true, true>(a, Pn, s)
                              : launch_leaf_on<float, double, kTriRows, 0, true, true>(a, Pn, s);
        if (e != cudaSuccess) return e;
        cur = bufs[which];
        cur64 = true;
        which ^= 1;
        Pc = Pn;
    }
    if (R) {
        const int nn = st.n * st.n;
        if (cur64) finalize_r_kernel<double><<<(nn + 255) / 256, 256, 0, s>>>(static_cast<const double*>(cur), st.n, R);
        else finalize_r_kernel<float><<<(nn + 255) / 256, 256, 0, s>>>(static_cast<const float*>(cur), st.n, R);
        count_launch();
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t pass_finish(PassState& st, int qr, double* R, double* colsum, double* GX, int* status, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (qr) {
        if (st.fp64) e = tree_and_finalize<double>(st, R, status, s);
        else if (st.tree64 && tree64_supported(st.n)) e = tree64_and_finalize(st, R, status, s);
        else e = tree_and_finalize<float>(st, R, status, s);
        if (e != cudaSuccess) return e;
    }
    const int kk = (GX && st.k > 0) ? st.k : 0;
    const int nout = st.n + kk * st.n;
    const int threads = 256;
    const int blocks = (nout * 32 + threads - 1) / threads;
    reduce_partials_kernel<<<blocks, threads, 0, s>>>(st.cs, st.gx, st.P, st.n, kk, colsum, GX, status);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mrnmf
