/*
 * mrnmf_oracle.c -- plain FP64 CPU oracle for the single-pass reduction of a
 * tall-and-skinny nonnegative X and the n-by-n separable step that follows it
 * (Benson, Lee, Rajwa, Gleich, "Scalable methods for nonnegative matrix
 * factorizations of near-separable tall-and-skinny matrices").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle: it is built and
 * called by tests/, by __graft_entry__.smoke() and by bench.py's cpu_baseline
 * leg, and by nothing else.  It shares no code, header, table or helper with
 * the CUDA path in paper_1402_6964_gb300/csrc, and the CUDA path never calls
 * it.  Every routine is written for a reader who wants to check it against the
 * paper by eye: no blocking, no fusion, no reordering beyond the definitions.
 *
 * Conventions: all matrices are dense row-major doubles.  X is m-by-n with
 * leading dimension ldx.  R is n-by-n (R[i*n+j] = R_ij).  H is r-by-n.
 * GX is k-by-n.  K holds 0-based column indices.
 *
 * Readings of the paper that the code fixes (the paper is silent on them):
 *  - Householder sign: beta = -sign(alpha)*||x||; at the end every row of R
 *    with a negative diagonal is negated so that diag(R) >= 0.
 *  - argmax / argmin ties go to the lowest column index.
 *  - SPA projects the chosen (normalised) column out of all columns.
 *  - Greedy XRAY scores with the residual Res = R - R(:,K)H (Res = R at the
 *    start) and recomputes H by NNLS after every pick.
 *  - GP walks the rows of GX D^-1 in order, appending argmax then argmin and
 *    skipping duplicates; K is the first r distinct indices.
 *  - NNLS is Lawson-Hanson in normal-equation form, with tolerance
 *    1e-12 * sqrt(max diag(A^T A) * b^T b) on the dual and at most 3r outer
 *    iterations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOMEM 3
#define ORC_ERR_NOT_CONVERGED 4
#define ORC_ERR_RANK 7

/* ------------------------------------------------------------------------ */
/* Thin QR, R factor only (Sec. 3.1, thin QR definition; Sec. 2.2, Q^T X).  */
/* Unblocked Householder on a column-major copy of the whole X.              */
/* ------------------------------------------------------------------------ */
int orc_qr_r(const double* X, int64_t m, int64_t ldx, int n, double* R)
{
    if (m < 1 || n < 1 || ldx < n) return ORC_ERR_ARG;
    double* A = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    if (!A) return ORC_ERR_NOMEM;
    for (int64_t i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) A[(size_t)j * m + i] = X[i * ldx + j];

    int64_t steps = m < n ? m : n;
    for (int64_t j = 0; j < steps; ++j) {
        double* x = A + (size_t)j * m;          /* column j, rows j..m-1 */
        double alpha = x[j];
        double tail = 0.0;                       /* sum of squares below the diagonal */
        for (int64_t i = j + 1; i < m; ++i) tail += x[i] * x[i];
        double nrm = sqrt(alpha * alpha + tail);
        if (nrm == 0.0) continue;                /* zero column: nothing to annihilate */
        double beta = (alpha >= 0.0) ? -nrm : nrm;
        /* v = x - beta e_1 (rows j..m-1);  H = I - 2 v v^T / (v^T v) */
        double v0 = alpha - beta;
        double vtv = v0 * v0 + tail;
        for (int c = (int)j + 1; c < n; ++c) {
            double* y = A + (size_t)c * m;
            double s = v0 * y[j];
            for (int64_t i = j + 1; i < m; ++i) s += x[i] * y[i];
            double f = 2.0 * s / vtv;
            y[j] -= f * v0;
            for (int64_t i = j + 1; i < m; ++i) y[i] -= f * x[i];
        }
        x[j] = beta;
        for (int64_t i = j + 1; i < m; ++i) x[i] = 0.0;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            R[i * n + j] = (j >= i && i < m) ? A[(size_t)j * m + i] : 0.0;
    free(A);
    /* make the diagonal nonnegative: R <- S R with S = diag(sign(R_ii)) */
    for (int i = 0; i < n; ++i)
        if (R[i * n + i] < 0.0)
            for (int j = i; j < n; ++j) R[i * n + j] = -R[i * n + j];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Column sums s_j = sum_i X_ij (Sec. 2.1 l1 scaling; Sec. 3.3), Kahan.      */
/* ------------------------------------------------------------------------ */
void orc_colsum(const double* X, int64_t m, int64_t ldx, int n, double* s)
{
    for (int j = 0; j < n; ++j) {
        double sum = 0.0, comp = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            double y = X[i * ldx + j] - comp;
            double t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        s[j] = sum;
    }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random        */
/* numbers: as easy as 1, 2, 3"): ten rounds of the 4x32 S-P network with    */
/* multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key bumps 0x9E3779B9,         */
/* 0xBB67AE85 applied between rounds.                                        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Entry G(i, l) of the m-by-k Gaussian matrix of Sec. 2.3 / Algorithm 1,
 * i = global row, l < k.  g_i ~ N(0, I_k) is drawn from a counter-based
 * generator keyed by the row, so any split of the rows sees the same G
 * (this settles the cross-processor correlation caveat of Sec. 3.2).
 *   key = (seed_lo, seed_hi), counter = (i_lo, i_hi, l / 4, 0x4D524E46)
 *   words w0..w3; pair p = (l % 4) / 2 uses (w_{2p}, w_{2p+1});
 *   u = ((w >> 9) + 0.5) * 2^-23  (an odd multiple of 2^-24: exact in
 *   binary32 as well as binary64, never 0 or 1);
 *   Box-Muller: rho = sqrt(-2 ln u1), z = rho cos(2 pi u2) for even l,
 *   rho sin(2 pi u2) for odd l.
 */
static double orc_u23(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

double orc_gauss_entry(uint64_t seed, int64_t row, int l)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)(uint64_t)row, (uint32_t)((uint64_t)row >> 32), (uint32_t)(l >> 2), 0x4D524E46u};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int p = (l & 3) >> 1;
    double u1 = orc_u23(w[2 * p]), u2 = orc_u23(w[2 * p + 1]);
    double rho = sqrt(-2.0 * log(u1));
    const double two_pi = 6.283185307179586476925286766559;
    return (l & 1) ? rho * sin(two_pi * u2) : rho * cos(two_pi * u2);
}

void orc_gauss_matrix(uint64_t seed, int64_t row0, int64_t rows, int k, double* G /* rows*k */)
{
    for (int64_t i = 0; i < rows; ++i)
        for (int l = 0; l < k; ++l) G[i * k + l] = orc_gauss_entry(seed, row0 + i, l);
}

/* GX = G^T X (k-by-n), summed row by row as Algorithm 1's reduce does (Sec. 3.2). */
void orc_gauss_project(const double* X, int64_t m, int64_t ldx, int n, int k, uint64_t seed,
                       int64_t row0, double* GX)
{
    double* g = (double*)malloc(sizeof(double) * (size_t)k);
    for (int64_t t = 0; t < (int64_t)k * n; ++t) GX[t] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        for (int l = 0; l < k; ++l) g[l] = orc_gauss_entry(seed, row0 + i, l);
        for (int l = 0; l < k; ++l)
            for (int j = 0; j < n; ++j) GX[(int64_t)l * n + j] += g[l] * X[i * ldx + j];
    }
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Lawson-Hanson NNLS on the normal equations (Sec. 2.4).                    */
/*   minimise ||A y - b||_2 over y >= 0, given AtA = A^T A (r-by-r),         */
/*   Atb = A^T b and btb = b^T b.                                            */
/* ------------------------------------------------------------------------ */
static int orc_chol_solve(const double* AtA, const double* Atb, int r, const int* idx, int p, double* z)
{
    /* Solve AtA[idx,idx] z = Atb[idx] by Cholesky; z has length p. */
    double* L = (double*)calloc((size_t)p * p, sizeof(double));
    double* y = (double*)malloc(sizeof(double) * (size_t)p);
    int ok = 1;
    for (int i = 0; i < p && ok; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = AtA[idx[i] * r + idx[j]];
            for (int q = 0; q < j; ++q) s -= L[i * p + q] * L[j * p + q];
            if (i == j) {
                if (!(s > 0.0)) { ok = 0; break; }
                L[i * p + i] = sqrt(s);
            } else {
                L[i * p + j] = s / L[j * p + j];
            }
        }
    }
    if (ok) {
        for (int i = 0; i < p; ++i) {
            double s = Atb[idx[i]];
            for (int q = 0; q < i; ++q) s -= L[i * p + q] * y[q];
            y[i] = s / L[i * p + i];
        }
        for (int i = p - 1; i >= 0; --i) {
            double s = y[i];
            for (int q = i + 1; q < p; ++q) s -= L[q * p + i] * z[q];
            z[i] = s / L[i * p + i];
        }
    }
    free(L);
    free(y);
    return ok ? ORC_OK : ORC_ERR_RANK;
}

int orc_nnls(const double* AtA, const double* Atb, double btb, int r, double* x)
{
    int* passive = (int*)calloc((size_t)r, sizeof(int));
    int* idx = (int*)malloc(sizeof(int) * (size_t)r);
    double* w = (double*)malloc(sizeof(double) * (size_t)r);
    double* z = (double*)malloc(sizeof(double) * (size_t)r);
    double* zp = (double*)malloc(sizeof(double) * (size_t)r);
    double maxdiag = 0.0;
    for (int i = 0; i < r; ++i) { x[i] = 0.0; if (AtA[i * r + i] > maxdiag) maxdiag = AtA[i * r + i]; }
    double tol = 1e-12 * sqrt(maxdiag * (btb > 0.0 ? btb : 0.0));
    int status = ORC_OK;
    int outer = 0;
    for (;;) {
        /* dual w = A^T (b - A x) */
        for (int i = 0; i < r; ++i) {
            double s = Atb[i];
            for (int j = 0; j < r; ++j) s -= AtA[i * r + j] * x[j];
            w[i] = s;
        }
        int t = -1;
        double wmax = tol;
        for (int i = 0; i < r; ++i)
            if (!passive[i] && w[i] > wmax) { wmax = w[i]; t = i; }
        if (t < 0) break;                       /* KKT satisfied */
        if (outer >= 3 * r) { status = ORC_ERR_NOT_CONVERGED; break; }
        ++outer;
        passive[t] = 1;
        for (int inner = 0; inner <= r + 1; ++inner) {
            int p = 0;
            for (int i = 0; i < r; ++i) if (passive[i]) idx[p++] = i;
            if (orc_chol_solve(AtA, Atb, r, idx, p, zp) != ORC_OK) { status = ORC_ERR_RANK; goto done; }
            for (int i = 0; i < r; ++i) z[i] = 0.0;
            int allpos = 1;
            for (int q = 0; q < p; ++q) { z[idx[q]] = zp[q]; if (zp[q] <= 0.0) allpos = 0; }
            if (allpos) { for (int i = 0; i < r; ++i) x[i] = z[i]; break; }
            /* step back to the boundary of the feasible set */
            double alpha = 2.0;
            int blocking = -1;
            for (int q = 0; q < p; ++q) {
                int i = idx[q];
                if (z[i] <= 0.0) {
                    double den = x[i] - z[i];          /* >= 0; 0 only if x_i = z_i = 0 */
                    double a = den > 0.0 ? x[i] / den : 0.0;
                    if (a < alpha) { alpha = a; blocking = i; }
                }
            }
            for (int i = 0; i < r; ++i) x[i] += alpha * (z[i] - x[i]);
            /* the blocking variable lands on the bound exactly; drop it and any
               other passive variable that is not strictly positive */
            x[blocking] = 0.0;
            for (int q = 0; q < p; ++q) {
                int i = idx[q];
                if (x[i] <= 0.0) { passive[i] = 0; x[i] = 0.0; }
            }
            if (inner == r + 1) { status = ORC_ERR_NOT_CONVERGED; goto done; }
        }
    }
done:
    free(passive); free(idx); free(w); free(z); free(zp);
    return status;
}

/* H(:, i) = argmin_{y >= 0} || R(:,K) y - R(:,i) ||_2, i = 0..n-1 (Sec. 2.4).
 * R is rows-by-n (rows = n for the reduced problem, rows = m to solve the
 * same problem on X itself). */
int orc_nnls_h(const double* R, int rows, int n, const int32_t* K, int r, double* H)
{
    double* AtA = (double*)malloc(sizeof(double) * (size_t)r * r);
    double* Atb = (double*)malloc(sizeof(double) * (size_t)r);
    double* x = (double*)malloc(sizeof(double) * (size_t)r);
    int status = ORC_OK;
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            double s = 0.0;
            for (int i = 0; i < rows; ++i) s += R[(int64_t)i * n + K[a]] * R[(int64_t)i * n + K[b]];
            AtA[a * r + b] = s;
        }
    for (int c = 0; c < n; ++c) {
        double btb = 0.0;
        for (int i = 0; i < rows; ++i) btb += R[(int64_t)i * n + c] * R[(int64_t)i * n + c];
        for (int a = 0; a < r; ++a) {
            double s = 0.0;
            for (int i = 0; i < rows; ++i) s += R[(int64_t)i * n + K[a]] * R[(int64_t)i * n + c];
            Atb[a] = s;
        }
        int st = orc_nnls(AtA, Atb, btb, r, x);
        if (st != ORC_OK && status == ORC_OK) status = st;
        for (int a = 0; a < r; ++a) H[(int64_t)a * n + c] = x[a];
    }
    free(AtA); free(Atb); free(x);
    return status;
}

/* ||R - R(:,K) H||_F and the relative error ||R - R(:,K)H||_F^2 / ||R||_F^2
 * (Sec. 2.4 reduced-space residual; Sec. 4 relative error). */
void orc_residual(const double* R, int rows, int n, const int32_t* K, int r, const double* H, double out[2])
{
    double e2 = 0.0, r2 = 0.0;
    for (int i = 0; i < rows; ++i)
        for (int c = 0; c < n; ++c) {
            double v = R[(int64_t)i * n + c];
            double s = v;
            for (int a = 0; a < r; ++a) s -= R[(int64_t)i * n + K[a]] * H[(int64_t)a * n + c];
            e2 += s * s;
            r2 += v * v;
        }
    out[0] = sqrt(e2);
    out[1] = r2 > 0.0 ? e2 / r2 : 0.0;
}

/* Helper for the selection rules: argmax of score over unchosen columns with
 * lowest-index ties; returns the index and writes the relative gap between
 * the best and the second best score. */
static int orc_pick(const double* score, const int* chosen, int n, double* gap)
{
    int best = -1;
    double b1 = -INFINITY, b2 = -INFINITY;
    for (int j = 0; j < n; ++j) {
        if (chosen[j]) continue;
        double s = score[j];
        if (best < 0 || s > b1) { b2 = b1; b1 = s; best = j; }
        else if (s > b2) { b2 = s; }
    }
    if (gap) {
        if (best < 0) *gap = -1.0;
        else if (b2 == -INFINITY) *gap = 1.0;
        else *gap = (b1 > 0.0) ? (b1 - b2) / b1 : 0.0;
    }
    return best;
}

/*
 * SPA on the l1-normalised columns (Sec. 2.1: XD^-1 with D_ii = ||X(:,i)||_1,
 * and the argmax_j ||Res(:,j)||_2^2 rule).  Y0 is rows-by-n (R, or X itself),
 * colsum the column sums of X.  gap[t] = relative gap of step t, or -1 when
 * the best remaining score is below 1e-24 of the first step's best (the
 * residual is zero to rounding, so the pick is not determined by the data).
 */
int orc_spa(const double* Y0, int rows, int n, const double* colsum, int r, int32_t* K, double* gap)
{
    if (r < 1 || r > n) return ORC_ERR_ARG;
    double* Y = (double*)malloc(sizeof(double) * (size_t)rows * n);
    double* f = (double*)malloc(sizeof(double) * (size_t)n);
    double* u = (double*)malloc(sizeof(double) * (size_t)rows);
    double* cj = (double*)malloc(sizeof(double) * (size_t)n);
    int* chosen = (int*)calloc((size_t)n, sizeof(int));
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < n; ++j) Y[(int64_t)i * n + j] = Y0[(int64_t)i * n + j] / colsum[j];
    double f0 = 0.0;
    for (int t = 0; t < r; ++t) {
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < rows; ++i) s += Y[(int64_t)i * n + j] * Y[(int64_t)i * n + j];
            f[j] = s;
        }
        double g;
        int p = orc_pick(f, chosen, n, &g);
        if (t == 0) f0 = f[p];
        if (!(f[p] > 1e-24 * f0)) g = -1.0;
        K[t] = p;
        if (gap) gap[t] = g;
        chosen[p] = 1;
        double nrm = sqrt(f[p]);
        if (!(nrm > 0.0)) continue;
        for (int i = 0; i < rows; ++i) u[i] = Y[(int64_t)i * n + p] / nrm;
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < rows; ++i) s += u[i] * Y[(int64_t)i * n + j];
            cj[j] = s;
        }
        for (int i = 0; i < rows; ++i)
            for (int j = 0; j < n; ++j) Y[(int64_t)i * n + j] -= cj[j] * u[i];
    }
    free(Y); free(f); free(u); free(cj); free(chosen);
    return ORC_OK;
}

/*
 * Greedy XRAY (Sec. 2.1): pick argmax_j ||Res^T R(:,j)||_2 / ||R(:,j)||_2 over
 * unchosen j, where Res = R - R(:,K) H and H = NNLS(R(:,K), R) is refreshed
 * after every pick (Res = R before the first pick).  Y0 is rows-by-n.
 */
int orc_xray(const double* Y0, int rows, int n, int r, int32_t* K, double* gap)
{
    if (r < 1 || r > n) return ORC_ERR_ARG;
    double* Res = (double*)malloc(sizeof(double) * (size_t)rows * n);
    double* H = (double*)malloc(sizeof(double) * (size_t)r * n);
    double* score = (double*)malloc(sizeof(double) * (size_t)n);
    double* cn = (double*)malloc(sizeof(double) * (size_t)n);
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    int* chosen = (int*)calloc((size_t)n, sizeof(int));
    int status = ORC_OK;
    memcpy(Res, Y0, sizeof(double) * (size_t)rows * n);
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < rows; ++i) s += Y0[(int64_t)i * n + j] * Y0[(int64_t)i * n + j];
        cn[j] = sqrt(s);
    }
    double s0 = 0.0;
    for (int t = 0; t < r; ++t) {
        for (int j = 0; j < n; ++j) {
            /* v = Res^T R(:,j) */
            for (int q = 0; q < n; ++q) {
                double s = 0.0;
                for (int i = 0; i < rows; ++i) s += Res[(int64_t)i * n + q] * Y0[(int64_t)i * n + j];
                v[q] = s;
            }
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += v[q] * v[q];
            score[j] = cn[j] > 0.0 ? sqrt(s) / cn[j] : 0.0;
        }
        double g;
        int p = orc_pick(score, chosen, n, &g);
        if (t == 0) s0 = score[p];
        if (!(score[p] > 1e-12 * s0)) g = -1.0;
        K[t] = p;
        if (gap) gap[t] = g;
        chosen[p] = 1;
        int st = orc_nnls_h(Y0, rows, n, K, t + 1, H);
        if (st != ORC_OK && status == ORC_OK) status = st;
        for (int i = 0; i < rows; ++i)
            for (int c = 0; c < n; ++c) {
                double s = Y0[(int64_t)i * n + c];
                for (int a = 0; a <= t; ++a) s -= Y0[(int64_t)i * n + K[a]] * H[(int64_t)a * n + c];
                Res[(int64_t)i * n + c] = s;
            }
    }
    free(Res); free(H); free(score); free(cn); free(v); free(chosen);
    return status;
}

/*
 * Gaussian-projection selection (Sec. 2.3 with the one-pass normalisation of
 * Sec. 3.3: G^T (X D^-1) = (G^T X) D^-1).  For each row l of Z = GX D^-1 in
 * order, append argmax_j Z(l,j) and then argmin_j Z(l,j) unless already
 * present.  cand receives up to 2k distinct indices (returned count in
 * *ncand); K = the first r of them (-1 where fewer than r exist).  gap[2l]
 * and gap[2l+1] are the relative gaps (to max_j |Z(l,j)|) of the max and min;
 * cand_gap[c] is the gap of the pick that added cand[c].
 */
int orc_gp_select(const double* GX, int k, int n, const double* colsum, int r, int32_t* K,
                  int32_t* cand, int* ncand, double* gap, double* cand_gap)
{
    int cnt = 0;
    for (int l = 0; l < k; ++l) {
        int jmax = 0, jmin = 0;
        double zmax = GX[(int64_t)l * n] / colsum[0], zmin = zmax, scale = fabs(zmax);
        for (int j = 1; j < n; ++j) {
            double z = GX[(int64_t)l * n + j] / colsum[j];
            if (z > zmax) { zmax = z; jmax = j; }
            if (z < zmin) { zmin = z; jmin = j; }
            if (fabs(z) > scale) scale = fabs(z);
        }
        double s2max = -INFINITY, s2min = INFINITY;
        for (int j = 0; j < n; ++j) {
            double z = GX[(int64_t)l * n + j] / colsum[j];
            if (j != jmax && z > s2max) s2max = z;
            if (j != jmin && z < s2min) s2min = z;
        }
        if (gap) {
            gap[2 * l] = (n > 1 && scale > 0.0) ? (zmax - s2max) / scale : 1.0;
            gap[2 * l + 1] = (n > 1 && scale > 0.0) ? (s2min - zmin) / scale : 1.0;
        }
        int picks[2] = {jmax, jmin};
        double pgap[2] = {(n > 1 && scale > 0.0) ? (zmax - s2max) / scale : 1.0,
                          (n > 1 && scale > 0.0) ? (s2min - zmin) / scale : 1.0};
        for (int q = 0; q < 2; ++q) {
            int dup = 0;
            for (int c = 0; c < cnt; ++c) if (cand[c] == picks[q]) dup = 1;
            if (!dup) {
                if (cand_gap) cand_gap[cnt] = pgap[q];
                cand[cnt++] = picks[q];
            }
        }
    }
    *ncand = cnt;
    for (int t = 0; t < r; ++t) K[t] = t < cnt ? cand[t] : -1;
    return cnt >= r ? ORC_OK : ORC_ERR_RANK;
}

/* ------------------------------------------------------------------------ */
/* R-SVD (Sec. 2.2 and Sec. 3.1, the R-SVD of a tall matrix): Sigma V' of   */
/* an n-by-n R, from R = U Sigma V'.  One-sided Jacobi (Hestenes): plane    */
/* rotations from the right make the columns of B = R' mutually orthogonal; */
/* then B = V Sigma, so column i of B is sigma_i v_i and its transpose is   */
/* row i of Sigma V'.  Pairs are visited in plain cyclic order (i < j, row  */
/* by row); each rotation uses Rutishauser's stable formulas.  Sweeps       */
/* repeat until one rotates nothing (at most 60).  Output rows are sorted   */
/* by descending sigma; each row is determined up to its sign.              */
/* ------------------------------------------------------------------------ */
int orc_r_svd(const double* R, int n, double* sigma, double* SVt)
{
    if (n < 1) return ORC_ERR_ARG;
    double* B = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n); /* B[k*n + i] = R[i*n + k] */
    int* order = (int*)malloc(sizeof(int) * (size_t)n);
    double* s = (double*)malloc(sizeof(double) * (size_t)n);
    if (!B || !order || !s) {
        free(B);
        free(order);
        free(s);
        return ORC_ERR_NOMEM;
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) B[(size_t)k * n + i] = R[(size_t)i * n + k];
    int converged = 0;
    for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
        int rotated = 0;
        for (int i = 0; i < n - 1; ++i) {
            for (int j = i + 1; j < n; ++j) {
                double a = 0.0, b = 0.0, g = 0.0; /* ||b_i||^2, ||b_j||^2, b_i' b_j */
                for (int k = 0; k < n; ++k) {
                    const double bi = B[(size_t)k * n + i], bj = B[(size_t)k * n + j];
                    a += bi * bi;
                    b += bj * bj;
                    g += bi * bj;
                }
                if (g == 0.0 || fabs(g) <= 1e-15 * sqrt(a * b)) continue;
                rotated = 1;
                const double zeta = (b - a) / (2.0 * g);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                for (int k = 0; k < n; ++k) {
                    const double bi = B[(size_t)k * n + i], bj = B[(size_t)k * n + j];
                    B[(size_t)k * n + i] = c * bi - sn * bj;
                    B[(size_t)k * n + j] = sn * bi + c * bj;
                }
            }
        }
        converged = !rotated;
    }
    for (int i = 0; i < n; ++i) {
        double a = 0.0;
        for (int k = 0; k < n; ++k) a += B[(size_t)k * n + i] * B[(size_t)k * n + i];
        s[i] = sqrt(a);
        order[i] = i;
    }
    /* descending sigma; equal values keep the lower column first */
    for (int i = 1; i < n; ++i) {
        const int o = order[i];
        int p = i;
        while (p > 0 && s[order[p - 1]] < s[o]) {
            order[p] = order[p - 1];
            --p;
        }
        order[p] = o;
    }
    for (int i = 0; i < n; ++i) {
        if (sigma) sigma[i] = s[order[i]];
        for (int k = 0; k < n; ++k) SVt[(size_t)i * n + k] = B[(size_t)k * n + order[i]];
    }
    free(B);
    free(order);
    free(s);
    return converged ? ORC_OK : ORC_ERR_NOT_CONVERGED;
}
