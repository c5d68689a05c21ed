/*
 * mrnmf.h -- C ABI of the GB300 single-pass reduction for near-separable NMF
 * of tall-and-skinny matrices (Benson, Lee, Rajwa, Gleich, arXiv 1402.6964).
 *
 * The method (Sec. 1.1, Sec. 2): a nonnegative m-by-n X (m >> n) is
 * near-separable, X ~ X(:,K) H with |K| = r.  One pass over X produces the
 * n-by-n triangular factor R of its thin QR (Sec. 3.1), the column sums of X
 * (Sec. 3.3) and, optionally, the Gaussian projection G^T X (Sec. 2.3,
 * Algorithm 1).  Because X = X(:,K)H implies R = R(:,K)H (Sec. 2.2), the
 * extreme columns K, the coefficients H and the residual are then computed
 * from R at n-by-n size (Sec. 2.1, Sec. 2.4).
 *
 * General rules for every entry point:
 *  - Pointers named "device" are CUDA device (or managed) memory owned by the
 *    caller; the library never frees or keeps them past the call's work.
 *  - Matrices are dense row-major: X[i*ldx + j], R[i*n + j] (upper
 *    triangular, diag >= 0, zeros below), H[t*n + j] (r-by-n), GX[l*n + j]
 *    (k-by-n).  K holds 0-based column indices.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it and the call returns without waiting.  Argument errors
 *    are returned at once and enqueue nothing.  Errors found on the device
 *    (negative / NaN / zero-sum input, NNLS not converged, a bounded wait
 *    that timed out) are recorded in a device status word of the handle and
 *    returned by mrnmf_sync_status().
 *  - A handle owns its device workspace and is not thread-safe: use one
 *    handle per host thread, or serialise calls on it.  Calls on one handle
 *    that overlap on the GPU (different streams) race on its workspace.
 *  - No entry point falls back to the CPU.
 *  - Limits: 1 <= n <= MRNMF_NMAX, m >= n, 1 <= r <= n, 1 <= k <= MRNMF_KMAX.
 */
#ifndef MRNMF_H
#define MRNMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRNMF_NMAX 256
#define MRNMF_KMAX 64

typedef enum {
    MRNMF_OK = 0,
    MRNMF_ERR_INVALID_ARG = 1,
    MRNMF_ERR_CUDA = 2,
    MRNMF_ERR_NO_MEMORY = 3,
    MRNMF_ERR_NOT_CONVERGED = 4,
    MRNMF_ERR_TIMEOUT = 5,
    MRNMF_ERR_BAD_INPUT = 6,       /* negative or NaN entry, or a zero column sum */
    MRNMF_ERR_RANK_DEFICIENT = 7   /* R(:,K) singular, or fewer than r GP candidates */
} mrnmf_status;

typedef enum { MRNMF_F32 = 0, MRNMF_F64 = 1 } mrnmf_dtype;

/* Arithmetic of the pass.  FP64: everything in binary64 (X must be F64).
 * FP32: binary32 SIMT Householder.  TF32X3 (F32 input, 16 < n <= 256, k <= 32
 * for n <= 64 and k <= 48 above, else MRNMF_ERR_INVALID_ARG): binary32
 * reflectors in 16-column panels with the compact-WY trailing update and the
 * Gaussian projection on tcgen05 tensor cores in 3-pass split TF32
 * (hi*hi + hi*lo + lo*hi, the main term and the corrections accumulated
 * apart in FP32); R within 1e-5 of the FP64 oracle, slower than FP32 on
 * GB300, so AUTO does not pick it.  AUTO picks FP64 for F64 input, otherwise
 * FP32.  TF32: the same tensor-core leaf with one TF32 product (hi*hi) in
 * place of three; its error is that of 10-bit mantissas, well above the FP32
 * form's (the tests state its bound).  BF16 is a form of the projection alone
 * (mrnmf_gauss_project_tc): G and X rounded to bfloat16, exact products, FP32
 * accumulation; the passes that form R reject it. */
typedef enum {
    MRNMF_PREC_AUTO = 0,
    MRNMF_PREC_FP64 = 1,
    MRNMF_PREC_FP32 = 2,
    MRNMF_PREC_TF32X3 = 3,
    MRNMF_PREC_BF16 = 4,
    MRNMF_PREC_TF32 = 5
} mrnmf_prec;

typedef enum { MRNMF_SPA = 0, MRNMF_XRAY = 1, MRNMF_GP = 2 } mrnmf_method;

typedef struct mrnmf_handle mrnmf_handle;

/* Create / destroy a handle.  mrnmf_create selects no device: the handle
 * works on the device that is current when each call is made. */
mrnmf_status mrnmf_create(mrnmf_handle** handle);
void mrnmf_destroy(mrnmf_handle* handle);

/* Human-readable text of the last error on this handle (never NULL). */
const char* mrnmf_last_error_string(const mrnmf_handle* handle);

/* Wait for `stream`, then return (and clear) the first error any kernel of
 * this handle recorded on the device since the last call. */
mrnmf_status mrnmf_sync_status(mrnmf_handle* handle, void* stream);

/*
 * R factor of the thin QR of X (Sec. 3.1: TSQR; only R is formed, Q stays
 * implicit) and the column sums of X (Sec. 3.3), in one read of X.
 *   X      device, m-by-n row-major, leading dimension ldx >= n, dtype F32/F64
 *   R      device, n*n doubles out: upper triangular, diag >= 0
 *   colsum device, n doubles out (nullable)
 * With a full-column-rank X, R is unique and matches the FP64 oracle to the
 * form's stated error.  X must be nonnegative (the method's NMF setting):
 * a negative or NaN entry sets MRNMF_ERR_BAD_INPUT on the device.
 */
mrnmf_status mrnmf_tsqr_r(mrnmf_handle* handle, const void* X, int64_t m, int32_t n, int64_t ldx,
                          int32_t dtype, int32_t prec, double* R, double* colsum, void* stream);

/*
 * Gaussian projection GX = G^T X (Sec. 2.3; Algorithm 1 with its combiner,
 * Sec. 3.2) and the column sums of X, in one read of X.  G is m-by-k with
 * i.i.d. N(0,1) entries drawn by Philox4x32-10 keyed by `seed` and the global
 * row index (row_offset + i), so G does not depend on how rows are split:
 *   key = (seed_lo, seed_hi), counter = (row_lo, row_hi, l/4, 0x4D524E46),
 *   u = ((w >> 9) + 0.5) 2^-23, Box-Muller pairs (w0,w1) -> l%4 = 0,1 and
 *   (w2,w3) -> l%4 = 2,3, cosine for even l and sine for odd l.
 *   GX     device, k*n doubles out
 *   colsum device, n doubles out (nullable)
 */
mrnmf_status mrnmf_gauss_project(mrnmf_handle* handle, const void* X, int64_t m, int32_t n, int64_t ldx,
                                 int32_t dtype, int32_t k, uint64_t seed, int64_t row_offset,
                                 double* GX, double* colsum, void* stream);

/*
 * The same projection with G^T X on the tcgen05 tensor cores in a named form
 * (Sec. 2.3 and Algorithm 1; the arithmetic form is this library's choice):
 *   form = MRNMF_PREC_TF32X3: split TF32, hi*hi + hi*lo + lo*hi, FP32
 *          accumulation (about binary32 accuracy);
 *   form = MRNMF_PREC_BF16:   every entry of G and of X rounded to bfloat16
 *          (round to nearest even) before the product; each product is then
 *          exact in FP32 and the sums are FP32 accumulations, so GX equals
 *          G_bf16^T X_bf16 up to FP32 summation error (binary64 across CTAs).
 * G is the Gaussian matrix of mrnmf_gauss_project (same seed and row keys).
 * The column sums are of X as read (binary32 tile sums, binary64 across).
 *   X      device, F32, m-by-n row-major, ldx >= n; n <= 128 and 1 <= k <= 64
 *   GX     device, k*n doubles out;  colsum device, n doubles out (nullable)
 * MRNMF_ERR_INVALID_ARG for another form, n > 128, k outside [1, 64], or the
 * argument errors of mrnmf_gauss_project.  A negative or NaN entry of X sets
 * MRNMF_ERR_BAD_INPUT on the device.
 */
mrnmf_status mrnmf_gauss_project_tc(mrnmf_handle* handle, const float* X, int64_t m, int32_t n, int64_t ldx,
                                    int32_t k, uint64_t seed, int64_t row_offset, int32_t form, double* GX,
                                    double* colsum, void* stream);

/*
 * The one-pass form of Sec. 3.5: R, the column sums and (if k > 0) GX from a
 * single read of X.  Arguments as in mrnmf_tsqr_r and mrnmf_gauss_project;
 * GX may be NULL when k == 0.
 */
mrnmf_status mrnmf_tsqr_gp(mrnmf_handle* handle, const void* X, int64_t m, int32_t n, int64_t ldx,
                           int32_t dtype, int32_t prec, double* R, double* colsum,
                           int32_t k, uint64_t seed, double* GX, void* stream);

/*
 * Extreme-column selection at n-by-n size (Sec. 2.1, Sec. 2.3).
 *   MRNMF_SPA : SPA on R D^-1 (D = diag(colsum)): repeatedly pick the column
 *               of largest 2-norm and project it out of all columns.
 *   MRNMF_XRAY: greedy XRAY on R: pick argmax_j ||Res^T R(:,j)|| / ||R(:,j)||,
 *               Res = R - R(:,K) H with H refreshed by NNLS after each pick.
 *   MRNMF_GP  : for each row l of GX D^-1 in order, append argmax then argmin,
 *               skipping duplicates; K = first r distinct.
 * Ties go to the lowest index.
 *   R      device n*n doubles (SPA, XRAY)      colsum device n doubles (SPA, GP)
 *   GX     device k*n doubles (GP only; NULL otherwise)
 *   K      device r int32 out                   gap device r doubles out (nullable):
 *          relative gap between the best and second-best score of each pick
 *          (GP: of the row's max), -1 where the best score is zero to rounding.
 */
mrnmf_status mrnmf_select_extreme(mrnmf_handle* handle, int32_t method, const double* R, int32_t n,
                                  const double* colsum, const double* GX, int32_t k, int32_t r,
                                  int32_t* K, double* gap, void* stream);

/*
 * H(:,i) = argmin_{y >= 0} || R(:,K) y - R(:,i) ||_2 for i = 0..n-1 (Sec. 2.4),
 * by Lawson-Hanson active sets on the FP64 normal equations.
 *   R device n*n, K device r int32, H device r*n doubles out.
 * MRNMF_ERR_NOT_CONVERGED / MRNMF_ERR_RANK_DEFICIENT surface at sync.
 */
mrnmf_status mrnmf_nnls_h(mrnmf_handle* handle, const double* R, int32_t n, const int32_t* K, int32_t r,
                          double* H, void* stream);

/*
 * out[0] = ||R - R(:,K) H||_F (= ||X - X(:,K)H||_F, Sec. 2.4),
 * out[1] = ||R - R(:,K) H||_F^2 / ||R||_F^2 (the relative error of Sec. 4).
 *   out device, 2 doubles.
 */
mrnmf_status mrnmf_residual(mrnmf_handle* handle, const double* R, int32_t n, const int32_t* K, int32_t r,
                            const double* H, double* out, void* stream);

/*
 * Rank sweep (Sec. 2.2 and Sec. 2.4: with R in hand, the residual of many
 * candidate separation ranks costs only n-by-n work; Sec. 5 picks r at an
 * elbow of this curve).  Selects r_max columns once with `method` (SPA,
 * greedy XRAY and GP all pick in a nested order, so the first r picks are the
 * rank-r selection), then for r = 1..r_max solves H_r by NNLS on K[0..r) and
 * writes curve[2(r-1)] = ||R - R(:,K_r) H_r||_F and
 * curve[2(r-1)+1] = ||R - R(:,K_r) H_r||_F^2 / ||R||_F^2.
 *   K     device r_max int32 out        curve device 2*r_max doubles out
 * Other arguments as in mrnmf_select_extreme; 1 <= r_max <= min(n, 64).
 */
mrnmf_status mrnmf_rank_sweep(mrnmf_handle* handle, int32_t method, const double* R, int32_t n,
                              const double* colsum, const double* GX, int32_t k, int32_t r_max, int32_t* K,
                              double* curve, void* stream);

/*
 * Follow-ups that read X a second time (optional: the method itself needs
 * only the one pass).
 *
 * mrnmf_gather_columns: W = X(:,K), the left factor of X ~ X(:,K) H (Sec. 2).
 *   X  device m-by-n row-major (ldx >= n), F32 or F64
 *   K  device r int32, each in [0, n)      W device m-by-r row-major (ldw >= r), same dtype as X
 * A K entry outside [0, n) sets MRNMF_ERR_INVALID_ARG on the device (column 0
 * is read in its place).  Bit-exact copy.
 *
 * mrnmf_full_residual: out[0] = ||X - X(:,K) H||_F and
 * out[1] = ||X - X(:,K) H||_F^2 / ||X||_F^2, formed row by row from X itself
 * (in X's precision, squares summed in binary64).  In exact arithmetic it
 * equals mrnmf_residual on R (Sec. 2.4), so it checks the reduced
 * computation.  H device r-by-n doubles (as from mrnmf_nnls_h), out device 2
 * doubles; 1 <= r <= n <= 256.
 */
/*
 * R-SVD form (Sec. 2.2: R = U Sigma V', so X = (QU) Sigma V'; the separable
 * step picks the same K on Sigma V' as on R, since K is invariant under a
 * left orthogonal factor).  One-sided Jacobi on R' in binary64.
 *   R      device n*n doubles, row-major (any square matrix; mrnmf_tsqr_r's R)
 *   sigma  device n doubles out, descending (nullable)
 *   SVt    device n*n doubles out, row-major: row i = sigma_i v_i' (each row
 *          determined up to sign)
 * MRNMF_ERR_NOT_CONVERGED surfaces at sync if 40 sweeps do not converge.
 */
mrnmf_status mrnmf_r_svd(mrnmf_handle* handle, const double* R, int32_t n, double* sigma, double* SVt,
                         void* stream);

mrnmf_status mrnmf_gather_columns(mrnmf_handle* handle, const void* X, int64_t m, int32_t n, int64_t ldx,
                                  int32_t dtype, const int32_t* K, int32_t r, void* W, int64_t ldw, void* stream);
mrnmf_status mrnmf_full_residual(mrnmf_handle* handle, const void* X, int64_t m, int32_t n, int64_t ldx,
                                 int32_t dtype, const int32_t* K, int32_t r, const double* H, double* out,
                                 void* stream);

/*
 * Streaming form of the pass (Sec. 3.4: one pass over data that arrives in
 * pieces).  begin() resets the handle's running state for n columns;
 * push() folds `rows` more rows into it (X_chunk device, row-major, ldx);
 * end() reduces the state to R / colsum / GX exactly as mrnmf_tsqr_gp would
 * for the concatenated rows.  Gaussian rows are keyed by the global row
 * index, so the result does not depend on how the rows were split.
 * Only one stream may be open per handle.
 */
mrnmf_status mrnmf_stream_begin(mrnmf_handle* handle, int32_t n, int32_t dtype, int32_t prec,
                                int32_t k, uint64_t seed, void* stream);
mrnmf_status mrnmf_stream_push(mrnmf_handle* handle, const void* X_chunk, int64_t rows, int64_t ldx,
                               void* stream);
mrnmf_status mrnmf_stream_end(mrnmf_handle* handle, double* R, double* colsum, double* GX, void* stream);

/*
 * Checkpoint of an open stream, between pushes (the analogue of re-running a
 * failed map task, Sec. 3.5; the paper has no device counterpart).  The state
 * is the running triangles, partial column sums and projections and the next
 * global row index: O(P n^2) bytes, independent of the rows pushed.
 *   state_size: bytes of the serialised state of the open stream.
 *   state_save: copies it into `host` (>= state_size bytes, caller-owned) and
 *               waits for `stream`.
 *   state_load: restores it into an open stream begun with the same n, dtype,
 *               prec, k and seed on the same device (else MRNMF_ERR_INVALID_ARG),
 *               and waits for `stream`.  Pushing the remaining chunks then
 *               gives bit for bit the result of the uninterrupted stream.
 */
mrnmf_status mrnmf_stream_state_size(mrnmf_handle* handle, size_t* bytes);
mrnmf_status mrnmf_stream_state_save(mrnmf_handle* handle, void* host, size_t bytes, void* stream);
mrnmf_status mrnmf_stream_state_load(mrnmf_handle* handle, const void* host, size_t bytes, void* stream);

/*
 * Batched pass: R (and colsum) of many independent problems of uneven m and n
 * (Sec. 3.1's TSQR applied to each), FP32 form, enqueued on `stream` as a
 * handful of launches for the whole batch: the row streams of all problems
 * with n <= 128 share one leaf launch per family (n <= 32, 33..64 and
 * 65..128), their trees one launch per level, and one launch writes every R
 * and colsum; problems with n > 128 run the one-problem pass in turn.  Each
 * problem's share of the streams is
 * planned on the host from its m and n (cost-balanced), tile height and tree
 * fan-in follow n.
 *   problems  host array of `count` descriptors (device X, R, colsum):
 *             X float32 m-by-n row-major (ldx >= n), 1 <= n <= MRNMF_NMAX,
 *             m >= n; R n*n doubles out; colsum n doubles out (nullable).
 * Once a call has sized the handle's buffers, a repeat of the same batch
 * issues no allocation or host synchronisation and can be captured in a CUDA
 * graph; a captured graph keeps reading the handle's descriptor staging area,
 * so make no batched call with a different batch on that handle while the
 * graph is replayed.
 */
typedef struct {
    const float* X;
    int64_t m;
    int64_t ldx;
    int32_t n;
    double* R;
    double* colsum;
} mrnmf_problem;

mrnmf_status mrnmf_tsqr_r_batched(mrnmf_handle* handle, const mrnmf_problem* problems, int32_t count, void* stream);

/*
 * End-to-end factorisation from HOST memory: streams X (host, row-major
 * float32, m-by-n, ldx) to the device in chunks with the copies overlapped
 * with the pass, then selects K by `method`, solves H and the residual, and
 * copies K (r int32), H (r*n doubles), resid (2 doubles) and, if non-NULL,
 * R (n*n doubles) back to host memory.  Synchronous: returns when the host
 * outputs are written (device-side errors are returned directly).
 * Pinned (page-locked) X gives the full copy bandwidth.
 */
mrnmf_status mrnmf_factorize_host(mrnmf_handle* handle, const float* X, int64_t m, int32_t n, int64_t ldx,
                                  int32_t prec, int32_t method, int32_t r, int32_t k, uint64_t seed,
                                  int32_t* K, double* H, double* resid, double* R, void* stream);

/*
 * The R / column-sum pass of mrnmf_tsqr_r (F32 input, FP32 form) for callers
 * that cannot allocate device memory -- e.g. code running inside a host
 * callback or an allocator hook, or under a memory pool the application owns
 * outright.  The paper has no counterpart: this is a deployment variant.
 * It needs no handle and allocates nothing (no cudaMalloc / cudaFree, no
 * allocating library call): its scratch is a fixed 32 MiB __device__ array
 * inside this library, held on every GPU that loads it until the process
 * exits.  Limits: 1 <= n <= MRNMF_NMAX, m >= n, ldx >= n; m is unbounded
 * (the pass uses fewer row streams when n is large so the scratch fits).
 *   X      device, m-by-n row-major float32      R device n*n doubles out
 *   colsum device n doubles out (nullable)
 *   status device int32 out (required): 0, or the first device-side error
 *          (MRNMF_ERR_BAD_INPUT), valid once the stream reaches it.  A NULL
 *          status is rejected with MRNMF_ERR_INVALID_ARG, because this entry
 *          has no handle to keep the error in.
 * Returns after enqueuing on `stream`; argument errors return at once.
 * All calls share the one array per device: calls that overlap on the GPU
 * race and give wrong results, so serialise them.  The array keeps the last
 * call's contents; every call clears what must start at zero.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress),
 * so make that first call before any stream capture.  That address is kept
 * for the life of the process: after cudaDeviceReset on a device, do not call
 * this entry point again in the same process.
 */
mrnmf_status mrnmf_tsqr_r_noalloc(const float* X, int64_t m, int32_t n, int64_t ldx, double* R, double* colsum,
                                  int32_t* status, void* stream);

/*
 * Instrumentation (no counterpart in the paper; used by benchmarks).
 * mrnmf_profile_events: when both are non-NULL, every later pass on this
 * handle records `ev_start` / `ev_stop` (cudaEvent_t created by the caller)
 * on its stream immediately before and after the leaf kernel -- the kernel
 * that reads X -- so its duration can be read with cudaEventElapsedTime.
 * Pass NULLs to stop.  mrnmf_kernel_launches: number of CUDA kernels this
 * library has launched in the calling process so far.
 */
mrnmf_status mrnmf_profile_events(mrnmf_handle* handle, void* ev_start, void* ev_stop);

/*
 * Diagnostics (no counterpart in the paper): one tcgen05 tensor-core GEMM
 * D = A B^T on a single CTA, the datapath of the tensor-core forms.
 *   A device 128-by-K float32 row-major, B device N-by-K float32 row-major,
 *   D device 128-by-N float32 row-major out; 16 <= N <= 256, N % 16 == 0,
 *   K in {32, 64}.
 *   kind 0: TF32 inputs; 1: 3-pass split TF32 (hi*hi + hi*lo + lo*hi);
 *   2: BF16 inputs.  FP32 accumulation in tensor memory.
 *   status device int32 out (nullable): MRNMF_ERR_TIMEOUT if the MMA never
 *   signalled completion within 1 s.
 */
mrnmf_status mrnmf_tc_selftest(const float* A, const float* B, float* D, int32_t N, int32_t K, int32_t kind,
                               int32_t* status, void* stream);
/*
 * Diagnostics (no counterpart in the paper): the scalars of one Householder
 * step of the leaves, beta = -sign(alpha) sqrt(alpha^2 + sigma), d = alpha -
 * beta, 1/beta, 1/d (Sec. 3.1), as the leaves compute them, next to the IEEE
 * square root and reciprocals.
 *   alpha, sigma device float[count] in (sigma > 0);
 *   out device float[8 count] out: per argument pair the leaves' beta, d,
 *   1/beta, 1/d, then the IEEE beta, d, 1/beta, 1/d.
 */
mrnmf_status mrnmf_hh_scalars_selftest(const float* alpha, const float* sigma, int64_t count, float* out,
                                       void* stream);

/*
 * Failure injection (no counterpart in the paper): the bounded mbarrier wait
 * of the warp-pipelined leaf, driven by a four-warp chain in one CTA in which
 * warp v waits for warp v - 1, for at most v * limit_ns (limit_ns in
 * [1e3, 1e9]).  The arrival on link `missing` (1..3; 0 = none) is left out,
 * so that wait runs out and the waits after it are abandoned through the
 * leaf's abort flag.  No fault, trap or hang is involved.
 *   out    device int32[4] out: per warp 0 completed, 1 ran out, 2 abandoned.
 *   status device int32 out: MRNMF_ERR_TIMEOUT when a wait ran out, else 0.
 */
mrnmf_status mrnmf_wait_selftest(int32_t missing, int64_t limit_ns, int32_t* out, int32_t* status, void* stream);
uint64_t mrnmf_kernel_launches(void);

/*
 * Tuning table (no counterpart in the paper; the paper's MapReduce runs leave
 * the number of map tasks to Hadoop).  Process-wide, not per handle.  Plain
 * text, one setting per line ('#' starts a comment):
 *     pass  <n_lo> <n_hi> <log2m_lo> <log2m_hi> <stream_factor>
 *     rows  <n_lo> <n_hi> <k_lo> <k_hi> <tile_rows>
 *     batch <family 1..3> <waves>
 * A pass of n columns over m rows scales its default number of row streams
 * (map tasks, Sec. 3.5) by the stream_factor of the first matching pass line
 * (n_lo <= n <= n_hi, log2m_lo <= log2(m) < log2m_hi; factor in (0, 64]).
 * A binary32 pass on the warp leaf (n <= 64; for n <= 16 only with k > 0,
 * since the lane-group leaf with its fixed super-tiles serves k = 0) with k
 * projection rows (0 without GX) stages tiles of the tile_rows of the first
 * matching rows line
 * (n_lo <= n <= n_hi, k_lo <= k <= k_hi; 32, 64 or 128), where the leaf's
 * form for n has that height (n <= 32: 64 or 128; 33..64: 32 or 64) and its
 * CTA fits in shared memory; otherwise the built-in height.  The variables
 * MRNMF_WARP_ROWS1 (n <= 32) and MRNMF_WARP_ROWS (33..64) override it.  A
 * batched call plans family f's streams (1: n <= 32, 2: 33..64, 3: 65..128)
 * for `waves` waves of resident CTAs (in [0.25, 256]).  Settings change only
 * the amount and shape of the parallel work: R is the same up to rounding
 * order.
 * The table is read from the file named by MRNMF_TUNE_FILE when first needed
 * (a malformed file is reported on stderr and ignored); paper_1402_6964_gb300/
 * tune.py writes one from measurements.
 * mrnmf_tune_load: replace the table with the file at `path` (NULL: clear
 * it).  MRNMF_ERR_INVALID_ARG if the file is unreadable or a line is
 * malformed (the table is then unchanged).  Host only; make no call that
 * runs a pass concurrently with it.
 * mrnmf_tune_query: the stream factor a pass of n columns over m rows would
 * use, and (batch_waves, 3 doubles, nullable) each family's planned waves
 * (0 = the built-in default).  Host only.
 * mrnmf_tune_leaf_rows: the tile height a binary32 pass of n columns with k
 * projection rows would stage on the warp leaf, after the variables, the
 * table and the default, or the lane-group leaf's super-tile (32 * 64/S rows,
 * S = 4, 8 or 16 lanes a stream) where that leaf serves (n, k); 0 where
 * neither does;
 * MRNMF_ERR_INVALID_ARG for a NULL tile_rows, n < 1 or k < 0.  Host only.
 */
mrnmf_status mrnmf_tune_load(const char* path);
mrnmf_status mrnmf_tune_query(int32_t n, int64_t m, double* stream_factor, double* batch_waves);
mrnmf_status mrnmf_tune_leaf_rows(int32_t n, int32_t k, int32_t* tile_rows);

#ifdef __cplusplus
}
#endif

#endif /* MRNMF_H */
