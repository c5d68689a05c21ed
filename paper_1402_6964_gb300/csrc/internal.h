// internal.h -- host-side interfaces between the C ABI (api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>

namespace mrnmf {

// Kernels launched by this library (mrnmf_kernel_launches).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Running state of one pass: P independent row streams ("mappers" of
// Sec. 3.5), each with its own n-by-n triangle and its partial column sums
// and Gaussian projection.
struct PassState {
    int n = 0;
    int k = 0;          // Gaussian rows (0 = no projection)
    int P = 0;          // number of row streams (partial-sum slots)
    int tri = 0;        // triangle slots the leaf leaves for the tree (P, or P / 4 when
                        // the warp leaf folds each CTA's four streams into one)
    int fp64 = 0;       // 1: triangles and reflectors in binary64, else binary32
    int tc = 0;         // tensor-core leaf: 1 = TF32X3 (three products), 2 = TF32 (one); 0 = none
    int tree64 = 0;     // 1: binary32 leaf triangles reduced by a binary64 tree
    int gp_form = 0;    // projection-only pass on tcgen05: MRNMF_PREC_TF32X3 or MRNMF_PREC_BF16
                        // (0: SIMT, or TF32X3 with MRNMF_GP_TC=1)
    void* R = nullptr;      // P * n * n (dense row-major, zeros below diag), T = float or double
    void* Rtmp = nullptr;   // ceil(P/2) * n * n binary64, ping-pong buffer of the tree
    double* cs = nullptr;   // P * n partial column sums
    double* gx = nullptr;   // P * k * n partial projections
    uint64_t seed = 0;
    int64_t rows_seen = 0;  // global row index of the next row (Gaussian key)
    cudaEvent_t ev_leaf_start = nullptr;  // optional timing events around the leaf kernel
    cudaEvent_t ev_leaf_stop = nullptr;
};

size_t pass_state_bytes(int n, int k, int P, int fp64);
void pass_state_carve(PassState& st, void* base);

// The binary64 tree over binary32 leaf triangles exists for this n (its
// packed triangle fits a CTA's shared memory).
bool tree64_supported(int n);
// MRNMF_TREE64=1 selects it for binary32 passes.
bool tree64_requested();

// The tuning table (tune.cu): a factor on the stream count of a pass of n
// columns over m rows (1 without an entry), and the waves a batch family's
// streams are planned for (`dflt` without an entry).
double tune_stream_factor(int n, int64_t m);
double tune_batch_waves(int family, double dflt);
int tune_leaf_rows(int n, int k);  // the table's warp-leaf tile height for (n, k); 0 without a `rows` line

// Number of streams for a pass over about `m` rows (0 = unknown / streaming).
int choose_streams(int n, int k, int fp64, int tc, int64_t m);

// The tensor-core form a projection-only pass takes: gp_form if nonzero, else
// MRNMF_PREC_TF32X3 under MRNMF_GP_TC=1, else 0 (the SIMT pass).
int gp_pass_form(int gp_form);

// Zero the state (triangles and partials) for a new pass.
cudaError_t pass_reset(const PassState& st, cudaStream_t s);

// Fold `rows` rows of X (row-major, ldx) into the state.  xf64: X is binary64.
// qr = 0 skips the triangle (Gaussian projection / column sums only).
cudaError_t pass_push(PassState& st, const void* X, int64_t rows, int64_t ldx, int xf64, int qr,
                      int* status, cudaStream_t s);

// Reduce the P triangles to one (tree over the stacked R's, Sec. 3.1), then
// write R (sign-normalised, binary64), colsum and GX (either may be NULL).
cudaError_t pass_finish(PassState& st, int qr, double* R, double* colsum, double* GX, int* status,
                        cudaStream_t s);

// ---- the n-by-n separable step (small_step.cu) ----
size_t small_ws_bytes(int n, int k, int r);
cudaError_t select_spa(const double* R, int n, const double* colsum, int r, int32_t* K, double* gap,
                       void* ws, int* status, cudaStream_t s);
cudaError_t select_xray(const double* R, int n, int r, int32_t* K, double* gap, void* ws, int* status,
                        cudaStream_t s);
cudaError_t select_gp(const double* GX, int k, int n, const double* colsum, int r, int32_t* K, double* gap,
                      void* ws, int* status, cudaStream_t s);
cudaError_t nnls_h(const double* R, int n, const int32_t* K, int r, double* H, void* ws, int* status,
                   cudaStream_t s);
cudaError_t residual(const double* R, int n, const int32_t* K, int r, const double* H, double* out, void* ws,
                     cudaStream_t s);

// ---- tensor-core leaf (tsqr_wy.cu) ----
bool tc_supported(int n, int k);   // the TF32X3 pass exists for this shape
bool tc_preferred(int n, int k);   // and MRNMF_PREC_AUTO picks it

// ---- tensor-core Gaussian projection pass (gp_tc.cu) ----
bool gp_tc_supported(int n, int k);
// bf16 = 1: bfloat16 operands (MRNMF_PREC_BF16), else split TF32 (MRNMF_PREC_TF32X3).
cudaError_t launch_gp_tc(const float* X, int64_t rows, int64_t ldx, int n, int k, int64_t row_base, uint64_t seed,
                         int max_ctas, double* cs, double* gx, int* status, int bf16, cudaStream_t s);

}  // namespace mrnmf
