// leaf.h -- arguments of the pass kernels, shared by the SIMT leaf
// translation units (tsqr_simt.cu, tsqr_warp.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mrnmf {

struct LeafArgs {
    const void* X;
    int64_t rows;          // rows of X in this launch
    int64_t ldx;
    int n;
    int64_t rows_per_cta;  // leaf: rows per stream (multiple of the tile height); tree: triangles per CTA
    int64_t row_base;      // global row index of X's row 0 (Gaussian key)
    const void* R_in;      // leaf: state to continue (nullptr = zeros); tree: input triangles
    void* R_out;
    int P_in;              // tree: number of input triangles
    double* cs;            // P * n (+=), nullptr = skip
    double* gx;            // P * k * n (+=), nullptr = skip
    int k;
    uint64_t seed;
    int check;             // reject negative / NaN entries
    int* status;
    int tile_rows;         // warp leaf: tile height the pass was planned with (0 = warp_leaf_rows_per_tile)
    int tc_split;          // tensor-core leaf: 1 = three TF32 products (hi*hi + hi*lo + lo*hi), 0 = one
    int ring_depth;        // pipelined leaf: tiles in flight in the reflector ring, 2 or 4 (0 = 2)
};

// Batched pass: one problem per entry, CTAs described one by one.
struct BatchProblem {
    const float* X;
    int64_t m;
    int64_t ldx;
    int n;
    int64_t rows_per_stream;  // multiple of the family's tile height
    float* tri;               // this problem's leaf triangles (one per CTA, n*n each)
    double* cs;               // this problem's partial column sums (one n-vector per stream)
};
struct BatchCta {
    int p;    // problem
    int cta;  // CTA index within the problem (warp families: streams 4*cta .. 4*cta+3; family 3: stream cta)
};

struct TreeCta {
    const float* in;  // `count` consecutive n*n triangles
    int count;        // 1 .. fan-in
    int n;
    float* out;       // one n*n triangle
};

// Warp-per-stream leaf (tsqr_warp.cu): binary32, n <= 64.  Streams = grid * warps_per_cta().
bool warp_leaf_supported(int n, int k);
int warp_leaf_rows_per_tile(int n, int k);
int warp_leaf_warps_per_cta();
int warp_leaf_ctas_per_sm(int n, int k);
cudaError_t launch_warp_leaf(const LeafArgs& a, int streams, cudaStream_t s);
// family 1: n <= 32 (64-row tiles), family 2: 33 <= n <= 64 (32-row tiles)
cudaError_t launch_warp_batched(const BatchCta* desc, int nctas, const BatchProblem* probs, int family, int max_n,
                                int* status, cudaStream_t s);
int warp_batched_rows_per_tile(int family);

// Lane-group leaf (tsqr_group.cu): binary32, n <= 28, no projection; four
// warps per CTA, one stream of the pass per warp (32/S Householder streams of
// S lanes inside it, folded at the end of the launch).  The warp leaf's
// functions dispatch to it; MRNMF_GROUP_LEAF=0 turns it off.
bool group_leaf_supported(int n, int k);
int group_leaf_rows_per_tile(int n);
int group_leaf_ctas_per_sm(int n);
cudaError_t launch_group_leaf(const LeafArgs& a, int streams, cudaStream_t s);

// CTA-per-stream leaf (tsqr_warp.cu): binary32, 64 < n <= 256.
bool cta_leaf_supported(int n, int k);
int cta_leaf_rows_per_tile(int k, int n);
int cta_leaf_ctas_per_sm(int n, int k);
cudaError_t launch_cta_leaf(const LeafArgs& a, int grid, cudaStream_t s);
int tree_fan_in(int family);

// Warp-pipelined leaf (tsqr_pipe.cu): binary32, 64 < n <= 256, one stream per CTA.
// MRNMF_PIPE_LEAF=0 falls back to the one-barrier-per-column CTA leaf.
bool pipe_leaf_supported(int n, int k);
int pipe_leaf_rows_per_tile();
int pipe_leaf_ctas_per_sm(int n, int k);
cudaError_t launch_pipe_leaf(const LeafArgs& a, int grid, cudaStream_t s);
// Batched form (batched.cu family 3): one stream per CTA, no projection.
cudaError_t launch_pipe_batched(const BatchCta* desc, int nctas, const BatchProblem* probs, int max_n, int* status,
                                cudaStream_t s);

// Projection-only pass (gp_simt.cu): binary32, n <= 64, 1 <= k <= 32, no
// triangle; one stream per warp, four per CTA.  MRNMF_GP_WARP=0 turns it off.
bool gp_warp_supported(int n, int k);
int gp_warp_rows_per_tile();
int gp_warp_streams_per_cta();
int gp_warp_streams(int n, int k, int64_t m);  // streams that fill the GPU for about m rows (0 = unknown)
cudaError_t launch_gp_warp(const LeafArgs& a, int streams, cudaStream_t s);

// Tensor-core leaf (tsqr_wy.cu): 16 < n <= 128; one stream per CTA.
int tc_leaf_rows_per_tile();
int tc_leaf_ctas_per_sm(int n);
cudaError_t launch_tc_leaf(const LeafArgs& a, int grid, cudaStream_t s);  // triangles folded per tree CTA
cudaError_t launch_tree_batched(const TreeCta* desc, int nctas, int family, cudaStream_t s);

// Wide tree level (binary32, n <= 128): P_in triangles -> *P_out = ceil(P_in / (S+1)).
bool wide_tree_supported(int n);
cudaError_t tree_wide_level(const float* Rin, int P_in, int n, float* Rout, cudaStream_t s, int* P_out);

}  // namespace mrnmf
