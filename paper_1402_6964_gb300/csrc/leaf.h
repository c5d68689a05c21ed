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
};

// Warp-per-stream leaf (tsqr_warp.cu): binary32, n <= 64.  Streams = grid * warps_per_cta().
bool warp_leaf_supported(int n, int k);
int warp_leaf_rows_per_tile(int n);
int warp_leaf_warps_per_cta();
int warp_leaf_ctas_per_sm(int n, int k);
cudaError_t launch_warp_leaf(const LeafArgs& a, int streams, cudaStream_t s);

// Wide tree level (binary32, n <= 64): P_in triangles -> *P_out = ceil(P_in / (S+1)).
bool wide_tree_supported(int n);
cudaError_t tree_wide_level(const float* Rin, int P_in, int n, float* Rout, cudaStream_t s, int* P_out);

}  // namespace mrnmf
