// tsqr_group.cu -- the lane-group leaf of the binary32 TSQR pass for narrow X
// (n <= 28, no projection).
//
// The local step of TSQR (Sec. 3.1) is a Householder QR of [R; A] for each
// row block A of a stream.  With one column per lane and one stream per warp
// (tsqr_warp.cu), a narrow X leaves most of a column step's cost fixed, and
// every lane has to receive the whole pivot column of its rows through shared
// memory: a tile's worth of shared-memory traffic per column step, which
// bounds that layout at small n.
//
// Here a warp runs 32/S independent Householder streams in lane groups of S
// lanes (S = 4, 8, 16 or 32, the smallest power of two >= max(n, 4)), and every
// lane holds whole rows: 64/S rows of the group's 64-row block, all n columns,
// in registers.  The pivot column of a step is then local to each lane; what
// crosses lanes is the vector of dot products g_c = A(:, j) . A(:, c) of the
// live columns c >= j and one scalar per column for the update.  Groups of 4
// and 8 lanes sum the dot products by xor shuffles and broadcast the scalars
// by shuffles; groups of 16 and 32 lanes pass both through shared memory
// (each lane's partials stored transposed and summed by the lane that owns
// the column, the scalars read back four at a time).  Lane s of a group also
// holds column s of the group's triangle (r[i] = R(i, s), i <= s).  n is a
// template parameter, so the finished columns c < j cost nothing, and the dot
// products and the update run on packed binary32 FMAs (two rows per
// instruction).
//
// The pass sees one stream per warp, as with the warp leaf: the warp stages
// super-tiles of 32 * 64/S consecutive rows by one bulk copy, lane l taking
// rows l, l + 32, l + 64, ... of each (any partition of the rows gives the same
// R up to rounding order).  At the end of a launch the CTA's 4 * 32/S
// triangles are folded into one by column steps in the column layout (each
// absorbed triangle is an n-row block), and the column sums of all lanes are
// added before each binary64 flush.
#include "group_leaf.cuh"

namespace mrnmf {

// One case per width n = 1 .. 16: CALL<n>(ARGS).
#define MRNMF_BY_WIDTH(n, CALL, ...)                 \
    switch (n) {                                     \
    case 1: return CALL<1>(__VA_ARGS__);         \
    case 2: return CALL<2>(__VA_ARGS__);         \
    case 3: return CALL<3>(__VA_ARGS__);         \
    case 4: return CALL<4>(__VA_ARGS__);         \
    case 5: return CALL<5>(__VA_ARGS__);         \
    case 6: return CALL<6>(__VA_ARGS__);         \
    case 7: return CALL<7>(__VA_ARGS__);         \
    case 8: return CALL<8>(__VA_ARGS__);         \
    case 9: return CALL<9>(__VA_ARGS__);         \
    case 10: return CALL<10>(__VA_ARGS__);       \
    case 11: return CALL<11>(__VA_ARGS__);       \
    case 12: return CALL<12>(__VA_ARGS__);       \
    case 13: return CALL<13>(__VA_ARGS__);       \
    case 14: return CALL<14>(__VA_ARGS__);       \
    case 15: return CALL<15>(__VA_ARGS__);       \
    default: return CALL<16>(__VA_ARGS__);       \
    }


cudaError_t group_launch_narrow(const LeafArgs& a, int streams, cudaStream_t s)
{
    MRNMF_BY_WIDTH(a.n, launch_group, a, streams, s)
}

int group_ctas_narrow(int n) { MRNMF_BY_WIDTH(n, group_ctas, ) }

#undef MRNMF_BY_WIDTH

bool group_leaf_supported(int n, int k)
{
    static const bool on = [] {
        const char* e = getenv("MRNMF_GROUP_LEAF");
        return !(e && e[0] == '0');
    }();
    // measured on GB300 against the warp leaf (k = 0, about 2 GB): 1264 / 933 GB/s
    // at n = 17, 970 / 850 at n = 25, 865 / 839 at n = 28, 683 / 825 at n = 32
    return on && n >= 1 && n <= 28 && k <= 0;
}

int group_leaf_rows_per_tile(int n) { return 32 * (64 / group_lanes(n)); }

int group_leaf_ctas_per_sm(int n) { return n <= 16 ? group_ctas_narrow(n) : group_ctas_wide(n); }

cudaError_t launch_group_leaf(const LeafArgs& a, int streams, cudaStream_t s)
{
    if (!group_leaf_supported(a.n, (a.gx != nullptr) ? a.k : 0)) return cudaErrorInvalidValue;
    const int TR = group_leaf_rows_per_tile(a.n);
    if ((a.tile_rows != 0 && a.tile_rows != TR) || a.rows_per_cta % TR != 0) return cudaErrorInvalidValue;
    return a.n <= 16 ? group_launch_narrow(a, streams, s) : group_launch_wide(a, streams, s);
}

}  // namespace mrnmf
