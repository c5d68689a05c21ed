// batched.cu -- many independent tall-and-skinny problems (uneven m and n) in
// one pass: mrnmf_tsqr_r_batched.
//
// Problems with n <= 128 go through one leaf launch per family, each CTA
// reading its problem from a descriptor table: the warp-per-stream leaf for
// n <= 32 (64-row tiles) and 33..64 (32-row tiles, four streams per CTA), the
// warp-pipelined leaf for 65..128 (one stream per CTA).  Then one launch per
// tree level per family folds each problem's triangles (fan-in 17, 9 or 4),
// and one launch writes every R and colsum.  Problems with n > 128 run the
// one-problem pass in turn on the same stream.
//
// Planning (the host side, done per call): each problem gets a share of the
// family's streams proportional to its estimated cost m * n * (issue cost per
// column of the family's tile shape), at least one CTA (4 streams), at most
// one tile per stream; rows per stream are then ceil(m / streams) rounded up
// to the tile height.  Tile height and tree fan-in follow from n.  All of it
// is enqueued on the caller's stream without host synchronisation once the
// handle's buffers are large enough, so a warmed-up call can be captured in a
// CUDA graph and replayed.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mrnmf.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"
#include "trace.h"
#include "leaf.h"

namespace mrnmf {

namespace {

struct FinalDesc {
    const float* Rfin;
    int n;
    double* R;
    const double* cs;
    int nstreams;
    double* colsum;
};

__global__ void __launch_bounds__(256) batched_finalize_kernel(const FinalDesc* __restrict__ desc, int* status)
{
    const FinalDesc d = desc[blockIdx.x];
    const int n = d.n, nn = n * n;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        double v = 0.0;
        if (j >= i) {
            v = (double)d.Rfin[e];
            if (d.Rfin[(size_t)i * n + i] < 0.f) v = -v;
        }
        d.R[e] = v;
    }
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < d.nstreams; ++q) s += d.cs[(size_t)q * n + c];
        if (!(s > 0.0)) set_status(status, MRNMF_ERR_BAD_INPUT);
        if (d.colsum) d.colsum[c] = s;
    }
}

size_t al16(size_t b) { return (b + 15) & ~size_t(15); }

constexpr int kFam = 3;  // n <= 32 and 33..64 (warp leaf), 65..128 (warp-pipelined leaf)

struct BatchPlan {
    std::vector<BatchProblem> probs[kFam];
    std::vector<BatchCta> ctas[kFam];
    std::vector<std::vector<TreeCta>> levels[kFam];
    std::vector<FinalDesc> finals;
    std::vector<int> big;  // problems left to the one-problem pass
};

// Build the plan with device pointers into `dev` (layout: descriptors, then
// triangles, then partial sums); returns the bytes needed.  With dev == nullptr
// only sizes are computed.
// Waves of resident CTAs the pipelined family's streams are planned for
// (MRNMF_PIPE_WAVES, default 32): its CTAs run long dependent chains, so
// many short streams balance the batch (measured on the 256-problem batch:
// 2 waves 496 ms, 8 waves 413 ms, 32 waves 390 ms).
const double kPipeWaves = [] {
    const char* v = getenv("MRNMF_PIPE_WAVES");
    const double x = v ? atof(v) : 32.0;
    return x >= 1.0 && x <= 64.0 ? x : 32.0;
}();

// streams per CTA and tile height of family f
int fam_spc(int f) { return f < 2 ? 4 : 1; }
int fam_rows(int f) { return f < 2 ? warp_batched_rows_per_tile(f + 1) : pipe_leaf_rows_per_tile(); }
double fam_cost(int f, const mrnmf_problem& q)
{
    const double mn = (double)q.m * q.n;
    return f == 0 ? 2.5 * mn : (f == 1 ? 6.0 * mn : mn * q.n / 16.0);
}

size_t plan_batched(const mrnmf_problem* pr, int count, int sms, int ctas_per_sm[kFam], BatchPlan& plan,
                    unsigned char* dev, size_t* desc_bytes, size_t* cs_off, size_t* cs_bytes)
{
    plan = BatchPlan();
    // split and cost
    std::vector<int> fam(count);
    double cost[kFam] = {0.0, 0.0, 0.0};
    for (int i = 0; i < count; ++i) {
        const int n = pr[i].n;
        fam[i] = n <= 32 ? 0 : (n <= 64 ? 1 : ((n <= 128 && pipe_leaf_supported(n, 0)) ? 2 : -1));
        if (fam[i] < 0) {
            plan.big.push_back(i);
            continue;
        }
        cost[fam[i]] += fam_cost(fam[i], pr[i]);
    }
    // streams: two waves of the family's resident streams
    std::vector<int> streams(count, 0);
    std::vector<int64_t> rps(count, 0);
    for (int i = 0; i < count; ++i) {
        if (fam[i] < 0) continue;
        const int f = fam[i];
        const int L = fam_rows(f), spc = fam_spc(f);
        const double waves = tune_batch_waves(f + 1, f < 2 ? 2.0 : kPipeWaves);
        const double budget = waves * sms * ctas_per_sm[f] * spc;
        const double share = cost[f] > 0 ? fam_cost(f, pr[i]) / cost[f] : 1.0;
        int64_t s = (int64_t)(budget * share + 0.5);
        const int64_t tiles = (pr[i].m + L - 1) / L;
        s = std::min<int64_t>(s, tiles);
        s = std::max<int64_t>(spc, (s + spc - 1) / spc * spc);
        streams[i] = (int)s;
        int64_t per = (pr[i].m + s - 1) / s;
        rps[i] = (per + L - 1) / L * L;
    }
    // triangle storage: leaf triangles, then each tree level's outputs
    size_t tri_floats = 0;
    std::vector<size_t> leaf_off(count, 0);
    for (int i = 0; i < count; ++i) {
        if (fam[i] < 0) continue;
        leaf_off[i] = tri_floats;
        tri_floats += (size_t)(streams[i] / fam_spc(fam[i])) * pr[i].n * pr[i].n;
    }
    // descriptor counts first (sizes only), then pointers once the layout is known
    int nprob[kFam] = {0, 0, 0}, nctas[kFam] = {0, 0, 0};
    for (int i = 0; i < count; ++i)
        if (fam[i] >= 0) {
            nprob[fam[i]]++;
            nctas[fam[i]] += streams[i] / fam_spc(fam[i]);
        }
    // tree levels: (problem, input offset, count, output offset) per tree CTA
    std::vector<size_t> final_off(count, 0);
    std::vector<std::vector<std::tuple<int, size_t, int, size_t>>> lv_raw[kFam];
    for (int i = 0; i < count; ++i) {
        if (fam[i] < 0) continue;
        const int f = fam[i], n = pr[i].n, F = tree_fan_in(f + 1);
        size_t in_off = leaf_off[i];
        int c = streams[i] / fam_spc(f);
        int level = 0;
        while (c > 1) {
            const int outs = (c + F - 1) / F;
            const size_t out_off = tri_floats;
            tri_floats += (size_t)outs * n * n;
            if ((int)lv_raw[f].size() <= level) lv_raw[f].resize(level + 1);
            for (int g = 0; g < outs; ++g) {
                const int cnt = std::min(F, c - g * F);
                lv_raw[f][level].emplace_back(i, in_off + (size_t)g * F * n * n, cnt, out_off + (size_t)g * n * n);
            }
            in_off = out_off;
            c = outs;
            ++level;
        }
        final_off[i] = in_off;
    }
    // descriptor area, in the order pack_plan writes it
    size_t off = 0;
    for (int f = 0; f < kFam; ++f) off = al16(off + sizeof(BatchProblem) * nprob[f]);
    for (int f = 0; f < kFam; ++f) off = al16(off + sizeof(BatchCta) * nctas[f]);
    for (int f = 0; f < kFam; ++f)
        for (auto& L : lv_raw[f]) off = al16(off + sizeof(TreeCta) * L.size());
    off = al16(off + sizeof(FinalDesc) * (nprob[0] + nprob[1] + nprob[2]));
    *desc_bytes = off;
    const size_t tri_off = off;
    off = al16(off + sizeof(float) * tri_floats);
    *cs_off = off;
    size_t cs_doubles = 0;
    std::vector<size_t> cs_at(count, 0);
    for (int i = 0; i < count; ++i)
        if (fam[i] >= 0) {
            cs_at[i] = cs_doubles;
            cs_doubles += (size_t)streams[i] * pr[i].n;
        }
    *cs_bytes = sizeof(double) * cs_doubles;
    off = al16(off + *cs_bytes);
    if (!dev) return off;

    float* tri = reinterpret_cast<float*>(dev + tri_off);
    double* csb = reinterpret_cast<double*>(dev + *cs_off);
    std::vector<int> pidx(count, -1);
    for (int i = 0; i < count; ++i) {
        if (fam[i] < 0) continue;
        const int f = fam[i];
        BatchProblem b;
        b.X = static_cast<const float*>(pr[i].X);
        b.m = pr[i].m;
        b.ldx = pr[i].ldx;
        b.n = pr[i].n;
        b.rows_per_stream = rps[i];
        b.tri = tri + leaf_off[i];
        b.cs = csb + cs_at[i];
        pidx[i] = (int)plan.probs[f].size();
        plan.probs[f].push_back(b);
        for (int c = 0; c < streams[i] / fam_spc(f); ++c) plan.ctas[f].push_back(BatchCta{pidx[i], c});
        FinalDesc fd;
        fd.Rfin = tri + final_off[i];
        fd.n = pr[i].n;
        fd.R = pr[i].R;
        fd.cs = b.cs;
        fd.nstreams = streams[i];
        fd.colsum = pr[i].colsum;
        plan.finals.push_back(fd);
    }
    for (int f = 0; f < kFam; ++f)
        for (auto& L : lv_raw[f]) {
            std::vector<TreeCta> v;
            for (auto& e : L) {
                const int i = std::get<0>(e);
                v.push_back(TreeCta{tri + std::get<1>(e), std::get<2>(e), pr[i].n, tri + std::get<3>(e)});
            }
            plan.levels[f].push_back(std::move(v));
        }
    return off;
}

// Serialise the plan's descriptors into `host` (desc_bytes long) in the layout
// plan_batched computed; returns device pointers of each table.
struct PlanPtrs {
    const BatchProblem* probs[kFam];
    const BatchCta* ctas[kFam];
    std::vector<const TreeCta*> levels[kFam];
    const FinalDesc* finals;
};

PlanPtrs pack_plan(const BatchPlan& plan, unsigned char* host, unsigned char* dev)
{
    PlanPtrs p;
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes) {
        std::memcpy(host + off, src, bytes);
        const unsigned char* d = dev + off;
        off = al16(off + bytes);
        return d;
    };
    for (int f = 0; f < kFam; ++f)
        p.probs[f] = reinterpret_cast<const BatchProblem*>(
            put(plan.probs[f].data(), sizeof(BatchProblem) * plan.probs[f].size()));
    for (int f = 0; f < kFam; ++f)
        p.ctas[f] = reinterpret_cast<const BatchCta*>(put(plan.ctas[f].data(), sizeof(BatchCta) * plan.ctas[f].size()));
    for (int f = 0; f < kFam; ++f)
        for (auto& L : plan.levels[f])
            p.levels[f].push_back(reinterpret_cast<const TreeCta*>(put(L.data(), sizeof(TreeCta) * L.size())));
    p.finals = reinterpret_cast<const FinalDesc*>(put(plan.finals.data(), sizeof(FinalDesc) * plan.finals.size()));
    return p;
}

cudaError_t run_batched_plan(const BatchPlan& plan, const PlanPtrs& p, int max_n[kFam], int* status, cudaStream_t s)
{
    cudaError_t e;
    for (int f = 0; f < 2; ++f) {
        e = launch_warp_batched(p.ctas[f], (int)plan.ctas[f].size(), p.probs[f], f + 1, max_n[f], status, s);
        if (e != cudaSuccess) return e;
    }
    e = launch_pipe_batched(p.ctas[2], (int)plan.ctas[2].size(), p.probs[2], max_n[2], status, s);
    if (e != cudaSuccess) return e;
    const size_t nlev = std::max({plan.levels[0].size(), plan.levels[1].size(), plan.levels[2].size()});
    for (size_t l = 0; l < nlev; ++l)
        for (int f = 0; f < kFam; ++f)
            if (l < plan.levels[f].size()) {
                e = launch_tree_batched(p.levels[f][l], (int)plan.levels[f][l].size(), f + 1, s);
                if (e != cudaSuccess) return e;
            }
    if (!plan.finals.empty()) {
        batched_finalize_kernel<<<(int)plan.finals.size(), 256, 0, s>>>(p.finals, status);
        count_launch();
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace
}  // namespace mrnmf

using namespace mrnmf::api;

extern "C" mrnmf_status mrnmf_tsqr_r_batched(mrnmf_handle* h, const mrnmf_problem* pr, int32_t count, void* stream)
{
    MRNMF_TRACE("mrnmf_tsqr_r_batched");
    if (!h) return MRNMF_ERR_INVALID_ARG;
    if (!pr || count < 1) return fail(h, MRNMF_ERR_INVALID_ARG, "need count >= 1 problems");
    for (int i = 0; i < count; ++i) {
        const mrnmf_problem& q = pr[i];
        if (!q.X || !q.R) return fail(h, MRNMF_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": X and R required");
        if (q.n < 1 || q.n > MRNMF_NMAX || q.m < q.n || q.ldx < q.n)
            return fail(h, MRNMF_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": need 1 <= n <= 256, m >= n, ldx >= n");
    }
    mrnmf_status st = bind_device(h);
    if (st != MRNMF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int max_n[3] = {1, 1, 65};
    for (int i = 0; i < count; ++i) {
        if (pr[i].n <= 32) max_n[0] = std::max(max_n[0], (int)pr[i].n);
        else if (pr[i].n <= 64) max_n[1] = std::max(max_n[1], (int)pr[i].n);
        else if (pr[i].n <= 128) max_n[2] = std::max(max_n[2], (int)pr[i].n);
    }
    int ctas[3] = {mrnmf::warp_leaf_ctas_per_sm(32, 0), mrnmf::warp_leaf_ctas_per_sm(64, 0),
                   mrnmf::pipe_leaf_ctas_per_sm(max_n[2], 0)};
    mrnmf::BatchPlan plan;
    size_t desc_bytes = 0, cs_off = 0, cs_bytes = 0;
    const size_t need = mrnmf::plan_batched(pr, count, sms, ctas, plan, nullptr, &desc_bytes, &cs_off, &cs_bytes);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if ((need > h->bws_bytes || desc_bytes > h->bstage_bytes) && capturing)
        return fail(h, MRNMF_ERR_INVALID_ARG, "run this batch once before capturing it (buffers must be sized)");
    if ((st = grow(h, &h->bws, &h->bws_bytes, need, "batched workspace")) != MRNMF_OK) return st;
    cudaError_t e;
    if (desc_bytes > h->bstage_bytes) {
        if (h->bstage) {
            cudaFreeHost(h->bstage);
            h->bstage = nullptr;
            h->bstage_bytes = 0;
        }
        if ((e = cudaHostAlloc(&h->bstage, desc_bytes, cudaHostAllocDefault)) != cudaSuccess)
            return cuda_fail(h, e, "batched staging");
        h->bstage_bytes = desc_bytes;
    }
    if (!h->ev_bstage && (e = cudaEventCreateWithFlags(&h->ev_bstage, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(h, e, "event");
    // the previous batched call's descriptor copy must have left the staging area
    if (!capturing && (e = cudaEventSynchronize(h->ev_bstage)) != cudaSuccess) return cuda_fail(h, e, "staging");
    unsigned char* devb = static_cast<unsigned char*>(h->bws);
    mrnmf::plan_batched(pr, count, sms, ctas, plan, devb, &desc_bytes, &cs_off, &cs_bytes);
    const mrnmf::PlanPtrs ptrs = mrnmf::pack_plan(plan, static_cast<unsigned char*>(h->bstage), devb);
    if ((e = cudaMemcpyAsync(devb, h->bstage, desc_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(h, e, "descriptor upload");
    // (not inside a stream capture: a captured record would leave the event
    // in the graph, and the next eager call could not wait on it)
    if (!capturing && (e = cudaEventRecord(h->ev_bstage, s)) != cudaSuccess) return cuda_fail(h, e, "event");
    if (cs_bytes && (e = cudaMemsetAsync(devb + cs_off, 0, cs_bytes, s)) != cudaSuccess)
        return cuda_fail(h, e, "partial sums");
    if ((e = mrnmf::run_batched_plan(plan, ptrs, max_n, h->d_status, s)) != cudaSuccess)
        return cuda_fail(h, e, "batched pass");
    for (int i : plan.big) {
        st = run_pass(h, pr[i].X, pr[i].m, pr[i].n, pr[i].ldx, MRNMF_F32, MRNMF_PREC_FP32, 1, pr[i].R, pr[i].colsum, 0,
                      0, 0, nullptr, s);
        if (st != MRNMF_OK) return st;
    }
    return MRNMF_OK;
}
