// tune.cu -- the tuning table: per (n bucket, log2 m bucket) a factor on the
// pass's stream count, per (n bucket, k bucket) the tile height of the warp
// leaf, and per batch family the number of waves of resident CTAs its streams
// are planned for.  The table is plain text, written by
// paper_1402_6964_gb300/tune.py from measurements on the GPU it serves:
//
//     # comment
//     pass  <n_lo> <n_hi> <log2m_lo> <log2m_hi> <stream_factor>
//     rows  <n_lo> <n_hi> <k_lo> <k_hi> <tile_rows 32|64|128>
//     batch <family 1..3> <waves>
//
// A pass of n columns and m rows uses the factor of the first `pass` line with
// n_lo <= n <= n_hi and log2m_lo <= log2(m) < log2m_hi (1 without one), and
// the warp leaf (n <= 64) with k projection rows the height of the first
// `rows` line with n_lo <= n <= n_hi and k_lo <= k <= k_hi, where its form has
// that height (64 or 128 rows for n <= 32, 32 or 64 above).  The table is read
// from MRNMF_TUNE_FILE on first use, or replaced at any time by
// mrnmf_tune_load; a pass keeps the height it was planned with.  Only the
// amount and shape of the parallel work change: every setting computes the
// same R up to rounding order.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/mrnmf.h"
#include "internal.h"
#include "leaf.h"

namespace mrnmf {
namespace {

struct PassEntry {
    int n_lo, n_hi;
    double lg_lo, lg_hi, factor;
};

struct RowsEntry {
    int n_lo, n_hi, k_lo, k_hi, rows;
};

struct Table {
    std::vector<PassEntry> pass;
    std::vector<RowsEntry> rows;
    double waves[3] = {0.0, 0.0, 0.0};  // 0: no entry
};

std::mutex g_mu;
bool g_init = false;
Table g_tab;

// Parse `path` into `t`; false on any malformed line.
bool parse(const char* path, Table& t)
{
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool ok = true;
    while (ok && fgets(line, sizeof line, f)) {
        char* s = line;
        while (*s == ' ' || *s == '\t') ++s;
        if (*s == '#' || *s == '\n' || *s == '\r' || *s == 0) continue;
        PassEntry e;
        RowsEntry r;
        int fam = 0;
        double w = 0.0;
        if (sscanf(s, "pass %d %d %lf %lf %lf", &e.n_lo, &e.n_hi, &e.lg_lo, &e.lg_hi, &e.factor) == 5) {
            ok = e.n_lo >= 1 && e.n_hi >= e.n_lo && e.lg_hi > e.lg_lo && e.factor > 0.0 && e.factor <= 64.0;
            if (ok) t.pass.push_back(e);
        } else if (sscanf(s, "rows %d %d %d %d %d", &r.n_lo, &r.n_hi, &r.k_lo, &r.k_hi, &r.rows) == 5) {
            ok = r.n_lo >= 1 && r.n_hi >= r.n_lo && r.k_lo >= 0 && r.k_hi >= r.k_lo &&
                 (r.rows == 32 || r.rows == 64 || r.rows == 128);
            if (ok) t.rows.push_back(r);
        } else if (sscanf(s, "batch %d %lf", &fam, &w) == 2) {
            ok = fam >= 1 && fam <= 3 && w >= 0.25 && w <= 256.0;
            if (ok) t.waves[fam - 1] = w;
        } else {
            ok = false;
        }
    }
    fclose(f);
    return ok;
}

void ensure_loaded()
{
    if (g_init) return;
    g_init = true;
    const char* p = getenv("MRNMF_TUNE_FILE");
    if (p && *p) {
        Table t;
        if (parse(p, t)) {
            g_tab = t;
        } else {
            fprintf(stderr, "libmrnmf: MRNMF_TUNE_FILE %s is unreadable or malformed; using the defaults\n", p);
        }
    }
}

}  // namespace

double tune_stream_factor(int n, int64_t m)
{
    if (m <= 0) return 1.0;
    std::lock_guard<std::mutex> lock(g_mu);
    ensure_loaded();
    const double lg = std::log2((double)m);
    for (const PassEntry& e : g_tab.pass)
        if (n >= e.n_lo && n <= e.n_hi && lg >= e.lg_lo && lg < e.lg_hi) return e.factor;
    return 1.0;
}

int tune_leaf_rows(int n, int k)
{
    std::lock_guard<std::mutex> lock(g_mu);
    ensure_loaded();
    for (const RowsEntry& e : g_tab.rows)
        if (n >= e.n_lo && n <= e.n_hi && k >= e.k_lo && k <= e.k_hi) return e.rows;
    return 0;
}

double tune_batch_waves(int family, double dflt)
{
    std::lock_guard<std::mutex> lock(g_mu);
    ensure_loaded();
    return (family >= 1 && family <= 3 && g_tab.waves[family - 1] > 0.0) ? g_tab.waves[family - 1] : dflt;
}

}  // namespace mrnmf

extern "C" mrnmf_status mrnmf_tune_load(const char* path)
{
    std::lock_guard<std::mutex> lock(mrnmf::g_mu);
    mrnmf::g_init = true;  // an explicit load replaces whatever MRNMF_TUNE_FILE said
    if (!path) {
        mrnmf::g_tab = mrnmf::Table();
        return MRNMF_OK;
    }
    mrnmf::Table t;
    if (!mrnmf::parse(path, t)) return MRNMF_ERR_INVALID_ARG;
    mrnmf::g_tab = t;
    return MRNMF_OK;
}

extern "C" mrnmf_status mrnmf_tune_query(int32_t n, int64_t m, double* stream_factor, double* batch_waves)
{
    if (!stream_factor && !batch_waves) return MRNMF_ERR_INVALID_ARG;
    if (stream_factor) *stream_factor = mrnmf::tune_stream_factor(n, m);
    if (batch_waves)
        for (int f = 1; f <= 3; ++f) batch_waves[f - 1] = mrnmf::tune_batch_waves(f, 0.0);
    return MRNMF_OK;
}

extern "C" mrnmf_status mrnmf_tune_leaf_rows(int32_t n, int32_t k, int32_t* tile_rows)
{
    if (!tile_rows || n < 1 || k < 0) return MRNMF_ERR_INVALID_ARG;
    *tile_rows = mrnmf::warp_leaf_supported(n, k) ? mrnmf::warp_leaf_rows_per_tile(n, k) : 0;
    return MRNMF_OK;
}
