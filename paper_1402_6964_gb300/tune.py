"""Write libmrnmf's tuning table for the GPU this runs on, from measurements.

    python -m paper_1402_6964_gb300.tune [--out PATH] [--reps N]

The table (format in include/mrnmf.h, "Tuning table") holds, per bucket of
(n, k) on the warp leaf (n <= 64), the tile height its tiles are staged in;
per bucket of (n, log2 m), a factor on the default number of row streams of a
pass; and per batch family the waves of resident CTAs its streams are planned
for.  This times, in that order: for every (n, k) bucket the FP32 pass
(mrnmf_tsqr_r, or mrnmf_tsqr_gp for k > 0) on uniform X of 2^24 rows with each
height the leaf's form has; for every (n, log2 m) bucket the FP32 pass
(k = 0) on uniform X of the bucket's representative shape with each candidate
factor, under the heights already chosen; for every batch family the batched
call on a drawn batch of that family's shapes with each candidate wave count.
A setting goes into the table only where it beats the built-in default by more
than 3 %, and again when the two are timed once more.  Candidates are loaded one at a time through mrnmf_tune_load, so the
measurement uses the library's own path.
"""
from __future__ import annotations

import argparse
import datetime
import math
import os
import statistics
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# warp-leaf tile heights: (n_lo, n_hi, representative n, heights, default first)
# and (k_lo, k_hi, representative k)
ROWS_N_BUCKETS = [(1, 16, 12, [64, 128]), (17, 32, 25, [64, 128]), (33, 48, 40, [32, 64]), (49, 64, 60, [32, 64])]
ROWS_K_BUCKETS = [(0, 0, 0), (1, 64, 20)]
ROWS_LOG2M = 24
# (n_lo, n_hi, representative n) and (log2 m lo, hi, representative log2 m)
N_BUCKETS = [(1, 16, 12), (17, 32, 25), (33, 64, 50), (65, 128, 100), (129, 256, 200)]
M_BUCKETS = [(0.0, 15.0, 14.0), (15.0, 18.0, 16.5), (18.0, 21.0, 19.5), (21.0, 24.0, 22.5), (24.0, 64.0, 24.0)]
FACTORS = [0.125, 0.25, 0.5, 1.0, 2.0]
WAVES = {1: [1.0, 2.0, 4.0], 2: [1.0, 2.0, 4.0], 3: [8.0, 16.0, 32.0, 64.0]}
MAX_BYTES = 4 << 30  # largest X drawn for one bucket
GAIN = 0.03


def _time(fn, reps, sync):
    """Median over `reps` of the time of one call; calls shorter than about
    2 ms are timed in back-to-back groups so that launch jitter averages out."""
    import torch
    for _ in range(2):
        fn()
    sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    b.record()
    sync()
    inner = max(1, min(64, math.ceil(2.0 / max(a.elapsed_time(b), 1e-3))))
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(inner):
            fn()
        b.record()
        sync()
        ts.append(a.elapsed_time(b) / inner)
    return statistics.median(ts)


def _pick(res, dflt, remeasure):
    """The fastest setting if it beats `dflt` by more than GAIN in `res` and
    again when both are measured once more (remeasure(setting) -> ms);
    otherwise `dflt`.  Returns (setting, default ms, setting ms)."""
    best = min(res, key=res.get)
    if best == dflt or res[best] >= (1.0 - GAIN) * res[dflt]:
        return dflt, res[dflt], res[dflt]
    t_d, t_b = remeasure(dflt), remeasure(best)
    if t_b >= (1.0 - GAIN) * t_d:
        return dflt, res[dflt], res[dflt]
    return best, t_d, t_b


def _with_table(lines):
    """Load a table of `lines` into the library (a temporary file)."""
    from paper_1402_6964_gb300 import mrnmf
    fd, path = tempfile.mkstemp(suffix=".txt")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    st = mrnmf.tune_load(path)
    os.unlink(path)
    if st != mrnmf.OK:
        raise RuntimeError(f"tune_load rejected {lines}")


def sweep_rows(h, reps, log):
    import torch

    from paper_1402_6964_gb300 import mrnmf
    out = []
    for n_lo, n_hi, n, heights in ROWS_N_BUCKETS:
        m = min(2 ** ROWS_LOG2M, MAX_BYTES // (4 * n))
        X = torch.rand(m, n, device="cuda")
        for k_lo, k_hi, k in ROWS_K_BUCKETS:
            res = {}
            for L in heights:
                _with_table([f"rows {n_lo} {n_hi} {k_lo} {k_hi} {L}"])
                if mrnmf.tune_leaf_rows(n, k) != L:
                    log(f"n={n} k={k}: height {L} does not fit; skipped")
                    continue
                if k:
                    res[L] = _time(lambda: h.tsqr_gp(X, k, seed=1, prec="fp32"), reps, h.sync)
                else:
                    res[L] = _time(lambda: h.tsqr_r(X, prec="fp32"), reps, h.sync)
            dflt = heights[0]
            if dflt not in res:
                log(f"rows n={n} k={k}: another leaf serves this shape (its tile height is not tuned); skipped")
                continue

            def again(L, k=k, n_lo=n_lo, n_hi=n_hi, k_lo=k_lo, k_hi=k_hi, X=X):
                _with_table([f"rows {n_lo} {n_hi} {k_lo} {k_hi} {L}"])
                if k:
                    return _time(lambda: h.tsqr_gp(X, k, seed=1, prec="fp32"), reps, h.sync)
                return _time(lambda: h.tsqr_r(X, prec="fp32"), reps, h.sync)
            best, t_d, t_b = _pick(res, dflt, again)
            _with_table([])
            log(f"rows n={n} k={k} m={m}: " + ", ".join(f"{L}: {t:.3f} ms" for L, t in res.items()) + f" -> {best}")
            if best != dflt:
                out.append((f"rows {n_lo} {n_hi} {k_lo} {k_hi} {best}",
                            f"n={n} k={k} m={m}: {dflt} rows {t_d:.3f} -> {best} rows {t_b:.3f} ms"))
        del X
        torch.cuda.empty_cache()
    return out


def sweep_passes(h, reps, log, fixed):
    """Stream factors per (n, log2 m) bucket, under the table lines `fixed`."""
    import torch
    out = []
    for n_lo, n_hi, n in N_BUCKETS:
        for lg_lo, lg_hi, lg in M_BUCKETS:
            m = max(int(2 ** lg), n)
            if 4 * m * n > MAX_BYTES:
                m = MAX_BYTES // (4 * n)
                if not lg_lo <= math.log2(m) < lg_hi:
                    log(f"n={n}: bucket [{lg_lo:g}, {lg_hi:g}) of log2 m needs more than {MAX_BYTES >> 30} GB; skipped")
                    continue
            X = torch.rand(m, n, device="cuda")
            res = {}
            for f in FACTORS:
                _with_table(fixed + [f"pass {n_lo} {n_hi} {lg_lo} {lg_hi} {f}"])
                res[f] = _time(lambda: h.tsqr_r(X, prec="fp32"), reps, h.sync)

            def again(f, n_lo=n_lo, n_hi=n_hi, lg_lo=lg_lo, lg_hi=lg_hi, X=X):
                _with_table(fixed + [f"pass {n_lo} {n_hi} {lg_lo} {lg_hi} {f}"])
                return _time(lambda: h.tsqr_r(X, prec="fp32"), reps, h.sync)
            best, t_d, t_b = _pick(res, 1.0, again)
            _with_table([])
            log(f"n={n} m={m}: " + ", ".join(f"{f}: {t:.3f} ms" for f, t in res.items()) + f" -> {best}")
            if best != 1.0:
                out.append((f"pass {n_lo} {n_hi} {lg_lo:g} {lg_hi:g} {best:g}", f"n={n} m={m}: {t_d:.3f} -> {t_b:.3f} ms"))
            del X
            torch.cuda.empty_cache()
    return out


def sweep_batches(h, reps, log):
    import torch

    from paper_1402_6964_gb300 import synth
    out = []
    ranges = {1: (10, 32), 2: (33, 64), 3: (65, 128)}
    for fam, (n_lo, n_hi) in ranges.items():
        specs = synth.batch_problems(48, seed=1402005 + fam, m_lo=1e4, m_hi=2e6, n_lo=n_lo, n_hi=n_hi)
        Xs = [synth.device_planted(m, n, r, seed=1402005 * 1000 + 97 * fam + i, noise=1e-3)[0]
              for i, (m, n, r) in enumerate(specs)]
        outs = [(torch.empty((X.shape[1], X.shape[1]), dtype=torch.float64, device="cuda"),
                 torch.empty(X.shape[1], dtype=torch.float64, device="cuda")) for X in Xs]
        res = {}
        for wv in WAVES[fam]:
            _with_table([f"batch {fam} {wv}"])
            res[wv] = _time(lambda: h.tsqr_r_batched(Xs, outs=outs), reps, h.sync)
        dflt = 2.0 if fam < 3 else 32.0

        def again(wv, fam=fam, Xs=Xs, outs=outs):
            _with_table([f"batch {fam} {wv}"])
            return _time(lambda: h.tsqr_r_batched(Xs, outs=outs), reps, h.sync)
        best, t_d, t_b = _pick(res, dflt, again)
        _with_table([])
        log(f"batch family {fam}: " + ", ".join(f"{w:g}: {t:.2f} ms" for w, t in res.items()) + f" -> {best:g}")
        if best != dflt:
            out.append((f"batch {fam} {best:g}", f"family {fam}: {t_d:.2f} -> {t_b:.2f} ms"))
        del Xs, outs
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_gb300.txt"))
    ap.add_argument("--reps", type=int, default=7)
    args = ap.parse_args()
    import torch

    from paper_1402_6964_gb300 import build, mrnmf
    build.build()
    torch.cuda.set_device(0)
    h = mrnmf.Handle()
    log = lambda s: print(s, file=sys.stderr, flush=True)
    rows = sweep_rows(h, args.reps, log)
    entries = rows + sweep_passes(h, args.reps, log, [line for line, _ in rows])
    entries += sweep_batches(h, max(3, args.reps // 2), log)
    h.close()
    name = torch.cuda.get_device_name(0)
    with open(args.out, "w") as f:
        f.write(f"# libmrnmf tuning table for {name}, written by paper_1402_6964_gb300/tune.py on "
                f"{datetime.date.today().isoformat()}\n")
        f.write("# each line: the setting, then the measurement that chose it (default -> tuned)\n")
        for line, why in entries:
            f.write(f"{line}\n# {why}\n")
    print(args.out)


if __name__ == "__main__":
    main()
