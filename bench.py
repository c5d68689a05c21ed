"""Benchmark of the single-pass TSQR reduction for near-separable NMF.

One step = the whole hot path over one resident synthetic X:
  the fused pass (R, column sums, Gaussian projection G^T X, Sec. 3.1-3.3),
  SPA, greedy XRAY and GP selection (Sec. 2.1, 2.3), and for each selection
  NNLS for H and the residual (Sec. 2.4).
Metric: GB/s of X read per step (4 m n bytes / step time).

Multi-GPU (torchrun): the pass has no exchange step on one box, so every rank
runs an independent replica on its own GPU; value = bytes all ranks read /
max over ranks of the timed region (CUDA events) ("scaling": "weak").

--impl reference times the FP64 CPU oracle (the only reference this project
has) on the host cores on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TSQR pass GB/s of X (% of HBM roofline), mixed vs FP32, at stated R error"
WORKLOAD = "near_sep_1e7x50"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def _fp32_simt_peak_tflops(sms: int, mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sms * 128 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms; start() waits
    for the first sample, begin() marks the start of the timed region, and
    stop() keeps the samples from the last one before begin() on."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5.0 and self._lines() == 0 and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        self.n0 = 0

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def begin(self):
        self.n0 = self._lines() if self.proc is not None else 0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()[max(0, self.n0 - 1):]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_step(X: np.ndarray, w, rows: int):
    """The oracle's whole path on the first `rows` rows of X; returns seconds."""
    import oracle
    oracle.build()
    Xs = X[:rows].astype(np.float64)
    t0 = time.perf_counter()
    R = oracle.qr_r(Xs)
    s = oracle.colsum(Xs)
    GX = oracle.gauss_project(Xs, w.k, w.seed)
    for K in (oracle.spa(R, s, w.r)[0], oracle.xray(R, w.r)[0], oracle.gp_select(GX, s, w.r)[0]):
        if np.all(K >= 0):
            H, _ = oracle.nnls_h(R, K)
            oracle.residual(R, K, H)
    return time.perf_counter() - t0


def run_reference(args):
    """The oracle as it stands on every host core: one spawned process per core,
    each step running the whole path on its own `ref_rows`-row chunk of the
    workload (a bounded sample); GB/s = rows of all processes / wall time."""
    import multiprocessing as mp

    from paper_1402_6964_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    rows = args.ref_rows
    cores, model = host_cpu_info()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        jobs = [(args.workload, c, rows) for c in range(cores)]
        for _ in range(args.warmup):
            pool.map(_oracle_chunk_worker, jobs)
        ts = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_chunk_worker, jobs)
            ts.append(time.perf_counter() - t0)
    t = sum(ts)
    gbs = 4.0 * rows * w.n * cores * args.steps / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "m": w.m, "n": w.n, "r": w.r, "k": w.k, "prec": args.prec,
                       "parallelism": "replicas" if args.gpus > 1 else "single GPU"},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "nproc": cores,
                             "cpu_model": model,
                             "sample": f"{cores} processes per step, each the whole path (pass + SPA/XRAY/GP + "
                                       f"NNLS + residual) on its own {rows}-row chunk of the {w.m}-row workload"},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gp_pass(args, quiet=False):
    """Projection-only pass: GB/s of X, SIMT (mrnmf_gauss_project) or a tensor-core
    form (mrnmf_gauss_project_tc, --gp-form tf32x3 | bf16)."""
    import torch

    from paper_1402_6964_gb300 import build, mrnmf, synth

    build.build()
    w = synth.WORKLOADS[args.workload]
    X, _ = synth.workload_matrix(w, m=args.rows)
    Xd = torch.from_numpy(X).cuda()
    h = mrnmf.Handle()
    if args.gp_form == "simt":
        proj = lambda: h.gauss_project(Xd, w.k, w.seed)
    else:
        proj = lambda: h.gauss_project_tc(Xd, w.k, w.seed, form=args.gp_form)
    for _ in range(args.warmup):
        proj()
    h.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        proj()
    b.record()
    torch.cuda.synchronize()
    h.sync()
    ms = a.elapsed_time(b) / args.steps
    hbm, _, src = _peaks()
    gbs = 4.0 * X.shape[0] * X.shape[1] / ms / 1e6
    line = {"mode": "gp", "metric": "Gaussian projection pass GB/s of X", "value": gbs, "unit": "GB/s",
            "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "path": ("tcgen05 " + args.gp_form) if args.gp_form != "simt"
            else ("tcgen05 tf32x3" if os.environ.get("MRNMF_GP_TC") == "1" else "simt"),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "peak_source": src},
            "config": {"workload": w.name, "m": X.shape[0], "n": w.n, "k": w.k}}
    h.close()
    del Xd
    torch.cuda.empty_cache()
    if not quiet:
        print(json.dumps(line), flush=True)
    return line


def run_pass(args):
    """The plain binary32 TSQR pass (mrnmf_tsqr_r, k = 0) on uniform X of
    --rows x --cols drawn on the device: pass and leaf time (library events),
    GB/s of X and the fraction of the HBM roofline."""
    import torch

    from paper_1402_6964_gb300 import build, mrnmf

    build.build()
    m, n = args.rows or 10_000_000, args.cols
    X = torch.rand(m, n, device="cuda")
    h = mrnmf.Handle()
    for _ in range(args.warmup):
        h.tsqr_r(X, prec="fp32")
    h.sync()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    l0, l1, a, b = ev(), ev(), ev(), ev()
    l0.record()
    l1.record()
    h.profile_events(l0, l1)
    tot = leaf = 0.0
    for _ in range(args.steps):
        a.record()
        h.tsqr_r(X, prec="fp32")
        b.record()
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
        leaf += l0.elapsed_time(l1)
    h.profile_events(None, None)
    h.sync()
    hbm, _, src = _peaks()
    ms, leaf_ms = tot / args.steps, leaf / args.steps
    gbs = 4.0 * m * n / leaf_ms / 1e6
    print(json.dumps({"mode": "pass", "metric": "TSQR pass GB/s of X (leaf)", "value": gbs, "unit": "GB/s",
                      "ms_per_step": ms, "leaf_ms": leaf_ms, "steps": args.steps, "warmup": args.warmup,
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                   "frac": gbs / hbm, "peak_source": src},
                      "config": {"workload": f"uniform {m}x{n}", "m": m, "n": n, "k": 0}}), flush=True)
    h.close()


def run_batched(args, quiet=False):
    """256 independent problems (m log-uniform in [1e4, 1e7], n uniform in
    10..128, r uniform in 3..min(16, n/2), sigma = 1e-3), drawn on the device:
    rows/s of per-matrix mrnmf_tsqr_r calls, of one mrnmf_tsqr_r_batched call,
    and of that call replayed as a CUDA graph."""
    import torch

    from paper_1402_6964_gb300 import build, mrnmf, synth

    build.build()
    torch.cuda.set_device(0)
    specs = synth.batch_problems(args.batch, seed=1402005)
    Xs = []
    for i, (m, n, r) in enumerate(specs):
        X, _ = synth.device_planted(m, n, r, seed=1402005 * 1000 + i, noise=1e-3)
        Xs.append(X)
    torch.cuda.synchronize()
    rows = sum(m for m, _, _ in specs)
    nbytes = sum(4.0 * m * n for m, n, _ in specs)
    h = mrnmf.Handle()
    outs = [(torch.empty((X.shape[1], X.shape[1]), dtype=torch.float64, device="cuda"),
             torch.empty(X.shape[1], dtype=torch.float64, device="cuda")) for X in Xs]
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def per_matrix():
        for X, (R, cs) in zip(Xs, outs):
            h.tsqr_r(X, prec="fp32")

    def batched():
        h.tsqr_r_batched(Xs, outs=outs)

    res = {}
    for name, fn in (("per_matrix", per_matrix), ("batched", batched)):
        for _ in range(args.warmup):
            fn()
        h.sync()
        a, b = ev(), ev()
        a.record()
        for _ in range(args.steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        h.sync()
        res[name] = a.elapsed_time(b) / args.steps
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            h.tsqr_r_batched(Xs, outs=outs, stream=st)
    torch.cuda.current_stream().wait_stream(st)
    for _ in range(args.warmup):
        g.replay()
    a, b = ev(), ev()
    a.record()
    for _ in range(args.steps):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    h.sync()
    res["batched_graph"] = a.elapsed_time(b) / args.steps
    line = {"mode": "batched", "metric": "batched TSQR pass rows/s (and GB/s of X)", "unit": "rows/s",
            "problems": len(specs), "rows": rows, "bytes": nbytes, "steps": args.steps, "warmup": args.warmup}
    for k, ms in res.items():
        line[k] = {"ms": ms, "rows_per_s": rows / ms * 1e3, "GBps": nbytes / ms / 1e6}
    line["value"] = line["batched_graph"]["rows_per_s"]
    h.close()
    del Xs, outs
    torch.cuda.empty_cache()
    if not quiet:
        print(json.dumps(line), flush=True)
    return line


def run_stream(args, quiet=False):
    """Flow-cytometry-shaped stream (1.6e9 x 25, r = 8, log-normal W,
    Dirichlet(0.5), sigma = 1e-2), or with --workload kron_fc_1p6e9x25 the
    Kronecker-structured A kron A (A: 40,000 x 5, r_A = 4, so r = 16): 64M-row
    chunks drawn on the device one at a time and pushed through
    mrnmf_stream_push (X is never resident whole).  GB/s counts the chunk reads
    of the pass; generation is timed apart."""
    import torch

    from paper_1402_6964_gb300 import build, mrnmf, synth

    build.build()
    kron = args.workload == "kron_fc_1p6e9x25"
    w = synth.WORKLOADS["kron_fc_1p6e9x25" if kron else "fc_stream_1p6e9x25"]
    m = args.rows or w.m
    chunk = min(64 << 20, m)
    if kron:
        A64, Kp = synth.kron_factor(w)
        A = torch.from_numpy(A64.astype(np.float32)).cuda()
        P = None
    else:
        P = synth.planted_structure(w.n, w.r, w.seed, w.alpha)
        Kp = P.K
    buf = torch.empty((chunk, w.n), dtype=torch.float32, device="cuda")
    h = mrnmf.Handle()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    gen_ms, push_ms = 0.0, 0.0
    nchunks = (m + chunk - 1) // chunk
    h.stream_begin(w.n, k=w.k, seed=w.seed)
    for c in range(nchunks):
        rows = min(chunk, m - c * chunk)
        a, b, d = ev(), ev(), ev()
        a.record()
        if kron:
            X = synth.kron_rows(A, c * chunk, rows, out=buf[:rows])
        else:
            X, _ = synth.device_planted(rows, w.n, w.r, w.seed, noise=w.noise, alpha=w.alpha, w_dist=w.w_dist,
                                        chunk=c, P=P, out=buf[:rows])
        b.record()
        h.stream_push(X)
        d.record()
        torch.cuda.synchronize()
        gen_ms += a.elapsed_time(b)
        push_ms += b.elapsed_time(d)
    e0, e1 = ev(), ev()
    e0.record()
    R, cs, GX = h.stream_end(w.n, k=w.k)
    K, gap = h.select_extreme("spa", R=R, colsum=cs, r=w.r)
    H = h.nnls_h(R, K)
    out = h.residual(R, K, H)
    e1.record()
    torch.cuda.synchronize()
    h.sync()
    end_ms = e0.elapsed_time(e1)
    nbytes = 4.0 * m * w.n
    hbm, _, src = _peaks()
    gbs = nbytes / (push_ms + end_ms) / 1e6
    line = {"mode": "stream", "metric": "streamed TSQR pass GB/s of X (chunk reads)", "value": gbs,
            "unit": "GB/s", "ms_pass": push_ms + end_ms, "ms_generation": gen_ms, "chunks": nchunks,
            "chunk_rows": chunk, "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm,
                                              "unit": "GB/s", "frac": gbs / hbm, "peak_source": src},
            "K_spa": sorted(K.cpu().numpy().tolist()), "K_planted": Kp.tolist(),
            "residual_rel": float(out[1].item()),
            "config": {"workload": w.name, "m": m, "n": w.n, "r": w.r, "k": w.k}}
    h.close()
    del buf
    torch.cuda.empty_cache()
    if not quiet:
        print(json.dumps(line), flush=True)
    return line


def tc_form_available(n: int, k: int) -> bool:
    """The tensor-core pass (TF32X3 or TF32) exists for this shape (the library's rule)."""
    return 16 < n <= 256 and k <= (32 if n <= 64 else 48)


def run_illcond_forms(args, quiet=False):
    """The 1e8 x 200 ill-conditioned workload (80 GB, drawn on the device):
    the fused pass (R, column sums, GX with k = 40) in each arithmetic form,
    with each form's R error by the Gram identity (binary64 X'X accumulated on
    the device)."""
    import torch

    from paper_1402_6964_gb300 import build, mrnmf, synth

    build.build()
    w = synth.WORKLOADS["illcond_1e8x200"]
    m = args.rows or w.m
    P = synth.planted_structure(w.n, w.r, w.seed, w.alpha, w.decades)
    Xd = torch.empty((m, w.n), dtype=torch.float32, device="cuda")
    ch = 1 << 23
    for c0 in range(0, m, ch):
        rows = min(ch, m - c0)
        synth.device_planted(rows, w.n, w.r, w.seed, noise=w.noise, alpha=w.alpha, w_dist=w.w_dist,
                             chunk=c0 // ch, P=P, out=Xd[c0:c0 + rows])
    torch.cuda.synchronize()
    Gd = torch.zeros((w.n, w.n), dtype=torch.float64, device="cuda")
    for c0 in range(0, m, 1 << 21):
        Xc = Xd[c0:c0 + (1 << 21)].double()
        Gd += Xc.T @ Xc
        del Xc
    Gram = Gd.cpu().numpy()
    del Gd
    h = mrnmf.Handle()
    n, k = w.n, w.k
    R = torch.empty((n, n), dtype=torch.float64, device="cuda")
    cs = torch.empty(n, dtype=torch.float64, device="cuda")
    GX = torch.empty((k, n), dtype=torch.float64, device="cuda")
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0.record()
    l1.record()
    forms = {}
    nbytes = 4.0 * m * n
    for form in ("fp32", "tf32x3", "tf32"):
        if form != "fp32" and not tc_form_available(n, k):
            continue
        h.tsqr_gp(Xd, k, w.seed, prec=form, out=(R, cs, GX))  # warm-up
        h.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        h.profile_events(l0, l1)
        leaf = 0.0
        a.record()
        for _ in range(reps):
            h.tsqr_gp(Xd, k, w.seed, prec=form, out=(R, cs, GX))
        b.record()
        torch.cuda.synchronize()
        leaf = l0.elapsed_time(l1)
        h.profile_events(None, None)
        h.sync()
        ms = a.elapsed_time(b) / reps
        Rh = R.cpu().numpy()
        forms[form] = {"pass_ms": ms, "GBps": nbytes / ms / 1e6, "leaf_ms": leaf,
                       "r_error_gram_identity": float(np.linalg.norm(Rh.T @ Rh - Gram) / np.linalg.norm(Gram))}
    h.close()
    del Xd, R, cs, GX
    torch.cuda.empty_cache()
    line = {"mode": "illcond", "workload": w.name, "m": m, "n": n, "k": k, "forms": forms}
    if "tf32x3" in forms:
        line["mixed_over_fp32"] = forms["fp32"]["pass_ms"] / forms["tf32x3"]["pass_ms"]
    if "tf32" in forms:
        line["tf32_over_fp32"] = forms["fp32"]["pass_ms"] / forms["tf32"]["pass_ms"]
    if not quiet:
        print(json.dumps(line), flush=True)
    return line


def per_n_sweep(sms: int, mhz: float, hbm: float):
    """The plain FP32 pass (k = 0, the metric's TSQR pass) at n = 4 .. 64 on
    about 2 GB of uniform X drawn on the device: leaf time from the library's
    events, GB/s, and the fraction of the HBM roofline and of the binary32
    SIMT peak (2 n^2 flops per row)."""
    import torch

    from paper_1402_6964_gb300 import mrnmf
    h = mrnmf.Handle()
    out = {}
    peak = _fp32_simt_peak_tflops(sms, mhz)
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0.record()
    l1.record()
    for n in (4, 8, 12, 16, 25, 32, 50, 64):
        m = int(5e8 // n)
        X = torch.rand(m, n, device="cuda")
        for _ in range(3):
            h.tsqr_r(X, prec="fp32")
        h.sync()
        h.profile_events(l0, l1)
        reps, leaf = 5, 0.0
        for _ in range(reps):
            h.tsqr_r(X, prec="fp32")
            torch.cuda.synchronize()
            leaf += l0.elapsed_time(l1)
        h.profile_events(None, None)
        h.sync()
        ms = leaf / reps
        gbs = 4.0 * m * n / ms / 1e6
        tf = 2.0 * m * n * n / ms / 1e9
        out[str(n)] = {"m": m, "leaf_ms": ms, "GBps": gbs, "hbm_frac": gbs / hbm, "tflops": tf,
                       "simt_frac": tf / peak}
        del X
    h.close()
    torch.cuda.empty_cache()
    return out


def host_link():
    """Pinned host -> device copy bandwidth (GB/s) at a few transfer sizes."""
    import torch
    out = {}
    for mb in (64, 256, 1024):
        hsrc = torch.empty(mb << 18, dtype=torch.float32).pin_memory()
        d = torch.empty(mb << 18, dtype=torch.float32, device="cuda")
        d.copy_(hsrc, non_blocking=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(5):
            d.copy_(hsrc, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        out[f"{mb}MiB"] = 5 * (mb << 20) / a.elapsed_time(b) / 1e6
        del hsrc, d
    return out


def host_cpu_info():
    """Core count and model of the host the oracle runs on (nproc, lscpu)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def _oracle_chunk_worker(job):
    """One host core's share of the all-cores baseline: the oracle's whole
    path on rows chunk*CHUNK .. of the workload (drawn here, untimed)."""
    wname, chunk, rows = job
    sys.path.insert(0, ROOT)
    from paper_1402_6964_gb300 import synth
    w = synth.WORKLOADS[wname]
    P = synth.planted_structure(w.n, w.r, w.seed, w.alpha, w.decades)
    X = synth.rows_chunk(P, w.seed, chunk, rows, w.noise, w.w_dist)
    return cpu_oracle_step(X, w, rows)


def cpu_baseline_all_cores(wname: str, rows: int, cores: int):
    """The oracle as it stands on every host core at once: `cores` spawned
    processes, each running the whole path on its own `rows`-row chunk of the
    workload; GB/s = all rows / wall time of the slowest."""
    import multiprocessing as mp
    from paper_1402_6964_gb300 import synth
    w = synth.WORKLOADS[wname]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_chunk_worker, [(wname, c, 2000) for c in range(cores)])  # start-up, page-in
        t0 = time.perf_counter()
        secs = pool.map(_oracle_chunk_worker, [(wname, c, rows) for c in range(cores)])
        wall = time.perf_counter() - t0
    return {"value": 4.0 * rows * w.n * cores / wall / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each the whole path on its own {rows}-row chunk of the workload; "
                      f"wall {wall:.1f} s (slowest process {max(secs):.1f} s)"}


def time_over_ranks(t_local: float, world: int, device=None) -> float:
    """The job's time: the slowest rank's timed region (max over ranks)."""
    if world <= 1:
        return t_local
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_gbs(bytes_per_step_per_rank: float, steps: int, world: int, t_max: float) -> float:
    """Whole-job throughput: every rank (replica) reads its own X each step."""
    return bytes_per_step_per_rank * steps * world / t_max / 1e9


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1402_6964_gb300 import build, mrnmf, synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    w = synth.WORKLOADS[args.workload]
    m_req = args.rows or w.m
    big = m_req * w.n * 4 > 16e9  # too large to draw on the host: draw it on the device
    if big:
        P = synth.planted_structure(w.n, w.r, w.seed, w.alpha, w.decades)
        Xd = torch.empty((m_req, w.n), dtype=torch.float32, device="cuda")
        ch = 1 << 23
        for c0 in range(0, m_req, ch):
            rows = min(ch, m_req - c0)
            synth.device_planted(rows, w.n, w.r, w.seed, noise=w.noise, alpha=w.alpha, w_dist=w.w_dist,
                                 chunk=c0 // ch, P=P, out=Xd[c0:c0 + rows])
        torch.cuda.synchronize()
        X = None
    else:
        X, P = synth.workload_matrix(w, m=args.rows)
        Xd = torch.from_numpy(X).cuda()
    m, n, r, k = Xd.shape[0], w.n, w.r, w.k
    dev = Xd.device
    h = mrnmf.Handle()
    stream = torch.cuda.current_stream()
    # Two sets of step outputs (R, column sums, GX, and each selection's K, H
    # and residual): step i writes set i mod 2.
    sets = []
    for _ in range(2):
        Ks = {mth: (torch.empty(r, dtype=torch.int32, device=dev), torch.empty(r, dtype=torch.float64, device=dev))
              for mth in ("spa", "xray", "gp")}
        sets.append({"R": torch.empty((n, n), dtype=torch.float64, device=dev),
                     "cs": torch.empty(n, dtype=torch.float64, device=dev),
                     "GX": torch.empty((k, n), dtype=torch.float64, device=dev), "Ks": Ks,
                     "Hs": {mth: torch.empty((r, n), dtype=torch.float64, device=dev) for mth in Ks},
                     "outs": {mth: torch.empty(2, dtype=torch.float64, device=dev) for mth in Ks}})

    # The three selections (and their NNLS and residual) depend only on R,
    # the column sums and GX: each runs on its own CUDA stream with its own
    # handle (a handle's small-step workspace serves one stream at a time),
    # forked from the stream `on` and joined back to it.
    side = {mth: (torch.cuda.Stream(device=dev), mrnmf.Handle()) for mth in ("spa", "xray", "gp")}
    ev_fork = torch.cuda.Event()
    ev_side = {mth: torch.cuda.Event() for mth in side}

    def selections(on, b):
        st = sets[b]
        ev_fork.record(on)
        for mth in ("xray", "spa", "gp"):
            s, hm = side[mth]
            s.wait_event(ev_fork)
            hm.select_extreme(mth, R=st["R"], colsum=st["cs"], GX=st["GX"] if mth == "gp" else None, r=r,
                              out=st["Ks"][mth], stream=s)
            hm.nnls_h(st["R"], st["Ks"][mth][0], out=st["Hs"][mth], stream=s)
            hm.residual(st["R"], st["Ks"][mth][0], st["Hs"][mth], out=st["outs"][mth], stream=s)
            ev_side[mth].record(s)
        for mth in ("xray", "spa", "gp"):
            on.wait_event(ev_side[mth])

    # Overlap (default): the selections of step i run on their own stream
    # while the pass of step i+1 runs; the pass of step i+2, which rewrites
    # set i mod 2, waits for them.  Every step still does all of its work.
    chain = torch.cuda.Stream(device=dev)
    ev_pass = [torch.cuda.Event(), torch.cuda.Event()]
    ev_chain = [torch.cuda.Event(), torch.cuda.Event()]
    graphs = [None, None]
    graph_launches = 0
    mode = {"overlap": not args.no_overlap}
    counter = [0]

    def step():
        b = counter[0] & 1
        counter[0] += 1
        st = sets[b]
        if mode["overlap"]:
            stream.wait_event(ev_chain[b])  # the selections of step i-2 read this set
        # the pass runs eagerly (its leaf kernel is timed by events around it);
        # the selection chains replay as one CUDA graph once captured
        h.tsqr_gp(Xd, k, w.seed, prec=args.prec, out=(st["R"], st["cs"], st["GX"]))
        on = stream
        if mode["overlap"]:
            ev_pass[b].record(stream)
            chain.wait_event(ev_pass[b])
            on = chain
        if graphs[b] is not None:
            with torch.cuda.stream(on):
                graphs[b].replay()
        else:
            selections(on, b)
        if mode["overlap"]:
            ev_chain[b].record(chain)

    def drain():
        stream.wait_stream(chain)

    for _ in range(max(args.warmup, 2)):
        step()
    drain()
    h.sync()
    for _, hm in side.values():
        hm.sync()
    if not args.eager:
        # every buffer and workspace is in place after the warm-up, so the
        # chains capture without allocations; graph b reads set b's R, column
        # sums and GX on every replay
        for b in range(2):
            cap = torch.cuda.Stream(device=dev)
            cap.wait_stream(stream)
            g = torch.cuda.CUDAGraph()
            l0 = mrnmf.kernel_launches()
            with torch.cuda.graph(g, stream=cap):
                selections(cap, b)
            graph_launches = mrnmf.kernel_launches() - l0
            stream.wait_stream(cap)
            graphs[b] = g
        torch.cuda.synchronize()
        for _ in range(2):
            step()
        drain()
        h.sync()
        for _, hm in side.values():
            hm.sync()

    leaf_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in leaf_ev:  # torch creates the CUDA event on first record; the library re-records it
        a.record(stream)
        b.record(stream)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = mrnmf.kernel_launches()
    clocks.begin()
    t_wall0 = time.perf_counter()
    step_ev[0].record(stream)
    for i in range(args.steps):
        h.profile_events(*leaf_ev[i])
        step()
        if i + 1 == args.steps:
            drain()  # the last step's selections end inside the timed region
        step_ev[i + 1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = mrnmf.kernel_launches() - launches0 + graph_launches * args.steps
    h.profile_events(None, None)
    h.sync()
    for _, hm in side.values():
        hm.sync()
    last = sets[(counter[0] - 1) & 1]
    R, Ks = last["R"], last["Ks"]
    t_dev = step_ev[0].elapsed_time(step_ev[-1]) / 1e3  # seconds
    # the same steps without the overlap, for the record
    seq_ms = None
    if mode["overlap"]:
        mode["overlap"] = False
        nseq = max(3, min(args.steps, 20))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(nseq):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms = e0.elapsed_time(e1) / nseq
        h.sync()
        mode["overlap"] = True
    leaf_ms = [a.elapsed_time(b) for a, b in leaf_ev]
    t_max = time_over_ranks(t_dev, world, dev)

    bytes_step = 4.0 * m * n
    value = job_gbs(bytes_step, args.steps, world, t_max)
    hbm, mhz, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    leaf_s = statistics.mean(leaf_ms) / 1e3
    leaf_gbs = bytes_step / leaf_s / 1e9
    # the leaf's algorithmic work: 2n^2 flops of Householder per row plus the
    # fused projection's 2kn (G'X accumulated in the same kernel)
    flops = 2.0 * m * n * n + 2.0 * m * n * k
    simt_peak = _fp32_simt_peak_tflops(sms, mhz)
    leaf_tflops = flops / leaf_s / 1e12
    # DRAM bytes of one leaf launch from the ncu capture recorded in
    # profiles/leaf_traffic.json (a smaller case of the same kernel, scaled by
    # rows); null once the kernel's source has changed since the capture
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "leaf_traffic.json")
    if os.path.exists(tfile):
        try:
            import hashlib
            td = json.load(open(tfile))
            src = open(os.path.join(ROOT, td["source"]), "rb").read()
            if (hashlib.sha256(src).hexdigest() == td["source_sha256"] and td["n"] == n and td["k"] == k
                    and args.prec != "tf32x3"):
                traffic = td["bytes_per_row"] * m
        except Exception:
            traffic = None
    roof_hbm = {"bound": "hbm", "achieved": leaf_gbs, "peak": hbm, "unit": "GB/s", "frac": leaf_gbs / hbm,
                "traffic": traffic, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"}
    roof_alu = {"bound": "alu", "achieved": leaf_tflops, "peak": simt_peak, "unit": "TFLOP/s",
                "frac": leaf_tflops / simt_peak, "traffic": traffic, "flops_per_row": 2 * n * n + 2 * n * k,
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"}
    roofline = roof_hbm if roof_hbm["frac"] >= roof_alu["frac"] else roof_alu

    # R error of this pass vs the unique R (Cholesky of the binary64 Gram X'X,
    # accumulated in row chunks on the device for device-drawn X)
    Rg = R.cpu().numpy()
    if big:
        Gd = torch.zeros((n, n), dtype=torch.float64, device=dev)
        for c0 in range(0, m, 1 << 20):
            Xc = Xd[c0:c0 + (1 << 20)].double()
            Gd += Xc.T @ Xc
            del Xc
        Gram = Gd.cpu().numpy()
        del Gd
    else:
        G = X.astype(np.float64)
        Gram = G.T @ G
        del G
    r_err = {"gram_identity": float(np.linalg.norm(Rg.T @ Rg - Gram) / np.linalg.norm(Gram))}
    # chol(X'X)' is a usable reference only while cond(X'X) is far below
    # 1/eps(binary64); beyond that (the ill-conditioned workload) the Gram
    # identity alone is reported
    cond_gram = float(np.linalg.cond(Gram))
    r_err["cond_gram"] = cond_gram
    if cond_gram < 1e10:
        try:
            Rc = np.linalg.cholesky(Gram).T
            r_err["rel_fro_vs_chol_gram"] = float(np.linalg.norm(Rg - Rc) / np.linalg.norm(Rc))
        except np.linalg.LinAlgError:
            pass
    K_spa = sorted(Ks["spa"][0].cpu().numpy().tolist())

    # ---- the pass alone in each arithmetic form available for this n (the
    # metric's "mixed vs FP32 at stated R error"), same resident X
    forms = {}
    for form in ("fp32", "tf32x3", "tf32"):
        if form != "fp32" and not tc_form_available(n, k):
            continue
        Rf = torch.empty((n, n), dtype=torch.float64, device=dev)
        csf = torch.empty(n, dtype=torch.float64, device=dev)
        GXf = torch.empty((k, n), dtype=torch.float64, device=dev)
        h.tsqr_gp(Xd, k, w.seed, prec=form, out=(Rf, csf, GXf))
        h.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            h.tsqr_gp(Xd, k, w.seed, prec=form, out=(Rf, csf, GXf))
        e1.record(stream)
        h.sync()
        ms = e0.elapsed_time(e1) / reps
        Rh = Rf.cpu().numpy()
        forms[form] = {"pass_ms": ms, "GBps": bytes_step / ms / 1e6,
                       "r_error_gram_identity": float(np.linalg.norm(Rh.T @ Rh - Gram) / np.linalg.norm(Gram))}

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e and not big:
        Xp = torch.from_numpy(X).pin_memory()
        h.factorize_host(Xp, r, method="spa", k=0, seed=w.seed, prec=args.prec)  # warm-up
        ne = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(ne):
            h.factorize_host(Xp, r, method="spa", k=0, seed=w.seed, prec=args.prec)
        te = (time.perf_counter() - t0) / ne
        e2e = {"value": bytes_step / te / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(bytes_step),
               "d2h_bytes_per_step": int(4 * r + 8 * r * n + 16), "ms_per_step": te * 1e3,
               "call": "mrnmf_factorize_host (SPA, H, residual)"}
        del Xp
        try:
            e2e["host_link_h2d_GBps"] = host_link()
        except Exception as ex:
            e2e["host_link_h2d_GBps"] = {"error": str(ex)[:200]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rows = args.cpu_rows
        Xh = X if X is not None else Xd[:rows].cpu().numpy()
        tcpu = cpu_oracle_step(Xh, w, rows)
        one = {"value": 4.0 * rows * n / tcpu / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {rows} rows of the workload (pass + SPA/XRAY/GP + NNLS + residual), "
                         f"{tcpu:.1f} s"}
        ncores, model = host_cpu_info()
        cpu = one
        if ncores > 1:
            try:
                cpu = cpu_baseline_all_cores(args.workload, args.cpu_rows_per_core, ncores)
                cpu["single_core"] = one
            except Exception as ex:  # the one-core figure stands alone
                one["all_cores_error"] = str(ex)[:200]
        cpu["nproc"] = ncores
        cpu["cpu_model"] = model

    # ---- the other workloads of the metric, measured after the main one
    other = None
    if rank == 0 and world == 1 and not args.no_other and args.rows is None:
        del Xd
        torch.cuda.empty_cache()
        other = {}
        try:
            other["per_n_fp32_pass"] = per_n_sweep(sms, mhz, hbm)
        except Exception as ex:
            other["per_n_fp32_pass"] = {"error": str(ex)[:300]}
        # the projection-only pass (GP alone) on the benchmarked workload, in the
        # default SIMT form and the tcgen05 BF16 form
        for form in ("simt", "bf16"):
            try:
                sub = argparse.Namespace(**vars(args))
                sub.rows, sub.steps, sub.warmup, sub.gp_form = None, 10, 3, form
                other[f"gp_projection_{form}"] = run_gp_pass(sub, quiet=True)
            except Exception as ex:
                other[f"gp_projection_{form}"] = {"error": str(ex)[:300]}
        for name, fn in (("illcond_1e8x200_forms", run_illcond_forms), ("fc_stream_1p6e9x25", run_stream),
                         ("batch_256", run_batched)):
            try:
                sub = argparse.Namespace(**vars(args))
                sub.rows, sub.steps, sub.warmup = None, 3, 3
                sub.workload = "fc_stream_1p6e9x25"
                other[name] = fn(sub, quiet=True)
            except Exception as ex:
                other[name] = {"error": str(ex)[:300]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "m": m, "n": n, "r": r, "k": k, "prec": args.prec,
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "selections": ("eager" if graphs[0] is None else "CUDA graph") + ", three streams, "
                           + ("overlapping the next step's pass (double-buffered outputs)" if not args.no_overlap
                              else "after the pass"),
                           "l2": f"input ({bytes_step / 1e9:.2f} GB) larger than L2 (129 MB); no flush needed",
                           "tune_file": os.path.relpath(os.environ["MRNMF_TUNE_FILE"], ROOT)
                           if os.environ.get("MRNMF_TUNE_FILE") else None},
                "roofline": roofline, "roofline_other": roof_alu if roofline is roof_hbm else roof_hbm,
                "leaf_ms": statistics.mean(leaf_ms), "sequential_ms_per_step": seq_ms, "r_error": r_err,
                "K_spa": K_spa, "K_planted": P.K.tolist(), "forms": forms,
                "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "cpu_baseline": cpu,
                "wall_s_timed": t_wall, "other_configs": other}
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


TUNE_FILE = os.path.join(ROOT, "paper_1402_6964_gb300", "tune_gb300.txt")


def main():
    # the library reads its tuning table from MRNMF_TUNE_FILE on first use;
    # the committed table (paper_1402_6964_gb300/tune.py wrote it) is the default
    if "MRNMF_TUNE_FILE" not in os.environ and os.path.exists(TUNE_FILE):
        os.environ["MRNMF_TUNE_FILE"] = TUNE_FILE
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["step", "gp", "pass", "batched", "stream", "illcond"], default="step",
                    help="step: the whole hot path (default); gp: the projection-only pass; "
                         "pass: the plain FP32 TSQR pass on uniform X of --rows x --cols; "
                         "batched: 256 independent problems; stream: 1.6e9 x 25 in 64M-row chunks; "
                         "illcond: the 1e8 x 200 workload in each arithmetic form")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--prec", choices=["auto", "fp32", "tf32x3", "tf32"], default="auto")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--rows", type=int, default=None, help="first ROWS rows only (profiling a smaller case)")
    ap.add_argument("--cols", type=int, default=8, help="columns of X in --mode pass")
    ap.add_argument("--gp-form", choices=["simt", "tf32x3", "bf16"], default="simt",
                    help="--mode gp: the SIMT projection, or mrnmf_gauss_project_tc in a tensor-core form")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--eager", action="store_true", help="launch the selection chains eagerly (no CUDA graph)")
    ap.add_argument("--no-overlap", action="store_true",
                    help="run each step's selections after its pass, before the next pass starts")
    ap.add_argument("--cpu-rows", type=int, default=1_000_000)
    ap.add_argument("--cpu-rows-per-core", type=int, default=500_000,
                    help="rows per process of the all-cores oracle baseline")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the 1e8 x 200 forms, the 1.6e9 x 25 stream and the 256-problem batch")
    ap.add_argument("--ref-rows", type=int, default=250_000, help="rows per process and step of --impl reference")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "gp":
        run_gp_pass(args)
    elif args.mode == "pass":
        run_pass(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "stream":
        run_stream(args)
    elif args.mode == "illcond":
        run_illcond_forms(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
