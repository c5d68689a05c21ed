"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in a copy of the oracle's C source (a
dropped term, a wrong sign, a transposed or wrong index, a skipped step),
builds it with gcc into a temporary directory, routes the oracle's wrappers to
that build, and requires that at least one pin fails.  The unmodified source,
built the same way, must pass every pin.  The pins are the facts of
test_oracle_pins.py (hand-worked fixtures, exact integer arithmetic, closed
forms, library routines of a different algorithm, brute force), restated here
as checks that return False instead of raising.
"""
import os
import subprocess

import numpy as np
import pytest

from paper_1402_6964_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
SRC = os.path.join(os.path.dirname(HERE), "oracle", "mrnmf_oracle.c")


def _read(name):
    cases = [{}]
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line == "---":
            cases.append({})
            continue
        tag, *vals = line.split()
        cases[-1].setdefault(tag, []).append([float(v) for v in vals])
    return cases


# ------------------------------------------------------------------ the pins

def pin_qr_gram(orc):
    X = synth.random_nonneg(300, 9, seed=11, dtype=np.float64, integer=True)
    R = orc.qr_r(X)
    G = (X.astype(np.int64).T @ X.astype(np.int64)).astype(np.float64)
    return np.allclose(R.T @ R, G, rtol=1e-13, atol=1e-10) and np.all(np.tril(R, -1) == 0)


def pin_qr_cholesky(orc):
    X = synth.random_nonneg(500, 12, seed=12, dtype=np.float64)
    return np.allclose(orc.qr_r(X), np.linalg.cholesky(X.T @ X).T, rtol=1e-10, atol=1e-10)


def pin_colsum_exact(orc):
    X = synth.random_nonneg(1000, 6, seed=17, dtype=np.float64, integer=True)
    return np.array_equal(orc.colsum(X), X.astype(np.int64).sum(0).astype(np.float64))


def pin_philox_kat(orc):
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        if [int(x) for x in orc.philox4x32_10(v[0:4], v[4:6])] != v[6:10]:
            return False
    return True


def pin_gauss_moments(orc):
    z = orc.gauss_matrix(seed=99, row0=0, rows=50000, k=8).ravel()
    return abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01


def pin_gx_matmul(orc):
    X = synth.random_nonneg(700, 9, seed=18, dtype=np.float64)
    G = orc.gauss_matrix(7, 100, 700, 6)
    return np.allclose(orc.gauss_project(X, 6, 7, row0=100), G.T @ X, rtol=1e-12, atol=1e-12)


def _brute_nnls(A, b):
    r = A.shape[1]
    best, bx = np.inf, None
    for mask in range(1 << r):
        S = [i for i in range(r) if mask >> i & 1]
        y = np.zeros(r)
        if S:
            ys, *_ = np.linalg.lstsq(A[:, S], b, rcond=None)
            if np.any(ys < 0):
                continue
            y[S] = ys
        res = np.sum((A @ y - b) ** 2)
        if bx is None or res < best - 1e-15 * max(1.0, best):
            best, bx = res, y
    return bx


def pin_nnls_brute(orc):
    for seed in range(6):
        g = np.random.default_rng(100 + seed)
        A = g.standard_normal((15, 7))
        b = g.standard_normal(15)
        x, st = orc.nnls(A.T @ A, A.T @ b, b @ b)
        if st != 0 or not np.allclose(x, _brute_nnls(A, b), rtol=1e-9, atol=1e-11):
            return False
    return True


def pin_nnls_scipy(orc):
    from scipy.optimize import nnls as sp_nnls
    for seed in range(4):
        g = np.random.default_rng(200 + seed)
        A = g.standard_normal((60, 24))
        b = g.standard_normal(60)
        x, st = orc.nnls(A.T @ A, A.T @ b, b @ b)
        if st != 0 or not np.allclose(x, sp_nnls(A, b)[0], rtol=1e-8, atol=1e-10):
            return False
    return True


def pin_spa_hand(orc):
    c = _read("spa_hand.txt")[0]
    X = np.array(c["X"])
    K, gap = orc.spa(X, X.sum(0), 2)
    return list(K) == [int(v) for v in c["K"][0]] and np.allclose(gap, c["GAP"][0], rtol=1e-12)


def pin_xray_hand(orc):
    c = _read("xray_hand.txt")[0]
    X = np.array(c["X"])
    K, gap, st = orc.xray(X, 2)
    return st == 0 and list(K) == [int(v) for v in c["K"][0]]


def pin_xray_first_pick(orc):
    X, P = synth.planted_separable(900, 15, 5, seed=27, noise=1e-3, dtype=np.float64)
    G = X.T @ X
    scores = np.linalg.norm(G, axis=0) / np.sqrt(np.diag(G))
    K, gap, st = orc.xray(orc.qr_r(X), 3)
    return K[0] == int(np.argmax(scores))


def pin_xray_scores(orc):
    from scipy.optimize import nnls as sp_nnls
    X, P = synth.planted_separable(400, 12, 5, seed=40, noise=1e-2, dtype=np.float64)
    K, gap, st = orc.xray(X, 5)
    chosen, Res = [], X.copy()
    for t in range(5):
        scores = np.linalg.norm(Res.T @ X, axis=0) / np.linalg.norm(X, axis=0)
        scores[chosen] = -np.inf
        order = np.argsort(-scores, kind="stable")
        if (scores[order[0]] - scores[order[1]]) / scores[order[0]] > 1e-9 and K[t] != order[0]:
            return False
        chosen.append(int(K[t]))
        A = X[:, chosen]
        Res = X - A @ np.stack([sp_nnls(A, X[:, c])[0] for c in range(X.shape[1])], axis=1)
    return st == 0


def pin_residual_full(orc):
    X, P = synth.planted_separable(2500, 16, 5, seed=32, noise=1e-2, dtype=np.float64)
    R = orc.qr_r(X)
    H, _ = orc.nnls_h(R, P.K)
    full = np.linalg.norm(X - X[:, P.K] @ H)
    ab, rel = orc.residual(R, P.K, H)
    return np.isclose(ab, full, rtol=1e-9) and np.isclose(rel, full ** 2 / np.linalg.norm(X) ** 2, rtol=1e-9)


def pin_gp_hand(orc):
    c = _read("gp_hand.txt")[0]
    K, cand, gap = orc.gp_select(np.array(c["GX"]), np.array(c["S"][0]), 4)
    return list(cand) == [int(v) for v in c["CAND"][0]]


def pin_r_svd(orc):
    X = synth.random_nonneg(400, 12, seed=41, dtype=np.float64)
    R = orc.qr_r(X)
    sig, S, st = orc.r_svd(R)
    sl = np.linalg.svd(R, compute_uv=False)
    G = R.T @ R
    return (st == 0 and np.allclose(sig, sl, rtol=0, atol=1e-12 * sl[0])
            and np.linalg.norm(S.T @ S - G) <= 1e-12 * np.linalg.norm(G))


PINS = [pin_qr_gram, pin_qr_cholesky, pin_colsum_exact, pin_philox_kat, pin_gauss_moments, pin_gx_matmul,
        pin_nnls_brute, pin_nnls_scipy, pin_spa_hand, pin_xray_hand, pin_xray_first_pick, pin_xray_scores, pin_residual_full, pin_gp_hand,
        pin_r_svd]

# ---------------------------------------------------------------- the mistakes

MUTANTS = {
    "qr: pivot-row term dropped from the reflector's dot": (
        "double s = v0 * y[j];", "double s = 0.0;"),
    "qr: factor 2 of the reflector dropped": (
        "double f = 2.0 * s / vtv;", "double f = s / vtv;"),
    "qr: diagonal sign normalisation skipped": (
        "if (R[i * n + i] < 0.0)", "if (0)"),
    "colsum: sign of the compensation": (
        "comp = (t - sum) - y;", "comp = (t - sum) + y;"),
    "philox: a round multiplier": (
        "(uint64_t)0xD2511F53u * (uint64_t)c0", "(uint64_t)0xD2511F55u * (uint64_t)c0"),
    "gauss: Box-Muller radius without the factor 2": (
        "double rho = sqrt(-2.0 * log(u1));", "double rho = sqrt(-log(u1));"),
    "GX: transposed accumulation": (
        "GX[(int64_t)l * n + j] += g[l] * X[i * ldx + j];", "GX[(int64_t)j * k + l] += g[l] * X[i * ldx + j];"),
    "nnls: sign of the dual": (
        "for (int j = 0; j < r; ++j) s -= AtA[i * r + j] * x[j];",
        "for (int j = 0; j < r; ++j) s += AtA[i * r + j] * x[j];"),
    "spa: projection step skipped": (
        "for (int j = 0; j < n; ++j) Y[(int64_t)i * n + j] -= cj[j] * u[i];",
        "for (int j = 0; j < n; ++j) Y[(int64_t)i * n + j] -= 0.0 * cj[j] * u[i];"),
    "spa: l1 column scaling dropped": (
        "Y[(int64_t)i * n + j] = Y0[(int64_t)i * n + j] / colsum[j];",
        "Y[(int64_t)i * n + j] = Y0[(int64_t)i * n + j];"),
    "xray: score not divided by the column norm": (
        "score[j] = cn[j] > 0.0 ? sqrt(s) / cn[j] : 0.0;", "score[j] = sqrt(s);"),
    "xray: residual not refreshed after a pick": (
        "Res[(int64_t)i * n + c] = s;", "Res[(int64_t)i * n + c] = Y0[(int64_t)i * n + c];"),
    "xray: newest pick left out of the residual": (
        "for (int a = 0; a <= t; ++a) s -= Y0[(int64_t)i * n + K[a]] * H[(int64_t)a * n + c];",
        "for (int a = 0; a < t; ++a) s -= Y0[(int64_t)i * n + K[a]] * H[(int64_t)a * n + c];"),
    "residual: wrong term in the denominator": (
        "r2 += v * v;", "r2 += s * s;"),
    "r-svd: rotation sign flipped": (
        "B[(size_t)k * n + i] = c * bi - sn * bj;", "B[(size_t)k * n + i] = c * bi + sn * bj;"),
    "r-svd: rotation angle from the wrong difference": (
        "const double zeta = (b - a) / (2.0 * g);", "const double zeta = (a - b) / (2.0 * g);"),
    "gp: min before max": (
        "int picks[2] = {jmax, jmin};", "int picks[2] = {jmin, jmax};"),
}


def _build(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    lib = tmp_path / f"{name}.so"
    src.write_text(text)
    subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                    "-o", str(lib), str(src), "-lm"], check=True)
    return str(lib)


def _results(oracle, lib):
    out = {}
    with oracle.substituted(lib):
        for pin in PINS:
            try:
                out[pin.__name__] = bool(pin(oracle))
            except (RuntimeError, np.linalg.LinAlgError):
                out[pin.__name__] = False
    return out


def test_unmodified_source_passes_every_pin(oracle, tmp_path):
    res = _results(oracle, _build(tmp_path, "orig", open(SRC).read()))
    assert all(res.values()), res


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(oracle, tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {old}"
    lib = _build(tmp_path, "mutant", text.replace(old, new))
    res = _results(oracle, lib)
    assert not all(res.values()), f"{name}: no pin failed"
