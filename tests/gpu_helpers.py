"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare by the acceptance rules.

Acceptance (6-bit min-sum): decisions, update counts, final LLRs and the full
edge-selection trace bit-exact.  FP32 sum-product: per-value |d| <= 1e-4
max(1, |m|) against FP64; dynamic-schedule traces identical up to the first
step whose oracle top-2 metric gap (relative to max(1, |metric|)) is below
1e-5; FER inside the oracle's 95% Clopper-Pearson interval on the same frames.
"""
from __future__ import annotations

import math
import os

import numpy as np

import oracle
import paper_2102_11089_gb300 as L
from paper_2102_11089_gb300 import workloads as wl

TOL_REL = 1e-4
NEAR_TIE = 1e-5
THREADS = max(1, os.cpu_count() or 1)

_codes = {}


class Spec(tuple):
    """(check_idx, var_idx, M, N, K, punct) of a test code.  Codes lifted from a
    protograph also carry the protograph (`base`, `Z`, `punct_cols`): the
    library builds them through ldpc_code_build_qc, whose protograph view is
    what the decode kernels of the benchmark read."""
    base = None
    Z = None
    punct_cols = None


def regular96():
    if "reg" not in _codes:
        c, v, m = wl.regular_code(96, 3, 6, 1)
        _codes["reg"] = (c, v, m, 96, 48, None)
    return _codes["reg"]


def qc(which, Z):
    key = (which, Z)
    if key not in _codes:
        d = wl.design(which)
        base = d.shifts(Z)
        c, v = oracle.qc_lift(base, Z)
        M, N = base.shape[0] * Z, base.shape[1] * Z
        punct = d.punct_mask(Z) if d.punct_cols else None
        s = Spec((c, v, M, N, d.info_cols * Z, punct))
        s.base, s.Z, s.punct_cols = base, Z, list(d.punct_cols)
        _codes[key] = s
    return _codes[key]


def make_code(spec):
    """The library's handle of a test code: through ldpc_code_build_qc for a
    lifted code (checked to hold the oracle's edge set), else through
    ldpc_code_create."""
    c, v, m, n, k, punct = spec
    if getattr(spec, "base", None) is None:
        return L.Code.from_edges(c, v, m, n, k, punct)
    code = L.Code.from_protograph(spec.base, spec.Z, k, spec.punct_cols or None)
    assert code.info.qc_lifting == spec.Z, "no protograph view"
    gc, gv = code.edges()
    order = np.lexsort((v, c))
    assert np.array_equal(gc, c[order]) and np.array_equal(gv, v[order]), "lift differs from the oracle's"
    return code


def make_code_edges(spec):
    """The same code through ldpc_code_create (CSR tables, no protograph view)."""
    c, v, m, n, k, punct = spec
    return L.Code.from_edges(c, v, m, n, k, punct)


def rate(spec):
    c, v, m, n, k, punct = spec
    ntx = n - (0 if punct is None else int(np.sum(punct)))
    return k / ntx


def llrs(spec, batch, ebn0, seed):
    c, v, m, n, k, punct = spec
    return wl.seeded_llrs(n, batch, wl.sigma2_from_ebn0(ebn0, rate(spec)), seed, punct)


def run_gpu(code, x, torch, **kw):
    dev = torch.device("cuda:0")
    kw.setdefault("want_trace", True)
    out = L.decode(code, torch.from_numpy(np.ascontiguousarray(x)).to(dev), want_llr=True, **kw)
    torch.cuda.synchronize()
    return {k: t.cpu().numpy() for k, t in out.items()}


def run_oracle(spec, x, arith, **kw):
    c, v, m, n, k, punct = spec
    if arith == "int6":
        return oracle.decode(c, v, m, n, qllr=x, want_trace=True, threads=THREADS, **kw)
    return oracle.decode(c, v, m, n, llr=x.astype(np.float64), want_trace=True, threads=THREADS, **kw)


def assert_bitexact(g, o, schedule):
    assert np.array_equal(g["updates"], o["updates"]), "updates"
    assert np.array_equal(g["converged"] & 1, o["converged"]), "converged"
    assert np.array_equal(g["hard"], o["hard"]), "hard"
    assert np.array_equal(g["llr"].astype(np.float64), o["llr"]), "llr"
    if schedule != "flooding":
        B = len(o["updates"])
        for b in range(B):
            u = int(o["updates"][b])
            assert np.array_equal(g["trace"][b, :u], o["trace"][b, :u]), f"trace of frame {b}"


def within_tol(got, ref):
    return np.abs(got.astype(np.float64) - ref) <= TOL_REL * np.maximum(1.0, np.abs(ref))


def trace_prefix_ok(g, o):
    """Traces equal up to the first oracle near-tie; returns matched lengths."""
    lens = []
    B = len(o["updates"])
    for b in range(B):
        u = int(min(o["updates"][b], g["updates"][b]))
        gaps = o["gap"][b, :u]
        tie = np.flatnonzero(gaps < NEAR_TIE)
        lim = int(tie[0]) if len(tie) else u
        gt, ot = g["trace"][b, :lim], o["trace"][b, :lim]
        if not np.array_equal(gt, ot):
            bad = int(np.flatnonzero(gt != ot)[0])
            raise AssertionError(f"frame {b}: trace differs at step {bad} before the first near-tie "
                                 f"at {lim} (gap {gaps[bad]:.3g})")
        lens.append(lim)
    return np.array(lens)


def clopper_pearson(k, n, alpha=0.05):
    from scipy import stats
    lo = 0.0 if k == 0 else stats.beta.ppf(alpha / 2, k, n - k + 1)
    hi = 1.0 if k == n else stats.beta.ppf(1 - alpha / 2, k + 1, n - k)
    return lo, hi


def fer_in_interval(g, o):
    errs_o = int((o["hard"].sum(1) > 0).sum())
    errs_g = int((g["hard"].sum(1) > 0).sum())
    n = len(o["updates"])
    lo, hi = clopper_pearson(errs_o, n)
    return lo <= errs_g / n <= hi, (errs_g / n, errs_o / n, lo, hi)


def fmt(x):
    return f"{x:.4g}" if isinstance(x, float) and math.isfinite(x) else str(x)
