"""Parity at the benchmark's full size and launch configuration.

The bench decodes 65,536 frames of the WiFi-like n = 2304 code at Eb/N0 1.5 dB with
ME-LMD-CIRBP (N_P 64, N_G 16, budget 3E, syndrome after every step) in one
`ldpc_decode` launch, default form.  Here the same launch runs on seeded inputs
(shared generator), with the edge trace requested (stores only: the schedule
and results are those of the timed launch), and is checked

  * on sampled frames against the oracle, run frame by frame with the same frame
    index (the random fill of Algorithm 4 is keyed by it): 6-bit mode bit-exact
    (trace, updates, decisions, final LLRs); FP32 traces equal up to the oracle's
    first near-tie, and decisions and convergence equal for the frames that meet
    none (beyond a near-tie FP32 and FP64 may legitimately part);
  * on every frame by properties that hold at any size: a frame is reported
    converged exactly when its decisions satisfy every check, the decisions are
    the signs of the final LLRs, and the budget bounds the update count (a frame
    that did not converge used all of it).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2102_11089_gb300 as L
from paper_2102_11089_gb300 import workloads as wl

from gpu_helpers import NEAR_TIE, make_code, qc, rate

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BATCH = 65536
EBN0 = 1.5
SEED_IN = 2102
KW = dict(schedule="me-lmd-cirbp", n_p=64, n_g=16, check_interval=1, seed=1234, gamma=0.1)


def _syndrome_ok(spec, hard):
    """Per frame: every check of H satisfied by the decisions (chunked)."""
    c, v, m, n, k, punct = spec
    order = np.argsort(c, kind="stable")
    cs, vs = c[order], v[order]
    starts = np.flatnonzero(np.r_[True, cs[1:] != cs[:-1]])
    ok = np.empty(hard.shape[0], dtype=bool)
    for b0 in range(0, hard.shape[0], 4096):
        h = hard[b0:b0 + 4096, vs].astype(np.uint8)
        par = np.bitwise_xor.reduceat(h, starts, axis=1)
        ok[b0:b0 + 4096] = ~par.any(axis=1)
    return ok


def _run(arith):
    spec = qc("wifi", 96)
    code = make_code(spec)
    budget = 3 * code.E
    lam = wl.seeded_llrs(code.N, BATCH, wl.sigma2_from_ebn0(EBN0, rate(spec)), SEED_IN)
    x = wl.quantize_llrs(lam, 0.5) if arith == "int6" else lam
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    out = L.decode(code, xt, arith=arith, max_updates=budget, want_trace=True, want_llr=True, **KW)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    idx = np.unique(np.r_[0, BATCH - 1, rng.choice(BATCH, 22, replace=False)])
    sel = torch.from_numpy(idx).to(dev)
    g = {"hard": out["hard"].cpu().numpy(), "updates": out["updates"].cpu().numpy(),
         "converged": out["converged"].cpu().numpy(), "llr": out["llr"].cpu().numpy(),
         "trace": out["trace"].index_select(0, sel).cpu().numpy()}
    del out, xt
    torch.cuda.empty_cache()
    return spec, code, budget, x, idx, g


def _oracle_frame(spec, x, b, arith, budget):
    c, v, m, n, k, punct = spec
    kw = dict(KW, max_updates=budget, frame_offset=int(b), want_trace=True)
    if arith == "int6":
        return oracle.decode(c, v, m, n, qllr=x[b:b + 1], **kw)
    return oracle.decode(c, v, m, n, llr=x[b:b + 1].astype(np.float64), **kw)


def _whole_batch_properties(spec, budget, g):
    conv = (g["converged"] & 1).astype(bool)
    assert np.array_equal(conv, _syndrome_ok(spec, g["hard"])), "converged flag vs zero syndrome"
    assert np.array_equal(g["hard"], (g["llr"] < 0).astype(np.uint8)), "decisions vs signs of L"
    assert (g["updates"] >= 0).all() and (g["updates"] <= budget).all()
    assert (g["updates"][~conv] == budget).all(), "a frame that did not converge stopped early"


def test_bench_workload_int6_sampled_frames_bitexact():
    spec, code, budget, x, idx, g = _run("int6")
    _whole_batch_properties(spec, budget, g)
    for r, b in enumerate(idx):
        o = _oracle_frame(spec, x, b, "int6", budget)
        u = int(o["updates"][0])
        assert int(g["updates"][b]) == u, f"frame {b}: updates"
        assert int(g["converged"][b] & 1) == int(o["converged"][0]), f"frame {b}: converged"
        assert np.array_equal(g["hard"][b], o["hard"][0]), f"frame {b}: decisions"
        assert np.array_equal(g["llr"][b].astype(np.float64), o["llr"][0]), f"frame {b}: final LLRs"
        assert np.array_equal(g["trace"][r, :u], o["trace"][0, :u]), f"frame {b}: trace"


def test_bench_workload_fp32_sampled_frames_match_oracle():
    spec, code, budget, x, idx, g = _run("fp32")
    _whole_batch_properties(spec, budget, g)
    assert (g["converged"] & 1).mean() > 0.97  # FER about 1 % at this operating point
    matched = []
    for r, b in enumerate(idx):
        o = _oracle_frame(spec, x, b, "fp32", budget)
        u = int(min(o["updates"][0], g["updates"][b]))
        tie = np.flatnonzero(o["gap"][0, :int(o["updates"][0])] < NEAR_TIE)
        if len(tie) == 0:
            assert int(g["converged"][b] & 1) == int(o["converged"][0]), f"frame {b}: converged"
            assert np.array_equal(g["hard"][b], o["hard"][0]), f"frame {b}: decisions"
        elif (g["converged"][b] & 1) and o["converged"][0]:
            # both found a codeword by different paths: the same one
            assert np.array_equal(g["hard"][b], o["hard"][0]), f"frame {b}: decisions"
        lim = int(tie[0]) if len(tie) and tie[0] < u else u
        gt, ot = g["trace"][r, :lim], o["trace"][0, :lim]
        assert np.array_equal(gt, ot), f"frame {b}: trace differs before the first near-tie at {lim}"
        matched.append(lim)
    # the comparison covers hundreds of committed updates per frame
    assert np.median(matched) >= 256, matched
