"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
derived by hand on a toy graph, exact MAP / max-marginals on cycle-free graphs
(brute force over all codewords), brute-force ML on a tiny loopy code, codeword
symmetry, bit-exact agreement of the incremental refresh with a full
recomputation, the per-update operation counts of Table I / Table II, hand-made
cases of Algorithm 4 and the published Philox known-answer vectors.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2102_11089_gb300 import workloads as wl

TOY_CHK = np.array([0, 0, 0, 1, 1, 1], dtype=np.int32)
TOY_VAR = np.array([0, 1, 2, 1, 2, 3], dtype=np.int32)


def _ev(expr):
    return float(eval(expr, {"log": math.log, "abs": abs}))


def _golden(golden_dir):
    with open(os.path.join(golden_dir, "toy_graph_steps.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# P8: Philox4x32-10 known answers, channel statistics


def test_philox_known_answers(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_channel_llr_statistics():
    # y = 1 + w, w ~ N(0, s2): lambda = 2y/s2 ~ N(2/s2, 4/s2)  (Sec. 2.A, Sec. 5)
    rate = 0.5
    eb = np.full(64, 2.0)
    lam = oracle.awgn_llr(4096, rate, eb, seed=11)
    s2 = wl.sigma2_from_ebn0(2.0, rate)
    assert abs(s2 - 1.0 / (2 * 0.5 * 10 ** 0.2)) < 1e-15
    m, v = lam.mean(), lam.var()
    n = lam.size
    assert abs(m - 2 / s2) < 5 * math.sqrt(4 / s2 / n)
    assert abs(v / (4 / s2) - 1) < 5 * math.sqrt(2 / n)
    from scipy import stats
    z = (lam.ravel() - 2 / s2) / math.sqrt(4 / s2)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # independent frames and positions: correlation between neighbours ~ 0
    assert abs(np.corrcoef(lam[:, :-1].ravel(), lam[:, 1:].ravel())[0, 1]) < 0.02


def test_channel_puncturing_and_frames():
    punct = np.zeros(64, np.uint8)
    punct[:8] = 1
    a = oracle.awgn_llr(64, 0.5, [1.0, 1.0], seed=5, frame_offset=0, punct=punct)
    b = oracle.awgn_llr(64, 0.5, [1.0], seed=5, frame_offset=1, punct=punct)
    assert np.all(a[:, :8] == 0)
    assert np.array_equal(a[1], b[0])           # counter = global frame index
    assert not np.array_equal(a[0], a[1])


def test_quantiser_rounding_decision_in_float32():
    lam = np.array([0.24, 0.25, 0.26, -0.75, 15.4, 16.0, -100.0, 0.0], np.float32)
    q = oracle.quantize(lam, 0.5)
    # rint(x/0.5): 0.48->0, 0.5->0 (half to even), 0.52->1, -1.5->-2, 30.8->31, 32->31 (sat)
    assert list(q) == [0, 0, 1, -2, 31, 31, -31, 0]


# ---------------------------------------------------------------------------
# P1: hand-derived steps on the toy graph


def test_toy_fp_initial_state_and_first_cirbp_step(golden_dir):
    g = _golden(golden_dir)["fp"]
    lam = np.array([[_ev(x) for x in g["lam"]]])
    o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule="cirbp", gamma=0.1,
                      max_updates=0, check_interval=0, want_state=True)
    st = o["state"]
    np.testing.assert_allclose(st["P"][0], [_ev(x) for x in g["init_P"]], rtol=0, atol=1e-13)
    np.testing.assert_allclose(st["Lt"][0], [_ev(x) for x in g["init_Lt"]], rtol=0, atol=1e-13)
    np.testing.assert_allclose(st["D"][0], [_ev(x) for x in g["init_D"]], rtol=0, atol=1e-13)
    o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule="cirbp", gamma=0.1,
                      max_updates=1, check_interval=0, want_state=True, want_trace=True)
    assert list(o["trace"][0]) == g["cirbp_trace"][:1]
    for key in ["C", "P", "L", "Lt", "D"]:
        np.testing.assert_allclose(o["state"][key][0], [_ev(x) for x in g["after_step1"][key]],
                                   rtol=0, atol=1e-13, err_msg=key)
    for sch, key in [("cirbp", "cirbp_trace"), ("lmd-cirbp", "lmd_cirbp_trace"),
                     ("rbp", "rbp_trace")]:
        o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule=sch, gamma=0.1,
                          max_updates=2, check_interval=0, want_trace=True)
        assert list(o["trace"][0]) == g[key], sch


def test_toy_fp_lmdrbp(golden_dir):
    # Algorithm 2: line 9's residual argmax over the refreshed checks, then line 10
    # re-selects the check into n' (LMDRBP) or not (sLMDRBP); hand-derived traces
    g = _golden(golden_dir)
    lam = np.array([[_ev(x) for x in g["fp"]["lam"]]])
    for sch, key in [("lmdrbp", "lmdrbp_trace"), ("slmdrbp", "slmdrbp_trace")]:
        o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule=sch, max_updates=2,
                          check_interval=0, want_trace=True)
        assert list(o["trace"][0]) == g["fp"][key], sch
    # degree-1 rule of Sec. 5.A (VN 0 and VN 3 have one check each)
    d1 = g["fp_degree1"]
    lam = np.array([[_ev(x) for x in d1["lam"]]])
    o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule="rbp", max_updates=0,
                      check_interval=0, want_state=True)
    np.testing.assert_allclose(o["state"]["P"][0], [_ev(x) for x in d1["init_P"]], rtol=0, atol=1e-13)
    for sch, key in [("lmdrbp", "lmdrbp_trace"), ("slmdrbp", "slmdrbp_trace")]:
        o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule=sch, max_updates=3,
                          check_interval=0, want_trace=True)
        assert list(o["trace"][0]) == d1[key], sch
        o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule=sch, max_updates=2,
                          check_interval=0, want_state=True)
        np.testing.assert_allclose(o["state"]["P"][0], [_ev(x) for x in d1["P_after_step2"]],
                                   rtol=0, atol=1e-13)


def test_toy_fp_flooding_first_iteration_equals_precompute(golden_dir):
    # P6: one flooding iteration sends exactly the precomputed messages of eq. (2)
    g = _golden(golden_dir)["fp"]
    lam = np.array([[_ev(x) for x in g["lam"]]])
    o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule="flooding", max_updates=6,
                      check_interval=0)
    np.testing.assert_allclose(o["llr"][0], [_ev(x) for x in g["flooding_L_after_1_iteration"]],
                               rtol=0, atol=1e-13)


def test_toy_fp_cirbp_fallback_branch(golden_dir):
    # gamma above every D: Alg. 1 line 6 takes the global residual argmax (= RBP)
    g = _golden(golden_dir)["fp"]
    lam = np.array([[_ev(x) for x in g["lam"]]])
    o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, llr=lam, schedule="cirbp", gamma=0.9,
                      max_updates=2, check_interval=0, want_trace=True)
    assert list(o["trace"][0]) == g["rbp_trace"]
    assert o["counters"]["fallback"][0] == 2


def test_toy_int_schedules(golden_dir):
    g = _golden(golden_dir)["int"]
    q = np.array([g["q"]], np.int8)
    o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, qllr=q, schedule="cirbp", max_updates=0,
                      check_interval=0, want_state=True, q_step=g["q_step"])
    assert list(o["state"]["P"][0]) == g["init_P"]
    assert list(o["state"]["Lt"][0]) == g["init_Lt"]
    for sch, key, ci in [("cirbp", "cirbp", 0), ("cirbp", "cirbp_stop", 1),
                         ("lmd-cirbp", "lmd_cirbp", 0), ("rbp", "rbp", 0)]:
        exp = g[key]
        o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, qllr=q, schedule=sch, gamma=0.1,
                          max_updates=2, check_interval=ci, want_trace=True,
                          q_step=g["q_step"])
        n = exp["updates"]
        assert list(o["trace"][0][:n]) == exp["trace"], key
        assert o["updates"][0] == n and o["converged"][0] == exp["converged"], key
        assert list(o["llr"][0]) == exp["L"], key
    f = g["flooding"]
    o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, qllr=q, schedule="flooding", max_updates=f["updates"],
                      check_interval=1)
    assert o["updates"][0] == f["updates"] and o["converged"][0] == f["converged"]
    assert list(o["llr"][0]) == f["L"]
    o = oracle.decode(TOY_CHK, TOY_VAR, 2, 4, qllr=q, schedule="flooding", max_updates=6,
                      check_interval=0)
    assert list(o["llr"][0]) == f["L_after_1_iteration"]


def test_ci_equals_paper_definition():
    # eq. (8) with p0(L) = e^L / (1 + e^L), on the oracle's own L and L~
    c, v, m = wl.regular_code(96, 3, 6, 1)
    lam = wl.seeded_llrs(96, 8, wl.sigma2_from_ebn0(1.0, 0.5), 3)
    o = oracle.decode(c, v, m, 96, llr=lam, schedule="lmd-cirbp", max_updates=50,
                      check_interval=0, want_state=True)
    st = o["state"]

    def p0(x):
        return np.exp(x) / (1.0 + np.exp(x))
    np.testing.assert_allclose(st["D"], np.abs(p0(st["L"]) - p0(st["Lt"])), rtol=0, atol=1e-15)
    assert np.all(st["D"] >= 0) and np.all(st["D"] < 1)


# ---------------------------------------------------------------------------
# P2: cycle-free graphs -> exact bitwise MAP (sum-product) / max-marginals (min-sum)


def _random_tree(rng, n_target):
    """Random cycle-free Tanner graph; every check has degree >= 2."""
    chk, var = [], []
    n_v, n_c = 1, 0
    while n_v < n_target:
        anchor = int(rng.integers(n_v))
        k = int(min(rng.integers(1, 4), n_target - n_v))
        chk.append(n_c); var.append(anchor)
        for _ in range(k):
            chk.append(n_c); var.append(n_v)
            n_v += 1
        n_c += 1
    return np.array(chk, np.int32), np.array(var, np.int32), n_c, n_v


def _codewords(chk, var, m, n):
    H = np.zeros((m, n), np.int64)
    H[chk, var] = 1
    words = np.array(list(itertools.product([0, 1], repeat=n)), np.int64)
    ok = ((words @ H.T) % 2 == 0).all(1)
    return words[ok]


def _map_llr(cw, lam):
    x = 1 - 2 * cw
    metric = (x * lam[None, :]).sum(1) / 2.0
    out = np.zeros(len(lam))
    for i in range(len(lam)):
        a = metric[cw[:, i] == 0]
        b = metric[cw[:, i] == 1]
        out[i] = (np.logaddexp.reduce(a) - np.logaddexp.reduce(b))
    return out


def _max_marginal(cw, q):
    x = 1 - 2 * cw
    metric = (x * q[None, :]).sum(1)
    return np.array([(metric[cw[:, i] == 0].max() - metric[cw[:, i] == 1].max()) // 2
                     for i in range(len(q))])


@pytest.mark.parametrize("schedule", ["flooding", "rbp", "cirbp", "me-cirbp"])
def test_tree_sum_product_is_exact_map(schedule):
    rng = np.random.default_rng(100)
    for trial in range(6):
        chk, var, m, n = _random_tree(rng, int(rng.integers(6, 13)))
        cw = _codewords(chk, var, m, n)
        lam = rng.normal(1.0, 1.2, n) * 2.0
        o = oracle.decode(chk, var, m, n, llr=lam[None], schedule=schedule, gamma=0.1,
                          n_p=2, n_g=4, max_updates=200 * len(chk), check_interval=0,
                          stop_on_quiescence=True)
        np.testing.assert_allclose(o["llr"][0], _map_llr(cw, lam), rtol=0, atol=1e-9,
                                   err_msg=f"trial {trial}")


@pytest.mark.parametrize("schedule", ["flooding", "rbp", "cirbp"])
def test_tree_min_sum_is_exact_max_marginal(schedule):
    rng = np.random.default_rng(200)
    for trial in range(6):
        chk, var, m, n = _random_tree(rng, int(rng.integers(5, 10)))
        cw = _codewords(chk, var, m, n)
        q = rng.integers(-3, 4, n).astype(np.int8)
        o = oracle.decode(chk, var, m, n, qllr=q[None], schedule=schedule, gamma=0.1,
                          max_updates=200 * len(chk), check_interval=0, stop_on_quiescence=True)
        assert list(o["llr"][0].astype(int)) == list(_max_marginal(cw, q.astype(np.int64))), trial


# ---------------------------------------------------------------------------
# P3: brute-force ML on a tiny loopy code


def test_bp_never_beats_ml_on_tiny_code():
    c, v, m = wl.regular_code(24, 3, 6, 9, girth6=False)
    cw = _codewords(c, v, m, 24)
    assert len(cw) >= 2 ** 12
    s2 = wl.sigma2_from_ebn0(1.0, 0.5)
    lam = wl.seeded_llrs(24, 400, s2, 4)
    x = 1 - 2 * cw
    ml = np.argmax(lam.astype(np.float64) @ x.T, axis=1)
    ml_err = (cw[ml].sum(1) > 0)
    for sch in ["flooding", "lmd-cirbp", "cirbp"]:
        o = oracle.decode(c, v, m, 24, llr=lam, schedule=sch, max_updates=20 * len(c))
        bp_err = o["hard"].sum(1) > 0
        # a decoded codeword can never have a larger correlation than the ML word
        corr_bp = ((1 - 2 * o["hard"].astype(np.int64)) * lam).sum(1)
        corr_ml = (x[ml] * lam).sum(1)
        conv = o["converged"].astype(bool)
        assert np.all(corr_bp[conv] <= corr_ml[conv] + 1e-9)
        # and ML errors are a subset of frame errors up to the rare BP-lucky case
        assert bp_err.sum() >= ml_err.sum() - 2, sch


# ---------------------------------------------------------------------------
# P4: invariants -- incremental == definitional, Table I counts, budgets


@pytest.mark.parametrize("schedule", ["rbp", "cirbp", "lmd-cirbp", "me-cirbp", "me-lmd-cirbp", "lmdrbp",
                                      "slmdrbp"])
@pytest.mark.parametrize("arith", ["fp", "int"])
def test_incremental_refresh_equals_definition(schedule, arith):
    c, v, m = wl.regular_code(48, 3, 6, 2)
    lam = wl.seeded_llrs(48, 6, wl.sigma2_from_ebn0(1.5, 0.5), 8)
    kw = dict(schedule=schedule, max_updates=600, n_p=4, n_g=8, selfcheck=True)
    if arith == "fp":
        o = oracle.decode(c, v, m, 48, llr=lam, **kw)
    else:
        o = oracle.decode(c, v, m, 48, qllr=wl.quantize_llrs(lam, 0.5), **kw)
    assert o["counters"]["selfcheck"].sum() == 0
    assert np.all(o["updates"] <= 600)
    # a fully definitional run takes the same decisions
    kw.pop("selfcheck")
    if arith == "fp":
        d = oracle.decode(c, v, m, 48, llr=lam, definitional=True, **kw)
    else:
        d = oracle.decode(c, v, m, 48, qllr=wl.quantize_llrs(lam, 0.5), definitional=True, **kw)
    assert np.array_equal(d["llr"], o["llr"]) and np.array_equal(d["updates"], o["updates"])


def test_table1_per_update_counts_regular_code():
    # (3,6)-regular: every update pre-updates (dv-1)(dc-1) = 10 C2V messages, does 10 CI
    # updates, dv-1 = 2 V2C updates; LMD-CIRBP compares (dv-1)dc-1 = 11 values per update
    # (after the first global search of N-1), CIRBP N + (dv-1) or N + E - 1 (Table I).
    c, v, m = wl.regular_code(96, 3, 6, 1)
    N, E = 96, 288
    lam = wl.seeded_llrs(N, 20, wl.sigma2_from_ebn0(1.0, 0.5), 12)
    for sch in ["lmd-cirbp", "cirbp", "rbp"]:
        o = oracle.decode(c, v, m, N, llr=lam, schedule=sch, max_updates=2000)
        ct, U = o["counters"], o["updates"]
        assert np.array_equal(ct["prop"], U)
        assert np.array_equal(ct["c2v_pre"], 10 * U)
        assert np.array_equal(ct["v2c"], 2 * U)
        assert np.array_equal(ct["ci"], 10 * U)
        assert np.array_equal(ct["ci_extra"], U)
        if sch == "lmd-cirbp":
            stopped_early = U < 2000
            exp = 11 * U + (N - 1) - np.where(stopped_early & (U > 0), 9, 0)
            assert np.array_equal(ct["cmp"], exp)
        elif sch == "cirbp":
            fb = ct["fallback"]
            assert np.array_equal(ct["cmp"], U * N + (U - fb) * 2 + fb * (E - 1))
        else:
            assert np.array_equal(ct["cmp"], U * (E - 1))


def test_table2_me_counts():
    # ME-CIRBP: each selected VN costs dv-1 residual comparisons and dv-1 V2C updates;
    # one Algorithm-4 call per step with at most N_G integer comparisons (Table II).
    c, v, m = wl.regular_code(96, 3, 6, 1)
    lam = wl.seeded_llrs(96, 10, wl.sigma2_from_ebn0(1.0, 0.5), 13)
    for ng in [4, 8, 16]:
        o = oracle.decode(c, v, m, 96, llr=lam, schedule="me-cirbp", n_p=8, n_g=ng,
                          max_updates=960)
        ct, U = o["counters"], o["updates"]
        assert np.array_equal(ct["cmp"], 2 * U)
        assert np.array_equal(ct["v2c"], 2 * U)
        assert np.all(ct["icmp"] <= ng * ct["steps"])
        assert np.all(U <= ct["steps"] * 8)


def test_committed_edge_has_zero_residual_and_budget_truncation():
    c, v, m = wl.regular_code(96, 3, 6, 1)
    lam = wl.seeded_llrs(96, 4, wl.sigma2_from_ebn0(0.5, 0.5), 14)
    for sch in ["rbp", "cirbp", "lmd-cirbp"]:
        for T in [1, 7, 31]:
            o = oracle.decode(c, v, m, 96, llr=lam, schedule=sch, max_updates=T, check_interval=0,
                              want_trace=True, want_state=True)
            st = o["state"]
            for b in range(4):
                e = o["trace"][b][T - 1]
                assert st["C"][b][e] == st["P"][b][e]
            assert np.all(o["updates"] == T)
    o = oracle.decode(c, v, m, 96, llr=lam, schedule="me-cirbp", n_p=8, n_g=4, max_updates=13,
                      check_interval=0)
    assert np.all(o["updates"] == 13)   # last step truncated to the remaining budget


def test_lmd_next_vn_is_in_two_hop_set_or_degree1_rule():
    # Alg. 3 line 11 / Sec. 5.A: the next VN lies in U(m*,n*), or N(m*)\n* when d_v(n*) = 1.
    d = wl.bg2_like(3)
    chk, var = oracle.qc_lift(d.shifts(16), 16)
    M, N = d.base.shape[0] * 16, d.base.shape[1] * 16
    lam = wl.seeded_llrs(N, 3, wl.sigma2_from_ebn0(1.0, 0.2), 15, d.punct_mask(16))
    o = oracle.decode(chk, var, M, N, llr=lam, schedule="lmd-cirbp", max_updates=3000,
                      check_interval=0, want_trace=True)
    order = np.lexsort((var, chk))
    e_cn, e_vn = chk[order], var[order]
    nb_c = {}
    for cc, vv in zip(e_cn, e_vn):
        nb_c.setdefault(cc, set()).add(vv)
    nb_v = {}
    for cc, vv in zip(e_cn, e_vn):
        nb_v.setdefault(vv, set()).add(cc)
    seen_deg1 = 0
    for b in range(3):
        tr = o["trace"][b]
        for t in range(len(tr) - 1):
            e, e2 = tr[t], tr[t + 1]
            n, mm, n2 = e_vn[e], e_cn[e], e_vn[e2]
            if len(nb_v[n]) == 1:
                seen_deg1 += 1
                cand = nb_c[mm] - {n}
            else:
                cand = set().union(*[nb_c[i] for i in nb_v[n] - {mm}]) - {n}
            assert n2 in cand
    assert seen_deg1 > 0


# ---------------------------------------------------------------------------
# P5: codeword symmetry


def _random_codeword(chk, var, m, n, rng):
    H = np.zeros((m, n), np.uint8)
    H[chk, var] = 1
    A = H.copy()
    piv = []
    r = 0
    for col in range(n):
        rows = np.flatnonzero(A[r:, col]) + r
        if len(rows) == 0:
            continue
        A[[r, rows[0]]] = A[[rows[0], r]]
        for rr in np.flatnonzero(A[:, col]):
            if rr != r:
                A[rr] ^= A[r]
        piv.append(col)
        r += 1
        if r == m:
            break
    free = [c for c in range(n) if c not in piv]
    x = np.zeros(n, np.uint8)
    x[free] = rng.integers(0, 2, len(free))
    for i, col in enumerate(piv):
        x[col] = (A[i, free].astype(int) @ x[free].astype(int)) % 2
    assert not ((H.astype(int) @ x) % 2).any()
    return x


@pytest.mark.parametrize("schedule", ["flooding", "rbp", "cirbp", "lmd-cirbp", "me-cirbp",
                                      "me-lmd-cirbp"])
def test_codeword_symmetry(schedule):
    c, v, m = wl.regular_code(96, 3, 6, 1)
    rng = np.random.default_rng(21)
    cw = _random_codeword(c, v, m, 96, rng)
    assert cw.sum() > 0
    lam = wl.seeded_llrs(96, 6, wl.sigma2_from_ebn0(1.5, 0.5), 16).astype(np.float64)
    flip = lam * (1 - 2 * cw.astype(np.float64))
    kw = dict(schedule=schedule, max_updates=1500, n_p=8, n_g=8, want_trace=True)
    a = oracle.decode(c, v, m, 96, llr=lam, **kw)
    b = oracle.decode(c, v, m, 96, llr=flip, **kw)
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["updates"], b["updates"])
    assert np.array_equal(a["hard"] ^ cw, b["hard"])
    # 6-bit mode: L can be exactly 0, where bsgn breaks the symmetry; compare |L| and trace
    q = wl.quantize_llrs(lam.astype(np.float32), 0.5)
    qf = (q * (1 - 2 * cw.astype(np.int8))).astype(np.int8)
    kw["check_interval"] = 0
    kw["max_updates"] = 400
    a = oracle.decode(c, v, m, 96, qllr=q, **kw)
    b = oracle.decode(c, v, m, 96, qllr=qf, **kw)
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["llr"] * (1 - 2 * cw.astype(np.int64)), b["llr"])


# ---------------------------------------------------------------------------
# P7: Algorithm 4


def test_alg4_hand_cases():
    D = np.array([0.9, 0.8, 0.1, 0.6, 0.3])
    allS = np.ones(5, np.uint8)
    # groups floor(4 D) = (3, 3, 0, 2, 1): |Q(1)| = 2, |Q(2)| = 3, |Q(3)| = 4
    P, icmp = oracle.alg4(D, allS, n_g=4, n_p=3)
    assert list(P) == [0, 1, 3] and icmp <= 4
    P, _ = oracle.alg4(D, allS, n_g=4, n_p=2)
    assert list(P) == [0, 1]
    P, _ = oracle.alg4(D, allS, n_g=4, n_p=4)
    assert list(P) == [0, 1, 3, 4]
    # k* = 0: random fill of one element of the top group {0, 1}
    P, _ = oracle.alg4(D, allS, n_g=4, n_p=1, seed=7, frame=3, step=5)
    w = oracle.philox4x32_10([0, 5, 3, 0], [7, 0])  # VNs 0..3 share counter (0, step, frame)
    k0, k1 = w[0], w[1]
    assert list(P) == [0 if (k0, 0) < (k1, 1) else 1]
    # |S| <= N_P: everything is selected
    S = np.array([1, 0, 1, 0, 0], np.uint8)
    P, _ = oracle.alg4(D, S, n_g=4, n_p=3)
    assert list(P) == [0, 2]
    # all in one group: N_P drawn from it, D -> 1 stays in the top group
    P, _ = oracle.alg4(np.full(10, 0.999999999), np.ones(10, np.uint8), n_g=8, n_p=3, seed=1)
    assert len(P) == 3 and len(set(P)) == 3
    P, _ = oracle.alg4(np.array([65534.0, 0, 32767, 16383]), np.ones(4, np.uint8), n_g=4,
                       n_p=1, arith=oracle.INT)
    assert list(P) == [0]
    # integer groups: floor(D * N_G / 65534) = (3, 0, 1, 0)
    P, _ = oracle.alg4(np.array([65534.0, 0, 32767, 16383]), np.ones(4, np.uint8), n_g=4,
                       n_p=2, arith=oracle.INT)
    assert list(P) == [0, 2]


def test_alg4_random_fill_is_uniform():
    D = np.full(12, 0.5)
    counts = np.zeros(12)
    for step in range(3000):
        P, _ = oracle.alg4(D, np.ones(12, np.uint8), n_g=4, n_p=3, seed=99, step=step)
        counts[P] += 1
    from scipy import stats
    assert stats.chisquare(counts).pvalue > 1e-4


# ---------------------------------------------------------------------------
# QC lifting: two independent lifts agree and obey the circulant rule


def test_qc_lift_agrees_with_circulant_definition():
    for d, Z in [(wl.wifi_like(2, 96), 96), (wl.bg2_like(3), 32), (wl.bg1_like(5), 16)]:
        base = d.shifts(Z)
        c1, v1 = oracle.qc_lift(base, Z)
        c2, v2 = wl.qc_edges_reference_free(d, Z)
        assert sorted(zip(c1.tolist(), v1.tolist())) == sorted(zip(c2.tolist(), v2.tolist()))
        r, c = c1 // Z, v1 // Z
        assert np.all(base[r, c] >= 0)
        assert np.all((v1 % Z - c1 % Z - base[r, c]) % Z == 0)
        assert len(c1) == int((base >= 0).sum()) * Z


def test_regular_code_has_girth_at_least_six():
    c, v, m = wl.regular_code(96, 3, 6, 1)
    H = np.zeros((m, 96), np.int64)
    np.add.at(H, (c, v), 1)
    assert H.max() == 1
    assert np.all(H.sum(0) == 3) and np.all(H.sum(1) == 6)
    ov = H @ H.T
    np.fill_diagonal(ov, 0)
    assert ov.max() <= 1


# ---------------------------------------------------------------------------
# Multi-edge steps (Alg. 4, 5, 6) on a hand-derived toy graph


def _me_golden(golden_dir):
    with open(os.path.join(golden_dir, "me_toy_steps.json")) as f:
        return json.load(f)


def _me_run(g, schedule, budget):
    H = np.array(g["H"])
    chk, var = np.nonzero(H)  # row-major: (check, variable) order = the edge ids
    q = np.array([g["q"]], dtype=np.int8)
    return oracle.decode(chk.astype(np.int32), var.astype(np.int32), H.shape[0], H.shape[1], qllr=q,
                         schedule=schedule, n_p=g["n_p"], n_g=g["n_g"], q_step=g["q_step"],
                         max_updates=budget, check_interval=0, want_trace=True, want_state=True)


def _me_check_state(o, want):
    for k in ("C", "P", "L", "Lt", "D"):
        assert o["state"][k][0].tolist() == [float(x) for x in want[k]], k


def test_me_toy_table_and_initial_selection(golden_dir):
    g = _me_golden(golden_dir)
    for k, expr in g["T"].items():  # the integer CI table of the hand derivation
        assert eval(expr, {"round": round, "tanh": math.tanh}) == {1: 8025, 2: 15142, 3: 20812, 4: 24955,
                                                                     5: 27796}[int(k)]
    D = np.array(g["init"]["D"], dtype=np.float64)
    assert [min(int(d) * 8 // 65534, 7) for d in D] == g["init"]["groups"]
    sel, _ = oracle.alg4(D, np.ones(6, np.uint8), g["n_g"], g["n_p"], arith=oracle.INT)
    assert sel.tolist() == g["init"]["selected"]


@pytest.mark.parametrize("schedule", ["me-cirbp", "me-lmd-cirbp"])
def test_me_toy_first_step(golden_dir, schedule):
    # Alg. 5 / Alg. 6 line 5 on P = {2, 4, 5}: per-p residual argmax on the
    # pre-step state, all commits, then the refresh of checks c0 and c2
    g = _me_golden(golden_dir)
    o = _me_run(g, schedule, 3)
    want = g["after_step1"]
    assert o["updates"][0] == 3
    assert o["trace"][0].tolist() == want["trace"]
    _me_check_state(o, want)
    assert [min(int(d) * 8 // 65534, 7) for d in o["state"]["D"][0]] == want["groups"]


def test_me_lmd_toy_second_selection_and_step(golden_dir):
    # Alg. 6 lines 6-14: P' = {argmax_{U(m*_p, p)} D} = {1, 4} (p = 2 and p = 5 both
    # name VN 4; p = 4 has degree 1), top-up of N_P - |P'| = 1 VN over O_N \ P'
    # gives {3}; the second step commits on {1, 3, 4}
    g = _me_golden(golden_dir)
    o = _me_run(g, "me-lmd-cirbp", 6)
    want = g["me_lmd_cirbp"]["after_step2"]
    assert o["trace"][0].tolist() == want["trace"]
    H = np.array(g["H"])
    chk, var = np.nonzero(H)
    assert sorted(var[o["trace"][0][3:6]].tolist()) == g["me_lmd_cirbp"]["selected_step2"]
    _me_check_state(o, want)


def test_me_cirbp_toy_second_step(golden_dir):
    # Alg. 5: the second selection is Alg. 4 over O_N again: {0, 3, 4}
    g = _me_golden(golden_dir)
    o = _me_run(g, "me-cirbp", 6)
    want = g["me_cirbp"]["after_step2"]
    assert o["trace"][0].tolist() == want["trace"]
    _me_check_state(o, want)
