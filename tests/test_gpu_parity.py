"""GPU parity: the CUDA decoders (called through the C ABI) against the CPU
oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle
import paper_2102_11089_gb300 as L
from paper_2102_11089_gb300 import workloads as wl

from gpu_helpers import (assert_bitexact, fer_in_interval, llrs, make_code, make_code_edges, qc, regular96,
                         run_gpu, run_oracle, trace_prefix_ok, within_tol)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ALL = ["flooding", "rbp", "cirbp", "lmd-cirbp", "me-cirbp", "me-lmd-cirbp", "lmdrbp", "slmdrbp"]
DYN = ["rbp", "cirbp", "lmd-cirbp", "me-cirbp", "me-lmd-cirbp", "lmdrbp", "slmdrbp"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# ---------------------------------------------------------------------------
# 6-bit min-sum: bit-exact


@pytest.mark.parametrize("schedule", ALL)
def test_int6_bitexact_regular_n96(schedule):
    spec = regular96()
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 300, 2.0, 2021), 0.5)
    kw = dict(schedule=schedule, max_updates=10 * code.E, gamma=0.1, n_p=8, n_g=8, seed=5)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)


@pytest.mark.parametrize("schedule", DYN)
@pytest.mark.parametrize("ci,budget", [(0, 1000), (7, 1001), (288, 2880)])
def test_int6_bitexact_check_intervals_and_ragged_budgets(schedule, ci, budget):
    spec = regular96()
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 64, 1.5, 77), 0.5)
    kw = dict(schedule=schedule, max_updates=budget, check_interval=ci, gamma=0.15, n_p=5, n_g=4,
              seed=9, frame_offset=123)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)


@pytest.mark.parametrize("schedule", ALL)
@pytest.mark.parametrize("N,dv,dc", [(102, 3, 6), (99, 3, 9)])
def test_int6_bitexact_n_not_a_multiple_of_four(schedule, N, dv, dc):
    # the last VN quad of Algorithm 4's pass (and the last bitmap word) is partial
    c, v, m = wl.regular_code(N, dv, dc, 3)
    spec = (c, v, m, N, N - m, None)
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 200, 1.75, 515), 0.5)
    kw = dict(schedule=schedule, max_updates=10 * code.E, gamma=0.1, n_p=7, n_g=6, seed=11)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)


@pytest.mark.parametrize("schedule", ["me-cirbp", "me-lmd-cirbp"])
@pytest.mark.parametrize("n_g", [200, 255])
def test_int6_bitexact_many_groups(schedule, n_g):
    # group indices past a nibble: Algorithm 4's per-byte group tests up to N_G - 1 = 254
    spec = regular96()
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 200, 1.5, 4242), 0.5)
    kw = dict(schedule=schedule, max_updates=10 * code.E, gamma=0.1, n_p=6, n_g=n_g, seed=13)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)
    lam = llrs(spec, 100, 1.5, 4243)
    g = run_gpu(code, lam, torch, arith="fp32", **kw)
    o = run_oracle(spec, lam, "fp32", **kw)
    trace_prefix_ok(g, o)


@pytest.mark.parametrize("schedule,n_p", [("flooding", 0), ("rbp", 0), ("cirbp", 0),
                                          ("lmd-cirbp", 0), ("me-cirbp", 64),
                                          ("me-lmd-cirbp", 4), ("me-lmd-cirbp", 16),
                                          ("me-lmd-cirbp", 64), ("lmdrbp", 0), ("slmdrbp", 0)])
def test_int6_bitexact_wifi_n2304(schedule, n_p):
    spec = qc("wifi", 96)
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 6, 1.5, 31), 0.5)
    kw = dict(schedule=schedule, max_updates=2 * code.E, gamma=0.1, n_p=max(n_p, 1), n_g=16, seed=3)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)


@pytest.mark.parametrize("schedule", ["lmd-cirbp", "cirbp", "me-lmd-cirbp", "flooding", "lmdrbp", "slmdrbp"])
def test_int6_bitexact_bg2_degree1_and_punctured(schedule):
    spec = qc("bg2", 16)
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 8, 1.0, 41), 0.5)
    kw = dict(schedule=schedule, max_updates=3 * code.E, gamma=0.1, n_p=16, n_g=8, seed=1)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)


@pytest.mark.parametrize("which,Z", [("wifi", 96), ("bg2", 16)])
@pytest.mark.parametrize("schedule", ALL)
@pytest.mark.parametrize("arith", ["int6", "fp32"])
def test_protograph_view_equals_csr_tables(which, Z, schedule, arith):
    # the same lifted code built from its protograph (neighbours and edge ids
    # computed from the circulant shifts) and from its edge list (CSR tables):
    # every output identical, FP32 included (same arithmetic in the same order)
    spec = qc(which, Z)
    code_qc, code_tab = make_code(spec), make_code_edges(spec)
    assert code_qc.info.qc_lifting == Z and code_tab.info.qc_lifting == 0
    lam = llrs(spec, 24, 1.25, 606)
    x = wl.quantize_llrs(lam, 0.5) if arith == "int6" else lam
    kw = dict(schedule=schedule, max_updates=2 * code_qc.E, gamma=0.1, n_p=16, n_g=16, seed=21)
    a = run_gpu(code_qc, x, torch, arith=arith, **kw)
    b = run_gpu(code_tab, x, torch, arith=arith, **kw)
    for k in ["hard", "updates", "converged", "llr", "trace"]:
        assert np.array_equal(a[k], b[k]), k


# ---------------------------------------------------------------------------
# FP32 sum-product: tolerance, trace prefix, FER interval


@pytest.mark.parametrize("which", ["reg", "wifi", "bg2"])
@pytest.mark.parametrize("iters", [1, 2, 5])
def test_fp32_flooding_messages_within_tolerance(which, iters):
    # every C2V message of flooding iteration `iters` (and the total LLRs) within
    # 1e-4 max(1, |m|) of the FP64 oracle's
    spec = regular96() if which == "reg" else (qc("wifi", 96) if which == "wifi" else qc("bg2", 16))
    code = make_code(spec)
    lam = llrs(spec, 32, 1.5, 5)
    kw = dict(schedule="flooding", max_updates=iters * code.E, check_interval=0)
    g = run_gpu(code, lam, torch, arith="fp32", want_msgs=True, want_trace=False, **kw)
    o = oracle_state(spec, lam, "fp32", **kw)
    ok = within_tol(g["c2v"], o["state"]["C"])
    assert ok.all(), f"{(~ok).sum()} messages, max |d| {np.max(np.abs(g['c2v'] - o['state']['C']))}"
    ok = within_tol(g["llr"], o["llr"])
    assert ok.all(), f"max excess {np.max(np.abs(g['llr'] - o['llr']))}"


def oracle_state(spec, x, arith, **kw):
    c, v, m, n, k, punct = spec
    if arith == "int6":
        return oracle.decode(c, v, m, n, qllr=x, want_trace=True, want_state=True, threads=8, **kw)
    return oracle.decode(c, v, m, n, llr=x.astype(np.float64), want_trace=True, want_state=True, threads=8, **kw)


@pytest.mark.parametrize("schedule", ALL)
@pytest.mark.parametrize("which", ["reg", "bg2"])
def test_int6_final_message_state_bitexact(which, schedule):
    # the whole final message state (L^C and, for the dynamic schedules, L~^C),
    # not only the decisions, equals the oracle's; CIRBP also its fallback count
    spec = regular96() if which == "reg" else qc("bg2", 16)
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 40, 1.25, 808), 0.5)
    kw = dict(schedule=schedule, max_updates=2 * code.E, gamma=0.2, n_p=8, n_g=8, seed=7)
    g = run_gpu(code, q, torch, arith="int6", want_msgs=True, want_fallbacks=True, **kw)
    o = oracle_state(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)
    assert np.array_equal(g["c2v"], o["state"]["C"])
    if schedule != "flooding":
        assert np.array_equal(g["pre"], o["state"]["P"])
    assert np.array_equal(g["fallbacks"], o["counters"]["fallback"])
    if schedule == "cirbp":
        assert g["fallbacks"].sum() > 0


@pytest.mark.parametrize("schedule", ["cirbp", "lmd-cirbp", "me-lmd-cirbp", "rbp"])
def test_fp32_message_state_before_first_near_tie(schedule):
    # frames whose oracle run meets no near-tie: same trace, and every final
    # message within 1e-4 max(1, |m|) of the oracle's
    spec = qc("wifi", 96)
    code = make_code(spec)
    lam = llrs(spec, 48, 1.5, 4711)
    T = 256
    kw = dict(schedule=schedule, max_updates=T, check_interval=0, gamma=0.1, n_p=16, n_g=16, seed=3)
    g = run_gpu(code, lam, torch, arith="fp32", want_msgs=True, want_fallbacks=True, **kw)
    o = oracle_state(spec, lam, "fp32", **kw)
    clean = (o["gap"][:, :T] >= 1e-5).all(1)
    assert clean.sum() >= 8, clean.sum()
    assert np.array_equal(g["trace"][clean, :T], o["trace"][clean, :T])
    assert within_tol(g["c2v"][clean], o["state"]["C"][clean]).all()
    assert within_tol(g["pre"][clean], o["state"]["P"][clean]).all()
    assert np.array_equal(g["fallbacks"][clean], o["counters"]["fallback"][clean])


@pytest.mark.parametrize("schedule", DYN)
def test_fp32_trace_prefix_and_fer_regular_n96(schedule):
    spec = regular96()
    code = make_code(spec)
    lam = llrs(spec, 1000, 2.0, 2021)
    kw = dict(schedule=schedule, max_updates=10 * code.E, gamma=0.1, n_p=8, n_g=8, seed=5)
    g = run_gpu(code, lam, torch, arith="fp32", **kw)
    o = run_oracle(spec, lam, "fp32", **kw)
    lens = trace_prefix_ok(g, o)
    assert np.median(lens) > 20
    ok, info = fer_in_interval(g, o)
    assert ok, info


@pytest.mark.parametrize("schedule", ["rbp", "cirbp", "lmd-cirbp", "lmdrbp", "slmdrbp"])
def test_fp32_llr_tolerance_before_first_near_tie(schedule):
    spec = regular96()
    code = make_code(spec)
    lam = llrs(spec, 64, 1.0, 99)
    T = 25
    kw = dict(schedule=schedule, max_updates=T, check_interval=0, gamma=0.1)
    g = run_gpu(code, lam, torch, arith="fp32", **kw)
    o = run_oracle(spec, lam, "fp32", **kw)
    clean = (o["gap"][:, :T] >= 1e-5).all(1)
    assert clean.sum() > 32
    assert np.array_equal(g["trace"][clean, :T], o["trace"][clean, :T])
    assert within_tol(g["llr"][clean], o["llr"][clean]).all()


@pytest.mark.parametrize("schedule", ["lmd-cirbp", "me-lmd-cirbp"])
def test_fp32_wifi_fer_interval(schedule):
    # 2,048 frames at 1.25 dB with a budget of 3E (the paper's I_max = 3 regime):
    # FER near 10%, so the 95% interval of the oracle's FER is a real constraint
    spec = qc("wifi", 96)
    code = make_code(spec)
    lam = llrs(spec, 2048, 1.25, 12)
    kw = dict(schedule=schedule, max_updates=3 * code.E, gamma=0.1, n_p=16, n_g=16, seed=2)
    g = run_gpu(code, lam, torch, arith="fp32", **kw)
    o = run_oracle(spec, lam, "fp32", **kw)
    trace_prefix_ok(g, o)
    ok, info = fer_in_interval(g, o)
    assert ok, info
    assert info[1] > 0.02, info  # the oracle's FER: the point is not error-free


# ---------------------------------------------------------------------------
# channel kernel


@pytest.mark.parametrize("which", ["reg", "bg2"])
def test_channel_matches_oracle(which):
    spec = regular96() if which == "reg" else qc("bg2", 16)
    c, v, m, n, k, punct = spec
    code = make_code(spec)
    eb = np.linspace(0.5, 3.0, 40).astype(np.float32)
    dev = torch.device("cuda:0")
    lam, qv = L.awgn_llr(code, torch.from_numpy(eb).to(dev), seed=77, frame_offset=1000,
                         quantize=True, q_step=0.5)
    torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    qv = qv.cpu().numpy()
    ref = oracle.awgn_llr(n, k / (n - (0 if punct is None else int(punct.sum()))),
                          eb.astype(np.float64), seed=77, frame_offset=1000, punct=punct)
    assert within_tol(lam, ref).all(), np.max(np.abs(lam - ref))
    if punct is not None:
        assert np.all(lam[:, punct.astype(bool)] == 0)
    # the quantiser decision is taken in float32; compare away from rounding boundaries
    qref = oracle.quantize(ref.astype(np.float32), 0.5)
    frac = np.abs(ref / 0.5 - np.floor(ref / 0.5) - 0.5)
    safe = frac > 1e-3
    assert np.array_equal(qv[safe], qref[safe])


def test_channel_ragged_length_and_statistics():
    # N = 99 is not a multiple of the 4-sample Philox block
    c = np.repeat(np.arange(33), 3).astype(np.int32)
    v = np.arange(99).astype(np.int32)
    code = L.Code.from_edges(c, v, 33, 99, 33)
    eb = np.full(2000, 2.0, np.float32)
    lam, _ = L.awgn_llr(code, torch.from_numpy(eb).cuda(), seed=3)
    lam = lam.cpu().numpy().astype(np.float64)
    ref = oracle.awgn_llr(99, 1 / 3, eb.astype(np.float64), seed=3)
    assert within_tol(lam, ref).all()
    s2 = wl.sigma2_from_ebn0(2.0, 1 / 3)
    assert abs(lam.mean() - 2 / s2) < 0.02 * 2 / s2


# ---------------------------------------------------------------------------
# robustness and degenerate cases


def test_nonfinite_and_out_of_range_inputs_are_flagged():
    spec = regular96()
    code = make_code(spec)
    lam = llrs(spec, 8, 2.0, 1)
    lam[3, 10] = np.nan
    lam[5, 0] = np.inf
    for sch in ["lmd-cirbp", "flooding", "me-cirbp"]:
        g = run_gpu(code, lam, torch, arith="fp32", schedule=sch, max_updates=288, n_p=4, n_g=4)
        assert g["converged"][3] == 2 and g["converged"][5] == 2 and g["updates"][3] == 0
        assert np.all(g["converged"][[0, 1, 2, 4, 6, 7]] != 2)
        with pytest.raises(L.LdpcError) as e:
            L.sync()
        assert e.value.name == "LDPC_ERR_NONFINITE_LLR"
        L.sync()  # cleared
    q = wl.quantize_llrs(llrs(spec, 4, 2.0, 1), 0.5)
    q[1, 7] = 40
    g = run_gpu(code, q, torch, arith="int6", schedule="cirbp", max_updates=288)
    assert g["converged"][1] == 2
    with pytest.raises(L.LdpcError):
        L.sync()


@pytest.mark.parametrize("schedule", ALL)
def test_zero_budget_and_clean_frames(schedule):
    spec = regular96()
    code = make_code(spec)
    lam = np.full((4, 96), 5.0, np.float32)  # every hard decision 0: valid at count 0
    lam[1, :10] = -1.0
    g = run_gpu(code, lam, torch, arith="fp32", schedule=schedule, max_updates=0, n_p=4, n_g=4)
    assert np.all(g["updates"] == 0)
    assert g["converged"][0] == 1 and g["converged"][1] == 0
    o = run_oracle(spec, lam, "fp32", schedule=schedule, max_updates=0, n_p=4, n_g=4)
    assert np.array_equal(g["hard"], o["hard"])


def test_empty_batch_is_a_noop():
    spec = regular96()
    code = make_code(spec)
    x = torch.empty((0, 96), dtype=torch.float32, device="cuda:0")
    out = L.decode(code, x, schedule="lmd-cirbp", max_updates=10)
    assert out["updates"].numel() == 0
