"""Execution forms: frame state in global-memory slots (large codes, or on
request) must give the same results as the shared-memory form and the oracle."""
import numpy as np
import pytest

import paper_2102_11089_gb300 as L
from paper_2102_11089_gb300 import workloads as wl

from gpu_helpers import (NEAR_TIE, assert_bitexact, fer_in_interval, llrs, make_code, qc, regular96, run_gpu,
                         run_oracle, trace_prefix_ok, within_tol)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ALL = ["flooding", "rbp", "cirbp", "lmd-cirbp", "me-cirbp", "me-lmd-cirbp", "lmdrbp", "slmdrbp"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("schedule", ALL)
def test_global_form_equals_shared_form_and_oracle(schedule):
    spec = regular96()
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 700, 1.5, 5), 0.5)  # more frames than state slots
    kw = dict(schedule=schedule, max_updates=6 * code.E, gamma=0.1, n_p=8, n_g=8, seed=4)
    g_s = run_gpu(code, q, torch, arith="int6", form=L.FORM_SMEM, **kw)
    g_g = run_gpu(code, q, torch, arith="int6", form=L.FORM_GLOBAL, **kw)
    for k in ["hard", "updates", "converged", "llr", "trace"]:
        assert np.array_equal(g_s[k], g_g[k]), k
    if schedule not in ("flooding", "me-cirbp", "me-lmd-cirbp"):  # single-edge: VN arrays in smem, edges global
        g_p = run_gpu(code, q, torch, arith="int6", form=L.FORM_SPLIT, **kw)
        for k in ["hard", "updates", "converged", "llr", "trace"]:
            assert np.array_equal(g_s[k], g_p[k]), k
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g_g, o, schedule)


@pytest.mark.parametrize("schedule", ["lmd-cirbp", "cirbp", "rbp", "lmdrbp", "me-lmd-cirbp", "flooding"])
def test_global_form_fp32_wifi(schedule):
    spec = qc("wifi", 96)
    code = make_code(spec)
    lam = llrs(spec, 24, 1.75, 8)
    kw = dict(schedule=schedule, max_updates=3 * code.E, gamma=0.1, n_p=16, n_g=16, seed=2)
    g_s = run_gpu(code, lam, torch, arith="fp32", form=L.FORM_SMEM, **kw)
    g_g = run_gpu(code, lam, torch, arith="fp32", form=L.FORM_GLOBAL, **kw)
    for k in ["hard", "updates", "converged", "llr", "trace"]:
        assert np.array_equal(g_s[k], g_g[k]), k
    if schedule not in ("flooding", "me-lmd-cirbp"):
        for tune in (0, 1 << 2, 3 << 2):  # frames per CTA of the split form: as many as fit, 2, 8
            g_p = run_gpu(code, lam, torch, arith="fp32", form=L.FORM_SPLIT, tune=tune, **kw)
            for k in ["hard", "updates", "converged", "llr", "trace"]:
                assert np.array_equal(g_s[k], g_p[k]), (tune, k)


def test_split_form_refuses_other_schedules():
    spec = regular96()
    code = make_code(spec)
    x = torch.zeros((1, 96), dtype=torch.float32, device="cuda:0")
    for sch in ["flooding", "me-lmd-cirbp"]:
        with pytest.raises(L.LdpcError) as e:
            L.decode(code, x, schedule=sch, max_updates=10, form=L.FORM_SPLIT)
        assert e.value.name == "LDPC_ERR_UNSUPPORTED"


@pytest.mark.parametrize("schedule,n_p", [("lmd-cirbp", 0), ("me-lmd-cirbp", 64), ("me-cirbp", 64),
                                          ("flooding", 0)])
def test_large_bg2_z128_int6_bitexact(schedule, n_p):
    # n = 6656: FP32 and 6-bit state exceed one SM for the single-edge and flooding forms
    spec = qc("bg2", 128)
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 4, 1.0, 17), 0.5)
    kw = dict(schedule=schedule, max_updates=2 * code.E, gamma=0.1, n_p=max(n_p, 1), n_g=16, seed=6)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)


@pytest.mark.parametrize("form", ["global", "cluster"])
@pytest.mark.parametrize("schedule", ["me-lmd-cirbp", "me-cirbp"])
def test_two_degree_classes_at_largest_n_p_int6_bitexact(schedule, form):
    # BG2-shaped Z = 64 (checks of degree 4 to 10, VNs up to degree 23): the
    # affected checks and pairs of a step fill both degree-class lists, and at
    # N_P = 384 the lists come close to their shared capacity N_P (d_v,max - 1)
    spec = qc("bg2", 64)
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 3, 1.25, 41), 0.5)
    kw = dict(schedule=schedule, max_updates=2 * code.E, gamma=0.1, n_p=384, n_g=16, seed=12,
              form=L.FORM_GLOBAL if form == "global" else L.FORM_CLUSTER)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **{k: v for k, v in kw.items() if k != "form"})
    assert_bitexact(g, o, schedule)


@pytest.mark.parametrize("schedule", ["me-lmd-cirbp", "lmd-cirbp"])
def test_large_bg1_z384_n26112(schedule):
    # the 26,112-bit BG1-shaped code: frame state ~1.3 MB (FP32), global-memory form
    spec = qc("bg1", 384)
    code = make_code(spec)
    assert code.N == 26112 and code.E == 122496
    q = wl.quantize_llrs(llrs(spec, 2, 1.2, 23), 0.5)
    kw = dict(schedule=schedule, max_updates=code.E // 2, gamma=0.1, n_p=256, n_g=16, seed=8)
    g = run_gpu(code, q, torch, arith="int6", **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, schedule)
    lam = llrs(spec, 2, 1.2, 23)
    g = run_gpu(code, lam, torch, arith="fp32", **kw)
    o = run_oracle(spec, lam, "fp32", **kw)
    trace_prefix_ok(g, o)


def test_shared_form_refuses_too_large_code():
    spec = qc("bg1", 384)
    code = make_code(spec)
    x = torch.zeros((1, code.N), dtype=torch.float32, device="cuda:0")
    with pytest.raises(L.LdpcError) as e:
        L.decode(code, x, schedule="lmd-cirbp", max_updates=10, form=L.FORM_SMEM)
    assert e.value.name == "LDPC_ERR_UNSUPPORTED"


def _all_outputs(code, x, torch, **kw):
    p = L.make_params(**kw)
    out = L.decode(code, x, p, want_trace=True, want_llr=True)
    L.sync()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("arith", ["int6", "fp32"])
@pytest.mark.parametrize("schedule", ["me-lmd-cirbp", "me-cirbp"])
def test_cluster_form_equals_global_form_bg2_z128(schedule, arith):
    # n = 6656: frame state spread over the shared memory of a cluster
    spec = qc("bg2", 128)
    code = make_code(spec)
    lam = llrs(spec, 40, 1.0, 31)
    x = torch.from_numpy(wl.quantize_llrs(lam, 0.5) if arith == "int6" else lam).cuda()
    kw = dict(schedule=schedule, arith=arith, max_updates=2 * code.E, gamma=0.1, n_p=64, n_g=16, seed=5)
    ref = _all_outputs(code, x, torch, form=L.FORM_GLOBAL, **kw)
    for tune in [0, 1 << 6, 2 << 6]:
        got = _all_outputs(code, x, torch, form=L.FORM_CLUSTER, tune=tune, **kw)
        for k in ref:
            assert np.array_equal(ref[k], got[k]), (tune, k)
    got = _all_outputs(code, x, torch, form=L.FORM_AUTO, **kw)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k


def test_cluster_form_small_code_and_sixteen_ctas():
    # a code that fits one CTA, forced onto a cluster of 2 (smallest) and of 16
    # (non-portable size: either it runs and agrees, or it is refused)
    spec = qc("wifi", 96)
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 300, 1.5, 9), 0.5)
    x = torch.from_numpy(q).cuda()
    kw = dict(schedule="me-lmd-cirbp", arith="int6", max_updates=3 * code.E, gamma=0.1, n_p=32, n_g=16, seed=2)
    ref = _all_outputs(code, x, torch, form=L.FORM_SMEM, **kw)
    got = _all_outputs(code, x, torch, form=L.FORM_CLUSTER, **kw)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    try:
        got = _all_outputs(code, x, torch, form=L.FORM_CLUSTER, tune=3 << 6, **kw)
    except L.LdpcError as e:
        assert e.name == "LDPC_ERR_UNSUPPORTED"
    else:
        for k in ref:
            assert np.array_equal(ref[k], got[k]), k


def test_cluster_form_bg1_z384_matches_oracle_int6():
    spec = qc("bg1", 384)
    code = make_code(spec)
    q = wl.quantize_llrs(llrs(spec, 2, 1.2, 41), 0.5)
    kw = dict(schedule="me-lmd-cirbp", max_updates=code.E // 2, gamma=0.1, n_p=256, n_g=16, seed=8)
    g = run_gpu(code, q, torch, arith="int6", form=L.FORM_CLUSTER, **kw)
    o = run_oracle(spec, q, "int6", **kw)
    assert_bitexact(g, o, "me-lmd-cirbp")


def test_cluster_form_bg1_z384_fp32_matches_oracle():
    # FP32 on the cluster form of the 26,112-bit code: the edge trace equals the
    # oracle's up to its first near-tie; over the first steps (before any near-tie)
    # every final message L^C, L~^C within 1e-4 max(1, |m|) of FP64
    import oracle
    spec = qc("bg1", 384)
    code = make_code(spec)
    c, v, m, n, k, punct = spec
    lam = llrs(spec, 4, 1.2, 43)
    kw = dict(schedule="me-lmd-cirbp", max_updates=code.E // 4, gamma=0.1, n_p=256, n_g=16, seed=8)
    g = run_gpu(code, lam, torch, arith="fp32", form=L.FORM_CLUSTER, **kw)
    o = run_oracle(spec, lam, "fp32", **kw)
    lens = trace_prefix_ok(g, o)
    assert lens.max() >= 256
    kw["max_updates"] = 512
    g = run_gpu(code, lam, torch, arith="fp32", form=L.FORM_CLUSTER, want_msgs=True, **kw)
    o = oracle.decode(c, v, m, n, llr=lam.astype(np.float64), want_trace=True, want_state=True, threads=8, **kw)
    clean = (o["gap"][:, :512] >= NEAR_TIE).all(1)
    assert clean.sum() >= 1, o["gap"][:, :512].min(1)
    assert np.array_equal(g["trace"][clean, :512], o["trace"][clean, :512])
    assert within_tol(g["c2v"][clean], o["state"]["C"][clean]).all()
    assert within_tol(g["pre"][clean], o["state"]["P"][clean]).all()


def test_smem_stream_measures_a_plausible_peak():
    # ldpc_smem_stream: the folded words are deterministic and the bandwidth lies
    # between a quarter and 1.5x of 152 SMs x 128 B/clk at 2.07 GHz
    dev = torch.device("cuda:0")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(sms * 2 * 1024, dtype=torch.int32, device=dev)
    L.smem_stream(sms * 2, 1024, 64, sink)
    torch.cuda.synchronize()
    first = sink.clone()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    nbytes = L.smem_stream(sms * 2, 1024, 2048, sink)
    b.record()
    torch.cuda.synchronize()
    assert nbytes == sms * 2 * 1024 * 2048 * 64
    gbs = nbytes / (a.elapsed_time(b) * 1e-3) / 1e9
    nominal = sms * 128 * 2.07e9 / 1e9
    assert 0.25 * nominal < gbs < 1.5 * nominal, gbs
    L.smem_stream(sms * 2, 1024, 64, sink)
    torch.cuda.synchronize()
    assert torch.equal(sink, first)
    with pytest.raises(L.LdpcError):
        L.smem_stream(1, 33, 1, sink)
