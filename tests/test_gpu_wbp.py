"""Weighted BP along a recorded schedule and its adjoint kernel, against the
FP64 oracle (whose adjoint is pinned to central finite differences)."""
import numpy as np
import pytest

import oracle
import paper_2102_11089_gb300 as L
from paper_2102_11089_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _c4(batch, T_mult, ebn0=2.0, seed=5):
    d = wl.wifi_like(2, 24)
    code = L.Code.from_protograph(d.shifts(24), 24, d.info_cols * 24, d.punct_cols)
    lam = wl.seeded_llrs(code.N, batch, wl.sigma2_from_ebn0(ebn0, 0.5), seed)
    x = torch.from_numpy(lam).cuda()
    from paper_2102_11089_gb300.wbp import record_schedule
    trace, upd = record_schedule(code, x, T_mult * code.E, n_p=16)
    return code, lam, x, trace, upd


def test_unit_weights_reproduce_the_decoder():
    from paper_2102_11089_gb300.wbp import weighted_bp
    code, lam, x, trace, upd = _c4(32, 2)
    T = trace.shape[1]
    assert int(upd.min()) == T
    p = L.make_params("lmd-cirbp", "fp32", max_updates=T, check_interval=0)
    ref = L.decode(code, x, p, want_llr=True)["llr"]
    out = weighted_bp(code, x, trace, torch.ones(T, device="cuda"))
    torch.cuda.synchronize()
    err = (out - ref).abs() / ref.abs().clamp(min=1.0)
    assert float(err.max()) <= 1e-4


def _oracle_case(batch=8, T_mult=2, seed=3):
    code, lam, x, trace, upd = _c4(batch, T_mult, ebn0=1.5, seed=seed)
    T = trace.shape[1]
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, T).astype(np.float32)
    c, v = code.edges()
    return code, lam, x, trace, w, c, v


def test_forward_and_adjoint_match_the_oracle():
    from paper_2102_11089_gb300.wbp import weighted_bp
    code, lam, x, trace, w, c, v = _oracle_case()
    tr = trace.cpu().numpy()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    xt = x.clone().requires_grad_(True)
    out = weighted_bp(code, xt, trace, wt)
    dL = (-torch.sigmoid(-out)).detach()  # d/dL of sum softplus(-L)
    out.backward(dL)
    torch.cuda.synchronize()
    L64, dw64, dl64 = oracle.wbp(c, v, code.M, code.N, lam.astype(np.float64), tr, w.astype(np.float64),
                                 dL=dL.cpu().numpy().astype(np.float64), threads=8)
    Lg = out.detach().cpu().numpy()
    assert np.max(np.abs(Lg - L64) / np.maximum(1.0, np.abs(L64))) <= 1e-3
    g64 = dw64.sum(0)
    g32 = wt.grad.cpu().numpy()
    assert np.linalg.norm(g32 - g64) <= 1e-3 * np.linalg.norm(g64)
    d32 = xt.grad.cpu().numpy()
    assert np.linalg.norm(d32 - dl64) <= 1e-3 * np.linalg.norm(dl64)


def test_counts_limit_the_replay_and_zero_weights():
    from paper_2102_11089_gb300.wbp import weighted_bp
    code, lam, x, trace, w, c, v = _oracle_case(batch=4)
    T = trace.shape[1]
    counts = torch.tensor([0, 1, T // 2, T], dtype=torch.int64, device="cuda")
    wt = torch.from_numpy(w).cuda()
    out = weighted_bp(code, x, trace, wt, counts=counts).cpu().numpy()
    L64 = oracle.wbp(c, v, code.M, code.N, lam.astype(np.float64), trace.cpu().numpy(), w.astype(np.float64),
                     counts=counts.cpu().numpy())
    assert np.array_equal(out[0], lam[0])
    assert np.max(np.abs(out - L64) / np.maximum(1.0, np.abs(L64))) <= 1e-3
    z = weighted_bp(code, x, trace, torch.zeros(T, device="cuda"))
    assert torch.equal(z, x)


def test_invalid_trace_entry_is_flagged():
    from paper_2102_11089_gb300.wbp import weighted_bp
    code, lam, x, trace, w, c, v = _oracle_case(batch=2)
    bad = trace.clone()
    bad[1, 5] = code.E + 3
    weighted_bp(code, x, bad, torch.ones(bad.shape[1], device="cuda"))
    with pytest.raises(L.LdpcError) as e:
        L.sync()
    assert e.value.name == "LDPC_ERR_INVALID_ARG"
    L.sync()


def test_config4_sized_training_step():
    # 12x24 protograph, Z=24 (n=576), T = 8E, 1,024 frames at 2.0 dB: the
    # directional derivative along the gradient matches central differences of
    # the loss, and a small step against the gradient lowers it.  The step is
    # small because the truncation error of central differences grows with
    # eps^2 times the third derivative of the loss, large for the exponential
    # terms of the BCE and of phi; at 1e-3 the FP32 loss still resolves the
    # difference (about 1e-5 on a loss of about 1e-3)
    from paper_2102_11089_gb300.wbp import bce_all_zero, weighted_bp
    code, lam, x, trace, upd = _c4(1024, 8, ebn0=2.0, seed=11)
    T = trace.shape[1]
    w = torch.ones(T, device="cuda", requires_grad=True)
    loss = bce_all_zero(weighted_bp(code, x, trace, w))
    loss.backward()
    g = w.grad.double()
    assert torch.isfinite(g).all() and float(g.abs().max()) > 0
    gn = float(g.norm())
    d = (-g / gn).float()
    eps = 1e-3
    with torch.no_grad():
        lp = float(bce_all_zero(weighted_bp(code, x, trace, w + eps * d)).double())
        lm = float(bce_all_zero(weighted_bp(code, x, trace, w - eps * d)).double())
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - (-gn)) <= 0.05 * gn, (fd, -gn)
    assert lp < float(loss)
