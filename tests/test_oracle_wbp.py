"""Pins of the oracle's weighted BP and its adjoint (the differentiable decoder
built on a recorded CI schedule): with unit weights the replay reproduces the
decoder's final LLRs, and the adjoint's gradients agree with FP64 central
finite differences (h = 1e-6)."""
import numpy as np
import pytest

import oracle
from paper_2102_11089_gb300 import workloads as wl


def _case(batch=3, T_mult=3, seed=4):
    c, v, m = wl.regular_code(24, 3, 6, 1, girth6=False)
    lam = wl.seeded_llrs(24, batch, wl.sigma2_from_ebn0(1.0, 0.5), seed)
    E = len(c)
    o = oracle.decode(c, v, m, 24, llr=lam.astype(np.float64), schedule="lmd-cirbp", max_updates=T_mult * E,
                      check_interval=0, want_trace=True)
    return c, v, m, lam.astype(np.float64), o


def test_unit_weights_replay_the_decoder():
    c, v, m, lam, o = _case()
    T = o["trace"].shape[1]
    assert np.all(o["updates"] == T)
    L = oracle.wbp(c, v, m, 24, lam, o["trace"], np.ones(T))
    assert np.array_equal(L, o["llr"])


def test_zero_updates_and_zero_weights():
    c, v, m, lam, o = _case(batch=2)
    T = o["trace"].shape[1]
    L = oracle.wbp(c, v, m, 24, lam, o["trace"], np.ones(T), counts=np.zeros(2, np.int64))
    assert np.array_equal(L, lam)
    L = oracle.wbp(c, v, m, 24, lam, o["trace"], np.zeros(T))
    assert np.array_equal(L, lam)  # every committed message is scaled to 0


def _loss(L):
    # BCE of the all-zero codeword's bits on the posteriors p0 = sigmoid(L)
    return np.logaddexp(0.0, -L).sum()


def _dloss(L):
    return -1.0 / (1.0 + np.exp(L))


@pytest.mark.parametrize("seed", [4, 9])
def test_adjoint_matches_central_differences(seed):
    c, v, m, lam, o = _case(batch=2, T_mult=2, seed=seed)
    tr = o["trace"]
    T = tr.shape[1]
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.6, 1.4, T)
    L, dw, dl = oracle.wbp(c, v, m, 24, lam, tr, w, dL=_dloss(oracle.wbp(c, v, m, 24, lam, tr, w)))
    h = 1e-6
    gw = dw.sum(0)
    for t in rng.choice(T, 24, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[t] += h
        wm[t] -= h
        fd = (_loss(oracle.wbp(c, v, m, 24, lam, tr, wp)) - _loss(oracle.wbp(c, v, m, 24, lam, tr, wm))) / (2 * h)
        assert abs(fd - gw[t]) <= 1e-6 * max(1.0, abs(fd)), (t, fd, gw[t])
    for b, n in [(0, 0), (0, 7), (1, 13), (1, 23)]:
        lp, lm = lam.copy(), lam.copy()
        lp[b, n] += h
        lm[b, n] -= h
        fd = (_loss(oracle.wbp(c, v, m, 24, lp, tr, w)) - _loss(oracle.wbp(c, v, m, 24, lm, tr, w))) / (2 * h)
        assert abs(fd - dl[b, n]) <= 1e-6 * max(1.0, abs(fd)), (b, n, fd, dl[b, n])


def test_per_frame_gradients_are_independent():
    c, v, m, lam, o = _case(batch=3)
    tr = o["trace"]
    T = tr.shape[1]
    w = np.linspace(0.8, 1.2, T)
    L = oracle.wbp(c, v, m, 24, lam, tr, w)
    _, dw, dl = oracle.wbp(c, v, m, 24, lam, tr, w, dL=_dloss(L), threads=3)
    _, dw1, dl1 = oracle.wbp(c, v, m, 24, lam[1:2], tr[1:2], w, dL=_dloss(L[1:2]))
    assert np.array_equal(dw[1], dw1[0]) and np.array_equal(dl[1], dl1[0])
