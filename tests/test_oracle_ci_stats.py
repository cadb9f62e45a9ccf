"""Pins of the oracle's CI counters (Properties 1 and 2, Sec. 3.A): hand cases
from the closed form of eq. (8), the cumulation into J(gamma) and F(gamma), and
Property 1 (J decreasing in gamma) on flooding BP of the regular (3,6) code."""
import math

import numpy as np

import oracle
from paper_2102_11089_gb300 import workloads as wl


def p0(x):
    return 1.0 / (1.0 + math.exp(-x))


def test_hand_cases():
    L = [0.0, -1.0, -1.0, 2.0, -3.0, 5.0]
    Lt = [0.0, 2.0, -4.0, 2.5, -0.5, -5.0]
    c = oracle.ci_counts(L, Lt, 10)
    # D = |p0(L) - p0(L~)|: 0 -> bin 0 correct; 0.6119 -> bin 6, wrong, toward truth;
    # |0.2689 - 0.0180| = 0.2510 -> bin 2, wrong, away; |0.8808 - 0.9241| = 0.0433 -> bin 0
    # correct; |0.0474 - 0.3775| = 0.3301 -> bin 3, wrong, toward; |0.9933 - 0.0067| -> bin 9
    d = [abs(p0(a) - p0(b)) for a, b in zip(L, Lt)]
    assert [min(int(x * 10), 9) for x in d] == [0, 6, 2, 0, 3, 9]
    exp = np.zeros((10, 4), np.int64)
    exp[0, 0] = 2
    exp[6, 1] = exp[6, 2] = 1
    exp[2, 1] = exp[2, 3] = 1
    exp[3, 1] = exp[3, 2] = 1
    exp[9, 0] = 1
    assert np.array_equal(c, exp)


def test_cumulation_into_j_and_f():
    torch = __import__("pytest").importorskip("torch")
    from paper_2102_11089_gb300.ci_stats import j_and_f
    c = np.array([[10, 1, 1, 0], [4, 2, 2, 0], [1, 3, 2, 1]], np.int64)
    J, F = j_and_f(c)
    assert np.allclose(J, [15 / 6, 5 / 5, 1 / 3])
    assert np.allclose(F, [5.0, 4.0, 2.0])
    J, F = j_and_f(np.array([[3, 0, 0, 0]], np.int64))
    assert J[0] == np.inf and np.isnan(F[0])
    del torch


def test_property1_j_decreases_on_flooding():
    # regular (3,6) n = 96 at 2.5 dB, 3,000 frames, iterations 0 and 1: J(gamma) falls
    # over the bins that hold at least 40 incorrect decisions
    c, v, m = wl.regular_code(96, 3, 6, 1)
    lam = wl.seeded_llrs(96, 3000, wl.sigma2_from_ebn0(2.5, 0.5), 21).astype(np.float64)
    E = len(c)
    Ls = [lam]
    for k in (1, 2):
        o = oracle.decode(c, v, m, 96, llr=lam, schedule="flooding", max_updates=k * E, check_interval=0,
                          threads=8)
        Ls.append(o["llr"])
    for k in (0, 1):
        cnt = oracle.ci_counts(Ls[k], Ls[k + 1], 10)
        cum = np.cumsum(cnt[::-1], axis=0)[::-1]
        ok = cum[:, 1] >= 40
        J = cum[ok, 0] / cum[ok, 1]
        assert len(J) >= 3
        assert np.all(np.diff(J) < 0), (k, J)
