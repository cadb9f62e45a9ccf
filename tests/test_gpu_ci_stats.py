"""CI counters kernel (Properties 1 and 2, Sec. 3.A) against the oracle."""
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


def test_counts_equal_the_oracle_on_the_same_pairs():
    from paper_2102_11089_gb300.ci_stats import pair_counts
    rng = np.random.default_rng(3)
    a = rng.normal(1.0, 3.0, 1_000_003).astype(np.float32)
    b = (a + rng.normal(0.0, 2.0, a.size)).astype(np.float32)
    a[:5] = [0.0, -0.0, 30.0, -30.0, 1e-8]
    b[:5] = [0.0, 1.0, -30.0, 30.0, -1e-8]
    # the bin of D is decided in FP32 on the GPU and in FP64 by the oracle: only
    # samples whose D lies within rounding distance of a bin edge may move
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    D = np.abs(np.tanh(a64 / 2) - np.tanh(b64 / 2)) / 2
    for nb in (1, 20, 1000):
        g = pair_counts(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), nb)
        o = oracle.ci_counts(a, b, nb)
        assert g.sum() == o.sum()
        assert np.array_equal(g[:, 1].sum(), o[:, 1].sum())  # correct / incorrect is exact
        x = D * nb
        near = int(np.sum(np.abs(x - np.rint(x)) < 1e-6 * nb))
        assert np.abs(g - o).sum() <= 2 * near, (nb, np.abs(g - o).sum(), near)


def test_flooding_counters_match_the_oracle_and_property1():
    from paper_2102_11089_gb300.ci_stats import flooding_counts, j_and_f
    d = wl.wifi_like(2, 96)
    code = L.Code.from_protograph(d.shifts(96), 96, d.info_cols * 96, d.punct_cols)
    lam = wl.seeded_llrs(code.N, 2048, wl.sigma2_from_ebn0(2.0, 0.5), 9)
    g = flooding_counts(code, torch.from_numpy(lam).cuda(), 3, n_bins=10)
    c, v = code.edges()
    Ls = [lam.astype(np.float64)]
    for k in (1, 2, 3):
        o = oracle.decode(c, v, code.M, code.N, llr=lam.astype(np.float64), schedule="flooding",
                          max_updates=k * code.E, check_interval=0, threads=8)
        Ls.append(o["llr"])
    for k in range(3):
        o = oracle.ci_counts(Ls[k], Ls[k + 1], 10)
        assert np.abs(g[k] - o).sum() <= 1e-4 * o.sum() + 4, k
    J, F = j_and_f(g)
    for k in range(3):
        cum = np.cumsum(g[k][::-1], axis=0)[::-1]
        ok = cum[:, 1] >= 100
        assert ok.sum() >= 3
        assert np.all(np.diff(J[k][ok]) < 0), (k, J[k])
