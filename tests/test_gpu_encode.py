"""Encoder and codeword channel: codewords satisfy every check and carry the
info bits; decoding is symmetric in the codeword (same trace, negated LLRs),
which exposes only the bsgn(0) convention of Sec. 2.A."""
import numpy as np
import pytest

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


def _code(which, Z):
    d = wl.design(which)
    return d, L.Code.from_protograph(d.shifts(Z), Z, d.info_cols * Z, d.punct_cols)


def _syndromes(code, cw):
    c, v = code.edges()
    ptr = np.concatenate([[0], np.cumsum(np.bincount(c, minlength=code.M))])
    return np.add.reduceat(cw[:, v].astype(np.int64), ptr[:-1], axis=1) % 2


@pytest.mark.parametrize("which,Z", [("wifi", 24), ("wifi", 96), ("bg2", 16), ("bg2", 128), ("bg2", 384),
                                     ("bg1", 384)])
def test_codewords_satisfy_every_check(which, Z):
    d, code = _code(which, Z)
    rng = np.random.default_rng(Z)
    info = rng.integers(0, 2, (33, code.K), dtype=np.uint8)
    cw = L.encode(code, torch.from_numpy(info).cuda()).cpu().numpy()
    assert cw.shape == (33, code.N) and set(np.unique(cw)) <= {0, 1}
    assert np.array_equal(cw[:, :code.K], info)
    assert not _syndromes(code, cw).any()
    if code.M <= 1200:  # the parity part has full rank: the codeword is unique
        c, v = code.edges()
        par = v >= code.K
        assert wl.gf2_rank(c[par], v[par] - code.K, code.M) == code.M


@pytest.mark.parametrize("schedule", ["lmd-cirbp", "me-lmd-cirbp", "flooding", "lmdrbp"])
@pytest.mark.parametrize("arith", ["int6", "fp32"])
def test_decoding_is_symmetric_in_the_codeword(schedule, arith):
    d, code = _code("wifi", 96)
    B = 64
    rng = np.random.default_rng(7)
    info = torch.from_numpy(rng.integers(0, 2, (B, code.K), dtype=np.uint8)).cuda()
    cw = L.encode(code, info)
    eb = torch.full((B,), 1.75, dtype=torch.float32, device="cuda")
    lam, q = L.awgn_llr_codewords(code, eb, cw, seed=5, quantize=arith == "int6")
    x = q if arith == "int6" else lam
    sgn = 1 - 2 * cw.to(x.dtype)
    x0 = (x * sgn).contiguous()  # the all-zero word seen through the same (reflected) noise
    # no syndrome stop: the stop rule sees the decisions bsgn(L), where bsgn(0) = 0
    # breaks the symmetry (see the next test)
    p = L.make_params(schedule, arith, max_updates=3 * code.E, n_p=32, n_g=16, seed=2, check_interval=0)
    a = L.decode(code, x, p, want_trace=schedule != "flooding", want_llr=True)
    b = L.decode(code, x0, p, want_trace=schedule != "flooding", want_llr=True)
    assert torch.equal(a["updates"], b["updates"])
    if schedule != "flooding":
        assert torch.equal(a["trace"], b["trace"])
    assert torch.equal(a["llr"], b["llr"] * sgn.float())
    zero = b["llr"] == 0
    flip = a["hard"] ^ b["hard"]
    assert torch.equal(flip[~zero], cw[~zero])  # decisions mirror the codeword except at L = 0


def test_bsgn_zero_bias_of_the_stop_rule_int6():
    # with the syndrome stop, a 6-bit frame and its reflected all-zero twin may
    # stop at different updates: only through VNs with L = 0 (bsgn(0) = 0)
    d, code = _code("wifi", 96)
    B = 256
    rng = np.random.default_rng(8)
    info = torch.from_numpy(rng.integers(0, 2, (B, code.K), dtype=np.uint8)).cuda()
    cw = L.encode(code, info)
    eb = torch.full((B,), 1.5, dtype=torch.float32, device="cuda")
    _, q = L.awgn_llr_codewords(code, eb, cw, seed=6, quantize=True)
    sgn = 1 - 2 * cw.to(torch.int8)
    p = L.make_params("lmd-cirbp", "int6", max_updates=3 * code.E)
    a = L.decode(code, q, p, want_llr=True)
    b = L.decode(code, (q * sgn).contiguous(), p, want_llr=True)
    differ = (a["updates"] != b["updates"]).cpu().numpy()
    zero_a = (a["llr"] == 0).any(1).cpu().numpy()
    zero_b = (b["llr"] == 0).any(1).cpu().numpy()
    assert not np.any(differ & ~(zero_a | zero_b))  # every divergence involves some L = 0
