"""ldpc_decode_noalloc, the entry point for callers that must not allocate
device memory when they decode (real-time loops kept out of the CUDA allocator,
processes whose memory belongs to another allocator or to a fixed budget):
through the C ABI its outputs must equal those of ldpc_decode, on two calls in
a row (the second call finds the first call's leftovers in the shared static
array), and in 6-bit mode equal the oracle's bit for bit.  Lifted codes run the
protograph-view kernels, edge-list codes the CSR-table kernels.  This file is
collected last on purpose."""
import numpy as np
import pytest

import paper_2102_11089_gb300 as L
from paper_2102_11089_gb300 import workloads as wl

from gpu_helpers import assert_bitexact, llrs, make_code, make_code_edges, qc, regular96, run_oracle, within_tol

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _outputs(B, N, budget, dev):
    return dict(hard=torch.full((B, N), 7, dtype=torch.uint8, device=dev),
                updates=torch.full((B,), -1, dtype=torch.int64, device=dev),
                converged=torch.full((B,), 9, dtype=torch.uint8, device=dev),
                trace=torch.full((B, budget), -1, dtype=torch.int32, device=dev),
                llr=torch.full((B, N), float("nan"), dtype=torch.float32, device=dev))


CASES = [("reg", "lmd-cirbp", "int6"), ("reg", "cirbp", "fp32"), ("wifi", "me-lmd-cirbp", "fp32"),
         ("wifi", "me-cirbp", "int6"), ("wifi", "me-lmd-cirbp", "int6"), ("bg2", "flooding", "fp32"),
         ("bg2", "flooding", "int6"), ("bg2", "rbp", "int6"), ("bg2", "lmd-cirbp", "fp32"),
         ("wifi-tab", "me-lmd-cirbp", "int6")]


@pytest.mark.parametrize("which,schedule,arith", CASES)
def test_noalloc_matches_decode_on_two_calls(which, schedule, arith):
    spec = {"reg": regular96, "wifi": lambda: qc("wifi", 96), "wifi-tab": lambda: qc("wifi", 96),
            "bg2": lambda: qc("bg2", 16)}[which]()
    code = make_code_edges(spec) if which == "wifi-tab" else make_code(spec)
    assert (code.info.qc_lifting > 0) == (which in ("wifi", "bg2"))
    dev = torch.device("cuda:0")
    lam = llrs(spec, 40, 1.5, 314)
    x = wl.quantize_llrs(lam, 0.5) if arith == "int6" else lam
    x = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    budget = 3 * code.E
    p = L.make_params(schedule, arith, max_updates=budget, n_p=16, n_g=8, seed=11)
    ref = L.decode(code, x, p, want_trace=True, want_llr=True)
    for call in range(2):
        out = L.decode_noalloc(code, x, p, _outputs(x.shape[0], code.N, budget, dev))
        torch.cuda.synchronize()
        for k in ["hard", "updates", "converged", "trace"]:
            assert torch.equal(out[k], ref[k]), (call, k)
        assert within_tol(out["llr"].cpu().numpy(), ref["llr"].cpu().numpy().astype(np.float64)).all()
    if arith == "int6":
        kw = dict(schedule=schedule, max_updates=budget, n_p=16, n_g=8, seed=11, gamma=0.1)
        o = run_oracle(spec, x.cpu().numpy(), "int6", **kw)
        assert_bitexact({k: v.cpu().numpy() for k, v in out.items()}, o, schedule)


def test_noalloc_rejects_state_beyond_static_scratch():
    # the WiFi-like protograph lifted with Z = 40,000 (n = 960,000): the state of a
    # single FP32 single-edge frame is ~41 MB, beyond the 32 MiB array
    d = wl.wifi_like(2, 96)
    code = L.Code.from_protograph(d.shifts(40000), 40000, 12 * 40000)
    assert code.N == 960000
    dev = torch.device("cuda:0")
    x = torch.zeros((1, code.N), dtype=torch.float32, device=dev)
    out = dict(hard=torch.empty((1, code.N), dtype=torch.uint8, device=dev),
               updates=torch.empty(1, dtype=torch.int64, device=dev),
               converged=torch.empty(1, dtype=torch.uint8, device=dev))
    p = L.make_params("lmd-cirbp", "fp32", max_updates=10)
    with pytest.raises(L.LdpcError) as e:
        L.decode_noalloc(code, x, p, out)
    assert e.value.name == "LDPC_ERR_UNSUPPORTED"
    assert "static scratch" in e.value.detail
