"""C-ABI contract tests that need no GPU: the library loads, exports every
function of include/ldpc.h, has the struct layouts the header declares,
validates arguments and builds codes (host side) identically to the oracle."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import paper_2102_11089_gb300 as L
from paper_2102_11089_gb300 import _build
from paper_2102_11089_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ldpc.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return L._load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ldpc_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", L.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (ldpc_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_struct_layouts_match_header(lib):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "ldpc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(ldpc_decode_params_t), offsetof(ldpc_decode_params_t, gamma),
         offsetof(ldpc_decode_params_t, max_updates), offsetof(ldpc_decode_params_t, seed),
         offsetof(ldpc_decode_params_t, form), sizeof(ldpc_code_info_t));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    P = L.DecodeParams
    assert vals == [ctypes.sizeof(P), P.gamma.offset, P.max_updates.offset, P.seed.offset,
                    P.form.offset, ctypes.sizeof(L.CodeInfo)]


def test_status_strings(lib):
    for code, name in [(0, "LDPC_OK"), (-1, "LDPC_ERR_INVALID_ARG"), (-2, "LDPC_ERR_DUPLICATE_EDGE"),
                       (-3, "LDPC_ERR_INDEX_RANGE"), (-4, "LDPC_ERR_EMPTY_NODE"),
                       (-5, "LDPC_ERR_UNSUPPORTED"), (-9, "LDPC_ERR_NONFINITE_LLR")]:
        assert lib.ldpc_status_string(code).decode() == name


def test_code_create_validation(lib):
    with pytest.raises(L.LdpcError) as e:
        L.Code.from_edges([0, 0], [1, 1], 1, 2, 1)
    assert e.value.name == "LDPC_ERR_DUPLICATE_EDGE"
    with pytest.raises(L.LdpcError) as e:
        L.Code.from_edges([0, 1], [0, 5], 2, 2, 1)
    assert e.value.name == "LDPC_ERR_INDEX_RANGE"
    with pytest.raises(L.LdpcError) as e:
        L.Code.from_edges([0, 0], [0, 1], 2, 2, 1)  # check 1 has no edge
    assert e.value.name == "LDPC_ERR_EMPTY_NODE"
    with pytest.raises(L.LdpcError) as e:
        L.Code.from_edges([0, 0], [0, 1], 1, 3, 1)  # variable 2 has no edge
    assert e.value.name == "LDPC_ERR_EMPTY_NODE"
    with pytest.raises(L.LdpcError) as e:
        L.Code.from_edges([0], [0], 1, 1, 0)
    assert e.value.name == "LDPC_ERR_INVALID_ARG"
    out = ctypes.c_void_p()
    assert lib.ldpc_code_create(None, None, 3, 1, 1, None, 1, ctypes.byref(out)) == -1
    with pytest.raises(L.LdpcError) as e:
        L.Code.from_protograph(np.array([[0, 5]]), 4, 1)  # shift >= Z
    assert e.value.name == "LDPC_ERR_INVALID_ARG"


def test_canonical_edge_order_and_info(lib):
    c, v, m = wl.regular_code(96, 3, 6, 1)
    perm = np.random.default_rng(0).permutation(len(c))
    code = L.Code.from_edges(c[perm], v[perm], m, 96, 48)
    cc, vv = code.edges()
    order = np.lexsort((v, c))
    assert np.array_equal(cc, c[order]) and np.array_equal(vv, v[order])
    assert code.info.max_vn_degree == 3 and code.info.max_cn_degree == 6
    assert code.info.max_two_hop == 18


@pytest.mark.parametrize("which,Z", [("wifi", 96), ("bg2", 16), ("bg2", 384), ("bg1", 384)])
def test_qc_lift_matches_oracle(lib, which, Z):
    d = wl.design(which)
    base = d.shifts(Z)
    code = L.Code.from_protograph(base, Z, d.info_cols * Z, d.punct_cols)
    cc, vv = code.edges()
    oc, ov = oracle.qc_lift(base, Z)
    order = np.lexsort((ov, oc))
    assert np.array_equal(cc, oc[order]) and np.array_equal(vv, ov[order])
    sz = d.sizes(Z)
    assert (code.M, code.N, code.E, code.K) == (sz["M"], sz["N"], sz["E"], sz["K"])
    assert code.info.n_punctured == 2 * Z * (len(d.punct_cols) > 0)
    assert code.info.qc_lifting == Z


def test_decode_validation_needs_no_gpu(lib):
    c, v, m = wl.regular_code(96, 3, 6, 1)
    code = L.Code.from_edges(c, v, m, 96, 48)
    p = L.make_params("lmd-cirbp", max_updates=10)
    null = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    # batch 0 is a no-op
    assert lib.ldpc_decode(code._h, null, 0, ctypes.byref(p), null, null, null, null, null, null) == 0
    bad = [("schedule", 9), ("arith", 5), ("max_updates", -1), ("gamma", 1.5), ("llr_clip", 0.0), ("llr_clip", 2e4),
           ("tune", 0x200), ("tune", 3), ("check_interval", -2)]
    for field, val in bad:
        q = L.make_params("lmd-cirbp", max_updates=10)
        setattr(q, field, val)
        assert lib.ldpc_decode(code._h, dummy, 4, ctypes.byref(q), null, null, null, null, null,
                               null) == -1, field
    for n_p in (0, 385):
        q = L.make_params("me-cirbp", max_updates=10, n_p=n_p)
        assert lib.ldpc_decode(code._h, dummy, 4, ctypes.byref(q), null, null, null, null, null,
                               null) == -1
    q = L.make_params("lmd-cirbp", max_updates=10, form=L.FORM_CLUSTER)  # single-edge: no cluster form
    assert lib.ldpc_decode(code._h, dummy, 4, ctypes.byref(q), null, null, null, null, null,
                           null) == -5
    q = L.make_params("me-cirbp", max_updates=10, form=L.FORM_SPLIT)  # multi-edge: no split form
    assert lib.ldpc_decode(code._h, dummy, 4, ctypes.byref(q), null, null, null, null, null,
                           null) == -5
    q = L.make_params("me-cirbp", max_updates=10, form=5)
    assert lib.ldpc_decode(code._h, dummy, 4, ctypes.byref(q), null, null, null, null, null,
                           null) == -1
    q = L.make_params("rbp", "int6", max_updates=10, q_step=0.0)
    assert lib.ldpc_decode(code._h, dummy, 4, ctypes.byref(q), null, null, null, null, null,
                           null) == -1
    assert lib.ldpc_decode(code._h, null, 4, ctypes.byref(p), null, null, null, null, null,
                           null) == -1
    assert lib.ldpc_decode(None, dummy, 4, ctypes.byref(p), null, null, null, null, null,
                           null) == -1
    assert lib.ldpc_awgn_llr(code._h, null, 0, 0, 0, null, null, ctypes.c_float(0.5), null) == 0
    assert lib.ldpc_awgn_llr(code._h, null, 3, 0, 0, null, null, ctypes.c_float(0.5), null) == -1


def test_decode_degree_limits_need_no_gpu(lib):
    """Lane teams hold a check (every schedule) or a variable (dynamic schedules)
    within one warp: degrees above 32 are refused before any device work."""
    null = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    # variable 0 in 33 checks (plus a second edge per check so no check is degree 1)
    chk = [m for m in range(33) for _ in range(2)]
    var = [v for m in range(33) for v in (0, 1 + m)]
    wide_v = L.Code.from_edges(np.array(chk, np.int32), np.array(var, np.int32), 33, 34, 1)
    # check 0 on 33 variables
    chk2 = [0] * 33 + list(range(1, 34))
    var2 = list(range(33)) + list(range(33))
    wide_c = L.Code.from_edges(np.array(chk2, np.int32), np.array(var2, np.int32), 34, 33, 1)
    for sched in ("me-cirbp", "me-lmd-cirbp", "lmd-cirbp", "cirbp", "rbp", "lmdrbp"):
        q = L.make_params(sched, max_updates=10)
        assert lib.ldpc_decode(wide_v._h, dummy, 4, ctypes.byref(q), null, null, null, null, null, null) == -5, sched
    for sched in ("flooding", "me-lmd-cirbp", "lmd-cirbp"):
        q = L.make_params(sched, max_updates=10)
        assert lib.ldpc_decode(wide_c._h, dummy, 4, ctypes.byref(q), null, null, null, null, null, null) == -5, sched
    # the no-allocation entry point applies the same limits
    for code, sched in ((wide_v, "me-lmd-cirbp"), (wide_v, "lmd-cirbp"), (wide_c, "flooding")):
        q = L.make_params(sched, max_updates=10)
        assert lib.ldpc_decode_noalloc(code._h, dummy, 4, ctypes.byref(q), null, null, null, null, null,
                                       null) == -5, sched


def test_default_params(lib):
    p = L.DecodeParams()
    assert lib.ldpc_default_params(ctypes.byref(p)) == 0
    assert p.schedule == L.LMD_CIRBP and p.arith == L.FP32_SUMPRODUCT
    assert abs(p.gamma - 0.1) < 1e-12 and p.check_interval == 1 and p.llr_clip == 25.0
    assert lib.ldpc_default_params(None) == -1


def test_queue_validation_needs_no_gpu(lib):
    d = wl.design("bg2")
    code = L.Code.from_protograph(d.shifts(16), 16, d.info_cols * 16, d.punct_cols)
    null = ctypes.c_void_p()
    dummy = ctypes.c_void_p(64)
    one = (ctypes.c_void_p * 1)(code._h)
    p = L.make_params("me-lmd-cirbp")
    q = lib.ldpc_decode_queue
    assert q(one, 1, null, 0, null, ctypes.byref(p), null, null, null, L.QUEUE_PERSISTENT, null) == 0
    assert q(one, 0, dummy, 1, dummy, ctypes.byref(p), null, null, null, 1, null) == -1  # no codes
    assert q(one, 17, dummy, 1, dummy, ctypes.byref(p), null, null, null, 1, null) == -1
    assert q(one, 1, dummy, 1, dummy, ctypes.byref(p), null, null, null, 2, null) == -1  # mode
    assert q(one, 1, dummy, -1, dummy, ctypes.byref(p), null, null, null, 1, null) == -1
    assert q(one, 1, dummy, 1 << 31, dummy, ctypes.byref(p), null, null, null, 1, null) == -5
    assert q(one, 1, null, 1, dummy, ctypes.byref(p), null, null, null, 1, null) == -1  # no items
    for sched in ["flooding", "rbp", "cirbp"]:
        r = L.make_params(sched)
        assert q(one, 1, dummy, 1, dummy, ctypes.byref(r), null, null, null, 1, null) == -5
    r = L.make_params("me-cirbp", n_p=0)
    assert q(one, 1, dummy, 1, dummy, ctypes.byref(r), null, null, null, 1, null) == -1
    r = L.make_params("me-cirbp", tune=0x200)
    assert q(one, 1, dummy, 1, dummy, ctypes.byref(r), null, null, null, 1, null) == -1
    assert L.WORK_ITEM_DTYPE.itemsize == 40


def test_ci_stats_validation_needs_no_gpu(lib):
    null = ctypes.c_void_p()
    dummy = ctypes.c_void_p(64)
    for nb in (0, 1025):
        assert lib.ldpc_ci_stats(dummy, dummy, 10, nb, dummy, null) == -1
    assert lib.ldpc_ci_stats(null, dummy, 10, 8, dummy, null) == -1
    assert lib.ldpc_ci_stats(dummy, dummy, -1, 8, dummy, null) == -1


def test_encode_plan_needs_no_gpu(lib):
    null = ctypes.c_void_p()
    for which, Z in [("wifi", 96), ("wifi", 24), ("bg2", 16), ("bg2", 384), ("bg1", 384)]:
        d = wl.design(which)
        code = L.Code.from_protograph(d.shifts(Z), Z, d.info_cols * Z, d.punct_cols)
        assert lib.ldpc_encode(code._h, null, 0, null, null) == 0, (which, Z)  # plan accepted
    c, v, m = wl.regular_code(96, 3, 6, 1)
    tab = L.Code.from_edges(c, v, m, 96, 48)
    assert lib.ldpc_encode(tab._h, null, 0, null, null) == -5  # no protograph
    base = np.zeros((3, 6), np.int32)  # all-ones protograph: no dual-diagonal core
    qc = L.Code.from_protograph(base, 4, 12)
    assert lib.ldpc_encode(qc._h, null, 0, null, null) == -5


@pytest.mark.parametrize("n,dv,dc", [(96, 3, 6), (2304, 3, 6), (1000, 4, 8), (99, 3, 9)])
def test_build_regular_code_is_regular_with_girth_six(lib, n, dv, dc):
    # ldpc_code_build_regular: exact degrees, no double edge, no 4-cycle (two
    # checks share at most one variable), deterministic for a seed
    code = L.Code.regular(n, dv, dc, 7)
    assert (code.N, code.M, code.E, code.K) == (n, n * dv // dc, n * dv, n - n * dv // dc)
    c, v = code.edges()
    H = np.zeros((code.M, code.N), np.int64)
    np.add.at(H, (c, v), 1)
    assert H.max() == 1
    assert set(H.sum(0)) == {dv} and set(H.sum(1)) == {dc}
    ov = H @ H.T
    np.fill_diagonal(ov, 0)
    assert ov.max() <= 1
    c2, v2 = L.Code.regular(n, dv, dc, 7).edges()
    assert np.array_equal(c, c2) and np.array_equal(v, v2)
    c3, v3 = L.Code.regular(n, dv, dc, 8).edges()
    assert not (np.array_equal(c, c3) and np.array_equal(v, v3))


def test_build_regular_rejects_bad_shapes(lib):
    for args in [(97, 3, 6), (96, 0, 6), (96, 3, 1), (96, 3, 40), (4, 3, 6)]:
        with pytest.raises(L.LdpcError) as e:
            L.Code.regular(*args, 1)
        assert e.value.name == "LDPC_ERR_INVALID_ARG"


def test_decode_ex_validation_needs_no_gpu(lib):
    # ldpc_decode_ex: outputs struct required; flooding keeps no L~^C (pre_out);
    # the split form runs only the single-edge schedules
    c, v, m = wl.regular_code(96, 3, 6, 1)
    code = L.Code.from_edges(c, v, m, 96, 48)
    dummy = ctypes.c_void_p(16)
    o = L.DecodeOutputs()
    p = L.make_params("flooding", max_updates=288)
    assert lib.ldpc_decode_ex(code._h, dummy, 4, ctypes.byref(p), None, None) == -1
    o.pre_out = 16
    assert lib.ldpc_decode_ex(code._h, dummy, 4, ctypes.byref(p), ctypes.byref(o), None) == -1
    assert lib.ldpc_decode_ex(code._h, dummy, 0, ctypes.byref(L.make_params("cirbp", max_updates=9)),
                              ctypes.byref(o), None) == 0  # batch 0: no-op
    q = L.make_params("flooding", max_updates=288, form=L.FORM_SPLIT)
    assert lib.ldpc_decode_ex(code._h, dummy, 4, ctypes.byref(q), ctypes.byref(L.DecodeOutputs()), None) == -5
    assert ctypes.sizeof(L.DecodeOutputs) == 8 * ctypes.sizeof(ctypes.c_void_p)
