"""CPU oracle for the dynamic-schedule BP decoders -- TEST INFRASTRUCTURE ONLY.

Loads ``ldpc_oracle.c`` (plain C, FP64 / exact integers) through ctypes.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
use it; the CUDA library never imports or links it.  See the header of
``ldpc_oracle.c`` for the readings of the paper it implements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldpc_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libldpc_oracle.so")
_lock = threading.Lock()
_handle = None

FLOODING, RBP, CIRBP, LMD_CIRBP, ME_CIRBP, ME_LMD_CIRBP, LMDRBP, SLMDRBP = range(8)
SCHEDULES = {"flooding": FLOODING, "rbp": RBP, "cirbp": CIRBP, "lmd-cirbp": LMD_CIRBP,
             "me-cirbp": ME_CIRBP, "me-lmd-cirbp": ME_LMD_CIRBP, "lmdrbp": LMDRBP, "slmdrbp": SLMDRBP}
FP, INT = 0, 1

COUNTERS = ["prop", "v2c", "c2v_pre", "ci", "ci_extra", "cmp", "icmp", "steps", "selfcheck",
            "fallback"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_lib/libldpc_oracle.so`` (gcc)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-Wall", "-Wno-unused-function", "-o", tmp, _SRC, "-lm", "-lpthread"],
                       check=True)
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class Params(ctypes.Structure):
    _fields_ = [
        ("schedule", ctypes.c_int32), ("arith", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("n_p", ctypes.c_int32), ("n_g", ctypes.c_int32),
        ("max_updates", ctypes.c_int64), ("check_interval", ctypes.c_int64),
        ("llr_clip", ctypes.c_double), ("q_step", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("frame_offset", ctypes.c_uint64),
        ("definitional", ctypes.c_int32), ("stale_dn", ctypes.c_int32),
        ("selfcheck", ctypes.c_int32), ("stop_on_quiescence", ctypes.c_int32),
    ]


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            h = ctypes.CDLL(_LIBPATH)
            P = ctypes.c_void_p
            h.orc_decode.restype = ctypes.c_int
            h.orc_decode.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(Params), P, P, ctypes.c_int64,
                                     P, P, P, P, P, P, P, P, ctypes.c_int]
            h.orc_philox4x32_10.restype = None
            h.orc_philox4x32_10.argtypes = [P, P, P]
            h.orc_awgn_llr.restype = None
            h.orc_awgn_llr.argtypes = [ctypes.c_int, P, ctypes.c_double, P, ctypes.c_int64,
                                       ctypes.c_uint64, ctypes.c_uint64, P]
            h.orc_quantize.restype = None
            h.orc_quantize.argtypes = [P, ctypes.c_int64, ctypes.c_float, P]
            h.orc_alg4.restype = ctypes.c_int
            h.orc_alg4.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_int64, P, P]
            h.orc_qc_lift.restype = ctypes.c_int64
            h.orc_qc_lift.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P]
            h.orc_wbp.restype = ctypes.c_int
            h.orc_wbp.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int64,
                                  P, P, ctypes.c_int64, P, ctypes.c_double, P, P, P, P, ctypes.c_int]
            h.orc_counters_count.restype = ctypes.c_int
            _handle = h
    return _handle


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    _lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def awgn_llr(n: int, rate: float, ebn0_db, seed: int, frame_offset: int = 0,
             punct=None) -> np.ndarray:
    eb = np.ascontiguousarray(np.atleast_1d(ebn0_db), dtype=np.float64)
    out = np.zeros((len(eb), n), dtype=np.float64)
    pm = None if punct is None else np.ascontiguousarray(punct, dtype=np.uint8)
    _lib().orc_awgn_llr(n, _ptr(pm), rate, _ptr(eb), len(eb), seed, frame_offset, _ptr(out))
    return out


def quantize(lam32: np.ndarray, q_step: float) -> np.ndarray:
    lam = np.ascontiguousarray(lam32, dtype=np.float32)
    q = np.zeros(lam.shape, dtype=np.int8)
    _lib().orc_quantize(_ptr(lam), lam.size, q_step, _ptr(q))
    return q


def qc_lift(base: np.ndarray, Z: int):
    b = np.ascontiguousarray(base, dtype=np.int32)
    rows, cols = b.shape
    e = _lib().orc_qc_lift(_ptr(b), rows, cols, Z, None, None)
    chk = np.zeros(e, dtype=np.int32)
    var = np.zeros(e, dtype=np.int32)
    _lib().orc_qc_lift(_ptr(b), rows, cols, Z, _ptr(chk), _ptr(var))
    return chk, var


def wbp(check_idx, var_idx, n_checks: int, n_vars: int, llr, trace, w, *, counts=None, llr_clip=25.0,
        dL=None, threads=1):
    """Weighted BP along recorded schedules (FP64): update t commits
    w[t] * (clipped eq. 2 C2V) on edge trace[b, t].  Returns the final LLRs
    [batch, N]; with dL (dloss/dL) also (dloss/dw per frame [batch, T],
    dloss/dllr [batch, N]) by the adjoint."""
    chk = np.ascontiguousarray(check_idx, dtype=np.int32)
    var = np.ascontiguousarray(var_idx, dtype=np.int32)
    lam = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
    tr = np.ascontiguousarray(np.atleast_2d(trace), dtype=np.int32)
    wt = np.ascontiguousarray(w, dtype=np.float64)
    B, T = tr.shape
    assert lam.shape == (B, n_vars) and wt.shape == (T,)
    cnt = None if counts is None else np.ascontiguousarray(counts, dtype=np.int64)
    L = np.zeros((B, n_vars))
    dw = dl = None
    dLa = None
    if dL is not None:
        dLa = np.ascontiguousarray(np.atleast_2d(dL), dtype=np.float64)
        dw = np.zeros((B, T))
        dl = np.zeros((B, n_vars))
    rc = _lib().orc_wbp(_ptr(chk), _ptr(var), len(chk), n_checks, n_vars, _ptr(lam), B, _ptr(tr),
                        None if cnt is None else _ptr(cnt), T, _ptr(wt), llr_clip, _ptr(L),
                        None if dLa is None else _ptr(dLa), None if dw is None else _ptr(dw),
                        None if dl is None else _ptr(dl), threads)
    if rc != 0:
        raise RuntimeError(f"orc_wbp failed: {rc}")
    return L if dL is None else (L, dw, dl)


def ci_counts(L, Lt, n_bins: int) -> np.ndarray:
    """Counters of Properties 1 and 2 (Sec. 3.A) for the all-zero codeword, in
    FP64 from the definitions: D = |p0(L) - p0(L~)| (eq. 8), p0(x) = 1/(1 + e^-x),
    bin min(floor(D n_bins), n_bins - 1); per bin [#(L >= 0), #(L < 0),
    #(L < 0 and p0(L~) >= p0(L)), #(L < 0 and p0(L~) < p0(L))]."""
    L = np.asarray(L, dtype=np.float64).ravel()
    Lt = np.asarray(Lt, dtype=np.float64).ravel()
    p0 = 0.5 + 0.5 * np.tanh(L / 2.0)     # = 1 / (1 + e^-L), exact form
    p0t = 0.5 + 0.5 * np.tanh(Lt / 2.0)
    D = np.abs(np.tanh(L / 2.0) - np.tanh(Lt / 2.0)) / 2.0
    b = np.minimum(np.floor(D * n_bins).astype(np.int64), n_bins - 1)
    out = np.zeros((n_bins, 4), dtype=np.int64)
    wrong = L < 0
    np.add.at(out[:, 0], b[~wrong], 1)
    np.add.at(out[:, 1], b[wrong], 1)
    up = wrong & (p0t >= p0)
    np.add.at(out[:, 2], b[up], 1)
    np.add.at(out[:, 3], b[wrong & ~up], 1)
    return out


def alg4(D, in_set, n_g: int, n_p: int, arith: int = FP, seed: int = 0, frame: int = 0,
         step: int = 0):
    D = np.ascontiguousarray(D, dtype=np.float64)
    s = np.ascontiguousarray(in_set, dtype=np.uint8)
    out = np.zeros(len(D), dtype=np.int32)
    icmp = np.zeros(1, dtype=np.int64)
    k = _lib().orc_alg4(_ptr(D), _ptr(s), len(D), arith, n_g, n_p, seed, frame, step,
                        _ptr(out), _ptr(icmp))
    return out[:k].copy(), int(icmp[0])


def decode(check_idx, var_idx, n_checks: int, n_vars: int, llr=None, qllr=None, *,
           schedule="lmd-cirbp", arith=None, gamma=0.1, n_p=16, n_g=16,
           max_updates=None, check_interval=1, llr_clip=25.0, q_step=0.5, seed=0,
           frame_offset=0, definitional=False, stale_dn=False, selfcheck=False,
           stop_on_quiescence=False, want_trace=False, want_state=False, threads=1):
    """Decode a batch; returns a dict of numpy arrays (hard, updates, converged,
    llr (final L_n), counters, and optionally trace, gap, state)."""
    chk = np.ascontiguousarray(check_idx, dtype=np.int32)
    var = np.ascontiguousarray(var_idx, dtype=np.int32)
    E = len(chk)
    if qllr is not None:
        q = np.ascontiguousarray(np.atleast_2d(qllr), dtype=np.int8)
        B = q.shape[0]
        lam = None
        if arith is None:
            arith = INT
    else:
        lam = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
        B = lam.shape[0]
        q = None
        if arith is None:
            arith = FP
    if max_updates is None:
        max_updates = 10 * E
    sch = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    p = Params(sch, arith, gamma, n_p, n_g, max_updates, check_interval, llr_clip, q_step,
               seed, frame_offset, int(definitional), int(stale_dn), int(selfcheck),
               int(stop_on_quiescence))
    nct = _lib().orc_counters_count()
    hard = np.zeros((B, n_vars), dtype=np.uint8)
    upd = np.zeros(B, dtype=np.int64)
    conv = np.zeros(B, dtype=np.uint8)
    llr_out = np.zeros((B, n_vars), dtype=np.float64)
    ctr = np.zeros((B, nct), dtype=np.int64)
    trace = np.full((B, max_updates), -1, dtype=np.int32) if want_trace else None
    gap = np.full((B, max_updates), np.inf, dtype=np.float64) if want_trace else None
    state = (np.zeros((B, 2 * E + 3 * n_vars), dtype=np.float64) if want_state else None)
    rc = _lib().orc_decode(_ptr(chk), _ptr(var), E, n_checks, n_vars, ctypes.byref(p),
                           _ptr(lam), _ptr(q), B, _ptr(hard), _ptr(upd), _ptr(conv),
                           _ptr(trace), _ptr(gap), _ptr(llr_out), _ptr(ctr), _ptr(state),
                           threads)
    if rc != 0:
        raise ValueError(f"oracle decode failed with status {rc}")
    out = dict(hard=hard, updates=upd, converged=conv, llr=llr_out,
               counters={name: ctr[:, i] for i, name in enumerate(COUNTERS)})
    if want_trace:
        out["trace"], out["gap"] = trace, gap
    if want_state:
        out["state"] = dict(C=state[:, :E], P=state[:, E:2 * E],
                            L=state[:, 2 * E:2 * E + n_vars],
                            Lt=state[:, 2 * E + n_vars:2 * E + 2 * n_vars],
                            D=state[:, 2 * E + 2 * n_vars:])
    return out
