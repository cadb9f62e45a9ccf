"""Python binding of the GB300 dynamic-schedule LDPC decoder (C ABI of include/ldpc.h).

Argument marshalling only: every step of the decoding path runs in the CUDA
library ``_lib/libldpc_gb300.so``.  PyTorch provides device memory and streams.
There is no fallback: if the library cannot be loaded, importing the decoding
functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "LdpcError", "Code", "DecodeParams", "decode", "decode_noalloc", "decode_queue", "make_items", "awgn_llr",
    "sync", "library_path", "QUEUE_STATIC", "QUEUE_PERSISTENT",
    "SCHEDULES", "FLOODING", "RBP", "CIRBP", "LMD_CIRBP", "ME_CIRBP", "ME_LMD_CIRBP",
    "FP32_SUMPRODUCT", "INT6_MINSUM", "FORM_AUTO", "FORM_SMEM", "FORM_GLOBAL", "FORM_CLUSTER", "FORM_SPLIT",
]

FLOODING, RBP, CIRBP, LMD_CIRBP, ME_CIRBP, ME_LMD_CIRBP, LMDRBP, SLMDRBP = range(8)
SCHEDULES = {"flooding": FLOODING, "rbp": RBP, "cirbp": CIRBP, "lmd-cirbp": LMD_CIRBP,
             "me-cirbp": ME_CIRBP, "me-lmd-cirbp": ME_LMD_CIRBP, "lmdrbp": LMDRBP, "slmdrbp": SLMDRBP}
FP32_SUMPRODUCT, INT6_MINSUM = 0, 1
FORM_AUTO, FORM_SMEM, FORM_GLOBAL, FORM_CLUSTER, FORM_SPLIT = 0, 1, 2, 3, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "_lib", "libldpc_gb300.so")
_lock = threading.Lock()
_handle = None


def library_path() -> str:
    return _LIB


class LdpcError(RuntimeError):
    def __init__(self, status: int, name: str, detail: str):
        super().__init__(f"{name}: {detail}")
        self.status = status
        self.name = name
        self.detail = detail


class DecodeParams(ctypes.Structure):
    _fields_ = [
        ("schedule", ctypes.c_int32), ("arith", ctypes.c_int32), ("gamma", ctypes.c_double),
        ("n_p", ctypes.c_int32), ("n_g", ctypes.c_int32),
        ("max_updates", ctypes.c_int64), ("check_interval", ctypes.c_int64),
        ("llr_clip", ctypes.c_float), ("q_step", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("frame_offset", ctypes.c_uint64),
        ("form", ctypes.c_int32), ("tune", ctypes.c_int32),
    ]


class DecodeOutputs(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("hard", "updates", "converged", "trace", "llr_out", "c2v_out", "pre_out", "fallbacks")]


class CodeInfo(ctypes.Structure):
    _fields_ = [
        ("n_checks", ctypes.c_int32), ("n_vars", ctypes.c_int32), ("n_edges", ctypes.c_int64),
        ("k_info", ctypes.c_int32), ("n_punctured", ctypes.c_int32),
        ("max_vn_degree", ctypes.c_int32), ("max_cn_degree", ctypes.c_int32),
        ("max_two_hop", ctypes.c_int32), ("qc_lifting", ctypes.c_int32),
    ]


def _load():
    global _handle
    with _lock:
        if _handle is not None:
            return _handle
        if not os.path.exists(_LIB):
            raise ImportError(f"CUDA library not built: {_LIB} (run __graft_entry__.build())")
        h = ctypes.CDLL(_LIB)
        P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        h.ldpc_status_string.restype = ctypes.c_char_p
        h.ldpc_status_string.argtypes = [I32]
        h.ldpc_last_error_detail.restype = ctypes.c_char_p
        h.ldpc_last_error_detail.argtypes = []
        for name, args in [
            ("ldpc_default_params", [P]),
            ("ldpc_code_create", [P, P, I64, I32, I32, P, I32, P]),
            ("ldpc_code_build_qc", [P, I32, I32, I32, P, I32, P]),
            ("ldpc_code_build_regular", [I32, I32, I32, U64, I32, I32, P]),
            ("ldpc_code_destroy", [P]),
            ("ldpc_code_info", [P, P]),
            ("ldpc_code_edges", [P, P, P]),
            ("ldpc_awgn_llr", [P, P, I64, U64, U64, P, P, ctypes.c_float, P]),
            ("ldpc_decode", [P, P, I64, P, P, P, P, P, P, P]),
            ("ldpc_decode_noalloc", [P, P, I64, P, P, P, P, P, P, P]),
            ("ldpc_decode_ex", [P, P, I64, P, P, P]),
            ("ldpc_smem_stream", [I32, I32, I32, P, P, P]),
            ("ldpc_decode_queue", [P, I32, P, I64, P, P, P, P, P, I32, P]),
            ("ldpc_wbp_forward", [P, P, I64, P, P, I64, P, ctypes.c_float, P, P, P, P]),
            ("ldpc_ci_stats", [P, P, I64, I32, P, P]),
            ("ldpc_encode", [P, P, I64, P, P]),
            ("ldpc_awgn_llr_codewords", [P, P, I64, U64, U64, P, P, P, ctypes.c_float, P]),
            ("ldpc_wbp_backward", [P, P, I64, P, P, I64, P, ctypes.c_float, P, P, P, P, P, P, P]),
            ("ldpc_sync", [P]),
        ]:
            f = getattr(h, name)
            f.restype = I32
            f.argtypes = args
        _handle = h
        return h


def _check(status: int):
    if status != 0:
        h = _load()
        raise LdpcError(status, h.ldpc_status_string(status).decode(),
                        h.ldpc_last_error_detail().decode())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Code:
    """An LDPC code handle (ldpc_code_t)."""

    def __init__(self, handle):
        self._h = handle
        self.info = CodeInfo()
        _check(_load().ldpc_code_info(self._h, ctypes.byref(self.info)))

    @classmethod
    def from_edges(cls, check_idx, var_idx, n_checks: int, n_vars: int, k_info: int,
                   punctured=None) -> "Code":
        c = np.ascontiguousarray(check_idx, dtype=np.int32)
        v = np.ascontiguousarray(var_idx, dtype=np.int32)
        p = None if punctured is None else np.ascontiguousarray(punctured, dtype=np.uint8)
        out = ctypes.c_void_p()
        _check(_load().ldpc_code_create(_np_ptr(c), _np_ptr(v), len(c), n_checks, n_vars,
                                        _np_ptr(p), k_info, ctypes.byref(out)))
        return cls(out)

    @classmethod
    def from_protograph(cls, base, Z: int, k_info: int, punct_cols=None) -> "Code":
        b = np.ascontiguousarray(base, dtype=np.int32)
        rows, cols = b.shape
        pc = None
        if punct_cols is not None:
            pc = np.zeros(cols, np.uint8)
            pc[list(punct_cols)] = 1
        out = ctypes.c_void_p()
        _check(_load().ldpc_code_build_qc(_np_ptr(b), rows, cols, Z, _np_ptr(pc), k_info,
                                          ctypes.byref(out)))
        return cls(out)

    @classmethod
    def regular(cls, n: int, dv: int, dc: int, seed: int, *, girth6: bool = True, k_info: int = 0) -> "Code":
        """ldpc_code_build_regular: seeded (dv, dc)-regular code, double edges
        (and 4-cycles) removed."""
        out = ctypes.c_void_p()
        _check(_load().ldpc_code_build_regular(n, dv, dc, seed, int(girth6), k_info, ctypes.byref(out)))
        return cls(out)

    @property
    def M(self):
        return self.info.n_checks

    @property
    def N(self):
        return self.info.n_vars

    @property
    def E(self):
        return self.info.n_edges

    @property
    def K(self):
        return self.info.k_info

    def edges(self):
        c = np.zeros(self.E, np.int32)
        v = np.zeros(self.E, np.int32)
        _check(_load().ldpc_code_edges(self._h, _np_ptr(c), _np_ptr(v)))
        return c, v

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _handle is not None:
            _handle.ldpc_code_destroy(h)
            self._h = None


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_params(schedule="lmd-cirbp", arith="fp32", *, gamma=0.1, n_p=16, n_g=16,
                max_updates=0, check_interval=1, llr_clip=25.0, q_step=0.5, seed=0,
                frame_offset=0, form=FORM_AUTO, tune=0) -> DecodeParams:
    p = DecodeParams()
    _check(_load().ldpc_default_params(ctypes.byref(p)))
    p.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    p.arith = {"fp32": FP32_SUMPRODUCT, "int6": INT6_MINSUM}.get(arith, arith)
    p.gamma, p.n_p, p.n_g = gamma, n_p, n_g
    p.max_updates, p.check_interval = max_updates, check_interval
    p.llr_clip, p.q_step, p.seed, p.frame_offset, p.form = llr_clip, q_step, seed, frame_offset, form
    p.tune = tune
    return p


def decode(code: Code, llr, params: DecodeParams | None = None, *, want_trace=False,
           want_llr=False, want_msgs=False, want_fallbacks=False, stream=None, out=None, **kw):
    """Decode a [batch, N] device tensor of channel LLRs (float32, or int8 for
    INT6).  Returns a dict of device tensors: hard, updates, converged and
    optionally trace / llr; with want_msgs the final messages c2v [batch, E]
    (L^C) and, for the dynamic schedules, pre [batch, E] (L~^C); with
    want_fallbacks the CIRBP fallback counts [batch] (ldpc_decode_ex)."""
    import torch
    if params is None:
        params = make_params(**kw)
    if not llr.is_cuda or not llr.is_contiguous():
        raise ValueError("llr must be a contiguous CUDA tensor")
    want = torch.int8 if params.arith == INT6_MINSUM else torch.float32
    if llr.dtype != want:
        raise ValueError(f"llr must be {want} for this arithmetic")
    B = llr.shape[0]
    dev = llr.device
    if out is None:
        out = dict(hard=torch.empty((B, code.N), dtype=torch.uint8, device=dev),
                   updates=torch.empty(B, dtype=torch.int64, device=dev),
                   converged=torch.empty(B, dtype=torch.uint8, device=dev))
        if want_trace:
            out["trace"] = torch.full((B, max(1, params.max_updates)), -1, dtype=torch.int32,
                                      device=dev)
        if want_llr:
            out["llr"] = torch.empty((B, code.N), dtype=torch.float32, device=dev)
        if want_msgs:
            out["c2v"] = torch.empty((B, code.E), dtype=torch.float32, device=dev)
            if params.schedule != FLOODING:
                out["pre"] = torch.empty((B, code.E), dtype=torch.float32, device=dev)
        if want_fallbacks:
            out["fallbacks"] = torch.empty(B, dtype=torch.int64, device=dev)

    def ptr(name):
        t = out.get(name)
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    if any(k in out for k in ("c2v", "pre", "fallbacks")):
        o = DecodeOutputs(*[None if t is None else t.value for t in
                            (ptr("hard"), ptr("updates"), ptr("converged"), ptr("trace"), ptr("llr"),
                             ptr("c2v"), ptr("pre"), ptr("fallbacks"))])
        _check(_load().ldpc_decode_ex(code._h, ctypes.c_void_p(llr.data_ptr()), B, ctypes.byref(params),
                                      ctypes.byref(o), _stream_ptr(stream)))
        return out
    _check(_load().ldpc_decode(code._h, ctypes.c_void_p(llr.data_ptr()), B, ctypes.byref(params),
                               ptr("hard"), ptr("updates"), ptr("converged"), ptr("trace"),
                               ptr("llr"), _stream_ptr(stream)))
    return out


def decode_noalloc(code: Code, llr, params: DecodeParams, out: dict, stream=None):
    """ldpc_decode_noalloc: like decode(), for callers that must not allocate.
    Every output tensor is supplied by the caller in `out` (keys hard, updates,
    converged and optionally trace, llr); nothing is allocated, neither here nor
    in the library, which works in its fixed 32 MiB device array."""
    def ptr(name):
        t = out.get(name)
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    _check(_load().ldpc_decode_noalloc(code._h, ctypes.c_void_p(llr.data_ptr()), llr.shape[0],
                                       ctypes.byref(params), ptr("hard"), ptr("updates"),
                                       ptr("converged"), ptr("trace"), ptr("llr"),
                                       _stream_ptr(stream)))
    return out


QUEUE_STATIC, QUEUE_PERSISTENT = 0, 1
WORK_ITEM_DTYPE = np.dtype([("code", "<i4"), ("flags", "<i4"), ("llr_offset", "<i8"),
                            ("out_offset", "<i8"), ("max_updates", "<i8"), ("frame_index", "<u8")])


def make_items(code, llr_offset, out_offset, max_updates, frame_index, device="cuda"):
    """Device array of ldpc_work_item_t (40 bytes each) from per-item columns."""
    import torch
    n = len(code)
    a = np.zeros(n, dtype=WORK_ITEM_DTYPE)
    a["code"], a["llr_offset"], a["out_offset"] = code, llr_offset, out_offset
    a["max_updates"], a["frame_index"] = max_updates, frame_index
    return torch.from_numpy(a.view(np.uint8).copy()).to(device)


def decode_queue(codes, items, n_items: int, llr, params: DecodeParams, *, hard=None, updates=None,
                 converged=None, mode=QUEUE_PERSISTENT, stream=None):
    """ldpc_decode_queue: frames of several lifted codes, each with its own
    budget, from a device work queue (see make_items)."""
    arr = (ctypes.c_void_p * len(codes))(*[c._h for c in codes])

    def ptr(t):
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    _check(_load().ldpc_decode_queue(arr, len(codes), ptr(items), n_items, ptr(llr), ctypes.byref(params),
                                     ptr(hard), ptr(updates), ptr(converged), mode, _stream_ptr(stream)))


def awgn_llr(code: Code, ebn0_db, seed: int, frame_offset: int = 0, *, quantize=False,
             q_step=0.5, stream=None, out=None, qout=None):
    """Channel LLRs of the all-zero codeword for a [batch] device tensor of
    Eb/N0 values (dB).  Returns (llr float32 [batch, N], qllr int8 or None)."""
    import torch
    B = ebn0_db.shape[0]
    dev = ebn0_db.device
    if out is None:
        out = torch.empty((B, code.N), dtype=torch.float32, device=dev)
    if quantize and qout is None:
        qout = torch.empty((B, code.N), dtype=torch.int8, device=dev)
    _check(_load().ldpc_awgn_llr(code._h, ctypes.c_void_p(ebn0_db.data_ptr()), B, seed,
                                 frame_offset, ctypes.c_void_p(out.data_ptr()),
                                 None if qout is None else ctypes.c_void_p(qout.data_ptr()),
                                 q_step, _stream_ptr(stream)))
    return out, qout


def encode(code: Code, info, stream=None):
    """Codewords [batch, N] (uint8 0/1) of the info bits [batch, K] (uint8)."""
    import torch
    if not info.is_cuda or info.dtype != torch.uint8 or not info.is_contiguous():
        raise ValueError("info must be a contiguous CUDA uint8 tensor")
    B = info.shape[0]
    cw = torch.empty((B, code.N), dtype=torch.uint8, device=info.device)
    _check(_load().ldpc_encode(code._h, ctypes.c_void_p(info.data_ptr()), B, ctypes.c_void_p(cw.data_ptr()),
                               _stream_ptr(stream)))
    return cw


def awgn_llr_codewords(code: Code, ebn0_db, codewords, seed: int, frame_offset: int = 0, *, quantize=False,
                       q_step=0.5, stream=None):
    """Channel LLRs of `codewords` ([batch, N] uint8, CUDA); as awgn_llr."""
    import torch
    B = ebn0_db.shape[0]
    dev = ebn0_db.device
    out = torch.empty((B, code.N), dtype=torch.float32, device=dev)
    qout = torch.empty((B, code.N), dtype=torch.int8, device=dev) if quantize else None
    _check(_load().ldpc_awgn_llr_codewords(code._h, ctypes.c_void_p(ebn0_db.data_ptr()), B, seed, frame_offset,
                                           ctypes.c_void_p(codewords.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           None if qout is None else ctypes.c_void_p(qout.data_ptr()), q_step,
                                           _stream_ptr(stream)))
    return out, qout


def smem_stream(blocks: int, threads: int, iters: int, sink, stream=None) -> int:
    """ldpc_smem_stream: launch the shared-memory read stream on `stream`;
    `sink` is a CUDA uint32/int32 tensor of blocks * threads words.  Returns the
    bytes the launch reads."""
    if sink.numel() < blocks * threads:
        raise ValueError("sink too small")
    nb = ctypes.c_int64(0)
    _check(_load().ldpc_smem_stream(blocks, threads, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(nb),
                                    _stream_ptr(stream)))
    return int(nb.value)


def sync(stream=None):
    _check(_load().ldpc_sync(_stream_ptr(stream)))
