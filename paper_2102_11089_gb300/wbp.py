"""Weighted BP along a recorded schedule, differentiable through the library's
adjoint kernel (ldpc_wbp_forward / ldpc_wbp_backward).

Not a step of the paper: the training-side use of its schedules.  A CI decoder
records which edge it commits at each update; `weighted_bp` replays that
schedule with one weight per update (update t commits w[t] times the eq. (2)
C2V of the edge) and returns the final LLRs.  Gradients with respect to the
weights and the channel LLRs come from the hand-written adjoint, which walks
the updates backwards from a tape of the values each update overwrote.  The
discrete schedule is an input: it is not differentiated.
"""
from __future__ import annotations

import ctypes

import torch

from . import Code, _check, _load, _stream_ptr, decode, make_params


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class _WeightedBP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, llr, code, trace, counts, clip):
        B, N = llr.shape
        T = trace.shape[1]
        dev = llr.device
        L = torch.empty((B, N), dtype=torch.float32, device=dev)
        C = torch.empty((B, code.E), dtype=torch.float32, device=dev)
        tape = torch.empty((B, max(T, 1)), dtype=torch.float32, device=dev)
        s = torch.cuda.current_stream(dev)
        _check(_load().ldpc_wbp_forward(code._h, _p(llr), B, _p(trace), _p(counts), T, _p(w),
                                        ctypes.c_float(clip), _p(L), _p(C), _p(tape), _stream_ptr(s)))
        ctx.save_for_backward(w, llr, trace, C, tape)
        ctx.code, ctx.counts, ctx.clip = code, counts, clip
        return L

    @staticmethod
    def backward(ctx, gL):
        w, llr, trace, C, tape = ctx.saved_tensors
        B, N = llr.shape
        T = trace.shape[1]
        dev = llr.device
        gL = gL.contiguous().float()
        dwf = torch.empty((B, max(T, 1)), dtype=torch.float32, device=dev)
        dw = torch.empty(max(T, 1), dtype=torch.float32, device=dev)
        dllr = torch.empty((B, N), dtype=torch.float32, device=dev) if ctx.needs_input_grad[1] else None
        s = torch.cuda.current_stream(dev)
        _check(_load().ldpc_wbp_backward(ctx.code._h, _p(llr), B, _p(trace), _p(ctx.counts), T, _p(w),
                                         ctypes.c_float(ctx.clip), _p(C), _p(tape), _p(gL), _p(dwf), _p(dw),
                                         _p(dllr), _stream_ptr(s)))
        return dw[:T], dllr, None, None, None, None


def weighted_bp(code: Code, llr: torch.Tensor, trace: torch.Tensor, weights: torch.Tensor, *,
                counts: torch.Tensor | None = None, clip: float = 25.0) -> torch.Tensor:
    """Final LLRs [batch, N] of the weighted replay of `trace` ([batch, T] int32
    edge ids) with `weights` ([T] float32); differentiable in `weights` and
    `llr` (float32 [batch, N])."""
    for name, t, dt in [("llr", llr, torch.float32), ("trace", trace, torch.int32), ("weights", weights, torch.float32)]:
        if not t.is_cuda or not t.is_contiguous() or t.dtype != dt:
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor")
    if counts is not None and (not counts.is_cuda or counts.dtype != torch.int64):
        raise ValueError("counts must be a CUDA int64 tensor")
    return _WeightedBP.apply(weights, llr, code, trace, counts, float(clip))


def bce_all_zero(L: torch.Tensor) -> torch.Tensor:
    """Mean binary cross-entropy of the bit posteriors p0 = sigmoid(L) against
    the all-zero codeword: mean(log(1 + e^-L))."""
    return torch.nn.functional.softplus(-L).mean()


def record_schedule(code: Code, llr: torch.Tensor, updates: int, schedule: str = "lmd-cirbp", **kw):
    """Run a CI schedule for exactly `updates` committed messages (no syndrome
    stop) and return its trace [batch, updates] (int32)."""
    p = make_params(schedule, "fp32", max_updates=updates, check_interval=0, **kw)
    out = decode(code, llr, p, want_trace=True)
    return out["trace"], out["updates"]
