"""Empirical J(gamma) and F(gamma) of the CI metric (Properties 1 and 2,
Sec. 3.A) on flooding BP, through the library's counter kernel.

In flooding BP the precomputed total LLR of a variable node after iteration k
is its total after iteration k + 1, so the pair (L, L~) of iteration k is
(L^(k), L^(k+1)) with L^(0) = lambda.  The all-zero codeword is sent.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import Code, _check, _load, _stream_ptr, decode, make_params


def pair_counts(llr_now: torch.Tensor, llr_pre: torch.Tensor, n_bins: int) -> np.ndarray:
    """ldpc_ci_stats over two equal-shape float32 CUDA tensors: [n_bins, 4] counts."""
    a, b = llr_now.contiguous(), llr_pre.contiguous()
    if a.shape != b.shape or a.dtype != torch.float32 or b.dtype != torch.float32 or not a.is_cuda:
        raise ValueError("two float32 CUDA tensors of one shape are required")
    out = torch.empty((n_bins, 4), dtype=torch.int64, device=a.device)
    s = torch.cuda.current_stream(a.device)
    _check(_load().ldpc_ci_stats(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), a.numel(), n_bins,
                                 ctypes.c_void_p(out.data_ptr()), _stream_ptr(s)))
    return out.cpu().numpy()


def flooding_counts(code: Code, llr: torch.Tensor, iterations: int, n_bins: int = 20) -> np.ndarray:
    """Counts [iterations, n_bins, 4] for iterations k = 0 .. iterations-1."""
    Ls = [llr.float()]
    for k in range(1, iterations + 1):
        p = make_params("flooding", "fp32", max_updates=k * code.E, check_interval=0)
        Ls.append(decode(code, llr, p, want_llr=True)["llr"])
    return np.stack([pair_counts(Ls[k], Ls[k + 1], n_bins) for k in range(iterations)])


def j_and_f(counts: np.ndarray):
    """Cumulate from the top bin: J[b] = #correct / #incorrect and
    F[b] = #(incorrect, moving toward the truth) / #(incorrect, moving away)
    over D >= b / n_bins (inf where the denominator is 0, nan where both are)."""
    c = np.cumsum(counts[..., ::-1, :], axis=-2)[..., ::-1, :].astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return c[..., 0] / c[..., 1], c[..., 2] / c[..., 3]
