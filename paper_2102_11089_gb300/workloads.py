"""Seeded synthetic workloads: stand-in LDPC code designs and channel LLR batches.

This module holds no decoding arithmetic.  It produces the *inputs* that both the
CUDA library and the CPU oracle consume:

* parity-check graphs as edge lists (a seeded random regular code) or as
  protographs with circulant shifts (the QC codes; lifting them into edge lists
  is done separately by the library and by the oracle);
* batches of channel LLRs drawn with numpy's PCG64 generator (BPSK over AWGN,
  all-zero codeword), used as common inputs for parity tests.

The paper evaluates on the IEEE 802.11 (1944,972) code and on 5G NR base-graph
codes (Sec. 5).  Their base matrices are not reproduced here; the designs below
are seeded stand-ins with the same shapes: a 12x24 dual-diagonal rate-1/2
protograph (WiFi-like), a 42x52 BG2-shaped and a 46x68 BG1-shaped protograph
with two punctured systematic columns and degree-1 extension parity columns.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "QCDesign", "regular_code", "wifi_like", "bg2_like", "bg1_like",
    "sigma2_from_ebn0", "seeded_llrs", "quantize_llrs", "gf2_rank",
    "qc_edges_reference_free", "WORKLOADS",
]


# ---------------------------------------------------------------------------
# helpers


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _four_cycle_cost(cn: np.ndarray, vn: np.ndarray, m: int, n: int,
                     cycles_too: bool = True) -> tuple[int, np.ndarray]:
    """Number of double edges (+ 4-cycles), and a mask of edges that take part in one."""
    cnt = np.zeros((m, n), dtype=np.int64)
    np.add.at(cnt, (cn, vn), 1)
    doubles = int(np.maximum(cnt - 1, 0).sum())
    b = (cnt > 0).astype(np.int64)
    ov = b @ b.T
    np.fill_diagonal(ov, 0)
    cycles = int((ov * (ov - 1) // 2).sum() // 2)
    badpair = (ov >= 2).astype(np.int64)
    bad_cell = ((badpair @ b) > 0) & (b > 0)
    if not cycles_too:
        return doubles, cnt[cn, vn] > 1
    bad = bad_cell[cn, vn] | (cnt[cn, vn] > 1)
    return doubles + cycles, bad


# ---------------------------------------------------------------------------
# config 1: seeded regular code


def regular_code(n: int, dv: int, dc: int, seed: int, max_iter: int = 200000,
                 girth6: bool = True):
    """Random (dv, dc)-regular Tanner graph by socket permutation, with double
    edges (and, if ``girth6``, 4-cycles) removed by seeded endpoint swaps
    (degrees are kept).

    Returns ``(check_idx, var_idx, n_checks)`` as int32 arrays of the edges.
    """
    if (n * dv) % dc:
        raise ValueError("n*dv must be a multiple of dc")
    m = n * dv // dc
    rng = _rng(seed)
    vn = np.repeat(np.arange(n), dv)
    cn = np.repeat(np.arange(m), dc)[rng.permutation(n * dv)]
    cost, bad = _four_cycle_cost(cn, vn, m, n, girth6)
    it = 0
    while cost > 0 and it < max_iter:
        it += 1
        cand = np.flatnonzero(bad)
        a = int(cand[rng.integers(len(cand))])
        b = int(rng.integers(len(cn)))
        if cn[a] == cn[b]:
            continue
        trial = cn.copy()
        trial[a], trial[b] = cn[b], cn[a]
        c2, bad2 = _four_cycle_cost(trial, vn, m, n, girth6)
        if c2 <= cost:
            cn, cost, bad = trial, c2, bad2
    if cost > 0:
        raise RuntimeError(f"could not remove 4-cycles (cost {cost}) for n={n}")
    order = np.lexsort((vn, cn))
    return cn[order].astype(np.int32), vn[order].astype(np.int32), m


# ---------------------------------------------------------------------------
# QC designs


@dataclass
class QCDesign:
    """A protograph: ``base[r, c]`` is -1 (zero block) or a circulant shift.

    Shifts are stored for the largest lifting size and reduced modulo Z when a
    smaller lifting size is used (as the 5G NR base graphs do).
    """
    name: str
    base: np.ndarray
    punct_cols: list = field(default_factory=list)
    info_cols: int = 0

    def shifts(self, Z: int) -> np.ndarray:
        b = self.base.copy()
        nz = b >= 0
        b[nz] = b[nz] % Z
        return b.astype(np.int32)

    def sizes(self, Z: int) -> dict:
        rows, cols = self.base.shape
        n = cols * Z
        n_tx = n - len(self.punct_cols) * Z
        return dict(M=rows * Z, N=n, E=int((self.base >= 0).sum()) * Z,
                    K=self.info_cols * Z, N_tx=n_tx)

    def punct_mask(self, Z: int) -> np.ndarray:
        rows, cols = self.base.shape
        m = np.zeros(cols * Z, dtype=np.uint8)
        for c in self.punct_cols:
            m[c * Z:(c + 1) * Z] = 1
        return m


def _qc_cycles(base: np.ndarray, Z: int, redrawable: np.ndarray):
    """4-cycles of the lifted graph: rows r1<r2, cols c1<c2 all nonzero with
    s11 - s12 + s22 - s21 = 0 (mod Z).  Returns a list of redrawable cells."""
    rows, cols = base.shape
    out = []
    nz = base >= 0
    for r1 in range(rows):
        for r2 in range(r1 + 1, rows):
            common = np.flatnonzero(nz[r1] & nz[r2])
            if len(common) < 2:
                continue
            for i in range(len(common)):
                for j in range(i + 1, len(common)):
                    c1, c2 = common[i], common[j]
                    d = base[r1, c1] - base[r1, c2] + base[r2, c2] - base[r2, c1]
                    if d % Z == 0:
                        cells = [(r, c) for r, c in ((r1, c1), (r1, c2), (r2, c1), (r2, c2))
                                 if redrawable[r, c]]
                        out.append(cells)
    return out


def _draw_shifts(base: np.ndarray, redrawable: np.ndarray, Zmax: int, check_Z: list,
                 rng: np.random.Generator, max_rounds: int = 20000) -> np.ndarray:
    base = base.copy()
    idx = np.argwhere(redrawable)
    for r, c in idx:
        base[r, c] = rng.integers(Zmax)
    for _ in range(max_rounds):
        bad = []
        for Z in check_Z:
            bad += _qc_cycles(base, Z, redrawable)
        if not bad:
            return base
        for cells in bad:
            if cells:
                r, c = cells[rng.integers(len(cells))]
                base[r, c] = rng.integers(Zmax)
    raise RuntimeError("could not draw 4-cycle-free shifts")


def wifi_like(seed: int = 2, Z: int = 96) -> QCDesign:
    """12x24 rate-1/2 protograph: info columns of weight {6 (x7), 3 (x4), 2 (x1)},
    a weight-3 first parity column (top and bottom shifts equal, middle 0) and a
    dual-diagonal staircase of shift-0 blocks.  81 nonzero blocks."""
    rng = _rng(seed)
    B = -np.ones((12, 24), dtype=np.int64)
    s1 = int(rng.integers(1, Z))
    B[0, 12], B[6, 12], B[11, 12] = s1, 0, s1
    for k in range(1, 12):
        B[k - 1, 12 + k] = 0
        B[k, 12 + k] = 0
    weights = rng.permutation([6] * 7 + [3] * 4 + [2])
    rowcount = (B >= 0).sum(1)
    redraw = np.zeros_like(B, dtype=bool)
    for c, w in enumerate(weights):
        order = np.lexsort((rng.random(12), rowcount))
        rows = order[:w]
        B[rows, c] = 0
        redraw[rows, c] = True
        rowcount[rows] += 1
    B = _draw_shifts(B, redraw, Z, [Z], rng)
    return QCDesign("wifi-like-12x24", B, [], 12)


def _extension_design(rows: int, cols: int, n_info: int, core_info: int, ext_heavy: int,
                      k_heavy: int, k_light: int, seed: int, Zmax: int, name: str) -> QCDesign:
    """5G-NR-shaped protograph: 4 core rows over the info + 4 core parity
    columns, then (rows-4) extension rows each with its own degree-1 parity
    column.  The first two info columns are punctured and take part in most
    extension rows."""
    rng = _rng(seed)
    B = -np.ones((rows, cols), dtype=np.int64)
    redraw = np.zeros_like(B, dtype=bool)
    p0 = n_info  # first core parity column
    for r in range(4):
        others = rng.permutation(np.arange(2, n_info))[:core_info - 2]
        for c in [0, 1, *others]:
            B[r, c] = 0
            redraw[r, c] = True
    s = int(rng.integers(1, 16))
    B[0, p0], B[2, p0], B[3, p0] = s, 0, s
    for k in range(3):
        B[k, p0 + 1 + k] = 0
        B[k + 1, p0 + 1 + k] = 0
    for r in range(4, rows):
        B[r, p0 + 4 + (r - 4)] = 0
        k = k_heavy if r < 4 + ext_heavy else k_light
        first = (r - 4) % 2
        pool = rng.permutation(np.arange(2, p0 + 4))[:k - 1]
        for c in [first, *pool]:
            B[r, c] = 0
            redraw[r, c] = True
    B = _draw_shifts(B, redraw, Zmax, [Zmax], rng)
    return QCDesign(name, B, [0, 1], n_info)


def bg2_like(seed: int = 3) -> QCDesign:
    """42x52, 10 info columns (2 punctured), rate 1/5 after puncturing."""
    return _extension_design(42, 52, 10, 7, 10, 4, 3, seed, 384, "bg2-like-42x52")


def bg1_like(seed: int = 5) -> QCDesign:
    """46x68, 22 info columns (2 punctured), rate 1/3 after puncturing."""
    return _extension_design(46, 68, 22, 19, 12, 6, 4, seed, 384, "bg1-like-46x68")


def qc_edges_reference_free(design: QCDesign, Z: int):
    """Edge list of a lifted protograph, for building a code from Python when
    neither library is at hand (used by tests of the input module only)."""
    base = design.shifts(Z)
    chk, var = [], []
    rows, cols = base.shape
    z = np.arange(Z)
    for r in range(rows):
        for c in range(cols):
            if base[r, c] >= 0:
                chk.append(r * Z + z)
                var.append(c * Z + (z + base[r, c]) % Z)
    return np.concatenate(chk).astype(np.int32), np.concatenate(var).astype(np.int32)


# ---------------------------------------------------------------------------
# channel inputs for tests


def sigma2_from_ebn0(ebn0_db: float, rate: float) -> float:
    """Noise variance of unit-energy BPSK at Eb/N0 (N0/2 = sigma^2, Sec. 5)."""
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def seeded_llrs(n: int, batch: int, sigma2: float, seed: int,
                punct: np.ndarray | None = None) -> np.ndarray:
    """Channel LLRs 2y/sigma^2 of the all-zero codeword (x = +1) over AWGN,
    float32 [batch, n]; punctured positions carry 0."""
    rng = _rng(seed)
    y = 1.0 + math.sqrt(sigma2) * rng.standard_normal((batch, n))
    lam = (2.0 * y / sigma2).astype(np.float32)
    if punct is not None:
        lam[:, np.asarray(punct, dtype=bool)] = 0.0
    return lam


def quantize_llrs(lam: np.ndarray, q_step: float) -> np.ndarray:
    """6-bit symmetric quantiser q = clamp(rint(lam / step), -31, 31), taken in
    float32 like the channel kernel."""
    q = np.rint(lam.astype(np.float32) / np.float32(q_step))
    return np.clip(q, -31, 31).astype(np.int8)


def gf2_rank(check_idx, var_idx, m: int) -> int:
    """Rank of H over GF(2) (rows as Python integers)."""
    rows = [0] * m
    for c, v in zip(np.asarray(check_idx).tolist(), np.asarray(var_idx).tolist()):
        rows[c] ^= 1 << v
    rank = 0
    pivots = {}
    for r in rows:
        while r:
            h = r.bit_length() - 1
            if h in pivots:
                r ^= pivots[h]
            else:
                pivots[h] = r
                rank += 1
                break
    return rank


# ---------------------------------------------------------------------------
# named workloads (the synthetic stand-ins of the paper's evaluation setups)

WORKLOADS = {
    # regular (3,6), n=96: all-zero codeword at 2.0 dB, 1000 frames, budget 10 E
    "regular-3-6-n96": dict(kind="regular", n=96, dv=3, dc=6, seed=1, k_info=48,
                            ebn0_db=2.0, frames=1000, budget_iters=10),
    # WiFi-like rate-1/2 QC code, Z=96 (n=2304)
    "wifi-like-n2304": dict(kind="qc", design="wifi", seed=2, Z=96,
                            ebn0_sweep=[1.0, 1.25, 1.5, 1.75, 2.0, 2.25, 2.5],
                            frames=65536, n_p=[4, 16, 64], n_g=[4, 8, 16]),
    # BG2-shaped, lifting sizes mixed, n up to 19,968
    "bg2-like-mixed": dict(kind="qc", design="bg2", seed=3, Z=[16, 32, 64, 128, 256, 384],
                           ebn0_range=[0.5, 3.0], budget_iters=[2, 20], frames=10 ** 6),
    # BG1-shaped, Z=384 (n=26,112)
    "bg1-like-n26112": dict(kind="qc", design="bg1", seed=5, Z=384,
                            ebn0_sweep=[0.8, 1.0, 1.2, 1.4, 1.6], n_p=[64, 256]),
}


def design(name: str, seed: int | None = None, Z: int | None = None) -> QCDesign:
    if name == "wifi":
        return wifi_like(2 if seed is None else seed, 96 if Z is None else Z)
    if name == "bg2":
        return bg2_like(3 if seed is None else seed)
    if name == "bg1":
        return bg1_like(5 if seed is None else seed)
    raise KeyError(name)
