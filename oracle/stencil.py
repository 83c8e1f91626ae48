"""Finite-difference operators of Sec. 2.2 (oracle; test infrastructure only).

* ``D``: the standard 8th-order centred first derivative (the paper uses a
  "standard 8th order stencil" for first derivatives; its weights are the
  Taylor-series ones 4/5, -1/5, 4/105, -1/280).
* ``narrow``: (a u_x)_x ~ (H_{i+1/2} - H_{i-1/2}) / dx^2 with
  H_{i+1/2} = sum_{m,n=-s+1..s} a_{i+m} M_{mn} u_{i+n}   (eqs. DaDu, H),
  M the 8x8 matrix of Sec. 2.2 (s = 4) or the 6x6 one (s = 3).

Arrays carry ``g`` ghost cells on each side of the differenced axis; the
result covers the interior only (``g`` cells trimmed from each end).
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np

# Default free parameters of the 8th-order stencil ("SMC", Sec. 2.2) and the
# two alternatives of App. A ("ZERO", "OPTIMAL").
M47_SMC, M48_SMC = Fr(3557, 44100), Fr(-2083, 117600)
M47_ZERO, M48_ZERO = Fr(0), Fr(0)
M47_OPT, M48_OPT = Fr(1059283, 13608000), Fr(-856481, 40824000)
M36_SMC = Fr(281, 3600)

D8 = (Fr(4, 5), Fr(-1, 5), Fr(4, 105), Fr(-1, 280))


def narrow8_exact(m47=M47_SMC, m48=M48_SMC):
    """The 8x8 M of Sec. 2.2 as exact rationals; rows m = -3..4, cols n = -3..4.

    Upper four rows from the printed m_ij formulas; the lower four rows are
    the printed sign-flipped reversals of the upper ones.
    """
    m47, m48 = Fr(m47), Fr(m48)
    m = {}
    m[1, 1] = Fr(5, 336) + m48
    m[1, 2] = Fr(-83, 3600) - Fr(1, 5) * m47 - Fr(14, 5) * m48
    m[1, 3] = Fr(299, 50400) + Fr(2, 5) * m47 + Fr(13, 5) * m48
    m[1, 4] = Fr(17, 12600) - Fr(1, 5) * m47 - Fr(4, 5) * m48
    m[1, 5] = Fr(1, 1120)
    m[2, 1] = Fr(-11, 560) - 2 * m48
    m[2, 2] = Fr(-31, 360) + m47 + 3 * m48
    m[2, 3] = Fr(41, 200) - Fr(9, 5) * m47 + Fr(4, 5) * m48
    m[2, 4] = Fr(-5927, 50400) + Fr(4, 5) * m47 - Fr(9, 5) * m48
    m[2, 5] = Fr(17, 600) - Fr(1, 5) * m47 - Fr(4, 5) * m48
    m[2, 6] = Fr(-503, 50400) + Fr(1, 5) * m47 + Fr(4, 5) * m48
    m[3, 1] = Fr(-1, 280)
    m[3, 2] = Fr(1097, 5040) - 2 * m47 + 6 * m48
    m[3, 3] = Fr(-1349, 10080) + 3 * m47 - 12 * m48
    m[3, 4] = Fr(-887, 5040) - m47 + 6 * m48
    m[3, 5] = Fr(3613, 50400) + Fr(4, 5) * m47 - Fr(9, 5) * m48
    m[3, 6] = Fr(467, 25200) - Fr(3, 5) * m47 + Fr(18, 5) * m48
    m[3, 7] = Fr(139, 25200) - Fr(1, 5) * m47 - Fr(9, 5) * m48
    m[4, 1] = Fr(17, 1680) + 2 * m48
    m[4, 2] = Fr(-319, 2520) + 2 * m47 - 8 * m48
    m[4, 3] = Fr(-919, 5040) - 2 * m47 + 6 * m48
    m[4, 4] = Fr(-445, 2016)
    m[4, 5] = Fr(583, 720) - m47 + 6 * m48
    m[4, 6] = Fr(-65, 224) - 7 * m48
    m[4, 7] = m47
    m[4, 8] = m48
    M = [[Fr(0)] * 8 for _ in range(8)]
    for (r, c), v in m.items():
        M[r - 1][c - 1] = v
    # rows 5..8: row 9-r is minus row r read backwards
    for r in range(4):
        for c in range(8):
            M[7 - r][7 - c] = -M[r][c]
    return M


def narrow6_exact(m36=M36_SMC):
    """The 6x6 M of Sec. 2.2 (6th order, s = 3) as exact rationals."""
    m36 = Fr(m36)
    m = {}
    m[1, 1] = Fr(-11, 180) + m36
    m[1, 2] = Fr(1, 9) - 2 * m36
    m[1, 3] = Fr(-1, 18) + m36
    m[1, 4] = Fr(1, 180)
    m[2, 1] = Fr(7, 60) - 3 * m36
    m[2, 2] = Fr(-1, 120) + 5 * m36
    m[2, 3] = Fr(-17, 90) - 2 * m36
    m[2, 4] = Fr(5, 72) + m36
    m[2, 5] = Fr(1, 90) - m36
    m[3, 1] = Fr(-1, 15) + 3 * m36
    m[3, 2] = Fr(-11, 60) - 3 * m36
    m[3, 3] = Fr(-101, 360)
    m[3, 4] = Fr(137, 180) - 2 * m36
    m[3, 5] = Fr(-83, 360) + m36
    m[3, 6] = m36
    M = [[Fr(0)] * 6 for _ in range(6)]
    for (r, c), v in m.items():
        M[r - 1][c - 1] = v
    for r in range(3):
        for c in range(6):
            M[5 - r][5 - c] = -M[r][c]
    return M


def to_float(M, dtype=np.float64) -> np.ndarray:
    """Exact rationals -> floating point (float64, or np.longdouble for the
    extended-precision check of ill-conditioned components)."""
    t = np.dtype(dtype).type
    return np.array([[t(v.numerator) / t(v.denominator) for v in row] for row in M], dtype=dtype)


def _take(f: np.ndarray, axis: int, start: int, length: int) -> np.ndarray:
    idx = [slice(None)] * f.ndim
    idx[axis] = slice(start, start + length)
    return f[tuple(idx)]


def D(f: np.ndarray, axis: int, h: float, g: int = 4) -> np.ndarray:
    """8th-order centred first derivative along ``axis``; trims g ghosts."""
    n = f.shape[axis] - 2 * g
    t = f.dtype.type
    out = np.zeros(_take(f, axis, g, n).shape, dtype=f.dtype)
    for k, c in enumerate(D8, start=1):
        out = out + (t(c.numerator) / t(c.denominator)) * (_take(f, axis, g + k, n) - _take(f, axis, g - k, n))
    return out / h


def narrow(a: np.ndarray, u: np.ndarray, axis: int, h: float, M: np.ndarray,
           g: int = 4) -> np.ndarray:
    """(a u_x)_x by eqs. DaDu/H with a 2s x 2s matrix M; trims g >= s ghosts.

    Interior cell i (0-based) has faces i-1/2 and i+1/2.  Face i+1/2 uses
    cells i-s+1 .. i+s.  The 1/dx^2 of eq. DaDu is applied last.
    """
    s = M.shape[0] // 2
    n = a.shape[axis] - 2 * g
    nf = n + 1                       # faces -1/2 .. n-1/2
    H = np.zeros(_take(a, axis, 0, nf).shape, dtype=np.result_type(a, u, M))
    # face f (= i+1/2 with i = f-1) sits between ghosted indices g+f-1 and g+f
    for mi in range(2 * s):
        m = mi - s + 1
        a_m = _take(a, axis, g - 1 + m, nf)
        for ni in range(2 * s):
            if M[mi, ni] == 0.0:
                continue
            nn = ni - s + 1
            H = H + a_m * M[mi, ni] * _take(u, axis, g - 1 + nn, nf)
    return (_take(H, axis, 1, n) - _take(H, axis, 0, n)) / (h * h)


def wide(a: np.ndarray, u: np.ndarray, axis: int, h: float) -> np.ndarray:
    """The wide alternative D(a D u) (Sec. 1), needs 8 ghosts; comparison only."""
    du = D(u, axis, h, g=4)          # 4 ghosts left
    return D(_take(a, axis, 4, du.shape[axis]) * du, axis, h, g=4)
