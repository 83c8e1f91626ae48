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


# ------------------------------------------------------------ boundaries
# Near a non-periodic boundary (Sec. 2.2, boundary paragraph) the stencils
# are lowered: the fourth cell from the boundary (index 3 counted from it)
# uses 6th-order centred stencils, the third (index 2) 4th-order centred
# ones, the second (index 1) the centred 2nd-order diffusion and a biased
# 3rd-order advection stencil, and the boundary cell (index 0) completely
# biased stencils: 2nd order for diffusion, 3rd order for advection.  Only
# cells inside the domain are read.

D6 = (Fr(3, 4), Fr(-3, 20), Fr(1, 60))
D4 = (Fr(2, 3), Fr(-1, 12))
# one-sided first derivatives from the four cells nearest the boundary,
# exact on cubics: at the cell next to it (biased) and at it (completely biased)
DB1 = (Fr(-2, 6), Fr(-3, 6), Fr(6, 6), Fr(-1, 6))
DB0 = (Fr(-11, 6), Fr(18, 6), Fr(-9, 6), Fr(2, 6))

# Free parameters of the 4th-order narrow stencil.  Polynomial exactness
# (deg a + deg u <= 5), zero row sums and the antisymmetry of the 8th- and
# 6th-order matrices leave two parameters p = M[3][1], q = M[3][2].  The
# paper's rule (minimise the sum of the absolute leading truncation
# coefficients) reproduces its own 6th- and 8th-order choices but leaves a
# triangle of optima here; minimising the next-order coefficients on it
# leaves an edge (q = 1/72), whose midpoint p = -1/9 is taken.
M4_P, M4_Q = Fr(-1, 9), Fr(1, 72)


def narrow4_exact(p=M4_P, q=M4_Q):
    """The 4x4 M of the 4th-order narrow stencil (s = 2), rows and columns
    -1..2, in terms of its two free parameters."""
    p, q = Fr(p), Fr(q)
    return [[-q, -p, 2 * p + 3 * q + Fr(1, 12), -p - 2 * q - Fr(1, 12)],
            [p + 4 * q + Fr(1, 6), -3 * q - Fr(3, 4), -3 * p - 6 * q + Fr(5, 12), 2 * p + 5 * q + Fr(1, 6)],
            [-2 * p - 5 * q - Fr(1, 6), 3 * p + 6 * q - Fr(5, 12), 3 * q + Fr(3, 4), -p - 4 * q - Fr(1, 6)],
            [p + 2 * q + Fr(1, 12), -2 * p - 3 * q - Fr(1, 12), p, q]]


def narrow2_exact():
    """The centred 2nd-order flux H_{i+1/2} = (a_i + a_{i+1})/2 (u_{i+1} - u_i)
    as a 2x2 M."""
    return [[Fr(-1, 2), Fr(1, 2)], [Fr(-1, 2), Fr(1, 2)]]


def _last(f, axis):
    return np.moveaxis(f, axis, -1)


def D_bc(f: np.ndarray, axis: int, h: float, g: int = 4) -> np.ndarray:
    """First derivative along ``axis`` whose two ends are non-periodic
    boundaries: D8 in the interior, lowered at the four cells next to each
    end.  ``f`` carries g ghosts along the axis, which are never read by
    the lowered cells (the interior cells never reach them either)."""
    out = D(f, axis, h, g)
    n = out.shape[axis]
    t = f.dtype.type
    c = lambda r: t(r.numerator) / t(r.denominator)
    fi = _last(_take(f, axis, g, n), axis)        # the domain's cells, axis last
    o = _last(out, axis)                          # a view: writes go to out
    for side in (0, 1):
        v = fi if side == 0 else fi[..., ::-1]    # mirrored for the high end
        sgn = 1.0 if side == 0 else -1.0
        k = (lambda j: j) if side == 0 else (lambda j: n - 1 - j)
        o[..., k(0)] = sgn * sum(c(w) * v[..., j] for j, w in enumerate(DB0)) / h
        o[..., k(1)] = sgn * sum(c(w) * v[..., j] for j, w in enumerate(DB1)) / h
        o[..., k(2)] = sgn * sum(c(w) * (v[..., 2 + j + 1] - v[..., 2 - j - 1]) for j, w in enumerate(D4)) / h
        o[..., k(3)] = sgn * sum(c(w) * (v[..., 3 + j + 1] - v[..., 3 - j - 1]) for j, w in enumerate(D6)) / h
    return out


def narrow_bc(a: np.ndarray, u: np.ndarray, axis: int, h: float, M8: np.ndarray,
              g: int = 4) -> np.ndarray:
    """(a u_x)_x along ``axis`` with non-periodic ends: the 8th-order narrow
    stencil in the interior, the 6th-, 4th- and 2nd-order narrow stencils at
    the fourth, third and second cells from each end, and at the end cell
    a u_xx + a_x u_x from one-sided 2nd-order differences,
      u_xx ~ (2 u0 - 5 u1 + 4 u2 - u3)/h^2,  u_x ~ (-3 u0 + 4 u1 - u2)/(2h),
    the same for a_x (mirrored at the high end)."""
    out = narrow(a, u, axis, h, M8, g)
    n = out.shape[axis]
    dt = np.result_type(a, u, M8)
    ai = _take(a, axis, g, n)
    ui = _take(u, axis, g, n)
    o = _last(out, axis)
    for s, M in ((3, narrow6_exact()), (2, narrow4_exact()), (1, narrow2_exact())):
        r = _last(narrow(ai, ui, axis, h, to_float(M, dt), g=s), axis)   # cells s .. n-1-s
        o[..., s] = r[..., 0]
        o[..., n - 1 - s] = r[..., -1]
    al, ul = _last(ai, axis), _last(ui, axis)
    for side in (0, 1):
        av = al if side == 0 else al[..., ::-1]
        uv = ul if side == 0 else ul[..., ::-1]
        uxx = 2 * uv[..., 0] - 5 * uv[..., 1] + 4 * uv[..., 2] - uv[..., 3]
        ux = -3 * uv[..., 0] + 4 * uv[..., 1] - uv[..., 2]
        ax_ = -3 * av[..., 0] + 4 * av[..., 1] - av[..., 2]
        o[..., 0 if side == 0 else n - 1] = (av[..., 0] * uxx + 0.25 * ax_ * ux) / (h * h)
    return out
