"""Seeded synthetic inputs: mechanisms, box layouts and primitive fields.

This module only *draws* inputs.  It evaluates none of the method's
arithmetic (no equation of state, no thermodynamic or transport property,
no rate, no stencil).  Both the CUDA library and the CPU oracle receive
what it produces as plain arrays.

Everything is CGS: cm, g, s, K, erg; activation energies in cal/mol.

Synthetic mechanisms stand in for the named mechanisms of the paper's
experiments (9-species H2/O2, GRI-Mech 3.0, DME-39), which are not used.

Recipe (all draws from ``numpy.random.default_rng(seed)``):

* Species are abstract molecules built from abstract elements.  With at most
  four species one element is used (A, A2, A3, A4); up to 15 species, two
  elements with compositions drawn from the lattice {0..3}^2; otherwise
  three elements from {0,1,2}^3 ({0..3}^3 beyond 26 species).  The single
  atoms are always present.  Molecular weights are the sums of the element
  weights, so every element-balanced reaction conserves mass exactly.
* Reactions have one or two distinct species per side, stoichiometric
  coefficients in {1, 2} and at most three molecules per side; both sides
  carry the same element counts.  Each reaction is written in the direction
  whose enthalpy offsets sum (``sum nu * a6``) is not positive.
* NASA-7 (single range): ``cp/R = c0 + c1 tau (1 - tau/7) + c3 tau^3 + c4
  tau^4`` with ``tau = T/1000``, ``c0 = 2.5 + 0.4 (atoms - 1) + U[0.15, 0.6]``,
  ``c1 ~ U[0, 1]``, ``c3 ~ U[0, 0.01]``, ``c4 ~ U[-0.001, 0]``; this keeps
  cp/R inside [2.5, 8] on 200..3500 K by construction.  ``a6`` (enthalpy
  offset, K) is element-additive plus U[-2500, 2500] K; ``a7`` is
  ``s0 - a1 ln(1000)`` with ``s0`` element-additive plus U[-1, 1].
* Arrhenius parameters: log10 A ~ U[8, 14] (mol, cm, s units), b ~ U[-1, 2],
  Ea ~ U[0, 40000] cal/mol.  A draw is kept only if the forward pseudo
  first-order rate bound ``A T^b exp(-Ea/(Rc T)) * ctot^(order-1)`` stays
  below ``kmax`` (default 1e6 1/s) for T on a 300..2000 K grid, ``ctot`` the
  ideal-gas molar concentration at 1 atm; otherwise all three are redrawn.
  This screen keeps the explicit (forward-Euler-substepped) integrators
  stable at acoustic time steps.
* Transport: Lewis numbers ~ U[0.3, 2]; eta_ref = 1.85e-4 g/(cm s) at
  T_ref = 300 K, exponent 0.7; Prandtl number 0.72.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

P_ATM = 1.01325e6            # dyn/cm^2
R_CAL = 1.98720425864083     # cal/(mol K), used only by the stiffness screen
R_ERG = 8.31446261815324e7   # erg/(mol K), used only by the stiffness screen


# --------------------------------------------------------------------------
# mechanisms
# --------------------------------------------------------------------------

@dataclass
class Mechanism:
    W: np.ndarray            # [ns] g/mol
    nasa7: np.ndarray        # [ns, 7]
    nu_f: np.ndarray         # [nr, ns] int32, reactant coefficients
    nu_r: np.ndarray         # [nr, ns] int32, product coefficients
    A: np.ndarray            # [nr]
    b: np.ndarray            # [nr]
    Ea: np.ndarray           # [nr] cal/mol
    Le: np.ndarray           # [ns]
    eta_ref: float = 1.85e-4
    T_ref: float = 300.0
    eta_exp: float = 0.7
    Pr: float = 0.72
    composition: np.ndarray = field(default=None)  # [ns, ne] element counts

    @property
    def ns(self) -> int:
        return int(self.W.shape[0])

    @property
    def nr(self) -> int:
        return int(self.A.shape[0])


def _compositions(ns: int, rng) -> tuple[np.ndarray, np.ndarray]:
    if ns <= 4:
        weights = np.array([14.007])
        comps = [(k + 1,) for k in range(ns)]
        return np.array(comps, dtype=np.int64), weights
    if ns <= 15:
        weights = np.array([1.008, 15.999])
        ne, span = 2, 4
    else:
        weights = np.array([1.008, 12.011, 15.999])
        ne, span = 3, (3 if ns <= 26 else 4 if ns <= 63 else 5)
    atoms = [tuple(1 if i == j else 0 for i in range(ne)) for j in range(ne)]
    lattice = [v for v in itertools.product(range(span), repeat=ne)
               if sum(v) > 0 and v not in atoms]
    order = rng.permutation(len(lattice))
    chosen = atoms + [lattice[i] for i in order[: ns - ne]]
    if len(chosen) < ns:
        raise ValueError(f"cannot draw {ns} distinct species compositions")
    return np.array(chosen, dtype=np.int64), weights


def _sides(ns: int):
    """All reaction sides: 1 or 2 distinct species, coefficients 1..2, <= 3 molecules."""
    out = []
    for k in range(ns):
        for c in (1, 2):
            out.append(((k, c),))
    for k, l in itertools.combinations(range(ns), 2):
        for ck in (1, 2):
            for cl in (1, 2):
                if ck + cl <= 3:
                    out.append(((k, ck), (l, cl)))
    return out


def _side_vector(side, comp):
    v = np.zeros(comp.shape[1], dtype=np.int64)
    for k, c in side:
        v += c * comp[k]
    return tuple(int(x) for x in v)


def _candidate_reactions(comp: np.ndarray):
    ns = comp.shape[0]
    by_elements: dict[tuple, list] = {}
    for s in _sides(ns):
        by_elements.setdefault(_side_vector(s, comp), []).append(s)
    cands = []
    for group in by_elements.values():
        for s1, s2 in itertools.combinations(group, 2):
            sp1 = {k for k, _ in s1}
            sp2 = {k for k, _ in s2}
            if sp1 & sp2:
                continue
            cands.append((s1, s2))
    return cands


def _thermo(comp: np.ndarray, rng) -> np.ndarray:
    ns, ne = comp.shape
    atoms = comp.sum(axis=1)
    beta_h = rng.uniform(-4000.0, 4000.0, size=ne)   # element enthalpy offsets, K
    beta_s = rng.uniform(5.0, 12.0, size=ne)         # element entropy offsets
    nasa = np.zeros((ns, 7))
    for k in range(ns):
        c0 = 2.5 + 0.4 * (atoms[k] - 1) + rng.uniform(0.15, 0.6)
        c1 = rng.uniform(0.0, 1.0)
        c3 = rng.uniform(0.0, 0.01)
        c4 = rng.uniform(-0.001, 0.0)
        a1 = c0
        a2 = c1 / 1.0e3
        a3 = -c1 / 7.0e6
        a4 = c3 / 1.0e9
        a5 = c4 / 1.0e12
        a6 = float(comp[k] @ beta_h) + rng.uniform(-2500.0, 2500.0)
        s0 = float(comp[k] @ beta_s) + rng.uniform(-1.0, 1.0)
        a7 = s0 - a1 * math.log(1000.0)
        nasa[k] = (a1, a2, a3, a4, a5, a6, a7)
    return nasa


def _rate_ok(logA10: float, b: float, Ea: float, order: int, kmax: float) -> bool:
    for T in np.linspace(300.0, 2000.0, 18):
        ctot = P_ATM / (R_ERG * T)
        lg = (logA10 + b * math.log10(T) - Ea / (R_CAL * T) / math.log(10.0)
              + (order - 1) * math.log10(ctot))
        if lg > math.log10(kmax):
            return False
    return True


def make_mechanism(ns: int, nr: int, seed: int, kmax: float = 1.0e6) -> Mechanism:
    """Seeded element-balanced reversible mechanism with ns species, nr reactions."""
    rng = np.random.default_rng(seed)
    comp, elw = _compositions(ns, rng)
    W = comp.astype(np.float64) @ elw
    nasa = _thermo(comp, rng)
    cands = _candidate_reactions(comp)
    if len(cands) < nr:
        raise ValueError(f"only {len(cands)} balanced reactions exist for {ns} species")
    pick = rng.permutation(len(cands))[:nr]
    nu_f = np.zeros((nr, ns), dtype=np.int32)
    nu_r = np.zeros((nr, ns), dtype=np.int32)
    A = np.zeros(nr)
    b = np.zeros(nr)
    Ea = np.zeros(nr)
    for r, ci in enumerate(pick):
        s1, s2 = cands[ci]
        d6 = sum(c * nasa[k, 5] for k, c in s2) - sum(c * nasa[k, 5] for k, c in s1)
        react, prod = (s1, s2) if d6 <= 0.0 else (s2, s1)
        for k, c in react:
            nu_f[r, k] = c
        for k, c in prod:
            nu_r[r, k] = c
        order = int(nu_f[r].sum())
        while True:
            lA = rng.uniform(8.0, 14.0)
            bb = rng.uniform(-1.0, 2.0)
            ea = rng.uniform(0.0, 40000.0)
            if _rate_ok(lA, bb, ea, order, kmax):
                break
        A[r] = 10.0 ** lA
        b[r] = bb
        Ea[r] = ea
    Le = rng.uniform(0.3, 2.0, size=ns)
    return Mechanism(W=W, nasa7=nasa, nu_f=nu_f, nu_r=nu_r, A=A, b=b, Ea=Ea,
                     Le=Le, composition=comp)


# --------------------------------------------------------------------------
# box layouts
# --------------------------------------------------------------------------

@dataclass
class Grid:
    domain: tuple            # (nx, ny, nz) global cells
    dx: tuple                # (hx, hy, hz) cm
    lo: np.ndarray           # [nboxes, 3] inclusive global lower corner (x, y, z)
    hi: np.ndarray           # [nboxes, 3] inclusive global upper corner

    @property
    def nboxes(self) -> int:
        return int(self.lo.shape[0])

    def box_shape(self, b: int) -> tuple:
        n = self.hi[b] - self.lo[b] + 1
        return int(n[0]), int(n[1]), int(n[2])

    def box_cells(self, b: int) -> int:
        nx, ny, nz = self.box_shape(b)
        return nx * ny * nz

    @property
    def ncells(self) -> int:
        return sum(self.box_cells(b) for b in range(self.nboxes))

    def offsets(self) -> np.ndarray:
        """Starting cell offset of each box in the concatenated box layout."""
        off = [0]
        for b in range(self.nboxes):
            off.append(off[-1] + self.box_cells(b))
        return np.array(off, dtype=np.int64)


def single_box(n, h) -> Grid:
    n = tuple(int(v) for v in (n if hasattr(n, "__len__") else (n, n, n)))
    h = tuple(float(v) for v in (h if hasattr(h, "__len__") else (h, h, h)))
    return Grid(domain=n, dx=h, lo=np.zeros((1, 3), dtype=np.int64),
                hi=np.array([[n[0] - 1, n[1] - 1, n[2] - 1]], dtype=np.int64))


def tiled_boxes(per_axis: int, edge_lo: int, edge_hi: int, h: float, seed: int) -> Grid:
    """per_axis^3 boxes tiling a periodic domain; each axis cut into seeded
    widths drawn uniformly from edge_lo..edge_hi (a BoxLib-style box array)."""
    rng = np.random.default_rng(seed)
    widths = [rng.integers(edge_lo, edge_hi + 1, size=per_axis) for _ in range(3)]
    starts = [np.concatenate([[0], np.cumsum(w)[:-1]]) for w in widths]
    lo, hi = [], []
    for kz in range(per_axis):
        for ky in range(per_axis):
            for kx in range(per_axis):
                l = (starts[0][kx], starts[1][ky], starts[2][kz])
                w = (widths[0][kx], widths[1][ky], widths[2][kz])
                lo.append(l)
                hi.append(tuple(a + b - 1 for a, b in zip(l, w)))
    domain = tuple(int(w.sum()) for w in widths)
    return Grid(domain=domain, dx=(h, h, h), lo=np.array(lo, dtype=np.int64),
                hi=np.array(hi, dtype=np.int64))


def global_to_boxes(grid: Grid, g: np.ndarray) -> np.ndarray:
    """[nc, Nz, Ny, Nx] global array -> [nc, ncells] concatenated box layout
    (each box [z][y][x], x fastest)."""
    nc = g.shape[0]
    out = np.empty((nc, grid.ncells), dtype=g.dtype)
    off = grid.offsets()
    for b in range(grid.nboxes):
        (x0, y0, z0), (x1, y1, z1) = grid.lo[b], grid.hi[b]
        blk = g[:, z0:z1 + 1, y0:y1 + 1, x0:x1 + 1]
        out[:, off[b]:off[b + 1]] = blk.reshape(nc, -1)
    return out


def boxes_to_global(grid: Grid, a: np.ndarray) -> np.ndarray:
    nc = a.shape[0]
    nx, ny, nz = grid.domain
    g = np.full((nc, nz, ny, nx), np.nan)
    off = grid.offsets()
    for b in range(grid.nboxes):
        (x0, y0, z0), (x1, y1, z1) = grid.lo[b], grid.hi[b]
        bx, by, bz = grid.box_shape(b)
        g[:, z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] = a[:, off[b]:off[b + 1]].reshape(nc, bz, by, bx)
    return g


# --------------------------------------------------------------------------
# primitive fields: prim = [u, v, w, T, p, Y_1..Y_ns] on the global grid
# --------------------------------------------------------------------------

def _coords(grid: Grid):
    nx, ny, nz = grid.domain
    hx, hy, hz = grid.dx
    x = (np.arange(nx) + 0.5) * hx
    y = (np.arange(ny) + 0.5) * hy
    z = (np.arange(nz) + 0.5) * hz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    L = (nx * hx, ny * hy, nz * hz)
    return X, Y, Z, L


def _smooth_mode(rng, X, Y, Z, L, kmax=2):
    """Product of sin/cos of integer modes 1..kmax with random phases; in [-1, 1]."""
    f = np.ones_like(X)
    for C, Ld in ((X, L[0]), (Y, L[1]), (Z, L[2])):
        k = rng.integers(1, kmax + 1)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        f = f * np.sin(2.0 * math.pi * k * C / Ld + ph)
    return f


def smooth_fields(grid: Grid, ns: int, seed: int, T0=1250.0, T1=250.0,
                  umax=5000.0, p_amp=0.0) -> np.ndarray:
    """Smooth periodic sinusoidal fields: T in T0 +- T1, p = 1 atm (times
    1 + p_amp * mode), |u| <= umax, Y_k positive sinusoids normalised to 1."""
    rng = np.random.default_rng(seed)
    X, Y, Z, L = _coords(grid)
    prim = np.empty((5 + ns,) + X.shape)
    for c in range(3):
        prim[c] = umax * _smooth_mode(rng, X, Y, Z, L)
    prim[3] = T0 + T1 * _smooth_mode(rng, X, Y, Z, L)
    prim[4] = P_ATM * (1.0 + p_amp * _smooth_mode(rng, X, Y, Z, L))
    raw = np.empty((ns,) + X.shape)
    for k in range(ns):
        raw[k] = rng.uniform(1.2, 2.0) + _smooth_mode(rng, X, Y, Z, L)
    prim[5:] = raw / raw.sum(axis=0)
    return prim


def bump_fields(grid: Grid, ns: int, seed: int, T0=1100.0, T1=400.0,
                v0=300.0, r0_frac=0.1) -> np.ndarray:
    """Gaussian temperature / pressure / composition bump with a Taylor-Green
    like velocity, after the design of the paper's convergence problem
    (Sec. 5.1), in a domain centred on the origin."""
    rng = np.random.default_rng(seed)
    X, Y, Z, L = _coords(grid)
    Xc, Yc, Zc = X - L[0] / 2, Y - L[1] / 2, Z - L[2] / 2
    r0 = r0_frac * L[0]
    g = np.exp(-(Xc ** 2 + Yc ** 2 + Zc ** 2) / r0 ** 2)
    prim = np.empty((5 + ns,) + X.shape)
    kx, ky, kz = (2 * math.pi / L[0], 2 * math.pi / L[1], 2 * math.pi / L[2])
    prim[0] = v0 * np.sin(kx * Xc) * np.cos(ky * Yc) * np.cos(kz * Zc)
    prim[1] = -v0 * np.cos(kx * Xc) * np.sin(ky * Yc) * np.cos(kz * Zc)
    prim[2] = 0.0
    prim[3] = T0 + T1 * g
    prim[4] = P_ATM * (1.0 + 0.1 * g)
    base = rng.uniform(0.5, 1.5, size=ns)
    amp = rng.uniform(-0.3, 0.3, size=ns)
    raw = base[:, None, None, None] * (1.0 + amp[:, None, None, None] * g[None])
    prim[5:] = raw / raw.sum(axis=0)
    return prim


def flame_fields(grid: Grid, ns: int, seed: int, Tu=300.0, Tb=2000.0,
                 delta_cells=8.0, ubase=1000.0, pert=0.03) -> np.ndarray:
    """Premixed planar-flame-like hot slab: two tanh fronts normal to x (so the
    profile is periodic), composition blended between seeded unburnt and burnt
    mixtures, base velocity ubase in x plus seeded perturbations of relative
    size pert."""
    rng = np.random.default_rng(seed)
    X, Y, Z, L = _coords(grid)
    d = delta_cells * grid.dx[0]
    phi = 0.5 * (np.tanh((X - 0.25 * L[0]) / d) - np.tanh((X - 0.75 * L[0]) / d))
    prim = np.empty((5 + ns,) + X.shape)
    prim[3] = Tu + (Tb - Tu) * phi
    prim[4] = P_ATM
    for c in range(3):
        base = ubase if c == 0 else 0.0
        prim[c] = base + pert * ubase * _smooth_mode(rng, X, Y, Z, L, kmax=3)
    yu = rng.uniform(0.2, 1.0, size=ns)
    yb = rng.uniform(0.2, 1.0, size=ns)
    yu /= yu.sum()
    yb /= yb.sum()
    prim[5:] = (yu[:, None, None, None] * (1.0 - phi[None])
                + yb[:, None, None, None] * phi[None])
    return prim


def spectral_velocity(grid: Grid, seed: int, rms: float, slope: float = -5.0 / 3.0,
                      kmin: int = 1, kmax: int | None = None) -> np.ndarray:
    """A seeded random-phase solenoidal velocity field [3, nz, ny, nx] on the
    periodic box with energy spectrum E(k) ~ k^slope on kmin <= |k| <= kmax
    (mode numbers), scaled to the given rms (over the three components, one
    factor, so the field stays divergence-free).  Fourier
    amplitudes |u(k)| ~ sqrt(E(k) / (4 pi k^2)); the divergence-free part is
    kept by projecting out k (k . u(k))/|k|^2."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid.domain
    kx = np.fft.fftfreq(nx, 1.0 / nx)
    ky = np.fft.fftfreq(ny, 1.0 / ny)
    kz = np.fft.rfftfreq(nz, 1.0 / nz)
    KY, KX, KZ = np.meshgrid(ky, kx, kz, indexing="ij")    # [ny, nx, nz//2+1]
    kmag = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    kmax = kmax or max(1, min(nx, ny, nz) // 4)
    amp = np.zeros_like(kmag)
    band = (kmag >= kmin) & (kmag <= kmax)
    amp[band] = np.sqrt(kmag[band] ** slope / (4.0 * np.pi * kmag[band] ** 2))
    uh = []
    for _ in range(3):
        ph = rng.uniform(0.0, 2.0 * np.pi, size=kmag.shape)
        uh.append(amp * np.exp(1j * ph))
    k2 = np.where(kmag > 0, kmag ** 2, 1.0)
    div = (KX * uh[0] + KY * uh[1] + KZ * uh[2]) / k2
    uh = [uh[0] - KX * div, uh[1] - KY * div, uh[2] - KZ * div]
    out = np.empty((3, nz, ny, nx))
    for c in range(3):
        # the transform runs over [y][x][z]; the result is laid out [z][y][x]
        f = np.fft.irfftn(uh[c], s=(ny, nx, nz), axes=(0, 1, 2))
        out[c] = np.transpose(f, (2, 0, 1))
    out *= rms / np.sqrt(np.mean(out ** 2))
    return out


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    grid: Grid
    mech: Mechanism
    prim: np.ndarray         # [NV, ncells] concatenated box layout
    dt: float
    nodes: int
    sweeps: int
    reaction_substeps: int
    steps: int
    precision: str
    x_outflow: bool = False  # non-periodic x ends (boundary-lowered stencils)


def _acoustic_dt(h: float, umax: float, Tmax: float, cfl: float = 0.5) -> float:
    # sound-speed bound for cp/R >= 2.5 gases of molecular weight >= 1
    c = math.sqrt(1.67 * R_ERG * Tmax / 1.0)
    return cfl * h / (umax + c)


def workload(name: str, seed: int = 1, n: int | None = None) -> Workload:
    """The five configurations, by name:

    c1  16^3 periodic, h = 1/16 cm, 3 species / 2 reactions, smooth fields,
        one RHS plus one SDC step (3 Gauss-Lobatto nodes, 4 sweeps), FP64.
    c2  64^3 periodic (n overrides), 9 species / 21 reactions, Gaussian bump,
        10 SDC steps, FP64.
    c3  256^3 periodic (n overrides), 9 species, planar hot slab, mixed
        precision, 20 steps.
    c4  64 boxes of 16..64 cells per edge tiling a periodic domain, 21 species
        / 84 reactions, smooth fields, MRSDC 3 coarse / 5 fine Gauss-Lobatto.
    c5  512 x 256 x 256, 21 species, hot slab (x outflow planned), mixed.
    """
    if name == "c1":
        nn = n or 16
        grid = single_box(nn, 1.0 / nn)
        mech = make_mechanism(3, 2, seed)
        g = smooth_fields(grid, 3, seed + 100, T0=1250.0, T1=250.0, umax=5000.0)
        dt = 0.5 * _acoustic_dt(grid.dx[0], 5000.0, 1500.0)
        return Workload(name, grid, mech, global_to_boxes(grid, g),
                        dt, 3, 4, 0, 1, "fp64")
    if name == "c2":
        nn = n or 64
        L = 0.1
        grid = single_box(nn, L / nn)
        mech = make_mechanism(9, 21, seed)
        g = bump_fields(grid, 9, seed + 100)
        dt = 0.5 * _acoustic_dt(grid.dx[0], 300.0, 1500.0)
        return Workload(name, grid, mech, global_to_boxes(grid, g), dt, 3, 4, 0, 10, "fp64")
    if name == "c3":
        nn = n or 256
        grid = single_box(nn, 1.0 / 256)
        mech = make_mechanism(9, 21, seed)
        g = flame_fields(grid, 9, seed + 100)
        dt = 0.5 * _acoustic_dt(grid.dx[0], 1100.0, 2000.0)
        return Workload(name, grid, mech, global_to_boxes(grid, g), dt, 3, 4, 0, 20, "mixed")
    if name == "c4":
        grid = tiled_boxes(4, 16, 64, 1.0 / 64, seed)
        if n is not None:
            grid = tiled_boxes(2, max(8, n // 2), n, 1.0 / 64, seed)
        mech = make_mechanism(21, 84, seed)
        g = smooth_fields(grid, 21, seed + 100, T0=1250.0, T1=250.0, umax=5000.0,
                          p_amp=0.02)
        dt = 0.5 * _acoustic_dt(grid.dx[0], 5000.0, 1500.0)
        return Workload(name, grid, mech, global_to_boxes(grid, g), dt, 3, 4, 5, 10, "mixed")
    if name == "c5":
        if n is None:
            grid = single_box((512, 256, 256), 1.0 / 256)
        else:
            grid = single_box((2 * n, n, n), 1.0 / 256)
        mech = make_mechanism(21, 84, seed)
        g = flame_fields(grid, 21, seed + 100, ubase=0.0, pert=0.0)
        # turbulent-like velocity: k^-5/3 spectrum, 10 m/s rms, over the flame
        g[0:3] = spectral_velocity(grid, seed + 200, rms=1000.0)
        dt = 0.5 * _acoustic_dt(grid.dx[0], 4000.0, 2000.0)
        return Workload(name, grid, mech, global_to_boxes(grid, g), dt, 5, 8, 5, 50, "mixed",
                        x_outflow=True)
    raise ValueError(f"unknown workload {name!r}")


# ------------------------------------------------------------------ App. A
def heat_fields(problem: str, N: int) -> dict:
    """Inputs of the appendix heat problems on the periodic square
    [0, 2 pi]^2 with x_i = 2 pi i / N (row-major [y][x]):
      T1: a = b = 1 + 0.1 cos x cos y, source exp(-t) G with
          G = (1 + 0.4 cos x cos y) sin x sin y (exact u = exp(-t) sin x sin y);
      T2: a = 1 + 0.9 cos 2x sin(2y + pi/3), b = 1 + 0.9 cos(2x + pi/3) sin 2y,
          no source.
    u0 = sin x sin y for both.  Returns dict(h, a, b, G (or None), u0)."""
    x = 2.0 * np.pi * np.arange(N) / N
    Y, X = np.meshgrid(x, x, indexing="ij")
    h = 2.0 * np.pi / N
    ss = np.sin(X) * np.sin(Y)
    if problem == "T1":
        cc = np.cos(X) * np.cos(Y)
        a = 1.0 + 0.1 * cc
        return dict(h=h, a=a, b=a.copy(), G=(1.0 + 0.4 * cc) * ss, u0=ss.copy())
    if problem == "T2":
        a = 1.0 + 0.9 * np.cos(2 * X) * np.sin(2 * Y + np.pi / 3)
        b = 1.0 + 0.9 * np.cos(2 * X + np.pi / 3) * np.sin(2 * Y)
        return dict(h=h, a=a, b=b, G=None, u0=ss.copy())
    raise ValueError(problem)
