"""Right-hand side of the reacting compressible Navier-Stokes equations
(eq. cns, Sec. 2.1) discretised as in Sec. 2.2 and Sec. 2.4.

Oracle, test infrastructure only.  Plain NumPy, FP64, no fusion.

Discretisation (readings of the paper where it is silent):

* Convective terms: -D_d applied to the pointwise fluxes (rho u_d,
  rho u_c u_d + p delta_cd, (rho E + p) u_d, rho Y_k u_d), D the 8th-order
  centred first derivative.
* Second-derivative terms (d/dx_d)(a d/dx_d u) use the narrow stencil
  (eqs. DaDu/H).  Mixed derivatives use D_d(c D_e u), e != d.
* Viscous stress tau (Sec. 2.1) split per direction d, with e, f the other
  two directions, c43 = 4/3 eta + xi and c23 = xi - 2/3 eta:
    momentum d:  narrow(c43, u_d) + D_d(c23 (D_e u_e + D_f u_f))
    momentum e:  narrow(eta, u_e) + D_d(eta D_e u_d)
    energy:      narrow(c43, u_d^2/2) + narrow(eta, (u_e^2 + u_f^2)/2)
                 + D_d(c23 (D_e u_e + D_f u_f) u_d + eta (D_e u_d) u_e
                       + eta (D_f u_d) u_f)
  i.e. div(tau . u) kept in flux form via u u_x = (u^2/2)_x.
* Heat conduction: narrow(lambda, T).
* Species diffusion, eq. fbar: -div Fbar_k = sum_d narrow(rho D_k, X_k)
  + narrow(rho D_k (X_k - Y_k)/p, p).
* Correction-velocity mode (eq. Vc, Sec. 2.4), the default:
    V_c,d = sum_l Fbar_l,d at cell centres from D derivatives,
    div V_c = sum_l div Fbar_l from the narrow stencils,
    -div(F_k) = -div Fbar_k + Y_k div V_c + grad Y_k . V_c,
    energy: -div sum_k F_k h_k = -div sum_k Fbar_k h_k
            + h div V_c + grad h . V_c,   h = sum_k Y_k h_k,
  where -div sum_k Fbar_k h_k = sum_d [sum_k narrow(rho D_k h_k, X_k)
            + narrow(sum_k h_k rho D_k (X_k - Y_k)/p, p)].
* Reference-species mode (Sec. 2.1, Sec. 2.4), species ``ref``: F_k = Fbar_k
  for k != ref, F_ref = -sum_{k != ref} F_k, and the energy flux uses
  h_k - h_ref.
* Chemistry: rho omega_k from ``chem.production_rates``.
* Options.terms selects which groups of terms are added (all by default), so
  that each can be checked on its own against the continuous operator:
    "conv"  -div of the convective fluxes (every component),
    "visc"  div tau (momentum),
    "work"  div(tau . u) (energy),
    "heat"  div(lambda grad T) (energy),
    "diff"  -div Fbar_k (species) and -div sum_k Fbar_k h_k (energy); in
            reference-species mode the whole species diffusion,
    "vc"    the correction-velocity terms div(Y_k V_c), div(h V_c),
    "chem"  rho omega_k.
* Non-periodic x ends (Options.x_outflow): every x derivative -- convective,
  narrow, mixed, velocity gradients, correction velocity -- uses the
  boundary-lowered stencils of ``stencil.D_bc`` / ``stencil.narrow_bc`` in
  the four cells next to each end (Sec. 2.2, boundary paragraph); no
  characteristic boundary correction.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import chem, stencil, thermo, transport

G = 4                               # ghost cells per side
AX = {0: -1, 1: -2, 2: -3}          # direction -> array axis (x fastest)


@dataclass
class Options:
    m47: object = stencil.M47_SMC
    m48: object = stencil.M48_SMC
    xi_ratio: float = 0.0           # bulk viscosity xi = xi_ratio * eta
    mode: str = "vc"                # "vc": correction velocity, "ref": reference species
    ref: int = -1                   # reference species index (mode "ref")
    T0: float = 1000.0              # Newton first guess
    reactions: bool = True
    x_outflow: bool = False         # x ends are non-periodic boundaries (lowered stencils)
    terms: frozenset = frozenset(("conv", "visc", "work", "heat", "diff", "vc", "chem"))


def _inner(f, dirs):
    idx = [slice(None)] * f.ndim
    for d in dirs:
        idx[AX[d]] = slice(G, -G)
    return f[tuple(idx)]


def _others(d):
    return [e for e in range(3) if e != d]


def rhs_ghosted(Ug: np.ndarray, mech, dx, opt: Options | None = None,
                parts: bool = False):
    """dU/dt at the interior cells of a box carried with 4 ghost cells on every
    side (faces, edges and corners filled).  Ug: [NV, nz+8, ny+8, nx+8].

    Returns [NV, nz, ny, nx]; with ``parts`` returns (transport, chemistry)
    whose sum is the full right-hand side.
    """
    opt = opt or Options()
    ns = mech.W.shape[0]
    W = np.asarray(mech.W, dtype=np.float64)
    P = thermo.primitives(Ug, mech.nasa7, W, T0=opt.T0)
    if not P["converged"].all():
        raise FloatingPointError("temperature Newton iteration did not converge")
    tr = transport.coefficients(P["T"], P["cp"], np.asarray(mech.Le), mech.eta_ref,
                                mech.T_ref, mech.eta_exp, mech.Pr, opt.xi_ratio)
    rho, vel, T, p = P["rho"], P["vel"], P["T"], P["p"]
    Y, X, h = P["Y"], P["X"], P["h"]
    eta, xi, lam, rhoD = tr["eta"], tr["xi"], tr["lam"], tr["rhoD"]
    c43 = 4.0 / 3.0 * eta + xi
    c23 = xi - 2.0 / 3.0 * eta
    hmix = np.sum(Y * h, axis=0)
    B = rhoD * (X - Y) / p[None]
    M = stencil.to_float(stencil.narrow8_exact(opt.m47, opt.m48), Ug.dtype)

    terms = opt.terms
    interior = _inner(_inner(_inner(Ug, [0]), [1]), [2]).shape
    out = np.zeros(interior, dtype=Ug.dtype)
    Nsum = np.zeros((ns,) + interior[1:], dtype=Ug.dtype)
    ref = opt.ref % ns

    for d in range(3):
        ax, hd = AX[d], dx[d]
        e, f = _others(d)

        def lin(a):                         # ghosted along d only
            return _inner(a, [e, f])

        bc = opt.x_outflow and d == 0

        def Dd(a):                          # D_d of a field ghosted along d
            return stencil.D_bc(a, ax, hd) if bc else stencil.D(a, ax, hd)

        def nd(a, u):                       # narrow along d
            if bc:
                return stencil.narrow_bc(lin(a), lin(u), ax, hd, M)
            return stencil.narrow(lin(a), lin(u), ax, hd, M)

        def grad(comp, along):
            """D_along of vel[comp] on cells interior except along d."""
            third = [k for k in range(3) if k not in (along, d)]
            arr = _inner(vel[comp], third)
            if opt.x_outflow and along == 0:
                return stencil.D_bc(arr, AX[along], dx[along])
            return stencil.D(arr, AX[along], dx[along])

        ud = vel[d]
        # convective fluxes
        if "conv" in terms:
            out[0] -= Dd(lin(Ug[1 + d]))
            for c in range(3):
                flux = Ug[1 + c] * ud + (p if c == d else 0.0)
                out[1 + c] -= Dd(lin(flux))
            out[4] -= Dd(lin((Ug[4] + p) * ud))
            out[5:] -= Dd(lin(Ug[5:] * ud[None]))

        # viscous stress
        Gee, Gff = grad(e, e), grad(f, f)
        Ged, Gfd = grad(d, e), grad(d, f)
        if "visc" in terms:
            out[1 + d] += nd(c43, vel[d]) + Dd(lin(c23) * (Gee + Gff))
            out[1 + e] += nd(eta, vel[e]) + Dd(lin(eta) * Ged)
            out[1 + f] += nd(eta, vel[f]) + Dd(lin(eta) * Gfd)
        if "work" in terms:
            out[4] += nd(c43, 0.5 * vel[d] ** 2) + nd(eta, 0.5 * (vel[e] ** 2 + vel[f] ** 2))
            out[4] += Dd(lin(c23) * (Gee + Gff) * lin(vel[d])
                         + lin(eta) * Ged * lin(vel[e]) + lin(eta) * Gfd * lin(vel[f]))
        # heat conduction
        if "heat" in terms:
            out[4] += nd(lam, T)

        # species diffusion
        if opt.mode == "vc":
            Nd = nd(rhoD, X) + nd(B, p[None])
            Nsum += Nd
            if "diff" in terms:
                out[5:] += Nd
                out[4] += np.sum(nd(rhoD * h, X), axis=0) + nd(np.sum(h * B, axis=0), p)
            rD_c = _inner(rhoD, [d])
            B_c = _inner(B, [d])
            Vc = -(np.sum(_inner(rD_c, [e, f]) * Dd(lin(X)), axis=0)
                   + np.sum(_inner(B_c, [e, f]), axis=0) * Dd(lin(p)))
            if "vc" in terms:
                out[5:] += Dd(lin(Y)) * Vc[None]
                out[4] += Dd(lin(hmix)) * Vc
        elif opt.mode == "ref":
            hr = h - h[ref][None]
            keep = [k for k in range(ns) if k != ref]
            if "diff" in terms:
                Nd = nd(rhoD[keep], X[keep]) + nd(B[keep], p[None])
                out[5 + np.array(keep)] += Nd
                out[5 + ref] -= np.sum(Nd, axis=0)
                out[4] += (np.sum(nd(rhoD[keep] * hr[keep], X[keep]), axis=0)
                           + nd(np.sum(hr[keep] * B[keep], axis=0), p))
        else:
            raise ValueError(opt.mode)

    if opt.mode == "vc" and "vc" in terms:
        divVc = -np.sum(Nsum, axis=0)
        Yi = _inner(_inner(_inner(Y, [0]), [1]), [2])
        hi = _inner(_inner(_inner(hmix, [0]), [1]), [2])
        out[5:] += Yi * divVc[None]
        out[4] += hi * divVc

    ch = np.zeros(interior, dtype=Ug.dtype)
    if opt.reactions and "chem" in terms and mech.A.shape[0] > 0:
        ri = _inner(_inner(_inner(rho, [0]), [1]), [2])
        Ti = _inner(_inner(_inner(T, [0]), [1]), [2])
        Yi = _inner(_inner(_inner(Y, [0]), [1]), [2])
        ch[5:] = chem.production_rates(ri, Ti, Yi, mech)
    if parts:
        return out, ch
    return out + ch


def pad_periodic(U: np.ndarray) -> np.ndarray:
    """Fill 4 ghost cells on every side by periodic wrap ([NV, nz, ny, nx])."""
    return np.pad(U, ((0, 0), (G, G), (G, G), (G, G)), mode="wrap")


def rhs_periodic(U: np.ndarray, mech, dx, opt: Options | None = None, parts=False):
    """Right-hand side on a triply periodic domain, U: [NV, nz, ny, nx].
    With ``opt.x_outflow`` the x ends are boundaries instead: the lowered
    stencils never read the wrapped x ghosts."""
    return rhs_ghosted(pad_periodic(U), mech, dx, opt, parts)


def patch(U: np.ndarray, z: int, y: int, x: int) -> np.ndarray:
    """The periodic 9x9x9 neighbourhood that determines dU/dt at one cell."""
    nz, ny, nx = U.shape[1:]
    iz = (np.arange(z - G, z + G + 1)) % nz
    iy = (np.arange(y - G, y + G + 1)) % ny
    ix = (np.arange(x - G, x + G + 1)) % nx
    return U[:, iz][:, :, iy][:, :, :, ix]


def rhs_at(U: np.ndarray, cells, mech, dx, opt: Options | None = None) -> np.ndarray:
    """dU/dt of a periodic field at a list of (z, y, x) cells, one by one."""
    out = np.empty((U.shape[0], len(cells)), dtype=U.dtype)
    for i, (z, y, x) in enumerate(cells):
        out[:, i] = rhs_ghosted(patch(U, z, y, x), mech, dx, opt)[:, 0, 0, 0]
    return out
