"""The oracle's right-hand side against the continuous operator of eq. cns.

On a smooth, triply periodic manufactured state (closed-form primitive
fields rho, u, T, Y_k), every group of terms of eq. cns (Sec. 2.1) is
differentiated exactly with sympy, here in the test and from the paper's
equations, not from the oracle:

* convection: -div(rho u), -div(rho u u + p I), -div((rho E + p) u),
  -div(rho Y_k u);
* viscous stress: div tau with
  tau_ij = eta (d_j u_i + d_i u_j - 2/3 delta_ij div u) + xi delta_ij div u;
* viscous work: div(tau . u);
* heat conduction: div(lambda grad T);
* species diffusion, eq. fbar: Fbar_k = -rho D_k (grad X_k + (X_k - Y_k)
  grad p / p), the terms -div Fbar_k and -div sum_k Fbar_k h_k;
* correction velocity (eq. Vc): V_c = sum_l Fbar_l, F_k = Fbar_k - Y_k V_c,
  whose extra terms are div(Y_k V_c) and div(h V_c), h = sum_k Y_k h_k;
* the reference-species mode: F_k = Fbar_k (k != ref), F_ref = -sum of the
  others.

The oracle evaluates each group alone (Options.terms) on 16^3, 32^3 and 64^3
cells, and must converge to the exact values at the 8th order of Sec. 2.2
(error ratio near 2^8 = 256 per halving of h).  The mutation test plants
plausible mistakes in copies of the oracle's source and checks that each
one fails this pin.

Thermodynamics (NASA-7, ideal gas) and the transport model (power-law
viscosity, constant Prandtl and Lewis numbers) are the readings the library
documents; the transport model is also pinned by hand-computed values.
"""
import sys
import types

import numpy as np
import pytest

from oracle import rhs as orhs
from oracle import transport
from paper_1309_7327_gb300 import synth

sp = pytest.importorskip("sympy")

R_U = 8.31446261815324e7          # erg / (mol K)
XI_RATIO = 0.6                    # bulk viscosity on, so that xi is exercised
NS = 3


class Exact:
    """Closed-form primitive fields and the exact terms of eq. cns, as numpy
    functions of cell-centre coordinates on the unit periodic cube."""

    def __init__(self, mech, seed=11):
        rng = np.random.default_rng(seed)
        xs = sp.symbols("x y z", real=True)
        x, y, z = xs
        k = 2 * sp.pi

        def wave(amp):
            ph = [sp.Float(v) for v in rng.uniform(0.0, 2.0 * np.pi, 6)]
            return amp * (sp.sin(k * x + ph[0]) * sp.cos(k * y + ph[1])
                          + sp.cos(k * y + ph[2]) * sp.sin(k * z + ph[3])
                          + sp.Rational(1, 2) * sp.sin(k * z + ph[4]) * sp.cos(k * x + ph[5]))

        ns = mech.ns
        rho = 2.5e-4 * (1 + wave(0.05))
        vel = [wave(3000.0) for _ in range(3)]
        T = 1200 + wave(150.0)
        Yraw = [sp.Float(1.5) + wave(0.4) for _ in range(ns)]       # > 0
        Ysum = sum(Yraw)
        Y = [v / Ysum for v in Yraw]
        W = [float(w) for w in mech.W]
        a = np.asarray(mech.nasa7, dtype=float)
        # ideal-gas mixture, NASA-7 polynomials (per unit mass)
        h = [R_U / W[i] * T * (a[i, 0] + a[i, 1] * T / 2 + a[i, 2] * T ** 2 / 3
                               + a[i, 3] * T ** 3 / 4 + a[i, 4] * T ** 4 / 5 + a[i, 5] / T)
             for i in range(ns)]
        cpk = [R_U / W[i] * (a[i, 0] + a[i, 1] * T + a[i, 2] * T ** 2 + a[i, 3] * T ** 3
                             + a[i, 4] * T ** 4) for i in range(ns)]
        winv = sum(Y[i] / W[i] for i in range(ns))
        p = rho * R_U * T * winv
        X = [Y[i] / W[i] / winv for i in range(ns)]
        cp = sum(Y[i] * cpk[i] for i in range(ns))
        e = sum(Y[i] * (h[i] - R_U * T / W[i]) for i in range(ns))
        E = e + sum(v ** 2 for v in vel) / 2
        # transport model
        eta = mech.eta_ref * (T / mech.T_ref) ** mech.eta_exp
        xi = XI_RATIO * eta
        lam = cp * eta / mech.Pr
        rD = [lam / (cp * float(mech.Le[i])) for i in range(ns)]

        def d(f, j):
            return sp.diff(f, xs[j])

        def div(F):
            return sum(d(F[j], j) for j in range(3))

        divu = div(vel)
        tau = [[eta * (d(vel[i], j) + d(vel[j], i)) + (xi - sp.Rational(2, 3) * eta) * divu
                * (1 if i == j else 0) for j in range(3)] for i in range(3)]
        Fbar = [[-rD[i] * (d(X[i], j) + (X[i] - Y[i]) * d(p, j) / p) for j in range(3)]
                for i in range(ns)]
        Vc = [sum(Fbar[i][j] for i in range(ns)) for j in range(3)]
        hmix = sum(Y[i] * h[i] for i in range(ns))
        ref = ns - 1
        zero = sp.Integer(0)
        nv = 5 + ns

        def comp(**kw):
            out = [zero] * nv
            for c, v in kw.items():
                out[int(c[1:])] = v
            return out

        terms = {}
        conv = [-div([rho * v for v in vel])]
        conv += [-div([rho * vel[i] * vel[j] + (p if i == j else 0) for j in range(3)])
                 for i in range(3)]
        conv += [-div([(rho * E + p) * v for v in vel])]
        conv += [-div([rho * Y[i] * v for v in vel]) for i in range(ns)]
        terms["conv"] = conv
        terms["visc"] = comp(c1=div(tau[0]), c2=div(tau[1]), c3=div(tau[2]))
        terms["work"] = comp(c4=div([sum(tau[i][j] * vel[i] for i in range(3)) for j in range(3)]))
        terms["heat"] = comp(c4=div([lam * d(T, j) for j in range(3)]))
        diff = [zero] * nv
        diff[4] = -div([sum(h[i] * Fbar[i][j] for i in range(ns)) for j in range(3)])
        for i in range(ns):
            diff[5 + i] = -div(Fbar[i])
        terms["diff"] = diff
        vct = [zero] * nv
        vct[4] = div([hmix * Vc[j] for j in range(3)])
        for i in range(ns):
            vct[5 + i] = div([Y[i] * Vc[j] for j in range(3)])
        terms["vc"] = vct
        dref = [zero] * nv
        for i in range(ns):
            if i != ref:
                dref[5 + i] = -div(Fbar[i])
        dref[5 + ref] = sum(div(Fbar[i]) for i in range(ns) if i != ref)
        dref[4] = -div([sum((h[i] - h[ref]) * Fbar[i][j] for i in range(ns) if i != ref)
                        for j in range(3)])
        terms["diff_ref"] = dref
        U = [rho] + [rho * v for v in vel] + [rho * E] + [rho * v for v in Y]
        self.nv = nv
        self.U = sp.lambdify(xs, U, modules="numpy", cse=True)
        self.terms = {k: (sp.lambdify(xs, v, modules="numpy", cse=True),
                          [c for c in range(nv) if v[c] != 0]) for k, v in terms.items()}

    @staticmethod
    def _grid(n):
        c = (np.arange(n) + 0.5) / n
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        return X, Y, Z

    @staticmethod
    def _full(vals, n):
        return np.stack([np.broadcast_to(np.asarray(v, dtype=float), (n, n, n)) for v in vals])

    def state(self, n):
        return self._full(self.U(*self._grid(n)), n)

    def term(self, name, n):
        f, comps = self.terms[name]
        return self._full(f(*self._grid(n)), n), comps


@pytest.fixture(scope="module")
def mech():
    return synth.make_mechanism(NS, 2, 7)


@pytest.fixture(scope="module")
def exact(mech):
    return Exact(mech)


ORACLE_TERM = {"conv": ("conv", "vc"), "visc": ("visc", "vc"), "work": ("work", "vc"),
               "heat": ("heat", "vc"), "diff": ("diff", "vc"), "vc": ("vc", "vc"),
               "diff_ref": ("diff", "ref")}


def term_errors(rhs_module, exact, mech, name, n, state_cache={}):
    """Per-component max|oracle - exact| / max|exact| of one term group on n^3."""
    key = (id(exact), n)
    if key not in state_cache:
        state_cache[key] = exact.state(n)
    U = state_cache[key]
    group, mode = ORACLE_TERM[name]
    opt = rhs_module.Options(xi_ratio=XI_RATIO, mode=mode, terms=frozenset([group]),
                             reactions=False)
    got = rhs_module.rhs_periodic(U, mech, (1.0 / n,) * 3, opt)
    want, comps = exact.term(name, n)
    return {c: float(np.abs(got[c] - want[c]).max() / np.abs(want[c]).max()) for c in comps}


TERMS = ["conv", "visc", "work", "heat", "diff", "vc", "diff_ref"]


@pytest.mark.parametrize("name", TERMS)
def test_each_term_converges_to_the_continuous_operator_at_order_8(exact, mech, name):
    e = [term_errors(orhs, exact, mech, name, n) for n in (16, 32, 64)]
    for c in e[0]:
        e16, e32, e64 = e[0][c], e[1][c], e[2][c]
        assert e32 < 1e-5, (name, c, e16, e32, e64)
        assert e64 < 5e-8, (name, c, e16, e32, e64)
        assert e16 / e32 > 100.0, (name, c, e16, e32, e64)       # pre-asymptotic: order > 6.6
        assert e32 / e64 > 190.0, (name, c, e16, e32, e64)       # order > 7.5


def test_transport_coefficients_at_hand_computed_points():
    """eta = eta_ref (T/T_ref)^0.7, lambda = cp eta / Pr, rho D_k =
    lambda / (cp Le_k), xi = xi_ratio eta, at T = 600 K (T/T_ref = 2,
    2^0.7 = 1.624504792712471) and T = 300 K, cp = 1.3e7 erg/(g K)."""
    T = np.array([600.0, 300.0])
    cp = np.array([1.3e7, 1.3e7])
    Le = np.array([1.5, 0.5])
    c = transport.coefficients(T, cp, Le, 1.85e-4, 300.0, 0.7, 0.72, xi_ratio=0.25)
    eta = np.array([3.005333866518071e-4, 1.85e-4])
    lam = np.array([5426.297258990962, 3340.277777777778])
    assert np.allclose(c["eta"], eta, rtol=1e-12)
    assert np.allclose(c["xi"], 0.25 * eta, rtol=1e-12)
    assert np.allclose(c["lam"], lam, rtol=1e-12)
    # rho D_k = lambda / (cp Le_k) = eta / (Pr Le_k)
    assert np.allclose(c["rhoD"][:, 0], [2.782716543072288e-4, 8.348149629216865e-4], rtol=1e-12)
    assert np.allclose(c["rhoD"][:, 1], [1.712962962962963e-4, 5.138888888888889e-4], rtol=1e-12)


# --------------------------------------------------------------- mutations
def _load(name, src, extra=None):
    mod = types.ModuleType(f"oracle._mutant_{name}")
    mod.__package__ = "oracle"
    sys.modules[mod.__name__] = mod
    try:
        exec(compile(src, f"<mutant {name}>", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    for k, v in (extra or {}).items():
        setattr(mod, k, v)
    return mod


def _mutant(file, old, new):
    import os

    import oracle
    base = os.path.dirname(oracle.__file__)
    rsrc = open(os.path.join(base, "rhs.py")).read()
    tsrc = open(os.path.join(base, "transport.py")).read()
    if file == "rhs":
        assert rsrc.count(old) == 1, old
        rsrc = rsrc.replace(old, new)
        return _load("rhs", rsrc)
    assert tsrc.count(old) == 1, old
    tr = _load("transport", tsrc.replace(old, new))
    return _load("rhs", rsrc, {"transport": tr})


MUTATIONS = [
    ("rhs", "c23 = xi - 2.0 / 3.0 * eta", "c23 = xi + 2.0 / 3.0 * eta", ["visc", "work"]),
    ("rhs", "c43 = 4.0 / 3.0 * eta + xi", "c43 = 4.0 / 3.0 * eta - xi", ["visc", "work"]),
    ("rhs", "out[1 + e] += nd(eta, vel[e]) + Dd(lin(eta) * Ged)",
     "out[1 + e] += nd(eta, vel[e])", ["visc"]),
    ("rhs", "out[4] += nd(c43, 0.5 * vel[d] ** 2) + nd(eta, 0.5 * (vel[e] ** 2 + vel[f] ** 2))",
     "out[4] += nd(eta, 0.5 * vel[d] ** 2) + nd(c43, 0.5 * (vel[e] ** 2 + vel[f] ** 2))", ["work"]),
    ("rhs", "B = rhoD * (X - Y) / p[None]", "B = rhoD * (Y - X) / p[None]", ["diff", "vc"]),
    ("rhs", "out[5:] += Yi * divVc[None]", "pass", ["vc"]),
    ("rhs", "out[4] -= Dd(lin((Ug[4] + p) * ud))", "out[4] -= Dd(lin(Ug[4] * ud))", ["conv"]),
    ("rhs", "hr = h - h[ref][None]", "hr = h", ["diff_ref"]),
    ("transport", "lam = cp_mix * eta / Pr", "lam = cp_mix * eta * Pr", ["heat", "diff"]),
]


@pytest.mark.parametrize("file,old,new,caught_by", MUTATIONS,
                         ids=[m[2][:40] for m in MUTATIONS])
def test_planted_mistakes_fail_the_pin(exact, mech, file, old, new, caught_by):
    mod = _mutant(file, old, new)
    for name in caught_by:
        good = max(term_errors(orhs, exact, mech, name, 16).values())
        bad = max(term_errors(mod, exact, mech, name, 16).values())
        assert good < 1e-3
        assert bad > 1e-2 and bad > 100 * good, (name, good, bad)
