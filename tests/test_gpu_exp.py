"""The library's exponentials (table-driven, Tang 1989) against the extended-
precision exp: within 2 ulp over the range the production rates use, and the
documented clamping outside it.  Variant 0 computes in FP64; variant 1 takes
the same decomposition through 128-bit fixed point, float pairs and 64-bit
fixed point (the integer and FP32 pipes).  Either one in the production rates
gives the oracle's right-hand side and multirate step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


def gpu_exp(S, x, variant=0):
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to("cuda:0")
    yd = torch.empty_like(xd)
    S.smc_exp(xd, yd, variant)
    return yd.cpu().numpy()


def ulp_error(y, x):
    ref = np.exp(x.astype(np.longdouble))
    ulp = np.spacing(ref.astype(np.float64))
    return np.abs((y.astype(np.longdouble) - ref) / ulp.astype(np.longdouble)).astype(np.float64)


@pytest.mark.parametrize("variant", [0, 1])
def test_exp_within_two_ulp(smc, variant):
    rng = np.random.default_rng(11)
    ln2_2048 = np.log(2.0) / 2048
    x = np.concatenate([
        rng.uniform(-700.0, 700.0, 400_000),
        rng.uniform(-5.0, 5.0, 400_000),
        # table-interval boundaries, where the rounding of n switches
        (np.arange(-40_000, 40_000) + 0.5) * ln2_2048,
        np.arange(-40_000, 40_000) * ln2_2048,
        np.array([0.0, -0.0, 1e-300, -1e-300, 1e-17, 511.9, -511.9, 709.0, -708.0]),
        # either side of the small-argument hand-over (|x| = 2^-20) and powers of two
        np.array([2.0 ** -20, -(2.0 ** -20), np.nextafter(2.0 ** -20, 0), 2.0 ** -19, 0.5, -0.5,
                  1.0, -1.0, 256.0, -256.0]),
        rng.uniform(-1e-3, 1e-3, 100_000),
    ])
    y = gpu_exp(smc, x, variant)
    err = ulp_error(y, x)
    assert np.all(np.isfinite(y))
    print("variant", variant, "max error", err.max(), "ulp, mean", err.mean())
    assert err.max() <= 2.0, (err.max(), x[np.argmax(err)])
    assert gpu_exp(smc, np.array([0.0]), variant)[0] == 1.0


@pytest.mark.parametrize("variant", [0, 1])
def test_exp_clamps_and_propagates_nan(smc, variant):
    x = np.array([800.0, 1e6, -800.0, -1e6, np.inf, -np.inf, np.nan])
    y = gpu_exp(smc, x, variant)
    assert np.all(ulp_error(y[:2], np.array([709.0, 709.0])) <= 2.0)
    assert np.all(ulp_error(y[2:4], np.array([-708.0, -708.0])) <= 2.0)
    assert y[4] == y[0] and y[5] == y[2]
    assert np.isnan(y[6])


def test_exp_rejects_bad_arguments(smc):
    x = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    with pytest.raises(smc.SmcError):
        smc.smc_exp(x.cpu(), x)
    y = torch.empty_like(x)
    smc.smc_exp(x[:0], y[:0])      # n = 0 is a no-op
    with pytest.raises(smc.SmcError):
        smc.smc_exp(x, y, 2)


def test_dmul_matches_the_fp64_product_bit_for_bit(smc):
    """The integer-pipe product against IEEE double multiplication (NumPy):
    random operands over the whole exponent range, constructed ties (both
    parities of the last bit), significands of all ones, signs, and every
    operand class the FP64 unit takes over (zero, subnormal, inf, NaN,
    products at the ends of the normal range)."""
    rng = np.random.default_rng(5)
    n = 400_000
    a = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-600, 600, n).astype(np.float64))
    b = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-600, 600, n).astype(np.float64))
    a *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
    i = np.arange(1, 20_001, dtype=np.float64)
    ties_a = 1.0 + i * 2.0 ** -52                    # x 1.5: exactly half an ulp over
    ties_b = np.full_like(ties_a, 1.5)
    ones = np.nextafter(2.0, 0.0) * np.exp2(rng.integers(-30, 30, 1000).astype(np.float64))
    tiny, big = np.finfo(np.float64).tiny, np.finfo(np.float64).max
    special_a = np.array([0.0, -0.0, 5e-324, tiny, 1.0, np.inf, -np.inf, np.nan, 2.0 ** 600,
                          2.0 ** -600, 1.5 * 2.0 ** 511, tiny * 2, big, 3.0])
    special_b = np.array([3.0, 3.0, 7.0, 0.5, 5e-324, 2.0, 2.0, 1.0, 2.0 ** 500, 2.0 ** -500,
                          1.5 * 2.0 ** 512, 0.75, 0.5, np.nan])
    A = np.concatenate([a, ties_a, ties_a * 3.0, ones, special_a])
    B = np.concatenate([b, ties_b, ties_b, ones[::-1], special_b])
    Ad = torch.from_numpy(A).to("cuda:0")
    Bd = torch.from_numpy(B).to("cuda:0")
    Yd = torch.empty_like(Ad)
    smc.smc_dmul(Ad, Bd, Yd)
    got = Yd.cpu().numpy()
    want = A * B
    same = (got.view(np.int64) == want.view(np.int64)) | (np.isnan(got) & np.isnan(want))
    assert same.all(), (A[~same][:5], B[~same][:5], got[~same][:5], want[~same][:5])


def test_rates_with_either_exponential_match_the_oracle(smc):
    """21 species / 84 reactions on eight uneven boxes: the FP64 right-hand
    side and one multirate step with the rate arithmetic on the FP64 pipe
    (alu 0), with the integer-pipe exponentials (1), and with the integer-pipe
    products too (2); 1 and 2 agree bit for bit (the products round alike)."""
    from oracle import rhs as orhs
    from oracle import sdc as osdc
    from oracle import thermo
    from paper_1309_7327_gb300 import synth
    from util import relerr
    wl = synth.workload("c4", seed=4, n=12)
    prim_g = synth.boxes_to_global(wl.grid, wl.prim)
    U_g = thermo.conserved(prim_g, wl.mech.nasa7, wl.mech.W)
    U = synth.global_to_boxes(wl.grid, U_g)
    ref = synth.global_to_boxes(wl.grid, orhs.rhs_periodic(U_g, wl.mech, wl.grid.dx))

    def part(which):
        def f(u):
            tr, ch = orhs.rhs_periodic(u, wl.mech, wl.grid.dx, parts=True)
            return tr if which == 0 else ch
        return f
    dt = 2e-9
    step = osdc.mrsdc_step(U_g, part(0), part(1), dt, coarse=3, fine=3, sweeps=2)[0]
    step = synth.global_to_boxes(wl.grid, step)
    out = {}
    for variant in (0, 1, 2):
        with smc.Smc(wl.grid, wl.mech, {"alu": variant}) as h:
            Ud = torch.from_numpy(U).to("cuda:0")
            F = torch.empty_like(Ud)
            h.rhs(Ud, F)
            h.sdc_step(Ud, dt, nodes=3, sweeps=2, reaction_substeps=3)
            h.synchronize()
            out[variant] = (F.cpu().numpy(), Ud.cpu().numpy())
            err = relerr(out[variant][0], ref)
            assert err.max() < 1e-12, (variant, err.max())
            err = relerr(out[variant][1] - U, step - U)
            assert err.max() < 1e-10, (variant, err.max())
    assert np.array_equal(out[1][0], out[2][0]) and np.array_equal(out[1][1], out[2][1])
