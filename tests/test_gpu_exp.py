"""The library's exponential (table-driven, Tang 1989) against the extended-
precision exp: within 2 ulp over the range the production rates use, and the
documented clamping outside it."""
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


def gpu_exp(S, x):
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to("cuda:0")
    yd = torch.empty_like(xd)
    S.smc_exp(xd, yd)
    return yd.cpu().numpy()


def ulp_error(y, x):
    ref = np.exp(x.astype(np.longdouble))
    ulp = np.spacing(ref.astype(np.float64))
    return np.abs((y.astype(np.longdouble) - ref) / ulp.astype(np.longdouble)).astype(np.float64)


def test_exp_within_two_ulp(smc):
    rng = np.random.default_rng(11)
    ln2_2048 = np.log(2.0) / 2048
    x = np.concatenate([
        rng.uniform(-700.0, 700.0, 400_000),
        rng.uniform(-5.0, 5.0, 400_000),
        # table-interval boundaries, where the rounding of n switches
        (np.arange(-40_000, 40_000) + 0.5) * ln2_2048,
        np.arange(-40_000, 40_000) * ln2_2048,
        np.array([0.0, -0.0, 1e-300, -1e-300, 1e-17, 511.9, -511.9, 709.0, -708.0]),
    ])
    y = gpu_exp(smc, x)
    err = ulp_error(y, x)
    assert np.all(np.isfinite(y))
    assert err.max() <= 2.0, (err.max(), x[np.argmax(err)])
    assert gpu_exp(smc, np.array([0.0]))[0] == 1.0


def test_exp_clamps_and_propagates_nan(smc):
    x = np.array([800.0, 1e6, -800.0, -1e6, np.inf, -np.inf, np.nan])
    y = gpu_exp(smc, x)
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
