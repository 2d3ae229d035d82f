"""The face kernels' FP64 time-integration coefficients (gks_probe_time_coefs: the device
function itself) against their definition evaluated with 80 significant digits.

The non-equilibrium branch of Eq. 3rd-simplify-flux decays as e^{-t/tau}; its time integrals
E0(d) = int_0^d e^{-t/tau} dt = tau (1 - e^{-d/tau}) and
E1(d) = int_0^d t e^{-t/tau} dt = tau^2 (1 - e^{-d/tau} (1 + d/tau)) over [0, dt/2] and
[0, dt], fitted linearly in t (Sec. 2.2), give the coefficients
a0 = (4 E0(dt/2) - E0(dt))/dt, a1 = (4 E1(dt/2) - E1(dt))/dt,
b0 = 4 (E0(dt) - 2 E0(dt/2))/dt^2, b1 = 4 (E1(dt) - 2 E1(dt/2))/dt^2.
Each is a difference of terms of similar size; the error is measured against the size of
those terms (for b1, which changes sign near dt/(2 tau) = 1.26, a relative error would
be meaningless there) and must stay below 1e-14 for theta = tau/dt from 1e-8 to 1e8,
across both branches of the device function (series below dt/(2 tau) = 1/2, closed form
above, e^{-x} = 0 beyond 40).  The reference uses the standard library's decimal module.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

from paper_1901_00261_gb300 import gks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gks.lib()


def reference(theta, dt):
    getcontext().prec = 80
    th, D = Decimal(float(theta)), Decimal(float(dt))
    tau = th * D

    def phi(y):
        return 1 - (-y).exp() * (1 + y)

    def E0(d):
        return tau * (1 - (-d / tau).exp())

    def E1(d):
        return tau * tau * phi(d / tau)

    h = D / 2
    x = h / tau
    val = [(4 * E0(h) - E0(D)) / D, (4 * E1(h) - E1(D)) / D,
           4 * (E0(D) - 2 * E0(h)) / (D * D), 4 * (E1(D) - 2 * E1(h)) / (D * D)]
    scale = [4 * E0(h) / D, th * th * D * (4 * phi(x) + phi(2 * x)),
             4 * (E0(D) + 2 * E0(h)) / (D * D), 4 * th * th * (phi(2 * x) + 2 * phi(x))]
    return val, scale


THETAS = np.concatenate([np.logspace(-8, 8, 161),
                         [1 / 80 * (1 - 1e-9), 1 / 80 * (1 + 1e-9), 0.398, 0.4,
                          1.0 - 1e-12, 1.0, 1.0 + 1e-12, 0.3, 0.7, 2.0]])


@pytest.mark.parametrize("dt", [1e-3, 0.25])
def test_time_coefficients_match_their_definition(dt):
    got = gks.probe_time_coefs(THETAS, dt)
    worst = 0.0
    for th, row in zip(THETAS, got):
        val, scale = reference(th, dt)
        for g, v, s in zip(row, val, scale):
            worst = max(worst, float(abs(Decimal(float(g)) - v) / s))
    assert worst < 1e-14, worst


@pytest.mark.parametrize("dt", [1e-3, 0.25])
def test_single_precision_time_coefficients(dt):
    """The single-precision form's coefficients (rounded to float after this): shorter series,
    whose truncation stays below 1e-9 of each coefficient itself (where the series branch
    runs, dt/(2 tau) < 1/2, no coefficient changes sign), and the same closed form above."""
    got = gks.probe_time_coefs(THETAS, dt, single=True)
    worst = 0.0
    for th, row in zip(THETAS, got):
        val, scale = reference(th, dt)
        for g, v, s in zip(row, val, scale):
            bound = max(Decimal(1e-9) * abs(v), Decimal(1e-14) * s)
            worst = max(worst, float(abs(Decimal(float(g)) - v) / bound))
    assert worst < 1.0, worst


def test_time_coefficient_probe_rejects_bad_theta():
    with pytest.raises(gks.GksError):
        gks.probe_time_coefs(np.array([1.0, 0.0]), 0.1)


def test_rcp64_within_two_ulp_of_the_reciprocal():
    """The FP64 reciprocal of the single-precision sweeps (a float seed and two Newton-Raphson
    steps in FP64) against the correctly rounded 1/x, over the float-normal range where it is
    used (densities and their products): at most 2 ulp of 1/x."""
    rng = np.random.default_rng(3)
    x = np.concatenate([np.logspace(-37, 37, 741), rng.uniform(0.05, 20.0, 4000),
                        [1.0, 2.0, 0.1, 3.0, 7.0, 1.0 - 2.0 ** -52, 1.0 + 2.0 ** -52]])
    got = gks.probe_rcp64(x)
    want = 1.0 / x
    ulp = np.spacing(want)
    assert np.max(np.abs(got - want) / ulp) <= 2.0


def test_rcp64_probe_rejects_null():
    L = gks.lib()
    assert L.gks_probe_rcp64(None, 1, None) == gks.GKS_EINVAL


def test_d2f_rounds_to_nearest_even():
    """The integer-pipe double -> float rounding of the FP32-bulk slope mirror equals IEEE
    round-to-nearest-even (numpy's float32 conversion) bit for bit: random values across the
    float range, exact ties between neighbouring floats (both parities), values next to the
    largest float and rounding to infinity, subnormal results, signed zeros, inf and nan."""
    rng = np.random.default_rng(17)
    mant = rng.uniform(1.0, 2.0, 20000)
    expo = rng.integers(-140, 128, 20000)
    x = mant * np.exp2(expo.astype(float)) * np.where(rng.random(20000) < 0.5, -1.0, 1.0)
    f = rng.uniform(1.0, 2.0, 4000).astype(np.float32) * np.float32(2.0) ** rng.integers(-120, 120, 4000).astype(np.float32)
    nxt = np.nextafter(f, np.float32(np.inf))
    ties = (f.astype(np.float64) + nxt.astype(np.float64)) / 2.0
    fmax = float(np.finfo(np.float32).max)
    edge = [fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24), 2.0 ** 128, 2.0 ** -126,
            2.0 ** -126 * (1 - 2.0 ** -30), 2.0 ** -149, 2.0 ** -150, 1e-300, 0.0, -0.0,
            np.inf, -np.inf, 1.0, -1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 0.1, 1.0 / 3.0]
    xs = np.concatenate([x, ties, -ties, np.array(edge)])
    got = gks.probe_d2f(xs)
    with np.errstate(over="ignore"):   # values beyond the float range round to inf
        want = xs.astype(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    nan = gks.probe_d2f(np.array([np.nan]))
    assert np.isnan(nan[0])
