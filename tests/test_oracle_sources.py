"""Pins of the oracle's moderator guns (§3.2: UniModeratorGun, MaxwellianGun).

Each gun starts a neutron at a point uniform on the moderator rectangle and
aims it at a point uniform on the slit; the wavelength is uniform on
[mean - range, mean + range] (UniModeratorGun) or follows the Maxwell-Boltzmann
energy distribution at temperature T (MaxwellianGun).  The checks below use
only closed forms:

* at the slit plane the hit point IS the aim point: uniform inside the slit,
  nothing outside (pins the slit sizes and their axes);
* further downstream, at twice the moderator-slit distance, x = 2 s_x - r_x is
  the sum of two independent uniforms: a trapezoid in x and in y (pins that
  the direction runs from the sampled source point, not from the centre);
* the uniform gun's spectrum is flat on its interval;
* the Maxwellian spectrum: E / kT ~ Gamma(3/2), so
  P(Lambda <= lambda) = Q(3/2, C / (kT lambda^2)) with C = h^2 / (2 m_n)
  = 81.8042 meV A^2 and Q the regularised upper incomplete gamma function.
  A dropped or wrong Box-Muller factor, a wrong kT or C, or a sampled energy
  taken for a wavelength moves this distribution.

Counts are multinomial; each check is a chi-square over the bins that hold an
expected count of at least 5, plus exact zeros where the probability is zero."""
import math

import numpy as np
import pytest

import workloads as W
from stats import chi2_sf

N = 400_000


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def run(orc, **kw):
    desc = W.moderator_test(n_histories=N, precision="f64", **kw)
    out = orc.OracleScene(desc).run(N, threads=8)
    psd = out["sum"][:1600].reshape(40, 40)        # [x bin][y bin]
    spec = out["sum"][1600:1660]
    return desc, psd, spec


def chi2_check(counts, probs, p_min=1e-4):
    counts = np.asarray(counts, dtype=np.float64).ravel()
    probs = np.asarray(probs, dtype=np.float64).ravel()
    exp = N * probs
    zero = probs == 0.0
    assert counts[zero].sum() == 0.0, "counts where the probability is zero"
    use = exp >= 5.0
    chi2 = float((((counts[use] - exp[use]) ** 2) / exp[use]).sum())
    p = chi2_sf(chi2, int(use.sum()) - 1)
    assert p >= p_min, (chi2, int(use.sum()), p)
    return p


def uniform_cdf(a, b):
    return lambda x: np.clip((x - a) / (b - a), 0.0, 1.0)


def sum_uniform_cdf(a, b):
    """CDF of U(-a, a) + U(-b, b) with a <= b (a trapezoid density):
    P(X + Y <= x) = (H(x + b) - H(x - b)) / (2 b), H the antiderivative of the
    CDF of U(-a, a)."""
    def H(t):
        t = np.asarray(t, dtype=np.float64)
        tc = np.clip(t, -a, a)
        return (tc + a) ** 2 / (4 * a) + np.maximum(t - a, 0.0)

    return lambda x: (H(np.asarray(x) + b) - H(np.asarray(x) - b)) / (2 * b)


def bin_probs(F, edges):
    c = F(edges)
    return np.diff(c)


def test_uniform_gun_hits_the_slit_uniformly(orc):
    desc, psd, spec = run(orc)
    src = desc["source"]
    sx, sy = src["slit_half"]
    edges = np.linspace(-1.0, 1.0, 41)
    px = bin_probs(uniform_cdf(-sx, sx), edges)
    py = bin_probs(uniform_cdf(-sy, sy), edges)
    chi2_check(psd, np.outer(px, py))
    assert psd.sum() == N


def test_uniform_gun_spectrum_is_flat_on_its_interval(orc):
    import json
    from pathlib import Path
    g = json.loads((Path(__file__).parent / "golden" / "uni_moderator_gun.json").read_text())
    src = W.moderator_source(mean_wl=g["parameters"]["mean_wl"], range_wl=g["parameters"]["range_wl"])
    assert math.isclose(src["lambda"][0], g["printed"]["lambda_min"])
    assert math.isclose(src["lambda"][1], g["printed"]["lambda_max"])
    desc, psd, spec = run(orc)
    lo, hi = desc["source"]["lambda"]
    assert (lo, hi) == src["lambda"]
    edges = np.linspace(0.2, 8.2, 61)
    chi2_check(spec, bin_probs(uniform_cdf(lo, hi), edges))


def test_downstream_plane_is_a_trapezoid_from_the_source_rectangle(orc):
    desc, psd, spec = run(orc, detector_z=40.0)
    src = desc["source"]
    # plane at z = +40 with moderator at -40 and slit at 0: x = 2 s_x - r_x
    ax, ay = 2 * src["slit_half"][0], 2 * src["slit_half"][1]
    bx, by = src["half"]
    edges = np.linspace(-8.0, 8.0, 41)
    px = bin_probs(sum_uniform_cdf(ax, bx), edges)
    py = bin_probs(sum_uniform_cdf(ay, by), edges)
    assert abs(px.sum() - 1) < 1e-12 and abs(py.sum() - 1) < 1e-12
    chi2_check(psd, np.outer(px, py))


@pytest.mark.parametrize("T", [293.15, 40.0])
def test_maxwellian_gun_spectrum_follows_the_maxwell_boltzmann_law(orc, T):
    from scipy.special import gammaincc
    desc, psd, spec = run(orc, temperature=T)
    C = 81.80420                  # h^2 / (2 m_n) in meV A^2
    kT = 0.08617333 * T           # meV
    edges = np.linspace(0.2, 8.2, 61)
    cdf = gammaincc(1.5, C / (kT * edges ** 2))
    chi2_check(spec, np.diff(cdf))
    # and the slit is still hit uniformly
    sx, sy = desc["source"]["slit_half"]
    e2 = np.linspace(-1.0, 1.0, 41)
    chi2_check(psd, np.outer(bin_probs(uniform_cdf(-sx, sx), e2), bin_probs(uniform_cdf(-sy, sy), e2)))


def test_trapezoid_cdf_helper_against_brute_force():
    rng = np.random.default_rng(7)
    x = rng.uniform(-0.5, 0.5, 2_000_000) + rng.uniform(-5.0, 5.0, 2_000_000)
    edges = np.linspace(-6, 6, 25)
    h = np.histogram(x, edges)[0] / x.size
    p = bin_probs(sum_uniform_cdf(0.5, 5.0), edges)
    assert np.abs(h - p).max() < 2e-3
