"""Per-scattering-order scorers (MultiScat, DeltaMomentum; Appendix C) in the
oracle, pinned by closed forms and by the probability-conservation claim of
§4.1 (biased and unbiased runs agree order by order)."""
import math

import numpy as np
import pytest

import workloads as W
from stats import compare_tallies, stats


def _sigma_t(oracle_mod, desc, lam):
    return oracle_mod.OracleScene(desc).sigma(0, lam).sum()


def test_unscattered_fraction_is_exp_minus_two_r_sigma(oracle_mod, threads):
    """A pencil along a diameter crosses 2R of sample: P(0 scatterings) = exp(-2 R Sigma_t)."""
    n = 400_000
    desc = W.total_scattering(n_histories=n, precision="f64")
    r = oracle_mod.OracleScene(desc).run(n, threads=threads)
    m, e = stats(r["sum"], r["sumsq"], n)
    st = _sigma_t(oracle_mod, desc, 1.0)
    assert abs(m[0] - math.exp(-2 * 1.2 * st)) < 4 * e[0], (m[0], math.exp(-2 * 1.2 * st))
    # every detected neutron is in exactly one MultiScat bin (orders >= 8 are rare)
    sc = oracle_mod.OracleScene(desc)
    q_all = r["sum"][sc.tally_off[1]:sc.tally_off[2]].sum() / n
    assert abs(m[:8].sum() - q_all) < 1e-3


def test_single_bragg_scatter_q_is_two_pi_over_d(oracle_mod, threads):
    """Bragg's law: one coherent elastic scatter off line d transfers
    Q = 2k sin(theta_B) = 2 pi / d, whatever the wavelength."""
    lines = W.fcc_bragg_lines()
    for lam in (0.9, 1.7):
        desc = W.total_scattering(n_histories=1, precision="f64", radius=0.05, lam=lam, nq=4000)
        desc["materials"][0]["sigma_inc"] = 0.0
        desc["materials"][0]["sigma_abs_ref"] = 0.0
        desc["bias"][0] = [1.0, 1.0, 200.0]      # make single scatters common; weights compensate
        n = 200_000
        sc = oracle_mod.OracleScene(desc)
        r = sc.run(n, threads=threads)
        off = sc.tally_off[2]                     # Q of neutrons scattered exactly once
        q1 = r["sum"][off:off + 4000]
        qmax = 4 * math.pi / lam
        edges = np.linspace(0, qmax, 4001)
        centres = 0.5 * (edges[1:] + edges[:-1])
        d = np.asarray(lines["d"])
        taus = 2 * math.pi / d[2 * d >= lam]
        near = np.zeros(4000, dtype=bool)
        for tq in taus:
            near |= np.abs(centres - tq) < 3 * (edges[1] - edges[0])
        assert q1.sum() > 0
        assert q1[near].sum() / q1.sum() > 0.999, lam


def test_biased_and_unbiased_agree_per_scattering_order(oracle_mod, threads):
    n = 1_000_000
    res = []
    for g in (1.0, 3.0):
        d = W.total_scattering(g=g, n_histories=n)
        r = oracle_mod.OracleScene(d).run(n, threads=threads)
        res.append(stats(r["sum"], r["sumsq"], n))
    (m1, e1), (m3, e3) = res
    ok, info = compare_tallies(m1, e1, m3, e3)
    assert ok, info


def test_absorption_bias_conserves_and_smooths_the_image(oracle_mod, threads):
    """§4.4: with abs_bias = 0.1 the transmission image is the same and less noisy."""
    n = 300_000
    out = {}
    for ab in (None, 0.1):
        d = W.imaging(n_histories=n, n_prims=150, psd_bins=8, abs_bias=ab, g_thin=1.0)
        r = oracle_mod.OracleScene(d).run(n, threads=threads)
        out[ab] = stats(r["sum"], r["sumsq"], n)
    (m1, e1), (m2, e2) = out[None], out[0.1]
    ok, info = compare_tallies(m1, e1, m2, e2)
    assert ok, info
    # implicit capture never adds noise (here the pixel choice dominates the noise)
    assert np.median(e2 / np.maximum(e1, 1e-300)) < 1.0


@pytest.mark.parametrize("g", [0.1, 0.5, 1.0])
def test_absorption_bias_second_moment_closed_form(oracle_mod, threads, g):
    """Pure absorber of optical depth S t with absorption bias g: a history
    passes with probability exp(-g S t) carrying w = exp((g-1) S t), so
    E[w] = exp(-S t) and E[w^2] = exp((g-2) S t) exactly."""
    n = 400_000
    S = 0.5
    d = W.slab(g=1.0, n_histories=n, sigma_s=0.0, sigma_a=S)
    d["bias"][0] = [g, 1.0, 1.0]
    r = oracle_mod.OracleScene(d).run(n, threads=threads)
    m1 = r["sum"][1] / n
    m2 = r["sumsq"][1] / n
    e1 = math.sqrt(max(m2 - m1 * m1, 0) / n)
    assert abs(m1 - math.exp(-S)) < 4 * e1 + 1e-12
    expect2 = math.exp((g - 2) * S)
    # the second moment's own standard error: w^2 takes one value
    w2 = math.exp(2 * (g - 1) * S)
    e2 = w2 * math.sqrt(math.exp(-g * S) * (1 - math.exp(-g * S)) / n)
    assert abs(m2 - expect2) < 4 * e2 + 1e-12, (m2, expect2)
