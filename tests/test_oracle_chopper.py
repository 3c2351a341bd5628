"""Pins of the oracle's disk chopper (ray-tracing mode, Eq. eRayTracing, §3.5)
and time-of-flight scorer (TOF, Appendix C).

A pencil beam meets the disk at one radius rho0 and angle phi0, so
everything has a closed form:

* before the chopper the time of flight is t = L lambda / (h / m_n) with L
  the flight path: a uniform wavelength gives a flat spectrum on
  [L lambda_lo, L lambda_hi] / (h / m_n), a Maxwellian one
  P(T <= t) = Q(3/2, C / (kT lambda(t)^2)) (C = h^2 / (2 m_n));
* in turns tau = f t, the chopper is open at the beam for tau within
  theta0 / (4 pi) of alpha - j / n (any integer j), alpha = (phi0 - phase) /
  (2 pi): the transmitted spectrum is the flat one restricted to that set,
  and the transmitted fraction its measure.  This is computed from the open
  intervals in time, not from the per-neutron mask the oracle evaluates;
* inside r_black the disk is black.

The chopper study of §4.5 gives the golden values (tests/golden/
chopper_study.json): the peaks behind the chopper repeat at the window rate."""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import workloads as W
from stats import chi2_sf

N = 400_000
H_OVER_MN = 395603.4012      # cm/s at 1 A: CODATA h / m_n
GOLDEN = json.loads((Path(__file__).parent / "golden" / "chopper_study.json").read_text())


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def run(orc, desc, n=N):
    out = orc.OracleScene(desc).run(n, threads=8)
    nb = desc["tallies"][0]["bins"][0]
    s = out["sum"]
    return s[:nb], s[nb:2 * nb], s[2 * nb], out


def chi2_check(counts, probs, n, p_min=1e-4):
    counts = np.asarray(counts, dtype=np.float64)
    exp = n * np.asarray(probs, dtype=np.float64)
    assert counts[exp == 0.0].sum() == 0.0
    use = exp >= 5.0
    chi2 = float((((counts[use] - exp[use]) ** 2) / exp[use]).sum())
    p = chi2_sf(chi2, int(use.sum()) - 1)
    assert p >= p_min, (chi2, int(use.sum()), p)


def flight_path(desc):
    """Gun to the front face of the disk (the ENTRY point)."""
    return W.CHOPPER_DISTANCE - desc["prims"][0]["params"][2]


def open_measure(t_lo, t_hi, desc):
    """Measure of {t in [t_lo, t_hi] : a window is on the beam}."""
    ch = desc["prims"][0]["chopper"]
    cx, cy = desc["prims"][0]["centre"][:2]
    phi0 = math.atan2(0.0 - cy, 0.0 - cx)
    f, n, h = ch["freq"], ch["n"], ch["theta0"] / (4 * math.pi)
    alpha = (phi0 - ch["phase"]) / (2 * math.pi)
    if f == 0.0:
        d = (alpha * n - round(alpha * n)) / n
        return (t_hi - t_lo) if abs(d) <= h else 0.0
    s_lo, s_hi = sorted((f * t_lo, f * t_hi))
    total = 0.0
    for j in range(math.floor((alpha - s_hi) * n) - 2, math.ceil((alpha - s_lo) * n) + 3):
        c = alpha - j / n
        total += max(0.0, min(s_hi, c + h) - max(s_lo, c - h))
    return total / abs(f)


def test_tof_before_the_chopper_is_flat_for_a_uniform_wavelength(orc):
    desc = W.chopper_pencil(n_histories=N)
    before, after, trans, out = run(orc, desc)
    L = flight_path(desc)
    t1, t2 = (L * lam / H_OVER_MN for lam in desc["source"]["lambda"])
    edges = np.linspace(0.0, 0.025, 201)
    probs = np.clip((np.minimum(edges[1:], t2) - np.maximum(edges[:-1], t1)) / (t2 - t1), 0.0, None)
    chi2_check(before, probs, N)
    assert before.sum() == N


@pytest.mark.parametrize("T", [293.0, 60.0])
def test_tof_before_the_chopper_of_a_maxwellian_pencil(orc, T):
    from scipy.special import gammaincc
    desc = W.chopper_pencil(n_histories=N, temperature=T)
    before, after, trans, out = run(orc, desc)
    L = flight_path(desc)
    edges = np.linspace(0.0, 0.025, 201)
    lam = edges[1:] * H_OVER_MN / L
    cdf = np.concatenate([[0.0], gammaincc(1.5, 81.80420 / (0.08617333 * T * lam ** 2))])
    chi2_check(before, np.diff(cdf), N)


@pytest.mark.parametrize("phase_deg,centre", [(17.0, (-10.0, -16.0)), (-40.0, (12.0, 9.0)),
                                              (3.0, (0.0, -19.0))])
def test_transmitted_fraction_and_spectrum_follow_the_open_intervals(orc, phase_deg, centre):
    desc = W.chopper_pencil(n_histories=N, phase_deg=phase_deg, disk_centre=centre)
    before, after, trans, out = run(orc, desc)
    L = flight_path(desc)
    t1, t2 = (L * lam / H_OVER_MN for lam in desc["source"]["lambda"])
    p = open_measure(t1, t2, desc) / (t2 - t1)
    sd = math.sqrt(p * (1 - p) / N)
    assert abs(trans / N - p) <= 4.5 * sd, (trans / N, p, sd)
    assert after.sum() == trans
    edges = np.linspace(0.0, 0.025, 201)
    probs = np.array([open_measure(max(a, t1), min(b, t2), desc) if b > t1 and a < t2 else 0.0
                      for a, b in zip(edges[:-1], edges[1:])]) / (t2 - t1)
    chi2_check(after, probs, N)


def test_disk_is_black_inside_its_inner_radius(orc):
    desc = W.chopper_pencil(n_histories=20_000, disk_centre=(0.0, -12.0))   # rho0 = 12 < 13
    before, after, trans, out = run(orc, desc, n=20_000)
    assert before.sum() == 20_000 and trans == 0 and after.sum() == 0


def test_static_disk_is_open_or_closed_by_its_phase(orc):
    # freq 0: window 0 at `phase`; the beam sits at 90 degrees
    for phase, expect in ((90.0, 1.0), (80.5, 1.0), (79.0, 0.0), (45.0, 0.0), (0.0, 1.0)):
        desc = W.chopper_pencil(n_histories=5_000, disk_centre=(0.0, -19.0), phase_deg=phase, freq=0.0)
        before, after, trans, out = run(orc, desc, n=5_000)
        assert trans / 5_000 == expect, phase


def test_chopper_study_peaks_repeat_at_the_window_rate(orc):
    """§4.5: eight peaks behind the chopper, one per window passage."""
    g = GOLDEN
    desc = W.chopper(n_histories=N, precision="f64")
    assert desc["prims"][0]["chopper"]["n"] == g["setup"]["n_windows"]
    assert desc["prims"][0]["chopper"]["freq"] == g["setup"]["freq_hz"]
    before, after, trans, out = run(orc, desc)
    dt = 0.025 / after.size
    nz = np.nonzero(after)[0]
    # peaks: runs of non-empty bins, gaps shorter than 0.4 ms merged
    runs, start = [], nz[0]
    for a, b in zip(nz[:-1], nz[1:]):
        if (b - a) * dt > 4e-4:
            runs.append((start, a))
            start = b
    runs.append((start, nz[-1]))
    peaks = [((lo + hi + 1) * 0.5 * dt, after[lo:hi + 1].sum()) for lo, hi in runs]
    peaks = [t for t, c in peaks if c >= 100]
    spacing = g["peak_spacing_s"]
    assert abs(1.0 / (g["setup"]["n_windows"] * g["setup"]["freq_hz"]) - spacing) < 1e-12
    assert abs(g["printed"]["window_rate_hz"] * spacing - 1.0) < 1e-12
    in_range = [t for t in peaks if spacing * 0.8 <= t <= spacing * g["printed"]["n_peaks"] * 1.05]
    assert len(in_range) == g["printed"]["n_peaks"], peaks
    assert np.all(np.abs(np.diff(in_range) - spacing) < 1e-4), np.diff(in_range)
    # the chopper passes about n theta0 / 2 pi of a beam much narrower than a window period
    assert 0.15 < trans / N < 0.3
