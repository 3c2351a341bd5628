"""The oracle's radius derivative with its interface term (reading R9), pinned
on a scattering cylinder against common-random-number finite differences of
the oracle's own plain runs -- nothing of the gradient machinery takes part in
the finite differences.

The sample cylinder sits in a can that follows its radius (inner R, outer
R + 0.15, a stronger scatterer than the sample), so moving R by dR turns a
layer of can into sample and a layer of vacuum into can.  The score-function part alone (the exponent term
-(Sigma_t,in - Sigma_t,out)/|n.u| per crossing) misses the collisions that
now happen in that layer; the oracle adds them as a derivative secondary per
crossing, weight w sign(c) C/|n.u|, transported to the detector.  Its
estimate of dTally/dR, accumulated in J, must equal
(Tally(R+h) - Tally(R-h)) / 2h bin by bin, where both runs use the same
history ids and seed (Philox keyed by history id), so the paired per-history
differences have a small variance.  Planted mistakes in the interface term
must fail the comparison."""
import math

import numpy as np
import pytest

import workloads as W
from planted import planted

R0, H = 0.5, 0.02
NBINS = 6
N = 1_500_000


def scatter_cylinder():
    world = {"shape": "box", "centre": (0, 0, 0), "params": (40, 40, 40)}
    prims = [W.prim("tube", (0, 0, 0), (0.0, R0, 1.0), material=0, axis=1, bind_rmax=True),
             W.prim("tube", (0, 0, 0), (R0, R0 + 0.15, 1.0), material=1, axis=1, bind_rmin=True, bind_rmax=True),
             W.prim("tube", (0, 0, 0), (10.0, 11.0, 30.0), role="detector", axis=1)]
    mats = [W.material(sigma_abs_ref=0.2, abs_mode="const", sigma_inc=0.6),
            W.material(sigma_abs_ref=0.05, abs_mode="const", sigma_inc=0.9)]
    src = {"kind": "rect", "centre": (0.0, 0.0, -5.0), "half": (1.0, 0.8), "lambda": (1.8, 1.8),
           "div": (0.0, 0.0), "aperture": None}
    tallies = [W.tally("angular", "entry", 2, bins=(NBINS, 1), lo=(0.0, 0.0), hi=(math.pi, 1.0),
                       origin=(0.0, 0.0, 0.0), axis=(0.0, 0.0, 1.0))]
    return W._scene("scatter-cyl", world, prims, mats, [[1, 1, 1], [1, 1, 1]], src, tallies, "f64", N,
                    instances={"params": np.array([[R0]]), "counts": np.array([N]), "radius_nominal": R0},
                    params=[{"kind": "radius", "target": -1}])


def per_history_bins(rec):
    """Detector bin of each history (-1 if not detected) and its weight."""
    det = rec["end"] == 2
    p = rec["final_pos"]
    ang = np.arccos(np.clip(p[:, 2] / np.linalg.norm(p, axis=1), -1.0, 1.0))
    b = np.minimum((ang / math.pi * NBINS).astype(int), NBINS - 1)
    return np.where(det, b, -1), np.where(det, rec["w_final"], 0.0)


def _compare(orc, n=N):
    sc = orc.OracleScene(scatter_cylinder())
    g = sc.run(n, threads=8, want_grad=True)
    J, J2 = g["J"][0], g["J2"][0]
    jm = J / n
    je = np.sqrt(np.maximum(J2 / n - jm * jm, 0.0) / (n - 1))
    runs = []
    for R in (R0 + H, R0 - H):
        r = sc.run(n, threads=8, params=[R], records=True)
        runs.append(per_history_bins(r["records"]))
    fd = np.zeros((n, NBINS))
    for sgn, (b, w) in zip((1.0, -1.0), runs):
        hit = b >= 0
        fd[np.nonzero(hit)[0], b[hit]] += sgn * w[hit] / (2 * H)
    fm = fd.mean(axis=0)
    fe = fd.std(axis=0, ddof=1) / math.sqrt(n)
    z = (jm - fm) / np.sqrt(je ** 2 + fe ** 2)
    return z, jm, fm


def test_radius_gradient_matches_crn_finite_differences(oracle_mod):
    z, jm, fm = _compare(oracle_mod)
    assert np.abs(z).max() < 4.5, (z, jm, fm)
    # the derivative is far from zero in the bins that carry the sample's scattering
    assert np.abs(fm).max() > 0.02


PLANTS = {
    "no derivative secondary": ("  transport(c, &S, hid, NULL, nsec);\n}", "  (void)S;\n}"),
    "secondary weight without its sign": ("S.w = P->w * (term[pick] > 0.0 ? 1.0 : -1.0) * C / cosn;",
                                          "S.w = P->w * C / cosn;"),
    "exponent term of the wrong sign": ("P->A[c->radius_par] -= (st_in - st_out) / cosn;",
                                        "P->A[c->radius_par] += (st_in - st_out) / cosn;"),
    "no obliquity factor": ("S.w = P->w * (term[pick] > 0.0 ? 1.0 : -1.0) * C / cosn;",
                            "S.w = P->w * (term[pick] > 0.0 ? 1.0 : -1.0) * C;"),
}


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_radius_gradient_pin_catches_planted_mistakes(name):
    with planted([PLANTS[name]]) as orc:
        z, jm, fm = _compare(orc, n=600_000)
        assert np.abs(z).max() > 6, (name, z)
