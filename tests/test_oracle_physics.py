"""Pins of the oracle's transport against closed forms, invariants and
independent enumerations (nothing here re-calls the oracle's own formulas)."""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads as W
from stats import compare_tallies, stats

PENCIL = {"kind": "pencil", "centre": (0.0, 0.0, -1.0), "half": (0.0, 0.0), "lambda": (1.8, 1.8),
          "div": (0.0, 0.0), "aperture": None}


# ---------------------------------------------------------------------------
# T1: Lambert-Beer (Eq. eDistribition) for the uncollided beam, biased or not
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("g", [1.0, 3.0, 0.4])
def test_uncollided_slab_transmission_is_lambert_beer(oracle_mod, threads, g):
    n = 400_000
    sc = oracle_mod.OracleScene(W.slab(g=g, n_histories=n))
    r = sc.run(n, threads=threads)
    m, e = stats(r["sum"], r["sumsq"], n)
    expect = math.exp(-0.6)
    assert abs(m[0] - expect) < 4 * e[0], (m[0], e[0])


# ---------------------------------------------------------------------------
# T2: a bias factor of 0 removes the process (§3.5); for absorption that is
# implicit capture, exact per history
# ---------------------------------------------------------------------------
def test_zero_absorption_bias_is_exact_implicit_capture(oracle_mod, threads):
    n = 20_000
    d = W.slab(g=1.0, n_histories=n, sigma_s=0.0, sigma_a=0.1)
    d["bias"][0] = [0.0, 1.0, 1.0]
    sc = oracle_mod.OracleScene(d)
    r = sc.run(n, threads=threads, records=True)
    w = r["records"]["w_final"]
    # identical for every history (zero variance); equal to exp(-Sigma_a t) up to
    # the 1e-9 cm step taken off the path where the neutron enters the slab
    assert w.max() - w.min() == 0.0
    assert np.all(np.abs(w / math.exp(-0.1) - 1.0) < 2e-10)
    m, e = stats(r["sum"], r["sumsq"], n)
    # the stderr is zero up to the cancellation floor of sum(w^2)/N - mean^2
    assert abs(m[0] / math.exp(-0.1) - 1) < 2e-10 and e[0] < 1e-8
    assert abs(m[1] / math.exp(-0.1) - 1) < 2e-10


def test_zero_absorption_bias_with_scattering_matches_unbiased(oracle_mod, threads):
    n = 400_000
    a = oracle_mod.OracleScene(W.slab(g=1.0, n_histories=n)).run(n, threads=threads)
    d = W.slab(g=1.0, n_histories=n)
    d["bias"][0] = [0.0, 1.0, 1.0]
    b = oracle_mod.OracleScene(d).run(n, threads=threads)
    ma, ea = stats(a["sum"], a["sumsq"], n)
    mb, eb = stats(b["sum"], b["sumsq"], n)
    ok, info = compare_tallies(ma, ea, mb, eb)
    assert ok, info
    # implicit capture cannot increase the variance of the transmission
    assert eb[1] <= ea[1] * 1.02


# ---------------------------------------------------------------------------
# T3: probability conservation -- biased and unbiased tallies agree (§4.1)
# ---------------------------------------------------------------------------
def test_biased_and_unbiased_slab_tallies_agree(oracle_mod, threads):
    n = 600_000
    res = []
    for g in (1.0, 3.0):
        r = oracle_mod.OracleScene(W.slab(g=g, n_histories=n)).run(n, threads=threads)
        res.append(stats(r["sum"], r["sumsq"], n))
    (m1, e1), (m3, e3) = res
    # Escape near 90 degrees runs along the 10 cm wide slab: with g = 3 a path of
    # x cm survives with probability exp(-3 Sigma_t x) and carries the weight
    # exp(2 Sigma_t x), so those bins are heavy-tailed and their sample variance
    # understates the error.  Compare them only through the integrated total.
    keep = np.ones_like(m1, dtype=bool)
    keep[2 + 80:2 + 100] = False
    ok, info = compare_tallies(m1[keep], e1[keep], m3[keep], e3[keep])
    assert ok, info
    # integrated escape over all angles
    assert abs(m1[2:].sum() - m3[2:].sum()) < 4 * math.sqrt((e1[2:] ** 2).sum() + (e3[2:] ** 2).sum()) + 1e-3


# ---------------------------------------------------------------------------
# T4/T5: infinite medium with isotropic scattering.  Per history: collisions
# N ~ geometric with mean Sigma_t/Sigma_a, flights ~ Exp(Sigma_t), directions
# after a scatter isotropic and independent:
#   E[nscat] = Sigma_s/Sigma_a,  E[z] = 1/Sigma_t (first flight along +z),
#   E[x^2] = E[y^2] = (2/Sigma_t^2) E[nscat] / 3,  E[r^2] = 2/(Sigma_a Sigma_t).
# With bias g the weighted means are the same (Eq. eWeight).
# ---------------------------------------------------------------------------
def _infinite_medium(g):
    world = {"shape": "sphere", "centre": (0, 0, 0), "params": (0.0, 1e4, 0.0)}
    prims = [W.prim("sphere", (0, 0, 0), (0.0, 1e3, 0.0), material=0)]
    src = dict(PENCIL, centre=(0.0, 0.0, 0.0))
    d = W._scene("inf", world, prims, [W.material(sigma_abs_ref=0.1, abs_mode="const",
                                                  sigma_inc=0.5)],
                 [[g, g, g]], src, [], "f64", 1)
    return d


@pytest.mark.parametrize("g", [1.0, 2.0])
def test_infinite_medium_moments(oracle_mod, threads, g):
    n = 200_000
    sc = oracle_mod.OracleScene(_infinite_medium(g))
    rec = sc.run(n, threads=threads, records=True)["records"]
    assert np.all(rec["end"] == 1)   # absorbed
    w = rec["w_final"]
    r = rec["final_pos"]
    st, sa = 0.6, 0.1
    checks = {
        "nscat": (rec["nscat"].astype(float), 0.5 / 0.1),
        "z": (r[:, 2], 1.0 / st),
        "x": (r[:, 0], 0.0),
        "y": (r[:, 1], 0.0),
        "x2": (r[:, 0] ** 2, (2 / st ** 2) * (0.5 / 0.1) / 3),
        "y2": (r[:, 1] ** 2, (2 / st ** 2) * (0.5 / 0.1) / 3),
        "r2": ((r ** 2).sum(1), 2 / (sa * st)),
    }
    for name, (v, expect) in checks.items():
        x = w * v
        mean = x.mean()
        err = x.std() / math.sqrt(n)
        assert abs(mean - expect) < 4.5 * err + 1e-12, (name, mean, expect, err)


# ---------------------------------------------------------------------------
# T7: powder Bragg lines
# ---------------------------------------------------------------------------
def _reflections(a=3.6, dmin=0.5):
    """Every individual fcc reflection (h,k,l) with d >= dmin, by enumeration."""
    out = []
    nmax = (a / dmin) ** 2
    for h in range(-8, 9):
        for k in range(-8, 9):
            for l in range(-8, 9):
                if (h, k, l) == (0, 0, 0) or len({h % 2, k % 2, l % 2}) != 1:
                    continue
                N = h * h + k * k + l * l
                if N <= nmax + 1e-9:
                    out.append(N)
    return out


def _powder_material_scene(lines, inc=0.0, g=1.0):
    world = {"shape": "sphere", "centre": (0, 0, 0), "params": (0.0, 1e4, 0.0)}
    prims = [W.prim("sphere", (0, 0, 0), (0.0, 1e3, 0.0), material=0)]
    src = dict(PENCIL, centre=(0.0, 0.0, 0.0), **{"lambda": (1.5, 1.5)})
    return W._scene("powder-inf", world, prims,
                    [W.material(sigma_inc=inc, bragg=lines)], [[g, g, g]], src, [], "f64", 1)


def test_bragg_sigma_against_reflection_enumeration(oracle_mod):
    lines = W.fcc_bragg_lines()
    assert len(lines["d"]) == 18 and sum(lines["mult"]) == 386
    f2_of_N = dict(zip(lines["hkl_N"], lines["F2"]))
    refl = _reflections()
    a = 3.6
    sc = oracle_mod.OracleScene(_powder_material_scene(lines))
    V0 = a ** 3
    for lam in (0.9, 1.2, 1.5, 1.8, 2.5, 3.0, 4.0, 4.15, 4.16, 5.0):
        s = sum(f2_of_N[N] * a / math.sqrt(N) for N in refl if 2 * a / math.sqrt(N) >= lam)
        expect = lam ** 2 / (2 * V0 ** 2) * s
        got = sc.sigma(0, lam)[2]
        assert got == pytest.approx(expect, rel=1e-12, abs=1e-15), lam
    # the Bragg edge: nothing beyond lambda = 2 d_max
    dmax = a / math.sqrt(3)
    assert sc.sigma(0, 2 * dmax * (1 + 1e-9))[2] == 0.0
    assert sc.sigma(0, 2 * dmax * (1 - 1e-9))[2] > 0.0
    # order of magnitude quoted for this workload: ~0.07/cm at 1.5 A for |F|^2 ~ 1 b
    unit = dict(lines, F2=[1.0] * 18)
    s1 = oracle_mod.OracleScene(_powder_material_scene(unit)).sigma(0, 1.5)[2]
    assert 0.05 < s1 < 0.08


def test_bragg_first_scatter_lines_and_frequencies(oracle_mod, threads):
    """First collisions in an infinite pure-Bragg medium: the deflection takes
    only the values 2 asin(lambda/2d) of the active lines, with frequencies
    proportional to m |F|^2 d, and a uniform azimuth."""
    lines = W.fcc_bragg_lines()
    n = 300_000
    sc = oracle_mod.OracleScene(_powder_material_scene(lines))
    rec = sc.run(n, threads=threads, records=True)["records"]
    u = rec["dir_after_first"]
    assert not np.isnan(u).any()
    lam = 1.5
    d = np.asarray(lines["d"])
    active = 2 * d >= lam
    cos2t = 1 - 2 * (lam / (2 * d[active])) ** 2
    idx = np.argmin(np.abs(u[:, 2][:, None] - cos2t[None, :]), axis=1)
    assert np.max(np.abs(u[:, 2] - cos2t[idx])) < 1e-12
    p = (np.asarray(lines["mult"]) * np.asarray(lines["F2"]) * d)[active]
    p = p / p.sum()
    counts = np.bincount(idx, minlength=active.sum())
    chi2 = ((counts - n * p) ** 2 / (n * p)).sum()
    from stats import chi2_sf
    assert chi2_sf(chi2, active.sum() - 1) > 1e-3, (counts, n * p)
    phi = np.arctan2(u[:, 1], u[:, 0])
    assert abs(np.cos(phi).mean()) < 4 / math.sqrt(2 * n)
    assert abs(np.sin(phi).mean()) < 4 / math.sqrt(2 * n)


# ---------------------------------------------------------------------------
# T8: supermirror (§2.5)
# ---------------------------------------------------------------------------
def test_mirror_reflectivity_properties(oracle_mod):
    t = W.MIRROR_TABLE
    for m in (1.0, 2.0, 3.0):
        R = lambda Q: oracle_mod.mirror_R(Q, m, t["R0"], t["Qc"], t["alpha"], t["W"])
        # below the critical wavenumber: the low-angle reflectivity of the table
        for Q in (0.0, 0.01, t["Qc"]):
            assert R(Q) == t["R0"]
        # continuous at Qc for m > 1
        if m > 1:
            assert abs(R(t["Qc"] * (1 + 1e-9)) - t["R0"]) < 1e-5
        # at Q = m Qc the cut-off factor is exactly one half of its plateau
        Qm = m * t["Qc"]
        plateau = t["R0"] * (1 - t["alpha"] * (Qm - t["Qc"]))
        if m > 1:
            assert R(Qm) == pytest.approx(0.5 * plateau, rel=1e-12)
        # non-increasing above Qc, non-negative, vanishing far above m Qc
        Qs = np.linspace(t["Qc"], 0.5, 2000)
        vals = np.array([R(q) for q in Qs])
        assert np.all(np.diff(vals) <= 1e-15) and np.all(vals >= 0.0)
        assert R(m * t["Qc"] + 20 * t["W"]) < 1e-12


def _guide_1d(length=300.0, lam=5.0, div_deg=1.0):
    d = W.guide(n_histories=1, length=length)
    d["source"] = dict(d["source"], **{"lambda": (lam, lam), "div": (math.radians(div_deg), 0.0),
                                        "aperture": (2.5, 2.5), "half": (2.5, 2.5)})
    return d


def test_guide_bounce_count_closed_form(oracle_mod, threads):
    """1-D divergence in a straight guide: unfolding the reflections, a neutron
    starting at x0 with angle theta meets floor((X + a)/(2a)) walls (in absolute
    value) for X = x0 + L tan(theta); its final weight is R(Q)^N with
    Q = 4 pi sin(theta)/lambda, and it leaves at the folded X."""
    L, lam, a = 300.0, 5.0, 2.5
    desc = _guide_1d(L, lam)
    sc = oracle_mod.OracleScene(desc)
    n = 3000
    rec = sc.run(n, threads=threads, records=True)["records"]
    key = (W.SEED_TRANSPORT & 0xffffffff, W.SEED_TRANSPORT >> 32)
    mir = desc["prims"][0]["mirror"]
    checked = 0
    for h in range(n):
        o = oracle_mod.philox((0, 0, h, 0), key)
        u01 = [(v + 0.5) / 2 ** 32 for v in o]
        x0 = 2.5 * (2 * u01[0] - 1)
        y0 = 2.5 * (2 * u01[1] - 1)
        th = math.radians(1.0) * (2 * u01[3] - 1)
        X = x0 + L * math.tan(th)
        N = abs(math.floor((X + a) / (2 * a)))
        Q = 4 * math.pi * abs(math.sin(th)) / lam
        R = oracle_mod.mirror_R(Q, mir["m"], mir["R0"], mir["Qc"], mir["alpha"], mir["W"])
        # folded exit position
        k = math.floor((X + a) / (2 * a))
        xf = X - 2 * a * k
        if k % 2:
            xf = -xf
        assert rec["end"][h] == 2   # detected
        assert rec["w_final"][h] == pytest.approx(R ** N, rel=1e-9, abs=1e-300)
        assert rec["final_pos"][h][0] == pytest.approx(xf, abs=1e-6)
        assert rec["final_pos"][h][1] == pytest.approx(y0, abs=1e-9)
        checked += N > 0
    assert checked > 500


# ---------------------------------------------------------------------------
# T10: score-function gradients against closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("g", [1.0, 3.0])
def test_density_gradient_of_uncollided_transmission(oracle_mod, threads, g):
    """T = exp(-n Sigma_t t)  =>  dT/dln n = -n Sigma_t t T."""
    n = 400_000
    d = W.slab(g=g, n_histories=n)
    d["materials"][0]["density_param"] = 0
    d["params"] = [{"kind": "density", "target": 0}]
    d["instances"] = {"params": np.ones((1, 1)), "counts": np.array([n])}
    sc = oracle_mod.OracleScene(d)
    r = sc.run(n, threads=threads, want_grad=True)
    gm, ge = stats(r["J"][0], r["J2"][0], n)
    expect = -0.6 * math.exp(-0.6)
    assert abs(gm[0] - expect) < 4 * ge[0], (gm[0], ge[0], expect)


def _cylinder_uncollided_scene(R, sig, b=1.0, g=1.0):
    world = {"shape": "box", "centre": (0, 0, 0), "params": (20, 20, 20)}
    prims = [W.prim("tube", (0, 0, 0), (0.0, R, 5.0), material=0, axis=1, bind_rmax=True),
             W.prim("box", (0, 0, 10.0), (5.0, 5.0, 0.1), role="detector")]
    src = {"kind": "rect", "centre": (0.0, 0.0, -5.0), "half": (b, 1.0), "lambda": (1.8, 1.8),
           "div": (0.0, 0.0), "aperture": None}
    tallies = [W.tally("count", "entry", 1, scat=0, name="uncollided")]
    d = W._scene("cyl", world, prims, [W.material(sigma_abs_ref=sig, abs_mode="const")],
                 [[g, g, g]], src, tallies, "f64", 1,
                 instances={"params": np.array([[R]]), "counts": np.array([1]),
                            "radius_nominal": R},
                 params=[{"kind": "radius", "target": -1}])
    return d


def test_radius_gradient_of_uncollided_cylinder_transmission(oracle_mod, threads):
    """Parallel beam of half-width b on a cylinder of radius R (pure absorber):
    T(R) = 1 - [2R - int_{-R}^{R} exp(-2 S sqrt(R^2-x^2)) dx] / 2b, so
    dT/dR = (1/2b) int_{-pi/2}^{pi/2} -2 S R exp(-2 S R cos p) dp."""
    R, S, b = 0.5, 0.8, 1.0
    n = 400_000
    sc = oracle_mod.OracleScene(_cylinder_uncollided_scene(R, S, b))
    r = sc.run(n, threads=threads, want_grad=True)
    m, e = stats(r["sum"], r["sumsq"], n)
    T_ref = 1 - (2 * R - integrate.quad(lambda x: math.exp(-2 * S * math.sqrt(R * R - x * x)),
                                        -R, R)[0]) / (2 * b)
    assert abs(m[0] - T_ref) < 4 * e[0]
    dT_ref = integrate.quad(lambda p: -2 * S * R * math.exp(-2 * S * R * math.cos(p)),
                            -math.pi / 2, math.pi / 2)[0] / (2 * b)
    gm, ge = stats(r["J"][0], r["J2"][0], n)
    assert abs(gm[0] - dT_ref) < 4 * ge[0], (gm[0], ge[0], dT_ref)


@pytest.mark.parametrize("lam", [1.5, 2.5])
def test_powder_bragg_prefactor_from_orientation_averaged_single_crystal(lam):
    """The absolute powder Bragg cross section of the oracle (the powder
    average of Eq. eCohEla) against an independent route: the kinematic
    single-crystal cross section of one reflection, lambda^3 |F|^2 /
    (V0 sin 2theta_B) times a narrow rocking profile (Gaussian, width eta) in
    the glancing angle, averaged by Monte Carlo over uniformly random crystal
    orientations (random lattice-plane normals on the sphere).  Summed over
    the reflections (a +-G pair reflects at most once per orientation) and
    divided by V0, it must give the oracle's Sigma_Bragg(lambda)."""
    from oracle import oracle as O
    O.build()
    desc = W.powder(n_histories=1)
    lines = W.fcc_bragg_lines()
    d = np.asarray(lines["d"]); m = np.asarray(lines["mult"]); F2 = np.asarray(lines["F2"]); V0 = lines["V0"]
    rng = np.random.default_rng(2024)
    n = rng.normal(size=(8_000_000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    theta = np.arcsin(np.abs(n[:, 2]))          # glancing angle of a beam along z on the planes
    eta = 0.003
    sigma_cell = 0.0                             # barn per unit cell
    for di, mi, fi in zip(d, m, F2):
        s = lam / (2.0 * di)
        if s >= 1.0:
            continue                             # no Bragg angle: beyond the edge
        tb = np.arcsin(s)
        w = np.exp(-0.5 * ((theta - tb) / eta) ** 2) / (math.sqrt(2 * math.pi) * eta)
        per_pair = lam ** 3 * fi / (V0 * math.sin(2 * tb)) * w.mean()
        sigma_cell += 0.5 * mi * per_pair
    expect = sigma_cell / V0                     # barn / A^3 = 1/cm
    got = O.OracleScene(desc).sigma(0, lam)[2]
    assert abs(got - expect) <= 0.01 * expect, (got, expect)
