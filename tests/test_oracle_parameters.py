"""Pins of the oracle's wavelength law and parameter multipliers, each with
planted mistakes that must fail.

* 1/v absorption (§2.2): Sigma_a(lambda) = Sigma_a(1.8 A) lambda / 1.8.  With
  the absorption bias 0 (§3.5: a factor 0 removes the process from the
  sampling, reading R4) and no scattering, every neutron crosses the slab
  uncollided and its weight is exactly exp(-Sigma_a(lambda) t): a
  zero-variance pin at wavelengths where lambda/1.8 and 1.8/lambda differ.
* Multipliers (reading R10): the number density n multiplies every process of
  its material, the Bragg scale s only the Bragg term.  With every bias 0 the
  weight is exactly exp(-Sigma_t(n, s) t), so L(n, s) = -ln(T)/t must equal
  n (Sigma_a + Sigma_inc) + n s Sigma_B, with Sigma_B from the enumeration of
  individual reflections (independent of the oracle's line table).
* The radius binding: a tube whose radii follow the radius parameter must
  measure exactly like an explicit tube of the moved radii, inside and on
  rays, and its uncollided transmission must follow the chord-length
  integral of the moved radius."""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads as W
from planted import planted

T_SLAB = 1.0


def _absorber_slab(lam, sig_a=0.1, n=2000):
    d = W.slab(g=1.0, n_histories=n, precision="f64", sigma_s=0.0, sigma_a=sig_a, thickness=T_SLAB)
    d["source"] = dict(d["source"], **{"lambda": (lam, lam)})
    d["bias"] = np.array([[0.0, 1.0, 1.0]])
    return d


def _weights(orc, desc, n=2000):
    r = orc.OracleScene(desc).run(n, threads=2, records=True)
    return r["records"]["w_final"], r


LAMBDAS = (0.9, 1.8, 3.6, 5.4)


def _check_1v(orc):
    bad = []
    for lam in LAMBDAS:
        w, r = _weights(orc, _absorber_slab(lam))
        expect = math.exp(-0.1 * lam / 1.8 * T_SLAB)
        # the nudge into the slab shortens the path by 1e-9 cm
        if not np.allclose(w, expect, rtol=1e-9, atol=0):
            bad.append((lam, float(w.mean()), expect))
        # every history is scored once, uncollided, with that weight
        if abs(r["sum"][0] / len(w) - expect) > 1e-9 * expect:
            bad.append(("tally", lam))
    return bad


def test_one_over_v_absorption_is_exact(oracle_mod):
    assert _check_1v(oracle_mod) == []


@pytest.mark.parametrize("old,new", [
    ("m->sig_abs_ref * lambda / 1.8", "m->sig_abs_ref * 1.8 / lambda"),     # v instead of 1/v
    ("m->sig_abs_ref * lambda / 1.8", "m->sig_abs_ref"),                   # no wavelength law
    ("m->sig_abs_ref * lambda / 1.8", "m->sig_abs_ref * lambda * lambda / 3.24"),
])
def test_one_over_v_pin_catches_planted_mistakes(old, new):
    with planted([(old, new)]) as orc:
        assert _check_1v(orc) != []


# ---------------------------------------------------------------------------
# density and Bragg-scale multipliers
# ---------------------------------------------------------------------------
LAM = 1.5
SIG_A, SIG_INC = 0.05, 0.2


def _param_slab():
    lines = W.fcc_bragg_lines()
    world = {"shape": "sphere", "centre": (0, 0, 0.5), "params": (0.0, 100.0, 0.0)}
    prims = [W.prim("box", (0, 0, 0.5), (5.0, 5.0, 0.5), material=0)]
    mats = [W.material(sigma_abs_ref=SIG_A, abs_mode="const", sigma_inc=SIG_INC, bragg=lines,
                       density_param=0, scale_param=1)]
    src = {"kind": "pencil", "centre": (0.0, 0.0, -1.0), "half": (0.0, 0.0), "lambda": (LAM, LAM),
           "div": (0.0, 0.0), "aperture": None}
    tallies = [W.tally("count", "exit", 0, face=5, scat=0)]
    return W._scene("param-slab", world, prims, mats, [[0.0, 0.0, 0.0]], src, tallies, "f64", 1,
                    instances={"params": np.array([[1.0, 1.0]]), "counts": np.array([1])},
                    params=[{"kind": "density", "target": 0}, {"kind": "scale", "target": 0}])


def _bragg_by_reflections(lam, a=3.6, dmin=0.5):
    """Sigma_B(lambda) at n = s = 1 summed reflection by reflection."""
    lines = W.fcc_bragg_lines()
    f2 = dict(zip(lines["hkl_N"], lines["F2"]))
    nmax = (a / dmin) ** 2
    tot = 0.0
    for h in range(-8, 9):
        for k in range(-8, 9):
            for l in range(-8, 9):
                if (h, k, l) == (0, 0, 0) or len({h % 2, k % 2, l % 2}) != 1:
                    continue
                N = h * h + k * k + l * l
                d = a / math.sqrt(N)
                if N <= nmax + 1e-9 and 2 * d >= lam:
                    tot += f2[N] * d
    return lam ** 2 / (2 * a ** 6) * tot


PARAMS = [(1.0, 1.0), (2.0, 1.0), (0.5, 1.0), (1.0, 2.0), (1.0, 0.5), (2.0, 0.5), (0.5, 3.0)]


def _check_multipliers(orc):
    sb = _bragg_by_reflections(LAM)
    sc = orc.OracleScene(_param_slab())
    bad = []
    for n, s in PARAMS:
        r = sc.run(500, threads=2, params=[n, s], records=True)
        w = r["records"]["w_final"]
        L = -np.log(w) / T_SLAB
        expect = n * (SIG_A + SIG_INC) + n * s * sb
        if not np.allclose(L, expect, rtol=1e-8, atol=0):
            bad.append((n, s, float(L.mean()), expect))
    return bad


def test_density_and_scale_multipliers(oracle_mod):
    assert _bragg_by_reflections(LAM) > 0.05
    assert _check_multipliers(oracle_mod) == []


@pytest.mark.parametrize("old,new", [
    # density applied to absorption only
    ("  for (int i = 0; i < OR_NPROC; ++i) sig[i] *= dens;", "  sig[OR_P_ABS] *= dens;"),
    # scale applied to every process
    ("  for (int i = 0; i < OR_NPROC; ++i) sig[i] *= dens;", "  for (int i = 0; i < OR_NPROC; ++i) sig[i] *= dens * (i < 2 ? scale : 1.0);"),
    # scale forgotten
    ("(m->nlines > 0) ? scale * lambda", "(m->nlines > 0) ? lambda"),
    # scale squared (mistaken for an amplitude factor)
    ("(m->nlines > 0) ? scale * lambda", "(m->nlines > 0) ? scale * scale * lambda"),
])
def test_multiplier_pin_catches_planted_mistakes(old, new):
    with planted([(old, new)]) as orc:
        assert _check_multipliers(orc) != []


# ---------------------------------------------------------------------------
# radius binding
# ---------------------------------------------------------------------------
R_NOM = 0.5


def _bound_scene(R, explicit=False):
    """A shell tube (rmin bound) inside a solid tube of the same axis (rmax
    bound), both following the radius parameter; or, explicit, the same tubes
    sized for radius R without binding."""
    world = {"shape": "box", "centre": (0, 0, 0), "params": (20, 20, 20)}
    dR = R - R_NOM
    if explicit:
        prims = [W.prim("tube", (0, 0, 0), (0.0, R_NOM + dR, 2.0), material=0, axis=1),
                 W.prim("tube", (0, 0, 0), (R_NOM + dR, R_NOM + 0.1 + dR, 2.0), material=0, axis=1),
                 W.prim("sphere", (3, 0, 0), (0.2 + dR, 0.6 + dR, 0.0), material=0)]
    else:
        prims = [W.prim("tube", (0, 0, 0), (0.0, R_NOM, 2.0), material=0, axis=1, bind_rmax=True),
                 W.prim("tube", (0, 0, 0), (R_NOM, R_NOM + 0.1, 2.0), material=0, axis=1,
                        bind_rmin=True, bind_rmax=True),
                 W.prim("sphere", (3, 0, 0), (0.2, 0.6, 0.0), material=0, bind_rmin=True, bind_rmax=True)]
    src = {"kind": "rect", "centre": (0.0, 0.0, -5.0), "half": (1.0, 1.0), "lambda": (1.8, 1.8),
           "div": (0.0, 0.0), "aperture": None}
    return W._scene("bound", world, prims, [W.material(sigma_abs_ref=0.8, abs_mode="const")], [[1, 1, 1]],
                    src, [], "f64", 1,
                    instances={"params": np.array([[R]]), "counts": np.array([1]), "radius_nominal": R_NOM},
                    params=[{"kind": "radius", "target": -1}])


def _check_binding(orc, R):
    bound = orc.OracleScene(_bound_scene(R))
    expl = orc.OracleScene(_bound_scene(R, explicit=True))
    rng = np.random.Generator(np.random.PCG64(11))
    bad = 0
    for i in range(3):
        c = np.array([3.0, 0.0, 0.0]) if i == 2 else np.zeros(3)
        for _ in range(300):
            x = c + rng.uniform(-1.2, 1.2, size=3)
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            if bound.prim_inside(i, x, params=[R]) != expl.prim_inside(i, x):
                bad += 1
            for fn in ("prim_exit", "prim_entry"):
                if fn == "prim_exit" and not expl.prim_inside(i, x):
                    continue
                t1, f1 = getattr(bound, fn)(i, x, u, params=[R])
                t2, f2 = getattr(expl, fn)(i, x, u)
                if f1 != f2 or not (t1 == t2 or abs(t1 - t2) <= 1e-12 * max(1.0, abs(t2))):
                    bad += 1
    return bad


@pytest.mark.parametrize("R", [0.3, 0.5, 0.8])
def test_bound_radii_measure_like_explicit_radii(oracle_mod, R):
    assert _check_binding(oracle_mod, R) == 0


@pytest.mark.parametrize("old,new", [
    ("dR = ip[i] - s->radius_nominal", "dR = s->radius_nominal - ip[i]"),   # sign
    ("  if (p->bind_rmin) R.r0 += dR;\n", ""),                               # rmin not bound
])
def test_binding_pin_catches_planted_mistakes(old, new):
    with planted([(old, new)]) as orc:
        assert _check_binding(orc, 0.8) > 0


def test_uncollided_transmission_of_a_moved_cylinder(oracle_mod, threads):
    """A beam of half-width b on the bound solid tube at radius R != nominal
    (pure absorber Sigma = 0.8): T = 1 - [2R - int exp(-2 S sqrt(R^2-x^2)) dx]/2b."""
    S, b, R, n = 0.8, 1.0, 0.75, 400_000
    world = {"shape": "box", "centre": (0, 0, 0), "params": (20, 20, 20)}
    prims = [W.prim("tube", (0, 0, 0), (0.0, R_NOM, 5.0), material=0, axis=1, bind_rmax=True),
             W.prim("box", (0, 0, 10.0), (5.0, 5.0, 0.1), role="detector")]
    src = {"kind": "rect", "centre": (0.0, 0.0, -5.0), "half": (b, 1.0), "lambda": (1.8, 1.8),
           "div": (0.0, 0.0), "aperture": None}
    d = W._scene("cyl", world, prims, [W.material(sigma_abs_ref=S, abs_mode="const")], [[1, 1, 1]], src,
                 [W.tally("count", "entry", 1, scat=0)], "f64", 1,
                 instances={"params": np.array([[R]]), "counts": np.array([1]), "radius_nominal": R_NOM},
                 params=[{"kind": "radius", "target": -1}])
    r = oracle_mod.OracleScene(d).run(n, threads=threads)
    m = r["sum"][0] / n
    e = math.sqrt(max(r["sumsq"][0] / n - m * m, 0.0) / (n - 1))
    T_ref = 1 - (2 * R - integrate.quad(lambda x: math.exp(-2 * S * math.sqrt(R * R - x * x)), -R, R)[0]) / (2 * b)
    T_nom = 1 - (2 * R_NOM - integrate.quad(lambda x: math.exp(-2 * S * math.sqrt(R_NOM ** 2 - x * x)),
                                            -R_NOM, R_NOM)[0]) / (2 * b)
    assert abs(m - T_ref) < 4 * e, (m, T_ref, e)
    assert abs(T_ref - T_nom) > 20 * e    # the binding moved the result by far more than the noise
