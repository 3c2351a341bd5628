"""T6: the rod model through a finite slab -- the pin of the
scatter-and-continue loop in a bounded medium.

In the rod model (the oracle's test mode) every incoherent scattering sends
the neutron along +z or -z with probability 1/2 each.  A pencil beam normal to
a slab z in [0, t] then stays on the z axis, and the forward and backward
fluxes obey the two-stream equations (§2.2's Lambert-Beer attenuation between
collisions, Eq. eDistribition, with half the scattered flux turned around):

    d psi+/dz = -S_t psi+ + (S_s/2)(psi+ + psi-)
   -d psi-/dz = -S_t psi- + (S_s/2)(psi+ + psi-),   psi+(0) = 1, psi-(t) = 0,

a linear system solved exactly with a matrix exponential: transmission
T = psi+(t), reflection R = psi-(0).  The oracle must reproduce both, unbiased
and with biased flights (§2.4, Eqs. eStepLength2 and eWeight: the
probability-conserving weights keep the same expectation), and the planted
mistakes below must fail."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from planted import planted

T, S_S, S_A = 1.5, 0.8, 0.3
N = 400_000


def two_stream(t=T, ss=S_S, sa=S_A):
    st = ss + sa
    M = np.array([[-st + ss / 2, ss / 2], [-ss / 2, st - ss / 2]])
    E = expm(M * t)
    R = -E[1, 0] / E[1, 1]
    return E[0, 0] + E[0, 1] * R, R


def rod_slab(g):
    world = {"shape": "sphere", "centre": (0, 0, T / 2), "params": (0.0, 50.0, 0.0)}
    prims = [W.prim("box", (0, 0, T / 2), (5.0, 5.0, T / 2), material=0)]
    mat = W.material(sigma_abs_ref=S_A, abs_mode="const", sigma_inc=S_S)
    mat["rod"] = True
    src = {"kind": "pencil", "centre": (0.0, 0.0, -1.0), "half": (0.0, 0.0), "lambda": (1.8, 1.8),
           "div": (0.0, 0.0), "aperture": None}
    tallies = [W.tally("count", "exit", 0, face=5, name="T"), W.tally("count", "exit", 0, face=4, name="R"),
               W.tally("count", "exit", 0, name="any face")]
    return W._scene("rod", world, prims, [mat], [g], src, tallies, "f64", N)


BIASES = ([1.0, 1.0, 1.0], [3.0, 3.0, 3.0], [0.4, 0.4, 0.4], [0.5, 2.0, 1.0])


def _zscores(orc, g, n=N):
    r = orc.OracleScene(rod_slab(g)).run(n, threads=8)
    m = r["sum"] / n
    e = np.sqrt(np.maximum(r["sumsq"] / n - m * m, 0.0) / (n - 1))
    Tx, Rx = two_stream()
    return (m[0] - Tx) / e[0], (m[1] - Rx) / e[1], m, e


def test_closed_form_is_a_two_stream_solution():
    Tx, Rx = two_stream()
    # no scattering: Lambert-Beer; no absorption: T + R = 1 (conservation)
    assert two_stream(ss=0.0)[0] == pytest.approx(math.exp(-S_A * T), rel=1e-12)
    t0, r0 = two_stream(sa=0.0)
    assert t0 + r0 == pytest.approx(1.0, rel=1e-12)
    assert t0 == pytest.approx(1.0 / (1.0 + S_S * T / 2), rel=1e-12)   # pure scatterer: 1/(1 + S t/2)
    assert 0 < Tx < 1 and 0 < Rx < 1 and Tx + Rx < 1


@pytest.mark.parametrize("g", BIASES)
def test_rod_model_transmission_and_reflection(oracle_mod, g):
    zt, zr, m, e = _zscores(oracle_mod, g)
    assert abs(zt) < 4 and abs(zr) < 4, (zt, zr, m[:2], two_stream())
    # a rod neutron leaves only through the two faces it moves along
    assert m[2] == pytest.approx(m[0] + m[1], rel=1e-12)


PLANTS = {
    "no weight compensation": ("P->w *= exp((sig_g - sig_t) * x);", "P->w *= 1.0;"),
    "compensation of the wrong sign": ("P->w *= exp((sig_g - sig_t) * x);", "P->w *= exp((sig_t - sig_g) * x);"),
    "no division by g at a collision": ("P->w /= s->bias[mat * OR_NPROC + j];", "P->w /= 1.0;"),
    "rod turned back too often": ("(xi[2] < 0.5) ? -1.0 : 1.0", "(xi[2] < 0.6) ? -1.0 : 1.0"),
    "unbiased step length": ("double l = (sig_g > 0.0) ? -log(xi[0]) / sig_g : INFINITY;",
                             "double l = (sig_g > 0.0) ? -log(xi[0]) / sig_t : INFINITY;"),
}


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_rod_pin_catches_planted_mistakes(name):
    with planted([PLANTS[name]]) as orc:
        worst = 0.0
        for g in BIASES:
            zt, zr, _, _ = _zscores(orc, g, n=200_000)
            worst = max(worst, abs(zt), abs(zr))
        assert worst > 6, (name, worst)
