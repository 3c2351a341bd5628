"""Every oracle pin catches a plausible mistake.

For each function of the oracle this file plants one mistake of the kind a
reader could overlook -- a swapped constant, a dropped factor, a wrong sign or
index -- into a copy of oracle.c (tests/planted.py), runs the pin that covers
that function against the copy, and requires the pin to fail.  The pins are
the very test functions of the other oracle test files, called unchanged; the
planted copy replaces the oracle only for the duration of the call.  (The
newer pins -- 1/v law, parameter multipliers, radius binding, rod model,
radius-gradient interface term -- carry their planted variants in their own
files.)"""
import pytest

import test_oracle_chopper as CH
import test_oracle_orders as OR
import test_oracle_physics as PH
import test_oracle_rng_geometry as RG
import test_oracle_sources as SO
from planted import planted

THREADS = 8

# (name, (old, new) in oracle.c, the pin(s) that must fail: callables of the planted oracle module)
CASES = [
    ("Philox multipliers swapped",
     ("const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;", "const uint32_t M0 = 0xCD9E8D57u, M1 = 0xD2511F53u;"),
     [lambda o: RG.test_philox_matches_curand_host_generator(o, 4096)]),
    ("uniform without the half offset (0 reachable)",
     ("return ((double)a + 0.5) * (1.0 / 4294967296.0);", "return ((double)a) * (1.0 / 4294967296.0);"),
     [lambda o: RG.test_uniform_strictly_inside_unit_interval(o)]),
    ("box exit through the wrong slab",
     ("else if (v[a] < 0.0) { double t = (-p->p[a] - q[a]) / v[a];",
      "else if (v[a] < 0.0) { double t = (p->p[a] - q[a]) / v[a];"),
     [lambda o: RG.test_entry_and_exit_distances_match_ray_marching(o, 0)]),
    ("tube treated as a sphere in its exit distance",
     ("    double A = v[0] * v[0] + v[1] * v[1] + (is_tube ? 0.0 : v[2] * v[2]);\n    double B = q[0] * v[0] + q[1] * v[1] + (is_tube ? 0.0 : q[2] * v[2]);\n    double C2 = q[0] * q[0] + q[1] * q[1] + (is_tube ? 0.0 : q[2] * q[2]);\n    double t0, t1;",
      "    double A = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];\n    double B = q[0] * v[0] + q[1] * v[1] + q[2] * v[2];\n    double C2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];\n    double t0, t1;"),
     [lambda o: RG.test_entry_and_exit_distances_match_ray_marching(o, 1)]),
    ("box entry faces swapped",
     ("int fa = 2 * a, fb = 2 * a + 1;", "int fa = 2 * a + 1, fb = 2 * a;"),
     [lambda o: RG.test_box_entry_faces_enumerated(o)]),
    ("rotation with a sign slip",
     ("out[2] = mu * u[2] - st * t * cp;", "out[2] = mu * u[2] + st * t * cp;"),
     [lambda o: RG.test_rotation_preserves_norm_and_angle(o)]),
    ("weight compensation halved",
     ("P->w *= exp((sig_g - sig_t) * x);", "P->w *= exp(0.5 * (sig_g - sig_t) * x);"),
     [lambda o: PH.test_uncollided_slab_transmission_is_lambert_beer(o, THREADS, 3.0),
      lambda o: PH.test_zero_absorption_bias_is_exact_implicit_capture(o, THREADS)]),
    ("isotropic scattering only forward",
     ("double mu = 2.0 * xi[2] - 1.0, phi = 2.0 * PI * xi[3];", "double mu = xi[2], phi = 2.0 * PI * xi[3];"),
     [lambda o: PH.test_infinite_medium_moments(o, THREADS, 1.0)]),
    ("Bragg cut-off at d instead of 2d",
     ("if (2.0 * m->d[i] >= lambda) sum += m->mult[i] * m->F2[i] * m->d[i];",
      "if (m->d[i] >= lambda) sum += m->mult[i] * m->F2[i] * m->d[i];"),
     [lambda o: PH.test_bragg_sigma_against_reflection_enumeration(o)]),
    ("Bragg deflection by theta instead of 2 theta",
     ("        double mu = 1.0 - 2.0 * sb * sb;\n        double un[3];",
      "        double mu = sqrt(1.0 - sb * sb);\n        double un[3];"),
     [lambda o: PH.test_bragg_first_scatter_lines_and_frequencies(o, THREADS)]),
    ("mirror reflectivity without the one-half",
     ("else R = 0.5 * m->R0 * (1.0 - m->alpha", "else R = m->R0 * (1.0 - m->alpha"),
     [lambda o: PH.test_mirror_reflectivity_properties(o)]),
    ("half-strength specular reflection",
     ("for (int i = 0; i < 3; ++i) P->u[i] -= 2.0 * n[i] * un;", "for (int i = 0; i < 3; ++i) P->u[i] -= 1.0 * n[i] * un;"),
     [lambda o: PH.test_guide_bounce_count_closed_form(o, THREADS)]),
    ("density score function from absorption only",
     ("m->density_par == p) P->A[p] -= sig_t * x;", "m->density_par == p) P->A[p] -= sig[OR_P_ABS] * x;"),
     [lambda o: PH.test_density_gradient_of_uncollided_transmission(o, THREADS, 1.0)]),
    ("scatnum filter off by one",
     ("if (T->scat >= 0 && T->scat != P->nscat) continue;", "if (T->scat >= 0 && T->scat != P->nscat + 1) continue;"),
     [lambda o: OR.test_single_bragg_scatter_q_is_two_pi_over_d(o, THREADS)]),
    ("process chosen without its bias factor",
     ("cum += s->bias[mat * OR_NPROC + i] * sig[i];", "cum += sig[i];"),
     [lambda o: OR.test_biased_and_unbiased_agree_per_scattering_order(o, THREADS)]),
    ("one bias factor for every process of a material",
     ("sig_g += (mat >= 0 ? s->bias[mat * OR_NPROC + i] : 1.0) * sig[i];",
      "sig_g += (mat >= 0 ? s->bias[mat * OR_NPROC + 0] : 1.0) * sig[i];"),
     [lambda o: PH.test_zero_absorption_bias_with_scattering_matches_unbiased(o, THREADS)]),
    ("slit axes swapped in the moderator gun",
     ("g->c[0] + g->slit_half[0] * (2.0 * b[1] - 1.0) - P.r[0]", "g->c[0] + g->slit_half[1] * (2.0 * b[1] - 1.0) - P.r[0]"),
     [lambda o: SO.test_uniform_gun_hits_the_slit_uniformly(o)]),
    ("Maxwellian without the squared Box-Muller cosine",
     ("const double E = kT * (-log(a[2]) - log(a[3]) * c * c);", "const double E = kT * (-log(a[2]) - log(a[3]) * c);"),
     [lambda o: SO.test_maxwellian_gun_spectrum_follows_the_maxwell_boltzmann_law(o, 293.15)]),
    ("time of flight with h/m_n in m/s instead of cm/s",
     ("return path * lambda / 395603.4012;", "return path * lambda / 3956.034012;"),
     [lambda o: CH.test_tof_before_the_chopper_is_flat_for_a_uniform_wavelength(o)]),
    ("chopper turning the wrong way",
     ("const double centre = ch->phase + 2.0 * PI * ch->freq * t", "const double centre = ch->phase - 2.0 * PI * ch->freq * t"),
     [lambda o: CH.test_transmitted_fraction_and_spectrum_follow_the_open_intervals(o, 17.0, (-10.0, -16.0))]),
]


@pytest.mark.parametrize("name,plant,pins", CASES, ids=[c[0] for c in CASES])
def test_pin_fails_on_planted_mistake(name, plant, pins):
    with planted([plant]) as orc:
        for pin in pins:
            with pytest.raises(AssertionError):
                pin(orc)


def test_every_case_is_a_real_change():
    for name, (old, new), _ in CASES:
        assert old != new, name
