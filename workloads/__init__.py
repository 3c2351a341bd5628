"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only *describes* workloads: geometry, material constants, Bragg line
lists, source and tally definitions, per-instance parameters.  It contains none of
the transport arithmetic (no cross-section evaluation, no sampling, no weights);
both sides turn these plain-Python descriptions into their own structures.

Units: lengths in cm, wavelengths in Angstrom, macroscopic cross sections in 1/cm,
|F|^2 in barn, unit-cell volume in Angstrom^3, angles in radians.

The five workloads stand in for the paper's experiments (the datasets those used
are not available): a slab for the total-scattering biasing study (§4.1), a powder
diffractometer for §4.2, a supermirror guide for §4.3, a batched powder study with
gradients, and a CSG imaging scene for the complex-geometry study (§4.4).
"""
from __future__ import annotations

import math
from typing import Any

import numpy as np

# Seeds (the transport seed mirrors the launcher default of §3, Table "tableLaunch").
SEED_TRANSPORT = 4096
SEED_TABLE = 12345
SEED_SCENE = 2024

BOX, TUBE, SPHERE = "box", "tube", "sphere"
ABS, INC, BRAGG = 0, 1, 2          # process order used on both sides
NPROC = 3

# Mirror constants of §2.5, Table "tableMirror" (alpha there is 6.07; the guide
# workload uses 3.0).
MIRROR_TABLE = {"R0": 0.99, "Qc": 0.0219, "alpha": 6.07, "W": 0.003}


# ----------------------------------------------------------------------------
# Bragg line list of a synthetic fcc powder
# ----------------------------------------------------------------------------
def fcc_bragg_lines(a: float = 3.6, dmin: float = 0.5, seed: int = SEED_TABLE,
                    sigma_ln: float = 0.5) -> dict[str, Any]:
    """Distinct reflection families of an fcc lattice (h,k,l all even or all odd)
    with d = a/sqrt(h^2+k^2+l^2) >= dmin, merged by N = h^2+k^2+l^2.

    Returns d (descending), multiplicity m (count of integer triples with that N)
    and |F|^2 in barn drawn lognormal(0, sigma_ln), one per line in ascending N.
    For a=3.6, dmin=0.5: 18 lines, 386 reflections.
    """
    nmax = int(math.floor((a / dmin) ** 2 + 1e-9))
    hmax = int(math.isqrt(nmax)) + 1
    counts: dict[int, int] = {}
    for h in range(-hmax, hmax + 1):
        for k in range(-hmax, hmax + 1):
            for l in range(-hmax, hmax + 1):
                if h == 0 and k == 0 and l == 0:
                    continue
                if len({h & 1, k & 1, l & 1}) != 1:
                    continue
                n = h * h + k * k + l * l
                if n <= nmax:
                    counts[n] = counts.get(n, 0) + 1
    ns = sorted(counts)
    rng = np.random.Generator(np.random.PCG64(seed))
    f2 = rng.lognormal(0.0, sigma_ln, size=len(ns))
    return {
        "V0": a ** 3,
        "d": [a / math.sqrt(n) for n in ns],
        "mult": [float(counts[n]) for n in ns],
        "F2": [float(x) for x in f2],
        "hkl_N": ns,
    }


# ----------------------------------------------------------------------------
# Helpers building plain dict descriptions
# ----------------------------------------------------------------------------
def prim(shape, centre, params, material=-1, role="bulk", axis=2, mirror=None,
         bind_rmin=False, bind_rmax=False, chopper=None):
    """One CSG primitive.  params: box -> half extents (hx,hy,hz); tube ->
    (rmin, rmax, half_height) along `axis`; sphere -> (rmin, rmax, 0).
    role: 'bulk' (transport inside), 'detector' (terminal: scored on entry, then
    removed), 'black' (terminal, absorbing, not scored)."""
    return {"shape": shape, "centre": tuple(float(c) for c in centre),
            "params": tuple(float(p) for p in params), "material": int(material),
            "role": role, "axis": int(axis), "mirror": mirror,
            "bind_rmin": bool(bind_rmin), "bind_rmax": bool(bind_rmax), "chopper": chopper}


def disk_chopper(r_black, n=4, freq=100.0, theta0_deg=20.0, phase_deg=0.0):
    """DiskChopper parameters of §3.5 (Table tableDiskChopper): black inner
    radius (cm), number of windows, rotation frequency (Hz), opening angle and
    phase (given in degrees as in the table, stored in radians)."""
    return {"r_black": float(r_black), "n": int(n), "freq": float(freq),
            "theta0": math.radians(theta0_deg), "phase": math.radians(phase_deg)}


def material(sigma_abs_ref=0.0, abs_mode="1/v", sigma_inc=0.0, bragg=None,
             density_param=-1, scale_param=-1):
    """Macroscopic cross sections of one material.  sigma_abs_ref is Sigma_a at
    1.8 A (abs_mode '1/v') or the constant Sigma_a (abs_mode 'const')."""
    return {"sigma_abs_ref": float(sigma_abs_ref), "abs_mode": abs_mode,
            "sigma_inc": float(sigma_inc), "bragg": bragg,
            "density_param": int(density_param), "scale_param": int(scale_param)}


def tally(kind, trigger, volume, bins=(1, 1), lo=(0.0, 0.0), hi=(1.0, 1.0),
          origin=(0.0, 0.0, 0.0), axis=(0.0, 0.0, 1.0), face=-1, scat=-1, name=""):
    """kind: 'count' | 'angular' | 'psd' (x,y) | 'wlx' (lambda, x) | 'multiscat' |
    'dq' | 'tof' (time of flight in s).
    trigger: 'entry' | 'exit' (particle tracing states of §3.4).
    volume: primitive index or -1 for the world.  face: -1 any, else face id.
    scat: scattering-number filter (-1 any, n >= 0 exactly n scatters)."""
    return {"kind": kind, "trigger": trigger, "volume": int(volume),
            "bins": (int(bins[0]), int(bins[1])), "lo": tuple(map(float, lo)),
            "hi": tuple(map(float, hi)), "origin": tuple(map(float, origin)),
            "axis": tuple(map(float, axis)), "face": int(face), "scat": int(scat),
            "name": name}


def _scene(name, world, prims, materials, bias, source, tallies, precision,
           n_histories, instances=None, params=None, seed=SEED_TRANSPORT):
    nmat = len(materials)
    if instances is None:
        instances = {"params": np.zeros((1, 0)), "counts": np.array([n_histories], dtype=np.int64)}
    return {"name": name, "world": world, "prims": prims, "materials": materials,
            "bias": np.asarray(bias, dtype=np.float64).reshape(nmat, NPROC),
            "source": source, "tallies": tallies, "precision": precision,
            "instances": instances, "params": params or [], "seed": int(seed),
            "event_cap": 4096}


# ----------------------------------------------------------------------------
# Workload 1: slab (stand-in for the §4.1 biasing study)
# ----------------------------------------------------------------------------
def slab(g: float = 1.0, n_histories: int = 1_000_000, precision: str = "f64",
         sigma_s: float = 0.5, sigma_a: float = 0.1, thickness: float = 1.0):
    """1.8 A pencil beam normal to a 1 x 10 x 10 cm slab (z in [0, t]), isotropic
    incoherent Sigma_s, 1/v absorption Sigma_a(1.8 A); bias g on every process.
    Tallies: 0 uncollided and 1 total transmission through the rear face, 2 escape
    angle in 180 bins on a 4 pi sphere of radius 100 cm around the slab centre."""
    zc = 0.5 * thickness
    world = {"shape": SPHERE, "centre": (0.0, 0.0, zc), "params": (0.0, 100.0, 0.0)}
    prims = [prim(BOX, (0, 0, zc), (5.0, 5.0, 0.5 * thickness), material=0)]
    mats = [material(sigma_abs_ref=sigma_a, abs_mode="1/v", sigma_inc=sigma_s)]
    source = {"kind": "pencil", "centre": (0.0, 0.0, -1.0), "half": (0.0, 0.0),
              "lambda": (1.8, 1.8), "div": (0.0, 0.0), "aperture": None}
    tallies = [
        tally("count", "exit", 0, face=5, scat=0, name="T_uncollided"),
        tally("count", "exit", 0, face=5, scat=-1, name="T_total"),
        tally("angular", "exit", -1, bins=(180, 1), lo=(0.0, 0.0), hi=(math.pi, 1.0),
              origin=(0.0, 0.0, zc), axis=(0.0, 0.0, 1.0), name="escape_angle"),
    ]
    return _scene("slab", world, prims, mats, [[g, g, g]], source, tallies,
                  precision, n_histories)


# ----------------------------------------------------------------------------
# Workload 2: powder diffractometer (stand-in for §4.2)
# ----------------------------------------------------------------------------
POWDER_RADIUS = 0.5
CAN_THICKNESS = 0.1


def _powder_geometry(radius=POWDER_RADIUS, bind=False):
    world = {"shape": BOX, "centre": (0.0, 0.0, 0.0), "params": (120.0, 120.0, 120.0)}
    prims = [
        prim(TUBE, (0, 0, 0), (0.0, radius, 1.0), material=0, axis=1, bind_rmax=bind),
        prim(TUBE, (0, 0, 0), (radius, radius + CAN_THICKNESS, 1.0), material=1, axis=1,
             bind_rmin=bind, bind_rmax=bind),
        prim(TUBE, (0, 0, 0), (100.0, 101.0, 25.0), material=-1, axis=1, role="detector"),
    ]
    return world, prims


def _powder_materials(params=False):
    lines = fcc_bragg_lines()
    sample = material(sigma_abs_ref=0.0, sigma_inc=0.3, bragg=lines,
                      density_param=2 if params else -1, scale_param=1 if params else -1)
    can = material(sigma_inc=0.1)
    return [sample, can]


def _powder_source():
    return {"kind": "rect", "centre": (0.0, 0.0, -5.0), "half": (0.5, 1.0),
            "lambda": (1.5, 1.5), "div": (0.0, 0.0), "aperture": None}


def _powder_tallies(nbins=3600):
    return [tally("angular", "entry", 2, bins=(nbins, 1), lo=(0.0, 0.0),
                  hi=(math.pi, 1.0), origin=(0, 0, 0), axis=(0, 0, 1), name="two_theta")]


def powder(n_histories: int = 100_000_000, precision: str = "f32", g=(1.0, 1.0, 1.0),
           nbins: int = 3600):
    """1.5 A, 1 x 2 cm parallel beam on a vertical (y-axis) cylinder r=0.5 cm,
    h=2 cm of a synthetic fcc powder (Bragg lines + incoherent 0.3/cm) inside a
    1 mm can (incoherent 0.1/cm); 2-theta in 0.05 deg bins on a cylindrical
    detector of radius 100 cm, |y| <= 25 cm."""
    world, prims = _powder_geometry()
    mats = _powder_materials()
    return _scene("powder", world, prims, mats, [list(g), [1.0, 1.0, 1.0]],
                  _powder_source(), _powder_tallies(nbins), precision, n_histories)


# ----------------------------------------------------------------------------
# Workload 3: supermirror guide (stand-in for §4.3)
# ----------------------------------------------------------------------------
def guide(n_histories: int = 100_000_000, precision: str = "f32", m: float = 2.0,
          alpha: float = 3.0, length: float = 2000.0, nbins=(100, 100)):
    """Straight 5 x 5 cm guide of `length` cm (four mirror walls), source 10 x 10 cm
    at the entrance with lambda ~ U(1,10) A and divergence ~ U(-1,1) deg per axis;
    neutrons outside the 5 x 5 cm opening are stopped.  Exit monitor: lambda x x."""
    mir = {"m": float(m), "R0": 0.99, "Qc": 0.0219, "alpha": float(alpha), "W": 0.003}
    L = float(length)
    zc = 0.5 * L
    world = {"shape": BOX, "centre": (0.0, 0.0, zc), "params": (10.0, 10.0, zc + 10.0)}
    prims = [
        prim(BOX, (0, 3.75, zc), (5.0, 1.25, zc), mirror=mir),     # top wall
        prim(BOX, (0, -3.75, zc), (5.0, 1.25, zc), mirror=mir),    # bottom wall
        prim(BOX, (3.75, 0, zc), (1.25, 2.5, zc), mirror=mir),     # right wall
        prim(BOX, (-3.75, 0, zc), (1.25, 2.5, zc), mirror=mir),    # left wall
        prim(BOX, (0, 0, L + 0.05), (2.5, 2.5, 0.05), role="detector"),
    ]
    source = {"kind": "rect", "centre": (0.0, 0.0, 0.0), "half": (5.0, 5.0),
              "lambda": (1.0, 10.0), "div": (math.radians(1.0), math.radians(1.0)),
              "aperture": (2.5, 2.5)}
    tallies = [tally("wlx", "entry", 4, bins=nbins, lo=(1.0, -2.5), hi=(10.0, 2.5),
                     name="exit_lambda_x")]
    return _scene("guide", world, prims, [], np.zeros((0, NPROC)), source, tallies,
                  precision, n_histories)


# ----------------------------------------------------------------------------
# Workload 4: batched powder instances with gradients
# ----------------------------------------------------------------------------
def batched(n_instances: int = 256, count_lo: float = 1e5, count_hi: float = 1e7,
            seed: int = SEED_SCENE, precision: str = "f32", nbins: int = 3600):
    """`n_instances` powder diffractometers (workload 2 geometry) with sample radius
    ~U(0.2,1.0) cm, Bragg scale ~U(0.5,2), density multiplier 1, and history counts
    exp(U(ln count_lo, ln count_hi)) rounded.  Parameters per instance:
    [radius, scale, density]; the can follows the radius (inner R, outer R+0.1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    radius = rng.uniform(0.2, 1.0, size=n_instances)
    scale = rng.uniform(0.5, 2.0, size=n_instances)
    counts = np.rint(np.exp(rng.uniform(math.log(count_lo), math.log(count_hi),
                                        size=n_instances))).astype(np.int64)
    params = np.stack([radius, scale, np.ones(n_instances)], axis=1)
    world, prims = _powder_geometry(POWDER_RADIUS, bind=True)
    mats = _powder_materials(params=True)
    pdesc = [{"kind": "radius", "target": -1}, {"kind": "scale", "target": 0},
             {"kind": "density", "target": 0}]
    return _scene("batched", world, prims, mats, [[1.0, 1.0, 1.0], [1.0, 1.0, 1.0]],
                  _powder_source(), _powder_tallies(nbins), precision, int(counts.sum()),
                  instances={"params": params, "counts": counts,
                             "radius_nominal": POWDER_RADIUS},
                  params=pdesc)


# ----------------------------------------------------------------------------
# Workload 5: CSG imaging scene (stand-in for §4.4)
# ----------------------------------------------------------------------------
def imaging_primitives(n: int = 1000, half: float = 5.0, seed: int = SEED_SCENE,
                       rmin: float = 0.15, rmax: float = 0.5):
    """Random non-overlapping boxes / cylinders / spheres in a cube of half-width
    `half`, placed by rejection on bounding spheres of radius ~U(rmin, rmax)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = np.zeros((n, 3))
    radii = np.zeros(n)
    out = []
    placed = 0
    tries = 0
    while placed < n:
        tries += 1
        if tries > 200 * n:
            raise RuntimeError("imaging scene: rejection sampling did not converge")
        rho = rng.uniform(rmin, rmax)
        c = rng.uniform(-half + rho, half - rho, size=3)
        if placed and np.any(np.linalg.norm(centres[:placed] - c, axis=1) < radii[:placed] + rho):
            continue
        kind = int(rng.integers(0, 3))
        mat = int(rng.integers(0, 3))
        if kind == 0:
            v = rng.uniform(0.5, 1.0, size=3)
            h = rho * v / np.linalg.norm(v)
            out.append(prim(BOX, c, h, material=mat))
        elif kind == 1:
            beta = rng.uniform(0.3, 1.2)
            axis = int(rng.integers(0, 3))
            out.append(prim(TUBE, c, (0.0, rho * math.cos(beta), rho * math.sin(beta)),
                            material=mat, axis=axis))
        else:
            out.append(prim(SPHERE, c, (0.0, rho, 0.0), material=mat))
        centres[placed] = c
        radii[placed] = rho
        placed += 1
    return out


def imaging(n_histories: int = 1_000_000_000, precision: str = "f32", n_prims: int = 1000,
            g_thin: float = 5.0, psd_bins: int = 512, seed: int = SEED_SCENE, abs_bias: float = None):
    """1000 random primitives in a 10 cm cube, 3 materials with Sigma_t
    (0.2, 1, 3)/cm and scatter fractions (0.9, 0.5, 0.1) (constant absorption),
    parallel 10 x 10 cm beam lambda ~ U(0.5, 6) A, bias 5 on the thinnest
    material, 512^2 PSD behind the cube; parameters: the three densities."""
    world = {"shape": BOX, "centre": (0.0, 0.0, 0.0), "params": (8.0, 8.0, 8.0)}
    prims = imaging_primitives(n_prims, seed=seed)
    det = prim(BOX, (0, 0, 5.55), (5.0, 5.0, 0.05), role="detector")
    prims.append(det)
    sig_t = (0.2, 1.0, 3.0)
    frac = (0.9, 0.5, 0.1)
    mats = [material(sigma_abs_ref=(1 - f) * s, abs_mode="const", sigma_inc=f * s,
                     density_param=i) for i, (s, f) in enumerate(zip(sig_t, frac))]
    bias = [[g_thin] * 3, [1.0] * 3, [1.0] * 3]
    if abs_bias is not None:
        # separate absorption bias (the abs_bias of §3.5, 0.1 in the §4.4 imaging study)
        for b in bias:
            b[ABS] = abs_bias
    source = {"kind": "rect", "centre": (0.0, 0.0, -6.0), "half": (5.0, 5.0),
              "lambda": (0.5, 6.0), "div": (0.0, 0.0), "aperture": None}
    tallies = [tally("psd", "entry", len(prims) - 1, bins=(psd_bins, psd_bins),
                     lo=(-5.0, -5.0), hi=(5.0, 5.0), name="psd")]
    pdesc = [{"kind": "density", "target": 0}, {"kind": "density", "target": 1},
             {"kind": "density", "target": 2}]
    inst = {"params": np.ones((1, 3)), "counts": np.array([n_histories], dtype=np.int64)}
    return _scene("imaging", world, prims, mats, bias, source, tallies, precision,
                  n_histories, instances=inst, params=pdesc)


# ----------------------------------------------------------------------------
# Moderator guns (§3.2: UniModeratorGun, MaxwellianGun)
# ----------------------------------------------------------------------------
def moderator_source(src_w=10.0, src_h=5.0, src_z=-40.0, slit_w=0.5, slit_h=1.0, slit_z=0.1,
                     mean_wl=3.39, range_wl=0.3, temperature=None):
    """Moderator rectangle (full sizes, cm) at src_z aiming at a slit at slit_z.
    Wavelength uniform on [mean_wl - range_wl, mean_wl + range_wl] (the reading
    of the UniModeratorGun listing, whose caption gives 3.09-3.69 A for 3.39 and
    0.3), or Maxwellian at `temperature` (K)."""
    lo, hi = mean_wl - range_wl, mean_wl + range_wl
    return {"kind": "moderator", "centre": (0.0, 0.0, float(src_z)), "half": (src_w / 2, src_h / 2),
            "lambda": (lo, hi), "div": (0.0, 0.0), "aperture": None, "slit_z": float(slit_z),
            "slit_half": (slit_w / 2, slit_h / 2), "temperature": float(temperature or 0.0)}


def moderator_test(n_histories=1_000_000, precision="f32", temperature=None, lam_bins=60,
                   detector_z=0.0):
    """An empty world with a moderator gun (moderator 10 x 5 cm at z = -40 cm,
    slit 0.5 x 1 cm at z = 0) and a detector face at `detector_z` carrying a
    PSD (40 x 40 bins over +-1 cm at the slit, +-8 cm further out) and a
    wavelength spectrum (checks of the guns)."""
    world = {"shape": BOX, "centre": (0.0, 0.0, 0.0), "params": (100.0, 100.0, 100.0)}
    src = moderator_source(src_z=-40.0, slit_z=0.0, temperature=temperature)
    prims = [prim(BOX, (0, 0, detector_z + 0.05), (20.0, 20.0, 0.05), role="detector")]
    half = 1.0 if detector_z == 0.0 else 8.0
    tallies = [tally("psd", "entry", 0, bins=(40, 40), lo=(-half, -half), hi=(half, half), name="slit_psd"),
               tally("wlx", "entry", 0, bins=(lam_bins, 1), lo=(0.2, -10.0), hi=(8.2, 10.0),
                     name="spectrum")]
    return _scene("moderator", world, prims, [], np.zeros((0, NPROC)), src, tallies, precision,
                  n_histories)


# ----------------------------------------------------------------------------
# Disk chopper in ray-tracing mode with time-of-flight scorers (§4.5)
# ----------------------------------------------------------------------------
CHOPPER_DISTANCE = 1000.0   # cm from the gun to the chopper plane


def chopper(n_histories: int = 10_000_000, precision: str = "f32", tof_bins: int = 1000,
            tof_max: float = 0.025):
    """The chopper study of §4.5: a 293 K MaxwellianGun with a 1 mm x 1 mm
    opening aimed at a 45 mm x 45 mm opening 10 m away, where a disk chopper
    (4 windows of 20 degrees, 100 Hz, inner radius 13 cm, outer 25 cm) turns.
    The chopper plane is z = 0 (gun at z = -10 m) and the beam crosses the disk
    at radius 19 cm, at 90 degrees from the first in-plane axis, so that a
    window is centred on the beam at t = 0.  Time-of-flight scorers on the
    chopper's ENTRY (just before it) and EXIT (just after it), 25 us bins."""
    world = {"shape": BOX, "centre": (0.0, 0.0, -495.0), "params": (50.0, 50.0, 510.0)}
    src = moderator_source(src_w=0.1, src_h=0.1, src_z=-CHOPPER_DISTANCE, slit_w=4.5, slit_h=4.5,
                           slit_z=0.0, temperature=293.0)
    disk = disk_chopper(r_black=13.0, n=4, freq=100.0, theta0_deg=20.0, phase_deg=0.0)
    prims = [prim(TUBE, (0.0, -19.0, 0.0), (0.0, 25.0, 0.05), axis=2, chopper=disk)]
    tallies = [tally("tof", "entry", 0, bins=(tof_bins, 1), lo=(0.0, 0.0), hi=(tof_max, 1.0), name="tof_before"),
               tally("tof", "exit", 0, bins=(tof_bins, 1), lo=(0.0, 0.0), hi=(tof_max, 1.0), name="tof_after"),
               tally("count", "exit", 0, name="transmitted")]
    return _scene("chopper", world, prims, [], np.zeros((0, NPROC)), src, tallies, precision, n_histories)


def chopper_pencil(n_histories: int = 400_000, precision: str = "f64", disk_centre=(-10.0, -16.0),
                   phase_deg=17.0, lam=(1.0, 3.0), temperature=None, freq=100.0, tof_bins=200,
                   tof_max=0.025):
    """A pencil beam along +z from (0, 0, -10 m) through a disk chopper in the
    plane z = 0 centred at `disk_centre` (x, y): the beam meets the disk at a
    single radius and angle, so that the transmitted fraction and the
    time-of-flight spectra have closed forms."""
    world = {"shape": BOX, "centre": (0.0, 0.0, -495.0), "params": (60.0, 60.0, 510.0)}
    src = {"kind": "pencil", "centre": (0.0, 0.0, -CHOPPER_DISTANCE), "half": (0.0, 0.0),
           "lambda": (float(lam[0]), float(lam[1])), "div": (0.0, 0.0), "aperture": None,
           "temperature": float(temperature or 0.0)}
    disk = disk_chopper(r_black=13.0, n=4, freq=freq, theta0_deg=20.0, phase_deg=phase_deg)
    prims = [prim(TUBE, (disk_centre[0], disk_centre[1], 0.0), (0.0, 25.0, 0.05), axis=2, chopper=disk)]
    tallies = [tally("tof", "entry", 0, bins=(tof_bins, 1), lo=(0.0, 0.0), hi=(tof_max, 1.0), name="tof_before"),
               tally("tof", "exit", 0, bins=(tof_bins, 1), lo=(0.0, 0.0), hi=(tof_max, 1.0), name="tof_after"),
               tally("count", "exit", 0, name="transmitted")]
    return _scene("chopper_pencil", world, prims, [], np.zeros((0, NPROC)), src, tallies, precision,
                  n_histories)


# ----------------------------------------------------------------------------
# Total scattering with per-scattering-order tallies (stand-in for §4.1)
# ----------------------------------------------------------------------------
def total_scattering(g: float = 1.0, n_histories: int = 10_000_000, precision: str = "f32",
                     radius: float = 1.2, lam: float = 1.0, max_order: int = 3, nq: int = 200):
    """Pencil beam of wavelength `lam` on a sphere of radius `radius` cm of the
    synthetic fcc powder (Bragg lines + incoherent 0.3/cm) inside a 4 pi
    spherical detector shell (radius 200 cm); bias g on every process of the
    sample.  Tallies: the scattering-number spectrum (MultiScat) and the
    elastic momentum transfer Q of all neutrons and of those scattered exactly
    1 .. max_order times (DeltaMomentum with its scatnum filter)."""
    world = {"shape": BOX, "centre": (0.0, 0.0, 0.0), "params": (250.0, 250.0, 250.0)}
    lines = fcc_bragg_lines()
    prims = [prim(SPHERE, (0, 0, 0), (0.0, radius, 0.0), material=0),
             prim(SPHERE, (0, 0, 0), (200.0, 201.0, 0.0), role="detector")]
    mats = [material(sigma_abs_ref=0.05, abs_mode="1/v", sigma_inc=0.3, bragg=lines)]
    source = {"kind": "pencil", "centre": (0.0, 0.0, -100.0), "half": (0.0, 0.0),
              "lambda": (lam, lam), "div": (0.0, 0.0), "aperture": None}
    qmax = 4 * math.pi / lam
    tallies = [tally("multiscat", "entry", 1, bins=(8, 1), lo=(0.0, 0.0), hi=(8.0, 1.0),
                     name="scattering_number")]
    for order in [-1] + list(range(1, max_order + 1)):
        tallies.append(tally("dq", "entry", 1, bins=(nq, 1), lo=(0.0, 0.0), hi=(qmax, 1.0),
                             origin=(0, 0, 0), axis=(0, 0, 1), scat=order,
                             name="Q_all" if order < 0 else f"Q_{order}"))
    return _scene("total_scattering", world, prims, mats, [[g, g, g]], source, tallies,
                  precision, n_histories)


WORKLOADS = {"slab": slab, "powder": powder, "guide": guide, "batched": batched,
             "imaging": imaging, "total_scattering": total_scattering, "moderator": moderator_test,
             "chopper": chopper}
