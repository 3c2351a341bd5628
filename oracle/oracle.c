/*
 * oracle.c -- plain FP64 CPU reference of the probability-conserved
 * cross-section-biasing neutron history loop (arxiv 2304.06226).
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline timing).  It shares
 * no code with the CUDA path.  Everything is written for reading, not speed:
 * brute-force geometry over every primitive, direct sums over Bragg lines, no
 * tables, no blocking.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 * (seed low word, seed high word), counter = (event k, sub-stream, history id,
 * instance).  Event k uses sub-stream 0 (flight, process, cos, azimuth) and
 * sub-stream 1 (Bragg line); the source is event 0.  A derivative secondary
 * (radius gradient) spawned at primary event k draws its set-up numbers from
 * (k, 2, ..); secondary number s of a history uses sub-streams 4+2s and 5+2s
 * for its own events.  Uniforms are (a + 1/2) 2^-32, strictly inside (0,1),
 * so the logarithm of the step-length equation is always finite.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition.                             */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* Weyl key increments */
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0; k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double or_u01(uint32_t a) { return ((double)a + 0.5) * (1.0 / 4294967296.0); }

static void draw4(const or_scene* s, uint32_t k, uint32_t sub, uint64_t hid, int inst,
                  double xi[4]) {
  uint32_t ctr[4] = {k, sub, (uint32_t)hid, (uint32_t)inst};
  uint32_t key[2] = {(uint32_t)(s->seed & 0xffffffffu), (uint32_t)(s->seed >> 32)};
  uint32_t o[4];
  or_philox4x32_10(ctr, key, o);
  for (int i = 0; i < 4; ++i) xi[i] = or_u01(o[i]);
}

/* ------------------------------------------------------------------------ */
/* Small vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ------------------------------------------------------------------------ */
/* Cross sections (§2.2, §2.3)                                               */
/* ------------------------------------------------------------------------ */
/* Macroscopic cross sections of material `mat` at wavelength lambda (A):
 *   absorption  Sigma_a(lambda) = Sigma_a(1.8 A) * lambda / 1.8 (1/v law, §2.2)
 *               or a constant;
 *   incoherent elastic: constant (isotropic, Eq. eIncEla);
 *   coherent elastic (powder Bragg, Eq. eCohEla averaged over orientations):
 *     Sigma = lambda^2 / (2 V0^2) * sum over lines with 2 d >= lambda of m |F|^2 d.
 * Instance parameters multiply: density -> every process, scale -> Bragg. */
void or_sigma(const or_scene* s, int mat, const double* ip, double lambda,
              double sig[OR_NPROC]) {
  sig[0] = sig[1] = sig[2] = 0.0;
  if (mat < 0) return;
  const or_material* m = &s->mats[mat];
  double dens = (m->density_par >= 0) ? ip[m->density_par] : 1.0;
  double scale = (m->scale_par >= 0) ? ip[m->scale_par] : 1.0;
  sig[OR_P_ABS] = m->abs_1v ? m->sig_abs_ref * lambda / 1.8 : m->sig_abs_ref;
  sig[OR_P_INC] = m->sig_inc;
  double sum = 0.0;
  for (int i = 0; i < m->nlines; ++i)
    if (2.0 * m->d[i] >= lambda) sum += m->mult[i] * m->F2[i] * m->d[i];
  sig[OR_P_BRAGG] = (m->nlines > 0) ? scale * lambda * lambda / (2.0 * m->V0 * m->V0) * sum : 0.0;
  for (int i = 0; i < OR_NPROC; ++i) sig[i] *= dens;
}

/* ------------------------------------------------------------------------ */
/* Mirror reflectivity (§2.5, Eq. eMirrowRef; McStas form)                   */
/* ------------------------------------------------------------------------ */
double or_mirror_R(const or_mirror* m, double Q) {
  double R;
  if (Q <= m->Qc) R = m->R0;
  else R = 0.5 * m->R0 * (1.0 - m->alpha * (Q - m->Qc)) * (1.0 - tanh((Q - m->m * m->Qc) / m->W));
  return R > 0.0 ? R : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Geometry: boxes, tubes (cylindrical shells with flat caps), sphere shells */
/* ------------------------------------------------------------------------ */
typedef struct { double r0, r1, h; } radii;

static radii prim_radii(const or_scene* s, const or_prim* p, const double* ip) {
  radii R = {p->p[0], p->p[1], p->p[2]};
  double dR = 0.0;
  for (int i = 0; i < s->npar; ++i)
    if (s->par_kind[i] == OR_PAR_RADIUS) dR = ip[i] - s->radius_nominal;
  if (p->bind_rmin) R.r0 += dR;
  if (p->bind_rmax) R.r1 += dR;
  return R;
}

/* local coordinates: q[0],q[1] transverse, q[2] along the axis (tubes) */
static void to_local(const or_prim* p, const double r[3], const double u[3],
                     double q[3], double v[3]) {
  double d[3] = {r[0] - p->c[0], r[1] - p->c[1], r[2] - p->c[2]};
  if (p->shape == OR_TUBE) {
    int a = p->axis, b = (a + 1) % 3, c = (a + 2) % 3;
    q[0] = d[b]; q[1] = d[c]; q[2] = d[a];
    v[0] = u[b]; v[1] = u[c]; v[2] = u[a];
  } else {
    for (int i = 0; i < 3; ++i) { q[i] = d[i]; v[i] = u[i]; }
  }
}

/* roots of A t^2 + 2 B t + C = 0; returns 0 if none */
static int roots(double A, double B, double C, double* t0, double* t1) {
  if (A <= 0.0) return 0;
  double disc = B * B - A * C;
  if (disc < 0.0) return 0;
  double sq = sqrt(disc);
  *t0 = (-B - sq) / A;
  *t1 = (-B + sq) / A;
  return 1;
}

int or_prim_inside(const or_scene* s, const or_prim* p, const double* ip, const double r[3]) {
  double q[3], v[3], u0[3] = {0, 0, 1};
  to_local(p, r, u0, q, v);
  if (p->shape == OR_BOX)
    return fabs(q[0]) <= p->p[0] && fabs(q[1]) <= p->p[1] && fabs(q[2]) <= p->p[2];
  radii R = prim_radii(s, p, ip);
  if (p->shape == OR_TUBE) {
    double rho2 = q[0] * q[0] + q[1] * q[1];
    return rho2 >= R.r0 * R.r0 && rho2 <= R.r1 * R.r1 && fabs(q[2]) <= R.h;
  }
  double r2 = dot3(q, q);
  return r2 >= R.r0 * R.r0 && r2 <= R.r1 * R.r1;
}

/* Face ids: box 2*axis + (1 if the + face); tube 0 outer, 1 inner, 2 -cap,
 * 3 +cap; sphere 0 outer, 1 inner. */

/* Distance from a point inside prim p to its boundary along u. */
double or_prim_exit(const or_scene* s, const or_prim* p, const double* ip,
                    const double r[3], const double u[3], int* face) {
  double q[3], v[3];
  to_local(p, r, u, q, v);
  double best = INFINITY;
  int bf = -1;
  if (p->shape == OR_BOX) {
    for (int a = 0; a < 3; ++a) {
      if (v[a] > 0.0) { double t = (p->p[a] - q[a]) / v[a]; if (t < best) { best = t; bf = 2 * a + 1; } }
      else if (v[a] < 0.0) { double t = (-p->p[a] - q[a]) / v[a]; if (t < best) { best = t; bf = 2 * a; } }
    }
  } else {
    radii R = prim_radii(s, p, ip);
    int is_tube = (p->shape == OR_TUBE);
    double A = v[0] * v[0] + v[1] * v[1] + (is_tube ? 0.0 : v[2] * v[2]);
    double B = q[0] * v[0] + q[1] * v[1] + (is_tube ? 0.0 : q[2] * v[2]);
    double C2 = q[0] * q[0] + q[1] * q[1] + (is_tube ? 0.0 : q[2] * q[2]);
    double t0, t1;
    if (roots(A, B, C2 - R.r1 * R.r1, &t0, &t1) && t1 >= 0.0 && t1 < best) { best = t1; bf = 0; }
    if (R.r0 > 0.0 && roots(A, B, C2 - R.r0 * R.r0, &t0, &t1) && t0 >= 0.0 && t0 < best) { best = t0; bf = 1; }
    if (is_tube) {
      if (v[2] > 0.0) { double t = (R.h - q[2]) / v[2]; if (t < best) { best = t; bf = 3; } }
      else if (v[2] < 0.0) { double t = (-R.h - q[2]) / v[2]; if (t < best) { best = t; bf = 2; } }
    }
  }
  if (best < 0.0) best = 0.0;
  if (face) *face = bf;
  return best;
}

/* Distance from a point outside prim p to where the ray enters it (INFINITY if
 * it never does).  The solid along the ray is the set of t where the point is
 * inside; the entry is the start of its first piece that ends ahead. */
double or_prim_entry(const or_scene* s, const or_prim* p, const double* ip,
                     const double r[3], const double u[3], int* face) {
  double q[3], v[3];
  to_local(p, r, u, q, v);
  if (face) *face = -1;
  if (p->shape == OR_BOX) {
    double tn = -INFINITY, tf = INFINITY;
    int fn = -1;
    for (int a = 0; a < 3; ++a) {
      if (v[a] == 0.0) {
        if (fabs(q[a]) > p->p[a]) return INFINITY;
        continue;
      }
      double ta = (-p->p[a] - q[a]) / v[a], tb = (p->p[a] - q[a]) / v[a];
      int fa = 2 * a, fb = 2 * a + 1;
      if (ta > tb) { double t = ta; ta = tb; tb = t; int f = fa; fa = fb; fb = f; }
      if (ta > tn) { tn = ta; fn = fa; }
      if (tb < tf) tf = tb;
    }
    if (tn > tf || tf <= 0.0) return INFINITY;
    if (face) *face = fn;
    return tn > 0.0 ? tn : 0.0;
  }
  radii R = prim_radii(s, p, ip);
  int is_tube = (p->shape == OR_TUBE);
  double A = v[0] * v[0] + v[1] * v[1] + (is_tube ? 0.0 : v[2] * v[2]);
  double B = q[0] * v[0] + q[1] * v[1] + (is_tube ? 0.0 : q[2] * v[2]);
  double C2 = q[0] * q[0] + q[1] * q[1] + (is_tube ? 0.0 : q[2] * q[2]);
  /* outer solid [o0, o1] */
  double o0, o1;
  if (A == 0.0) {
    if (C2 > R.r1 * R.r1) return INFINITY;
    o0 = -INFINITY; o1 = INFINITY;
  } else if (!roots(A, B, C2 - R.r1 * R.r1, &o0, &o1)) {
    return INFINITY;
  }
  /* axial slab [z0, z1] (tubes only) */
  double z0 = -INFINITY, z1 = INFINITY;
  int fz0 = -1;
  if (is_tube) {
    if (v[2] == 0.0) {
      if (fabs(q[2]) > R.h) return INFINITY;
    } else {
      double ta = (-R.h - q[2]) / v[2], tb = (R.h - q[2]) / v[2];
      if (ta < tb) { z0 = ta; z1 = tb; fz0 = 2; }
      else { z0 = tb; z1 = ta; fz0 = 3; }
    }
  }
  /* hole (i0, i1) where the radius is below rmin */
  double seg_s[2], seg_e[2];
  int seg_f[2], nseg = 0;
  double i0, i1;
  if (R.r0 > 0.0 && A > 0.0 && roots(A, B, C2 - R.r0 * R.r0, &i0, &i1)) {
    seg_s[0] = o0; seg_e[0] = i0; seg_f[0] = 0;
    seg_s[1] = i1; seg_e[1] = o1; seg_f[1] = 1;
    nseg = 2;
  } else if (R.r0 > 0.0 && A == 0.0 && C2 < R.r0 * R.r0) {
    return INFINITY;  /* travelling along the axis inside the hole */
  } else {
    seg_s[0] = o0; seg_e[0] = o1; seg_f[0] = 0;
    nseg = 1;
  }
  for (int i = 0; i < nseg; ++i) {
    double a = seg_s[i], b = seg_e[i];
    int f = seg_f[i];
    if (z0 > a) { a = z0; f = fz0; }
    if (z1 < b) b = z1;
    if (a < b && b > 0.0) {
      if (face) *face = f;
      return a > 0.0 ? a : 0.0;
    }
  }
  return INFINITY;
}

static double world_exit(const or_scene* s, const double r[3], const double u[3]) {
  or_prim w;
  memset(&w, 0, sizeof w);
  w.mirror = w.chopper = -1;
  w.shape = s->world_shape;
  for (int i = 0; i < 3; ++i) { w.c[i] = s->world_c[i]; w.p[i] = s->world_p[i]; }
  w.axis = 2;
  int f;
  return or_prim_exit(s, &w, NULL, r, u, &f);
}

static int world_inside(const or_scene* s, const double r[3]) {
  or_prim w;
  memset(&w, 0, sizeof w);
  w.mirror = w.chopper = -1;
  w.shape = s->world_shape;
  for (int i = 0; i < 3; ++i) { w.c[i] = s->world_c[i]; w.p[i] = s->world_p[i]; }
  w.axis = 2;
  return or_prim_inside(s, &w, NULL, r);
}

/* Outward unit normal of prim p's face `face` at point r. */
static void prim_normal(const or_scene* s, const or_prim* p, const double* ip,
                        const double r[3], int face, double n[3]) {
  n[0] = n[1] = n[2] = 0.0;
  if (p->shape == OR_BOX) {
    n[face / 2] = (face & 1) ? 1.0 : -1.0;
    return;
  }
  double d[3] = {r[0] - p->c[0], r[1] - p->c[1], r[2] - p->c[2]};
  if (p->shape == OR_TUBE) {
    int a = p->axis;
    if (face >= 2) { n[a] = (face == 3) ? 1.0 : -1.0; return; }
    d[a] = 0.0;
  }
  double len = sqrt(dot3(d, d));
  double sgn = (face == 1) ? -1.0 : 1.0;   /* inner surface: outward = towards the axis */
  for (int i = 0; i < 3; ++i) n[i] = sgn * d[i] / len;
  (void)s; (void)ip;
}

/* Point location: the primitive containing r, -1 for the world region, -2 if
 * outside the world. */
static int locate(const or_scene* s, const double* ip, const double r[3]) {
  if (!world_inside(s, r)) return -2;
  for (int i = 0; i < s->nprim; ++i)
    if (or_prim_inside(s, &s->prims[i], ip, r)) return i;
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Direction change for a deflection by polar angle acos(mu), azimuth phi    */
/* ------------------------------------------------------------------------ */
void or_rotate(const double u[3], double mu, double phi, double out[3]) {
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  double cp = cos(phi), sp = sin(phi);
  double t2 = 1.0 - u[2] * u[2];
  if (t2 > 1e-20) {
    double t = sqrt(t2);
    out[0] = mu * u[0] + st * (u[0] * u[2] * cp - u[1] * sp) / t;
    out[1] = mu * u[1] + st * (u[1] * u[2] * cp + u[0] * sp) / t;
    out[2] = mu * u[2] - st * t * cp;
  } else {
    out[0] = st * cp;
    out[1] = st * sp;
    out[2] = (u[2] >= 0.0 ? 1.0 : -1.0) * mu;
  }
}

/* ------------------------------------------------------------------------ */
/* Tallies (§3.4 scorers)                                                    */
/* ------------------------------------------------------------------------ */
int or_total_bins(const or_scene* s) {
  int n = 0;
  for (int t = 0; t < s->ntally; ++t) n += s->tallies[t].nb[0] * s->tallies[t].nb[1];
  return n;
}

static int bin1(double x, double lo, double hi, int n) {
  if (!(x >= lo) || !(x < hi)) return -1;
  int b = (int)floor((x - lo) / (hi - lo) * n);
  return (b >= 0 && b < n) ? b : -1;
}

/* Angle between (r - origin) and the tally axis. */
static double tally_angle(const or_tally* T, const double r[3]) {
  double v[3] = {r[0] - T->origin[0], r[1] - T->origin[1], r[2] - T->origin[2]};
  double len = sqrt(dot3(v, v));
  double al = sqrt(dot3(T->axis, T->axis));
  double c = dot3(v, T->axis) / (len * al);
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  return acos(c);
}

/* Bin of tally t for a particle at r with wavelength lambda after nscat
 * scatterings, or -1. */
/* Time of flight (s) of a neutron born at t = 0 that has flown `path` cm at
 * wavelength lambda (A): its speed is v = h / (m_n lambda), h / m_n =
 * 3956.034 m^2/s per A of wavelength (CODATA h and m_n), i.e.
 * 395603.4 cm/s at 1 A.  Every process here is elastic, so the speed is
 * constant along a history. */
static double time_of_flight(double path, double lambda) {
  return path * lambda / 395603.4012;
}

static int tally_bin(const or_tally* T, const double r[3], double lambda, int nscat, double path) {
  switch (T->kind) {
    case OR_T_TOF: return bin1(time_of_flight(path, lambda), T->lo[0], T->hi[0], T->nb[0]);
    case OR_T_COUNT: return 0;
    case OR_T_ANGULAR: return bin1(tally_angle(T, r), T->lo[0], T->hi[0], T->nb[0]);
    case OR_T_MULTISCAT: return bin1((double)nscat, T->lo[0], T->hi[0], T->nb[0]);
    case OR_T_DQ: {
      /* elastic momentum transfer Q = 2 k sin(theta/2), k = 2 pi / lambda (Eq. eQelastic) */
      double Q = 4.0 * PI * sin(0.5 * tally_angle(T, r)) / lambda;
      return bin1(Q, T->lo[0], T->hi[0], T->nb[0]);
    }
    case OR_T_PSD: {
      int bx = bin1(r[0], T->lo[0], T->hi[0], T->nb[0]);
      int by = bin1(r[1], T->lo[1], T->hi[1], T->nb[1]);
      return (bx < 0 || by < 0) ? -1 : bx * T->nb[1] + by;
    }
    case OR_T_WLX: {
      int bl = bin1(lambda, T->lo[0], T->hi[0], T->nb[0]);
      int bx = bin1(r[0], T->lo[1], T->hi[1], T->nb[1]);
      return (bl < 0 || bx < 0) ? -1 : bl * T->nb[1] + bx;
    }
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* One history                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  double r[3], u[3], lambda, w;
  double A[OR_MAX_PAR];
  double path;        /* length flown since the source (cm), for the time of flight */
  int vol, nscat;
  int secondary;      /* 1 for a radius-derivative secondary */
  uint32_t sub0;      /* sub-stream of its events */
} particle;

typedef struct {
  const or_scene* s;
  int inst;
  const double* ip;
  int want_grad;
  or_accum* acc;
  int* tally_off;
  int radius_par;     /* index of the radius parameter, -1 if none */
} ctx;

static void score(ctx* c, const particle* P, int trigger, int volume, int face) {
  const or_scene* s = c->s;
  for (int t = 0; t < s->ntally; ++t) {
    const or_tally* T = &s->tallies[t];
    if (T->trigger != trigger || T->volume != volume) continue;
    if (T->face >= 0 && T->face != face) continue;
    if (T->scat >= 0 && T->scat != P->nscat) continue;
    int b = tally_bin(T, P->r, P->lambda, P->nscat, P->path);
    if (b < 0) continue;
    int idx = c->tally_off[t] + b;
    int tb = or_total_bins(s);
    if (!P->secondary) {
      c->acc->sum[idx] += P->w;
      c->acc->sumsq[idx] += P->w * P->w;
      if (c->want_grad && c->acc->J) {
        for (int k = 0; k < s->npar; ++k) {
          double g = P->w * P->A[k];
          c->acc->J[(size_t)k * tb + idx] += g;
          c->acc->J2[(size_t)k * tb + idx] += g * g;
        }
      }
    } else if (c->want_grad && c->acc->J && c->radius_par >= 0) {
      double g = P->w;
      c->acc->J[(size_t)c->radius_par * tb + idx] += g;
      c->acc->J2[(size_t)c->radius_par * tb + idx] += g * g;
    }
  }
}

/* Disk chopper in ray-tracing mode (§2.1, Eq. eRayTracing; §2.5 and §3.5,
 * DiskChopper): the factor epsilon is 1 if, at the moment the neutron reaches
 * the (infinitely thin) disk, its position lies in an opening window, else 0.
 * In the plane of the disk, with in-plane axes e1 = axis+1, e2 = axis+2
 * (cyclic) about the tube centre, the neutron is at radius rho and angle phi.
 * At time t window k (k = 0..n-1) is centred at phase + 2 pi f t + 2 pi k / n
 * and spans theta0; the disk is black for rho < r_black.  Written as the
 * plain definition: the angular distance to each window centre in turn. */
static int chopper_open(const or_scene* s, const or_prim* pt, const particle* P) {
  const or_chopper* ch = &s->choppers[pt->chopper];
  const int a1 = (pt->axis + 1) % 3, a2 = (pt->axis + 2) % 3;
  const double q1 = P->r[a1] - pt->c[a1], q2 = P->r[a2] - pt->c[a2];
  const double rho = sqrt(q1 * q1 + q2 * q2);
  if (rho < ch->r_black) return 0;
  const double phi = atan2(q2, q1);
  const double t = time_of_flight(P->path, P->lambda);
  for (int k = 0; k < ch->n; ++k) {
    const double centre = ch->phase + 2.0 * PI * ch->freq * t + 2.0 * PI * k / ch->n;
    double d = fmod(phi - centre, 2.0 * PI);          /* in (-2 pi, 2 pi) */
    if (d > PI) d -= 2.0 * PI;
    if (d < -PI) d += 2.0 * PI;
    if (fabs(d) <= 0.5 * ch->theta0) return 1;
  }
  return 0;
}

static double nudge_len(const double r[3]) {
  double m = fmax(fabs(r[0]), fmax(fabs(r[1]), fabs(r[2])));
  return 1e-9 * fmax(1.0, m);
}

static int material_of(const or_scene* s, int vol) {
  return vol >= 0 ? s->prims[vol].material : -1;
}

/* Is prim p's face a lateral surface that moves with the radius parameter?
 * Returns +1 if it is the rmax surface, -1 if the rmin surface, 0 otherwise. */
static int radius_face(const or_prim* p, int face) {
  if (p->shape == OR_BOX) return 0;
  if (face == 0 && p->bind_rmax) return 1;
  if (face == 1 && p->bind_rmin) return -1;
  return 0;
}

static void transport(ctx* c, particle* P, uint64_t hid, or_record* rec, uint32_t* nsec);

/* Radius derivative at the crossing of a moving lateral surface.  The layer of
 * thickness dR outside the surface changes from the outer material to the inner
 * one; a path crossing it at |n.u| spends dR/|n.u| in it.  (1) The score
 * function of the continuing path gains -(Sigma_t,in - Sigma_t,out)/|n.u|.
 * (2) Collisions inside the layer, absent from the sampled paths, are added as a
 * derivative secondary starting at the crossing with weight
 * w sign(c) C/|n.u|, colliding by a term chosen with probability |c|/C among
 * c = +Sigma_j,in and -Sigma_j,out (scattering processes j). */
static void radius_crossing(ctx* c, particle* P, int mat_in, int mat_out, const double n[3],
                            uint32_t k, uint64_t hid, uint32_t* nsec) {
  const or_scene* s = c->s;
  double cosn = fabs(dot3(P->u, n));
  if (cosn < 1e-12) return;   /* grazing: measure zero */
  double sin_[OR_NPROC], sout[OR_NPROC];
  or_sigma(s, mat_in, c->ip, P->lambda, sin_);
  or_sigma(s, mat_out, c->ip, P->lambda, sout);
  double st_in = sin_[0] + sin_[1] + sin_[2];
  double st_out = sout[0] + sout[1] + sout[2];
  P->A[c->radius_par] -= (st_in - st_out) / cosn;
  /* derivative secondary */
  double term[4] = {sin_[OR_P_INC], sin_[OR_P_BRAGG], -sout[OR_P_INC], -sout[OR_P_BRAGG]};
  double C = 0.0;
  for (int i = 0; i < 4; ++i) C += fabs(term[i]);
  if (C <= 0.0) return;
  double xi[4];
  draw4(s, k, 2u, hid, c->inst, xi);
  double acc = 0.0;
  int pick = 3;
  for (int i = 0; i < 4; ++i) {
    acc += fabs(term[i]);
    if (xi[0] * C < acc) { pick = i; break; }
  }
  while (term[pick] == 0.0 && pick > 0) --pick;   /* guard against rounding at the end */
  int mat = (pick < 2) ? mat_in : mat_out;
  int proc = (pick % 2 == 0) ? OR_P_INC : OR_P_BRAGG;
  particle S = *P;
  S.secondary = 1;
  S.w = P->w * (term[pick] > 0.0 ? 1.0 : -1.0) * C / cosn;
  S.nscat = P->nscat + 1;
  S.sub0 = 4u + 2u * (*nsec);
  (*nsec)++;
  if (proc == OR_P_INC) {
    double mu = 2.0 * xi[1] - 1.0, phi = 2.0 * PI * xi[2];
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    S.u[0] = st * cos(phi); S.u[1] = st * sin(phi); S.u[2] = mu;
  } else {
    const or_material* m = &s->mats[mat];
    double tot = 0.0;
    for (int i = 0; i < m->nlines; ++i)
      if (2.0 * m->d[i] >= P->lambda) tot += m->mult[i] * m->F2[i] * m->d[i];
    double a = 0.0;
    int line = -1;
    for (int i = 0; i < m->nlines; ++i) {
      if (2.0 * m->d[i] < P->lambda) continue;
      a += m->mult[i] * m->F2[i] * m->d[i];
      line = i;
      if (xi[3] * tot < a) break;
    }
    double sb = P->lambda / (2.0 * m->d[line]);
    double mu = 1.0 - 2.0 * sb * sb;   /* cos(2 theta_B) */
    double un[3];
    or_rotate(P->u, mu, 2.0 * PI * xi[2], un);
    S.u[0] = un[0]; S.u[1] = un[1]; S.u[2] = un[2];
  }
  c->acc->counters[7]++;
  /* place it on the side its new direction points to */
  double e = nudge_len(S.r);
  double rn[3] = {S.r[0] + e * S.u[0], S.r[1] + e * S.u[1], S.r[2] + e * S.u[2]};
  int v = locate(s, c->ip, rn);
  if (v < -1) return;
  S.r[0] = rn[0]; S.r[1] = rn[1]; S.r[2] = rn[2];
  S.vol = v;
  if (v >= 0 && s->prims[v].role != OR_ROLE_BULK) return;  /* no transport in a detector */
  transport(c, &S, hid, NULL, nsec);
}

/* Transport one particle until it ends (§3.1).  Derivative secondaries are
 * transported to completion as soon as they are created. */
static void transport(ctx* c, particle* P, uint64_t hid, or_record* rec, uint32_t* nsec) {
  const or_scene* s = c->s;
  or_accum* acc = c->acc;
  const int grad = c->want_grad;
  int end = OR_END_LOST;
  uint32_t k;
  for (k = 1; ; ++k) {
    if ((int)k > s->event_cap) { end = OR_END_TRUNCATED; acc->counters[4]++; break; }
    acc->counters[1]++;
    double xi[4];
    draw4(s, k, P->sub0, hid, c->inst, xi);
    /* cross sections of the current volume, true and biased */
    int mat = material_of(s, P->vol);
    double sig[OR_NPROC];
    or_sigma(s, mat, c->ip, P->lambda, sig);
    double sig_t = 0.0, sig_g = 0.0;
    for (int i = 0; i < OR_NPROC; ++i) {
      sig_t += sig[i];
      sig_g += (mat >= 0 ? s->bias[mat * OR_NPROC + i] : 1.0) * sig[i];
    }
    /* biased step length, Eq. eStepLength2 */
    double l = (sig_g > 0.0) ? -log(xi[0]) / sig_g : INFINITY;
    /* distance to the next boundary */
    double db;
    int target = -1, face = -1;   /* target: prim entered (world region), or -1 */
    if (P->vol >= 0) {
      db = or_prim_exit(s, &s->prims[P->vol], c->ip, P->r, P->u, &face);
    } else {
      db = world_exit(s, P->r, P->u);
      target = -3;   /* world exit */
      for (int i = 0; i < s->nprim; ++i) {
        int f;
        double t = or_prim_entry(s, &s->prims[i], c->ip, P->r, P->u, &f);
        if (t < db) { db = t; target = i; face = f; }
      }
    }
    double x = (l >= db) ? db : l;
    if (!isfinite(x)) { end = OR_END_LOST; acc->counters[5]++; break; }
    /* move and compensate the weight, Eq. eWeight: exp(sum_i (g_i-1) Sigma_i x) */
    for (int i = 0; i < 3; ++i) P->r[i] += x * P->u[i];
    P->path += x;
    P->w *= exp((sig_g - sig_t) * x);
    if (grad && mat >= 0 && !P->secondary) {
      for (int p = 0; p < s->npar; ++p) {
        const or_material* m = &s->mats[mat];
        if (s->par_kind[p] == OR_PAR_DENSITY && m->density_par == p) P->A[p] -= sig_t * x;
        if (s->par_kind[p] == OR_PAR_SCALE && m->scale_par == p) P->A[p] -= sig[OR_P_BRAGG] * x;
      }
    }
    if (l >= db) {
      /* ---- relocation: the particle reached a boundary ---- */
      acc->counters[3]++;
      if (P->vol >= 0) {
        int from = P->vol;
        const or_prim* pf = &s->prims[from];
        score(c, P, OR_PTS_EXIT, from, face);
        double e = nudge_len(P->r);
        double rn[3] = {P->r[0] + e * P->u[0], P->r[1] + e * P->u[1], P->r[2] + e * P->u[2]};
        int v = locate(s, c->ip, rn);
        int rf = grad && !P->secondary && c->radius_par >= 0 ? radius_face(pf, face) : 0;
        if (rf != 0) {
          double n[3];
          prim_normal(s, pf, c->ip, P->r, face, n);
          int mat_next = (v >= 0) ? s->prims[v].material : -1;
          int mi = rf > 0 ? pf->material : mat_next;
          int mo = rf > 0 ? mat_next : pf->material;
          radius_crossing(c, P, mi, mo, n, k, hid, nsec);
        }
        for (int i = 0; i < 3; ++i) P->r[i] = rn[i];
        if (v == -2) { score(c, P, OR_PTS_EXIT, -1, -1); end = OR_END_ESCAPED; break; }
        P->vol = v;
        if (v >= 0) {
          const or_prim* pt = &s->prims[v];
          score(c, P, OR_PTS_ENTRY, v, -1);
          if (pt->role == OR_ROLE_DETECTOR) { end = OR_END_DETECTED; break; }
          if (pt->role == OR_ROLE_BLACK) { end = OR_END_BLACK; break; }
          if (pt->chopper >= 0 && !chopper_open(s, pt, P)) { end = OR_END_BLACK; break; }
        }
      } else if (target == -3) {
        score(c, P, OR_PTS_EXIT, -1, -1);
        end = OR_END_ESCAPED;
        break;
      } else {
        const or_prim* pt = &s->prims[target];
        if (pt->mirror >= 0) {
          /* mirror (§2.5): weight R(Q), specular reflection, Eq. eMirrowNewDir */
          double n[3];
          prim_normal(s, pt, c->ip, P->r, face, n);
          double un = dot3(P->u, n);
          double Q = 4.0 * PI * fabs(un) / P->lambda;
          double R = or_mirror_R(&s->mirrors[pt->mirror], Q);
          acc->counters[6]++;
          P->w *= R;
          if (R <= 0.0) { end = OR_END_MIRROR; break; }
          for (int i = 0; i < 3; ++i) P->u[i] -= 2.0 * n[i] * un;
          double e = nudge_len(P->r);
          for (int i = 0; i < 3; ++i) P->r[i] += e * P->u[i];
        } else {
          int rf = grad && !P->secondary && c->radius_par >= 0 ? radius_face(pt, face) : 0;
          if (rf != 0) {
            double n[3];
            prim_normal(s, pt, c->ip, P->r, face, n);
            int mi = rf > 0 ? pt->material : -1;
            int mo = rf > 0 ? -1 : pt->material;
            radius_crossing(c, P, mi, mo, n, k, hid, nsec);
          }
          double e = nudge_len(P->r);
          for (int i = 0; i < 3; ++i) P->r[i] += e * P->u[i];
          P->vol = target;
          score(c, P, OR_PTS_ENTRY, target, face);
          if (pt->role == OR_ROLE_DETECTOR) { end = OR_END_DETECTED; break; }
          if (pt->role == OR_ROLE_BLACK) { end = OR_END_BLACK; break; }
          if (pt->chopper >= 0 && !chopper_open(s, pt, P)) { end = OR_END_BLACK; break; }
        }
      }
    } else {
      /* ---- interaction: choose the process with probability g_j Sigma_j / Sigma_g ---- */
      acc->counters[2]++;
      if (rec && P->nscat == 0 && isnan(rec->first_collision[0]))
        for (int i = 0; i < 3; ++i) rec->first_collision[i] = P->r[i];
      int j = -1;
      double cum = 0.0;
      for (int i = 0; i < OR_NPROC; ++i) {
        cum += s->bias[mat * OR_NPROC + i] * sig[i];
        if (xi[1] * sig_g < cum) { j = i; break; }
      }
      if (j < 0) {   /* rounding at the top end: last process with a non-zero share */
        for (int i = OR_NPROC - 1; i >= 0; --i)
          if (s->bias[mat * OR_NPROC + i] * sig[i] > 0.0) { j = i; break; }
      }
      P->w /= s->bias[mat * OR_NPROC + j];
      if (grad && !P->secondary) {
        const or_material* m = &s->mats[mat];
        for (int p = 0; p < s->npar; ++p) {
          if (s->par_kind[p] == OR_PAR_DENSITY && m->density_par == p) P->A[p] += 1.0;
          if (s->par_kind[p] == OR_PAR_SCALE && m->scale_par == p && j == OR_P_BRAGG) P->A[p] += 1.0;
        }
      }
      if (j == OR_P_ABS) { end = OR_END_ABSORBED; break; }
      if (j == OR_P_INC && s->mats[mat].rod) {
        /* rod model (test mode): forward or backward along z, 1/2 each */
        P->u[0] = 0.0; P->u[1] = 0.0; P->u[2] = (xi[2] < 0.5) ? -1.0 : 1.0;
      } else if (j == OR_P_INC) {
        /* isotropic: cos theta uniform on [-1,1], azimuth uniform */
        double mu = 2.0 * xi[2] - 1.0, phi = 2.0 * PI * xi[3];
        double st = sqrt(fmax(0.0, 1.0 - mu * mu));
        P->u[0] = st * cos(phi); P->u[1] = st * sin(phi); P->u[2] = mu;
      } else {
        /* powder Bragg: line i with probability m_i |F_i|^2 d_i over the lines
         * with 2 d_i >= lambda; deflection 2 theta_B, sin theta_B = lambda/(2 d_i) */
        double xb[4];
        draw4(s, k, P->sub0 + 1u, hid, c->inst, xb);
        const or_material* m = &s->mats[mat];
        double tot = 0.0;
        for (int i = 0; i < m->nlines; ++i)
          if (2.0 * m->d[i] >= P->lambda) tot += m->mult[i] * m->F2[i] * m->d[i];
        double a = 0.0;
        int line = -1;
        for (int i = 0; i < m->nlines; ++i) {
          if (2.0 * m->d[i] < P->lambda) continue;
          a += m->mult[i] * m->F2[i] * m->d[i];
          line = i;
          if (xb[0] * tot < a) break;
        }
        double sb = P->lambda / (2.0 * m->d[line]);
        double mu = 1.0 - 2.0 * sb * sb;
        double un[3];
        or_rotate(P->u, mu, 2.0 * PI * xi[3], un);
        for (int i = 0; i < 3; ++i) P->u[i] = un[i];
      }
      if (rec && P->nscat == 0 && !P->secondary)
        for (int i = 0; i < 3; ++i) rec->dir_after_first[i] = P->u[i];
      P->nscat++;
    }
  }
  if (rec) {
    for (int i = 0; i < 3; ++i) rec->final_pos[i] = P->r[i];
    rec->w_final = P->w;
    for (int i = 0; i < OR_MAX_PAR; ++i) rec->A_final[i] = P->A[i];
    rec->nscat = P->nscat;
    rec->nevents = (int)k;
    rec->end = end;
  }
}

static void history(ctx* c, uint64_t hid, or_record* rec) {
  const or_scene* s = c->s;
  or_accum* acc = c->acc;
  acc->counters[0]++;
  particle P;
  memset(&P, 0, sizeof P);
  if (rec) {
    memset(rec, 0, sizeof *rec);
    for (int i = 0; i < 3; ++i) rec->first_collision[i] = rec->dir_after_first[i] = NAN;
  }
  /* source, event 0 (§3.2 guns) */
  double a[4], b[4];
  draw4(s, 0u, 0u, hid, c->inst, a);
  draw4(s, 0u, 1u, hid, c->inst, b);
  const or_source* g = &s->src;
  P.r[0] = g->c[0]; P.r[1] = g->c[1]; P.r[2] = g->c[2];
  if (g->kind == OR_SRC_RECT || g->kind == OR_SRC_MODERATOR) {
    P.r[0] += g->half[0] * (2.0 * a[0] - 1.0);
    P.r[1] += g->half[1] * (2.0 * a[1] - 1.0);
  }
  if (g->temperature > 0.0) {
    /* MaxwellianGun (§3.2): kinetic energy from the Maxwell-Boltzmann
     * distribution sqrt(E) exp(-E/kT), i.e. E/kT ~ Gamma(3/2): the sum of an
     * exponential variate and half the square of a normal one, the latter by
     * the Box-Muller construction; then lambda = sqrt((h^2/2m_n) / E). */
    const double kT = 0.08617333 * g->temperature;          /* meV */
    const double c = cos(0.5 * PI * b[3]);
    const double E = kT * (-log(a[2]) - log(a[3]) * c * c);   /* meV */
    P.lambda = sqrt(81.80420 / E);                           /* A */
  } else {
    P.lambda = (g->lam_hi > g->lam_lo) ? g->lam_lo + (g->lam_hi - g->lam_lo) * a[2] : g->lam_lo;
  }
  if (g->kind == OR_SRC_MODERATOR) {
    /* UniModeratorGun / MaxwellianGun: aim at a point uniform on the slit */
    double t[3] = {g->c[0] + g->slit_half[0] * (2.0 * b[1] - 1.0) - P.r[0],
                   g->c[1] + g->slit_half[1] * (2.0 * b[2] - 1.0) - P.r[1], g->slit_z - P.r[2]};
    double n = sqrt(dot3(t, t));
    P.u[0] = t[0] / n; P.u[1] = t[1] / n; P.u[2] = t[2] / n;
  } else if (g->div[0] > 0.0 || g->div[1] > 0.0) {
    double tx = tan(g->div[0] * (2.0 * a[3] - 1.0));
    double ty = tan(g->div[1] * (2.0 * b[0] - 1.0));
    double n = sqrt(tx * tx + ty * ty + 1.0);
    P.u[0] = tx / n; P.u[1] = ty / n; P.u[2] = 1.0 / n;
  } else {
    P.u[0] = 0.0; P.u[1] = 0.0; P.u[2] = 1.0;
  }
  P.w = 1.0;
  P.sub0 = 0u;
  /* a history can end at its source: the record then holds the birth point */
  if (rec)
    for (int i = 0; i < 3; ++i) rec->final_pos[i] = P.r[i];
  if (g->has_aperture &&
      (fabs(P.r[0] - g->c[0]) > g->aperture[0] || fabs(P.r[1] - g->c[1]) > g->aperture[1])) {
    if (rec) { rec->end = OR_END_APERTURE; rec->w_final = 0.0; }
    return;
  }
  P.vol = locate(s, c->ip, P.r);
  if (P.vol == -2) { if (rec) { rec->end = OR_END_LOST; rec->w_final = P.w; } acc->counters[5]++; return; }
  if (P.vol >= 0 && s->prims[P.vol].role != OR_ROLE_BULK) {
    if (rec) { rec->end = OR_END_BLACK; rec->w_final = P.w; }
    return;
  }
  uint32_t nsec = 0;
  transport(c, &P, hid, rec, &nsec);
}

/* ------------------------------------------------------------------------ */
/* Threaded driver: contiguous history ranges per thread, summed in order    */
/* ------------------------------------------------------------------------ */
typedef struct {
  ctx c;
  or_accum acc;
  uint64_t first, n;
  or_record* records;
} job;

static void* worker(void* arg) {
  job* J = (job*)arg;
  J->c.acc = &J->acc;
  for (uint64_t i = 0; i < J->n; ++i)
    history(&J->c, J->first + i, J->records ? &J->records[i] : NULL);
  return NULL;
}

int or_run(const or_scene* s, int inst, const double* ip, uint64_t first, uint64_t n,
           int threads, int want_grad, or_accum* acc, or_record* records) {
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > n && n > 0) threads = (int)n;
  if (n == 0) return 0;
  int tb = or_total_bins(s);
  int* off = (int*)calloc((size_t)s->ntally + 1, sizeof(int));
  for (int t = 0, o = 0; t < s->ntally; ++t) { off[t] = o; o += s->tallies[t].nb[0] * s->tallies[t].nb[1]; }
  int radius_par = -1;
  for (int i = 0; i < s->npar; ++i) if (s->par_kind[i] == OR_PAR_RADIUS) radius_par = i;
  job* jobs = (job*)calloc((size_t)threads, sizeof(job));
  pthread_t* th = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
  size_t np = (size_t)(s->npar > 0 ? s->npar : 1);
  for (int t = 0; t < threads; ++t) {
    job* J = &jobs[t];
    J->c.s = s; J->c.inst = inst; J->c.ip = ip; J->c.want_grad = want_grad;
    J->c.tally_off = off; J->c.radius_par = radius_par;
    J->first = first + n * (uint64_t)t / (uint64_t)threads;
    J->n = first + n * (uint64_t)(t + 1) / (uint64_t)threads - J->first;
    J->records = records ? records + (J->first - first) : NULL;
    J->acc.sum = (double*)calloc((size_t)tb, sizeof(double));
    J->acc.sumsq = (double*)calloc((size_t)tb, sizeof(double));
    if (want_grad && acc->J) {
      J->acc.J = (double*)calloc(np * (size_t)tb, sizeof(double));
      J->acc.J2 = (double*)calloc(np * (size_t)tb, sizeof(double));
    }
  }
  for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, worker, &jobs[t]);
  for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  for (int t = 0; t < threads; ++t) {
    job* J = &jobs[t];
    for (int i = 0; i < tb; ++i) { acc->sum[i] += J->acc.sum[i]; acc->sumsq[i] += J->acc.sumsq[i]; }
    if (J->acc.J) {
      for (size_t i = 0; i < np * (size_t)tb; ++i) { acc->J[i] += J->acc.J[i]; acc->J2[i] += J->acc.J2[i]; }
    }
    for (int i = 0; i < 8; ++i) acc->counters[i] += J->acc.counters[i];
    free(J->acc.sum); free(J->acc.sumsq); free(J->acc.J); free(J->acc.J2);
  }
  free(jobs); free(th); free(off);
  return 0;
}
