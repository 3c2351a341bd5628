/*
 * oracle.h -- plain FP64 CPU reference of the probability-conserved
 * cross-section-biasing neutron history loop (arxiv 2304.06226).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code, header,
 * table or constant with the CUDA path; the two meet only in the seeded workload
 * descriptions (module `workloads`) that both sides read.
 *
 * What it computes, in the paper's order (§3.1, "Simulation flow"):
 *   source -> locate volume -> { mirror at a boundary (§2.5) ->
 *   total and biased macroscopic cross section -> biased step
 *   l_g = -ln(xi)/(g rho sigma) (§2.4, Eq. eStepLength2) -> relocation to the
 *   boundary or move to an interaction point -> weight compensation
 *   (§2.4, Eq. eWeight) -> propagation (scatter) or absorption } -> scorers (§3.4).
 *
 * Units: cm, Angstrom, 1/cm, barn, Angstrom^3.
 *
 * Parity status per function (see also the test files that pin them):
 *   or_philox4x32_10         pinned (cuRAND host generator output)
 *   geometry distances       pinned (brute-force ray marching, enumeration)
 *   weight / step sampling   pinned (Lambert-Beer closed forms, zero-variance
 *                            implicit capture, biased-vs-unbiased equality)
 *   isotropic scattering     pinned (angular moments, infinite-medium closed forms)
 *   powder Bragg sigma       pinned in its lambda and line dependence against a
 *                            reflection-by-reflection enumeration, and in its
 *                            absolute prefactor lambda^2/(2 V0^2) against the
 *                            kinematic single-crystal cross section averaged by
 *                            Monte Carlo over random crystal orientations
 *   mirror R(Q), reflection  pinned (Table tableMirror values, bounce-count closed form)
 *   score-function gradients pinned (closed-form uncollided derivatives, finite
 *                            differences on common random numbers)
 */
#ifndef TP_ORACLE_H
#define TP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BOX = 0, OR_TUBE = 1, OR_SPHERE = 2 };
enum { OR_ROLE_BULK = 0, OR_ROLE_DETECTOR = 1, OR_ROLE_BLACK = 2 };
enum { OR_P_ABS = 0, OR_P_INC = 1, OR_P_BRAGG = 2, OR_NPROC = 3 };
enum { OR_T_COUNT = 0, OR_T_ANGULAR = 1, OR_T_PSD = 2, OR_T_WLX = 3, OR_T_MULTISCAT = 4, OR_T_DQ = 5,
       OR_T_TOF = 6 };
enum { OR_PTS_ENTRY = 0, OR_PTS_EXIT = 1 };
enum { OR_PAR_RADIUS = 0, OR_PAR_SCALE = 1, OR_PAR_DENSITY = 2 };
enum { OR_SRC_PENCIL = 0, OR_SRC_RECT = 1, OR_SRC_MODERATOR = 2 };
/* how a history ended */
enum { OR_END_ESCAPED = 0, OR_END_ABSORBED = 1, OR_END_DETECTED = 2, OR_END_BLACK = 3,
       OR_END_MIRROR = 4, OR_END_TRUNCATED = 5, OR_END_APERTURE = 6, OR_END_LOST = 7 };

#define OR_MAX_PAR 4

typedef struct {
  int shape, axis, material, role, mirror, bind_rmin, bind_rmax;
  int chopper;      /* index into or_scene.choppers or -1 */
  double c[3];      /* centre */
  double p[3];      /* box: half extents; tube: rmin, rmax, half height; sphere: rmin, rmax, - */
} or_prim;

typedef struct { double m, R0, Qc, alpha, W; } or_mirror;

/* Disk chopper (§3.5, Table tableDiskChopper) on a vacuum tube: black below
 * radius r_black, n windows of full opening theta0 (rad) evenly spread over
 * 2 pi, rotating at freq (Hz, right-hand rule about the tube axis), window 0
 * at angle phase (rad) from the first in-plane axis at time zero. */
typedef struct { double r_black; int n; double freq, theta0, phase; } or_chopper;

typedef struct {
  double sig_abs_ref;   /* Sigma_a at 1.8 A (abs_1v) or constant */
  int abs_1v;
  double sig_inc;
  int nlines;           /* Bragg lines; 0 = none */
  double V0;            /* unit cell volume, A^3 */
  const double *d, *mult, *F2;   /* per line: d (A), multiplicity, |F|^2 (barn) */
  int density_par, scale_par;    /* parameter index or -1 */
  int rod;              /* test mode, 0 normally: incoherent scattering sends the neutron
                           along +z or -z with probability 1/2 each (the rod model whose
                           two-stream closed form pins the scatter-and-continue loop) */
} or_material;

typedef struct {
  int kind, trigger, volume, face, scat;
  int nb[2];
  double lo[2], hi[2];
  double origin[3], axis[3];
} or_tally;

typedef struct {
  int kind;
  double c[3];
  double half[2];
  double lam_lo, lam_hi;
  double div[2];
  int has_aperture;
  double aperture[2];
  double slit_z;        /* moderator gun: slit plane and half sizes */
  double slit_half[2];
  double temperature;   /* > 0: Maxwell-Boltzmann energies at this temperature (K) */
} or_source;

typedef struct {
  int world_shape;
  double world_c[3], world_p[3];
  int nprim;   const or_prim* prims;
  int nmirror; const or_mirror* mirrors;
  int nchopper; const or_chopper* choppers;
  int nmat;    const or_material* mats;
  const double* bias;          /* [nmat][3] */
  or_source src;
  int ntally;  const or_tally* tallies;
  int npar;    const int* par_kind;   /* [npar] */
  double radius_nominal;
  uint64_t seed;
  int event_cap;
} or_scene;

/* Per-history record used for history-by-history comparisons. */
typedef struct {
  double first_collision[3];   /* NaN if the history never collided */
  double dir_after_first[3];   /* direction leaving the first collision (NaN if none) */
  double final_pos[3];
  double w_final;
  double A_final[OR_MAX_PAR];
  int nscat, nevents, end;
  int pad;
} or_record;

typedef struct {
  double* sum;     /* [total_bins] */
  double* sumsq;   /* [total_bins] */
  double* J;       /* [npar][total_bins] or NULL */
  double* J2;      /* [npar][total_bins] or NULL */
  int64_t counters[8];  /* histories, events, collisions, crossings, truncated, lost, mirror hits, secondaries */
} or_accum;

/* Run histories [first, first+n) of instance `inst` with parameters
 * inst_params[npar]; accumulates into acc (caller zeroes it).  Uses `threads`
 * POSIX threads over contiguous history ranges.  records (optional, [n]). */
int or_run(const or_scene* s, int inst, const double* inst_params,
           uint64_t first, uint64_t n, int threads, int want_grad,
           or_accum* acc, or_record* records);

/* Building blocks exposed for pins. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01(uint32_t a);
void or_sigma(const or_scene* s, int mat, const double* inst_params, double lambda,
              double sig[OR_NPROC]);
double or_mirror_R(const or_mirror* m, double Q);
double or_prim_exit(const or_scene* s, const or_prim* p, const double* inst_params,
                    const double r[3], const double u[3], int* face);
double or_prim_entry(const or_scene* s, const or_prim* p, const double* inst_params,
                     const double r[3], const double u[3], int* face);
int or_prim_inside(const or_scene* s, const or_prim* p, const double* inst_params,
                   const double r[3]);
void or_rotate(const double u[3], double mu, double phi, double out[3]);
int or_total_bins(const or_scene* s);

#ifdef __cplusplus
}
#endif
#endif
