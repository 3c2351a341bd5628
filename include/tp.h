/*
 * tp.h -- C ABI of the GB300 (sm_103a) neutron history engine with
 * probability-conserved cross-section biasing (arxiv 2304.06226).
 *
 * The problem (§2.1, Eq. eTransport): estimate detection probabilities
 * f_det = integral of G f_src by Monte Carlo histories.  Each history (§3.1,
 * "Simulation flow") is born at a particle gun (§3.2), is located in a volume of
 * a CSG geometry (§3.3), samples a flight length from the *biased* macroscopic
 * cross section Sigma_g = sum_i g_i Sigma_i (§2.4, Eq. eStepLength2), moves to the
 * boundary (relocation) or to an interaction point, multiplies its weight by the
 * true-to-biased likelihood ratio (§2.4, Eq. eWeight), is reflected by
 * supermirrors (§2.5, Eqs. eMirrowRef and eMirrowNewDir), scatters (isotropic
 * incoherent, Eq. eIncEla; powder Bragg lines, Eq. eCohEla) or is absorbed
 * (1/v law, §2.2), and is scored at particle-tracing states ENTRY / EXIT (§3.4).
 *
 * Conventions (every call):
 *  - No call aborts or throws.  Every call returns a tp_status; on failure
 *    tp_last_error() gives a message (thread-local, valid until the next call on
 *    the same thread).  A status other than TP_OK leaves the scene usable unless
 *    it is TP_ERR_CUDA (the CUDA context may then be unusable).
 *  - Input arrays are copied; the caller keeps ownership and may free them
 *    after the call returns.
 *  - Outputs go to caller-owned buffers, on the host or on the device as the
 *    `on_device` flag of the call says.
 *  - GPU work is ordered on the CUDA stream passed in tp_run.stream (the
 *    caller's current stream).  Host-output calls synchronise that stream.
 *  - Units: cm, Angstrom, 1/cm, barn, Angstrom^3, radians.
 *  - The library allocates its own device memory (cudaMalloc) for a scene.
 */
#ifndef TP_H
#define TP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tp_scene tp_scene; /* opaque, library-owned */

typedef enum {
  TP_OK = 0,
  TP_ERR_INVALID_ARG = 1, /* a bad argument or description (message says which) */
  TP_ERR_GEOMETRY = 2,    /* overlapping primitives, primitive outside the world */
  TP_ERR_CUDA = 3,        /* a CUDA runtime error */
  TP_ERR_OOM = 4,         /* device allocation failed */
  TP_ERR_TIMEOUT = 5,     /* a device-side wait or iteration cap gave up */
  TP_ERR_STATE = 6,       /* call out of order (e.g. run before tp_set_materials) */
  TP_ERR_ABORTED = 7      /* the run was stopped by tp_abort; its tallies are partial */
} tp_status;

/* Solids (Appendix A: Box, Tube, Orb/Sphere with full phi). */
enum { TP_BOX = 0, TP_TUBE = 1, TP_SPHERE = 2 };
/* Volume roles: transport inside; terminal scorer volume; terminal absorber. */
enum { TP_ROLE_BULK = 0, TP_ROLE_DETECTOR = 1, TP_ROLE_BLACK = 2 };
/* Processes, in the order they are sampled. */
enum { TP_PROC_ABS = 0, TP_PROC_INC = 1, TP_PROC_BRAGG = 2, TP_NPROC = 3 };
/* Scorers (§3.4, Table tableScorer): a count, Angular, PSD (x,y), a
 * wavelength x position monitor (WlSpectrum crossed with a PSD axis),
 * MultiScat (number of scatterings), DeltaMomentum (elastic momentum
 * transfer, Eq. eQelastic) and TOF (time of flight). */
enum { TP_TALLY_COUNT = 0, TP_TALLY_ANGULAR = 1, TP_TALLY_PSD = 2, TP_TALLY_WLX = 3,
       TP_TALLY_MULTISCAT = 4, TP_TALLY_DQ = 5, TP_TALLY_TOF = 6 };
/* Particle tracing states that trigger scorers (§3.4). */
enum { TP_PTS_ENTRY = 0, TP_PTS_EXIT = 1 };
/* Differentiable instance parameters. */
enum { TP_PAR_RADIUS = 0, TP_PAR_SCALE = 1, TP_PAR_DENSITY = 2 };
/* Particle guns (§3.2): a pencil (SimpleThermalGun with a fixed direction), a
 * rectangle emitting along +z with uniform divergence, and a moderator
 * rectangle aiming at a slit (UniModeratorGun / MaxwellianGun). */
enum { TP_SRC_PENCIL = 0, TP_SRC_RECT = 1, TP_SRC_MODERATOR = 2 };
/* Transport arithmetic. */
enum { TP_FP32 = 0, TP_FP64 = 1 };

#define TP_MAX_PARAMS 4
#define TP_MAX_TALLIES 16

/* One CSG primitive, placed in the world with no rotation.
 * shape TP_BOX: params = half extents (x, y, z).
 * shape TP_TUBE: params = (rmin, rmax, half height), axis 0/1/2 = x/y/z.
 * shape TP_SPHERE: params = (rmin, rmax, unused).
 * material: index into tp_set_materials' array, -1 = vacuum.
 * mirror: index into tp_scene_desc.mirrors or -1.  A neutron arriving at the
 *   boundary of a mirror primitive is reflected (§2.5) and never enters it.
 * bind_rmin / bind_rmax: the radius moves with the TP_PAR_RADIUS instance
 *   parameter, by (value - radius_nominal).
 * chopper: index into tp_scene_desc.choppers or -1.  The primitive is then a
 *   vacuum (material -1) bulk TP_TUBE and no mirror: the disk of a chopper
 *   (§3.5, DiskChopper), whose outer radius is the tube's rmax. */
typedef struct {
  int shape, axis, material, role, mirror, bind_rmin, bind_rmax, chopper;
  double centre[3];
  double params[3];
} tp_prim;

/* Supermirror (§2.5, Eq. eMirrowRef, Table tableMirror): m, R0, Qc (1/A),
 * alpha (A), W (1/A). */
typedef struct { double m, R0, Qc, alpha, W; } tp_mirror;

/* Disk chopper in ray-tracing mode (§2.1, Eq. eRayTracing; §3.5, Table
 * tableDiskChopper).  The disk is infinitely thin: a neutron entering its
 * tube keeps its weight (epsilon = 1) if, at the entry point and time, it is
 * at radius >= r_black from the tube axis and inside an opening window, and is
 * stopped (epsilon = 0, end code "black") otherwise.  There are n_windows
 * windows of full opening theta0 (rad), evenly spread over 2 pi, turning at
 * freq (Hz; positive = right-hand rule about the tube axis); at time zero
 * window 0 is centred at angle phase (rad) from the first in-plane axis
 * (axis+1 mod 3, towards axis+2 mod 3).  Time is the time of flight since the
 * source (see TP_TALLY_TOF).  ENTRY scorers of the tube see the neutron before
 * the mask, EXIT scorers after it. */
typedef struct {
  double r_black;
  int n_windows;
  double freq, theta0, phase;
} tp_chopper;

/* A scorer.  kind TP_TALLY_ANGULAR bins the angle between (position - origin)
 * and axis over [lo[0], hi[0]) in nbins[0] bins; TP_TALLY_PSD bins x over
 * [lo[0],hi[0]) and y over [lo[1],hi[1]); TP_TALLY_WLX bins the wavelength over
 * [lo[0],hi[0]) and x over [lo[1],hi[1]); TP_TALLY_MULTISCAT bins the number of
 * scatterings over [lo[0], hi[0]); TP_TALLY_DQ bins Q = 4 pi sin(theta/2)/lambda
 * (1/A) over [lo[0], hi[0]), theta being the angle between (position - origin)
 * and axis (origin = sample position, axis = beam direction: the elastic
 * momentum transfer of Eq. eQelastic); TP_TALLY_TOF bins the time of flight
 * t (s) over [lo[0], hi[0]): sources emit at t = 0 and a neutron that has flown
 * a path L (cm) at wavelength lambda (A) is at t = L lambda / 395603.4 (its
 * speed h / (m_n lambda); every process is elastic).  Bins are laid out
 * axis-0 major.
 * trigger TP_PTS_ENTRY / TP_PTS_EXIT of `volume` (primitive index, -1 = world).
 * face: -1 any, else the face id (box 2*axis + (1 for the + face); tube 0
 *   outer, 1 inner, 2 -cap, 3 +cap; sphere 0 outer, 1 inner).
 * scat: -1 any, else only neutrons scattered exactly `scat` times (the
 *   scatnum filter of the DeltaMomentum scorer, Appendix C). */
typedef struct {
  int kind, trigger, volume, face, scat;
  int nbins[2];
  double lo[2], hi[2];
  double origin[3], axis[3];
} tp_tally_desc;

/* Source.  TP_SRC_PENCIL: at centre, direction +z.  TP_SRC_RECT: uniform on the
 * rectangle centre +- half (x, y), direction +z tilted by angles uniform in
 * +-div (x, y).  TP_SRC_MODERATOR: uniform on the rectangle centre +- half
 * (x, y) at z = centre[2], aimed at a point uniform on the slit rectangle
 * (centre.x, centre.y) +- slit_half at z = slit_z (> centre[2]).
 * Wavelength uniform on [lambda_lo, lambda_hi], or, if temperature > 0, from
 * the Maxwell-Boltzmann energy distribution sqrt(E) exp(-E/kT) at that
 * temperature (K); a Maxwellian source with an angular divergence must be
 * TP_SRC_MODERATOR (the two would share random numbers otherwise), and
 * tp_create_scene rejects the combination with TP_ERR_INVALID_ARG.  With
 * has_aperture, neutrons born outside centre +- aperture are stopped.
 * (§3.2: ParticleGun, UniModeratorGun, MaxwellianGun.) */
typedef struct {
  int kind;
  double centre[3];
  double half[2];
  double lambda_lo, lambda_hi;
  double div[2];
  int has_aperture;
  double aperture[2];
  double slit_z;
  double slit_half[2];
  double temperature;
} tp_source;

/* Scene description.  The world is a vacuum box (params = half extents) or
 * sphere (params = (0, radius, 0)) containing every primitive; leaving it ends
 * a history (EXIT of volume -1).  Primitives must not overlap (touching is
 * allowed); at most TP_MAX_PRIMS of them.  inst_params is
 * [n_instances][n_params]; param_kind[n_params]. */
#define TP_MAX_PRIMS 16777214
typedef struct {
  int world_shape;
  double world_centre[3], world_params[3];
  int n_prims;     const tp_prim* prims;
  int n_mirrors;   const tp_mirror* mirrors;
  tp_source source;
  int n_tallies;   const tp_tally_desc* tallies;
  int n_instances; const double* inst_params;
  int n_params;    const int* param_kind;
  double radius_nominal;
  int precision;   /* TP_FP32 | TP_FP64 */
  int event_cap;   /* events per history before it is truncated (counted); 0 = 4096 */
  int n_choppers;  const tp_chopper* choppers;
} tp_scene_desc;

/* Creates a scene: validates the description (TP_ERR_INVALID_ARG,
 * TP_ERR_GEOMETRY) and uploads it to the current CUDA device.  *out receives a
 * library-owned handle, freed by tp_destroy_scene. */
tp_status tp_create_scene(const tp_scene_desc* desc, tp_scene** out);

/* Material macroscopic cross sections (§2.2, §2.3):
 *   absorption Sigma_a(lambda) = sigma_abs_ref * lambda/1.8 (abs_1v = 1, the
 *     1/v law with the reference at 1.8 A) or sigma_abs_ref (abs_1v = 0);
 *   isotropic incoherent elastic sigma_inc (Eq. eIncEla);
 *   powder Bragg lines (Eq. eCohEla averaged over orientations):
 *     Sigma(lambda) = lambda^2/(2 V0^2) sum_{2 d_i >= lambda} mult_i F2_i d_i
 *     with d in A, F2 = |F|^2 in barn per cell, V0 in A^3.
 * density_param / scale_param: instance parameter index multiplying every
 *   process / the Bragg term, or -1.  Lines may come in any order.
 * Replaces previous materials; resets bias factors to 1. */
typedef struct {
  double sigma_abs_ref;
  int abs_1v;
  double sigma_inc;
  int n_lines;
  double V0;
  const double* d;
  const double* mult;
  const double* F2;
  int density_param, scale_param;
} tp_material;

tp_status tp_set_materials(tp_scene* s, const tp_material* m, int n);

/* Per-process bias factors g[TP_NPROC] of one material (§3.5: scatter_bias,
 * abs_bias; §2.4): flights are sampled from sum_i g_i Sigma_i and the weight is
 * compensated by Eq. eWeight.  g_i >= 0; g_i = 0 removes process i from the
 * sampling (its Sigma still attenuates the weight); 1 = unbiased. */
tp_status tp_set_bias(tp_scene* s, int material, const double g[TP_NPROC]);

/* Optional per-history record (first collision, final state), written for
 * the first n_records histories of instance 0 of a run: history id
 * first_history[0] + i goes to records[i]. */
typedef struct {
  double first_collision[3];
  double dir_after_first[3];
  double final_pos[3];
  double w_final;
  double A_final[TP_MAX_PARAMS];
  int nscat, nevents, end, pad;
} tp_record;

/* One batch of histories.  n_histories[n_instances] (host array) histories per
 * instance with ids first_history[i] .. first_history[i]+n_histories[i]-1
 * (first_history may be NULL: 0).  Random numbers are Philox4x32-10 keyed by
 * (seed, event, sub-stream, history id, instance), so results do not depend on
 * the launch shape and runs over disjoint id ranges add up.
 * want_grad accumulates the score-function tallies for tp_backward.
 * stream: a cudaStream_t (NULL = legacy default stream).
 * kernel: TP_KERNEL_HISTORY (one neutron per thread until it ends),
 *   TP_KERNEL_EVENT (neutrons regrouped by event type every event in a
 *   shared-memory bank per block), TP_KERNEL_WARPQ (a pool of neutrons per
 *   warp; each step runs the event type most of them wait for), or 0: the
 *   autotuner times the variants (and block sizes) on the scene's first run
 *   with and without gradients and keeps the fastest.
 * block_size / ctas_per_sm: 0 = autotuned / the most that fit on an SM.  The
 *   FP32 kernels exist in an 80-register and a 64-register build; a request
 *   for more CTAs per SM than the 80-register build allows (more than 3 of 256
 *   threads) selects the 64-register one.  kernel 0 lets the autotuner pick
 *   the variant, block size, build and table staging on the scene's first run
 *   (with and without gradients separately).
 * use_graph: 1 = run as a CUDA graph [work-description copies, work-counter
 *   reset, persistent kernel] captured on the first call with a given launch
 *   (kernel, block, CTAs, gradients, seed, total histories, records) and
 *   replayed afterwards; history counts and first ids may change between
 *   replays (they are read from the scene's pinned staging buffer).
 * records: device array of n_records tp_record, or NULL.
 * secondaries (gradient runs with a radius parameter): the radius-derivative
 *   secondaries are transported 1 = where they are made, while their primary
 *   waits, or 2 = queued in device memory and transported by a second pass of
 *   the plain kernel, the run going through the histories in chunks whose
 *   secondaries fit the queue (6 records per history, at most 2^31 records
 *   of 56 bytes in FP32 and at most half the free device memory, sized at the
 *   first such run; a secondary finding the queue full is transported in
 *   place); 0 =
 *   chosen by the autotuner with kernel 0, else 1.  Results do not depend on
 *   the choice (each secondary has its own random numbers).
 * regroup (event kernel, plain runs): the bank is regrouped every `regroup`
 *   events -- sorted into queues by event type (advance inside a primitive,
 *   advance in the world region, collision, refill), so that a warp runs one
 *   kind of event -- and in between each thread runs the next events of the
 *   neutron it holds; 0 = chosen by the autotuner with kernel 0 (1 or 4),
 *   else 1.  Results do not depend on it.
 * stage (explicit kernel): where the kernel reads the scene tables from: 0 =
 *   copied into shared memory when they fit (at most 96 KiB beside the
 *   neutron bank), 1 = copied into shared memory (TP_ERR_INVALID_ARG if they
 *   do not fit), 2 = read from device memory through L1/L2 (leaves room for
 *   more blocks per SM).  With kernel 0 the autotuner decides and stage must
 *   be 0.  Results do not depend on it. */
typedef struct {
  uint64_t seed;
  const uint64_t* n_histories;
  const uint64_t* first_history;
  int want_grad;
  void* stream;
  int block_size;
  int ctas_per_sm;
  tp_record* records;
  uint64_t n_records;
  int kernel;
  int use_graph;
  int secondaries;
  int regroup;
  int stage;
} tp_run;

enum { TP_KERNEL_AUTO = 0, TP_KERNEL_HISTORY = 1, TP_KERNEL_EVENT = 2, TP_KERNEL_WARPQ = 3 };

/* Runs histories and accumulates their scores into the scene's tallies
 * (sum w, sum w^2 per bin per instance, and the gradient tallies).  Returns
 * after the launch is queued on the stream, so errors raised on the device
 * (a bounded wait that gave up: TP_ERR_TIMEOUT; a run stopped by tp_abort:
 * TP_ERR_ABORTED) are reported by the next tp_get_counters, together with the
 * per-run counts (truncated histories, lost particles). */
tp_status tp_run_histories(tp_scene* s, const tp_run* r);

/* Mean and standard error per source history of every bin of `tally` for
 * `instance`: mean = sum w / N, stderr = sqrt((sum w^2/N - mean^2)/(N-1)),
 * N = histories run for that instance.  mean / stderr_ receive nbins[0]*nbins[1]
 * doubles (device pointers if on_device, else host; the call then
 * synchronises).  stderr_ may be NULL. */
tp_status tp_read_tallies(tp_scene* s, int tally, int instance, double* mean, double* stderr_,
                          int on_device);

/* Raw accumulators of one instance: sum w and sum w^2 over every bin of every
 * tally (concatenated in tally order); J and J2 (may be NULL) receive
 * [n_params][total bins] of sum w A_p and sum (w A_p)^2. */
tp_status tp_read_raw(tp_scene* s, int instance, double* sum, double* sumsq, double* J, double* J2,
                      int on_device);

/* Overwrites the raw accumulators of one instance -- sum, sumsq
 * ([total bins]), J, J2 ([n_params][total bins], may be NULL) -- and its
 * history count, the layout of tp_read_raw.  For combining runs made
 * elsewhere: after the partial accumulators of several GPUs (disjoint history
 * ids) are summed, writing the sums back makes tp_read_tallies and
 * tp_backward give the statistics of all histories (§2.1: the estimate is a
 * mean over independent histories, so partial sums add).  Synchronises. */
tp_status tp_write_raw(tp_scene* s, int instance, const double* sum, const double* sumsq, const double* J,
                       const double* J2, double n_histories, int on_device);

/* Backward pass of the tallies with respect to the instance parameters:
 *   grad_params[i][p] = sum_b grad_tallies[i][b] * dmean_b/dtheta_p
 * over all bins b of all tallies of instance i, where dmean/dtheta comes from
 * the score-function (likelihood-ratio) accumulators of the forward run (plus
 * the interface term for radii).  grad_tallies: [n_instances][total bins];
 * grad_params: [n_instances][n_params]; both on the device if on_device.
 * The derivative is per unit of the parameter (radius: per cm; scale and
 * density: per unit multiplier). */
tp_status tp_backward(tp_scene* s, const double* grad_tallies, double* grad_params, int on_device,
                      void* stream);

/* Replaces the instance parameters ([n_instances][n_params], same layout as
 * tp_scene_desc.inst_params) and re-validates the geometry (TP_ERR_GEOMETRY
 * leaves the old values in place).  Tallies are not reset. */
tp_status tp_set_params(tp_scene* s, const double* inst_params);

/* Zeroes every tally and history count. */
tp_status tp_reset_tallies(tp_scene* s);

/* Counters since the last reset: histories, events, collisions, boundary
 * crossings, truncated histories, lost neutrons, mirror reflections, derivative
 * secondaries.  Synchronises the device, fills `out` in every case, then returns
 * the status the kernels recorded since the last reset: TP_OK,
 * TP_ERR_TIMEOUT (a block's bounded wait for its copy of the scene tables gave
 * up; that block transported nothing) or TP_ERR_ABORTED (tp_abort). */
tp_status tp_get_counters(tp_scene* s, int64_t out[8]);

/* Asks every run of the scene that is queued or running to stop: the kernels
 * poll a flag in mapped host memory whenever they claim new histories, claim
 * none once it is set, finish the neutrons they hold and record
 * TP_ERR_ABORTED.  Callable from any host thread, also while another thread
 * waits for the run; it does not wait itself.  The scene stays aborted (later
 * runs stop at once) until tp_reset_tallies, which clears the flag along with
 * the partial tallies.  No device call is made. */
tp_status tp_abort(tp_scene* s);

/* Test hooks, for the failure-detection tests only (0 = normal operation).
 * TP_TEST_SKIP_TABLE_COPY: the kernels arm their wait for the bulk copy of the
 * scene tables into shared memory but issue no copy, so that the bounded wait
 * (about half a second) runs out: each block records TP_ERR_TIMEOUT and
 * returns with nothing in flight and nothing transported.  s = NULL sets the
 * flags of tp_run_histories_noalloc, which has no scene.
 * TP_TEST_FULL_BUILD: the scene runs the kernels' complete feature build even
 * if the lean one serves it (the two must agree; the test of that uses it).
 * TP_TEST_SMALL_SEC_QUEUE: the queue of radius-derivative secondaries holds at
 * most 2^20 records, so that a short run goes through several chunks. */
enum { TP_TEST_SKIP_TABLE_COPY = 1, TP_TEST_FULL_BUILD = 2, TP_TEST_SMALL_SEC_QUEUE = 4 };
tp_status tp_set_test_flags(tp_scene* s, int flags);

/* Launch configuration of the last run: kernel (TP_KERNEL_*), block size and
 * CTAs per SM. */
tp_status tp_get_launch(tp_scene* s, int* kernel, int* block_size, int* ctas_per_sm);

/* Transport kernels the last tp_run_histories launched: 1, or with queued
 * secondaries two per chunk of histories (first pass, second pass); 0 before
 * any run or if the run had no histories.  No device work. */
int tp_get_launch_count(const tp_scene* s);

/* The complete launch configuration of the scene's last tp_run_histories
 * (after the autotuner, if it ran): transport kernel (TP_KERNEL_*), threads
 * per block, CTAs per SM, tables staged in shared memory (1) or read from
 * device memory (0), register build (80 or 64 registers per thread: the
 * kernels are compiled for 3 and for 4 blocks of 256 threads per SM), full
 * build (1: mirrors, choppers, per-order scorers, moderator guns and
 * separate absorption factors compiled in; 0: the lean build for scenes
 * without them), regrouping interval of the event kernel, secondaries queued
 * for a second pass (1) or transported in place (0), and transport kernels
 * launched.  All zero before the first run.  Errors: TP_ERR_INVALID_ARG for
 * NULL arguments. */
typedef struct {
  int kernel, block_size, ctas_per_sm, staged, registers, full_build, regroup, queued_secondaries, launches;
} tp_launch_info;
tp_status tp_get_launch_info(const tp_scene* s, tp_launch_info* out);

/* Total bins over all tallies (per instance). */
int tp_total_bins(const tp_scene* s);

/* ------------------------------------------------------------------------
 * Allocation-free run (the paper has no counterpart: this is a deployment
 * entry point of this library).
 *
 * Some callers cannot call cudaMalloc: code whose device memory is owned by
 * another allocator, or that runs where new device allocations are not
 * allowed.  tp_run_histories_noalloc runs the same transport kernel as
 * tp_run_histories for a scene given as a description, without creating a
 * scene and without allocating device or pinned host memory.  The scene
 * tables, the per-run work description and the kernel's work counter, event
 * counters and status word are kept in one fixed device array of
 * TP_NOALLOC_SCRATCH_BYTES bytes that every GPU loading this library holds
 * until the process exits.
 *  - desc, mats[n_mats], bias ([n_mats][TP_NPROC], NULL = all 1) and r are
 *    read as in tp_create_scene, tp_set_materials, tp_set_bias and
 *    tp_run_histories, with these restrictions (TP_ERR_INVALID_ARG
 *    otherwise): r->want_grad, r->records, r->use_graph and r->secondaries
 *    must be 0/NULL, r->regroup 0 or 1, r->stage 0 or 1, and r->kernel 0 or TP_KERNEL_HISTORY: the call always
 *    runs the history-based kernel with the tables staged when they fit, and
 *    builds no uniform grid, so a scene of many primitives tests all of them
 *    at every step of the world region (same results, more work).
 *  - sum, sumsq: caller-owned device arrays of [n_instances][total bins]
 *    doubles; the call ADDS sum w and sum w^2 of every bin into them.
 *  - counters_out (host, may be NULL): the counters of this call.
 *  - The call waits for its work and then reads the status word the kernel
 *    leaves, whether or not counters_out is given: a bounded device wait that
 *    gave up returns TP_ERR_TIMEOUT (the sums then hold nothing of this
 *    call).
 *  - Limits: at most TP_NOALLOC_MAX_INSTANCES instances and
 *    TP_NOALLOC_MAX_TABLE_BYTES bytes of scene tables (checked first:
 *    TP_ERR_INVALID_ARG with a message naming the limit).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - The call waits for its own work on r->stream before returning.  Every
 *    call shares the one array, which keeps the last call's contents (each
 *    call clears what must start at zero): calls that overlap on the GPU, from
 *    several threads or streams, race and give wrong results. */
#define TP_NOALLOC_MAX_INSTANCES 64
#define TP_NOALLOC_MAX_TABLE_BYTES 65536
#define TP_NOALLOC_SCRATCH_BYTES (65536 + 4096 + 256)
tp_status tp_run_histories_noalloc(const tp_scene_desc* desc, const tp_material* mats, int n_mats,
                                   const double* bias, const tp_run* r, double* sum, double* sumsq,
                                   int64_t counters_out[8]);

/* ------------------------------------------------------------------------
 * Measured hardware rates of the current device (no counterpart in the paper:
 * the denominators of this library's roofline).  The history loop is bound by
 * instruction issue -- FP32 and integer arithmetic, the special-function unit
 * for its logarithms, exponentials and sines, FP64 atomics into the tallies --
 * not by HBM or tensor cores, so its roofline fraction is taken against these
 * rates, measured by short bounded microbenchmarks (each a fixed number of
 * iterations of independent dependency chains at full occupancy, timed with
 * CUDA events on `stream` after a warm-up launch).  Rates are lane operations
 * per second over the whole device, at whatever clock the device runs
 * (sm_clock_mhz, measured during the FP32 kernel from clock64 and the global
 * timer).  Allocates and frees about 35 MB of device scratch; synchronises
 * `stream`; takes well under a second. */
typedef struct {
  double fp32_fma;          /* FP32 fused multiply-adds */
  double int32_imad;        /* 32-bit integer multiply-adds */
  double int32_logic;       /* 32-bit three-input logic operations */
  double mufu_lg2, mufu_ex2, mufu_sin;   /* special-function unit, approximate */
  double fp64_fma;          /* FP64 fused multiply-adds */
  double atomic_f64_spread; /* FP64 global atomic adds into 3600 bins (one detector) */
  double atomic_f64_hot;    /* FP64 global atomic adds piled on 32 bins */
  double l2_read_bytes;     /* bytes per second read from an L2-resident buffer */
  double sm_clock_mhz;
  int sm_count;
} tp_peaks;
tp_status tp_measure_peaks(tp_peaks* out, void* stream);

void tp_destroy_scene(tp_scene* s);
const char* tp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
