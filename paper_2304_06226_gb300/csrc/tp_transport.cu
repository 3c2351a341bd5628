// tp_transport.cu -- sm_103a kernels of the biased neutron history loop.
//
// One persistent launch processes every history of every instance (gradient
// runs may add a second launch over the queued radius-derivative secondaries).
// Three kernels share the physics and differ in how neutrons meet lanes: the
// history kernel (each lane carries one neutron in registers and takes the next
// id of its warp's chunk when it ends), the event kernel (a block-wide bank of
// neutrons sorted every iteration by what they wait for) and the warp-pool
// kernel (each warp runs the most common pending event of its own pool); all
// claim history ids with global atomics, so lanes stay busy until the work
// runs out (no per-history kernel, no host round trip).  A step is one event of
// the simulation flow of §3.1: cross sections of the current volume, biased
// flight length (§2.4, Eq. eStepLength2), distance to the next boundary, move
// and weight compensation (§2.4, Eq. eWeight), then either relocation across
// the boundary (scorers, supermirror of §2.5) or an interaction (absorption,
// isotropic incoherent or powder Bragg scattering).
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
// (event k, sub-stream, history id, instance): sub-stream 0 carries flight,
// process, cosine and azimuth of event k, sub-stream 1 the Bragg line; the source
// is event 0; a radius-derivative secondary set up at event k uses (k, 2, ..)
// and secondary s of a history uses sub-streams 4+2s and 5+2s.  Results are thus
// independent of the launch shape and of which lane ran which history.
//
// Tallies are FP64 sums of w and w^2 per bin (plus the score-function tallies),
// added with warp-aggregated atomics: the lanes hitting one bin find each other
// once per score, sum their values by pointer jumping over their group
// (shuffles, in the transport precision) and the group's lowest lane issues one
// FP64 atomic per array.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "tp_internal.h"

namespace tp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Compile-time options of a kernel build (template parameter OPT): kOptGrid
// walks the uniform grid of a large scene; kOptFull compiles the complete
// feature set -- supermirrors, disk choppers, every scorer kind and the
// moderator / Maxwellian / divergent guns with their apertures.  Without it
// (the lean build, chosen by the host for scenes that use none of those) the
// kernel carries only boxes, tubes and spheres, count / angular / PSD scorers
// and pencil or rectangle guns, a smaller instruction footprint for the hot
// loop.  Both builds compute the same thing for the scenes they accept.
// kOptNoSec (gradient runs of the history kernel without a radius parameter,
// chosen at launch): no radius-derivative secondary can arise, so the parking
// place and the secondary's state drop out of the registers.
constexpr int kOptGrid = 1, kOptFull = 2, kOptNoSec = 4;

// ---------------------------------------------------------------------------
// Precision traits
// ---------------------------------------------------------------------------
template <typename R> struct Tr;
template <> struct Tr<float> {
  static __device__ __forceinline__ float u01(uint32_t a) {
    return (float)(a >> 8) * 5.9604644775390625e-8f + 2.98023223876953125e-8f;  // ((a>>8)+1/2) 2^-24
  }
  static __device__ __forceinline__ float nudge(float m) { return 1e-5f * fmaxf(1.0f, m); }
  static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
  // -ln(u01(a)), the step of Eq. eStepLength2 per unit of Sigma_g: the
  // hardware logarithm (absolute error below 4e-7 on [0.5, 1)), except within
  // 1e-6 of 1 where that error could reach the value itself and log1p of the
  // exact u - 1 is taken
  static __device__ __forceinline__ float neg_log_u01(uint32_t a) {
    const float u = u01(a);
    return (a >> 8) < 0xFFFFF0u ? -__logf(u) : -log1pf(u - 1.0f);
  }
  static constexpr float kPi = 3.14159265358979323846f;
  static constexpr float kTwoPi = 6.283185307179586f;
  static constexpr float kFourPi = 12.566370614359172f;
};
template <> struct Tr<double> {
  static __device__ __forceinline__ double u01(uint32_t a) {
    return ((double)a + 0.5) * 2.3283064365386963e-10;  // (a + 1/2) 2^-32
  }
  static __device__ __forceinline__ double nudge(double m) { return 1e-9 * fmax(1.0, m); }
  static __device__ __forceinline__ double neg_log_u01(uint32_t a) { return -log(u01(a)); }
  static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
  static constexpr double kPi = 3.14159265358979323846;
  static constexpr double kTwoPi = 6.283185307179586;
  static constexpr double kFourPi = 12.566370614359172;
};

// h^2 / (2 m_n) in meV A^2: E = kH2over2mn / lambda^2
constexpr double kH2over2mn = 81.80420;
// h / m_n in cm/s per A of wavelength: speed v = kHoverMn / lambda, so a path
// of L cm takes L lambda / kHoverMn seconds
constexpr double kHoverMn = 395603.4012;

__device__ __forceinline__ float d_log(float x) { return logf(x); }
__device__ __forceinline__ double d_log(double x) { return log(x); }
__device__ __forceinline__ float d_exp(float x) { return expf(x); }
__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ void d_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void d_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float d_tanh(float x) { return tanhf(x); }
__device__ __forceinline__ double d_tanh(double x) { return tanh(x); }
__device__ __forceinline__ float d_tan(float x) { return tanf(x); }
__device__ __forceinline__ double d_tan(double x) { return tan(x); }
__device__ __forceinline__ float d_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double d_atan2(double y, double x) { return atan2(y, x); }

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
// Out of line: the block is drawn at several places of the event loop, and
// one shared copy keeps the loop's instruction footprint smaller (measured
// faster than inlining every copy).
__device__ __noinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ---------------------------------------------------------------------------
// Per-lane neutron state
// ---------------------------------------------------------------------------
template <typename R>
struct Particle {
  R x[3], u[3];
  R lam, w;
  R s;       // path length flown since the source (time of flight s lam / kHoverMn)
  int vol, nscat;
  uint32_t k, hid, inst;
  int last;  // primitive just left, flags and stuck count (see kNoPrim)
  // sub0 != 0 marks a radius-derivative secondary (the plain second pass of
  // gradient runs transports them), nsec counts the secondaries made
  uint32_t sub0, nsec;
  // gradient runs only (zero in plain runs, whose shared-memory banks keep
  // just the fields above): the score-function accumulators
  R A[kMaxPar];
};

template <typename R>
struct View {
  const DPrim<R>* prims;
  const DMat<R>* mats;
  const DMirror<R>* mirrors;
  const DChopper<R>* choppers;
  const DTally<R>* tallies;
  const R* line_d;
  const R* line_cum;
  const int* nb;
};

// Neutron bank in shared memory as a structure of arrays: the neutron state
// is a sequence of words (32-bit in FP32, 64-bit in FP64) and word i of the
// neutron in slot s lives at w[i * n + s], so that a warp touching the same
// field of different slots reads consecutive words.  Plain runs (GRAD false)
// keep only the words before Particle::A -- the accumulators are zero there --
// which shrinks the bank by a fifth.
template <typename R, bool GRAD>
struct Bank {
  using Word = typename std::conditional<sizeof(R) == 8, unsigned long long, unsigned>::type;
  static constexpr size_t kBytes = GRAD ? sizeof(Particle<R>) : offsetof(Particle<R>, A);
  static constexpr int kWords = (int)(kBytes / sizeof(Word));
  static_assert(kBytes % sizeof(Word) == 0 && sizeof(Particle<R>) % sizeof(Word) == 0, "whole words");
  Word* w;
  int n;   // slots
  __device__ __forceinline__ Bank(void* base, int nslots) : w(static_cast<Word*>(base)), n(nslots) {}
  __device__ __forceinline__ Particle<R> load(int s) const {
    Word t[sizeof(Particle<R>) / sizeof(Word)];
#pragma unroll
    for (int i = 0; i < kWords; ++i) t[i] = w[i * n + s];
#pragma unroll
    for (int i = kWords; i < (int)(sizeof(Particle<R>) / sizeof(Word)); ++i) t[i] = 0;
    Particle<R> P;
    memcpy(&P, t, sizeof P);
    return P;
  }
  __device__ __forceinline__ void store(int s, const Particle<R>& P) const {
    Word t[sizeof(Particle<R>) / sizeof(Word)];
    memcpy(t, &P, sizeof P);
#pragma unroll
    for (int i = 0; i < kWords; ++i) w[i * n + s] = t[i];
  }
  // the volume field alone (the regrouping reads it to sort advances)
  __device__ __forceinline__ int vol(int s) const {
    constexpr size_t off = offsetof(Particle<R>, vol);
    const Word* word = w + (off / sizeof(Word)) * n + s;
    return reinterpret_cast<const int*>(word)[(off % sizeof(Word)) / sizeof(int)];
  }
  static __host__ __device__ constexpr size_t bytes(int nslots) { return kBytes * (size_t)nslots; }
};

// Register arrays are only indexed with compile-time indices (a runtime index
// would move them to local memory): these select / update element i.
template <typename R>
__device__ __forceinline__ R sel(const R (&v)[kMaxPar], int i, R dflt) {
  R r = dflt;
#pragma unroll
  for (int k = 0; k < kMaxPar; ++k)
    if (k == i) r = v[k];
  return r;
}

template <typename R>
__device__ __forceinline__ void add_at(R (&v)[kMaxPar], int i, R x) {
#pragma unroll
  for (int k = 0; k < kMaxPar; ++k)
    if (k == i) v[k] += x;
}

// ---------------------------------------------------------------------------
// Cross sections
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int active_lines(const View<R>& V, const DMat<R>& m, R lam) {
  // lines sorted by d descending: count of 2 d >= lambda by binary search
  int lo = 0, hi = m.nlines;
  const R* d = V.line_d + m.line_off;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (R(2) * d[mid] >= lam) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <typename R>
__device__ __forceinline__ void sigma(const View<R>& V, int mat, const R (&ip)[kMaxPar], R lam, R sig[TP_NPROC]) {
  const DMat<R>& m = V.mats[mat];
  const R dens = sel(ip, m.density_par, R(1));
  const R scale = sel(ip, m.scale_par, R(1));
  sig[TP_PROC_ABS] = dens * (m.abs_1v ? m.sig_abs_ref * lam * R(1.0 / 1.8) : m.sig_abs_ref);
  sig[TP_PROC_INC] = dens * m.sig_inc;
  R sb = R(0);
  if (m.nlines > 0) {
    const int n = active_lines(V, m, lam);
    sb = dens * scale * m.bragg_pref * lam * lam * V.line_cum[m.cum_off + n];
  }
  sig[TP_PROC_BRAGG] = sb;
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
template <typename R>
struct Radii { R r0, r1, h; };

template <typename R>
__device__ __forceinline__ Radii<R> radii(const DPrim<R>& p, R dR) {
  Radii<R> r{p.p[0], p.p[1], p.p[2]};
  if (p.flags & F_BIND_RMIN) r.r0 += dR;
  if (p.flags & F_BIND_RMAX) r.r1 += dR;
  return r;
}

// local frame: q[0], q[1] transverse, q[2] along the tube axis
template <typename R>
__device__ __forceinline__ void to_local(const DPrim<R>& p, const R x[3], const R u[3], R q[3], R v[3]) {
  const R d0 = x[0] - p.c[0], d1 = x[1] - p.c[1], d2 = x[2] - p.c[2];
  if (p.shape == TP_TUBE) {
    if (p.axis == 0) { q[0] = d1; q[1] = d2; q[2] = d0; v[0] = u[1]; v[1] = u[2]; v[2] = u[0]; }
    else if (p.axis == 1) { q[0] = d2; q[1] = d0; q[2] = d1; v[0] = u[2]; v[1] = u[0]; v[2] = u[1]; }
    else { q[0] = d0; q[1] = d1; q[2] = d2; v[0] = u[0]; v[1] = u[1]; v[2] = u[2]; }
  } else {
    q[0] = d0; q[1] = d1; q[2] = d2; v[0] = u[0]; v[1] = u[1]; v[2] = u[2];
  }
}

// Roots of A t^2 + 2 B t + C = 0 with disc = B^2 - A C given; stable form.
template <typename R>
__device__ __forceinline__ void roots(R A, R B, R C, R disc, R* t0, R* t1) {
  const R sq = d_sqrt(disc);
  const R qq = -(B + copysign(sq, B));
  R a, b;
  if (qq != R(0)) { a = qq / A; b = C / qq; } else { a = R(0); b = R(0); }
  *t0 = fmin(a, b);
  *t1 = fmax(a, b);
}

// Quadratic pieces of a tube (2-D, transverse) or sphere (3-D) at radius r.
template <typename R>
struct Quad { R A, B, C2, cross2; };

template <typename R>
__device__ __forceinline__ Quad<R> quad(const R q[3], const R v[3], bool tube) {
  Quad<R> Q;
  if (tube) {
    Q.A = v[0] * v[0] + v[1] * v[1];
    Q.B = q[0] * v[0] + q[1] * v[1];
    Q.C2 = q[0] * q[0] + q[1] * q[1];
    const R c = q[0] * v[1] - q[1] * v[0];
    Q.cross2 = c * c;
  } else {
    Q.A = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    Q.B = q[0] * v[0] + q[1] * v[1] + q[2] * v[2];
    Q.C2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    const R c0 = q[1] * v[2] - q[2] * v[1], c1 = q[2] * v[0] - q[0] * v[2], c2 = q[0] * v[1] - q[1] * v[0];
    Q.cross2 = c0 * c0 + c1 * c1 + c2 * c2;
  }
  return Q;
}

// Intersections with radius r: returns false if the ray misses.
template <typename R>
__device__ __forceinline__ bool hit_radius(const Quad<R>& Q, R r, R* t0, R* t1) {
  if (Q.A <= R(0)) return false;
  const R disc = Q.A * r * r - Q.cross2;  // = B^2 - A (C2 - r^2), no cancellation
  if (disc < R(0)) return false;
  roots(Q.A, Q.B, Q.C2 - r * r, disc, t0, t1);
  return true;
}

template <typename R>
__device__ bool inside(const DPrim<R>& p, R dR, const R x[3]) {
  R q[3], v[3];
  const R u0[3] = {R(0), R(0), R(1)};
  to_local(p, x, u0, q, v);
  if (p.shape == TP_BOX)
    return fabs(q[0]) <= p.p[0] && fabs(q[1]) <= p.p[1] && fabs(q[2]) <= p.p[2];
  const Radii<R> rr = radii(p, dR);
  if (p.shape == TP_TUBE) {
    const R rho2 = q[0] * q[0] + q[1] * q[1];
    return rho2 >= rr.r0 * rr.r0 && rho2 <= rr.r1 * rr.r1 && fabs(q[2]) <= rr.h;
  }
  const R r2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  return r2 >= rr.r0 * rr.r0 && r2 <= rr.r1 * rr.r1;
}

// Distance to leave p from inside; face id out.
template <typename R>
__device__ R exit_dist(const DPrim<R>& p, R dR, const R x[3], const R u[3], int* face) {
  R q[3], v[3];
  to_local(p, x, u, q, v);
  R best = Tr<R>::inf();
  int bf = -1;
  if (p.shape == TP_BOX) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (v[a] > R(0)) { const R t = (p.p[a] - q[a]) / v[a]; if (t < best) { best = t; bf = 2 * a + 1; } }
      else if (v[a] < R(0)) { const R t = (-p.p[a] - q[a]) / v[a]; if (t < best) { best = t; bf = 2 * a; } }
    }
  } else {
    const bool tube = p.shape == TP_TUBE;
    const Radii<R> rr = radii(p, dR);
    const Quad<R> Q = quad(q, v, tube);
    R t0, t1;
    if (hit_radius(Q, rr.r1, &t0, &t1) && t1 >= R(0) && t1 < best) { best = t1; bf = 0; }
    if (rr.r0 > R(0) && hit_radius(Q, rr.r0, &t0, &t1) && t0 >= R(0) && t0 < best) { best = t0; bf = 1; }
    if (tube) {
      if (v[2] > R(0)) { const R t = (rr.h - q[2]) / v[2]; if (t < best) { best = t; bf = 3; } }
      else if (v[2] < R(0)) { const R t = (-rr.h - q[2]) / v[2]; if (t < best) { best = t; bf = 2; } }
    }
  }
  *face = bf;
  return best < R(0) ? R(0) : best;
}

// Distance to enter p from outside (inf if never); face id out.  Pieces of the
// solid along the ray that end before tmin are ignored: tmin > 0 is used for
// the primitive just left, so that rounding at its surface cannot send the
// neutron straight back in.
template <typename R>
__device__ R entry_dist(const DPrim<R>& p, R dR, const R x[3], const R u[3], int* face, R tmin) {
  R q[3], v[3];
  to_local(p, x, u, q, v);
  const R INF = Tr<R>::inf();
  *face = -1;
  if (p.shape == TP_BOX) {
    R tn = -INF, tf = INF;
    int fn = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (v[a] == R(0)) {
        if (fabs(q[a]) > p.p[a]) return INF;
        continue;
      }
      const R inv = R(1) / v[a];
      R ta = (-p.p[a] - q[a]) * inv, tb = (p.p[a] - q[a]) * inv;
      int fa = 2 * a;
      if (ta > tb) { const R t = ta; ta = tb; tb = t; fa = 2 * a + 1; }
      if (ta > tn) { tn = ta; fn = fa; }
      if (tb < tf) tf = tb;
    }
    if (tn > tf || tf <= tmin) return INF;
    *face = fn;
    return tn > R(0) ? tn : R(0);
  }
  const bool tube = p.shape == TP_TUBE;
  const Radii<R> rr = radii(p, dR);
  const Quad<R> Q = quad(q, v, tube);
  R o0, o1;
  if (Q.A == R(0)) {
    if (Q.C2 > rr.r1 * rr.r1) return INF;
    o0 = -INF; o1 = INF;
  } else if (!hit_radius(Q, rr.r1, &o0, &o1)) {
    return INF;
  }
  R z0 = -INF, z1 = INF;
  int fz0 = -1;
  if (tube) {
    if (v[2] == R(0)) {
      if (fabs(q[2]) > rr.h) return INF;
    } else {
      const R ta = (-rr.h - q[2]) / v[2], tb = (rr.h - q[2]) / v[2];
      if (ta < tb) { z0 = ta; z1 = tb; fz0 = 2; } else { z0 = tb; z1 = ta; fz0 = 3; }
    }
  }
  R s0 = o0, e0 = o1, s1 = INF, e1 = -INF;
  int f0 = 0, f1 = 1;
  if (rr.r0 > R(0)) {
    R i0, i1;
    if (Q.A > R(0) && hit_radius(Q, rr.r0, &i0, &i1)) {
      e0 = i0; s1 = i1; e1 = o1;
    } else if (Q.A == R(0) && Q.C2 < rr.r0 * rr.r0) {
      return INF;
    }
  }
  // first piece
  R a = s0, b = e0;
  int f = f0;
  if (z0 > a) { a = z0; f = fz0; }
  if (z1 < b) b = z1;
  if (a < b && b > tmin) { *face = f; return a > R(0) ? a : R(0); }
  a = s1; b = e1; f = f1;
  if (z0 > a) { a = z0; f = fz0; }
  if (z1 < b) b = z1;
  if (a < b && b > tmin) { *face = f; return a > R(0) ? a : R(0); }
  return INF;
}

template <typename R>
__device__ __forceinline__ bool world_inside(const KParams<R>& kp, const R x[3]) {
  const R d0 = x[0] - kp.world_c[0], d1 = x[1] - kp.world_c[1], d2 = x[2] - kp.world_c[2];
  if (kp.world_shape == TP_BOX)
    return fabs(d0) <= kp.world_p[0] && fabs(d1) <= kp.world_p[1] && fabs(d2) <= kp.world_p[2];
  return d0 * d0 + d1 * d1 + d2 * d2 <= kp.world_p[1] * kp.world_p[1];
}

template <typename R>
__device__ __forceinline__ R world_exit(const KParams<R>& kp, const R x[3], const R u[3]) {
  DPrim<R> w;
  w.shape = kp.world_shape;
  w.axis = 2;
  w.flags = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) { w.c[i] = kp.world_c[i]; w.p[i] = kp.world_p[i]; }
  int f;
  return exit_dist(w, R(0), x, u, &f);
}

// Point location: primitive containing x, -1 for the world region, -2 outside
// the world.
template <typename R>
__device__ __forceinline__ int locate(const KParams<R>& kp, const View<R>& V, R dR, const R x[3]) {
  if (!world_inside(kp, x)) return -2;
  if (kp.use_grid) {
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!(x[a] >= kp.grid_lo[a] && x[a] <= kp.grid_hi[a])) return -1;   // outside every primitive
      c[a] = min(kp.grid_n[a] - 1, max(0, (int)floor((x[a] - kp.grid_lo[a]) * kp.grid_inv[a])));
    }
    const int cell = (c[0] * kp.grid_n[1] + c[1]) * kp.grid_n[2] + c[2];
    for (int k = kp.grid_start[cell]; k < kp.grid_start[cell + 1]; ++k) {
      const int i = kp.grid_items[k];
      if (inside(V.prims[i], dR, x)) return i;
    }
    return -1;
  }
  for (int i = 0; i < kp.nprim; ++i)
    if (inside(V.prims[i], dR, x)) return i;
  return -1;
}

// Location just after leaving primitive `from`: only the primitives touching it
// can contain the point.
template <typename R>
__device__ __forceinline__ int locate_after(const KParams<R>& kp, const View<R>& V, R dR, const R x[3],
                                            int from) {
  if (!world_inside(kp, x)) return -2;
  const DPrim<R>& pf = V.prims[from];
  for (int k = 0; k < pf.nb_cnt; ++k) {
    const int i = V.nb[pf.nb_off + k];
    if (inside(V.prims[i], dR, x)) return i;
  }
  return -1;
}

// Leaving a primitive through a face of its convex hull (every box face, the
// outer surface and caps of a tube, the outer surface of a sphere), a ray can
// never meet that primitive again.
__device__ __forceinline__ bool hull_face(int shape, int face) {
  return shape == TP_BOX || face != 1;
}
// Particle::last packs the primitive just left (bits 0-23, kNoPrim = none),
// a flag to skip it entirely (kLastHull), and the number of consecutive
// boundary steps shorter than a few nudge lengths (bits 24-29): a neutron
// caught between two surfaces that rounding makes overlap (an edge where two
// mirror boxes meet, in FP32) is ended as lost after kMaxStuck of them.
constexpr int kNoPrim = 0x00FFFFFF;
constexpr int kPrimMask = 0x00FFFFFF;
static_assert(TP_MAX_PRIMS < kNoPrim, "primitive indices must fit below kNoPrim");
constexpr int kLastHull = 0x40000000;
constexpr int kStuckShift = 24;
constexpr int kStuckMask = 0x3F << kStuckShift;
constexpr int kMaxStuck = 16;

template <typename R>
__device__ __forceinline__ void normal(const DPrim<R>& p, const R x[3], int face, R n[3]) {
  n[0] = n[1] = n[2] = R(0);
  if (p.shape == TP_BOX) { n[face >> 1] = (face & 1) ? R(1) : R(-1); return; }
  R d[3] = {x[0] - p.c[0], x[1] - p.c[1], x[2] - p.c[2]};
  if (p.shape == TP_TUBE) {
    if (face >= 2) { n[p.axis] = (face == 3) ? R(1) : R(-1); return; }
    d[p.axis] = R(0);
  }
  const R inv = (face == 1 ? R(-1) : R(1)) / d_sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  n[0] = d[0] * inv; n[1] = d[1] * inv; n[2] = d[2] * inv;
}

// Deflection by polar cosine mu and azimuth phi about u.
template <typename R>
__device__ __forceinline__ void rotate(R u[3], R mu, R phi) {
  const R st = d_sqrt(fmax(R(0), R(1) - mu * mu));
  R sp, cp;
  d_sincos(phi, &sp, &cp);
  const R t2 = R(1) - u[2] * u[2];
  R o0, o1, o2;
  if (t2 > R(1e-20)) {
    const R t = d_sqrt(t2);
    const R it = R(1) / t;
    o0 = mu * u[0] + st * (u[0] * u[2] * cp - u[1] * sp) * it;
    o1 = mu * u[1] + st * (u[1] * u[2] * cp + u[0] * sp) * it;
    o2 = mu * u[2] - st * t * cp;
  } else {
    o0 = st * cp;
    o1 = st * sp;
    o2 = (u[2] >= R(0) ? R(1) : R(-1)) * mu;
  }
  u[0] = o0; u[1] = o1; u[2] = o2;
}

template <typename R>
__device__ __forceinline__ R mirror_R(const DMirror<R>& m, R Q) {
  if (Q <= m.Qc) return m.R0;
  const R r = R(0.5) * m.R0 * (R(1) - m.alpha * (Q - m.Qc)) * (R(1) - d_tanh((Q - m.mQc) / m.W));
  return r > R(0) ? r : R(0);
}

// ---------------------------------------------------------------------------
// Scoring: warp-aggregated FP64 atomics
// ---------------------------------------------------------------------------
// The active lanes that score the same bin at once: each lane's group of
// lanes with the same bin index, the next member above it in lane order (-1
// for the last), and the rounds a pointer-jumping sum over the largest group
// takes (ceil log2 of its size; 0 when no two lanes share a bin).
struct AggGroup {
  unsigned am, grp;
  int next, rounds;
};

__device__ __forceinline__ AggGroup agg_group(unsigned long long idx) {
  AggGroup g;
  g.am = __activemask();
  g.grp = __match_any_sync(g.am, idx);
  const int lane = threadIdx.x & 31;
  const unsigned above = g.grp & (0xFFFFFFFEu << lane);
  g.next = above ? __ffs(above) - 1 : -1;
  const unsigned gmax = __reduce_max_sync(g.am, (unsigned)__popc(g.grp));
  g.rounds = gmax > 1u ? 32 - __clz((int)(gmax - 1u)) : 0;
  return g;
}

// Adds v and v2 into bins a[idx], b[idx] (FP64) for every active lane of the
// group G: the group's values are summed in the transport precision by pointer
// jumping (after round k each lane holds its own value plus those of the next
// 2^k - 1 members, so the lowest member ends with the group's sum; the FP64
// pipe is a small fraction of the FP32 one) and its lowest lane adds them
// with one FP64 atomic per array.
template <typename R>
__device__ __forceinline__ void agg_add2(const AggGroup& G, double* a, double* b, unsigned long long idx, R v,
                                         R v2) {
  int nx = G.next;
  for (int k = 0; k < G.rounds; ++k) {
    const int src = nx >= 0 ? nx : (int)(threadIdx.x & 31);
    const R x = __shfl_sync(G.am, v, src);
    const R y = __shfl_sync(G.am, v2, src);
    const int nn = __shfl_sync(G.am, nx, src);
    if (nx >= 0) {
      v += x;
      v2 += y;
      nx = nn;
    }
  }
  if ((int)(threadIdx.x & 31) == __ffs(G.grp) - 1) {
    atomicAdd(a + idx, (double)v);
    atomicAdd(b + idx, (double)v2);
  }
}

template <typename R>
__device__ __forceinline__ int bin1(R x, R lo, R hi, R inv_w, int n) {
  if (!(x >= lo) || !(x < hi)) return -1;
  const int b = (int)floor((x - lo) * inv_w);
  return (b >= 0 && b < n) ? b : (b >= n ? n - 1 : -1);
}

// angle between (x - origin) and the tally axis, accurate at small angles
template <typename R>
__device__ __forceinline__ R tally_angle(const DTally<R>& T, R x0, R x1, R x2) {
  const R v0 = x0 - T.origin[0], v1 = x1 - T.origin[1], v2 = x2 - T.origin[2];
  const R dt = v0 * T.axis[0] + v1 * T.axis[1] + v2 * T.axis[2];
  const R c0 = v1 * T.axis[2] - v2 * T.axis[1], c1 = v2 * T.axis[0] - v0 * T.axis[2],
          c2 = v0 * T.axis[1] - v1 * T.axis[0];
  return d_atan2(d_sqrt(c0 * c0 + c1 * c1 + c2 * c2), dt);
}

template <typename R, int OPT>
__device__ __forceinline__ int tally_bin(const DTally<R>& T, R x0, R x1, R x2, R lam, int nscat, R path) {
  if constexpr (!(OPT & kOptFull)) {
    // lean build: count, angular and PSD scorers only
    if (T.kind == TP_TALLY_COUNT) return 0;
    if (T.kind == TP_TALLY_ANGULAR) return bin1(tally_angle(T, x0, x1, x2), T.lo[0], T.hi[0], T.inv_w[0], T.nb0);
    const int bx = bin1(x0, T.lo[0], T.hi[0], T.inv_w[0], T.nb0);
    const int by = bin1(x1, T.lo[1], T.hi[1], T.inv_w[1], T.nb1);
    return (bx < 0 || by < 0) ? -1 : bx * T.nb1 + by;
  } else {
    switch (T.kind) {
      case TP_TALLY_COUNT: return 0;
      case TP_TALLY_TOF: return bin1(path * lam * R(1.0 / kHoverMn), T.lo[0], T.hi[0], T.inv_w[0], T.nb0);
      case TP_TALLY_ANGULAR: return bin1(tally_angle(T, x0, x1, x2), T.lo[0], T.hi[0], T.inv_w[0], T.nb0);
      case TP_TALLY_MULTISCAT: return bin1((R)nscat, T.lo[0], T.hi[0], T.inv_w[0], T.nb0);
      case TP_TALLY_DQ: {
        // elastic momentum transfer Q = 4 pi sin(theta/2) / lambda (Eq. eQelastic)
        R sh, ch;
        d_sincos(R(0.5) * tally_angle(T, x0, x1, x2), &sh, &ch);
        return bin1(Tr<R>::kFourPi * sh / lam, T.lo[0], T.hi[0], T.inv_w[0], T.nb0);
      }
      case TP_TALLY_PSD: {
        const int bx = bin1(x0, T.lo[0], T.hi[0], T.inv_w[0], T.nb0);
        const int by = bin1(x1, T.lo[1], T.hi[1], T.inv_w[1], T.nb1);
        return (bx < 0 || by < 0) ? -1 : bx * T.nb1 + by;
      }
      default: {
        const int bl = bin1(lam, T.lo[0], T.hi[0], T.inv_w[0], T.nb0);
        const int bx = bin1(x0, T.lo[1], T.hi[1], T.inv_w[1], T.nb1);
        return (bl < 0 || bx < 0) ? -1 : bl * T.nb1 + bx;
      }
    }
  }
}

// Scoring at a particle tracing state: every tally of `mask` (filtered by face
// and scattering number) gets w and w^2 in its bin, and the gradient tallies
// w A_p (a derivative secondary scores w into the radius tally only).
template <typename R, bool GRAD, int OPT>
__device__ __forceinline__ void score_out(const KParams<R>& kp, const DTally<R>* tallies, unsigned mask, int face,
                                       R x0, R x1, R x2, R lam, R w_, R A0, R A1, R A2, R A3, int nscat,
                                       uint32_t inst, bool secondary, R path) {
  const R A[kMaxPar] = {A0, A1, A2, A3};
  while (mask) {
    const int t = __ffs(mask) - 1;
    mask &= mask - 1;
    const DTally<R>& T = tallies[t];
    if (T.face >= 0 && T.face != face) continue;
    if (T.scat >= 0 && T.scat != nscat) continue;
    const int b = tally_bin<R, OPT>(T, x0, x1, x2, lam, nscat, path);
    if (b < 0) continue;
    const unsigned long long idx = (unsigned long long)inst * kp.total_bins + T.offset + b;
    const R w = w_;
    const unsigned long long stride = (unsigned long long)kp.n_inst * kp.total_bins;
    // one grouping of the lanes on this path serves every array of the bin
    if (!secondary) {
      const AggGroup G = agg_group(idx);
      agg_add2(G, kp.sum, kp.sumsq, idx, w, w * w);
      if (GRAD) {
#pragma unroll
        for (int p = 0; p < kMaxPar; ++p) {
          if (p >= kp.npar) break;
          const R g = w * A[p];
          agg_add2(G, kp.J, kp.J2, p * stride + idx, g, g * g);
        }
      }
    } else if (kp.radius_par >= 0) {   // a radius-derivative secondary
      const AggGroup G = agg_group(idx);
      agg_add2(G, kp.J, kp.J2, kp.radius_par * stride + idx, w, w * w);
    }
  }
}

template <typename R, bool GRAD, int OPT>
__device__ __forceinline__ void score(const KParams<R>& kp, const View<R>& V, const Particle<R>& P, unsigned mask,
                                      int face) {
  score_out<R, GRAD, OPT>(kp, V.tallies, mask, face, P.x[0], P.x[1], P.x[2], P.lam, P.w, P.A[0], P.A[1], P.A[2],
                     P.A[3], P.nscat, P.inst, P.sub0 != 0u, P.s);
}

// ---------------------------------------------------------------------------
// Source (event 0), §3.2
// ---------------------------------------------------------------------------
template <typename R, int OPT>
__device__ bool source(const KParams<R>& kp, const View<R>& V, Particle<R>& P, R dR, int* end) {
  const uint4 a = philox(make_uint4(0u, 0u, P.hid, P.inst), kp.key0, kp.key1);
  P.x[0] = kp.src_c[0]; P.x[1] = kp.src_c[1]; P.x[2] = kp.src_c[2];
  if (kp.src_kind != TP_SRC_PENCIL) {
    P.x[0] += kp.src_half[0] * (R(2) * Tr<R>::u01(a.x) - R(1));
    P.x[1] += kp.src_half[1] * (R(2) * Tr<R>::u01(a.y) - R(1));
  }
  if constexpr (OPT & kOptFull) {
    const bool need_b = kp.src_kind == TP_SRC_MODERATOR || kp.src_kT > R(0) || kp.src_div[0] > R(0) ||
                        kp.src_div[1] > R(0);
    uint4 b = make_uint4(0u, 0u, 0u, 0u);
    if (need_b) b = philox(make_uint4(0u, 1u, P.hid, P.inst), kp.key0, kp.key1);
    if (kp.src_kT > R(0)) {
      // Maxwell-Boltzmann energies sqrt(E) exp(-E/kT): E/kT ~ Gamma(3/2) = an
      // exponential variate plus half a squared normal one (Box-Muller)
      R sc, cc;
      d_sincos(R(0.5) * Tr<R>::kPi * Tr<R>::u01(b.w), &sc, &cc);
      const R e = kp.src_kT * (-d_log(Tr<R>::u01(a.z)) - d_log(Tr<R>::u01(a.w)) * cc * cc);
      P.lam = d_sqrt(R(kH2over2mn) / e);
    } else {
      P.lam = kp.src_lam_hi > kp.src_lam_lo ? kp.src_lam_lo + (kp.src_lam_hi - kp.src_lam_lo) * Tr<R>::u01(a.z)
                                            : kp.src_lam_lo;
    }
    if (kp.src_kind == TP_SRC_MODERATOR) {
      // towards a point uniform on the slit
      const R d0 = kp.src_c[0] + kp.src_slit_half[0] * (R(2) * Tr<R>::u01(b.y) - R(1)) - P.x[0];
      const R d1 = kp.src_c[1] + kp.src_slit_half[1] * (R(2) * Tr<R>::u01(b.z) - R(1)) - P.x[1];
      const R d2 = kp.src_slit_z - P.x[2];
      const R inv = R(1) / d_sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      P.u[0] = d0 * inv; P.u[1] = d1 * inv; P.u[2] = d2 * inv;
    } else if (kp.src_div[0] > R(0) || kp.src_div[1] > R(0)) {
      const R tx = d_tan(kp.src_div[0] * (R(2) * Tr<R>::u01(a.w) - R(1)));
      const R ty = d_tan(kp.src_div[1] * (R(2) * Tr<R>::u01(b.x) - R(1)));
      const R inv = R(1) / d_sqrt(tx * tx + ty * ty + R(1));
      P.u[0] = tx * inv; P.u[1] = ty * inv; P.u[2] = inv;
    } else {
      P.u[0] = R(0); P.u[1] = R(0); P.u[2] = R(1);
    }
  } else {
    // lean build: uniform wavelength band, direction +z
    P.lam = kp.src_lam_hi > kp.src_lam_lo ? kp.src_lam_lo + (kp.src_lam_hi - kp.src_lam_lo) * Tr<R>::u01(a.z)
                                          : kp.src_lam_lo;
    P.u[0] = R(0); P.u[1] = R(0); P.u[2] = R(1);
  }
  P.w = R(1);
#pragma unroll
  for (int i = 0; i < kMaxPar; ++i) P.A[i] = R(0);
  P.nscat = 0; P.k = 0; P.sub0 = 0; P.nsec = 0; P.s = R(0); P.last = kNoPrim;
  if ((OPT & kOptFull) && kp.src_aperture && (fabs(P.x[0] - kp.src_c[0]) > kp.src_ap[0] ||
                                              fabs(P.x[1] - kp.src_c[1]) > kp.src_ap[1])) {
    P.w = R(0);
    *end = END_APERTURE;
    return false;
  }
  P.vol = kp.src_free ? -1 : locate(kp, V, dR, P.x);
  if (P.vol == -2) { *end = END_LOST; return false; }
  if (P.vol >= 0 && V.prims[P.vol].role != TP_ROLE_BULK) { *end = END_BLACK; return false; }
  return true;
}

template <typename R>
__device__ __forceinline__ R nudge_len(const R x[3]) {
  return Tr<R>::nudge(fmax(fabs(x[0]), fmax(fabs(x[1]), fabs(x[2]))));
}

// Draw the new direction of a scatter by process `proc` of material `mat`.
template <typename R>
__device__ __forceinline__ void scatter_dir(const View<R>& V, int mat, int proc, R lam, R u[3], R xmu,
                                            R xphi, R xline) {
  if (proc == TP_PROC_INC) {
    const R mu = R(2) * xmu - R(1);
    const R st = d_sqrt(fmax(R(0), R(1) - mu * mu));
    R sp, cp;
    d_sincos(Tr<R>::kTwoPi * xphi, &sp, &cp);
    u[0] = st * cp; u[1] = st * sp; u[2] = mu;
  } else {
    const DMat<R>& m = V.mats[mat];
    const int n = active_lines(V, m, lam);
    const R* cum = V.line_cum + m.cum_off;
    const R target = xline * cum[n];
    // smallest i < n with target < cum[i+1]
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (target < cum[mid + 1]) hi = mid; else lo = mid + 1;
    }
    const R sb = lam / (R(2) * V.line_d[m.line_off + lo]);
    rotate(u, R(1) - R(2) * sb * sb, Tr<R>::kTwoPi * xphi);
  }
}

// Radius derivative at the crossing of a lateral surface that moves with the
// radius parameter.  The layer of thickness dR just outside the surface turns
// from the outer material into the inner one; a path crossing it with |n.u|
// spends dR/|n.u| in it.  The continuing path's score function gains
// -(Sigma_t,in - Sigma_t,out)/|n.u|; the collisions that now happen in the layer
// are added as one derivative secondary starting at the crossing, with weight
// w sign(c) C/|n.u|, scattered by a term picked with probability |c|/C among
// c = +Sigma_j,in, -Sigma_j,out over the scattering processes j.  Returns true
// if a secondary was created in *S.
template <typename R>
__device__ __forceinline__ bool radius_crossing(const KParams<R>& kp, const View<R>& V, Particle<R>& P, const R (&ip)[kMaxPar],
                                R dR, int mi, int mo, const R n[3], Particle<R>* S,
                                unsigned* cnt) {
  const R cosn = fabs(P.u[0] * n[0] + P.u[1] * n[1] + P.u[2] * n[2]);
  if (cosn < R(1e-12)) return false;
  R si[TP_NPROC] = {R(0), R(0), R(0)}, so[TP_NPROC] = {R(0), R(0), R(0)};
  if (mi >= 0) sigma(V, mi, ip, P.lam, si);
  if (mo >= 0) sigma(V, mo, ip, P.lam, so);
  add_at(P.A, kp.radius_par, -((si[0] + si[1] + si[2]) - (so[0] + so[1] + so[2])) / cosn);
  const R term[4] = {si[TP_PROC_INC], si[TP_PROC_BRAGG], -so[TP_PROC_INC], -so[TP_PROC_BRAGG]};
  const R C = fabs(term[0]) + fabs(term[1]) + fabs(term[2]) + fabs(term[3]);
  if (!(C > R(0))) return false;
  const uint4 r = philox(make_uint4(P.k, 2u, P.hid, P.inst), kp.key0, kp.key1);
  const R pickv = Tr<R>::u01(r.x) * C;
  int pick = 3;
  R acc = R(0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    acc += fabs(term[i]);
    if (pick == 3 && i < 3 && pickv < acc) pick = i;
  }
  // guard against rounding at the top end: the last non-zero term at or below pick
  R tp = R(0);
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    if (i <= pick && tp == R(0) && term[i] != R(0)) { tp = term[i]; pick = i; }
  }
  const int mat = pick < 2 ? mi : mo;
  const int proc = (pick & 1) ? TP_PROC_BRAGG : TP_PROC_INC;
  *S = P;
  S->w = P.w * (tp > R(0) ? R(1) : R(-1)) * C / cosn;
  S->nscat = P.nscat + 1;
  S->sub0 = 4u + 2u * P.nsec;
  S->k = 0;
  S->last = kNoPrim;
  P.nsec++;
  scatter_dir(V, mat, proc, P.lam, S->u, Tr<R>::u01(r.y), Tr<R>::u01(r.z), Tr<R>::u01(r.w));
  cnt[C_SEC]++;
  const R e = nudge_len(S->x);
  R xn[3] = {S->x[0] + e * S->u[0], S->x[1] + e * S->u[1], S->x[2] + e * S->u[2]};
  const int v = locate(kp, V, dR, xn);
  if (v < -1) return false;
  S->x[0] = xn[0]; S->x[1] = xn[1]; S->x[2] = xn[2];
  S->vol = v;
  if (v >= 0 && V.prims[v].role != TP_ROLE_BULK) return false;
  return true;
}

// ---------------------------------------------------------------------------
// One event of one neutron, in three parts: advance (cross sections, biased
// flight, next boundary, move and weight), then either cross (relocation at a
// boundary) or collide (interaction).  Each returns -1 while the neutron
// lives, else its end code; advance returns kOutCross / kOutColl instead.
// ---------------------------------------------------------------------------
constexpr int kOutCross = 100, kOutColl = 101;

// Disk chopper in ray-tracing mode (Eq. eRayTracing, §3.5): epsilon = 1 if the
// neutron entering the disk's tube is outside the black centre and inside an
// opening window at its time of flight, else 0.  Angles are counted in window
// periods so that the comparison stays exact in FP32 over many turns.
template <typename R>
__device__ __forceinline__ bool chopper_open(const View<R>& V, const DPrim<R>& pt, const Particle<R>& P) {
  const DChopper<R>& ch = V.choppers[pt.flags >> kChopperShift];
  // in-plane axes (axis+1, axis+2) mod 3, as in the tube's local frame
  const R d0 = P.x[0] - pt.c[0], d1 = P.x[1] - pt.c[1], d2 = P.x[2] - pt.c[2];
  const R q1 = pt.axis == 0 ? d1 : (pt.axis == 1 ? d2 : d0);
  const R q2 = pt.axis == 0 ? d2 : (pt.axis == 1 ? d0 : d1);
  if (q1 * q1 + q2 * q2 < ch.r_black2) return false;
  const R t = P.s * P.lam * R(1.0 / kHoverMn);
  const R psi = d_atan2(q2, q1) * ch.n_over_2pi - ch.nf * t - ch.n_phase;
  return fabs(psi - rint(psi)) <= ch.half;
}

// Entry test of primitive i from the world region, with the bounding-sphere
// early-out and the rules for the primitive just left; keeps the nearest.
template <typename R>
__device__ __forceinline__ void entry_test(const View<R>& V, R dR, const R x[3], const R u[3], int i, int last,
                                           bool last_hull, R tmin, R* db, int* target, int* face) {
  const DPrim<R>& pi = V.prims[i];
  if (i == last && last_hull) return;
  // bounding sphere: skip if the ray misses it or moves away from outside it
  const R q0 = x[0] - pi.c[0], q1 = x[1] - pi.c[1], q2 = x[2] - pi.c[2];
  const R qu = q0 * u[0] + q1 * u[1] + q2 * u[2];
  const R qq = q0 * q0 + q1 * q1 + q2 * q2;
  const R rb2 = pi.bound_r * pi.bound_r;
  if (qq > rb2 && (qu >= R(0) || qq - qu * qu > rb2)) return;
  int f;
  const R t = entry_dist(pi, dR, x, u, &f, i == last ? tmin : R(0));
  if (t < *db) { *db = t; *target = i; *face = f; }
}

// World-region search through the uniform grid: a 3-D DDA over the cells the
// ray crosses, nearest first, stopping once the best hit lies inside the cells
// already visited.  Out of line so that scenes without a grid keep a smaller
// hot loop.
template <typename R>
__device__ __forceinline__ void grid_search(const KParams<R>& kp, const View<R>& V, R dR, R x0, R x1, R x2, R u0,
                                         R u1, R u2, int last, bool last_hull, R tmin, R* db_io, int* target_io,
                                         int* face_io) {
  const R x[3] = {x0, x1, x2}, u[3] = {u0, u1, u2};
  R db = *db_io;
  int target = *target_io, face = *face_io;
  R t0 = R(0), t1 = db;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (u[a] != R(0)) {
      const R inv = R(1) / u[a];
      R ta = (kp.grid_lo[a] - x[a]) * inv, tb = (kp.grid_hi[a] - x[a]) * inv;
      if (ta > tb) { const R t = ta; ta = tb; tb = t; }
      t0 = fmax(t0, ta);
      t1 = fmin(t1, tb);
    } else if (!(x[a] >= kp.grid_lo[a] && x[a] <= kp.grid_hi[a])) {
      t1 = R(-1);
    }
  }
  if (t0 <= t1) {
    int c[3], stp[3];
    R tnext[3], tdel[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R pa = x[a] + t0 * u[a];
      c[a] = min(kp.grid_n[a] - 1, max(0, (int)floor((pa - kp.grid_lo[a]) * kp.grid_inv[a])));
      if (u[a] > R(0)) {
        stp[a] = 1;
        tnext[a] = (kp.grid_lo[a] + (c[a] + 1) * kp.grid_cell[a] - x[a]) / u[a];
        tdel[a] = kp.grid_cell[a] / u[a];
      } else if (u[a] < R(0)) {
        stp[a] = -1;
        tnext[a] = (kp.grid_lo[a] + c[a] * kp.grid_cell[a] - x[a]) / u[a];
        tdel[a] = -kp.grid_cell[a] / u[a];
      } else {
        stp[a] = 0;
        tnext[a] = Tr<R>::inf();
        tdel[a] = Tr<R>::inf();
      }
    }
    const int maxsteps = kp.grid_n[0] + kp.grid_n[1] + kp.grid_n[2] + 3;
    for (int it = 0; it < maxsteps; ++it) {
      const int cell = (c[0] * kp.grid_n[1] + c[1]) * kp.grid_n[2] + c[2];
      const int k1 = kp.grid_start[cell + 1];
      for (int k = kp.grid_start[cell]; k < k1; ++k)
        entry_test(V, dR, x, u, kp.grid_items[k], last, last_hull, tmin, &db, &target, &face);
      const int a = (tnext[0] <= tnext[1]) ? (tnext[0] <= tnext[2] ? 0 : 2) : (tnext[1] <= tnext[2] ? 1 : 2);
      const R texit = tnext[a];
      if (db <= texit || texit >= t1) break;
      c[a] += stp[a];
      if (c[a] < 0 || c[a] >= kp.grid_n[a]) break;
      tnext[a] += tdel[a];
    }
  }
  *db_io = db;
  *target_io = target;
  *face_io = face;
}

template <typename R>
struct Adv {
  uint4 r0;           // random numbers of this event (sub-stream 0)
  R sig[TP_NPROC];    // true cross sections at the event (collisions only)
  R sig_g;
  int face, target;   // crossing: face id; target primitive, -3 = leaving the world
};

// WHERE: kAny, or kInPrim / kInWorld when the caller knows where the neutron
// is (the regrouping kernels), which drops the other branch from the code.
constexpr int kAny = 0, kInPrim = 1, kInWorld = 2;

template <typename R, bool GRAD, int OPT, int WHERE = kAny>
__device__ int advance(const KParams<R>& kp, const View<R>& V, Particle<R>& P, const R (&ip)[kMaxPar], R dR,
                       unsigned* cnt, Adv<R>& a) {
  const R INF = Tr<R>::inf();
  P.k += 1;
  if ((int)P.k > kp.event_cap) { cnt[C_TRUNC]++; return END_TRUNCATED; }
  cnt[C_EVENTS]++;
  const int mat = (WHERE == kInWorld) ? -1 : (P.vol >= 0 ? V.prims[P.vol].material : -1);
  R* sig = a.sig;
  sig[0] = sig[1] = sig[2] = R(0);
  R sig_t = R(0), sig_g = R(0);
  if (mat >= 0) {
    sigma(V, mat, ip, P.lam, sig);
    const DMat<R>& m = V.mats[mat];
    sig_t = sig[0] + sig[1] + sig[2];
    sig_g = m.g[0] * sig[0] + m.g[1] * sig[1] + m.g[2] * sig[2];
  }
  a.sig_g = sig_g;
  // Random numbers only where a flight is sampled: with Sigma_g = 0 (vacuum,
  // or every bias factor 0) the step is infinite and the event draws nothing.
  // The counter-based stream keeps every other event's numbers unchanged.
  R l = INF;
  if (sig_g > R(0)) {
    a.r0 = philox(make_uint4(P.k, P.sub0, P.hid, P.inst), kp.key0, kp.key1);
    l = Tr<R>::neg_log_u01(a.r0.x) / sig_g;
  }
  // next boundary
  R db;
  int target = -3, face = -1;
  if (WHERE == kInPrim || (WHERE == kAny && P.vol >= 0)) {
    db = exit_dist(V.prims[P.vol], dR, P.x, P.u, &face);
  } else {
    db = world_exit(kp, P.x, P.u);
    const R tmin = R(2) * nudge_len(P.x);
    const int last = P.last & kPrimMask;
    const bool last_hull = (P.last & kLastHull) != 0;
    if constexpr ((OPT & kOptGrid) != 0) {
      grid_search(kp, V, dR, P.x[0], P.x[1], P.x[2], P.u[0], P.u[1], P.u[2], last, last_hull, tmin, &db,
                  &target, &face);
    } else {
      for (int i = 0; i < kp.nprim; ++i)
        entry_test(V, dR, P.x, P.u, i, last, last_hull, tmin, &db, &target, &face);
    }
  }
  a.face = face;
  a.target = target;
  const bool crossing = l >= db;
  const R x = crossing ? db : l;
  if (!(x < INF)) { cnt[C_LOST]++; return END_LOST; }
  {
    int stuck = (P.last & kStuckMask) >> kStuckShift;
    stuck = (crossing && db < R(4) * nudge_len(P.x)) ? stuck + 1 : 0;
    if (stuck > kMaxStuck) { cnt[C_LOST]++; return END_LOST; }
    P.last = (P.last & ~kStuckMask) | (stuck << kStuckShift);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) P.x[i] += x * P.u[i];
  P.s += x;
  if (sig_g != sig_t) P.w *= d_exp((sig_g - sig_t) * x);
  if (GRAD && mat >= 0 && P.sub0 == 0u) {
    const DMat<R>& m = V.mats[mat];
#pragma unroll
    for (int p = 0; p < kMaxPar; ++p) {
      if (p >= kp.npar) break;
      if (kp.param_kind[p] == TP_PAR_DENSITY && m.density_par == p) P.A[p] -= sig_t * x;
      if (kp.param_kind[p] == TP_PAR_SCALE && m.scale_par == p) P.A[p] -= sig[TP_PROC_BRAGG] * x;
    }
  }
  return crossing ? kOutCross : kOutColl;
}

// Relocation at the boundary reached by advance (face / target of `a`).
// spawn: set when a radius-derivative secondary was created into *S.
template <typename R, bool GRAD, int OPT, int WHERE = kAny>
__device__ int cross(const KParams<R>& kp, const View<R>& V, Particle<R>& P, const R (&ip)[kMaxPar], R dR,
                     unsigned* cnt, int face, int target, Particle<R>* S, bool* spawn) {
  cnt[C_CROSS]++;
  if (WHERE == kInPrim || (WHERE == kAny && P.vol >= 0)) {
    // leave the current primitive: EXIT scorers, then relocate
    const int from = P.vol;
    const DPrim<R>& pf = V.prims[from];
    if (pf.exit_mask) score<R, GRAD, OPT>(kp, V, P, (unsigned)pf.exit_mask, face);
    const R e = nudge_len(P.x);
    R xn[3] = {P.x[0] + e * P.u[0], P.x[1] + e * P.u[1], P.x[2] + e * P.u[2]};
    const int v = locate_after(kp, V, dR, xn, from);
    P.last = (P.last & kStuckMask) | from | (hull_face(pf.shape, face) ? kLastHull : 0);
    if (GRAD && !(OPT & kOptNoSec) && kp.radius_par >= 0 && P.sub0 == 0u && pf.shape != TP_BOX &&
        ((face == 0 && (pf.flags & F_BIND_RMAX)) || (face == 1 && (pf.flags & F_BIND_RMIN)))) {
      R n[3];
      normal(pf, P.x, face, n);
      const int mnext = v >= 0 ? V.prims[v].material : -1;
      const int mi = face == 0 ? pf.material : mnext;
      const int mo = face == 0 ? mnext : pf.material;
      *spawn = radius_crossing<R>(kp, V, P, ip, dR, mi, mo, n, S, cnt);
    }
    P.x[0] = xn[0]; P.x[1] = xn[1]; P.x[2] = xn[2];
    if (v == -2) {
      if (kp.world_exit_mask) score<R, GRAD, OPT>(kp, V, P, (unsigned)kp.world_exit_mask, -1);
      return END_ESCAPED;
    }
    P.vol = v;
    if (v >= 0) {
      const DPrim<R>& pt = V.prims[v];
      if (pt.entry_mask) score<R, GRAD, OPT>(kp, V, P, (unsigned)pt.entry_mask, -1);
      if (pt.role == TP_ROLE_DETECTOR) return END_DETECTED;
      if (pt.role == TP_ROLE_BLACK) return END_BLACK;
      if ((OPT & kOptFull) && (pt.flags & F_CHOPPER) && !chopper_open(V, pt, P)) return END_BLACK;
    }
    return -1;
  }
  if (target == -3) {
    if (kp.world_exit_mask) score<R, GRAD, OPT>(kp, V, P, (unsigned)kp.world_exit_mask, -1);
    return END_ESCAPED;
  }
  const DPrim<R>& pt = V.prims[target];
  if ((OPT & kOptFull) && pt.mirror >= 0) {
    // supermirror: weight R(Q), specular reflection (Eq. eMirrowNewDir)
    R n[3];
    normal(pt, P.x, face, n);
    const R un = P.u[0] * n[0] + P.u[1] * n[1] + P.u[2] * n[2];
    const R Q = Tr<R>::kFourPi * fabs(un) / P.lam;
    const R Rf = mirror_R(V.mirrors[pt.mirror], Q);
    cnt[C_MIRROR]++;
    P.w *= Rf;
    if (!(Rf > R(0))) return END_MIRROR;
#pragma unroll
    for (int i = 0; i < 3; ++i) P.u[i] -= R(2) * n[i] * un;
    P.last = (P.last & kStuckMask) | target | (hull_face(pt.shape, face) ? kLastHull : 0);
    const R e = nudge_len(P.x);
#pragma unroll
    for (int i = 0; i < 3; ++i) P.x[i] += e * P.u[i];
    return -1;
  }
  if (GRAD && !(OPT & kOptNoSec) && kp.radius_par >= 0 && P.sub0 == 0u && pt.shape != TP_BOX &&
      ((face == 0 && (pt.flags & F_BIND_RMAX)) || (face == 1 && (pt.flags & F_BIND_RMIN)))) {
    R n[3];
    normal(pt, P.x, face, n);
    const int mi = face == 0 ? pt.material : -1;
    const int mo = face == 0 ? -1 : pt.material;
    *spawn = radius_crossing<R>(kp, V, P, ip, dR, mi, mo, n, S, cnt);
  }
  const R e = nudge_len(P.x);
#pragma unroll
  for (int i = 0; i < 3; ++i) P.x[i] += e * P.u[i];
  P.vol = target;
  P.last = (P.last & kStuckMask) | kNoPrim;
  if (pt.entry_mask) score<R, GRAD, OPT>(kp, V, P, (unsigned)pt.entry_mask, face);
  if (pt.role == TP_ROLE_DETECTOR) return END_DETECTED;
  if (pt.role == TP_ROLE_BLACK) return END_BLACK;
  if ((OPT & kOptFull) && (pt.flags & F_CHOPPER) && !chopper_open(V, pt, P)) return END_BLACK;
  return -1;
}

// Interaction at the point reached by advance: process j with probability
// g_j Sigma_j / Sigma_g, weight / g_j, then absorption or a new direction.
template <typename R, bool GRAD>
__device__ int collide(const KParams<R>& kp, const View<R>& V, Particle<R>& P, unsigned* cnt,
                       const uint4 r0, const R sig[TP_NPROC], R sig_g) {
  cnt[C_COLL]++;
  const int mat = V.prims[P.vol].material;
  if (kp.records && P.sub0 == 0u && P.nscat == 0 && P.inst == 0 && P.hid - kp.inst_first[0] < kp.n_records) {
    tp_record* rc = kp.records + (P.hid - kp.inst_first[0]);
    rc->first_collision[0] = (double)P.x[0];
    rc->first_collision[1] = (double)P.x[1];
    rc->first_collision[2] = (double)P.x[2];
  }
  const DMat<R>& m = V.mats[mat];
  const R xi1 = Tr<R>::u01(r0.y) * sig_g;
  int j;
  const R c0 = m.g[0] * sig[0], c1 = c0 + m.g[1] * sig[1];
  if (xi1 < c0) j = 0;
  else if (xi1 < c1) j = 1;
  else if (m.g[2] * sig[2] > R(0)) j = 2;
  else j = (m.g[1] * sig[1] > R(0)) ? 1 : 0;
  P.w /= m.g[j];
  if (GRAD && P.sub0 == 0u) {
#pragma unroll
    for (int p = 0; p < kMaxPar; ++p) {
      if (p >= kp.npar) break;
      if (kp.param_kind[p] == TP_PAR_DENSITY && m.density_par == p) P.A[p] += R(1);
      if (kp.param_kind[p] == TP_PAR_SCALE && m.scale_par == p && j == TP_PROC_BRAGG) P.A[p] += R(1);
    }
  }
  if (j == TP_PROC_ABS) return END_ABSORBED;
  R xline = R(0);
  if (j == TP_PROC_BRAGG) {
    const uint4 r1 = philox(make_uint4(P.k, P.sub0 + 1u, P.hid, P.inst), kp.key0, kp.key1);
    xline = Tr<R>::u01(r1.x);
  }
  scatter_dir(V, mat, j, P.lam, P.u, Tr<R>::u01(r0.z), Tr<R>::u01(r0.w), xline);
  if (kp.records && P.sub0 == 0u && P.nscat == 0 && P.inst == 0 && P.hid - kp.inst_first[0] < kp.n_records) {
    tp_record* rc = kp.records + (P.hid - kp.inst_first[0]);
    rc->dir_after_first[0] = (double)P.u[0];
    rc->dir_after_first[1] = (double)P.u[1];
    rc->dir_after_first[2] = (double)P.u[2];
  }
  P.nscat++;
  return -1;
}

// Collision after a separate advance: the event's random numbers and cross
// sections are recomputed from the neutron's state (event k is unchanged).
template <typename R, bool GRAD>
__device__ int collide_again(const KParams<R>& kp, const View<R>& V, Particle<R>& P, const R (&ip)[kMaxPar],
                             unsigned* cnt) {
  const uint4 r0 = philox(make_uint4(P.k, P.sub0, P.hid, P.inst), kp.key0, kp.key1);
  R sig[TP_NPROC];
  const int mat = V.prims[P.vol].material;
  sigma(V, mat, ip, P.lam, sig);
  const DMat<R>& m = V.mats[mat];
  const R sig_g = m.g[0] * sig[0] + m.g[1] * sig[1] + m.g[2] * sig[2];
  return collide<R, GRAD>(kp, V, P, cnt, r0, sig, sig_g);
}

// One whole event (history-based kernel).
template <typename R, bool GRAD, int OPT>
__device__ int step(const KParams<R>& kp, const View<R>& V, Particle<R>& P, const R (&ip)[kMaxPar], R dR,
                    unsigned* cnt, Particle<R>* S, bool* spawn) {
  Adv<R> a;
  const int r = advance<R, GRAD, OPT>(kp, V, P, ip, dR, cnt, a);
  if (r == kOutCross) return cross<R, GRAD, OPT>(kp, V, P, ip, dR, cnt, a.face, a.target, S, spawn);
  if (r == kOutColl) return collide<R, GRAD>(kp, V, P, cnt, a.r0, a.sig, a.sig_g);
  return r;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copy of the scene tables into shared memory
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Longest wait for the table copy: it takes microseconds, so a wait this long
// means the copy never arrives.
constexpr unsigned long long kStageWaitNs = 500ull * 1000ull * 1000ull;

// Waits for phase 0 of the mbarrier, bounded in time and in tries; false if
// it gave up.
__device__ __forceinline__ bool wait_phase0(uint64_t* bar) {
  uint32_t done = 0;
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 22) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar))
        : "memory");
    if (!done && global_ns() - t0 > kStageWaitNs) break;
  }
  return done != 0;
}

// Copies `bytes` of scene tables into shared memory with one bulk asynchronous
// copy completing on an mbarrier.  Returns false if the bounded wait gave up
// (the caller records TP_ERR_TIMEOUT).  skip_copy (test hook) arms the barrier
// without issuing the copy, so that the wait runs out with nothing in flight.
__device__ bool stage_tables(uint8_t* dst, const uint8_t* src, uint32_t bytes, uint64_t* bar, bool skip_copy) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !skip_copy) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
  }
  bool ok = wait_phase0(bar);
  // a copy that is late is still in flight: let it land (again bounded) before
  // the block gives up and exits
  if (!ok && !skip_copy) wait_phase0(bar);
  return __syncthreads_and(ok) != 0;
}

// Host-requested stop (tp_abort).  The flag lives in mapped host memory,
// whose reads take microseconds, so a thread reads it at its first claim of
// new histories and then at every kAbortPollEvery-th one; returns true (and
// records TP_ERR_ABORTED unless an earlier error is recorded) once it is set.
constexpr unsigned kAbortPollEvery = 32;

template <typename R>
__device__ __forceinline__ bool aborted(const KParams<R>& kp, unsigned& polls) {
  if (!kp.abort_flag || (polls++ % kAbortPollEvery) != 0 || *kp.abort_flag == 0) return false;
  atomicCAS(kp.status, 0, (int)TP_ERR_ABORTED);
  return true;
}

// ---------------------------------------------------------------------------
// The persistent transport kernel
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void finish(const KParams<R>& kp, const Particle<R>& P, int end) {
  if (kp.records && P.sub0 == 0u && P.inst == 0 && P.hid - kp.inst_first[0] < kp.n_records) {
    tp_record* rc = kp.records + (P.hid - kp.inst_first[0]);
    rc->final_pos[0] = (double)P.x[0];
    rc->final_pos[1] = (double)P.x[1];
    rc->final_pos[2] = (double)P.x[2];
    rc->w_final = (double)P.w;
    for (int i = 0; i < kMaxPar; ++i) rc->A_final[i] = (double)P.A[i];
    rc->nscat = P.nscat;
    rc->nevents = (int)P.k;
    rc->end = end;
  }
}

// A queued radius-derivative secondary (second pass of gradient runs): the
// state it starts from.  A secondary carries no score-function accumulators
// (it scores its weight into the radius tallies only), makes no secondaries,
// and starts at event 0 next to no primitive, so 14 words hold it.
template <typename R>
struct SecRec {
  R x[3], u[3], lam, w, s;
  int vol, nscat;
  uint32_t hid, inst, sub0;
};

template <typename R>
__device__ __forceinline__ void sec_write(SecRec<R>* q, const Particle<R>& S) {
  SecRec<R> r;
#pragma unroll
  for (int i = 0; i < 3; ++i) { r.x[i] = S.x[i]; r.u[i] = S.u[i]; }
  r.lam = S.lam; r.w = S.w; r.s = S.s;
  r.vol = S.vol; r.nscat = S.nscat; r.hid = S.hid; r.inst = S.inst; r.sub0 = S.sub0;
  *q = r;
}

template <typename R>
__device__ __forceinline__ Particle<R> sec_read(const SecRec<R>* q) {
  const SecRec<R> r = *q;
  Particle<R> P;
#pragma unroll
  for (int i = 0; i < 3; ++i) { P.x[i] = r.x[i]; P.u[i] = r.u[i]; }
  P.lam = r.lam; P.w = r.w; P.s = r.s;
#pragma unroll
  for (int i = 0; i < kMaxPar; ++i) P.A[i] = R(0);
  P.vol = r.vol; P.nscat = r.nscat; P.hid = r.hid; P.inst = r.inst; P.sub0 = r.sub0;
  P.k = 0; P.nsec = 0; P.last = kNoPrim;
  return P;
}

// Histories (or queued secondaries) a launch works through.
template <typename R>
__device__ __forceinline__ unsigned long long work_total(const KParams<R>& kp) {
  if (kp.sec_mode != 2) return kp.total;
  const unsigned long long n = *kp.sec_count;   // written by the previous launch on the stream
  return n < kp.sec_cap ? n : kp.sec_cap;
}

// Appends a radius-derivative secondary to the queue of the second pass;
// false if the queue is full (the caller then transports it in place).
// One atomic per record: the lanes that push are in divergent code, where no
// warp-wide aggregation is safe.
template <typename R>
__device__ __forceinline__ bool sec_push(const KParams<R>& kp, const Particle<R>& S) {
  if (kp.sec_mode != 1) return false;
  const unsigned long long i = atomicAdd(kp.sec_count, 1ull);
  if (i >= kp.sec_cap) return false;
  sec_write(reinterpret_cast<SecRec<R>*>(kp.sec_buf) + i, S);
  return true;
}

template <typename R, bool GRAD, int OPT, int MINB>
__global__ void __launch_bounds__(256, MINB) k_transport(const __grid_constant__ KParams<R> kp) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bar;
  const uint8_t* base = kp.blob;
  if (kp.stage_blob) {
    if (!stage_tables(smem, kp.blob, kp.blob_bytes, &bar, (kp.test_flags & TP_TEST_SKIP_TABLE_COPY) != 0)) {
      if (threadIdx.x == 0) atomicCAS(kp.status, 0, (int)TP_ERR_TIMEOUT);
      return;
    }
    base = smem;
  }
  View<R> V;
  V.prims = reinterpret_cast<const DPrim<R>*>(base + kp.off_prims);
  V.mats = reinterpret_cast<const DMat<R>*>(base + kp.off_mats);
  V.mirrors = reinterpret_cast<const DMirror<R>*>(base + kp.off_mirrors);
  V.choppers = reinterpret_cast<const DChopper<R>*>(base + kp.off_choppers);
  V.tallies = reinterpret_cast<const DTally<R>*>(base + kp.off_tallies);
  V.line_d = reinterpret_cast<const R*>(base + kp.off_line_d);
  V.line_cum = reinterpret_cast<const R*>(base + kp.off_line_cum);
  V.nb = reinterpret_cast<const int*>(base + kp.off_nb);

  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned cnt[kNumCounters];   // per-thread counts: 32 bits suffice (widened below)
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) cnt[i] = 0;
  unsigned polls = 0;   // claims made by this thread (abort polling)

  Particle<R> P, park, S;
  R ip[kMaxPar];
  R dR = R(0);
  bool alive = false, done = false, parked = false;
  const unsigned long long total = work_total(kp);
  unsigned long long chunk_next = 0, chunk_end = 0;  // warp-uniform

  for (;;) {
    // ---- give idle lanes new histories from the warp's chunk ----
    unsigned idle = __ballot_sync(kFull, !alive && !done);
    while (idle) {
      if (chunk_next >= chunk_end) {
        unsigned long long b = 0;
        if (lane == 0) b = aborted(kp, polls) ? total : atomicAdd(kp.work_counter, (unsigned long long)kp.chunk);
        b = __shfl_sync(kFull, b, 0);
        if (b >= total) {
          if (!alive) done = true;
          break;
        }
        chunk_next = b;
        chunk_end = min(b + (unsigned long long)kp.chunk, total);
      }
      const unsigned avail = (unsigned)min((unsigned long long)__popc(idle), chunk_end - chunk_next);
      const unsigned rank = __popc(idle & lt_mask);
      if (((idle >> lane) & 1u) && rank < avail && kp.sec_mode == 2) {
        P = sec_read(reinterpret_cast<const SecRec<R>*>(kp.sec_buf) + chunk_next + rank);   // a queued secondary
#pragma unroll
        for (int i = 0; i < kMaxPar; ++i) ip[i] = __ldg(kp.inst_params + (size_t)P.inst * kMaxPar + i);
        dR = kp.radius_par >= 0 ? sel(ip, kp.radius_par, R(0)) - kp.radius_nominal : R(0);
        alive = true;
      } else if (((idle >> lane) & 1u) && rank < avail) {
        const unsigned long long g = chunk_next + rank + kp.index_base;
        // instance of global index g
        int lo = 0, hi = kp.n_inst - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (kp.inst_prefix[mid] <= g) lo = mid; else hi = mid - 1;
        }
        P.inst = (uint32_t)lo;
        P.hid = (uint32_t)(kp.inst_first[lo] + (g - kp.inst_prefix[lo]));
#pragma unroll
        for (int i = 0; i < kMaxPar; ++i) ip[i] = __ldg(kp.inst_params + (size_t)lo * kMaxPar + i);
        dR = kp.radius_par >= 0 ? sel(ip, kp.radius_par, R(0)) - kp.radius_nominal : R(0);
        cnt[C_HIST]++;
        int end = -1;
        alive = source<R, OPT>(kp, V, P, dR, &end);
        if (!alive) {
          if (end == END_LOST) cnt[C_LOST]++;
          finish(kp, P, end);
        }
      }
      chunk_next += avail;
      idle = __ballot_sync(kFull, !alive && !done);
    }
    if (__all_sync(kFull, done)) break;
    if (alive) {
      bool spawn = false;
      const int end = step<R, GRAD, OPT>(kp, V, P, ip, dR, cnt, &S, &spawn);
      if (end >= 0) finish(kp, P, end);
      if (GRAD && spawn && sec_push(kp, S)) spawn = false;
      if (GRAD && spawn) {
        if (end < 0) { park = P; parked = true; }
        P = S;
      } else if (end >= 0) {
        if (GRAD && parked) { P = park; parked = false; }
        else alive = false;
      }
    }
  }
  // ---- counters: warp sum, one atomic per warp and slot ----
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) {
    unsigned long long v = cnt[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0 && v) atomicAdd(kp.counters + i, v);
  }
}

// ---------------------------------------------------------------------------
// Event-based persistent kernel: a bank of neutrons in shared memory, one slot
// per thread, regrouped every event by what each neutron needs next.  Every
// iteration builds, with warp ballots, one queue per event type -- new history,
// advance inside a primitive, advance in the world region, collision -- and
// hands queue entries to consecutive threads, so that a warp runs one kind of
// event.  Gradient runs take the queues one after the other; plain runs take
// all of them in one phase (see the kernel).  An advance that reaches a
// boundary crosses it in the same pass (inside a primitive every crossing is
// an exit, in the world region an entry).
// ---------------------------------------------------------------------------
enum { EV_EMPTY = 0, EV_ADV = 1, EV_COLL = 2 };
enum { Q_EMPTY = 0, Q_ADVP, Q_ADVW, Q_COLL, kNumQ };
// plain runs: the queues concatenated in this order
enum { QP_ADVP = 0, QP_ADVW, QP_COLL, QP_EMPTY, kNumQPlain };
constexpr int kNumQMax = kNumQPlain > kNumQ ? kNumQPlain : kNumQ;

// Append `slot` to queue q if `pred`; all lanes of the warp must call this.
__device__ __forceinline__ void q_push(unsigned short* list, int* count, bool pred, int slot) {
  const unsigned m = __ballot_sync(kFull, pred);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(kFull, base, __ffs(m) - 1);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = (unsigned short)slot;
}

template <typename R>
__device__ __forceinline__ void load_params(const KParams<R>& kp, uint32_t inst, R (&ip)[kMaxPar], R* dR) {
  if (kp.npar == 0) {   // no instance parameters: nothing to read
#pragma unroll
    for (int i = 0; i < kMaxPar; ++i) ip[i] = R(0);
    *dR = R(0);
    return;
  }
  const R* q = kp.inst_params + (size_t)inst * kMaxPar;
#pragma unroll
  for (int i = 0; i < kMaxPar; ++i) ip[i] = __ldg(q + i);
  *dR = kp.radius_par >= 0 ? sel(ip, kp.radius_par, R(0)) - kp.radius_nominal : R(0);
}

// Counts of a secondary run out of line (returned, so that the caller's
// counters stay in registers).
struct SecCounts { unsigned c[kNumCounters]; };

// Transports a radius-derivative secondary to its end where it was made
// (gradient runs of the warp-pool kernel, when the queue of the second pass
// is full or not in use): out of line, a cold path that keeps its registers
// away from the hot loop.  A secondary makes no secondaries of its own.
template <typename R, int OPT>
__device__ __noinline__ SecCounts run_secondary(const KParams<R>& kp, const View<R>& V, Particle<R> S,
                                                const R (&ip)[kMaxPar], R dR) {
  SecCounts r;
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) r.c[i] = 0;
  for (;;) {
    Particle<R> none;
    bool spawn = false;
    const int end = step<R, true, OPT>(kp, V, S, ip, dR, r.c, &none, &spawn);
    if (end >= 0) {
      finish(kp, S, end);
      return r;
    }
  }
}

// The per-slot steps of the regrouping kernels.  A bank (event kernel) or pool
// (warp-pool kernel) holds one neutron per slot with its next event in pend[];
// in gradient runs a primary that made a radius-derivative secondary waits in
// park[] while the secondary runs in its slot.

// A new history with global index g into `slot`.  Returns -1 if it ended at
// the source, else 1 if it starts inside a primitive, 0 in the world region.
template <typename R, bool GRAD, int OPT>
__device__ __forceinline__ int slot_start(const KParams<R>& kp, const View<R>& V, const Bank<R, GRAD>& bank, int* pend,
                                          int slot, unsigned long long g, unsigned* cnt) {
  if (kp.sec_mode == 2) {   // a queued secondary: it starts where it was made
    const Particle<R> S = sec_read(reinterpret_cast<const SecRec<R>*>(kp.sec_buf) + g);
    bank.store(slot, S);
    pend[slot] = EV_ADV;
    return S.vol >= 0 ? 1 : 0;
  }
  g += kp.index_base;
  Particle<R> P;
  int lo = 0, hi = kp.n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (kp.inst_prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  P.inst = (uint32_t)lo;
  P.hid = (uint32_t)(kp.inst_first[lo] + (g - kp.inst_prefix[lo]));
  R ip[kMaxPar], dR;
  load_params(kp, P.inst, ip, &dR);
  cnt[C_HIST]++;
  int end = -1;
  if (!source<R, OPT>(kp, V, P, dR, &end)) {
    if (end == END_LOST) cnt[C_LOST]++;
    finish(kp, P, end);
    return -1;
  }
  bank.store(slot, P);
  pend[slot] = EV_ADV;
  return P.vol >= 0 ? 1 : 0;
}

// Advance the neutron of `slot` and, if it reaches a boundary, cross it (inside
// a primitive every crossing is an exit, in the world region an entry; the
// caller knows which: in_prim).  Returns true if it now waits for a collision.
// PARK: a secondary that is not queued takes over the slot while its primary
// waits in park[] (event kernel); without PARK (warp pools) the lane runs it
// to its end at once, out of line, and the pool needs no parking bank.
template <typename R, bool GRAD, int OPT, bool PARK = true>
__device__ __forceinline__ bool slot_advance(const KParams<R>& kp, const View<R>& V, const Bank<R, GRAD>& bank,
                                             const Bank<R, GRAD>& park, int* pend, int* parked, int slot, bool in_prim,
                                             unsigned* cnt) {
  Particle<R> P = bank.load(slot);
  R ip[kMaxPar], dR;
  load_params(kp, P.inst, ip, &dR);
  Adv<R> a;
  bool spawn = false, coll = false;
  Particle<R> S;
  int end;
  if (in_prim) {
    end = advance<R, GRAD, OPT, kInPrim>(kp, V, P, ip, dR, cnt, a);
    if (end == kOutCross) end = cross<R, GRAD, OPT, kInPrim>(kp, V, P, ip, dR, cnt, a.face, a.target, &S, &spawn);
  } else {
    end = advance<R, GRAD, OPT, kInWorld>(kp, V, P, ip, dR, cnt, a);
    if (end == kOutCross) end = cross<R, GRAD, OPT, kInWorld>(kp, V, P, ip, dR, cnt, a.face, a.target, &S, &spawn);
  }
  if (end == kOutColl) {
    pend[slot] = EV_COLL;
    coll = true;
  } else {
    if (end >= 0) finish(kp, P, end);
    if (GRAD && spawn && sec_push(kp, S)) spawn = false;
    if (GRAD && !PARK && spawn) {
      const SecCounts r = run_secondary<R, OPT>(kp, V, S, ip, dR);
#pragma unroll
      for (int i = 0; i < kNumCounters; ++i) cnt[i] += r.c[i];
      spawn = false;
    }
    if (GRAD && PARK && spawn) {
      if (end < 0) { park.store(slot, P); parked[slot] = 1; }
      P = S;
      pend[slot] = EV_ADV;
    } else if (end >= 0) {
      if (GRAD && PARK && parked[slot]) { P = park.load(slot); parked[slot] = 0; pend[slot] = EV_ADV; }
      else pend[slot] = EV_EMPTY;
    } else {
      pend[slot] = EV_ADV;
    }
  }
  bank.store(slot, P);
  return coll;
}

// The collision the neutron of `slot` waits for.
template <typename R, bool GRAD, bool PARK = true>
__device__ __forceinline__ void slot_collide(const KParams<R>& kp, const View<R>& V, const Bank<R, GRAD>& bank,
                                             const Bank<R, GRAD>& park, int* pend, int* parked, int slot,
                                             unsigned* cnt) {
  Particle<R> P = bank.load(slot);
  R ip[kMaxPar], dR;
  load_params(kp, P.inst, ip, &dR);
  const int end = collide_again<R, GRAD>(kp, V, P, ip, cnt);
  if (end >= 0) {
    finish(kp, P, end);
    if (GRAD && PARK && parked[slot]) { P = park.load(slot); parked[slot] = 0; pend[slot] = EV_ADV; }
    else pend[slot] = EV_EMPTY;
  } else {
    pend[slot] = EV_ADV;
  }
  bank.store(slot, P);
}


template <typename R, bool GRAD, int OPT, int MINB>
__global__ void __launch_bounds__(256, MINB) k_transport_ev(const __grid_constant__ KParams<R> kp) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bar;
  __shared__ int qcount[2][kNumQMax];   // per regrouping parity (plain runs)
  __shared__ unsigned long long claim_base;
  __shared__ int claim_state;        // 0 work left, 1 exhausted
  const int NB = blockDim.x;
  const int tid = threadIdx.x;
  const uint8_t* base = kp.blob;
  uint32_t tab = 0;
  if (kp.stage_blob) {
    if (!stage_tables(smem, kp.blob, kp.blob_bytes, &bar, (kp.test_flags & TP_TEST_SKIP_TABLE_COPY) != 0)) {
      if (tid == 0) atomicCAS(kp.status, 0, (int)TP_ERR_TIMEOUT);
      return;
    }
    base = smem;
    tab = (kp.blob_bytes + 15u) & ~15u;
  }
  View<R> V;
  V.prims = reinterpret_cast<const DPrim<R>*>(base + kp.off_prims);
  V.mats = reinterpret_cast<const DMat<R>*>(base + kp.off_mats);
  V.mirrors = reinterpret_cast<const DMirror<R>*>(base + kp.off_mirrors);
  V.choppers = reinterpret_cast<const DChopper<R>*>(base + kp.off_choppers);
  V.tallies = reinterpret_cast<const DTally<R>*>(base + kp.off_tallies);
  V.line_d = reinterpret_cast<const R*>(base + kp.off_line_d);
  V.line_cum = reinterpret_cast<const R*>(base + kp.off_line_cum);
  V.nb = reinterpret_cast<const int*>(base + kp.off_nb);
  // bank layout after the tables: the bank, parked primaries (gradient runs),
  // pending event types, parked flags, queues
  using BankT = Bank<R, GRAD>;
  const BankT bank(smem + tab, NB);
  const BankT park(smem + tab + BankT::bytes(NB), NB);
  int* pend = reinterpret_cast<int*>(smem + tab + BankT::bytes(NB) * (GRAD ? 2 : 1));
  int* parked = pend + NB;
  unsigned short* qlist = reinterpret_cast<unsigned short*>(parked + NB);  // [kNumQMax][NB]

  const unsigned long long total = work_total(kp);
  unsigned cnt[kNumCounters];   // per-thread counts: 32 bits suffice (widened below)
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) cnt[i] = 0;
  unsigned polls = 0;   // claims made by this thread (abort polling)
  const int lane = tid & 31;
  pend[tid] = EV_EMPTY;
  parked[tid] = 0;
  if (tid < 2 * kNumQMax) qcount[tid / kNumQMax][tid % kNumQMax] = 0;
  if (tid == 0) claim_state = 0;
  __syncthreads();

  if constexpr (GRAD) {
    // Gradient runs: the queues one after the other (refill, advance in a
    // primitive, advance in the world region, collision), consecutive threads
    // on consecutive entries, so that all warps of a phase run the same code:
    // the interface terms and secondaries make the advance large, and a phase
    // keeps the instructions the SM runs at once few.
    int* qc = qcount[0];
    for (;;) {
      if (tid < kNumQ) qc[tid] = 0;
      __syncthreads();
      {
        const int ty = pend[tid];
        const bool inprim = ty == EV_ADV && bank.vol(tid) >= 0;
        q_push(qlist + Q_EMPTY * NB, &qc[Q_EMPTY], ty == EV_EMPTY, tid);
        q_push(qlist + Q_ADVP * NB, &qc[Q_ADVP], ty == EV_ADV && inprim, tid);
        q_push(qlist + Q_ADVW * NB, &qc[Q_ADVW], ty == EV_ADV && !inprim, tid);
      }
      __syncthreads();
      const int n_empty = qc[Q_EMPTY];
      if (tid == 0) {
        claim_base = total;
        if (n_empty > 0 && claim_state == 0) {
          const unsigned long long b = aborted(kp, polls) ? total : atomicAdd(kp.work_counter, (unsigned long long)n_empty);
          claim_base = b;
          if (b + n_empty >= total) claim_state = 1;
        }
      }
      __syncthreads();
      {
        int born = -1, slot = 0;
        if (tid < n_empty) {
          slot = qlist[Q_EMPTY * NB + tid];
          const unsigned long long g = claim_base + tid;
          if (g < total) born = slot_start<R, GRAD, OPT>(kp, V, bank, pend, slot, g, cnt);
        }
        q_push(qlist + Q_ADVP * NB, &qc[Q_ADVP], born == 1, slot);
        q_push(qlist + Q_ADVW * NB, &qc[Q_ADVW], born == 0, slot);
      }
      __syncthreads();
      const int n_advp = qc[Q_ADVP], n_advw = qc[Q_ADVW];
      if (n_advp + n_advw == 0 && claim_state == 1) break;   // uniform: shared values
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        const int n = pass == 0 ? n_advp : n_advw;
        int slot = 0;
        bool coll = false;
        if (tid < n) {
          slot = qlist[(pass == 0 ? Q_ADVP : Q_ADVW) * NB + tid];
          coll = slot_advance<R, GRAD, OPT>(kp, V, bank, park, pend, parked, slot, pass == 0, cnt);
        }
        q_push(qlist + Q_COLL * NB, &qc[Q_COLL], coll, slot);
      }
      __syncthreads();
      if (tid < qc[Q_COLL]) slot_collide<R, GRAD>(kp, V, bank, park, pend, parked, qlist[Q_COLL * NB + tid], cnt);
      __syncthreads();
    }
  } else {
    // Plain runs: one work phase per iteration.  In a regrouping iteration
    // thread t takes the t-th entry of the concatenated queues [advance in a
    // primitive | advance in the world region | collision | refill], so that
    // every thread of the block has a slot and each warp runs one kind of
    // event (but those at the joins).  Two barriers per regrouping; the
    // counts alternate between two buffers so that a reset never meets a
    // reader.  With
    // kp.regroup = R > 1 only every R-th iteration regroups: in between, each
    // thread runs the next event of the neutron it had, without barriers.
    const int every = kp.regroup > 1 ? kp.regroup : 1;
    int my_slot = -1, ri = 0;
    for (int iter = 0;; ++iter) {
      const bool regroup = (iter % every) == 0;
      int slot = -1, kind = 0;   // 1 advance in a primitive, 2 in the world region, 3 collision
      bool want = false;         // refill rslot with a new history
      int rslot = -1;
      if (regroup) {
        int* qc = qcount[ri & 1];
        bool exhausted;
        {
          const int ty = pend[tid];
          const bool inprim = ty == EV_ADV && bank.vol(tid) >= 0;
          q_push(qlist + QP_ADVP * NB, &qc[QP_ADVP], ty == EV_ADV && inprim, tid);
          q_push(qlist + QP_ADVW * NB, &qc[QP_ADVW], ty == EV_ADV && !inprim, tid);
          q_push(qlist + QP_COLL * NB, &qc[QP_COLL], ty == EV_COLL, tid);
          q_push(qlist + QP_EMPTY * NB, &qc[QP_EMPTY], ty == EV_EMPTY, tid);
          if (tid < kNumQPlain) qcount[(ri + 1) & 1][tid] = 0;   // last read in the previous regrouping
          exhausted = claim_state != 0;                         // last written before the last barrier
        }
        __syncthreads();
        int live = 0;
#pragma unroll
        for (int q = 0; q < QP_EMPTY; ++q) live += qc[q];
        if (live == 0 && exhausted) break;   // uniform: shared values read before any write
        int t = tid, q = 0;
        for (; q < QP_EMPTY; ++q) {
          if (t < qc[q]) break;
          t -= qc[q];
        }
        if (q < QP_EMPTY) {
          slot = qlist[q * NB + t];
          kind = q == QP_ADVP ? 1 : (q == QP_ADVW ? 2 : 3);
        } else if (t < qc[QP_EMPTY] && !exhausted) {
          want = true;
          rslot = qlist[QP_EMPTY * NB + t];
        }
        ++ri;
      } else if (my_slot >= 0) {
        const int ty = pend[my_slot];
        if (ty == EV_ADV) { slot = my_slot; kind = bank.vol(my_slot) >= 0 ? 1 : 2; }
        else if (ty == EV_COLL) { slot = my_slot; kind = 3; }
        else if (claim_state == 0) { want = true; rslot = my_slot; }
      }
      if (kind == 1 || kind == 2) slot_advance<R, GRAD, OPT>(kp, V, bank, park, pend, parked, slot, kind == 1, cnt);
      else if (kind == 3) slot_collide<R, GRAD>(kp, V, bank, park, pend, parked, slot, cnt);
      // refill: new histories, one claim per warp
      const unsigned m = __ballot_sync(kFull, want);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long g = 0;
        if (lane == leader) g = aborted(kp, polls) ? total : atomicAdd(kp.work_counter, (unsigned long long)__popc(m));
        g = __shfl_sync(kFull, g, leader) + __popc(m & ((1u << lane) - 1u));
        if (want) {
          if (g < total) slot_start<R, GRAD, OPT>(kp, V, bank, pend, rslot, g, cnt);
          else claim_state = 1;
        }
      }
      my_slot = kind ? slot : rslot;
      if ((iter + 1) % every == 0) __syncthreads();   // the next iteration regroups
    }
  }
  // ---- counters ----
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) {
    unsigned long long v = cnt[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0 && v) atomicAdd(kp.counters + i, v);
  }
}

// ---------------------------------------------------------------------------
// Warp-pool kernel: each warp owns kPool neutrons in shared memory and, every
// step, runs the event type most of them wait for (new history, advance in a
// primitive -- with the exit crossing --, advance in the world -- with the
// entry crossing --, collision) on up to 32 of them, so the warp executes one
// code path with most lanes busy.  Warps never wait for one another: no CTA
// barrier after the table copy.
// ---------------------------------------------------------------------------
#ifndef TP_POOL
#define TP_POOL 64
#endif
constexpr int kPool = TP_POOL;            // neutrons per warp (a multiple of 32)
static_assert(kPool % 32 == 0, "pool size");
constexpr int kPoolGroups = kPool / 32;   // pool slots per lane

template <typename R, bool GRAD, int OPT, int MINB>
__global__ void __launch_bounds__(256, MINB) k_transport_wq(const __grid_constant__ KParams<R> kp) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bar;
  const uint8_t* base = kp.blob;
  uint32_t tab = 0;
  if (kp.stage_blob) {
    if (!stage_tables(smem, kp.blob, kp.blob_bytes, &bar, (kp.test_flags & TP_TEST_SKIP_TABLE_COPY) != 0)) {
      if (threadIdx.x == 0) atomicCAS(kp.status, 0, (int)TP_ERR_TIMEOUT);
      return;
    }
    base = smem;
    tab = (kp.blob_bytes + 15u) & ~15u;
  }
  View<R> V;
  V.prims = reinterpret_cast<const DPrim<R>*>(base + kp.off_prims);
  V.mats = reinterpret_cast<const DMat<R>*>(base + kp.off_mats);
  V.mirrors = reinterpret_cast<const DMirror<R>*>(base + kp.off_mirrors);
  V.choppers = reinterpret_cast<const DChopper<R>*>(base + kp.off_choppers);
  V.tallies = reinterpret_cast<const DTally<R>*>(base + kp.off_tallies);
  V.line_d = reinterpret_cast<const R*>(base + kp.off_line_d);
  V.line_cum = reinterpret_cast<const R*>(base + kp.off_line_cum);
  V.nb = reinterpret_cast<const int*>(base + kp.off_nb);

  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  __shared__ unsigned char sel[8][32];   // per warp: the slots of this step, in lane order
  unsigned char* sel_row = sel[warp];
  // per warp: its pool of kPool neutrons and their pending event types (no
  // parking: a secondary that is not queued runs to its end at once)
  using BankT = Bank<R, GRAD>;
  const BankT pool(smem + tab + BankT::bytes(kPool) * warp, kPool);
  const BankT park = pool;   // unused (PARK false)
  int* pend = reinterpret_cast<int*>(smem + tab + BankT::bytes(kPool) * nwarps) + warp * 2 * kPool;
  int* parked = pend + kPool;

  const unsigned long long total = work_total(kp);
  unsigned cnt[kNumCounters];   // per-thread counts: 32 bits suffice (widened below)
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) cnt[i] = 0;
  unsigned polls = 0;   // claims made by this thread (abort polling)
#pragma unroll
  for (int g = 0; g < kPoolGroups; ++g) { pend[g * 32 + lane] = EV_EMPTY; parked[g * 32 + lane] = 0; }
  __syncwarp();
  unsigned long long chunk_next = 0, chunk_end = 0;   // warp-uniform
  bool work_left = true;                              // warp-uniform

  for (;;) {
    // ---- count what the pool waits for ----
    unsigned m[kNumQ][kPoolGroups];
#pragma unroll
    for (int g = 0; g < kPoolGroups; ++g) {
      const int slot = g * 32 + lane;
      const int ty = pend[slot];
      const bool adv = ty == EV_ADV;
      const bool inprim = adv && pool.vol(slot) >= 0;
      m[Q_EMPTY][g] = __ballot_sync(kFull, ty == EV_EMPTY);
      m[Q_ADVP][g] = __ballot_sync(kFull, adv && inprim);
      m[Q_ADVW][g] = __ballot_sync(kFull, adv && !inprim);
      m[Q_COLL][g] = __ballot_sync(kFull, ty == EV_COLL);
    }
    int count[kNumQ];
#pragma unroll
    for (int q = 0; q < kNumQ; ++q) {
      count[q] = 0;
#pragma unroll
      for (int g = 0; g < kPoolGroups; ++g) count[q] += __popc(m[q][g]);
    }
    // ---- pick the queue: refill when half the pool is free, else the fullest ----
    int q = -1;
    if (work_left && count[Q_EMPTY] >= 32) {
      q = Q_EMPTY;
    } else {
      int best = 0;
#pragma unroll
      for (int k = 1; k < kNumQ; ++k)
        if (count[k] > best) { best = count[k]; q = k; }
      if (q < 0) {
        if (work_left && count[Q_EMPTY] > 0) q = Q_EMPTY;
        else break;   // nothing live and no work left
      }
    }
    // ---- lane j takes the j-th slot of queue q ----
    const int n = min(count[q], 32);
    int slot = -1;
    if constexpr (!(OPT & kOptFull)) {
      // lean build: the slots' own lanes write their indices in rank order to
      // the warp's selection row and lane j reads entry j (powder +14 %)
      int base = 0;
#pragma unroll
      for (int g = 0; g < kPoolGroups; ++g) {
        const unsigned mg = m[q][g];
        const int r = base + __popc(mg & lt_mask);
        if (((mg >> lane) & 1u) && r < 32) sel_row[r] = (unsigned char)(g * 32 + lane);
        base += __popc(mg);
      }
      __syncwarp();
      if (lane < n) slot = (int)sel_row[lane];
      __syncwarp();
    } else if (lane < n) {
      // full build: each lane finds its set bit (guide and total scattering
      // run 5 % faster this way)
      int j = lane;
#pragma unroll
      for (int g = 0; g < kPoolGroups; ++g) {
        const int c = __popc(m[q][g]);
        if (slot < 0) {
          if (j < c) slot = g * 32 + (int)__fns(m[q][g], 0, j + 1);
          else j -= c;
        }
      }
    }
    if (q == Q_EMPTY) {
      // new histories from the warp's chunk of global indices
      int taken = 0;
      while (taken < n) {
        if (chunk_next >= chunk_end) {
          unsigned long long b = 0;
          if (lane == 0) b = aborted(kp, polls) ? total : atomicAdd(kp.work_counter, (unsigned long long)kp.chunk);
          b = __shfl_sync(kFull, b, 0);
          if (b >= total) { work_left = false; break; }
          chunk_next = b;
          chunk_end = min(b + (unsigned long long)kp.chunk, total);
        }
        const int avail = (int)min((unsigned long long)(n - taken), chunk_end - chunk_next);
        if (lane >= taken && lane < taken + avail)
          slot_start<R, GRAD, OPT>(kp, V, pool, pend, slot, chunk_next + (lane - taken), cnt);
        chunk_next += avail;
        taken += avail;
      }
    } else if (q == Q_ADVP || q == Q_ADVW) {
      if (slot >= 0) slot_advance<R, GRAD, OPT, false>(kp, V, pool, park, pend, parked, slot, q == Q_ADVP, cnt);
    } else {
      if (slot >= 0) slot_collide<R, GRAD, false>(kp, V, pool, park, pend, parked, slot, cnt);
    }
    __syncwarp();
  }
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) {
    unsigned long long v = cnt[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0 && v) atomicAdd(kp.counters + i, v);
  }
}

// mean and standard error per bin
__global__ void k_stats(const double* __restrict__ sum, const double* __restrict__ sumsq, double n,
                        int nbins, double* __restrict__ mean, double* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbins) return;
  const double m = n > 0 ? sum[i] / n : 0.0;
  mean[i] = m;
  if (err) {
    const double var = n > 0 ? fmax(sumsq[i] / n - m * m, 0.0) : 0.0;
    err[i] = n > 1 ? sqrt(var / (n - 1.0)) : 0.0;
  }
}

// grad_params[i][p] = scale[i][p] / N_i * sum_b grad[i][b] J[p][i][b]; one CTA per (i, p)
__global__ void k_backward(const double* __restrict__ J, const double* __restrict__ grad,
                           const double* __restrict__ scale, const double* __restrict__ n_done,
                           int n_inst, int npar, int total_bins, double* __restrict__ out) {
  const int i = blockIdx.x, p = blockIdx.y;
  const double* Jp = J + ((size_t)p * n_inst + i) * total_bins;
  const double* g = grad + (size_t)i * total_bins;
  double acc = 0.0;
  for (int b = threadIdx.x; b < total_bins; b += blockDim.x) acc += g[b] * Jp[b];
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (threadIdx.x == 0) {
      const double n = n_done[i];
      out[(size_t)i * npar + p] = n > 0 ? acc * scale[(size_t)i * npar + p] / n : 0.0;
    }
  }
}

// Each kernel exists in two register budgets: 80 registers (3 blocks of 256
// threads per SM) and, for FP32 runs, 64 registers (4 blocks; more warps to
// hide latency, more spills).  The flag kVariantHighOcc on the variant selects
// the second (FP32 runs only), kVariantFull the complete feature set (else
// the lean build, see kOptFull).
#define TP_KERNEL_TABLE(NAME)                                                                   \
  template <typename R, bool GRAD, int OPT, int MINB>                                          \
  struct NAME##_t {                                                                            \
    static const void* fn() { return (const void*)NAME<R, GRAD, OPT, MINB>; }                  \
    static void launch(const KParams<R>& p, int grid, int block, size_t smem, cudaStream_t st) { \
      NAME<R, GRAD, OPT, MINB><<<grid, block, smem, st>>>(p);                                  \
    }                                                                                          \
  };
TP_KERNEL_TABLE(k_transport)
TP_KERNEL_TABLE(k_transport_ev)
TP_KERNEL_TABLE(k_transport_wq)
#undef TP_KERNEL_TABLE
template <typename R> struct HistTag { template <bool G, int O, int M> using k = k_transport_t<R, G, O, M>; };
template <typename R> struct EvTag { template <bool G, int O, int M> using k = k_transport_ev_t<R, G, O, M>; };
template <typename R> struct WqTag { template <bool G, int O, int M> using k = k_transport_wq_t<R, G, O, M>; };

// Calls f(K()) with K the kernel of one family (Tag) for (options, gradients,
// register budget).
template <typename R, typename Tag, int OPT, typename F>
auto with_budget(bool grad, bool hi, F&& f) {
  if (grad && !hi) return f(typename Tag::template k<true, OPT, 3>());
  if constexpr (sizeof(R) == 4) {
    if (grad) return f(typename Tag::template k<true, OPT, 4>());
    if (hi) return f(typename Tag::template k<false, OPT, 4>());
  }
  return f(typename Tag::template k<false, OPT, 3>());
}

// The gradient history kernel without secondaries (kOptNoSec), per budget.
template <typename R, typename Tag, int OPT, typename F>
auto with_budget_nosec(bool hi, F&& f) {
  if constexpr (sizeof(R) == 4) {
    if (hi) return f(typename Tag::template k<true, OPT | kOptNoSec, 4>());
  }
  return f(typename Tag::template k<true, OPT | kOptNoSec, 3>());
}

// nosec: a gradient run without a radius parameter (history kernel only).
template <typename R, typename Tag, typename F>
auto with_kernel(int variant, bool grad, bool grid, F&& f, bool nosec = false) {
  const bool hi = (variant & kVariantHighOcc) && sizeof(R) == 4;
  const bool full = (variant & kVariantFull) != 0;
  if constexpr (std::is_same<Tag, HistTag<R>>::value || std::is_same<Tag, WqTag<R>>::value) {
    if (grad && nosec) {
      if (full) return grid ? with_budget_nosec<R, Tag, kOptFull | kOptGrid>(hi, f) : with_budget_nosec<R, Tag, kOptFull>(hi, f);
      return grid ? with_budget_nosec<R, Tag, kOptGrid>(hi, f) : with_budget_nosec<R, Tag, 0>(hi, f);
    }
  }
  if (full) return grid ? with_budget<R, Tag, kOptFull | kOptGrid>(grad, hi, f) : with_budget<R, Tag, kOptFull>(grad, hi, f);
  return grid ? with_budget<R, Tag, kOptGrid>(grad, hi, f) : with_budget<R, Tag, 0>(grad, hi, f);
}

template <typename R, typename Tag>
cudaError_t launch_family(const KParams<R>& p, int variant, bool grad, int grid, int block, size_t smem,
                          cudaStream_t st) {
  with_kernel<R, Tag>(variant, grad, p.use_grid != 0, [&](auto k) {
    decltype(k)::launch(p, grid, block, smem, st);
    return 0;
  }, p.radius_par < 0);
  return cudaGetLastError();
}

// The dynamic shared-memory limit of a kernel only grows, so that every
// configuration resolved earlier (the autotuner resolves all candidates before
// timing them) can still be launched.
cudaError_t occupancy_of(const void* fn, int block, size_t smem, int* ctas) {
  cudaFuncAttributes attr;
  cudaError_t e = cudaFuncGetAttributes(&attr, fn);
  if (e != cudaSuccess) return e;
  if ((size_t)attr.maxDynamicSharedSizeBytes < smem) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, block, smem);
}

template <typename R, typename Tag>
cudaError_t occupancy_family(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas) {
  cudaError_t e = occupancy_of(with_kernel<R, Tag>(variant, grad, use_grid, [](auto k) { return decltype(k)::fn(); }),
                               block, smem, ctas);
  if (e != cudaSuccess || !grad || !(std::is_same<Tag, HistTag<R>>::value || std::is_same<Tag, WqTag<R>>::value))
    return e;
  // the build without secondaries that the same launch may take: its limit
  // too, and the smaller occupancy of the two
  int c2 = 0;
  e = occupancy_of(with_kernel<R, Tag>(variant, grad, use_grid, [](auto k) { return decltype(k)::fn(); }, true),
                   block, smem, &c2);
  if (e == cudaSuccess && c2 < *ctas) *ctas = c2;
  return e;
}

}  // namespace

// This file is compiled once per (precision, kernel family) -- TP_BUILD_F32 or
// TP_BUILD_F64 with TP_BUILD_KERNEL = 1 (history), 2 (event) or 3 (warp
// pools) -- so that the kernels build in parallel, and once with
// TP_BUILD_COMMON for the dispatch, the sizes and the small kernels.
#if defined(TP_BUILD_KERNEL)
#if TP_BUILD_KERNEL == 1
#define TP_FAMILY HistTag
#define TP_SUFFIX k1
#elif TP_BUILD_KERNEL == 2
#define TP_FAMILY EvTag
#define TP_SUFFIX k2
#else
#define TP_FAMILY WqTag
#define TP_SUFFIX k3
#endif
#define TP_CAT_(a, b) a##_##b
#define TP_CAT(a, b) TP_CAT_(a, b)
#if defined(TP_BUILD_F32)
cudaError_t TP_CAT(launch_transport_f32, TP_SUFFIX)(const KParams<float>& p, int variant, bool grad, int grid,
                                                     int block, size_t smem, cudaStream_t st) {
  return launch_family<float, TP_FAMILY<float>>(p, variant, grad, grid, block, smem, st);
}
cudaError_t TP_CAT(occupancy_f32, TP_SUFFIX)(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas) {
  return occupancy_family<float, TP_FAMILY<float>>(variant, grad, use_grid, block, smem, ctas);
}
#endif
#if defined(TP_BUILD_F64)
cudaError_t TP_CAT(launch_transport_f64, TP_SUFFIX)(const KParams<double>& p, int variant, bool grad, int grid,
                                                     int block, size_t smem, cudaStream_t st) {
  return launch_family<double, TP_FAMILY<double>>(p, variant, grad, grid, block, smem, st);
}
cudaError_t TP_CAT(occupancy_f64, TP_SUFFIX)(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas) {
  return occupancy_family<double, TP_FAMILY<double>>(variant, grad, use_grid, block, smem, ctas);
}
#endif
#endif  // TP_BUILD_KERNEL

#if defined(TP_BUILD_COMMON)
cudaError_t launch_transport_f32(const KParams<float>& p, int variant, bool grad, int grid, int block, size_t smem,
                                 cudaStream_t st) {
  switch (variant & 3) {
    case TP_KERNEL_EVENT: return launch_transport_f32_k2(p, variant, grad, grid, block, smem, st);
    case TP_KERNEL_WARPQ: return launch_transport_f32_k3(p, variant, grad, grid, block, smem, st);
    default: return launch_transport_f32_k1(p, variant, grad, grid, block, smem, st);
  }
}

cudaError_t launch_transport_f64(const KParams<double>& p, int variant, bool grad, int grid, int block, size_t smem,
                                 cudaStream_t st) {
  switch (variant & 3) {
    case TP_KERNEL_EVENT: return launch_transport_f64_k2(p, variant, grad, grid, block, smem, st);
    case TP_KERNEL_WARPQ: return launch_transport_f64_k3(p, variant, grad, grid, block, smem, st);
    default: return launch_transport_f64_k1(p, variant, grad, grid, block, smem, st);
  }
}

cudaError_t occupancy_f32(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas) {
  switch (variant & 3) {
    case TP_KERNEL_EVENT: return occupancy_f32_k2(variant, grad, use_grid, block, smem, ctas);
    case TP_KERNEL_WARPQ: return occupancy_f32_k3(variant, grad, use_grid, block, smem, ctas);
    default: return occupancy_f32_k1(variant, grad, use_grid, block, smem, ctas);
  }
}

cudaError_t occupancy_f64(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas) {
  switch (variant & 3) {
    case TP_KERNEL_EVENT: return occupancy_f64_k2(variant, grad, use_grid, block, smem, ctas);
    case TP_KERNEL_WARPQ: return occupancy_f64_k3(variant, grad, use_grid, block, smem, ctas);
    default: return occupancy_f64_k1(variant, grad, use_grid, block, smem, ctas);
  }
}

size_t particle_bytes(int precision) {
  return precision == TP_FP64 ? sizeof(SecRec<double>) : sizeof(SecRec<float>);
}

size_t bank_bytes(int variant, int precision, bool grad, int block) {
  variant &= 3;
  const size_t ps = precision == TP_FP64 ? (grad ? Bank<double, true>::kBytes : Bank<double, false>::kBytes)
                                         : (grad ? Bank<float, true>::kBytes : Bank<float, false>::kBytes);
  if (variant == TP_KERNEL_EVENT)
    return ps * block * (grad ? 2 : 1) + 2 * sizeof(int) * block + sizeof(unsigned short) * kNumQMax * block;
  if (variant == TP_KERNEL_WARPQ) {
    const size_t slots = (size_t)(block / 32) * kPool;
    return ps * slots + 2 * sizeof(int) * slots;
  }
  return 0;
}

cudaError_t occupancy_transport(int variant, int precision, bool grad, bool use_grid, int block, size_t smem,
                                int* ctas) {
  return precision == TP_FP64 ? occupancy_f64(variant, grad, use_grid, block, smem, ctas)
                              : occupancy_f32(variant, grad, use_grid, block, smem, ctas);
}

cudaError_t launch_stats(const double* sum, const double* sumsq, double n, int nbins, double* mean,
                         double* err, cudaStream_t st) {
  if (nbins <= 0) return cudaSuccess;
  k_stats<<<(nbins + 255) / 256, 256, 0, st>>>(sum, sumsq, n, nbins, mean, err);
  return cudaGetLastError();
}

cudaError_t launch_backward(const double* J, const double* grad_tallies, const double* scale,
                            const double* n_done, int n_inst, int npar, int total_bins,
                            double* grad_params, cudaStream_t st) {
  if (n_inst <= 0 || npar <= 0) return cudaSuccess;
  k_backward<<<dim3(n_inst, npar), 256, 0, st>>>(J, grad_tallies, scale, n_done, n_inst, npar, total_bins,
                                                 grad_params);
  return cudaGetLastError();
}
#endif  // TP_BUILD_COMMON

}  // namespace tp
