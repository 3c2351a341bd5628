// tp_api.cu -- host runtime behind the C ABI of include/tp.h: scene validation,
// device tables, launch configuration, tallies, backward pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "tp_internal.h"

using namespace tp;

namespace {

thread_local std::string g_err;

tp_status fail(tp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define TP_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
  } while (0)

// The status word the kernels leave (0 = fine) as a tp_status with a message.
tp_status device_status(int status) {
  if (status == 0) return TP_OK;
  if (status == TP_ERR_TIMEOUT)
    return fail(TP_ERR_TIMEOUT, "a block's bounded wait for its copy of the scene tables gave up");
  if (status == TP_ERR_ABORTED) return fail(TP_ERR_ABORTED, "the run was stopped by tp_abort");
  return fail((tp_status)status, "device status %d", status);
}

// Test flags of the allocation-free call (tp_set_test_flags with no scene).
std::atomic<int> g_noalloc_test_flags{0};

bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

constexpr double kBoltzmann_meV = 0.08617333;   // k_B in meV/K

// Instance parameters [n][kMaxPar] in the transport precision (what the kernels read).
std::vector<uint8_t> params_bytes(const std::vector<double>& p, int precision) {
  std::vector<uint8_t> out(p.size() * (precision == TP_FP64 ? sizeof(double) : sizeof(float)));
  if (precision == TP_FP64) {
    std::memcpy(out.data(), p.data(), out.size());
  } else {
    float* f = reinterpret_cast<float*>(out.data());
    for (size_t i = 0; i < p.size(); ++i) f[i] = (float)p[i];
  }
  return out;
}

// Source checks shared by both ways of describing a scene.
bool source_ok(const tp_source& src) {
  if (src.kind < TP_SRC_PENCIL || src.kind > TP_SRC_MODERATOR) return false;
  if (!(src.temperature >= 0) || !std::isfinite(src.temperature)) return false;
  if (src.temperature == 0 && (!(src.lambda_lo > 0) || !(src.lambda_hi >= src.lambda_lo) || !std::isfinite(src.lambda_hi)))
    return false;
  if (!(src.div[0] >= 0 && src.div[0] < 1.5 && src.div[1] >= 0 && src.div[1] < 1.5)) return false;
  if (src.temperature > 0 && src.kind != TP_SRC_MODERATOR && (src.div[0] > 0 || src.div[1] > 0)) return false;
  if (src.kind == TP_SRC_MODERATOR &&
      (!(src.slit_z > src.centre[2]) || !(src.slit_half[0] >= 0) || !(src.slit_half[1] >= 0) ||
       !std::isfinite(src.slit_z) || !std::isfinite(src.slit_half[0]) || !std::isfinite(src.slit_half[1])))
    return false;
  return finite_all(src.centre, 3) && finite_all(src.half, 2);
}

struct Mat {
  tp_material m;
  std::vector<double> d, mult, F2;  // sorted by d descending
  double g[TP_NPROC] = {1.0, 1.0, 1.0};
};

}  // namespace

// A launch configuration: kernel variant, block size, CTAs per SM and options.
struct LaunchCfg {
  int kernel, block, ctas;
  int stage;   // copy the scene tables into shared memory
  int hi;      // the 64-register build (FP32 runs only)
  int defer;   // gradient runs: secondaries queued and transported in a second pass
  int full = 1;  // the build with every feature (else the lean one)
  int regroup = 1;  // event kernel, plain runs: events between regroupings
  int variant() const { return kernel | (hi ? kVariantHighOcc : 0) | (full ? kVariantFull : 0); }
};

struct tp_scene {
  int device = 0;
  int sm_count = 0;
  int precision = TP_FP32;
  int event_cap = 4096;
  // 1 if the scene needs the kernels' full feature set (mirrors, choppers,
  // scorers other than count / angular / PSD, moderator / Maxwellian /
  // divergent guns or an aperture), 0 if the lean build serves it
  int full = 1;
  int full_needed = 1;   // what the description needs (full may be forced by a test flag)
  int src_free = 0;      // every source point in the world region (set with the tables)
  // description (owned copies)
  int world_shape = TP_BOX;
  double world_c[3] = {0, 0, 0}, world_p[3] = {0, 0, 0};
  std::vector<tp_prim> prims;
  std::vector<tp_mirror> mirrors;
  std::vector<tp_chopper> choppers;
  tp_source source{};
  std::vector<tp_tally_desc> tallies;
  std::vector<int> tally_off;
  int total_bins = 0;
  int n_inst = 1, n_par = 0;
  std::vector<double> inst_params;  // [n_inst][kMaxPar]
  std::vector<int> param_kind;
  double radius_nominal = 0.0;
  std::vector<Mat> mats;
  bool have_materials = false;
  // device tables
  uint8_t* d_blob = nullptr;
  size_t blob_cap = 0;
  uint32_t blob_bytes = 0;
  uint32_t off_prims = 0, off_mats = 0, off_mirrors = 0, off_choppers = 0, off_tallies = 0, off_line_d = 0,
           off_line_cum = 0, off_nb = 0;
  bool blob_dirty = true;
  // uniform grid (scenes with more than kGridMinPrims primitives)
  int* d_grid = nullptr;   // [ncells + 1] starts, then items
  int grid_n[3] = {0, 0, 0};
  double grid_lo[3] = {0, 0, 0}, grid_hi[3] = {0, 0, 0};
  int grid_cells = 0;
  // tallies
  double *d_sum = nullptr, *d_sumsq = nullptr, *d_J = nullptr, *d_J2 = nullptr;
  std::vector<double> n_done;  // histories run per instance
  // per-run work description
  unsigned long long *d_prefix = nullptr, *d_first = nullptr, *h_stage = nullptr;
  void* d_params = nullptr;   // instance parameters in the transport precision
  double* d_aux = nullptr;  // backward: [n_inst][n_par] scale + [n_inst] n_done
  double* h_aux = nullptr;
  unsigned long long* d_work = nullptr;
  unsigned long long* d_counters = nullptr;
  int* d_status = nullptr;
  // abort request: host-written flag in mapped pinned memory (tp_abort)
  volatile int* h_abort = nullptr;
  int* d_abort = nullptr;
  int test_flags = 0;   // tp_set_test_flags
  cudaEvent_t stage_done = nullptr;
  bool stage_pending = false;
  // launch configuration: last used, and the autotuned choice per gradient mode
  int kernel = 0, block = 0, ctas_per_sm = 0;
  LaunchCfg last_cfg{};   // the last run's complete configuration
  int launches = 0;   // transport kernels of the last run
  int smem_optin = 0; // shared memory a block may use on this device (queried once)
  int tuned_kernel[2] = {0, 0}, tuned_block[2] = {0, 0}, tuned_stage[2] = {-1, -1}, tuned_hi[2] = {-1, -1};
  int tuned_defer = 0;   // gradient runs: secondaries queued for a second pass
  int tuned_regroup[2] = {1, 1};   // event kernel: events between regroupings
  // queue of radius-derivative secondaries for the second pass (gradient runs)
  uint8_t* d_sec = nullptr;
  unsigned long long* d_sec_count = nullptr;
  unsigned long long sec_cap = 0;
  LaunchCfg sec_cfg{0, 0, 0, 0, 0, 0};   // the second pass (plain warp-pool kernel)
  // CUDA graph of the last graph run and the launch it was captured for
  cudaGraphExec_t graph = nullptr;
  cudaStream_t capture_stream = nullptr;
  unsigned long long graph_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

// ---------------------------------------------------------------------------
// Validation helpers
// ---------------------------------------------------------------------------
struct Box3 { double lo[3], hi[3]; };

double bound_r0(const tp_scene* s, const tp_prim& p, int inst) {
  double r = p.params[0];
  if (p.bind_rmin) {
    for (int i = 0; i < s->n_par; ++i)
      if (s->param_kind[i] == TP_PAR_RADIUS) r += s->inst_params[(size_t)inst * kMaxPar + i] - s->radius_nominal;
  }
  return r;
}
double bound_r1(const tp_scene* s, const tp_prim& p, int inst) {
  double r = p.params[1];
  if (p.bind_rmax) {
    for (int i = 0; i < s->n_par; ++i)
      if (s->param_kind[i] == TP_PAR_RADIUS) r += s->inst_params[(size_t)inst * kMaxPar + i] - s->radius_nominal;
  }
  return r;
}

Box3 aabb(const tp_scene* s, const tp_prim& p, int inst) {
  Box3 b;
  double h[3];
  if (p.shape == TP_BOX) {
    for (int i = 0; i < 3; ++i) h[i] = p.params[i];
  } else if (p.shape == TP_TUBE) {
    const double r = bound_r1(s, p, inst);
    for (int i = 0; i < 3; ++i) h[i] = r;
    h[p.axis] = p.params[2];
  } else {
    const double r = bound_r1(s, p, inst);
    for (int i = 0; i < 3; ++i) h[i] = r;
  }
  for (int i = 0; i < 3; ++i) { b.lo[i] = p.centre[i] - h[i]; b.hi[i] = p.centre[i] + h[i]; }
  return b;
}

bool point_inside(const tp_scene* s, const tp_prim& p, int inst, const double x[3], double shrink) {
  double d[3] = {x[0] - p.centre[0], x[1] - p.centre[1], x[2] - p.centre[2]};
  if (p.shape == TP_BOX)
    return std::fabs(d[0]) < p.params[0] - shrink && std::fabs(d[1]) < p.params[1] - shrink &&
           std::fabs(d[2]) < p.params[2] - shrink;
  const double r0 = bound_r0(s, p, inst), r1 = bound_r1(s, p, inst);
  if (p.shape == TP_TUBE) {
    double rho2 = 0;
    for (int i = 0; i < 3; ++i)
      if (i != p.axis) rho2 += d[i] * d[i];
    const double rho = std::sqrt(rho2);
    return rho > r0 + shrink && rho < r1 - shrink && std::fabs(d[p.axis]) < p.params[2] - shrink;
  }
  const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  return r > r0 + shrink && r < r1 - shrink;
}

// true if primitives a and b share interior volume (exact for boxes, coaxial
// tubes and concentric spheres; otherwise a sampling test on a 9^3 grid)
bool overlap(const tp_scene* s, const tp_prim& a, const tp_prim& b, int inst) {
  const Box3 A = aabb(s, a, inst), B = aabb(s, b, inst);
  for (int i = 0; i < 3; ++i)
    if (A.hi[i] <= B.lo[i] || B.hi[i] <= A.lo[i]) return false;
  if (a.shape == TP_BOX && b.shape == TP_BOX) return true;
  const double eps = 1e-12;
  if (a.shape == TP_TUBE && b.shape == TP_TUBE && a.axis == b.axis) {
    bool coaxial = true;
    for (int i = 0; i < 3; ++i)
      if (i != a.axis && std::fabs(a.centre[i] - b.centre[i]) > eps) coaxial = false;
    if (coaxial) {
      const double ra0 = bound_r0(s, a, inst), ra1 = bound_r1(s, a, inst);
      const double rb0 = bound_r0(s, b, inst), rb1 = bound_r1(s, b, inst);
      return ra0 < rb1 - eps && rb0 < ra1 - eps;  // axial overlap already implied by the boxes
    }
  }
  if (a.shape == TP_SPHERE && b.shape == TP_SPHERE) {
    const double dx = a.centre[0] - b.centre[0], dy = a.centre[1] - b.centre[1], dz = a.centre[2] - b.centre[2];
    const double dc = std::sqrt(dx * dx + dy * dy + dz * dz);
    const double ra0 = bound_r0(s, a, inst), ra1 = bound_r1(s, a, inst);
    const double rb0 = bound_r0(s, b, inst), rb1 = bound_r1(s, b, inst);
    if (dc < eps) return ra0 < rb1 - eps && rb0 < ra1 - eps;
    if (dc >= ra1 + rb1) return false;
  }
  // sampling test over the intersection of the two boxes
  double lo[3], hi[3];
  for (int i = 0; i < 3; ++i) { lo[i] = std::max(A.lo[i], B.lo[i]); hi[i] = std::min(A.hi[i], B.hi[i]); }
  const int n = 9;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        const double x[3] = {lo[0] + (hi[0] - lo[0]) * (i + 0.5) / n, lo[1] + (hi[1] - lo[1]) * (j + 0.5) / n,
                             lo[2] + (hi[2] - lo[2]) * (k + 0.5) / n};
        if (point_inside(s, a, inst, x, 1e-9) && point_inside(s, b, inst, x, 1e-9)) return true;
      }
  return false;
}

bool inside_world(const tp_scene* s, const tp_prim& p, int inst) {
  const Box3 b = aabb(s, p, inst);
  if (s->world_shape == TP_BOX) {
    for (int i = 0; i < 3; ++i)
      if (b.lo[i] <= s->world_c[i] - s->world_p[i] || b.hi[i] >= s->world_c[i] + s->world_p[i]) return false;
    return true;
  }
  double far2 = 0;
  for (int i = 0; i < 3; ++i) {
    const double e = std::max(std::fabs(b.lo[i] - s->world_c[i]), std::fabs(b.hi[i] - s->world_c[i]));
    far2 += e * e;
  }
  return std::sqrt(far2) < s->world_p[1];
}

tp_status validate_geometry(tp_scene* s) {
  const int np = (int)s->prims.size();
  // insts to check: every instance when the radius moves and the scene is small
  bool moving = false;
  for (const auto& p : s->prims) moving |= (p.bind_rmin || p.bind_rmax);
  const int ninst = (moving && np <= 64) ? s->n_inst : 1;
  for (int q = 0; q < ninst; ++q) {
    for (int i = 0; i < np; ++i) {
      const tp_prim& p = s->prims[i];
      if (p.shape != TP_BOX) {
        const double r0 = bound_r0(s, p, q), r1 = bound_r1(s, p, q);
        if (!(r0 >= 0.0) || !(r1 > r0))
          return fail(TP_ERR_GEOMETRY, "primitive %d (instance %d): radii %g..%g invalid", i, q, r0, r1);
      }
      if (!inside_world(s, p, q)) return fail(TP_ERR_GEOMETRY, "primitive %d (instance %d) not inside the world", i, q);
    }
    // pairwise: bounding-sphere rejection first
    std::vector<double> bc(3 * (size_t)np), br(np);
    for (int i = 0; i < np; ++i) {
      const Box3 b = aabb(s, s->prims[i], q);
      double r2 = 0;
      for (int k = 0; k < 3; ++k) {
        bc[3 * i + k] = 0.5 * (b.lo[k] + b.hi[k]);
        const double h = 0.5 * (b.hi[k] - b.lo[k]);
        r2 += h * h;
      }
      br[i] = std::sqrt(r2);
    }
    for (int i = 0; i < np; ++i)
      for (int j = i + 1; j < np; ++j) {
        const double dx = bc[3 * i] - bc[3 * j], dy = bc[3 * i + 1] - bc[3 * j + 1], dz = bc[3 * i + 2] - bc[3 * j + 2];
        if (dx * dx + dy * dy + dz * dz >= (br[i] + br[j]) * (br[i] + br[j])) continue;
        if (overlap(s, s->prims[i], s->prims[j], q))
          return fail(TP_ERR_GEOMETRY, "primitives %d and %d overlap (instance %d)", i, j, q);
      }
  }
  return TP_OK;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// ---------------------------------------------------------------------------
// Device scene tables in precision R
// ---------------------------------------------------------------------------
// Bounding radius about the centre over every instance, with a margin, and
// the lists of touching primitives (boxes grown by a tolerance intersect).
// True if no point of the box [lo, hi] is within m of primitive p (instance
// inst): apart from its bounding box, or -- for tubes and spheres -- wholly
// beyond the outer radius or wholly inside the inner one (a detector ring
// around the source).
bool box_clear_of(const tp_scene* s, const tp_prim& p, int inst, const double lo[3], const double hi[3], double m) {
  const Box3 b = aabb(s, p, inst);
  for (int k = 0; k < 3; ++k)
    if (hi[k] + m < b.lo[k] || lo[k] - m > b.hi[k]) return true;
  if (p.shape == TP_BOX) return false;
  // nearest and farthest distance of the box from the centre (sphere) or the axis (tube)
  double near2 = 0, far2 = 0;
  for (int k = 0; k < 3; ++k) {
    if (p.shape == TP_TUBE && k == p.axis) continue;
    const double a = lo[k] - p.centre[k], c = hi[k] - p.centre[k];
    const double nk = (a <= 0 && c >= 0) ? 0.0 : std::min(std::fabs(a), std::fabs(c));
    const double fk = std::max(std::fabs(a), std::fabs(c));
    near2 += nk * nk;
    far2 += fk * fk;
  }
  const double r0 = bound_r0(s, p, inst), r1 = bound_r1(s, p, inst);
  return std::sqrt(near2) >= r1 + m || (r0 > 0 && std::sqrt(far2) <= r0 - m);
}

void neighbours(const tp_scene* s, std::vector<double>& bound, std::vector<int>& off, std::vector<int>& cnt,
                std::vector<int>& list) {
  const int np = (int)s->prims.size();
  bool moving = false;
  for (const auto& p : s->prims) moving |= (p.bind_rmin || p.bind_rmax);
  const int ninst = moving ? s->n_inst : 1;
  bound.assign(np, 0.0);
  std::vector<Box3> box(np);
  for (int i = 0; i < np; ++i) {
    for (int q = 0; q < ninst; ++q) {
      const Box3 b = aabb(s, s->prims[i], q);
      double r2 = 0;
      for (int k = 0; k < 3; ++k) {
        const double h = std::max(std::fabs(b.hi[k] - s->prims[i].centre[k]), std::fabs(b.lo[k] - s->prims[i].centre[k]));
        r2 += h * h;
      }
      bound[i] = std::max(bound[i], std::sqrt(r2));
      if (q == 0) box[i] = b;
      for (int k = 0; k < 3; ++k) { box[i].lo[k] = std::min(box[i].lo[k], b.lo[k]); box[i].hi[k] = std::max(box[i].hi[k], b.hi[k]); }
    }
    double scale = 1.0;
    for (int k = 0; k < 3; ++k) scale = std::max(scale, std::fabs(s->prims[i].centre[k]));
    bound[i] = bound[i] * (1.0 + 1e-5) + 1e-5 * scale;
  }
  off.assign(np, 0);
  cnt.assign(np, 0);
  list.clear();
  for (int i = 0; i < np; ++i) {
    off[i] = (int)list.size();
    // i's box grown by more than the nudge past a surface: the point just
    // outside i lies in it
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      const double tol = 1e-4 * std::max({1.0, std::fabs(box[i].lo[k]), std::fabs(box[i].hi[k])});
      lo[k] = box[i].lo[k] - tol;
      hi[k] = box[i].hi[k] + tol;
    }
    double scale = 1.0;
    for (int k = 0; k < 3; ++k) scale = std::max(scale, std::fabs(s->prims[i].centre[k]));
    for (int j = 0; j < np; ++j) {
      if (j == i) continue;
      // the point lies within i's bounding sphere grown by the nudge: j's
      // bounding sphere must reach it
      double d2 = 0;
      for (int k = 0; k < 3; ++k) d2 += (s->prims[j].centre[k] - s->prims[i].centre[k]) * (s->prims[j].centre[k] - s->prims[i].centre[k]);
      if (std::sqrt(d2) > bound[i] + bound[j] + 1e-4 * scale) continue;
      // j may hold that point unless its solid keeps clear of the grown box
      // for every instance (apart, or -- a ring or shell about i -- i's box in
      // its hole)
      bool touch = false;
      for (int q = 0; q < ninst && !touch; ++q) touch = !box_clear_of(s, s->prims[j], q, lo, hi, 0.0);
      if (touch) list.push_back(j);
    }
    cnt[i] = (int)list.size() - off[i];
  }
}

// True if every point the gun can start a neutron at -- the rectangle centre
// +- half at the source plane, or the pencil's point -- lies inside the world
// and outside the bounding box of every primitive (every instance), with a
// margin far above the transport precision's rounding: the source volume is
// then the world region without a point location.
bool source_in_free_space(const tp_scene* s) {
  const tp_source& g = s->source;
  double lo[3], hi[3];
  for (int k = 0; k < 3; ++k) lo[k] = hi[k] = g.centre[k];
  if (g.kind != TP_SRC_PENCIL)
    for (int k = 0; k < 2; ++k) { lo[k] -= g.half[k]; hi[k] += g.half[k]; }
  double scale = 1.0;
  for (int k = 0; k < 3; ++k) scale = std::max({scale, std::fabs(lo[k]), std::fabs(hi[k])});
  const double m = 1e-4 * scale;
  if (s->world_shape == TP_BOX) {
    for (int k = 0; k < 3; ++k)
      if (lo[k] - m <= s->world_c[k] - s->world_p[k] || hi[k] + m >= s->world_c[k] + s->world_p[k]) return false;
  } else {
    double f2 = 0;
    for (int k = 0; k < 3; ++k) {
      const double e = std::max(std::fabs(lo[k] - s->world_c[k]), std::fabs(hi[k] - s->world_c[k])) + m;
      f2 += e * e;
    }
    if (std::sqrt(f2) >= s->world_p[1]) return false;
  }
  bool moving = false;
  for (const auto& p : s->prims) moving |= (p.bind_rmin || p.bind_rmax);
  const int ninst = moving ? s->n_inst : 1;
  for (const auto& p : s->prims)
    for (int q = 0; q < ninst; ++q)
      if (!box_clear_of(s, p, q, lo, hi, m)) return false;
  return true;
}

template <typename R>
std::vector<uint8_t> build_blob(tp_scene* s) {
  s->src_free = source_in_free_space(s) ? 1 : 0;
  const int np = (int)s->prims.size(), nm = (int)s->mats.size(), nmir = (int)s->mirrors.size(),
            nch = (int)s->choppers.size(), nt = (int)s->tallies.size();
  int nl = 0;
  for (const auto& m : s->mats) nl += (int)m.d.size();
  std::vector<double> bound;
  std::vector<int> nb_off, nb_cnt, nb_list;
  neighbours(s, bound, nb_off, nb_cnt, nb_list);
  size_t off = 0;
  s->off_prims = (uint32_t)off; off = align16(off + sizeof(DPrim<R>) * np);
  s->off_mats = (uint32_t)off; off = align16(off + sizeof(DMat<R>) * std::max(nm, 1));
  s->off_mirrors = (uint32_t)off; off = align16(off + sizeof(DMirror<R>) * std::max(nmir, 1));
  s->off_choppers = (uint32_t)off; off = align16(off + sizeof(DChopper<R>) * std::max(nch, 1));
  s->off_tallies = (uint32_t)off; off = align16(off + sizeof(DTally<R>) * std::max(nt, 1));
  s->off_line_d = (uint32_t)off; off = align16(off + sizeof(R) * std::max(nl, 1));
  s->off_line_cum = (uint32_t)off; off = align16(off + sizeof(R) * (nl + std::max(nm, 1)));
  s->off_nb = (uint32_t)off; off = align16(off + sizeof(int) * std::max<size_t>(nb_list.size(), 1));
  std::vector<uint8_t> blob(off, 0);
  if (!nb_list.empty()) std::memcpy(blob.data() + s->off_nb, nb_list.data(), nb_list.size() * sizeof(int));
  auto* P = reinterpret_cast<DPrim<R>*>(blob.data() + s->off_prims);
  for (int i = 0; i < np; ++i) {
    const tp_prim& p = s->prims[i];
    DPrim<R> d{};
    for (int k = 0; k < 3; ++k) { d.c[k] = (R)p.centre[k]; d.p[k] = (R)p.params[k]; }
    d.shape = p.shape; d.axis = p.axis; d.material = p.material; d.role = p.role;
    d.mirror = p.mirror; d.flags = (p.bind_rmin ? F_BIND_RMIN : 0) | (p.bind_rmax ? F_BIND_RMAX : 0);
    if (p.chopper >= 0) d.flags |= F_CHOPPER | (p.chopper << kChopperShift);
    d.entry_mask = 0; d.exit_mask = 0;
    d.bound_r = (R)bound[i];
    d.nb_off = nb_off[i];
    d.nb_cnt = nb_cnt[i];
    for (int t = 0; t < nt; ++t) {
      if (s->tallies[t].volume != i) continue;
      if (s->tallies[t].trigger == TP_PTS_ENTRY) d.entry_mask |= 1 << t;
      else d.exit_mask |= 1 << t;
    }
    P[i] = d;
  }
  auto* M = reinterpret_cast<DMat<R>*>(blob.data() + s->off_mats);
  auto* LD = reinterpret_cast<R*>(blob.data() + s->off_line_d);
  auto* LC = reinterpret_cast<R*>(blob.data() + s->off_line_cum);
  int lo = 0;
  for (int i = 0; i < nm; ++i) {
    const Mat& m = s->mats[i];
    DMat<R> d{};
    d.sig_abs_ref = (R)m.m.sigma_abs_ref;
    d.sig_inc = (R)m.m.sigma_inc;
    d.bragg_pref = m.d.empty() ? R(0) : (R)(1.0 / (2.0 * m.m.V0 * m.m.V0));
    for (int k = 0; k < TP_NPROC; ++k) d.g[k] = (R)m.g[k];
    d.abs_1v = m.m.abs_1v;
    d.nlines = (int)m.d.size();
    d.line_off = lo;
    d.cum_off = lo + i;
    d.density_par = m.m.density_param;
    d.scale_par = m.m.scale_param;
    double acc = 0.0;
    LC[d.cum_off] = R(0);
    for (int k = 0; k < d.nlines; ++k) {
      LD[lo + k] = (R)m.d[k];
      acc += m.mult[k] * m.F2[k] * m.d[k];
      LC[d.cum_off + k + 1] = (R)acc;
    }
    lo += d.nlines;
    M[i] = d;
  }
  auto* MI = reinterpret_cast<DMirror<R>*>(blob.data() + s->off_mirrors);
  for (int i = 0; i < nmir; ++i) {
    const tp_mirror& m = s->mirrors[i];
    MI[i] = DMirror<R>{(R)m.m, (R)m.R0, (R)m.Qc, (R)m.alpha, (R)m.W, (R)(m.m * m.Qc), R(0), R(0)};
  }
  auto* CH = reinterpret_cast<DChopper<R>*>(blob.data() + s->off_choppers);
  for (int i = 0; i < nch; ++i) {
    const tp_chopper& c = s->choppers[i];
    const double n = c.n_windows, two_pi = 2.0 * M_PI;
    CH[i] = DChopper<R>{(R)(c.r_black * c.r_black), (R)(n / two_pi), (R)(n * c.freq), (R)(n * c.phase / two_pi),
                        (R)(n * c.theta0 / (2.0 * two_pi)), R(0), R(0), R(0)};
  }
  auto* T = reinterpret_cast<DTally<R>*>(blob.data() + s->off_tallies);
  for (int t = 0; t < nt; ++t) {
    const tp_tally_desc& d = s->tallies[t];
    DTally<R> x{};
    for (int k = 0; k < 2; ++k) {
      x.lo[k] = (R)d.lo[k];
      x.hi[k] = (R)d.hi[k];
      x.inv_w[k] = (R)(d.nbins[k] / (d.hi[k] - d.lo[k]));
    }
    double an = std::sqrt(d.axis[0] * d.axis[0] + d.axis[1] * d.axis[1] + d.axis[2] * d.axis[2]);
    if (!(an > 0)) an = 1.0;
    for (int k = 0; k < 3; ++k) { x.origin[k] = (R)d.origin[k]; x.axis[k] = (R)(d.axis[k] / an); }
    x.kind = d.kind; x.trigger = d.trigger; x.volume = d.volume; x.face = d.face; x.scat = d.scat;
    x.nb0 = d.nbins[0]; x.nb1 = d.nbins[1]; x.offset = s->tally_off[t];
    T[t] = x;
  }
  return blob;
}

constexpr int kGridMinPrims = 24;
// Cells per primitive of the uniform grid: one walks fewer cells per flight
// than finer grids at little cost in primitives per cell (the fastest of 0.5
// to 32 on the 1000-primitive scene).
constexpr double kGridCellsPerPrim = 1.0;

// Uniform grid over the bounding box of the primitives, about one cell per
// primitive with cubic cells; each cell lists the primitives whose bounding box
// (over every instance) meets it.
tp_status upload_grid(tp_scene* s) {
  if (s->d_grid) { cudaFree(s->d_grid); s->d_grid = nullptr; }
  s->grid_cells = 0;
  const int np = (int)s->prims.size();
  if (np < kGridMinPrims) return TP_OK;
  bool moving = false;
  for (const auto& p : s->prims) moving |= (p.bind_rmin || p.bind_rmax);
  const int ninst = moving ? s->n_inst : 1;
  std::vector<Box3> box(np);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < np; ++i) {
    box[i] = aabb(s, s->prims[i], 0);
    for (int q = 1; q < ninst; ++q) {
      const Box3 b = aabb(s, s->prims[i], q);
      for (int k = 0; k < 3; ++k) { box[i].lo[k] = std::min(box[i].lo[k], b.lo[k]); box[i].hi[k] = std::max(box[i].hi[k], b.hi[k]); }
    }
    for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], box[i].lo[k]); hi[k] = std::max(hi[k], box[i].hi[k]); }
  }
  double vol = 1.0;
  for (int k = 0; k < 3; ++k) {
    const double pad = 1e-4 * std::max(1.0, hi[k] - lo[k]);
    lo[k] -= pad; hi[k] += pad;
    vol *= hi[k] - lo[k];
  }
  const double h = std::cbrt(vol / (kGridCellsPerPrim * np));
  // pad every box by a small fraction of a cell so that rounding at cell faces
  // during the walk cannot skip a primitive
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < 3; ++k) { box[i].lo[k] -= 1e-3 * h; box[i].hi[k] += 1e-3 * h; }
  // and a sphere about each centre holding the primitive (every instance),
  // padded alike: a cell that its box meets but its sphere misses (a box
  // corner of a sphere, cylinder or tilted-looking box) does not list it
  std::vector<double> ball(np, 0.0);
  for (int i = 0; i < np; ++i) {
    double r2 = 0;
    for (int k = 0; k < 3; ++k) {
      const double e = std::max(box[i].hi[k] - s->prims[i].centre[k], s->prims[i].centre[k] - box[i].lo[k]);
      r2 += e * e;
    }
    ball[i] = std::sqrt(r2);
    if (s->prims[i].shape != TP_BOX) {   // a tube or sphere: its own radius bounds it more tightly
      double rmax = 0;
      for (int q = 0; q < ninst; ++q) rmax = std::max(rmax, bound_r1(s, s->prims[i], q));
      const double hh = s->prims[i].shape == TP_TUBE ? s->prims[i].params[2] : 0.0;
      ball[i] = std::min(ball[i], std::sqrt(rmax * rmax + hh * hh) + 2e-3 * h);
    }
  }
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    s->grid_n[k] = (int)std::max(1.0, std::min(256.0, std::round((hi[k] - lo[k]) / h)));
    ncell *= s->grid_n[k];
    s->grid_lo[k] = lo[k];
    s->grid_hi[k] = hi[k];
  }
  std::vector<int> count(ncell + 1, 0);
  auto range = [&](const Box3& b, int k, int* a0, int* a1) {
    const double inv = s->grid_n[k] / (s->grid_hi[k] - s->grid_lo[k]);
    *a0 = std::max(0, std::min(s->grid_n[k] - 1, (int)std::floor((b.lo[k] - s->grid_lo[k]) * inv)));
    *a1 = std::max(0, std::min(s->grid_n[k] - 1, (int)std::floor((b.hi[k] - s->grid_lo[k]) * inv)));
  };
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int> fill;
    if (pass == 1) {
      for (long long c = 0; c < ncell; ++c) count[c + 1] += count[c];
      fill.assign(count.begin(), count.end() - 1);
    }
    std::vector<int> items(pass == 1 ? count[ncell] : 0);
    for (int i = 0; i < np; ++i) {
      int r[3][2];
      for (int k = 0; k < 3; ++k) range(box[i], k, &r[k][0], &r[k][1]);
      for (int a = r[0][0]; a <= r[0][1]; ++a)
        for (int b = r[1][0]; b <= r[1][1]; ++b)
          for (int c = r[2][0]; c <= r[2][1]; ++c) {
            const int ic[3] = {a, b, c};
            double d2 = 0;   // squared distance from the centre to the cell
            for (int k = 0; k < 3; ++k) {
              const double w = (s->grid_hi[k] - s->grid_lo[k]) / s->grid_n[k];
              const double lo = s->grid_lo[k] + ic[k] * w, hi = lo + w;
              const double x = s->prims[i].centre[k];
              const double e = x < lo ? lo - x : (x > hi ? x - hi : 0.0);
              d2 += e * e;
            }
            if (std::sqrt(d2) > ball[i]) continue;
            const long long cell = ((long long)a * s->grid_n[1] + b) * s->grid_n[2] + c;
            if (pass == 0) count[cell + 1]++;
            else items[fill[cell]++] = i;
          }
    }
    if (pass == 1) {
      std::vector<int> all(count.begin(), count.end());
      all.insert(all.end(), items.begin(), items.end());
      TP_CUDA(cudaMalloc(&s->d_grid, all.size() * sizeof(int)));
      TP_CUDA(cudaMemcpy(s->d_grid, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  s->grid_cells = (int)ncell;
  return TP_OK;
}

tp_status upload_blob(tp_scene* s) {
  tp_status gst = upload_grid(s);
  if (gst != TP_OK) return gst;
  std::vector<uint8_t> blob = s->precision == TP_FP64 ? build_blob<double>(s) : build_blob<float>(s);
  if (blob.size() > s->blob_cap) {
    if (s->d_blob) cudaFree(s->d_blob);
    s->d_blob = nullptr;
    TP_CUDA(cudaMalloc(&s->d_blob, blob.size()));
    s->blob_cap = blob.size();
  }
  TP_CUDA(cudaMemcpy(s->d_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  s->blob_bytes = (uint32_t)blob.size();
  s->blob_dirty = false;
  return TP_OK;
}

constexpr uint32_t kMaxStagedBlob = 96 * 1024;  // larger tables are read through L1/L2
// The sparse regrouping interval the autotuner tries beside regrouping every
// event (event kernel, plain runs).
constexpr int kRegroupSparse = 4;

template <typename R>
void fill_common(const tp_scene* s, KParams<R>& k) {
  k.blob = s->d_blob;
  k.blob_bytes = s->blob_bytes;
  k.off_prims = s->off_prims; k.off_mats = s->off_mats; k.off_mirrors = s->off_mirrors;
  k.off_choppers = s->off_choppers;
  k.off_tallies = s->off_tallies; k.off_line_d = s->off_line_d; k.off_line_cum = s->off_line_cum;
  k.off_nb = s->off_nb;
  k.stage_blob = s->blob_bytes <= kMaxStagedBlob ? 1 : 0;
  k.nprim = (int)s->prims.size();
  k.nmat = (int)s->mats.size();
  k.ntally = (int)s->tallies.size();
  k.npar = s->n_par;
  k.radius_par = -1;
  for (int i = 0; i < kMaxPar; ++i) k.param_kind[i] = i < s->n_par ? s->param_kind[i] : -1;
  for (int i = 0; i < s->n_par; ++i)
    if (s->param_kind[i] == TP_PAR_RADIUS) k.radius_par = i;
  k.radius_nominal = (R)s->radius_nominal;
  k.world_shape = s->world_shape;
  for (int i = 0; i < 3; ++i) { k.world_c[i] = (R)s->world_c[i]; k.world_p[i] = (R)s->world_p[i]; }
  k.world_entry_mask = 0;
  k.world_exit_mask = 0;
  for (int t = 0; t < (int)s->tallies.size(); ++t)
    if (s->tallies[t].volume == -1) {
      if (s->tallies[t].trigger == TP_PTS_EXIT) k.world_exit_mask |= 1 << t;
      else k.world_entry_mask |= 1 << t;
    }
  const tp_source& src = s->source;
  k.src_kind = src.kind;
  k.src_aperture = src.has_aperture;
  for (int i = 0; i < 3; ++i) k.src_c[i] = (R)src.centre[i];
  for (int i = 0; i < 2; ++i) {
    k.src_half[i] = (R)src.half[i];
    k.src_div[i] = (R)src.div[i];
    k.src_ap[i] = (R)src.aperture[i];
  }
  k.src_lam_lo = (R)src.lambda_lo;
  k.src_lam_hi = (R)src.lambda_hi;
  k.src_slit_z = (R)src.slit_z;
  k.src_slit_half[0] = (R)src.slit_half[0];
  k.src_slit_half[1] = (R)src.slit_half[1];
  k.src_kT = (R)(kBoltzmann_meV * src.temperature);
  k.src_free = s->src_free;
  k.event_cap = s->event_cap;
  k.use_grid = s->grid_cells > 0 ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    k.grid_n[i] = s->grid_n[i];
    k.grid_lo[i] = (R)s->grid_lo[i];
    k.grid_hi[i] = (R)s->grid_hi[i];
    k.grid_cell[i] = s->grid_n[i] > 0 ? (R)((s->grid_hi[i] - s->grid_lo[i]) / s->grid_n[i]) : R(1);
    k.grid_inv[i] = s->grid_n[i] > 0 ? (R)(s->grid_n[i] / (s->grid_hi[i] - s->grid_lo[i])) : R(0);
  }
  k.grid_start = s->d_grid;
  k.grid_items = s->d_grid ? s->d_grid + s->grid_cells + 1 : nullptr;
  k.n_inst = s->n_inst;
  k.inst_prefix = s->d_prefix;
  k.inst_first = s->d_first;
  k.inst_params = static_cast<const R*>(s->d_params);
  k.work_counter = s->d_work;
  k.sum = s->d_sum; k.sumsq = s->d_sumsq; k.J = s->d_J; k.J2 = s->d_J2;
  k.total_bins = s->total_bins;
  k.counters = s->d_counters;
  k.status = s->d_status;
  k.abort_flag = s->d_abort;
  k.test_flags = s->test_flags;
}

size_t smem_bytes(const tp_scene* s) { return s->blob_bytes <= kMaxStagedBlob ? align16(s->blob_bytes) : 0; }

tp_status pick_launch(tp_scene* s, bool grad, int req_block, int req_ctas, int* block, int* ctas) {
  int b = req_block > 0 ? req_block : (s->block > 0 ? s->block : 256);
  if (b % 32 != 0 || b < 32 || b > 256) return fail(TP_ERR_INVALID_ARG, "block_size %d: need a multiple of 32 in [32, 256]", b);
  int occ = 0;
  TP_CUDA(occupancy_transport(TP_KERNEL_HISTORY | (s->full ? kVariantFull : 0), s->precision, grad,
                              s->grid_cells > 0, b, smem_bytes(s), &occ));
  if (occ < 1) return fail(TP_ERR_INVALID_ARG, "block_size %d does not fit on an SM", b);
  int c = req_ctas > 0 ? std::min(req_ctas, occ) : occ;
  *block = b;
  *ctas = c;
  return TP_OK;
}

size_t smem_variant(const tp_scene* s, int variant, bool grad, int block, int stage) {
  return (stage ? align16(s->blob_bytes) : 0) + align16(bank_bytes(variant, s->precision, grad, block));
}

// Tables larger than this are offered to the autotuner unstaged as well
// (read through L1/L2), which leaves room for more blocks per SM.
constexpr uint32_t kStageChoiceBytes = 16 * 1024;

// Completes a launch configuration (CTAs per SM from the occupancy).
// stage: -1 = stage the tables when they fit (<= kMaxStagedBlob).
// hi: -1 = the 80-register build unless req_ctas asks for more CTAs per SM
// than it allows and the 64-register build allows more; 0 / 1 = that build.
tp_status resolve(tp_scene* s, bool grad, int kernel, int req_block, int req_ctas, LaunchCfg* c, int stage = -1,
                  int hi = -1) {
  const int b = req_block > 0 ? req_block : 256;
  if (b % 32 != 0 || b < 32 || b > 256)
    return fail(TP_ERR_INVALID_ARG, "kernel %d block_size %d: need a multiple of 32 in [32, 256]", kernel, b);
  if (s->smem_optin == 0) {
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    TP_CUDA(cudaDeviceGetAttribute(&s->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  }
  const size_t limit = (size_t)s->smem_optin;
  // stage the tables when they are small enough and fit beside the neutron bank
  if (stage < 0) stage = s->blob_bytes <= kMaxStagedBlob && smem_variant(s, kernel, grad, b, 1) <= limit ? 1 : 0;
  if (stage && s->blob_bytes > kMaxStagedBlob) return fail(TP_ERR_INVALID_ARG, "tables too large to stage");
  if (smem_variant(s, kernel, grad, b, stage) > limit)
    return fail(TP_ERR_INVALID_ARG, "kernel %d block_size %d needs %zu bytes of shared memory; a block may use %zu",
                kernel, b, smem_variant(s, kernel, grad, b, stage), limit);
  const bool can_hi = s->precision == TP_FP32;
  if (hi > 0 && !can_hi) return fail(TP_ERR_INVALID_ARG, "the 64-register build serves FP32 runs only");
  int h = hi > 0 ? 1 : 0, occ = 0;
  const size_t sm = smem_variant(s, kernel, grad, b, stage);
  const int fbit = s->full ? kVariantFull : 0;
  TP_CUDA(occupancy_transport(kernel | (h ? kVariantHighOcc : 0) | fbit, s->precision, grad, s->grid_cells > 0, b, sm, &occ));
  if (hi < 0 && can_hi && req_ctas > occ) {
    int occ_hi = 0;
    TP_CUDA(occupancy_transport(kernel | kVariantHighOcc | fbit, s->precision, grad, s->grid_cells > 0, b, sm, &occ_hi));
    if (occ_hi > occ) { h = 1; occ = occ_hi; }
  }
  if (occ < 1) return fail(TP_ERR_INVALID_ARG, "kernel %d block_size %d does not fit on an SM", kernel, b);
  *c = LaunchCfg{kernel, b, req_ctas > 0 ? std::min(req_ctas, occ) : occ, stage, h, 0, s->full};
  return TP_OK;
}

struct Outputs {
  double *sum, *sumsq, *J, *J2;
  unsigned long long* counters;
};

// One launch.  sec_mode: see KParams; index_base: global index of its first
// history (a chunk of a longer run).
template <typename R>
cudaError_t launch_one(tp_scene* s, const LaunchCfg& c, bool grad, uint64_t seed, unsigned long long total,
                       tp_record* records, unsigned long long n_records, const Outputs& o, cudaStream_t st,
                       int sec_mode = 0, unsigned long long index_base = 0) {
  KParams<R> k{};
  fill_common(s, k);
  k.sec_mode = sec_mode;
  k.sec_buf = s->d_sec;
  k.sec_count = s->d_sec_count;
  k.sec_cap = s->sec_cap;
  k.index_base = index_base;
  k.key0 = (uint32_t)(seed & 0xffffffffu);
  k.key1 = (uint32_t)(seed >> 32);
  k.total = total;
  k.records = records;
  k.n_records = records ? n_records : 0;
  k.sum = o.sum; k.sumsq = o.sumsq; k.J = o.J; k.J2 = o.J2; k.counters = o.counters;
  k.stage_blob = c.stage;
  k.regroup = c.regroup;
  const int grid = s->sm_count * c.ctas;
  const long long warps = (long long)grid * (c.block / 32);
  k.chunk = sec_mode == 2 ? 16 : (int)std::max(1ll, std::min(256ll, (long long)(total / (unsigned long long)(warps * 8))));
  cudaError_t e = cudaMemsetAsync(s->d_work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const size_t sm = smem_variant(s, c.kernel, grad, c.block, c.stage);
  if constexpr (std::is_same<R, double>::value) return launch_transport_f64(k, c.variant(), grad, grid, c.block, sm, st);
  else return launch_transport_f32(k, c.variant(), grad, grid, c.block, sm, st);
}

// Histories a chunk of a queued-secondaries run may hold: the queue takes
// kSecPerHistory secondaries per history (the batched powder workload makes
// 3.5 on average); a fuller queue transports the rest in place.  Records are
// 56 bytes in FP32, so the largest queue (2^31) holds 120 GB: the 5.9e8
// histories of the batched workload go through in two chunks.
constexpr unsigned long long kSecPerHistory = 6;
constexpr unsigned long long kSecCapMin = 1ull << 16, kSecCapMax = 1ull << 31;

// The queue of secondaries for runs of up to `total` histories (allocated
// outside any stream capture; a larger one drops the captured graph).
tp_status ensure_sec(tp_scene* s, unsigned long long total) {
  // at most half of the free device memory
  size_t free_b = 0, total_b = 0;
  TP_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const unsigned long long mem_cap = (unsigned long long)(free_b / 2 / particle_bytes(s->precision));
  const unsigned long long cap = (s->test_flags & TP_TEST_SMALL_SEC_QUEUE) ? (1ull << 20) : kSecCapMax;
  unsigned long long want = kSecCapMin;
  while (want < cap && want < kSecPerHistory * total && 2 * want <= mem_cap) want <<= 1;
  if (s->sec_cfg.kernel == 0) {
    tp_status st = resolve(s, false, TP_KERNEL_WARPQ, 256, 0, &s->sec_cfg, -1, s->precision == TP_FP32 ? 1 : 0);
    if (st != TP_OK) return st;
  }
  if (s->d_sec && s->sec_cap >= want && s->sec_cap <= cap) return TP_OK;
  if (s->stage_pending) { TP_CUDA(cudaEventSynchronize(s->stage_done)); s->stage_pending = false; }
  TP_CUDA(cudaDeviceSynchronize());
  cudaFree(s->d_sec);
  s->d_sec = nullptr;
  s->sec_cap = 0;
  if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
  TP_CUDA(cudaMalloc(&s->d_sec, want * particle_bytes(s->precision)));
  if (!s->d_sec_count) TP_CUDA(cudaMalloc(&s->d_sec_count, sizeof(unsigned long long)));
  s->sec_cap = want;
  return TP_OK;
}

// The launch (or, for queued secondaries, the sequence of launches) of a run:
// chunks of histories whose secondaries fit the queue, each followed by a
// second pass of the plain warp-pool kernel over the queue.
template <typename R>
cudaError_t launch_run(tp_scene* s, const LaunchCfg& c, bool grad, uint64_t seed, unsigned long long total,
                       tp_record* records, unsigned long long n_records, const Outputs& o, cudaStream_t st) {
  if (!grad || !c.defer) return launch_one<R>(s, c, grad, seed, total, records, n_records, o, st);
  if (!s->d_sec || s->sec_cfg.kernel == 0) return cudaErrorInvalidValue;   // ensure_sec comes first
  const LaunchCfg& sc = s->sec_cfg;
  const unsigned long long chunk = std::max(1ull, s->sec_cap / kSecPerHistory);
  for (unsigned long long c0 = 0; c0 < total; c0 += chunk) {
    const unsigned long long n = std::min(chunk, total - c0);
    cudaError_t e = cudaMemsetAsync(s->d_sec_count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_one<R>(s, c, true, seed, n, records, n_records, o, st, 1, c0);
    if (e == cudaSuccess) e = launch_one<R>(s, sc, false, seed, 0, nullptr, 0, o, st, 2, 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_cfg(tp_scene* s, const LaunchCfg& c, bool grad, uint64_t seed, unsigned long long total,
                       tp_record* records, unsigned long long n_records, const Outputs& o, cudaStream_t st) {
  if (s->precision == TP_FP64) return launch_run<double>(s, c, grad, seed, total, records, n_records, o, st);
  return launch_run<float>(s, c, grad, seed, total, records, n_records, o, st);
}

// Times every candidate (kernel, block size) on up to 2^22 of this run's
// histories, scoring into scratch tallies, and keeps the fastest.
// Times every launch candidate on scratch tallies in two rounds: all of them
// on up to 2^22 histories, then the four fastest on up to 2^25 (short trials
// of fast scenes are dominated by the launch and the tail of the last wave).
tp_status autotune(tp_scene* s, bool grad, uint64_t seed, unsigned long long total, cudaStream_t st) {
  const size_t nb = (size_t)s->n_inst * std::max(1, s->total_bins);
  const size_t per = grad ? 2 + 2 * (size_t)s->n_par : 2;
  double* scratch = nullptr;
  unsigned long long* cnt = nullptr;
  TP_CUDA(cudaMalloc(&scratch, per * nb * sizeof(double)));
  cudaError_t ce = cudaMalloc(&cnt, kNumCounters * sizeof(unsigned long long));
  if (ce != cudaSuccess) { cudaFree(scratch); return fail(TP_ERR_OOM, "autotune scratch"); }
  Outputs o{scratch, scratch + nb, grad ? scratch + 2 * nb : nullptr,
            grad ? scratch + (2 + s->n_par) * nb : nullptr, cnt};
  const int cand[][2] = {{TP_KERNEL_EVENT, 256}, {TP_KERNEL_EVENT, 128}, {TP_KERNEL_HISTORY, 128},
                         {TP_KERNEL_HISTORY, 256}, {TP_KERNEL_WARPQ, 256}, {TP_KERNEL_WARPQ, 128}};
  const int nhi = s->precision == TP_FP32 ? 2 : 1;   // both register builds
  const int nstage = s->blob_bytes > kStageChoiceBytes && s->blob_bytes <= kMaxStagedBlob ? 2 : 1;
  std::vector<LaunchCfg> cfgs;
  for (int ci = 0; ci < (int)(sizeof cand / sizeof cand[0]) * nstage * nhi; ++ci) {
    const int* c = cand[ci / (nstage * nhi)];
    const int stage = nstage == 2 ? ((ci / nhi) % 2 == 0 ? 1 : 0) : -1;
    LaunchCfg cfg;
    if (resolve(s, grad, c[0], c[1], 0, &cfg, stage, ci % nhi) != TP_OK) continue;   // does not fit
    cfgs.push_back(cfg);
    if (grad && s->d_sec) {   // and with the secondaries queued for a second pass
      cfg.defer = 1;
      cfgs.push_back(cfg);
    }
    if (!grad && c[0] == TP_KERNEL_EVENT) {   // and regrouped every kRegroupSparse events
      cfg.regroup = kRegroupSparse;
      cfgs.push_back(cfg);
    }
  }
  if (cfgs.empty()) {
    cudaFree(scratch);
    cudaFree(cnt);
    return fail(TP_ERR_INVALID_ARG, "no launch configuration fits");
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  tp_status result = TP_OK;
  std::vector<float> ms(cfgs.size(), 1e30f);
  auto time_all = [&](const std::vector<int>& which, unsigned long long trial) {
    for (int i : which) {
      for (int rep = 0; rep < 2; ++rep) {   // the first repetition warms up
        cudaEventRecord(a, st);
        ce = launch_cfg(s, cfgs[i], grad, seed, trial, nullptr, 0, o, st);
        cudaEventRecord(b, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(b);
        if (ce != cudaSuccess) return false;
      }
      cudaEventElapsedTime(&ms[i], a, b);
    }
    return true;
  };
  std::vector<int> order(cfgs.size());
  std::iota(order.begin(), order.end(), 0);
  const unsigned long long trial1 = std::min(total, 1ull << 22), trial2 = std::min(total, 1ull << 25);
  bool ok = time_all(order, trial1);
  if (ok && trial2 > trial1 && order.size() > 1) {
    std::sort(order.begin(), order.end(), [&](int x, int y) { return ms[x] < ms[y]; });
    order.resize(std::min<size_t>(4, order.size()));
    ok = time_all(order, trial2);
  }
  if (!ok) result = fail(TP_ERR_CUDA, "autotune: %s", cudaGetErrorString(ce));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(scratch);
  cudaFree(cnt);
  if (result != TP_OK) return result;
  const int best = *std::min_element(order.begin(), order.end(), [&](int x, int y) { return ms[x] < ms[y]; });
  const LaunchCfg& pick = cfgs[best];
  s->tuned_kernel[grad] = pick.kernel;
  s->tuned_block[grad] = pick.block;
  s->tuned_stage[grad] = pick.stage;
  s->tuned_hi[grad] = pick.hi;
  s->tuned_regroup[grad] = pick.regroup;
  if (grad) s->tuned_defer = pick.defer;
  return TP_OK;
}

// Runs [work-description copies, work-counter reset, kernel] as a CUDA graph,
// captured on a private stream the first time a launch key is seen and
// replayed on `st` afterwards.  The copies read the pinned staging buffer at
// replay time, so counts and first ids may change between replays.
tp_status run_graph(tp_scene* s, const LaunchCfg& cfg, bool grad, const tp_run* r, unsigned long long total,
                    const Outputs& o, cudaStream_t st) {
  const unsigned long long key[8] = {(unsigned long long)cfg.variant(), (unsigned long long)cfg.block,
                                     (unsigned long long)(cfg.ctas * 256 + cfg.regroup * 4 + cfg.stage * 2 + cfg.defer),
                                     (unsigned long long)grad,
                                     r->seed, total,
                                     (unsigned long long)(uintptr_t)r->records, r->records ? r->n_records : 0};
  if (!s->graph || std::memcmp(key, s->graph_key, sizeof key) != 0) {
    if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
    if (!s->capture_stream) TP_CUDA(cudaStreamCreateWithFlags(&s->capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = s->capture_stream;
    TP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaMemcpyAsync(s->d_prefix, s->h_stage, (s->n_inst + 1) * sizeof(unsigned long long),
                                     cudaMemcpyHostToDevice, cs);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(s->d_first, s->h_stage + s->n_inst + 1, s->n_inst * sizeof(unsigned long long),
                           cudaMemcpyHostToDevice, cs);
    if (ce == cudaSuccess) ce = launch_cfg(s, cfg, grad, r->seed, total, r->records, r->n_records, o, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &g);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&s->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ce != cudaSuccess) { s->graph = nullptr; return fail(TP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce)); }
    std::memcpy(s->graph_key, key, sizeof key);
  }
  TP_CUDA(cudaGraphLaunch(s->graph, st));
  TP_CUDA(cudaEventRecord(s->stage_done, st));
  s->stage_pending = true;
  return TP_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

// Checks a scene description and copies it into the host side of *s (no
// device work).  Shared by tp_create_scene and the allocation-free call.
static tp_status describe(const tp_scene_desc* d, tp_scene* s) {
  if (d->precision != TP_FP32 && d->precision != TP_FP64) return fail(TP_ERR_INVALID_ARG, "precision %d", d->precision);
  if (d->world_shape != TP_BOX && d->world_shape != TP_SPHERE) return fail(TP_ERR_INVALID_ARG, "world shape %d", d->world_shape);
  if (!finite_all(d->world_centre, 3) || !finite_all(d->world_params, 3)) return fail(TP_ERR_INVALID_ARG, "world not finite");
  if (d->world_shape == TP_BOX && !(d->world_params[0] > 0 && d->world_params[1] > 0 && d->world_params[2] > 0))
    return fail(TP_ERR_INVALID_ARG, "world half extents must be positive");
  if (d->world_shape == TP_SPHERE && !(d->world_params[1] > 0)) return fail(TP_ERR_INVALID_ARG, "world radius must be positive");
  if (d->n_prims < 0 || (d->n_prims > 0 && !d->prims)) return fail(TP_ERR_INVALID_ARG, "prims");
  if (d->n_prims > TP_MAX_PRIMS) return fail(TP_ERR_INVALID_ARG, "%d primitives: at most %d", d->n_prims, TP_MAX_PRIMS);
  if (d->n_mirrors < 0 || (d->n_mirrors > 0 && !d->mirrors)) return fail(TP_ERR_INVALID_ARG, "mirrors");
  if (d->n_choppers < 0 || (d->n_choppers > 0 && !d->choppers)) return fail(TP_ERR_INVALID_ARG, "choppers");
  if (d->n_tallies < 0 || d->n_tallies > TP_MAX_TALLIES || (d->n_tallies > 0 && !d->tallies))
    return fail(TP_ERR_INVALID_ARG, "n_tallies %d (max %d)", d->n_tallies, TP_MAX_TALLIES);
  if (d->n_instances < 1) return fail(TP_ERR_INVALID_ARG, "n_instances must be >= 1");
  if (d->n_params < 0 || d->n_params > TP_MAX_PARAMS) return fail(TP_ERR_INVALID_ARG, "n_params %d (max %d)", d->n_params, TP_MAX_PARAMS);
  if (d->n_params > 0 && (!d->inst_params || !d->param_kind)) return fail(TP_ERR_INVALID_ARG, "inst_params / param_kind");
  if (d->event_cap < 0) return fail(TP_ERR_INVALID_ARG, "event_cap");

  s->precision = d->precision;
  s->event_cap = d->event_cap > 0 ? d->event_cap : 4096;
  s->world_shape = d->world_shape;
  for (int i = 0; i < 3; ++i) { s->world_c[i] = d->world_centre[i]; s->world_p[i] = d->world_params[i]; }
  s->prims.assign(d->prims, d->prims + d->n_prims);
  s->mirrors.assign(d->mirrors, d->mirrors + d->n_mirrors);
  s->choppers.assign(d->choppers, d->choppers + d->n_choppers);
  s->source = d->source;
  s->tallies.assign(d->tallies, d->tallies + d->n_tallies);
  s->n_inst = d->n_instances;
  s->n_par = d->n_params;
  s->param_kind.assign(d->param_kind, d->param_kind + d->n_params);
  s->radius_nominal = d->radius_nominal;
  s->inst_params.assign((size_t)s->n_inst * kMaxPar, 0.0);
  int n_radius = 0;
  for (int p = 0; p < s->n_par; ++p) {
    if (s->param_kind[p] < TP_PAR_RADIUS || s->param_kind[p] > TP_PAR_DENSITY) return (fail(TP_ERR_INVALID_ARG, "param_kind[%d]", p));
    n_radius += s->param_kind[p] == TP_PAR_RADIUS;
  }
  if (n_radius > 1) return (fail(TP_ERR_INVALID_ARG, "at most one radius parameter"));
  for (int q = 0; q < s->n_inst; ++q)
    for (int p = 0; p < s->n_par; ++p) {
      const double v = d->inst_params[(size_t)q * s->n_par + p];
      if (!std::isfinite(v)) return (fail(TP_ERR_INVALID_ARG, "inst_params[%d][%d] not finite", q, p));
      if (s->param_kind[p] != TP_PAR_RADIUS && !(v > 0)) return (fail(TP_ERR_INVALID_ARG, "inst_params[%d][%d] must be > 0", q, p));
      s->inst_params[(size_t)q * kMaxPar + p] = v;
    }
  // primitives
  for (int i = 0; i < d->n_prims; ++i) {
    const tp_prim& p = s->prims[i];
    if (p.shape < TP_BOX || p.shape > TP_SPHERE) return (fail(TP_ERR_INVALID_ARG, "prim %d: shape %d", i, p.shape));
    if (p.axis < 0 || p.axis > 2) return (fail(TP_ERR_INVALID_ARG, "prim %d: axis %d", i, p.axis));
    if (p.role < TP_ROLE_BULK || p.role > TP_ROLE_BLACK) return (fail(TP_ERR_INVALID_ARG, "prim %d: role %d", i, p.role));
    if (p.mirror < -1 || p.mirror >= d->n_mirrors) return (fail(TP_ERR_INVALID_ARG, "prim %d: mirror %d", i, p.mirror));
    if (p.material < -1) return (fail(TP_ERR_INVALID_ARG, "prim %d: material %d", i, p.material));
    if (!finite_all(p.centre, 3) || !finite_all(p.params, 3)) return (fail(TP_ERR_INVALID_ARG, "prim %d: not finite", i));
    if (p.shape == TP_BOX && !(p.params[0] > 0 && p.params[1] > 0 && p.params[2] > 0))
      return (fail(TP_ERR_INVALID_ARG, "prim %d: box half extents must be positive", i));
    if (p.shape == TP_TUBE && !(p.params[2] > 0)) return (fail(TP_ERR_INVALID_ARG, "prim %d: tube half height", i));
    if ((p.bind_rmin || p.bind_rmax) && (p.shape == TP_BOX || n_radius == 0))
      return (fail(TP_ERR_INVALID_ARG, "prim %d: radius binding needs a tube/sphere and a radius parameter", i));
    if (p.chopper < -1 || p.chopper >= d->n_choppers) return (fail(TP_ERR_INVALID_ARG, "prim %d: chopper %d", i, p.chopper));
    if (p.chopper >= 0 && (p.shape != TP_TUBE || p.material != -1 || p.role != TP_ROLE_BULK || p.mirror != -1 ||
                           p.bind_rmin || p.bind_rmax))
      return (fail(TP_ERR_INVALID_ARG, "prim %d: a chopper is a vacuum bulk tube, no mirror, no radius binding", i));
  }
  for (int i = 0; i < d->n_choppers; ++i) {
    const tp_chopper& c = s->choppers[i];
    if (!(c.r_black >= 0) || c.n_windows < 1 || c.n_windows > (1 << 20) || !(c.theta0 > 0) ||
        !(c.theta0 <= 2.0 * M_PI) || !finite_all(&c.r_black, 1) || !finite_all(&c.freq, 1) ||
        !finite_all(&c.phase, 1))
      return (fail(TP_ERR_INVALID_ARG, "chopper %d: need r_black >= 0, n_windows >= 1, theta0 in (0, 2 pi], "
                                       "finite freq and phase", i));
  }
  for (int i = 0; i < d->n_mirrors; ++i) {
    const tp_mirror& m = s->mirrors[i];
    if (!(m.R0 >= 0 && m.Qc >= 0 && m.W > 0 && m.alpha >= 0 && m.m >= 0) ||
        !finite_all(&m.m, 1) || !finite_all(&m.R0, 1))
      return (fail(TP_ERR_INVALID_ARG, "mirror %d: need R0, Qc, alpha, m >= 0 and W > 0", i));
  }
  // source
  if (!source_ok(s->source))
    return (fail(TP_ERR_INVALID_ARG, "source: kind, wavelength range (> 0, lo <= hi) or temperature (>= 0), "
                                         "divergence in [0, 1.5) rad (none with a temperature unless "
                                         "TP_SRC_MODERATOR), slit beyond the moderator"));
  // tallies
  s->tally_off.resize(s->tallies.size() + 1);
  long long tb = 0;
  for (int t = 0; t < d->n_tallies; ++t) {
    const tp_tally_desc& T = s->tallies[t];
    if (T.kind < TP_TALLY_COUNT || T.kind > TP_TALLY_TOF) return (fail(TP_ERR_INVALID_ARG, "tally %d: kind", t));
    if (T.trigger != TP_PTS_ENTRY && T.trigger != TP_PTS_EXIT) return (fail(TP_ERR_INVALID_ARG, "tally %d: trigger", t));
    if (T.volume < -1 || T.volume >= d->n_prims) return (fail(TP_ERR_INVALID_ARG, "tally %d: volume %d", t, T.volume));
    if (T.volume == -1 && T.trigger == TP_PTS_ENTRY) return (fail(TP_ERR_INVALID_ARG, "tally %d: the world has no ENTRY", t));
    if (T.nbins[0] < 1 || T.nbins[1] < 1) return (fail(TP_ERR_INVALID_ARG, "tally %d: bins", t));
    if (T.kind == TP_TALLY_COUNT && (T.nbins[0] != 1 || T.nbins[1] != 1)) return (fail(TP_ERR_INVALID_ARG, "tally %d: a count has one bin", t));
    if ((T.kind == TP_TALLY_ANGULAR || T.kind == TP_TALLY_MULTISCAT || T.kind == TP_TALLY_DQ ||
         T.kind == TP_TALLY_TOF) && T.nbins[1] != 1)
      return (fail(TP_ERR_INVALID_ARG, "tally %d: a 1-D scorer has nbins[1] = 1", t));
    const int dims = (T.kind == TP_TALLY_PSD || T.kind == TP_TALLY_WLX) ? 2 : (T.kind == TP_TALLY_COUNT ? 0 : 1);
    for (int k = 0; k < dims; ++k)
      if (!(T.hi[k] > T.lo[k]) || !std::isfinite(T.hi[k]) || !std::isfinite(T.lo[k]))
        return (fail(TP_ERR_INVALID_ARG, "tally %d: range of axis %d", t, k));
    s->tally_off[t] = (int)tb;
    tb += (long long)T.nbins[0] * T.nbins[1];
  }
  if (tb > (1ll << 30)) return (fail(TP_ERR_INVALID_ARG, "too many bins"));
  s->total_bins = (int)tb;
  {
    bool full = d->n_mirrors > 0 || d->n_choppers > 0;
    for (const tp_prim& p : s->prims) full = full || p.mirror >= 0 || p.chopper >= 0;
    for (const tp_tally_desc& T : s->tallies)
      full = full || !(T.kind == TP_TALLY_COUNT || T.kind == TP_TALLY_ANGULAR || T.kind == TP_TALLY_PSD);
    const tp_source& g = s->source;
    full = full || g.kind == TP_SRC_MODERATOR || g.temperature > 0 || g.div[0] > 0 || g.div[1] > 0 || g.has_aperture;
    s->full_needed = full ? 1 : 0;
    s->full = s->full_needed;
  }
  s->tally_off[s->tallies.size()] = (int)tb;
  return validate_geometry(s);
}

const char* tp_last_error(void) { return g_err.c_str(); }

int tp_total_bins(const tp_scene* s) { return s ? s->total_bins : 0; }

tp_status tp_create_scene(const tp_scene_desc* d, tp_scene** out) {
  g_err.clear();
  if (!d || !out) return fail(TP_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  tp_scene* s = new tp_scene();
  auto bail = [&](tp_status st) { tp_destroy_scene(s); return st; };
  tp_status st = describe(d, s);
  if (st != TP_OK) return bail(st);
  // device
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  if (e != cudaSuccess) return bail(fail(TP_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e)));
  const size_t nb = (size_t)s->n_inst * std::max(1, s->total_bins);
  auto alloc = [&](void** p, size_t bytes) -> bool {
    cudaError_t r = cudaMalloc(p, bytes);
    if (r != cudaSuccess) { fail(r == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(r)); return false; }
    return true;
  };
  if (!alloc((void**)&s->d_sum, nb * sizeof(double)) || !alloc((void**)&s->d_sumsq, nb * sizeof(double)))
    return bail(TP_ERR_OOM);
  if (s->n_par > 0) {
    if (!alloc((void**)&s->d_J, nb * s->n_par * sizeof(double)) || !alloc((void**)&s->d_J2, nb * s->n_par * sizeof(double)))
      return bail(TP_ERR_OOM);
  }
  if (!alloc((void**)&s->d_prefix, (s->n_inst + 1) * sizeof(unsigned long long)) ||
      !alloc((void**)&s->d_first, s->n_inst * sizeof(unsigned long long)) ||
      !alloc((void**)&s->d_params, (size_t)s->n_inst * kMaxPar * sizeof(double)) ||
      !alloc((void**)&s->d_aux, ((size_t)s->n_inst * (kMaxPar + 1)) * sizeof(double)) ||
      !alloc((void**)&s->d_work, sizeof(unsigned long long)) ||
      !alloc((void**)&s->d_counters, kNumCounters * sizeof(unsigned long long)) ||
      !alloc((void**)&s->d_status, sizeof(int)))
    return bail(TP_ERR_OOM);
  if (cudaMallocHost((void**)&s->h_stage, (2 * (size_t)s->n_inst + 1) * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost((void**)&s->h_aux, ((size_t)s->n_inst * (kMaxPar + 1)) * sizeof(double)) != cudaSuccess)
    return bail(fail(TP_ERR_OOM, "pinned staging buffers"));
  if (cudaEventCreateWithFlags(&s->stage_done, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(TP_ERR_CUDA, "event"));
  {
    void* hp = nullptr;
    void* dp = nullptr;
    if (cudaHostAlloc(&hp, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
      return bail(fail(TP_ERR_OOM, "mapped abort flag"));
    s->h_abort = static_cast<volatile int*>(hp);
    *s->h_abort = 0;
    if (cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess) return bail(fail(TP_ERR_CUDA, "abort flag address"));
    s->d_abort = static_cast<int*>(dp);
  }
  const std::vector<uint8_t> pb = params_bytes(s->inst_params, s->precision);
  if (cudaMemcpy(s->d_params, pb.data(), pb.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(TP_ERR_CUDA, "upload instance parameters"));
  s->n_done.assign(s->n_inst, 0.0);
  st = tp_reset_tallies(s);
  if (st != TP_OK) return bail(st);
  *out = s;
  return TP_OK;
}

tp_status tp_set_materials(tp_scene* s, const tp_material* m, int n) {
  g_err.clear();
  if (!s || (n > 0 && !m) || n < 0) return fail(TP_ERR_INVALID_ARG, "null argument");
  std::vector<Mat> mats(n);
  for (int i = 0; i < n; ++i) {
    const tp_material& x = m[i];
    if (!(x.sigma_abs_ref >= 0) || !(x.sigma_inc >= 0) || !std::isfinite(x.sigma_abs_ref) || !std::isfinite(x.sigma_inc))
      return fail(TP_ERR_INVALID_ARG, "material %d: cross sections must be finite and >= 0", i);
    if (x.n_lines < 0 || (x.n_lines > 0 && (!x.d || !x.mult || !x.F2)))
      return fail(TP_ERR_INVALID_ARG, "material %d: Bragg line arrays", i);
    if (x.n_lines > 0 && !(x.V0 > 0)) return fail(TP_ERR_INVALID_ARG, "material %d: V0 must be > 0", i);
    for (int k = 0; k < x.n_lines; ++k)
      if (!(x.d[k] > 0) || !(x.mult[k] >= 0) || !(x.F2[k] >= 0) || !std::isfinite(x.d[k]) || !std::isfinite(x.F2[k]))
        return fail(TP_ERR_INVALID_ARG, "material %d line %d: need d > 0, mult >= 0, F2 >= 0", i, k);
    for (int which = 0; which < 2; ++which) {
      const int p = which ? x.scale_param : x.density_param;
      if (p < -1 || p >= s->n_par) return fail(TP_ERR_INVALID_ARG, "material %d: parameter index %d", i, p);
      if (p >= 0 && s->param_kind[p] != (which ? TP_PAR_SCALE : TP_PAR_DENSITY))
        return fail(TP_ERR_INVALID_ARG, "material %d: parameter %d has the wrong kind", i, p);
    }
    mats[i].m = x;
    std::vector<int> idx(x.n_lines);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return x.d[a] > x.d[b]; });
    for (int k : idx) { mats[i].d.push_back(x.d[k]); mats[i].mult.push_back(x.mult[k]); mats[i].F2.push_back(x.F2[k]); }
    mats[i].m.d = mats[i].m.mult = mats[i].m.F2 = nullptr;
  }
  for (size_t i = 0; i < s->prims.size(); ++i)
    if (s->prims[i].material >= n) return fail(TP_ERR_INVALID_ARG, "prim %zu uses material %d of %d", i, s->prims[i].material, n);
  s->mats = std::move(mats);
  s->have_materials = true;
  s->blob_dirty = true;
  return TP_OK;
}

tp_status tp_set_bias(tp_scene* s, int material, const double g[TP_NPROC]) {
  g_err.clear();
  if (!s || !g) return fail(TP_ERR_INVALID_ARG, "null argument");
  if (!s->have_materials) return fail(TP_ERR_STATE, "tp_set_materials first");
  if (material < 0 || material >= (int)s->mats.size()) return fail(TP_ERR_INVALID_ARG, "material %d", material);
  for (int i = 0; i < TP_NPROC; ++i)
    if (!(g[i] >= 0) || !std::isfinite(g[i])) return fail(TP_ERR_INVALID_ARG, "bias factor %d must be finite and >= 0", i);
  for (int i = 0; i < TP_NPROC; ++i) s->mats[material].g[i] = g[i];
  s->blob_dirty = true;
  return TP_OK;
}

tp_status tp_set_params(tp_scene* s, const double* inst_params) {
  g_err.clear();
  if (!s || (!inst_params && s->n_par > 0)) return fail(TP_ERR_INVALID_ARG, "null argument");
  std::vector<double> old = s->inst_params;
  for (int q = 0; q < s->n_inst; ++q)
    for (int p = 0; p < s->n_par; ++p) {
      const double v = inst_params[(size_t)q * s->n_par + p];
      if (!std::isfinite(v) || (s->param_kind[p] != TP_PAR_RADIUS && !(v > 0))) {
        s->inst_params = old;
        return fail(TP_ERR_INVALID_ARG, "inst_params[%d][%d] = %g", q, p, v);
      }
      s->inst_params[(size_t)q * kMaxPar + p] = v;
    }
  tp_status st = validate_geometry(s);
  if (st != TP_OK) {
    s->inst_params = old;
    return st;
  }
  TP_CUDA(cudaDeviceSynchronize());
  const std::vector<uint8_t> pb = params_bytes(s->inst_params, s->precision);
  TP_CUDA(cudaMemcpy(s->d_params, pb.data(), pb.size(), cudaMemcpyHostToDevice));
  s->blob_dirty = true;   // bounding radii and neighbour lists depend on the radii
  return TP_OK;
}

tp_status tp_reset_tallies(tp_scene* s) {
  if (!s) return fail(TP_ERR_INVALID_ARG, "null scene");
  // a run still draining after tp_abort must have stopped before the flag clears
  TP_CUDA(cudaDeviceSynchronize());
  if (s->h_abort) *s->h_abort = 0;
  const size_t nb = (size_t)s->n_inst * std::max(1, s->total_bins);
  TP_CUDA(cudaMemset(s->d_sum, 0, nb * sizeof(double)));
  TP_CUDA(cudaMemset(s->d_sumsq, 0, nb * sizeof(double)));
  if (s->d_J) {
    TP_CUDA(cudaMemset(s->d_J, 0, nb * s->n_par * sizeof(double)));
    TP_CUDA(cudaMemset(s->d_J2, 0, nb * s->n_par * sizeof(double)));
  }
  TP_CUDA(cudaMemset(s->d_counters, 0, kNumCounters * sizeof(unsigned long long)));
  TP_CUDA(cudaMemset(s->d_status, 0, sizeof(int)));
  std::fill(s->n_done.begin(), s->n_done.end(), 0.0);
  return TP_OK;
}

tp_status tp_run_histories(tp_scene* s, const tp_run* r) {
  g_err.clear();
  if (!s || !r || !r->n_histories) return fail(TP_ERR_INVALID_ARG, "null argument");
  if (!s->have_materials) return fail(TP_ERR_STATE, "tp_set_materials first");
  if (r->want_grad && s->n_par == 0) return fail(TP_ERR_INVALID_ARG, "want_grad without parameters");
  if (r->kernel < TP_KERNEL_AUTO || r->kernel > TP_KERNEL_WARPQ) return fail(TP_ERR_INVALID_ARG, "kernel %d", r->kernel);
  const bool grad = r->want_grad != 0;
  cudaStream_t st = (cudaStream_t)r->stream;
  if (s->blob_dirty) {
    tp_status e = upload_blob(s);
    if (e != TP_OK) return e;
  }
  // work description
  if (s->stage_pending) {
    TP_CUDA(cudaEventSynchronize(s->stage_done));
    s->stage_pending = false;
  }
  unsigned long long total = 0;
  for (int i = 0; i < s->n_inst; ++i) {
    const unsigned long long first = r->first_history ? r->first_history[i] : 0ull;
    if (r->n_histories[i] > 0xffffffffull || first > 0x100000000ull - r->n_histories[i])
      return fail(TP_ERR_INVALID_ARG, "instance %d: history ids must stay below 2^32", i);
    s->h_stage[i] = total;
    s->h_stage[s->n_inst + 1 + i] = first;
    total += r->n_histories[i];
  }
  s->h_stage[s->n_inst] = total;
  if (total == 0) return TP_OK;
  if (r->secondaries < 0 || r->secondaries > 2) return fail(TP_ERR_INVALID_ARG, "secondaries %d", r->secondaries);
  if (r->stage < 0 || r->stage > 2) return fail(TP_ERR_INVALID_ARG, "stage %d: need 0, 1 or 2", r->stage);
  if (r->stage != 0 && r->kernel == TP_KERNEL_AUTO)
    return fail(TP_ERR_INVALID_ARG, "stage %d needs an explicit kernel (the autotuner picks the staging)", r->stage);
  const bool tune = r->kernel == TP_KERNEL_AUTO && s->tuned_kernel[grad] == 0;
  if (grad && (r->secondaries == 2 || (r->secondaries == 0 && (tune || (r->kernel == TP_KERNEL_AUTO && s->tuned_defer))))) {
    tp_status e = ensure_sec(s, total);   // before any capture: it may allocate
    if (e != TP_OK) return e;
  }
  int kernel = r->kernel, block = r->block_size;
  if (kernel == TP_KERNEL_AUTO) {
    if (s->tuned_kernel[grad] == 0) {
      // the trials read this run's work description
      TP_CUDA(cudaMemcpyAsync(s->d_prefix, s->h_stage, (s->n_inst + 1) * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
      TP_CUDA(cudaMemcpyAsync(s->d_first, s->h_stage + s->n_inst + 1, s->n_inst * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
      tp_status e = autotune(s, grad, r->seed, total, st);
      if (e != TP_OK) return e;
      if (grad && !s->tuned_defer && r->secondaries != 2 && s->d_sec) {   // not needed: give it back
        TP_CUDA(cudaStreamSynchronize(st));
        cudaFree(s->d_sec);
        s->d_sec = nullptr;
        s->sec_cap = 0;
      }
    }
    kernel = s->tuned_kernel[grad];
    if (block == 0) block = s->tuned_block[grad];
  }
  LaunchCfg cfg;
  const int stage = r->kernel == TP_KERNEL_AUTO ? s->tuned_stage[grad] : (r->stage == 0 ? -1 : (r->stage == 1 ? 1 : 0));
  tp_status e = resolve(s, grad, kernel, block, r->ctas_per_sm, &cfg, stage,
                        r->kernel == TP_KERNEL_AUTO && r->ctas_per_sm == 0 ? s->tuned_hi[grad] : -1);
  if (e != TP_OK) return e;
  if (grad) cfg.defer = r->secondaries == 2 || (r->secondaries == 0 && r->kernel == TP_KERNEL_AUTO && s->tuned_defer);
  if (r->regroup < 0 || r->regroup > 64) return fail(TP_ERR_INVALID_ARG, "regroup %d: need 0..64", r->regroup);
  cfg.regroup = r->regroup > 0 ? r->regroup : (r->kernel == TP_KERNEL_AUTO ? s->tuned_regroup[grad] : 1);
  Outputs o{s->d_sum, s->d_sumsq, s->d_J, s->d_J2, s->d_counters};
  if (r->use_graph) {
    e = run_graph(s, cfg, grad, r, total, o, st);
    if (e != TP_OK) return e;
  } else {
    TP_CUDA(cudaMemcpyAsync(s->d_prefix, s->h_stage, (s->n_inst + 1) * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    TP_CUDA(cudaMemcpyAsync(s->d_first, s->h_stage + s->n_inst + 1, s->n_inst * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    TP_CUDA(cudaEventRecord(s->stage_done, st));
    s->stage_pending = true;
    cudaError_t ce = launch_cfg(s, cfg, grad, r->seed, total, r->records, r->n_records, o, st);
    if (ce != cudaSuccess) return fail(TP_ERR_CUDA, "transport launch: %s", cudaGetErrorString(ce));
  }
  for (int i = 0; i < s->n_inst; ++i) s->n_done[i] += (double)r->n_histories[i];
  s->kernel = cfg.kernel;
  s->block = cfg.block;
  s->ctas_per_sm = cfg.ctas;
  s->last_cfg = cfg;
  if (grad && cfg.defer) {
    const unsigned long long chunk = std::max(1ull, s->sec_cap / kSecPerHistory);
    s->launches = (int)(2 * ((total + chunk - 1) / chunk));
  } else {
    s->launches = 1;
  }
  return TP_OK;
}

tp_status tp_read_tallies(tp_scene* s, int tally, int instance, double* mean, double* err, int on_device) {
  g_err.clear();
  if (!s || !mean) return fail(TP_ERR_INVALID_ARG, "null argument");
  if (tally < 0 || tally >= (int)s->tallies.size()) return fail(TP_ERR_INVALID_ARG, "tally %d", tally);
  if (instance < 0 || instance >= s->n_inst) return fail(TP_ERR_INVALID_ARG, "instance %d", instance);
  const int nb = s->tallies[tally].nbins[0] * s->tallies[tally].nbins[1];
  const size_t off = (size_t)instance * s->total_bins + s->tally_off[tally];
  const double n = s->n_done[instance];
  if (on_device) {
    TP_CUDA(launch_stats(s->d_sum + off, s->d_sumsq + off, n, nb, mean, err, 0));
    return TP_OK;
  }
  double *dm = nullptr, *de = nullptr;
  TP_CUDA(cudaMalloc(&dm, 2 * (size_t)nb * sizeof(double)));
  de = dm + nb;
  cudaError_t e = launch_stats(s->d_sum + off, s->d_sumsq + off, n, nb, dm, de, 0);
  if (e == cudaSuccess) e = cudaMemcpy(mean, dm, nb * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && err) e = cudaMemcpy(err, de, nb * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dm);
  if (e != cudaSuccess) return fail(TP_ERR_CUDA, "read tallies: %s", cudaGetErrorString(e));
  return TP_OK;
}

tp_status tp_read_raw(tp_scene* s, int instance, double* sum, double* sumsq, double* J, double* J2, int on_device) {
  g_err.clear();
  if (!s) return fail(TP_ERR_INVALID_ARG, "null scene");
  if (instance < 0 || instance >= s->n_inst) return fail(TP_ERR_INVALID_ARG, "instance %d", instance);
  const size_t nb = (size_t)s->total_bins;
  const size_t off = (size_t)instance * nb;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  TP_CUDA(cudaDeviceSynchronize());
  if (sum) TP_CUDA(cudaMemcpy(sum, s->d_sum + off, nb * sizeof(double), kind));
  if (sumsq) TP_CUDA(cudaMemcpy(sumsq, s->d_sumsq + off, nb * sizeof(double), kind));
  for (int p = 0; p < s->n_par; ++p) {
    const size_t src = ((size_t)p * s->n_inst + instance) * nb;
    if (J) TP_CUDA(cudaMemcpy(J + p * nb, s->d_J + src, nb * sizeof(double), kind));
    if (J2) TP_CUDA(cudaMemcpy(J2 + p * nb, s->d_J2 + src, nb * sizeof(double), kind));
  }
  return TP_OK;
}

tp_status tp_write_raw(tp_scene* s, int instance, const double* sum, const double* sumsq, const double* J,
                       const double* J2, double n_histories, int on_device) {
  g_err.clear();
  if (!s || !sum || !sumsq) return fail(TP_ERR_INVALID_ARG, "null argument");
  if (instance < 0 || instance >= s->n_inst) return fail(TP_ERR_INVALID_ARG, "instance %d", instance);
  if (!(n_histories >= 0) || !std::isfinite(n_histories)) return fail(TP_ERR_INVALID_ARG, "n_histories %g", n_histories);
  if ((J || J2) && s->n_par == 0) return fail(TP_ERR_INVALID_ARG, "scene has no parameters");
  const size_t nb = (size_t)s->total_bins;
  const size_t off = (size_t)instance * nb;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  TP_CUDA(cudaDeviceSynchronize());
  TP_CUDA(cudaMemcpy(s->d_sum + off, sum, nb * sizeof(double), kind));
  TP_CUDA(cudaMemcpy(s->d_sumsq + off, sumsq, nb * sizeof(double), kind));
  for (int p = 0; p < s->n_par; ++p) {
    const size_t dst = ((size_t)p * s->n_inst + instance) * nb;
    if (J) TP_CUDA(cudaMemcpy(s->d_J + dst, J + p * nb, nb * sizeof(double), kind));
    if (J2) TP_CUDA(cudaMemcpy(s->d_J2 + dst, J2 + p * nb, nb * sizeof(double), kind));
  }
  s->n_done[instance] = n_histories;
  return TP_OK;
}

tp_status tp_backward(tp_scene* s, const double* grad_tallies, double* grad_params, int on_device, void* stream) {
  g_err.clear();
  if (!s || !grad_tallies || !grad_params) return fail(TP_ERR_INVALID_ARG, "null argument");
  if (s->n_par == 0 || !s->d_J) return fail(TP_ERR_STATE, "scene has no parameters");
  cudaStream_t st = (cudaStream_t)stream;
  const int ni = s->n_inst, np = s->n_par;
  // d/dtheta: radius per cm; scale and density are log-parameters in the
  // accumulators, divided by the parameter value here
  TP_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < ni; ++i) {
    for (int p = 0; p < np; ++p) {
      const double v = s->inst_params[(size_t)i * kMaxPar + p];
      s->h_aux[(size_t)i * np + p] = s->param_kind[p] == TP_PAR_RADIUS ? 1.0 : 1.0 / v;
    }
    s->h_aux[(size_t)ni * np + i] = s->n_done[i];
  }
  TP_CUDA(cudaMemcpyAsync(s->d_aux, s->h_aux, ((size_t)ni * np + ni) * sizeof(double), cudaMemcpyHostToDevice, st));
  const size_t gt_bytes = (size_t)ni * s->total_bins * sizeof(double);
  const size_t gp_bytes = (size_t)ni * np * sizeof(double);
  const double* d_gt = grad_tallies;
  double* d_gp = grad_params;
  double* tmp = nullptr;
  if (!on_device) {
    TP_CUDA(cudaMalloc(&tmp, gt_bytes + gp_bytes));
    TP_CUDA(cudaMemcpyAsync(tmp, grad_tallies, gt_bytes, cudaMemcpyHostToDevice, st));
    d_gt = tmp;
    d_gp = tmp + (size_t)ni * s->total_bins;
  }
  cudaError_t e = launch_backward(s->d_J, d_gt, s->d_aux, s->d_aux + (size_t)ni * np, ni, np, s->total_bins, d_gp, st);
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(grad_params, d_gp, gp_bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(TP_ERR_CUDA, "backward: %s", cudaGetErrorString(e));
  return TP_OK;
}

tp_status tp_get_counters(tp_scene* s, int64_t out[8]) {
  g_err.clear();
  if (!s || !out) return fail(TP_ERR_INVALID_ARG, "null argument");
  unsigned long long h[kNumCounters];
  int status = 0;
  TP_CUDA(cudaDeviceSynchronize());
  TP_CUDA(cudaMemcpy(h, s->d_counters, sizeof h, cudaMemcpyDeviceToHost));
  TP_CUDA(cudaMemcpy(&status, s->d_status, sizeof status, cudaMemcpyDeviceToHost));
  for (int i = 0; i < kNumCounters; ++i) out[i] = (int64_t)h[i];
  return device_status(status);
}

tp_status tp_abort(tp_scene* s) {
  if (!s || !s->h_abort) return fail(TP_ERR_INVALID_ARG, "null scene");
  *s->h_abort = 1;
  return TP_OK;
}

tp_status tp_set_test_flags(tp_scene* s, int flags) {
  g_err.clear();
  if (flags & ~(TP_TEST_SKIP_TABLE_COPY | TP_TEST_FULL_BUILD | TP_TEST_SMALL_SEC_QUEUE))
    return fail(TP_ERR_INVALID_ARG, "unknown test flags %#x", flags);
  if (!s) {
    g_noalloc_test_flags.store(flags & TP_TEST_SKIP_TABLE_COPY);
    return TP_OK;
  }
  s->test_flags = flags;
  s->full = (s->full_needed || (flags & TP_TEST_FULL_BUILD)) ? 1 : 0;
  for (int g = 0; g < 2; ++g) s->tuned_kernel[g] = 0;   // the autotuner's choice was for the other build
  if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }   // the flags are baked into it
  return TP_OK;
}

int tp_get_launch_count(const tp_scene* s) { return s ? s->launches : 0; }

tp_status tp_get_launch_info(const tp_scene* s, tp_launch_info* out) {
  if (!s || !out) return fail(TP_ERR_INVALID_ARG, "null argument");
  *out = tp_launch_info{};
  if (s->kernel == 0) return TP_OK;
  const LaunchCfg& c = s->last_cfg;
  out->kernel = c.kernel;
  out->block_size = c.block;
  out->ctas_per_sm = c.ctas;
  out->staged = c.stage ? 1 : 0;
  out->registers = c.hi ? 64 : 80;
  out->full_build = c.full ? 1 : 0;
  out->regroup = c.regroup;
  out->queued_secondaries = c.defer ? 1 : 0;
  out->launches = s->launches;
  return TP_OK;
}

tp_status tp_get_launch(tp_scene* s, int* kernel, int* block, int* ctas) {
  if (!s || !kernel || !block || !ctas) return fail(TP_ERR_INVALID_ARG, "null argument");
  *kernel = s->kernel;
  *block = s->block;
  *ctas = s->ctas_per_sm;
  return TP_OK;
}

void tp_destroy_scene(tp_scene* s) {
  if (!s) return;
  if (s->stage_pending) cudaEventSynchronize(s->stage_done);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->capture_stream) cudaStreamDestroy(s->capture_stream);
  cudaFree(s->d_blob);
  cudaFree(s->d_grid);
  cudaFree(s->d_sum); cudaFree(s->d_sumsq); cudaFree(s->d_J); cudaFree(s->d_J2);
  cudaFree(s->d_prefix); cudaFree(s->d_first); cudaFree(s->d_params); cudaFree(s->d_aux);
  cudaFree(s->d_work); cudaFree(s->d_counters); cudaFree(s->d_status);
  cudaFree(s->d_sec); cudaFree(s->d_sec_count);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  if (s->h_aux) cudaFreeHost(s->h_aux);
  if (s->h_abort) cudaFreeHost(const_cast<int*>(s->h_abort));
  if (s->stage_done) cudaEventDestroy(s->stage_done);
  delete s;
}

}  // extern "C"

// ===========================================================================
// Allocation-free variant of tp_run_histories
// ===========================================================================
// For callers that cannot allocate device memory (code running where the device
// memory is owned by another allocator, or where cudaMalloc is not allowed):
// everything the transport kernel needs besides its inputs and outputs -- the
// scene tables, the per-run work description and the work counter, event
// counters and status word -- lives in one file-scope device array that every
// GPU loading this library holds until the process exits.
namespace {

constexpr size_t kNaBlobBytes = TP_NOALLOC_MAX_TABLE_BYTES;
constexpr size_t kNaWorkOff = kNaBlobBytes;                      // prefix, first ids, params
constexpr size_t kNaWorkBytes = 4096;
constexpr size_t kNaCtlOff = kNaWorkOff + kNaWorkBytes;         // work counter, counters, status
constexpr size_t kNaCtlBytes = 256;
static_assert(kNaCtlOff + kNaCtlBytes == TP_NOALLOC_SCRATCH_BYTES, "scratch layout");
static_assert((TP_NOALLOC_MAX_INSTANCES + 1) * 8 + TP_NOALLOC_MAX_INSTANCES * 8 +
                  TP_NOALLOC_MAX_INSTANCES * kMaxPar * 8 <= kNaWorkBytes, "work section");

static __device__ __align__(256) unsigned char g_noalloc_scratch[TP_NOALLOC_SCRATCH_BYTES];

constexpr int kNaMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
tp_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  TP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail(TP_ERR_INVALID_ARG, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    TP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_addr[dev];
  return TP_OK;
}

}  // namespace

extern "C" tp_status tp_run_histories_noalloc(const tp_scene_desc* d, const tp_material* mats, int n_mats,
                                              const double* bias, const tp_run* r, double* sum, double* sumsq,
                                              int64_t counters_out[8]) {
  g_err.clear();
  if (!d || !r || !r->n_histories || !sum || !sumsq || (n_mats > 0 && !mats) || n_mats < 0)
    return fail(TP_ERR_INVALID_ARG, "null argument");
  if (r->want_grad || r->records) return fail(TP_ERR_INVALID_ARG, "no gradients or records in the allocation-free call");
  if (r->kernel != TP_KERNEL_AUTO && r->kernel != TP_KERNEL_HISTORY)
    return fail(TP_ERR_INVALID_ARG, "kernel %d: the allocation-free call runs the history kernel only", r->kernel);
  if (r->use_graph || r->secondaries || r->regroup > 1 || r->stage == 2)
    return fail(TP_ERR_INVALID_ARG, "the allocation-free call takes no graph, secondaries, regroup or unstaged-table option");
  if (d->n_instances < 1 || d->n_instances > TP_NOALLOC_MAX_INSTANCES)
    return fail(TP_ERR_INVALID_ARG, "n_instances %d: the allocation-free call takes 1..%d", d->n_instances,
                TP_NOALLOC_MAX_INSTANCES);
  // host-side scene: the same checks and tables as tp_create_scene, no device memory
  tp_scene s;
  tp_status st = describe(d, &s);
  if (st != TP_OK) return st;
  st = tp_set_materials(&s, mats, n_mats);
  if (st != TP_OK) return st;
  if (bias)
    for (int m = 0; m < n_mats; ++m)
      if ((st = tp_set_bias(&s, m, bias + (size_t)m * TP_NPROC)) != TP_OK) return st;
  std::vector<uint8_t> blob = s.precision == TP_FP64 ? build_blob<double>(&s) : build_blob<float>(&s);
  if (blob.size() > kNaBlobBytes)
    return fail(TP_ERR_INVALID_ARG, "scene tables need %zu bytes; the allocation-free call holds at most %zu",
                blob.size(), kNaBlobBytes);
  s.blob_bytes = (uint32_t)blob.size();
  unsigned long long total = 0;
  std::vector<unsigned long long> work((size_t)2 * s.n_inst + 1);
  for (int i = 0; i < s.n_inst; ++i) {
    const unsigned long long first = r->first_history ? r->first_history[i] : 0ull;
    if (r->n_histories[i] > 0xffffffffull || first > 0x100000000ull - r->n_histories[i])
      return fail(TP_ERR_INVALID_ARG, "instance %d: history ids must stay below 2^32", i);
    work[i] = total;
    work[(size_t)s.n_inst + 1 + i] = first;
    total += r->n_histories[i];
  }
  work[s.n_inst] = total;

  unsigned char* base = nullptr;
  if ((st = noalloc_scratch(&base)) != TP_OK) return st;
  cudaStream_t strm = (cudaStream_t)r->stream;
  s.d_blob = base;
  s.d_prefix = reinterpret_cast<unsigned long long*>(base + kNaWorkOff);
  s.d_first = s.d_prefix + (s.n_inst + 1);
  s.d_params = s.d_first + s.n_inst;
  s.d_work = reinterpret_cast<unsigned long long*>(base + kNaCtlOff);
  s.d_counters = s.d_work + 1;
  s.d_status = reinterpret_cast<int*>(s.d_counters + kNumCounters);
  s.d_sum = sum;
  s.d_sumsq = sumsq;
  // the array keeps the previous call's contents: clear the work counter,
  // counters and status, then copy this call's tables in
  TP_CUDA(cudaMemsetAsync(base + kNaCtlOff, 0, kNaCtlBytes, strm));
  TP_CUDA(cudaMemcpyAsync(s.d_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice, strm));
  TP_CUDA(cudaMemcpyAsync(s.d_prefix, work.data(), work.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, strm));
  const std::vector<uint8_t> pb = params_bytes(s.inst_params, s.precision);
  TP_CUDA(cudaMemcpyAsync(s.d_params, pb.data(), pb.size(), cudaMemcpyHostToDevice, strm));
  if (total > 0) {
    int dev = 0, sms = 0;
    TP_CUDA(cudaGetDevice(&dev));
    TP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    s.sm_count = sms;
    int block = 0, ctas = 0;
    if ((st = pick_launch(&s, false, r->block_size, r->ctas_per_sm, &block, &ctas)) != TP_OK) return st;
    const int grid = sms * ctas;
    long long chunk = (long long)(total / (unsigned long long)((long long)grid * (block / 32) * 8));
    chunk = std::max(1ll, std::min(256ll, chunk));
    cudaError_t ce;
    if (s.precision == TP_FP64) {
      KParams<double> k{};
      fill_common(&s, k);
      k.key0 = (uint32_t)(r->seed & 0xffffffffu); k.key1 = (uint32_t)(r->seed >> 32);
      k.total = total; k.chunk = (int)chunk;
      k.test_flags = g_noalloc_test_flags.load();
      ce = launch_transport_f64(k, TP_KERNEL_HISTORY | (s.full ? kVariantFull : 0), false, grid, block, smem_bytes(&s), strm);
    } else {
      KParams<float> k{};
      fill_common(&s, k);
      k.key0 = (uint32_t)(r->seed & 0xffffffffu); k.key1 = (uint32_t)(r->seed >> 32);
      k.total = total; k.chunk = (int)chunk;
      k.test_flags = g_noalloc_test_flags.load();
      ce = launch_transport_f32(k, TP_KERNEL_HISTORY | (s.full ? kVariantFull : 0), false, grid, block, smem_bytes(&s), strm);
    }
    if (ce != cudaSuccess) return fail(TP_ERR_CUDA, "transport launch: %s", cudaGetErrorString(ce));
  }
  // the host copies above read pageable memory that dies with this call
  TP_CUDA(cudaStreamSynchronize(strm));
  int status = 0;
  TP_CUDA(cudaMemcpy(&status, s.d_status, sizeof status, cudaMemcpyDeviceToHost));
  if (counters_out) {
    unsigned long long h[kNumCounters];
    TP_CUDA(cudaMemcpy(h, s.d_counters, sizeof h, cudaMemcpyDeviceToHost));
    for (int i = 0; i < kNumCounters; ++i) counters_out[i] = (int64_t)h[i];
  }
  return device_status(status);
}
