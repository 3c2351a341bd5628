// tp_internal.h -- device data layout shared by the host runtime (tp_api.cu) and
// the kernels (tp_transport.cu).  Not part of the public ABI (include/tp.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tp.h"

namespace tp {

constexpr int kMaxPar = TP_MAX_PARAMS;
constexpr int kMaxTallies = TP_MAX_TALLIES;
constexpr int kNumCounters = 8;
// Counter slots (also the order of tp_get_counters).
enum { C_HIST = 0, C_EVENTS, C_COLL, C_CROSS, C_TRUNC, C_LOST, C_MIRROR, C_SEC };
// History end codes (tp_record.end).
enum { END_ESCAPED = 0, END_ABSORBED, END_DETECTED, END_BLACK, END_MIRROR, END_TRUNCATED,
       END_APERTURE, END_LOST };
// Primitive flag bits; a chopper primitive also keeps its chopper index in
// flags >> kChopperShift.
enum { F_BIND_RMIN = 1, F_BIND_RMAX = 2, F_CHOPPER = 4 };
constexpr int kChopperShift = 8;

// One primitive as the kernels see it.  Lengths in the transport precision R.
// entry_mask / exit_mask: bit t set if tally t listens to ENTRY / EXIT here.
// bound_r: radius of a sphere about c containing the primitive for every
// instance (with a margin).  nb_off / nb_cnt: the primitives that touch this one
// (the only candidates for the volume entered when leaving it).
template <typename R>
struct alignas(16) DPrim {
  R c[3];
  R p[3];
  R bound_r;
  int shape, axis, material, role;
  int mirror, flags, entry_mask, exit_mask;
  int nb_off, nb_cnt;
};

// Material: cross sections, bias factors and the location of its Bragg table.
// Lines are sorted by d descending; cum[cum_off + i] = sum_{j<i} m_j F2_j d_j.
template <typename R>
struct alignas(16) DMat {
  R sig_abs_ref, sig_inc, bragg_pref;  // bragg_pref = 1 / (2 V0^2)
  R g[TP_NPROC];
  int abs_1v, nlines, line_off, cum_off;
  int density_par, scale_par, pad0, pad1;
};

template <typename R>
struct alignas(16) DMirror {
  R m, R0, Qc, alpha, W, mQc, pad0, pad1;
};

// Disk chopper, in units of the window period: a neutron at angle phi (rad)
// and time t (s) is at psi = phi * n_over_2pi - nf * t - n_phase periods from
// window centres (integers) and passes if |psi - rint(psi)| <= half.
template <typename R>
struct alignas(16) DChopper {
  R r_black2;     // black inner radius squared
  R n_over_2pi;   // n / (2 pi)
  R nf;           // n * freq
  R n_phase;      // n * phase / (2 pi)
  R half;         // n * theta0 / (4 pi)
  R pad0, pad1, pad2;
};

template <typename R>
struct alignas(16) DTally {
  R lo[2], hi[2];
  R inv_w[2];  // nbins / (hi - lo)
  R origin[3], axis[3];  // axis normalised
  int kind, trigger, volume, face, scat, nb0, nb1, offset;
};

// Everything a transport launch needs.  The scene tables live in one blob in
// global memory (16-byte aligned sections) that each CTA stages into shared
// memory with a bulk asynchronous copy when it fits.
template <typename R>
struct KParams {
  const uint8_t* blob;
  uint32_t blob_bytes;
  uint32_t off_prims, off_mats, off_mirrors, off_choppers, off_tallies, off_line_d, off_line_cum, off_nb;
  int stage_blob;  // 1: copy the blob into shared memory
  int nprim, nmat, ntally, npar;
  int param_kind[kMaxPar];
  int radius_par;  // index of the radius parameter or -1
  R radius_nominal;
  // world
  int world_shape;
  R world_c[3], world_p[3];
  int world_entry_mask, world_exit_mask;
  // source
  int src_kind, src_aperture;
  R src_c[3], src_half[2], src_lam_lo, src_lam_hi, src_div[2], src_ap[2];
  R src_slit_z, src_slit_half[2], src_kT;   // moderator slit; kT in meV (0: uniform wavelength)
  int src_free;   // 1: every source point lies in the world region, outside every primitive (no locate)
  // uniform grid over the primitives (large scenes): cell (i,j,k) lists the
  // primitives whose bounding box meets it, in CSR form (grid_start / grid_items)
  int use_grid;
  int grid_n[3];
  R grid_lo[3], grid_hi[3], grid_cell[3], grid_inv[3];
  const int* grid_start;
  const int* grid_items;
  // random numbers
  uint32_t key0, key1;
  int event_cap;
  // work: n_inst instances, global history index g in [0, total)
  int n_inst;
  const unsigned long long* inst_prefix;  // [n_inst + 1], device
  const unsigned long long* inst_first;   // [n_inst], device: first history id
  const R* inst_params;                   // [n_inst][kMaxPar], device, transport precision
  unsigned long long total;
  unsigned long long* work_counter;
  int chunk;  // histories a warp claims at once
  // event kernel, plain runs: the bank is regrouped every `regroup` events
  // (1 = every event); in between, each thread continues its own neutron
  int regroup;
  unsigned long long index_base;  // global index of claim 0 (one chunk of a longer run)
  // Radius-derivative secondaries of gradient runs: 0 = transported where
  // they are made; 1 = appended to sec_buf (transported in place only when it
  // is full); 2 = this launch transports the sec_buf records instead of new
  // histories.
  int sec_mode;
  uint8_t* sec_buf;                 // [sec_cap] neutron records
  unsigned long long* sec_count;    // records appended (may pass sec_cap)
  unsigned long long sec_cap;
  // outputs
  double* sum;    // [n_inst][total_bins]
  double* sumsq;
  double* J;      // [npar][n_inst][total_bins]
  double* J2;
  int total_bins;
  unsigned long long* counters;  // [kNumCounters]
  tp_record* records;
  unsigned long long n_records;
  int* status;
  // Host-written abort request (mapped pinned memory, may be null): once it is
  // non-zero the kernels claim no new histories, finish the ones they hold and
  // set *status to TP_ERR_ABORTED.
  const volatile int* abort_flag;
  // TP_TEST_* flags of tp_set_test_flags (0 in normal runs).
  int test_flags;
};

// Launchers (tp_transport.cu).  variant: TP_KERNEL_HISTORY / _EVENT / _WARPQ,
// optionally with kVariantHighOcc (the 64-register build of an FP32 kernel: 4
// blocks of 256 threads per SM instead of 3) and kVariantFull (the build with
// every feature: mirrors, choppers, all scorer kinds and guns; without it the
// lean build, for scenes that use none of them).
constexpr int kVariantHighOcc = 16;
constexpr int kVariantFull = 32;
cudaError_t launch_transport_f32(const KParams<float>& p, int variant, bool grad, int grid, int block,
                                 size_t smem, cudaStream_t st);
cudaError_t launch_transport_f64(const KParams<double>& p, int variant, bool grad, int grid, int block,
                                 size_t smem, cudaStream_t st);
// one per kernel family (k1 history, k2 event, k3 warp pools), each in its own
// translation unit
#define TP_DECLARE_FAMILY(K)                                                                                \
  cudaError_t launch_transport_f32_##K(const KParams<float>& p, int variant, bool grad, int grid, int block, \
                                       size_t smem, cudaStream_t st);                                       \
  cudaError_t launch_transport_f64_##K(const KParams<double>& p, int variant, bool grad, int grid, int block, \
                                       size_t smem, cudaStream_t st);                                       \
  cudaError_t occupancy_f32_##K(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas);  \
  cudaError_t occupancy_f64_##K(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas);
TP_DECLARE_FAMILY(k1)
TP_DECLARE_FAMILY(k2)
TP_DECLARE_FAMILY(k3)
#undef TP_DECLARE_FAMILY
// Shared memory of the neutron bank of a variant (added to the staged tables).
size_t bank_bytes(int variant, int precision, bool grad, int block);
// Bytes of one queued neutron record (sec_buf).
size_t particle_bytes(int precision);
cudaError_t occupancy_transport(int variant, int precision, bool grad, bool use_grid, int block, size_t smem,
                                int* ctas);
cudaError_t occupancy_f32(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas);
cudaError_t occupancy_f64(int variant, bool grad, bool use_grid, int block, size_t smem, int* ctas);
cudaError_t launch_stats(const double* sum, const double* sumsq, double n, int nbins, double* mean,
                         double* err, cudaStream_t st);
cudaError_t launch_backward(const double* J, const double* grad_tallies, const double* scale,
                            const double* n_done, int n_inst, int npar, int total_bins,
                            double* grad_params, cudaStream_t st);

}  // namespace tp
