// pic_internal.cuh -- context layout and launcher declarations shared by the
// CUDA translation units of libpic.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pic.h"

#define PIC_MAX_SPECIES 4
#define PIC_MAX_GL 8
#define PIC_MAX_ANDERSON 8

// Status bits raised by the particle kernels (one word per evaluation).
#define PIC_ST_NOCONV 1u      // inner limit reached
#define PIC_ST_NONFINITE 2u   // non-finite orbit velocity
#define PIC_ST_SUPERLUM 4u    // |vbar| >= kappa
#define PIC_ST_PIECES 8u      // orbit crosses more knots than the kernel handles
#define PIC_ST_WAIT 16u       // a bounded device wait (staging copies) gave up

// reals per gather record: [grad phi^{1/2} (d), A^n (3), A^{n+1} (3)] padded
// to a multiple of four so that records load with 16-byte vector loads
inline int node_record_len(int d) { return (d + 6 + 3) / 4 * 4; }

struct Geom {
  int dim;
  int n[3];
  int logn[3];
  int Ng;
  double L[3], x0[3], dx[3], dV;
};

// Scalars the particle kernels read; passed by value.
struct StepConst {
  double dt, kappa;
  double qs[PIC_MAX_SPECIES], ms[PIC_MAX_SPECIES];
  double tau_r, tau_a;  // inner tolerances
  int inner_max;
  int ngl;
  int warm;  // start the inner iteration from vbar instead of v^0
  int order;       // shape degree: 2, or 1
  int refine_max;  // convergence-triggered refinement depth (0 = off)
  double gl_t[PIC_MAX_GL], gl_w[PIC_MAX_GL];  // nodes and weights on [0, 1]
};

// Per-evaluation counters written by the particle kernel.
struct EvalCounters {
  unsigned int status;
  int inner_max;
  unsigned long long inner_sum;
  unsigned long long pieces;
  unsigned long long refined;  // particles solved with substeps
  unsigned int chunk_next;     // chunk queue of the persistent FP64 map kernel
};

// The spectral field state (accepted, candidate, or a tangent of either).
struct SpecState {
  double2 *rho, *phi, *psi, *A, *U;  // Ng, Ng, Ng, 3Ng, 3Ng modes
};

// Forward sensitivity of the state (pic_tangent_begin): the tangents of the
// particle offsets and canonical momenta in slot order, of the spectral
// field state, and the scratch of the tangent solve of one step.
struct TangentState {
  double *off;           // [dim][cap] tangent of the offset, node units
  double *P;             // [3][cap]
  SpecState f, f1;       // accepted and candidate field tangents
  double *A_real;        // 3Ng tangent of A^n in real space
  double *A1_real;       // 3Ng tangent of A^{n+1} of the last tangent evaluation
  double2 *jh;           // 3Ng transform of the tangent trial current
  double2 *work;         // (dim + 3) Ng tangent gather spectra
  double *rec;           // Ng * nvp tangent gather records
  void *drec;            // Ng * nvp dual records
  void *dpart;           // (dim + 15) * cap dual particle arrays
  double *Jd;            // 6Ng orbit current and its tangent
  double *V;             // 21 * 3Ng Krylov basis
  double *x, *b, *w, *Tx;  // 3Ng each
  int gmres_iters;       // Krylov iterations of the last tangent solve
  void *block;           // the single allocation behind all of the above
};

// Reduction partials returned to the host after the residual kernel.
struct ResidSums {
  double r2, H2, j2, smax;
};

struct pic_ctx {
  Geom g;
  int nspecies;
  double qs[PIC_MAX_SPECIES], ms[PIC_MAX_SPECIES];
  double dt;
  pic_options opt;
  cudaStream_t st;
  std::string err;
  int started;     // pic_start done (or state restored)
  int have_particles;
  int pending_mech;
  double E0;
  long long steps_done;

  // ---- particles (SoA, capacity cap) -------------------------------------
  int64_t np, cap;
  int rsize;          // sizeof(real) of particle storage: 8 (FP64) or 4 (mixed)
  int32_t *cell;      // [3][cap] nearest node per active dim
  void *off;          // [3][cap] offset in node units, [-1/2, 1/2)
  void *P;            // [3][cap] canonical momentum
  double *w;          // [cap]
  int32_t *sp;        // [cap]
  int64_t *id;        // [cap] load order index
  void *Am, *v0, *vbar, *Pnew;  // [3][cap] step work
  int32_t *iters;     // [cap]
  float4 *dep_rec;    // [2 cap] deposit records of the FP32 map (mixed contexts), or null
  double *u_in;       // [3][cap] mechanical input awaiting pic_start
  // sort scratch
  int32_t *keys;      // [cap] sort keys
  int32_t *cnt_sort;  // [Ng] per-cell counts / cursors of the sort
  void *tmp_r;        // [3][cap] scratch of particle reals
  double *tmp_d;      // [3][cap]
  int32_t *tmp_i;     // [4][cap]: staged species, then staged node indices
  int64_t *tmp_l;

  // ---- mesh: accepted state (spectral primary + real copies) ------------
  double2 *phi_h, *psi_h, *rho_h, *A_h, *U_h;   // Ng, Ng, Ng, 3Ng, 3Ng
  double *A_real;     // 3Ng  A^n in real space (gather)
  void *A_real_f;     // 3Ng  float copy of A^n (mixed path only)
  double *J_acc;      // 3Ng  accepted current (seed of the next outer solve)
  // ---- mesh: one map evaluation -----------------------------------------
  double2 *phi1_h, *psi1_h, *rho1_h, *A1_h, *U1_h;  // n+1 candidates
  double2 *jh;        // 3Ng  transform of the trial current
  double2 *work_h;    // (d + 6) * Ng spectral scratch for inverse transforms
  double *A1_real;    // 3Ng  A^{n+1} of the last evaluation in real space
  double *scr_r;      // 4Ng  real scratch (start, get/set)
  void *nodes;        // Ng * NV gather records in the particle real type
  void *nodes_u;      // Ng * 3 U^{n+1/2} records (final pass diagnostics)
  float *nodes_f;     // Ng * NV FP32 gather records (option fp32_first), or null
  float *nodes_u_f;   // Ng * 4 their U^{n+1/2} records
  int eval_f32;       // the queued evaluations use FP32 arithmetic on FP64 storage
  double *Jorb;       // 3Ng deposited orbit current
  double2 *Jorb_h;    // 3Ng its projected transform
  double *H;          // 3Ng  H(j)
  // ---- outer solver ------------------------------------------------------
  double *j, *r, *jt, *Ht, *rt, *dir;   // 3Ng each
  double *dJ, *dR;    // M * 3Ng
  // ---- FFT ---------------------------------------------------------------
  double2 *tw[3];     // twiddle table per axis: exp(-2 pi i k / n), k < n
  // ---- reductions ------------------------------------------------------
  double *red;        // block partials
  double *red_host;   // pinned
  double *rep_dev;    // 8 device slots of the queued commit-time sums
  EvalCounters *cnt_dev, *cnt_host;
  double *psum;       // per-block particle sums (work, chain, K)
  double *psum_host;  // pinned copy of the final-pass partials
  int map_final;      // the queued particle map is a final (diagnostic) pass
  // ---- device-controlled step (control.cu) ------------------------------
  int loop_capture;              // capturing the controlled step's graphs
  unsigned long long *map_timer; // [2] first start, last end of the map launch (ns)
  struct SCtl *sctl;             // controller state (device)
  struct SCtl *sctl_host;        // pinned copy read after the step
  double *sred;                  // block partials of the residual and Gram sums
  struct StepGraphs {
    const void *phi, *A;
    double tr, ta, itr, ita;
    int64_t np;
    int f32;  // FP32-stage evaluations
    cudaGraphExec_t loop, verify;
    int nk_round, nk_verify;  // kernels per loop round, in the verification
  } sgraphs[4];
  int nsgraphs;
  int sgraphs_off;               // the graphs could not be built: the host drives the step
  int f32_stage_off;             // the FP32 stage's graph could not be built: no FP32 stage
  // ---- statistics (pic_stats) ------------------------------------------
  long long launches;          // kernels launched by this context
  long long map_launches;      // particle-map kernel launches
  double map_ms;               // their summed device time (CUDA events)
  long long pushes;            // particles x map evaluations
  long long inner_iters;       // summed inner iterations
  long long pieces;            // summed knot-split orbit pieces walked
  long long refined;           // particle solves that needed substeps
  cudaEvent_t ev0, ev1;
  int num_sms;
  // ---- execution -----------------------------------------------------------
  cudaStream_t own_st;  // created when the caller passed no stream
  struct GraphEntry {
    const void *j, *H, *r, *phi, *A;
    int final_pass;
    double tr, ta, itr, ita;
    int64_t np;
    int nkern;  // kernels in the graph
    cudaGraphExec_t exec;
  };
  GraphEntry graphs[16];
  int ngraphs;
  int graphs_off;  // capture failed once: launch directly
  TangentState *tan;  // forward sensitivity, or null
  // deterministic deposit (option deterministic_deposit): per-cell particle
  // lists and the deposit's reach
  int32_t *det_count = nullptr, *det_cursor = nullptr, *det_start = nullptr, *det_list = nullptr;
  int *det_reach = nullptr;
  int64_t det_cap = 0;
};

// Gauss-Legendre nodes t and weights w of an n-point rule on [0, 1]
void gauss_legendre01(int n, double *t, double *w);

// outer and inner tolerances of a step at tolerance tol (reading R9), and
// the particle-map constants built from the inner ones
void tolerances(const pic_ctx *ctx, double tol, double *tr, double *ta, double *itr,
                double *ita);
StepConst make_sc(const pic_ctx *ctx, double itr, double ita);

// drop every captured graph (buffers or sizes changed)
void graphs_clear(pic_ctx *ctx);

// every kernel launch is followed by KCHECK(): it counts the launch and
// turns a launch error into PIC_ECUDA
#define KCHECK()                                                              \
  do {                                                                        \
    ctx->launches++;                                                          \
    CK(cudaGetLastError());                                                   \
  } while (0)

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return PIC_ECUDA;                                                       \
    }                                                                         \
  } while (0)

// ---------------------------------------------------------------- fft.cu
// In-place unnormalised complex FFT of `batch` consecutive mesh arrays of
// Ng values each, along every active axis; sign -1 forward, +1 inverse.
int fft_nd(pic_ctx *ctx, double2 *data, int batch, int sign);
int fft_init(pic_ctx *ctx);

// ---------------------------------------------------------------- field.cu
int field_real_to_complex(pic_ctx *ctx, const double *src, double2 *dst, int ncomp);
int field_complex_to_real(pic_ctx *ctx, const double2 *src, double *dst, int ncomp,
                          double scale);
int field_project_h(pic_ctx *ctx, double2 *f, int ncomp);
int field_cn_update(pic_ctx *ctx, const double2 *jh, int want_uhalf);
int field_pack_nodes(pic_ctx *ctx, int want_uhalf);
// The whole spectral field step of one map evaluation at the trial current
// jdev (real, 3Ng): transforms, projection, continuity and CN update into the
// candidate spectra, gather records (final pass: with U^{n+1/2}), and J_orb
// cleared for the deposit.  Fused launches on 2D meshes (field2d.cu).
int field_evaluate(pic_ctx *ctx, const double *jdev, int final_pass);
int field_initial_constraints(pic_ctx *ctx);
// The CN update from any field state `in` into `out` and the gather spectra
// `spec`; the update is linear in (j, state) jointly, so a tangent state and a
// tangent current give the tangent of the field step.
int field_cn_update_into(pic_ctx *ctx, const double2 *jh, const SpecState &in,
                         const SpecState &out, double2 *spec, int want_uhalf);
// FP64 gather records from the gather spectra `spec` (inverse-transformed in
// place) and A^n in real space; A^{n+1} in real space goes to A1_real
int field_pack_nodes_into(pic_ctx *ctx, double2 *spec, const double *A_n, double *A1_real,
                          double *nodes);
// phi from Gauss's law and psi from the Lorenz gauge of the state st
int field_initial_constraints_into(pic_ctx *ctx, const SpecState &st);
// transpose of the gather spectra's dependence on the trial current:
// jbar^ (3 Ng modes) from the cotangents sbar^ of [i k phi^{1/2} (dim),
// A^{n+1} (3)], times scale
int field_cn_adjoint(pic_ctx *ctx, const double2 *sbar, double2 *jbar, double scale);
// The transpose of the whole field step (adjoint of a step): ybar the 9
// spectral cotangents of the next state [phi, psi, A (3), U (3), rho], rbar
// the dim + 3 of the gather spectra [i k phi^{1/2}, A^{n+1}]; out receives
// 12 spectra [phi, psi, A (3), U (3), rho, j (3)] of the current state and
// the trial current, times scale.
int field_cn_state_adjoint(pic_ctx *ctx, const double2 *ybar, const double2 *rbar,
                           double2 *out, double scale);

// ---------------------------------------------------------------- checkpoint.cu
// A device-side snapshot of the accepted state in the checkpoint image's
// layout (no header, no validation), and its restore into the same context
// with the same particle count (drops a forward sensitivity).
uint64_t state_snapshot_bytes(const pic_ctx *ctx);
int state_snapshot(pic_ctx *ctx, void *dev);
int state_restore(pic_ctx *ctx, const void *dev, int64_t np, long long steps_done,
                  int sort_every, double E0);
// tangent of the field energy: dW = sum d W / d(phi, A, U) . (dphi, dA, dU)
int field_energy_tangent(pic_ctx *ctx, const SpecState &st, const SpecState &dst, double *dW);
int field_energy(pic_ctx *ctx, const double2 *phi_h, const double2 *A_h,
                 const double2 *U_h, double *W);
int field_constraints(pic_ctx *ctx, double *gauss_rms, double *lorenz_rms);
int field_mesh_work(pic_ctx *ctx, double *work);
// Nyquist projection of ncomp real mesh arrays (src may equal dst)
int field_project_real(pic_ctx *ctx, const double *src, double *dst, int ncomp);
int field_mesh_work_real(pic_ctx *ctx, const double *H, double *work);
// Queued forms of the commit-time sums (no synchronisation): raw sums into
// device slots (energy: 1, constraints: 2, mesh work: 1), scaled by the
// caller after one copy and one synchronisation for all of them.
int field_energy_queued(pic_ctx *ctx, double *dout);
int field_constraints_queued(pic_ctx *ctx, double *dout);
int field_mesh_work_real_queued(pic_ctx *ctx, const double *H, double *dout);

// ---------------------------------------------------------------- particle.cu
int particles_alloc(pic_ctx *ctx, int64_t n);
int particles_load(pic_ctx *ctx, const int32_t *sp, const int32_t *cell_in, const double *x,
                   const double *uP, int canonical, const double *w, int on_device);
int particles_form_P(pic_ctx *ctx);
int particles_point_deposit(pic_ctx *ctx, double *rho, double *J);
int particles_step_start(pic_ctx *ctx);
// queue the particle map and the copies of its counters and sums to pinned
// host memory; particles_map_finish reads them after the stream is synced
int particles_map_launch(pic_ctx *ctx, const StepConst &sc, int final_pass);
int particles_map_finish(pic_ctx *ctx, double *work_sum, double *chain_sum, EvalCounters *cnt);
// the final pass's work and chain-rule sums from the pinned partials
void particles_final_sums(const pic_ctx *ctx, double *work, double *chain);
int particles_commit(pic_ctx *ctx);
int particles_kinetic(pic_ctx *ctx, double *K);
int particles_kinetic_queued(pic_ctx *ctx);           // partials to psum_host, no sync
double particles_kinetic_collect(const pic_ctx *ctx);  // after the caller's sync
// refresh the particle-precision copy of A^n after A_real changed
int particles_refresh_A(pic_ctx *ctx);
int particles_export(pic_ctx *ctx, double *x, double *P, double *w, int32_t *sp,
                     int on_device);
int particles_export_eval(pic_ctx *ctx, double *vbar, double *Pnew, int32_t *iters,
                          int on_device);
int particles_export_u(pic_ctx *ctx, double *u, int on_device);
int particles_sort(pic_ctx *ctx);

// ---------------------------------------------------------------- det.cu
// buffers of the deterministic deposit (pic_start, pic_set_state); free them
int det_alloc(pic_ctx *ctx);
void det_free(pic_ctx *ctx);
// the orbit current of the last map evaluation, summed node by node in a
// fixed order from the particles' vbar, into J (overwriting it)
int det_deposit(pic_ctx *ctx, double *J, const StepConst &sc);
// pic_start's point deposits of rho (added to its contents) and J, in a fixed order
int det_point_deposit(pic_ctx *ctx, double *rho, double *J, const StepConst &sc);
// the particle sort's slots in the deterministic order
int det_sort_slots(pic_ctx *ctx, int64_t *slot);

// ---------------------------------------------------------------- tangent.cu
// advance the tangent through the converged step (before the commit) and
// commit it (after the state's commit); free it
int tangent_solve(pic_ctx *ctx, const StepConst &sc, double tol);
int tangent_commit(pic_ctx *ctx);
void tangent_free(pic_ctx *ctx);
// Newton-Krylov outer solver: scratch for the step (dual particle inputs at
// the step start), the inexact Newton direction (I - H'(j)) x = r by
// GMRES to relative residual eta (*iters: tangent map evaluations), release
struct NkState;
int nk_begin(pic_ctx *ctx, const StepConst &sc, NkState **out);
int nk_direction(pic_ctx *ctx, NkState *nk, const double *r, double eta, double *x, int *iters);
void nk_end(NkState *nk);

// ---------------------------------------------------------------- control.cu
// Algorithm 1's outer iteration decided on the device (one context)
struct StepOutcome {
  int status, why, outer_iters, map_evals, inner_max;
  int converged;  // the loop ended with the outer tests passed
  unsigned long long inner_sum, refined;  // of the final (verification) evaluation
  double res_srms, res_smax, work_p, chain;
};
int control_alloc(pic_ctx *ctx);
void control_free(pic_ctx *ctx);
void control_graphs_clear(pic_ctx *ctx);
// Runs the outer iteration of one step from the accepted current J_acc with
// the graphs of control.cu; *ran = 0 when they cannot be used (the caller
// then drives the step from the host).  On success of the step ctx->j holds
// the accepted current, ctx->H its map value from the final evaluation.
// from_j: start from the iterate already in ctx->j (a second stage) instead
// of J_acc; verify: run the verifying evaluation after the loop (without
// it the loop ends at the first iterate that passes the tests).
int step_control_device(pic_ctx *ctx, const StepConst &sc, double tr, double ta, StepOutcome *out,
                        int *ran, int from_j, int verify);

// ---------------------------------------------------------------- reduce.cu
// queue r = H - j and its test sums (copied to pinned host memory);
// resid_finish reads them after the stream is synced
int resid_launch(pic_ctx *ctx, const double *Hv, const double *jv, double *rv, double tau_r,
                 double tau_a);
void resid_finish(pic_ctx *ctx, ResidSums *out);
int dots(pic_ctx *ctx, const double *const *a, const double *const *b, int npairs, double *out);
int axpy_dir(pic_ctx *ctx, double *dir, const double *r, double beta,
             const double *const *dJ, const double *const *dR, const double *gam, int mh,
             size_t N3);
int lincomb(pic_ctx *ctx, double *out, const double *a, double alpha, const double *b,
            double beta_c, size_t N);
int diff_into(pic_ctx *ctx, double *out, const double *a, const double *b, size_t N);
