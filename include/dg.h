/*
 * dg.h -- C ABI of the GB300 (sm_103a) implementation of one explicit time step
 * of the second-order centroidal-Taylor discontinuous Galerkin (DG) scheme for the
 * Euler and ideal-MHD equations on a periodic Cartesian mesh
 * (Mocz, Vogelsberger, Sijacki, Pakmor & Hernquist 2013).
 *
 * Method (paper sections):
 *   Sec. 2.1  conservative system U = (rho, rho v, rho e, B), eq. `cons`;
 *             p_gas = (gamma - 1) rho u,  rho e = rho u + rho v^2/2 + B^2/2.
 *   Sec. 2.2  weak form (eq. `dg`); per cell a Taylor polynomial about the
 *             centroid, U = U_avg + dU/dx x + dU/dy y [+ dU/dz z]; evolution of
 *             averages (eq. `fv`, `fv3d`) and derivatives (eq. `dgderiv`,
 *             `dgderiv3d`) with the cell mass matrix; the magnetic field uses the
 *             locally divergence-free bases, V1..V5 in 2D:
 *             Bx = b1 + a3 x + a1 y,  By = b2 + a2 x - a3 y,
 *             and V1..V11 in 3D:
 *             Bx = b1 + (a10 + a11) x + a4 y + a5 z,  By = b2 + a6 x - a10 y + a7 z,
 *             Bz = b3 + a8 x + a9 y - a11 z.
 *   Sec. 2.3  face fluxes from the exact Riemann solver (Euler) or HLLD (MHD).
 *   Sec. 2.4  time integration: the two-stage SSP Runge-Kutta method (Gauss face
 *             rules), or the paper's MUSCL-Hancock step (half-step primitive
 *             prediction, one update; face-centroid or Gauss face rule).
 *   Sec. 2.5  slope limiting on primitive variables at every stage input: the
 *             min/max limiter or the WENO-type limiter.
 *   Sec. 2.6  the normal field at a face is the average of both sides.
 *   Time step dt = CFL / max_cells sum_d (|v_d| + c_d)/dx_d (c: sound speed, or
 *   the fast magnetosonic speed along d).
 *
 * Interchange layout (every state buffer crossing this ABI): float64, one plane
 * per coefficient, planes variable-major, each plane [nz][ny][nx] with x fastest.
 *   Taylor variables, in order: 2D Euler (rho, mx, my, E), 3D Euler
 *   (rho, mx, my, mz, E), 2D MHD (rho, mx, my, E), 3D MHD (rho, mx, my, mz, E);
 *   per variable the coefficients (average, d/dx, d/dy[, d/dz]) in physical
 *   units -> plane v*(dim+1)+k.  MHD then appends the magnetic block:
 *   (b1, b2, a1, a2, a3) in 2D, (b1, b2, b3, a4, ..., a11) in 3D.
 *   Number of planes: 12 (2D Euler), 20 (3D Euler), 17 (2D MHD), 31 (3D MHD);
 *   see dg_num_planes().
 *
 * Ownership: the caller owns every buffer it passes; the library copies in and
 * out and owns its device state.  Streams: all device work is enqueued on the
 * stream given to dg_init (NULL = legacy default stream).  Errors: functions never
 * abort or trap; they return a dg_status and keep a per-context message
 * (dg_last_error).  Device-side problems (non-physical states, Riemann-solver
 * failure) set a sticky device word that the next synchronising call reports as
 * DG_ENONPHYS.  A context is not thread safe: calls on one context must not
 * overlap.  Different contexts may be driven from different host threads at the
 * same time (the process-wide tile-shape tuning is serialised inside the library).
 */
#ifndef DG_H
#define DG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx; /* opaque, owned by the library */

typedef enum {
  DG_OK = 0,
  DG_EINVAL = 1,    /* invalid argument or configuration */
  DG_ENOMEM = 2,    /* device or host allocation failed */
  DG_ECUDA = 3,     /* a CUDA runtime call failed */
  DG_ENONPHYS = 4,  /* rho <= 0 or p <= 0 met, Riemann vacuum, or Newton failure */
  DG_ETIMEOUT = 5,  /* a bounded device wait ran out */
  DG_ESTATE = 6     /* call not valid in the context's current state */
} dg_status;

enum { DG_EULER = 0, DG_MHD = 1 };
enum { DG_FP64 = 0, DG_FP32 = 1 }; /* FP32: FP32 arithmetic and slopes, FP64 averages */
enum { DG_EXACT = 0, DG_HLLD = 1 };
/* Time integrators: the two-stage SSP Runge-Kutta method with 2-point Gauss face
 * rules, or the MUSCL-Hancock step of Sec. 2.4 (half-step prediction of the
 * primitive values from the cell centroid and the limited gradients, then one
 * update of the averages and moments by eq. `GalerkUpdate`: one kernel and one
 * read and write of the state per step). */
enum { DG_SSPRK2 = 0, DG_MUSCL_HANCOCK = 1 };

typedef struct {
  int eq;           /* DG_EULER | DG_MHD (3D MHD: limiter 0 or 1) */
  int dim;          /* 2 | 3 */
  int n[3];         /* cells per axis (n[2] ignored in 2D) */
  double box[3];    /* box lengths; cell size box[a]/n[a] */
  double gamma;     /* adiabatic index, > 1 */
  double cfl;       /* Courant number for the time step, > 0 */
  int limiter;      /* 0 off, 1 min/max limiter of Sec. 2.5, 2 the WENO-type
                       limiter of Sec. 2.5 (DG and min/max-limited stencil
                       gradients weighted by their oscillation factors) */
  int precision;    /* DG_FP64 | DG_FP32 */
  int riemann;      /* DG_EXACT (Euler) | DG_HLLD (MHD); must match eq */
  int ckpt_every;   /* adjoint checkpoint stride k (>= 1); 0 = no recording */
  int integrator;   /* DG_SSPRK2 | DG_MUSCL_HANCOCK */
  int face_points;  /* MUSCL-Hancock face rule: 1 (or 0) = one flux at the face
                       centroid with weight the face area (eq. `GalerkUpdate`),
                       2 = 2-point Gauss rule per face dimension; SSP-RK2 always
                       uses the Gauss rule and needs 0 or 2 */
} dg_config;

/* Number of interchange planes of a configuration, or -1 if it is invalid. */
int dg_num_planes(const dg_config* cfg);

/* Create a context: validates cfg, allocates the device state (three state
 * buffers in the internal layout: FP64 averages and FP64 or FP32 derivative
 * coefficients), binds `cuda_stream` (a cudaStream_t, may be NULL).
 * On success *out owns the context (free with dg_destroy).  DG_EINVAL on a bad
 * configuration, DG_ENOMEM / DG_ECUDA on allocation failure (*out = NULL). */
dg_status dg_init(const dg_config* cfg, void* cuda_stream, dg_ctx** out);

/* Create one context for `nprob` independent problems (same eq, dim, precision,
 * gamma, cfl, limiter; grid sizes and boxes may differ) that are stepped together
 * by one launch per Runge-Kutta stage, each with its own time step.  The state
 * buffers of dg_set_state / dg_get_state are then the concatenation of the
 * problems' interchange arrays in order. */
dg_status dg_init_batch(const dg_config* cfgs, int nprob, void* cuda_stream, dg_ctx** out);

void dg_destroy(dg_ctx* ctx);

/* Message describing the last failure of this context ("" if none).  The string
 * is owned by the context and valid until its next call. */
const char* dg_last_error(const dg_ctx* ctx);

/* Copy a state in (interchange layout, float64).  on_device != 0: `coeffs` is a
 * device pointer, else host memory (page-locked host memory is read in place by
 * the layout kernels; pageable memory is staged plane by plane).  Resets time and
 * step counters, clears the device error word and computes the first Courant
 * time step.  Synchronises the stream. */
dg_status dg_set_state(dg_ctx* ctx, const double* coeffs, int on_device);

/* Copy the current state out (interchange layout, float64; page-locked host
 * memory is written in place, pageable memory through device staging).
 * Synchronises. */
dg_status dg_get_state(dg_ctx* ctx, double* coeffs, int on_device);

/* Advance `nsteps` steps of the configured integrator.  dt_override > 0: every
 * step uses that time step; otherwise each step uses the Courant time step of
 * its input state, computed on the device (fused into the last kernel of the
 * previous step).
 * t_out (may be NULL) receives the simulation time after the steps (problem 0
 * of a batch).  Returns after enqueueing when t_out is NULL and no error is
 * pending; otherwise synchronises and reports the device error word. */
dg_status dg_step(dg_ctx* ctx, int nsteps, double dt_override, double* t_out);

/* Synchronise, then report the device error word (DG_OK or DG_ENONPHYS). */
dg_status dg_sync(dg_ctx* ctx);

/* Per-problem simulation time and the time step the next step would use
 * (host arrays of nprob entries; either may be NULL).  Synchronises. */
dg_status dg_get_times(dg_ctx* ctx, double* t, double* dt_next);

/* Totals V * sum_cells(average) of every conserved variable, FP64 with
 * compensated (Neumaier) summation: Taylor variables then, for MHD, the field
 * averages b1, b2 (2D) or b1, b2, b3 (3D).  `out` is a host array of
 * (nvar * nprob) doubles, nvar = 4 (2D) or 5 (3D) Taylor variables + 0, 2 or 3
 * field averages.  Synchronises. */
dg_status dg_totals(dg_ctx* ctx, double* out);

/* Sec. 2.6 Stokes estimate of div B per cell, (1/V) sum_faces B.n A with the
 * face-normal field averaged between the two sides and integrated with the
 * face Gauss rule.  MHD only.  `out`: ncell doubles ([ny][nx]); host or device
 * by on_device.  Synchronises. */
dg_status dg_divb(dg_ctx* ctx, double* out, int on_device);

/* Vector-Jacobian product of one SSP-RK2 step with the time step held fixed
 * (the reverse of dg_step for gradients of an objective of the final state;
 * DG_SSPRK2 contexts only):
 *   lam_prev = (d U^{n+1} / d U^n)^T lam_next,   U^{n+1} = step(U^n; dt).
 * u_n, lam_next, lam_prev: device pointers, interchange layout, float64; lam_prev
 * may not alias the other two.  One 2D problem, Euler or planar MHD (HLLD, the
 * divergence-free field basis), limiter 0 or 1 (the limiter contributes the
 * derivative of its active branch).  Other configurations: DG_EINVAL.  The context's own state is not changed.  Enqueued on the context
 * stream. */
dg_status dg_adjoint_step(dg_ctx* ctx, const double* lam_next, double* lam_prev,
                          const double* u_n, double dt);

/* Forward steps that record the trajectory for dg_adjoint: like dg_step, plus a
 * device checkpoint of the state every cfg.ckpt_every steps and the time step of
 * every step.  Successive calls extend one recording.  Any other change of the
 * state ends it: dg_set_state, or dg_step with nsteps > 0 (a later dg_record then
 * starts a new recording from the state reached, and dg_adjoint returns
 * DG_ESTATE until it does). */
dg_status dg_record(dg_ctx* ctx, int nsteps, double dt_override, double* t_out);

/* A counter that changes whenever the recorded trajectory changes (extended by
 * dg_record, ended by dg_step or dg_set_state), so that a caller that keeps a
 * recording for a later dg_adjoint can check that it is still the same one.
 * -1 for a null context.  No device work. */
long long dg_record_generation(const dg_ctx* ctx);

/* Gradient of an objective of the final recorded state with respect to the
 * state at the start of the recording, by reverse sweeps over the recorded
 * segments, recomputing each segment's states from its checkpoint:
 *   lam_0 = (d U^N / d U^0)^T lam_N.
 * Device pointers, interchange layout, float64.  Time steps are those recorded
 * (held fixed).  The context's current state is restored afterwards. */
dg_status dg_adjoint(dg_ctx* ctx, const double* lam_N, double* lam_0);

/* Conservation totals of a state held by the caller, for callers that may not
 * allocate device memory (the paper has no counterpart: this is a service of the
 * library, not a step of the method).  Same result as dg_totals -- V * sum of the
 * cell averages of every conserved variable, FP64 with compensated summation,
 * Taylor variables then (MHD) b1, b2[, b3] -- but without a context and without any
 * cudaMalloc/cudaFree: the per-block partial sums live in one fixed 512 KiB
 * static device array that every GPU loading the library keeps until exit.
 *   cfg: grid and equations of the state (precision, limiter and cfl unused).
 *   u: device pointer, interchange layout, float64.
 *   out: nvar doubles, device (out_on_device != 0) or host memory; a host
 *        result is waited for, a device one is only enqueued.
 *   cuda_stream: stream for the work (NULL = legacy default stream).
 * Limit: at most 16,777,216 cells (e.g. 256^3 or 4096^2); larger grids return
 * DG_EINVAL.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race, so
 * enqueue them one after another.  Failures are described by
 * dg_last_error(NULL). */
dg_status dg_totals_noalloc(const dg_config* cfg, const double* u, double* out,
                            int out_on_device, void* cuda_stream);

/* Measured fused multiply-add throughput of the current device (a diagnostic for
 * roofline fractions; the paper has no counterpart): every SM runs independent
 * FMA chains in FP64 (precision DG_FP64) or FP32 (DG_FP32) for ~20 ms, timed
 * with CUDA events on a private stream; *flops_per_s = 2 x FMAs per second, the
 * best of several runs.  The FP64 stage kernels are bound by the FP64 pipe, and
 * this is the peak their FP64 flop rate is reported against.  Allocates a small
 * buffer; synchronises.  Failures are described by dg_last_error(NULL). */
dg_status dg_peak_fma(int precision, double* flops_per_s);

/* Kernel timing with CUDA events recorded on the context stream around every
 * stage-kernel launch (enable != 0), or stop (0).  Enabling clears the record
 * and disables CUDA-graph replay for the recorded steps. */
dg_status dg_profile(dg_ctx* ctx, int enable);

/* Per-phase SM cycles of the stage kernels (2D and 3D SSP-RK2 stage kernels with
 * per-element staging) summed over their CTAs since profiling was last enabled.
 * Only the library's profiling build (compiled with DG_PHASE_PROFILE) counts
 * them; the normal build returns DG_EINVAL.  cycles[s * 16 + k] for stage s = 0, 1
 * and phase k; n >= 32.  2D phases: 0 staging, 1 primitives, 2 limiter, 3 faces,
 * 4 per-cell right-hand side and combination, 5 Courant reduction; 3D phases:
 * 0 staging and primitives, 1 limiter, 2 volume integral, 3/5/7 x/y/z faces,
 * 4/6/8 their gathers, 9 combination, 10 Courant reduction.  Synchronises. */
dg_status dg_phase_cycles(dg_ctx* ctx, double* cycles, int n);

/* Totals of the recorded kernel times: ms[k] and launches[k] for k = 0 (stage 1)
 * and 1 (stage 2 incl. the fused time-step reduction).  A batch of 2D problems
 * runs both stages in one launch per step, and a MUSCL-Hancock step is one
 * launch; both are counted under k = 1.  Synchronises. */
dg_status dg_profile_read(dg_ctx* ctx, double ms[2], long long launches[2]);

/* Name of the stage kernel and tile shape this context launches (chosen by the
 * autotuner when the state is first set), e.g. "stage2d_tma_kernel 16x16 fp32".
 * Owned by the context. */
const char* dg_kernel_name(const dg_ctx* ctx);

/* Algorithmic DRAM bytes of one stage-kernel launch on the whole grid (all
 * problems): stage 1 reads and writes one state, stage 2 reads two and writes
 * one (a batch of 2D problems: 0 for stage 1, both stages for stage 2; a
 * MUSCL-Hancock step: 0 for stage 1, one state read and one written for stage
 * 2).  Used for roofline figures. */
double dg_stage_bytes(const dg_ctx* ctx, int stage);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
