/*
 * lbm.h -- C ABI of the GB300 LBM-RANS wall-function solver.
 *
 * The library advances the lattice Boltzmann equation (Section 2.1, Eqs. 1-8)
 * on a uniform D2Q9 or D3Q19 lattice with the local relaxation time set by
 * molecular plus Spalart-Allmaras eddy viscosity (Section 2.2, Eqs. 10-14),
 * and imposes turbulent walls with either of the paper's two schemes:
 *   - slip-velocity half-way bounce-back (Section 3.2, Eqs. 31-35), and
 *   - the hybrid regularized condition with the blended wall-normal gradient
 *     (HRFD, Section 3.1, Eqs. 17-28),
 * both closed by the SA-consistent wall function (Eqs. 15-16) or the log law,
 * inverted for u_tau by an FP64 Newton iteration.
 *
 * Conventions
 *   - Every function returns an lbm_status; nothing throws across the ABI.
 *   - All physical inputs and outputs are SI; the library converts to lattice
 *     units with the acoustic scaling dt = M dx / (sqrt(3) U_ref) (Section 4.1.1).
 *   - Field arrays are float64, x fastest: index (z*ny + y)*nx + x; vector
 *     fields are component-major: comp*(nz*ny*nx) + cell.
 *   - Wall-node arrays of a y face hold one value per (z, x) node of the face,
 *     index z*nx + x, zero where the face is not a wall (x < x_start).
 *   - The library owns every device buffer it allocates (through cfg.alloc if
 *     given, else cudaMalloc) and never frees caller memory.
 *   - Work is enqueued on cfg.stream; lbm_step returns as soon as the work is
 *     enqueued. Functions that copy results to the caller synchronise that
 *     stream and report device-side failure flags.
 *   - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,        /* invalid argument or configuration */
  LBM_ENOMEM = 2,        /* device or host allocation failed */
  LBM_ECUDA = 3,         /* a CUDA runtime call failed (see lbm_last_error) */
  LBM_ENONFINITE = 4,    /* a population, velocity or nu_tilde became NaN/Inf */
  LBM_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  LBM_ENEWTON = 6,       /* the u_tau inversion did not converge at some node */
  LBM_EUNSUPPORTED = 7   /* valid request this build does not implement */
} lbm_status;

enum { LBM_D2Q9 = 9, LBM_D3Q19 = 19 };
enum { LBM_BGK = 0, LBM_REGULARIZED = 1 };
enum { LBM_FP32 = 0, LBM_FP16_SHIFTED = 1, LBM_BF16_SHIFTED = 2, LBM_FP64 = 3 };
enum { LBM_SA = 0, LBM_LAMINAR = 1 };
enum { LBM_LAW_SA_ANALYTIC = 0, LBM_LAW_LOG = 1 };

/* boundary kinds (lbm_bc.kind) */
enum {
  LBM_BC_PERIODIC = 0,
  LBM_BC_WALL_SLIP_BB = 1,     /* Section 3.2: Eq. 31 with the slip velocity of Eq. 35 */
  LBM_BC_WALL_HRFD = 2,        /* Section 3.1: Eq. 19 with Eqs. 23, 26-28 */
  LBM_BC_SYMMETRY = 3,         /* specular reflection (free slip) */
  LBM_BC_INLET_ZOUHE = 4,      /* Zou-He velocity inlet (xmin only) */
  LBM_BC_OUTLET_ZEROGRAD = 5,  /* zero-gradient outlet (xmax only) */
  LBM_BC_FREESTREAM = 6,       /* incoming populations at f^eq(rho0, u_in) */
  LBM_BC_WALL_CAI_DEGRIGNY = 7 /* Section 3.1.2: regularized wall (Eqs. 19, 23, 26) whose
                                  wall-normal gradient is the third-order difference of
                                  the wall function, Eqs. 29-30 */
};

/* bounce-back wall whose boundary nodes are not half-way from the wall
   (lbm_bc.interp; Section 3.2): the reflected population of each crossing link
   is interpolated along the link at the wall fraction q = d_w */
enum {
  LBM_IBB_NONE = 0,            /* half-way bounce-back, Eq. 31 (d_w must be 1/2) */
  LBM_IBB_BOUZIDI = 1,         /* Bouzidi et al., Eq. 36 (two branches at q = 1/2) */
  LBM_IBB_YU = 2               /* Yu et al., Eq. 37 (one expression for every q) */
};

/* faces (lbm_set_bc face argument) */
enum { LBM_XMIN = 0, LBM_XMAX = 1, LBM_YMIN = 2, LBM_YMAX = 3, LBM_ZMIN = 4, LBM_ZMAX = 5 };

/* lbm_fields masks; dst[k] receives the k-th set bit in this order */
enum {
  LBM_FIELD_RHO = 1u << 0,      /* nz*ny*nx, kg/m^3 */
  LBM_FIELD_U = 1u << 1,        /* 3*nz*ny*nx, m/s */
  LBM_FIELD_NU_T = 1u << 2,     /* nz*ny*nx, m^2/s, nu_tilde * f_v1 (Eq. 10) */
  LBM_FIELD_NU_TILDE = 1u << 3, /* nz*ny*nx, m^2/s */
  LBM_FIELD_UTAU_YMIN = 1u << 4,/* nz*nx, m/s */
  LBM_FIELD_UTAU_YMAX = 1u << 5,/* nz*nx, m/s */
  LBM_FIELD_CF_YMIN = 1u << 6,  /* nz*nx, 2 (u_tau / U_ref)^2 */
  LBM_FIELD_CF_YMAX = 1u << 7
};

typedef struct {
  int lattice;                 /* LBM_D2Q9 | LBM_D3Q19 */
  int nx, ny, nz;              /* cells; nz = 1 for D2Q9 */
  double dx;                   /* m */
  double nu;                   /* m^2/s */
  double rho0;                 /* kg/m^3 */
  double u_ref;                /* m/s, sets dt with mach */
  double mach;                 /* dt = mach*dx/(sqrt(3)*u_ref) */
  double force[3];             /* body acceleration g (m/s^2); F = rho0 g */
  double origin[3];            /* physical coordinates of the domain's low corner */
  int collision;               /* LBM_BGK | LBM_REGULARIZED */
  int storage;                 /* LBM_FP32 | LBM_FP16_SHIFTED | LBM_BF16_SHIFTED | LBM_FP64 */
  int turbulence;              /* LBM_SA | LBM_LAMINAR */
  int wall_law;                /* LBM_LAW_SA_ANALYTIC (Eq. 16) | LBM_LAW_LOG */
  double kappa, B;             /* log-law constants */
  double u_shift;              /* m/s, x velocity U of the stored deviations: populations are
                                  kept as f_i - f_i^eq(rho0, U x) (0: f_i - w_i rho0); set it
                                  to the mean flow to keep the stored values small */
  int staging;                 /* inner-row population loads: 0 = direct loads through L1
                                  (default, fastest measured); 1 = TMA tiles staged in shared
                                  memory, double-buffered over z planes */
  void* (*alloc)(size_t bytes, void* user);  /* optional device allocator */
  void (*free)(void* ptr, void* user);
  void* alloc_user;
  void* stream;                /* cudaStream_t; NULL = legacy default stream */
} lbm_config;

typedef struct {
  int kind;                    /* LBM_BC_* */
  double beta;                 /* HRFD blend of Eq. 27 (0.28 calibrated) */
  int ref_node;                /* bounce-back: 1 = B, 2 = F; HRFD requires 2 (F) */
  double x_start;              /* walls: active where cell-centre x >= x_start;
                                  cells before it behave as a symmetry plane */
  double u_in[3];              /* inlet / free-stream velocity, m/s */
  double nut_ratio_in;         /* inlet / free-stream nu_tilde / nu */
  double d_w;                  /* walls: distance from the wall to the boundary nodes in
                                  lattice spacings, (0, 1]; 0 selects the half-way 1/2.
                                  It sets y_B = d_w Delta in the wall function, Delta_w
                                  in Eq. 35, Newton's reference height, the SA wall
                                  distance and the bounce-back link fraction q
                                  (Section 4.1.2.5) */
  int interp;                  /* bounce-back walls: LBM_IBB_*; d_w != 1/2 needs
                                  LBM_IBB_BOUZIDI or LBM_IBB_YU */
} lbm_bc;

typedef struct {
  double mass;                 /* sum of populations (lattice units, rho0 = 1) */
  double momentum[3];          /* sum of c_i f_i over the lattice (lattice units) */
  double mean_u_tau[2];        /* m/s, mean over wall nodes of ymin / ymax */
  double max_rel_du_tau;       /* max |u_tau - u_tau_prev| / u_tau over wall nodes since
                                  the previous lbm_diagnostics call (Section 4.1.1 criterion) */
  int nonfinite;               /* 1 if any population was NaN/Inf */
  int newton_failures;         /* wall-node updates whose Newton iteration reached its
                                  100-iteration limit since the state was set (a count
                                  summed over steps and nodes; the last iterate is used) */
} lbm_diag;

typedef struct lbm_ctx lbm_ctx;

/* Create a solver for one lattice (Section 2.1: the D2Q9 / D3Q19 velocity sets
   of Eq. 3; Eq. 8 for the relaxation time; the acoustic scaling of Section
   4.1.1, dt = M dx / (sqrt(3) U_ref), converts cfg's SI inputs to lattice units).
   All faces start periodic.  Validates the configuration: tau0 = 1/2 + 3 nu_lb
   must exceed 1/2, sizes positive (nz = 1 for D2Q9), Q x padded cells < 2^31,
   enum values known; returns LBM_EINVAL (or LBM_EUNSUPPORTED for a lattice too
   large for 32-bit indexing) with the reason in lbm_last_error(NULL).
   cfg is copied; the caller keeps ownership of it.  On success *out owns all
   device state (allocated through cfg->alloc if set, else cudaMalloc); on
   failure *out is NULL and nothing is leaked (LBM_ENOMEM, LBM_ECUDA). */
lbm_status lbm_create(const lbm_config* cfg, lbm_ctx** out);

/* Set the condition of one face (LBM_XMIN..LBM_ZMAX) before the first
   lbm_set_fields/lbm_step.  Rejects combinations the method does not define:
   walls only on y faces, inlet only on xmin, outlet only on xmax, z periodic,
   periodic faces paired, HRFD needs ny >= 3 (B, F, FF) per wall. */
lbm_status lbm_set_bc(lbm_ctx* ctx, int face, const lbm_bc* bc);

/* Initial state from physical fields rho (nz*ny*nx), u (3*nz*ny*nx), nu_tilde
   (nz*ny*nx): post-collision populations f* = f^eq(rho, u) (Eq. 17), u^0 = u.
   on_device != 0: the pointers are device memory; else host memory. */
lbm_status lbm_set_fields(lbm_ctx* ctx, const double* rho, const double* u,
                          const double* nu_tilde, int on_device);

/* Enqueue nsteps full steps on cfg.stream, each in the order SA update
   (Section 2.2, Eqs. 10-14, explicit Euler), bounce-back wall pre-pass (Section
   3.2, Eqs. 31-35 with the Newton inversion of Eq. 16 or the log law), pull
   streaming (Eq. 3) with the face conditions, regularized wall reconstruction
   (Section 3.1, Eqs. 19-28, or Eq. 29), moments (Eqs. 4-5) and collision with
   omega from nu + nu_t (Eq. 8).  Returns once the work is enqueued (no host
   synchronisation).  A lattice with walls and at least 2^21 cells launches each
   step's three kernels directly, so that the wall pre-pass overlaps the inner
   rows on a high-priority stream; other lattices replay pairs of steps from
   captured CUDA graphs (one per buffer parity).  Errors: LBM_EINVAL for nsteps < 0 or
   no state yet (lbm_set_fields / lbm_set_state first), face validation errors
   of the first step, LBM_ECUDA for a failed launch or capture.  Device-side
   failures (non-finite values, Newton limit) are reported by the next call
   that synchronises (lbm_fields, lbm_diagnostics). */
lbm_status lbm_step(lbm_ctx* ctx, int nsteps);

/* Same steps launched without a graph, one kernel after the other, with CUDA
   events around them; summed over the nsteps: kernel_ms[0] the bulk rows
   (inner rows, then wall rows; every row of a lattice without walls),
   kernel_ms[1] the wall pre-pass, kernel_ms[2] the inner rows alone (the
   face-free kernel; equal to kernel_ms[0] without walls).  Synchronises
   cfg.stream.  Bookkeeping for benchmarks: the paper has no counterpart. */
lbm_status lbm_step_timed(lbm_ctx* ctx, int nsteps, float kernel_ms[3]);

/* Copy the fields selected by mask (LBM_FIELD_*) into caller buffers dst[k]
   (float64, physical units), in increasing bit order: rho = sum f_i (Eq. 4) and
   u (Eq. 5, with the F/2 shift) of the last collision, nu_t = nu_tilde f_v1
   (Eq. 10), nu_tilde, and per wall node u_tau (Newton on Eq. 16 / the log law)
   and C_f = 2 (u_tau / U_ref)^2 (the skin-friction coefficient of Section 4.2.2
   with U_ref the reference speed of cfg).  dst_on_device != 0: device pointers,
   else host pointers; the caller owns them and sizes them as the LBM_FIELD_*
   comments state.  Synchronises cfg.stream.  Returns LBM_ENONFINITE if the
   state holds NaN/Inf and LBM_ENEWTON if the u_tau inversion reached its
   iteration limit at some wall node since the state was set (the fields are
   copied in both cases); LBM_EINVAL for unknown mask bits, a NULL dst entry or
   no state yet. */
lbm_status lbm_fields(lbm_ctx* ctx, unsigned mask, void* const* dst, int dst_on_device);

/* FP64 reductions over the lattice (deterministic order) into *out, host
   memory: total mass and momentum of the post-collision populations (the
   quantities Eq. 23 of Section 3.1 is built to conserve), mean u_tau per wall
   and the relative u_tau change of the convergence criterion (Section 4.1.1).
   Synchronises cfg.stream.  Non-finite values and Newton failures are reported
   in *out (nonfinite, newton_failures) with LBM_OK; LBM_ETIMEOUT if a bounded
   device-side wait gave up. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, lbm_diag* out);

/* Convergence-driven run (Section 4.1.1: runs are converged when the relative
   change of u_tau falls below 1e-4).  Advances in chunks of check_every steps
   (the last chunk may be shorter); after each chunk the largest relative change
   of u_tau over the wall nodes since the previous check,
   max |u_tau - u_tau_prev| / u_tau, is compared with tol, and the run stops at
   the first check below tol or after max_steps steps.  The paper states the
   criterion per iteration; a chunk of m steps applies it to the change over m
   steps (m = 1 is the literal per-step form).  The u_tau of the state at entry
   is the first reference, so a run stops after one chunk at the earliest.
   *steps_done receives the steps taken and *residual the last checked change
   (converged if and only if *residual < tol; INFINITY before the first check).
   Synchronises cfg.stream once per chunk.  Errors: LBM_EINVAL for tol <= 0,
   check_every < 1, max_steps < 0, NULL outputs, no state yet, or a lattice
   without walls; LBM_ENONFINITE when a wall u_tau is NaN/Inf; step errors as
   lbm_step.  Resets the reference of lbm_diagnostics' max_rel_du_tau. */
lbm_status lbm_run_to_convergence(lbm_ctx* ctx, double tol, int check_every, long long max_steps,
                                  long long* steps_done, double* residual);

/* Raw state for checkpointing: the post-collision populations in storage
   precision (bytes reported by lbm_state_bytes), the per-cell records of
   velocity and nu_tilde (u_x, u_y, u_z, nu_tilde) in compute precision and
   u_tau in FP64, concatenated.  dst and src
   are host buffers of lbm_state_bytes(ctx) bytes. */
size_t lbm_state_bytes(const lbm_ctx* ctx);
lbm_status lbm_get_state(lbm_ctx* ctx, void* dst);
lbm_status lbm_set_state(lbm_ctx* ctx, const void* src);

/* Release everything the context owns (after synchronising its stream):
   device buffers through cfg.free (or cudaFree), captured graphs, the side
   streams and events.  Caller memory is never freed.  NULL is allowed.  A batch
   that holds the context must be destroyed first. */
void lbm_destroy(lbm_ctx* ctx);

/* Message of the last failure of this context (static storage if ctx is NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Number of kernels this context has put on the GPU since lbm_create: every
   launch of lbm_set_fields, lbm_step (the kernels of replayed graphs
   included), lbm_step_timed, lbm_fields and lbm_diagnostics.  A host-side
   count that never synchronises; 0 for NULL.  Bookkeeping for benchmarks: the
   paper has no counterpart. */
unsigned long long lbm_kernel_launches(const lbm_ctx* ctx);

/* Steps advanced since lbm_create (lbm_step, lbm_step_timed, lbm_run_to_convergence
   and batch launches that include the context); -1 for NULL.  Bookkeeping: the
   paper has no counterpart. */
long long lbm_steps_done(const lbm_ctx* ctx);

/* Polls a bounded device-side wait of this context's kernels makes before it
   gives up (default 2^24, about a second): the waits of the TMA-staged
   inner-row kernel (cfg.staging = 1) for its tiles.  A wait that gives up makes
   its block wait (with the default bound) for its copies in flight and leave;
   the next synchronising call returns LBM_ETIMEOUT and the state is not valid.
   polls = 0 makes every such wait give up at once: a test of that failure path,
   with no fault and no hang.  LBM_EINVAL for polls < 0.  The paper has no
   counterpart. */
lbm_status lbm_set_wait_limit(lbm_ctx* ctx, long long polls);

/* Lattice parameters after unit conversion: out[0] = dt (s), out[1] = nu
   (lattice), out[2] = tau0, out[3..5] = F (lattice). */
lbm_status lbm_lattice_params(const lbm_ctx* ctx, double out[6]);

/* Mass and momentum (lattice units: out[0] = sum of populations, out[1..3] =
   sum of c_i f_i) of a caller-owned population array, computed without
   allocating any memory.  The paper has no counterpart: this serves callers
   that cannot allocate device memory at the point of the call (applications
   that hand the library fixed buffers, allocators that forbid growth, loops
   where an allocation would synchronise the device).
   f: device pointer to Q * pitch*ny*nz populations in `storage` precision,
      laid out as lbm_get_state's population block (shifted deviations
      f_i - w_i, x fastest, rows of `pitch` >= nx elements).  For a state
      created with a nonzero u_shift the block holds f_i - f_i^eq(rho0, U x)
      and out[1] then lacks the constant U (lattice units) per cell.
   out: device pointer to 4 doubles, written asynchronously on `stream`.
   Partial sums live in one fixed 128 KiB static device array shared by all
   calls (held on every GPU that loads the library until exit): lattices above
   16,777,216 cells are rejected with LBM_EINVAL, calls that overlap on the GPU
   race and must be serialised by the caller, and the first call on each device
   looks up the array's address (make it before any stream capture).  That
   address is kept for the life of the process: after a cudaDeviceReset it is
   stale, so do not call this entry point on a device that has been reset.
   Devices with index >= 64 are rejected with LBM_EUNSUPPORTED.  Errors are
   described by lbm_last_error(NULL). */
lbm_status lbm_moments_noalloc(const void* f, int lattice, int storage, int nx, int ny, int nz,
                               int pitch, double* out, void* stream);

/* ------------------------------------------------------------------------
 * Batched sweeps (a mesh-sensitivity sweep of many channel and plate
 * instances; the paper runs its grid and Reynolds-number studies of Sections
 * 4.1.2.4 and 4.1.2.6 as separate runs).  Many independent contexts are
 * advanced together, in one of two modes.  Mode 0: one persistent, cooperative
 * kernel launch per lbm_batch_step call, replayed from a captured CUDA graph;
 * work items, each taken by one warp in a fixed order from a ticket counter,
 * are chunks of 32 wall nodes (the wall pre-pass) and ranges of cells of one
 * instance; an item waits only for the items of its own instance it depends
 * on (the previous step, or this step's wall pre-pass for the wall rows), with
 * bounded waits that report LBM_ETIMEOUT.  Mode 1: per step, one launch per
 * kind of item over every instance (wall pre-pass, then wall rows, beside the
 * face-free cells), one CTA per item, launched directly (the wall branch's
 * stream priority holds only for direct launches); no device-side waits.  The autotuner picks the faster mode.  Each
 * step of an instance computes what lbm_step computes.  Instances keep their own configurations and boundary conditions;
 * the contexts must have been created and initialised (lbm_set_fields) first,
 * must share one storage type and one stream, and are read back with
 * lbm_fields / lbm_diagnostics.  The batch does not own the contexts; destroy
 * it before them.
 * ---------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* ctxs: n distinct contexts (host array, copied).  LBM_EINVAL for n < 1, NULL
   or repeated contexts, a context without state or mixed storage types. */
lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, lbm_batch** out);
/* Advance every instance by nsteps (enqueued on the contexts' stream; returns
   without waiting for the GPU).  The tile size (cells per work item, one warp
   each) and threads per CTA are chosen by the built-in autotuner on the first
   call unless lbm_batch_tune fixed them; the autotuner advances every instance
   while it times (28 steps).  A bounded wait of an earlier launch that gave up
   is reported here (LBM_ETIMEOUT) once that launch has finished, or by
   lbm_batch_wait, also when later launches were enqueued meanwhile; the
   instances' states are then not valid.  Each launch's failure record is copied
   to its own host slot; with four launches of the persistent kernel still in
   flight, the next call first waits for the oldest. */
lbm_status lbm_batch_step(lbm_batch* b, int nsteps);
/* Time the candidate tile sizes (64, 256, 1024 cells per warp item) and block
   sizes (128, 256 threads) of mode 0 and the launches of mode 1 once, keep the
   fastest configuration of mode 0 and the faster mode (unless
   lbm_batch_set_mode fixed it); best[0] = threads per CTA, best[1] = cells per
   tile of mode 0 (best may be NULL).  Advances every instance by 28 steps.
   Synchronises. */
lbm_status lbm_batch_tune(lbm_batch* b, int best[2]);
/* mode 0: the persistent ticketed kernel, 1: per-step multi-instance launches,
   -1: the autotuner's choice (default).  The paper has no counterpart. */
lbm_status lbm_batch_set_mode(lbm_batch* b, int mode);
/* Wait for the batch's launches to finish; LBM_ETIMEOUT if a bounded wait of
   the last launch gave up. */
lbm_status lbm_batch_wait(lbm_batch* b);
/* Polls a waiting warp makes before it gives up (default 2^24, about a
   second).  polls = 0 makes every wait that would have to poll give up at once
   (every warp then leaves the kernel and lbm_batch_wait reports LBM_ETIMEOUT):
   a test of that failure path, with no fault and no hang.  The paper has no
   counterpart. */
lbm_status lbm_batch_set_wait_limit(lbm_batch* b, long long polls);
/* out[0] = threads per CTA, out[1] = cells per work item, out[2] = 1 if the
   launches are replayed from a captured graph (mode 0; 0 in mode 1, whose
   launches are direct, or if capture was refused), out[3] = work items per
   step, out[4] = the mode the steps run in (0 or 1, see lbm_batch_set_mode). */
lbm_status lbm_batch_info(const lbm_batch* b, int out[5]);
void lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
