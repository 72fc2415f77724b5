/*
 * lbmd.h -- C ABI of the GB300 (sm_103a) coupled lattice-Boltzmann / polymer
 * molecular-dynamics step of Fyta, Melchionna, Kaxiras and Succi,
 * "Coupling Lattice Boltzmann with Atomistic Dynamics for the multiscale
 * simulation of nano-biological flows" (arXiv:0710.1272).
 *
 * One call of lbmd_step advances the coupled system by one LB time step
 * (Delta t = 1) following the four-stage scheme of Sec. II:
 *   (1) interpolate the fluid velocity u(x) to the beads,
 *   (2) run M MD substeps (Delta t_MD = 1/M) with u frozen,
 *   (3) extrapolate the bead friction + random forces back to the grid,
 *   (4) advance the D3Q19 populations by one stream-collide (Eq. 5).
 *
 * Conventions shared by every entry point:
 *  - All functions return an int status: LBMD_OK (0) or a negative LBMD_E*
 *    code.  A CUDA failure inside a context is sticky: later calls on that
 *    context return LBMD_ECUDA until it is destroyed.
 *  - The library never allocates device memory.  The caller passes one device
 *    workspace (size from lbmd_workspace_size, 256-byte aligned) and a CUDA
 *    stream (a context also keeps a small pinned host buffer, 48 n_beads + 64
 *    bytes, for host read-outs of the beads); every kernel runs on that stream or on a private second stream
 *    that is forked from and joined back into it.  The caller owns the
 *    workspace, the stream and every output buffer.
 *  - Work is asynchronous on the stream unless a function says it
 *    synchronises.
 *  - Lattice arrays are structure-of-arrays, x fastest: a scalar field is
 *    [z][y][x] (V = nx*ny*nz entries); a vector field is [3][z][y][x]; the
 *    populations are [19][z][y][x].
 *  - D3Q19 population order: 0 rest; 1/2 = +x/-x; 3/4 = +y/-y; 5/6 = +z/-z;
 *    7/8 = (+1,+1,0)/(-1,-1,0); 9/10 = (+1,-1,0)/(-1,+1,0);
 *    11/12 = (+1,0,+1)/(-1,0,-1); 13/14 = (+1,0,-1)/(-1,0,+1);
 *    15/16 = (0,+1,+1)/(0,-1,-1); 17/18 = (0,+1,-1)/(0,-1,+1).
 *  - Not thread-safe per context; separate contexts are independent.
 */
#ifndef LBMD_H
#define LBMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LBMD_OK 0
#define LBMD_EINVAL (-1)       /* a parameter or argument is out of range    */
#define LBMD_ESIZE (-2)        /* workspace too small or misaligned          */
#define LBMD_ECUDA (-3)        /* a CUDA runtime call failed (sticky)        */
#define LBMD_EUNSUPPORTED (-4) /* valid for the method, not built here       */

/* ---- per-chain state word (lbmd_status) -------------------------------- */
#define LBMD_RUNNING 0
#define LBMD_TRANSLOCATED 1 /* every bead on the trans side x < wall_x      */
#define LBMD_RETRACTED 2    /* crossed, then all beads back past the pore   */
#define LBMD_NAN 3          /* a bead position or velocity, or a population
                               after a stream-collide, is not finite        */
#define LBMD_SHAKE_FAIL 4   /* the constraint solve did not converge        */

/* ---- option values ----------------------------------------------------- */
#define LBMD_STORE_F32 0  /* populations stored as float deviations        */
#define LBMD_STORE_F16 1  /* ... as IEEE half deviations f - w_p rho0      */
#define LBMD_STORE_BF16 2 /* ... as bfloat16 deviations                    */
#define LBMD_FORCING_PAPER 0 /* first-order source (w_p/c_s^2) c_p.F, Eq. 10 */
#define LBMD_FORCING_GUO 1   /* Guo second-order forcing for the body force  */
#define LBMD_COUPLING_TRILINEAR 0 /* 8-node trilinear gather / spread        */
#define LBMD_COUPLING_NGP 1       /* nearest grid point (the paper's choice) */
#define LBMD_STREAM_PULL 0 /* two population buffers, pull streaming (A -> B) */
#define LBMD_STREAM_AA 1   /* one buffer, in-place AA-pattern streaming      */

/* Largest chain one context accepts (one GPU thread block per chain). */
#define LBMD_MAX_BEADS 1024

/*
 * Problem statement of Sec. III plus the method parameters of Sec. II.
 * All lengths and times are in lattice units (Delta x = Delta t = 1).
 * Host pointers in this struct are read during lbmd_create only.
 */
typedef struct lbmd_params {
  int32_t nx, ny, nz;          /* box; periodic in every direction          */
  int32_t wall_x;              /* first x-layer of the wall; -1: no wall    */
  int32_t wall_thickness;      /* wall layers (paper: 1)                    */
  int32_t pore_d;              /* side of the square pore (paper: 3); 0: closed */
  int32_t pore_y0, pore_z0;    /* lowest pore node; -1: centred, (n - d)/2  */
  int32_t y_walls;             /* 1: solid rows y = 0 and y = ny-1          */
  int32_t storage;             /* LBMD_STORE_*                              */
  int32_t forcing;             /* LBMD_FORCING_*                            */
  int32_t coupling;            /* LBMD_COUPLING_*                           */
  int32_t n_beads;             /* 0 .. LBMD_MAX_BEADS                       */
  int32_t md_substeps;         /* M of Sec. II (paper: 5), 1 .. 255         */
  int32_t n_constraints;       /* -1: linear chain of n_beads-1 bonds of
                                  bond_length; 0: free beads; >0: the bonds
                                  below (must form the linear chain k, k+1) */
  int32_t shake_max_iter;      /* Newton iterations per constraint solve    */
  int32_t solvent_free;        /* 0: beads coupled to the LB solvent (Sec. II);
                                  1: no solvent (Sec. III's comparison run):
                                  u_i = 0, no LB step, no back-reaction; the
                                  beads keep drag, noise, wall and drive.
                                  Needs n_beads >= 1.                        */
  int32_t diag_every;          /* record the chain diagnostics (lbmd_diag)
                                  at the end of every diag_every-th step;
                                  0: never                                  */
  int32_t diag_capacity;       /* records kept (later ones are dropped)     */
  int32_t streaming;           /* LBMD_STREAM_*: how Eq. 5's free streaming
                                  moves the populations.  PULL keeps two
                                  buffers; AA (in-place, Bailey et al. 2009)
                                  keeps one, halving the population memory,
                                  with the same results and the same bytes
                                  moved per node update.  Single-box contexts
                                  only.                                     */
  double tau;                  /* BGK relaxation time, nu = (tau - 1/2)/3   */
  double rho0;                 /* reference density (paper: 1)              */
  double body_force[3];        /* uniform force density g                   */
  double bead_mass;            /* m (paper: unspecified; 1)                 */
  double gamma;                /* friction coefficient of Eq. 4 (paper 0.1) */
  double kT;                   /* 1/beta (paper: 1e-4)                      */
  double lj_sigma, lj_eps;     /* Eq. 2, truncated at 2^(1/6) sigma         */
  double kappa_phi;            /* bending stiffness of Eq. 3                */
  double f_drive;              /* pulling force in the pore (paper: 0.02)   */
  double bond_length;          /* b (paper: 1.2) for n_constraints == -1    */
  double shake_tol;            /* max |d^2 - b^2| / b^2 accepted            */
  double init_tg_amp;          /* Taylor-Green amplitude if init_u == NULL  */
  double kT_fluid;             /* temperature of the thermal source F_p of
                                  Eq. 5 (fluctuating LB); 0: no source.
                                  Single-box contexts only.                 */
  uint64_t seed;               /* Philox key of the bead and fluid noise    */
  const int32_t *bond_i;       /* host, n_constraints entries               */
  const int32_t *bond_j;
  const double *bond_len;
  const double *init_pos;      /* host, 3*n_beads, unwrapped [i][xyz]; NULL:
                                  the library's seeded start (Sec. III: the
                                  chain on the cis side, one end in the pore):
                                  bead 0 at (wall_x + wall_thickness, pore
                                  centre), bead 1 one bond along +x, then a
                                  self-avoiding walk of Philox-drawn random
                                  directions (keyed by seed), every bead
                                  after the first two at least 2^(1/6) sigma
                                  from the wall plane, from every solid node
                                  and from beads two or more places away
                                  (minimum image).  lbmd_create fails with
                                  LBMD_EINVAL if no such walk fits the box.  */
  const double *init_vel;      /* host, 3*n_beads or NULL (zero)             */
  const double *init_rho;      /* host, V or NULL (rho0)                     */
  const double *init_u;        /* host, 3*V SoA or NULL                      */
} lbmd_params;

typedef struct lbmd_ctx lbmd_ctx; /* opaque */

/*
 * Chain diagnostics of Sec. III at the end of an LB step.  Untranslocated
 * beads are those with unwrapped x >= wall_x, translocated ones x < wall_x
 * (every bead is untranslocated without a wall).
 */
typedef struct lbmd_diag {
  int64_t step;      /* LB steps completed                                   */
  int32_t n_trans;   /* N_T                                                  */
  int32_t reserved;
  double r_u, r_t;   /* radii of gyration of the untranslocated and the
                        translocated beads (0 for an empty part)             */
  double r_e;        /* effective radius (R_T^(1/mu) + R_U^(1/mu))^mu, mu = 0.6 */
  double s_h;        /* m gamma sum_i v_i . u_i: work rate of the fluid (Eq. 13) */
  double s_e;        /* sum_i F_drive,i . v_i: work rate of the drive (Eq. 14) */
  double kinetic;    /* m/2 sum_i |v_i|^2                                    */
} lbmd_diag;

/*
 * Bytes of device workspace lbmd_create needs for these parameters: the
 * state of the Sec. II scheme -- the D3Q19 populations of Eq. 5 (two buffers,
 * one with LBMD_STREAM_AA), the Sec. III wall as a solid bitfield and link
 * masks, the bead positions, velocities and neighbour lists of Eqs. 1-4, the
 * transfer weights and impulse sums of the coupling (Eq. 10) -- and read-out
 * staging.
 * Validates the parameters; no CUDA call, callable without a GPU.
 * Errors: LBMD_EINVAL (bad parameter, message in lbmd_last_message).
 */
int lbmd_workspace_size(const lbmd_params *params, size_t *bytes);

/*
 * Build the geometry of Sec. III (wall at x = wall_x, centred d x d pore,
 * optional y-walls), the equilibrium populations f = f_eq(rho, u) of the
 * initial fields, and the bead state; everything is written into the caller's
 * workspace on `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * The call synchronises the stream before it returns.  With beads it marks
 * the chain's buffers (about 1 MB for 400 beads) as an L2-persisting access
 * window for the context's own kernels, raising the CUDA context's
 * persisting-L2 limit (cudaLimitPersistingL2CacheSize) to that size if it is
 * lower; nothing else of the device's state is changed.
 * Errors: LBMD_EINVAL, LBMD_ESIZE (bytes too small or workspace not 256-byte
 * aligned), LBMD_EUNSUPPORTED (constraint topology other than a linear
 * chain), LBMD_ECUDA.  On error *out is NULL and nothing is leaked.
 */
int lbmd_create(const lbmd_params *params, void *dev_workspace, size_t bytes,
                void *cuda_stream, lbmd_ctx **out);

/*
 * Advance n_steps coupled LB steps (Sec. II scheme above), asynchronously on
 * the context's stream.  The steps replay a CUDA graph captured at the first
 * call (disabled while kernel timing is on).  n_steps >= 0.
 * Errors: LBMD_EINVAL, LBMD_ECUDA.
 */
int lbmd_step(lbmd_ctx *ctx, int64_t n_steps);

/*
 * Density rho (V floats) and velocity u = sum_p f_p c_p / rho (3*V floats,
 * [3][z][y][x]) of the current pre-collision populations (Eqs. 7-8; with Guo
 * forcing u carries the +g/(2 rho) shift).  Solid nodes read 0.
 * dst_is_device: 1 if rho/u are device pointers (stream-ordered, async);
 * 0 for host memory (the call synchronises).  Either pointer may be NULL.
 */
int lbmd_read_fields(lbmd_ctx *ctx, float *rho, float *u, int dst_is_device);

/*
 * The 19 pre-collision populations f_p(x, t) of Eq. 5 (19*V floats,
 * [19][z][y][x]), i.e. after streaming and bounce-back, before the next
 * collision; the density and velocity of Eqs. 7-8 are their moments.  Solid
 * nodes read 0.  dst_is_device as above.
 */
int lbmd_read_populations(lbmd_ctx *ctx, float *f, int dst_is_device);

/*
 * Bead positions (unwrapped, 3*n_beads doubles [i][xyz]) and velocities: the
 * state advanced by the MD substeps of Sec. II (Eqs. 1-4); unwrapped x is what
 * the Sec. III translocation count N_T compares with wall_x.
 * dst_is_device as above.  Either pointer may be NULL.  A host read-out also
 * fetches the status word in the same synchronisation, so an lbmd_status
 * call before the next lbmd_step does not synchronise again.
 */
int lbmd_read_beads(lbmd_ctx *ctx, double *pos, double *vel, int dst_is_device);

/* Status word at the start of the block of lbmd_read_beads_async (fields as
 * lbmd_status). */
typedef struct lbmd_status_word {
  int64_t step;        /* LB steps completed                               */
  int64_t t_transloc;  /* first step with N_T = N, -1 before               */
  int32_t n_trans;     /* N_T                                              */
  int32_t state;       /* LBMD_RUNNING, ...                                */
} lbmd_status_word;

/* Bytes of the block of lbmd_read_beads_async for n_beads beads. */
#define LBMD_BEAD_BLOCK_BYTES(n_beads) (32 + 48 * (size_t)(n_beads))

/*
 * Asynchronous host read-out for pipelined loops: enqueues on the context's
 * stream one kernel that fills `dst` (caller-owned page-locked host memory:
 * cudaHostAlloc / cudaHostRegister) -- writing it directly when the device
 * can address it (cudaHostAlloc memory on a unified-addressing system,
 * mapped registrations), else through the context's staging buffer and one
 * copy -- with
 *   offset 0:            lbmd_status_word,
 *   offset 32:           unwrapped positions, 3*n_beads doubles [i][xyz],
 *   offset 32 + 24 n:    velocities, 3*n_beads doubles,
 * LBMD_BEAD_BLOCK_BYTES(n_beads) bytes in all.  Nothing is synchronised: the
 * block is valid once the stream has passed this point (synchronise it, or an
 * event recorded on it after this call).  A following lbmd_step may be
 * enqueued at once; its kernels run after the read-out.  With pageable memory
 * the call may block until the copy is done.  The staging buffer is used
 * only for a dst the device cannot address; read-outs enqueued later on the
 * stream do not disturb it.
 * Errors: LBMD_EINVAL (dst NULL or bytes too small), LBMD_ECUDA.
 */
int lbmd_read_beads_async(lbmd_ctx *ctx, void *dst, size_t bytes);

/*
 * One coupled step (Sec. II: interpolate, M MD substeps, spread, stream and
 * collide; Sec. III bookkeeping) and the read-out of its bead block, as
 * lbmd_step(ctx, 1) followed by lbmd_read_beads_async(ctx, dst, bytes) -- same
 * block layout, same asynchrony, same requirements on dst -- but as one graph
 * launch when the device can address dst: the read-out kernel is a node of
 * the step's graph, and its destination is set before each launch.  For other
 * memory, and while kernel timing is on, it makes the two calls.
 * Errors: LBMD_EINVAL (dst NULL or bytes too small), LBMD_ECUDA.
 */
int lbmd_step_read_async(lbmd_ctx *ctx, void *dst, size_t bytes);

/*
 * Of the last step: the fluid velocity interpolated at each bead, u_i, and the
 * impulse J_i = sum over substeps of Delta t_MD (F_drag + F_r) that was handed
 * to the fluid (with the opposite sign).  3*n_beads doubles each.
 */
int lbmd_read_bead_aux(lbmd_ctx *ctx, double *u_i, double *impulse, int dst_is_device);

/*
 * Step counter, number of translocated beads N_T (x < wall_x, Sec. III), the
 * chain state word (LBMD_RUNNING, ...) and the first step with N_T = N (-1 if
 * none).  Synchronises the stream.  Any pointer may be NULL.
 */
int lbmd_status(lbmd_ctx *ctx, int64_t *step, int32_t *n_trans, int32_t *state,
                int64_t *t_transloc);

/*
 * Constraint-solver counters: Newton iterations (summed over the M substeps)
 * of the last LB step, and the number of LB steps in which a SHAKE solve hit
 * the iteration cap with a residual above 1e-3 (Sec. II, SHAKE/RATTLE).
 * Synchronises the stream.  Either pointer may be NULL.
 */
int lbmd_solver_stats(lbmd_ctx *ctx, int32_t *newton_iters_last_step, int32_t *failed_steps);

/*
 * Kernel timing for benchmarks: while enabled, each lbmd_step call captures
 * its n_steps steps into one CUDA graph in which event-record nodes bracket
 * every stream-collide (and the MD cycle and the spread apply), and launches
 * it; the times are those of the graph's execution on the device.
 * lbmd_lb_kernel_time synchronises and returns the summed duration (ms) and
 * count of those stream-collide launches since timing was enabled.
 * n_steps <= 2^20 per call while timing.
 */
int lbmd_set_kernel_timing(lbmd_ctx *ctx, int enable);
int lbmd_lb_kernel_time(lbmd_ctx *ctx, double *total_ms, int64_t *launches);

/*
 * Same timing, per kernel of the step: summed ms of the stream-collide (stage
 * 4), the MD cycle with the gather (stages 1-2) and the spread (stage 3), and
 * the number of timed steps.  Synchronises.  Any pointer may be NULL.
 */
int lbmd_kernel_times(lbmd_ctx *ctx, double *lb_ms, double *md_ms, double *spread_ms,
                      int64_t *steps);

/*
 * One D3Q19 stream-collide step (pure solvent, no beads) on caller-owned
 * populations, for callers that cannot allocate device memory: code whose
 * device memory is fully owned by another framework's pool, code running while
 * another thread captures a CUDA graph in global mode (cudaMalloc is then
 * prohibited), or a real-time loop that must not call the allocator.  It needs
 * no context and no workspace and allocates nothing.  The paper has no
 * counterpart: this is a convenience of this library.
 *   params:  box, wall/pore geometry, y_walls, tau, rho0, body_force, forcing;
 *            storage must be LBMD_STORE_F32, n_beads 0 and kT_fluid 0
 *            (LBMD_EUNSUPPORTED otherwise; other fields ignored)
 *   f_in:    device, 19*V floats [19][z][y][x], the pre-collision populations
 *            f_p(x, t) (absolute values, not deviations); solid nodes ignored
 *   f_out:   device, 19*V floats, receives f_p(x, t+1); solid nodes set to 0;
 *            must not overlap f_in
 *   cuda_stream: stream of the work (cudaStream_t; NULL = legacy default)
 * The geometry scratch (solid bitfield + tile flags) lives in one fixed device
 * array inside the library, 5 MiB per GPU that loads the library, held until
 * the process exits; it limits the box to ny * nz * ceil(nx / 32) <= 2^20
 * (e.g. 256^3).  Each call rebuilds it on the stream, so nothing carries over
 * from the previous call, but every call shares it: calls that may overlap on
 * the GPU (unordered streams) race and must be serialised by the caller.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture.  A device reset (cudaDeviceReset)
 * may move the array: after one, this entry point must not be called again
 * in the same process.
 * Asynchronous; errors: LBMD_EINVAL (bad parameter, f_in == f_out,
 * ny > 524280), LBMD_EUNSUPPORTED (see params), LBMD_ESIZE (box beyond the
 * scratch limit), LBMD_ECUDA (a launch failed; the status is that of this
 * call's own launches).
 */
int lbmd_lb_step_noalloc(const lbmd_params *params, const float *f_in, float *f_out,
                         void *cuda_stream);

/*
 * The diagnostic records written so far (params.diag_every, at most
 * params.diag_capacity of them), oldest first: copies min(count, max_records)
 * to `records` (host) and sets *n_records (may be NULL) to the count.
 * Values are computed in FP32 on the device.  Synchronises.
 */
int lbmd_read_diagnostics(lbmd_ctx *ctx, lbmd_diag *records, int32_t max_records,
                          int32_t *n_records);

/* Release the context's host resources (not the caller's workspace). */
int lbmd_destroy(lbmd_ctx *ctx);

/* ---- ensembles of independent realisations ------------------------------
 * The translocation statistics of Sec. III (duration histograms, the
 * time-versus-length exponent) come from ensembles of 100-1000 realisations
 * per chain length, each started from a different initial chain.  An
 * ensemble context advances many independent realisations -- each with its
 * own box, wall/pore geometry, chain, parameters and seed, all with the same
 * storage type and forcing -- through one set of launches per LB step: the
 * gather and the spread over every bead of every realisation, one MD block
 * per chain (chains grouped by block size, the groups run concurrently) and
 * one stream-collide kernel over a shared list of tiles (32 x rows
 * consecutive nodes of one z-plane) of every live realisation.  Steps are replayed from
 * CUDA graphs of 1, 2 and 16 steps.
 *
 * A realisation is live while its state word is LBMD_RUNNING and it has taken
 * fewer steps than the current cap (lbmd_ensemble_run; no cap before the first
 * run).  The decision is taken on the device at the end of every step, so a
 * realisation stops exactly at its translocation (or retraction, NaN, SHAKE
 * failure) step or at the cap; its state then stays as it was.  Every step of
 * a live realisation is the step lbmd_step would take for the same params.
 *
 * Same conventions as the single-box context: one caller workspace (256-byte
 * aligned), the caller's stream, no device allocation, sticky CUDA errors.
 */
typedef struct lbmd_ensemble lbmd_ensemble;

/*
 * Workspace bytes for `count` realisations members[0 .. count-1].  Each member
 * is validated as by lbmd_workspace_size and must further have
 * n_beads >= 1, 19 * nx*ny*nz < 2^31, nx*ny < 2^22, kT_fluid = 0 and
 * streaming = LBMD_STREAM_PULL; all members must share storage, forcing and solvent_free (LBMD_EUNSUPPORTED
 * otherwise).  count must be >= 1.
 */
int lbmd_ensemble_workspace_size(const lbmd_params *members, int32_t count, size_t *bytes);

/*
 * Create the ensemble: uploads every member's geometry, initial populations
 * (f_eq(rho0, 0), or init_rho / init_u) and chain as lbmd_create does.  The
 * host arrays in members are read during the call only.  Synchronises the
 * stream.  Errors as lbmd_create.
 */
int lbmd_ensemble_create(const lbmd_params *members, int32_t count, void *dev_workspace,
                         size_t bytes, void *cuda_stream, lbmd_ensemble **out);

/* Advance every live realisation by n_steps LB steps (asynchronous). */
int lbmd_ensemble_step(lbmd_ensemble *ens, int64_t n_steps);

/*
 * Run until no realisation is live, with the step cap set to max_steps (total
 * steps per realisation, counted from creation).  Realisations stopped only by
 * an earlier, lower cap resume.  Every check_every steps (rounded up to a
 * multiple of 16; <= 0 means 1024) the host counts the live realisations, stops
 * when there are none and drops finished realisations from the tile list.
 * Synchronises.  *steps_run (may be NULL) receives the LB steps enqueued by
 * this call, i.e. those of its longest-running realisation rounded up to the
 * check interval.
 */
int lbmd_ensemble_run(lbmd_ensemble *ens, int64_t max_steps, int64_t check_every,
                      int64_t *steps_run);

/*
 * Per realisation (arrays of `count` entries; any pointer may be NULL): state
 * word, first step with N_T = N (-1 if none), steps taken and N_T of the last
 * step.  Synchronises.
 */
int lbmd_ensemble_results(lbmd_ensemble *ens, int32_t *state, int64_t *t_transloc,
                          int64_t *steps, int32_t *n_trans);

/* Number of realisations that take part in the next step.  Synchronises. */
int lbmd_ensemble_live(lbmd_ensemble *ens, int32_t *n_live);

/*
 * Read-outs of realisation `member` (0-based), with the layout and
 * dst_is_device meaning of lbmd_read_beads / lbmd_read_populations.  The
 * populations are those after the realisation's last step.  Synchronise.
 */
int lbmd_ensemble_read_beads(lbmd_ensemble *ens, int32_t member, double *pos, double *vel,
                             int dst_is_device);
int lbmd_ensemble_read_populations(lbmd_ensemble *ens, int32_t member, float *f,
                                   int dst_is_device);
int lbmd_ensemble_read_diagnostics(lbmd_ensemble *ens, int32_t member, lbmd_diag *records,
                                   int32_t max_records, int32_t *n_records);

/*
 * Launch shape of the ensemble stream-collide: tile height rows (4, 8 or 16
 * rows of 32 consecutive nodes), register budget for warps resident warps per
 * SM (32: 64 registers, or 48: 40 registers), tiles per block `claim`
 * (1 .. 64; one block per claim tiles of the live realisations) and cells
 * per thread: 1; 2, the nodes at the same
 * (x, y) on two consecutive z-planes; or LBMD_ENS_XPAIR, two x-adjacent
 * nodes whose 16-bit deviations share one 32-bit word (16-bit storage only;
 * tiles of 64 x rows nodes).  The two-cell shapes need warps = 32 and rows 4
 * or 8.  Default (8, 48, 2, 1).  The CUDA graphs are re-captured at the next
 * step.
 */
#define LBMD_ENS_XPAIR 3
int lbmd_ensemble_set_tuning(lbmd_ensemble *ens, int32_t rows, int32_t warps, int32_t claim,
                             int32_t cells_per_thread);
int lbmd_ensemble_get_tuning(lbmd_ensemble *ens, int32_t *rows, int32_t *warps, int32_t *claim,
                             int32_t *cells_per_thread);

/*
 * Autotuner: times the stream-collide alone, `trials` launches per shape, for
 * every shape above (cells per thread 1, 2 or LBMD_ENS_XPAIR, rows, warps, claim in
 * {1, 2, 4, 8}) on the live realisations' current populations, and keeps the
 * fastest.  The trial launches write exactly what the next step's
 * stream-collide writes (from the same input), so the simulation is
 * unchanged.  *best_ms (may be NULL) receives the fastest average launch time
 * (0 for a solvent-free ensemble, which has no stream-collide).  Synchronises.
 */
int lbmd_ensemble_autotune(lbmd_ensemble *ens, int32_t trials, double *best_ms);

/*
 * Kernel timing for benchmarks: while enabled, lbmd_ensemble_step launches
 * kernels directly (no graph) with CUDA events around each step and around
 * its stream-collide.  lbmd_ensemble_kernel_times synchronises and returns the
 * summed ms of the stream-collide launches, of the whole steps, and the number
 * of timed steps since timing was enabled.  Any pointer may be NULL.
 */
int lbmd_ensemble_set_kernel_timing(lbmd_ensemble *ens, int enable);
int lbmd_ensemble_kernel_times(lbmd_ensemble *ens, double *lb_ms, double *step_ms,
                               int64_t *steps);

/* Release the ensemble's host resources (not the caller's workspace). */
int lbmd_ensemble_destroy(lbmd_ensemble *ens);

/* Static description of a status code. */
const char *lbmd_strerror(int status);

/* Thread-local text of the last LBMD_EINVAL / LBMD_ECUDA cause. */
const char *lbmd_last_message(void);

/* ABI version: (major << 16) | minor. */
int lbmd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBMD_H */
