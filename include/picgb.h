/*
 * picgb.h -- C ABI of the GB300-native 2D electrostatic PIC step loop.
 *
 * The library advances the paper's two-dimensional electrostatic
 * particle-in-cell model (Lin & Nishimura, arXiv:1610.03918): kinetic
 * electrons and one ion species in Debye-length / inverse-plasma-frequency
 * units (Sec. II), between a grounded plate at x = 0 and an electrode at
 * x = nx, optionally periodic in y (Sec. III-B), with a trench cut into the
 * electrode (Sec. III-C).  One step is
 *
 *   gather E^n -> leapfrog kick + drift (Eqs. 1-4) -> absorption at walls
 *   and conductors with per-wall tallies and bottom surface charge
 *   (Sec. III-A, III-C, III-D) -> cloud-in-cell deposit of rho^{n+1} ->
 *   Poisson solve of Eq. 5 on the conductor-masked grid -> E^{n+1} = -grad Phi
 *   (central differences inside, two-point at boundaries, Sec. II).
 *
 * Conventions: x is normal to the plates, y runs along them.  A bounded
 * direction with N cells has N + 1 nodes, a periodic one N nodes.  Node and
 * cell arrays are row-major [i_x][j_y], y fastest.  Positions are absolute
 * (a particle at x lies in cell floor(x)).
 *
 * Ownership: every pointer argument is owned by the caller.  Host arrays
 * are copied in or out before the call returns.  Device memory is owned by
 * the library (allocated in pic_init through cfg->alloc, or cudaMalloc when
 * alloc is NULL) and released by pic_free.
 *
 * Errors: every entry point returns a pic_status.  Kernels record
 * conditions they detect (non-convergence, full hit buffer, particle moved
 * farther than the walk limit, out-of-range input) as sticky bits of a
 * device status word; the next synchronising call (pic_diag, or pic_step
 * when it polls the Poisson solver) returns the matching status, and
 * PIC_DIAG_STATUS reads and clears the word.  No entry point is thread-safe
 * for one context; distinct contexts are independent.
 */
#ifndef PICGB_H
#define PICGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
  PIC_OK = 0,
  PIC_EINVAL = 1,     /* bad argument or configuration */
  PIC_ENOMEM = 2,     /* allocation failed */
  PIC_ECUDA = 3,      /* a CUDA call failed */
  PIC_ENOCONV = 4,    /* Poisson solve hit its iteration cap above rtol */
  PIC_EOVERFLOW = 5,  /* capacity of a particle store exceeded */
  PIC_ECFL = 6,       /* a particle moved farther than the face-walk limit */
  PIC_ETIMEOUT = 7,   /* reserved: a bounded device wait gave up */
  PIC_EFULL = 8,      /* hit-record buffer full (tallies stay exact) */
  PIC_ESTATE = 9,     /* call not valid in the current state */
  PIC_ERANGE = 10,    /* pic_load got a particle outside the plasma region */
  PIC_ESIZE = 11      /* grid larger than the fixed scratch of pic_deposit_static */
} pic_status;

/* Status-word bits (PIC_DIAG_STATUS). */
#define PIC_ST_NOCONV   (1u << 0)
#define PIC_ST_FULL     (1u << 1)
#define PIC_ST_CFL      (1u << 2)
#define PIC_ST_RANGE    (1u << 3)
#define PIC_ST_CAPACITY (1u << 4)

/* Wall identifiers of the absorption tallies.  A particle's move is the
 * straight segment x^n -> x^{n+1}; the first crossed face whose far cell is
 * a conductor or outside a bounded direction absorbs it (x face first on an
 * exact tie; ending exactly on a face counts as being in the higher cell). */
#define PIC_WALL_XMIN     0 /* x = 0 plate */
#define PIC_WALL_XMAX     1 /* x = nx plate; the trench bottom inside the trench */
#define PIC_WALL_YMIN     2 /* y = 0 wall (bounded y only) */
#define PIC_WALL_YMAX     3 /* y = ny wall (bounded y only) */
#define PIC_WALL_COND_PX  4 /* conductor entered moving +x (electrode top) */
#define PIC_WALL_COND_MX  5 /* conductor entered moving -x */
#define PIC_WALL_COND_PY  6 /* conductor entered moving +y (trench wall at its upper y) */
#define PIC_WALL_COND_MY  7 /* conductor entered moving -y (trench wall at its lower y) */
#define PIC_NWALLS        8

typedef struct {
  int32_t nx, ny;                 /* cells along x (normal to the plates) and y */
  int32_t periodic_x, periodic_y; /* 1 = periodic (Sec. III-B), 0 = bounded */
  double dt;                      /* time step in 1/omega_e (Sec. III-A: 0.1) */
  double phi_top;                 /* Dirichlet value of the x = 0 plate, T_e/e */
  double phi_electrode;           /* x = nx plate and electrode slab value */
  int32_t trench_depth;           /* electrode slab thickness: cells i >= nx - depth */
  int32_t trench_y0;              /* first open column of the trench */
  int32_t trench_width;           /* open columns (0: flat slab) */
  int32_t surface_charge;         /* 1: charge collected on the x = nx face feeds rho */
  double alpha[2];                /* Eqs. 1-2: alpha_e = -1, alpha_i = (m_e/m_i)(q_i/e) */
  double charge[2];               /* species charge in units of e: {-1, +1} */
  int32_t ppc[2];                 /* particles per cell at density n_0: weight = 1/ppc */
  int64_t capacity[2];            /* maximum particles per species */
  int32_t sort_every;             /* steps between tile sorts (>= 1); 0: chosen by the library --
                                     it sorts, times the particle kernel on each of the next 48
                                     steps (waiting for each of them), and keeps the interval
                                     S in [4, 48] that minimises (sort time + particle time of
                                     the S steps after a sort) / S.  Results do not depend on
                                     it (the deposit is exact and the reductions run in a fixed
                                     order).  pic_batch_init requires >= 1. */
  int32_t poisson_maxit;          /* cap on inner PCG iterations per solve */
  double poisson_rtol;            /* target ||b - A phi||_2 / ||b||_2 (A phi in double-float) */
  int32_t warm_start;             /* 0: zero initial guess each solve, 1: previous phi,
                                     2: extrapolated 2 phi^n - phi^{n-1}, 3: learned -- the
                                     warm-start network's guess phi_L + s U(rho / s, mask)
                                     (see unet_weights and pic_set_learned_start), 4: the
                                     lift start -- phi_L, the potential of the empty box
                                     (solved once), on the free nodes */
  int32_t device;                 /* CUDA device ordinal */
  int32_t timing;                 /* 1: each step records its phase boundaries in CUDA
                                     events (a pool of 64 steps, read back when it fills or
                                     at pic_diag) for the per-phase device times of
                                     PIC_DIAG_TIMING */
  int32_t graphs;                 /* 1: each step is one launch of a captured CUDA graph whose
                                     Poisson loops are device-side conditional nodes;
                                     0: kernels launched from a host loop that polls the solver */
  int32_t poisson_method;         /* inner solver of the iterative refinement of Eq. 5:
                                     0: automatic -- a direct FFT / tridiagonal / capacitance
                                     solve when the box is periodic in y with a power-of-two
                                     ny <= 2048, bounded in x, and its free nodes form a full
                                     slab with at most one slot below it (the trench and the
                                     plate geometries), else 1;
                                     1: conjugate gradient preconditioned by a multigrid V-cycle */
  int64_t hit_capacity;           /* hit records kept (PIC_DIAG_HITS) */
  void *stream;                   /* cudaStream_t to run on; NULL: a library-owned stream */
  /* optional device allocator: called with the context's stream (the memory
     is used in stream order on it); NULL: cudaMalloc / cudaFree.  Blocks
     must be aligned to 16 bytes at least; a misaligned block is released
     again and the call fails with PIC_ENOMEM. */
  void *(*alloc)(size_t bytes, void *stream, void *user);
  void (*free)(void *ptr, void *stream, void *user);      /* its release function */
  void *alloc_user;
  /* RF bias of the electrode (Sec. III-B: Phi = Phi_0 sin(omega_RF t) on the
     biased plate): every node held at the electrode potential takes
     phi_electrode + phi_rf_amp sin(omega_rf t) in the solve of time level
     n, t = n dt.  phi_rf_amp = 0: a fixed bias. */
  double phi_rf_amp;
  double omega_rf;
  /* ion recycling (Sec. III-A: a lost ion is replaced by a thermal ion in the
     bulk, as ionisation of the neutral gas; Sec. III-C: ionisation only in
     the bulk region).  With recycle = 1, every ion absorbed during step n
     (tallied and recorded as usual) re-enters in the same step, with its id,
     at a uniform position in the cell rows [source_x0, source_x1) (all y;
     source_x1 = 0: nx - trench_depth, the rows above the electrode) and with
     a Maxwellian velocity of standard deviation recycle_vth per component,
     taken as its v^{n+1/2}.  The draws are Philox4x32-10 keyed by seed with
     counter (id, n, 1, k): k = 0 gives the row source_x0 + floor(r0 L / 2^32),
     the column floor(r1 ny / 2^32) and the offsets (r2 >> 8) 2^-24,
     (r3 >> 8) 2^-24; k = 1 the Box-Muller pair of u1 = ((q0 >> 8) + 1) 2^-24,
     u2 = (q1 >> 8) 2^-24.  Electrons are not recycled. */
  int32_t recycle;
  int32_t source_x0, source_x1;
  double recycle_vth;
  uint64_t seed;                  /* key of the counter-based draws */
  /* warm_start = 3: file of the warm-start network's parameters (the flat
     FP32 vector of pic_unet_save); the network then gives the initial guess
     of every solve inside the step.  NULL otherwise. */
  const char *unet_weights;
  /* 1: this context is one rank of a run split by particles (each rank holds
     a share of the particles and the whole grid); it is advanced by
     pic_step_particles, an all-reduce of its exchange buffer, and
     pic_step_fields, not by pic_step.  Requires sort_every >= 1. */
  int32_t decomposed;
  /* tile variant of the particle store (shape of the sort's tiles and of the
     particle kernel's shared-memory windows, CTA size): 0: 16 x 16 cells,
     128 threads; 1: 32 (x) x 16 (y), 128; 2: 16 x 32, 128; 3: 32 x 32, 256;
     halo 4 cells.  pic_autotune chooses one by timing.  Results do not
     depend on it. */
  int32_t tile_variant;
} pic_config;

/* One absorbed particle (PIC_DIAG_HITS): velocity is v^{n+1/2}. */
typedef struct {
  uint32_t id;
  int16_t species;
  int16_t wall;     /* PIC_WALL_* */
  int32_t cell;     /* cell index along the wall: y index for x faces, x index for y faces */
  int32_t step;     /* step during which the particle was absorbed (0-based) */
  float vx, vy;
} pic_hit;

/* Load flags */
#define PIC_LOAD_V_AT_T0 1u /* velocities are v^0: back-kick by dt/2 before the first step */

/* Diagnostic kinds for pic_diag.  Unless stated, out receives doubles. */
enum {
  PIC_DIAG_ENERGY = 0,   /* [KE_e, KE_i, FE, n]: of the last step, time level n (see below) */
  PIC_DIAG_MOMENTUM = 1, /* [Px_e, Py_e, Px_i, Py_i] = m_s w_s sum v^{n+1/2} */
  PIC_DIAG_COUNTS = 2,   /* int64[2*8 + 2]: wall tallies [species][wall], then live counts */
  PIC_DIAG_SURFACE = 3,  /* int64[2*ny]: hits on the x = nx face per species per y cell */
  PIC_DIAG_HITS = 4,     /* pic_hit[n_out] (the first hit_capacity records) */
  PIC_DIAG_RHO = 5,      /* [nxn*nyn]: net charge density of the last deposit */
  PIC_DIAG_PHI = 6,      /* [nxn*nyn]: potential (held as a double-float pair, ~48 bits) */
  PIC_DIAG_E = 7,        /* [2*nxn*nyn]: Ex then Ey at the nodes */
  PIC_DIAG_STATE_E = 8,  /* [5*n]: x, y, vx, vy, id blocks of live electrons (into pinned
                            host memory the export kernel writes directly) */
  PIC_DIAG_STATE_I = 9,  /* same for ions */
  PIC_DIAG_POISSON = 10, /* [inner iterations, outer iterations, rel residual, ms] of the last solve,
                            and (with room for a fifth double) the rel residual at its first check:
                            that of the initial guess with the multigrid inner solver, that after
                            the first correction with the direct one (whose first pass always
                            corrects) */
  PIC_DIAG_STATUS = 11,  /* uint32: status word; reading clears it */
  PIC_DIAG_TIMING = 12,  /* [steps, ms particle kernel, ms sort, ms Poisson (the solve's
                            residual passes also form E), ms rho,
                            sorts, kernel launches, particle slots processed]: device time
                            from CUDA events on the context stream, accumulated over
                            pic_step calls since the last read; reading resets it */
  PIC_DIAG_PHI_VACUUM = 13, /* [nxn*nyn]: potential of the empty box (Dirichlet values only),
                               solved once to 1e-10 */
  PIC_DIAG_SOLVER = 14,     /* int32: inner Poisson solver in use, 0 direct, 1 multigrid PCG
                               (pic_config.poisson_method) */
  PIC_DIAG_SORT = 15,       /* int32[2]: steps between tile sorts in use (0 while it is being
                               tuned), and 1 if it was chosen by the tuning of sort_every = 0 */
  PIC_DIAG_TILE = 16        /* int32[5]: tile variant in use, its tile cells along x and y,
                               halo cells, particle-kernel threads per CTA */
};

/* Create a context from cfg.  Builds the conductor mask, Dirichlet nodes and
 * multigrid hierarchy of the geometry (Sec. III), allocates device memory.
 * Returns PIC_EINVAL for an inconsistent configuration. */
pic_status pic_init(const pic_config *cfg, pic_ctx **out);

/* Replace the particles of species s (0 electrons, 1 ions) by n particles at
 * absolute positions (x, y) with velocities (vx, vy); ids may be NULL
 * (0..n-1).  All arrays are host memory of length n.  Initial state per
 * Sec. III-A (uniform positions, Eq. 6 velocities) is the caller's choice.
 * With flags & PIC_LOAD_V_AT_T0 the velocities are taken at t = 0 and the
 * species is back-kicked by dt/2 in the field of the full loaded state
 * before the next step (leapfrog start).
 * species == -1 loads a fixed external charge density rho_ext (Sec. III-D)
 * from x[nxn*nyn]; species == -2 sets the potential (the initial guess of the
 * next solve; Dirichlet nodes keep their values) from x[nxn*nyn]; the other
 * pointers are then ignored.
 * Particles outside the domain or in a conductor are dropped and counted
 * in the PIC_ST_RANGE bit; n > capacity returns PIC_EOVERFLOW. */
pic_status pic_load(pic_ctx *ctx, int32_t species, int64_t n, const double *x,
                    const double *y, const double *vx, const double *vy,
                    const uint32_t *ids, uint32_t flags);

/* Advance nsteps leapfrog steps (Sec. II).  nsteps == 0 only brings the
 * fields up to date with the loaded state (deposit, Poisson solve, E) and
 * applies pending dt/2 back-kicks (this part polls the solver from the host).
 * With cfg->graphs the steps are queued as graph launches and the call
 * returns without waiting (with cfg->timing it waits once every 64 steps, to
 * read back the phase events; while the sort interval is being tuned, once
 * per step); a solve that fails to reach rtol sets PIC_ST_NOCONV, reported by
 * the next pic_diag.  Without graphs the call waits on each solve and
 * returns PIC_ENOCONV directly. */
pic_status pic_step(pic_ctx *ctx, int32_t nsteps);

/* Autotuner of the particle store's tile variant (pic_config.tile_variant).
 * With cache_path naming a file that holds an entry for this GPU (device
 * name), grid, geometry and particles per cell, that entry's variant is
 * taken.  Otherwise every variant is timed on the live run: the particles
 * are sorted into its tiles, then `steps` steps run with no further sort and
 * the particle kernel's mean device time (CUDA events) is recorded; the
 * fastest variant is kept and, with cache_path, stored in the file (a JSON
 * array, one object per line: key, tile_variant, particle_ms of every
 * variant).  The timed steps advance the run; results do not depend on the
 * variant.  A tuned sort interval (sort_every = 0) is chosen again for the
 * new tiles.  *chosen (may be NULL) receives the variant.  Synchronous;
 * PIC_EINVAL for a decomposed context or a cache file that cannot be
 * written. */
pic_status pic_autotune(pic_ctx *c, int32_t steps, const char *cache_path, int32_t *chosen);

/* Turn the per-phase timing of cfg->timing on (1) or off (0) for the steps
 * that follow; totals already recorded are kept until PIC_DIAG_TIMING reads
 * them.  Graph steps with timing carry event nodes between the phases, which
 * also end the programmatic overlap of one phase's kernels with the next;
 * the first step of each kind captures its graph.  Returns PIC_EINVAL for
 * other values of on. */
pic_status pic_set_timing(pic_ctx *ctx, int32_t on);

/* Copy a diagnostic to host memory out (cap_bytes long); *n_out receives the
 * element count written (may be NULL).  Synchronises the stream.
 * ENERGY: KE_s = 1/2 m_s w_s sum v^{n-1/2}.v^{n+1/2}, FE = 1/2 sum_nodes |E^n|^2,
 * m_s = charge_s / alpha_s, w_s = 1/ppc_s.  Too small a buffer: PIC_EINVAL. */
pic_status pic_diag(pic_ctx *ctx, int32_t kind, void *out, int64_t cap_bytes,
                    int64_t *n_out);

/* Checkpoint and restart (no counterpart in the paper; a service for long
 * runs).  pic_save writes the complete state of the run into the host buffer
 * buf of cap_bytes: the live particles in their stored form (cell index,
 * FP32 in-cell offsets and half-step velocities, id), the potential (and the
 * previous step's, for the warm start), the field, rho, rho_ext and the
 * Dirichlet data as stored (double-float pairs), the wall tallies, the
 * trench-bottom counts, the hit records kept and the total hit count, the
 * step counter, the status word and the solver's last scalars.  *n_out
 * receives the size; buf == NULL only reports it.  The particles are
 * compacted through a temporary device buffer of 24 bytes per particle
 * slot drawn from the context's allocator.  PIC_ESTATE after a pic_load that
 * no step has brought up to date.  Synchronous.
 *
 * pic_restore loads such a checkpoint into a context created with the same
 * configuration (grid, geometry, capacities at least the live counts, hit
 * capacity at least the records kept; PIC_EINVAL / PIC_EOVERFLOW
 * otherwise).  The next pic_step (or pic_batch_step of a batch member)
 * sorts the particles and continues the run bit for bit as if it had not
 * been interrupted: N steps, save, restore into a new context, N steps give
 * the particles, fields, tallies and hit records of 2N uninterrupted steps.
 * PIC_DIAG_ENERGY reports the kinetic energy again from the next step on. */
pic_status pic_save(pic_ctx *ctx, void *buf, int64_t cap_bytes, int64_t *n_out);
pic_status pic_restore(pic_ctx *ctx, const void *buf, int64_t n_bytes);

/* ---- One run split by particles across ranks (GPUs) ---------------------
 * The paper's model has one grid and many particles; a run too large for one
 * GPU is split by particles.  Every rank (a context with decomposed = 1, the
 * same configuration on every rank, its own share of the particles through
 * pic_load) keeps the whole grid.  One step is
 *   pic_step_particles   [tile sort] gather, push, absorption with this
 *                        rank's tallies and hit records, and the fixed-point
 *                        deposit of this rank's particles (Eqs. 1-5);
 *   all-reduce           the caller sums the rank's exchange buffer in place
 *                        over all ranks (int64 addition; e.g. NCCL ncclInt64
 *                        ncclSum on the context's stream): the deposit sums
 *                        [2][nodes] and the bottom counts [2][ny];
 *   pic_step_fields      rho from the summed deposit and surface charge, the
 *                        Poisson solve and the field (identical on every
 *                        rank: same inputs, deterministic kernels).
 * Integer sums are exact and order-free, so an R-rank run gives, bit for bit,
 * the rho, phi, E and particles (as a union) of the same particles in one
 * context.  After pic_load the first pic_step_particles / pic_step_fields
 * pair brings the fields up to date (as pic_step(ctx, 0) does).  Per-rank
 * diagnostics (COUNTS, SURFACE, HITS, STATE, the kinetic energies of ENERGY)
 * cover the rank's own particles; fields (RHO, PHI, E, FE) are global.
 * pic_step_particles and pic_step_fields queue work on the context's stream
 * and return; calling them out of order returns PIC_ESTATE. */
pic_status pic_step_particles(pic_ctx *ctx);
pic_status pic_step_fields(pic_ctx *ctx);
/* The rank's exchange buffer: *buf (device, int64, *count elements). */
pic_status pic_exchange_buffer(pic_ctx *ctx, int64_t **buf, int64_t *count);
/* The all-reduce of n ranks' exchange buffers when all are contexts of this
 * process on one device (a single-GPU stand-in for the collective): waits for
 * each context's stream, writes the element-wise sum into every buffer,
 * synchronously.  n <= 64. */
pic_status pic_exchange_sum(pic_ctx *const *ctxs, int32_t n);

/* Release the context and all its device memory. */
pic_status pic_free(pic_ctx *ctx);

/* Static description of a status code. */
const char *pic_strerror(pic_status st);

/* Text of the last failure recorded on the calling thread (the failing CUDA
 * call and its error string), or "" if none. */
const char *pic_last_error(void);

/* Ensemble of independent runs on one GPU (the trench-width sweep of
 * Sec. III-C run as a batch).  Each member is a full context built from
 * cfgs[k] (its own grid size, trench, particles and tallies); all members
 * share one CUDA stream (`stream`, or a library-owned one when NULL) and one
 * tile-sort schedule (equal sort_every, else PIC_EINVAL).  One ensemble step
 * is one launch of a captured CUDA graph in which every member's step (sort
 * when due, particle kernel, rho, Poisson solve with its own device-side
 * convergence loop, field) is an independent branch, so the members' phases
 * overlap on the GPU.  Load and read members with pic_load / pic_diag on
 * pic_batch_member(b, k); advance them only through pic_batch_step. */
typedef struct pic_batch pic_batch;

pic_status pic_batch_init(const pic_config *cfgs, int32_t n, void *stream, pic_batch **out);

/* Member k's context (owned by the batch), or NULL for an invalid index. */
pic_ctx *pic_batch_member(pic_batch *b, int32_t k);

/* Advance every member by nsteps.  Members whose fields are out of date
 * (after pic_load) are brought up to date first, as pic_step(ctx, 0) does.
 * Returns once the steps are queued; with cfgs[0].timing it waits for each
 * step and accumulates its device time. */
pic_status pic_batch_step(pic_batch *b, int32_t nsteps);

/* out[0] = ensemble steps and out[1] = their device milliseconds (CUDA
 * events around each ensemble graph launch) since the last call. */
pic_status pic_batch_timing(pic_batch *b, double *out);

/* Release the batch and all its members. */
pic_status pic_batch_free(pic_batch *b);

/* ---- Learned warm start for the Poisson solve of Eq. 5 ------------------
 * The paper solves Eq. 5 by Gauss-Seidel / Jacobi and names a faster field
 * solver as future work (Sec. II, Sec. IV).  A U-Net U maps (rho / s, conductor
 * mask) to (phi - phi_L) / s, s = max |rho|, phi_L the potential of the empty
 * box; phi_L + s U(...) is the initial guess of the solve, which still runs to
 * its tolerance.  Four levels (32/64/128/256 channels), two 3x3 conv + ReLU per
 * level, 2x2 average pool down, 2x2 stride-2 transposed conv up with skip
 * concatenation, 1x1 head; BF16 activations and weights, FP32 accumulation
 * and master weights.  All arrays are DEVICE memory, NHWC, FP32:
 * x [batch][height][width][2], y and targets [batch][height][width].
 * height and width are multiples of 8 (at least 16), and 2 batch height width
 * < 2^31 (PIC_EINVAL otherwise).  Parameters travel as
 * one flat FP32 vector (layer by layer: enc0a..enc3b conv weights [out][3][3][in]
 * and biases, then per decoder level the transposed conv [2][2][in][out] and
 * bias and the two convs, then the head weight [32] and bias). */
typedef struct pic_unet pic_unet;

pic_status pic_unet_create(int32_t batch, int32_t height, int32_t width, void *stream, pic_unet **out);
int64_t pic_unet_num_params(const pic_unet *u);
pic_status pic_unet_set_params(pic_unet *u, const float *host_params); /* resets Adam state */
pic_status pic_unet_get_params(pic_unet *u, float *host_params);
/* y = U(x) (queued on the net's stream) */
pic_status pic_unet_forward(pic_unet *u, const float *x, float *y);
/* MSE loss of U(x) against t and the gradient of every parameter (host copy,
 * may be NULL); synchronous */
pic_status pic_unet_gradients(pic_unet *u, const float *x, const float *t, float *host_grad,
                              double *loss);
/* one Adam step (lr, beta 0.9 / 0.999) on the MSE loss; *loss (host, may be
 * NULL) receives the loss once the stream reaches it */
pic_status pic_unet_train_step(pic_unet *u, const float *x, const float *t, float lr, double *loss);
pic_status pic_unet_free(pic_unet *u);

/* The U-Net's contractions -- the 3x3 and transposed 2x2 convolutions, their
 * data gradients and their weight gradients -- run on the fifth-generation
 * tensor cores (tcgen05.mma, FP32 accumulators in tensor memory, operands
 * staged by TMA) wherever the shapes allow (the network's own shapes always
 * do when each level is at least 8 wide), and on the mma.sync / CUDA-core
 * kernels otherwise; impl 1 selects those for all of them (impl 0: the
 * default).  Synchronous. */
pic_status pic_unet_set_conv_impl(pic_unet *u, int32_t impl);
/* PIC_ETIMEOUT (and clears it) if a bounded wait of a tensor-core kernel of
 * this network gave up since the last call; waits for the net's stream. */
pic_status pic_unet_status(pic_unet *u);

/* One 3x3 convolution with zero padding (the U-Net's layer):
 * out[b][h][w][out_off + n] = act(bias[n] + sum_{dy, dx, c}
 *   in[b][h + dy - 1][w + dx - 1][in_off + c] * w[n][3 dy + dx][c]),
 * dy, dx in {0, 1, 2}, act = ReLU when relu, else identity.  in, out: DEVICE
 * BF16 NHWC with channel strides in_cs, out_cs; w: DEVICE BF16 [cout][9][cin];
 * bias: DEVICE FP32 [cout] or NULL.  impl 0: tcgen05 tensor cores (shapes as
 * above, else PIC_EINVAL); impl 1: mma.sync (cout 32 with cin 16 or a
 * multiple of 32, or cout a multiple of 64 with cin a multiple of 32).
 * FP32 accumulation, BF16 rounding of the result.  Synchronous on `stream`;
 * PIC_ETIMEOUT if a bounded wait of the tensor-core kernel gave up. */
pic_status pic_conv3x3_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *in, int32_t in_cs,
                            int32_t in_off, int32_t cin, const void *w, const float *bias, int32_t relu,
                            void *out, int32_t out_cs, int32_t out_off, int32_t cout, void *stream);

/* The weight gradient of one 3x3 convolution with zero padding (the U-Net's
 * layer): dw[n][3 dy + dx][c] += sum_{b, h, w} dpre[b][h][w][n] *
 *   in[b][h + dy - 1][w + dx - 1][in_off + c], dy, dx in {0, 1, 2}.
 * dpre: DEVICE BF16 [B][H][W][cout] (the gradient before the activation);
 * in: DEVICE BF16 NHWC with channel stride in_cs; dw: DEVICE FP32
 * [cout][9][cin], ADDED to (zero it first), 16-byte aligned for impl 0.
 * impl 0: tcgen05 tensor cores (cout 32 or a multiple of 64, cin 16, 32 or a
 * multiple of 64, in_cs and in_off multiples of 8, else PIC_EINVAL); impl 1:
 * mma.sync (channel counts, in_cs and in_off multiples of 8).  FP32 products
 * of the BF16 values, summed in FP32 with atomic adds (the order of the sum
 * varies from run to run).  Synchronous on `stream`; PIC_ETIMEOUT if a
 * bounded wait of the tensor-core kernel gave up. */
pic_status pic_conv3x3_wgrad_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *dpre,
                                  const void *in, int32_t in_cs, int32_t in_off, int32_t cin, int32_t cout,
                                  float *dw, void *stream);

/* The U-Net's 2x2 average pool: out[b][y][x][c] = BF16(0.25 * sum_{a, d in
 * {0, 1}} in[b][2y + a][2x + d][in_off + c]) (FP32 sum).  in: DEVICE BF16
 * NHWC [B][H][W] with channel stride in_cs; out: DEVICE BF16
 * [B][H/2][W/2][C] (contiguous).  H and W even; C, in_cs and in_off
 * multiples of 8; both pointers 16-byte aligned; else PIC_EINVAL.
 * Synchronous on `stream`. */
pic_status pic_avgpool2_bf16(int32_t B, int32_t H, int32_t W, const void *in, int32_t in_cs, int32_t in_off,
                             int32_t C, void *out, void *stream);
/* The U-Net's 1x1 head on its 32 last channels: y[p] = b[0] + sum_{c < 32}
 * hin[p][c] w[c] (FP32).  hin: DEVICE BF16 [npix][32], 16-byte aligned; w:
 * DEVICE FP32 [32]; b: DEVICE FP32 [1]; y: DEVICE FP32 [npix].  Synchronous
 * on `stream`. */
pic_status pic_head_bf16(int64_t npix, const void *hin, const float *w, const float *b, float *y, void *stream);
/* Its backward: gh[p][c] = BF16(dy[p] w[c]), dw[c] += sum_p dy[p] hin[p][c],
 * db[0] += sum_p dy[p] (FP32, atomic adds in a varying order).  dy: DEVICE
 * FP32 [npix]; gh: DEVICE BF16 [npix][32], 16-byte aligned; dw, db: DEVICE
 * FP32, ADDED to.  Synchronous on `stream`. */
pic_status pic_head_back_bf16(int64_t npix, const float *dy, const void *hin, const float *w, void *gh, float *dw,
                              float *db, void *stream);
/* Backward through a ReLU, with the bias gradient of the convolution before
 * it: dpre[p][c] = y[p][off_y + c] > 0 ? t[p][c] : 0 and db[c] += sum_p
 * dpre[p][c], where t = g[p][g_off + c], or, with gp (the gradient of the
 * 2x2 average pool that follows y, DEVICE BF16 [B][H/2][W/2][C]),
 * t = BF16(g[p][g_off + c] + 0.25 gp[parent of p][c]).  g, y: DEVICE BF16
 * NHWC [B][H][W] with channel strides g_cs, y_cs; dpre: DEVICE BF16
 * [B][H][W][C]; db: DEVICE FP32 [C], ADDED to (atomic adds in a varying
 * order).  C 8, 16, 32, 64, 128 or 256; strides and offsets multiples of 8;
 * pointers 16-byte aligned; H and W even with gp; else PIC_EINVAL.
 * Synchronous on `stream`. */
pic_status pic_relu_back_bf16(int32_t B, int32_t H, int32_t W, const void *g, int32_t g_cs, int32_t g_off,
                              const void *y, int32_t y_cs, int32_t y_off, const void *gp, void *dpre, int32_t C,
                              float *db, void *stream);

/* The U-Net's 2x2 stride-2 transposed convolution (its upsampling layer):
 * out[b][2y + a][2x + c][out_off + co] = bias[co] + sum_{ci}
 *   in[b][y][x][ci] * w[a][c][ci][co],  a, c in {0, 1}.
 * in: DEVICE BF16 [B][H][W][cin] (contiguous); w: DEVICE FP32
 * [2][2][cin][cout] (the layer's parameter order); bias: DEVICE FP32 [cout];
 * out: DEVICE BF16 NHWC [B][2H][2W] with channel stride out_cs.  impl 0:
 * tcgen05 tensor cores on a BF16 copy of w (a temporary device buffer; cin a
 * multiple of 16, cout 16, 32 or a multiple of 64, out_cs and out_off
 * multiples of 8, W >= 8, else PIC_EINVAL); impl 1: CUDA cores with the
 * FP32 weights.  FP32
 * accumulation, BF16 rounding of the result.  Synchronous on `stream`;
 * PIC_ETIMEOUT if a bounded wait of the tensor-core kernel gave up. */
pic_status pic_upconv_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *in, int32_t cin,
                           const float *w, const float *bias, void *out, int32_t out_cs, int32_t out_off,
                           int32_t cout, void *stream);

/* The weight and bias gradients of the U-Net's 2x2 stride-2 transposed
 * convolution: dw[a][c][ci][co] += sum_{b, y, x} in[b][y][x][ci] *
 *   gout[b][2y + a][2x + c][gout_off + co], db[co] += sum over all gout
 * pixels of gout[..][gout_off + co].  in: DEVICE BF16 [B][H][W][cin]
 * (contiguous); gout: DEVICE BF16 NHWC [B][2H][2W] with channel stride
 * gout_cs; dw: DEVICE FP32 [2][2][cin][cout], db: DEVICE FP32 [cout], both
 * ADDED to.  impl 0: tcgen05 tensor cores and a vector column sum (cin a
 * multiple of 64, cout 32, 64, 128 or 256, gout_cs and gout_off multiples
 * of 8, else PIC_EINVAL); impl 1: CUDA cores.  FP32 sums with atomic adds
 * (their order varies from run to run).  Synchronous on `stream`;
 * PIC_ETIMEOUT if a bounded wait of the tensor-core kernel gave up. */
pic_status pic_upconv_wgrad_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *in, int32_t cin,
                                 const void *gout, int32_t gout_cs, int32_t gout_off, int32_t cout, float *dw,
                                 float *db, void *stream);

/* The data gradient of the U-Net's 2x2 stride-2 transposed convolution (the
 * input-side gradient of its upsampling layer):
 * gin[b][y][x][n] = sum_{a, c in {0, 1}} sum_{k < cout}
 *   gout[b][2y + a][2x + c][gout_off + k] * w[2a + c][n][k].
 * gout: DEVICE BF16 NHWC [B][2H][2W] with channel stride gout_cs; w: DEVICE
 * FP32 [2][2][cin][cout] (the layer's parameter order); gin: DEVICE BF16
 * [B][H][W][cin].  impl 0: tcgen05 tensor cores on a BF16 copy of w (a
 * temporary device buffer of 8 cin cout bytes; cin 32, 64, 128 or 256, cout a
 * multiple of 16, gout_cs and gout_off multiples of 8, W >= 8, else
 * PIC_EINVAL); impl 1: CUDA cores with the FP32 weights.  FP32 accumulation,
 * BF16 rounding of the result.  Synchronous on `stream`; PIC_ETIMEOUT if a
 * bounded wait of the tensor-core kernel gave up. */
pic_status pic_upconv_back_bf16(int32_t impl, int32_t B, int32_t H, int32_t W, const void *gout,
                                int32_t gout_cs, int32_t gout_off, int32_t cout, const float *w, void *gin,
                                int32_t cin, void *stream);

/* He initialisation of every weight (He et al., ICCV 2015: N(0, 2 / fan_in)
 * for the layers followed by a ReLU, N(0, 1 / fan_in) for the linear head;
 * fan_in = 9 x input channels for a 3x3 convolution, the input channels for
 * a transposed one), zero biases, Adam state reset.  Weight e of layer k
 * (layers in parameter order) takes the cosine half of the Box-Muller pair of
 * Philox4x32-10 with key = seed and counter (e, k, 2, 0).  Synchronous. */
pic_status pic_unet_init(pic_unet *u, uint64_t seed);
/* The flat FP32 parameter vector to / from a file (raw, native byte order,
 * pic_unet_num_params values).  Synchronous. */
pic_status pic_unet_save(pic_unet *u, const char *path);
pic_status pic_unet_load(pic_unet *u, const char *path);

/* Use a copy of the parameters of net for the learned initial guess of every
 * later solve of the context (its warm_start becomes 3): inside each step the
 * guess phi_L + s U(rho / s, mask) is formed on the device (s = max |rho|, the
 * input and the network's forward pass on the context's stream, captured in
 * the step graph) and the solve runs from it to its tolerance.  net must have
 * batch 1, height >= nxn (nxn rounded up to a multiple of 8) and width nyn.
 * Computes the empty-box potential phi_L if not done yet.  Synchronous. */
pic_status pic_set_learned_start(pic_ctx *c, const pic_unet *net);

/* Change the initial guess of the solves that follow (pic_config.warm_start:
 * 0 zero, 1 previous, 2 extrapolated, 3 learned -- only once
 * pic_set_learned_start has given the context a network -- 4 lift, whose
 * empty-box potential is solved on the first switch); the step graphs are
 * captured again.  Synchronous. */
pic_status pic_set_warm_start(pic_ctx *c, int32_t mode);

/* Training target of the warm-start network for the context's current
 * potential: t [hpad][nyn] (device, FP32) = (phi - phi_L) / scale, rows
 * nxn..hpad-1 zero.  Synchronous. */
pic_status pic_learned_target(pic_ctx *c, int32_t hpad, double scale, float *t);

/* Input of the warm-start network for the context's current charge density:
 * x [hpad][nyn][2] (device, FP32) = (rho / s, 1 on Dirichlet nodes), rows
 * nxn..hpad-1 filled as conductor; *scale = s = max |rho| (host).
 * hpad >= nxn.  Synchronous. */
pic_status pic_learned_input(pic_ctx *c, int32_t hpad, float *x, double *scale);

/* Solve Eq. 5 again for the context's current charge density, to the
 * configured tolerance, from the initial guess `guess`: 0 zero, 1 the current
 * potential (the previous step's), 2 the empty-box potential phi_L, 3 the
 * learned guess phi_L + scale * y (y device FP32, row-major over the nodes
 * with row pitch nyn, e.g. the network's output).  The field is recomputed.
 * stats (host, may be NULL) = [PCG iterations, refinement passes, relative
 * residual, device ms from the guess to the solution].  Synchronous. */
pic_status pic_poisson(pic_ctx *c, int32_t guess, const float *y, double scale, double *stats);

/* Cloud-in-cell deposit that allocates no device memory.  The paper has no
 * counterpart; this is a service for callers that cannot allocate at the
 * point where they deposit -- a program whose device memory is owned by
 * another runtime's pool, or a latency-critical loop that cannot take the
 * device-wide synchronisation an allocation or release may cause.
 *
 * Computes rho[n] = weight * (sum over particles of their bilinear shares at
 * node n), with the same fixed-point arithmetic as the context-based deposit
 * (shares quantised to 2^-20 of a particle, summed exactly), for n particles
 * at absolute positions x[k], y[k] on a grid of nx x ny cells (N + 1 nodes
 * in a bounded direction, N in a periodic one; periodic coordinates wrap).
 * x, y (n doubles each) and rho (nodes, row-major, y fastest) are DEVICE
 * pointers owned by the caller.  Particles outside the grid in a bounded
 * direction, and particles with a NaN coordinate, are dropped without any
 * report: the call still returns PIC_OK, and their charge is missing from rho.
 * Work is queued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * of the current device and the call returns once it is queued.  PIC_ECUDA
 * means one of this call's own launches failed; errors left by earlier,
 * unrelated CUDA calls are neither reported nor cleared.
 *
 * Scratch: one fixed array of 2^20 64-bit accumulators (8 MiB), a static
 * device variable of the library that every GPU loading the library holds
 * until the process exits.  Grids with more than 2^20 nodes return
 * PIC_ESIZE.  Each call looks up the array's device address in the context
 * current on the calling thread (so a caller may switch contexts, or reset
 * the device, between calls); make the first call on a device before any
 * stream capture, since that first lookup loads the library's module there.
 * Every call clears and reuses the same array, so calls whose work overlaps
 * on one GPU (different streams, or different host threads) race and must
 * be serialised by the caller. */
pic_status pic_deposit_static(int32_t nx, int32_t ny, int32_t periodic_x, int32_t periodic_y,
                              int64_t n, const double *x, const double *y, double weight,
                              double *rho, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PICGB_H */
