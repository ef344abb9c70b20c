/*
 * lbib.h -- C ABI of the GB300 lattice-Boltzmann / dynamic immersed-boundary
 * library (liblbib.so).
 *
 * Method: Coclite, Ranaldo, Pascazio, de Tullio, "A Lattice Boltzmann
 * dynamic-Immersed Boundary scheme for the transport of deformable inertial
 * capsules in low-Re flows" (arXiv 2207.06029).  A D3Q19 BGK lattice with the
 * Guo forcing term (Sec. 2.1, Eqs. e_i, evoleq, eqfunc, forcing) and Zou-He
 * velocity walls is coupled to immersed bodies through moving-least-squares
 * interpolation and spreading (Sec. 2.2, Eqs. uLag, l2norm, intKernel,
 * bodyforce).  Membranes feel spring, bending and volume forces plus the
 * probe-based hydrodynamic stresses and move by the Verlet update; rigid
 * bodies follow the Newton-Euler update (Sec. 2.3, Eqs. strainPot..
 * angularVelRig).
 *
 * Units: lattice units, dx = dt = 1, reference density 1.  Node (x, y, z)
 * sits at position (x, y, z); the linear cell index is
 * idx = x + nx * (y + ny * z).
 *
 * Ownership: the library owns all device state of a context.  Every array
 * argument is owned by the caller and is only read or written during the
 * call (inputs are copied).  Pointers flagged "on_device" are CUDA device
 * pointers (e.g. torch tensor data); otherwise they are host pointers.
 *
 * Errors: every call returns LBIB_OK (0) or a negative code and never aborts
 * or traps the device.  lbib_last_error() gives a message.  Errors raised on
 * the device (a body support reaching a wall) surface at the next call that
 * synchronises (lbib_sync, lbib_get_*); after any error the context is
 * sticky: further lbib_step calls return the same code.
 *
 * Calls on one context are not thread-safe; different contexts are
 * independent.  All device work of a context runs on its stream.
 */
#ifndef LBIB_H
#define LBIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LBIB_OK = 0,
    LBIB_EINVAL = -1,      /* invalid argument or parameter */
    LBIB_ENOMEM = -2,      /* device or host allocation failed */
    LBIB_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed */
    LBIB_EDIVERGED = -4,   /* the run diverged (see lbib_set_watchdog) */
    LBIB_EBODY_WALL = -5,  /* an MLS support (marker or probe) reached a wall node */
    LBIB_ETIMEOUT = -6,    /* a bounded device wait expired (persistent batched step) */
    LBIB_ETOOBIG = -7      /* a size exceeds a fixed maximum (lbib_mesh_measures_noalloc) */
};

/* Storage precision of the populations.  FP64 stores and computes in
 * double; FP32 stores and computes in float; FP16_DEV / BF16_DEV store the
 * deviations f_i - w_i in half / bfloat16 and compute in float. */
typedef enum { LBIB_FP64 = 0, LBIB_FP32 = 1, LBIB_FP16_DEV = 2, LBIB_BF16_DEV = 3 } lbib_prec;

/* Boundary kind per axis: PERIODIC wraps; WALL makes the first and last
 * nodes of the axis Zou-He velocity-wall nodes (Sec. 2.1). */
typedef enum { LBIB_PERIODIC = 0, LBIB_WALL = 1 } lbib_bc;

typedef struct {
    int nx, ny, nz;          /* lattice nodes per axis; >= 3 on walled axes */
    double tau;              /* BGK relaxation time, > 0.5; nu = (tau - 1/2)/3 (Sec. 2.1) */
    double body_force[3];    /* uniform fluid body force g_ext (not applied on wall nodes) */
    int bc[3];               /* lbib_bc per axis */
    double wall_u[6][3];     /* wall velocity per face: -x, +x, -y, +y, -z, +z; on an edge or
                              * corner node the component along each of its faces' normals
                              * is that face's own, the others the mean over its faces */
    int precision;           /* lbib_prec */
    void *stream;            /* cudaStream_t to run on, or NULL for a library-owned stream */
    /* optional device allocator (e.g. a PyTorch caching allocator); both NULL
     * means cudaMalloc / cudaFree.  Blocks must be 256-byte aligned, as
     * cudaMalloc's are (the kernels use 16-byte vector accesses); a
     * misaligned block is handed back to free and counts as a failed
     * allocation (LBIB_ENOMEM) */
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *alloc_user;
} lbib_params;

typedef struct {
    int rigid;               /* 1: rigid body (Newton-Euler); 0: membrane (Verlet) */
    double ks0;              /* membrane: global stiffness k_s0 (Ca = rho nu u_ref / k_s0, Sec. 2.3) */
    double Eb;               /* membrane: bending ratio Eb = k_b / (k_s,l r^2) */
    double kv;               /* membrane: volume-penalty constant k_v (Eq. volFor) */
    double thickness;        /* membrane thickness T (springs and mass), lattice units */
    double density_ratio;    /* rho_s / rho_f: membrane mass or rigid-body density */
    double ref_radius;       /* r in the bending constant */
    double gravity[3];       /* rigid: gravity acceleration (adds (rho_s - rho_f) V g) */
    double u0[3], omega0[3]; /* rigid: initial linear and angular velocity */
    int bend_variant;        /* 0: k_b [1 - cos(theta - theta0)]; 1: k_b/2 (theta - theta0)^2 */
    int kinematic;           /* membrane: 1 advects the markers with the interpolated fluid velocity
                              * (the kinematic IB of Sec. 3.4) and spreads the internal forces
                              * alone; 0 the dynamic IB (Newton + Verlet) */
    int rigid_force;         /* rigid: 0 the hydrodynamic force and moment of the probe stress jumps
                              * (Eqs. hydroForP, hydroForNu, as printed); 1 momentum exchange: minus
                              * the previous step's IB force sum_l A_l F_l (and its moment) plus the
                              * inertia of the fluid inside the body, rho_f V du/dt and I_f dw/dt */
    int centroid_markers;    /* 0: the IB markers are the mesh vertices, each carrying a third of its
                              * triangles' area; 1: the IB markers are the triangle centroids (as
                              * printed in Sec. 2.3), each carrying its triangle's area, the vertices
                              * moving with the area-weighted mean of their triangles' centroid
                              * velocities */
    int mass_model;          /* membrane: the mass spread uniformly over the vertices (Eq. newtonSoft)
                              * is 0 that of a shell of thickness T and density rho_s, rho_s T A / N_v
                              * (Sec. 3.5), or 1 that of a capsule of density rho_s, rho_s V / N_v with
                              * V the enclosed volume (Sec. 3.4) */
} lbib_body_params;

typedef struct {
    double xc[3];            /* rigid: centre of mass; membrane: mean of the vertices */
    double u[3];             /* rigid: velocity; membrane: mean marker boundary velocity */
    double omega[3];         /* rigid: angular velocity; membrane: 0 */
    double q[4];             /* rigid: orientation quaternion (w, x, y, z); membrane: (1,0,0,0) */
    double volume, area;     /* enclosed volume and surface area of the current mesh */
} lbib_body_state;

/* Creates a context: allocates the two population buffers, the force field
 * and its tile flags, and sets the fluid at rest (f = f^eq(1, 0)).
 * out receives the context; returns LBIB_EINVAL for bad sizes, tau <= 1/2,
 * an unknown precision or bc; LBIB_ENOMEM / LBIB_ECUDA otherwise. */
int lbib_create(const lbib_params *p, void **out);

/* Sets the fluid to density 1 and the linear shear profile
 * u = (u_lo + (u_hi - u_lo) z / (nz - 1), 0, 0), the steady Couette flow
 * between z walls moving along x at u_lo and u_hi, as equilibrium
 * populations (Eq. eqfunc) formed on the device (nz = 1: at rest).
 * Asynchronous on the context stream.  LBIB_EINVAL for non-finite
 * velocities. */
int lbib_set_shear_fields(void *ctx, double u_lo, double u_hi);

/* Sets the fluid to equilibrium f = f^eq(rho(x), u(x)) (Eq. eqfunc).
 * rho[ncell], u[3*ncell] (x, y, z per cell), host or device doubles. */
int lbib_set_fields(void *ctx, const double *rho, const double *u, int on_device);

/* Sets the post-collision populations directly: f[ncell*19], 19 values per
 * cell in the order of Eq. (e_i).  Host or device doubles. */
int lbib_set_populations(void *ctx, const double *f, int on_device);

/* Adds an immersed body given its vertices (the Lagrangian markers,
 * verts[3*nv]) and outward, counter-clockwise triangles (tris[3*nt]) of a
 * closed manifold mesh (Sec. 2.2, Fig. IB).  The rest state (spring
 * constants, rest lengths and dihedral angles, volume, mass, inertia) is
 * computed here in FP64.  Host arrays.  body_id receives the body index.
 * LBIB_EINVAL for an open or inverted mesh or bad parameters. */
int lbib_add_body(void *ctx, const double *verts, int nv, const int *tris, int nt,
                  const lbib_body_params *bp, int *body_id);

/* Advances nsteps time steps, asynchronously on the context stream.  One
 * step: MLS interpolation at markers and hydrodynamic probes, structure
 * forces and update, spreading of the IB force (Eq. bodyforce), then the
 * fused stream + wall + collide sweep (Eq. evoleq).  Returns the sticky
 * error if one is recorded. */
int lbib_step(void *ctx, int nsteps);

/* Waits for the context stream and reports device-side errors. */
int lbib_sync(void *ctx);

/* Divergence detection (no counterpart in the paper; an explicit scheme
 * run outside its stability range produces NaN or runaway values, which
 * must fail the run instead of finishing it silently).  The run fails with
 * the sticky LBIB_EDIVERGED when:
 *  - every step, on the device: a marker (or probe) coordinate is non-finite
 *    or beyond 1e9, or a membrane vertex moves a lattice unit or more in one
 *    step (lattice velocities stay far below the speed of sound 0.577);
 *  - every `every` steps (a multiple of the context's step count; default
 *    1000, 0 turns it off), after that step, a watchdog kernel reads the
 *    whole lattice: some node's density is non-finite or not positive, or
 *    its speed |u| reaches the lattice speed of sound 1/sqrt(3), or the
 *    total mass, reduced in FP64 in a fixed order, differs from that of the
 *    first check after lbib_create / lbib_set_fields / lbib_set_populations
 *    by more than mass_tol relative (default 0.1).
 * The error surfaces at the next synchronising call, like LBIB_EBODY_WALL;
 * the state stays readable (lbib_get_*).  In a batch the watchdog of each
 * context runs after the lbib_batch_step call during which its cadence
 * fell.  Each check reads the populations once (76 B per node in FP32).
 * LBIB_EINVAL for every < 0 or mass_tol <= 0. */
int lbib_set_watchdog(void *ctx, int every, double mass_tol);

/* Runs the watchdog check on the current state now (queued after the steps
 * already queued), synchronises and returns the context's error:
 * LBIB_EDIVERGED if this or an earlier check failed, LBIB_OK otherwise. */
int lbib_check(void *ctx);

/* Density and velocity u = (sum f e + f_lb/2)/rho of the last collision
 * (Sec. 2.1): rho[ncell], u[3*ncell]; either may be NULL.  Synchronises. */
int lbib_get_fields(void *ctx, double *rho, double *u, int on_device);

/* Global mass and momentum of the post-collision populations, reduced on
 * the GPU in FP64 in a fixed order: out[0] = sum over nodes of sum_i f_i,
 * out[1..3] = sum over nodes of sum_i f_i e_i (host doubles).  Synchronises. */
int lbib_get_totals(void *ctx, double *out);

/* Post-collision populations, f[ncell*19] doubles.  Synchronises. */
int lbib_get_populations(void *ctx, double *f, int on_device);

/* Marker positions after the last step (X), the boundary velocity U_b
 * imposed in that step (V) and the Lagrangian IB force F_l (F), each
 * [3*nv] host doubles; any may be NULL.  Synchronises. */
int lbib_get_markers(void *ctx, int body, double *X, double *V, double *F);

/* The same three arrays, copied asynchronously: the copies are queued on the
 * context's stream after the steps already queued, and the call returns at
 * once.  The host arrays must stay valid until the stream reaches the
 * copies, and are read only after a synchronisation (lbib_sync, or an event
 * recorded on the context's stream after this call); page-locked host
 * memory makes the copies overlap later steps.  Device errors of the steps
 * surface at the next synchronising call.  LBIB_EINVAL for a bad body. */
int lbib_get_markers_async(void *ctx, int body, double *X, double *V, double *F);

/* Advances the context by nsteps steps and records body `body`'s markers
 * after each step k into X + 3 nv k, V + 3 nv k and F + 3 nv k (host arrays
 * of nsteps * 3 * nv doubles; any may be NULL): a trajectory recorded
 * without a host round trip per step.  Each step's markers are staged on the
 * device by one small kernel queued behind the step (in a context-owned
 * buffer of 3 * nsteps * 3 nv doubles, kept for later calls and grown when
 * needed); the device-to-host copies, one per requested array, are queued
 * after the last step.  The fields are stored as lbib_step(ctx, nsteps)
 * stores them (lbib_set_output), and steps that store none run from the
 * step graphs.  The same rules as lbib_get_markers_async apply to the host
 * arrays.  Errors as lbib_step; LBIB_ENOMEM if the staging buffer cannot be
 * allocated. */
int lbib_step_markers(void *ctx, int nsteps, int body, double *X, double *V, double *F);

/* Body summary after the last step.  Synchronises. */
int lbib_get_body(void *ctx, int body, lbib_body_state *out);

/* Number of steps taken and number of kernels launched so far. */
int lbib_counters(void *ctx, long long *steps, long long *launches);

/* Enables (1) or disables (0) CUDA-event timing of the kernels of each
 * step, recorded on the context stream. */
int lbib_profile(void *ctx, int enable);

/* Timing since profiling was enabled or last read: ms[0] total
 * milliseconds of the MLS stage (support-region moments, interpolation and
 * probes), ms[1] of the structure update and spreading, ms[2] of the
 * collide-stream sweeps (both parts when they overlap the IB stage), ms[3]
 * of the steps from start to end; nsteps receives the number of steps
 * timed.  ms has 4 entries.  Synchronises and resets the accumulators. */
int lbib_get_profile(void *ctx, double *ms, long long *nsteps);

/* Times the step in several launch configurations and keeps the fastest:
 * the sweep kernel and its block shape (the row-tile kernel with 128-bit
 * loads and stores where rows are whole 16-byte vectors, or the one-node
 * kernel in several shapes), then (single-body contexts) the overlap of the far-field
 * sweep with the IB stage.  Each trial runs
 * 1 + 2 * `steps` real time steps, so the simulation advances by about
 * 16 * `steps` steps.  choice (optional, 5 ints) receives block x, block y (0, 0: whole
 * x-rows), the overlap flag, the row-tile flag and the far-field blocks per
 * SM (0: full grid).  With overlap it also chooses the IB kernels' blocks
 * per SM (0, 1 or 2; lbib_get_launch_config reports it). */
int lbib_autotune(void *ctx, int steps, int *choice);

/* Sets the sweep launch configuration (what lbib_autotune chooses):
 * row_tiles = 1 selects the row-tile kernel (x-rows staged in shared memory
 * with 128-bit loads and stores; any precision with rows of whole 16-byte
 * vectors: nx a multiple of 4 in FP32/FP64, of 8 in FP16/BF16, else
 * ignored), 0 the one-node kernel with blocks of block_x * block_y threads
 * (0, 0: whole x-rows); far_per_sm > 0 runs the far-field sweep (overlap
 * on) with that many resident blocks per SM striding over the lattice, so
 * that the IB kernels beside it find free SMs, 0 on its full grid.  Results
 * are the same in every configuration. */
int lbib_set_sweep_config(void *ctx, int row_tiles, int block_x, int block_y, int far_per_sm);

/* Resident blocks per SM of the IB kernels (MLS, structure update and
 * spreading): 0 (default) launches their full grids; k > 0 launches at
 * most k blocks per SM, each taking its share of the work in turn, so that
 * a far-field sweep running beside them keeps the rest of every SM (the IB
 * kernels hold up to all of an SM's registers otherwise).  Results are the
 * same in every configuration.  LBIB_EINVAL outside [0, 64]. */
int lbib_set_ib_blocks(void *ctx, int per_sm);

/* The launch configuration in use, 6 ints: block_x, block_y, overlap,
 * row_tiles, far_per_sm (as lbib_autotune's choice) and the IB blocks per
 * SM (lbib_set_ib_blocks). */
int lbib_get_launch_config(void *ctx, int *cfg);

/* With a single body, the sweep of the nodes outside the body's support
 * box runs on a second stream concurrently with the IB stage (default 1);
 * 0 runs one whole-lattice sweep after the IB stage.  Results are the same
 * either way. */
int lbib_set_overlap(void *ctx, int enable);

/* Steps that do not store the fields run as CUDA graphs captured on first
 * use (one per phase of the six-step rotation of the population, position
 * and support-box buffers) and launched into the context stream (enable = 1,
 * default); 0 enqueues every kernel of every step.  Results are identical.
 * Adding a body, changing the overlap or autotuning recaptures. */
int lbib_set_graphs(void *ctx, int enable);

/* When the sweep also writes the macroscopic fields read by
 * lbib_get_fields: fields_every = 0 (default) on the last step of each
 * lbib_step call, k > 0 on every k-th step, < 0 never (lbib_get_fields then
 * returns the fields of the last step that wrote them). */
int lbib_set_output(void *ctx, int fields_every);

/* Checkpoint: the context's device state (populations, IB force and its
 * tile flags, fields, bodies' positions, velocities, forces, transfer
 * weights and rigid states, counters) and its step counters, into a host
 * buffer.  buf == NULL: *size receives the bytes needed.  Otherwise *size is
 * the buffer's capacity on entry and the bytes written on return.
 * Synchronises. */
int lbib_save(void *ctx, void *buf, size_t *size);

/* Restores a checkpoint into a context set up the same way (same lattice,
 * precision and bodies added in the same order); the run continues exactly
 * where the saved one stood.  Clears a sticky error.  LBIB_EINVAL for a
 * buffer from a differently set-up context (nothing is changed then). */
int lbib_load(void *ctx, const void *buf, size_t size);

/* Bytes of device memory held by the context. */
int lbib_device_bytes(void *ctx, size_t *bytes);

/* ---- batches -----------------------------------------------------------
 * A batch advances the lattices and bodies of several contexts with common
 * launches: per step one support-moments, one MLS, one membrane (and rigid)
 * and one collide-stream launch cover every lattice of the batch, each
 * launch splitting its blocks over the lattices or bodies by prefix sums.
 * Steps run six at a time from one captured CUDA graph (one graph per batch;
 * six steps bring every buffer rotation back to its start).  Each context
 * computes exactly what lbib_step would (up to the order of the atomic
 * spreading sums).  Used for many small, uneven runs at once. */

/* Creates a batch of n contexts (same precision; each context in at most
 * one live batch).  stream: cudaStream_t of the batch, or NULL for a
 * library-owned one.  Waits for the contexts' queued work.  out receives
 * the batch.  LBIB_EINVAL for mixed precisions, repeated or NULL contexts;
 * the message is lbib_batch_last_error(NULL). */
int lbib_batch_create(void *const *ctxs, int n, void *stream, void **out);

/* Advances every context of the batch by nsteps (asynchronously on the
 * batch stream, ordered after each context's queued work; later work on a
 * context's stream is ordered after it).  The fields of the last step are
 * stored, as with lbib_step.  A context stepped on its own since the batch
 * was built makes this return LBIB_EINVAL (rebuild the batch). */
int lbib_batch_step(void *batch, int nsteps);

/* Waits for the batch and reports the first context error. */
int lbib_batch_sync(void *batch);

/* Steps taken through the batch and kernels launched by it. */
int lbib_batch_counters(void *batch, long long *steps, long long *launches);

/* Times `steps` six-step graph launches and one field-storing step (what
 * a long lbib_batch_step runs) for each sweep configuration and keeps the
 * fastest:
 * the batched sweep with 128, 256 or 512 threads a block and 1 or 4 cells a
 * thread, one one-lattice sweep launch per lattice spread over side
 * streams, or the persistent kernel (lbib_batch_set_persistent) with sweep
 * tiles of 256 x 4, 8 or 16 cells, each with the lattices as given or
 * largest first; the contexts advance by 20 * (24 + 12 * steps) steps.
 * choice (optional, 3 ints): threads (0: one launch per lattice, -1: the
 * persistent kernel), order, cells per thread. */
int lbib_batch_autotune(void *batch, int steps, int *choice);

/* Persistent mode (enable = 1): every six-step chunk of lbib_batch_step
 * runs as one kernel launch (captured once as a CUDA graph with the reset
 * of its counters) instead of one launch per kernel and step.  The launch
 * keeps as many blocks resident as fit on the GPU; they take work items
 * in a fixed order from a global ticket counter -- per body the support
 * moments, MLS, structure-update and spreading blocks, per lattice the
 * sweep tiles (256 x cells_per_thread cells, lbib_batch_set_config), step
 * after step -- and start an item once the items it depends on (its
 * lattice's earlier phases of the step, and its previous sweep) have
 * finished, so one lattice's IB work runs beside other lattices' sweeps.
 * An item only waits for items taken before it, by blocks already
 * running, so the queue cannot deadlock; each wait is still bounded by
 * wait_limit_s (2 s is ample: a whole chunk takes milliseconds), after
 * which the launch ends and every context of the batch holds the sticky
 * LBIB_ETIMEOUT (0 gives up at the first wait that finds its items
 * unfinished: a way to exercise that path).  Results are those of the
 * per-kernel launches (up to the order of the atomic spreading sums).
 * Waits for the batch's queued work and rebuilds its tables.  LBIB_EINVAL
 * for enable not 0 or 1 or a wait limit outside [0, 60] s. */
int lbib_batch_set_persistent(void *batch, int enable, double wait_limit_s);

/* Sets what lbib_batch_autotune chooses: threads a block of the batched
 * sweep (a multiple of 32 up to 512; 0: one one-lattice sweep launch per
 * lattice on side streams), order (0 lattices as given, 1 largest first)
 * and cells a sweep thread (1 to 16).  Waits for the batch's queued work
 * and rebuilds its tables.  LBIB_EINVAL for values out of range (the batch
 * is unchanged then).  Results are the same in every configuration. */
int lbib_batch_set_config(void *batch, int threads, int order, int cells_per_thread);

/* Releases the batch (not its contexts). */
void lbib_batch_destroy(void *batch);

/* Message of the last error of a batch (NULL: of the last failed create). */
const char *lbib_batch_last_error(const void *batch);

/* ---- serving --------------------------------------------------------------
 * A server runs submitted requests (a lattice, its initial state, bodies and
 * a step count) to completion on the current GPU.  A worker thread admits
 * queued requests in arrival order while the estimated device memory of the
 * admitted ones fits hbm_budget, and advances all admitted runs together as
 * one batch (lbib_batch_*), chunk_steps steps at a time or fewer: a chunk
 * ends when the run with the fewest remaining steps finishes.  A chunk that
 * advances a single run steps it with lbib_step.  Finished runs
 * leave the batch, arrivals join it, and the batch is rebuilt (continuous
 * batching).  LBIB_SERVE_PLAIN instead runs one request at a time with
 * lbib_step, in arrival order.  A run that diverges (lbib_set_watchdog, at
 * its context's default cadence, and lbib_check when its steps are done)
 * fails with LBIB_EDIVERGED and leaves the batch; the other runs go on.  A finished run's context stays resident (and
 * counts against the budget) until the caller takes it. */
enum { LBIB_REQ_QUEUED = 0, LBIB_REQ_RUNNING = 1, LBIB_REQ_DONE = 2, LBIB_REQ_FAILED = 3 };
enum { LBIB_SERVE_BATCHED = 0, LBIB_SERVE_PLAIN = 1 };
enum { LBIB_SERVE_SHORTEST = 0, LBIB_SERVE_OLDEST = 1 };

typedef struct {
    size_t hbm_budget;  /* bytes of device memory the admitted runs may hold */
    int chunk_steps;    /* longest chunk between admissions (> 0) */
    int max_active;     /* most runs in the batch at once (>= 1) */
    int mode;           /* LBIB_SERVE_BATCHED or LBIB_SERVE_PLAIN */
    long long batch_cells; /* batched mode: 0 advances every admitted run in each chunk; > 0 advances
                            * up to this many lattice cells of runs (at least one run), chosen in
                            * batch_order, the others waiting resident */
    int batch_order;       /* with batch_cells > 0: LBIB_SERVE_SHORTEST the runs with the least
                            * remaining work (cells x steps) first, LBIB_SERVE_OLDEST the earliest
                            * submitted first.  LBIB_EINVAL for other values. */
} lbib_serve_params;

typedef struct {
    double submit_s;    /* submission time since the server started */
    double queued_s;    /* submission to admission */
    double latency_s;   /* submission to completion */
    double done_s;      /* completion time since the server started */
    char error[160];    /* message of a failed run ("" otherwise) */
} lbib_serve_times;

typedef struct {
    long long runs_done, runs_failed, queued, active, chunks, rebuilds;
    double cell_updates;  /* lattice-cell updates performed */
    double busy_s;        /* wall time the worker spent advancing runs */
    size_t bytes_in_use, peak_bytes;  /* memory estimate of admitted runs */
} lbib_serve_summary;

/* A request: lattice parameters (p->stream, p->alloc and p->free are
 * ignored), nsteps steps, init = 0 fluid at rest, 1 the linear shear
 * profile between the z walls (x velocity from the -z to the +z wall
 * velocity).  Host arrays are copied. */
int lbib_request_create(const lbib_params *p, long long nsteps, int init, void **req);
int lbib_request_add_body(void *req, const double *verts, int nv, const int *tris, int nt,
                          const lbib_body_params *bp);
/* Frees a request that was never submitted. */
void lbib_request_destroy(void *req);

/* Starts a server on the current device with its own stream and worker
 * thread. */
int lbib_serve_create(const lbib_serve_params *sp, void **server);
/* Queues a request (the server takes ownership); id receives its ticket. */
int lbib_serve_submit(void *server, void *req, long long *id);
/* Waits until the request is done or failed (timeout_s < 0: no limit);
 * state receives LBIB_REQ_*.  Returns LBIB_ETIMEOUT if still running, the
 * run's error code if it failed (LBIB_ENOMEM: larger than the budget). */
int lbib_serve_wait(void *server, long long id, double timeout_s, int *state);
/* Hands a finished request's context to the caller (who destroys it with
 * lbib_destroy) and releases its ticket; t (optional) receives its times. */
int lbib_serve_take(void *server, long long id, void **ctx, lbib_serve_times *t);
int lbib_serve_stats(void *server, lbib_serve_summary *out);
/* Drops queued requests, lets running ones finish, frees everything left
 * (including contexts not taken). */
void lbib_serve_destroy(void *server);

/* Largest triangle count lbib_mesh_measures_noalloc accepts. */
#define LBIB_NOALLOC_MAX_TRIS (1 << 20)

/* Enclosed volume and surface area of a closed triangle mesh, computed on
 * the GPU without allocating any memory.  The paper has no counterpart: it
 * is a stand-alone, allocation-free variant of the membrane-volume reduction
 * the step performs (and gives the volume and area lbib_get_body reports).
 *
 * For callers that cannot call cudaMalloc: code that runs while another
 * thread captures a CUDA graph in global capture mode (cudaMalloc is then
 * an error), code whose device memory is reserved up front by a pool or a
 * budget, and latency-bound loops where an allocation would synchronise
 * the device.  No context is needed.
 *
 * X[3*nv] (vertex x, y, z) and tris[3*nt] (vertex indices of outward,
 * counter-clockwise triangles) are device arrays; out[2] (device) receives
 * the volume (sum over triangles of X0 . (X1 x X2) / 6) and the area.
 * Asynchronous on `stream` (a cudaStream_t); the caller owns every array.
 * NULL means the legacy default stream, whose work synchronises implicitly
 * with every blocking stream: a caller running while another thread
 * captures a graph must pass a stream created with cudaStreamNonBlocking,
 * or cudaStreamPerThread, or the implicit synchronisation invalidates that
 * capture.  A vertex index outside [0, nv) is skipped and makes both
 * outputs NaN.  nt = 0 gives zeros.
 *
 * Scratch: a 64 KiB file-scope device array (plus a counter), held on every
 * GPU that loads the library until the process exits, so nt is limited to
 * LBIB_NOALLOC_MAX_TRIS; larger nt returns LBIB_ETOOBIG, negative sizes or
 * NULL arrays LBIB_EINVAL, a failed CUDA call LBIB_ECUDA.  Every call looks
 * up the array's device address in the current device's context
 * (cudaGetSymbolAddress; nothing is cached, so a reset device is handled);
 * the first call in a process may also load the library's device code, so
 * make it before any stream capture.  Each call then issues one
 * cudaMemsetAsync and one kernel launch on `stream`.
 * Every call shares the array (each clears its counter first), so calls
 * that overlap on the GPU -- on different streams, or from different host
 * threads -- race and must be serialised by the caller.  Allocates nothing:
 * no cudaMalloc, cudaFree or allocating library routine. */
int lbib_mesh_measures_noalloc(const double *X, int nv, const int *tris, int nt, double *out, void *stream);

/* Fused multiply-add throughput of the current device in flops/s (two per
 * FMA), FP64 (fp64 = 1) or FP32 (0), measured by a short kernel of
 * independent FMA chains (a few blocks per SM, about 10 ms): the arithmetic
 * peak for the roofline of FP64 kernels, which GB300 issues at a small
 * fraction of its FP32 rate.  Allocates and frees a few bytes; synchronises
 * its own stream.  LBIB_EINVAL for a NULL output, LBIB_ECUDA on a CUDA
 * error.  Not part of the method (a measurement aid). */
int lbib_measure_fma(int fp64, double *flops_per_s);

/* Releases all device and host memory of the context (NULL is a no-op). */
void lbib_destroy(void *ctx);

/* Message of the last error of ctx (or of the last failed lbib_create when
 * ctx is NULL).  Valid until the next call on the context. */
const char *lbib_last_error(const void *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBIB_H */
