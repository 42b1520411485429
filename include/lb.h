/*
 * lb.h -- C ABI of the GB300 lattice Boltzmann library for capillary filling.
 *
 * The library advances the D2Q9 free-energy multiple-relaxation-time lattice
 * Boltzmann scheme of Pooley, Kusumaatmaja & Yeomans, "Modelling capillary
 * filling dynamics using lattice Boltzmann simulations", for two models:
 *   - the van der Waals liquid-gas model (one distribution f; Sec. 2, Eq. (pt),
 *     p0 = rho T / (1 - b rho) - a rho^2), and
 *   - the binary model (f for the density, g for the order parameter phi;
 *     Sec. 3.1, Eq. (chempot), Eq. (latbolt2), viscosity nu(phi) of Eq. (nu)),
 * with the evolution of Eq. (latbolt), the matrices M and S and the equilibria
 * of Appendix A, the stencils of Eq. (best), bounce-back walls whose boundary
 * nodes are set to rest after streaming, and a prescribed wall gradient
 * d_n rho|_b or d_n phi|_b that sets the contact angle (Sec. 2.2).
 *
 * Conventions for every call:
 *   - Every function returns lb_status (or nothing); no C++ exception crosses
 *     this boundary.  On failure lb_last_error() describes the cause.
 *   - Host arrays are row-major (ny, nx) doubles, x contiguous; population
 *     arrays are plane-major (9, ny, nx).  The caller owns them; the library
 *     only reads or writes them during the call.
 *   - Device memory belongs to the context.  It is obtained through the
 *     optional lb_alloc callbacks, or cudaMalloc when none are given, and is
 *     released by lb_destroy.
 *   - Work is issued on the stream passed to lb_create (a cudaStream_t, NULL for
 *     the default stream).  lb_step returns without waiting; every call that
 *     returns data to the host waits for the stream.
 *   - After LB_ERR_NONFINITE or LB_ERR_TIMEOUT, lb_step and lb_autotune return
 *     LB_ERR_STATE until the state is replaced (lb_init_fields,
 *     lb_set_populations or lb_load_state, which clear the condition); the reading calls
 *     (lb_fields, lb_get_populations, lb_get_moments, lb_filled_length),
 *     lb_last_error and lb_destroy remain available.
 *
 * Geometry (Sec. 2.2, Fig. 1b): the grid is periodic in x and y.  The tube
 * occupies the columns [tube_x0, tube_x0 + tube_len) (mod nx); inside them the
 * rows [tube_y0, tube_y0 + tube_h) (mod ny) are fluid and the other rows are
 * solid, so one block of solid forms both walls through the y-wrap.  Columns
 * outside the tube are reservoirs, periodic in y.  tube_len = 0: no solid at
 * all; tube_len = nx: walls along the whole length.  Valid geometries have
 * tube_h >= 2, a solid thickness ny - tube_h >= 1 and, when 0 < tube_len < nx,
 * at least 2 reservoir columns.
 */
#ifndef LB_GB300_H
#define LB_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
  LB_OK = 0,
  LB_ERR_ARG = 1,       /* invalid argument; nothing was changed */
  LB_ERR_CUDA = 2,      /* a CUDA call failed; see lb_last_error */
  LB_ERR_NONFINITE = 3, /* a reduction found a NaN or Inf in the state */
  LB_ERR_TIMEOUT = 4,   /* a device-side wait gave up (staged or persistent kernel) */
  LB_ERR_STATE = 5,     /* call not allowed in the context's current state */
  LB_ERR_NOMEM = 6      /* device allocation failed */
} lb_status;

typedef enum { LB_MODEL_LIQUID_GAS = 0, LB_MODEL_BINARY = 1 } lb_model;

/* Storage of the distributions.  Arithmetic is FP64 for LB_STORAGE_F64 and FP32
 * otherwise.  LB_STORAGE_F16DEV keeps f_i - w_i rho0 and g_1..g_8 in FP16 and
 * g_0 in FP32, with rho0 = 1 and w_i the rest weights of the binary model's
 * equilibrium (Eq. (equilibrium), App. A) in the bulk phases, where
 * P0 = 1/3 + A/4: w_0 = 1 - 5 P0/3, w_1..w_4 = P0/3, w_5..w_8 = P0/12 (the
 * standard 4/9, 1/9, 1/36 for A = 0).
 *
 * LB_STORAGE_MOMENTS (binary model only) keeps six FP32 numbers per node
 * instead of the populations: rho, jx, jy, pxx - pyy, pxy of f and phi of g.
 * With the relaxation matrix of App. A every other mode of f, and every mode
 * of g, relaxes fully to equilibrium in one collision (Sec. 3.1), so the next
 * state depends on nothing else: the update is the population scheme's in
 * exact arithmetic, with 48 instead of 144 bytes moved per node update.  The
 * populations themselves are not kept (lb_get_populations returns LB_ERR_ARG;
 * lb_get_moments reads the state), and lb_set_populations stores their
 * moments.  The density is held as rho - 1 (the binary model keeps rho near
 * 1), which lb_get_moments, lb_fields and the reductions add back in FP64.  At
 * most 715827882 nodes (6 nx ny < 2^32).
 *
 * LB_STORAGE_MOMENTS_F16 (binary model only) keeps the same six moments with
 * rho - 1, jx, jy, pxx - pyy and pxy in FP16 and phi in FP32 (FP32 arithmetic):
 * 28 bytes per node update.  Like LB_STORAGE_MOMENTS it keeps no populations.
 *
 * LB_STORAGE_F32_GELIM (binary model only) keeps the nine f populations in FP32,
 * as deviations f_i - w_i from w = 4/9, 1/9, 1/36, and phi in place of the nine
 * g populations, which all relax fully to g^eq (App. A, Eq. (latbolt2)):
 * 80 bytes per node update.  lb_get_populations returns f and, for g, the
 * populations (phi, 0, ..., 0), whose phi is the only moment of g a step uses.
 * At most 429496729 nodes (10 nx ny < 2^32).
 *
 * LB_STORAGE_F32_BLOCKED (binary model only) keeps the eighteen FP32
 * populations, with the values and arithmetic of LB_STORAGE_F32 (the two give
 * identical results), in blocks of 32 consecutive nodes n = y nx + x: block
 * b = n / 32 holds, for i = 0..8, the pairs (f_i, g_i) of its 32 nodes in node
 * order, so f_i of node n is float element 576 b + 64 i + 2 (n % 32) of the
 * state and g_i the element after it; the last block is padded, so the state
 * holds 18 * 32 * ceil(nx ny / 32) floats
 * (lb_save_state writes this layout).  A row of a tile with its neighbour
 * columns is then one contiguous range of blocks, which the staged step kernel
 * fetches with one bulk copy per row (plus one block at an x-wrap) instead of one
 * copy per population plane; any nx.  At most 238609280 nodes
 * (18 * 32 * ceil(nx ny / 32) < 2^32).
 *
 * LB_STORAGE_F16_BLOCKED (binary model only) keeps the values of
 * LB_STORAGE_F16DEV (FP16 f_i - w_i rho0 and g_1..g_8, FP32 g_0; the two give
 * identical results) in blocks of 32 consecutive nodes: block b = n / 32 is
 * 1216 bytes: f_0 less its offset (FP16, 32 values), then for i = 1..8 the pairs
 * (f_i less its offset, g_i) of the 32 nodes (FP16), then g_0 (FP32), so f_0 of
 * node n is half element 608 b + n % 32 of the state, f_i (i >= 1) half
 * 608 b + 32 + 64 (i - 1) + 2 (n % 32), g_i the half after it and g_0 float
 * 304 b + 272 + n % 32; the last block is padded (the state is
 * 1216 ceil(nx ny / 32) bytes; lb_save_state writes this layout).  One bulk copy
 * per staged row, as for LB_STORAGE_F32_BLOCKED; any nx.  At most 226050880 nodes
 * (19 * 32 * ceil(nx ny / 32) < 2^32). */
typedef enum {
  LB_STORAGE_F64 = 0,
  LB_STORAGE_F32 = 1,
  LB_STORAGE_F16DEV = 2,
  LB_STORAGE_MOMENTS = 3,
  LB_STORAGE_MOMENTS_F16 = 4,
  LB_STORAGE_F32_GELIM = 5,
  LB_STORAGE_F32_BLOCKED = 6,
  LB_STORAGE_F16_BLOCKED = 7
} lb_storage;

typedef struct {
  int nx, ny;
} lb_grid;

typedef struct {
  int tube_x0, tube_len; /* tube columns [tube_x0, tube_x0 + tube_len) mod nx */
  int tube_y0, tube_h;   /* fluid band [tube_y0, tube_y0 + tube_h) mod ny inside the tube */
  int gas_cols;          /* default initial state: gas in x < gas_cols (Sec. 2.2 reservoirs) */
  double wall_grad;      /* d_n rho|_b (liquid-gas) or d_n phi|_b (binary), n = inward normal */
} lb_walls;

typedef struct {
  int model;               /* lb_model */
  int storage;             /* lb_storage */
  double kappa, a, b, T;   /* liquid-gas: kappa = 0.02, a = 9/49, b = 2/21, T = 0.56 (Sec. 2) */
  double A, M;             /* binary: A (= kappa = 0.04, Sec. 3.1) and mobility M (Eq. diff) */
  double nu_l, nu_g;       /* binary: bulk kinematic viscosities of Eq. (nu) */
  double nu;               /* liquid-gas kinematic viscosity; omega = 2/(6 nu + 1) (App. A) */
  double lambda_scale;     /* lambda of Eq. (equilibrium) = lambda_scale * local nu */
  double rho_l, rho_g;     /* liquid-gas: densities of the default initial state and of the
                              l(t) threshold (rho_l + rho_g)/2 */
  int l0;                  /* default initial state: liquid in [gas_cols, tube_x0 + l0) */
  int nu_table;            /* binary: 0 = omega from the exact local nu; K >= 2 = from the
                              nearest of K viscosities evenly spaced over [nu_g, nu_l], the
                              look-up table of App. A (the paper uses ~10^4) */
} lb_params;

/* Optional device allocator.  malloc_fn returns device memory of at least bytes
 * bytes usable on stream, or NULL; free_fn releases it. */
typedef struct {
  void *(*malloc_fn)(size_t bytes, void *stream, void *user);
  void (*free_fn)(void *ptr, void *stream, void *user);
  void *user;
} lb_alloc;

/* Create a lattice and set the default initial state (Sec. 2.2: u = 0, liquid
 * in [gas_cols, tube_x0 + l0), gas elsewhere, tanh profiles of width 2 for the
 * liquid-gas model and sqrt(2) for phi, f = f^eq and g = g^eq of Appendix A).
 * stream is a cudaStream_t or NULL.  *out is set only on LB_OK. */
lb_status lb_create(const lb_grid *grid, const lb_walls *walls, const lb_params *params,
                    const lb_alloc *alloc, void *stream, lb_ctx **out);

/* Release every device buffer and the context.  NULL is ignored. */
void lb_destroy(lb_ctx *ctx);

/* Reset the state to equilibrium with the given macroscopic host fields
 * ((ny, nx) doubles; phi may be NULL for the liquid-gas model and is required
 * for the binary model).  Values at solid nodes are ignored.  Sets time to 0. */
lb_status lb_init_fields(lb_ctx *ctx, const double *rho, const double *ux, const double *uy,
                         const double *phi);

/* Advance n >= 0 time steps of Eq. (latbolt) (and Eq. (latbolt2)): stencils,
 * equilibria, collision, streaming with bounce-back, rest of boundary nodes.
 * Asynchronous on the context's stream. */
lb_status lb_step(lb_ctx *ctx, long n);

/* Copy the macroscopic fields rho, u = j/rho and phi to host arrays ((ny, nx)
 * doubles, any may be NULL; phi is 0 for the liquid-gas model).  Boundary nodes
 * report u after the rest rule.  Solid nodes report 0.  Waits for the stream. */
lb_status lb_fields(lb_ctx *ctx, double *rho, double *ux, double *uy, double *phi);

/* FP64 reductions (Sec. 1 defines l): l_centre = distance from tube_x0 to the
 * first sign change of phi (binary) or rho - (rho_l + rho_g)/2 (liquid-gas)
 * along the tube's middle row (mean of the two middle rows for even tube_h),
 * linearly interpolated, 0 if the inlet is already gas and tube_len if there is
 * no change; l_vol = sum over tube nodes of the liquid fraction / tube_h;
 * mass = sum of rho and phi_sum = sum of phi over fluid nodes.  Any pointer may
 * be NULL.  Returns LB_ERR_NONFINITE (and poisons the context) if mass or
 * phi_sum is not finite.  Waits for the stream. */
lb_status lb_filled_length(lb_ctx *ctx, double *l_centre, double *l_vol, double *mass,
                           double *phi_sum);

/* Copy the populations to host arrays (9, ny, nx) of doubles (g may be NULL;
 * it is left untouched for the liquid-gas model).  rested != 0 applies the
 * boundary-node rest rule of Sec. 2.2 to f on the way out; rested = 0 returns
 * the stored state exactly (the library applies that rule when it next reads a
 * boundary node).  Waits for the stream. */
lb_status lb_get_populations(lb_ctx *ctx, double *f, double *g, int rested);

/* Replace the populations (plane-major host doubles, rounded to the storage
 * type).  g is required for the binary model.  Solid nodes are ignored. */
lb_status lb_set_populations(lb_ctx *ctx, const double *f, const double *g);

/* The six moments of the stored state, host array (6, ny, nx) of doubles in
 * the order rho, jx, jy, pxx - pyy, pxy (of f), phi (sum of g; 0 for the
 * liquid-gas model): for the population storages they are summed in FP64
 * from the stored populations (LB_STORAGE_F32_GELIM: from f, and phi), for the
 * moment storages they are the state.  As
 * lb_get_populations with rested = 0, boundary nodes are returned before the
 * rest rule (which would set j = 0).  Solid nodes give zeros.  Waits for the
 * stream. */
lb_status lb_get_moments(lb_ctx *ctx, double *m);

/* Checkpoints: the stored state exactly as the storage holds it (the f
 * planes, then the g planes, then the FP32 g_0 plane of LB_STORAGE_F16DEV; for
 * the storages advanced by the pull kernel their planes as the device holds
 * them), lb_state_bytes bytes in host
 * memory the caller owns.  lb_load_state takes such bytes from a lattice of the
 * same grid, walls and params (LB_ERR_ARG if the size differs), sets the step
 * counter to time and clears a non-finite or timed-out condition; the
 * continued run is bit for bit the run that was saved.  Both wait for the
 * stream. */
size_t lb_state_bytes(const lb_ctx *ctx);
lb_status lb_save_state(lb_ctx *ctx, void *host, size_t bytes);
lb_status lb_load_state(lb_ctx *ctx, const void *host, size_t bytes, long time);

/* Bounds-checked debug build of the library (compiled with -DLB_CHECK): every
 * global load and store of the step kernels checks its index against its
 * buffer; an index outside is counted, the first one recorded and the access
 * skipped (a load reads 0), with no trap.  This call returns the count of such
 * accesses and the first offending element index + 1 since the last call (the
 * counters are then cleared), with *enabled = 1.  The counters belong to the
 * kernels of the context's model and storage and count every lattice of that
 * model and storage in the process.  In the normal build *enabled, *bad and
 * *first_bad are 0.  Any pointer may be NULL.  Waits for the device. */
lb_status lb_check_report(lb_ctx *ctx, int *enabled, unsigned long long *bad,
                          unsigned long long *first_bad);

/* Wait for all work issued on the context's stream; LB_ERR_TIMEOUT if a
 * device-side wait of the step kernel gave up since the state was set. */
lb_status lb_sync(lb_ctx *ctx);

/* Failure injection on the host, for tests of the recovery path: marks the
 * context's device error word exactly as a staged-kernel wait that gave up
 * marks it, with no kernel running.  The next call that waits (lb_sync,
 * lb_filled_length) returns LB_ERR_TIMEOUT and poisons the context; a new
 * state (lb_init_fields, lb_set_populations, lb_load_state) clears both the
 * word and the condition.  Waits for the stream. */
lb_status lb_inject_wait_timeout(lb_ctx *ctx);

/* Time steps taken since the last initialisation. */
long lb_time(const lb_ctx *ctx);

/* Fluid (non-solid) node count. */
long lb_fluid_nodes(const lb_ctx *ctx);

/* Choose the tile of the step kernel: tile_x threads per block along x (64,
 * 128 or 256) and tile_y rows per block (1 .. ny).  Invalidates the captured
 * step graph. */
lb_status lb_set_tile(lb_ctx *ctx, int tile_x, int tile_y);
lb_status lb_get_tile(const lb_ctx *ctx, int *tile_x, int *tile_y);

/* Choose the step kernel: 0 = automatic (the staged kernel whenever it fits,
 * else the sliding-window kernel), 1 = sliding-window kernel (rows held in
 * registers), 2 = staged kernel (rows brought into shared memory by bulk
 * copies; fits when nx % 8 == 0 and nx * ny <= 477218588, and at any nx for
 * the block storages, else LB_ERR_ARG)
 * with its shallow ring of row stages, 3 = staged kernel with its deep ring.
 * All compute the same update bit for bit.  LB_STORAGE_MOMENTS,
 * LB_STORAGE_MOMENTS_F16 and LB_STORAGE_F32_GELIM have one kernel of their own,
 * the pull kernel over the reduced state (variant 4; 0 and 4 are accepted).  Invalidates the captured step
 * graph. */
lb_status lb_set_kernel(lb_ctx *ctx, int variant);
/* The kernel variant in use (1, 2, 3 or 4; automatic selection resolved). */
lb_status lb_get_kernel(const lb_ctx *ctx, int *variant);

/* Time each candidate kernel variant and tile on this lattice (the state is
 * saved and restored) and keep the fastest.  Returns the choice and its time per step in
 * microseconds.  Waits for the stream. */
lb_status lb_autotune(lb_ctx *ctx, int *tile_x, int *tile_y, double *us_per_step);

/* Description of the last error on ctx (or of the last failed lb_create when
 * ctx is NULL).  Never NULL. */
const char *lb_last_error(const lb_ctx *ctx);

/* Diagnostic: the FP64 fused multiply-add rate of the current device in
 * TFLOP/s (2 flops per FMA), measured on `stream` (a cudaStream_t; NULL for the
 * legacy default stream) by a kernel of independent FMA chains, 8 CTAs of 256
 * threads per SM, best of three launches after one warm-up (tens of
 * milliseconds; waits for the stream).  The liquid-gas model computes in FP64
 * (the van der Waals pins of Sec. 2 and the densities near 4 want its
 * precision), and on this GPU FP64 arithmetic, not HBM, bounds that path; this
 * is the ceiling its roofline is quoted against.  LB_ERR_ARG if tflops is
 * NULL, LB_ERR_CUDA if a CUDA call fails (*tflops is then 0). */
lb_status lb_fp64_fma_rate(void *stream, double *tflops);

/* ------------------------------------------------------------------------
 * Batched sweeps: many binary capillaries of different sizes and parameters
 * advanced together by one persistent kernel (every lattice of a batch takes
 * the same number of steps).  The paper runs its capillaries one at a time; a
 * batch exists to fill the GPU with the parameter sweeps behind Figs. 5 and 6
 * and behind the l(t) surrogate.  Each lattice evolves exactly as it would in
 * its own lb_ctx with the same parameters (bit for bit).
 * ------------------------------------------------------------------------ */
typedef struct lb_batch lb_batch;

/* n lattices, each described as for lb_create (all binary, one common
 * storage: LB_STORAGE_F64, LB_STORAGE_F32, LB_STORAGE_F32_BLOCKED,
 * LB_STORAGE_F16DEV, LB_STORAGE_F16_BLOCKED or LB_STORAGE_MOMENTS), each set to
 * the default initial
 * state.  *out set only on LB_OK. */
lb_status lb_batch_create(int n, const lb_grid *grids, const lb_walls *walls, const lb_params *params,
                          const lb_alloc *alloc, void *stream, lb_batch **out);
void lb_batch_destroy(lb_batch *b);

/* Advance every lattice by n steps: one cooperative persistent launch whose
 * CTAs take the tiles of all lattices in turn and meet at a grid barrier after
 * each step.  A barrier that does not complete within its time limit makes the
 * next call that waits return LB_ERR_TIMEOUT.  Asynchronous. */
lb_status lb_batch_step(lb_batch *b, long n);

/* out[i*4 + k] = {l_centre, l_vol, mass, phi_sum} of lattice i (definitions as
 * in lb_filled_length).  Waits for the stream. */
lb_status lb_batch_lengths(lb_batch *b, double *out);

/* Run to each of nsamples step counts at[k] (counted from now, non-decreasing)
 * and record the four reductions of every lattice there: out[(i*nsamples + k)*4
 * + j].  The whole sequence (persistent launches and reductions) is captured
 * as one CUDA graph and launched once.  Waits for the stream. */
lb_status lb_batch_run_sampled(lb_batch *b, int nsamples, const long *at, double *out);

/* Populations of lattice i, as lb_get_populations (LB_ERR_ARG for
 * LB_STORAGE_MOMENTS), and its six moments, as lb_get_moments. */
lb_status lb_batch_populations(lb_batch *b, int i, double *f, double *g, int rested);
lb_status lb_batch_moments(lb_batch *b, int i, double *m);

/* Tile of the persistent kernel (tile_x = 64, 128, 256 consumer threads along
 * x, tile_y rows), and a tuner that times every candidate (body, ring depth and
 * tile) on the batch itself for 2*steps steps each (this advances the state). */
lb_status lb_batch_set_tile(lb_batch *b, int tile_x, int tile_y);
lb_status lb_batch_autotune(lb_batch *b, int steps, int *tile_x, int *tile_y, double *ms_per_step);

/* Checkpoints of the whole batch, as lb_save_state / lb_load_state: every
 * lattice's state in the batch's own arena layout (lattices one after the
 * other, offsets padded to 64 elements), for a batch created with the same
 * lattices and storage.  lb_batch_load_state does not clear a timed-out batch. */
size_t lb_batch_state_bytes(const lb_batch *b);
lb_status lb_batch_save_state(lb_batch *b, void *host, size_t bytes);
lb_status lb_batch_load_state(lb_batch *b, const void *host, size_t bytes, long time);

/* Body of the persistent kernel, as lb_set_kernel: 0 = automatic (staged when
 * the staged kernel fits every lattice, else sliding-window), 1 = sliding-window
 * body, 2 / 3 = staged body with its shallow / deep ring (bulk copies into a
 * shared-memory ring that runs on across tiles and steps; every lattice with
 * nx % 8 == 0 and nx * ny <= 477218588, else LB_ERR_ARG).  All give the same result bit for bit.  A batch in
 * LB_STORAGE_MOMENTS has one body (4), the single-lattice moment kernel's
 * strips.  get returns the body in use (1, 2, 3 or 4). */
lb_status lb_batch_set_kernel(lb_batch *b, int variant);
lb_status lb_batch_get_kernel(const lb_batch *b, int *variant);

/* Grid-barrier settings: the wait limit in seconds (default 2) and a number of
 * arrivals that never come.  A nonzero absent_blocks makes every barrier wait
 * run out (failure injection on the host, for tests): the kernel returns, the
 * state is unreliable and the next waiting call returns LB_ERR_TIMEOUT.  The
 * staged body's shared-memory waits use a fixed 2 s limit. */
lb_status lb_batch_set_barrier(lb_batch *b, unsigned int absent_blocks, double limit_seconds);

/* As lb_check_report, for the persistent batch kernels (every batch in the
 * process). */
lb_status lb_batch_check_report(lb_batch *b, int *enabled, unsigned long long *bad,
                                unsigned long long *first_bad);

long lb_batch_time(const lb_batch *b);
/* Fluid nodes of lattice i, or of the whole batch for i < 0. */
long lb_batch_fluid_nodes(const lb_batch *b, int i);
const char *lb_batch_last_error(const lb_batch *b);

/* ------------------------------------------------------------------------
 * Allocation-free reductions.  The paper has no counterpart: this entry point
 * exists for callers of this library that cannot allocate device memory --
 * for example a host framework that owns every device buffer through its own
 * fixed pool, or a loop that must not take the implicit synchronisation and the
 * possible failure of cudaMalloc/cudaFree while it runs.  It computes the same
 * four values as lb_filled_length from a state the caller holds, without a
 * context, and calls no allocator (neither cudaMalloc/cudaFree nor any library
 * routine that allocates).
 *
 * Inputs: grid, walls and params describe the lattice exactly as for lb_create
 * (only the geometry, model, storage, rho_l and rho_g are used).  f, g and g0
 * are device pointers to a state in the library's layout for params->storage:
 * plane-major (9, ny, nx) arrays of double (LB_STORAGE_F64) or float
 * (LB_STORAGE_F32); for LB_STORAGE_F16DEV, f holds 9 FP16 planes of
 * f_i - w_i (w_i the rest weights of params->A, as for LB_STORAGE_F16DEV
 * above), g holds 8 FP16 planes g_1..g_8 and g0 one
 * FP32 plane of g_0; for the block storages (LB_STORAGE_F32_BLOCKED,
 * LB_STORAGE_F16_BLOCKED) f holds the whole state in that storage's block
 * layout (the bytes lb_save_state writes), at least 4-byte aligned, and g and g0
 * are ignored.  g is ignored for the liquid-gas model, g0 unless the storage is
 * LB_STORAGE_F16DEV.  out is a device pointer to 4 doubles that
 * receives {l_centre, l_vol, mass, phi_sum} (definitions as in
 * lb_filled_length).  nblocks is the number of blocks of the first reduction
 * pass, each of which leaves one partial sum in the scratch.
 *
 * Scratch: a file-scope device array of LB_NOALLOC_MAX_BLOCKS x 4 doubles
 * (64 KiB) that every GPU which loads the library holds until the process
 * exits.  nblocks outside [1, LB_NOALLOC_MAX_BLOCKS] is rejected with
 * LB_ERR_ARG.  Every call shares that array and it keeps the last call's
 * contents; each call writes every slot it later reads, so nothing has to be
 * cleared between calls.  Calls whose kernels overlap on the GPU (issued on
 * different streams or from different host threads without ordering) race on
 * the scratch and may return wrong values: issue them in order on one stream.
 *
 * The first call in a CUDA context looks up the scratch array's device address
 * in that context (cudaGetSymbolAddress on the current device) and keeps it,
 * keyed by the device and the context's unique ID, for later calls; make that
 * first call before any stream capture begins.  A call made in another
 * context of the same device (after cudaDeviceReset, or under a context the
 * caller made current through the driver API) sees a different ID and looks
 * the address up again, so the same rule applies to its first call there.
 *
 * Asynchronous on stream (a cudaStream_t or NULL); out is valid once the stream
 * reaches the call.  No NaN check is made (there is no context to poison):
 * inspect mass and phi_sum.  Returns LB_ERR_ARG for a NULL required pointer, an
 * invalid geometry, model or storage, nblocks out of range, or (liquid-gas
 * model) densities that are not finite with rho_l > rho_g, and LB_ERR_CUDA if
 * the device or context query, the address lookup or a kernel launch fails.
 * ------------------------------------------------------------------------ */
#define LB_NOALLOC_MAX_BLOCKS 2048

lb_status lb_filled_length_noalloc(const lb_grid *grid, const lb_walls *walls, const lb_params *params,
                                   const void *f, const void *g, const void *g0, int nblocks,
                                   double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LB_GB300_H */
