/*
 * lbm.h - C ABI of the GB300 (sm_103a) LBM-LES channel solver with the
 * wall-function bounce (WFB) boundary of Han, Ooka & Kikumoto,
 * "A wall function approach in lattice Boltzmann method: algorithm and
 * validation using turbulent channel flow" (arXiv 2009.04352).
 *
 * One call of lbm_step advances the lattice Boltzmann equation (Eq. 1) by one
 * time step per iteration: a single fused CUDA kernel gathers the 19 D3Q19
 * populations of every cell (streaming, Eq. 1 left side), forms the moments
 * (Eq. 2), relaxes them with BGK plus a standard Smagorinsky eddy viscosity
 * (Sec. 3.1) and the Guo body force F_a (Eq. 1 right side), and at the two wall
 * layers applies bounce-back or the WFB reassignment (Eqs. 14-15) with the wall
 * stress from Spalding's law (Eqs. 16-17) solved by Newton's method (Sec. 2.3).
 *
 * Conventions shared by every entry point:
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3, reference density 1.
 *  - Grid nx * ny * nz: x streamwise and periodic, y wall-normal, z spanwise
 *    and periodic (the channel of Sec. 3.1, Fig. 3). All ny layers are fluid;
 *    the walls lie half a link outside them (y = -1/2 and y = ny - 1/2).
 *  - D3Q19 velocities are numbered as in Table A-1 (Appendix A).
 *  - Dense cell arrays are [nz][ny][nx] with x fastest; population arrays are
 *    [19][nz][ny][nx]; wall arrays are [2 walls: bottom, top][nz][nx][2: x, z].
 *  - Every call is ordered on the handle's CUDA stream. Calls that write to
 *    host memory synchronise that stream before returning; calls that write to
 *    device memory do not.
 *  - Return value: LBM_OK (0) or a negative LBM_ERR_* code. Nothing throws
 *    across the ABI. lbm_last_error() returns a message for the most recent
 *    failure on the calling thread.
 *  - Ownership: the library owns every device buffer it allocates and frees
 *    them in lbm_destroy. Pointers passed in stay owned by the caller and are
 *    not retained after the call returns.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_Q 19
#define LBM_K_STATS 11   /* plane statistics per layer, see lbm_plane_stats */
#define LBM_K_WALL 4     /* wall statistics per wall, see lbm_plane_stats */

enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,       /* invalid argument; nothing was changed */
    LBM_ERR_CUDA = -2,      /* a CUDA runtime call failed */
    LBM_ERR_OOM = -3,       /* device allocation failed */
    LBM_ERR_DIVERGED = -4,  /* a conservation check found NaN/Inf */
    LBM_ERR_STATE = -5      /* call not valid in the handle's current state */
};

typedef struct { int nx, ny, nz; } lbm_grid;

/* Wall treatment of the two walls y = const.
 *   BB, WFB, FREESLIP: halfway walls at y = -1/2 and y = ny - 1/2, every layer
 *     is fluid (half height D = ny / 2); the WFB correction rides on the
 *     reflected populations of the first layer.
 *   WFB_NODE: the full-way form of the WFB with wall nodes (the geometry of
 *     Eq. 14 and Table 1): layers 0 and ny - 1 are wall nodes, the fluid is
 *     layers 1 .. ny - 2 (D = (ny - 1) / 2). A wall node does not collide; it
 *     takes tau_w from the wall function at the first fluid node (y1 = its
 *     distance, 1 in lattice units), sends back into the fluid the specular
 *     partners of the populations that arrived from it plus (tau_w . e) / 2
 *     (Eqs. 13, 14a,b), and reverses all others. Needs ny >= 3, the two-lattice
 *     layout and the CELL or PAIR kernel (AUTO picks PAIR for even nx); the
 *     moments and statistics of layers 0 and ny - 1 are those of the wall
 *     nodes' own populations. */
typedef enum {
    LBM_WALL_BB = 0,        /* halfway bounce-back: the no-slip reference (Sec. 2.1, Eq. 3) */
    LBM_WALL_WFB = 1,       /* wall-function bounce (Sec. 2.2, Eqs. 14-15) */
    LBM_WALL_FREESLIP = 2,  /* specular reflection (Sec. 2.1, Eq. 4); WFB with tau_w = 0 */
    LBM_WALL_WFB_NODE = 3   /* wall-function bounce on wall nodes (full-way form) */
} lbm_wall_kind;

/* Wall function that gives tau_w to the WFB layer. Sec. 2.3 uses Spalding's
 * law; the WFB frame takes any law that returns tau_w, and the introduction
 * names the logarithmic law and the two-layer power law of Werner and Wengle.
 * Each is solved for u+ from R = y+ u+ = y1 |u_t| / nu (Eq. 17):
 *   SPALDING  y+ = u+ + e^{-kappa B} (e^{kappa u+} - 1 - kappa u+ - (kappa u+)^2/2
 *             - (kappa u+)^3/6) (Eq. 16), Newton;
 *   LOG       u+ = y+ below the crossing y_c of y+ and ln(y+)/kappa + B,
 *             u+ = ln(y+)/kappa + B above it, Newton on the log branch;
 *   POWER     u+ = y+ below 8.3^(7/6) (11.81), u+ = 8.3 (y+)^(1/7) above it,
 *             explicit: u+ = 8.3^(7/8) R^(1/8). */
typedef enum {
    LBM_LAW_SPALDING = 0,
    LBM_LAW_LOG = 1,
    LBM_LAW_POWER = 2
} lbm_wall_law;

/* Wall model of the WFB boundary (Sec. 2.3). kappa and B are the constants of
 * Spalding's law (Eq. 16; the paper uses 0.41 and 5.5) and of the log law. y1
 * is the wall distance entering y+ = y1 u_tau / nu (Eq. 17); 1.0 reproduces
 * the first-layer y+ printed in Table 1. nu is the molecular viscosity used by
 * the wall law; a value <= 0 selects (tau - 1/2) / 3. newton_iters caps the
 * Newton iterations per wall cell and step (<= 0 selects 12); each cell keeps
 * its value from its first relative step below 1e-7 on (the result does not
 * depend on the kernel form). law is an
 * lbm_wall_law (0, the zero-initialised default, is Spalding's law); another
 * value, or a log law whose two branches never cross (B <= (1 + ln kappa) /
 * kappa), makes lbm_create / lbm_batch_create fail with LBM_ERR_ARG. */
typedef struct {
    int kind;            /* lbm_wall_kind */
    double kappa;
    double B;
    double y1;
    double nu;
    int newton_iters;
    int law;             /* lbm_wall_law */
} lbm_wall_model;

typedef enum {
    LBM_FP32 = 0,          /* populations stored as FP32 deviations f_a - w_a */
    LBM_FP16_SHIFTED = 1   /* populations stored as FP16 deviations f_a - w_a */
} lbm_precision;

/* Storage layout of the populations (both move 19 reads + 19 writes per cell
 * and step and give bitwise the same results; the paper fixes neither).
 *   PULL2  two lattices: each step gathers from the neighbours of one array
 *          and writes the own cell of the other.
 *   AA     one lattice updated in place (the AA pattern of Bailey et al.
 *          2009): steps alternate between reading and rewriting the own
 *          cell's slots and gathering from the neighbours / pushing to them,
 *          which halves the population memory. Runs the CELL, PAIR and QUAD
 *          kernel forms; selecting TMA fails with LBM_ERR_ARG. Not available
 *          for batches. */
typedef enum {
    LBM_PULL2 = 0,
    LBM_AA = 1
} lbm_layout;

/* Form of the fused step kernel (all compute the same update).
 *   CELL: one thread per cell, any grid.
 *   PAIR: two cells per thread, 2-wide loads and packed FP32 math; even nx.
 *   TMA:  two cells per thread; each CTA streams whole source rows into a
 *         shared-memory ring with bulk asynchronous copies (full/empty
 *         mbarriers, 2-4 stages); nx a multiple of 64 whose rows fit the ring.
 *   QUAD: four cells per thread, 8-byte loads and stores; FP16 storage and nx a
 *         multiple of 4. With the two-lattice layout and BGK (or wall nodes)
 *         a step is two launches, the interior rows and then the two wall
 *         rows, the latter with the two-cell tile (the same bits); with MRT
 *         and halfway walls one launch whose wall rows call a separately
 *         compiled four-cell wall tile.
 *   AUTO: QUAD where allowed, else PAIR for even nx, else CELL. */
typedef enum {
    LBM_KERNEL_AUTO = 0,
    LBM_KERNEL_CELL = 1,
    LBM_KERNEL_PAIR = 2,
    LBM_KERNEL_TMA = 3,
    LBM_KERNEL_QUAD = 4
} lbm_kernel;

typedef struct lbm_handle lbm_handle;

/* Create a lattice at rest (f_a = w_a, rho = 1, u = 0).
 *   g          grid; nx >= 1, ny >= 2, nz >= 1, nx * ny * nz <= 2^31 - 1 cells.
 *   tau        BGK relaxation time tau0 > 1/2 (molecular viscosity (tau0 - 1/2)/3).
 *   C_s        Smagorinsky constant (>= 0; 0 turns the LES model off).
 *   force      body force per unit volume (F_x, F_y, F_z), host pointer.
 *   wm         wall model of both walls.
 *   precision  lbm_precision.
 *   layout     lbm_layout.
 *   cuda_stream  cudaStream_t to order all work on; NULL selects the legacy
 *              default stream.
 *   out        receives the handle.
 * Allocates 2 * 19 * cells populations (PULL2) or 19 * cells (AA), plus small
 * wall and statistics buffers, on the current device. Errors: LBM_ERR_ARG,
 * LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_create(lbm_grid g, double tau, double C_s, const double force[3],
               lbm_wall_model wm, int precision, int layout, void *cuda_stream,
               lbm_handle **out);

/* Bytes of one population lattice of grid g stored at `precision`: 19 planes of
 * ny * nz rows, each row padded to a multiple of 32 cells. 0 for an invalid
 * grid or precision. Host arithmetic only. (No counterpart in the paper: the
 * storage is this library's.) */
size_t lbm_population_bytes(lbm_grid g, int precision);

/* lbm_create on population arrays the caller owns, for example tensors of a
 * framework's caching allocator, so that the big arrays come out of the
 * caller's memory pool. pop0 (and pop1 for LBM_PULL2; NULL for LBM_AA) are
 * device pointers on the current device, at least 16-byte aligned, each of
 * lbm_population_bytes(g, precision) bytes. The handle reads and writes them
 * on its stream until lbm_destroy, which does not free them; the caller keeps
 * them alive until then and does not touch them while steps are in flight.
 * Their contents are undefined until lbm_init_channel or lbm_set_populations.
 * The library still allocates its small wall, statistics and partial-sum
 * buffers. Other arguments and errors as lbm_create; a NULL pop0, a wrong
 * pop1 for the layout or a misaligned pointer give LBM_ERR_ARG. */
int lbm_create_from_buffers(lbm_grid g, double tau, double C_s, const double force[3],
                            lbm_wall_model wm, int precision, int layout, void *cuda_stream,
                            void *pop0, void *pop1, lbm_handle **out);

/* Seeded channel initial field: f = f^eq(rho = 1, u0) (second-order D3Q19
 * equilibrium) with u0_x = u_mean_x[y] + a (2 U_0 - 1), u0_y = a (2 U_1 - 1),
 * u0_z = a (2 U_2 - 1), a = noise_amp, and U_c the uniform [0,1) variate
 * (top 53 bits x 2^-53) of the first SplitMix64 output for state
 * seed XOR (3 * cell + c), cell = (z * ny + y) * nx + x.
 *   u_mean_x  host array [ny]. Resets the step counter to 0. */
int lbm_init_channel(lbm_handle *h, const double *u_mean_x, double noise_amp, uint64_t seed);

/* Replace the populations by host_in (FP64, [19][nz][ny][nx], not shifted).
 * Rounded once to the storage precision. Resets the step counter to 0. */
int lbm_set_populations(lbm_handle *h, const double *host_in);

/* Copy the current populations f_a(x, t) to host_out (FP64, [19][nz][ny][nx],
 * not shifted). Synchronises the stream. */
int lbm_populations(lbm_handle *h, double *host_out);

/* Sample plane statistics at every step whose index t (before the step) is a
 * multiple of `every` (0 = never). Sampling is fused into that step's kernel. */
int lbm_set_stats_every(lbm_handle *h, int every);

/* Advance n >= 0 time steps (Eq. 1 with the wall treatment of Eqs. 14-17).
 * Asynchronous on the handle's stream; steps without sampling are replayed
 * from CUDA graphs of 16 steps. The first call with n > 0 after lbm_create,
 * lbm_set_kernel, lbm_set_les or lbm_set_wait_limit captures, instantiates and
 * uploads both of those graphs (one per start phase), whatever n is, so a
 * short warm-up call leaves nothing to build inside a later timed run; make
 * that first call outside any stream capture of the caller's own. */
int lbm_step(lbm_handle *h, int n);

/* Number of steps taken since the last (re)initialisation. */
long long lbm_get_step(lbm_handle *h);

/* Choose the step kernel form (lbm_kernel). Synchronises the stream; returns
 * LBM_ERR_ARG if the grid does not allow the form. lbm_create selects AUTO.
 * The populations and statistics are kept; only the launch changes. */
int lbm_set_kernel(lbm_handle *h, int kernel);

/* The kernel form in use (never LBM_KERNEL_AUTO), -1 for a NULL handle. */
int lbm_get_kernel(lbm_handle *h);

/* Tile-shape autotuner of a single channel (no counterpart in the paper): time
 * every kernel form the grid allows (CELL, PAIR, TMA, QUAD: one, two or four
 * cells per thread, or the row-pipelined CTA) for `steps` >= 1 steps each,
 * after 2 warm-up steps and its graph build, with CUDA events on the handle's
 * stream, and keep the fastest. best_ms and best_kernel (nullable) receive its
 * time per step and its lbm_kernel value. The timed steps advance the state
 * like lbm_step (all forms compute the same update), so the step count grows
 * by (steps + 2) per form tried. Synchronises. Errors: LBM_ERR_ARG (NULL
 * handle, steps < 1), LBM_ERR_STATE (batch member), LBM_ERR_CUDA. */
int lbm_autotune(lbm_handle *h, int steps, double *best_ms, int *best_kernel);

typedef enum {
    LBM_COLLISION_BGK = 0,  /* single relaxation time (default) */
    LBM_COLLISION_MRT = 1   /* D3Q19 multiple relaxation times (ref. [40] of Sec. 3.1) */
} lbm_collision;

/* LES model (Sec. 3.1). collision: BGK, or the D3Q19 MRT of d'Humieres et al.
 * (2002) (moments rho, e, eps, j, q, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz,
 * p_xz, m; rates s_e = 1.19, s_eps = 1.4, s_q = 1.99, s_m = 1.98, and the
 * five stress moments 3p_xx, p_ww, p_xy, p_yz, p_xz with the two pi moments
 * 3pi_xx, pi_ww at 1/tau_eff (d'Humieres' s_q = 1.2 and s_pi = 1.4 make the
 * scheme linearly unstable at the tau0 of the channels, tau0 - 1/2 ~ 1e-4);
 * equilibrium moments M f^eq; Guo forcing in moment space).
 * Both use the Smagorinsky tau_eff. u_tau_ref > 0 and a_plus > 0 add van Driest
 * damping of the Smagorinsky length, C_s (1 - exp(-y+/A+)), with y the layer
 * centre's distance to the nearer wall (j + 1/2) and y+ = y u_tau_ref / nu (nu
 * of the wall model); both 0 turn it off. Synchronises; keeps the state. */
int lbm_set_les(lbm_handle *h, int collision, double u_tau_ref, double a_plus);

/* Density rho [nz][ny][nx] and velocity u [3][nz][ny][nx] of the current
 * populations (Eq. 2 with the Guo half-force shift, u = (sum e f + F/2)/rho),
 * FP32. on_device != 0: rho and u are device pointers and the call is
 * asynchronous; otherwise host pointers and the stream is synchronised.
 * Either pointer may be NULL. */
int lbm_moments(lbm_handle *h, float *rho, float *u, int on_device);

/* Wall stress of the most recent step, [2][nz][nx][2] FP32: the tangential
 * momentum (x, z) the wall treatment added to each wall cell in that step.
 * For WFB this is (tau_w,x, tau_w,z) of Eq. 15 (dt = dy = 1); for bounce-back
 * the momentum exchanged by the reflection; zero for free-slip. */
int lbm_wall_stress(lbm_handle *h, float *tau, int on_device);

/* Accumulated plane statistics (FP64), summed over the cells of each layer and
 * over the sampled steps (time and plane averaging of Sec. 3.1):
 *   out [ny][LBM_K_STATS] = rho, u_x, u_y, u_z, u_x^2, u_y^2, u_z^2, u_x u_y,
 *                           rho u_x, rho u_y, rho u_z  (u as in lbm_moments)
 *   wall_out [2][LBM_K_WALL] = sum of tau_w,x, tau_w,z, |tau_w|, |tau_w|^2
 *   n_samples = number of sampled steps.
 * Host pointers (each may be NULL); synchronises. reset != 0 clears the sums. */
int lbm_plane_stats(lbm_handle *h, double *out, double *wall_out, long long *n_samples,
                    int reset);

/* Global mass and raw momentum of the current populations, out[4] =
 * (sum f, sum e_x f, sum e_y f, sum e_z f), reduced in FP64 (host pointer;
 * synchronises). Returns LBM_ERR_DIVERGED if any sum is NaN or Inf. */
int lbm_conservation(lbm_handle *h, double *out);

/* Instantaneous plane sums of the current populations, written without any
 * device allocation. The paper has no counterpart: this is a library service
 * for callers that must not allocate device memory when they take the
 * measurement, e.g. code running under a fixed memory budget or a pool that
 * must not grow, or a host loop that has to avoid allocation calls because
 * they can synchronise the device.
 *   out_dev  caller-owned DEVICE array [ny][LBM_K_STATS] receiving, for each
 *            layer, the sums over its cells of rho, u_x, u_y, u_z, u_x^2,
 *            u_y^2, u_z^2, u_x u_y, rho u_x, rho u_y, rho u_z (the columns of
 *            lbm_plane_stats, for the current state only, nothing accumulated).
 * Asynchronous on the handle's stream. The block partial sums live in one
 * fixed array of 1.44 MB that the library keeps in device memory on every GPU
 * that loads it, until the process exits; it holds at most ny = 2048 layers,
 * and larger grids are rejected with LBM_ERR_ARG. The array used is the one of
 * the CURRENT device, so the handle's device must be current when calling. The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current, so make the first call
 * before any stream capture. Every call overwrites the part of the array it
 * uses, so nothing needs clearing between calls; calls whose work overlaps on
 * the GPU (other streams or handles) race on the shared array and must be
 * ordered by the caller. */
int lbm_plane_profile_noalloc(lbm_handle *h, double *out_dev);

/* ---------------------------------------------------------------------------
 * Batched ensemble: independent channels of uneven sizes and parameters
 * advanced together by one persistent kernel launch per time step (plain
 * steps replayed from a CUDA graph). Each member is the channel lbm_create
 * would build from the same arguments; its populations live in one pool owned
 * by the batch.
 * ------------------------------------------------------------------------- */

typedef struct {
    lbm_grid grid;          /* nx even and >= 2 */
    double tau;
    double C_s;
    double force[3];
    lbm_wall_model wall;
} lbm_member;

typedef struct lbm_batch lbm_batch;

/* Create n >= 1 members (at rest) in one population pool on the current
 * device, all with the given storage precision, ordered on cuda_stream.
 * Errors: LBM_ERR_ARG (a member's grid or parameters), LBM_ERR_OOM. */
int lbm_batch_create(int n, const lbm_member *members, int precision, void *cuda_stream, lbm_batch **out);

/* Member i as an lbm_handle view (NULL if out of range). Every call of the
 * single-channel API that does not advance time works on it (initial field,
 * populations in/out, moments, wall stress, plane statistics, conservation);
 * lbm_step and lbm_set_kernel return LBM_ERR_STATE, lbm_destroy ignores it.
 * The view stays valid until lbm_batch_destroy. */
lbm_handle *lbm_batch_member(lbm_batch *b, int i);

/* Total cells of all members. */
long long lbm_batch_cells(lbm_batch *b);

/* Plane statistics of every member at steps whose index is a multiple of
 * `every` (0 = never), accumulated in each member's lbm_plane_stats. */
int lbm_batch_set_stats_every(lbm_batch *b, int every);

/* Advance every member by n steps. Asynchronous. */
int lbm_batch_step(lbm_batch *b, int n);

/* Form of the batch step (no counterpart in the paper; both give every member
 * bitwise the populations of the same channel run alone with the kernel named
 * below):
 *   PERSISTENT     one launch of the persistent batch kernel per step over the
 *                  work list of all members' two-cell tiles (any even nx; the
 *                  members run the PAIR kernel's arithmetic).
 *   MEMBER_GRIDS   every member runs the single-channel step kernels its grid
 *                  selects (AUTO: QUAD for FP16 storage and nx a multiple of
 *                  4, else PAIR), its members spread over `streams` capture
 *                  streams (1 .. 32; 0 selects 8) balanced by cell count, and
 *                  each 16-step chunk of all members captured as one CUDA
 *                  graph, so that the members' grids run concurrently.
 * lbm_batch_create selects MEMBER_GRIDS (8 streams); the autotuner searches
 * both. */
typedef enum {
    LBM_BATCH_PERSISTENT = 1,
    LBM_BATCH_MEMBER_GRIDS = 2
} lbm_batch_form;

/* Select the form (and, for MEMBER_GRIDS, the number of capture streams).
 * Synchronises; the state is kept. LBM_ERR_ARG for an unknown form or a
 * stream count outside 0 .. 32. */
int lbm_batch_set_form(lbm_batch *b, int form, int streams);

/* The form in use (-1 for a NULL batch); *streams (nullable) receives the
 * capture streams of the member-grid form. */
int lbm_batch_get_form(lbm_batch *b, int *streams);

/* Launch shape of the persistent form: threads per CTA (64 or 128; a tile is
 * 2 * threads cells of one row) and CTAs per SM (<= 0 or above the occupancy
 * limit selects the limit). */
int lbm_batch_set_config(lbm_batch *b, int threads, int ctas_per_sm);
int lbm_batch_get_config(lbm_batch *b, int *threads, int *ctas_per_sm, int *grid, long long *tiles);

/* Time every form (lbm_batch_set_form) with its launch shapes (threads per
 * CTA x CTAs per SM; 4, 8 or 16 streams) for `steps` steps each (after 2
 * warm-up steps) and keep the fastest; best_ms (nullable) receives its time
 * per step. The timed steps advance all members like lbm_batch_step, so tune
 * before initialising the members. Synchronises. */
int lbm_batch_autotune(lbm_batch *b, int steps, double *best_ms);

/* Block until the batch's work has finished. */
int lbm_batch_sync(lbm_batch *b);

/* Free the batch, its pool and its member views. NULL is ignored. */
void lbm_batch_destroy(lbm_batch *b);

/* Block until all work queued on the handle's stream has finished. Returns
 * LBM_ERR_CUDA if a wait inside the pipelined kernel timed out (the kernel then
 * stops early and leaves the step incomplete, so the populations are no longer
 * a valid state). A timeout is reported once: the call clears the device flag
 * after reading it, so the next call succeeds unless another wait timed out. */
int lbm_sync(lbm_handle *h);

/* Clock cycles each shared-memory pipeline wait of the pipelined (TMA) kernel
 * may take before it gives up and sets the error flag that lbm_sync reports
 * (failure detection, no counterpart in the paper). cycles <= 0 restores the
 * default of 2^32 (about 2 s at 2 GHz). Whatever the limit, a CTA that gives
 * up first waits, for at most the default, until the copies it has issued have
 * landed, so that none arrives after it has exited. Other kernel forms have
 * no waits. Synchronises the stream and drops the captured step graphs. */
int lbm_set_wait_limit(lbm_handle *h, long long cycles);

/* Free every device resource of the handle. NULL is ignored. */
void lbm_destroy(lbm_handle *h);

/* Message of the last failed call on this thread ("" if none). */
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
