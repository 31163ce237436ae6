/*
 * lbm_pf.h -- C ABI of the GB300 (sm_103a) phase-field lattice Boltzmann
 * library: the per-time-step lattice update of the two-distribution model of
 * Liang, Xu, Chen, Wang, Chai & Shi, "Phase-field-based lattice Boltzmann
 * modeling of large-density-ratio two-phase flows" (arXiv:1710.09541, 2018),
 * Sec. II, on a D2Q9 grid.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid: nx * ny nodes, node (x, y) at linear index y*nx + x (x fastest).
 *    Lattice units: dx = dt = 1, c_s^2 = 1/3 (Eq. 10).
 *  - x is always periodic.  y is periodic (bc_y = LBM_BC_PERIODIC), closed
 *    by half-way bounce-back walls at y = -1/2 and y = ny - 1/2
 *    (LBM_BC_WALLS; Sec. III B), or closed by the bottom wall only with an
 *    open top (LBM_BC_WALL_OPEN; the impact case of Sec. III D, whose "open
 *    boundary" the paper does not define).  The open top is read as a
 *    zero-gradient outflow: populations leaving through it are lost, the top
 *    row's incoming populations (c_y = -1) take the values of the row below,
 *    and the phi stencil's ghost row repeats the top row.  It needs ny >= 2,
 *    and the rule also holds for the initial state and for a restored one
 *    (the top row's c_y = -1 populations of a state passed to lbm_set_state
 *    are replaced by the row below's).
 *  - Host arrays passed in or out are double precision, N = nx*ny entries,
 *    owned by the caller; the library copies them and keeps no pointer.
 *  - All device memory is owned by the handle: allocated by lbm_create
 *    (stream-ordered, cudaMallocAsync on params.stream), released by
 *    lbm_destroy (cudaFreeAsync, then a synchronisation of that stream);
 *    lbm_create_in places it in a caller's buffer instead.  All GPU work is
 *    enqueued on params.stream (NULL = the legacy default stream).
 *  - Every call returns an lbm_status; nothing aborts, traps or exits.  After
 *    a failure lbm_last_error(h) returns a one-line description.
 *  - A handle is not thread-safe: one host thread per handle.
 *  - Arithmetic on the device is FP32 (no fast-math): every addition,
 *    multiplication and fused multiply-add is an explicit IEEE
 *    round-to-nearest operation.  The step has no division or square root;
 *    its five reciprocals, 1/rho (Eq. 22a), 1/tau_g (Eq. 23), the 1/nu
 *    inversion of Eq. 25, 1/|grad phi| (Eq. 2) and 1/|C| (Eq. 29), use the
 *    hardware approximations rcp.approx / rsqrt.approx (relative error below
 *    2^-22, deterministic).  Diagnostics that sum over the grid accumulate in
 *    FP64.
 */
#ifndef LBM_PF_H
#define LBM_PF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_handle lbm_handle;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID = -1,   /* bad argument or parameter set */
    LBM_ERR_CUDA = -2,      /* a CUDA runtime call failed (message kept) */
    LBM_ERR_STATE = -3,     /* step/get called before lbm_init */
    LBM_ERR_NONFINITE = -4, /* a NaN/Inf appeared in phi, u or p */
    LBM_ERR_OOM = -5        /* device or host allocation failed */
} lbm_status;

/* viscosity rule across the interface (visc_mode) */
enum {
    LBM_VISC_LINEAR_NU = 0,  /* nu = phi (nu_l - nu_g) + nu_g            Eq. 24 */
    LBM_VISC_INVERSE_NU = 1, /* 1/nu = phi (1/nu_l - 1/nu_g) + 1/nu_g     Eq. 25 */
    LBM_VISC_STEP_MU = 2     /* mu = rho_l nu_l if phi >= 1/2 else rho_g nu_g,
                                nu = mu / rho(phi)                        Eq. 26 */
};
enum { LBM_BC_PERIODIC = 0, LBM_BC_WALLS = 1, LBM_BC_WALL_OPEN = 2 };
/* unit normal n of the sharpening term (normal_scheme) */
enum {
    LBM_NORMAL_CENTRAL = 0, /* n = grad phi / |grad phi|, grad by Eq. 27  (Eq. 2) */
    LBM_NORMAL_LOCAL = 1    /* n from the non-equilibrium of f_i           (Eq. 29) */
};
/* population storage in HBM (storage); arithmetic is FP32 in every format */
enum {
    LBM_STORE_FP32 = 0,         /* f, g: 9 FP32 planes each (72 B/node) */
    LBM_STORE_FP16_SHIFTED = 1, /* f_0 FP32 (takes the rounding of the others, so sum phi is
                                   conserved); f_1..8 FP16 of f_i/w_i - 1/2; g FP16 of
                                   2^10 g_i/w_i (38 B/node) */
    LBM_STORE_BF16_SHIFTED = 2, /* as FP16_SHIFTED with BF16 and g unscaled */
    LBM_STORE_BF16_SHIFTED_SR = 3 /* the BF16_SHIFTED layout; each step rounds the nine g codes
                                   stochastically (up with probability equal to the discarded
                                   fraction, so the stored code is right on average), which keeps
                                   the slow viscous change of g that rounding to nearest stalls
                                   at large tau_g.  The dithers come from a counter-based hash of
                                   the node index and the handle's step count since lbm_init:
                                   runs are reproducible, and a checkpoint restored into the
                                   handle that saved it (lbm_set_state keeps the count) resumes
                                   bit for bit; restored elsewhere it resumes with other dithers.
                                   Not available in batches (LBM_ERR_INVALID). */
};
/* step kernel (kernel) */
enum {
    LBM_KERNEL_AUTO = 0,    /* the library's choice: currently LBM_KERNEL_GENERIC */
    LBM_KERNEL_GENERIC = 1  /* tiles of 32 x 4 threads, direct loads, phi ring recomputed
                               in shared memory; one node per thread with FP32 storage,
                               two with 16-bit storage; any grid */
};

typedef struct {
    double rho_l, rho_g;  /* liquid / gas densities, Eq. 13; rho_g > 0 */
    double nu_l, nu_g;    /* kinematic viscosities of the pure phases, Eqs. 24-26; > 0 */
    int visc_mode;        /* LBM_VISC_* */
    double sigma;         /* surface tension; k = 3 sigma W / 2, beta = 12 sigma / W (Eq. 7); >= 0 */
    double W;             /* interface thickness, Eqs. 3 and 7; > 0 */
    double tau_h;         /* Allen-Cahn relaxation time (tau_f of Eq. 8); > 1/2;
                             mobility M = (tau_h - 1/2)/3 (Eq. 14) */
    double Gx, Gy;        /* body-force density G (Eqs. 4b, 19), same in both phases */
    int bc_y;             /* LBM_BC_PERIODIC, LBM_BC_WALLS or LBM_BC_WALL_OPEN */
    int normal_scheme;    /* LBM_NORMAL_* */
    int storage;          /* LBM_STORE_*: how populations are stored between steps */
    int check_every;      /* > 0: every check_every steps lbm_step synchronises the
                             stream and returns LBM_ERR_NONFINITE if any node produced
                             a non-finite phi, u or p since the last check; 0: off */
    void* stream;         /* cudaStream_t for all work; NULL = default stream */
    int kernel;           /* LBM_KERNEL_* */
} lbm_params;

/*
 * lbm_create -- validate the parameters and allocate the device state for an
 * nx x ny grid: two buffers of 9 FP32 planes for each of f_i (Allen-Cahn,
 * Eq. 8) and g_i (Navier-Stokes, Eq. 15), two FP32 planes holding (phi u) of
 * the previous step (for d_t(phi u) in Eq. 11), and staging for host I/O.
 * Requires nx >= 1, ny >= 1 (ny >= 2 with walls), nx*ny < 2^31, and the
 * parameter ranges listed in lbm_params.  On success *out owns everything.
 * Errors: LBM_ERR_INVALID, LBM_ERR_OOM, LBM_ERR_CUDA (then *out == NULL).
 */
lbm_status lbm_create(int nx, int ny, const lbm_params* p, lbm_handle** out);

/*
 * Handles whose device memory belongs to the caller (for example a PyTorch
 * tensor, so that the framework's caching allocator owns and accounts for
 * it).  The same state as lbm_create describes, laid out in one buffer.
 *
 * lbm_workspace_bytes -- validate the parameters as lbm_create does and write
 *   to *bytes the size of the device workspace an nx x ny handle needs.  Makes
 *   no CUDA call.  Errors: LBM_ERR_INVALID.
 * lbm_create_in -- create a handle whose device buffers are carved from
 *   d_workspace: device (or managed) memory of the current device, 256-byte
 *   aligned, at least lbm_workspace_bytes long.  The handle never frees it;
 *   the caller keeps it alive, and untouched by other work, until
 *   lbm_destroy.  Otherwise the handle behaves exactly as one from lbm_create.
 *   Errors: LBM_ERR_INVALID (bad parameters, NULL, too small, misaligned, or
 *   not device memory of the current device), LBM_ERR_CUDA.
 */
lbm_status lbm_workspace_bytes(int nx, int ny, const lbm_params* p, size_t* bytes);
lbm_status lbm_create_in(int nx, int ny, const lbm_params* p, void* d_workspace, size_t bytes,
                         lbm_handle** out);

/*
 * lbm_init -- set the state to equilibrium: f_i = f_i^eq(phi0, u0) (Eq. 9),
 * g_i = g_i^eq(p0, rho(phi0), u0) (Eqs. 13, 16, 17), and the previous-step
 * (phi u) to phi0 * u0.  phi0 is required; ux0, uy0, p0 may be NULL (= 0).
 * Host arrays of N doubles.  Enqueued on the stream; the host arrays may be
 * reused when the call returns (the copies are synchronous to the host).
 */
lbm_status lbm_init(lbm_handle* h, const double* phi0, const double* ux0,
                    const double* uy0, const double* p0);

/*
 * lbm_step -- advance nsteps >= 0 time steps.  One step is, per node: stream
 * f_i and g_i (pull; Eqs. 8, 15 left-hand sides) with periodic or half-way
 * bounce-back links; phi = sum f_i (Eq. 12); rho (Eq. 13); grad phi and
 * lap phi (Eqs. 27, 28); mu_phi (Eqs. 6, 7); F = mu_phi grad phi + G
 * (Eqs. 5, 19); u and p (Eq. 22); tau_g from nu (Eqs. 23-26); the Allen-Cahn
 * collision with source F_i (Eqs. 2, 3, 8, 9, 11; d_t(phi u) as the backward
 * difference over one step); the Navier-Stokes collision with forcing G_i
 * (Eqs. 15-17, 20).  Asynchronous on the stream unless check_every triggers
 * a check.  Errors: LBM_ERR_STATE (no init), LBM_ERR_NONFINITE, LBM_ERR_CUDA.
 */
lbm_status lbm_step(lbm_handle* h, int nsteps);

/*
 * lbm_get_fields -- phi, rho, ux, uy, p of the current state, computed by the
 * same formulas as the step (Eqs. 12, 13, 22).  Any output may be NULL.
 * Host arrays of N doubles; synchronises the stream before returning.
 */
lbm_status lbm_get_fields(lbm_handle* h, double* phi, double* rho, double* ux,
                          double* uy, double* p);

/*
 * lbm_state_bytes -- size of the checkpoint: 20 * N * sizeof(float).
 * lbm_get_state / lbm_set_state -- copy the complete state to / from a host
 * buffer of exactly that size, laid out as FP32 f[9][ny][nx], g[9][ny][nx]
 * (pre-collision populations of the current time, i.e. after streaming,
 * velocity index i in the order of Eq. 10), then (phi u_x, phi u_y) of the
 * previous step [2][ny][nx].  Restoring a saved state and stepping reproduces
 * the uninterrupted run bit for bit.  Both synchronise the stream.
 */
size_t lbm_state_bytes(const lbm_handle* h);
lbm_status lbm_get_state(lbm_handle* h, void* host_buf, size_t bytes);
lbm_status lbm_set_state(lbm_handle* h, const void* host_buf, size_t bytes);

/*
 * lbm_diag -- grid reductions of the current state: sum of phi (FP64
 * accumulation; conserved by the scheme, Eqs. 8-12), max |u|, min p, max p.
 * Any output may be NULL.  Synchronises the stream.
 */
lbm_status lbm_diag(lbm_handle* h, double* sum_phi, double* umax, double* pmin,
                    double* pmax);

/*
 * lbm_diag_fields_noalloc -- the reductions of lbm_diag (sum of phi in FP64,
 * max |u|, min p, max p) over fields the caller already holds on the device,
 * without allocating anything.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory at this point, such
 * as a process whose device memory belongs to its own pool or runtime (a
 * cudaMalloc behind its back breaks its accounting or fails), or a stepping
 * loop that must not synchronise the device (cudaMalloc/cudaFree can).
 *   d_fields  device array of 5*n doubles: planes phi, rho, ux, uy, p of n
 *             nodes each (the layout lbm_get_fields fills; rho is not read).
 *   n         node count, 0 <= n <= 16,777,216 (4096^2); larger n returns
 *             LBM_ERR_INVALID and explains the limit in err.
 *   d_out     device array of 4 doubles receiving sum phi, max |u|, min p,
 *             max p (for n = 0: 0, 0, +inf, -inf).
 *   stream    cudaStream_t to enqueue on (NULL = default stream); the call
 *             returns after enqueueing, d_out is ready when the stream is.
 *   err, err_len  optional host buffer for a one-line error message.
 * The block partials live in a fixed 128 KiB array inside the library image,
 * which every GPU that loads the library holds until the process exits.
 * Set-up: the first call on each device, and the first call after that
 * device was reset (cudaDeviceReset makes a new primary context), looks up
 * the array's device address with the device current and loads the call's
 * two kernels.  Under lazy module loading (the CUDA default) that set-up can
 * load the library's device code, which allocates device memory for it and
 * may synchronise: exactly what these callers avoid.  So make one warm-up
 * call (n = 0 and any 4-double d_out will do) during your own set-up, before
 * a memory pool takes over the device or a stream capture begins; later
 * calls allocate nothing.  All calls on a device share the array: calls
 * whose kernels overlap on the GPU (on different streams, or from different
 * threads) race and must be ordered by the caller.  The array keeps the
 * previous call's partials; each call rewrites every slot it reads, so
 * nothing needs clearing.  Errors: LBM_ERR_INVALID (NULL pointer, n too
 * large), LBM_ERR_CUDA (no device, a CUDA error already pending from earlier
 * work -- reported and left pending, nothing launched --, set-up or launch
 * failure).
 */
lbm_status lbm_diag_fields_noalloc(const double* d_fields, size_t n, double* d_out, void* stream,
                                   char* err, size_t err_len);

/*
 * Batched stepping of many independent cases: drops and impacts of uneven
 * grid sizes, Reynolds numbers and density ratios advanced together.  A batch
 * groups existing handles that share one device, one stream and one storage
 * format; it does not own them (create, init, read back, checkpoint and
 * destroy them as usual).  The paper runs one case at a time; batching is an
 * addition of this library.
 *
 * lbm_batch_create -- build the batch over ncases handles (1 <= ncases <= 200,
 *   each initialised, none repeated, each with at most 65535 x 32767 tiles of
 *   the smallest tile shape, none with LBM_STORE_BF16_SHIFTED_SR storage).  The batch owns a case table, device tile
 *   lists (8 bytes per tile per tile shape and class) and two private
 *   streams; handles must outlive the batch.
 *   Errors: LBM_ERR_INVALID, LBM_ERR_OOM, LBM_ERR_CUDA (then *out == NULL).
 * lbm_batch_step -- advance every case by nsteps time steps (the same update as
 *   lbm_step, Sec. II, bit for bit).  The cases form two classes, periodic in y
 *   and walled in y; each class has a kernel compiled for its boundary and its
 *   own stream, and one launch per step covers the tiles of all its cases.  The
 *   two classes share no data, so their launch chains run concurrently.  Steps
 *   run as replays of a CUDA graph of 32 steps per class.  The first call with
 *   nsteps >= 140 times five tile shapes (32x4, 32x8, 32x16, 64x2, 64x4 nodes)
 *   for each class on its own first 140 steps (per shape 4 warm-up steps and
 *   the faster of two windows of 12) and keeps the fastest.
 *   Ordered after earlier work on the cases' stream, and later work on that
 *   stream waits for it.  A case may also be stepped on its own between batch
 *   steps.  If any case was created with check_every > 0, the call ends by
 *   synchronising and returns LBM_ERR_NONFINITE (the first such case named by
 *   lbm_batch_last_error) when a case with check_every > 0 produced a
 *   non-finite phi, u or p during the call; all cases' flags are cleared.
 *   Otherwise the call is asynchronous.  If a CUDA call fails after work was
 *   enqueued (LBM_ERR_CUDA), the call orders the cases' stream after what was
 *   enqueued and marks the batch and every case as failed: the cases answer
 *   LBM_ERR_STATE until lbm_init or lbm_set_state restores them, and the
 *   batch answers LBM_ERR_STATE to every further step (build a new one).
 * lbm_batch_info -- for class cls (0: periodic cases, 1: walled cases): the
 *   number of cases, the tile shape in use, its measured microseconds per
 *   step (0 before tuning or for an empty class) and whether tuning ran; any
 *   output pointer may be NULL.  Errors: LBM_ERR_INVALID (NULL batch, cls not
 *   0 or 1).
 */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(int ncases, lbm_handle* const* cases, lbm_batch** out);
lbm_status lbm_batch_step(lbm_batch* b, int nsteps);
lbm_status lbm_batch_info(const lbm_batch* b, int cls, int* ncases, int* tile_tx, int* tile_ty,
                          double* us_per_step, int* tuned);
void lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/*
 * Impact-case tooling (Sec. III D).  Both read the current state on the device
 * with the step's own arithmetic, so their values equal lbm_get_fields' at
 * the same nodes bit for bit, and both block until the result is on the host.
 *
 * lbm_spreading_radius -- the spreading radius r of an impacting drop (the
 *   quantity of Fig. 8, r/D against t U/D): half the x-extent of the run of
 *   nodes with phi >= 1/2 that contains column xc on row y, counted in nodes
 *   (x_right - x_left + 1) / 2; 0 when phi(xc, y) < 1/2.  The run does not
 *   wrap around the periodic x edges.  The paper gives neither the row nor
 *   the rule; the row is the caller's (the tests use the row W above the film
 *   surface).  r_interp (may be NULL) places each end at the phi = 1/2
 *   crossing by linear interpolation between the run's end node and its gas
 *   neighbour (an end at the grid edge lies half a node beyond it).
 *   Errors: LBM_ERR_INVALID (NULL handle, (xc, y) outside the grid),
 *   LBM_ERR_STATE (before lbm_init), LBM_ERR_CUDA.
 * lbm_probe -- phi, rho, u and p (Eqs. 12, 13, 22) at npts nodes (x[j], y[j]),
 *   0 <= npts <= nx*ny, written to caller-owned host arrays of npts doubles
 *   (any output may be NULL).  A Laplace pressure jump or a velocity at a few
 *   nodes costs a few KB of traffic instead of a full read-back.
 *   Errors: LBM_ERR_INVALID (NULL handle or coordinates, npts out of range, a
 *   node outside the grid: nothing is written), LBM_ERR_STATE, LBM_ERR_CUDA.
 */
lbm_status lbm_spreading_radius(lbm_handle* h, int y, int xc, double* r, double* r_interp);

/*
 * lbm_laplace_jump -- the pressure jump of a drop (the Laplace law, p_in -
 *   p_out = sigma / R, that Eqs. 5-7 and 22 reproduce for a resolved
 *   interface): the mean of p (Eq. 22b) over the nodes closer than r_in to
 *   (xc, yc) minus its mean over the nodes farther than r_out, summed in FP64
 *   on the device.  Node (i, j) sits at (i, j); distances take the nearest
 *   periodic image along periodic directions.  Averaging over the inner
 *   region rather than reading the centre node matters: with the central
 *   normal (Eq. 2 with Eq. 27) phi dips at the centre of larger drops and the
 *   pressure spikes there.  Blocks until the result is on the host.
 *   Errors: LBM_ERR_INVALID (NULL handle or output, r_in <= 0, r_out < r_in,
 *   non-finite centre, or an empty region), LBM_ERR_STATE, LBM_ERR_CUDA.
 */
lbm_status lbm_laplace_jump(lbm_handle* h, double xc, double yc, double r_in, double r_out,
                            double* dp);
lbm_status lbm_probe(lbm_handle* h, int npts, const int* x, const int* y, double* phi, double* rho,
                     double* ux, double* uy, double* p);

/* lbm_synchronize -- wait for all work enqueued by this handle. */
lbm_status lbm_synchronize(lbm_handle* h);

/* lbm_destroy -- free everything the handle owns; NULL is a no-op. */
void lbm_destroy(lbm_handle* h);

/* lbm_last_error -- description of the last failure on h (never NULL). */
const char* lbm_last_error(const lbm_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_PF_H */
