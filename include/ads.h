/*
 * ads.h -- C ABI of the GB300 alternating-direction isogeometric wave solver.
 *
 * The method (Los, Behnoudfar, Paszynski, Calo, "Fast isogeometric solvers
 * for hyperbolic wave propagation problems"):
 *   - space: tensor-product B-splines of degree p on [0,L0]x[0,L1]x[0,L2],
 *     open uniform knots, n_a = n_elem[a] + p functions per axis (Sec. 2);
 *     homogeneous Dirichlet boundary (the first and last function per axis
 *     are fixed at zero) or the natural (traction-free) boundary of Sec. 5
 *     (ads_grid_t.boundary); n_elem[2] = 0 makes a 2D problem on
 *     [0,L0]x[0,L1] (one constant function along z, n_2 = 1);
 *   - scalar wave u_tt - c2 Lap u = f (Sec. 2): implicit Newmark step with
 *     the Kronecker split operator (eq. pwave2)
 *         (Mx+eta Kx)(x)(My+eta Ky)(x)(Mz+eta Kz) a_{n+1}
 *             = F_{n+1} - K (u_n + tau v_n + eta a_n),   eta = c2 tau^2/4,
 *         u_{n+1} = u_n + tau v_n + eta (a_n + a_{n+1}),
 *         v_{n+1} = v_n + tau/2 (a_n + a_{n+1}),
 *     K = c2 (Kx.My.Mz + Mx.Ky.Mz + Mx.My.Kz); the split inverse is three
 *     directional banded solves (Appendix);
 *   - linear elasticity rho u_tt = div sigma + f (Sec. 5): three-level
 *     alternating-triangular scheme (eqs. decom, pre, corr, spill, gen),
 *         D (U^{n+1} - 2U^n + U^{n-1}) / tau^2 + Ups U^n = f^n,
 *         D = (rho M + tau^2/2 Ups1~)(rho M)^{-1}(rho M + tau^2/2 Ups2~).
 *
 * Conventions for every call:
 *   - Return ADS_OK (0) or a negative ADS_ERR_* code; ads_last_error() gives
 *     a message (thread-local, valid until the next call on that thread).
 *   - Field arrays cross the boundary as FP64 coefficient arrays of the FULL
 *     space, [comp][z][y][x] with x fastest, count = comps*n0*n1*n2 doubles
 *     (n from ads_dims); with the Dirichlet restriction the boundary
 *     coefficients are ignored on input and zero on output.
 *   - mem = ADS_HOST: plain host pointers (pageable or pinned); the caller
 *     owns them, the library copies and keeps no reference.
 *     mem = ADS_DEVICE: device pointers on the simulation's device.
 *   - Device memory of a simulation is owned by the library; it comes from
 *     the allocator in ads_options_t (e.g. a framework's caching allocator)
 *     or from cudaMalloc.
 *   - Work is ordered on the simulation's CUDA stream; ads_step returns
 *     without waiting, ads_get_state / ads_energy / ads_sync wait.
 *   - A simulation is not thread-safe: one caller thread at a time.  Distinct
 *     simulations may be driven from distinct threads (ads_batch_step and
 *     ads_autotune serialise their shared process-wide state).
 */
#ifndef ADS_H
#define ADS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADS_OK 0
#define ADS_ERR_INVALID_ARG (-1)
#define ADS_ERR_OOM (-2)
#define ADS_ERR_CUDA (-3)
#define ADS_ERR_TIMEOUT (-4)
#define ADS_ERR_UNSUPPORTED (-5)

enum { ADS_SCALAR_WAVE = 0, ADS_ELASTIC = 1 };   /* ads_material_t.kind */
enum { ADS_FP64 = 0, ADS_FP32 = 1 };             /* ads_options_t.precision */
enum { ADS_HOST = 0, ADS_DEVICE = 1 };           /* memory kind of a pointer */

/* ads_apply operators (all FP64, on one scalar field of the full space) */
enum {
    ADS_OP_MASS = 0,        /* out = (Mx.My.Mz) in                          */
    ADS_OP_STIFF = 1,       /* out = K in, K = c2 (Kx.My.Mz + Mx.Ky.Mz + Mx.My.Kz) */
    ADS_OP_MASS_SOLVE = 2,  /* out = (Mx.My.Mz)^{-1} in, exact (Appendix)    */
    ADS_OP_SPLIT_SOLVE = 3  /* out = ((Mx+eta Kx).(My+eta Ky).(Mz+eta Kz))^{-1} in */
};

typedef struct ads_sim ads_sim_t;     /* opaque, library-owned */

typedef struct {
    int n_elem[3];        /* elements along x, y, z (>= 1) */
    double length[3];     /* domain extents (> 0) */
    int boundary;         /* ADS_DIRICHLET: homogeneous Dirichlet, the first and
                             last B-spline per axis are dropped (n_elem + p - 2
                             unknowns per axis, full arrays carry zero boundary
                             coefficients); ADS_NATURAL: traction-free / natural
                             boundary (Sec. 5), every B-spline is an unknown
                             (n_elem + p per axis, full array = unknowns) */
} ads_grid_t;

enum { ADS_DIRICHLET = 0, ADS_NATURAL = 1 };

typedef struct {
    int kind;             /* ADS_SCALAR_WAVE or ADS_ELASTIC */
    double c2;            /* scalar wave speed squared (u_tt - c2 Lap u = f) */
    double lambda, mu;    /* Lame parameters (elasticity) */
    double rho;           /* density (elasticity) */
} ads_material_t;

typedef void *(*ads_alloc_fn)(size_t bytes, void *ctx);
typedef void (*ads_free_fn)(void *ptr, void *ctx);

typedef struct {
    int precision;        /* ADS_FP64, or ADS_FP32: FP32 state and sweeps,
                             1D factors computed in FP64 and rounded */
    int device;           /* CUDA device ordinal; -1 = the current device */
    void *stream;         /* cudaStream_t for all work (not the legacy
                             default stream: steps are replayed as CUDA
                             graphs); NULL = a stream the library creates */
    ads_alloc_fn alloc;   /* device allocator; NULL = cudaMalloc */
    ads_free_fn free;     /* matching free; required when alloc is set */
    void *alloc_ctx;      /* passed to alloc/free */
    int tile_lines;       /* y rows per CTA of the RHS + x-sweep kernel (a
                             tile of one z-plane); 0 = library choice */
    int residual_correction; /* scalar wave, ADS_FP32 only: after the FP32
                             sweeps give a, form the residual
                             r = F - K p - G~ a in FP64 from the FP32 state,
                             solve G~ d = r with the FP32 sweeps and take
                             a + d (one step of iterative refinement); the
                             update then uses the corrected a.  0 = off */
} ads_options_t;

/* Gaussian g(x) = amp * exp(-|x - center|^2 / den); for elasticity the
 * vector field is dir * g (dir ignored for the scalar wave). */
typedef struct {
    double amp;
    double dir[3];
    double center[3];
    double den;
} ads_gaussian_t;

/* Source f(x, t) = r(t) g(x): Ricker wavelet
 * r(t) = (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2) times a Gaussian. */
typedef struct {
    ads_gaussian_t shape;
    double freq;
    double t0;
} ads_source_t;

/* Create a simulation (setup of Sec. 2 / Appendix): builds the 1D knot
 * vectors, Gauss rules and banded 1D matrices in FP64, factors the 1D
 * directional operators (banded LU without pivoting; all are SPD), uploads
 * them and allocates the state on the device.  p in 1..4; tau > 0;
 * opts may be NULL (FP64, current device, library stream, cudaMalloc).
 * State starts at zero with step counter 0.  Errors: INVALID_ARG (sizes,
 * tau, material), UNSUPPORTED (p, or a grid beyond the kernels' limits:
 * at most 512 unknowns per axis: n_elem + p - 2, or n_elem + p with the
 * natural boundary), OOM, CUDA. */
int ads_create(const ads_grid_t *grid, int p, double tau, const ads_material_t *mat,
               const ads_options_t *opts, ads_sim_t **out);

/* Free all device memory of the simulation (waits for its stream). */
void ads_destroy(ads_sim_t *sim);

/* Full basis counts per axis (n[3]) and field components (1 or 3). */
int ads_dims(const ads_sim_t *sim, int *n, int *comps);

/* Source term f(x,t) = r(t) g(x) (Sec. 2: F_{n+1} = (f(t_{n+1}), w)); its
 * load vector is integrated with the (p+1)-point Gauss rule.  NULL removes
 * the source.  Scalar wave: F_{n+1} enters step n -> n+1; elasticity: f^n
 * at level n (eq. gen). */
int ads_set_source(ads_sim_t *sim, const ads_source_t *src);

/* Source with a general spatial profile: F(t) = r(t) g, with g[i] = (f, N_i)
 * the load vector of an arbitrary (non-separable) f, integrated by the caller
 * and given as a full coefficient array (count = n0*n1*n2; boundary entries
 * are ignored with the Dirichlet restriction), r the Ricker wavelet of
 * (freq, t0).  Elasticity: the body force of component c is r(t) dir[c] g
 * (dir may be NULL = no force).  K1 adds r(t_{n+1}) g while it forms the
 * right-hand side (one extra read of g per unknown).  mem: ADS_HOST or
 * ADS_DEVICE.  Replaces any source set before.  Waits. */
int ads_set_source_field(ads_sim_t *sim, const double *g, size_t count, int mem, const double *dir, double freq,
                         double t0);

/* Set the state from L2 projections (Appendix: isogeometric L2 projection,
 * exact Kronecker mass solve) of Gaussian initial displacement u0 and
 * velocity v0 (either may be NULL = zero); resets the step counter to 0.
 * Scalar wave: a0 = M^{-1}(F(0) - K u0).  Elasticity: U^{-1} = U0 - tau V0
 * + tau^2/2 A0, A0 = (rho M)^{-1}(f^0 - Ups U0). */
int ads_set_gaussian_state(ads_sim_t *sim, const ads_gaussian_t *u0, const ads_gaussian_t *v0);

/* Set the state from coefficient arrays (count = comps*n0*n1*n2 each): the
 * B-spline coefficients of the discrete fields of Sec. 2 (u = sum_abc
 * N_a N_b N_c U_abc; the Newmark state u_n, v_n, a_n of eq. pwave2) or of
 * Sec. 5 (the three-level state U^n, U^{n-1} of eq. gen).
 * Scalar wave: u, v required; a may be NULL (then a = M^{-1}(F(t_n) - K u),
 * the consistent acceleration of the first line of eq. scheme at t_n).
 * Elasticity: u = U^n, v = V^n; a must be NULL; U^{n-1} as in
 * ads_set_gaussian_state.  The step counter is left unchanged.  The FP32
 * path rounds the state to FP32 here.  Errors: INVALID_ARG (null sim, u or
 * v, wrong count, a given for elasticity, unknown mem), OOM (staging
 * memory), CUDA. */
int ads_set_state(ads_sim_t *sim, const double *u, const double *v, const double *a, size_t count,
                  int mem);

/* Read the state (B-spline coefficient arrays, layout as ads_set_state);
 * any output may be NULL.  Scalar wave: u_n, v_n, a_n of the Newmark update
 * of eq. pwave2 (u_n = p - q + eta a_n, tau v_n = q - tau^2/2 a_n from the
 * two device arrays p = u + tau v + eta a, q = tau v + tau^2/2 a).
 * Elasticity: u = U^n, v = (U^n - U^{n-1})/tau (the difference quotient of
 * the three-level scheme, eq. gen); a must be NULL.  Waits for the stream;
 * reports a device-side error (ADS_ERR_TIMEOUT for an expired bounded wait)
 * recorded by earlier steps. */
int ads_get_state(ads_sim_t *sim, double *u, double *v, double *a, size_t count, int mem);

/* Advance nsteps >= 0 time steps (asynchronous on the stream).
 * Scalar wave, one step (Sec. 2, eq. pwave2, read as average-acceleration
 * Newmark with the split operator):
 *   R = F_{n+1} - K (u_n + tau v_n + eta a_n), K by sum factorisation of the
 *   Gauss-quadrature integrals (Sec. 2, eqs. for M_x, K_x);
 *   a_{n+1} = (Ax (x) Ay (x) Az)^{-1} R by three directional banded solves
 *   over every grid line (Appendix);  u, v updated as in eq. pwave2.
 * Elasticity, one step of the alternating-triangular scheme (Sec. 5, eqs.
 *   decom, pre, corr, spill, gen with sigma = 1/2): block-lower sweep,
 *   rho M, block-upper sweep, U^{n+1} = 2U^n - U^{n-1} + delta.
 * Runs of 16 steps replay a captured CUDA graph.  Errors: INVALID_ARG,
 * CUDA; device-side errors surface at the next waiting call. */
int ads_step(ads_sim_t *sim, int nsteps);

/* Advance `count` distinct simulations (same device) by nsteps each.
 * Scalar-wave simulations of equal precision and degree, whatever their
 * grids, tiles and sources, advance together: each time step is one grouped
 * launch of K1 over all their z-planes per segment length and CTA layout
 * present among them (up to 32 simulations per launch), one of the y sweep
 * for those whose K1 tile does not span y, and one of the z sweep + update
 * per segment length; runs of 16 steps replay a captured CUDA graph (cached
 * per member set).  Each (precision, degree) group runs on a stream of its
 * own: every group starts after the work already queued on its members'
 * streams, and those streams wait for their groups before any later work.
 * All groups join before any completion is queued, and elasticity
 * simulations step on their own streams after the joins, so groups and
 * elasticity overlap on the device even when every member shares one
 * stream.  Every result equals what ads_step gives the simulation alone
 * (the members share no data).  Errors: INVALID_ARG (null or repeated
 * simulation, mixed devices, nsteps < 0), CUDA. */
int ads_batch_step(ads_sim_t *const *sims, int count, int nsteps);

/* Autotuner of the K1 line tile: times every layout K1 can take for this
 * grid (whole z-plane with the fused y sweep in one CTA when it fits shared
 * memory; FP32 only: the z-plane split over a 2-CTA cluster, the y sweep
 * reading the partner's rows through distributed shared memory, when two
 * such CTAs fit one SM; 8, 16, 32 or 64 rows with a separate y sweep) for
 * trial_steps steps each on the simulation itself, restores its state and
 * step counter after every trial, and keeps the fastest.  The choice is
 * cached for the process per (grid, p, precision, kind): later calls for
 * the same shape apply it without timing.  trial_steps = 0 takes the
 * default layout.  *tile_rows (nullable) receives the rows one CTA holds
 * (for a cluster pair: its larger half).  Waits. */
int ads_autotune(ads_sim_t *sim, int trial_steps, int *tile_rows);

/* Wait for the simulation's stream; reports asynchronous CUDA errors. */
int ads_sync(ads_sim_t *sim);

/* Step counter n (time t_n = n tau). */
int ads_get_step(const ads_sim_t *sim, long long *n);

/* Energies at step n.  Scalar wave: kinetic 1/2 v^T M v, potential
 * 1/2 u^T K u; modified kinetic 1/2 v^T (G~ - eta K) v (with potential, the
 * exactly conserved invariant when f = 0).  Elasticity: kinetic
 * 1/2 rho V^T M V with V = (U^n - U^{n-1})/tau, potential 1/2 U^T Ups U,
 * kin_mod = the conserved invariant of the three-level scheme at n-1/2
 * (Sec. 5.1, eq. equality).  Reductions in FP64 with compensated summation.  Any output
 * may be NULL.  Waits for the stream. */
int ads_energy(ads_sim_t *sim, double *kinetic, double *potential, double *kin_mod);

/* Apply one of the ADS_OP_* operators of this simulation's space to a
 * scalar field (count = n0*n1*n2 doubles), in FP64 on the device.  Waits. */
int ads_apply(ads_sim_t *sim, int op, const double *in, double *out, size_t count, int mem);

/* ads_apply for callers that cannot allocate device memory during the call:
 * a host application whose device memory is handed out in full up front (a
 * pool owned by another framework, a fixed per-process budget), or a loop
 * that cannot take the synchronisation and latency cudaMalloc and cudaFree
 * may cost.  ads_apply allocates two scratch fields per call; this variant
 * calls no cudaMalloc, cudaFree or allocating library routine.  The paper
 * has no counterpart: this is a property of the library, not of the method.
 *   in, out: DEVICE pointers on the simulation's device to FP64 fields of
 *            the full space (count = n0*n1*n2, boundary coefficients ignored
 *            / written as zero); other memory is rejected with
 *            ADS_ERR_INVALID_ARG.
 *   Scratch: a fixed array compiled into the library, two fields of at most
 *            524288 doubles each (8 MiB, held by every GPU that loads the
 *            library until the process exits); spaces whose padded interior
 *            is larger are rejected with ADS_ERR_UNSUPPORTED.
 *   The first call on a device resolves the array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 *   All calls share the one array and each leaves its contents behind (a
 *   call clears what it reads first): calls whose work overlaps on the GPU
 *   (two streams, two simulations at once) race; serialise them.  The call
 *   waits for the simulation's stream and then reads the simulation's
 *   device error word (a blocking copy). */
int ads_apply_noalloc(ads_sim_t *sim, int op, const double *in, double *out, size_t count);

/* Checkpoint: the raw device state (all precisions bit-exact) plus the
 * step counter.  bytes = ads_checkpoint_bytes(); save waits for the stream. */
size_t ads_checkpoint_bytes(const ads_sim_t *sim);
int ads_checkpoint_save(ads_sim_t *sim, void *host_buf, size_t bytes);
int ads_checkpoint_load(ads_sim_t *sim, const void *host_buf, size_t bytes);

/* Device bytes held by the simulation (state, scratch, factors). */
size_t ads_device_bytes(const ads_sim_t *sim);

/* Upper bound of the device bytes a simulation of this shape holds once
 * created with a source set (state and tables, each allocation rounded up as
 * a caching allocator rounds it), for admission control before creating it.
 * kind: ADS_SCALAR_WAVE | ADS_ELASTIC; precision: ADS_FP64 | ADS_FP32.
 * Returns 0 for invalid arguments.  Host only, no device access. */
size_t ads_estimate_bytes(const ads_grid_t *grid, int p, int kind, int precision);

/* Measurement: run ONE time step with CUDA events recorded on the
 * simulation's stream between its kernels; fills names[i] (static strings)
 * and ms[i] (device time of kernel i) for i < min(cap, *count).  The stream
 * is held by a 2 ms device-side sleep while the step is queued, so the
 * intervals hold no host launch latency.  Advances the state like
 * ads_step(sim, 1).  Waits. */
int ads_profile_step(ads_sim_t *sim, const char **names, float *ms, int cap, int *count);

/* Measurement of the fused RHS kernel alone (Sec. 2, eq. pwave2: the
 * right-hand side F_{n+1} - K p by sum factorisation, then the x and y
 * directional solves of the Appendix): `reps` back-to-back launches
 * on the simulation's stream, input the displacement-like state p, output
 * the work field (overwritten; the state is not changed), bracketed by one
 * pair of CUDA events after a 2 ms device-side sleep.  *ms_per_launch: the
 * average device time per launch.  Scalar-wave simulations only
 * (ADS_ERR_UNSUPPORTED otherwise); reps in [1, 10000].  Waits. */
int ads_profile_rhs(ads_sim_t *sim, int reps, float *ms_per_launch);

/* Measurement of the device's CUDA-core arithmetic peak (the paper has no
 * counterpart; it gives the compute ceiling beside the HBM one for the
 * line sweeps): one launch of 8 CTAs x 256 threads per SM, each thread
 * running 8 independent FMA chains for `iters` rounds (1 .. 2^24), timed
 * with CUDA events on a stream of its own after one warm-up launch.
 * kind 0: FP64 DFMA; 1: FP32 FFMA; 2: packed FP32 FFMA2 (two FMAs per
 * instruction).  *tflops = 2 x FMAs / device time (TFLOP/s); *ms (nullable)
 * = the device time.  device < 0: the current device.  The clocks are
 * whatever the device runs at: this call changes no setting.  Allocates 64
 * bytes for the duration of the call.  Waits. */
int ads_measure_fma_peak(int device, int kind, int iters, double *tflops, double *ms);

/* Kernel launches issued by this library since load (all simulations). */
long long ads_launch_count(void);

/* Self-test of the device-side timeout path: one CTA waits on an mbarrier
 * whose transaction bytes never arrive (no copy is issued) for at most
 * `cycles` SM cycles (1 .. 4e9); the wait runs out, the kernel records the
 * timeout in a device error word and returns, as every bounded wait of the
 * library does.  Returns ADS_ERR_TIMEOUT when that happened (the expected
 * outcome), ADS_OK if the wait completed, ADS_ERR_CUDA on a launch error.
 * The CUDA context stays usable.  device < 0: the current device.  Waits. */
int ads_selftest_timeout(int device, long long cycles);

const char *ads_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ADS_H */
