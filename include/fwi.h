/*
 * fwi.h -- C ABI of the GB300 (sm_103a) likelihood-guidance gradient library
 * for "Robust Physics-Guided Diffusion for Full-Waveform Inversion"
 * (arXiv 2603.16393).
 *
 * The library computes, for a batch of B velocity models and Ns shots each:
 *   fwi_forward       d_syn = F(v): 2D constant-density acoustic FD solve
 *                     (Eq. 1; 2nd order in time, 4th order in space, absorbing
 *                     layer, Ricker source, receiver restriction R; Sec. 2.1, 6.1)
 *   fwi_w2_prepare    the observation-only quantities of the misfit (Sec. 5.1:
 *                     weight omega, shift c', observed quantiles, S_obs)
 *   fwi_w2_misfit     J(v) = sum_{s,r} W2 / S_obs (Eq. final_objective) and the
 *                     adjoint source dJ/dd_syn
 *   fwi_adjoint_grad  dJ/dv by the time-reversed discrete adjoint solve
 *                     (the F'* of Eq. dps_baseline_step, Sec. 4.2)
 *   fwi_guided_step   v_{i-1} = v'_{i-1} - rho_i D_i h (Eq. precond_step,
 *                     Eq. tv, Eq. rho, Eq. kappa; Algorithm 2)
 *
 * Conventions shared by every call
 *   - Array arguments are DEVICE pointers to contiguous float32 (int32 where
 *     stated) buffers owned and allocated by the caller.  The library never
 *     allocates device memory and never frees caller memory.
 *   - Layouts are row-major with the last index fastest:
 *       v, grad           [B][nz][nx]          m/s and 1/(m/s); row = depth z
 *       d_obs, d_syn, adj [B][ns][nr][nt]      traces, sample n at t_n = n dt
 *       w2                [B][ns][nr]
 *       J, rho            [B]
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls only enqueue work; they return before it runs.
 *   - Argument checks happen on the host before anything is enqueued; a
 *     failing check returns an error code and enqueues nothing.  Launch
 *     failures return FWI_ERR_CUDA.  Conditions only the device can see
 *     (a velocity above the declared v_max or not positive) are written to a
 *     status word in the workspace; fwi_check() reads it.
 *   - fwi_last_error() returns a message for the last failing call of the
 *     calling thread.
 *   - Results are deterministic: the same inputs give bitwise-identical
 *     outputs (no floating-point atomics; fixed reduction orders).
 */
#ifndef FWI_H
#define FWI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FWI_VERSION 11400  /* major*10000 + minor*100 + patch */

#if defined(__GNUC__)
#define FWI_API __attribute__((visibility("default")))
#else
#define FWI_API
#endif

/* Limits of this library. */
#define FWI_MAX_SHOTS 256
#define FWI_MAX_RECEIVERS 1024

typedef enum fwi_status {
    FWI_OK = 0,
    FWI_ERR_INVALID_ARG = 1,    /* a pointer, size or parameter is invalid      */
    FWI_ERR_UNSTABLE_CFL = 2,   /* v_max dt sqrt(1/dx^2+1/dz^2) > sqrt(3)/2, or a
                                   velocity above v_max / not positive was found
                                   on the device                                   */
    FWI_ERR_UNSUPPORTED = 3,    /* valid but outside what this library implements */
    FWI_ERR_CUDA = 4,           /* a CUDA runtime call or launch failed         */
    FWI_ERR_DEVICE_TIMEOUT = 5, /* a device-side wait ran out of its budget     */
    FWI_ERR_OOM = 6             /* a caller buffer is too small                 */
} fwi_status;

/* Discretisation and acquisition (Sec. 2.1, 6.1; see the readings listed with
 * each field).  Host struct; fwi_plan_create copies everything it needs,
 * including the index arrays.  Physical scalars are double: the kernels form
 * their per-cell coefficients from them in double and round once, so that a
 * float32 time step (0.001 is not a float) does not bias every velocity. */
typedef struct fwi_problem {
    int nz, nx;          /* physical grid (rows = depth), >= 1                      */
    double dz, dx;       /* grid spacing in m, > 0                                  */
    int nb;              /* absorbing-layer width in cells on left, right, bottom   */
    int top_bc;          /* 0: zero ghosts above row 0; 1: mirror (du/dn = 0, Eq. 1) */
    int nt;              /* time steps, >= 2                                        */
    double dt;           /* time step in s, > 0                                     */
    int ns, nr;          /* shots (<= FWI_MAX_SHOTS), receivers (<= FWI_MAX_RECEIVERS) */
    const int *src_iz, *src_ix;   /* HOST arrays [ns]: source cell per shot          */
    const int *rec_iz, *rec_ix;   /* HOST arrays [nr]: receivers shared by all shots */
    double f_peak;       /* Ricker peak frequency in Hz (Sec. 6.1: 15)              */
    double t0;           /* Ricker delay in s; <= 0 selects 1.1 / f_peak (Sec. 6.1) */
    double v_ref;        /* speed the damping is designed for, m/s (not differentiated) */
    double refl_R;       /* nominal two-way amplitude reflection of the layer, (0,1] */
    double v_max;        /* declared upper bound of every velocity passed in, m/s  */
    int batch;           /* B models per call, >= 1                                 */
    int checkpoint_every; /* 0: fwi_forward keeps the whole wavefield record for the
                            adjoint; K >= 1: it keeps the propagator state every K
                            steps and fwi_adjoint_grad recomputes each K-step segment
                            from it (same arithmetic, bitwise-identical gradient,
                            about nt/K times less memory, one extra forward pass) */
    int space_order;     /* 0 or 4: 4th-order Laplacian (the default); 8: the 8th-order
                            stencil of the paper's solver (Sec. 6.1), run on the
                            global-memory tiled kernels for every grid size         */
    int kernels;         /* propagator family: FWI_KERNELS_AUTO (0) picks by grid size;
                            the others force one and fail with FWI_ERR_UNSUPPORTED
                            where it cannot run the plan.  Every family computes the
                            same recurrences (Sec. 2.1, Eq. 2) to float rounding.   */
    int absorber;        /* FWI_ABSORBER_SPONGE (0): the damping layer of Eq. (1)
                            with A, B (the default); FWI_ABSORBER_CPML (1): a
                            convolutional PML in the same nb cells (the paper's
                            solver absorbs with a PML, Sec. 6.1): the layer stretches
                            d/dx, d/dz by s = 1 + sigma/(i omega), sigma = d0 (d/nb)^2,
                            d0 = 3 v_ref ln(1/refl_R) / (2 nb h), each 1/s a memory
                            variable advanced per step.  CPML plans: 4th order,
                            top_bc = 0, checkpoint_every = 0, distinct receiver cells;
                            they run on FWI_KERNELS_CPML.                           */
    int shape;           /* thread shape inside the family: FWI_SHAPE_DEFAULT (0) or one
                            of the FWI_SHAPE_* of the family the plan runs on (the
                            others fail with FWI_ERR_UNSUPPORTED); every shape computes
                            the same results.  fwi_autotune_kernels measures them. */
} fwi_problem;

/* Thread shapes (fwi_problem.shape); the default is marked. */
enum {
    FWI_SHAPE_DEFAULT = 0,
    FWI_SHAPE_RESIDENT_PAIRS = 1,    /* resident: two columns x 11 rows a thread, packed
                                        f32x2 arithmetic (default where the padded width
                                        is even and NZ <= 110)                          */
    FWI_SHAPE_RESIDENT_COLUMNS = 2,  /* resident: one column x 22 rows a thread        */
    FWI_SHAPE_CLUSTER_RS13 = 3,      /* cluster: one column x 13-row thread strips     */
    FWI_SHAPE_CLUSTER_RS19 = 4,      /* cluster: one column x 19-row thread strips     */
    FWI_SHAPE_TILED_ROWS8 = 5,       /* tiled: 8 rows a thread, 256 threads a 32 x 64 tile */
    FWI_SHAPE_TILED_ROWS4 = 6,       /* tiled: 4 rows a thread, 512 threads a tile      */
    FWI_SHAPE_CLUSTER_PAIRS = 7,     /* cluster: two columns x 10 rows a thread, packed
                                        f32x2 arithmetic, the adjoint's per-cell arrays
                                        in tensor memory (default where the padded width
                                        is even and the strips fit 672 threads; else 13-,
                                        then 19-row single-column strips)               */
    FWI_SHAPE_TILED_QUADS = 8        /* tiled: four columns x 2 rows a thread, 256 threads
                                        a tile, 16-byte (float4) loads and stores
                                        (default; the same bits as the row shapes)     */
};

/* Absorbing layers (fwi_problem.absorber). */
enum { FWI_ABSORBER_SPONGE = 0, FWI_ABSORBER_CPML = 1 };

/* Propagator families (fwi_problem.kernels). */
enum {
    FWI_KERNELS_AUTO = 0,
    FWI_KERNELS_RESIDENT = 1, /* one CTA holds a (model, shot)'s whole padded grid in
                                 shared memory; 4th order; grids up to ~150 x 340 cells  */
    FWI_KERNELS_TILED = 2,    /* global-memory fields, TMA-staged halo tiles, one launch
                                 per time step; any grid, 4th or 8th order               */
    FWI_KERNELS_CLUSTER = 3,  /* a cluster of 2-8 CTAs holds the grid in their shared
                                 memories, halo rows through distributed shared memory;
                                 4th order, whole record (checkpoint_every = 0), padded
                                 width <= 337                                           */
    FWI_KERNELS_CPML = 4      /* global-memory kernels of the CPML absorber (the only
                                 family of absorber = FWI_ABSORBER_CPML plans)         */
};

/* Misfit hyperparameters (Sec. 5.1, 6.2, 6.3): k = 100, c' factor 1.1,
 * eps' = 1e-9, N_xi = 1000. */
typedef struct fwi_w2_params {
    double k;            /* Eq. omega_def, >= 0                                     */
    double cshift_factor; /* c' = cshift_factor |min_t omega d_obs|, >= 0           */
    double eps_density;  /* eps' in the density denominator, >= 0                   */
    int n_xi;            /* quantile nodes xi_j = j/(n_xi-1), >= 2                  */
    int squared;         /* 0: J = sum W2 / S_obs (Eq. final_objective); 1: the raw
                            objective of the W2+TV baseline (Sec. 6.3, Baseline 1),
                            J = sum W2^2 / sum int_0^1 |Q_obs|^2, per-trace output W2^2
                            (pass k = 0 for its unenhanced traces)                  */
} fwi_w2_params;

/* Guided-step hyperparameters (Eq. rho, Eq. kappa; Sec. 6.3: c = 0.1, tau = 0,
 * eps = 1e-4, gamma and rho0 per dataset in Table 1).  kappa is clipped to
 * [kappa_min, kappa_max] only when kappa_min < kappa_max.
 * unit (> 0): the size of one unit of the diffusion's normalised space in the
 * units of the arrays passed (1 when they are already normalised; 1500 for
 * velocities in m/s with the normalisation (v - 3000)/1500).  The update is
 * then exactly the normalised-space update mapped back: TV is taken on
 * v0hat/unit, kappa on unit*g, and the step is rho kappa unit^2 h. */
typedef struct fwi_guide_params {
    double rho0, c, tau, gamma, eps, kappa_min, kappa_max;
    double unit;
} fwi_guide_params;

typedef struct fwi_plan fwi_plan;   /* opaque, host memory only */

/* Validate a problem and build a plan (host only; no CUDA call).
 * Checks every field above, the CFL bound for v_max (v_max dt sqrt(1/dx^2 +
 * 1/dz^2) <= 2 / sqrt(lambda), lambda the largest symbol of the 1D stencil:
 * 16/3 at 4th order (bound sqrt(3)/2), 6.5016 at 8th order (bound 0.7844)),
 * that sources and receivers lie on the physical grid, and that this library
 * can run the grid (FWI_ERR_UNSUPPORTED otherwise).  *out receives the plan
 * or NULL.  Errors: FWI_ERR_INVALID_ARG, FWI_ERR_UNSTABLE_CFL,
 * FWI_ERR_UNSUPPORTED. */
FWI_API fwi_status fwi_plan_create(const fwi_problem *prob, const fwi_w2_params *w2,
                           fwi_plan **out);

/* Release a plan (NULL is ignored). */
FWI_API void fwi_plan_destroy(fwi_plan *plan);

/* Bytes the caller must provide:
 *   workspace: device scratch passed to fwi_forward / fwi_w2_misfit /
 *              fwi_adjoint_grad / fwi_check; its first 256 bytes hold the
 *              device status word (with checkpoint_every = K it also holds
 *              the K-step record of one segment and the adjoint state);
 *   obs_ctx:   filled by fwi_w2_prepare, read by fwi_w2_misfit;
 *   snapshots: what fwi_forward keeps for fwi_adjoint_grad: the wavefield
 *              record (nt time levels of the padded grid per model and shot)
 *              when checkpoint_every = 0, else ceil(nt/K) checkpoints of the
 *              propagator state (two padded grids per model and shot each).
 * The workspace and snapshot buffers must start on a 16-byte boundary (the
 * record planes and checkpoints are moved in 16-byte units); every entry
 * point that takes them returns FWI_ERR_INVALID_ARG otherwise.
 * Any output pointer may be NULL. */
FWI_API fwi_status fwi_plan_sizes(const fwi_plan *plan, size_t *workspace_bytes,
                          size_t *obs_ctx_bytes, size_t *snapshot_bytes);

/* Padded grid of the plan: NZ = nz + nb, NX = nx + 2 nb. */
FWI_API fwi_status fwi_plan_padded(const fwi_plan *plan, int *NZ, int *NX);

/* Propagator family the plan runs: *family = FWI_KERNELS_RESIDENT, _TILED,
 * _CLUSTER or _CPML (the automatic choice resolved, or the one forced).
 * Host only. */
FWI_API fwi_status fwi_plan_kernels(const fwi_plan *plan, int *family);

/* Forward solve of Eq. (1) for every model and shot (Sec. 2.1, 6.1).
 *   v         [B][nz][nx] device, m/s; every value must be in (0, v_max]
 *   d_syn     [B][ns][nr][nt] device, written: sample n = field at step n+1
 *             at each receiver
 *   snapshots device buffer of fwi_plan_sizes' snapshot_bytes, written with
 *             the record fwi_adjoint_grad needs; NULL to skip it (e.g. when
 *             only data are wanted)
 *   workspace device buffer of workspace_bytes; its status word is reset
 * A velocity outside (0, v_max] sets FWI_ERR_UNSTABLE_CFL in the status word
 * and leaves that model's outputs undefined. */
FWI_API fwi_status fwi_forward(const fwi_plan *plan, const float *v, float *d_syn,
                       float *snapshots, void *workspace, void *stream);

/* Self-check of the propagators' bounded waits (failure detection without a
 * fault): fwi_forward on a plan that runs FWI_KERNELS_CLUSTER (every halo row
 * withheld, each wait bounded by 20 ms) or FWI_KERNELS_TILED (no halo tile
 * loaded, each wait bounded by 1024 mbarrier polls), so that the waits run
 * out.  The kernels finish (their outputs are not meaningful) and the status
 * word in the workspace reads FWI_ERR_DEVICE_TIMEOUT, which fwi_check()
 * returns; the device stays usable.  Arguments as fwi_forward.  Errors:
 * FWI_ERR_INVALID_ARG, FWI_ERR_UNSUPPORTED for plans of other families,
 * FWI_ERR_CUDA. */
FWI_API fwi_status fwi_forward_wait_check(const fwi_plan *plan, const float *v, float *d_syn,
                                          float *snapshots, void *workspace, void *stream);

/* Observation-only part of the misfit for B observed data cubes
 * (Sec. 5.1 (I)-(III), Sec. 6.2):
 *   M = max_{s,r,t} |d_obs|, omega = 1/(1 + k |d_obs| / M)      (Eq. omega_def)
 *   c'(s,r) = cshift_factor |min_t omega d_obs|                  (Sec. 6.2)
 *   Q_obs = quantiles of P(omega d_obs + c')                     (Eq. pdf_map, Wp_1d)
 *   S_obs = sum_{s,r} (int_0^1 |Q_obs|^2)^(1/2)                  (Sec. 5.1 (III))
 *   d_obs   [B][ns][nr][nt] device
 *   obs_ctx device buffer of obs_ctx_bytes, written (opaque layout). */
FWI_API fwi_status fwi_w2_prepare(const fwi_plan *plan, const float *d_obs, void *obs_ctx,
                          void *stream);

/* Weighted, normalised W2 misfit (Eq. final_objective; Sec. 6.2 numerics:
 * trapezoid CDF, interpolated generalised-inverse quantiles, trapezoid in xi)
 * and its exact derivative.
 *   obs_ctx  from fwi_w2_prepare (same plan)
 *   d_syn    [B][ns][nr][nt] device
 *   J        [B] device, written
 *   w2       [B][ns][nr] device, written per-trace W2; NULL to skip
 *   adj_src  [B][ns][nr][nt] device, written dJ/dd_syn; NULL to skip
 *   workspace device buffer of workspace_bytes (per-trace scratch) */
FWI_API fwi_status fwi_w2_misfit(const fwi_plan *plan, const void *obs_ctx, const float *d_syn,
                         float *J, float *w2, float *adj_src, void *workspace,
                         void *stream);

/* dJ/dv by the discrete adjoint of fwi_forward (time-reversed solve with the
 * adjoint source injected at the receivers, imaging condition, fold of the
 * absorbing layer onto the edge cells, sum over shots in a fixed order).
 * With checkpoint_every = K the time loop runs as ceil(nt/K) segments, last
 * first: each recomputes its K forward steps from its checkpoint into the
 * workspace, then runs them backwards (2 ceil(nt/K) + 1 launches).
 *   v         [B][nz][nx] device, the same models fwi_forward was given
 *   adj_src   [B][ns][nr][nt] device (from fwi_w2_misfit)
 *   snapshots what fwi_forward wrote for these models (record or checkpoints)
 *   grad      [B][nz][nx] device, written, 1/(m/s)
 *   workspace device buffer of workspace_bytes */
FWI_API fwi_status fwi_adjoint_grad(const fwi_plan *plan, const float *v, const float *adj_src,
                            const float *snapshots, float *grad, void *workspace,
                            void *stream);

/* Preconditioned guided update of Algorithm 2 for B instances of nz x nx:
 *   TV  = (1/N_g) sum |forward differences| of v0hat        (Eq. tv; a
 *         difference leaving the grid counts as 0)
 *   rho = rho0 exp(-(TV - tau)_+ / c)                        (Eq. rho)
 *   kappa_j = ((||g||_inf + eps)/(|g_j| + eps))^gamma         (Eq. kappa)
 *   v_out = v_prime - rho kappa . h                          (Eq. precond_step)
 *   (with params->unit != 1, see fwi_guide_params)
 *   v_prime, v0hat, g (= grad wrt v0hat), h (= grad wrt v_i): [B][nz][nx] device
 *   v_out  [B][nz][nx] device, written (may alias v_prime)
 *   rho_out [B] device, written; NULL to skip
 * TV is taken on v0hat as passed (callers pass the normalised field). */
FWI_API fwi_status fwi_guided_step(int batch, int nz, int nx, const fwi_guide_params *params,
                           const float *v_prime, const float *v0hat, const float *g,
                           const float *h, float *v_out, float *rho_out, void *stream);

/* Least-squares data potential of the DPS baseline (Phi_l2 of Eq.
 * dps_baseline_step, Sec. 4.2; Baseline 3 of Sec. 6.3), per instance b:
 *   J[b]    = (1/2) sum_{s,r,t} (d_syn - d_obs)^2 / sigma^2
 *   adj_src = dJ/dd_syn = (d_syn - d_obs) / sigma^2   (the adjoint source of
 *             fwi_adjoint_grad for this potential)
 *   plan    gives the sizes B, ns, nr, nt
 *   d_obs, d_syn [B][ns][nr][nt] device; J [B] device, written;
 *   adj_src [B][ns][nr][nt] device, written, or NULL; sigma finite, > 0.
 * Errors: FWI_ERR_INVALID_ARG before any launch, FWI_ERR_CUDA. */
FWI_API fwi_status fwi_l2_misfit(const fwi_plan *plan, const float *d_obs, const float *d_syn,
                                 double sigma, float *J, float *adj_src, void *stream);

/* Total variation of Eq. tv on the field v / unit (forward differences, a
 * difference leaving the grid counts as 0, divided by N_g = nz nx) and the
 * (sub)gradient step direction of the TV-regularised baselines (Sec. 6.3,
 * Baselines 1 and 2):
 *   h  = g + alpha dTV(v / unit)/dv,  taking sign(0) = 0 for a tie
 *   tv[b] = TV(v_b / unit)
 *   v, g, h [batch][nz][nx] device (g may be NULL: taken as 0; h may alias g);
 *   tv [batch] device or NULL; alpha finite, unit > 0.
 * Errors: FWI_ERR_INVALID_ARG, FWI_ERR_UNSUPPORTED (grid above 2^30 cells),
 * FWI_ERR_CUDA. */
FWI_API fwi_status fwi_tv_grad(int batch, int nz, int nx, double alpha, double unit,
                               const float *v, const float *g, float *h, float *tv,
                               void *stream);

/* Reconstruction measures of Sec. 6.3 per instance, out[b][3]:
 *   [0] ||v_true - v_rec||_2 / ||v_true||_2
 *   [1] PSNR = 10 log10(R^2 / mean (v_true - v_rec)^2), R = data_range
 *   [2] SSIM averaged over every 11 x 11 window inside the grid, Gaussian
 *       weights (sigma 1.5) normalised to 1, C1 = (0.01 R)^2, C2 = (0.03 R)^2;
 *       NaN if the grid is smaller than a window
 *   v_true, v_rec [batch][nz][nx] device; out [batch][3] device, written.
 * Errors: FWI_ERR_INVALID_ARG, FWI_ERR_UNSUPPORTED, FWI_ERR_CUDA. */
FWI_API fwi_status fwi_image_metrics(int batch, int nz, int nx, double data_range,
                                     const float *v_true, const float *v_rec, float *out,
                                     void *stream);

/* Largest batch x ns x nr that fwi_w2_misfit_static accepts. */
#define FWI_STATIC_MAX_TRACES 65536

/* fwi_w2_misfit without a workspace argument (the paper has no counterpart:
 * this is a deployment variant).  For callers that cannot provide device
 * memory of their own -- code that runs inside a host framework owning every
 * device allocation through its own pool, or a steady-state loop in which no
 * allocation may happen -- the per-trace scratch of the misfit comes from an
 * array compiled into the library (FWI_STATIC_MAX_TRACES floats of device
 * global memory on every GPU that loads the library, held until the process
 * exits).  The call itself allocates nothing.
 *   Arguments and results are those of fwi_w2_misfit.  The array holds the
 *   per-trace W2 values only when w2 is NULL; a caller that passes w2 gets
 *   them there and the array is not used (nor the size limit applied).
 *   The first call on a device looks up the array's device address with
 *   that device current; make that first call before any stream capture.
 *   The address belongs to the device's context: after cudaDeviceReset the
 *   next call looks it up again (make that call before any capture too).
 *   All calls on a device share the one array and it keeps the last call's
 *   contents; every value a call reads is written by that same call first,
 *   so nothing needs clearing.  Calls whose GPU work overlaps (different
 *   streams or threads on the same device) race on the array: serialise them.
 * Errors: FWI_ERR_INVALID_ARG for NULL arguments, FWI_ERR_UNSUPPORTED when
 * w2 is NULL and batch x ns x nr exceeds FWI_STATIC_MAX_TRACES, FWI_ERR_CUDA
 * otherwise. */
FWI_API fwi_status fwi_w2_misfit_static(const fwi_plan *plan, const void *obs_ctx,
                                        const float *d_syn, float *J, float *w2,
                                        float *adj_src, void *stream);

/* Measured choice of the propagator family and thread shape (a tuning
 * utility; the paper has no counterpart).  For every family that can run the
 * problem (resident, tiled, cluster, CPML; see fwi_problem.kernels) and every
 * shape of that family (fwi_problem.shape) it creates plans on T =
 * trial_steps and min(2T, nt) steps, times a gradient pass on each (the
 * faster of two after an untimed one: fwi_forward with the record, then
 * fwi_adjoint_grad with the synthetic data as adjoint source) in `scratch`,
 * and predicts the pass at the problem's nt as fixed cost + nt x cost per
 * step from the two timings (the families differ in both).  Reports the
 * family and shape with the smallest prediction.  Blocks the host until the
 * trial work on the stream is done.
 *   prob, w2     the problem (its `kernels` and `shape` fields are ignored)
 *   v            [B][nz][nx] device, representative models in (0, v_max]
 *   trial_steps  steps per trial, in [2, prob->nt]
 *   scratch      device buffer, 256-byte aligned, of at least
 *                fwi_autotune_scratch_bytes; overwritten
 *   family       written: FWI_KERNELS_RESIDENT, _TILED, _CLUSTER or _CPML
 *   shape        written: the FWI_SHAPE_* of the chosen family measured fastest
 *   ms           [4] host, written: predicted milliseconds of one pass at nt
 *                steps for resident, tiled, cluster, CPML, each at its fastest
 *                shape (-1 where the family cannot run the problem); NULL to skip
 *   shapes       [4] host, written: those fastest shapes (-1 where the family
 *                cannot run the problem); NULL to skip
 * Set kernels = *family and shape = *shape in the problem before
 * fwi_plan_create.  Errors: those of fwi_plan_create for the problem,
 * FWI_ERR_INVALID_ARG, FWI_ERR_OOM (scratch too small), FWI_ERR_CUDA, and
 * device statuses of the trials (fwi_check). */
FWI_API fwi_status fwi_autotune_kernels(const fwi_problem *prob, const fwi_w2_params *w2,
                                        const float *v, int trial_steps, void *scratch,
                                        size_t scratch_bytes, int *family, int *shape, float *ms,
                                        int *shapes, void *stream);

/* Scratch bytes fwi_autotune_kernels needs for this problem and trial length
 * (the largest over the families of workspace + snapshots + data + gradient
 * of the min(2 trial_steps, nt)-step trial plan).  Host only.  Errors: as fwi_plan_create, and
 * FWI_ERR_INVALID_ARG for trial_steps outside [2, nt]. */
FWI_API fwi_status fwi_autotune_scratch_bytes(const fwi_problem *prob, const fwi_w2_params *w2,
                                              int trial_steps, size_t *bytes);

/* Plan groups: uneven instances as one unit (a batching utility; the paper
 * has no counterpart).  A group holds plans of any grid sizes and propagator
 * families; fwi_group_gradient runs every plan's whole gradient (fwi_forward
 * with its record or checkpoints, fwi_w2_misfit, fwi_adjoint_grad) on a
 * stream of its own, forked from `stream` by an event and joined back to it,
 * so that the plans' kernels overlap on the GPU and a capture of `stream`
 * (cudaStreamBeginCapture) records the whole uneven set as one CUDA graph,
 * replayed with one launch.  Results are those of the per-plan calls.
 * fwi_group_create needs the current CUDA device (it creates the streams and
 * events, owned by the group); the plans stay owned by the caller and must
 * outlive the group.  Errors: FWI_ERR_INVALID_ARG, FWI_ERR_CUDA. */
typedef struct fwi_group fwi_group;
FWI_API fwi_status fwi_group_create(const fwi_plan *const *plans, int n, fwi_group **out);
FWI_API void fwi_group_destroy(fwi_group *group);

/* Every list has one entry per plan of the group, with the layout of the
 * corresponding single-plan call: v [B][nz][nx]; obs_ctx from fwi_w2_prepare;
 * d_syn and adj_src [B][ns][nr][nt] (written); snapshots of snapshot_bytes;
 * grad [B][nz][nx] and J [B] (written); workspace of workspace_bytes.  The
 * plans' buffers must not overlap.  Errors: FWI_ERR_INVALID_ARG for a NULL
 * list or entry, otherwise those of the single-plan calls. */
FWI_API fwi_status fwi_group_gradient(fwi_group *group, const float *const *v,
                                      const void *const *obs_ctx, float *const *d_syn,
                                      float *const *adj_src, float *const *snapshots,
                                      float *const *grad, float *const *J,
                                      void *const *workspace, void *stream);

/* Persistent passes over uneven instances (a batching utility; the paper has
 * no counterpart).  The forward (record on) or the adjoint of up to
 * FWI_QUEUE_MAX_PLANS plans of different grid sizes in ONE launch: every
 * (model, shot) unit of every plan goes on one numbered list (plan by plan, in
 * the order given: put the largest first), and each CTA of the resident
 * column-pair propagators draws the next unit from *counter until the list is
 * done, so units of different grids run side by side and no SM waits for the
 * tail of one plan.  Results are bitwise those of fwi_forward /
 * fwi_adjoint_grad on each plan.
 *   plans     store-all plans (checkpoint_every 0) of the resident column-pair
 *             kernels (padded NZ <= 110 and an even padded width <= 156) with one
 *             physics: the same dx, dz, dt, nb, top_bc, v_ref, refl_R, f_peak and
 *             t0 (grids, batches, shots and receivers may differ); others fail
 *             with FWI_ERR_UNSUPPORTED
 *   lists     one entry per plan, with the layout of the single-plan call
 *   counter   one int of device memory, owned by the caller; the call zeroes it
 *             on the stream before the launch (no allocation)
 * fwi_queue_adjoint also sums each plan's shots into grad.
 * Errors: FWI_ERR_INVALID_ARG, FWI_ERR_UNSUPPORTED, FWI_ERR_CUDA. */
#define FWI_QUEUE_MAX_PLANS 4
FWI_API fwi_status fwi_queue_forward(const fwi_plan *const *plans, int n, const float *const *v,
                                     float *const *d_syn, float *const *snapshots,
                                     void *const *workspace, int *counter, void *stream);
FWI_API fwi_status fwi_queue_adjoint(const fwi_plan *const *plans, int n, const float *const *v,
                                     const float *const *adj_src, const float *const *snapshots,
                                     float *const *grad, void *const *workspace, int *counter,
                                     void *stream);

/* Wait for `stream` and return the device status word of `workspace`
 * (FWI_OK, FWI_ERR_UNSTABLE_CFL, FWI_ERR_DEVICE_TIMEOUT), then clear it. */
FWI_API fwi_status fwi_check(const fwi_plan *plan, void *workspace, void *stream);

/* ---------------------------------------------------------------- convolutional score model
 * Elementwise pieces of a convolutional score model built on
 * fwi_conv3x3_bf16: s(x, i) = -eps(x) / sqrt(1 - abar_i) from a
 * noise-prediction network eps (Sec. 3.4), and its vector-Jacobian product
 * for Eq. chain_rule.  Activations are NHWC bf16 with `channels` channels per
 * pixel; npix = B nz nx.  Errors: FWI_ERR_INVALID_ARG before any launch,
 * FWI_ERR_CUDA. */

/* X[p][0] = bf16(scale x[p]), X[p][c] = 0 for c >= 1; x [npix] fp32, X
 * [npix][channels] bf16 (16-byte aligned, channels a multiple of 8). */
FWI_API fwi_status fwi_pack_channel0(long long npix, int channels, float scale, const float *x,
                                     void *X, void *stream);

/* y[p] = scale Y[p][0]; Y [npix][channels] fp32, y [npix] fp32. */
FWI_API fwi_status fwi_unpack_channel0(long long npix, int channels, float scale, const float *Y,
                                       float *y, void *stream);

/* A = bf16(silu(P)), silu(p) = p / (1 + e^-p); P, A [n] bf16 (may alias). */
FWI_API fwi_status fwi_silu_bf16(long long n, const void *P, void *A, void *stream);

/* dP = bf16(dA silu'(P)), silu'(p) = sg (1 + p (1 - sg)), sg = 1 / (1 + e^-p);
 * dA, P, dP [n] bf16 (dP may alias dA). */
FWI_API fwi_status fwi_silu_grad_bf16(long long n, const void *dA, const void *P, void *dP,
                                      void *stream);

/* Self-check of the convolution's bounded waits (failure detection without a
 * fault): the same launch as fwi_conv3x3_bf16 with the weight blocks never
 * loaded and a wait bound of 20 ms, so that every device-side wait runs out.
 * The kernel then waits (bounded) for the input copies it started, releases
 * its tensor memory, writes nothing to y and sets *status (device int, not
 * NULL) to FWI_ERR_DEVICE_TIMEOUT; the device stays usable.  Arguments as for
 * fwi_conv3x3_bf16.  Errors: as fwi_conv3x3_bf16, FWI_ERR_INVALID_ARG for a
 * NULL status. */
FWI_API fwi_status fwi_conv3x3_bf16_wait_check(int n, int h, int w, int cin, int cout,
                                               const void *x, const void *wt, void *y, int y_bf16,
                                               int *status, void *stream);

/* Denoising score matching (Sec. 3.4, Eq. L2_rewrite) of the convolutional
 * score model: with x_t = sqrt(abar) x_0 + sqrt(1 - abar) z the conditional
 * score is -z / sqrt(1 - abar), and with the weight kappa(t) = 1 - abar the
 * objective is the regression of eps(x_t, t) on z.  Float32 device arrays
 * unless stated; bf16 tensors are NHWC with `channels` per pixel.  Errors:
 * FWI_ERR_INVALID_ARG before any launch, FWI_ERR_CUDA. */

/* xt = sqrt(abar) x0 + sqrt(1 - abar) z over n elements, 0 < abar < 1. */
FWI_API fwi_status fwi_dsm_noisy(long long n, double abar, const float *x0, const float *z,
                                 float *xt, void *stream);

/* *loss = mean over n of (eps - z)^2 (one device float) and grad = d loss /
 * d eps = 2 (eps - z) / n.  The sum runs over per-CTA partials written to
 * `work` (up to 608 of them, work_floats floats, caller-owned; NULL: one CTA)
 * and added in order: a fixed summation order for given n and work_floats. */
FWI_API fwi_status fwi_dsm_loss(long long n, const float *eps, const float *z, float *loss,
                                float *grad, float *work, long long work_floats, void *stream);

/* Weight gradient of the 3x3 convolution (stride 1, zero padding 1):
 * dW[co][ky][kx][ci] = sum_{b,y,x} dP[b][y][x][co] X[b][y+ky-1][x+kx-1][ci],
 * X bf16 [n][h][w][cin], dP bf16 [n][h][w][cout], dW float32 [cout][3][3][cin]
 * (written), cin and cout multiples of 64; X, dP, dW and work 16-byte aligned.
 * On the CUDA cores (64 x 64 register-tiled outputs).  The pixels are split
 * into fwi_conv3x3_wgrad_splits(...) contiguous ranges whose partial sums go
 * to `work` (work_floats floats, caller-owned; NULL or too small for two
 * splits means one range written straight to dW) and are then added in range
 * order: a fixed summation order for given sizes, work_floats and SM count. */
FWI_API fwi_status fwi_conv3x3_wgrad(int n, int h, int w, int cin, int cout, const void *X,
                                     const void *dP, float *dW, float *work,
                                     long long work_floats, void *stream);

/* The number of pixel ranges fwi_conv3x3_wgrad uses (1..16; about four CTAs
 * per SM, at most work_floats / (9 cin cout)); 0 for invalid sizes. */
FWI_API int fwi_conv3x3_wgrad_splits(int n, int h, int w, int cin, int cout,
                                     long long work_floats);

/* The same weight gradient on the tensor cores (tcgen05, BF16 products, FP32
 * accumulation), cin and cout multiples of 64 (a 64-channel remainder of a
 * 128-channel block is computed on zero rows).  Over the zero-padded pixel
 * domain q (rows of wp = w + 2 rounded up to a multiple of 8 pixels) the
 * operands are first staged K-major in `stage` (caller-owned, at least
 * fwi_conv3x3_wgrad_tc_stage_bytes(...) bytes): dP^T[co][q] and three copies
 * X_s^T[ci][q] = Xpad(q + s), s = -1, 0, 1; each tap (ky, kx) is then the
 * GEMM sum_q dP^T[co][q] X_{kx-1}^T[ci][q + (ky-1) wp].  The padded pixels
 * are split into fwi_conv3x3_wgrad_tc_splits(...) ranges whose partial tiles
 * go to `work` (NULL: one range) and are added in range order.  *status (may
 * be NULL) receives FWI_ERR_DEVICE_TIMEOUT if a device-side wait ran out. */
FWI_API fwi_status fwi_conv3x3_wgrad_tc(int n, int h, int w, int cin, int cout, const void *X,
                                        const void *dP, float *dW, void *stage,
                                        long long stage_bytes, float *work,
                                        long long work_floats, int *status, void *stream);

/* Self-check of fwi_conv3x3_wgrad_tc's bounded waits: the same launch with
 * every copy withheld and a 20 ms bound, so that the MMA issuer's first wait
 * runs out; the kernel then frees its TMEM and returns, and *status (needed)
 * reads FWI_ERR_DEVICE_TIMEOUT.  dW is left unspecified; one range. */
FWI_API fwi_status fwi_conv3x3_wgrad_tc_wait_check(int n, int h, int w, int cin, int cout,
                                                   const void *X, const void *dP, float *dW,
                                                   void *stage, long long stage_bytes,
                                                   int *status, void *stream);

/* Bytes of the K-major staging buffer, (cout + 3 cin) x padded pixels x 2
 * (0 for invalid sizes). */
FWI_API long long fwi_conv3x3_wgrad_tc_stage_bytes(int n, int h, int w, int cin, int cout);

/* Pixel ranges of fwi_conv3x3_wgrad_tc: about one CTA per SM, at most
 * work_floats / (9 cin cout); 0 for invalid sizes. */
FWI_API int fwi_conv3x3_wgrad_tc_splits(int n, int h, int w, int cin, int cout,
                                        long long work_floats);

/* db[c] = sum_p dP[p][c] over npix pixels (dP bf16 [npix][channels]): the
 * pixels split into up to 4 x SM-count ranges whose partial sums go to `work`
 * (work_floats / channels ranges at most; NULL: one range) and are added in
 * range order. */
FWI_API fwi_status fwi_channel_sum(long long npix, int channels, const void *dP, float *db,
                                   float *work, long long work_floats, void *stream);

/* One Adam step (step >= 1) on n float32 parameters: m = b1 m + (1 - b1) g,
 * v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
FWI_API fwi_status fwi_adam_step(long long n, double lr, double beta1, double beta2, double eps,
                                 int step, float *param, const float *grad, float *m, float *v,
                                 void *stream);

/* bf16 weights Wb = W and their transpose for the backward pass,
 * WTb[ci][ky][kx][co] = W[co][2-ky][2-kx][ci]; W float32 [cout][3][3][cin]. */
FWI_API fwi_status fwi_conv3x3_weights_prep(int cout, int cin, const float *W, void *Wb,
                                            void *WTb, void *stream);

/* Per-step biases of a layer: out[i][c] = b[c] + sum_k E[c][k] phi[i][k]
 * (b [channels], E [channels][dim], phi [nsteps][dim], out [nsteps][channels]). */
FWI_API fwi_status fwi_time_bias(int nsteps, int channels, int dim, const float *b, const float *E,
                                 const float *phi, float *out, void *stream);

/* dE[c][k] = db[c] phi[k]: the gradient with respect to E of a bias b + E phi. */
FWI_API fwi_status fwi_time_bias_grad(int channels, int dim, const float *db, const float *phi,
                                      float *dE, void *stream);

/* U-Net resampling (the score model of Sec. 6 is a U-Net), NHWC bf16, FP32
 * arithmetic, channels a multiple of 8, arrays 16-byte aligned.
 * fwi_pool2_bf16: y [n][(h+1)/2][(w+1)/2][C] = s * the sum of x [n][h][w][C]
 *   over each 2 x 2 block inside the image, s = 1 / (cells in the block) for
 *   mode 0 (the mean) and 1 for mode 1 (the sum: the adjoint of mode-0 up2).
 * fwi_up2_bf16: y [n][ho][wo][C] = s * x[n][i/2][j/2] with x [n][(ho+1)/2][(wo+1)/2][C],
 *   s = 1 for mode 0 (nearest neighbour) and 1 / (cells of the block inside
 *   ho x wo) for mode 1 (the adjoint of mode-0 pooling).
 * fwi_add_bf16: z = x + y over `count` elements (a multiple of 8).
 * Errors: FWI_ERR_INVALID_ARG before any launch, FWI_ERR_CUDA. */
FWI_API fwi_status fwi_pool2_bf16(int n, int h, int w, int channels, int mode, const void *x,
                                  void *y, void *stream);
FWI_API fwi_status fwi_up2_bf16(int n, int ho, int wo, int channels, int mode, const void *x,
                                void *y, void *stream);
FWI_API fwi_status fwi_add_bf16(long long count, const void *x, const void *y, void *z,
                                void *stream);

/* ---------------------------------------------------------------- low-fidelity guidance
 * Grid transfers of the low-fidelity guidance surrogate (the multi-fidelity
 * route to cheaper physics guidance, Sec. 7): the W2 potential of the problem
 * coarsened by two (grid spacing and time step doubled, sources and the even
 * receivers at the coarse cells index / 2, nb and nz, nx rounded up, nt / 2
 * samples) is evaluated at R v, and its gradient with respect to v is R^T of
 * the coarse gradient.  All arrays are float32 device arrays; outputs may not
 * alias inputs.  Errors: FWI_ERR_INVALID_ARG before any launch, FWI_ERR_CUDA. */

/* R: vc[b][I][J] = mean of v[b][2I..2I+1][2J..2J+1] inside the grid;
 * v [B][nz][nx], vc [B][ceil(nz/2)][ceil(nx/2)]. */
FWI_API fwi_status fwi_restrict2(int batch, int nz, int nx, const float *v, float *vc,
                                 void *stream);

/* R^T: g[b][i][j] = gc[b][i/2][j/2] / (the number of fine cells averaged into
 * that coarse cell); gc [B][ceil(nz/2)][ceil(nx/2)], g [B][nz][nx]. */
FWI_API fwi_status fwi_restrict2_transpose(int batch, int nz, int nx, const float *gc, float *g,
                                           void *stream);

/* Observations of the coarse problem: dc[b][s][r][m] = d[b][s][2r][2m + 1] for
 * m < nt/2 (fine sample n holds the field at (n+1) dt, coarse sample m at
 * (m+1) 2 dt); d [B][ns][nr][nt], dc [B][ns][ceil(nr/2)][nt/2]. */
FWI_API fwi_status fwi_decimate2(int batch, int ns, int nr, int nt, const float *d, float *dc,
                                 void *stream);

/* The coarse problem itself (host only; no CUDA call): *coarse = *fine with
 * nz, nx, nb halved and rounded up, dz, dx, dt doubled, nt / 2 steps and
 * checkpoint_every halved (rounded up; 0 stays 0); shot i at cell
 * (src_iz[i] / 2, src_ix[i] / 2); the receivers of even index k at
 * (rec_iz[k] / 2, rec_ix[k] / 2), ceil(nr / 2) of them.  Every other field is
 * copied.  The index arrays are the caller's HOST arrays (src_iz, src_ix of
 * fine->ns entries, rec_iz, rec_ix of ceil(fine->nr / 2)); the coarse
 * problem's pointers point into them, so they must outlive its use.
 * The coarse problem is passed to fwi_plan_create, which validates it (CFL
 * with the doubled dt included).
 * Errors: FWI_ERR_INVALID_ARG for NULL arguments, counts out of range or
 * nt < 4. */
FWI_API fwi_status fwi_coarse_problem(const fwi_problem *fine, fwi_problem *coarse, int *src_iz,
                                      int *src_ix, int *rec_iz, int *rec_ix);

/* ---------------------------------------------------------------- tensor-core convolution
 * 3x3 convolution, stride 1, zero padding 1, the dense contraction of a
 * convolutional score model or surrogate used for the guidance of
 * Algorithms 1-2 (the paper's score network is a U-Net, Sec. 6; its surrogate
 * idea is in Sec. 7):
 *   y[b][p][co] = act(bias[co] + sum_{t in 3x3, ci} x[b][p + t][ci] w[co][t][ci])
 * with x outside the image read as 0; act 0: identity, 1: SiLU v / (1 + e^-v).
 * Runs on the tcgen05 tensor cores: BF16 operands, FP32 accumulation.
 *   x    [n][h][w][cin]  bf16 device (NHWC), 16-byte aligned
 *   wt   [cout][3][3][cin] bf16 device (tap t = 3 ky + kx, offsets ky-1, kx-1)
 *   bias [cout] fp32 device, or NULL
 *   y    [n][h][w][cout] device, fp32 (y_bf16 = 0) or bf16 (y_bf16 = 1, round to
 *        nearest even), 16-byte aligned, not aliasing x
 *   status  device int, or NULL: set to FWI_ERR_DEVICE_TIMEOUT if a device-side
 *        wait ran out (the outputs are then not written)
 * cin and cout are positive multiples of 64 (a cout that is a multiple of 256 runs
 * the widest, fastest MMA shape).
 * Errors: FWI_ERR_INVALID_ARG, FWI_ERR_UNSUPPORTED before any launch,
 * FWI_ERR_CUDA. */
FWI_API fwi_status fwi_conv3x3_bf16(int n, int h, int w, int cin, int cout, const void *x,
                                    const void *wt, const float *bias, int act, void *y,
                                    int y_bf16, int *status, void *stream);

/* The same convolution writing a layer's two bf16 outputs at once: the
 * pre-activation p = bf16(bias + sum ...) and its SiLU a = bf16(q / (1 + e^-q))
 * with q = p widened to float -- bit for bit what fwi_conv3x3_bf16 (act 0,
 * bf16 output) followed by fwi_silu_bf16 give, without the second pass over
 * p.  The paper gives no architecture for its networks (Sec. 6); this is the
 * layer of the score networks above (a 3x3 convolution and SiLU).
 *   p, a [n][h][w][cout] bf16 device, 16-byte aligned, neither aliasing x
 * Other arguments and errors as fwi_conv3x3_bf16. */
FWI_API fwi_status fwi_conv3x3_bf16_silu(int n, int h, int w, int cin, int cout, const void *x,
                                         const void *wt, const float *bias, void *p, void *a,
                                         int *status, void *stream);

/* The convolution (no bias) that carries a gradient back through a layer,
 * followed by the SiLU derivative of the layer below in the same epilogue:
 *   dp = bf16(g silu'(q)),  g = bf16(sum ...) widened,  q = p widened,
 *   silu'(q) = sg (1 + q (1 - sg)),  sg = 1 / (1 + e^-q)
 * -- bit for bit fwi_conv3x3_bf16 (act 0, bf16 output) followed by
 * fwi_silu_grad_bf16 on that output and p.
 *   p   [n][h][w][cout] bf16 device: the pre-activation, read only
 *   dp  [n][h][w][cout] bf16 device, written; 16-byte aligned, aliasing neither x nor p
 * Other arguments and errors as fwi_conv3x3_bf16. */
FWI_API fwi_status fwi_conv3x3_bf16_silu_grad(int n, int h, int w, int cin, int cout,
                                              const void *x, const void *wt, const void *p,
                                              void *dp, int *status, void *stream);

/* ---------------------------------------------------------------- reverse diffusion
 * The elementwise steps of one reverse step i -> i-1 of Algorithm 1 (DPS) and
 * Algorithm 2 (OT-guided preconditioned DPS) around the physics gradient:
 *   s      = score of v_i (given, or of a Gaussian prior, below)
 *   v0hat  = (v_i + (1 - abar_i) s) / sqrt(abar_i)                  (Eq. v0hat)
 *   v'     = c_v v_i + c_0 v0hat + sigma_i z                (Algorithms 1-2)
 *   v_phys = clamp(shift + unit v0hat, v_lo, v_hi)          (the physics model)
 *   then, after the caller's fwi_forward -> misfit -> fwi_adjoint_grad at v_phys:
 *   g      = unit dPhi/dv_phys [v_lo <= shift + unit v0hat <= v_hi]  (dPhi/dv0hat)
 *   h      = (g + (1 - abar_i) (ds/dv_i)^T g) / sqrt(abar_i)    (Eq. chain_rule)
 *   and fwi_guided_step(v', v0hat, g, h) with unit = 1 gives v_{i-1}
 *   (Algorithm 2); rho0 = zeta, gamma = 0 and an unreachable tau give
 *   P_i = zeta I, the DPS step of Algorithm 1 (Sec. 5.2).
 * The diffusion state v_i, v0hat, v', g and h live in the normalised space
 * x = (v - shift) / unit; v_phys and dPhi/dv_phys are in m/s.
 * Gaussian prior (a closed-form score model): x_0 ~ N(mu, diag tau2), with
 * the step-i marginal N(sqrt(abar_i) mu, abar_i tau2 + 1 - abar_i) of
 * Eq. vp_transition, so s = -(v_i - sqrt(abar_i) mu) / (abar_i tau2 + 1 - abar_i)
 * and (ds/dv_i)^T g = -g / (abar_i tau2 + 1 - abar_i); the kernels evaluate
 * its v0hat and h in the equivalent cancellation-free forms
 * (sqrt(abar_i) tau2 v_i + (1 - abar_i) mu) / D and sqrt(abar_i) tau2 g / D,
 * D = abar_i tau2 + 1 - abar_i, because the forms above lose most float32
 * digits at high noise (abar_i near 0). */
typedef struct fwi_ddpm_step {
    double abar;    /* abar_i = prod_{j<=i} (1 - beta_j), in (0, 1)              */
    double c_v;     /* sqrt(alpha_i) (1 - abar_{i-1}) / (1 - abar_i)             */
    double c_0;     /* sqrt(abar_{i-1}) beta_i / (1 - abar_i)                    */
    double sigma;   /* sigma_i >= 0                                              */
} fwi_ddpm_step;

typedef struct fwi_diffusion_space {
    double shift, unit;   /* v = shift + unit x (3000, 1500 map 1500..4500 to [-1, 1]) */
    double v_lo, v_hi;    /* clamp of the physics model, v_lo < v_hi                    */
} fwi_diffusion_space;

#define FWI_SIGMA_POSTERIOR 0   /* sigma_i^2 = (1 - abar_{i-1}) beta_i / (1 - abar_i) */
#define FWI_SIGMA_BETA 1        /* sigma_i^2 = beta_i                                 */

/* Coefficients of reverse step i (1 <= i <= n_steps) from the schedule
 * betas[0..n_steps) = beta_1..beta_N (host memory, each in (0, 1)), formed in
 * FP64 on the host (no CUDA call).  Errors: FWI_ERR_INVALID_ARG. */
FWI_API fwi_status fwi_ddpm_coefficients(const double *betas, int n_steps, int i,
                                         int sigma_mode, fwi_ddpm_step *out);

/* v0hat, v' and v_phys of reverse step `step` for B instances of ncell cells
 * (all [B][ncell] device arrays, float32).
 *   v_i    the current state; z the standard normal draws of this step
 *   score  the score at v_i, or NULL for the Gaussian prior of mu, tau2
 *          ([ncell] device arrays shared by the batch; ignored when score is
 *          given; tau2 >= 0)
 *   v0hat, v_prime, v_phys  written (none may alias an input)
 * Errors: FWI_ERR_INVALID_ARG before any launch, FWI_ERR_CUDA. */
FWI_API fwi_status fwi_ddpm_proposal(int batch, int ncell, const fwi_ddpm_step *step,
                                     const fwi_diffusion_space *space, const float *v_i,
                                     const float *score, const float *mu, const float *tau2,
                                     const float *z, float *v0hat, float *v_prime,
                                     float *v_phys, void *stream);

/* g and h of reverse step `step` ([B][ncell] device arrays, float32).
 *   v0hat   from fwi_ddpm_proposal; g_phys = dPhi/dv at v_phys (1/(m/s))
 *   vjp     (ds/dv_i)^T g of the caller's score model, or NULL: then the
 *           Gaussian prior's, from tau2 ([ncell]), or 0 when tau2 is NULL too
 *           (a score that does not depend on v_i).  A network's vjp needs g
 *           first: call once with both NULL, form the vjp from g, call again.
 *   g, h    written (may not alias an input)
 * Errors: FWI_ERR_INVALID_ARG before any launch, FWI_ERR_CUDA. */
FWI_API fwi_status fwi_ddpm_guidance(int batch, int ncell, const fwi_ddpm_step *step,
                                     const fwi_diffusion_space *space, const float *v0hat,
                                     const float *g_phys, const float *vjp, const float *tau2,
                                     float *g, float *h, void *stream);

/* A reverse step whose launches replay from one CUDA graph: the step index
 * lives in device memory and the coefficients in a device table, so the same
 * launches serve every step of a chain.
 * fwi_ddpm_table (host only): table [(n_steps + 1) x FWI_DDPM_RECORD_FLOATS]
 *   floats of host memory receives record i (1 <= i <= n_steps) = the float
 *   coefficients fwi_ddpm_proposal / fwi_ddpm_guidance use at step i with
 *   this space (record 0 is zero); the caller copies it to the device.
 * fwi_ddpm_proposal_at / fwi_ddpm_guidance_at: fwi_ddpm_proposal /
 *   fwi_ddpm_guidance at step i = *step (a device int), coefficients from the
 *   device table, the draws of the proposal at z + i z_stride; when i lies
 *   outside 1..n_steps the kernels write nothing.
 * fwi_ddpm_step_down: *step -= 1 (one thread), the last launch of a step.
 * Errors: FWI_ERR_INVALID_ARG before any launch, FWI_ERR_CUDA. */
#define FWI_DDPM_RECORD_FLOATS 12
FWI_API fwi_status fwi_ddpm_table(const double *betas, int n_steps, int sigma_mode,
                                  const fwi_diffusion_space *space, float *table);
FWI_API fwi_status fwi_ddpm_proposal_at(int batch, int ncell, const float *table, const int *step,
                                        int n_steps, const float *v_i, const float *score,
                                        const float *mu, const float *tau2, const float *z,
                                        long long z_stride, float *v0hat, float *v_prime,
                                        float *v_phys, void *stream);
FWI_API fwi_status fwi_ddpm_guidance_at(int batch, int ncell, const float *table, const int *step,
                                        int n_steps, const float *v0hat, const float *g_phys,
                                        const float *vjp, const float *tau2, float *g, float *h,
                                        void *stream);
FWI_API fwi_status fwi_ddpm_step_down(int *step, void *stream);

/* Score of a low-rank Gaussian prior x_0 ~ N(mu, U^T diag(lam) U + s2 I) at
 * step i = *step of a table (fwi_ddpm_table): the step-i marginal is
 * N(sqrt(abar_i) mu, C), C = abar_i Sigma + (1 - abar_i) I (Eq. vp_transition),
 * and with the rows of U orthonormal
 *   out = -C^-1 (x - sqrt(abar_i) mu)     (mu given: the score s_i(x))
 *   out = -C^-1 x                        (mu NULL: (ds_i/dx)^T x, the score's
 *                                          vector-Jacobian product applied to x)
 * through the eigenvalues c_j = abar (lam_j + s2) + 1 - abar along the rows of
 * U and c_perp = abar s2 + 1 - abar across them.  A stand-in for a trained
 * score (the paper's is a U-Net, Sec. 6) whose samples are smooth.
 *   U [k][ncell], lam [k], mu [ncell], x and out [batch][ncell] (fp32, device;
 *   out may not alias x); work: batch x k floats of device scratch; k = 0 is
 *   the isotropic prior N(mu, s2 I).  Outside 1..n_steps nothing is written.
 * Sums in a fixed order: a second call gives the same bits.
 * Errors: FWI_ERR_INVALID_ARG (s2 > 0, sizes, NULL pointers), FWI_ERR_CUDA. */
FWI_API fwi_status fwi_lowrank_score_at(int batch, int ncell, int k, const float *U,
                                        const float *lam, double s2, const float *x,
                                        const float *mu, const float *table, const int *step,
                                        int n_steps, float *work, float *out, void *stream);

/* ---------------------------------------------------------------- learned forward surrogate
 * Data-side steps of a convolutional encoder-decoder that maps a velocity model
 * to the seismograms of the FD solver: the surrogate route to cheaper guidance
 * that Sec. 7 proposes, used in the early reverse steps of Algorithm 2 (Sec.
 * 5.2), with the FD solver as its check and fallback.  The six convolutions run
 * on fwi_conv3x3_bf16 (with fwi_silu_bf16, fwi_silu_grad_bf16, fwi_add_bf16,
 * fwi_conv3x3_wgrad_tc, fwi_channel_sum and fwi_adam_step for training).
 * Layout: model b is column (b mod m) of image (b / m), an image being nx pixels
 * high (the model's columns x) and m pixels wide; the convolution weights keep
 * their horizontal taps at zero (fwi_sur_weights_prep), so each model only
 * couples its own columns x - 1, x, x + 1 and the m models of an image never
 * mix.  nimg = ceil(nmod / m).  All arrays are device arrays; bf16 tensors are
 * NHWC and 16-byte aligned where the convolution reads them.
 * Errors: FWI_ERR_INVALID_ARG before any launch, FWI_ERR_CUDA. */

/* X [nimg][nx][m][c0] bf16 = in_scale v[b][c][x] + in_shift for channel c < nz,
 * G[x][c] (fp32 [nx][c0], the geometry channels) above; columns past nmod are 0.
 * c0 is a multiple of 64 and >= nz.  v [nmod][nz][nx] fp32. */
FWI_API fwi_status fwi_sur_pack(int nmod, int m, int nz, int nx, int c0, float in_scale,
                                float in_shift, const float *v, const float *G, void *X,
                                void *stream);

/* dv[b][z][x] = in_scale dX[b / m][x][b mod m][z]: the gradient at the models
 * from the fp32 gradient dX [nimg][nx][m][c0] at the packed input. */
FWI_API fwi_status fwi_sur_unpack_grad(int nmod, int m, int nz, int nx, int c0, float in_scale,
                                       const float *dX, float *dv, void *stream);

/* d[b][s][r][t] = amp sign(y) (e^|y| - 1) with y = Y[b / m][rec_ix[r]][b mod m][s nt + t]:
 * the traces from the fp32 output Y [nimg][nx][m][cout] (ns nt <= cout, amp > 0),
 * rec_ix [nr] device ints (the receivers' columns, distinct). */
FWI_API fwi_status fwi_sur_traces(int nmod, int m, int ns, int nr, int nt, int nx, int cout,
                                  float amp, const int *rec_ix, const float *Y, float *d,
                                  void *stream);

/* dY [nimg][nx][m][cout] bf16 = scale adj[b][s][r][t] amp e^|y| at column
 * x = rec_ix[r], channel s nt + t, and 0 at every other entry: the transpose of
 * the derivative of fwi_sur_traces at Y applied to adj [nmod][ns][nr][nt].
 * col_rec [nx] device ints: the receiver at column x, or -1. */
FWI_API fwi_status fwi_sur_output_grad(int nmod, int m, int ns, int nr, int nt, int nx,
                                       int cout, float amp, float scale, const int *col_rec,
                                       const float *Y, const float *adj, void *dY,
                                       void *stream);

/* Yt [nimg][nx][m][cout] fp32 = sign(d) log(1 + |d| / amp) at the entries
 * fwi_sur_traces reads (the regression target of Y), 0 elsewhere. */
FWI_API fwi_status fwi_sur_target(int nmod, int m, int ns, int nr, int nt, int nx, int cout,
                                  float amp, const int *col_rec, const float *d, float *Yt,
                                  void *stream);

/* loss[0] = mean over the n entries of (Y - Yt)^2 and dY = bf16(2 (Y - Yt) / n);
 * work: fp32 scratch for up to 608 per-CTA partials, added in a fixed order. */
FWI_API fwi_status fwi_sur_loss(long long n, const float *Y, const float *Yt, float *loss,
                                void *dY, float *work, long long work_floats, void *stream);

/* Along the image only (bf16 NHWC, channels a multiple of 8):
 * fwi_pool_h_bf16: y [n][(h+1)/2][w][C] = s * (x[2I] + x[2I+1]) over the rows
 *   inside the image, s = 1 / rows (mode 0, mean) or 1 (mode 1, the adjoint of
 *   mode-0 upsampling);
 * fwi_up_h_bf16: y [n][ho][w][C] = s * x[i / 2], s = 1 (mode 0) or 1 / (the rows
 *   of block i / 2 inside ho) (mode 1, the adjoint of mean pooling). */
FWI_API fwi_status fwi_pool_h_bf16(int n, int h, int w, int channels, int mode, const void *x,
                                   void *y, void *stream);
FWI_API fwi_status fwi_up_h_bf16(int n, int ho, int w, int channels, int mode, const void *x,
                                 void *y, void *stream);

/* From three-tap fp32 weights W3 [cout][3][cin] (tap k couples pixel x + k - 1):
 * W [cout][3][3][cin] bf16 with W[co][ky][1][ci] = W3[co][ky][ci] and the
 * horizontal taps zero, and its transpose WT [cin][3][3][cout] (WT[ci][ky][kx][co]
 * = W[co][2-ky][2-kx][ci], the weights of the backward convolution). */
FWI_API fwi_status fwi_sur_weights_prep(int cout, int cin, const float *W3, void *W, void *WT,
                                        void *stream);

/* dW3[co][ky][ci] = dW[co][ky][1][ci]: the gradient of the three-tap weights
 * from a 3 x 3 weight gradient dW [cout][3][3][cin] (fp32). */
FWI_API fwi_status fwi_sur_wgrad_centre(int cout, int cin, const float *dW, float *dW3,
                                        void *stream);

/* The FD solver as the check of a surrogate's guidance gradient (Sec. 7's
 * surrogate route, gated per noise level of Algorithm 2): per model b,
 *   err[b] = ||g_b - g_ref_b||_2 / ||g_ref_b||_2
 * over the n floats of model b (g, g_ref [nmod][n] fp32, device; err [nmod]
 * fp32, device).  Sums in double in a fixed order (one CTA a model): a second
 * call gives the same bits.  A zero reference gives 0 if g_b is zero too,
 * else +inf.  nmod, n >= 1 and non-NULL pointers, else FWI_ERR_INVALID_ARG. */
FWI_API fwi_status fwi_rel_error(int nmod, long long n, const float *g, const float *g_ref,
                                 float *err, void *stream);

/* Message of the last failing call on this thread ("" if none). */
FWI_API const char *fwi_last_error(void);

/* FWI_VERSION of the loaded library. */
FWI_API int fwi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FWI_H */
