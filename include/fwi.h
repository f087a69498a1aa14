/*
 * fwi.h -- C ABI of libfwi.so, the GB300 (sm_103a) Scheme III hot path of
 *   Bharadwaj, Mulder & Drijkoningen, "A parameterization analysis for acoustic
 *   full-waveform inversion of sub-wavelength anomalies" (arXiv:1804.01184).
 *
 * Time-domain staggered-grid finite-difference modelling of the 2-D variable-density
 * acoustic wave equation (Sec. "Scheme III"; the operator of eq. param_full), its Born
 * linearisation, and the adjoint wavefield with the zero-lag cross-correlation fused into
 * the gradient, converted by the chain rule to every parameterization of Table 1
 * (Sec. "Modelling and Inversion").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every array argument is a DEVICE pointer owned by the caller, except the fwi_grid,
 *    fwi_sources and fwi_receivers structs themselves (host memory, read during the call).
 *  - The library allocates nothing.  Scratch memory is the caller's `work` buffer of
 *    `work_bytes` bytes (256-byte aligned); fwi_workspace_bytes() says how much an
 *    operation needs.  A larger buffer lets fwi_gradient keep more wavefield history
 *    (fewer recomputed forward steps); the plan is a deterministic function of the sizes.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *    default stream).  Results are valid once the stream has reached them.  Argument errors
 *    that the host can see return an error code at once; errors that need the data (a
 *    contrast with 1 + xi <= 0, a CFL violation, a position outside the grid) are recorded
 *    in the workspace and returned by fwi_status().
 *  - Grids are row-major [nz][nx], x fastest.  The physical node (ix, iz) sits at
 *    x = ix*dx, z = iz*dx metres.  The computational grid adds `sponge` absorbing cells on
 *    every side; those cells take the model of the nearest physical cell.
 *  - Return value: FWI_OK (0) or a negative FWI_E* code; fwi_last_error() gives a message
 *    (thread-local, valid until the next call on the same thread).
 *  - Work on different streams must use different workspaces.
 */
#ifndef FWI_H_
#define FWI_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FWI_OK        0
#define FWI_EINVAL   -1   /* bad size, null pointer, 1 + xi <= 0, position off the grid */
#define FWI_ECFL     -2   /* dt above the stability limit of the stencil for the model */
#define FWI_ENOMEM   -3   /* workspace smaller than the operation's minimum             */
#define FWI_ETIMEOUT -4   /* a bounded device-side wait expired (fwi_fborn_status) */
#define FWI_ECUDA    -5   /* a CUDA runtime call failed                                 */

/* Parameterizations of Table 1; contrasts xi = (m - m_o)/m_o of the named pair. */
typedef enum {
    FWI_VP_RHO = 0,      /* (A) P-wave speed, density            */
    FWI_IP_RHO = 1,      /* (B) impedance Ip = rho vp, density   */
    FWI_VP_IP = 2,       /* (C) P-wave speed, impedance          */
    FWI_K_RHO = 3,       /* (D) bulk modulus K = rho vp^2, density */
    FWI_INVK_INVRHO = 4  /* (E) 1/K, 1/rho                        */
} fwi_param;

/* Operations, for fwi_workspace_bytes(). */
typedef enum { FWI_OP_MODEL = 0, FWI_OP_BORN = 1, FWI_OP_ADJOINT = 2, FWI_OP_GRADIENT = 3 } fwi_op;

typedef struct {
    int nx, nz;        /* physical nodes (>= 2 each)                                      */
    int sponge;        /* absorbing cells added on each side (>= 0)                       */
    int order;         /* spatial order of the staggered stencil: 4 or 8                  */
    int nt;            /* time steps (>= 1)                                               */
    double dx;         /* grid spacing [m], the same in x and z                           */
    double dt;         /* time step [s]                                                   */
    double vp_o;       /* reference P-wave speed [m/s] (homogeneous reference medium)     */
    double rho_o;      /* reference density [kg/m^3]                                      */
    double sponge_v;   /* speed used for the sponge profile [m/s] (<= 0: vp_o)            */
    double sponge_R;   /* target reflection of the sponge (0 < R < 1; <= 0: 1e-3)         */
} fwi_grid;

/* One point source per shot (explosive: volume injection into the pressure equation,
 * scaled by the local bulk modulus, bilinear weights / dx^2).  wavelet[n] is the source
 * time function at t = (n + 1/2) dt, shared by all shots. */
typedef struct {
    int ns;                 /* shots                                                   */
    const float *xy;        /* device [ns][2]: (x, z) in metres                        */
    const float *wavelet;   /* device [nt]                                             */
} fwi_sources;

/* Pressure receivers, shared by all shots; sample n of a trace is the bilinear
 * interpolation of p at time (n + 1) dt. */
typedef struct {
    int nr;
    const float *xy;        /* device [nr][2]: (x, z) in metres                        */
} fwi_receivers;

/* Bytes of workspace an operation needs.  budget_bytes = 0 asks for the minimum; otherwise
 * the result is the largest plan that fits in budget_bytes (at least the minimum).  Returns
 * 0 on invalid arguments. */
size_t fwi_workspace_bytes(const fwi_grid *g, int ns, int nr, fwi_op op, size_t budget_bytes);

/* Forward modelling (Sec. Scheme III: the forward wavefield of eq. param_full).
 *   xi_a, xi_b : [nz][nx] float32 contrasts of the model in parameterization pz (Table 1)
 *   traces     : [ns][nr][nt] float32 output pressure traces
 * Computes in FP32. */
int fwi_model(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b,
              const fwi_sources *src, const fwi_receivers *rec, float *traces,
              void *work, size_t work_bytes, void *stream);

/* Born modelling: the exact linearisation of fwi_model's discrete scheme around (xi_a, xi_b)
 * applied to the contrast perturbation (dxi_a, dxi_b) (the Born idea of eq. param_born,
 * applied to Scheme III's discretisation).  dtraces: [ns][nr][nt] float32. */
int fwi_born(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b,
             const float *dxi_a, const float *dxi_b, const fwi_sources *src,
             const fwi_receivers *rec, float *dtraces, void *work, size_t work_bytes,
             void *stream);

/* Adjoint modelling: for a trace-space vector residual [ns][nr][nt] (float32) returns the
 * gradient of sum(residual * traces) w.r.t. the contrasts of all five parameterizations,
 * grads [5][2][nz][nx] float64 (index [pz][0] = first parameter of pair pz, [pz][1] the
 * second), evaluated at the model (pz, xi_a, xi_b).  The adjoint wavefield is
 * cross-correlated with the forward wavefield at every step inside the adjoint kernels
 * (Sec. "Modelling and Inversion": gradient by adjoint modelling, then the chain rule).
 * Accumulation: each adjoint step's products go into FP32 per-shot fields; after every
 * chunk of steps (64 by default, fwi_set_accumulation) and after the last step those fields
 * are flushed into FP64 running sums over shots and cleared, so no FP32 sum spans more than
 * one chunk.  The flush adds a chunk's per-shot values with a compensated (TwoSum) FP32 sum,
 * exact to about twice FP32 precision, and adds that to the FP64 sum; its order is fixed, so
 * results are bitwise reproducible.  The density chain rule and the parameterization chain
 * rules run in FP64. */
int fwi_adjoint(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b,
                const fwi_sources *src, const fwi_receivers *rec, const float *residual,
                double *grads, void *work, size_t work_bytes, void *stream);

/* Misfit and gradient (Sec. "Modelling and Inversion"): J = 1/2 sum (d_mod - data)^2 over
 * shots, receivers and samples (time-domain reading of the least-squares misfit), written
 * to misfit (device, 1 float64), and its gradient for all five parameterizations, grads
 * [5][2][nz][nx] float64.  data: [ns][nr][nt] float32 observed traces. */
int fwi_gradient(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b,
                 const fwi_sources *src, const fwi_receivers *rec, const float *data,
                 double *misfit, double *grads, void *work, size_t work_bytes, void *stream);

/* Least-squares misfit of one set of traces (Sec. "Modelling and Inversion"): writes
 * J = 1/2 sum_k (traces[k] - data[k])^2, accumulated in FP64 in a fixed order, to *misfit
 * (device, 1 float64).  traces, data: `count` float32 values (device).  Allocates nothing;
 * asynchronous on `stream`.  Used for misfit surfaces over many forward models (error bowls). */
int fwi_misfit(const float *traces, const float *data, long long count, double *misfit, void *stream);

/* fwi_gradient with a weight per trace: J = 1/2 sum_{s,r,n} w[s][r] (d_mod - data)^2, whose
 * adjoint source is w (d_mod - data).  weights: [ns][nr] float32 (device), null = all 1 (then
 * identical to fwi_gradient).  A 0/1 weight selects the traces of a limited aperture, e.g. a
 * range of scattering angles (Sec. "Hierarchical Inversion"). */
int fwi_gradient_weighted(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b,
                          const fwi_sources *src, const fwi_receivers *rec, const float *data,
                          const float *weights, double *misfit, double *grads, void *work, size_t work_bytes,
                          void *stream);

/* fwi_misfit with a weight per trace: J = 1/2 sum_t w[t] sum_n (traces[t][n] - data[t][n])^2
 * over ntraces traces of nt samples; weights null = all 1. */
int fwi_misfit_weighted(const float *traces, const float *data, long long ntraces, int nt, const float *weights,
                        double *misfit, void *stream);

/* Waits for `stream` and returns the data-dependent status recorded by the last operation
 * that used `work` (FWI_OK, FWI_EINVAL, FWI_ECFL), then clears it. */
int fwi_status(void *work, void *stream);

/* Message for the last error on this thread ("" if none). */
const char *fwi_last_error(void);

/* Kernels launched by the last operation on this thread (for launch accounting). */
long long fwi_launch_count(void);

/* Forward modelling without any device allocation (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc or any allocating routine where they need a
 * forward model: a service whose device memory is fixed at start-up, a plugin inside a
 * framework that owns all device memory, code where an allocation may block on other work.
 * Same arguments and results as fwi_model, without work/work_bytes: the scratch is a
 * file-scope __device__ array of FWI_NOALLOC_SCRATCH_BYTES (64 MiB) in the library image,
 * which every GPU that loads the library holds until the process exits.
 *  - Limit: the grid, shot and receiver counts must fit that scratch with one shot at a
 *    time (fwi_workspace_bytes(g, ns, nr, FWI_OP_MODEL, 0) <= FWI_NOALLOC_SCRATCH_BYTES,
 *    e.g. 201 x 201 + 40-cell sponge with 64 shots); larger problems return FWI_ENOMEM
 *    with a message in fwi_last_error().
 *  - The first call on a device resolves the scratch address on that device (the device
 *    must be current); make that first call before any stream capture.
 *  - All calls share the one scratch array per device and it keeps the last call's
 *    contents; the call clears what must start at zero.  Calls whose work overlaps on the
 *    GPU (different streams, or different host threads) race on the scratch: serialise them.
 *  - The data-dependent checks fwi_model records in its workspace (1 + xi <= 0, CFL, points
 *    off the grid) land in the scratch; fwi_status_noalloc() reads them.  Host-visible
 *    argument errors are returned as usual.
 */
#define FWI_NOALLOC_SCRATCH_BYTES (64u << 20)
int fwi_model_noalloc(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b,
                      const fwi_sources *src, const fwi_receivers *rec, float *traces, void *stream);

/* fwi_status for fwi_model_noalloc (no counterpart in the paper): waits for `stream` and
 * returns the data-dependent status the last fwi_model_noalloc call on the current device
 * recorded in the built-in scratch (FWI_OK, FWI_EINVAL, FWI_ECFL), then clears it; FWI_OK
 * when no such call has run on this device.  Allocates nothing. */
int fwi_status_noalloc(void *stream);

/* Wavefield checkpointing (no counterpart in the paper: the adjoint needs the forward
 * wavefield, Sec. "Scheme III").  every > 0: plans made afterwards for fwi_adjoint and
 * fwi_gradient keep (p, vx, vz) checkpoints every `every` steps and recompute each segment's
 * pressure history before its adjoint, whatever the budget allows; 0 (default): the planner
 * keeps the whole history when it fits and otherwise checkpoints every ~sqrt(3 nt) steps.
 * Gradients are identical either way. */
int fwi_set_checkpoint(int every);

/* Phase ranges for timeline tools (no counterpart in the paper).  enable = 1: every operation
 * marks the host thread's enqueueing of its phases with NVTX ranges ("fwi:model_build",
 * "fwi:forward", "fwi:recompute", "fwi:adjoint", "fwi:reduce", "fwi:born",
 * "fwi:engine_iteration"), visible to timeline profilers; 0 (default): none.  Results are
 * identical either way. */
int fwi_trace(int enable);

/* Ranges opened per phase since the last report, one "name count" line each, written to buf
 * (at most len - 1 bytes, NUL-terminated; buf may be NULL to only reset); returns the length of
 * the full report. */
int fwi_trace_report(char *buf, size_t len);

/* Length of the FP32 accumulation chunks of the gradient (no counterpart in the paper; the
 * time integral of the zero-lag cross-correlation of Sec. "Modelling and Inversion" is a sum
 * over all steps).  steps > 0: plans made afterwards flush the FP32 per-shot accumulators
 * into the FP64 sums after every `steps` adjoint steps (and after the last); 0 restores the
 * default of 64.  A value of at least nt keeps one FP32 sum over the whole record.  Returns
 * FWI_EINVAL for steps < 0. */
int fwi_set_accumulation(int steps);

/* Launch-shape tuning (no counterpart in the paper: the tile-shape autotuner's hook).  By
 * default the strip height of the streaming kernels is tuned online: for each launch shape
 * the first launches try the height an occupancy rule picks (strips that just fill the warps
 * the GPU holds at once) and a few others, each timed twice with CUDA events on the
 * launching stream without blocking, and the shape then keeps its fastest height (launches
 * under stream capture are not timed).  tz > 0 (any number of rows) fixes the height instead,
 * for plans made afterwards by any thread (0 restores tuning); variant picks the register
 * budget per thread of the single-job kernels (0 = default: unbounded, 170 for the forward
 * kernel; 1 = 128; 2 = 170).  Results are
 * bitwise identical for every setting; only speed changes. */
int fwi_set_tile(int tz, int variant);

/* ---------------------------------------------------------------------------------------
 * Batching engine (no counterpart in the paper: the throughput layer for many independent
 * problems -- shots of different surveys, line searches, sweeps over models).
 *
 * An engine owns a caller-allocated device arena (256-byte aligned; the engine never
 * allocates device memory) and one stream.  fwi_engine_submit() queues a job; jobs are
 * admitted first-in first-out whenever their workspace (the plan the job's work_budget
 * gives) fits into the free part of the arena (first-fit), and it returns to the arena
 * when they finish, so new jobs join while earlier ones still run.
 * fwi_engine_run() advances every admitted job by one time step per iteration; the steps of
 * all running jobs of one kind go out as one batched kernel launch (up to 96 jobs per
 * launch, larger batches split).  Each job computes exactly what the matching single-job
 * call (fwi_model, fwi_born, fwi_gradient) computes with a workspace of
 * fwi_workspace_bytes(grid, ns, nr, op, work_budget) bytes: its results are bitwise
 * independent of the other jobs it runs beside.
 *
 * A job's input arrays (contrasts, geometry, wavelet, data) and outputs stay owned by the
 * caller and must stay valid until the job's ticket comes back as done.  Data-dependent
 * errors (CFL, points off the grid) are recorded in the job's workspace and are not
 * reported by the engine: check inputs with the single-job API first.  An engine is used
 * from one host thread at a time.
 * ------------------------------------------------------------------------------------- */
typedef enum { FWI_JOB_MODEL = 0, FWI_JOB_BORN = 1, FWI_JOB_GRADIENT = 2 } fwi_job_kind;

typedef struct {
    fwi_job_kind kind;
    fwi_grid grid;
    fwi_param pz;
    const float *xi_a, *xi_b;      /* [nz][nx] contrasts (device) */
    const float *dxi_a, *dxi_b;    /* BORN: [nz][nx] perturbation (device) */
    fwi_sources src;               /* device pointers, as for fwi_model */
    fwi_receivers rec;
    float *traces;                 /* MODEL, BORN: [ns][nr][nt] output (device) */
    const float *data;             /* GRADIENT: [ns][nr][nt] observed traces (device) */
    double *misfit;                /* GRADIENT: 1 float64 output (device) */
    double *grads;                 /* GRADIENT: [5][2][nz][nx] float64 output (device) */
    size_t work_budget;            /* the job runs the plan fwi_workspace_bytes(grid, ns, nr, op,
                                      work_budget) gives (0: the smallest plan) */
} fwi_job;

typedef struct fwi_engine fwi_engine;

/* Creates an engine over `arena` (device, arena_bytes, 256-byte aligned) and `stream`. */
int fwi_engine_create(fwi_engine **engine, void *arena, size_t arena_bytes, void *stream);

/* Validates and queues a copy of *job; *ticket receives its id (1, 2, ...).  FWI_EINVAL for
 * invalid arguments, FWI_ENOMEM when the job's workspace exceeds the arena. */
int fwi_engine_submit(fwi_engine *engine, const fwi_job *job, long long *ticket);

/* Runs up to `iterations` engine iterations (admission, one time step of every running job,
 * retirement), enqueued on the engine's stream without waiting for the GPU.  Writes to
 * done[0 .. *ndone) the tickets (at most max_done per call; the rest come back on later
 * calls) of jobs whose results are complete on the device.  When no job is left queued or
 * running, the call waits for the GPU to finish the outstanding ones.  A call first waits
 * for the GPU to finish the work of the call before the previous one, so the host never
 * runs more than one call's iterations ahead of the GPU (what bounds the wait of a job
 * submitted between calls).  Returns FWI_OK or the first failure (FWI_ECUDA, ...) of the work
 * it enqueued; after a failure the engine's jobs are undefined: destroy it. */
int fwi_engine_run(fwi_engine *engine, int iterations, long long *done, int max_done, int *ndone);

/* Cancels a job that is queued or running (a request the caller no longer wants; no
 * counterpart in the paper).  A queued job leaves the queue.  A running job stops being
 * advanced and its arena block returns to the free list at once: the work already enqueued
 * for it on the engine's stream still runs, before anything enqueued later, so the block is
 * reused safely; its outputs are left incomplete and its ticket never comes back as done.
 * The job's input and output arrays stay in use until the engine's stream has passed this
 * call (synchronise it, or record an event, before freeing them).  The other jobs' results
 * do not change.  Returns FWI_EINVAL for a ticket that is not queued or running. */
int fwi_engine_cancel(fwi_engine *engine, long long ticket);

/* Jobs queued, running (admitted, not retired) and retired but not yet reported as done;
 * bytes of the arena in use. */
int fwi_engine_info(fwi_engine *engine, int *queued, int *running, int *pending, size_t *arena_used);

/* Waits for the engine's stream and frees the engine (not the arena). */
int fwi_engine_destroy(fwi_engine *engine);

/* Per-launch timing (no counterpart in the paper: measurement support).  While enabled
 * (enable = 1), every kernel launch of the library is bracketed by a CUDA event pair recorded
 * on the launching stream; enable = N > 1 samples one launch in N of each kernel (the first of
 * every N since the call), which keeps the events' own cost off a timed loop; 0 disables.
 * fwi_profile_report() waits for those events, writes one line per kernel
 * "name launches timed_launches timed_ms\n" (launches since profiling was enabled or last
 * reported; the device time summed over the timed ones) into buf (at most len bytes, NUL-terminated), resets the
 * record and returns the report length (or a negative FWI_E* code). */
int fwi_profile(int enable);
int fwi_profile_report(char *buf, size_t len);

/* ---------------------------------------------------------------------------------------
 * Frequency-domain Born modelling of Schemes I and II (Sec. "Modelling and Inversion",
 * eqn:param_born and eqn:param_pfreq1; Sec. "Point-scatterer Analysis", eqn:param_Hker).
 *
 * The reference medium is homogeneous (vp_o, rho_o, K_o = rho_o vp_o^2).  Its Green function
 * is G_o(x; p) = (i rho_o / 4) H_0^(1)(k |x - p|), k = 2 pi f / vp_o (e^{-i w t} convention;
 * the sign that makes the printed Lippmann-Schwinger equation exact; misfits, gradients and
 * Hessians do not depend on it).  The modelling vector of node x for source s and receiver r
 * is W = [w^2/K_o G_o(x; r) G_o(x; s),  -(1/rho_o) grad G_o(x; r) . grad G_o(x; s)], and the
 * Born data are
 *     p[f][s][r] = S_f ( G_o(x_r; x_s) + dx^2 sum_x W(x) . (xi_{1/K}(x), xi_{1/rho}(x)) ),
 * where (xi_{1/K}, xi_{1/rho}) are the contrasts of parameterization pz mapped LINEARLY
 * (scheme FWI_FB_LINEAR, Scheme I: the linearization at zero contrast behind Table 3; for the
 * impedance -(xi_{1/K} + xi_{1/rho})/2) or EXACTLY (FWI_FB_NONLINEAR, Scheme II: Table 2).
 * The misfit is J = 1/2 sum_{f,s,r} |p - q|^2 over the given frequencies (all w > 0).
 *
 * Model grid: nx x nz nodes, x fastest, node (i, j) at (x0 + i dx, z0 + j dx) metres;
 * sources and receivers are points anywhere at least dx/2 from every node.
 * Complex arrays are interleaved float pairs (re, im).  Device pointers as elsewhere,
 * except the host arrays of fwi_fborn_tables. */
typedef struct {
    int nx, nz;          /* model nodes */
    int nf;              /* frequencies */
    double dx;           /* node spacing (m) */
    double x0, z0;       /* coordinates of node (0, 0) (m) */
    double vp_o, rho_o;  /* homogeneous reference medium (m/s, kg/m^3) */
} fwi_fgrid;

#define FWI_FB_LINEAR    1   /* Scheme I map  */
#define FWI_FB_NONLINEAR 2   /* Scheme II map */

/* Bytes of the workspace of a geometry of ns sources and nr receivers on grid g (0 if the
 * sizes are invalid): Green tables G_o and dG_o/dr for every (frequency, point, node) --
 * 16 nf (ns + nr) nx nz bytes -- plus per-call scratch. */
size_t fwi_fborn_workspace_bytes(const fwi_fgrid *g, int ns, int nr);

/* Fills the workspace for one acquisition: freqs [nf] (Hz, > 0), spectrum [nf] complex
 * S(w_f), src_xy [ns][2], rec_xy [nr][2] -- HOST arrays, copied before the call returns --
 * and the Green tables of every source and receiver at every node and frequency (double-
 * precision Bessel functions, stored as float pairs).  FWI_EINVAL for a point within dx/2 of
 * a node, a non-positive frequency or bad sizes; FWI_ENOMEM if work_bytes is too small.  The
 * other fwi_fborn_* calls read this workspace with the same (g, ns, nr). */
int fwi_fborn_tables(const fwi_fgrid *g, const double *freqs, const float *spectrum, const float *src_xy, int ns,
                     const float *rec_xy, int nr, void *work, size_t work_bytes, void *stream);

/* Born data p [nf][ns][nr] complex (eqn:param_pfreq1) of the contrasts xi_a, xi_b [nz][nx] of
 * parameterization pz under `scheme`; incident != 0 adds the direct field S_f G_o(x_r; x_s)
 * (0: the scattered part only).  FWI_EINVAL for bad arguments (a contrast with 1 + xi <= 0 under
 * the exact map gives non-finite data). */
int fwi_fborn_model(const fwi_fgrid *g, int ns, int nr, int scheme, fwi_param pz, const float *xi_a,
                    const float *xi_b, int incident, void *work, float *data, void *stream);

/* Misfit J (one double) and its gradient grad [2][nz][nx] (double; dJ/dxi_a then dJ/dxi_b)
 * at the contrasts xi_a, xi_b of pz under `scheme`, against observed data q [nf][ns][nr]
 * complex (with the direct field, as fwi_fborn_model(incident = 1) gives it):
 * dJ/dxi_{1/K,1/rho}(x) = Re sum conj(p - q) S_f W(x) dx^2, then the chain rule through
 * the map's Jacobian at each node. */
int fwi_fborn_gradient(const fwi_fgrid *g, int ns, int nr, int scheme, fwi_param pz, const float *xi_a,
                       const float *xi_b, const float *data_obs, void *work, double *misfit, double *grad,
                       void *stream);

/* fwi_fborn_gradient and fwi_fborn_hessian(pz, jx, jz) in one call: misfit, gradient [2][nz][nx]
 * and the Scheme I Hessian terms H [2][2][nz][nx] of node (jx, jz), both as the two calls give
 * them, with the Hessian's sums formed in the gradient's pass over the Green tables (one table
 * pass instead of two).  FWI_EINVAL for bad arguments, a node off the grid or more than 2048
 * sources + receivers. */
int fwi_fborn_gradient_hessian(const fwi_fgrid *g, int ns, int nr, int scheme, fwi_param pz, const float *xi_a,
                               const float *xi_b, const float *data_obs, int jx, int jz, void *work, double *misfit,
                               double *grad, double *H, void *stream);

/* The misfit J alone (one double), as fwi_fborn_gradient computes it: the data contraction,
 * the residual and the reduction, without the gradient pass (line searches). */
int fwi_fborn_misfit(const fwi_fgrid *g, int ns, int nr, int scheme, fwi_param pz, const float *xi_a,
                     const float *xi_b, const float *data_obs, void *work, double *misfit, void *stream);

/* Scheme I Hessian terms H [2][2][nz][nx] (double): H[a][b][i] = d^2 J / d xi_a(x_i) d xi_b(x_j)
 * for the fixed node j = (jx, jz) and every node i -- the real part of
 * dx^4 sum_f |S_f|^2 sum_{s,r} conj(W_a(x_i)) W_b(x_j) taken through the linear map of pz (the
 * Gauss-Newton Hessian, exact for Scheme I).  H[.][.][j] is the reduced Hessian of
 * eqn:param_Hker.  FWI_EINVAL for a node off the grid or more than 2048 sources + receivers. */
int fwi_fborn_hessian(const fwi_fgrid *g, int ns, int nr, fwi_param pz, int jx, int jz, void *work, double *H,
                      void *stream);

/* Device-side status of the acquisition's workspace since the last call of this function
 * (synchronizes `stream`, then clears it): FWI_ETIMEOUT if a bounded wait inside the tensor-core
 * data contraction of fwi_fborn_model / _gradient / _misfit expired (its results are then
 * invalid; the kernel still released its tensor memory), else FWI_OK. */
int fwi_fborn_status(const fwi_fgrid *g, int ns, int nr, void *work, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FWI_H_ */
