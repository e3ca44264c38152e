/*
 * se1p.h - C ABI of the GB300 (sm_103a) singly periodic Spectral Ewald library.
 *
 * The library evaluates the electrostatic potential, force and energy of N
 * point charges in a box [0,L1) x [0,L2) x [0,L3) that is periodic in z and
 * free in x and y, by the SE1P method of Saffar Shamshirgar & Tornberg ("The
 * Spectral Ewald method for singly periodic domains"):
 *
 *   phi = phi^R + phi^F + phi^self                                (Eq. 2.1)
 *   phi^R    : erfc real-space sum over a cell list, r <= rc      (Eq. 2.2)
 *   phi^F    : Algorithm 1 - Gaussian gridding (Eq. 3.4), adaptive FFT
 *              (Algorithm 2), scaling with the Ewald Green's function and the
 *              truncated 2-D kernel at k3 = 0 (Eqs. 3.5-3.10), inverse
 *              adaptive FFT (Algorithm 3), Gaussian gathering (Eq. 3.11) and
 *              its analytic gradient for the force (Eq. 3.25)
 *   phi^self : -2 xi/sqrt(pi) q_m                                 (Eq. 2.5)
 *   F_m      : -q_m grad phi(x_m); U = 1/2 sum_m q_m phi_m        (Section 3.5)
 *
 * Conventions shared by every entry point:
 *   - Particle arrays are caller-owned and never freed by the library.
 *     x is [n][3] doubles (x, y, z interleaved), q is [n] doubles, phi is [n],
 *     force is [n][3], energy is one double.  Results follow the caller's
 *     particle order.  Entry points named *_host take host pointers; all
 *     others take device pointers of the current CUDA device.
 *   - x and y must lie in [0, L1) and [0, L2); z is wrapped into [0, L3).
 *     sum(q) must vanish: |sum q| <= 1e-12 sum |q| (Section 2.1).
 *   - Device-side checks (box, finiteness, neutrality) cannot stop an
 *     asynchronous call: the call runs to completion on sanitised values and
 *     records the problem in the plan's status word.  se1p_plan_sync_status()
 *     synchronises the stream and returns (then clears) that word.
 *   - A plan owns all of its device workspace; it may be used by one stream at
 *     a time.  Calls are asynchronous on `stream` (a cudaStream_t passed as
 *     void*; NULL = legacy default stream) unless stated otherwise.
 *   - Host-side argument errors are returned immediately and launch nothing.
 */
#ifndef SE1P_H
#define SE1P_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SE1P_OK = 0,
    SE1P_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter                        */
    SE1P_ERR_NOT_NEUTRAL = 2, /* |sum q| > 1e-12 sum |q|                                 */
    SE1P_ERR_OUT_OF_BOX = 3,  /* some x or y outside [0, L)                              */
    SE1P_ERR_ALLOC = 4,       /* device or pinned-host allocation failed                 */
    SE1P_ERR_CUDA = 5,        /* a CUDA runtime call or kernel launch failed             */
    SE1P_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                           */
    SE1P_ERR_NAN = 7,         /* non-finite position or charge                           */
    SE1P_ERR_CAPACITY = 8     /* n larger than the plan's n_max, or a cell too crowded   */
} se1p_status;

typedef enum { SE1P_FP64 = 0, SE1P_MIXED = 1 } se1p_precision;

/*
 * Problem and method parameters (Algorithm 1 INPUT; Section 4.3 recipe).
 * Fields marked "0 = auto" are chosen by the plan:
 *   Mt  : smallest 2^a 3^b 5^c 7^d >= M + P (extra points are zero padding)
 *   n0  : smallest such size >= s0 Mt, s0 defaulting to 2 sqrt(2) >= 1 + sqrt(2)
 *   nI  : smallest such size >= sl Mt, sl defaulting to the smallest value with
 *         e^{-2 pi sl} < tol (Eq. 4.8)
 *   nl  : round(M3 / 10) (Eq. 4.9), at least 1
 */
typedef struct {
    double L[3];   /* box lengths; x, y free, z periodic                                */
    double xi;     /* Ewald splitting parameter                                         */
    int M[3];      /* grid points: M[0] = M[1] over [0, L) in x, y; M[2] along z        */
    int P;         /* Gaussian support in grid points per axis, 2 <= P <= min(M[2], 32) */
    int Mt;        /* grid points per free axis incl. the extension; 0 = auto          */
    int n0;        /* padded 2-D FFT size of the k3 = 0 slab; 0 = auto                 */
    int nI;        /* padded 2-D FFT size of the slabs in the set I; 0 = auto          */
    int nl;        /* local pad size: I = {0 < |k3| <= 2 pi nl / L1}; < 0 = auto        */
    double s0;     /* k3 = 0 upsampling used when n0 == 0 (<= 0: 2 sqrt 2)             */
    double sl;     /* I-set upsampling used when nI == 0 (<= 0: from tol)              */
    double rc;     /* real-space cutoff; <= 0 skips phi^R (k-space and self only)      */
    double tol;    /* tolerance for the automatic choices (<= 0: 1e-10)                */
    int precision; /* se1p_precision                                                    */
    int flags;     /* 0, or SE1P_FLAG_TRIPLY_PERIODIC                                  */
} se1p_params;

/*
 * SE1P_FLAG_TRIPLY_PERIODIC selects the triply periodic Spectral Ewald method
 * (SE3P), the method the paper measures SE1P against (Section 1, Example 6.5):
 * x and y are periodic as well, with periods L[0] = L[1], and the Green's
 * function is 1/k^2 for every k != 0 with no k = 0 term (a neutral system in a
 * conducting medium).  No axis is padded: the FFTs run on the M[0] x M[1] x M[2]
 * periodic grid (M[0] a 2^a 3^b 5^c 7^d size); Mt, n0, nI, nl, s0, sl are
 * ignored.  Gridding and gathering run on the same M + P extended grid as SE1P
 * and the P-wide overhang is folded onto the periodic grid (and unfolded before
 * gathering).  Requires an even P and rc <= min(L).  x and y are wrapped into
 * [0, L) like z.  The single-step entry points se1p_spread, se1p_fourier and
 * se1p_gather are not available for such plans (SE1P_ERR_INVALID_ARG).
 */
#define SE1P_FLAG_TRIPLY_PERIODIC 1

/* Resolved plan geometry (read-only view). */
typedef struct {
    int Mt, M3, n0, nI, nl;
    int n_I_modes;          /* number of k3 > 0 modes in the set I                         */
    int P, precision;
    double h, hz;           /* grid spacing in x,y and in z                               */
    double eta, etaz;       /* Gaussian shape eta = P xi^2 h^2/(c^2 pi), c = 0.95 (Eq. 3.3) */
    double R;               /* truncation radius of the 2-D kernel, sqrt(2) Mt h          */
    int cells[3];           /* real-space cell list dimensions                            */
    int features;           /* bit 0: the z forward pass loads its pencils by bulk tensor copies */
    size_t workspace_bytes; /* device memory owned by the plan                            */
} se1p_plan_info;

typedef struct se1p_plan se1p_plan;

/* Create a plan for systems of up to n_max particles on the current device.
 * Validates params (SE1P_ERR_INVALID_ARG), resolves the automatic fields,
 * allocates the workspace (SE1P_ERR_ALLOC) and precomputes, in FP64 on the
 * device, the k3 = 0 scaling table 4 pi e^{-(1-eta) kappa^2/4 xi^2} G_R(kappa)
 * (Eqs. 3.9-3.10).  Synchronous.  *plan is NULL on failure; a failed allocation
 * frees everything the call allocated before it.  For tests of that path, the
 * environment variable SE1P_TEST_FAIL_ALLOC=k (k >= 1) makes the k-th workspace
 * allocation of every plan creation fail (SE1P_ERR_ALLOC) without asking CUDA. */
se1p_status se1p_plan_create(const se1p_params *params, int n_max, se1p_plan **plan);

/* Free a plan and its workspace (synchronises the device first).  NULL is a no-op. */
se1p_status se1p_plan_destroy(se1p_plan *plan);

/* Fill *info with the resolved geometry. */
se1p_status se1p_plan_get_info(const se1p_plan *plan, se1p_plan_info *info);

/* Full evaluation (Algorithm 1 + Eq. 2.2 + Eq. 2.5 + Section 3.5), device pointers.
 * Any of phi, force, energy may be NULL.  0 <= n <= n_max; n == 0 writes a zero
 * energy and nothing else.  energy receives U = 1/2 sum q_m phi_m (FP64 reduction). */
se1p_status se1p_eval(se1p_plan *plan, int n, const double *x, const double *q, double *phi,
                      double *force, double *energy, void *stream);

/* Same as se1p_eval with host pointers: copies x, q to the plan's device buffers,
 * evaluates, copies the results back and synchronises `stream`.  Returns the
 * device status word (as se1p_plan_sync_status) when the launches succeeded. */
se1p_status se1p_eval_host(se1p_plan *plan, int n, const double *x, const double *q,
                           double *phi, double *force, double *energy, void *stream);

/* Adjoint (vector-Jacobian product) of phi, for reverse-mode differentiation.
 * Given the cotangent v_phi = dl/dphi of a loss l(phi), returns
 *   grad_q[n]    = dl/dq_n = phi[v](x_n)              (the method applied to charges v)
 *   grad_x[n][3] = dl/dx_n = -(v_n E[q](x_n) + q_n E[v](x_n)),   E = -grad phi (target side)
 * exactly for the discrete SE1P operator: gridding and gathering use the same
 * window (Eqs. 3.4, 3.11), so phi_m = sum_n q_n K(x_m, x_n) with K symmetric and
 * the source-side derivative equals the target-side one with the roles swapped
 * (Eq. 3.25 gives the latter); the real-space kernel is symmetric as well.
 * The grid is recomputed for q and for v (two evaluations), never stored.
 * v_phi need not be neutral; since phi of a neutral system is defined only for
 * neutral charge changes, grad_q is meaningful up to a constant shift.
 * Either output may be NULL.  Device pointers; asynchronous on `stream`.
 * Energy gradients need no adjoint: dU/dq = phi and dU/dx = -F (se1p_eval). */
se1p_status se1p_eval_vjp(se1p_plan *plan, int n, const double *x, const double *q, const double *v_phi,
                          double *grad_x, double *grad_q, void *stream);

/* ---- single steps, for verification of one stage at a time (device pointers) ---- */

/* Gridding, Algorithm 1 step 2 (Eq. 3.4): H on the M3 x Mt x Mt grid, written
 * as grid[(z * Mt + y) * Mt + x] in doubles (converted from FP32 in mixed mode).
 * The free-axis grid origin is at -P h/2, i.e. particle x sits at x + P h/2. */
se1p_status se1p_spread(se1p_plan *plan, int n, const double *x, const double *q, double *grid,
                        void *stream);

/* Algorithm 1 steps 3-5: AFT (Algorithm 2), scaling (Eq. 3.5), AIFT (Algorithm 3),
 * from grid_in (H) to grid_out (the scaled-and-filtered grid), same layout as
 * se1p_spread.  grid_in and grid_out may alias. */
se1p_status se1p_fourier(se1p_plan *plan, const double *grid_in, double *grid_out, void *stream);

/* Algorithm 1 step 6 (Eq. 3.11) and Eq. 3.25: phi^F and F^F at the particles from
 * a grid in the se1p_spread layout.  Writes (does not accumulate) phi and force;
 * either may be NULL. */
se1p_status se1p_gather(se1p_plan *plan, int n, const double *x, const double *q,
                        const double *grid, double *phi, double *force, void *stream);

/* Real-space part, Eq. 2.2 and its force (Eq. 3.22), over a cell list whose cells
 * have an edge of at least rc/3 where a particle expects at least 800 neighbours
 * within rc (n_max at uniform density), rc/2 otherwise (a target's sources lie
 * within ceil(rc / edge) cells per axis).  Writes (does not accumulate) phi and force.  Requires
 * params.rc > 0 and rc <= L3. */
se1p_status se1p_real_space(se1p_plan *plan, int n, const double *x, const double *q, double *phi,
                            double *force, void *stream);

/* ---- per-stage timing ---- */

/* Stages of se1p_eval timed by the profiling events (one CUDA event pair per
 * stage, recorded on the evaluation stream). */
typedef enum {
    SE1P_STAGE_PACK = 0,    /* validation, counting sort, window tables          */
    SE1P_STAGE_SPREAD = 1,  /* gridding, Eq. 3.4                                  */
    SE1P_STAGE_FOURIER = 2, /* AFT + scaling + AIFT (Algorithms 2-3, Eq. 3.5)     */
    SE1P_STAGE_GATHER = 3,  /* gathering of phi and F, Eqs. 3.11 and 3.25         */
    SE1P_STAGE_REAL = 4,    /* real-space sum, Eq. 2.2                            */
    SE1P_STAGE_FINAL = 5,   /* outputs in caller order and the energy reduction   */
    SE1P_NUM_STAGES = 6
} se1p_stage;

/* Enable (1) or disable (0) per-stage event recording for subsequent se1p_eval
 * calls (at most 4096 evaluations are kept).  With 2, recording is on and the
 * evaluation runs its stages one after another on the caller's stream instead of
 * overlapping the real space with the grid path, so that each stage's time is
 * its time alone (same results).  Enabling clears earlier records.  Synchronous.
 * Other values: SE1P_ERR_INVALID_ARG. */
se1p_status se1p_plan_set_profiling(se1p_plan *plan, int enable);

/* Synchronise the device and return, per stage, the summed elapsed milliseconds
 * over all recorded evaluations (ms[SE1P_NUM_STAGES]) and their number
 * (*n_evals); then clear the records. */
se1p_status se1p_plan_stage_times(se1p_plan *plan, double *ms, int *n_evals);

/* Synchronise `stream` and return the device status word (SE1P_OK or the first
 * error recorded since the last call), then clear it. */
se1p_status se1p_plan_sync_status(se1p_plan *plan, void *stream);

/* ---- parameter selection (Section 4.3) ---- */

typedef struct {
    double L[3];   /* box; L[0] == L[1]                                       */
    double xi;     /* Ewald splitting parameter                              */
    double Q;      /* sum of q^2 of the system                               */
    int n;         /* number of particles                                    */
    double tol;    /* requested rms error (absolute, per Eqs. 2.7-2.8, 4.3)  */
    int precision; /* copied into the result                                 */
} se1p_tune_request;

/* Choose every field of *out for a requested tolerance, following Section 4.3:
 *   rc from Eq. 2.9 and k_inf from Eq. 2.10 (Lambert W), M = 2 k_inf per axis
 *   (scaled by the axis length; even 2^a 3^b 5^c 7^d sizes), P from Eq. 4.3 (even,
 *   at most 32); k_inf and P are taken for tol/100 (the printed estimates undershoot
 *   the measured k-space error by 5-20x), s_l at the lowest mode k3 = 2 pi/L3 from
 *   sqrt(Q/V) exp(-|k3| (s_l Mt h - L)) <= tol (the trapezoidal rule's error of Section 4.2: its
 *   nearest implied images lie s_l Mt h - L away, its amplitude grows with the charge content) and
 *   at least exp(-|k3| s_l L) <= tol (Eq. 4.8 when L3 = L), n_l = ceil(M/10) (Eq. 4.9), s0 = 2 sqrt 2;
 *   Mt, n0, nI are then fixed to smooth sizes.  Host only, no GPU work.
 *   SE1P_ERR_INVALID_ARG for non-positive lengths, xi, Q, n or tol outside (0,1). */
se1p_status se1p_autotune(const se1p_tune_request *req, se1p_params *out);

/* ---- batched evaluation (many independent systems) ----
 *
 * A batch owns one plan per system (params[i], n_max[i]).  se1p_batch_eval
 * evaluates all systems from packed arrays: system i occupies particles
 * offsets[i] .. offsets[i+1]-1 (host array of count+1 ints) of x [*][3], q, phi,
 * force; energy[i] receives its U.  The work of all systems is captured once
 * into a CUDA graph (nodes spread over up to 32 streams, so small systems run
 * concurrently) and replayed with one graph launch per call; the graph is
 * re-captured when the sizes or the pointers change.  Device pointers;
 * asynchronous on `stream`.  se1p_batch_sync_status synchronises and returns
 * the first device status of any system (then clears them). */
typedef struct se1p_batch se1p_batch;
se1p_status se1p_batch_create(int count, const se1p_params *params, const int *n_max, se1p_batch **batch);
se1p_status se1p_batch_destroy(se1p_batch *batch);
se1p_status se1p_batch_eval(se1p_batch *batch, const int *offsets, const double *x, const double *q,
                            double *phi, double *force, double *energy, void *stream);
se1p_status se1p_batch_sync_status(se1p_batch *batch, void *stream);
/* The plan of system i (owned by the batch), e.g. for se1p_plan_get_info; NULL if out of range. */
se1p_plan *se1p_batch_plan(se1p_batch *batch, int i);

/* ---- allocation-free variant ----
 *
 * se1p_real_space_noalloc: the real-space part (phi^R and F^R, as
 * se1p_real_space) for callers that cannot allocate device memory, e.g. code
 * that runs while a framework owns the device allocator, embedded hosts whose
 * device memory is handed out up front, or plugins in processes that forbid
 * allocation after start-up.  The paper has no counterpart: this is a
 * deployment variant of the same sum.
 *
 * It takes the parameters directly (no plan: plan creation allocates) and uses
 * params->L, xi, rc (> 0, <= L3) and precision.  All scratch lives in one
 * file-scope __device__ array of about 2.2 MB that every GPU which loads the
 * library holds until the process exits; nothing is allocated or freed (no
 * cudaMalloc, cudaFree or allocating library routine).
 *   - n <= 16384 particles (larger n returns SE1P_ERR_CAPACITY); the cell list
 *     is capped at 4096 cells, made coarser (never finer than rc) if needed.
 *   - x, q, phi, force are device pointers; phi and force must be non-NULL.
 *     Writes (does not accumulate) phi and force.  Inputs are sanitised as in
 *     se1p_eval, but this entry point records no device status.
 *   - Every call made outside stream capture looks up the array's device
 *     address (cudaGetSymbolAddress) with the current device, so an address
 *     that a device reset made stale is never used.  A call made while `stream`
 *     is being captured uses the address found by the last uncaptured call on
 *     that device: make one call before any stream capture.
 *   - Every call shares the array and leaves its contents behind; calls whose
 *     work overlaps on the GPU race on it and must be serialised by the caller.
 * Asynchronous on `stream`. */
se1p_status se1p_real_space_noalloc(const se1p_params *params, int n, const double *x, const double *q,
                                    double *phi, double *force, void *stream);

/* ---- device arithmetic peaks (measurement) ----
 *
 * se1p_measure_fma_peak: FMA throughput of the current device in TFLOP/s
 * (2 flop per FMA), FP32 for SE1P_MIXED and FP64 for SE1P_FP64, from a
 * kernel of independent FMA chains on every SM (best of three ~10 ms launches
 * after a warm-up).  The gridding, gathering and real-space steps are bound by
 * this arithmetic rather than by HBM, so their roofline fractions are quoted
 * against it.  The paper has no counterpart: it times one CPU core.
 * *sm_count (may be NULL) receives the device's multiprocessor count.
 * Synchronous; uses the legacy default stream; allocates nothing. */
se1p_status se1p_measure_fma_peak(int precision, double *tflops, int *sm_count);

/* Static, human-readable name of a status code. */
const char *se1p_status_string(se1p_status status);

#ifdef __cplusplus
}
#endif

#endif /* SE1P_H */
