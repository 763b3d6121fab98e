/*
 * grape.h - C ABI of the GB300 open-GRAPE gradient library (libgrape.so).
 *
 * Open GRAPE without matrix exponentials (Boutin et al., arXiv:1609.03170):
 * the density matrix rho (d x d, complex128) is propagated under the Lindblad
 * master equation (Eq. master, Eq. disspation)
 *     d rho/dt = -i[H(t), rho] + sum_m gamma_m (c_m rho c_m^+ - {c_m^+ c_m, rho}/2),
 *     H(t) = H_0 + sum_k u_k(j) H_k on slice j             (Eq. Hamiltonian)
 * over N piecewise-constant control slices of length dt = T/N, each slice
 * integrated with n_RK classic RK4 substeps (Sec. 3, Eq. rkmaster).  The
 * performance index is Phi = sum_s Re Tr(sigma_s rho_s(T)) (Eq. phi, Eq. Phi0)
 * and its gradient dPhi/du_k(j) comes from a backward (adjoint) propagation
 * under the dual Lindbladian followed by per-slice trace products
 * (Sec. 2.2 Eq. lambda, Eq. dphidu; Sec. 3).
 *
 * Conventions
 *  - complex numbers are interleaved (re, im) doubles;
 *  - d x d matrices are row-major; rho0/sigma hold n_states (or 1) of them;
 *  - controls u are slice-major: u[j * n_controls + k];
 *  - pointers passed to grape_forward / grape_gradient may be host or device
 *    memory (told apart with cudaPointerGetAttributes); device pointers must
 *    be memory of the problem's device (another device's memory is rejected
 *    with GRAPE_EINVAL) and are only borrowed;
 *  - every call returns a grape_status; on failure grape_last_error() gives a
 *    thread-local message.  No call aborts, traps or waits without a bound.
 */
#ifndef GRAPE_H_
#define GRAPE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRAPE_OK = 0,
    GRAPE_EINVAL = 1,      /* invalid argument or descriptor */
    GRAPE_ENOMEM = 2,      /* device or host allocation failed */
    GRAPE_ECUDA = 3,       /* a CUDA runtime call failed */
    GRAPE_ETIMEOUT = 4,    /* a bounded wait ran out */
    GRAPE_EBUSY = 5,       /* resource (slot, memory budget) not available now */
    GRAPE_ENOTREADY = 6,   /* result not ready yet (grape_poll) */
    GRAPE_EINTERNAL = 7
} grape_status;

typedef enum {
    GRAPE_PREC_DF64 = 0,   /* double-float: pairs of FP32 numbers, ~48-bit significands,
                              on the FP32 pipes (default; GB300 issues FP32 ~67x faster
                              than FP64) */
    GRAPE_PREC_FP64 = 1    /* native FP64 */
} grape_precision;

typedef enum {
    GRAPE_GRAD_EXACT = 0,        /* exact derivative of the discrete RK4 map */
    GRAPE_GRAD_FIRST_ORDER = 1   /* the paper's Eq. (dphidu), first order in dt */
} grape_grad_mode;

/* A banded (DIA) operator: band b holds the entries Op[i][i + offsets[b]],
 * values[b * d + i] (complex), for i in [0, d); entries whose column falls
 * outside [0, d) are ignored. */
typedef struct {
    int32_t n_diag;
    const int32_t *offsets;   /* [n_diag] */
    const double *values;     /* [n_diag][d] complex interleaved */
} grape_band_op;

/* Problem descriptor.  grape_problem_create copies every array it points to. */
typedef struct {
    int32_t d;                  /* Hilbert-space dimension */
    int32_t n_controls;         /* R, number of control Hamiltonians */
    int32_t n_jumps;            /* number of dissipators c_m */
    int32_t n_states;           /* initial states propagated (n_s of Eq. RK) */
    int32_t n_slices;           /* N, piecewise-constant control slices */
    int32_t n_rk;               /* RK4 substeps per slice */
    double T;                   /* total duration */
    grape_band_op H0;           /* drift Hamiltonian (Hermitian) */
    const grape_band_op *Hc;    /* [n_controls] control Hamiltonians (Hermitian) */
    const grape_band_op *jumps; /* [n_jumps] jump operators c_m */
    const double *rates;        /* [n_jumps] gamma_m >= 0 */
    const double *rho0;         /* [n_states][d][d] complex, Hermitian */
    const double *sigma;        /* [n_states or 1][d][d] complex target/observable */
    int32_t sigma_broadcast;    /* 1: one sigma for all states */
    int32_t grad_mode;          /* grape_grad_mode */
    int32_t ckpt_stride;        /* slices per checkpoint segment of the gradient;
                                   0 = automatic (no recomputation when the stage
                                   storage fits in 60% of the free device memory) */
    int32_t precision;          /* grape_precision of the kernels */
    const int32_t *jump_control;/* NULL or [n_jumps]: -1 = fixed rate; k >= 0 = the
                                   dissipator's rate is rates[m] * u_k(j) in slice j
                                   (a control on a dissipation rate, the variant
                                   mentioned after Eq. partialuk; Hc[k] must then be
                                   empty and dL/du_k = rates[m] D[c_m]) */
} grape_problem_desc;

typedef struct grape_problem *grape_problem_t;

/* Builds the device tables of a problem on the current CUDA device.
 * Operators enter as band lists (Eq. Hamiltonian, Eq. disspation); the
 * non-Hermitian part -i/2 sum gamma_m c_m^+ c_m is formed here.  sigma enters
 * the cost only through its Hermitian part (rho(T) is Hermitian), so it is
 * stored Hermitianised.  Errors: GRAPE_EINVAL (sizes, band offsets beyond
 * +-(d-1), non-Hermitian rho0 or control, negative rates), GRAPE_ENOMEM. */
grape_status grape_problem_create(const grape_problem_desc *desc, grape_problem_t *out);

/* Frees everything the problem allocated.  NULL is accepted. */
grape_status grape_problem_destroy(grape_problem_t problem);

/* Forward propagation (Sec. 3, Eq. rkmaster) and the cost (Eq. phi).
 * u: [n_slices][n_controls] doubles, host or device.
 * F: one double (host or device) receiving Phi.
 * rhoT: NULL or [n_states][d][d] complex (host or device) receiving rho_s(T).
 * stream: a cudaStream_t (NULL = legacy default stream).  The call returns
 * once the results are in host memory when F is a host pointer; with device
 * outputs it only enqueues the work on the stream. */
grape_status grape_forward(grape_problem_t problem, const double *u, double *F,
                           double *rhoT, void *stream);

/* Phi and its gradient dPhi/du_k(j) (Sec. 2.2 Eq. dphidu; Sec. 3), in the
 * problem's grad_mode.  grad: [n_slices][n_controls] doubles, host or
 * device.  Same pointer and stream rules as grape_forward.  The cost is
 * linear in rho, so the adjoint sweep does not read the forward states: in
 * exact mode, with the whole problem in one segment on a cluster kernel, the
 * two sweeps run at the same time on the problem's own streams and the
 * trace of each chunk of slices waits for both (GRAPE_CONCURRENT=0: one
 * after the other; the results are the same bits either way). */
grape_status grape_gradient(grape_problem_t problem, const double *u, double *F,
                            double *grad, void *stream);

/* ---- Gaussian filtering of the controls (App. A, transfer matrix of the
 * erf form; chain rule for the gradient) ----
 * The n_steps piecewise-constant controls u (length Dt each) become n_sub
 * subpixel amplitudes s (length dt each) - the slices a problem propagates:
 *   s[n][k]  = sum_j T_k[n][j] u[j][k],
 *   T_k[n][j] = (erf(w0_k (n dt - j Dt) / 2) - erf(w0_k (n dt - (j+1) Dt) / 2)) / 2
 * with 0-based n, j and w0_k = wB_k / sqrt(-ln(1/sqrt 2)) for a 3 dB bandwidth
 * wB_k of control k.  grape_filter_adjoint applies the transpose,
 *   g_u[j][k] = sum_n T_k[n][j] g_s[n][k],
 * which turns dPhi/ds into dPhi/du.  u, s, g_s, g_u are device float64 arrays,
 * row-major [index][control]; omega0 is a host array of n_controls values.
 * Both run on `stream` in FP64 (one thread per output, only the band of
 * terms that can be non-zero: erf saturates to +-1 exactly).  Errors:
 * GRAPE_EINVAL (NULL or host data pointers, n_steps or n_sub < 1,
 * n_controls outside [1, 8], Dt, dt or an omega0 not positive and finite),
 * GRAPE_ECUDA. */
grape_status grape_filter_apply(int32_t n_steps, int32_t n_sub, int32_t n_controls, double Dt,
                                double dt, const double *omega0, const double *u, double *s,
                                void *stream);
grape_status grape_filter_adjoint(int32_t n_steps, int32_t n_sub, int32_t n_controls, double Dt,
                                  double dt, const double *omega0, const double *g_s, double *g_u,
                                  void *stream);

/* Phi and dPhi/du for n_steps filtered controls u [n_steps][n_controls]: the
 * problem's n_slices are the subpixels (dt = T / n_slices, Dt = T / n_steps),
 * s = filter(u) is propagated by grape_gradient and its gradient is mapped
 * back through the transposed filter into grad [n_steps][n_controls].  u, F
 * and grad may be host or device memory (host results are ready on return);
 * omega0: host, one value per control.  The problem keeps the subpixel
 * buffers (allocated on the first call).  Errors as grape_gradient and
 * grape_filter_apply. */
grape_status grape_gradient_filtered(grape_problem_t problem, int32_t n_steps, const double *omega0,
                                     const double *u, double *F, double *grad, void *stream);

/* Device memory the problem holds, in bytes (tables plus stage storage). */
grape_status grape_problem_memory(grape_problem_t problem, size_t *bytes);

/* Launch geometry chosen for the propagation kernels (cluster size, threads
 * per block, elements per thread).  For tests and benchmarks. */
grape_status grape_problem_geometry(grape_problem_t problem, int32_t *cluster,
                                    int32_t *threads, int32_t *elems_per_thread);

/* Running-cost penalty (Sec. 5 and App. B, the photon-number penalty):
 * the performance index becomes Phi = Phi_0 - beta Phi_p with
 *   Phi_p = dt * sum over initial states and boundaries n = 0..n_slices of
 *           Re Tr(A rho_n),   dt = T / n_slices,
 * for an operator A diagonal in the basis (diag: host, d real values; a^dag a
 * is diag[n Q + q] = n).  The gradient comes from one modified backward
 * evolution: -beta dt A is added to the adjoint at every slice boundary and
 * at the final time, in the exact and the first-order gradient alike.
 * grape_forward and grape_gradient then return the penalised Phi (the
 * forward sweep runs in chunks of 64 slices to reach every boundary state).
 * beta = 0 or diag = NULL removes the penalty.  Waits for the device.
 * Errors: GRAPE_EINVAL (NULL problem, non-finite values), GRAPE_ENOMEM,
 * GRAPE_ECUDA.  grape_gradient_static rejects penalised problems. */
grape_status grape_problem_set_penalty(grape_problem_t problem, const double *diag, double beta);

/* Sets the propagation tile of a cluster-kernel problem: the cluster width
 * (1, 2, 4, 8 or 16 CTAs per initial state, each CTA owning an equal share
 * of the state's entries) and the threads per CTA (a multiple of 32 in
 * [64, 512]).  Every entry is computed by the same arithmetic whatever CTA
 * or thread owns it, so results do not change, bit for bit; only speed and
 * the SMs a call occupies do (narrow tiles leave room for other problems,
 * see grape_batch_create).  Errors: GRAPE_EINVAL (values out of range, a
 * grid-kernel problem, or a tile whose state window does not fit in shared
 * memory or of which no cluster can be resident; the tile is unchanged),
 * GRAPE_ECUDA.  The tile chosen at create is the widest useful cluster
 * (shortest stage latency) with 512 threads per CTA or, when one CTA holds
 * a whole state on the Hermitian kernel, the state's upper entries
 * rounded up to whole warps (at least 64 threads). */
grape_status grape_problem_set_tile(grape_problem_t problem, int32_t cluster, int32_t threads);

/* Which propagation kernel the problem runs on: 0 = Hermitian cluster kernel
 * (upper triangle, states in distributed shared memory), 1 = full-matrix
 * cluster kernel, 2 = grid kernel (states in global memory, one cooperative
 * grid, for states too large for a cluster's shared memory). */
grape_status grape_problem_kernel(grape_problem_t problem, int32_t *kind);

/* Waits for the device and reports whether a bounded wait of the
 * problem's kernels gave up since the last check (GRAPE_ETIMEOUT; the
 * results of that call are invalid): a grid barrier of the grid kernel, a
 * window wait of the Hermitian cluster kernel (which waits on mbarriers
 * for the values its peers push into its shared memory), or a copy wait of
 * the staged gradient-trace kernel (which waits on mbarriers for the bulk
 * copies of its operands into shared memory).  The flag is
 * cleared by the report.  Calls that return results to host memory do this
 * check themselves. */
grape_status grape_problem_status(grape_problem_t problem);

/* Per-launch timing with CUDA events recorded on the caller's stream around
 * every kernel the library launches (off by default).  grape_phase_times
 * waits for the recorded events, returns the summed milliseconds and launch
 * counts since the previous call per phase - [0] forward propagation,
 * [1] cost, [2] adjoint propagation, [3] gradient traces - and clears them. */
grape_status grape_set_profiling(grape_problem_t problem, int32_t on);
grape_status grape_phase_times(grape_problem_t problem, double ms[4], int32_t launches[4]);

/* grape_gradient without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need a gradient - code whose allocator owns all of
 * the device memory, host callbacks where cudaMalloc may not be called, or
 * latency-bound loops that must not wait on the allocator.  The problem is
 * created beforehand with grape_problem_create; the stage storage, the
 * propagated states, the partial traces and any checkpoints come from one
 * file-scope device array of 64 MiB per device, which stays held until the
 * process exits.  It is committed on a device when the first problem is
 * created there (grape_problem_create looks up its device address once per
 * device, with that device current; a failed lookup makes this call return
 * GRAPE_ECUDA), so this call itself makes no cudaMalloc/cudaFree, no
 * module load and no host allocation of its own; it only enqueues work on
 * `stream`.  u, F and grad must be device memory of the problem's device
 * (GRAPE_EINVAL otherwise, also for another device's memory).  The
 * checkpoint segment length is the longest whose scratch fits; a problem
 * that needs more than 64 MiB with every segment length is rejected with
 * GRAPE_EINVAL and a message giving the least bytes it needs, as is a
 * problem with a running-cost penalty.  All calls share the one array and
 * it keeps the last call's contents (nothing in it needs to start at zero:
 * every buffer is written before it is read), so calls whose GPU work
 * overlaps - on two streams, or from two threads - race and give wrong
 * results: serialise them.  Results equal those of grape_gradient bit for
 * bit (the traces are split and summed in the same order).  This call
 * cannot wait for the device, so after the stream has completed call
 * grape_problem_status: on GRAPE_ETIMEOUT a bounded wait of one of the
 * kernels (grid barrier, window wait, trace copy wait) gave up and F and
 * grad are invalid. */
grape_status grape_gradient_static(grape_problem_t problem, const double *u, double *F,
                                   double *grad, void *stream);

/* ---- Batching: many problems of different sizes in one graph launch ----
 * (the batched form of the hot path; the paper evaluates one problem at a
 * time).  grape_batch_create first tunes the propagation tile per bucket of
 * d (32 wide): for the bucket's largest problem it times every tile that
 * fits (cluster width x threads per CTA, see grape_problem_set_tile) on a
 * few slices of forward propagation run as concurrent copies, as many as
 * can be resident at once, and sets the tile of highest throughput on the
 * bucket's problems (their own tiles come back at grape_batch_destroy;
 * GRAPE_BATCH_TUNE=0 skips the tuning).  The problems are then spread over
 * n_lanes concurrent streams, longest
 * first to the least loaded lane; each lane owns stage storage sized for its
 * largest problem (with checkpoint segments that keep every lane within an
 * equal share of 60% of the free device memory) and runs its problems one
 * after another.  The first grape_batch_gradient call captures the whole
 * batch into a CUDA graph; later calls with the same pointers and stream
 * replay it, other pointers re-capture.  Results equal per-problem
 * grape_gradient calls bit for bit.  The problems must outlive the batch and
 * must not be used concurrently with it. */
typedef struct grape_batch *grape_batch_t;

/* n_lanes <= 0 picks the work-weighted mean number of copies of the
 * batch's problems that can be resident at once (at least 8, at most 128,
 * capped at n).  Errors: GRAPE_EINVAL (NULL pointers,
 * a problem listed twice, problems on different devices), GRAPE_ENOMEM. */
grape_status grape_batch_create(grape_problem_t *problems, int32_t n, int32_t n_lanes,
                                grape_batch_t *out);
grape_status grape_batch_destroy(grape_batch_t batch);
/* u[i]: problem i's controls, grad[i]: its gradient, F: n doubles - all
 * device memory.  Enqueues the work on `stream` and returns. */
grape_status grape_batch_gradient(grape_batch_t batch, const double *const *u, double *F,
                                  double *const *grad, void *stream);
/* Lanes, scratch bytes and kernel launches per grape_batch_gradient. */
grape_status grape_batch_info(grape_batch_t batch, int32_t *n_lanes, size_t *scratch_bytes,
                              int32_t *launches);

/* ---- Serving: pulse optimisations with continuous batching ----
 * A job maximises Phi of one problem with projected L-BFGS (the paper
 * optimises with BFGS, Sec. 2.1, Eq. update) over the box
 * u_min <= u <= u_max, starting from u0.  Each iteration is one gradient
 * evaluation at a trial point followed by one L-BFGS step on the device
 * (decrease of -Phi accepts the point, otherwise the step is halved).  The
 * server keeps every job's controls, gradient and L-BFGS history on the
 * device; a worker thread admits queued jobs (in order) whenever a slot is
 * free, their gradient storage fits the memory budget and the SMs their
 * clusters need (states x cluster width) are not taken - a job admitted
 * while others run or wait is first moved to the narrowest cluster width its
 * state fits (grape_problem_set_tile; results unchanged), widened again
 * between iterations when nothing waits and SMs are free, and given its own
 * tile back when it ends (GRAPE_SERVER_ELASTIC=0 keeps tiles) - runs each admitted job on
 * its own stream and launches its next iteration as soon as the previous one
 * completes, so iterations of different jobs overlap.  A job's result does
 * not depend on the other jobs (deterministic kernels). */
typedef struct grape_server *grape_server_t;

typedef struct {
    int32_t max_iters;   /* gradient evaluations (e.g. 50) */
    int32_t lbfgs_m;     /* curvature pairs kept (1..64, e.g. 10) */
    double u_min, u_max; /* box on every control amplitude */
    double step0;        /* first step: largest control change of the first move */
    double tol;          /* stop when max |P(u - grad) - u| <= tol (0: use max_iters) */
} grape_opt_params;

typedef struct {
    int32_t evaluations; /* gradient evaluations the job used */
    double queued_us;    /* submit -> admission */
    double latency_us;   /* submit -> result */
} grape_job_info;

/* hbm_budget_bytes = 0 uses 60% of the free device memory; max_slots jobs
 * run at once.  Starts the worker thread (device = the current device). */
grape_status grape_server_create(size_t hbm_budget_bytes, int32_t max_slots, grape_server_t *out);
/* Runs the jobs already admitted to completion, drops queued ones, joins the
 * worker.  Problems must outlive their jobs; a problem serves one job at a
 * time (jobs of a busy problem wait in the queue). */
grape_status grape_server_destroy(grape_server_t server);
/* Queues a job (u0: host, n_slices x n_controls; it is copied). */
grape_status grape_submit(grape_server_t server, grape_problem_t problem, const double *u0,
                          const grape_opt_params *params, uint64_t *ticket);
/* Waits up to timeout_us for the job; GRAPE_ENOTREADY while it runs.  On
 * completion copies the best controls (host) and Phi there, fills info (all
 * three nullable) and forgets the ticket. */
grape_status grape_poll(grape_server_t server, uint64_t ticket, int64_t timeout_us, double *u_out,
                        double *F_out, grape_job_info *info);

/* Kernel launches one grape_gradient call makes (for launch accounting);
 * -1 before the first gradient call has fixed the segment plan. */
int32_t grape_gradient_launches(grape_problem_t problem);

/* Thread-local message of the last failed call on this thread. */
const char *grape_last_error(void);

/* Measured FMA throughput of the current device, the denominator of the
 * propagation kernels' ALU roofline (a measurement helper; the paper has no
 * counterpart).  precision = GRAPE_PREC_DF64 measures the FP32 pipes that the
 * double-float kernels run on, GRAPE_PREC_FP64 the FP64 pipe of the native
 * kernels.  A kernel of independent multiply-add chains (8 per thread, all
 * SMs) runs once to warm up and three times timed with CUDA events on a
 * private stream; *tflops = 2 x multiply-adds / best time (TFLOP/s), *ms =
 * that time.  Allocates and frees a small output buffer; waits for the
 * device.  Errors: GRAPE_EINVAL (NULL outputs, unknown precision),
 * GRAPE_ECUDA. */
grape_status grape_fma_peak(int32_t precision, double *tflops, double *ms);

/* Library version string. */
const char *grape_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GRAPE_H_ */
