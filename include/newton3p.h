/*
 * newton3p.h — C ABI of the GB300 (sm_103a) three-precision Newton solver.
 *
 * Method: C. T. Kelley, "Newton's Method in Three Precisions" (arXiv
 * 2307.16051).  The nonlinear residual F is evaluated in double precision,
 * the Jacobian is stored in single precision (J32), a half-precision copy
 * J_h = I_s^h(J32) is factored with partial pivoting, and the Newton step is
 * computed by iterative refinement (IR) or GMRES-IR with those factors
 * (Algorithm 2.1 [newton3p], Section 2.2).  The test problem is the
 * composite-midpoint Chandrasekhar H-equation of Section 3, eq. (3.2):
 *     F(x)_i = x_i - (1 - c/(2N) sum_j x_j mu_i/(mu_j + mu_i))^{-1},
 *     mu_i = (i - 1/2)/N.
 *
 * Conventions for every function:
 *  - The return value is an nl_status.  On NL_EINVAL nothing is written.
 *    nl_last_error() gives a human-readable message for the calling thread.
 *  - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *    pointers are CUDA global memory on the current device, owned by the
 *    caller unless stated otherwise.
 *  - Matrices are row-major with a leading dimension `ld` (elements between
 *    the starts of consecutive rows), ld >= N.  Half-precision matrices are
 *    IEEE binary16 (`uint16_t` bit patterns, CUDA __half in memory).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Kernel
 *    entry points are asynchronous unless they return host data.
 *  - There is no CPU fallback: without a CUDA device every call that needs
 *    one returns NL_ECUDA.
 */
#ifndef NEWTON3P_H
#define NEWTON3P_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NL_OK = 0,
    NL_EINVAL = 1,     /* bad argument (N < 1, c outside [0,1), null pointer, ...) */
    NL_ENOMEM = 2,     /* device allocation failed */
    NL_ENOTCONV = 3,   /* Newton cap reached; the best iterate is returned */
    NL_ESINGULAR = 4,  /* exactly zero pivot in a factorisation */
    NL_ENUMERIC = 5,   /* NaN/Inf in F, or binary16 overflow of the Jacobian */
    NL_ETIMEOUT = 6,   /* a device-side bounded wait gave up (no hang, context intact) */
    NL_ECUDA = 7       /* CUDA runtime error, or no device / library */
} nl_status;

/* Linear solver for the Newton step.
 *  NL_FP64LU:    J in double, LU in double, one direct solve (Algorithm 1.1,
 *                column F64 of Tables 2-3): the on-GPU baseline.
 *  NL_IR16:      J32 + half-precision LU + IR (Algorithm IR, Section 2.2).
 *  NL_GMRESIR16: J32 + half-precision LU as left preconditioner of GMRES,
 *                wrapped in IR (GMRES-IR, Section 2.2).
 *  NL_IR16_GMRES: NL_IR16 until the first Newton step whose IR stalls (the
 *                failure rule of Section 3.1 fires, or ir_maxit corrections
 *                do not meet eta_j); that step's linear solve is redone with
 *                GMRES-IR from u0 = 0 and every later step uses GMRES-IR.
 *  NL_F32, NL_F16: the two-precision Newton methods the paper compares
 *                against (Section 1.3, columns F32 and F16 of Tables 2-3):
 *                the Jacobian stored and factored in single (J32, binary32
 *                LU with interchanges) or half (J16 = I_s^h(J32), the
 *                binary16 LU of NL_IR16) precision, and the step computed
 *                with ONE triangular-solve pair in that precision: binary32
 *                for F32; for F16 the right side fl16(-F/||F||) and every
 *                product and difference of both solves rounded to binary16.
 *                No refinement, so F16 converges slowly (Section 1.3). */
typedef enum {
    NL_FP64LU = 0,
    NL_IR16 = 1,
    NL_GMRESIR16 = 2,
    NL_IR16_GMRES = 3,
    NL_F32 = 4,
    NL_F16 = 5
} nl_mode;

/* Solver parameters (nl_config_default fills the defaults in brackets). */
typedef struct {
    double eta_j;        /* [1e-4] IR/GMRES-IR stops at ||J32 u - b|| <= eta_j ||b||, eq. (2.3) */
    int ir_maxit;        /* [20]  cap on IR (or GMRES-IR outer) corrections per Newton step */
    int gmres_restart;   /* [30]  GMRES restart length m */
    double gmres_tol;    /* [1e-4] inner GMRES tolerance, relative to the initial preconditioned residual */
    int gmres_maxcycles; /* [10]  GMRES restart cycles per outer correction */
    int newton_maxit;    /* [30]  cap on Newton steps */
    double tau_a;        /* [0]   absolute tolerance tau_a of Algorithm 1.1 */
    int lu_nb;           /* [0 = 128] outer block of the LU, also its binary16 rounding period: a multiple
                            of 16 up to 128 (one level of blocking), or 256, 384 or 512 (two levels: inner
                            panels of 128 carried in single precision, and one tensor-core update of
                            depth lu_nb of the rest of the matrix per outer block, so the trailing matrix
                            is read and written once per lu_nb columns; when partial pivoting needs
                            interchanges the factorisation is redone with 128).  -1 = autotune at
                            nl_create: the factorisation of the Jacobian at x0 = ones is timed for nb in
                            {512, 256, 128, 64} (the two-level ones when N >= 2 nb) and the fastest is
                            kept */
    int trailing_gemm;   /* [0 = auto] 1 = SIMT fp32-FMA trailing update, 2 = tcgen05 tensor-core update;
                            batches only (nl_batch_create): 3 / 4 = the grouped LU as one persistent
                            launch with 64 x 64 / 128 x 64 SIMT update tiles (nb <= 64), 5 = one
                            persistent launch with 128 x 128 tcgen05 update tiles (nb = 64) */
    int lu_path;         /* [0 = auto] no-interchange fast path with exact fallback; 1 = interchanging path only */
    int trsv_cluster;    /* [0 = auto] half-precision triangular solves: one thread-block cluster per
                            triangle of at most 16 CTAs (the largest of 16, 8, 4 the device can
                            co-schedule) for N <= 10240, else one launch of independent CTAs per
                            triangle that hand solved entries over global memory; 4, 8 or 16 caps
                            the cluster size (any N); -1 = always the global-memory hand-off */
    int lu_stream;       /* [0 = auto] half-precision fast path: the diagonal block and the off-diagonal
                            solves of a panel in one cooperative launch, the solves streaming one
                            column behind the diagonal block (when its CTAs fit on the GPU at once),
                            128 rows per CTA where possible; 256 = the same with 256 rows per CTA
                            (half the SMs, for solves that share the GPU); -1 = two launches per
                            panel.  Bitwise the same factors in every case */
    int ir_variant;      /* [0] IR correction (NL_IR16, and the IR part of NL_IR16_GMRES): 0 = on the
                            fly, d = U^{-1} L^{-1} r with the binary16 factors promoted to single
                            (eq. (2.16) applied to IR); 1 = the scaled half-precision correction of
                            eq. (2.19), d = ||r|| I_h^s(U^{-1} L^{-1} I_s^h(r/||r||)) with both
                            triangular solves in binary16 arithmetic (as nl_lusolve16h).  The
                            batched path accepts only 0 */
    int gmres_factors32; /* [0] GMRES-IR preconditioner: 0 = the binary16 factors promoted to single on the
                            fly (eq. (2.16)); 1 = a single-precision copy of the binary16 factors made
                            once per factorisation (Section 2.3: one more N x N copy, no interchange
                            of precision inside the solves; the same values, so the same
                            preconditioner up to the solves' summation order).  The batched path
                            accepts only 0 */
    int lu16_arith;      /* [0] arithmetic of the half-precision factorisation: 0 = binary32 arithmetic on
                            binary16 storage (lu_nb above); 1 = every operation rounded to binary16
                            (the arithmetic behind the paper's F16 column): right-looking partial
                            pivoting, one grid-wide step per column, slow (as nl_lu16 path 3); one
                            cooperative launch with a CTA on every SM, so it is meant for solves that
                            have the GPU to themselves (its barriers are bounded: NL_ETIMEOUT, not a
                            hang, if its CTAs cannot all run).  The batched path accepts only 0 */
    int wait_limit;      /* [0] bound of the device-side waits of the half-precision triangular solves:
                            0 = the default (about a second, then NL_ETIMEOUT); > 0 = that many polls
                            (cluster solve) or clock cycles (global-memory solve); < 0 = every such wait
                            gives up at once.  A test hook for the timeout path: the solve returns
                            NL_ETIMEOUT with the context intact */
    int scale_fp16;      /* [0] 1 = scale J into the binary16 range before the down-cast (Section 2.3 on
                            underflow when rounding to half precision): J_h = I_s^h(R J32) with power-of-two
                            row factors R (exact in binary32, nl_k_jacobian_scaled), so the factors are
                            those of R J and every triangular solve with them is applied to R v.  Three-
                            precision modes with the on-the-fly correction only: NL_EINVAL with
                            ir_variant = 1, gmres_factors32 = 1 or lu16_arith = 1 (nl_create) and with
                            NL_F16 (nl_solve).  The batched path accepts only 0 */
    int fft_f;           /* [0 = auto] evaluation of F (Section 3: O(N log N) with an FFT): 1 = FFT
                            convolution in double (nl_k_residual_fft: four launches, rounding-level
                            differences from the direct sum); -1 = the direct double sum over the Hankel
                            table (N^2 products); 0 = the FFT for N >= 4096, where it is the faster one
                            (45 against 61 us at N = 4096, 70 us against 2.1 ms at N = 32768), the direct
                            sum below */
    int lu_lookahead;    /* [0 = on] half-precision fast path with the tensor-core update (lu_nb <= 128):
                            after each panel only the trailing matrix's first 128-row and 128-column
                            tile strips (which hold the next panel) are updated on the solve's
                            stream, and the rest of the update runs on a second stream of the same
                            priority while the next panel is factored; the two are joined before
                            the next update.  -1 = one update per panel.  Bitwise the same factors */
} nl_config;

#define NL_MAX_HIST 128

/* Statistics of the last nl_solve on a handle (all host values). */
typedef struct {
    int status;                       /* nl_status of the solve */
    int mode;                         /* nl_mode */
    int newton_iters;                 /* Newton steps taken */
    int lu_nb;                        /* LU outer block used */
    double fnorm0;                    /* ||F(x0)||_2 */
    double fnorm;                     /* ||F||_2 of the returned iterate (the final one on NL_OK, else the best) */
    double hist[NL_MAX_HIST];         /* ||F(x_n)|| / ||F(x_0)||, n = 0..newton_iters */
    int lin_iters[NL_MAX_HIST];       /* per Newton step: IR corrections or GMRES Arnoldi steps
                                         (0 for the direct solves of NL_FP64LU, NL_F32, NL_F16) */
    int lin_outer[NL_MAX_HIST];       /* per Newton step: IR / GMRES-IR outer corrections */
    int lin_failed[NL_MAX_HIST];      /* per Newton step: IR failure rule fired (Section 3.1) */
    double lin_relres[NL_MAX_HIST];   /* per Newton step: final ||J32 u - b|| / ||b|| */
    double t_total_ms;                /* wall time of nl_solve (host clock) */
    double t_f_ms, t_jac_ms, t_lu_ms, t_lin_ms; /* device time per phase (CUDA events), summed */
    int gpu_launches;                 /* kernels launched by the solve */
    int lu_pivoted;                   /* factorisations that needed row interchanges (interchanging path) */
    int lu_tune_count;                /* autotuner candidates timed at nl_create (lu_nb = -1), else 0 */
    int lu_tune_nb[4];
    float lu_tune_ms[4];              /* factorisation time of each candidate */
    int reserved[5];
} nl_stats_t;

typedef struct nl_solver nl_solver;

/* Fill *cfg with the defaults.  Returns NL_EINVAL on NULL. */
nl_status nl_config_default(nl_config* cfg);

/* Create a solver for the H-equation of size N and albedo c (Section 3).
 * Allocates all device state for every mode except the double Jacobian
 * (allocated on the first NL_FP64LU solve) and the single-precision solve's
 * workspace (on the first NL_F32 solve).  N >= 1, 0 <= c < 1 (J(x*) is
 * singular at c = 1).  cfg may be NULL (defaults).  *out receives the handle,
 * owned by the caller until nl_destroy. */
nl_status nl_create(int64_t N, double c, const nl_config* cfg, nl_solver** out);

/* Use `stream` (cudaStream_t) for all later work of this handle. */
nl_status nl_set_stream(nl_solver* s, void* stream);

/* Newton solve from x0 (host, N doubles; NULL = ones) to
 * ||F(x)||_2 <= tol ||F(x0)||_2 + tau_a (Algorithm 1.1 / 2.1 with tau_r = tol).
 * The step uses the scaled right-hand side of eqs. (2.17)-(2.18): the linear
 * solver works on b = -F/||F|| and s = ||F|| u.  x_out (host, N doubles) gets
 * the final iterate on NL_OK; on any other status (NL_ENOTCONV, NL_ENUMERIC,
 * NL_ESINGULAR, NL_ETIMEOUT) the iterate with the smallest ||F|| seen, whose
 * norm is nl_stats_t.fnorm (after NL_ETIMEOUT the step that timed out is not
 * a candidate).  Blocks until done. */
nl_status nl_solve(nl_solver* s, const double* x0, double tol, nl_mode mode, double* x_out);

/* As nl_solve with x0 and x_out in device memory (x0 may be NULL = ones):
 * no host-device copy of vectors, only scalars are read back. */
nl_status nl_solve_device(nl_solver* s, const double* x0_dev, double tol, nl_mode mode, double* x_out_dev);

/* Copy the statistics of the last solve into *out (caller-owned). */
nl_status nl_stats(const nl_solver* s, nl_stats_t* out);

/* Bytes of device memory the handle holds. */
int64_t nl_device_bytes(const nl_solver* s);

/* Release the handle and its device memory.  NULL is a no-op. */
void nl_destroy(nl_solver* s);

/* Change the albedo c of an existing handle (its device state is reused; the
 * next solve starts from its own x0).  0 <= c < 1. */
nl_status nl_set_c(nl_solver* s, double c);

/* Device bytes a handle for N needs in `mode` (NL_FP64LU adds the double
 * Jacobian and its workspace, NL_F32 the single-precision solve's workspace,
 * gmres_factors32 with a GMRES-IR mode that workspace and the single-precision
 * factor copy), cfg as for nl_create (NULL = defaults).
 * -1 on invalid arguments.  Used for admission by memory footprint. */
int64_t nl_footprint_bytes(int64_t N, nl_mode mode, const nl_config* cfg);

/* Message of the last failing call on this thread ("" if none). */
const char* nl_last_error(void);

/* Per-kernel timing for measurement.  Returns the number of launches and the
 * summed device time (CUDA events on each launch's stream) of the kernel
 * class timed since the previous call, then starts timing `kernel_class`
 * (NULL or "" stops timing).  Classes: "k_panel16" (streaming panel),
 * "k_diag_lu16", "k_offdiag16" (half-precision LU, two-launch panel),
 * "k_diag_lu", "k_offdiag" (double LU), "k_tc_update32" (the two-level
 * LU's tensor-core inner updates), "k_lu_grouped_p" (the persistent grouped
 * LU), "k_tc_gemm" (tensor-core trailing
 * update), "k_tc_gemm_x" (its look-ahead part: the next panel's tile strips),
 * "k_invdiag" (diagonal-block inverses), "k_trsv_cl" (cluster
 * triangular solve), "k_trsv_mb" (mailbox triangular solve),
 * "k_lusolve16h" (binary16-arithmetic solve), "k_gemv_residual",
 * "k_residual" (F by the direct sum), "k_fft" (F by the FFT: its four
 * launches together).  Not
 * thread-safe against
 * concurrent solves on other threads.  Synchronises the recorded events. */
nl_status nl_kernel_timing(const char* kernel_class, int* launches, double* total_ms);

/* Library version string. */
const char* nl_version(void);

/* Test hook for the out-of-memory path: the next `count` device allocations
 * made for solver or batch handles (nl_create, the first NL_FP64LU / NL_F32
 * solve, nl_batch_create) fail as if the device were full, so those calls
 * return NL_ENOMEM and leave no handle behind.  0 turns it off.  NL_EINVAL
 * for count < 0. */
nl_status nl_debug_fail_allocs(int count);

/* ----------------------------------------------------------------------- */
/* Batched solves: many independent instances of eq. (3.2), each with its   */
/* own N and c, advanced together on the device.                            */
/* ----------------------------------------------------------------------- */

#define NL_BATCH_MAX_TUNE 48

/* Per-batch results of the last nl_batch_solve (host values). */
typedef struct {
    int count;              /* instances */
    int converged;          /* instances that met the tolerance */
    int parked_lu;          /* instances whose factorisation needed row interchanges (finished singly) */
    int parked_ir;          /* instances whose IR stalled (finished singly with GMRES-IR) */
    int newton_rounds;      /* executions of the batched Newton step */
    int ir_rounds;          /* executions of the batched IR correction */
    int lu_nb;              /* LU outer block of the bucket that holds the largest instance */
    int trailing_gemm;      /* that bucket's update: 1 SIMT, 2 tcgen05 (three launches per outer step);
                               3 / 4 one persistent launch, 64 x 64 / 128 x 64 SIMT update tiles;
                               5 one persistent launch, 128 x 128 tcgen05 update tiles */
    int gpu_launches;       /* kernels executed, including the single-instance completions */
    int graph_nodes_step;   /* kernel nodes in one batched Newton step (outside the IR loop) */
    int graph_nodes_ir;     /* kernel nodes in one IR correction */
    int tune_count;         /* autotuner candidates timed (all buckets) */
    int tune_bucket[NL_BATCH_MAX_TUNE];  /* the bucket each candidate was timed on */
    int tune_nb[NL_BATCH_MAX_TUNE];
    int tune_gemm[NL_BATCH_MAX_TUNE];
    double tune_ms[NL_BATCH_MAX_TUNE];   /* grouped LU time of the candidate on its bucket's first Jacobians */
    int nbuckets;           /* N buckets of the binary16 grouped LU, factored side by side */
    int bucket_nmax[8];     /* bucket b: bucket_nmax[b-1] < N <= bucket_nmax[b] (powers of two from 128) */
    int bucket_count[8];    /* instances in the bucket */
    int bucket_nb[8];       /* its outer block (the rounding period of its instances' factorisations) */
    int bucket_gemm[8];     /* its update / launch form, as trailing_gemm */
    int bucket_cached[8];   /* 1: the choice was read from the tuning table (NL_LU_TUNE_FILE) */
    double lu16_ms;         /* device time of one whole binary16 grouped LU of the batch (every bucket,
                               side by side) on the Jacobians at x0 = ones, best of 3 at creation */
    double t_total_ms;      /* host wall time of the solve */
    double t_graph_ms;      /* device time of the batched graph (CUDA events) */
    double t_single_ms;     /* host wall time of the single-instance completions */
    int reserved[16];
} nl_batch_info_t;

typedef struct nl_batch nl_batch;

/* Create a batch of `count` instances (N[i] in [1, 8192], 0 <= c[i] < 1).
 * All device state is allocated here (the double Jacobians on the first
 * NL_FP64LU solve).  cfg may be NULL; cfg->lu_path = 1 hands every instance to
 * the single-instance interchanging path at its first step (the batch then
 * factors nothing itself).  The instances are grouped by N into buckets
 * (N <= 128, 129..256, ..., 4097..8192); each bucket's binary16 grouped LU
 * runs on its own stream, side by side with the others, with its own outer
 * block nb (the rounding period of its instances' factorisations) and update.
 * cfg->lu_nb != 0 gives every bucket that nb (and cfg->trailing_gemm);
 * cfg->lu_nb = 0 lets the autotuner time each bucket alone, on the batch's
 * Jacobians at x0 = ones, for (nb, update) in {(128, tcgen05), (64, tcgen05),
 * (64, persistent tcgen05 128x128), (64, persistent SIMT 64x64), (64,
 * persistent SIMT 128x64), (32, persistent SIMT 64x64), (32, persistent SIMT
 * 128x64)} and keep the fastest (recorded in
 * nl_batch_info_t).  When the environment variable NL_LU_TUNE_FILE names a
 * file, the choices are kept there as JSON (one entry per device, SM count,
 * bucket range and instance count rounded up to a power of two), read by
 * later batches instead of timing, and written after tuning (a file that
 * cannot be read or written only costs the timing).  Vectors of the batch are packed:
 * instance i occupies entries [off_i, off_i + N[i]), off_i = N[0]+...+N[i-1]. */
nl_status nl_batch_create(int count, const int64_t* N, const double* c, const nl_config* cfg, nl_batch** out);

/* Solve every instance from x0 (host, packed; NULL = ones) to
 * ||F(x)|| <= tol ||F(x0)|| + tau_a.  mode: NL_IR16_GMRES (three precisions)
 * or NL_FP64LU.  The whole batched iteration is one CUDA graph with
 * conditional WHILE nodes (Newton steps, IR corrections); instances that need
 * row interchanges or whose IR stalls are finished on the single-instance
 * path (NL_IR16_GMRES semantics, or NL_FP64LU).  x_out: host, packed,
 * caller-owned.  Returns NL_OK when every instance met its tolerance,
 * otherwise the first failing instance's status. */
nl_status nl_batch_solve(nl_batch* b, const double* x0, double tol, nl_mode mode, double* x_out);

/* As nl_batch_solve with x0 (may be NULL) and x_out in device memory. */
nl_status nl_batch_solve_device(nl_batch* b, const double* x0_dev, double tol, nl_mode mode, double* x_out_dev);

/* Statistics of instance i in the last solve (hist relative to its own ||F(x0)||). */
nl_status nl_batch_stats(nl_batch* b, int i, nl_stats_t* out);

/* Batch-level results of the last solve. */
nl_status nl_batch_info(const nl_batch* b, nl_batch_info_t* out);

/* Use `stream` (cudaStream_t) for later solves of this batch. */
nl_status nl_batch_set_stream(nl_batch* b, void* stream);

/* Bytes of device memory the batch holds. */
int64_t nl_batch_device_bytes(const nl_batch* b);

/* Release the batch.  NULL is a no-op. */
void nl_batch_destroy(nl_batch* b);

/* ----------------------------------------------------------------------- */
/* Serving: a request loop that admits solves of different N and c as      */
/* device memory and execution slots free up, and runs them concurrently.  */
/* ----------------------------------------------------------------------- */

typedef struct {
    int64_t hbm_budget_bytes;  /* [64 GiB] device memory the server may hold (solver handles) */
    int max_inflight;          /* [8] requests on the device at once (one worker thread and stream each) */
    int mode;                  /* [NL_IR16_GMRES] nl_mode of every solve, NL_FP64LU .. NL_IR16_GMRES */
    double tol;                /* [1e-10] tau_r of every solve */
    int starve_ms;             /* [250] after the oldest waiting request has waited this long, no later
                                  request is admitted before it */
    int priority_n;            /* [1024] requests with N <= priority_n run on high-priority streams, so
                                  that their short kernels are scheduled ahead of large factorisations */
    int policy;                /* [1] admission order among arrived requests: 0 arrival order,
                                  1 smallest N first (shortest solve first) */
    nl_config solver;          /* solver parameters of every handle */
    int reserved[8];
} nl_server_config;

/* Per-request results. */
typedef struct {
    int status;          /* nl_status of the solve; -1 while pending or running */
    int N;
    double c;
    double t_arrive_s;   /* arrival, seconds after nl_server_start */
    double t_admit_s;    /* admission (handle and slot granted) */
    double t_done_s;     /* completion (x copied to the host) */
    double latency_ms;   /* t_done - t_arrive */
    int newton_iters;
    int handle_reused;   /* 1 if the solve ran on a cached handle (no allocation) */
    int reserved[6];
} nl_request_info_t;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t bytes_held, bytes_peak;  /* device bytes of the handles the server holds (now, peak) */
    int inflight_peak;               /* most requests on the device at once */
    int handles_created, handles_evicted;
    double p50_ms, p99_ms, mean_ms;  /* latency percentiles over completed requests */
    double span_s;                   /* first arrival to last completion */
    double solves_per_s;             /* completed / span_s */
    int reserved[8];
} nl_server_info_t;

typedef struct nl_server nl_server;

/* Defaults in brackets above (solver: nl_config_default). */
nl_status nl_server_config_default(nl_server_config* cfg);

/* Start a server (worker threads wait for nl_server_start).  The first call
 * initialises the library's kernels on the current device. */
nl_status nl_server_create(const nl_server_config* cfg, nl_server** out);

/* Queue a request for the H-equation of size N and albedo c, arriving
 * `arrival_s` seconds after nl_server_start (a negative value: now).  x0 =
 * ones.  *id receives the request id.  Thread-safe. */
nl_status nl_server_submit(nl_server* s, int64_t N, double c, double arrival_s, int64_t* id);

/* Start the arrival clock and admission.  Requests are admitted in arrival
 * order, skipping a request that does not fit in the memory budget for a
 * later one that does (until the starvation bound); each runs on its own
 * CUDA stream with its iterate, factors and Krylov basis on the device. */
nl_status nl_server_start(nl_server* s);

/* Result of request `id`.  wait != 0 blocks until it is done.  x_out (host,
 * N doubles) and stats may be NULL.  Returns NL_EINVAL for an unknown id. */
nl_status nl_server_result(nl_server* s, int64_t id, int wait, double* x_out, nl_stats_t* stats,
                           nl_request_info_t* info);

/* Wait until every submitted request is done (timeout_s <= 0: no limit);
 * NL_ETIMEOUT if the limit passed first. */
nl_status nl_server_drain(nl_server* s, double timeout_s);

/* Counters and latency percentiles so far. */
nl_status nl_server_info(nl_server* s, nl_server_info_t* out);

/* Stop the workers (pending requests are dropped) and release all memory. */
void nl_server_destroy(nl_server* s);

/* Grouped LU of `count` independent matrices (the batched factorisation of
 * Section 2's J_h, one launch per kernel class per outer step): A[i] (device,
 * N[i] x N[i], leading dimension ld[i], a multiple of 8) is factored in place
 * without row interchanges, checking exactly that partial pivoting would keep
 * every diagonal pivot (ipiv[i][k] = k).  flags_host[i] (host, count ints):
 * 0 = factored (identical to partial pivoting); 1 = partial pivoting would
 * interchange rows or a pivot is zero: A[i] is left partly factored and the
 * caller factors it with nl_lu16 / nl_lu64.  fp64 = 0: binary16 matrices,
 * arithmetic model as nl_lu16; fp64 = 1: double.  nb: multiple of 16 in
 * [16, 128] (0 = 128).  gemm: 0 auto, 1 SIMT, 2 tcgen05 (binary16, nb a
 * multiple of 64), 3 / 4 / 5: the whole factorisation as ONE persistent
 * launch (binary16, nb <= 64): CTAs take diagonal, off-diagonal and update
 * tasks from a device queue and wait (bounded) on per-matrix progress words;
 * the update tiles are 64 x 64 (3) or 128 x 64 (4) with the SIMT update's
 * arithmetic (factors bitwise those of gemm = 1), or 128 x 128 tcgen05 tiles
 * (5, nb = 64; factors bitwise those of gemm = 2).  A wait that gives up
 * returns NL_ETIMEOUT.  A, ipiv: host arrays of device pointers.
 * N[i] in [1, 32768].  With the tcgen05 update the entries of a row in
 * columns N[i] .. round_up(N[i], 8) - 1 (inside the leading dimension) may be
 * overwritten: the tensor-memory copies store whole 16-byte units at the
 * matrix's right edge.  Allocates its workspace with cudaMalloc.
 * Synchronises. */
nl_status nl_lu_grouped(int count, const int64_t* N, void* const* A, const int64_t* ld, int32_t* const* ipiv,
                        int fp64, int nb, int gemm, int32_t* flags_host, void* stream);

/* Test hook: the number of polls after which a dependency wait of the
 * persistent grouped LU gives up (0 = the default, about a second; negative =
 * at the first unmet poll).  A wait that gives up records a timeout in the
 * device error word, every later wait returns at once, the launch completes
 * (the tasks skip their work) and the call returns NL_ETIMEOUT; the context
 * stays usable.  Process-wide; for tests only. */
nl_status nl_debug_grouped_wait_limit(long long polls);

/* Per-task timing of the persistent grouped LU (nl_lu_grouped gemm 3 / 4 /
 * 5, batches with trailing_gemm 3 / 4 / 5), for measurement.  Returns in out9
 * (host, 9 doubles; may be NULL), for the task kinds diagonal block,
 * off-diagonal quad and update tile in that order, the tasks run and the
 * microseconds (SM clock cycles / the device's clock rate) summed over them
 * waiting for dependencies and working, since the previous call; then clears
 * the sums and switches the timing on (enable != 0) or off.  Synchronises the
 * device. */
nl_status nl_debug_grouped_task_times(int enable, double* out9);

/* Grouped b[i] <- U^{-1} L^{-1} P b[i] with the factors LU[i] (binary16
 * promoted to single on the fly, eq. (2.16), b single; or double), one CTA
 * per system, N[i] in [1, 8192].  LU, ipiv, b: host arrays of device pointers. */
nl_status nl_lusolve_grouped(int count, const int64_t* N, const void* const* LU, const int64_t* ld,
                             const int32_t* const* ipiv, void* const* b, int fp64, void* stream);

/* ----------------------------------------------------------------------- */
/* Kernel-level entry points (device pointers).  These expose each step of */
/* the hot path on its own, for tests and for callers with their own loop.  */
/* ----------------------------------------------------------------------- */

/* C <- C - A B on the tensor cores (tcgen05 kind::f16, binary32 accumulation
 * in tensor memory, one binary32 rounding per entry of C), the two-level
 * factorisation's inner update on its single-precision shadow (Section 2:
 * the elimination of J_h with binary16 multipliers and U entries, kept in
 * binary32 between roundings): C is M x Nc binary32, A is M x K and B is
 * K x Nc binary32 whose entries are binary16 values (other values are rounded
 * to binary16 on the way in); row-major device arrays, K <= 128, any M, Nc.
 * Rows and columns outside M x Nc are not touched. */
nl_status nl_k_update32(int64_t M, int64_t Nc, int64_t K, const float* A, int64_t lda, const float* B,
                        int64_t ldb, float* C, int64_t ldc, void* stream);

/* Residual of eq. (3.2) with the fused Newton update (Algorithm 1.1, last two
 * lines):  x_out = x + fnorm_scale * u  (u NULL: x_out = x), then
 *   r_i = (1 - c/(2N) sum_j x_out_j mu_i/(mu_j+mu_i))^{-1},  F_i = x_out_i - r_i,
 * all in double, and *fnorm_dev = ||F||_2.  u is single precision (the step
 * from the linear solver before unscaling, eq. (2.18)) or double when
 * u_is_double != 0.  x, x_out, F, r: N doubles; x_out must not alias x.
 * fnorm_dev: one device double. */
nl_status nl_k_residual(int64_t N, double c, const double* x, const void* u, int u_is_double,
                        double fnorm_scale, double* x_out, double* F, double* r, double* fnorm_dev,
                        void* stream);

/* The same residual, fused update and norm as nl_k_residual, with the sum of
 * eq. (3.2) evaluated in O(N log N) (Section 3): with z_m = x_(N-1-m) the sum
 * y_i = sum_j x_j h[i+j], h[k] = 1/(k+1), is the convolution (h * z)[i+N-1],
 * computed as a circular convolution of length L (the power of two >=
 * max(4, 2N)) by hand-written double-precision FFTs (four-step split into two
 * passes of radix-2 Stockham transforms in shared memory, twiddles from
 * sincospi).  Results differ from nl_k_residual by rounding only (about
 * 1e-14 relative to max|x| at N = 4096).  Allocates its workspace (16 L
 * doubles) with cudaMallocAsync; the transform of h is recomputed per call
 * (a solver handle keeps it). */
nl_status nl_k_residual_fft(int64_t N, double c, const double* x, const void* u, int u_is_double,
                            double fnorm_scale, double* x_out, double* F, double* r, double* fnorm_dev,
                            void* stream);

/* Analytic Jacobian of eq. (3.2) at x, given r from nl_k_residual:
 *   J_ij = delta_ij - (c/(2N)) r_i^2 mu_i/(mu_i+mu_j)   (Sections 1.1, 3),
 * written in one pass as J32 (single, computed in single from the double row
 * factor) and J16 = I_s^h(J32) (binary16, round to nearest even; Section 2).
 * Either output may be NULL.  Padding columns N..ld-1 are set to 0. */
nl_status nl_k_jacobian(int64_t N, double c, const double* r, float* J32, int64_t ld32, void* J16,
                        int64_t ld16, void* stream);

/* As nl_k_jacobian, with J16 scaled into the binary16 range row by row
 * (nl_config.scale_fp16; Section 2.3 on rounding into half precision):
 *   J16_ij = I_s^h(2^k_i J32_ij),  rs[i] = 2^k_i (device, N floats),
 * where 2^k_i is the largest power of two with 2^k_i B_i <= 2^13 for the row
 * bound B_i = 1 + c/(2N) r_i^2 >= max_j |J_ij|.  The factors of J16 then
 * factor R J; a solve with them is applied to R v to solve with J.
 * J32 is unscaled.  rs must not be NULL. */
nl_status nl_k_jacobian_scaled(int64_t N, double c, const double* r, float* J32, int64_t ld32, void* J16,
                               int64_t ld16, float* rs, void* stream);

/* The same Jacobian in double (for NL_FP64LU). */
nl_status nl_k_jacobian64(int64_t N, double c, const double* r, double* J64, int64_t ld, void* stream);

/* Half-precision LU with partial pivoting of A16 (N x N binary16, in place):
 * P A = L U with L unit lower (below the diagonal) and U upper, both binary16.
 * Arithmetic model: binary32 arithmetic, binary16 storage, L and U entries
 * rounded to binary16 as they are formed and the unfinished submatrix rounded
 * to binary16 every nb elimination steps (nb = outer block; the paper's
 * Section 2 says only that J_h is factored in half precision).
 * ipiv (device, N int32): LAPACK-style 0-based interchanges.  *info_host: 0,
 * or k+1 for the first exactly-zero pivot k (then NL_ESINGULAR).  nb: 0 = 128,
 * else a multiple of 16 in [16, 128], or 256, 384, 512 for the two-level
 * factorisation (nl_config.lu_nb; its workspace includes a single-precision
 * copy of the matrix).  gemm: 0 auto, 1 SIMT, 2 tcgen05.
 * path: 0 = factor first without interchanges, checking exactly that partial
 * pivoting keeps every diagonal pivot, and refactor with interchanges from a
 * saved copy of A if not (same result either way); 1 = interchanging path
 * only; 2 = as 0 with the diagonal block and the off-diagonal solves of each
 * panel in two launches instead of one streaming launch (same result);
 * 3 = every operation rounded to binary16 instead (l_ik = fl16(a_ik/a_kk),
 * a_ij <- fl16(a_ij - fl16(l_ik a_kj)) in increasing k, the first row of
 * largest |a_ik| as pivot): the arithmetic of the paper's F16 column; nb and
 * gemm are ignored, and *info_host is also set (to -1) after a binary16
 * overflow, returned as NL_ENUMERIC; 4 = as 0 with look-ahead
 * (nl_config.lu_lookahead; same result; the call creates and destroys a
 * second stream).
 * With the tcgen05 update the entries of a row in columns N ..
 * round_up(N, 8) - 1 (inside ld) may be overwritten (the tensor-memory copies
 * store whole 16-byte units at the matrix's right edge).
 * Allocates its workspace (and the copy) with cudaMallocAsync on
 * `stream`.  Synchronises the stream. */
nl_status nl_lu16(int64_t N, void* A16, int64_t ld, int32_t* ipiv, int nb, int gemm, int path, int32_t* info_host,
                  void* stream);

/* Double-precision LU with partial pivoting (the F64 baseline), same layout,
 * ipiv convention and path choice.  nb: 0 = 64, else a multiple of 16 in
 * [16, 128].  Synchronises the stream. */
nl_status nl_lu64(int64_t N, double* A, int64_t ld, int32_t* ipiv, int nb, int path, int32_t* info_host,
                  void* stream);

/* b <- U^{-1} L^{-1} P b with the binary16 factors of nl_lu16 promoted to
 * single on the fly (eq. (2.16)), b single precision (device, N floats).
 * Allocates its workspace with cudaMallocAsync.  Returns NL_ETIMEOUT if a
 * bounded wait gave up. Synchronises the stream. */
nl_status nl_lusolve16(int64_t N, const void* LU16, int64_t ld, const int32_t* ipiv, float* b, void* stream);

/* b <- U^{-1} L^{-1} P b in double with the factors of nl_lu64. */
nl_status nl_lusolve64(int64_t N, const double* LU, int64_t ld, const int32_t* ipiv, double* b, void* stream);

/* Single-precision LU with partial pivoting of A (N x N binary32, in place;
 * the F32 column of Section 1.3): binary32 storage and arithmetic (the
 * updates as fused multiply-adds), always the interchanging path.  Layout,
 * ipiv and info as nl_lu16.  nb: 0 = 128, else a multiple of 16 in
 * [16, 128].  Allocates its workspace with cudaMallocAsync; synchronises
 * the stream. */
nl_status nl_lu32(int64_t N, float* A, int64_t ld, int32_t* ipiv, int nb, int32_t* info_host, void* stream);

/* b <- U^{-1} L^{-1} P b in single with the factors of nl_lu32 (device, N
 * floats).  Returns NL_ETIMEOUT if a bounded wait gave up.  Synchronises the
 * stream. */
nl_status nl_lusolve32(int64_t N, const float* LU, int64_t ld, const int32_t* ipiv, float* b, void* stream);

/* b <- U^{-1} L^{-1} P b entirely in binary16 arithmetic with the factors of
 * nl_lu16 (the F16 column of Section 1.3): b16 binary16 (device, N values,
 * in place); the interchanges applied in order, then every product l_it x_t
 * and every difference rounded to binary16 (round to nearest even), the
 * forward solve taking row i's terms in increasing t, the backward solve in
 * decreasing t, and x_t = fl16(s_t / u_tt).  One CTA; synchronises the
 * stream. */
nl_status nl_lusolve16h(int64_t N, const void* LU16, int64_t ld, const int32_t* ipiv, void* b16, void* stream);

/* r = b - A u in single precision (Algorithm IR, residual line), A N x N
 * single row-major; *rnorm_dev = ||r||_2 (double, device). */
nl_status nl_k_gemv_residual(int64_t N, const float* A, int64_t ld, const float* b, const float* u, float* r,
                             double* rnorm_dev, void* stream);

/* out[i] = fl16(fl32(a[i] / b[i])) (device, n floats each): the multiplier
 * rounding l = fl16(a / u) of the half-precision LU (Section 2), as the LU
 * kernels compute it (a correctly rounded reciprocal, a product, and the IEEE
 * division wherever the product lies within a few single-precision units of a
 * binary16 rounding boundary).  For tests of that arithmetic. */
nl_status nl_k_div_round16(int64_t n, const float* a, const float* b, float* out, void* stream);

/* Trailing update of the half-precision LU:  C <- fl16(C - A B) with A M x K,
 * B K x Nc, C M x Nc binary16 row-major (lda, ldb, ldc), products accumulated
 * in single.  gemm: 1 SIMT (sequential fused multiply-adds over k),
 * 2 tcgen05 tensor cores (K a multiple of 64 up to 1024, lda/ldb/ldc multiples
 * of 8, pointers 16-byte aligned; the persistent kernel: one CTA per SM, TMA
 * loads of A, B and C and TMA stores of C, the K extent streamed through a
 * four-slot ring of 64-wide operand slabs while C stays in tensor memory, so
 * C is read and written once whatever K; loads and MMAs of one tile overlap
 * the epilogue of the previous one), 3 the same tensor-core arithmetic with
 * one CTA per 128 x 128 tile and K <= 256 (bitwise the same results as 2). */
nl_status nl_k_gemm16_update(int64_t M, int64_t Nc, int64_t K, const void* A, int64_t lda, const void* B,
                             int64_t ldb, void* C, int64_t ldc, int gemm, void* stream);

/* Same operation and results as nl_k_gemv_residual, for callers that cannot
 * allocate device memory: code running inside a fixed memory pool that owns
 * all of the device's memory, or a plug-in that must not grow the process's
 * device footprint.  The paper has no counterpart: this is a
 * packaging of the residual for such callers.
 * Scratch: a fixed 33 KB array inside the library image, held on every GPU
 * that loads the library until the process exits; no cudaMalloc or other
 * allocation happens.  Limit: 1 <= N <= 32768, else NL_EINVAL.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the one array per device, so calls whose work overlaps
 * on the GPU (different streams, no ordering between them) race and give
 * wrong norms; order them on one stream.  A, u: 16-byte aligned, ld a
 * multiple of 4, as for nl_k_gemv_residual. */
nl_status nl_k_gemv_residual_noalloc(int64_t N, const float* A, int64_t ld, const float* b, const float* u,
                                     float* r, double* rnorm_dev, void* stream);

/* IR / GMRES-IR for J32 u = b with given half-precision factors (Section 2.2):
 * u0 = 0; success at ||b - J32 u|| <= eta ||b||; failure when the residual
 * norm increases (the best iterate is returned, Section 3.1); at most maxit
 * outer corrections.  solver: 0 = IR, 2 = GMRES-IR (restart m, inner tol
 * gtol, gcycles cycles).  u: device, N floats (output).  stats_host (may be
 * NULL): int[4] = {linear iterations, outer corrections, failed, converged}
 * and relres_host (may be NULL): final relative residual.  Synchronises. */
nl_status nl_linsolve16(int64_t N, const float* J32, int64_t ld32, const void* LU16, int64_t ld16,
                        const int32_t* ipiv, const float* b, float* u, double eta, int maxit, int solver, int m,
                        double gtol, int gcycles, int32_t* stats_host, double* relres_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NEWTON3P_H */
