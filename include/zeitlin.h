/*
 * zeitlin.h -- C ABI of the GB300 (sm_103a) library for the per-time-step hot
 * path of the Zeitlin-Euler solver on the sphere with the isospectral midpoint
 * (IsoMP) integrator of Cifani, Viviani & Modin, "An efficient geometric method
 * for incompressible hydrodynamics on the sphere" (arXiv 2206.05466).
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Matrices are N x N complex128 in DEVICE memory, row-major, leading
 *    dimension N, real and imaginary parts interleaved: element (i, j) is
 *    ptr[2*(i*N + j)] + i*ptr[2*(i*N + j) + 1].  A pointer must be 16-byte
 *    aligned.  The caller owns every matrix; the library never frees one.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls that must read a device result to decide what to
 *    launch next (isomp_step, isomp_run) block the calling host thread.
 *  - The return value is a status: 0 success, > 0 a warning with the result
 *    written, < 0 an error.  zt_last_error() gives a message for the calling
 *    thread's last non-zero status.
 *  - A plan owns its workspace; calls on one plan must not run concurrently
 *    (on different streams or threads).  Different plans are independent.
 */
#ifndef ZEITLIN_H
#define ZEITLIN_H

#if defined(__GNUC__)
#define ZT_API __attribute__((visibility("default")))
#else
#define ZT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define ZT_OK              0
#define ZT_NOT_CONVERGED   1   /* maxit sweeps reached; W_{n+1} still written  */
#define ZT_EINVAL         -1   /* bad argument (size, pointer, alignment, h)   */
#define ZT_ENOMEM         -2   /* device or host allocation failed             */
#define ZT_ECUDA          -3   /* a CUDA runtime/driver call failed            */
#define ZT_ENONFINITE     -4   /* residual is NaN or Inf (input not finite)    */
#define ZT_ETIMEOUT       -5   /* a bounded device wait ran out                */

#define ZT_PRECISION_FP64   0  /* complex products in FP64 (DFMA)                 */
#define ZT_PRECISION_SPLIT  1  /* complex products as BF16 digit slices on tcgen05 */

#define ZT_FINAL_FRESH  0      /* W_{n+1} from products recomputed at the last iterate */
#define ZT_FINAL_REUSE  1      /* W_{n+1} from the products of the last sweep           */

#define ZT_FIRST_EXTRAPOLATED 0   /* first iterate W_n + (W_n - W_{n-1})/2 when the plan's previous
                                     step advanced the same W with the same h and converged; else W_n */
#define ZT_FIRST_WN           1   /* first iterate W_n                                             */

typedef struct zt_plan zt_plan;

/* Tuning knobs; zero fields take the library default. */
typedef struct zt_tuning {
    int slices;          /* SPLIT: digit slices per operand, 3..8 (default 7)        */
    int digit_bits;      /* SPLIT: bits per balanced digit, 6..8 (default 7)         */
    int exact_groups;    /* SPLIT: leading digit groups summed exactly (default 4)   */
    int final_mode;      /* ZT_FINAL_FRESH (default) or ZT_FINAL_REUSE               */
    int sweeps_per_sync; /* sweeps enqueued between host convergence checks, 1..64; 0 (default):
                            as many as the previous step took (4 for a plan's first step) */
    int dense;           /* SPLIT: 1 = multiply every digit pair; 0 (default) = skip digit-pair
                            tiles that are exactly zero (identical results)                  */
    int tile_order;      /* SPLIT launch order of output tiles: 0 (default) / 3 / 4 / 5 = column
                            blocks of 8 / 16 / 4 / 2 tiles, rows walked inside a block;
                            1 = row-major; 2 = tiles near the diagonal first; 6 = column
                            blocks of 8 from the last block to the first */
    int no_persistent;   /* SPLIT: 0 (default) = persistent product kernel (one CTA per SM working
                            through the tiles); 1 = one tile per CTA */
    int wait_us;         /* SPLIT: limit of each bounded wait inside the product kernel, in
                            microseconds (1 .. 60e6; default 2e6).  A wait that runs out makes
                            the call return ZT_ETIMEOUT; W is then unspecified */
    int debug_stall_loads; /* SPLIT, testing only: k > 0 stops the product kernel's operand
                            loads after k - 1 of them, so that its bounded waits run out and
                            the call returns ZT_ETIMEOUT (default 0: off) */
    int slices2;         /* SPLIT: digit slices of the second product of a sweep, B = Pt A^H
                            (Sec. 3.1), 2..slices; 0 (default) = slices.  B enters the update
                            (Eq. 9) and the final assembly (Eq. 8) scaled by h^2/4, so it needs
                            fewer digits than A = Pt Wt for the same error in W: Pt's digit
                            planes are truncated to their leading slices2 digits and A is split
                            into slices2 digits */
    int first_iterate;   /* ZT_FIRST_EXTRAPOLATED (default) or ZT_FIRST_WN: the fixed-point
                            iteration's starting point (Eq. 9 converges to the same Wt from either,
                            within tol; the extrapolated one is an O(h^2) guess and saves sweeps) */
    int second_form;     /* SPLIT: kernel form of the second product of a sweep: 0 (default) = that
                            of the first (no_persistent), 1 = one tile per CTA, 2 = persistent */
} zt_tuning;

typedef struct zt_step_stats {
    int    iters;        /* fixed-point sweeps taken                               */
    int    converged;    /* 1 if the residual fell below tol                       */
    double residual;     /* last ||Wt^{k+1} - Wt^k||_F                             */
} zt_step_stats;

typedef struct zt_run_stats {
    long   steps;        /* steps completed                                        */
    long   total_iters;  /* sweeps over all steps                                  */
    int    max_iters;    /* largest sweep count of one step                        */
    int    all_converged;/* 1 if every step converged                              */
    double max_residual; /* largest final residual of a step                       */
} zt_run_stats;

/* Create a plan for size N (1 <= N <= 16384) and precision ZT_PRECISION_*.
 * Plans allocate from the device's default stream-ordered memory pool; the
 * first plan on a device raises that pool's release threshold, so memory of
 * destroyed plans stays pooled for reuse (cudaMemPoolTrimTo returns it).
 * Precomputes, once, the tridiagonal blocks of Delta_N (Sec. 3.2, Eq.
 * 13) and their LDL^T factors (the factorisation behind the HPD
 * tridiagonal solve of Sec. 3.3), and allocates the step workspace (about
 * 6 N^2 complex values, plus the digit slices for ZT_PRECISION_SPLIT).
 * `opt` may be NULL.  On success *out receives the plan.  Errors: ZT_EINVAL,
 * ZT_ENOMEM, ZT_ECUDA.  Uses the current CUDA device. */
ZT_API int zt_plan_create(int N, int precision, const zt_tuning* opt, zt_plan** out);

/* Free a plan and its device workspace (NULL is ignored).  Synchronises the
 * device first. */
ZT_API void zt_plan_destroy(zt_plan* plan);

/* Message for the calling thread's last non-zero status ("" if none). */
ZT_API const char* zt_last_error(void);

/* W = Delta_N P (Sec. 3.2-3.3): the discrete Laplacian applied diagonal by
 * diagonal, each diagonal m (sub- and super-) through the tridiagonal block
 * -T_m of Eq. 13.  P is any complex N x N matrix; W must not alias P.
 * O(N^2).  Errors: ZT_EINVAL, ZT_ECUDA. */
ZT_API int zeitlin_laplacian_apply(zt_plan* plan, const double* P, double* W, void* stream);

/* P = Delta_N^{-1} W for W in su(N) (Sec. 3.3, Eq. 14): one
 * tridiagonal system per sub-diagonal m = 0..N-1, solved with the
 * precomputed factors; the l = 0 mode of the singular m = 0 block is
 * projected out (mean of the right-hand side and of the solution removed).
 * Only the lower triangle of W is read; the upper triangle of P is written as
 * -conj of the lower (skew-Hermitian), so P is in su(N).  W must not alias P.
 * O(N^2).  Errors: ZT_EINVAL, ZT_ECUDA. */
ZT_API int zeitlin_stream_solve(zt_plan* plan, const double* W, double* P, void* stream);

/* One IsoMP step in place, W = W_n on entry, W_{n+1} on return (Sec. 2,
 * Eqs. 8 and 9; products as in Sec. 3.1).  Fixed-point sweeps
 *   Pt = Delta_N^{-1} Wt,  A = Pt Wt,  B = A Pt,
 *   Wt <- W_n + h/2 (A - A^H) + h^2/4 B,   r = ||Wt_new - Wt_old||_F
 * until r < tol or maxit sweeps, then
 *   W_{n+1} = Wt + h/2 (A - A^H) - h^2/4 B.
 * The first iterate is W_n, or W_n + (W_n - W_{n-1})/2 when the plan's previous
 * step advanced this W buffer with this h and converged (zt_tuning.first_iterate,
 * zt_plan_reset_history): the fixed point, and W_{n+1}, are the same within tol.
 * W must be in su(N).  `stats` (host pointer, may be NULL) receives the sweep
 * count and last residual.  Blocks the host thread until the step is done.
 * Returns ZT_OK, ZT_NOT_CONVERGED (W_{n+1} written from the last iterate),
 * ZT_ENONFINITE, ZT_ETIMEOUT, ZT_EINVAL or ZT_ECUDA. */
ZT_API int isomp_step(zt_plan* plan, double* W, double h, double tol, int maxit,
               zt_step_stats* stats, void* stream);

/* nsteps IsoMP steps in place (same semantics as isomp_step for each step).
 * `stats` (host pointer, may be NULL) receives totals.  Stops at the first
 * error; a step that does not converge is reported in stats and in the
 * return value (ZT_NOT_CONVERGED) but the run continues. */
ZT_API int isomp_run(zt_plan* plan, double* W, double h, long nsteps, double tol,
              int maxit, zt_run_stats* stats, void* stream);

/* C = X Y for complex N x N X and skew-Hermitian Y (Y^H = -Y), in the plan's
 * precision: the product kernel of the step (Sec. 3.1, both factors of the
 * commutator products are in su(N)).  Only Y's skew-Hermitian structure is
 * used: C = -X conj(Y)^T.  Exposed for parity tests.  Errors: ZT_EINVAL,
 * ZT_ECUDA, ZT_ETIMEOUT. */
ZT_API int zt_zgemm_skew(zt_plan* plan, const double* X, const double* Y, double* C, void* stream);

/* Discrete Casimirs C_k = tr(W^k), k = 2..5 (Sec. 2, Eq. 7), computed on the
 * device with the plan's products (W^2 = W W and W^4 = W^2 W^2, split or FP64
 * as the plan) and FP64 conjugate dot products summed in a fixed order.
 * W: device, N x N complex128 row-major, skew-Hermitian (the identities used
 * rely on it).  C: HOST array of 8 doubles, (Re, Im) of C2, C3, C4, C5.  Uses
 * the plan's step workspace; waits for the stream before returning.  Status
 * as for the other calls (ZT_ETIMEOUT if a bounded device wait ran out). */
ZT_API int zeitlin_casimirs(zt_plan* plan, const double* W, double* C, void* stream);

/* Kinetic-energy spectrum (Sec. 4; basis of Sec. 3.2): E_l = sum_{|m| <= l}
 * |omega_lm|^2 / (2 l (l+1)) for l = 1 .. N-1 and E_0 = 0, with omega_lm the
 * coefficients of W in the quantised basis (Eq. 10) over every l <= N-1; the
 * E_l sum to the Hamiltonian (1/2) tr(P W), P = Delta_N^{-1} W.  W: device
 * N x N complex128 in su(N) (skew-Hermitian: only the lower triangle and the
 * diagonal are read, |omega_{l,-m}| = |omega_lm|); E: DEVICE array of N
 * doubles, caller-owned.  Asynchronous on the stream; uses the plan's step
 * workspace (not concurrently with a step of the same plan).  About N^3/6 FP64
 * recurrence steps, no eigenvector stored (GB300: ~0.26 s at N = 4096, growing
 * like N^3).  Errors: ZT_EINVAL (NULL plan, W not 16-byte or E not 8-byte
 * aligned), ZT_ECUDA (launch failure). */
ZT_API int zeitlin_energy_spectrum(zt_plan* plan, const double* W, double* E, void* stream);

/* ---- Quantised spherical-harmonic basis (Sec. 3.2, Eqs. 10-12) ----
 * T^_lm (0 <= m <= l) lies on the m-th lower diagonal; its entries there are
 * the unit eigenvector of the block -Delta^m for the eigenvalue l(l+1), with
 * the sign of Eq. 11 (last entry of the diagonal has the sign (-1)^m), and
 * T^_{l,-m} = (-1)^m T^_lm^T.  A basis holds T^_lm for l <= lmax on the plan's
 * device (about (lmax+1)(lmax+2)/2 * N doubles, twice during creation); the
 * plan is read only by zt_basis_create, so either may be destroyed first.
 * zt_basis_destroy waits for the launches that read the basis.  Coefficients
 * omega_lm are complex128 in a flat device array of (lmax+1)^2 entries at
 * l*l + l + m. */
typedef struct zt_basis zt_basis;
/* Computes the basis for 0 <= lmax <= N-1 and waits for it; *out receives the
 * handle (NULL on failure).  Errors: ZT_EINVAL (NULL plan or out, lmax out of
 * range), ZT_ENOMEM / ZT_ECUDA (device allocation or launch). */
ZT_API int zt_basis_create(zt_plan* plan, int lmax, zt_basis** out);
ZT_API void zt_basis_destroy(zt_basis* basis);   /* NULL: no-op */
/* Copies the N - m diagonal entries of T^_lm (0 <= m <= l <= lmax) to a HOST
 * array of N - m doubles (synchronous).  ZT_EINVAL outside that range. */
ZT_API int zt_basis_vector(zt_basis* basis, int l, int m, double* out);
/* W = sum_{l <= lmax, |m| <= l} i omega_lm T^_lm (Eq. 10); W: device N x N complex128,
 * overwritten (zero outside the band |m| <= lmax).  Asynchronous on the stream.
 * ZT_EINVAL for a NULL basis or a NULL / not 16-byte aligned pointer. */
ZT_API int zeitlin_w_from_omega(zt_basis* basis, const double* omega, double* W, void* stream);
/* omega_lm = -i tr(T^_lm^H W) for l <= lmax (the inverse of the above on the span of
 * the basis).  Asynchronous on the stream; errors as above. */
ZT_API int zeitlin_omega_from_w(zt_basis* basis, const double* W, double* omega, void* stream);

/* Device bytes a plan for (N, precision, tuning) allocates (for admission by
 * memory footprint); -1 for an invalid N.  `opt` may be NULL. */
ZT_API long long zt_plan_estimate_bytes(int N, int precision, const zt_tuning* opt);

/* Number of kernel launches the library enqueued since the plan was created
 * (every launch of every entry point on this plan). */
ZT_API long zt_plan_launch_count(const zt_plan* plan);

/* Forget the plan's step history (Eq. 9's first iterate, zt_tuning.first_iterate):
 * the next step starts from W_n.  For callers that rewrite W in place between
 * steps; the result is the same either way (within tol), only the sweep count
 * depends on the first iterate.  A NULL plan is ignored. */
ZT_API void zt_plan_reset_history(zt_plan* plan);

/* Measurement hook (no counterpart in the paper).  When enabled, the library
 * records a CUDA event pair on the launching stream around every launch of
 * the kernel classes below, and sums, per class, the elapsed time and the
 * algorithmic work of the launches that did work (sweeps skipped after
 * convergence are not counted).  Work units: ZT_KERNEL_PRODUCT -- tensor
 * FLOPs issued (SPLIT: 2 x 128 x 256 x 64 per digit-pair MMA unit actually
 * issued, counted on the device, so all-zero units skipped are not counted;
 * FP64: 8 flops per complex multiply-add over the computed tiles) and, in
 * work_alg, FP64-equivalent FLOPs of the complex product (8 N^3 for a full
 * product, 4 N^2 (N+1) for the lower triangle); ZT_KERNEL_SOLVE -- bytes
 * (lower triangle of W read, all of P written: 8 N (N+1) + 16 N^2);
 * ZT_KERNEL_SPLIT -- bytes read and written; ZT_KERNEL_UPDATE -- bytes.
 * zt_plan_set_timing(plan, 1) also clears the sums. */
#define ZT_KERNEL_PRODUCT 0
#define ZT_KERNEL_SOLVE   1
#define ZT_KERNEL_SPLIT   2
#define ZT_KERNEL_UPDATE  3
#define ZT_KERNEL_KINDS   4
ZT_API int zt_plan_set_timing(zt_plan* plan, int enable);
/* Totals for one kernel class since timing was enabled; synchronises on the
 * recorded events.  Any output pointer may be NULL. */
ZT_API int zt_plan_kernel_time(zt_plan* plan, int kind, long* launches, double* total_ms,
                               double* work, double* work_alg);

/* ---- Ensembles: grouped steps over many independent instances ----------
 *
 * A batch binds `count` existing plans (any mix of N and precision; split
 * instances must share the cluster shape, all must share the final mode),
 * their device state matrices W[i] (caller-owned, bound for the batch's
 * lifetime) and their time steps h[i].  One batched step advances every
 * instance by one IsoMP step exactly as isomp_step would, bit for bit, but
 * each kernel of the step is one grouped launch over all instances; each
 * instance keeps its own device convergence state, so instances that
 * converge early are masked off while the others keep sweeping (Sec. 2,
 * Eqs. 8-9, applied to an ensemble).  A plan may belong to one batch at a
 * time and must not be stepped on its own while the batch is in use. */
typedef struct zt_batch zt_batch;
ZT_API int zt_batch_create(int count, zt_plan* const* plans, double* const* W, const double* h, zt_batch** out);
ZT_API void zt_batch_destroy(zt_batch* batch);
/* Capture the step's launch sequence into CUDA graphs on the next step and
 * replay them afterwards (1 = on, 0 = off; default off). */
ZT_API int zt_batch_set_graph(zt_batch* batch, int enable);
/* One step of every instance.  `stats` (host array of `count`, may be NULL)
 * receives each instance's sweeps and residual.  Blocks the host thread until
 * the step is done (one synchronisation per step while all instances converge
 * within sweeps_per_sync sweeps).  Returns the worst status over instances. */
ZT_API int isomp_step_batched(zt_batch* batch, double tol, int maxit, zt_step_stats* stats, void* stream);
/* nsteps batched steps; `stats` receives totals over all instances and steps. */
ZT_API int isomp_run_batched(zt_batch* batch, long nsteps, double tol, int maxit, zt_run_stats* stats,
                             void* stream);
/* Kernel launches enqueued by the batch so far. */
ZT_API long zt_batch_launch_count(const zt_batch* batch);

/* Allocation-free split-precision product (no counterpart in the paper).
 *
 * Computes the same C = X Y, Y skew-Hermitian, as zt_zgemm_skew with a
 * ZT_PRECISION_SPLIT plan at the default tuning (7 slices of 7 bits), but
 * needs no plan and never allocates device or pinned memory: it is meant for
 * callers that cannot call cudaMalloc -- a serving process that reserved all
 * of the device memory for resident simulation state at start-up, code
 * embedded in a host application whose own allocator owns the device, or a
 * time-critical loop that must not hit the implicit device synchronisation
 * of cudaMalloc/cudaFree.
 *
 * Its scratch (digit planes, row exponents, a status word) is one file-scope
 * device array of ZT_NOALLOC_SCRATCH_BYTES (about 5.5 MB); every GPU that
 * loads the library holds it until the process exits.  N is limited to
 * 1 <= N <= ZT_NOALLOC_MAX_N; larger N returns ZT_EINVAL.  X, Y, C are
 * caller-owned device matrices as for zt_zgemm_skew (C must not alias X or
 * Y).  The first call on each device resolves the device address of the
 * array (cudaGetSymbolAddress) and sets the kernel's shared-memory limit;
 * make that first call before any stream capture.  Every call clears the
 * array on `stream` before use, so no state carries over between calls, but
 * all calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Blocks the host thread until the product is done.  Errors: ZT_EINVAL,
 * ZT_ECUDA, ZT_ETIMEOUT. */
#define ZT_NOALLOC_MAX_N 256
#define ZT_NOALLOC_SCRATCH_BYTES 5508352
ZT_API int zt_zgemm_skew_split_noalloc(int N, const double* X, const double* Y, double* C, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ZEITLIN_H */
