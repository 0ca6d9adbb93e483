/*
 * lgk.h -- C ABI of the batched-ADMM Gamma Knife planning library (liblgk.so).
 *
 * Solves the dual linear program of Lightning inverse planning (arXiv
 * 2509.08602, Eq. dual_problem and Appendix A)
 *
 *     minimize c^T x   subject to   A x <= b,   l <= x <= u
 *
 * for K objective weightings at once with the scaled-form ADMM of Sec. 2.B
 * (Eq. admm, with the x-step in the closed form of Eq. partial_elimination),
 * all K weightings sharing one matrix A and one cached inverse of
 * S = A A^T + I.  Everything runs on one CUDA device.
 *
 * Conventions (every entry point):
 *  - The return value is an lgk_status; 0 is success.  No C++ exception and no
 *    abort crosses this boundary.  On failure lgk_last_error() returns a
 *    thread-local message describing the last error.
 *  - Input arrays are HOST pointers owned by the caller; the library copies
 *    what it needs before returning and never keeps a caller pointer.
 *  - Output arrays are HOST pointers owned by the caller, sized as stated.
 *  - lgk_case and lgk_result are opaque and owned by the library until
 *    lgk_destroy_case / lgk_free_result.  A result keeps its case alive
 *    (a case may be destroyed while results of it exist).
 *  - One lgk_case may be used by one host thread at a time.  Different cases
 *    may be used concurrently from different threads.
 *  - All arrays are row-major (C order).
 */
#ifndef LGK_H
#define LGK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lgk_case lgk_case;
typedef struct lgk_result lgk_result;

typedef enum {
    LGK_OK = 0,
    LGK_EINVAL = 1,    /* invalid argument (sizes, NaN/Inf, class codes, ...)      */
    LGK_ENOMEM = 2,    /* device or host allocation failed                         */
    LGK_EBUDGET = 3,   /* case footprint exceeds lgk_params.hbm_budget             */
    LGK_ENOTPD = 4,    /* S = A A^T + I not positive definite in FP64 (Cholesky)   */
    LGK_ECUDA = 5,     /* CUDA runtime/driver error, or a device-side error flag   */
    LGK_ETIMEOUT = 6   /* a bounded wait (host poll or device barrier) ran out     */
} lgk_status;

/* Dose-point classes (Sec. 2.A; Appendix A block names TS, TI, R, LD, O). */
enum { LGK_TS = 0, LGK_TI = 1, LGK_R = 2, LGK_LD1 = 3, LGK_LD2 = 4, LGK_OAR = 5 };

/* Arithmetic of the ADMM iterations.
 *  LGK_PREC_FP32:   A, S^{-1} and the iterates in FP32, all GEMMs in FP32 on
 *                   CUDA cores through cuBLAS (the plain GPU form, the
 *                   paper's own precision: Sec. 3.A).  Comparison form.
 *  LGK_PREC_BF16:   A rounded once to BF16 (8 significant bits), iterates as
 *                   two BF16 terms, 2 tensor-core products per GEMM.  Fast,
 *                   but the LP solved is the one with the rounded matrix: on
 *                   the synthetic cases its plans' beam-on time moves ~1 %.
 *  LGK_PREC_BF16X3: A as two BF16 terms (hi + lo, ~16 bits) and the iterates
 *                   as two BF16 terms, 3 products per GEMM (hi.hi + hi.lo +
 *                   lo.hi); the plans match FP64 ones.  Product form, default.
 *  In both BF16 forms S^{-1} and the solve input are split into three BF16
 *  terms (6 products), accumulation is FP32 in tensor memory, and S is formed
 *  and inverted in FP64 from exactly the matrix the GEMMs use.               */
enum { LGK_PREC_FP32 = 0, LGK_PREC_BF16 = 1, LGK_PREC_BF16X3 = 2 };

typedef struct {
    int n_iso;               /* N isocenters; beam variables B = 24 N (8 sectors x 3 collimators) */
    int n_pts;               /* P dose points                                                   */
    int n_targets;           /* >= 1; TS/TI/R points carry a target index                       */
    int n_oars;              /* >= 0; OAR points carry an OAR index                             */
    const double* phi;       /* P x B dose-rate kernels, Gy/min.  Beam index
                                b = (i*8 + s)*3 + c (isocenter, sector, collimator)             */
    const uint8_t* kind;     /* P point classes LGK_TS..LGK_OAR                                 */
    const uint16_t* struct_id; /* P: target index (TS/TI/R), OAR index (OAR), ignored (LD)      */
    const double* d_presc;   /* n_targets prescription doses D_T (> 0), Gy                      */
    const double* q_area;    /* n_targets shares of total target area   (Appendix A, q_kA)      */
    const double* q_vol;     /* n_targets shares of total target volume (Appendix A, q_kV)      */
    const double* d_oar;     /* n_oars maximum doses D_O (> 0), Gy; may be NULL if n_oars = 0   */
    double d_ld1, d_ld2;     /* low-dose thresholds (> 0), Gy (Appendix A)                      */
    double phi_cal;          /* calibration dose rate, Gy/min (3 in Sec. 3.B)                   */
} lgk_case_desc;

typedef struct {
    int precision;           /* LGK_PREC_*; default LGK_PREC_BF16X3                             */
    int normalize_rows;      /* Sec. 3.C unit-norm rows of A (scales b too); default 1          */
    int scale_bot;           /* Sec. 3.C beta scaling of the BOT columns; default 1             */
    int check_every;         /* iterations between residual tests; default 10                   */
    double eps_abs;          /* absolute residual floor per sqrt(n+m); default 1e-12            */
    int device;              /* CUDA device ordinal; default 0                                   */
    void* stream;            /* cudaStream_t to run on, or NULL for a library-owned stream     */
    size_t hbm_budget;       /* bytes; 0 = no limit.  create_case fails with LGK_EBUDGET when
                                the case's resident footprint would exceed it                  */
    int timeout_ms;          /* bound on any single host wait; default 600000                   */
    int profile;             /* 1: time every kernel of every iteration with CUDA events
                                (read by lgk_fetch_profile); default 0                       */
    int lo_refresh;          /* LGK_PREC_BF16X3 only.  1 (default): iterate with the high BF16
                                term of A and add the low term's product from the last full
                                iteration (lo R1 and lo^T v, kept in FP32); the solve's first
                                iteration and every residual-test iteration use both terms
                                and refresh those products.  The fixed point, hence every
                                converged plan, is that of the two-term A; the heavy products
                                read half the bytes.
                                0: both terms every iteration (the literal iteration).      */
    int lo_refresh_iters;    /* with lo_refresh = 1: once a solve has run this many iterations
                                with columns still active (a stream: once its oldest running
                                column has), it continues with the literal iteration (a
                                safety net for columns the lagged products slow down);
                                0 = never.  Default 8000.                                   */
    int rho_adapt;           /* 1: adapt each column's rho during the solve by residual
                                balancing (Boyd et al., Sec. 3.4.1 of their ADMM monograph):
                                at every graph replay boundary (5 x check_every iterations),
                                with the relative residuals of that iteration's test, rho is
                                multiplied by 1.5 when rel_pri > 3 rel_dual and divided by
                                1.5 when rel_dual > 3 rel_pri, at most 40 times per column
                                (then fixed, so the iteration converges as with a fixed rho).
                                S = A A^T + I does not depend on rho (Sec. 2.B), so a change
                                only rescales the column's scaled duals y by rho_old/rho_new
                                (the multipliers rho y are unchanged).  The stop test and
                                the reported plans use the column's current rho.
                                0 (default): rho fixed per column (Eq. rho_rule or caller's). */
    int solve_refine;        /* BF16 forms: iterative refinement steps of the x-update's solve
                                per iteration, 0..2 (default 0; see also refine_after).  v = S^{-1} rhs is a product
                                with the explicit inverse whose FP32 sums lose accuracy when
                                rhs is large along the directions S magnifies (v is then
                                ~1000x smaller than rhs); each step computes the residual
                                e = rhs - S v (with S kept as three BF16 terms, 6 products)
                                and adds S^{-1} e, so A x1 - x2 = rhs - S v (Sec. 2.B) is
                                held to the product's accuracy instead.  Each step costs two
                                solve-sized products; S takes 6 m^2 more device bytes.      */
    int setup_fp64;          /* BF16 forms: 1 forms S = A A^T + I with FP64 products on the CUDA
                                cores (exact from the rounded A; slow on this GPU's FP64 rate);
                                0 (default): on the tensor cores from A's BF16 terms (exact
                                products, FP32 sums over 128 columns of A, FP64 sums of those;
                                about 1e-6 relative error per entry).  The FP32 form always
                                uses FP64 products.                                          */
    int check_fp64;          /* 1: the plan check (lgk_fetch_check, stream checks) forms A z1 and
                                A^T lam with FP64 products on the CUDA cores; 0 (default): on
                                the tensor cores from exact BF16 splits, FP32 sums over 64
                                columns, FP64 across them (two-term BF16 form only).        */
    int autotune;            /* 1: the first solve of a case at a given column count times each
                                GEMM configuration on one replay of the real iteration (256- or
                                128-row tiles for the A GEMMs where both exist; the solve's
                                column tile whole or halved) and keeps the fastest for later
                                solves of that case and count.  The configurations sum in
                                different orders, so plans then differ in rounding from an
                                untuned solve.  0 (default): the fixed rule.                 */
    int refine_after;        /* BF16 forms with solve_refine = 0: a column that has run this many
                                iterations of its weighting (counted from the weighting's own
                                start, also in a stream) continues with one refinement step of
                                the solve per iteration (as solve_refine = 1) until it stops.
                                The other columns feed a zero correction to the refinement
                                (their arithmetic is bitwise the unrefined one), so a
                                weighting's plan does not depend on the columns beside it.
                                Columns whose residuals level off above tol (the explicit-
                                inverse solve's accuracy floor, near 5e-5 on the 5000 x 61600
                                case) then converge.  The refined iteration costs two more
                                solve-sized products for every column once any column needs
                                it.  Needs S's three BF16 terms (6 m^2 device bytes, kept
                                whenever this is > 0).  0 = never.  Default 4000.             */
    int l2_keep_inverse;     /* BF16 forms: 1 keeps S^{-1}'s three BF16 terms (6 m^2 bytes) in L2
                                across iterations while a solve runs: a persisting L2 carve-out
                                of up to the device's limit (cudaLimitPersistingL2CacheSize, a
                                setting of the calling process's context, set back to 0 when
                                the solve returns) and evict-last loads of the inverse in the
                                solve.  Changes no result.  Concurrent solves in one process
                                share the carve-out.  0 (default): default L2 policy.         */
    int gemm2_tile_rows;     /* BF16 forms: rows of A^T per output tile of GEMM2 (the q1 step's
                                product), 128 or 256 (256 where the operand and the column
                                count allow it), or 0 (default) for GEMM1's height.  Changes the
                                summation order (results differ in rounding).  The autotuner
                                chooses it on its own.                                        */
    int accum_kblocks;       /* BF16 forms: GEMM1 (A . R1, a sum over all n columns of A) keeps at
                                most this many 64-column blocks in one tensor-memory
                                accumulator; longer k ranges are cut into more stream-K partial
                                sums, added in k order (round to nearest) by the next kernel.
                                The tensor cores' FP32 accumulation over a long chain drifts
                                (on the 8325 x 122664 case, chains of ~430 blocks left the
                                plans' FP64 duality gap at 1-3e-3; 64 brings it to ~1e-4).
                                Default 64; 0: no limit.                                     */
} lgk_params;

/* Fills *p with the defaults above.  Returns LGK_EINVAL if p is NULL. */
int lgk_default_params(lgk_params* p);

/*
 * lgk_create_case -- assemble and prepare one planning case on the device.
 *
 * Builds A of Appendix A (rows: 24 N beam variables then N isocenter rows;
 * columns: the P points in input order then 8 N BOT columns):
 *   A = [ phi_TS^T/D  phi_TI^T/D  -phi_R^T/D  -phi_LD^T/D_LD  -phi_O^T/D_O  -C_S^T ]
 *       [     0           0           0            0              0         T^T   ]
 * with C = I_N (x) I_8 (x) 1_{1x3}, T = I_N (x) 1_{8x1}, C_S = C phi_cal / D_T,mean;
 * normalises its rows and scales the BOT columns by
 * beta = (#non-OAR points)/2000 (Sec. 3.C); forms S = A A^T + I in FP64,
 * factors it (FP64 Cholesky, Sec. 2.B "cache a decomposition") and keeps its
 * inverse resident (Sec. 3.A keeps the explicit inverse).
 *
 * desc, p: host structs (p may be NULL for defaults).  *out receives the case.
 * Errors: LGK_EINVAL (bad sizes/classes/NaN), LGK_EBUDGET, LGK_ENOMEM,
 * LGK_ENOTPD, LGK_ECUDA.  On error *out is set to NULL.  The scalar fields
 * and the point classes are checked on the host before any CUDA call; the
 * dose rates phi (n_pts x 24 n_iso, up to GBs) are checked on the device as
 * A is assembled from them: a NaN, infinite or negative entry also returns
 * LGK_EINVAL, after the copy to the device.
 */
int lgk_create_case(const lgk_case_desc* desc, const lgk_params* p, lgk_case** out);

/* Sizes of a case: m rows, n columns of A, beta applied, device bytes held. */
int lgk_case_info(const lgk_case* cs, int* m, int* n, double* beta, size_t* bytes);

/*
 * lgk_solve_weightings -- run batched ADMM for K weightings (Sec. 2.B).
 *
 * W:   K x 4 host array (w_T, w_R, w_LD, w_BOT) >= 0 per weighting (Sec. 2.A).
 *      Bounds per Appendix A: u = (q_kA w_T / N_kTS, q_kV w_T / N_kTI,
 *      (w_R / n_targets) / N_kR, w_LD / N_LD1, w_LD / N_LD2, inf, inf),
 *      l = 0, b = (0, w_BOT) (times the row scale).
 * rho: K host values > 0, or NULL for the rule of Eq. rho_rule,
 *      rho = rho0 * sqrt(w0_bot / w_BOT) (w0_bot, rho0 > 0 then required).
 * tol: relative primal/dual residual tolerance of the stop test; 0 runs
 *      exactly max_iter iterations for every column.
 * max_iter: > 0.  State starts at zero (z = y = 0).
 * Stop test (every check_every iterations, per column): with r = x - z and
 *   s = rho (z - z_prev), stop once ||r|| <= eps_abs sqrt(n+m) + tol max(||x||,||z||)
 *   and ||s|| <= eps_abs sqrt(n+m) + tol ||rho y||.  A stopped column is frozen.
 * Blocks until every column has stopped or reached max_iter.
 * *out receives the result (library-owned).  Non-convergence is reported per
 * column by lgk_fetch_stats, not as an error.
 * Errors: LGK_EINVAL, LGK_ENOMEM, LGK_ECUDA, LGK_ETIMEOUT.
 */
int lgk_solve_weightings(lgk_case* cs, int K, const double* W, const double* rho,
                         double w0_bot, double rho0, double tol, int max_iter,
                         lgk_result** out);

/*
 * lgk_solve_group -- G (1..4) cases of different sizes solved together, each
 * with its own weighting set, every tensor-core product of an iteration one
 * persistent launch over all of them (the co-scheduled batched form: a small
 * case's products ride in the launches of a large one instead of paying
 * their own ramp and tail), captured in CUDA graphs.  Each case runs the
 * iteration of lgk_solve_weightings (Sec. 2.B, Eq. admm) on its own K columns
 * with its own control block and stop test; every case's products are cut
 * into the same stream-K runs and summed in the same order as in a solve of
 * that case alone, so each result is bitwise that of lgk_solve_weightings
 * with the same arguments, as long as the group runs on the tile heights the
 * case would take alone (256-row tiles need every case to allow them) and no
 * other member reaches lo_refresh_iters first: once the oldest running member
 * passes lo_refresh_iters, the whole group continues with the literal
 * iteration.  refine_after does not apply in a group, and autotune is
 * ignored.
 *   cases: G distinct cases on one device; all BF16 forms with the same
 *          lo_refresh, solve_refine and check_every (else LGK_EINVAL).
 *   K, W, rho: per case, as in lgk_solve_weightings (rho may be NULL, or
 *          rho[g] NULL, for Eq. rho_rule with w0_bot and rho0[g]).
 *   tol, max_iter: shared by the group.
 *   out: G result handles (host array), each freed with lgk_free_result.
 * The group runs on the first case's stream.  256-row tiles are used only
 * when every case can take them.  On error no result is returned.
 * Errors: LGK_EINVAL, LGK_ENOMEM, LGK_ECUDA, LGK_ETIMEOUT (the first case's
 * timeout_ms bounds the whole group).
 */
int lgk_solve_group(int G, lgk_case* const* cases, const int* K, const double* const* W,
                    const double* const* rho, double w0_bot, const double* rho0, double tol,
                    int max_iter, lgk_result** out);

/*
 * lgk_solve_weightings_async -- lgk_solve_weightings without blocking.
 *
 * Same arguments, checks and iteration (Sec. 2.B) as lgk_solve_weightings;
 * the solve runs on a library thread and *out is returned at once.  Until
 * lgk_wait(*out, ...) has returned LGK_OK, every fetch on *out returns
 * LGK_EINVAL, and the case is busy: another solve of it returns LGK_EINVAL.
 * W and rho are copied before the call returns.  Freeing the result while
 * the solve runs stops the solve at its next graph replay (within 5 residual-
 * test intervals) and waits for that.
 */
int lgk_solve_weightings_async(lgk_case* cs, int K, const double* W, const double* rho,
                               double w0_bot, double rho0, double tol, int max_iter,
                               lgk_result** out);

/*
 * lgk_wait -- wait at most timeout_ms (>= 0; 0 polls) for the asynchronous
 * solve of res.  LGK_OK once it finished successfully (the result may then be
 * fetched); LGK_ETIMEOUT if it is still running (call again later); the
 * solve's own error code if it failed.  A result from any other solve call
 * returns LGK_OK at once.
 */
int lgk_wait(lgk_result* res, int timeout_ms);

/* Sector times t (K x 24N, minutes) and isocenter beam-on times tau (K x N,
 * normalised units of the LP) of each plan: the multipliers rho * y2 of
 * A x <= b, unscaled by the row scale (Sec. 2.B: the primal solution is rho y*).
 * Either pointer may be NULL. */
int lgk_fetch_times(const lgk_result* res, double* t, double* tau);

/* Doses of each plan on caller points: dose = phi_eval t (Sec. 4: the dose is
 * the dose-rate kernels weighted by the sector times).  phi_eval is n_eval x 24N
 * (host), dose is K x n_eval (host).  Computed on the device in FP64. */
int lgk_fetch_doses(const lgk_result* res, const double* phi_eval, int n_eval, double* dose);

/*
 * lgk_fetch_doses_device -- allocation-free variant of lgk_fetch_doses.
 *
 * For callers that must not allocate device memory at run time: code whose
 * device memory is owned by another framework's pool or a fixed arena,
 * real-time loops that cannot afford an allocator's latency or its implicit
 * device synchronisation, and callers that have reserved all of the GPU's
 * memory up front.  Such callers pass their own device buffers and this call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * The paper has no counterpart of this entry point; it is a convenience of
 * this library.
 *
 * Computes dose = phi_eval t exactly as lgk_fetch_doses does (FP64, same
 * kernel), for the K plans of `res`:
 *   phi_eval_dev  DEVICE pointer, n_eval x 24N FP64 row-major, on the case's
 *                 device (checked; host or other-device pointers are rejected)
 *   dose_dev      DEVICE pointer, K x n_eval FP64 row-major, written
 * The plans' sector times (K x 24N FP64) are staged in a scratch array that
 * the library keeps in static device memory: LGK_NOALLOC_MAX_TIMES doubles
 * (32 MiB), held on every GPU that loads the library until the process exits.
 * K x 24N above that limit returns LGK_EINVAL (split the plans into smaller
 * batches).  Every element of the scratch that is read is first written by
 * the same call, so nothing carries over from one call to the next; but all
 * calls share the one array, so calls that overlap on the GPU (from several
 * host threads, or on several streams) race with each other and must be
 * serialised by the caller.
 * The first call on a device looks up the scratch array's device address;
 * make that first call before any stream capture.  Every later call made
 * outside a stream capture looks the address up again, so an address found
 * before a device reset is not reused after it.
 * Ordering: the call runs on the case's stream (lgk_params.stream, or the
 * library's own), not on the caller's.  The caller must finish writing
 * phi_eval_dev before the call (e.g. synchronise the stream that wrote it);
 * the call synchronises the case's stream before it returns, so dose_dev is
 * complete on return.  The caller's current device is unchanged on return.
 * Errors: LGK_EINVAL, LGK_ECUDA.
 */
#define LGK_NOALLOC_MAX_TIMES (1 << 22)
int lgk_fetch_doses_device(const lgk_result* res, const double* phi_eval_dev, int n_eval,
                           double* dose_dev);

/*
 * lgk_fetch_metrics -- clinical metrics of every plan, on the device.
 *
 * Definitions of Sec. 2.A with the conventions of Sec. 3.B, evaluated on
 * caller points (e.g. a regular grid) from the doses d = phi_eval t:
 *   coverage    = |target AND d >= D_k| / |target|      (D_k: the point's target)
 *   selectivity = |target AND d >= D_k| / |d >= min_k D_k|
 *   gi          = |d >= D/2| / |d >= D|  (NaN unless all prescriptions are equal)
 *   bot         = sum over isocenters of the longest sector time (its collimator
 *                 times summed), minutes
 * phi_eval: n_eval x 24N (host); label: n_eval target index per point, -1
 * outside every target (host).  Outputs: K values each (host; any may be
 * NULL).  Counts are exact integers on the device (FP64 doses), so the
 * metrics do not depend on the evaluation order.
 */
int lgk_fetch_metrics(const lgk_result* res, const double* phi_eval, int n_eval, const int* label,
                      double* coverage, double* selectivity, double* gi, double* bot);

/* Per-column statistics (each pointer may be NULL; arrays of K):
 * iterations run, dual objective c^T z1 (FP64 on the device), relative primal
 * and dual residuals at the last test, converged flag. */
int lgk_fetch_stats(const lgk_result* res, int* iters, double* obj, double* rel_pri,
                    double* rel_dual, uint8_t* converged);

/*
 * lgk_fetch_check -- FP64 check of each plan against its exact LP.
 *
 * Sec. 2.B recovers the plan (sector and isocenter times) from the scaled
 * multipliers rho y2 of the final iterate; the iterations themselves run in
 * BF16/FP32 and stop on FP32 residual sums.  This call re-evaluates every
 * column on the device in FP64, from z1 = clip(q1, 0, u) and
 * lam = rho max(q2 - b, 0) as the library holds them, against the LP of
 * Eq. dual_problem with its bounds u and b computed in FP64 (Appendix A), and
 * with A the matrix the iterations use (its BF16 terms summed exactly, or its
 * FP32 copy).  A z1 and A^T lam: for the two-term BF16 form on the tensor
 * cores from exact splits (z1 exactly, lam to 2^-24, in three BF16 terms),
 * exact products, FP32 sums over 64 columns and FP64 sums across them; for
 * the other forms, or with lgk_params.check_fp64, FP64 dot products on the
 * CUDA cores (slow on this part's FP64 rate).  Everything after the two
 * products is FP64.
 * out: K x LGK_CHECK_COUNT host array, per column:
 *   LGK_CHECK_OBJ        c^T z1 (the dual LP's objective)
 *   LGK_CHECK_PLAN       b^T lam + sum over finite-u columns of u (-(c + A^T lam))_+:
 *                        the weighted-sum objective of Sec. 2.A at the plan
 *   LGK_CHECK_GAP        (c^T z1 + plan) / max(1, |c^T z1|): relative duality gap
 *                        (the optimum lies between -plan and c^T z1 when both
 *                        points are feasible)
 *   LGK_CHECK_INFEAS     ||(A z1 - b)_+||_2 / ||b||_2
 *   LGK_CHECK_INFEAS_ABS ||(A z1 - b)_+||_2
 *   LGK_CHECK_HARD       max over u = inf columns (organ limits, BOT coupling)
 *                        of (-(c + A^T lam))_+, divided by max lam
 *   LGK_CHECK_BOUND      max over finite-u columns of (z1 - u)_+ (the iterations
 *                        clip to FP32 copies of u)
 *   LGK_CHECK_PRIMAL     ||(A z1 - b)_+||_2 / ((1 + ||A||_2) ||z||_2), z = (z1, min(q2, b)),
 *                        ||A||_2 estimated at set-up: a column that stopped at
 *                        relative primal residual tol with an accurate x-step
 *                        solve has this at most about tol (the violation is
 *                        A (z1 - x1) + (x2 - z2) + (A x1 - x2)); an inexact solve
 *                        (A x1 != x2) shows up here
 * Runs on the case's stream; device temporaries of about
 * 64 x (2 n + 2.5 m) doubles are allocated on first use and kept with the
 * result.  Errors: LGK_EINVAL, LGK_ENOMEM, LGK_ECUDA.
 */
enum { LGK_CHECK_OBJ = 0, LGK_CHECK_PLAN = 1, LGK_CHECK_GAP = 2, LGK_CHECK_INFEAS = 3,
       LGK_CHECK_INFEAS_ABS = 4, LGK_CHECK_HARD = 5, LGK_CHECK_BOUND = 6, LGK_CHECK_PRIMAL = 7,
       LGK_CHECK_COUNT = 8 };
int lgk_fetch_check(const lgk_result* res, double* out);

/*
 * lgk_solve_weightings_warm -- as lgk_solve_weightings, but starting from a
 * given ADMM state instead of zero (checkpoint / resume, or a warm start from
 * an earlier solve).  The state is the q-form of Eq. admm: q1 = z1 + y1
 * (K x n) and q2 = z2 + y2 (K x m) of the scaled problem, FP64 host arrays as
 * returned by lgk_fetch_state; z = projection of q (z1 = clip(q1, 0, u),
 * z2 = min(q2, b)) and y = q - z.  Either pointer may be NULL (zeros).
 */
int lgk_solve_weightings_warm(lgk_case* cs, int K, const double* W, const double* rho,
                              double w0_bot, double rho0, double tol, int max_iter,
                              const double* q1_init, const double* q2_init, lgk_result** out);

/*
 * lgk_solve_weightings_masked -- as lgk_solve_weightings_warm, with a
 * selection of dose points per weighting (Sec. 2.C: the second pass samples
 * its low-dose points per weighting from the union of all weightings'
 * low-dose volumes, and a weighting's LP leaves out the union points not
 * sampled for it by zeroing their upper bounds u).
 *   mask: n_pts x ceil(K/32) uint32 host array; point p belongs to weighting j
 *         when bit (j % 32) of mask[p * ceil(K/32) + j / 32] is set.  NULL:
 *         every point in every weighting.  Bits past K are ignored.
 * A point left out of weighting j gets u = 0 there (so its x is 0 and the
 * weighting solves the LP of its selected points only), and the point counts
 * N_alpha that normalise u (Appendix A) are weighting j's selected counts; a
 * class with no selected point drops out of that weighting's objective.
 * q1_init, q2_init: as in lgk_solve_weightings_warm (NULL: zero state).
 */
int lgk_solve_weightings_masked(lgk_case* cs, int K, const double* W, const double* rho,
                                double w0_bot, double rho0, double tol, int max_iter,
                                const uint32_t* mask, const double* q1_init, const double* q2_init,
                                lgk_result** out);

/*
 * lgk_solve_stream -- K_total weightings through `width` columns of one
 * resident case (continuous batching of a weighting set).  The first
 * min(width, K_total) weightings start together; whenever a column stops
 * (its residual test passes, or it has run max_iter iterations of its own),
 * its results are copied out at the next graph boundary (every 5 residual-
 * test intervals) and the next weighting, in the given order, takes the
 * column from q = 0.  Columns never interact, so each weighting runs the
 * iteration of lgk_solve_weightings (Eq. admm) from its own start; only
 * the lagged low term's refresh points fall at different iterations of its
 * trajectory (the fixed point is unchanged), and a refilled column's first
 * iterations before its first residual test add no low-term product.
 * A batch's time is set by its slowest column while every iteration streams
 * all of A for every column; refilling lets a set of weightings larger than
 * the batch width run at the cost of the mean iteration count instead.
 *   W:   K_total x 4 host array (w_T, w_R, w_LD, w_BOT), admitted in order.
 *   rho: K_total host array, or NULL for Eq. rho_rule (w0_bot, rho0 as in
 *        lgk_solve_weightings).
 *   max_iter: per weighting; a column is stopped within one graph replay
 *        (5 x check_every iterations) after reaching it.
 *   width: columns iterated at once, 1 <= width <= 4096.
 * Outputs (host arrays, each may be NULL), per weighting in input order:
 *   t (K_total x 24N), tau (K_total x N): as lgk_fetch_times;
 *   iters, obj, rel_pri, rel_dual, converged (K_total): as lgk_fetch_stats
 *        (the residuals of the weighting's last residual test; 0 with tol = 0,
 *        which runs none);
 *   prof_ms, prof_launches (LGK_K_COUNT): per-kernel CUDA-event time and
 *        launches as lgk_fetch_profile (only with lgk_params.profile = 1);
 *   check (K_total x LGK_CHECK_COUNT): the FP64 check of lgk_fetch_check,
 *        run on each weighting's column when it stops (before the column is
 *        refilled).
 * 1 <= K_total <= 1 << 20, and (ceil(K_total / width) + 1) x (max_iter
 * rounded up to a graph replay, plus one replay) <= 2^30 (the stream's
 * iteration counter is 32-bit).  LGK_EINVAL on bad arguments; on any error the
 * outputs are undefined.  lgk_params.timeout_ms bounds the whole stream.
 */
int lgk_solve_stream(lgk_case* cs, int K_total, const double* W, const double* rho, double w0_bot,
                     double rho0, double tol, int max_iter, int width, double* t, double* tau, int* iters,
                     double* obj, double* rel_pri, double* rel_dual, uint8_t* converged, double* prof_ms,
                     long long* prof_launches, double* check);

/* ------------------------------------------------------------------------
 * Two-pass optimisation (Sec. 2.C).  The first pass takes its low-dose
 * points from a geometric expansion of the targets; the second takes them,
 * per weighting, from the low-dose volume of that weighting's first-pass
 * plan: the candidate points whose dose lies in [D_LD, D_LD + Delta).  The
 * weightings' volumes differ, so their points are sampled with Algorithm 1
 * (non-redundant sampling: overlapping volumes share points) and the second
 * pass is one batched solve over the union of the samples, each weighting
 * masked to its own sample (lgk_solve_weightings_masked).
 * ------------------------------------------------------------------------ */

/*
 * lgk_low_dose_volumes -- the low-dose volumes of a result's plans.
 * Doses d = phi_cand t of every plan on n_cand candidate points (FP64, on the
 * device, the product lgk_fetch_doses computes), then for each of n_levels
 * ranges [d_lo[l], d_lo[l] + delta[l]) (the upper end computed in FP64 on the
 * host) the membership of every candidate:
 *   phi_cand: n_cand x 24N host array (>= 0); streamed to the device in chunks.
 *   member:   n_levels x K x ceil(n_cand/32) uint32 (host, output); candidate i
 *             is in volume (l, j) when bit (i % 32) of word i / 32 of row (l, j)
 *             is set.
 *   count:    n_levels x K (host, output): |V_lj|.
 * 1 <= n_levels <= 8, d_lo > 0, delta > 0; LGK_EINVAL otherwise.
 */
int lgk_low_dose_volumes(const lgk_result* res, const double* phi_cand, int n_cand, int n_levels,
                         const double* d_lo, const double* delta, uint32_t* member, int* count);

/*
 * lgk_sample_low_dose -- Algorithm 1 (Sec. 2.C), on the host.
 * Volumes V_j (j < K) are candidate bitsets (member: K x ceil(n_cand/32), as
 * lgk_low_dose_volumes writes one level).  Volume j wants n_desired[j] points
 * (capped at |V_j|), i.e. sampling density w_j = n_desired[j] / |V_j|.  The
 * volumes are visited by decreasing w_j (ties: smaller j; empty volumes are
 * skipped); at each one the union's current points are thinned to w_j times
 * the union volume, those inside V_j are reused, and w_j times the new part
 * of V_j is drawn fresh.  Counts are w_j x (a set size) rounded to nearest,
 * halves up, in exact integer arithmetic.  A draw of k items from a set takes
 * the k items with the smallest keys
 *     key(i) = f(f(f(f(seed) ^ level) ^ (2 j + s)) ^ i)
 * (f = the SplitMix64 output function of Steele, Lea and Flood, 2014; s = 0
 * for the thinning draw, 1 for the fresh draw; i = candidate index), so the
 * result is a deterministic function of the inputs.
 * Outputs (host): *n_union = |P|, P the union of the samples p_j;
 * union_idx[0..n_union) its candidate indices, ascending (capacity n_cand);
 * sel (may be NULL): n_union x ceil(K/32) uint32, bit j of row u set when
 * union point u belongs to p_j (capacity n_cand x ceil(K/32)).
 */
int lgk_sample_low_dose(int K, int n_cand, const uint32_t* member, const int* n_desired, uint64_t seed,
                        int level, int* n_union, int* union_idx, uint32_t* sel);

typedef struct {
    const double* phi_cand;  /* n_cand x 24N host: dose-rate kernels of the candidate points
                                of the second pass's low-dose volumes                        */
    int n_cand;
    double delta_ld1;        /* Delta of the LD1 and LD2 volumes [D_LD, D_LD + Delta), Gy    */
    double delta_ld2;
    int n_ld1, n_ld2;        /* desired points per weighting and level; <= 0: the first
                                pass's LD1 / LD2 point counts                                 */
    uint64_t seed;           /* Algorithm 1 draws (level 0: LD1, level 1: LD2)               */
} lgk_pass2_params;

/*
 * lgk_two_pass -- both passes in one call.
 * Pass 1: lgk_create_case(desc, p) and lgk_solve_weightings with the rho rule
 * (Eq. rho_rule) and rho0 = rho0_per_beta x beta of that case.  Then the
 * LD1 and LD2 volumes of every plan on the candidates, Algorithm 1 per level
 * (desired counts as above), and pass 2: a case whose points are desc's
 * non-low-dose points (in order), then the LD1 union points, then the LD2
 * union points (candidate order), solved with lgk_solve_weightings_masked
 * (rho0 = rho0_per_beta x beta of the second case, same W, tol, max_iter).
 * Outputs: *res1_out (may be NULL: freed), *case2_out and *res2_out (owned by
 * the caller), n_union[2] and union_idx[2][n_cand] (candidate indices of the
 * LD1 and LD2 union points; either may be NULL).  On error every output
 * handle is NULL.
 */
int lgk_two_pass(const lgk_case_desc* desc, const lgk_params* p, int K, const double* W, double w0_bot,
                 double rho0_per_beta, double tol, int max_iter, const lgk_pass2_params* p2,
                 lgk_result** res1_out, lgk_case** case2_out, lgk_result** res2_out, int* n_union,
                 int* union_idx);

/* ADMM state of the scaled problem in q-form: q1 = z1 + y1 (K x n) and
 * q2 = z2 + y2 (K x m), FP64 host arrays (either may be NULL).  Feeding them
 * back to lgk_solve_weightings_warm resumes the iteration. */
int lgk_fetch_state(const lgk_result* res, double* q1, double* q2);

/* Kernel classes of one ADMM iteration.  Launch order: [GEMM1_LO] GEMM1
 * REDUCE_RHS SOLVE REDUCE_SOLVE [GEMM2_LO] GEMM2 [Q1_UPDATE] FINALIZE.  The
 * BF16 forms run the q1 update inside the tensor-core GEMM2's epilogue
 * (LGK_K_Q1_UPDATE reports zero launches for them); the FP32 form launches
 * it.  GEMM1_LO / GEMM2_LO (lo R1 and lo^T v) run on the full iterations of
 * LGK_PREC_BF16X3 with lo_refresh = 1.  With solve_refine > 0 each refinement
 * step adds SV (S v), REDUCE_ERR (e = rhs - S v), SOLVE and REDUCE_SOLVE after
 * the first REDUCE_SOLVE. */
enum { LGK_K_GEMM1 = 0, LGK_K_REDUCE_RHS = 1, LGK_K_SOLVE = 2, LGK_K_REDUCE_SOLVE = 3,
       LGK_K_GEMM2 = 4, LGK_K_Q1_UPDATE = 5, LGK_K_FINALIZE = 6, LGK_K_GEMM1_LO = 7,
       LGK_K_GEMM2_LO = 8, LGK_K_SV = 9, LGK_K_REDUCE_ERR = 10, LGK_K_COUNT = 11 };

/* Per-kernel-class device time of a solve made with lgk_params.profile = 1:
 * ms[LGK_K_COUNT] total milliseconds between CUDA events recorded on the
 * solve's stream around each kernel, launches[LGK_K_COUNT] the number of
 * timed launches (iterations in which columns were still active).  Either
 * pointer may be NULL.  LGK_EINVAL if the solve was not profiled. */
int lgk_fetch_profile(const lgk_result* res, double* ms, long long* launches);

/* ------------------------------------------------------------------ serving
 * A request loop with continuous batching for planning requests that arrive
 * over time.  (The paper plans one case at a time; this is the serving form
 * of the library, not a step of the method.)
 *
 * A resident case is a case kept on the device (A, S^{-1} and the ADMM state
 * of its columns).  Cases are admitted first come, first served under a
 * device-memory budget: a case is set up once its estimated peak footprint
 * (set-up temporaries included) fits next to the cases in flight; one that
 * can never fit fails with LGK_EBUDGET.  Each admitted case runs on a worker
 * thread with its own CUDA stream as one streaming solve of `stream_width`
 * columns (lgk_solve_stream's iteration): every weighting submitted for the
 * case, by any request and at any time while it is resident, takes the next
 * column that frees up (at the next replay boundary, every 5 residual-test
 * intervals).  Requests that arrive while the case is on the GPU thus join
 * its running batch, and cases on different workers overlap on the device.
 * A weighting's result does not depend on what runs beside it or when it
 * entered (bitwise: columns never interact, every column starts alike, and
 * every reduction has a fixed order).
 * Per-weighting stop test, tolerance and iteration cap: those of
 * lgk_solve_stream with the server's tol and max_iter, rho by Eq. rho_rule.
 * A case that is continuously busy for 2^30 iterations of its stream (about
 * 60 hours at 200 us per iteration) fails its requests with LGK_EINVAL.
 */
typedef struct lgk_server lgk_server;

typedef struct {
    lgk_params case_params;  /* per-case parameters (its stream field is ignored)           */
    size_t hbm_budget;       /* bytes for the cases in flight; 0 = 90 % of free memory      */
    int workers;             /* resident cases on the device at once (>= 1)                 */
    double tol;              /* stop tolerance of every weighting                            */
    int max_iter;            /* iteration cap of every weighting                             */
    double w0_bot;           /* rho rule: rho = rho0_per_beta * beta * sqrt(w0_bot / w_BOT) */
    double rho0_per_beta;
    int stream_width;        /* columns of each case's streaming solve; 0 = 32              */
} lgk_server_params;

typedef struct {
    int status;              /* lgk_status of the request                                   */
    int K, n_iso;
    double queue_ms;         /* submit -> its first weighting takes a column                 */
    double setup_ms;         /* the case's set-up, if the request waited for it; else 0      */
    double solve_ms;         /* first weighting in a column -> last weighting done           */
    double total_ms;         /* submit -> done                                               */
    int max_iters;           /* iterations of the slowest weighting                          */
    int converged;           /* weightings that met the tolerance                            */
    size_t footprint;        /* estimated peak device bytes of the case (admission)          */
} lgk_request_info;

int lgk_server_create(const lgk_server_params* p, lgk_server** out);
/* One-shot request: a new resident case (desc copied) with the K weightings
 * W (K x 4, copied; w_BOT > 0); the case leaves the device once they are
 * done.  *id receives the request id. */
int lgk_server_submit(lgk_server* s, const lgk_case_desc* desc, int K, const double* W,
                      long long* id);
/* Queue a resident case (desc copied) for admission; *case_id receives its id.
 * It stays resident, taking weightings from lgk_server_submit_to, until
 * lgk_server_close.  LGK_EBUDGET if it can never fit the budget. */
int lgk_server_open(lgk_server* s, const lgk_case_desc* desc, long long* case_id);
/* A request of K weightings (W: K x 4, copied; w_BOT > 0) for resident case
 * case_id: they join its running stream as columns free up.  *id receives
 * the request id.  LGK_EINVAL if the case is unknown or closed. */
int lgk_server_submit_to(lgk_server* s, long long case_id, int K, const double* W, long long* id);
/* No more requests for case_id: it leaves the device once its queued
 * weightings are done. */
int lgk_server_close(lgk_server* s, long long case_id);
/* Waits (at most timeout_ms) for request id; fills *info and, if not NULL,
 * t (K x 24N) and tau (K x N) in the request's weighting order.  A request
 * can be waited for once. */
int lgk_server_wait(lgk_server* s, long long id, int timeout_ms, lgk_request_info* info,
                    double* t, double* tau);
/* Finishes the weightings in the cases' columns, fails the queued ones
 * (LGK_ETIMEOUT, "server destroyed"), joins the workers. */
void lgk_server_destroy(lgk_server* s);

void lgk_free_result(lgk_result* res);
void lgk_destroy_case(lgk_case* cs);
const char* lgk_last_error(void);

/* Number of kernel launches the library issued on this thread since the last
 * call (diagnostics for launch counting; graph replays count their nodes). */
long long lgk_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LGK_H */
