/*
 * fe.h -- C ABI of the GB300 (sm_103a) recursive Fermi-operator expansion
 * library: the projected density matrix D = f(Hp) and the band energy
 * tr(Hp D) from a dense symmetric projected Hamiltonian Hp.
 *
 * Method (arXiv 2301.04642, Khadatkar & Motamarri):
 *   - Sec. II-A: D = theta(mu I - Hp) at zero temperature (projector on the
 *     N_e lowest eigenvectors), D = [exp(beta (Hp - mu I)) + I]^{-1} at
 *     finite temperature, beta = 1/kT.
 *   - Sec. II-B1, Eq. (1): zero temperature by SP2, X_{k+1} = X_k^2 or
 *     2 X_k - X_k^2, the branch chosen from tr X and tr X^2 = ||X||_F^2
 *     (Sec. III-B) so that tr X -> N_e.  X_0 is Hp scaled into [0, 1] with
 *     spectral bounds (Sec. II-C): a Lanczos estimate, certified to contain
 *     the spectrum by three logistic steps (a Chebyshev T_8 filter), within
 *     the Gershgorin interval.
 *   - Sec. III-A: relative trace change RelTr as the convergence measure and a
 *     mixed-precision schedule (cheap products far from convergence, FP64-
 *     accurate products at the end).
 *   - Sec. II-B3, Eq. (2): finite temperature by a recursive expansion whose
 *     every step doubles the inverse temperature (see FE_METHOD_FERMI).
 *
 * Conventions for every function:
 *   - Matrices are dense, row-major, FP64, with a leading dimension ld >= n
 *     (elements between n and ld in a row are ignored / not written).
 *   - Hp must be symmetric with both triangles stored (rows are read whole).
 *   - Pointers are host or device pointers as the problem's flags say
 *     (FE_PTR_HOST / FE_PTR_DEVICE); device pointers must belong to the
 *     context's device.  The caller owns Hp and D.  A context's work is
 *     ordered only after earlier work on its own stream (fe_config's
 *     cuda_stream, else a non-blocking stream it creates): device inputs
 *     written on other streams must be complete before the call.
 *   - Every call returns an FE_* status; no call exits, throws or traps.
 *     fe_last_error_string() gives a one-line reason for the last failure.
 *   - A context is used by one host thread at a time, except fe_submit /
 *     fe_poll, which may be called from any thread.
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FE_API __attribute__((visibility("default")))
#else
#define FE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define FE_OK 0
#define FE_PENDING 1       /* fe_poll: solve still queued or running          */
#define FE_EINVAL (-1)     /* bad argument (see fe_problem), or NaN/Inf in Hp   */
#define FE_ENOMEM (-2)     /* does not fit the context's HBM budget at all      */
#define FE_ENOTCONV (-3)   /* iteration cap reached (e.g. degenerate HOMO/LUMO) */
#define FE_ETIMEOUT (-4)   /* a bounded device wait expired; context still usable */
#define FE_ECUDA (-5)      /* CUDA runtime/driver error                          */
#define FE_EBUSY (-6)      /* too many outstanding tickets                       */

/* ---- problem flags -------------------------------------------------------- */
#define FE_PTR_HOST 0x0u      /* Hp and D are host pointers (default)          */
#define FE_PTR_DEVICE 0x1u    /* Hp and D are device pointers                  */

#define FE_METHOD_AUTO 0x00u  /* SP2 if kT == 0 else FERMI                     */
#define FE_METHOD_SP2 0x10u   /* zero temperature, Sec. II-B1                   */
#define FE_METHOD_FERMI 0x20u /* finite temperature, doubling recursion         */
/* Zero temperature, accelerated SP2 (A-Z-RFOE, Sec. II-B2): the SP2
 * polynomials shifted and scaled with the caller's HOMO/LUMO estimates
 * (fe_problem.homo < fe_problem.lumo, e.g. the previous subspace iteration's
 * Rayleigh-Ritz eigenvalues), so that eigenvalues reach 0 or 1 in fewer
 * products.  The folds are valid when the estimates lie inside the true gap
 * (homo >= the HOMO eigenvalue, lumo <= the LUMO eigenvalue).  The device
 * checks after every product that the traces stay consistent with that
 * (N_e b <= tr X <= N_e + (n - N_e) a and tr(X - X^2) <= (n - N_e) a +
 * N_e (1 - b), a and b the folded interval ends, within 1/2); when they do
 * not, the solve starts again as plain SP2 (fe_result.iters counts both). */
#define FE_METHOD_ASP2 0x30u
/* Finite temperature, the truncated SP2 expansion as the paper prints it
 * (T-RFOE, Sec. II-B3, Eq. (2)): D = G_m(X0), the SP2 recursion with its
 * trace-driven branches stopped after m products, X0 from the Gershgorin
 * bounds.  m is the first step at which the step function G_m is as steep
 * at its midpoint (G_m = 1/2) as the Fermi-Dirac function at mu, i.e.
 * |dG_m/de| >= beta/4; fe_result.mu is the midpoint energy.  D is a smeared
 * step, not Fermi-Dirac (the paper quotes eps1 ~ 1e-3 against it), and
 * tr D is near but not equal to N_e.  The step function is steep
 * (|dG/dx| = beta w / 4 at its midpoint, w the Gershgorin width), so a
 * product's rounding error is amplified that much for the states near mu.
 * Precision: FE_PREC_MIXED (split FP16 until RelTr < 5e-4, the paper's
 * switch point, then FP64-accurate digit products), FE_PREC_FP32 (split FP16
 * only) or FE_PREC_FP64 (FP64-accurate digit products on the tensor cores
 * from an FP64 X0, for results within FP64 rounding times that slope). */
#define FE_METHOD_TRFOE 0x40u
#define FE_METHOD_MASK 0xF0u

/* Precision schedules (Sec. III-A).  Bits 8..11. */
#define FE_PREC_MIXED 0x000u  /* split FP16 tensor-core products, FP64 polish   */
#define FE_PREC_FP64 0x100u   /* every product in FP64 (the plain baseline)     */
#define FE_PREC_FP32 0x200u   /* split FP16 tensor-core products only, no polish */
#define FE_PREC_TRY_FP16 0x300u /* single FP16 products until RelTr < 5e-4, then MIXED */
#define FE_PREC_MASK 0xF00u

/* ---- context ---------------------------------------------------------------- */
typedef struct fe_ctx fe_ctx;

typedef struct {
    int device;               /* CUDA device ordinal                              */
    size_t hbm_budget_bytes;  /* pool limit; 0 = 80% of the device's free memory  */
    int max_iters;            /* cap on expansion products per phase; 0 = 100     */
    uint32_t precision_policy;/* default FE_PREC_* when a problem leaves it 0     */
    void *cuda_stream;        /* cudaStream_t to run on; NULL = library stream    */
    const char *autotune_path;/* tile-shape table file: loaded by fe_create when it
                                 exists, rewritten by fe_autotune; NULL = none    */
} fe_config;

typedef struct {
    const double *Hp;  /* n x n symmetric, row-major, leading dimension ld        */
    int64_t n;         /* dimension, >= 1                                           */
    int64_t ld;        /* leading dimension of Hp and D, >= n                       */
    double n_e;        /* electron count N_e (occupied states, no spin factor),
                          0 <= n_e <= n; integral when kT == 0                     */
    double kT;         /* smearing temperature in the units of Hp; 0 = zero T      */
    double tol;        /* RelTr stop |tr X_k - tr X_{k-1}| / N_e; 0 = 5e-8          */
    double *D;         /* output density matrix (n x n, ld), may be NULL           */
    uint32_t flags;    /* FE_PTR_* | FE_METHOD_* | FE_PREC_*                        */
    double homo;       /* FE_METHOD_ASP2: estimate of the highest occupied
                          eigenvalue of Hp (ignored by the other methods)          */
    double lumo;       /* FE_METHOD_ASP2: estimate of the lowest unoccupied
                          eigenvalue of Hp, > homo                                 */
} fe_problem;

typedef struct {
    int status;             /* FE_* of this solve                                  */
    int iters;              /* total expansion products                            */
    int iters_by_phase[4];  /* [0] single-FP16, [1] split-FP16, [2] FP64, [3] finite-T steps */
    double e_band;          /* tr(Hp D), FP64                                       */
    double trace;           /* tr D                                                 */
    double idem_fro;        /* ||X^2 - X||_F of the last product's input, measured in its
                               epilogue (0 T); D, its output, is closer to idempotent */
    double mu;              /* chemical potential (FE_METHOD_FERMI), midpoint energy
                               of the step function (FE_METHOD_TRFOE); NaN at zero T */
    double eps_min;         /* lower spectral bound the expansion used: a Lanczos
                               estimate widened by its certificate so that it
                               contains the spectrum, within the Gershgorin interval */
    double eps_max;         /* upper spectral bound, likewise                        */
    double ms;              /* fe_solve / fe_solve_batch: device time of the solve
                               (CUDA events); fe_poll: submit-to-done latency, ms   */
} fe_result;

typedef uint64_t fe_ticket;

/* One tile-shape table entry as fe_autotune reports it. */
typedef struct {
    int64_t n;       /* problem dimension                                          */
    int bn;          /* tensor-core tile width chosen: 256 (128 x 256 tiles) or 128 */
    double ms_256;   /* best device time (ms) per solve of a synthetic batch of this
                        size with 128 x 256 tiles                                  */
    double ms_128;   /* the same with 128 x 128 tiles                               */
} fe_tune;

/* Create a context on cfg->device.  cfg may be NULL (defaults).
 * Errors: FE_EINVAL (bad device, malformed autotune_path file; a file that
 * cannot be opened starts an empty table), FE_ECUDA. */
FE_API int fe_create(fe_ctx **out, const fe_config *cfg);

/* Wait for outstanding work, free all device memory.  NULL is accepted. */
FE_API int fe_destroy(fe_ctx *ctx);

/* Blocking solve of one problem.  Hp is read (copied into the pool first when
 * it is a host pointer, or when its ld is not the pool's layout); D (if not
 * NULL) is written on success: a page-locked host D (cudaHostAlloc,
 * cudaHostRegister) by the output kernel directly, other host memory through a
 * staging copy.  r receives the result even on failure.
 * Errors: FE_EINVAL (n < 1, ld < n, N_e out of [0, n], kT < 0, non-integral
 * N_e at kT == 0, tol < 0, NaN/Inf in Hp, FE_METHOD_ASP2 without finite
 * homo < lumo or with kT != 0, FE_METHOD_TRFOE with kT == 0), FE_ENOMEM,
 * FE_ENOTCONV (iteration cap, or a polish that cannot reach the trace and
 * idempotency targets, e.g. a degenerate HOMO/LUMO), FE_ETIMEOUT, FE_ECUDA. */
FE_API int fe_solve(fe_ctx *ctx, const fe_problem *p, fe_result *r);

/* Solve `count` independent problems (any mix of n) in one launch sequence:
 * each expansion step is one persistent launch over the tiles of all active
 * problems.  rs[i] receives problem i's result; the return value is FE_OK if
 * every problem succeeded, else the first failing status. */
FE_API int fe_solve_batch(fe_ctx *ctx, int count, const fe_problem *ps, fe_result *rs);

/* Non-blocking submission for continuous batching.  Hp is copied into the
 * pool before this returns (the caller may reuse it); D must stay valid until
 * fe_poll returns a final status for the ticket.  Requests that do not fit
 * the free part of the HBM budget wait in a queue; a request larger than the
 * whole budget fails with FE_ENOMEM. */
FE_API int fe_submit(fe_ctx *ctx, const fe_problem *p, fe_ticket *t);

/* FE_PENDING while the ticket's solve is queued or running; otherwise the
 * final status, with r filled.  Never blocks. */
FE_API int fe_poll(fe_ctx *ctx, fe_ticket t, fe_result *r);

/* Tile-shape autotuner.  The split-FP16 / single-FP16 symmetric products
 * (Sec. III-B: the matrix product is the cost) run over upper-triangle tiles of
 * 128 x 256 or 128 x 128 elements.  Wide tiles halve the operand traffic per
 * flop; narrow ones waste less work at the diagonal and the ragged edge and
 * give more tiles to balance over the SMs, which pays for small n.  The
 * context keeps a table from (number of 128-row panels, precision policy) to
 * the width; a problem uses the entry for its panel count, else the nearest
 * one under its policy, else 256.  Problems of different widths share one
 * launch in fe_solve_batch.
 * fe_autotune fills the table for the panel counts of ns[0..count): for each
 * it times `reps` batches of synthetic gapped solves of that size (N_e =
 * 0.85 n, device Hp, no output; enough copies per batch, at most 16, for two
 * waves of 128 x 256 tiles over the SMs, so that the time per solve measures
 * throughput as in a busy batch or server) with each width under precision
 * policy `prec` (0 = the context's default; FE_PREC_FP64 has no tiles), keeps
 * the width with the lower time per solve, and writes the table to the
 * context's autotune_path if one was given.  out (may be NULL) receives one
 * entry per ns[i].  The solves run on the context's stream like
 * fe_solve_batch; n must lie in [2, 2^20].
 * Errors: FE_EINVAL, FE_ENOMEM, any fe_solve status. */
FE_API int fe_autotune(fe_ctx *ctx, int count, const int64_t *ns, uint32_t prec, int reps, fe_tune *out);

/* Tile widths for a recurring batch.  fe_autotune times each size on its own
 * (copies of one problem); in a mixed batch the widths interact (one launch
 * holds every problem's tiles), so this tunes on the batch itself: it times
 * fe_solve_batch on ps[0..count) (outputs not written: every D is ignored)
 * with 128 x 256 tiles for every problem, then makes the problems of the
 * smallest panel count narrow (128 x 128), then those of the next one, and so
 * on while each step lowers the batch's device time by more than 0.5%; the
 * first step that does not is undone and ends the search.  The result is left
 * in the context's table (and its autotune_path file).  Each trial is one
 * untimed batch then the best of `reps` (< 1: 2).  trial_ms[0..max_trials)
 * receives the trials' batch times (ms; [0] = all 128 x 256), *ntrials their
 * number (both may be NULL / 0).
 * Errors: FE_EINVAL (count < 1, an invalid problem), any fe_solve_batch
 * status (the table is then left as it was). */
FE_API int fe_autotune_batch(fe_ctx *ctx, int count, const fe_problem *ps, int reps, double *trial_ms,
                             int max_trials, int *ntrials);

/* ---- the products either side of the expansion --------------------------
 * In Chebyshev-filtered subspace iteration (Sec. I, Sec. III-A) the
 * expansion replaces the diagonalisation of the projected Hamiltonian; the
 * step before it forms Hp from the filtered subspace by the Rayleigh-Ritz
 * projection, the step after it uses D for the density and the subspace
 * rotation.  Psi is the m x n block of filtered vectors (m grid points,
 * n vectors, m >> n), row-major with leading dimension ld (a grid point's n
 * values contiguous).  Both calls take DEVICE pointers on the context's
 * device, run on the context's stream and return when the result is ready.
 * Precision: the operands are split into FP16 hi + lo slices (22 bits, one
 * power-of-two scale per operand from its largest entry) and multiplied on
 * the tensor cores with FP32 accumulation per 64-wide K chunk, the chunks
 * summed in FP32 registers (at most 128 per part) and the parts in FP64:
 * |C_ij - (A B)_ij| <= (2^-21 + 2^-21 + c 2^-24) sum_k |A_ik| |B_kj|
 * + 2^-36 K max|A| max|B|, c the chunks of one part (the last term for
 * entries below 2^-25 of their operand's largest, whose low slice leaves the
 * FP16 normal range); an FP32-class result, as the FP32 Rayleigh-Ritz
 * products of mixed-precision subspace iteration.
 * Errors: FE_EINVAL (NULL pointer, m or n < 1, n > 2^20, m > 2^31 - 1, a
 * leading dimension below n), FE_ENOMEM (workspace of about 8 m n bytes for
 * fe_project, 4 (m + n) n for fe_rotate, beyond the HBM budget), FE_ETIMEOUT,
 * FE_ECUDA. */

/* Hp = Psi^T HPsi (n x n, leading dimension ldh), HPsi = H Psi given (m x n,
 * same leading dimension ld as Psi).  The product is symmetric in exact
 * arithmetic; the upper triangle is computed and mirrored, so Hp is exactly
 * symmetric. */
FE_API int fe_project(fe_ctx *ctx, const double *Psi, const double *HPsi, int64_t m, int64_t n, int64_t ld,
                      double *Hp, int64_t ldh);

/* Out = Psi D (m x n, leading dimension ldo) for a symmetric n x n D
 * (leading dimension ldd; its rows are read as its columns). */
FE_API int fe_rotate(fe_ctx *ctx, const double *Psi, int64_t m, int64_t n, int64_t ldpsi, const double *D,
                     int64_t ldd, double *Out, int64_t ldo);

/* One-line description of the last error on this context (or of the last
 * fe_create failure when ctx is NULL).  Valid until the next call. */
FE_API const char *fe_last_error_string(const fe_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FE_H */
