/*
 * lasso.h -- C ABI of the GB300 screened Lasso solver.
 *
 * The library solves   x* = argmin_x 1/2 ||A x - y||_2^2 + lambda ||x||_1          (eq:lasso)
 * with FISTA (or ISTA) restricted to the atoms that survive dynamic safe screening, while
 * iterating on a ladder of approximate dictionaries A~^0, ..., A~^I = A of increasing
 * precision (Algorithm 1, FastL1).  Screening uses the stable GAP Safe sphere of Theorem 1
 * (or the stable Dynamic Safe sphere of Table I) with per-atom error bounds
 * eps_j >= ||a~_j - a_j||_2, so every rejection is safe for the original problem; the
 * dictionary switches on gap saturation or on the speed criterion (Algorithm 2).
 *
 * Conventions
 *  - A dictionary has N rows (signal dimension) and K atoms (columns).  Dense inputs may be
 *    given atom-major (row j = atom j, length N, leading dimension ld >= N) or column-major
 *    (the usual N x K "columns are atoms" layout with leading dimension ld >= N, i.e. the
 *    same memory); both mean element (n, j) at A[j * ld + n].  Row-major N x K input is
 *    given with atom_major = 0 and ld >= K: element (n, j) at A[n * ld + j].
 *  - Kronecker dictionaries: A = (sum_{r<R} B_r (x) C_r) diag(d) with B_r: N1 x K1 and
 *    C_r: N2 x K2 row-major, N = N1 N2, K = K1 K2, atom k1 K2 + k2, row n1 N2 + n2, and
 *    d_j = 1 / ||(sum_r B_r (x) C_r) e_j||_2 computed by the library in FP64 (unit atoms).
 *  - "Relative gap" is G / ||y||^2 where G is an upper bound of the duality gap G(x, theta|A)
 *    of the returned point for the original problem over the whole dictionary (rounding of
 *    every kernel is folded in).  A signal stops when this bound is <= tol at the exact level.
 *  - Every call returns a status (lasso_status) and never aborts; on error the outputs are
 *    left as documented per call.  lasso_strerror() gives a message; when the most recent
 *    status-returning call on the same thread recorded a detail (the limit it refused, the
 *    CUDA call that failed), the message carries it.
 *  - Pointers named *_host are host memory; pointers named d_* are device memory of the
 *    current CUDA device.  The library owns every lasso_dict it creates.
 *  - Thread safety: a lasso_dict may be used by one call at a time.
 */
#ifndef LASSO_GB300_H
#define LASSO_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LASSO_OK = 0,
    LASSO_ERR_INVALID_ARG = -1,   /* bad size, null pointer, wrong order of calls         */
    LASSO_ERR_CUDA = -2,          /* a CUDA runtime call failed                           */
    LASSO_ERR_NONFINITE = -3,     /* NaN/Inf met in the data or in a gap                  */
    LASSO_ERR_MAXITER = -4,       /* max_iter passes without reaching tol (x is partial)  */
    LASSO_ERR_TIMEOUT = -5,       /* wall-clock budget exceeded (x is partial)            */
    LASSO_ERR_UNSUPPORTED = -6,   /* valid request this build does not handle             */
    LASSO_ERR_NOMEM = -7,         /* device allocation failed                             */
    LASSO_WARN_AUDIT = 1          /* full-dictionary certificate above tol (see gap)      */
} lasso_status;

typedef enum { LASSO_F64 = 0, LASSO_F32 = 1 } lasso_dtype;

/* Approximate-dictionary kinds for lasso_dict_add_level (Section III-A, "precision" levels). */
typedef enum {
    LASSO_LEVEL_BF16 = 2,         /* BF16 copy of A (round to nearest even)                    */
    LASSO_LEVEL_FP8 = 3,          /* E4M3 copy with per-atom scale s_j = max_i |a_ij| / 448     */
    LASSO_LEVEL_KRON = 4,         /* Kronecker truncation to the first `param` terms            */
    LASSO_LEVEL_F32 = 5,          /* FP32 copy of an FP64 dictionary                            */
    LASSO_LEVEL_FAUST = 6         /* product of sparse factors (lasso_dict_add_level_faust)     */
} lasso_level_kind;

typedef struct lasso_dict lasso_dict;

/* Create a dense dictionary: the exact A of the problem min_x 1/2 ||y - A x||^2 + lambda ||x||_1
 * (eq:lasso; atoms are the columns a_j).  dt gives the element type of A and
 * the precision of the exact level (FP64 data: FP64 arithmetic; FP32 data: FP32 products with
 * compensated accumulation).  normalize != 0 rescales every atom to unit l2 norm first (in
 * FP64, then rounded to dt); the problem solved is then the one with normalised atoms.
 * host_ptr != 0 if A is host memory.  The library copies A.  *out is NULL on error. */
int lasso_dict_create_dense(const void* A, lasso_dtype dt, int64_t N, int64_t K, int64_t ld,
                            int atom_major, int normalize, int host_ptr, lasso_dict** out);

/* Create a sum-of-Kronecker dictionary (SuKro, Section V-A: A = sum_r B_r (x) C_r) from its
 * factors (FP32, host memory if host_ptr != 0, else device memory; the library copies them).
 * B holds R row-major N1 x K1 factors, C holds R row-major N2 x K2 factors.  The exact A is the
 * FP64 Kronecker sum times diag(d): normalize != 0 gives unit atoms (d_j = 1 / ||column j||,
 * computed in FP64), normalize == 0 keeps the sum as given (d_j = 1).  The library stores a
 * dense FP32 rounding of A as the last level (its rounding error enters eps_j), and the
 * structured truncations are added with lasso_dict_add_level(LASSO_LEVEL_KRON, R').
 * Returns LASSO_ERR_INVALID_ARG for null factors, a non-positive size or R > 64 (*out = NULL). */
int lasso_dict_create_kron(const float* B, const float* C, int R, int N1, int K1, int N2, int K2,
                           int normalize, int host_ptr, lasso_dict** out);

/* Append an approximate dictionary below the exact one.  Levels must be added from the
 * coarsest to the finest; the exact dictionary always stays last (A~^I = A).  eps_j is
 * computed exactly in FP64 against the exact atoms.  param: number of Kronecker terms for
 * LASSO_LEVEL_KRON, ignored otherwise.  Up to 7 approximate levels. */
int lasso_dict_add_level(lasso_dict* dict, lasso_level_kind kind, int param);

/* Append a product of sparse factors A~ = S_0 S_1 ... S_{J-1} as an approximate level (the
 * FAuST dictionaries of Section VI, "multilayer sparse" approximations of A).  S_f has
 * dims[f] rows and dims[f+1] columns, dims[0] = N and dims[J] = K; the product approximates the
 * dictionary as stored (normalised atoms when the dictionary was created with normalize != 0),
 * so a column scale belongs in the last factor.  All arrays are HOST memory, read once and
 * copied:
 *   indptr   concatenation over f of the dims[f] + 1 CSR row pointers of S_f (each factor's
 *            own offsets, starting at 0 and non-decreasing);
 *   indices  concatenation over f of the nnz_f = indptr_f[dims[f]] column indices of S_f,
 *            strictly increasing within each row and in [0, dims[f+1]);
 *   values   the matching FP32 values (finite).
 * eps_j = ||a~_j - a_j||_2 is computed from the explicit FP64 product; the FP32 sparse
 * products of a solve add their rounding through kappa_j = ||(|S_0| ... |S_{J-1}|) e_j||_2.
 * RC defaults to (sum_f nnz_f) / (N K).  1 <= J <= 16, every nnz_f < 2^31.  Returns
 * LASSO_ERR_INVALID_ARG when a check fails (nothing is added), LASSO_ERR_NOMEM when the
 * explicit products (2 x K x max(dims) doubles, during the call only) do not fit. */
int lasso_dict_add_level_faust(lasso_dict* dict, int J, const int64_t* dims, const int64_t* indptr,
                               const int32_t* indices, const float* values);

/* Set the relative complexity RC of level `level` (eq:complexity_model_approx) used by the
 * speed criterion of Algorithm 2; by default RC is the level's bytes (dense) or FLOPs
 * (Kronecker) per full product over those of the exact dense product. */
int lasso_dict_set_rc(lasso_dict* dict, int level, double rc);

/* Step size: L = 1.001 max_i ||A~^i||_2^2 by 200 power iterations on the device, unless
 * L_override > 0 is given.  Called automatically by the first solve when not called. */
int lasso_dict_prepare(lasso_dict* dict, double L_override);

typedef struct {
    int64_t N, K;
    int n_levels;                 /* including the exact level (last)                   */
    double L;                     /* step constant (0 before prepare)                   */
    int kind[8];                  /* lasso_level_kind of each level; exact: -1 (F64) / -2 (F32) */
    double rc[8];
    double eps_mean[8], eps_max[8];
} lasso_dict_info_t;

int lasso_dict_info(const lasso_dict* dict, lasso_dict_info_t* info);

/* Copy level data back for inspection (tests): eps (K doubles) and, for dense levels, the
 * dequantised atoms as FP64 (K x N atom-major, row j = a~_j).  Either output may be NULL. */
int lasso_dict_level_host(const lasso_dict* dict, int level, double* eps_host, double* atoms_host);

void lasso_dict_destroy(lasso_dict* dict);

typedef enum { LASSO_FISTA = 0, LASSO_ISTA = 1 } lasso_algo;
/* Screening rules (Table I): stable GAP Safe (Theorem 1), stable Dynamic Safe, and the Static
 * Safe sphere B(y / lam, ||y|| |1/lam - 1/lam_max'|) of eq:static_sphere with lam_max' an upper
 * bound of lambda_max from the certified initial pass. */
typedef enum { LASSO_RULE_GAP = 0, LASSO_RULE_DST = 1, LASSO_RULE_STATIC = 2 } lasso_rule;

typedef struct {
    double Gamma;            /* switching threshold of Algorithm 2 (default 0.5)                */
    int algo;                /* lasso_algo (default FISTA)                                      */
    int rule;                /* lasso_rule (default stable GAP Safe)                            */
    int screen_every;        /* screen every k passes (default 1)                               */
    int max_iter;            /* per-signal pass limit (default 20000)                           */
    int lambda_relative;     /* 1: lambdas are lambda / lambda_max of each signal (default 0)   */
    int final_fp64;          /* 1: append an FP64-accumulation rung on the exact data and keep
                                FP64 iterates (tight tolerances; default 0).  The gaps certify
                                the FP64 iterates: lasso_solve returns them as they are, the
                                batch calls return their rounding to FP32.  Set automatically
                                for FP32 dictionaries when tol < 5e-7: an FP32 point cannot be
                                certified much below that (its dual point's gap is first order
                                in the point's rounding)                                      */
    int certify_full;        /* 1: audit with an explicit full-dictionary pass at exit (default
                                0): every atom recomputed with error-free products            */
    int passes_per_sync;     /* passes per captured CUDA graph replay (default 8)               */
    int tensor_cores;        /* 1: batched BF16/FP8 levels use the tcgen05 GEMMs (default 1)   */
    double tau;              /* rejection guard: reject iff test < 1 - tau (default 1e-9)       */
    double time_limit_s;     /* 0: none                                                          */
    int profile;             /* 1: time every kernel of the passes with CUDA events (stats)     */
    int full_gap;            /* 1: stop on the duality gap of the whole dictionary (default; the
                                rejected atoms' correlations are evaluated when the preserved-set
                                gap meets tol); 0: stop on the preserved-set gap, which bounds
                                P(x) - P* only                                                  */
    int tc_exact;            /* 1: with tensor_cores, the exact FP32 level's bulk correlation runs
                                on the tensor cores in split form a = a1 + a2 (+ bounded rest),
                                rho = r1 + r2 (+ bounded rest), three BF16 products in one FP32
                                accumulator; its error bound enters the stable test like an
                                approximation error, and the stopping certificate recomputes
                                the deciding atoms from the FP32 data.  Default 0: the tensor
                                cores' FP32 accumulation is too coarse for the last decades of
                                the gap (FISTA needs more passes, some signals stall near 1e-6) */
    int split_level;         /* 1 (default): with tensor_cores, a batch of at least 256 signals and an
                                FP32 dense exact level, one more approximate level runs just
                                before the exact one: the split BF16 pair a1 + a2 of the exact
                                atoms (a - a1 - a2 = e3, |e3| <= 2^-16 |a|), correlated on the
                                tensor cores as a1^T r1 + a1^T r2 + a2^T r1 with promoted
                                accumulation; its residual is the exact one, and the
                                correlation error (||e3_j||, the dropped terms, the rounding)
                                enters the stable test as an approximation error (Section III).
                                It takes the solve's middle decades off the exact level.  RC
                                0.02 (Algorithm 2).  Ignored with tc_exact.  0: no split level */
    int fp64_fallback;       /* 1 (default): a signal whose certificate stops improving on the exact
                                FP32 level (FP32 iterates at their precision floor, e.g. on very
                                coherent dictionaries) is stopped and solved again from scratch
                                with FP64 iterates and an FP64-accumulation rung, as final_fp64
                                does; its outputs replace the FP32 ones.  That second solve keeps
                                its extrapolated point (the certified one) FP32-representable, so
                                the returned gap covers the returned FP32 x.  With FISTA, a
                                signal of that second solve whose certificate has not improved
                                for max(2000, passes / 2) passes ends there with
                                LASSO_ERR_MAXITER, its best point and certificate (an FP32 point
                                can sit above tol for good).  0: such a signal ends with
                                LASSO_ERR_MAXITER.                                               */
    int autotune;            /* 1 (default): before the first FP32 batch of a size class (B rounded
                                up to a power of two), time the correlation pass for atom chunks
                                of 64 / 128 / 256 and 4 / 8 / 16 blocks per SM on a synthetic
                                exact-level state (K / 8 preserved atoms per signal) and keep the
                                fastest for the dictionary; 0: 128-atom chunks, 8 blocks per SM */
    uint8_t* kept_mask;      /* optional output of the batch calls (default NULL): B x K bytes, row b
                                = signal b, 1 where atom j is in the signal's preserved set at exit
                                and 0 where a safe test rejected it (Definition 2: a rejected atom
                                is zero in every solution).  Device memory for lasso_solve_batch,
                                host memory for lasso_solve_batch_host; ignored by lasso_solve,
                                which returns its preserved set as a sorted list.  A signal with
                                lambda >= lambda_max, or y = 0, has an empty set.               */
} lasso_opts;

/* Fill *opts with the defaults above. */
void lasso_opts_default(lasso_opts* opts);

typedef struct {
    int64_t passes;          /* passes executed (max over signals for a batch)                  */
    int64_t level_passes[8]; /* passes spent on each level, summed over signals                 */
    int64_t kept_final;      /* |A| at exit (single solve) or its sum over the batch            */
    double lambda_max;       /* lambda_max of the (first) signal                                */
    double lambda;           /* lambda used for the (first) signal                              */
    double seconds;          /* wall time of the call                                           */
    int64_t launches;        /* kernels launched by the call (all kinds)                        */
    /* per kernel kind (0 residual, 1 correlation + update, 2 screening, 3 schedule,
       4 structured products (Kronecker GEMMs, sparse factors), 5 tensor-core GEMMs):
       launches, device milliseconds (with opts.profile) and algorithmic bytes (dictionary
       rows, signals and iterates read or written by the definition of the step) */
    int64_t kernel_launches[6];
    double kernel_ms[6];
    double kernel_bytes[6];
    double level_atoms[8];   /* sum over passes and signals of |A_t| on each level              */
    int64_t fp64_resolved;   /* signals solved again with FP64 iterates (opts.fp64_fallback)     */
    int64_t corr_chunk;      /* atoms per correlation work item used by the solve              */
    int64_t corr_blocks_per_sm; /* correlation grid, in blocks per SM                           */
    double level_rc[8];      /* relative complexity each level of the solve's ladder used in
                                Algorithm 2: measured for the tensor-core levels (time per signal
                                of the batched product over every atom / that of the exact
                                level's gather over every atom, once per batch size class), else
                                the level's RC (lasso_dict_set_rc, or the byte / FLOP ratio)    */
} lasso_stats;

/* Solve one signal with FastL1 (Algorithm 1: FISTA / ISTA on the preserved atoms, stable safe
 * screening, SwitchDictionary of Algorithm 2 along the ladder) to the relative gap tol.  Host
 * buffers.  y: N values (rounded to the exact level's precision on
 * entry).  lambda: absolute, or relative to lambda_max if opts->lambda_relative.  Outputs:
 * x_host (K, zero outside the preserved set), gap_host (relative gap of the returned point),
 * kept_host (capacity K, sorted preserved set at exit, may be NULL), n_kept (may be NULL),
 * stats (may be NULL).  lambda >= lambda_max returns x = 0, gap = 0, n_kept = 0. */
int lasso_solve(lasso_dict* dict, const double* y_host, double lambda, double tol,
                const lasso_opts* opts, double* x_host, double* gap_host, int32_t* kept_host,
                int64_t* n_kept, lasso_stats* stats);

/* Solve B independent signals with Algorithm 1 in one batch on `stream` (a cudaStream_t, NULL =
 * default stream); each signal has its own lambda, preserved set and ladder level.  Device
 * buffers: d_Y (B x N FP32, row b = y_b), d_lambdas (B FP64), d_X (B x K FP32 output),
 * d_gaps (B FP64 output), d_status (B int32 output: lasso_status per signal), d_iters (B int32
 * output, may be NULL); opts->kept_mask optionally receives the preserved sets.
 * 1 <= B <= 65535 and N <= 24576 after padding (LASSO_ERR_UNSUPPORTED, with the limit in the
 * message, beyond that).
 * Synchronisation: the passes run as a CUDA graph of opts->passes_per_sync passes, replayed
 * until every signal has stopped; between replays the host reads a 4-byte count of finished
 * signals from the device (one stream synchronisation per replay), and the stream is
 * synchronised before the call returns.  The FP64 second solve of saturated signals
 * (opts->fp64_fallback) allocates and frees its own buffers.
 * Per-signal status: LASSO_OK, LASSO_ERR_MAXITER (pass limit), LASSO_ERR_TIMEOUT (the call's
 * wall-clock limit; every live signal stops at its next pass), LASSO_ERR_NONFINITE (NaN / Inf
 * in y_b or in its gap), LASSO_ERR_INVALID_ARG (lambda_b not positive and finite).  On
 * MAXITER and TIMEOUT, row b of d_X is the signal's current point and d_gaps[b] the certificate
 * evaluated at it (the relative gap of the reduced problem).  The call returns
 * LASSO_ERR_TIMEOUT when the wall-clock limit stopped it, else LASSO_OK once every signal has
 * a status (per-signal errors are reported in d_status only), or a call-level error. */
int lasso_solve_batch(lasso_dict* dict, const float* d_Y, const double* d_lambdas, int64_t B,
                      double tol, const lasso_opts* opts, float* d_X, double* d_gaps,
                      int32_t* d_status, int32_t* d_iters, void* stream, lasso_stats* stats);

/* Same with host buffers (opts->kept_mask, if set, is host memory too): copies inputs to the
 * device, solves (Algorithm 1), copies results back. */
int lasso_solve_batch_host(lasso_dict* dict, const float* Y_host, const double* lambdas_host,
                           int64_t B, double tol, const lasso_opts* opts, float* X_host,
                           double* gaps_host, int32_t* status_host, lasso_stats* stats);

/* lambda_max = ||A^T y||_inf of B signals (eq:DefLMax: for lambda >= lambda_max the solution is
 * x = 0).  Device buffers: d_Y (B x N FP32), d_out (B FP64 output); exact level, error-free
 * products; queued on `stream` (a cudaStream_t).  May allocate its workspace on first use.
 * 1 <= B <= 65535 (LASSO_ERR_UNSUPPORTED beyond). */
int lasso_lambda_max(lasso_dict* dict, const float* d_Y, int64_t B, double* d_out, void* stream);

/* Same values as lasso_lambda_max, for callers that cannot allocate device memory (their
 * device memory belongs to another allocator, or they cannot afford cudaMalloc's implicit
 * synchronisation).  The paper has no counterpart: this is a deployment variant.
 * It allocates nothing, not even on its first call for a dictionary: its scratch is a fixed
 * 8 MiB array inside the library (1048576 doubles, held by every GPU that loads the library
 * until the process exits), and it reads only the exact level's atom rows.  Limits, each
 * returning LASSO_ERR_UNSUPPORTED with a message: B * ceil(K / 256) <= 1048576, B <= 65535,
 * and the padded signal must fit the 200 KiB of shared memory it is staged in (N <= 51200 for
 * FP32 dictionaries, N <= 25600 for FP64).  The dictionary's device must be the current CUDA
 * device (else LASSO_ERR_INVALID_ARG).
 * Device buffers: d_Y (B x N FP32, rows contiguous), d_out (B FP64).  The work is queued on
 * `stream` (a cudaStream_t; the call does not wait for it).  The first call on each device
 * looks up the scratch address with that device current.  Every call shares the one scratch array: calls whose work overlaps on the
 * GPU (other streams, other threads) race and must be serialised by the caller. */
int lasso_lambda_max_noalloc(const lasso_dict* dict, const float* d_Y, int64_t B, double* d_out,
                             void* stream);

/* Derivative of L(x*(y, A)) through the support system (not in the paper; derived from the
 * KKT conditions of Section II): with S = supp(x_b), u = (A_S^T A_S)^{-1} g_S,
 * dL/dy_b = A_S u and dL/dA[:, S] += r u^T - (A_S u) x_S^T, r = y_b - A_S x_S.  lambda is held
 * fixed.  Device buffers: d_Y (B x N), d_X (B x K solution), d_G (B x K, dL/dx), outputs
 * d_dY (B x N) and d_dA (K x N atom-major, accumulated over the batch; may be NULL).  Uses
 * the exact level of a dense dictionary; supports up to 1024 nonzeros per signal.  d_dA is
 * accumulated over the signals with FP32 atomic adds in no fixed order, so its last bits can
 * differ between runs; d_dY is deterministic. */
int lasso_backward(lasso_dict* dict, const float* d_Y, const float* d_X, const float* d_G,
                   int64_t B, float* d_dY, float* d_dA, void* stream);

/* DIAGNOSTIC, not part of the solve path.
 * Check of the tensor-core GEMM behind the batched BF16 / FP8 levels and the split exact level:
 * B x K correlations of random operands (N terms each; signed values, and all-positive values
 * for the worst accumulation) through tcgen05, compared with an FP64 evaluation of the same
 * products.  max_rel_err: largest |error| / sum_i |a_i r_i|; max_err_over_bound: largest |error|
 * over the accumulation bound the stable test assumes: gamma_n(u_tc) sum_i |a_i r_i| with
 * n = N + N/k products and k-steps (u_tc = 2^-22 for BF16, 2^-19 for E4M3); in split mode the
 * promoted bound (each k-block of 128 products a tensor-core chain, the k-block sums added in
 * FP32 with round to nearest).  mode: 0 = BF16, 1 = E4M3, 2 = split BF16 (a1 r1 + a1 r2 + a2 r1
 * with promoted accumulation, as the split level runs).  The paper has no counterpart: it checks
 * an assumption of this build's rounding model (products treated as exact there).  Returns
 * LASSO_ERR_INVALID_ARG for a mode outside 0-2, non-positive sizes or K * B > 2^28. */
int lasso_tc_selftest(int mode, int64_t K, int64_t N, int64_t B, double* max_rel_err, double* max_err_over_bound);

/* DIAGNOSTIC, not part of the solve path (the benchmark's roofline denominator).
 * Read bandwidth (GB/s) of a buffer resident in L2 (bytes in [1 MiB, 96 MiB]), read `rounds`
 * times by one launch with 16-byte loads that bypass L1; the roofline denominator of kernels
 * whose operands stay in L2 across a batch.  The paper has no counterpart (hardware
 * measurement).  Allocates and frees its buffer; synchronises the device. */
int lasso_probe_l2_read(int64_t bytes, int rounds, double* gbs);

const char* lasso_strerror(int status);

/* Build information ("sm_103a ..."). */
const char* lasso_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* LASSO_GB300_H */
