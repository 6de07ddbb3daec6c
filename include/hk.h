/*
 * hk.h -- C ABI of libhk: the extended-precision Cholesky factorisation of a
 * Hankel moment matrix and inverse iteration for its smallest eigenvalue, on
 * one NVIDIA GB300 (sm_103a).
 *
 * The operation (Emmart, Weems and Chen, "Computing the smallest eigenvalue of
 * large ill-conditioned Hankel matrices"):
 *   - the matrix is M_ij = m_{i+j}, i, j = 0..N-1, with the moments
 *     m_k = Gamma((1+k)/beta)/beta of the weight exp(-x^beta) (Introduction,
 *     definition of M; section "Hankel matrices, the moment problem ...");
 *   - M = R^T R with R upper triangular: the submatrix-order LDL^T of section
 *     "The LDL^T Determinant Algorithm" written as Cholesky (R = D^1/2 L^T);
 *   - inverse iteration with two triangular solves per step, lambda_t the
 *     inverse of the Rayleigh quotient of M^-1 (section "M is extremely
 *     ill-conditioned" bounds the spectrum by the Rayleigh quotient).
 *
 * Number format (hk_mp): value = (-1)^sign * m * 2^exp with the mantissa
 * m = sum_l limbs[l] * 2^(32 l), l = 0..L-1, L = P/32, normalised so that
 * 2^(P-1) <= m < 2^P, or m = 0 (then sign = 0 and exp = 0).  P is a multiple
 * of 32.  Exponents are 64-bit and never overflow in practice.
 *
 * Semantics, exactly as the CPU oracle computes them:
 *   A_ij = m_{i+j} - sum_{t<i} R_ti R_tj       (exact, no rounding)
 *   S_ij = RNE_P(A_ij);  S_ii <= 0 -> HK_ERR_NOT_PD
 *   R_ii = RNE_P(sqrt(S_ii));  R_ij = RNE_P(S_ij / R_ii)   (correctly rounded)
 *   y_i = RNE(RNE(v_i - sum_{k<i} R_ki y_k) / R_ii),
 *   w_i = RNE(RNE(y_i - sum_{k>i} R_ik w_k) / R_ii),
 *   lambda_t = RNE(RNE(<v,v>) / RNE(<v,w>)),  v <- w 2^-E (max |v_i| in [1/2,1)),
 *   starting from v = (1, ..., 1).
 * Every sum is exact; RNE is round to nearest, ties to even mantissa.
 *
 * Threading and streams: an hk_ctx is used by one host thread at a time.  All
 * device work is issued on the context's stream; calls that return host data
 * synchronise that stream before returning.
 *
 * Errors: every int-returning call returns an hk_status.  No call aborts the
 * process; on error the context stays usable (a new hk_load_moments resets it).
 */
#ifndef HK_H
#define HK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HK_OK = 0,
  HK_ERR_ARG = 1,      /* bad argument (size, precision, null pointer, unnormalised value) */
  HK_ERR_NOT_PD = 2,   /* a rounded pivot S_ii <= 0: P too small or M not positive definite */
  HK_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  HK_ERR_OOM = 4,      /* device allocation failed or caller workspace too small */
  HK_ERR_TIMEOUT = 5,  /* a bounded device wait ran out (no hang; the kernel returned) */
  HK_ERR_STATE = 6,    /* call out of order (e.g. hk_factor before hk_load_moments) */
  HK_ERR_RANGE = 7     /* exact-accumulation window exhausted after all widenings */
} hk_status;

/* One P-bit number; the caller owns limbs[L]. */
typedef struct {
  int32_t sign;      /* 0 or 1 */
  int64_t exp;       /* value = (-1)^sign * m * 2^exp */
  uint32_t *limbs;   /* L little-endian 32-bit limbs of m */
} hk_mp;

typedef struct hk_ctx hk_ctx;

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream).  *ctx receives the handle. */
int hk_create(hk_ctx **ctx, int device, void *cuda_stream);

/* Release every device buffer the library allocated and the context. */
void hk_destroy(hk_ctx *ctx);

/* Human-readable text for a status code (static storage). */
const char *hk_strerror(int code);

/* Device bytes hk_factor + hk_smallest_eig need for order N at precision P
 * (one widening of the exact-accumulation window included). */
int hk_workspace_bytes(int N, int P, size_t *bytes);

/* Use caller-owned device memory [dev_ptr, dev_ptr + bytes) as workspace
 * instead of library allocations.  The caller keeps it alive until the
 * context is destroyed or another workspace is set.  Too small -> HK_ERR_OOM
 * at the first call that needs more. */
int hk_set_workspace(hk_ctx *ctx, void *dev_ptr, size_t bytes);

/* Load the 2N-1 moments m_0..m_{2N-2} (host array of hk_mp, copied to the
 * device), defining M_ij = m_{i+j} (Introduction).  beta = beta_num/beta_den
 * is recorded for reporting only; the moments define the matrix.  Requires
 * 1 <= N, P a positive multiple of 32, every value normalised.  Resets any
 * previous factorisation. */
int hk_load_moments(hk_ctx *ctx, int N, int beta_num, int beta_den, int P,
                    const hk_mp *moments);

/* Same, from flat arrays: sign[2N-1] (int32), exp[2N-1] (int64) and
 * limbs[(2N-1) * L] (uint32, moment k at limbs + k*L).  With on_device = 0
 * the pointers are host memory (copied in); with on_device = 1 they are
 * device memory already resident in HBM (copied device to device). */
int hk_load_moments_flat(hk_ctx *ctx, int N, int beta_num, int beta_den, int P,
                         const int32_t *sign, const int64_t *exp, const uint32_t *limbs,
                         int on_device);

/* Factor M = R^T R.  On HK_ERR_NOT_PD, *bad_row (if non-NULL) receives the
 * first row whose rounded pivot is <= 0, as the oracle reports it. */
int hk_factor(hk_ctx *ctx, int *bad_row);

/* Select the kernel of the factorisation's trailing update for later
 * hk_factor calls: path 0 (default) = exact product scanning on the integer
 * multiply-add pipe with Karatsuba pieces; path 1 = the same exact
 * contraction on the INT8 tensor path (mma.sync m16n8k32 u8 x u8 -> s32 over
 * the bytes of the aligned entries, 64-bit drains).  Both give bit-identical R
 * (the contraction is exact integer arithmetic either way).  Invalidates a
 * previous factorisation. */
int hk_set_update_path(hk_ctx *ctx, int path);

/* Options of a context (take effect at the next hk_factor):
 *   HK_OPT_UPDATE_PATH      0 IMAD product scanning (default), 1 INT8 mma.sync
 *   HK_OPT_KARATSUBA        Karatsuba levels of the IMAD update, 0..4, or -1
 *                           (default): the depth of least modelled update
 *                           cost for the window width (four levels only for
 *                           N >= 768 and windows of about 580 limbs or more)
 *   HK_OPT_GRAPH            1: capture each factorisation's launch sequence in a
 *                           CUDA graph and replay it (default 0)
 *   HK_OPT_AUTOTUNE         1: choose the update kernel's stripe width and chunk
 *                           length per operand shape by timing the candidates on
 *                           synthetic operands (cached per process; default 0,
 *                           a cost model)
 *   HK_OPT_PANEL_ROWS       rows per panel block, 1..256 (default 16)
 *   HK_OPT_MAX_ITERS        step cap of hk_smallest_eig with iters = 0,
 *                           1..100000 (default 200); keeps the factorisation
 *   HK_OPT_WAIT_NS          limit in nanoseconds of every bounded device wait
 *                           of this context's kernels (a pipeline stage that
 *                           never fills, a copy that never lands), 1000 ..
 *                           6e10 (default 2e9); a wait that runs out makes its
 *                           kernel record the timeout and return, and the call
 *                           returns HK_ERR_TIMEOUT; keeps the factorisation
 *   HK_OPT_LOOKAHEAD        1 (default): while block b's rows are finished one
 *                           by one (the sequential panel chain, on a high-
 *                           priority stream), the update of block b + 1 by all
 *                           rows up to block b - 1 runs on a low-priority
 *                           stream, and only the contribution of block b waits
 *                           for its panel; in the solves of hk_smallest_eig
 *                           the GEMV of block b + 1 against the entries known
 *                           before block b runs beside block b's entry chain
 *                           the same way; 0: one stream, strictly in order
 * None of the first five, nor the lookahead, changes any result: every sum is
 * exact. */
enum { HK_OPT_UPDATE_PATH = 0, HK_OPT_KARATSUBA = 1, HK_OPT_GRAPH = 2, HK_OPT_AUTOTUNE = 3, HK_OPT_PANEL_ROWS = 4,
       HK_OPT_MAX_ITERS = 5, HK_OPT_WAIT_NS = 6, HK_OPT_LOOKAHEAD = 7 };
int hk_set_option(hk_ctx *ctx, int option, long long value);

/* Failure-detection self-test (no counterpart in the paper): on the context's
 * stream, one block arms a shared-memory barrier for a transfer that is never
 * issued and waits on it with the same bounded wait the update kernels use,
 * limited by HK_OPT_WAIT_NS.  The wait runs out, the kernel records the
 * timeout in the context's device status word and returns -- no hang, no
 * fault -- and the call returns HK_ERR_TIMEOUT (HK_OK would mean the wait
 * was not bounded as designed).  The status word is cleared afterwards, so
 * the context and any factorisation it holds stay usable.  Requires loaded
 * moments (HK_ERR_STATE otherwise). */
int hk_selftest_wait(hk_ctx *ctx);

/* Solve `count` independent instances (moments[k] holds the 2N[k]-1 host
 * moments of instance k at precision P[k]); beta is recorded for reporting.
 * Workers (nthreads, <= 0 means 16) each own a context and a CUDA stream of
 * ctx's device and take instances largest first (N^3 P^2); the options of ctx
 * apply to all.  Per instance: status_out[k] (an hk_status; HK_ERR_NOT_PD means
 * P[k] is too small), lambda_out[k] (caller limbs of P[k]/32 words) after
 * `iters` steps of inverse iteration (0 = until converged), iters_out[k] (may
 * be NULL) the steps taken, negated when iters = 0 and the step cap
 * (HK_OPT_MAX_ITERS) ended the iteration before the convergence test was met.
 * Every status_out[k] is written: an instance no worker reached (no worker
 * could start) keeps HK_ERR_CUDA.  Returns HK_OK when at least one worker
 * started (each instance then carries its own status), HK_ERR_CUDA when none
 * could. */
int hk_batch_solve(hk_ctx *ctx, int count, const int *N, const int *beta_num, const int *beta_den,
                   const int *P, const hk_mp *const *moments, int iters, int nthreads,
                   hk_mp *lambda_out, int *status_out, int *iters_out);

/* ----- the paper's own method -------------------------------------------------
 * P(x) = det(M - xI) by the submatrix-order LDL^T of section "The LDL^T
 * Determinant Algorithm", with every trailing sum accumulated exactly and
 * rounded once to P bits (RNE), as the CPU oracle of the method computes it:
 *   D_t    = RNE(m_2t - x - sum_{s<t} C_s[t] Q_s[t])            (pivots)
 *   C_t[r] = RNE(m_{t+r} - sum_{s<t} C_s[t] Q_s[r]),  r > t      (columns)
 *   Q_t[r] = RNE(C_t[r] / D_t)                                  (CDivDiag)
 *   det    = RNE(...RNE(RNE(D_0 D_1) D_2)... D_{N-1})          (running product)
 * Negative pivots are allowed (above lambda_1, M - xI is indefinite); a zero
 * pivot ends the factorisation with det = 0.  The trailing sums run on the
 * same exact update kernel as hk_factor.  These calls overwrite the
 * context's factor buffers: hk_smallest_eig needs a new hk_factor after them.
 *
 * hk_ldlt_det: x is a host P-bit value (normalised or zero), copied in; *det
 * (caller limbs[L]) receives P(x); *neg_pivots (may be NULL) the number of
 * negative pivots (the eigenvalues of M below x, by Sylvester's law of inertia,
 * when no pivot is zero); *zero_row (may be NULL) the first zero pivot or -1.
 * HK_ERR_RANGE when the exact-accumulation window could not be widened
 * enough. */
int hk_ldlt_det(hk_ctx *ctx, const hk_mp *x, hk_mp *det, int *neg_pivots, int *zero_row);

/* After hk_ldlt_det (or within hk_secant, its last determinant): which = 0 the
 * N pivots D_t into flat host arrays of N entries; 1 the columns C_t[r] (the
 * packed upper triangle of N(N+1)/2 entries, layout as hk_get_R_flat, the
 * pivots on its diagonal); 2 the quotients Q_t[r] (same layout, zero
 * diagonal).  HK_ERR_STATE before any LDL^T. */
int hk_get_ldlt_flat(hk_ctx *ctx, int which, int32_t *sign, int64_t *exp, uint32_t *limbs);

/* The Secant root finder of section "The Secant Algorithm" on P(x):
 *   x_2 = 0, x_1 = -min_t D_t(0) (the smallest pivot of M itself, negated),
 *   x_{i+1} = RNE(x_i - RNE(RNE(RNE(x_i - x_{i-1}) / RNE(P(x_i) - P(x_{i-1}))) P(x_i)))
 * until |x_{i+1} - x_i| <= 2^-136 |x_{i+1}| exactly, P(x_i) = P(x_{i-1}), or
 * (after three steps) a step no shorter than the one before it; at most
 * max_steps steps.  Every determinant is hk_ldlt_det's; the recurrence runs in
 * single-block device kernels.  *root (caller limbs[L]) receives the last
 * iterate (lambda_1 to the working precision); *dets_used (may be NULL) the
 * number of determinants evaluated, which is also the number of iterates
 * x_1, x_2, ... that hk_get_secant_flat returns. */
int hk_secant(hk_ctx *ctx, int max_steps, hk_mp *root, int *dets_used);

/* The first `count` iterates x_1, x_2, ... and their determinants P(x_k) of
 * the last hk_secant, into flat host arrays of `count` entries each. */
int hk_get_secant_flat(hk_ctx *ctx, int count, int32_t *xsign, int64_t *xexp, uint32_t *xlimbs, int32_t *psign,
                       int64_t *pexp, uint32_t *plimbs);

/* Verification of a root (section "Interval Verification"): the shifted LDL^T
 * at x_lo = x (1 - 2^-bits) and x_hi = x (1 + 2^-bits), both exact at P2 bits
 * (P2 a multiple of 32, P2 >= P + bits + 1, <= 32768), on the context's
 * moments zero-extended to P2 bits.  out4[0], out4[1]: negative pivots at x_lo
 * and x_hi; out4[2], out4[3]: the signs of their determinants (1, -1, 0).
 * The root is accepted when out4 = {0, 1, 1, -1}: M - x_lo I has no negative
 * eigenvalue and M - x_hi I exactly one.  The pivots are rounded at P2 bits,
 * so this is the inertia of the once-rounded factorisation, not an interval
 * proof.  x must be nonzero and normalised.  Uses a temporary context on the
 * same device and stream. */
int hk_secant_verify(hk_ctx *ctx, const hk_mp *x, int bits, int P2, int *out4);

/* Copy R (row-major packed upper triangle, N(N+1)/2 entries, entry (t, j),
 * j >= t, at index t*N - t*(t-1)/2 + (j - t)) to host hk_mp values whose
 * limbs arrays the caller provides. */
int hk_get_R(hk_ctx *ctx, hk_mp *R);

/* Same into flat host arrays of N(N+1)/2 entries. */
int hk_get_R_flat(hk_ctx *ctx, int32_t *sign, int64_t *exp, uint32_t *limbs);

/* Inverse iteration after hk_factor.  iters > 0: exactly that many steps.
 * iters == 0: until |lambda_t - lambda_{t-1}| <= 2^-136 lambda_t or the step
 * cap (HK_OPT_MAX_ITERS, default 200); hk_get_stats out[5] says which.
 * *lambda_min receives lambda_T (caller-provided limbs[L]); *iters_used the
 * step count. */
int hk_smallest_eig(hk_ctx *ctx, int iters, hk_mp *lambda_min, int *iters_used);

/* Last hk_smallest_eig history lambda_1..lambda_T into flat host arrays of
 * `count` entries (count <= iters_used). */
int hk_get_history_flat(hk_ctx *ctx, int count, int32_t *sign, int64_t *exp, uint32_t *limbs);

/* Per-phase device times in milliseconds of the last hk_factor /
 * hk_smallest_eig: out[0] update kernels, out[1] panel (diagonal and row)
 * kernels, out[2] solve kernels, out[3] total factor, out[4] total
 * inverse iteration.  n = number of doubles provided (<= 8). */
int hk_get_timings(hk_ctx *ctx, double *out, int n);

/* Launch statistics of the last hk_factor + hk_smallest_eig: out[0] kernels
 * launched, out[1] exact-accumulation window width W in limbs, out[2]
 * widenings taken, out[3] Karatsuba levels of the factor update, out[4] limb
 * products the update executes per P-bit multiply-accumulate, out[5] 1 if the
 * last hk_smallest_eig with iters = 0 met the convergence test, out[6] and
 * out[7] the largest and mean window width in limbs of the solution vectors
 * in that hk_smallest_eig (the exact products of a solve cost W x that width),
 * out[8] how many window widenings of the last hk_factor resumed at the
 * failing block (re-aligning the finished rows) instead of restarting,
 * out[9] and out[10] how many solve blocks of that hk_smallest_eig used the
 * GEMV the lookahead prepared for them, and how many prepared GEMVs were
 * dropped because the block's vector range did not fit their grid.
 * n = number of int64 provided (entries past 10 are set to 0). */
int hk_get_stats(hk_ctx *ctx, int64_t *out, int n);

/* ----- measurement hook ------------------------------------------------------
 * Integer throughput of the device (a few ms on every SM): out[0] IMAD
 * (mad.lo.u32) per clock per SM and out[1] the SM clock in MHz seen by that
 * probe; out[2] exact 32x32->64 limb products per clock per SM in the 3-word
 * accumulation form of the update kernel (mad.lo.cc/madc.hi.cc/addc), out[3]
 * its clock; out[4] u8 multiply-adds per clock per SM of mma.sync m16n8k32
 * (the warp-level INT8 tensor instruction), out[5] its clock.  n >= 6.
 * There is no counterpart in the paper: it measures the roofline denominator.
 * Makes `device` current for the calling thread; its work runs on a private
 * non-blocking stream (events and copies ordered on it), so it neither waits
 * for nor blocks other streams, and several host threads may call it. */
int hk_probe_int_peaks(int device, double *out, int n);

/* Measurement hook (no counterpart in the paper): after hk_factor, re-runs the
 * exact update kernel for the contributions of the first `tsteps` panel steps
 * (rows t < tsteps of R) to every later entry -- sum_{t < min(i, tsteps)}
 * R_ti R_tj for all i <= j -- into scratch column sums that are discarded,
 * and returns the device time of those launches (*ms, CUDA events on the
 * context's stream) and their P-bit multiply-accumulates (*macs).  The factor
 * is not changed.  This is the slice of the factorisation that the CPU
 * oracle's timed sample computes. */
int hk_time_update_slice(hk_ctx *ctx, int tsteps, double *ms, double *macs);

/* ----- self-test hooks of the device multiprecision library ----------------
 * Run one single-CTA device operation on host operands (copied in and out) so
 * that tests can compare it with exact integer arithmetic:
 *   op 0: out = x * y                       (nx, ny limbs; out nx+ny limbs)
 *   op 1: out = floor(2^(2P+1) / x)          (x: L limbs normalised; out L+2)
 *   op 2: out = RNE_P(sqrt(x * 2^e)) mantissa, *eo exponent (x: L limbs)
 *   op 3: out = RNE_P((x 2^e) / (y 2^f)) mantissa, *eo exponent
 *   op 4: out = RNE_P(|x| 2^e) of an nx-limb integer, *eo exponent
 * `out` has room for the stated limbs.  Runs on the calling thread's current
 * device, on a private non-blocking stream (stream-ordered copies, then a
 * synchronisation of that stream only); safe from several host threads. */
int hk_selftest_mp(int op, int L, const uint32_t *x, int nx, int64_t ex,
                   const uint32_t *y, int ny, int64_t ey, uint32_t *out, int64_t *eo);

/* Self-test of the scalar P-bit operations of the Secant recurrence (the
 * kernels behind hk_secant), on host values of L limbs (copied in and out,
 * on a private stream): op 0: *out = RNE(a - b) (exact difference, rounded
 * once; an operand more than P + 64 bits below the other enters as a sticky
 * unit), op 1: *out = RNE(a b), op 2: *out = RNE(a / b) (b nonzero),
 * op 3: *cmp = -1, 0 or 1 as a < b, a = b, a > b (exact comparison). */
int hk_selftest_scalar(int op, int L, const hk_mp *a, const hk_mp *b, hk_mp *out, int *cmp);

/* ----- allocation-free multiprecision operation ----------------------------
 * The paper has no counterpart: this is a service for callers that must not
 * allocate device memory -- code whose device memory is owned by another
 * allocator (a framework's caching allocator holding the whole budget), or
 * latency-sensitive loops in which cudaMalloc/cudaFree would add implicit
 * device synchronisation.  Same operations and op codes as hk_selftest_mp,
 * but x, y, out and eo are DEVICE pointers and the work runs asynchronously
 * on `stream` (a cudaStream_t, NULL = legacy default stream); the results are
 * valid once the stream reaches this point.  out needs nx+ny+2 limbs (op 0),
 * L+2 (op 1) or L (ops 2-4); eo needs 2 int64 (exponent, and 1 if an exact
 * correction did not settle).  For ops 1 and 2, nx = L; for op 3, nx = ny = L.
 *
 * No memory is allocated: the work area is one fixed device array of about
 * 1.3 MB inside the library (every GPU that loads the library holds it until
 * the process exits), so sizes are limited to nx + ny + L <= 4096 limbs, and
 * ops 1-4 to P = 32 L <= 32768 bits (the range their error bounds cover);
 * larger requests return HK_ERR_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (concurrent streams or host threads)
 * race and must be serialised by the caller.  Each call clears the part of the
 * array it uses before its kernel runs. */
int hk_mp_op_noalloc(int op, int L, const uint32_t *x, int nx, int64_t ex,
                     const uint32_t *y, int ny, int64_t ey, uint32_t *out, int64_t *eo,
                     void *stream);

/* ----- precision predictor network ------------------------------------------
 * The paper has no learned component.  Its precision requirement grows with N
 * (Introduction; the K column of Table 2), and each P-bit multiply-accumulate
 * costs about (P/32)^2 limb products, so the library carries a small network
 * that predicts, from (N, beta), the working precision, log2 lambda_min and the
 * iteration count; the caller verifies each prediction by a rerun at P + 1024
 * bits.  Network: 2 -> 64 -> 64 -> 3, exact GELU z Phi(z) after both hidden
 * layers, float32.  Parameters are one flat device array of HK_MLP_NPARAMS
 * floats, row-major W[out][in]:
 *   W1[64][2], b1[64], W2[64][64], b2[64], W3[3][64], b3[3].
 * Loss of a batch of B samples (inputs x[B][2], targets t[B][3], per-output
 * weights w[3]):  (1/B) sum_b sum_k w_k (y_bk - t_bk)^2.
 * All pointers are DEVICE pointers; work runs asynchronously on `stream`
 * (a cudaStream_t, NULL = legacy default).  Sums run in a fixed order, so every
 * call is deterministic.  Errors: HK_ERR_ARG for B < 1 or a null pointer,
 * HK_ERR_OOM for a work area below hk_mlp_workspace_bytes(B), HK_ERR_CUDA for a
 * failed launch. */
#define HK_MLP_NPARAMS 4547
size_t hk_mlp_workspace_bytes(int B);
/* y[B][3] = network(x). */
int hk_mlp_forward(const float *params, const float *x, int B, float *y, void *stream);
/* *loss and grad[HK_MLP_NPARAMS] (d loss / d params) by back-propagation. */
int hk_mlp_loss_grad(const float *params, const float *x, const float *t, const float *w, int B,
                     float *grad, float *loss, void *work, size_t work_bytes, void *stream);
/* One Adam step (Kingma and Ba) on n parameters with moment arrays m, v,
 * step index `step` >= 1 (bias corrections 1 - beta^step). */
int hk_mlp_adam(float *params, const float *grad, float *m, float *v, int n, int step, float lr,
                float beta1, float beta2, float eps, void *stream);
/* `steps` full-batch Adam steps (indices step0+1 .. step0+steps) on the
 * HK_MLP_NPARAMS parameters; loss_hist (device, may be NULL) receives the loss
 * before each step.  grad is a device array of HK_MLP_NPARAMS floats. */
int hk_mlp_train(float *params, float *m, float *v, float *grad, const float *x, const float *t,
                 const float *w, int B, int steps, int step0, float lr, float beta1, float beta2,
                 float eps, float *loss_hist, void *work, size_t work_bytes, void *stream);

/* Host-side plan of the exact update kernel for an accumulation window of W
 * limbs: what hk_factor launches for that window when schedules are not
 * autotuned (HK_OPT_AUTOTUNE 0, the default).  No GPU work, no device memory;
 * for tests and tooling.  The plan expands every aligned entry a[0..W) into
 * Karatsuba pieces (lo, hi, lo + hi of a split, recursively), contracts piece k
 * of the X entries with piece k of the Y entries exactly, and adds that
 * contraction to the result at each of its terms (offset in limbs, sign).
 *   levels     Karatsuba depth 0..4, or -1 for the depth of least modelled
 *              update cost (the hk_factor default for N >= 768; smaller
 *              factorisations stop at three levels); four levels only where
 *              three update blocks still fit an SM, and windows below 64
 *              limbs take at most three
 *   info[9]    out: [0] depth, [1] pieces n, [2] expanded entry stride in
 *              limbs, [3] zero gap between pieces (limbs), [4] stripe width
 *              uc, [5] chunk length upc, [6] units, [7] blocks per output with
 *              their own operand window (0: blocks stage whole entries), [8]
 *              column-sum width C
 *   splits[40] out (may be NULL): the split points level by level -- [0] the
 *              level-1 split, [1..4) the level-2 splits of the lo, hi, lo+hi
 *              pieces, [4..13) the level-3 splits of the nine level-2 pieces,
 *              [13..40) the level-4 splits of the 27 level-3 pieces (unused
 *              levels 0)
 *   pieces     out (may be NULL, 3 x 81 ints): per piece k < n its offset in
 *              the expanded entry, width, number of terms
 *   terms      out (may be NULL, 2 x 16 x 81 ints): term t of piece k at
 *              [2(16k + t)] (offset in limbs) and [2(16k + t) + 1] (sign +-1)
 *   units      out (may be NULL, 2 x ucap ints): unit u = (piece << 24 |
 *              first result column of its stripe, first p of its chunk)
 *   win        out (may be NULL, 2 x 64 ints): block b's operand window
 *              (first limb, limbs) within the expanded entry
 * Returns HK_ERR_ARG for W < 1, levels outside -1..4, a NULL info, or ucap
 * below the unit count when units is given. */
int hk_update_plan(int W, int levels, int64_t *info, int32_t *splits, int32_t *pieces, int32_t *terms,
                   int32_t *units, int64_t ucap, int32_t *win);

/* Load a trained predictor network into the context: params = HK_MLP_NPARAMS
 * host floats (layout above), scales = 10 host doubles: feature means and
 * standard deviations (2 + 2; features log2 N - 8 and log2 beta) and target
 * means and standard deviations (3 + 3; targets (bits - 128)/N,
 * log2(lambda_min)/N and log2(iterations)).  Copied; the context keeps them. */
int hk_set_predictor(hk_ctx *ctx, const float *params, const double *scales);

/* Predict for `count` instances (host arrays N[count], beta[count] > 0): out3
 * (host, count x 3 floats) receives the required precision in bits (before any
 * safety margin), log2 lambda_min and the iteration count to convergence.
 * Runs the network on the context's device and stream; returns after the
 * results are on the host.  HK_ERR_STATE if no network was loaded. */
int hk_predict(hk_ctx *ctx, int count, const double *N, const double *beta, float *out3);

#ifdef __cplusplus
}
#endif

#endif /* HK_H */
