/*
 * pes.h -- C-ABI of libpes: evaluation and differentiation of a polynomial at
 * power series in multiple double precision, on one GB300 GPU (sm_103a).
 *
 * Method: J. Verschelde, "Accelerated Polynomial Evaluation and Differentiation
 * at Power Series in Multiple Double Precision" (2021).
 *   - A series is truncated at degree d: d+1 coefficients (Sec. 2).
 *   - A coefficient is a multiple double: an unevaluated sum of k doubles,
 *     k in {1, 2, 3, 4, 5, 8, 10} (Sec. 1, "Contributions").
 *   - The polynomial is p = a_0 + sum_{m=1..N} a_m x_{i_1} ... x_{i_{n_m}}
 *     (Eq. eqpolynomial) with coefficient series a_m and variable supports
 *     i_1 < ... < i_{n_m}; it is evaluated, with all n partial derivatives, at
 *     n input series z_1..z_n (problem statement of Sec. 5).
 *   - The work is the reverse mode of Sec. 3 (forward, backward and cross
 *     products of every monomial) as layered convolution jobs (Sec. 5), followed
 *     by the addition of the monomial contributions.
 *
 * Layout of every series buffer: limb-major, float64, contiguous:
 *   buffer[l][s][j] at ((l * n_series) + s) * (d + 1) + j,
 * limb l in [0, k), series s, coefficient j in [0, d].  Limb 0 holds the leading
 * double of every coefficient; outputs are normalised (nonoverlapping limbs,
 * each limb at most half an ulp of the previous one).
 *
 * Ownership: the caller owns every data buffer (device memory of the current
 * device).  A plan owns its job tables and its workspace in device memory.
 * Calls taking a stream are asynchronous on that stream (a cudaStream_t, NULL
 * for the legacy default stream); device-side failures (a bounded wait that
 * gave up) are recorded in the plan and returned by pes_check.  Calls on one
 * plan must not overlap in time (they share the plan's workspace).
 *
 * Every function returns PES_OK or an error code; nothing traps or aborts.
 */
#ifndef PES_H
#define PES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PES_OK = 0,
  PES_EINVAL = 1,            /* invalid argument (message in pes_last_error) */
  PES_EUNSUPPORTED_K = 2,    /* k not in {1,2,3,4,5,8,10} */
  PES_ENOMEM = 3,            /* device or host allocation failed */
  PES_ECUDA = 4,             /* a CUDA runtime call failed */
  PES_ETIMEOUT = 5,          /* a device-side wait gave up (see pes_check) */
  PES_EINTERNAL = 6,         /* inconsistent internal state */
  PES_EUNSUPPORTED_SIZE = 7  /* degree above 16383, a tile or thread count that does not fit, or a
                                problem above the static array of pes_eval_grad_static */
} pes_status;

typedef struct pes_plan_s* pes_plan_t;
typedef struct pes_batch_s* pes_batch_t;

/* Arithmetic of the convolution multiply-accumulate loop.  Both accumulate the
 * digit products of every output coefficient exactly and round the sum once to
 * k limbs (24-bit digits on the FP64 FMA pipe, 28-bit digits with 32x32->64-bit
 * integer multiply-add); results agree to within the last limb's rounding.
 * PES_ARITH_AUTO takes the integer pipe. */
enum { PES_ARITH_AUTO = -1, PES_ARITH_FP64 = 0, PES_ARITH_INT = 1 };

typedef struct {
  int32_t arith;       /* PES_ARITH_AUTO (default), PES_ARITH_FP64 or PES_ARITH_INT */
  int32_t threads;     /* threads per CTA of the convolution kernel (a multiple of 32), 0 = automatic.
                          Integer pipe: the lanes are spread evenly over the coefficient pairs (j, d-j),
                          automatic = two lanes per pair (one per output coefficient; three at k = 10),
                          at least one lane per pair; FP64 pipe: automatic = 128 */
  int32_t ctas_per_sm; /* persistent CTAs per SM; 0 = as many as fit */
  int32_t with_vjp;    /* 1: also build the tables of pes_vjp (default 1) */
  int64_t timeout_ms;  /* bound on every device-side wait; 0 = default (60000) */
  int32_t profile;     /* 1: record CUDA events around each launch of a call (see pes_last_timing) */
  int32_t autotune;    /* 1 = on the first call, time the candidate launch shapes of the convolution
                          kernel (threads per CTA, CTAs per SM, staging depth; for a batch, of every
                          group) on the caller's data and keep the fastest (cached in
                          $PES_AUTOTUNE_CACHE, else ~/.cache/pes_autotune.txt) */
  int32_t staging;     /* staging depth of the convolution kernel: 1 = a CTA stages a job's operands
                          after rounding the previous job; 2 = it claims the next job and, if that
                          job's operands are complete, stages them while rounding the current one
                          (a separate staging buffer: more shared memory); 0 = automatic (1, and both
                          are tried when autotuning) */
  int32_t split;       /* parts per convolution job (integer pipe): 1, 2, 4, 8 or 16; each part computes
                          the output coefficients of a contiguous range of coefficient pairs (j, d-j), so a
                          job's dependants wait for all its parts; more parts shorten the chains of long
                          monomials; 0 = automatic: the parts double while the table's average layer, times
                          the parts, holds fewer jobs than the launch has CTAs and every part keeps at
                          least 8 coefficient pairs (the p2-like workload at d=152, k=10: 1 for its 128
                          monomials, 2 for 64 of them, 4 for 32, 8 for 16 or fewer; p3: 1); when
                          autotuning, 1, 2 and the automatic choice, half and twice it, are tried */
  int32_t tile;        /* 0 = automatic: the whole series of a job's operands are staged in shared memory
                          when they fit (integer / FP64 pipe: d <= 471 / 359 at k=10, 543 / 447 at k=8,
                          839 / 607 at k=5, 991 / 815 at k=4, 1075 / 919 at k=3, 1351 / 1231 at k=2,
                          1535 / 1487 at k=1), else the tiled kernel with tiles of 128 coefficients.
                          > 0 (a multiple of 8 in [16, 1024]): always the tiled kernel with tiles of this
                          many coefficients: every job is split into output tiles, each accumulated tile
                          pair by tile pair from staged tiles of its operands (any degree up to 16383; the
                          same bits as the whole-series kernel) */
} pes_options;

/* Fill *opt with the defaults. */
void pes_default_options(pes_options* opt);

/* ---- plans ------------------------------------------------------------------ */

/* Compile the job tables of one polynomial (Sec. 5, data staging) and allocate
 * its workspace.
 *   supp_ptr: N+1 row pointers into supp_idx (supp_ptr[0] == 0);
 *   supp_idx: 0-based variable indices of monomials 1..N, strictly increasing
 *             within a monomial (the paper's i_1 < ... < i_{n_k}, 1-based);
 *   N >= 0 monomials (a_0 is implicit), n >= 1 variables, 0 <= d <= 16383, k as above.
 * Errors: PES_EINVAL (bad sizes, empty monomial, index out of range, unsorted or
 * repeated index), PES_EUNSUPPORTED_K, PES_EUNSUPPORTED_SIZE, PES_ENOMEM,
 * PES_ECUDA.  The supports are copied; the caller keeps ownership. */
pes_status pes_plan(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n, int32_t d,
                    int32_t k, pes_plan_t* out);
pes_status pes_plan_ex(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n, int32_t d,
                       int32_t k, const pes_options* opt, pes_plan_t* out);

/* Monomials with positive powers (Sec. 3): monomial m is
 * a_m prod_t x_{supp_idx[t]}^{supp_exp[t]} over its support entries t.
 * supp_exp holds one exponent in [1, 64] per support entry.  The common factor
 * prod z_v^(e_v - 1) is formed from a table of series powers (repeated
 * products) and folded into the coefficient series, the reverse mode runs on
 * the monomial of exponents one, and every partial derivative is added with
 * the variable's exponent as an integer factor; pes_eval_grad and pes_vjp then
 * work as for any plan.  Everything else as pes_plan_ex. */
pes_status pes_plan_powers(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp, int32_t N,
                           int32_t n, int32_t d, int32_t k, const pes_options* opt, pes_plan_t* out);

/* Complex coefficient and input series (Sec. 4 and 5 keep real and imaginary
 * parts in separate arrays).  pes_eval_grad on such a plan takes
 *   coeff [2][k][N+1][d+1], input [2][k][n][d+1], value [2][k][d+1], grad [2][k][n][d+1],
 * the real block followed by the imaginary block.  Every complex product is
 * four real ones combined exactly (the real part xr yr - xi yi, the imaginary
 * part xr yi + xi yr); the value and every partial are rounded once per
 * component.  supp_exp may be NULL (exponents 1) or as in pes_plan_powers.
 * pes_vjp on a complex plan takes upstream [2][k][d+1] and writes
 * grad_input [2][k][n][d+1] and grad_coeff [2][k][N+1][d+1]: the derivatives of
 * the real loss L = sum_j (Re u_j Re v_j + Im u_j Im v_j) with respect to the
 * real parts (first block) and the imaginary parts (second block) of every
 * series, i.e. the correlations of u with the conjugates of the gradient
 * series and of the monomial products. */
pes_status pes_plan_complex(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp, int32_t N,
                            int32_t n, int32_t d, int32_t k, const pes_options* opt, pes_plan_t* out);

/* A system of P polynomials in the same n variables, and its Jacobian matrix
 * (the value and Jacobian series that a Newton step on power series needs;
 * every entry is the gradient of Sec. 4 of one polynomial).  Polynomial p owns
 * the monomials poly_ptr[p] .. poly_ptr[p+1]-1 of supp_ptr / supp_idx /
 * supp_exp (exactly as in pes_plan_powers, N = poly_ptr[P] monomials in all,
 * supp_exp may be NULL) plus its own constant series.  All polynomials share
 * the input series and one job table; the products of every monomial are the
 * ones its own plan would compute, so every output is bit-identical to a plan
 * of that polynomial alone.  Evaluate with pes_eval_system (pes_eval_grad is
 * pes_eval_system with PES_LAYOUT_SERIES); pes_vjp takes one upstream series
 * per polynomial.
 *   P >= 1, poly_ptr: P+1 non-decreasing entries, poly_ptr[0] == 0.
 * Errors as pes_plan_ex, and PES_EINVAL for a bad poly_ptr. */
pes_status pes_plan_system(int32_t P, const int32_t* poly_ptr, const int32_t* supp_ptr, const int32_t* supp_idx,
                           const int32_t* supp_exp, int32_t n, int32_t d, int32_t k, const pes_options* opt,
                           pes_plan_t* out);
void pes_plan_destroy(pes_plan_t plan);

/* Value and gradient of the polynomial at the input series (Sec. 4 and 5).
 *   coeff: device, [k][N+1][d+1], index 0 is a_0;
 *   input: device, [k][n][d+1];
 *   value: device, [k][d+1]          (written);
 *   grad:  device, [k][n][d+1]       (written; series i is d p / d x_i).
 * Asynchronous on `stream`. */
pes_status pes_eval_grad(pes_plan_t plan, const double* coeff, const double* input, double* value, double* grad,
                         void* stream);

/* Output layouts of pes_eval_system. */
#define PES_LAYOUT_SERIES 0 /* value [k][P][d+1], jac [k][P][n][d+1]: one series per entry */
#define PES_LAYOUT_MATRIX 1 /* value [k][d+1][P], jac [k][d+1][P][n]: one row-major P x n matrix
                               (and P-vector) per power of t and limb, as a linearised
                               Newton step J_0 dx_j = r_j - sum_{i>=1} J_i dx_{j-i} reads them */

/* Values and Jacobian of a system plan (pes_plan_system) at the input series.
 *   coeff: device, [k][N+P][d+1]: for each polynomial p in order its constant
 *          series, then the coefficient series of its monomials (the constant
 *          of p at index poly_ptr[p] + p, monomial m of p at index m + p + 1);
 *   input: device, [k][n][d+1];
 *   value, jac: device, written in the chosen layout; jac entry (p, i) is
 *          d p / d x_i.
 * Asynchronous on `stream`.  PES_EINVAL for a plan that is not a system or an
 * unknown layout. */
pes_status pes_eval_system(pes_plan_t plan, const double* coeff, const double* input, double* value, double* jac,
                           int32_t layout, void* stream);

/* Vector-Jacobian product of the value series with an upstream series u:
 * for L = sum_j u_j v_j (v the value series),
 *   grad_coeff[0]  = u,
 *   grad_coeff[m]_j = sum_{l=j..d} u_l M_m[l-j],  M_m = prod_{i in S_m} z_i,
 *   grad_input[i]_j = sum_{l=j..d} u_l g_i[l-j],  g_i = d p / d x_i,
 * i.e. truncated correlations (transposed convolutions) of u with the monomial
 * products and with the gradient series (the derivative of a truncated series
 * product with respect to one factor is multiplication by the other, whose
 * transpose is the correlation); for monomials with powers M_m is the product
 * of the variables with their exponents.
 *   upstream:   device, [k][d+1];
 *   grad_input: device, [k][n][d+1] (written);
 *   grad_coeff: device, [k][N+1][d+1] (written).
 * On a system plan (pes_plan_system), L = sum_p sum_j u_{p,j} v_{p,j}:
 *   upstream [k][P][d+1] (one series per polynomial), grad_coeff [k][N+P][d+1]
 *   in the layout of the coefficient buffer (the constant of p receives u_p,
 *   monomial m of p the correlation of u_p with M_m), and grad_input[i] the sum
 *   over p of the correlations of u_p with the Jacobian series d p / d x_i,
 *   summed exactly and rounded once.
 * reuse_forward = 1: the plan's workspace still holds the forward, backward and
 * cross products of the last pes_eval_grad call on this plan with the same
 * coeff and input (no other call in between); only the correlations and the
 * monomial products are computed.  reuse_forward = 0: everything is recomputed.
 * Needs a plan built with with_vjp = 1.  Asynchronous on `stream`. */
pes_status pes_vjp(pes_plan_t plan, const double* coeff, const double* input, const double* upstream,
                   double* grad_input, double* grad_coeff, int32_t reuse_forward, void* stream);

/* Copy the plan's workspace (the forward, backward and cross products of the
 * last call) to a caller buffer (to_buffer = 1) or back from it (to_buffer = 0),
 * asynchronously on `stream`.  buffer: device, pes_plan_info.workspace_bytes
 * bytes.  Lets a caller keep the products of one call alive under its own
 * memory budget and reuse them later with pes_vjp(..., reuse_forward = 1). */
pes_status pes_workspace_io(pes_plan_t plan, void* buffer, int32_t to_buffer, void* stream);

/* Device time of the launches of the last pes_eval_grad / pes_vjp /
 * pes_eval_grad_batch call of a plan or batch built with profile = 1, measured
 * with CUDA events on the call's stream (waits for the events):
 *   ms[0] pack, ms[1] convolution kernel(s), ms[2] addition, ms[3] unpack
 * (for a batch ms[1] is the whole graph and the others are 0);
 * *launches receives the number of kernels the call launched. */
pes_status pes_last_timing(pes_plan_t plan, double* ms, int32_t* launches);
pes_status pes_batch_last_timing(pes_batch_t batch, double* ms, int32_t* launches);

/* Synchronise `stream`, then return (and clear) the device status of the plan:
 * PES_OK, or PES_ETIMEOUT when a bounded wait gave up during a call. */
pes_status pes_check(pes_plan_t plan, void* stream);

typedef struct {
  int64_t conv_jobs;       /* convolution jobs of pes_eval_grad (3n-3 per monomial of n >= 2 variables) */
  int64_t layers;          /* number of layers (largest monomial size) */
  int64_t add_terms;       /* series contributions summed by the addition stage */
  int64_t add_jobs;        /* pairwise additions of the paper's tree: add_terms - outputs with >=1 term */
  int64_t workspace_bytes; /* device workspace owned by the plan */
  int64_t vjp_conv_jobs;   /* extra convolutions of pes_vjp (monomial products) */
  int64_t vjp_corr_jobs;   /* correlations of pes_vjp (N + n) */
  int32_t digits;          /* digits per coefficient of the exact dot product */
  int32_t grid;            /* persistent CTAs of the convolution kernel */
  int32_t threads;         /* threads per CTA */
  int32_t smem_bytes;      /* dynamic shared memory per CTA */
  int32_t arith;           /* PES_ARITH_FP64 or PES_ARITH_INT: the pipe the plan uses */
  int32_t staging;         /* staging depth in use (1 or 2) */
  int32_t split;           /* parts per convolution job in use */
  int32_t complex_series;  /* 1 for a plan of pes_plan_complex */
  int32_t system_P;        /* polynomials of a plan of pes_plan_system, else 0 */
  int32_t tile;            /* coefficients per output tile of the tiled kernel; 0: whole-series kernel */
} pes_plan_info;

pes_status pes_get_plan_info(pes_plan_t plan, pes_plan_info* info);

/* ---- one polynomial split over ranks ---------------------------------------------
 *
 * The monomials of a polynomial are independent through the convolution layers;
 * only the addition jobs combine their contributions (Sec. 5).  So a polynomial
 * can be split over R ranks (one GPU each) by monomials: rank r plans the
 * polynomial of its own monomials (pes_plan / pes_plan_powers, the constant a_0
 * on one rank only, zero on the others) and the ranks exchange two exact integer
 * arrays.  With pes_partial_grids, an all-reduce (maximum) of the grids,
 * pes_partial_sums, an all-reduce (sum) of the digit sums and pes_round_sums,
 * every rank obtains the value and gradient that one plan of the whole polynomial
 * computes, bit for bit: the addition stage sums the contributions of every
 * output coefficient on the largest grid among them and rounds once, and both
 * the maximum and the sum of integers are exact in any order.  (A sum of the
 * ranks' rounded k-double limbs in floating point would not be.)
 *
 * Item o (d + 1) + j is coefficient j of the value (o = 0) or of d p / d x_i
 * (o = 1 + i); L is pes_plan_info.digits. */

/* The contiguous range [*m_begin, *m_end) of monomials (0-based, of supp_ptr's
 * N monomials) that rank `rank` of `world` takes: cut where the running sum of
 * the monomials' convolution jobs (3 n_m - 3, one for n_m = 1) crosses
 * r W / world, W the total, so no rank holds more than W / world plus one
 * monomial's jobs.  Host only.  PES_EINVAL for bad sizes or an empty monomial. */
pes_status pes_shard_range(const int32_t* supp_ptr, int32_t N, int32_t world, int32_t rank, int32_t* m_begin,
                           int32_t* m_end);

/* Run the plan's convolutions (as pes_eval_grad does) and write, for every item,
 * the largest grid of its contributions (a grid below -100000 when it has none).
 *   grids: device, int32 [(n+1)(d+1)] (written).
 * Real single-polynomial plans only (PES_EINVAL for complex or system plans).
 * Asynchronous on `stream`. */
pes_status pes_partial_grids(pes_plan_t plan, const double* coeff, const double* input, int32_t* grids,
                             void* stream);

/* Sum every item's contributions exactly on the grid `grids` gives it (the
 * elementwise maximum over all ranks of pes_partial_grids), dropping the digits
 * below its L digits as the addition stage does, and write the L digit sums
 * unrounded: acc[item * L + p] weighs 2^(28 (g - 1 - p)) (24 bits for the FP64
 * pipe), g = grids[item].  Uses the products of the last pes_partial_grids call
 * on this plan (no other call in between).
 *   grids: device, int32 [(n+1)(d+1)];  acc: device, int64 [(n+1)(d+1)][L] (written).
 * Asynchronous on `stream`. */
pes_status pes_partial_sums(pes_plan_t plan, const int32_t* grids, int64_t* acc, void* stream);

/* Round digit sums (pes_partial_sums summed over the ranks) on their grids to k
 * limbs, once per item, as the addition stage rounds: value [k][d+1] and grad
 * [k][n][d+1] (device, written).  Asynchronous on `stream`. */
pes_status pes_round_sums(pes_plan_t plan, const int32_t* grids, const int64_t* acc, double* value, double* grad,
                          void* stream);

/* The same rounding on the host (host buffers; no GPU needed), for k limbs and
 * the digits of `arith` (PES_ARITH_INT or PES_ARITH_FP64), n variables, degree d. */
pes_status pes_round_sums_host(int32_t k, int32_t arith, int32_t n, int32_t d, const int32_t* grids,
                               const int64_t* acc, double* value, double* grad);

/* ---- batches: many polynomials in one persistent launch (CUDA graph) ---------- */

/* count instances; instance b has n[b] variables, N[b] monomials and degree
 * d[b]; its supports are rows supp_ptr[P_b .. P_b + N[b]] (each instance's row
 * pointers start at 0) with P_b = sum_{c<b} (N[c] + 1), indexing supp_idx from
 * Q_b = sum_{c<b} supp_ptr[P_c + N[c]].  All instances share k.
 * The buffers of pes_eval_grad_batch concatenate the instances' buffers in
 * order, each laid out as for pes_eval_grad; pes_batch_offsets gives where each
 * instance starts. */
pes_status pes_plan_batch(int32_t count, const int32_t* n, const int32_t* N, const int32_t* d,
                          const int32_t* supp_ptr, const int32_t* supp_idx, int32_t k, const pes_options* opt,
                          pes_batch_t* out);
/* The same for monomials with powers (as pes_plan_powers): supp_exp holds one
 * exponent in [1, 64] per entry of supp_idx (or is NULL: exponents 1). */
pes_status pes_plan_batch_powers(int32_t count, const int32_t* n, const int32_t* N, const int32_t* d,
                                 const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp,
                                 int32_t k, const pes_options* opt, pes_batch_t* out);
void pes_batch_destroy(pes_batch_t batch);

/* Offsets (in doubles) of instance b in the concatenated buffers, arrays of
 * count+1 entries (the last is the total length).  Any pointer may be NULL. */
pes_status pes_batch_offsets(pes_batch_t batch, int64_t* coeff_off, int64_t* input_off, int64_t* value_off,
                             int64_t* grad_off);

/* All instances at once.  Instances are grouped by the CTA shape their degree
 * needs; every group is one pack, one persistent convolution launch over its
 * concatenated job tables and one addition launch; the groups run on forked
 * streams; the whole call is captured once as a CUDA graph (re-captured when the
 * caller's buffers change) and replayed. */
pes_status pes_eval_grad_batch(pes_batch_t batch, const double* coeff, const double* input, double* value,
                               double* grad, void* stream);
pes_status pes_batch_check(pes_batch_t batch, void* stream);
pes_status pes_get_batch_info(pes_batch_t batch, pes_plan_info* info);

/* ---- multiple double numbers --------------------------------------------------- */

/* Elementwise out = x + y (op 0) or x * y (op 1) of `count` k-double numbers,
 * limb-major [k][count], device buffers (Sec. 1 arithmetic: FMA TwoSum/TwoProd
 * with renormalisation). */
pes_status pes_md_binary(int32_t op, int32_t k, const double* x, const double* y, double* out, int64_t count,
                         void* stream);

/* Double-precision-equivalent cost of one k-double multiplication and addition
 * (Sec. 6.2 gives 3089 and 397 for k = 10; other k use the FP64 operation
 * counts of this library's md_mul and md_add). */
pes_status pes_md_costs(int32_t k, double* mul_ops, double* add_ops);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (2 flops per
 * FMA), best of `repeats` timed launches over all SMs. */
pes_status pes_fp64_peak(int32_t repeats, double* tflops);

/* Measured throughput of 32x32->64-bit integer multiply-add (the digit product
 * of PES_ARITH_INT) on the current device, in tera-operations per second, in
 * the form the convolution kernel issues it: 64-bit accumulators and operands
 * read from shared memory (an 8 x 8 outer product per pair of 8-digit rows), so
 * that the compiler cannot replace the products by additions. */
pes_status pes_int_peak(int32_t repeats, double* tops);

/* ---- job compiler introspection (host only; no GPU needed) --------------------- */

/* stats[0] conv jobs, [1] layers, [2] add terms, [3] paper add jobs,
 * [4] slots of the data array, [5] add levels of the paper's tree, [6] vjp extra
 * convolutions, [7] correlations.  layer_sizes[0..cap) receives the number of
 * jobs per layer.  paper_layout = 1 counts the data array of Eq. (eqcountnum). */
pes_status pes_jobc_stats(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                          int32_t paper_layout, int64_t* stats, int32_t* layer_sizes, int32_t cap);
/* The same for monomials with powers (supp_exp as in pes_plan_powers). */
pes_status pes_jobc_stats_powers(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp, int32_t N,
                                 int32_t n, int32_t paper_layout, int64_t* stats, int32_t* layer_sizes, int32_t cap);

/* Convolution jobs in dispatch order: jobs[4 t + 0..3] = (input 1, input 2,
 * output, layer), inputs and outputs as slots of the data array (multiply by
 * d+1 for the paper's offsets of Sec. 5); at most cap jobs. */
pes_status pes_jobc_jobs(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                         int32_t paper_layout, int32_t* jobs, int64_t cap);
/* The same for monomials with powers (supp_exp as in pes_plan_powers). */
pes_status pes_jobc_jobs_powers(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp, int32_t N,
                                int32_t n, int32_t paper_layout, int32_t* jobs, int64_t cap);

/* Sizes of the levels of the paper's pairwise addition tree (Sec. 5 and the
 * launch counts of Sec. 6.1); at most cap levels, *nlevels receives the count. */
pes_status pes_jobc_add_levels(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                               int64_t* levels, int32_t cap, int32_t* nlevels);

/* Series summed by the addition stage: output 0 is the value, output 1+i the
 * partial derivative d p / d x_i; its terms are the slots
 * add_src[add_ptr[o] .. add_ptr[o+1]) of the data array (a coefficient slot a_m
 * for a monomial of one variable, else a forward, backward or cross product).
 * add_ptr: n+2 entries; at most cap terms are written. */
pes_status pes_jobc_add_terms(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                              int32_t* add_ptr, int32_t* add_src, int64_t cap);
/* The same for monomials with powers; add_mult[t] receives the integer factor
 * of term t (the exponent of the variable for a partial derivative, else 1). */
pes_status pes_jobc_add_terms_powers(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp,
                                     int32_t N, int32_t n, int32_t* add_ptr, int32_t* add_src, int32_t* add_mult,
                                     int64_t cap);
/* The whole program of a plan (host tables, to inspect or interpret them):
 * complex_series 1 for pes_plan_complex; P > 0 with poly_ptr (as in
 * pes_plan_system, poly_ptr[P] == N) for a system; with_vjp 1 to include the
 * VJP tables.
 *   counts[14]: [0] evaluation jobs, [1] addition outputs, [2] addition terms,
 *   [3] slots, [4] VJP jobs (the forward and monomial products, then the
 *   correlations and, for complex series, their add / subtract jobs), [5] VJP
 *   jobs before the correlations, [6] upstream slot, [7] first gradient slot,
 *   [8] first correlation slot (for complex series these three are numbered as
 *   in the real program, the parts living in 2s and 2s + 1), [9] input slots;
 *   systems: [10] first constant slot, [11] first upstream slot, [12] first
 *   Jacobian slot, [13] first slot of the Jacobian correlations (-1 otherwise);
 *   jobs: 5 ints per job (input 1, input 2, output, layer, kind: 0 convolution,
 *   1 correlation, 2 addition, 3 subtraction), the evaluation's jobs then the
 *   VJP's, counts[0] + counts[4] in all; add_ptr (counts[1] + 1), add_src and
 *   add_mult (counts[2]) as pes_jobc_add_terms_powers.
 * NULL arrays are not written (call once with NULL to size them). */
pes_status pes_jobc_program(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp, int32_t N,
                            int32_t n, int32_t complex_series, int32_t P, const int32_t* poly_ptr, int32_t with_vjp,
                            int64_t* counts, int32_t* jobs, int32_t* add_ptr, int32_t* add_src, int32_t* add_mult);
/* The same for a system (pes_plan_system): output p < P is the value of
 * polynomial p, output P + p*n + i the Jacobian entry d p / d x_i; *const0
 * receives the slot of the constant series of polynomial 0 (polynomial p's
 * is const0 + p); the other slots are those of pes_jobc_jobs_powers on the
 * concatenated supports.  add_ptr: P + P*n + 1 entries. */
pes_status pes_jobc_add_terms_system(int32_t P, const int32_t* poly_ptr, const int32_t* supp_ptr,
                                     const int32_t* supp_idx, const int32_t* supp_exp, int32_t n, int32_t* const0,
                                     int32_t* add_ptr, int32_t* add_src, int32_t* add_mult, int64_t cap);

/* Self-test of the failure path: runs the convolution kernel (the whole-series
 * kernel, then the tiled kernel) on one job that waits for a completion flag
 * nobody sets, with the given bound (ms).  Returns
 * PES_OK when the kernel gave up on its own and reported PES_ETIMEOUT through
 * the status word (written to *device_status), leaving the context usable. */
pes_status pes_selftest_timeout(int64_t timeout_ms, int32_t* device_status);

/* ---- evaluation without device allocation ------------------------------------ */

/* Same result as pes_plan + pes_eval_grad, for callers that cannot call
 * cudaMalloc (code running inside another framework's memory pool, plug-ins
 * whose host forbids device allocations, paths that must keep the device
 * footprint fixed after start-up).  It allocates nothing on the device: the
 * job tables, completion flags, control word and workspace of forward,
 * backward and cross products live in one file-scope static device array of
 * 64 MiB that is part of this library, so every GPU that loads the library
 * holds those 64 MiB until the process exits.  The paper has no counterpart.
 *
 * Arguments as pes_plan (supports of monomials with exponents one, N, n, d, k)
 * and pes_eval_grad (caller-owned device buffers coeff, input, value, grad;
 * asynchronous on `stream`); the outputs are bit for bit those of pes_plan +
 * pes_eval_grad.  The job tables are compiled on the host at every call and
 * copied into the array with cudaMemcpyAsync; nothing calls cudaMalloc,
 * cudaFree or an allocating library routine.  Limits, each rejected with
 * PES_EUNSUPPORTED_SIZE (message in pes_last_error):
 *   - d <= 1023, and the whole operand series of a job must fit one CTA's
 *     shared memory (there is no tiled kernel here): d <= 471 at k=10, 543 at
 *     k=8, 839 at k=5, 991 at k=4;
 *   - tables and workspace within the 64 MiB: at d=152, k=10 a series takes
 *     18,560 bytes of workspace (160 rows of 29 words), so about 3,600 series
 *     fit; the workspace holds 3 n_m - 2 series per monomial of n_m >= 2
 *     variables, a_0 and the n inputs.
 * Negative d or a NULL buffer is PES_EINVAL, k outside the set
 * PES_EUNSUPPORTED_K.
 *
 * The first call on a device takes the array's device address with
 * cudaGetSymbolAddress (with that device current), and so does the first call
 * in any other CUDA context of the device (a context the caller made current,
 * or the new primary context after cudaDeviceReset); make that first call
 * before any stream capture.  Every call reuses the same array and rewrites
 * its tables, flags and control word, so calls that overlap on the GPU (on
 * different streams or threads) race and give wrong results; serialise them.
 * status_out: NULL, or a host int32 that receives the device status (0, or
 * PES_ETIMEOUT if a bounded wait gave up) after the call synchronises the
 * stream. */
pes_status pes_eval_grad_static(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n, int32_t d,
                                int32_t k, const double* coeff, const double* input, double* value, double* grad,
                                void* stream, int32_t* status_out);

/* Human-readable name of a status code; never NULL. */
const char* pes_status_string(pes_status s);
/* Message of the last PES_EINVAL / PES_ECUDA on this thread ("" if none). */
const char* pes_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PES_H */
