/*
 * pes_oracle.c -- the ORACLE: a plain, slow CPU evaluator used only as test
 * infrastructure (tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs).  It is not part of the product path and shares no code with
 * the CUDA library.
 *
 * What it computes (Verschelde, "Accelerated Polynomial Evaluation and
 * Differentiation at Power Series in Multiple Double Precision", 2021):
 *
 *   * multiple double numbers are unevaluated sums of k doubles (Sec. 1,
 *     "Contributions"; k = 1,2,3,4,5,8,10);
 *   * the product of two series truncated at degree d is the convolution of
 *     Eq. (eqconvform), z_j = sum_{i=0..j} x_i y_{j-i};
 *   * the polynomial of Eq. (eqpolynomial), p = a_0 + sum_k a_k x_{i_1}...x_{i_{n_k}},
 *     is evaluated at the series z together with all n partial derivatives
 *     (Sec. 4 and the problem statement of Sec. 5).
 *
 * Arithmetic route (deliberately different from the CUDA path):
 *   - TwoSum (Knuth) and TwoProduct by Veltkamp/Dekker splitting, NO fused
 *     multiply-add (build with -ffp-contract=off);
 *   - exact sums are kept as nonoverlapping floating-point expansions grown one
 *     double at a time (Shewchuk's Grow-Expansion with zero elimination) and
 *     compressed (Shewchuk's Compress);
 *   - a result is rounded to k limbs by repeatedly taking the largest component
 *     of the compressed remainder (faithful rounding per limb).
 *
 * Every convolution coefficient is the exact sum of all k*k limb products of all
 * j+1 terms, rounded once to k limbs.  Value and gradient series are exact sums of
 * the rounded monomial contributions, rounded once.  Monomial products are formed
 * naively, left to right, a_k * z_{i_1} * z_{i_2} * ..., and every partial
 * derivative is its own product of a_k with all the other variables: there is no
 * reverse mode here (Sec. 3 is what the CUDA path implements).
 *
 * Layout of every series array: limb-major, [k][series][d+1] doubles, the same
 * layout the C-ABI of the library uses.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXK 10

/* ------------------------------------------------------------------------- */
/* error-free transformations without FMA                                     */
/* ------------------------------------------------------------------------- */

/* Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b). */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

/* Veltkamp splitting of a double into two halves of at most 26 bits each. */
static void split(double a, double *hi, double *lo)
{
    double c = 134217729.0 * a; /* 2^27 + 1 */
    double big = c - a;
    *hi = c - big;
    *lo = a - *hi;
}

/* Dekker's TwoProduct: p + e == a * b exactly, p = fl(a * b). */
static void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    double ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    double err1 = x - ah * bh;
    double err2 = err1 - al * bh;
    double err3 = err2 - ah * bl;
    *p = x;
    *e = al * bl - err3;
}

/* ------------------------------------------------------------------------- */
/* exact floating-point expansions                                            */
/* ------------------------------------------------------------------------- */

typedef struct {
    double *c; /* components, nonoverlapping, increasing magnitude, no zeros */
    int m;     /* number of components (0 means the value 0) */
    int cap;
} expn;

static int expn_init(expn *e, int cap)
{
    e->c = (double *)malloc(sizeof(double) * (size_t)cap);
    e->m = 0;
    e->cap = cap;
    return e->c != NULL;
}

static void expn_free(expn *e)
{
    free(e->c);
    e->c = NULL;
    e->m = e->cap = 0;
}

static void compress(expn *e);

/* Grow-Expansion with zero elimination: e := e + b, exactly. */
static void grow(expn *e, double b)
{
    if (b == 0.0)
        return;
    if (e->m + 2 > e->cap)
        compress(e);
    if (e->m + 2 > e->cap) {
        int ncap = e->cap * 2;
        double *nc = (double *)realloc(e->c, sizeof(double) * (size_t)ncap);
        if (!nc)
            abort();
        e->c = nc;
        e->cap = ncap;
    }
    double q = b;
    int out = 0;
    for (int i = 0; i < e->m; ++i) {
        double h;
        two_sum(q, e->c[i], &q, &h);
        if (h != 0.0)
            e->c[out++] = h;
    }
    if (q != 0.0)
        e->c[out++] = q;
    e->m = out;
}

/* Shewchuk's Compress: same value, fewer and larger components, still
 * nonoverlapping with increasing magnitude. */
static void compress(expn *e)
{
    int m = e->m;
    if (m <= 1)
        return;
    double *g = e->c;
    double q = g[m - 1];
    int bottom = m - 1;
    for (int i = m - 2; i >= 0; --i) {
        double qn = q + g[i]; /* Fast-Two-Sum(q, g[i]), |q| >= |g[i]| */
        double qq = g[i] - (qn - q);
        if (qq != 0.0) {
            g[bottom--] = qn;
            q = qq;
        } else {
            q = qn;
        }
    }
    g[bottom] = q;
    int top = 0;
    for (int i = bottom + 1; i < m; ++i) {
        double qn = g[i] + q; /* Fast-Two-Sum(g[i], q), |g[i]| >= |q| */
        double qq = q - (qn - g[i]);
        if (qq != 0.0)
            g[top++] = qq;
        q = qn;
    }
    if (q != 0.0)
        g[top++] = q;
    e->m = top;
}

/* Round an expansion to k limbs: limb l is the largest component of the
 * compressed remainder, which is then removed exactly. */
static void round_k(expn *e, int k, double *out, size_t stride)
{
    compress(e);
    for (int l = 0; l < k; ++l) {
        if (e->m == 0) {
            out[(size_t)l * stride] = 0.0;
            continue;
        }
        out[(size_t)l * stride] = e->c[e->m - 1];
        e->m -= 1;
        compress(e);
    }
}

/* e += x * y exactly, x and y given as k limbs with the given strides. */
static void add_product(expn *e, int k, const double *x, size_t sx, const double *y, size_t sy)
{
    for (int p = 0; p < k; ++p) {
        double xp = x[(size_t)p * sx];
        if (xp == 0.0)
            continue;
        for (int q = 0; q < k; ++q) {
            double yq = y[(size_t)q * sy];
            if (yq == 0.0)
                continue;
            double ph, pl;
            two_prod(xp, yq, &ph, &pl);
            grow(e, pl);
            grow(e, ph);
        }
    }
}

static void add_value(expn *e, int k, const double *x, size_t sx)
{
    for (int p = k - 1; p >= 0; --p)
        grow(e, x[(size_t)p * sx]);
}

/* ------------------------------------------------------------------------- */
/* scalar multiple-double operations (k limbs, contiguous)                    */
/* ------------------------------------------------------------------------- */

static int valid_k(int k)
{
    return k == 1 || k == 2 || k == 3 || k == 4 || k == 5 || k == 8 || k == 10;
}

/* out = round_k(x + y) */
int orc_md_add(int k, const double *x, const double *y, double *out)
{
    if (!valid_k(k))
        return 1;
    expn e;
    if (!expn_init(&e, 64))
        return 3;
    add_value(&e, k, x, 1);
    add_value(&e, k, y, 1);
    round_k(&e, k, out, 1);
    expn_free(&e);
    return 0;
}

/* out = round_k(x * y) */
int orc_md_mul(int k, const double *x, const double *y, double *out)
{
    if (!valid_k(k))
        return 1;
    expn e;
    if (!expn_init(&e, 4 * k * k + 16))
        return 3;
    add_product(&e, k, x, 1, y, 1);
    round_k(&e, k, out, 1);
    expn_free(&e);
    return 0;
}

/* round_k of an arbitrary list of n doubles (used by tests to pin round_k). */
int orc_round_sum(int k, int n, const double *v, double *out)
{
    if (!valid_k(k) || n < 0)
        return 1;
    expn e;
    if (!expn_init(&e, n + 16))
        return 3;
    for (int i = 0; i < n; ++i)
        grow(&e, v[i]);
    round_k(&e, k, out, 1);
    expn_free(&e);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* series: a series is d+1 coefficients, each of k limbs; "limb stride" is the  */
/* distance between limb l and limb l+1 of the same coefficient.              */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *p; /* coefficient 0, limb 0 */
    size_t ls;       /* limb stride */
} cser;

typedef struct {
    double *p;
    size_t ls;
} ser;

/* z = x * y truncated at degree d (Eq. eqconvform), each coefficient the exact sum
 * of its j+1 terms rounded once to k limbs.  z may not alias x or y. */
static void conv(int k, int d, cser x, cser y, ser z, expn *e)
{
    for (int j = 0; j <= d; ++j) {
        e->m = 0;
        for (int i = 0; i <= j; ++i)
            add_product(e, k, x.p + i, x.ls, y.p + (j - i), y.ls);
        round_k(e, k, z.p + j, z.ls);
    }
}

/* r_j = sum_{l=j..d} u_l * s_{l-j} (truncated correlation), rounded once. */
static void corr(int k, int d, cser u, cser s, ser r, expn *e)
{
    for (int j = 0; j <= d; ++j) {
        e->m = 0;
        for (int l = j; l <= d; ++l)
            add_product(e, k, u.p + l, u.ls, s.p + (l - j), s.ls);
        round_k(e, k, r.p + j, r.ls);
    }
}

int orc_conv(int k, int d, const double *x, const double *y, double *z)
{
    if (!valid_k(k) || d < 0)
        return 1;
    size_t S = (size_t)d + 1;
    expn e;
    if (!expn_init(&e, 4 * k * k + 64))
        return 3;
    cser cx = {x, S}, cy = {y, S};
    ser sz = {z, S};
    conv(k, d, cx, cy, sz, &e);
    expn_free(&e);
    return 0;
}

int orc_corr(int k, int d, const double *u, const double *s, double *r)
{
    if (!valid_k(k) || d < 0)
        return 1;
    size_t S = (size_t)d + 1;
    expn e;
    if (!expn_init(&e, 4 * k * k + 64))
        return 3;
    cser cu = {u, S}, cs = {s, S};
    ser sr = {r, S};
    corr(k, d, cu, cs, sr, &e);
    expn_free(&e);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* polynomial evaluation and differentiation, naive                           */
/* ------------------------------------------------------------------------- */

static int check_supports(int N, int n, const int32_t *ptr, const int32_t *idx)
{
    if (N < 0 || n <= 0 || ptr[0] != 0)
        return 1;
    for (int m = 0; m < N; ++m) {
        if (ptr[m + 1] <= ptr[m])
            return 1;
        for (int t = ptr[m]; t < ptr[m + 1]; ++t) {
            if (idx[t] < 0 || idx[t] >= n)
                return 1;
            if (t > ptr[m] && idx[t] <= idx[t - 1])
                return 1;
        }
    }
    return 0;
}

/* Exponents: NULL means every variable has exponent 1; else one positive
 * exponent per support entry, at most ORC_MAX_EXP. */
#define ORC_MAX_EXP 64
static int check_exponents(int N, const int32_t *ptr, const int32_t *ex)
{
    if (!ex)
        return 0;
    for (int t = 0; t < (N > 0 ? ptr[N] : 0); ++t)
        if (ex[t] < 1 || ex[t] > ORC_MAX_EXP)
            return 1;
    return 0;
}

/* Product of a start series with the input series of the variables of
 * monomial m, every variable repeated as often as its exponent (ex NULL: once),
 * variable `skip` once fewer (skip < 0: none), left to right.  The start series
 * is the coefficient a_m when m >= 1, else the constant series 1.  Result in
 * out (limb stride S).  t0/t1 are scratch series of k*S doubles. */
static void monomial_product(int k, int d, size_t S, const double *coeff, size_t cstride,
                             const double *input, size_t istride, const int32_t *vars,
                             const int32_t *ex, int nv, int m, int skip, double *out, double *t0,
                             double *t1, expn *e)
{
    double *cur = t0, *nxt = t1;
    if (m >= 1) {
        for (int l = 0; l < k; ++l)
            memcpy(cur + (size_t)l * S, coeff + (size_t)l * cstride + (size_t)m * S, sizeof(double) * S);
    } else {
        memset(cur, 0, sizeof(double) * (size_t)k * S);
        cur[0] = 1.0;
    }
    for (int v = 0; v < nv; ++v) {
        int reps = (ex ? ex[v] : 1) - (vars[v] == skip ? 1 : 0);
        for (int r = 0; r < reps; ++r) {
            cser a = {cur, S};
            cser b = {input + (size_t)vars[v] * S, istride};
            ser c = {nxt, S};
            conv(k, d, a, b, c, e);
            double *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
    }
    for (int l = 0; l < k; ++l)
        memcpy(out + (size_t)l * S, cur + (size_t)l * S, sizeof(double) * S);
}

static int used_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/*
 * value[k][d+1] = a_0 + sum_m a_m prod_{i in S_m} z_i^{e_i}
 * grad[k][n][d+1]: grad_i = sum_{m : i in S_m} e_i a_m z_i^{e_i - 1} prod_{j in S_m, j != i} z_j^{e_j}
 * (Eq. eqpolynomial; exponents e from supp_exp, all 1 when supp_exp is NULL;
 * every power is repeated multiplication, the factor e_i is e_i additions).
 * coeff: [k][N+1][d+1] (index 0 is a_0), input: [k][n][d+1].
 * supp_ptr: N+1 row pointers, supp_idx: 0-based variable ids, increasing per row.
 * grad may be NULL (value only).  nthreads <= 0 uses the OpenMP default.
 * Returns 0 on success, 1 on invalid arguments, 3 on allocation failure.
 */
int orc_eval_grad_pow(int k, int d, int N, int n, const int32_t *supp_ptr, const int32_t *supp_idx,
                      const int32_t *supp_exp, const double *coeff, const double *input, double *value,
                      double *grad, int nthreads)
{
    if (!valid_k(k) || d < 0 || check_supports(N, n, supp_ptr, supp_idx) ||
        check_exponents(N, supp_ptr, supp_exp))
        return 1;
    const size_t S = (size_t)d + 1;
    const size_t cstride = (size_t)(N + 1) * S; /* limb stride of coeff */
    const size_t istride = (size_t)n * S;       /* limb stride of input */
    int nth = used_threads(nthreads);
    int fail = 0;

    /* ---- value: exact accumulation over monomials, one expansion per coefficient ---- */
    expn *acc = (expn *)calloc(S, sizeof(expn));
    if (!acc)
        return 3;
    for (size_t j = 0; j < S; ++j)
        if (!expn_init(&acc[j], 64))
            fail = 1;
    for (size_t j = 0; j < S && !fail; ++j)
        add_value(&acc[j], k, coeff + j, cstride); /* a_0 */

#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
    {
        double *prod = (double *)malloc(sizeof(double) * (size_t)k * S * 3);
        expn e;
        expn *part = (expn *)calloc(S, sizeof(expn));
        int ok = prod && part && expn_init(&e, 4 * k * k + 64);
        for (size_t j = 0; ok && j < S; ++j)
            ok = expn_init(&part[j], 64);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int m = 0; m < N; ++m) {
            if (!ok)
                continue;
            const int32_t *vars = supp_idx + supp_ptr[m];
            const int32_t *ex = supp_exp ? supp_exp + supp_ptr[m] : NULL;
            int nv = supp_ptr[m + 1] - supp_ptr[m];
            monomial_product(k, d, S, coeff, cstride, input, istride, vars, ex, nv, m + 1, -1, prod,
                             prod + (size_t)k * S, prod + 2 * (size_t)k * S, &e);
            for (size_t j = 0; j < S; ++j)
                add_value(&part[j], k, prod + j, S);
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (!ok)
                fail = 1;
            for (size_t j = 0; ok && j < S; ++j)
                for (int c = 0; c < part[j].m; ++c)
                    grow(&acc[j], part[j].c[c]);
        }
        if (part)
            for (size_t j = 0; j < S; ++j)
                expn_free(&part[j]);
        free(part);
        free(prod);
        if (ok)
            expn_free(&e);
    }
    for (size_t j = 0; j < S; ++j) {
        if (!fail)
            round_k(&acc[j], k, value + j, S);
        expn_free(&acc[j]);
    }
    free(acc);
    if (fail)
        return 3;
    if (!grad)
        return 0;

    /* ---- gradient: one variable at a time, every partial formed afresh ---- */
#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
    {
        double *prod = (double *)malloc(sizeof(double) * (size_t)k * S * 3);
        expn e;
        expn *g = (expn *)calloc(S, sizeof(expn));
        int ok = prod && g && expn_init(&e, 4 * k * k + 64);
        for (size_t j = 0; ok && j < S; ++j)
            ok = expn_init(&g[j], 64);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int i = 0; i < n; ++i) {
            if (!ok)
                continue;
            for (size_t j = 0; j < S; ++j)
                g[j].m = 0;
            for (int m = 0; m < N; ++m) {
                const int32_t *vars = supp_idx + supp_ptr[m];
                const int32_t *ex = supp_exp ? supp_exp + supp_ptr[m] : NULL;
                int nv = supp_ptr[m + 1] - supp_ptr[m];
                int mult = 0; /* exponent of x_i in monomial m (0: absent) */
                for (int v = 0; v < nv; ++v)
                    if (vars[v] == i)
                        mult = ex ? ex[v] : 1;
                if (!mult)
                    continue;
                monomial_product(k, d, S, coeff, cstride, input, istride, vars, ex, nv, m + 1, i,
                                 prod, prod + (size_t)k * S, prod + 2 * (size_t)k * S, &e);
                for (int r = 0; r < mult; ++r) /* the factor e_i, added exactly */
                    for (size_t j = 0; j < S; ++j)
                        add_value(&g[j], k, prod + j, S);
            }
            for (size_t j = 0; j < S; ++j)
                round_k(&g[j], k, grad + (size_t)i * S + j, istride);
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (!ok)
                fail = 1;
        }
        if (g)
            for (size_t j = 0; j < S; ++j)
                expn_free(&g[j]);
        free(g);
        free(prod);
        if (ok)
            expn_free(&e);
    }
    return fail ? 3 : 0;
}

int orc_eval_grad(int k, int d, int N, int n, const int32_t *supp_ptr, const int32_t *supp_idx,
                  const double *coeff, const double *input, double *value, double *grad,
                  int nthreads)
{
    return orc_eval_grad_pow(k, d, N, n, supp_ptr, supp_idx, NULL, coeff, input, value, grad, nthreads);
}

/*
 * Vector-Jacobian product of the value series with an upstream series u (d+1
 * coefficients of k limbs, [k][d+1]):
 *   L = sum_l u_l v_l,   v = a_0 + sum_m a_m M_m,   M_m = prod_{i in S_m} z_i^{e_i}.
 * v is linear in every coefficient series, and the derivative of L along the
 * coefficients of an input series z_i is the correlation of u with the
 * partial derivative g_i (the chain rule for the truncated product), so
 *   dL/da_0[j] = u_j,
 *   dL/da_m[j] = sum_{l=j..d} u_l M_m[l-j],
 *   dL/dz_i[j] = sum_{l=j..d} u_l g_i[l-j],   g_i = dp/dx_i (z).
 * grad_coeff: [k][N+1][d+1]; grad_input: [k][n][d+1].  supp_exp as in
 * orc_eval_grad_pow.
 */
int orc_vjp_pow(int k, int d, int N, int n, const int32_t *supp_ptr, const int32_t *supp_idx,
                const int32_t *supp_exp, const double *coeff, const double *input, const double *upstream,
                double *grad_input, double *grad_coeff, int nthreads)
{
    if (!valid_k(k) || d < 0 || check_supports(N, n, supp_ptr, supp_idx) ||
        check_exponents(N, supp_ptr, supp_exp))
        return 1;
    const size_t S = (size_t)d + 1;
    const size_t cstride = (size_t)(N + 1) * S;
    const size_t istride = (size_t)n * S;
    int nth = used_threads(nthreads);
    double *value = (double *)malloc(sizeof(double) * (size_t)k * S);
    double *g = (double *)malloc(sizeof(double) * (size_t)k * istride);
    if (!value || !g) {
        free(value);
        free(g);
        return 3;
    }
    int rc = orc_eval_grad_pow(k, d, N, n, supp_ptr, supp_idx, supp_exp, coeff, input, value, g, nthreads);
    int fail = rc != 0;
    if (!fail) {
        for (int l = 0; l < k; ++l) /* dL/da_0 = u */
            memcpy(grad_coeff + (size_t)l * cstride, upstream + (size_t)l * S, sizeof(double) * S);
#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
        {
            double *prod = (double *)malloc(sizeof(double) * (size_t)k * S * 3);
            expn e;
            int ok = prod && expn_init(&e, 4 * k * k + 64);
            cser cu = {upstream, S};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int t = 0; t < N + n; ++t) {
                if (!ok)
                    continue;
                if (t < N) {
                    int m = t;
                    const int32_t *vars = supp_idx + supp_ptr[m];
                    const int32_t *ex = supp_exp ? supp_exp + supp_ptr[m] : NULL;
                    int nv = supp_ptr[m + 1] - supp_ptr[m];
                    /* M_m: the monomial without its coefficient, left to right from 1 */
                    monomial_product(k, d, S, coeff, cstride, input, istride, vars, ex, nv, 0, -1, prod,
                                     prod + (size_t)k * S, prod + 2 * (size_t)k * S, &e);
                    cser cm = {prod, S};
                    ser r = {grad_coeff + (size_t)(m + 1) * S, cstride};
                    corr(k, d, cu, cm, r, &e);
                } else {
                    int i = t - N;
                    cser cg = {g + (size_t)i * S, istride};
                    ser r = {grad_input + (size_t)i * S, istride};
                    corr(k, d, cu, cg, r, &e);
                }
            }
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (!ok)
                    fail = 1;
            }
            free(prod);
            if (ok)
                expn_free(&e);
        }
    }
    free(value);
    free(g);
    return fail ? (rc ? rc : 3) : 0;
}

int orc_vjp(int k, int d, int N, int n, const int32_t *supp_ptr, const int32_t *supp_idx,
            const double *coeff, const double *input, const double *upstream,
            double *grad_input, double *grad_coeff, int nthreads)
{
    return orc_vjp_pow(k, d, N, n, supp_ptr, supp_idx, NULL, coeff, input, upstream, grad_input, grad_coeff,
                       nthreads);
}

/* ------------------------------------------------------------------------- */
/* complex series (Re and Im each a k-double series)                          */
/* ------------------------------------------------------------------------- */

/* e -= x * y exactly (negating a double is exact) */
static void sub_product(expn *e, int k, const double *x, size_t sx, const double *y, size_t sy)
{
    for (int p = 0; p < k; ++p) {
        double xp = -x[(size_t)p * sx];
        if (xp == 0.0)
            continue;
        for (int q = 0; q < k; ++q) {
            double yq = y[(size_t)q * sy];
            if (yq == 0.0)
                continue;
            double ph, pl;
            two_prod(xp, yq, &ph, &pl);
            grow(e, pl);
            grow(e, ph);
        }
    }
}

/* A complex series: real and imaginary part, same limb stride. */
typedef struct {
    const double *re, *im;
    size_t ls;
} ccser;

typedef struct {
    double *re, *im;
    size_t ls;
} cpser;

/* z = x * y truncated at degree d, complex: coefficient j of Re z is the exact
 * sum of xr_i yr_{j-i} - xi_i yi_{j-i}, of Im z the exact sum of
 * xr_i yi_{j-i} + xi_i yr_{j-i}, each rounded once to k limbs. */
static void cconv(int k, int d, ccser x, ccser y, cpser z, expn *e)
{
    for (int j = 0; j <= d; ++j) {
        e->m = 0;
        for (int i = 0; i <= j; ++i) {
            add_product(e, k, x.re + i, x.ls, y.re + (j - i), y.ls);
            sub_product(e, k, x.im + i, x.ls, y.im + (j - i), y.ls);
        }
        round_k(e, k, z.re + j, z.ls);
        e->m = 0;
        for (int i = 0; i <= j; ++i) {
            add_product(e, k, x.re + i, x.ls, y.im + (j - i), y.ls);
            add_product(e, k, x.im + i, x.ls, y.re + (j - i), y.ls);
        }
        round_k(e, k, z.im + j, z.ls);
    }
}

/* Complex analogue of monomial_product: the start series (a_m, or 1 when
 * m < 1) times every variable's series as often as its exponent, `skip` once
 * fewer.  Real and imaginary parts of coeff and input are separate blocks
 * (cimag / iimag doubles after the real ones).  out: 2 k S doubles (Re, Im). */
static void cmonomial_product(int k, int d, size_t S, const double *coeff, size_t cstride, size_t cimag,
                              const double *input, size_t istride, size_t iimag, const int32_t *vars,
                              const int32_t *ex, int nv, int m, int skip, double *out, double *t0, double *t1,
                              expn *e)
{
    const size_t blk = (size_t)k * S;
    double *cur = t0, *nxt = t1; /* each: Re block then Im block, limb stride S */
    if (m >= 1) {
        for (int l = 0; l < k; ++l) {
            memcpy(cur + (size_t)l * S, coeff + (size_t)l * cstride + (size_t)m * S, sizeof(double) * S);
            memcpy(cur + blk + (size_t)l * S, coeff + cimag + (size_t)l * cstride + (size_t)m * S,
                   sizeof(double) * S);
        }
    } else {
        memset(cur, 0, sizeof(double) * 2 * blk);
        cur[0] = 1.0;
    }
    for (int v = 0; v < nv; ++v) {
        int reps = (ex ? ex[v] : 1) - (vars[v] == skip ? 1 : 0);
        for (int r = 0; r < reps; ++r) {
            ccser a = {cur, cur + blk, S};
            ccser b = {input + (size_t)vars[v] * S, input + iimag + (size_t)vars[v] * S, istride};
            cpser c = {nxt, nxt + blk, S};
            cconv(k, d, a, b, c, e);
            double *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
    }
    memcpy(out, cur, sizeof(double) * 2 * blk);
}

/*
 * Complex coefficients and inputs (the polynomial of orc_eval_grad_pow over
 * complex series): coeff [2][k][N+1][d+1], input [2][k][n][d+1], value
 * [2][k][d+1], grad [2][k][n][d+1], each the real block followed by the
 * imaginary block.  Every complex product is formed exactly per component and
 * rounded once; sums are exact per component, rounded once.  supp_exp may be
 * NULL.  grad may be NULL.
 */
int orc_eval_grad_complex(int k, int d, int N, int n, const int32_t *supp_ptr, const int32_t *supp_idx,
                          const int32_t *supp_exp, const double *coeff, const double *input, double *value,
                          double *grad)
{
    if (!valid_k(k) || d < 0 || check_supports(N, n, supp_ptr, supp_idx) ||
        check_exponents(N, supp_ptr, supp_exp))
        return 1;
    const size_t S = (size_t)d + 1;
    const size_t cstride = (size_t)(N + 1) * S, cimag = (size_t)k * cstride;
    const size_t istride = (size_t)n * S, iimag = (size_t)k * istride;
    const size_t blk = (size_t)k * S;
    int fail = 0;
    double *prod = (double *)malloc(sizeof(double) * 6 * blk);
    expn e;
    expn *acc = (expn *)calloc(2 * S, sizeof(expn));
    if (!prod || !acc || !expn_init(&e, 8 * k * k + 64)) {
        free(prod);
        free(acc);
        return 3;
    }
    for (size_t j = 0; j < 2 * S; ++j)
        if (!expn_init(&acc[j], 64))
            fail = 1;
    /* value: a_0 plus every monomial */
    for (size_t j = 0; j < S && !fail; ++j) {
        add_value(&acc[j], k, coeff + j, cstride);
        add_value(&acc[S + j], k, coeff + cimag + j, cstride);
    }
    for (int m = 0; m < N && !fail; ++m) {
        const int32_t *vars = supp_idx + supp_ptr[m];
        const int32_t *ex = supp_exp ? supp_exp + supp_ptr[m] : NULL;
        int nv = supp_ptr[m + 1] - supp_ptr[m];
        cmonomial_product(k, d, S, coeff, cstride, cimag, input, istride, iimag, vars, ex, nv, m + 1, -1, prod,
                          prod + 2 * blk, prod + 4 * blk, &e);
        for (size_t j = 0; j < S; ++j) {
            add_value(&acc[j], k, prod + j, S);
            add_value(&acc[S + j], k, prod + blk + j, S);
        }
    }
    for (size_t j = 0; j < S && !fail; ++j) {
        round_k(&acc[j], k, value + j, S);
        round_k(&acc[S + j], k, value + blk + j, S);
    }
    /* gradient: every partial afresh, added e_i times */
    for (int i = 0; i < n && grad && !fail; ++i) {
        for (size_t j = 0; j < 2 * S; ++j)
            acc[j].m = 0;
        for (int m = 0; m < N; ++m) {
            const int32_t *vars = supp_idx + supp_ptr[m];
            const int32_t *ex = supp_exp ? supp_exp + supp_ptr[m] : NULL;
            int nv = supp_ptr[m + 1] - supp_ptr[m];
            int mult = 0;
            for (int v = 0; v < nv; ++v)
                if (vars[v] == i)
                    mult = ex ? ex[v] : 1;
            if (!mult)
                continue;
            cmonomial_product(k, d, S, coeff, cstride, cimag, input, istride, iimag, vars, ex, nv, m + 1, i,
                              prod, prod + 2 * blk, prod + 4 * blk, &e);
            for (int r = 0; r < mult; ++r)
                for (size_t j = 0; j < S; ++j) {
                    add_value(&acc[j], k, prod + j, S);
                    add_value(&acc[S + j], k, prod + blk + j, S);
                }
        }
        for (size_t j = 0; j < S; ++j) {
            round_k(&acc[j], k, grad + (size_t)i * S + j, istride);
            round_k(&acc[S + j], k, grad + iimag + (size_t)i * S + j, istride);
        }
    }
    for (size_t j = 0; j < 2 * S; ++j)
        expn_free(&acc[j]);
    free(acc);
    free(prod);
    expn_free(&e);
    return fail ? 3 : 0;
}

/* r = correlation of u with the conjugate of s, truncated at degree d: for L =
 * sum_l (Re u_l Re v_l + Im u_l Im v_l) and v_l = sum_{j<=l} s_{l-j} w_j, the
 * derivatives of L with respect to Re w_j and Im w_j are the real and
 * imaginary parts of sum_{l>=j} u_l conj(s_{l-j}):
 *   Re r_j = sum_{l>=j} Re u_l Re s_{l-j} + Im u_l Im s_{l-j},
 *   Im r_j = sum_{l>=j} Im u_l Re s_{l-j} - Re u_l Im s_{l-j},
 * each an exact sum rounded once to k limbs. */
static void ccorr_conj(int k, int d, ccser u, ccser s, cpser r, expn *e)
{
    for (int j = 0; j <= d; ++j) {
        e->m = 0;
        for (int l = j; l <= d; ++l) {
            add_product(e, k, u.re + l, u.ls, s.re + (l - j), s.ls);
            add_product(e, k, u.im + l, u.ls, s.im + (l - j), s.ls);
        }
        round_k(e, k, r.re + j, r.ls);
        e->m = 0;
        for (int l = j; l <= d; ++l) {
            add_product(e, k, u.im + l, u.ls, s.re + (l - j), s.ls);
            sub_product(e, k, u.re + l, u.ls, s.im + (l - j), s.ls);
        }
        round_k(e, k, r.im + j, r.ls);
    }
}

/*
 * Vector-Jacobian product over complex series, with the real and imaginary
 * parts of every series as separate real variables: for the real loss
 * L = sum_j (Re u_j Re v_j + Im u_j Im v_j) (v the value series of
 * orc_eval_grad_complex), grad_coeff and grad_input hold dL/dRe and dL/dIm of
 * every coefficient series and input series as the real and imaginary block:
 *   grad_coeff[0] = u,  grad_coeff[m] = corr(u, conj(M_m)),  grad_input[i] = corr(u, conj(g_i)),
 * M_m the product of the variables of monomial m (with their exponents) and
 * g_i = d p / d x_i (the polynomial is holomorphic in every series, so the
 * derivative of v with respect to one series is multiplication by g_i or
 * M_m, and the transpose of multiplication by s is correlation with conj(s)
 * under this inner product).  upstream [2][k][d+1], grad_input [2][k][n][d+1],
 * grad_coeff [2][k][N+1][d+1].
 */
int orc_vjp_complex(int k, int d, int N, int n, const int32_t *supp_ptr, const int32_t *supp_idx,
                    const int32_t *supp_exp, const double *coeff, const double *input, const double *upstream,
                    double *grad_input, double *grad_coeff)
{
    if (!valid_k(k) || d < 0 || check_supports(N, n, supp_ptr, supp_idx) ||
        check_exponents(N, supp_ptr, supp_exp))
        return 1;
    const size_t S = (size_t)d + 1;
    const size_t cstride = (size_t)(N + 1) * S, cimag = (size_t)k * cstride;
    const size_t istride = (size_t)n * S, iimag = (size_t)k * istride;
    const size_t blk = (size_t)k * S;
    double *value = (double *)malloc(sizeof(double) * 2 * blk);
    double *g = (double *)malloc(sizeof(double) * 2 * (size_t)k * istride);
    double *prod = (double *)malloc(sizeof(double) * 6 * blk);
    expn e;
    if (!value || !g || !prod || !expn_init(&e, 8 * k * k + 64)) {
        free(value);
        free(g);
        free(prod);
        return 3;
    }
    int rc = orc_eval_grad_complex(k, d, N, n, supp_ptr, supp_idx, supp_exp, coeff, input, value, g);
    if (rc == 0) {
        ccser cu = {upstream, upstream + blk, S};
        for (int l = 0; l < k; ++l) { /* dL/da_0 = u */
            memcpy(grad_coeff + (size_t)l * cstride, upstream + (size_t)l * S, sizeof(double) * S);
            memcpy(grad_coeff + cimag + (size_t)l * cstride, upstream + blk + (size_t)l * S, sizeof(double) * S);
        }
        for (int m = 0; m < N; ++m) {
            const int32_t *vars = supp_idx + supp_ptr[m];
            const int32_t *ex = supp_exp ? supp_exp + supp_ptr[m] : NULL;
            int nv = supp_ptr[m + 1] - supp_ptr[m];
            /* M_m: the monomial without its coefficient, from 1 */
            cmonomial_product(k, d, S, coeff, cstride, cimag, input, istride, iimag, vars, ex, nv, 0, -1, prod,
                              prod + 2 * blk, prod + 4 * blk, &e);
            ccser cm = {prod, prod + blk, S};
            cpser r = {grad_coeff + (size_t)(m + 1) * S, grad_coeff + cimag + (size_t)(m + 1) * S, cstride};
            ccorr_conj(k, d, cu, cm, r, &e);
        }
        for (int i = 0; i < n; ++i) {
            ccser cg = {g + (size_t)i * S, g + iimag + (size_t)i * S, istride};
            cpser r = {grad_input + (size_t)i * S, grad_input + iimag + (size_t)i * S, istride};
            ccorr_conj(k, d, cu, cg, r, &e);
        }
    }
    free(value);
    free(g);
    free(prod);
    expn_free(&e);
    return rc;
}

/* number of threads the oracle would use for nthreads (for reporting) */
int orc_threads(int nthreads) { return used_threads(nthreads); }

/* count independent truncated products Z[c] = X[c] * Y[c] (Eq. eqconvform),
 * arrays [k][count][d+1]; the pairs are spread over threads. */
int orc_conv_many(int k, int d, int count, const double *X, const double *Y, double *Z, int nthreads)
{
    if (!valid_k(k) || d < 0 || count < 0)
        return 1;
    const size_t S = (size_t)d + 1;
    const size_t ls = (size_t)count * S;
    int fail = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(used_threads(nthreads))
#endif
    {
        expn e;
        int ok = expn_init(&e, 4 * k * k + 64);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int c = 0; c < count; ++c) {
            if (!ok)
                continue;
            cser x = {X + (size_t)c * S, ls}, y = {Y + (size_t)c * S, ls};
            ser z = {Z + (size_t)c * S, ls};
            conv(k, d, x, y, z, &e);
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (!ok)
                fail = 1;
        }
        if (ok)
            expn_free(&e);
    }
    return fail ? 3 : 0;
}
