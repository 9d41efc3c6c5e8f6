/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for successive-
 * cancellation (SC) decoding of polar codes in syndrome form, after
 * Jouguet & Kunz-Jacques, "High performance error correction for quantum key
 * distribution using polar codes" (arXiv 1204.5882).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * library under paper_1204_5882_gb300/csrc.
 *
 * Conventions (the paper gives no formula for the transform, Sec. 3):
 *   - one bit per uint8_t (0/1), index i = position in natural order;
 *   - x = u * F^{(x)n},  F = [[1,0],[1,1]], no bit-reversal permutation;
 *     splitting u = (a, b) in halves gives x = (aG' ^ bG', bG');
 *   - LLR L = ln P(y|x=0)/P(y|x=1); decision on an information leaf:
 *     u = 1 iff L < 0 (so L = +0.0 and L = -0.0 both decide 0).
 *
 * Parity pins (tests/test_oracle_*.py):
 *   encode          -- involution, N=2 closed form, explicit Kronecker product;
 *   f / g           -- N=2 closed form, literal 2*atanh(tanh*tanh);
 *   SC exact f      -- brute-force bit-channel LLR (sum over all future bits);
 *   SC min-sum      -- brute-force max-log bit-channel LLR, bit-exact on
 *                      small-integer LLRs, ties included;
 *   construction    -- BEC brute force of bit-channel erasure probabilities,
 *                      conservation, GA vs numerically integrated phi;
 *   capacity        -- closed forms and independent quadrature.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Arikan transform (Sec. 3: channels combined recursively).                */
/* x = u * F^{(x)n}: for every level the first half of each block of size   */
/* 2h is XORed with its second half.  Applied in place.                     */
/* ------------------------------------------------------------------------ */
OR_API void or_encode(uint8_t *v, int n)
{
    size_t N = (size_t)1 << n;
    for (size_t h = 1; h < N; h <<= 1)
        for (size_t base = 0; base < N; base += 2 * h)
            for (size_t j = 0; j < h; j++)
                v[base + j] ^= v[base + h + j];
}

/* ------------------------------------------------------------------------ */
/* Channel LLRs (Sec. 1 and Sec. 2.2: BSC for DV-QKD, BI-AWGN for CV-QKD).  */
/* BSC: L = (1-2y) * c with c = ln((1-p)/p) computed in double and rounded  */
/* once to float.  BIAWGN: L = y * s with s = 2/sigma^2 in double, the      */
/* product rounded to double and then once to float.  The double versions   */
/* keep the double values.                                                  */
/* ------------------------------------------------------------------------ */
OR_API void or_llr_bsc_f32(const uint8_t *y, size_t n, double p, float *L)
{
    double c = log((1.0 - p) / p);
    float cf = (float)c;
    for (size_t i = 0; i < n; i++) L[i] = y[i] ? -cf : cf;
}

OR_API void or_llr_bsc_f64(const uint8_t *y, size_t n, double p, double *L)
{
    double c = log((1.0 - p) / p);
    for (size_t i = 0; i < n; i++) L[i] = y[i] ? -c : c;
}

OR_API void or_llr_biawgn_f32(const double *y, size_t n, double sigma2, float *L)
{
    double s = 2.0 / sigma2;
    for (size_t i = 0; i < n; i++) L[i] = (float)(y[i] * s);
}

OR_API void or_llr_biawgn_f64(const double *y, size_t n, double sigma2, double *L)
{
    double s = 2.0 / sigma2;
    for (size_t i = 0; i < n; i++) L[i] = y[i] * s;
}

/* ------------------------------------------------------------------------ */
/* Check-node update f (Sec. 4: LLR update through phi).                    */
/* The paper names phi(x) = log(tanh(x/2)); its sign is garbled (that value */
/* is negative for x > 0).  Read as Gallager's phi(x) = -ln tanh(x/2),      */
/* which is its own inverse on (0, inf), so                                 */
/*   f(a, b) = sgn(a) sgn(b) phi(phi(|a|) + phi(|b|))                       */
/*           = 2 atanh(tanh(a/2) tanh(b/2)).                                */
/* With A = |a|, B = |b| the same quantity is also                          */
/*   ln((1 + e^(A+B)) / (e^A + e^B))                                        */
/*     = min(A,B) + ln(1 + e^-(A+B)) - ln(1 + e^-|A-B|)                     */
/* (divide numerator and denominator by e^max(A,B)).  The two forms are     */
/* used where each is accurate:                                             */
/*   - phi form while min(A,B) < F_SPLIT: phi(x) = log1p(2/expm1(x)) keeps  */
/*     full relative precision, so a tiny f (about A*B/2) keeps its value   */
/*     and sign;                                                            */
/*   - min form once min(A,B) >= F_SPLIT: there phi(A) and phi(B) are both  */
/*     below 2e^-F_SPLIT and would underflow to 0 for A, B beyond about 709 */
/*     (double) or 88 (float), turning phi(0) into +inf; the min form is    */
/*     finite everywhere and its result is at least F_SPLIT - ln 2, so its  */
/*     rounding error is a few ulp of the result.                           */
/* Min-sum replaces the magnitude by min(A, B).  The sign of f is taken as  */
/* - iff exactly one of a, b is negative (signbit); a zero magnitude gives  */
/* a zero f, whose sign no decision reads.                                  */
/* ------------------------------------------------------------------------ */
#define F_SPLIT 16.0
static double phi64(double x) { return log1p(2.0 / expm1(x)); }
static float phi32(float x) { return log1pf(2.0f / expm1f(x)); }

OR_API double or_f_exact_f64(double a, double b)
{
    double A = fabs(a), B = fabs(b), m;
    if (fmin(A, B) < F_SPLIT)
        m = phi64(phi64(A) + phi64(B));
    else
        m = fmin(A, B) + log1p(exp(-(A + B))) - log1p(exp(-fabs(A - B)));
    return (signbit(a) != signbit(b)) ? -m : m;
}

OR_API float or_f_exact_f32(float a, float b)
{
    float A = fabsf(a), B = fabsf(b), m;
    if (fminf(A, B) < (float)F_SPLIT)
        m = phi32(phi32(A) + phi32(B));
    else
        m = fminf(A, B) + log1pf(expf(-(A + B))) - log1pf(expf(-fabsf(A - B)));
    return (signbit(a) != signbit(b)) ? -m : m;
}

OR_API double or_f_minsum_f64(double a, double b)
{
    double m = fmin(fabs(a), fabs(b));
    return (signbit(a) != signbit(b)) ? -m : m;
}

OR_API float or_f_minsum_f32(float a, float b)
{
    float m = fminf(fabsf(a), fabsf(b));
    return (signbit(a) != signbit(b)) ? -m : m;
}

/* ------------------------------------------------------------------------ */
/* Recursive SC decoder (Sec. 1: deterministic, O(N log N); Sec. 4:         */
/* recursive).  Syndrome form (Sec. 1): frozen positions take Alice's       */
/* revealed values fval[i] instead of zeros.                                */
/*                                                                          */
/* node(k, L[0..2^k)):                                                      */
/*   k == 0 : u = frozen ? fval : (L < 0);  beta = u                        */
/*   else   : h = 2^(k-1)                                                   */
/*            Lc[j] = f(L[j], L[j+h])                    -> left child      */
/*            Lc[j] = beta_L[j] ? L[j+h]-L[j] : L[j+h]+L[j] -> right child  */
/*            beta  = (beta_L ^ beta_R, beta_R)                             */
/* The root beta is x_hat = u_hat * F^{(x)n}.                               */
/* ------------------------------------------------------------------------ */
#define OR_DEFINE_SC(T, SUF, FEXACT, FMINSUM)                                  \
    static void sc_node_##SUF(int k, const T *L, const uint8_t *frz,           \
                              const uint8_t *fval, uint8_t *u, uint8_t *beta,  \
                              int fkind, T *scratch, T *leaf)                  \
    {                                                                          \
        if (k == 0) {                                                          \
            uint8_t d = frz[0] ? fval[0] : (uint8_t)(L[0] < (T)0);             \
            u[0] = d;                                                          \
            beta[0] = d;                                                       \
            if (leaf) leaf[0] = L[0];                                          \
            return;                                                            \
        }                                                                      \
        size_t h = (size_t)1 << (k - 1);                                       \
        T *Lc = scratch;                                                       \
        for (size_t j = 0; j < h; j++)                                         \
            Lc[j] = fkind ? FEXACT(L[j], L[j + h]) : FMINSUM(L[j], L[j + h]);  \
        sc_node_##SUF(k - 1, Lc, frz, fval, u, beta, fkind, scratch + h,       \
                      leaf);                                                   \
        for (size_t j = 0; j < h; j++)                                         \
            Lc[j] = beta[j] ? (L[j + h] - L[j]) : (L[j + h] + L[j]);           \
        sc_node_##SUF(k - 1, Lc, frz + h, fval + h, u + h, beta + h, fkind,    \
                      scratch + h, leaf ? leaf + h : NULL);                    \
        for (size_t j = 0; j < h; j++) beta[j] ^= beta[j + h];                 \
    }                                                                          \
    OR_API int or_sc_decode_##SUF(int n, int fkind, const T *llr,             \
                                  const uint8_t *frozen, const uint8_t *fval,  \
                                  uint8_t *u_hat, uint8_t *x_hat, T *leaf)     \
    {                                                                          \
        size_t N = (size_t)1 << n;                                             \
        T *scratch = (T *)malloc(sizeof(T) * (N > 1 ? N : 1));                 \
        if (!scratch) return -1;                                               \
        sc_node_##SUF(n, llr, frozen, fval, u_hat, x_hat, fkind, scratch,      \
                      leaf);                                                   \
        free(scratch);                                                         \
        return 0;                                                              \
    }

OR_DEFINE_SC(double, f64, or_f_exact_f64, or_f_minsum_f64)
OR_DEFINE_SC(float, f32, or_f_exact_f32, or_f_minsum_f32)

/* ------------------------------------------------------------------------ */
/* Reduced-precision storage of the LLRs (the paper's fixed-point decoder,  */
/* Sec. 4, leaves the width open).  Reading: the LLRs that are stored in    */
/* bulk memory -- the channel LLRs on entry and every f and g output of the */
/* levels k >= min_level (nodes of 2^k leaves) -- are rounded to the        */
/* storage format; smaller nodes (min_level = the on-chip subtree size) and */
/* all f and g arithmetic stay in float:                                    */
/*   store 1 (half): clamp to +-65504, round to nearest even half;         */
/*   store 2 (int8): values are L * scale (scale a power of two chosen per  */
/*                   frame), rounded to nearest even integer, clamped to    */
/*                   +-127; exact f is evaluated on L = value / scale.      */
/* store 0 is plain float storage (identical to or_sc_decode_f32).          */
/* ------------------------------------------------------------------------ */
static float q_store(float v, int store)
{
    if (store == 1) {
        v = fminf(fmaxf(v, -65504.0f), 65504.0f);
        return (float)(_Float16)v;
    }
    if (store == 2) return fminf(fmaxf(rintf(v), -127.0f), 127.0f);
    return v;
}

static float f_store(float a, float b, int fkind, int store, float scale)
{
    if (!fkind) return q_store(or_f_minsum_f32(a, b), store);
    return q_store(scale * or_f_exact_f32(a / scale, b / scale), store);
}

static void sc_node_q(int k, const float *L, const uint8_t *frz, const uint8_t *fval,
                      uint8_t *u, uint8_t *beta, int fkind, int store, float scale,
                      int min_level, float *scratch, float *leaf)
{
    if (k == 0) {
        uint8_t d = frz[0] ? fval[0] : (uint8_t)(L[0] < 0.0f);
        u[0] = d;
        beta[0] = d;
        if (leaf) leaf[0] = L[0];
        return;
    }
    size_t h = (size_t)1 << (k - 1);
    int st = (k - 1 >= min_level) ? store : 0;   /* the children are stored? */
    float *Lc = scratch;
    for (size_t j = 0; j < h; j++) Lc[j] = f_store(L[j], L[j + h], fkind, st, scale);
    sc_node_q(k - 1, Lc, frz, fval, u, beta, fkind, store, scale, min_level, scratch + h, leaf);
    for (size_t j = 0; j < h; j++)
        Lc[j] = q_store(beta[j] ? (L[j + h] - L[j]) : (L[j + h] + L[j]), st);
    sc_node_q(k - 1, Lc, frz + h, fval + h, u + h, beta + h, fkind, store, scale, min_level,
              scratch + h, leaf ? leaf + h : NULL);
    for (size_t j = 0; j < h; j++) beta[j] ^= beta[j + h];
}

OR_API int or_sc_decode_store(int n, int fkind, int store, float scale, int min_level,
                              const float *llr, const uint8_t *frozen, const uint8_t *fval,
                              uint8_t *u_hat, uint8_t *x_hat, float *leaf)
{
    size_t N = (size_t)1 << n;
    float *buf = (float *)malloc(sizeof(float) * 2 * N);
    if (!buf) return -1;
    for (size_t i = 0; i < N; i++) buf[i] = q_store(store == 2 ? llr[i] * scale : llr[i], store);
    sc_node_q(n, buf, frozen, fval, u_hat, x_hat, fkind, store, scale, min_level, buf + N,
              leaf);
    free(buf);
    return 0;
}

/* Per-frame int8 scale: the power of two s = 2^e, e = round(log2(target /  */
/* mean |L|)), mean taken in double; s = 1 when every L is zero.            */
OR_API float or_int8_scale(const float *llr, size_t n, double target)
{
    double acc = 0.0;
    for (size_t i = 0; i < n; i++) acc += fabs((double)llr[i]);
    if (!(acc > 0.0)) return 1.0f;
    double e = nearbyint(log2(target / (acc / (double)n)));
    if (e > 100) e = 100;
    if (e < -100) e = -100;
    return (float)ldexp(1.0, (int)e);
}

/* ------------------------------------------------------------------------ */
/* Frozen-set construction (Sec. 3: density evolution selects the frozen    */
/* bits as the lowest-capacity bit-channels).  The paper uses the method of */
/* Mori-Tanaka; this oracle implements the two standard substitutes:        */
/*   BSC    -- Bhattacharyya parameters, Z- <= 2Z - Z^2 (upper bound),      */
/*             Z+ = Z^2, Z0 = 2 sqrt(p(1-p));                               */
/*   BIAWGN -- Gaussian approximation of density evolution, m0 = 2/sigma^2, */
/*             m+ = 2m, m- = phiGA^-1(1 - (1 - phiGA(m))^2),                */
/*             P_e = Q(sqrt(m/2)).                                           */
/* Index convention: z'[2j] = minus(z[j]), z'[2j+1] = plus(z[j]), so the    */
/* first polarisation step lands in the most significant index bit, which   */
/* is the top split (u first half / second half) of the natural-order       */
/* decoder above.  Everything is kept in the log domain (ln Z, ln phiGA) so */
/* that nothing underflows at N = 2^24.                                     */
/* ------------------------------------------------------------------------ */

/* ln(2Z - Z^2) = lz + ln(2 - e^lz) = lz + log1p(-expm1(lz)). */
static double bh_minus(double lz) { return lz + log1p(-expm1(lz)); }
static double bh_plus(double lz) { return 2.0 * lz; }

OR_API void or_bhatt_log_from(int n, double lz0, double *out)
{
    size_t N = (size_t)1 << n;
    double *tmp = (double *)malloc(sizeof(double) * N);
    out[0] = lz0;
    for (int s = 0; s < n; s++) {
        size_t len = (size_t)1 << s;
        for (size_t j = 0; j < len; j++) {
            tmp[2 * j] = bh_minus(out[j]);
            tmp[2 * j + 1] = bh_plus(out[j]);
        }
        memcpy(out, tmp, sizeof(double) * 2 * len);
    }
    free(tmp);
}

OR_API void or_bhatt_log_bsc(int n, double p, double *out)
{
    double lz0 = log(2.0) + 0.5 * (log(p) + log1p(-p));
    or_bhatt_log_from(n, lz0, out);
}

/* phi of the Gaussian approximation, in logs: the Chung-Richardson-Urbanke */
/* form (IEEE Trans. IT 47(2), 2001) completed by the small-x piece of Ha,  */
/* Kim and McLaughlin (IEEE Trans. IT 50(11), 2004, rate-compatible        */
/* puncturing of LDPC codes), so that phi(0) = 1 (the two-piece form       */
/* has phi(0) = e^0.0218 > 1, a fixed point of the minus step at m = 0.029, */
/* and then rates the "minus^k plus^j" channels of long codes as reliable): */
/*   x < 0.867      : phi(x) = exp(0.0564 x^2 - 0.48560 x)                  */
/*   0.867 <= x < 10: phi(x) = exp(-0.4527 x^0.86 + 0.0218)                 */
/*   x >= 10        : phi(x) = sqrt(pi/x) exp(-x/4) (1 - 10/(7x))           */
/* The first two pieces meet at 0.867 (to the printed precision).           */
OR_API double or_ga_lnphi(double x)
{
    if (x < 0.867) return 0.0564 * x * x - 0.48560 * x;
    if (x < 10.0) return -0.4527 * pow(x, 0.86) + 0.0218;
    return 0.5 * log(M_PI / x) - 0.25 * x + log1p(-10.0 / (7.0 * x));
}

/* Inverse of ln phiGA.  Each piece is decreasing; at x = 10 the pieces do  */
/* not meet (ln phi jumps up from -3.2576 to -3.2331), so targets inside    */
/* that gap have two preimages.  Reading taken: the lowest piece whose      */
/* range holds t is used -- the quadratic piece (smaller root, in the       */
/* cancellation-free form -2t / (b + sqrt(b^2 + 4at))) when t is above its  */
/* value at 0.867, else the middle piece in closed form when t is above its */
/* limit at 10, else the x >= 10 piece by bisection (bracket doubled until  */
/* it holds the root, then halved until it cannot shrink).                  */
OR_API double or_ga_lnphi_inv(double t)
{
    double q867 = 0.0564 * 0.867 * 0.867 - 0.48560 * 0.867;
    if (t > q867) {
        if (t >= 0.0) return 0.0;
        return -2.0 * t / (0.48560 + sqrt(0.48560 * 0.48560 + 4.0 * 0.0564 * t));
    }
    double left10 = -0.4527 * pow(10.0, 0.86) + 0.0218;
    if (t > left10) {
        double v = (0.0218 - t) / 0.4527;
        return v > 0.0 ? pow(v, 1.0 / 0.86) : 0.0;
    }
    double lo = 10.0, hi = 20.0;
    while (or_ga_lnphi(hi) > t) { lo = hi; hi *= 2.0; }
    for (;;) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (or_ga_lnphi(mid) > t) lo = mid; else hi = mid;
    }
    return hi;
}

/* m- : 1 - phi(m-) = (1 - phi(m))^2  <=>  phi(m-) = phi(m) (2 - phi(m)).  */
static double ga_minus(double m)
{
    double lp = or_ga_lnphi(m);
    double t = lp + log1p(-expm1(lp)); /* ln(phi (2 - phi)) */
    return or_ga_lnphi_inv(t);
}

OR_API void or_ga_mean(int n, double sigma2, double *out)
{
    size_t N = (size_t)1 << n;
    double *tmp = (double *)malloc(sizeof(double) * N);
    out[0] = 2.0 / sigma2;
    for (int s = 0; s < n; s++) {
        size_t len = (size_t)1 << s;
        for (size_t j = 0; j < len; j++) {
            tmp[2 * j] = ga_minus(out[j]);
            tmp[2 * j + 1] = 2.0 * out[j];
        }
        memcpy(out, tmp, sizeof(double) * 2 * len);
    }
    free(tmp);
}

/* ln Q(x) for x >= 0: erfc for moderate x, asymptotic series for large x.   */
OR_API double or_ln_q(double x)
{
    if (x < 30.0) return log(0.5 * erfc(x / M_SQRT2));
    double x2 = x * x;
    double s = 1.0 - 1.0 / x2 + 3.0 / (x2 * x2) - 15.0 / (x2 * x2 * x2);
    return -0.5 * x2 - log(x) - 0.5 * log(2.0 * M_PI) + log(s);
}

/* ln P_e of each bit-channel under the Gaussian approximation. */
OR_API void or_ga_lnpe(int n, double sigma2, double *out)
{
    size_t N = (size_t)1 << n;
    or_ga_mean(n, sigma2, out);
    for (size_t i = 0; i < N; i++) out[i] = or_ln_q(sqrt(out[i] / 2.0));
}

/* Selection: freeze the N-K least reliable bit-channels.  `bad[i]` grows   */
/* with unreliability (ln Z or ln P_e).  Order: bad descending, ties broken */
/* by index ascending (the lower index is frozen first).                    */
static const double *g_bad;
static int cmp_unrel(const void *pa, const void *pb)
{
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    if (g_bad[a] > g_bad[b]) return -1;
    if (g_bad[a] < g_bad[b]) return 1;
    return (a < b) ? -1 : (a > b);
}

OR_API void or_select_frozen(int n, const double *bad, uint64_t K, uint8_t *frozen)
{
    size_t N = (size_t)1 << n;
    uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * N);
    for (size_t i = 0; i < N; i++) idx[i] = (uint32_t)i;
    g_bad = bad;
    qsort(idx, N, sizeof(uint32_t), cmp_unrel);
    for (size_t i = 0; i < N; i++) frozen[i] = 0;
    for (size_t r = 0; r < N - K; r++) frozen[idx[r]] = 1;
    free(idx);
}

/* ------------------------------------------------------------------------ */
/* Degraded-channel construction: the density evolution of Sec. 3 made      */
/* finite (Tal & Vardy, "How to construct polar codes", IEEE Trans. IT      */
/* 2013, degrading merge).  A symmetric binary-input channel is held as at  */
/* most M conjugate output pairs (a, b), a >= b: a = W(y|0) = W(y'|1) and   */
/* b = W(y|1) = W(y'|0), y' the conjugate output; the pairs' a + b sum to 1 */
/* and the ML error probability is sum b.  With W^-(y1,y2|u1) =             */
/* 1/2 sum_u2 W(y1|u1^u2) W(y2|u2) and W^+(y1,y2,u1|u2) = 1/2 W(y1|u1^u2)   */
/* W(y2|u2), the outputs built from pairs i <= j of W group into:           */
/*   minus: (a_i a_j + b_i b_j, a_i b_j + b_i a_j)                          */
/*   plus:  (a_i a_j, b_i b_j) and (max, min)(a_i b_j, b_i a_j)             */
/* each counted twice when i < j (the orders (i, j) and (j, i)).  The pairs */
/* are then sorted by likelihood ratio a/b and, while more than M remain,   */
/* the two neighbours whose merger (a1+a2, b1+b2) loses the least mutual    */
/* information are merged (first such neighbour in ratio order on ties).    */
/* Merging outputs degrades the channel, so sum b of each bit-channel is an */
/* upper bound on its true error probability that tightens as M grows; with */
/* no merge it is exact.  Index convention as above: the first polarisation */
/* step is the most significant index bit.                                  */
/* BI-AWGN start: y >= 0 is cut into M0 intervals of equal capacity         */
/* contribution (in the LLR 2y/sigma^2), giving pairs                       */
/*   a = P(y in I | +1), b = P(y in I | -1) = P(-y in I | +1),              */
/* then merged down to M like any other step.                               */
/* ------------------------------------------------------------------------ */
typedef struct { double a, b; } tv_pair;

static double tv_info(tv_pair p) /* bits carried by a pair (a + b of them) */
{
    double s = p.a + p.b, r = 0.0;
    if (p.a > 0.0) r += p.a * log2(2.0 * p.a / s);
    if (p.b > 0.0) r += p.b * log2(2.0 * p.b / s);
    return r;
}

static int tv_cmp(const void *pa, const void *pb) /* a/b ascending, then a, then b */
{
    const tv_pair *x = (const tv_pair *)pa, *y = (const tv_pair *)pb;
    double l = x->a * y->b, r = y->a * x->b;
    if (l != r) return l < r ? -1 : 1;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return 0;
}

/* Drops empty pairs, sorts, merges down to at most M pairs; returns the     */
/* count.  info[] caches each pair's information, loss[k] that of merging    */
/* pairs k and k+1 (only the neighbours of a merger change).                 */
static int tv_reduce(tv_pair *p, int L, int M, double *info, double *loss)
{
    int c = 0;
    for (int k = 0; k < L; k++)
        if (p[k].a + p[k].b > 0.0) p[c++] = p[k];
    L = c;
    qsort(p, (size_t)L, sizeof(tv_pair), tv_cmp);
    if (L <= M) return L;
    for (int k = 0; k < L; k++) info[k] = tv_info(p[k]);
    for (int k = 0; k + 1 < L; k++) {
        tv_pair m = {p[k].a + p[k + 1].a, p[k].b + p[k + 1].b};
        loss[k] = info[k] + info[k + 1] - tv_info(m);
    }
    while (L > M) {
        int best = 0;
        for (int k = 1; k + 1 < L; k++)
            if (loss[k] < loss[best]) best = k;
        p[best].a += p[best + 1].a;
        p[best].b += p[best + 1].b;
        info[best] = tv_info(p[best]);
        for (int k = best + 1; k + 1 < L; k++) {
            p[k] = p[k + 1];
            info[k] = info[k + 1];
        }
        for (int k = best + 1; k + 2 < L; k++) loss[k] = loss[k + 1];
        L--;
        for (int k = best - 1; k <= best; k++) {
            if (k < 0 || k + 1 >= L) continue;
            tv_pair m = {p[k].a + p[k + 1].a, p[k].b + p[k + 1].b};
            loss[k] = info[k] + info[k + 1] - tv_info(m);
        }
    }
    return L;
}

static int tv_minus(const tv_pair *w, int L, tv_pair *out)
{
    int c = 0;
    for (int i = 0; i < L; i++)
        for (int j = i; j < L; j++) {
            double f = (i == j) ? 1.0 : 2.0;
            out[c].a = f * (w[i].a * w[j].a + w[i].b * w[j].b);
            out[c].b = f * (w[i].a * w[j].b + w[i].b * w[j].a);
            c++;
        }
    return c;
}

static int tv_plus(const tv_pair *w, int L, tv_pair *out)
{
    int c = 0;
    for (int i = 0; i < L; i++)
        for (int j = i; j < L; j++) {
            double f = (i == j) ? 1.0 : 2.0;
            double x = w[i].a * w[j].b, y = w[i].b * w[j].a;
            out[c].a = f * w[i].a * w[j].a;
            out[c].b = f * w[i].b * w[j].b;
            c++;
            out[c].a = f * (x > y ? x : y);
            out[c].b = f * (x > y ? y : x);
            c++;
        }
    return c;
}

/* Capacity contribution 1 - h2(1 / (1 + e^l)) of an output with LLR l >= 0. */
static double tv_cap_llr(double l)
{
    double q = 1.0 / (1.0 + exp(l));
    if (q <= 0.0) return 1.0;
    return 1.0 + q * log2(q) + (1.0 - q) * log2(1.0 - q);
}

static double tv_q(double x) { return 0.5 * erfc(x / M_SQRT2); }

/* Starting channel: returns its pair count (at most M0 before merging). */
static int tv_start(int channel, double param, int M0, tv_pair *p)
{
    if (channel == 0) { /* BSC(p) */
        p[0].a = 1.0 - param;
        p[0].b = param;
        return 1;
    }
    double s2 = param, sg = sqrt(param);
    double lo_y = 0.0;
    for (int k = 0; k < M0; k++) {
        double hi_y;
        if (k + 1 == M0) {
            hi_y = INFINITY;
        } else { /* LLR where the capacity contribution reaches (k+1)/M0 */
            double target = (double)(k + 1) / M0, lo = 0.0, hi = 1.0;
            while (tv_cap_llr(hi) < target) hi *= 2.0;
            for (int it = 0; it < 200; it++) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                if (tv_cap_llr(mid) < target) lo = mid; else hi = mid;
            }
            hi_y = hi * s2 / 2.0;
        }
        double qa_hi = isinf(hi_y) ? 0.0 : tv_q((hi_y - 1.0) / sg);
        double qb_hi = isinf(hi_y) ? 0.0 : tv_q((hi_y + 1.0) / sg);
        p[k].a = tv_q((lo_y - 1.0) / sg) - qa_hi;
        p[k].b = tv_q((lo_y + 1.0) / sg) - qb_hi;
        lo_y = hi_y;
    }
    return M0;
}

/* Upper bounds on the ML error probability of every bit-channel of a code  */
/* of length 2^n on the BSC (channel 0, param = p) or the BI-AWGN channel   */
/* (channel 1, param = sigma^2), with at most M = mu / 2 pairs per channel. */
/* Returns 0, or -1 for a bad argument.                                     */
OR_API int or_tv_pe(int n, int channel, double param, int mu, double *pe)
{
    int M = mu / 2, M0 = 4 * M;
    if (n < 0 || n > 24 || M < 1 || M > 64 || (channel != 0 && channel != 1)) return -1;
    size_t N = (size_t)1 << n;
    int cap = 2 * M * (M + 1) > M0 ? 2 * M * (M + 1) : M0;
    tv_pair *cur = (tv_pair *)malloc(sizeof(tv_pair) * N * M);
    tv_pair *nxt = (tv_pair *)malloc(sizeof(tv_pair) * N * M);
    int *cnt = (int *)malloc(sizeof(int) * N), *ncnt = (int *)malloc(sizeof(int) * N);
    tv_pair *tmp = (tv_pair *)malloc(sizeof(tv_pair) * cap);
    double *info = (double *)malloc(sizeof(double) * cap);
    double *loss = (double *)malloc(sizeof(double) * cap);
    int L0 = tv_start(channel, param, M0, tmp);
    cnt[0] = tv_reduce(tmp, L0, M, info, loss);
    memcpy(cur, tmp, sizeof(tv_pair) * cnt[0]);
    for (int s = 0; s < n; s++) {
        size_t len = (size_t)1 << s;
        for (size_t j = 0; j < len; j++) {
            for (int side = 0; side < 2; side++) {
                int L = side == 0 ? tv_minus(cur + j * M, cnt[j], tmp)
                                  : tv_plus(cur + j * M, cnt[j], tmp);
                L = tv_reduce(tmp, L, M, info, loss);
                memcpy(nxt + (2 * j + side) * M, tmp, sizeof(tv_pair) * L);
                ncnt[2 * j + side] = L;
            }
        }
        tv_pair *t = cur; cur = nxt; nxt = t;
        int *tc = cnt; cnt = ncnt; ncnt = tc;
    }
    for (size_t i = 0; i < N; i++) {
        double e = 0.0;
        for (int k = 0; k < cnt[i]; k++) e += cur[i * M + k].b;
        pe[i] = e;
    }
    free(cur); free(nxt); free(cnt); free(ncnt); free(tmp); free(info); free(loss);
    return 0;
}

/* Sec. 3's rule for the code rate: the frame error rate of SC is at most   */
/* the sum of the information bits' error probabilities, so K is the        */
/* largest count whose most reliable bit-channels sum to at most `target`.  */
/* Reliability order as in or_select_frozen (bad descending, lower index     */
/* first on ties, so the information set is the tail of that order).        */
OR_API uint64_t or_k_for_sum(int n, const double *bad, double target)
{
    size_t N = (size_t)1 << n;
    uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * N);
    for (size_t i = 0; i < N; i++) idx[i] = (uint32_t)i;
    g_bad = bad;
    qsort(idx, N, sizeof(uint32_t), cmp_unrel);
    double acc = 0.0;
    uint64_t K = 0;
    for (size_t r = N; r-- > 0;) {
        acc += bad[idx[r]];
        if (acc > target) break;
        K++;
    }
    free(idx);
    return K;
}

/* The same rule on log-domain reliabilities (ln Z or ln P_e): the order is   */
/* that of the logs, the sum is of their exponentials.                      */
OR_API uint64_t or_k_for_sum_log(int n, const double *lbad, double target)
{
    size_t N = (size_t)1 << n;
    uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * N);
    for (size_t i = 0; i < N; i++) idx[i] = (uint32_t)i;
    g_bad = lbad;
    qsort(idx, N, sizeof(uint32_t), cmp_unrel);
    double acc = 0.0;
    uint64_t K = 0;
    for (size_t r = N; r-- > 0;) {
        acc += exp(lbad[idx[r]]);
        if (acc > target) break;
        K++;
    }
    free(idx);
    return K;
}

/* ------------------------------------------------------------------------ */
/* Capacities for the efficiency beta = R / C (Sec. 2.1, Eq. 3).            */
/* BSC: C = 1 - h2(p).  BIAWGN with x = 0 sent (+1):                        */
/*   C = 1 - E[log2(1 + exp(-2Y/sigma^2))],  Y ~ N(1, sigma^2),             */
/* by the composite Simpson rule over +-12 sigma.                           */
/* ------------------------------------------------------------------------ */
OR_API double or_capacity_bsc(double p)
{
    if (p <= 0.0 || p >= 1.0) return 1.0;
    return 1.0 + p * log2(p) + (1.0 - p) * log2(1.0 - p);
}

static double log2_1p_exp(double z) /* log2(1 + e^z), no overflow */
{
    if (z > 0) return (z + log1p(exp(-z))) / M_LN2;
    return log1p(exp(z)) / M_LN2;
}

OR_API double or_capacity_biawgn(double sigma2)
{
    double sigma = sqrt(sigma2);
    const int M = 200000; /* even */
    double a = 1.0 - 12.0 * sigma, b = 1.0 + 12.0 * sigma, h = (b - a) / M;
    double acc = 0.0;
    for (int i = 0; i <= M; i++) {
        double y = a + i * h;
        double pdf = exp(-0.5 * (y - 1.0) * (y - 1.0) / sigma2) / (sigma * sqrt(2.0 * M_PI));
        double w = (i == 0 || i == M) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        acc += w * pdf * log2_1p_exp(-2.0 * y / sigma2);
    }
    return 1.0 - acc * h / 3.0;
}
