/*
 * FP64 (and double-double) CPU oracle for the general spherical harmonic transform of CMB lensing
 * (Reinecke, Belkner & Carron, arXiv:2304.10431).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * What it computes is the plain definition, by direct summation at every
 * point, in double precision with compensated (Neumaier) sums:
 *
 *   spin 0 forward  (Sect. 2, Eq. "forward"):
 *       T_i = sum_{l<=L} sum_{|m|<=l} a_lm Y_lm(theta_i, phi_i)
 *   spin 0 adjoint  (Sect. 2, Eq. "adjoint"):
 *       a_lm = sum_i T_i Y*_lm(theta_i, phi_i),             m >= 0
 *   spin s>0 forward (Sect. 2, Eq. "forwardpol"):
 *       (Q + iU)_i = - e^{i s chi_i} sum_lm (G_lm + i C_lm) sY_lm(n_i)
 *   spin s>0 adjoint (Sect. 2, the two equations after "forwardpol"):
 *       +-sA_lm = sum_i e^{-+ i s chi_i} (Q +- iU)_i  +-sY*_lm(n_i)
 *       G = -1/2 (sA + (-1)^s (-s)A),  C = -1/(2i) (sA - (-1)^s (-s)A)
 *   pointing (Sect. 3, the unlensed-direction formula and Fig. 1):
 *       n' = cos(a) n + sin(a)/a (a_theta e_theta + a_phi e_phi),
 *       chi = beta - beta'
 *
 * Conventions (the paper is silent; these are the readings used here):
 *   Y_lm orthonormal with the Condon-Shortley phase; real fields obey
 *   a_{l,-m} = (-1)^m conj(a_lm).  Spin-weighted harmonics follow
 *   sY_lm = sqrt((l-s)!/(l+s)!) eth^s Y_lm with
 *   eth f = -(sin th)^s (d_th + i/sin th d_ph)(sin th)^-s f, which equals
 *       sY_lm(th, ph) = (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(th) e^{i m ph}
 *   with Wigner's small-d matrix.  The theta part  s lambda_lm(th)  is built
 *   from the closed form at l0 = max(m,|s|) followed by the standard
 *   three-term recursion of d^l_{m1 m2} in l.  Negative m use
 *   s lambda_{l,-m} = (-1)^{s+m} (-s)lambda_{l,m}.
 *
 * Underflow of sin^m is handled by carrying an explicit power-of-two exponent
 * next to the recursion values; values whose true magnitude is below the
 * double range contribute exactly zero.
 *
 * The *_dd entry points evaluate the same definitions with the harmonics
 * (cos and sin of the angles, start values, recursion coefficients and
 * values, e^{i m phi}) in double-double arithmetic (~106 bits) and the sums
 * as above: at lmax ~ 5000 the FP64 recursion's own rounding reaches ~1e-12,
 * the level of the smallest accuracy targets.
 *
 * a_lm layout: index(l,m) = m(2 lmax + 1 - m)/2 + l for 0 <= m <= mmax,
 * m <= l <= lmax; complex numbers are (re, im) pairs of doubles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------- sums */
typedef struct { double s, c; } nsum;
static inline void ns_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static inline double ns_val(const nsum *a) { return a->s + a->c; }

static inline int64_t alm_index(int lmax, int l, int m)
{
    return (int64_t)m * (2 * lmax + 1 - m) / 2 + l;
}

int64_t oracle_nalm(int lmax, int mmax)
{
    return alm_index(lmax, mmax + 1, mmax + 1);
}

/* --------------------------------------------- scaled numbers  x = v*2^e */
typedef struct { double v; int e; } sdbl;
static inline sdbl sd_norm(double v, int e)
{
    int k; double f;
    if (v == 0.0) { sdbl r = {0.0, 0}; return r; }
    f = frexp(v, &k);
    { sdbl r = {f, e + k}; return r; }
}
static inline sdbl sd_mul(sdbl a, double b) { return sd_norm(a.v * b, a.e); }
static inline double sd_val(sdbl a) { return ldexp(a.v, a.e); }

/* x^n for 0 < x <= 1 as a scaled number (binary powering). */
static sdbl sd_pow(double x, int n)
{
    sdbl r = {0.5, 1}, b = sd_norm(x, 0);
    if (x == 0.0) { sdbl z = {0.0, 0}; return n == 0 ? r : z; }
    while (n > 0) {
        if (n & 1) r = sd_norm(r.v * b.v, r.e + b.e);
        b = sd_norm(b.v * b.v, 2 * b.e);
        n >>= 1;
    }
    return r;
}

/* Closed form of  sigma lambda_{l0, m}(theta)  at l0 = max(m, |sigma|), m >= 0.
 * From d^j_{m1 m2} with j = max(|m1|,|m2|) (a single term of Wigner's sum):
 *   m >= |sigma|:  (-1)^m  sqrt((2m+1)/4pi  C(2m, m+sigma)) c^(m-sigma) s^(m+sigma)
 *   m <  |sigma| = a, sigma > 0: (-1)^m sqrt((2a+1)/4pi C(2a, a+m)) c^(a-m) s^(a+m)
 *                     sigma < 0: (-1)^a sqrt((2a+1)/4pi C(2a, a+m)) c^(a+m) s^(a-m)
 * with c = cos(theta/2), s = sin(theta/2). */
static sdbl start_value(int m, int sigma, double theta)
{
    int a = sigma < 0 ? -sigma : sigma;
    int l0 = m >= a ? m : a;
    int n = 2 * l0, k = m >= a ? m + sigma : a + m;
    int pc, ps, sign;
    double c = cos(0.5 * theta), s = sin(0.5 * theta);
    sdbl bin = {0.5, 1}, r;
    int i;
    if (m >= a) { pc = m - sigma; ps = m + sigma; sign = (m & 1) ? -1 : 1; }
    else if (sigma > 0) { pc = a - m; ps = a + m; sign = (m & 1) ? -1 : 1; }
    else { pc = a + m; ps = a - m; sign = (a & 1) ? -1 : 1; }
    /* binomial C(n, k) as a scaled product */
    for (i = 1; i <= k; ++i) bin = sd_mul(bin, (double)(n - k + i) / (double)i);
    /* sqrt of a scaled number: make the exponent even first */
    if (bin.e & 1) { bin.v *= 2.0; bin.e -= 1; }
    r.v = sqrt(bin.v * (2.0 * l0 + 1.0) / (4.0 * OR_PI));
    r.e = bin.e / 2;
    r = sd_norm(r.v, r.e);
    if (pc > 0) { sdbl p = sd_pow(c, pc); r = sd_norm(r.v * p.v, r.e + p.e); }
    if (ps > 0) { sdbl p = sd_pow(s, ps); r = sd_norm(r.v * p.v, r.e + p.e); }
    r.v *= sign;
    return r;
}

/* sigma lambda_{l,m}(theta) for l = 0..lmax (zero below l0), m >= 0, given the
 * scaled start value at l0.  Three-term recursion of d^l_{m1,m2}, m1 = m,
 * m2 = -sigma, normalised by sqrt((2l+1)/4pi):
 *   lam_{l+1} = alpha_{l+1} (x - c_{l+1}) lam_l - beta_{l+1} lam_{l-1}
 *   alpha_{l+1} = (l+1) sqrt((2l+3)(2l+1) / (((l+1)^2-m1^2)((l+1)^2-m2^2)))
 *   c_{l+1}     = m1 m2 / (l (l+1))
 *   beta_{l+1}  = (l+1)/l sqrt((2l+3)/(2l-1)) sqrt((l^2-m1^2)(l^2-m2^2)
 *                                             / (((l+1)^2-m1^2)((l+1)^2-m2^2)))
 */
static void lambda_run(int lmax, int m, int sigma, double theta, sdbl st, double *out)
{
    int a = sigma < 0 ? -sigma : sigma;
    int l0 = m >= a ? m : a, l;
    double x = cos(theta);
    double m1 = m, m2 = -sigma;
    double prev = 0.0, cur;
    int E;
    for (l = 0; l <= lmax && l < l0; ++l) out[l] = 0.0;
    if (l0 > lmax) return;
    if (st.v == 0.0) { for (l = l0; l <= lmax; ++l) out[l] = 0.0; return; }
    /* keep values as cur * 2^E, E a multiple of 128 (or 0) */
    E = 0;
    cur = st.v;
    {
        int e = st.e;
        if (e < 0) { int q = -((-e + 127) / 128); E = q * 128; cur = ldexp(st.v, e - E); }
        else cur = ldexp(st.v, e);
    }
    out[l0] = E == 0 ? cur : ldexp(cur, E);
    for (l = l0; l < lmax; ++l) {
        double lp = l + 1.0, ll = l;
        double den = (lp * lp - m1 * m1) * (lp * lp - m2 * m2);
        double alpha = lp * sqrt((2.0 * ll + 3.0) * (2.0 * ll + 1.0) / den);
        double cc = (l > 0) ? m1 * m2 / (ll * lp) : 0.0;
        double beta = 0.0, nxt;
        if (l > 0) {
            double num = (ll * ll - m1 * m1) * (ll * ll - m2 * m2);
            beta = lp / ll * sqrt((2.0 * ll + 3.0) / (2.0 * ll - 1.0)) * sqrt(num / den);
        }
        nxt = alpha * (x - cc) * cur - beta * prev;
        prev = cur;
        cur = nxt;
        if (E < 0 && fabs(cur) > 0x1p128) {
            cur = ldexp(cur, -128); prev = ldexp(prev, -128); E += 128;
        }
        out[l + 1] = E == 0 ? cur : ldexp(cur, E);
    }
}

/* ------------------------------------------------- double-double mode
 * For targets near or below 1e-12 the FP64 recursion above is not accurate
 * enough at lmax ~ 5000 (cos(theta) and cos(theta/2)^m rounded to FP64, the
 * recursion's own rounding, cos(m phi) of a rounded argument: each ~1e-12).
 * The "precise" entry points therefore carry cos, sin, the start values, the
 * recursion coefficients and values, and e^{i m phi} as unevaluated sums of
 * two doubles (Dekker / Knuth error-free transformations, FMA products),
 * about 106 bits; each value is rounded to one double only where it enters a
 * compensated sum. */
typedef struct { double h, l; } dd;
static inline dd dd_make(double h, double l) { dd r = {h, l}; return r; }
static inline dd dd_fast(double a, double b) /* |a| >= |b| */
{
    double s = a + b;
    return dd_make(s, b - (s - a));
}
static inline dd dd_two_sum(double a, double b)
{
    double s = a + b, bb = s - a;
    return dd_make(s, (a - (s - bb)) + (b - bb));
}
static inline dd dd_add(dd a, dd b)
{
    dd s = dd_two_sum(a.h, b.h), t = dd_two_sum(a.l, b.l);
    s.l += t.h;
    s = dd_fast(s.h, s.l);
    s.l += t.l;
    return dd_fast(s.h, s.l);
}
static inline dd dd_neg(dd a) { return dd_make(-a.h, -a.l); }
static inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static inline dd dd_mul(dd a, dd b)
{
    double p = a.h * b.h;
    double e = fma(a.h, b.h, -p) + (a.h * b.l + a.l * b.h);
    return dd_fast(p, e);
}
static inline dd dd_mul_d(dd a, double b)
{
    double p = a.h * b;
    double e = fma(a.h, b, -p) + a.l * b;
    return dd_fast(p, e);
}
static inline dd dd_div(dd a, dd b)
{
    double q1 = a.h / b.h;
    dd r = dd_sub(a, dd_mul_d(b, q1));
    double q2 = r.h / b.h;
    r = dd_sub(r, dd_mul_d(b, q2));
    double q3 = r.h / b.h;
    dd q = dd_fast(q1, q2);
    return dd_add(q, dd_make(q3, 0.0));
}
static inline dd dd_sqrt(dd a)
{
    double s;
    dd r;
    if (a.h <= 0.0) return dd_make(0.0, 0.0);
    s = sqrt(a.h);
    r = dd_sub(a, dd_mul(dd_make(s, 0.0), dd_make(s, 0.0)));
    return dd_fast(s, r.h / (2.0 * s));
}
static inline dd dd_ldexp(dd a, int e) { return dd_make(ldexp(a.h, e), ldexp(a.l, e)); }
static const dd DD_PI = {3.141592653589793116e+00, 1.224646799147353207e-16};

/* sin and cos of an exact double t: Taylor series of t / 2^K (|t| / 2^K <=
 * 2^-9), then K angle doublings. */
static void dd_sincos(double t, dd *sn, dd *cs)
{
    int K = 12;
    while (fabs(ldexp(t, -K)) > 0x1p-9) ++K;
    dd u = dd_make(ldexp(t, -K), 0.0), u2 = dd_mul(u, u);
    dd s = u, c = dd_make(1.0, 0.0), ts = u, tc = dd_make(1.0, 0.0);
    int k;
    for (k = 1; k <= 10; ++k) {
        ts = dd_div(dd_mul(ts, u2), dd_make(-(double)((2 * k) * (2 * k + 1)), 0.0));
        tc = dd_div(dd_mul(tc, u2), dd_make(-(double)((2 * k - 1) * (2 * k)), 0.0));
        s = dd_add(s, ts);
        c = dd_add(c, tc);
    }
    for (k = 0; k < K; ++k) {
        dd s2 = dd_ldexp(dd_mul(s, c), 1);
        dd c2 = dd_mul(dd_sub(c, s), dd_add(c, s));
        s = s2;
        c = c2;
    }
    *sn = s;
    *cs = c;
}

/* scaled double-double x = v 2^e, |v.h| in [0.5, 1) */
typedef struct { dd v; int e; } sdd;
static inline sdd sdd_norm(dd v, int e)
{
    int k;
    sdd r;
    if (v.h == 0.0) { r.v = dd_make(0.0, 0.0); r.e = 0; return r; }
    frexp(v.h, &k);
    r.v = dd_ldexp(v, -k);
    r.e = e + k;
    return r;
}
static inline sdd sdd_mul(sdd a, sdd b) { return sdd_norm(dd_mul(a.v, b.v), a.e + b.e); }
static sdd sdd_pow(dd x, int n)
{
    sdd r = sdd_norm(dd_make(1.0, 0.0), 0), b = sdd_norm(x, 0);
    while (n > 0) {
        if (n & 1) r = sdd_mul(r, b);
        b = sdd_mul(b, b);
        n >>= 1;
    }
    return r;
}

/* start value (the closed form of start_value) and the recursion of
 * lambda_run, in double-double; out[l] receives the value rounded to double */
static void lambda_run_dd(int lmax, int m, int sigma, double theta, double *out)
{
    int a = sigma < 0 ? -sigma : sigma;
    int l0 = m >= a ? m : a, l, i;
    int n = 2 * l0, k = m >= a ? m + sigma : a + m, pc, ps, sign, E;
    dd sh, ch, x, prev, cur;
    sdd r, bin;
    double m1 = m, m2 = -sigma;
    for (l = 0; l <= lmax && l < l0; ++l) out[l] = 0.0;
    if (l0 > lmax) return;
    dd_sincos(0.5 * theta, &sh, &ch);
    x = dd_sub(dd_mul(ch, ch), dd_mul(sh, sh)); /* cos theta */
    if (m >= a) { pc = m - sigma; ps = m + sigma; sign = (m & 1) ? -1 : 1; }
    else if (sigma > 0) { pc = a - m; ps = a + m; sign = (m & 1) ? -1 : 1; }
    else { pc = a + m; ps = a - m; sign = (a & 1) ? -1 : 1; }
    if (ps > 0 && sh.h == 0.0) { for (l = l0; l <= lmax; ++l) out[l] = 0.0; return; }
    if (pc > 0 && ch.h == 0.0) { for (l = l0; l <= lmax; ++l) out[l] = 0.0; return; }
    bin = sdd_norm(dd_make(1.0, 0.0), 0);
    for (i = 1; i <= k; ++i)
        bin = sdd_norm(dd_div(dd_mul_d(bin.v, (double)(n - k + i)), dd_make((double)i, 0.0)), bin.e);
    /* sqrt(bin (2 l0 + 1) / (4 pi)) with an even exponent */
    if (bin.e & 1) { bin.v = dd_ldexp(bin.v, 1); bin.e -= 1; }
    r.v = dd_sqrt(dd_div(dd_mul_d(bin.v, 2.0 * l0 + 1.0), dd_ldexp(DD_PI, 2)));
    r = sdd_norm(r.v, bin.e / 2);
    if (pc > 0) r = sdd_mul(r, sdd_pow(ch, pc));
    if (ps > 0) r = sdd_mul(r, sdd_pow(sh, ps));
    if (sign < 0) r.v = dd_neg(r.v);
    /* values carried as cur * 2^E, E a multiple of 128 (or 0) */
    E = 0;
    if (r.e < 0) { E = -((-r.e + 127) / 128) * 128; }
    cur = dd_ldexp(r.v, r.e - E);
    prev = dd_make(0.0, 0.0);
    out[l0] = ldexp(cur.h + cur.l, E);
    for (l = l0; l < lmax; ++l) {
        double lp = l + 1.0, ll = l;
        dd den = dd_mul(dd_make((lp - m1) * (lp + m1), 0.0), dd_make((lp - m2) * (lp + m2), 0.0));
        dd alpha = dd_mul_d(dd_sqrt(dd_div(dd_make((2.0 * ll + 3.0) * (2.0 * ll + 1.0), 0.0), den)), lp);
        dd cc = dd_make(0.0, 0.0), beta = dd_make(0.0, 0.0), nxt;
        if (l > 0) {
            dd num = dd_mul(dd_make((ll - m1) * (ll + m1), 0.0), dd_make((ll - m2) * (ll + m2), 0.0));
            cc = dd_div(dd_make(m1 * m2, 0.0), dd_make(ll * lp, 0.0));
            beta = dd_mul(dd_div(dd_make(lp, 0.0), dd_make(ll, 0.0)),
                          dd_sqrt(dd_mul(dd_div(dd_make(2.0 * ll + 3.0, 0.0), dd_make(2.0 * ll - 1.0, 0.0)),
                                         dd_div(num, den))));
        }
        nxt = dd_sub(dd_mul(dd_mul(alpha, dd_sub(x, cc)), cur), dd_mul(beta, prev));
        prev = cur;
        cur = nxt;
        if (E < 0 && fabs(cur.h) > 0x1p128) {
            cur = dd_ldexp(cur, -128); prev = dd_ldexp(prev, -128); E += 128;
        }
        out[l + 1] = E == 0 ? cur.h + cur.l : ldexp(cur.h + cur.l, E);
    }
}

/* e^{i m phi}, m = 0..mmax, by repeated double-double multiplication */
static void eimphi_dd(int mmax, double phi, double *cm, double *sm)
{
    dd s1, c1, c = dd_make(1.0, 0.0), s = dd_make(0.0, 0.0);
    int m;
    dd_sincos(phi, &s1, &c1);
    for (m = 0; m <= mmax; ++m) {
        dd cn, sn;
        cm[m] = c.h + c.l;
        sm[m] = s.h + s.l;
        cn = dd_sub(dd_mul(c, c1), dd_mul(s, s1));
        sn = dd_add(dd_mul(s, c1), dd_mul(c, s1));
        c = cn;
        s = sn;
    }
}

/* sigma lambda_{l,m}(theta) for l = 0..lmax in FP64 or double-double */
static void lambda_any(int lmax, int m, int sigma, double theta, int precise, double *out)
{
    if (precise) lambda_run_dd(lmax, m, sigma, theta, out);
    else lambda_run(lmax, m, sigma, theta, start_value(m, sigma, theta), out);
}

/* Pin helper: sigma lambda_{l,m}(theta), l = 0..lmax, for any sign of m. */
static int slambda_impl(int lmax, int m, int sigma, double theta, int precise, double *out)
{
    int am = m < 0 ? -m : m;
    if (lmax < 0 || am > lmax) return 1;
    if (m >= 0) {
        lambda_any(lmax, m, sigma, theta, precise, out);
    } else {
        /* s lambda_{l,-m} = (-1)^{s+m} (-s) lambda_{l,m} */
        int l, sg = ((sigma + am) & 1) ? -1 : 1;
        lambda_any(lmax, am, -sigma, theta, precise, out);
        for (l = 0; l <= lmax; ++l) out[l] *= sg;
    }
    return 0;
}
int oracle_slambda(int lmax, int m, int sigma, double theta, double *out)
{
    return slambda_impl(lmax, m, sigma, theta, 0, out);
}
int oracle_slambda_dd(int lmax, int m, int sigma, double theta, double *out)
{
    return slambda_impl(lmax, m, sigma, theta, 1, out);
}

/* ------------------------------------------------------------- forward */
/* Ring/point Fourier coefficients:  for every point i and every m, the
 * coefficient of e^{i m phi} in the (pre-phase) field,
 *   spin 0:  F_m = sum_l a_lm lambda_lm(theta),                 m = 0..mmax
 *   spin s:  F_m = - sum_l (G_lm + i C_lm) s lambda_lm(theta),  m = -mmax..mmax
 * out: spin 0 [npts][mmax+1] complex; spin s [npts][2 mmax+1] complex with
 * column m + mmax.  Used by staged tests of the Legendre step. */
int oracle_ring_coeffs(int lmax, int mmax, int spin, int64_t npts, const double *theta,
                       const double *alm, double *out)
{
    int64_t nalm = oracle_nalm(lmax, mmax);
    int ncol = spin == 0 ? mmax + 1 : 2 * mmax + 1;
    int64_t i;
    if (lmax < 0 || mmax < 0 || mmax > lmax || spin < 0 || spin > lmax) return 1;
#pragma omp parallel
    {
        double *lp = (double *)malloc(sizeof(double) * (lmax + 1));
        double *lm = (double *)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
        for (i = 0; i < npts; ++i) {
            int m, l;
            double *o = out + 2 * (int64_t)ncol * i;
            for (m = 0; m <= mmax; ++m) {
                if (spin == 0) {
                    nsum re = {0, 0}, im = {0, 0};
                    lambda_run(lmax, m, 0, theta[i], start_value(m, 0, theta[i]), lp);
                    for (l = m; l <= lmax; ++l) {
                        const double *a = alm + 2 * alm_index(lmax, l, m);
                        ns_add(&re, a[0] * lp[l]);
                        ns_add(&im, a[1] * lp[l]);
                    }
                    o[2 * m] = ns_val(&re);
                    o[2 * m + 1] = ns_val(&im);
                } else {
                    nsum pr = {0, 0}, pi = {0, 0}, qr = {0, 0}, qi = {0, 0};
                    const double *G = alm, *C = alm + 2 * nalm;
                    int sg = (spin & 1) ? -1 : 1;
                    lambda_run(lmax, m, spin, theta[i], start_value(m, spin, theta[i]), lp);
                    lambda_run(lmax, m, -spin, theta[i], start_value(m, -spin, theta[i]), lm);
                    for (l = m; l <= lmax; ++l) {
                        const double *g = G + 2 * alm_index(lmax, l, m);
                        const double *c = C + 2 * alm_index(lmax, l, m);
                        /* m >= 0:  (G + iC) s lambda_lm */
                        ns_add(&pr, (g[0] - c[1]) * lp[l]);
                        ns_add(&pi, (g[1] + c[0]) * lp[l]);
                        /* -m: (G_{l,-m} + i C_{l,-m}) s lambda_{l,-m}
                         *   = (-1)^s (conj G + i conj C) (-s) lambda_lm */
                        ns_add(&qr, sg * (g[0] + c[1]) * lm[l]);
                        ns_add(&qi, sg * (-g[1] + c[0]) * lm[l]);
                    }
                    o[2 * (mmax + m)] = -ns_val(&pr);
                    o[2 * (mmax + m) + 1] = -ns_val(&pi);
                    if (m > 0) {
                        o[2 * (mmax - m)] = -ns_val(&qr);
                        o[2 * (mmax - m) + 1] = -ns_val(&qi);
                    }
                }
            }
        }
        free(lp);
        free(lm);
    }
    return 0;
}

/* Forward lensing operator at arbitrary points (direct summation).
 * alm: [ncomp][nalm] complex (ncomp = 1 for spin 0: T; 2 for spin s: G, C).
 * map: [ncomp][npts] real (spin 0: T; spin s: Q = Re, U = Im).
 * chi may be NULL (no phase). */
static int synthesis_impl(int lmax, int mmax, int spin, int64_t npts, const double *theta,
                          const double *phi, const double *chi, const double *alm, double *map, int precise)
{
    int64_t nalm = oracle_nalm(lmax, mmax);
    int64_t i;
    if (lmax < 0 || mmax < 0 || mmax > lmax || spin < 0 || spin > lmax) return 1;
#pragma omp parallel
    {
        double *lp = (double *)malloc(sizeof(double) * (lmax + 1));
        double *lm = (double *)malloc(sizeof(double) * (lmax + 1));
        double *cmv = (double *)malloc(sizeof(double) * (mmax + 1));
        double *smv = (double *)malloc(sizeof(double) * (mmax + 1));
#pragma omp for schedule(dynamic, 1)
        for (i = 0; i < npts; ++i) {
            int m, l;
            double th = theta[i], ph = phi[i];
            if (precise) eimphi_dd(mmax, ph, cmv, smv);
            else for (m = 0; m <= mmax; ++m) { cmv[m] = cos(m * ph); smv[m] = sin(m * ph); }
            if (spin == 0) {
                nsum tot = {0, 0};
                for (m = 0; m <= mmax; ++m) {
                    nsum re = {0, 0}, im = {0, 0};
                    double cm = cmv[m], sm = smv[m], w = m == 0 ? 1.0 : 2.0;
                    lambda_any(lmax, m, 0, th, precise, lp);
                    for (l = m; l <= lmax; ++l) {
                        const double *a = alm + 2 * alm_index(lmax, l, m);
                        ns_add(&re, a[0] * lp[l]);
                        ns_add(&im, a[1] * lp[l]);
                    }
                    /* a_{l,-m} Y_{l,-m} = conj(a_lm Y_lm): real part counted twice */
                    ns_add(&tot, w * (ns_val(&re) * cm - ns_val(&im) * sm));
                }
                map[i] = ns_val(&tot);
            } else {
                nsum tr = {0, 0}, ti = {0, 0};
                const double *G = alm, *C = alm + 2 * nalm;
                int sg = (spin & 1) ? -1 : 1;
                double ps, pc, zr, zi;
                for (m = 0; m <= mmax; ++m) {
                    nsum pr = {0, 0}, pi = {0, 0}, qr = {0, 0}, qi = {0, 0};
                    double cm = cmv[m], sm = smv[m];
                    lambda_any(lmax, m, spin, th, precise, lp);
                    lambda_any(lmax, m, -spin, th, precise, lm);
                    for (l = m; l <= lmax; ++l) {
                        const double *g = G + 2 * alm_index(lmax, l, m);
                        const double *c = C + 2 * alm_index(lmax, l, m);
                        ns_add(&pr, (g[0] - c[1]) * lp[l]);
                        ns_add(&pi, (g[1] + c[0]) * lp[l]);
                        ns_add(&qr, sg * (g[0] + c[1]) * lm[l]);
                        ns_add(&qi, sg * (-g[1] + c[0]) * lm[l]);
                    }
                    /* + m term times e^{i m phi} */
                    ns_add(&tr, ns_val(&pr) * cm - ns_val(&pi) * sm);
                    ns_add(&ti, ns_val(&pr) * sm + ns_val(&pi) * cm);
                    if (m > 0) { /* - m term times e^{-i m phi} */
                        ns_add(&tr, ns_val(&qr) * cm + ns_val(&qi) * sm);
                        ns_add(&ti, -ns_val(&qr) * sm + ns_val(&qi) * cm);
                    }
                }
                /* - e^{i s chi} * total */
                zr = ns_val(&tr); zi = ns_val(&ti);
                if (chi) { pc = cos(spin * chi[i]); ps = sin(spin * chi[i]); }
                else { pc = 1.0; ps = 0.0; }
                map[i] = -(pc * zr - ps * zi);
                map[npts + i] = -(ps * zr + pc * zi);
            }
        }
        free(lp);
        free(lm);
        free(cmv);
        free(smv);
    }
    return 0;
}

int oracle_synthesis(int lmax, int mmax, int spin, int64_t npts, const double *theta,
                     const double *phi, const double *chi, const double *alm, double *map)
{
    return synthesis_impl(lmax, mmax, spin, npts, theta, phi, chi, alm, map, 0);
}

int oracle_synthesis_dd(int lmax, int mmax, int spin, int64_t npts, const double *theta,
                        const double *phi, const double *chi, const double *alm, double *map)
{
    return synthesis_impl(lmax, mmax, spin, npts, theta, phi, chi, alm, map, 1);
}

/* ------------------------------------------------------------- adjoint */
/* Adjoint at arbitrary points, literal definitions (m >= 0 returned):
 *   spin 0:  a_lm = sum_i T_i Y*_lm(n_i)
 *   spin s:  +-sA_lm = sum_i e^{-+ i s chi_i} (Q_i +- i U_i) +-sY*_lm(n_i)
 *            G = -(sA + (-1)^s (-s)A)/2,  C = -(sA - (-1)^s (-s)A)/(2i)
 * Parallel over m; points are processed in blocks so that the per-point
 * start values (one scaled number per m and spin sign) fit in memory. */
static int adjoint_impl(int lmax, int mmax, int spin, int64_t npts, const double *theta,
                        const double *phi, const double *chi, const double *map, double *alm, int precise)
{
    int64_t nalm = oracle_nalm(lmax, mmax);
    int nsig = spin == 0 ? 1 : 2;
    int64_t blk = (int64_t)(1 << 22) / ((int64_t)(mmax + 1) * nsig);
    int64_t b0;
    nsum *acc;
    if (lmax < 0 || mmax < 0 || mmax > lmax || spin < 0 || spin > lmax) return 1;
    if (blk < 1) blk = 1;
    /* accumulators: per sign (+s, -s) per alm, complex */
    acc = (nsum *)calloc((size_t)(nsig * nalm * 2), sizeof(nsum));
    if (!acc) return 2;
    for (b0 = 0; b0 < npts; b0 += blk) {
        int64_t nb = npts - b0 < blk ? npts - b0 : blk;
        sdbl *st = (sdbl *)malloc(sizeof(sdbl) * (size_t)(nb * (mmax + 1) * nsig));
        double *ec = (double *)malloc(sizeof(double) * (size_t)(nb * (mmax + 1)));
        double *es = (double *)malloc(sizeof(double) * (size_t)(nb * (mmax + 1)));
        int64_t j;
        int m;
        if (!st || !ec || !es) { free(st); free(ec); free(es); free(acc); return 2; }
#pragma omp parallel for schedule(static)
        for (j = 0; j < nb; ++j) {
            int mm, sg;
            if (!precise)
                for (mm = 0; mm <= mmax; ++mm)
                    for (sg = 0; sg < nsig; ++sg)
                        st[(j * (mmax + 1) + mm) * nsig + sg] =
                            start_value(mm, sg == 0 ? spin : -spin, theta[b0 + j]);
            if (precise) eimphi_dd(mmax, phi[b0 + j], ec + j * (mmax + 1), es + j * (mmax + 1));
            else
                for (mm = 0; mm <= mmax; ++mm) {
                    ec[j * (mmax + 1) + mm] = cos(mm * phi[b0 + j]);
                    es[j * (mmax + 1) + mm] = sin(mm * phi[b0 + j]);
                }
        }
#pragma omp parallel
        {
            double *lp = (double *)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
            for (m = 0; m <= mmax; ++m) {
                int sg, l;
                for (sg = 0; sg < nsig; ++sg) {
                    int sigma = sg == 0 ? spin : -spin;
                    nsum *A = acc + 2 * (sg * nalm + alm_index(lmax, m, m));
                    int64_t jj;
                    for (jj = 0; jj < nb; ++jj) {
                        int64_t i = b0 + jj;
                        double cm = ec[jj * (mmax + 1) + m], sm = es[jj * (mmax + 1) + m];
                        double xr, xi, wr, wi;
                        if (spin == 0) { xr = map[i]; xi = 0.0; }
                        else {
                            /* e^{-+ i s chi} (Q +- i U) */
                            double q = map[i], u = map[npts + i];
                            double c = chi ? cos(spin * chi[i]) : 1.0;
                            double s = chi ? sin(spin * chi[i]) : 0.0;
                            if (sg == 0) { xr = c * q + s * u; xi = c * u - s * q; }
                            else { xr = c * q + s * u; xi = -(c * u - s * q); }
                        }
                        /* times e^{-i m phi} */
                        wr = xr * cm + xi * sm;
                        wi = xi * cm - xr * sm;
                        if (precise) lambda_run_dd(lmax, m, sigma, theta[i], lp);
                        else lambda_run(lmax, m, sigma, theta[i], st[(jj * (mmax + 1) + m) * nsig + sg], lp);
                        for (l = m; l <= lmax; ++l) {
                            ns_add(&A[2 * (l - m)], wr * lp[l]);
                            ns_add(&A[2 * (l - m) + 1], wi * lp[l]);
                        }
                    }
                }
            }
            free(lp);
        }
        free(st);
        free(ec);
        free(es);
    }
    {
        int64_t k;
        if (spin == 0) {
            for (k = 0; k < nalm; ++k) {
                alm[2 * k] = ns_val(&acc[2 * k]);
                alm[2 * k + 1] = ns_val(&acc[2 * k + 1]);
            }
        } else {
            double sg = (spin & 1) ? -1.0 : 1.0;
            for (k = 0; k < nalm; ++k) {
                double ar = ns_val(&acc[2 * k]), ai = ns_val(&acc[2 * k + 1]);
                double br = sg * ns_val(&acc[2 * (nalm + k)]), bi = sg * ns_val(&acc[2 * (nalm + k) + 1]);
                /* G = -(a + b)/2 ;  C = -(a - b)/(2i) = i (a - b)/2 */
                alm[2 * k] = -0.5 * (ar + br);
                alm[2 * k + 1] = -0.5 * (ai + bi);
                alm[2 * (nalm + k)] = -0.5 * (ai - bi);
                alm[2 * (nalm + k) + 1] = 0.5 * (ar - br);
            }
        }
    }
    free(acc);
    return 0;
}

int oracle_adjoint(int lmax, int mmax, int spin, int64_t npts, const double *theta,
                   const double *phi, const double *chi, const double *map, double *alm)
{
    return adjoint_impl(lmax, mmax, spin, npts, theta, phi, chi, map, alm, 0);
}

int oracle_adjoint_dd(int lmax, int mmax, int spin, int64_t npts, const double *theta,
                      const double *phi, const double *chi, const double *map, double *alm)
{
    return adjoint_impl(lmax, mmax, spin, npts, theta, phi, chi, map, alm, 1);
}

/* ------------------------------------------------------------ pointing */
/* Unlensed direction and spin phase (Sect. 3, pointing formula; Fig. 1):
 *   n' = cos(a) n + sin(a)/a (a_th e_th + a_ph e_ph),  a = |alpha|
 * beta  = angle of the deflection at n, measured from e_th towards e_ph;
 * beta' = angle of the geodesic's tangent at n' in the local (e_th', e_ph')
 *         basis; chi = beta - beta' wrapped to (-pi, pi]; chi = 0 if a = 0.
 * theta' in [0, pi], phi' in [0, 2pi). */
int oracle_pointing(int64_t n, const double *theta, const double *phi, const double *ath,
                    const double *aph, double *theta_out, double *phi_out, double *chi_out)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double st = sin(theta[i]), ct = cos(theta[i]), sp = sin(phi[i]), cp = cos(phi[i]);
        double nv[3] = {st * cp, st * sp, ct};
        double et[3] = {ct * cp, ct * sp, -st};
        double ep[3] = {-sp, cp, 0.0};
        double a = sqrt(ath[i] * ath[i] + aph[i] * aph[i]);
        double np_[3], tp[3], d[3], th2, ph2, chi = 0.0;
        int k;
        if (a == 0.0) {
            theta_out[i] = theta[i];
            ph2 = fmod(phi[i], 2.0 * OR_PI);
            if (ph2 < 0) ph2 += 2.0 * OR_PI;
            phi_out[i] = ph2;
            if (chi_out) chi_out[i] = 0.0;
            continue;
        }
        for (k = 0; k < 3; ++k) d[k] = (ath[i] * et[k] + aph[i] * ep[k]) / a;
        for (k = 0; k < 3; ++k) {
            np_[k] = cos(a) * nv[k] + sin(a) * d[k];
            tp[k] = -sin(a) * nv[k] + cos(a) * d[k];
        }
        th2 = atan2(sqrt(np_[0] * np_[0] + np_[1] * np_[1]), np_[2]);
        ph2 = atan2(np_[1], np_[0]);
        if (ph2 < 0) ph2 += 2.0 * OR_PI;
        if (ph2 >= 2.0 * OR_PI) ph2 -= 2.0 * OR_PI;
        theta_out[i] = th2;
        phi_out[i] = ph2;
        if (chi_out) {
            double st2 = sin(th2), ct2 = cos(th2), sp2 = sin(ph2), cp2 = cos(ph2);
            double et2[3] = {ct2 * cp2, ct2 * sp2, -st2};
            double ep2[3] = {-sp2, cp2, 0.0};
            double beta = atan2(aph[i], ath[i]);
            double bp = atan2(tp[0] * ep2[0] + tp[1] * ep2[1] + tp[2] * ep2[2],
                              tp[0] * et2[0] + tp[1] * et2[1] + tp[2] * et2[2]);
            chi = beta - bp;
            while (chi > OR_PI) chi -= 2.0 * OR_PI;
            while (chi <= -OR_PI) chi += 2.0 * OR_PI;
            chi_out[i] = chi;
        }
    }
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
