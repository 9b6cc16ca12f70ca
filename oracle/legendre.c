/*
 * ORACLE — test infrastructure only.  Plain FP64 CPU reference for the
 * Legendre part of the spherical harmonic transforms of the S2LET paper
 * (Leistedt, McEwen, Vandergheynst & Wiaux 2013).  Only tests/, the smoke
 * check and the CPU-baseline leg of bench.py may load this file; the GPU
 * library never does.
 *
 * Y_lm(theta, phi) = lambda_lm(theta) e^{i m phi} are the spherical harmonics
 * of Eq. (harmonicssynthesis) / (harmonicsanalysis), Sect. 2.1, with the
 * Condon-Shortley phase.  lambda_lm is computed with the textbook recurrences
 * for orthonormal associated Legendre functions:
 *
 *   lambda_mm      = (-1)^m sqrt((2m+1)/(4 pi) prod_{k=1..m} (2k-1)/(2k)) sin^m theta
 *   lambda_{m+1,m} = sqrt(2m+3) cos(theta) lambda_mm
 *   lambda_lm      = a_lm (cos(theta) lambda_{l-1,m} - b_lm lambda_{l-2,m})
 *       a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1))
 *   lambda_{l,-m}  = (-1)^m lambda_lm
 *
 * cos(theta) enters as sgn (1 - y), with sgn = +-1 the sign of cos(theta) and
 * y = 1 - |cos(theta)| given to full relative precision by the caller, so
 * cos(theta) lambda is evaluated as sgn (lambda - y lambda).  This is the same
 * recurrence; near the poles, where |cos(theta)| is close to 1, it keeps the
 * rounding error of every step relative to the small quantity y lambda
 * instead of to lambda.
 *
 * Near the poles the sectoral value underflows any floating-point format
 * (sin^2047 of pi/4095 is about 1e-6370), so the seed and the start of the
 * recurrence are carried as "extended numbers": an FP64 mantissa and a
 * separate int base-2 exponent.  Once the value exceeds 2^-900 the
 * recurrence continues in plain FP64.  Conversion to FP64 rounds values below
 * the FP64 range to 0, which is the correctly rounded FP64 result.
 *
 * The seed is computed from the product formula for every (m, theta), not
 * incrementally, so the code reads like the formula above.
 */
#include <math.h>
#include <stddef.h>

typedef struct {
    double f; /* mantissa, 0.5 <= |f| < 1, or 0 */
    int e;    /* value = f * 2^e */
} xnum;

static xnum xnorm(double f, int e)
{
    xnum r;
    int k = 0;
    if (f == 0.0) {
        r.f = 0.0;
        r.e = -(1 << 28);
        return r;
    }
    r.f = frexp(f, &k);
    r.e = e + k;
    return r;
}

static xnum xfrom(double v) { return xnorm(v, 0); }

/* a (sgn (x - y x) - b z), the recurrence step on extended numbers */
static xnum xstep(double a, double b, double sgn, double y, xnum x, xnum z)
{
    int e = x.e > z.e ? x.e : z.e;
    double xs = ldexp(x.f, x.e - e), zs = ldexp(z.f, z.e - e);
    double v = a * (sgn * (xs - y * xs) - b * zs);
    return xnorm(v, e);
}

static double xtod(xnum a)
{
    if (a.f == 0.0) return 0.0;
    if (a.e < -1100) return 0.0;
    return ldexp(a.f, a.e);
}

/* lambda_mm(theta) from the product formula, as an extended number.  The
 * running product is renormalised by 2^500 whenever it falls below 2^-500. */
static xnum sectoral(int m, double sin_t)
{
    const double PI = 3.14159265358979323846;
    double f = sqrt((2.0 * m + 1.0) / (4.0 * PI));
    int e = 0;
    for (int k = 1; k <= m; ++k) {
        f *= -sqrt((2.0 * k - 1.0) / (2.0 * k)) * sin_t;
        if (f != 0.0 && fabs(f) < 0x1p-500) {
            f = ldexp(f, 500);
            e -= 500;
        }
    }
    return xnorm(f, e);
}

static double coef_a(int l, int m)
{
    double L = l, M = m;
    return sqrt((4.0 * L * L - 1.0) / (L * L - M * M));
}

static double coef_b(int l, int m)
{
    double L1 = l - 1, M = m;
    return sqrt((L1 * L1 - M * M) / (4.0 * L1 * L1 - 1.0));
}

/*
 * lambda_lm(theta) for l = m .. N-1 (m >= 0) written to out[l - m].
 * sin_t: sin(theta); cos(theta) = sgn (1 - y) (the caller passes exact values
 * at the poles).  Optionally out_e (may be NULL) receives, for each l, the base-2
 * exponent of the extended number before conversion, and out_f its mantissa;
 * tests use them to pin values that FP64 cannot hold.
 */
void oracle_legendre_column(int m, int N, double sin_t, double sgn, double y,
                            double *out, double *out_f, int *out_e)
{
    if (m >= N) return;
    xnum p1 = sectoral(m, sin_t); /* lambda_{l-1} */
    xnum p0 = xfrom(0.0);         /* lambda_{l-2} */
    out[0] = xtod(p1);
    if (out_f) out_f[0] = p1.f;
    if (out_e) out_e[0] = p1.e;
    int l = m + 1;
    /* extended-number phase */
    for (; l < N && p1.e < -900; ++l) {
        xnum p2 = xstep(coef_a(l, m), coef_b(l, m), sgn, y, p1, p0);
        out[l - m] = xtod(p2);
        if (out_f) out_f[l - m] = p2.f;
        if (out_e) out_e[l - m] = p2.e;
        p0 = p1;
        p1 = p2;
    }
    /* plain FP64 phase */
    double d0 = xtod(p0), d1 = xtod(p1);
    for (; l < N; ++l) {
        double a = coef_a(l, m), b = coef_b(l, m);
        double d2 = a * (sgn * (d1 - y * d1) - b * d0);
        out[l - m] = d2;
        if (out_f || out_e) {
            xnum x = xfrom(d2);
            if (out_f) out_f[l - m] = x.f;
            if (out_e) out_e[l - m] = x.e;
        }
        d0 = d1;
        d1 = d2;
    }
}

/*
 * Legendre part of the inverse transform, Eq. (harmonicssynthesis):
 *   F_m(theta_t) = sum_{l=|m|}^{N-1} f_lm lambda_{l,m}(theta_t)
 * for the n_ord orders m = orders[k] and t = 0 .. nt-1.  One column
 * lambda_{l,|m|}(theta_t) serves m and -m (lambda_{l,-m} = (-1)^m lambda_lm).
 * flm: complex, interleaved re/im, index l*l + l + m (length N*N).
 * F:   complex, interleaved, [k][t], n_ord x nt.
 */
void oracle_legendre_inverse(int N, const double *flm, int nt, const double *sin_t,
                             const double *sgn, const double *y, int n_ord, const int *orders,
                             double *F)
{
    if (N > 8192) return;
#pragma omp parallel
    {
        double lam[8192];
#pragma omp for schedule(dynamic, 1)
        for (int am = 0; am < N; ++am) {
            int kp = -1, kn = -1; /* positions of +am and -am in the list */
            for (int k = 0; k < n_ord; ++k) {
                if (orders[k] == am) kp = k;
                if (am > 0 && orders[k] == -am) kn = k;
            }
            if (kp < 0 && kn < 0) continue;
            for (int t = 0; t < nt; ++t) {
                oracle_legendre_column(am, N, sin_t[t], sgn[t], y[t], lam, 0, 0);
                for (int s = 0; s < 2; ++s) {
                    int k = s ? kn : kp;
                    if (k < 0) continue;
                    int m = s ? -am : am;
                    double sg = (s && (am & 1)) ? -1.0 : 1.0;
                    double re = 0.0, im = 0.0;
                    for (int l = am; l < N; ++l) {
                        double v = sg * lam[l - am];
                        size_t idx = (size_t)l * l + l + m;
                        re += flm[2 * idx] * v;
                        im += flm[2 * idx + 1] * v;
                    }
                    size_t o = (size_t)k * nt + t;
                    F[2 * o] = re;
                    F[2 * o + 1] = im;
                }
            }
        }
    }
}

/*
 * Legendre contraction of the forward transform (last step of the MW
 * quadrature, Eq. (harmonicsanalysis) made a finite sum by the sampling
 * theorem of Sect. 2.1):
 *   out_lm = sum_{t=0}^{nt-1} lambda_{l,m}(theta_t) G_m(theta_t)
 * for the n_ord orders m = orders[k] and l = |m| .. N-1; other entries of out
 * are left as they are.  The caller applies the quadrature factor.
 * G:   complex, interleaved, [k][t], n_ord x nt.
 * out: complex, interleaved, index l*l + l + m.
 */
void oracle_legendre_forward(int N, const double *G, int nt, const double *sin_t,
                             const double *sgn, const double *y, int n_ord, const int *orders,
                             double *out)
{
    if (N > 8192) return;
#pragma omp parallel
    {
        double lam[8192];
#pragma omp for schedule(dynamic, 1)
        for (int am = 0; am < N; ++am) {
            int kp = -1, kn = -1;
            for (int k = 0; k < n_ord; ++k) {
                if (orders[k] == am) kp = k;
                if (am > 0 && orders[k] == -am) kn = k;
            }
            if (kp < 0 && kn < 0) continue;
            for (int s = 0; s < 2; ++s) {
                if ((s ? kn : kp) < 0) continue;
                int m = s ? -am : am;
                for (int l = am; l < N; ++l) {
                    size_t idx = (size_t)l * l + l + m;
                    out[2 * idx] = 0.0;
                    out[2 * idx + 1] = 0.0;
                }
            }
            for (int t = 0; t < nt; ++t) {
                oracle_legendre_column(am, N, sin_t[t], sgn[t], y[t], lam, 0, 0);
                for (int s = 0; s < 2; ++s) {
                    int k = s ? kn : kp;
                    if (k < 0) continue;
                    int m = s ? -am : am;
                    double sg = (s && (am & 1)) ? -1.0 : 1.0;
                    size_t o = (size_t)k * nt + t;
                    double gre = G[2 * o], gim = G[2 * o + 1];
                    for (int l = am; l < N; ++l) {
                        double v = sg * lam[l - am];
                        size_t idx = (size_t)l * l + l + m;
                        out[2 * idx] += v * gre;
                        out[2 * idx + 1] += v * gim;
                    }
                }
            }
        }
    }
}
