// Host-side FP64 tables: exact-argument trigonometry, a radix-2 FFT for the
// Bluestein and w-convolution kernels, the wavelet generating functions of
// Sect. 2.2 by composite Gauss-Legendre quadrature, and the per-ring values.
#include "host_tables.h"

#include <algorithm>
#include <cmath>

namespace s2h {

static const double PI = 3.14159265358979323846264338327950288;

void sincospi_rat(int64_t k, int64_t d, double *s, double *c)
{
    // angle = pi k / d, reduced to [0, 2 pi) as k in [0, 2d)
    int64_t K = k % (2 * d);
    if (K < 0) K += 2 * d;
    double ss = 1.0, cs = 1.0;
    if (K > d) {            // sin(2 pi - a) = -sin a
        K = 2 * d - K;
        ss = -1.0;
    }
    if (2 * K > d) {        // cos(pi - a) = -cos a
        K = d - K;
        cs = -1.0;
    }
    double sv, cv;
    if (4 * K <= d) {       // a = pi K / d in [0, pi/4]
        const double a = PI * (double)K / (double)d;
        sv = std::sin(a);
        cv = std::cos(a);
    } else {                // a = pi/2 - b, b = pi (d - 2K) / (2d)
        const double b = PI * (double)(d - 2 * K) / (2.0 * (double)d);
        sv = std::cos(b);
        cv = std::sin(b);
    }
    *s = ss * sv;
    *c = cs * cv;
}

void fft_pow2(std::vector<cd> &a, int sign)
{
    const size_t n = a.size();
    if (n < 2) return;
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const size_t half = len >> 1;
        for (size_t k = 0; k < half; ++k) {
            double s, c;
            sincospi_rat((int64_t)(2 * k), (int64_t)len, &s, &c);   // angle 2 pi k / len
            const cd w(c, sign * s);
            for (size_t i = k; i < n; i += len) {
                const cd u = a[i], v = w * a[i + half];
                a[i] = u + v;
                a[i + half] = u - v;
            }
        }
    }
}

// ------------------------------------------------------------ generating functions
static double bump(double t) { return (t > -1.0 && t < 1.0) ? std::exp(-1.0 / (1.0 - t * t)) : 0.0; }

static double s_lambda(double t, double lam) { return bump(2.0 * lam / (lam - 1.0) * (t - 1.0 / lam) - 1.0); }

struct GL {
    std::vector<double> x, w;
    explicit GL(int n) : x(n), w(n)
    {
        // Newton iteration on the Legendre polynomial P_n
        for (int i = 0; i < (n + 1) / 2; ++i) {
            double z = std::cos(PI * (i + 0.75) / (n + 0.5)), pp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p1 = 1.0, p2 = 0.0;
                for (int j = 1; j <= n; ++j) {
                    const double p3 = p2;
                    p2 = p1;
                    p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
                }
                pp = n * (z * p1 - p2) / (z * z - 1.0);
                const double z1 = z;
                z = z1 - p1 / pp;
                if (std::fabs(z - z1) < 1e-16) break;
            }
            x[i] = -z;
            x[n - 1 - i] = z;
            w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
        }
    }
};

// int_a^b s_lambda(u)^2 / u du, composite 24-point Gauss-Legendre on 64 panels
static double integral(double a, double b, double lam)
{
    static const GL gl(24);
    const int panels = 64;
    const double h = (b - a) / panels;
    double sum = 0.0;
    for (int p = 0; p < panels; ++p) {
        const double lo = a + p * h, mid = lo + 0.5 * h;
        double part = 0.0;
        for (size_t i = 0; i < gl.x.size(); ++i) {
            const double u = mid + 0.5 * h * gl.x[i];
            const double sv = s_lambda(u, lam);
            part += gl.w[i] * sv * sv / u;
        }
        sum += 0.5 * h * part;
    }
    return sum;
}

double k_lambda(double t, double lam)
{
    if (t <= 1.0 / lam) return 1.0;
    if (t >= 1.0) return 0.0;
    return integral(t, 1.0, lam) / integral(1.0 / lam, 1.0, lam);
}

// kappa^2 = k(t/lambda) - k(t): the two integrals of Eq. (smoothscaling) differ by
// the integral over [t/lambda, t] (within the support [1/lambda, 1]), taken directly
// so that nothing cancels where both k values are close to 1.
double kappa_lambda(double t, double lam)
{
    const double lo = std::max(t / lam, 1.0 / lam), hi = std::min(t, 1.0);
    if (hi <= lo) return 0.0;
    return std::sqrt(integral(lo, hi, lam) / integral(1.0 / lam, 1.0, lam));
}

double eta_lambda(double t, double lam) { return std::sqrt(k_lambda(t, lam)); }

// cubic B-spline as its two polynomial pieces: 2/3 - x^2 + |x|^3 / 2 on |x| <= 1,
// (2 - |x|)^3 / 6 on 1 < |x| < 2, zero beyond
static double bspline3(double x)
{
    const double a = std::fabs(x);
    if (a >= 2.0) return 0.0;
    if (a <= 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    const double b = 2.0 - a;
    return b * b * b / 6.0;
}

double bspline_k(double t, double lam, int L, int J)
{
    return 1.5 * bspline3(2.0 * t * std::pow(lam, J - 1) / L);
}

double bspline_eta(int l, int B, int J0, int L, int J)
{
    return std::sqrt(std::max(0.0, bspline_k(l / std::pow((double)B, J0), B, L, J)));
}

double bspline_kappa(int l, int B, int j, int L, int J)
{
    const double kj = bspline_k(l / std::pow((double)B, j), B, L, J);
    const double d = j < J ? bspline_k(l / std::pow((double)B, j + 1), B, L, J) - kj : 1.0 - kj;
    return std::sqrt(std::max(0.0, d));
}

void wav_bandlimits(int L, int B, int J0, int J, bool multires, bool bspline, int *n_scal, std::vector<int> &n_wav)
{
    auto ipow = [](long long b, int e) {
        long long r = 1;
        for (int i = 0; i < e; ++i) r = std::min<long long>(r * b, 1LL << 40);
        return r;
    };
    auto cap = [&](int e) -> int {               // min(L, ceil(L / B^e)), e may be <= 0
        if (e <= 0) return L;
        const long long d = ipow(B, e);
        return (int)std::min<long long>(L, (L + d - 1) / d);
    };
    *n_scal = !multires ? L : bspline ? cap(J - J0 - 1) : (int)std::min<long long>(L, ipow(B, J0));
    n_wav.clear();
    for (int j = J0; j <= J; ++j)
        n_wav.push_back(!multires ? L : bspline ? cap(J - j - 2) : (int)std::min<long long>(L, ipow(B, j + 1)));
}

void wav_kernel(int L, int B, int J0, int J, bool bspline, int k, std::vector<double> &fac)
{
    fac.assign(L, 0.0);
    for (int l = 0; l < L; ++l) {
        if (bspline)
            fac[l] = (k == 0) ? bspline_eta(l, B, J0, L, J) : bspline_kappa(l, B, J0 + k - 1, L, J);
        else
            fac[l] = (k == 0) ? eta_lambda(l / std::pow((double)B, J0), B)
                              : kappa_lambda(l / std::pow((double)B, J0 + k - 1), B);
    }
}

int jmax(int L, int B)
{
    int J = 0;
    long long p = 1;
    while (p < (long long)L - 1) {
        p *= B;
        ++J;
    }
    return J;
}

// ------------------------------------------------------------ band tables
// out[bitrev(k)] = a[k]: the layout the device FFTs multiply in.
static std::vector<cd> bit_reversed(const std::vector<cd> &a)
{
    const size_t n = a.size();
    int bits = 0;
    while (((size_t)1 << bits) < n) ++bits;
    std::vector<cd> out(n);
    for (size_t k = 0; k < n; ++k) {
        size_t r = 0;
        for (int b = 0; b < bits; ++b)
            if (k & ((size_t)1 << b)) r |= (size_t)1 << (bits - 1 - b);
        out[r] = a[k];
    }
    return out;
}

void build_band(int N, Band &bd)
{
    const int P = 2 * N - 1;
    int M = 2, logM = 1;
    while (M < 4 * N - 3) {
        M <<= 1;
        ++logM;
    }
    bd.N = N;
    bd.P = P;
    bd.M = M;
    bd.logM = logM;
    double s, c;
    bd.chirp.resize(P);
    for (int n = 0; n < P; ++n) {
        sincospi_rat((int64_t)n * n % (2 * (int64_t)P), P, &s, &c);
        bd.chirp[n] = cd(c, s);
    }
    std::vector<cd> b(M, cd(0.0, 0.0));
    for (int j = 0; j < P; ++j) b[j] = bd.chirp[j];
    for (int j = 1; j < P; ++j) b[M - j] = bd.chirp[j];
    fft_pow2(b, -1);
    bd.bhat = bit_reversed(b);
    // w(p) = int_0^pi e^{i p theta} sin(theta) dtheta
    std::vector<cd> v(M, cd(0.0, 0.0));
    for (int p = -(2 * N - 2); p <= 2 * N - 2; ++p) {
        cd w(0.0, 0.0);
        if ((p & 1) == 0) w = cd(2.0 / (1.0 - (double)p * p), 0.0);
        else if (p == 1) w = cd(0.0, PI / 2);
        else if (p == -1) w = cd(0.0, -PI / 2);
        v[((p % M) + M) % M] = w;
    }
    fft_pow2(v, -1);
    bd.what = bit_reversed(v);
    // per-stage twiddles, stacked: tw[M - 2h + k] = e^{-2 pi i k / (2h)}, k < h, h = M/2 .. 1
    bd.tw.assign(M, cd(0.0, 0.0));
    for (int h = M / 2; h >= 1; h >>= 1)
        for (int k = 0; k < h; ++k) {
            sincospi_rat((int64_t)k, h, &s, &c);     // angle pi k / h = 2 pi k / (2h)
            bd.tw[M - 2 * h + k] = cd(c, -s);
        }
    bd.phase.resize(2 * N - 1);
    for (int k = -(N - 1); k <= N - 1; ++k) {
        sincospi_rat(k, P, &s, &c);
        bd.phase[k + N - 1] = cd(c, s);
    }
    bd.sinth.resize(N);
    bd.sgn.resize(N);
    bd.y.resize(N);
    bd.xh.resize(N);
    bd.xl.resize(N);
    for (int t = 0; t < N; ++t) {
        const int k = 2 * t + 1;          // theta_t = pi k / P
        const bool north = 2 * k < P;
        const int kr = north ? k : P - k; // distance to the nearer pole, in units of pi/P
        double sh, ch;
        sincospi_rat(kr, P, &s, &c);
        sincospi_rat(kr, 2 * (int64_t)P, &sh, &ch);
        bd.sinth[t] = s;                  // sin(pi - a) = sin a; exactly 0 at the south pole
        bd.sgn[t] = north ? 1.0 : -1.0;
        bd.y[t] = 2.0 * sh * sh;          // 1 - |cos theta| = 2 sin^2(a/2)
        const double x = bd.sgn[t] * (1.0 - bd.y[t]);
        bd.xh[t] = (float)x;
        bd.xl[t] = (float)(x - (double)bd.xh[t]);
    }
}

void legendre_coefs(int L, std::vector<double> &a, std::vector<double> &ab)
{
    a.assign((size_t)L * L, 0.0);
    ab.assign((size_t)L * L, 0.0);
    for (int m = 0; m < L; ++m)
        for (int l = m + 1; l < L; ++l) {
            const double ll = l, mm = m, l1 = l - 1;
            const double av = std::sqrt((4.0 * ll * ll - 1.0) / (ll * ll - mm * mm));
            const double bv = std::sqrt((l1 * l1 - mm * mm) / (4.0 * l1 * l1 - 1.0));
            a[(size_t)m * L + l] = av;
            ab[(size_t)m * L + l] = av * bv;
        }
}

}  // namespace s2h
