// Host-side (FP64) tables of the S2LET GPU library.
#pragma once
#include <complex>
#include <cstdint>
#include <vector>

namespace s2h {

using cd = std::complex<double>;

// sin and cos of pi * k / d for integers k, d > 0, with exact reduction of k
// to the first octant in integers.
void sincospi_rat(int64_t k, int64_t d, double *s, double *c);

// In-place radix-2 FFT, a.size() a power of two; sign -1: e^{-2 pi i jk/M}.
void fft_pow2(std::vector<cd> &a, int sign);

// Generating functions of Sect. 2.2 (smooth construction of McEwen et al.).
double k_lambda(double t, double lam);
double kappa_lambda(double t, double lam);
double eta_lambda(double t, double lam);
// B-spline generating function of the footnote of Sect. 2.2:
// k(t) = 3/2 B_3(2 t lambda^(J-1) / L), B_3 the cubic B-spline (support (-2, 2))
double bspline_k(double t, double lam, int L, int J);
// kernel factors of the B-spline family for degree l: scaling eta(l / lambda^J0) =
// sqrt(k(l / lambda^J0)); wavelet j < J: sqrt(k(l / lambda^(j+1)) - k(l / lambda^j));
// the finest scale j = J: sqrt(1 - k(l / lambda^J)), so that the squared factors of
// all maps sum to one for every l (exact reconstruction)
double bspline_eta(int l, int B, int J0, int L, int J);
double bspline_kappa(int l, int B, int j, int L, int J);

// Band-limits of the scaling map and of wavelet scales J0..J (Sect. 3.1): every
// map at L without multiresolution; otherwise min(L, B^J0) and min(L, B^(j+1))
// for the smooth family, min(L, ceil(L / B^(J-J0-1))) and min(L, ceil(L /
// B^(J-j-2))) for the B-spline family (the ends of the kernels' supports).
void wav_bandlimits(int L, int B, int J0, int J, bool multires, bool bspline, int *n_scal, std::vector<int> &n_wav);
// Kernel factors of map k for degrees l < L: k = 0 the scaling function,
// sqrt(4 pi/(2l+1)) Phi_l0 = eta(l / B^J0); k >= 1 scale j = J0 + k - 1,
// sqrt(4 pi/(2l+1)) Psi^j_l0 = kappa(l / B^j) (Sect. 2.2).
void wav_kernel(int L, int B, int J0, int J, bool bspline, int k, std::vector<double> &fac);
int jmax(int L, int B);

// Per band-limit tables (see fft.cuh and legendre.cuh for their meaning);
// bhat and what are stored in bit-reversed order.
struct Band {
    int N, P, M, logM;
    std::vector<cd> chirp, bhat, what, tw, phase;
    std::vector<double> sinth, sgn, y;   // per ring; cos(theta) = sgn (1 - y)
    std::vector<float> xh, xl;           // cos(theta) as float-float
};
void build_band(int N, Band &b);

// Recurrence coefficients a_lm and a_lm b_lm, row-major [m][l], m, l < L.
void legendre_coefs(int L, std::vector<double> &a, std::vector<double> &ab);

}  // namespace s2h
