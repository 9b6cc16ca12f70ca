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
