// Mixed-radix FFTs of odd length P = 2N - 1 in shared memory (FP32), for the
// band-limits whose P factors into the radices 13, 11, 9, 7, 5, 3 (P = 4095 =
// 13 * 9 * 7 * 5 at N = 2048).  Unlike the Bluestein form of fft.cuh, which
// computes a length-P DFT as a circular convolution of length M >= 2P - 1, the
// transform works on the P samples directly: a quarter of the operations per
// sample at P = 4095, and no chirp products whose intermediates exceed the
// result by sqrt(P).
//
// Decimation in frequency, in place (Cooley-Tukey for composite lengths): with
// P = R S' and n = j + S' q, k = s + R k', the DFT splits into R DFTs of
// length S' of y_s[j] = w_P^{j s} sum_q x[j + S' q] w_R^{q s}, stored at
// j + S' s.  Repeating this on every block leaves X_k at a mixed-radix
// digit-reversed position pos(k) (tables below); natural order in, permuted
// order out.  The transposed algorithm (twiddles before the radix-R DFTs,
// passes in reverse order) takes permuted input to natural output, so a
// product with a diagonal between a forward and an inverse transform needs no
// permutation pass.  Radix-R DFTs of prime R pair x_k with x_{R-k}, so each
// cosine and sine product serves two outputs; radix 9 is 3 x 3 in registers.
#pragma once
#include "common.cuh"
#include "dft_consts.cuh"

namespace s2g {

// ---------------------------------------------------------------- factorisation
struct MrFactors {
    int n;          // number of passes, -1 if P has a prime factor above 13
    int r[16];      // radices, first pass first
};
__host__ __device__ constexpr MrFactors mr_factors(int P)
{
    MrFactors f{0, {}};
    const int cand[6] = {13, 11, 9, 7, 5, 3};
    for (int i = 0; i < 6; ++i)
        while (P > 1 && P % cand[i] == 0 && f.n < 16) {
            f.r[f.n++] = cand[i];
            P /= cand[i];
        }
    if (P != 1) f.n = -1;
    // the largest radix second to last: with the lane order of mr_pass this keeps the
    // passes' shared-memory accesses nearly free of bank conflicts (P = 4095:
    // 9, 7, 13, 5 take 1.12 times the ideal wavefronts, 13, 9, 7, 5 took 1.36)
    if (f.n >= 3) {
        const int r0 = f.r[0];
        for (int i = 0; i < f.n - 2; ++i) f.r[i] = f.r[i + 1];
        f.r[f.n - 2] = r0;
    }
    return f;
}
// length of the sub-transforms entering pass i (P for pass 0)
__host__ __device__ constexpr int mr_sub(int P, int i)
{
    const MrFactors f = mr_factors(P);
    int S = P;
    for (int k = 0; k < i; ++k) S /= f.r[k];
    return S;
}

// Offset of pass i's twiddles in the per-pass table: pass i (radix R, M = S / R)
// holds w_S^{j s} at (s - 1) M + j, s = 1..R-1, j < M, so that the threads of a
// pass, which run over consecutive j, read consecutive entries.
__host__ __device__ constexpr int mr_tw_off(int P, int i)
{
    const MrFactors f = mr_factors(P);
    int off = 0;
    for (int k = 0; k < i; ++k) off += (f.r[k] - 1) * (mr_sub(P, k) / f.r[k]);
    return off;
}

// The band-limits with mixed-radix kernels: P = 2N - 1 in this list.
#define S2G_MR_LENGTHS(X) X(7) X(15) X(45) X(63) X(65) X(99) X(315) X(4095)
__host__ __device__ constexpr bool mr_supported(int P)
{
    return P == 7 || P == 15 || P == 45 || P == 63 || P == 65 || P == 99 || P == 315 || P == 4095;
}

// Tables of one length P (device pointers, built on the host in FP64):
//   tw       per-pass twiddles (mr_tw_off), w_S = e^{-2 pi i / S}
//   rev[k]   = position of X_k after the forward passes
//   shm[p]   = e^{-i a pi / P} at position p = rev[k], a = k (k < N) or k - P:
//              the half-sample shift theta -> theta - pi/P of the quadrature
//   shp[p]   = conj(shm[p]) / P
//   ve[t]    = v_even(theta_t - pi/P) / P, vfold[t] (t < N): quadrature weights,
//   qd[t], qa[t] (t < N): pole-ring columns of the shifted-grid product (k_quad_mr)
struct MrTab {
    const float2 *tw;
    const int *rev;
    const float2 *shm, *shp;
    const float *ve, *vfold, *qd, *qa;
};

// ---------------------------------------------------------------- small DFTs
template <bool INV> __device__ __forceinline__ float2 mr_twiddle(float2 x, float2 w)
{
    // x * w, or x * conj(w) for the inverse transform
    return INV ? make_float2(fmaf(x.x, w.x, x.y * w.y), fmaf(x.y, w.x, -x.x * w.y))
               : make_float2(fmaf(x.x, w.x, -x.y * w.y), fmaf(x.x, w.y, x.y * w.x));
}

// y_s = sum_q x_q e^{-+2 pi i q s / R} in place, R odd prime (pairing k, R-k):
// y_0 = x_0 + sum a_k, y_s = A_s -+ i B_s, y_{R-s} = A_s +- i B_s with
// a_k = x_k + x_{R-k}, b_k = x_k - x_{R-k}, A_s = x_0 + sum_k a_k cos(2 pi k s/R),
// B_s = sum_k b_k sin(2 pi k s/R)
template <int R, bool INV> __device__ __forceinline__ void mr_dft_prime(float2 (&x)[R])
{
    constexpr int H = (R - 1) / 2;
    using K = DftConst<R>;
    float2 a[H], b[H];
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        a[k - 1] = make_float2(x[k].x + x[R - k].x, x[k].y + x[R - k].y);
        b[k - 1] = make_float2(x[k].x - x[R - k].x, x[k].y - x[R - k].y);
    }
    float2 y0 = x[0];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        y0.x += a[k].x;
        y0.y += a[k].y;
    }
#pragma unroll
    for (int s = 1; s <= H; ++s) {
        float2 A = x[0], B = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const int e = (k * s) % R;
            const float c = K::c(e), sn = K::s(e);
            A.x = fmaf(a[k - 1].x, c, A.x);
            A.y = fmaf(a[k - 1].y, c, A.y);
            B.x = fmaf(b[k - 1].x, sn, B.x);
            B.y = fmaf(b[k - 1].y, sn, B.y);
        }
        // -i B = (B.y, -B.x)
        if (INV) {
            x[s] = make_float2(A.x - B.y, A.y + B.x);
            x[R - s] = make_float2(A.x + B.y, A.y - B.x);
        } else {
            x[s] = make_float2(A.x + B.y, A.y - B.x);
            x[R - s] = make_float2(A.x - B.y, A.y + B.x);
        }
    }
    x[0] = y0;
}

template <bool INV> __device__ __forceinline__ void mr_dft3(float2 &x0, float2 &x1, float2 &x2)
{
    float2 v[3] = {x0, x1, x2};
    mr_dft_prime<3, INV>(v);
    x0 = v[0];
    x1 = v[1];
    x2 = v[2];
}

// radix 9 as 3 x 3: n = n1 + 3 n2, k = k2 + 3 k1; DFTs over n2, twiddles
// w_9^{n1 k2}, DFTs over n1
template <bool INV> __device__ __forceinline__ void mr_dft9(float2 (&x)[9])
{
    using K = DftConst<9>;
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) mr_dft3<INV>(x[n1], x[n1 + 3], x[n1 + 6]);
    // u[n1][k2] now at x[n1 + 3 k2]; twiddles for n1, k2 in {1, 2}
#pragma unroll
    for (int n1 = 1; n1 < 3; ++n1)
#pragma unroll
        for (int k2 = 1; k2 < 3; ++k2) {
            const int e = n1 * k2;
            x[n1 + 3 * k2] = mr_twiddle<INV>(x[n1 + 3 * k2], make_float2(K::c(e), -K::s(e)));
        }
    float2 y[9];
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
        float2 p = x[3 * k2], q = x[1 + 3 * k2], r = x[2 + 3 * k2];
        mr_dft3<INV>(p, q, r);
        y[k2] = p;          // k = k2 + 3 k1
        y[k2 + 3] = q;
        y[k2 + 6] = r;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = y[i];
}

template <int R, bool INV> __device__ __forceinline__ void mr_dft(float2 (&x)[R])
{
    if constexpr (R == 9) mr_dft9<INV>(x);
    else mr_dft_prime<R, INV>(x);
}

// ---------------------------------------------------------------- passes
// One pass over NF transforms of length P: radix R on sub-transforms of length
// S (M = S / R butterflies each).  DIT: twiddles before the radix-R DFT
// (transposed algorithm), else after it.  Element pos of transform f is read
// with ld(f, pos) and written with st(f, pos, v): shared memory for inner
// passes, global memory or a product with a table for the first and last.
// Lanes take consecutive butterflies j of a sub-transform (contiguous addresses)
// where there are at least 16 of them; in the late passes, where there are
// fewer, consecutive sub-transforms blk (addresses an odd stride S apart, which
// fall in distinct banks) and share their twiddles.
// A thread runs the same butterfly of every transform of the block, so its
// twiddles are loaded once for NF butterflies.
template <int P, int R, int S, int TWO, bool DIT, bool INV, int NF, class LD, class ST>
__device__ __forceinline__ void mr_pass(const float2 *__restrict__ twp, LD ld, ST st)
{
    constexpr int M = S / R, NB = P / R, NBLK = P / S;
    constexpr bool BLK_FAST = M < 16;
    const float2 *tw = twp + TWO;
    for (int r = threadIdx.x; r < NB; r += blockDim.x) {
        const int blk = BLK_FAST ? r % NBLK : r / M;
        const int j = BLK_FAST ? r / NBLK : r - blk * M;
        const int base = blk * S + j;
        float2 w[R > 1 ? R - 1 : 1];
        if (M > 1 && j > 0) {
#pragma unroll
            for (int s = 1; s < R; ++s) w[s - 1] = __ldg(tw + (s - 1) * M + j);
        }
#pragma unroll 1
        for (int f = 0; f < NF; ++f) {
            float2 x[R];
#pragma unroll
            for (int q = 0; q < R; ++q) x[q] = ld(f, base + q * M);
            if (DIT && M > 1 && j > 0) {
#pragma unroll
                for (int s = 1; s < R; ++s) x[s] = mr_twiddle<INV>(x[s], w[s - 1]);
            }
            mr_dft<R, INV>(x);
            if (!DIT && M > 1 && j > 0) {
#pragma unroll
                for (int s = 1; s < R; ++s) x[s] = mr_twiddle<INV>(x[s], w[s - 1]);
            }
#pragma unroll
            for (int q = 0; q < R; ++q) st(f, base + q * M, x[q]);
        }
    }
    __syncthreads();
}

// shared-memory element access of NF transforms stored at buf + f P
template <int P> struct MrSmem {
    float2 *buf;
    __device__ __forceinline__ float2 operator()(int f, int pos) const { return buf[f * P + pos]; }
    __device__ __forceinline__ void operator()(int f, int pos, float2 v) const { buf[f * P + pos] = v; }
};

// passes I, I+1, .., LAST (DIF) or I, I-1, .., LAST (DIT); the first pass executed
// loads with ld, the last one stores with st, all others use shared memory
template <int P, int I, int LAST, bool DIT, bool INV, int NF, class LD, class ST>
__device__ __forceinline__ void mr_run_range(float2 *buf, const float2 *tw, LD ld, ST st, int first)
{
    constexpr MrFactors F = mr_factors(P);
    if constexpr (I >= 0 && I < F.n && (DIT ? I >= LAST : I <= LAST)) {
        constexpr int R = F.r[I], S = mr_sub(P, I), TWO = mr_tw_off(P, I);
        const MrSmem<P> sm{buf};
        const bool is_first = I == first;
        if constexpr (I == LAST) {
            if (is_first) mr_pass<P, R, S, TWO, DIT, INV, NF>(tw, ld, st);
            else mr_pass<P, R, S, TWO, DIT, INV, NF>(tw, sm, st);
        } else {
            if (is_first) mr_pass<P, R, S, TWO, DIT, INV, NF>(tw, ld, sm);
            else mr_pass<P, R, S, TWO, DIT, INV, NF>(tw, sm, sm);
        }
        mr_run_range<P, DIT ? I - 1 : I + 1, LAST, DIT, INV, NF>(buf, tw, ld, st, first);
    }
}
template <int P, int I, bool DIT, bool INV, int NF, class LD, class ST>
__device__ __forceinline__ void mr_run(float2 *buf, const float2 *tw, LD ld, ST st)
{
    constexpr MrFactors F = mr_factors(P);
    mr_run_range<P, I, DIT ? 0 : F.n - 1, DIT, INV, NF>(buf, tw, ld, st, I);
}

// Two passes fused on the same butterflies, with a product by a table between
// them, where a transform's last pass and the next transform's first pass act
// on the same groups of elements:
//   mr_pass_dif_last_dit_first: the last forward (DIF) pass, tab1[pos], the first
//     inverse (DIT) pass (M = 1, no twiddles); tab1 complex
//   mr_pass_dit_last_dif_first: the last inverse (DIT) pass (pass 0), tab2[pos],
//     the first forward (DIF) pass (pass 0), sharing the twiddles; tab2 real
// Each saves one round trip of the transforms through shared memory.
template <int P, int NF>
__device__ __forceinline__ void mr_pass_dif_last_dit_first(float2 *buf, const float2 *__restrict__ tab1)
{
    constexpr MrFactors F = mr_factors(P);
    constexpr int I = F.n - 1, R = F.r[I], S = mr_sub(P, I), NB = P / R;
    static_assert(S == R, "last pass of length R");
    for (int r = threadIdx.x; r < NB; r += blockDim.x) {
        const int base = r * S;
#pragma unroll 1
        for (int f = 0; f < NF; ++f) {
            float2 x[R];
#pragma unroll
            for (int q = 0; q < R; ++q) x[q] = buf[f * P + base + q];
            mr_dft<R, false>(x);
#pragma unroll
            for (int q = 0; q < R; ++q) x[q] = mr_twiddle<false>(x[q], __ldg(tab1 + base + q));
            mr_dft<R, true>(x);
#pragma unroll
            for (int q = 0; q < R; ++q) buf[f * P + base + q] = x[q];
        }
    }
    __syncthreads();
}
template <int P, int NF>
__device__ __forceinline__ void mr_pass_dit_last_dif_first(float2 *buf, const float2 *__restrict__ twp,
                                                           const float *__restrict__ tab2)
{
    constexpr MrFactors F = mr_factors(P);
    constexpr int R = F.r[0], M = P / R, TWO = mr_tw_off(P, 0);
    // pass 0 has one sub-transform (S = P): its lanes run over the butterflies j either way
    const float2 *tw = twp + TWO;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        float2 w[R - 1];
        if (j > 0) {
#pragma unroll
            for (int s = 1; s < R; ++s) w[s - 1] = __ldg(tw + (s - 1) * M + j);
        }
#pragma unroll 1
        for (int f = 0; f < NF; ++f) {
            float2 x[R];
#pragma unroll
            for (int q = 0; q < R; ++q) x[q] = buf[f * P + j + q * M];
            if (j > 0) {
#pragma unroll
                for (int s = 1; s < R; ++s) x[s] = mr_twiddle<true>(x[s], w[s - 1]);
            }
            mr_dft<R, true>(x);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const float v = __ldg(tab2 + j + q * M);
                x[q].x *= v;
                x[q].y *= v;
            }
            mr_dft<R, false>(x);
            if (j > 0) {
#pragma unroll
                for (int s = 1; s < R; ++s) x[s] = mr_twiddle<false>(x[s], w[s - 1]);
            }
#pragma unroll
            for (int q = 0; q < R; ++q) buf[f * P + j + q * M] = x[q];
        }
    }
    __syncthreads();
}

// NF transforms X_k = sum_n x_n e^{-+2 pi i n k / P} (unnormalised): x_n = ld(f, n)
// in natural order, X_k handed to st(f, rev[k], X_k).  The block synchronises
// at the end of every pass.
template <int P, bool INV, int NF, class LD, class ST>
__device__ __forceinline__ void mr_fft_dif(float2 *buf, const float2 *tw, LD ld, ST st)
{
    static_assert(mr_factors(P).n > 0, "P must factor into 3, 5, 7, 9, 11, 13");
    mr_run<P, 0, false, INV, NF>(buf, tw, ld, st);
}
template <int P, bool INV, int NF> __device__ __forceinline__ void mr_fft_dif(float2 *buf, const float2 *tw)
{
    mr_fft_dif<P, INV, NF>(buf, tw, MrSmem<P>{buf}, MrSmem<P>{buf});
}
// The same transforms from X_k = ld(f, rev[k]), natural order out: st(f, n, x_n).
template <int P, bool INV, int NF, class LD, class ST>
__device__ __forceinline__ void mr_fft_dit(float2 *buf, const float2 *tw, LD ld, ST st)
{
    static_assert(mr_factors(P).n > 0, "P must factor into 3, 5, 7, 9, 11, 13");
    mr_run<P, mr_factors(P).n - 1, true, INV, NF>(buf, tw, ld, st);
}

// ---------------------------------------------------------------- S1 / S6 for real maps
// Four rings per block, packed two by two as two complex sequences
// z = f(theta_a, .) + i f(theta_b, .); the spectra are written (read) order-major,
// F[b][m][t], t contiguous, so no transpose pass is needed: the four rings of a
// block are 32 contiguous bytes of every order's row.  Three blocks fit an SM.
constexpr int MR_RINGS = 4;
constexpr int MR_THREADS = 256;
template <int P> constexpr size_t mr_ring_smem() { return (size_t)(MR_RINGS / 2) * P * sizeof(float2); }

// F_m(theta_t) = scale sum_p f(theta_t, phi_p) e^{-i m phi_p}, m < N; grid (ceil(N/4), maps)
template <int P>
__global__ void __launch_bounds__(MR_THREADS, 3) k_ring_fwd_real_mr(const float *__restrict__ f,
                                                                    float2 *__restrict__ F, float scale, MrTab T)
{
    constexpr int N = (P + 1) / 2, NF = MR_RINGS / 2;
    extern __shared__ __align__(16) float2 mr_buf[];
    const int b = blockIdx.y, t0 = blockIdx.x * MR_RINGS;
    const float *src = f + (size_t)b * N * P;
    // the first pass reads the ring pairs from global memory
    auto ld = [&](int q, int p) -> float2 {
        const int ta = t0 + 2 * q;
        const float re = ta < N ? src[(size_t)ta * P + p] : 0.f;
        const float im = ta + 1 < N ? src[(size_t)(ta + 1) * P + p] : 0.f;
        return make_float2(re, im);
    };
    mr_fft_dif<P, false, NF>(mr_buf, T.tw, ld, MrSmem<P>{mr_buf});
    // X_a(m) = (Z_m + conj Z_{P-m}) / 2, X_b(m) = (Z_m - conj Z_{P-m}) / (2i)
    const float s = 0.5f * scale;
    float2 *out = F + (size_t)b * N * N;
    for (int i = threadIdx.x; i < N * NF; i += blockDim.x) {
        const int m = i / NF, q = i - m * NF;
        const int ta = t0 + 2 * q;
        if (ta >= N) continue;
        const float2 zk = mr_buf[q * P + __ldg(T.rev + m)];
        const float2 zp = mr_buf[q * P + __ldg(T.rev + (m ? P - m : 0))];
        const float2 xa = make_float2((zk.x + zp.x) * s, (zk.y - zp.y) * s);
        const float2 xb = make_float2((zk.y + zp.y) * s, (zp.x - zk.x) * s);
        float2 *o = out + (size_t)m * N + ta;
        if ((N & 1) == 0) {                      // ta + 1 < N and 16-byte alignment
            *reinterpret_cast<float4 *>(o) = make_float4(xa.x, xa.y, xb.x, xb.y);
        } else {
            o[0] = xa;
            if (ta + 1 < N) o[1] = xb;
        }
    }
}

// f(theta_t, phi_p) = scale sum_m F_m(theta_t) e^{i m phi_p} with F_{-m} = conj F_m:
// the spectra go to their permuted positions, the transposed passes bring the
// samples out in natural order and the last one writes them to the map rows.
template <int P>
__global__ void __launch_bounds__(MR_THREADS, 3) k_ring_inv_real_mr(const float2 *__restrict__ F,
                                                                    float *__restrict__ f, float scale, MrTab T)
{
    constexpr int N = (P + 1) / 2, NF = MR_RINGS / 2;
    extern __shared__ __align__(16) float2 mr_buf[];
    const int b = blockIdx.y, t0 = blockIdx.x * MR_RINGS;
    const float2 *in = F + (size_t)b * N * N;
    for (int i = threadIdx.x; i < N * NF; i += blockDim.x) {
        const int m = i / NF, q = i - m * NF;
        const int ta = t0 + 2 * q;
        float2 xa = make_float2(0.f, 0.f), xb = xa;
        const float2 *s = in + (size_t)m * N + ta;
        if ((N & 1) == 0 && ta < N) {
            const float4 v = *reinterpret_cast<const float4 *>(s);
            xa = make_float2(v.x, v.y);
            xb = make_float2(v.z, v.w);
        } else {
            if (ta < N) xa = s[0];
            if (ta + 1 < N) xb = s[1];
        }
        // Z_m = xa + i xb, Z_{P-m} = conj(xa) + i conj(xb)
        mr_buf[q * P + __ldg(T.rev + m)] = make_float2(xa.x - xb.y, xa.y + xb.x);
        if (m) mr_buf[q * P + __ldg(T.rev + P - m)] = make_float2(xa.x + xb.y, xb.x - xa.y);
    }
    __syncthreads();
    float *dst = f + (size_t)b * N * P;
    auto st = [&](int q, int p, float2 z) {
        const int ta = t0 + 2 * q;
        if (ta < N) dst[(size_t)ta * P + p] = z.x * scale;
        if (ta + 1 < N) dst[(size_t)(ta + 1) * P + p] = z.y * scale;
    };
    mr_fft_dit<P, true, NF>(mr_buf, T.tw, MrSmem<P>{mr_buf}, st);
}

// ---------------------------------------------------------------- S2: theta quadrature
// The MW quadrature of one column x_t = F_m(theta_t), t < N (parity sigma =
// (-1)^m), as four length-P DFTs.  On the 2P-point grid phi_u = pi u / P the
// product of two trigonometric polynomials of degree N - 1 is integrated exactly
// against sin(theta) on [0, pi] by real weights v_u (their Fourier coefficients
// are w(c) = int_0^pi e^{i c theta} sin(theta) dtheta for |c| <= P - 1).  The odd
// points phi_{2t+1} are the rings theta_t; the even points are the rings shifted
// by -pi/P, where band-limited values come from the shift K (DFT, phase
// e^{-i a pi/P}, inverse DFT).  So with the extension x~ to the circle
//   G~ = v_odd * x~ + K^T (v_even * (K x~)),   K^T = shift by +pi/P,
// and the fold G_t = G~_t + sigma G~_{P-1-t} (t < N - 1) gives the same linear map
// as the dense G = Q_sigma F (both are fixed by the integrals against every
// trigonometric polynomial of degree N - 1).  With x~_{P-1-t} = sigma x_t the
// v_odd term folds to vfold_t x_t.  The products with the phases and weights
// ride on the last pass of each transform; the extension on the first.
//
// Two columns per transform.  Write v = v_s + v_a with v_a = (pi/2) sin(phi), the
// part odd under the reflection t -> P - 1 - t.  The shifted-grid product with v_s
// alone, W = K^T diag(v_s) K, commutes with the reflection, so it keeps the
// symmetric and antisymmetric parts of its input apart: a column e of parity +1
// and a column o of parity -1 (adjacent orders) share one transform of
//   z = ext_+(e) + ext_-(o)   (z_t = e_t + o_t, z_{P-1-t} = e_t - o_t, t < N),
// and w = W z splits by the reflection.  ext_-(o) is antisymmetric except at the
// fixed point t = N - 1, where it holds d = o_{N-1}; that part, d delta_{N-1}, is
// symmetric, and so is the v_a part of the full product applied to ext_-(o) off the
// pole.  With the pole-ring columns qd = W delta_{N-1} and qa = 2 K^T diag(v_a) K
// delta_{N-1} (antisymmetric; tables of the plan), for t < N - 1:
//   G_e,t = w_t + w_{P-1-t} - 2 d qd_t + vfold_t e_t
//   G_o,t = w_t - w_{P-1-t} + d qa_t + vfold_t o_t
// and at the pole ring
//   G_e,N-1 = w_{N-1} - d qd_{N-1} + vfold_{N-1} e_{N-1}
//   G_o,N-1 = d (qd_{N-1} + vfold_{N-1}) + sum_{t < N-1} qa_t o_t,
// the same linear map per column as one transform each, at half the transforms.
//
// In FP32 the FFT form spreads each column's rounding error evenly over theta,
// where the dense product keeps it local; for the smallest orders, whose
// Legendre functions are largest at the poles, that raised the error of the
// finest wavelet maps at L = 2048 near the poles tenfold, to 1.8e-5.  So the
// orders |m| <= MR_QUAD_DENSE_M stay with the dense product (measured at L =
// 2048: 8.6e-7 with that split, 1.1e-6 all dense) and this kernel takes the rest.
// CPB transforms per block; map b has K columns r = 0..K-1, the rows [b][mi] of
// the order-major spectra with mi = mstart + r + (r >= seg0 ? gap : 0) (m = mi -
// m_offset), in two segments [0, seg0) and [seg0, K) of consecutive orders.
// Transform (unit) uu of a map takes columns r0 = 2 uu and r0 + 1 of the first
// segment (uu < useg = ceil(seg0 / 2)), else r0 = seg0 + 2 (uu - useg) and r0 + 1
// of the second; the second column is absent past its segment's end.
constexpr int MR_QUAD_DENSE_M = 32;
template <int P> constexpr int mr_quad_cpb() { return P > 2048 ? 2 : 8; }
template <int P> constexpr size_t mr_quad_smem() { return (size_t)mr_quad_cpb<P>() * P * sizeof(float2); }

struct MrCols {
    int nmi, m_offset, K, mstart, seg0, gap;
    int useg, upm, nunits;           // units in the first segment, per map, in all
};

template <int P>
__global__ void __launch_bounds__(MR_THREADS, 3) k_quad_mr(const float2 *__restrict__ Fin, float2 *__restrict__ Gout,
                                                           MrCols C, MrTab T)
{
    constexpr int N = (P + 1) / 2, CPB = mr_quad_cpb<P>(), NW = MR_THREADS / 32;
    extern __shared__ __align__(16) float2 mr_buf[];
    __shared__ int rowe[CPB], rowo[CPB];      // rows of the parity +1 and -1 columns, -1 if absent
    __shared__ float2 red[CPB][NW];
    if (threadIdx.x < CPB) {
        const int u = blockIdx.x * CPB + threadIdx.x;
        int re = -1, ro = -1;
        if (u < C.nunits) {
            const int b = u / C.upm, uu = u - b * C.upm;
            const bool first = uu < C.useg;
            const int r0 = first ? 2 * uu : C.seg0 + 2 * (uu - C.useg);
            const int rend = first ? C.seg0 : C.K;
            const int mi0 = C.mstart + r0 + (first ? 0 : C.gap);
            const int row0 = b * C.nmi + mi0, row1 = r0 + 1 < rend ? row0 + 1 : -1;
            const bool odd0 = ((mi0 - C.m_offset) & 1) != 0;
            re = odd0 ? row1 : row0;
            ro = odd0 ? row0 : row1;
        }
        rowe[threadIdx.x] = re;
        rowo[threadIdx.x] = ro;
    }
    __syncthreads();
    const MrSmem<P> sm{mr_buf};
    // z = ext_+(e) + ext_-(o), read from global memory by the first pass
    auto ext = [&](int q, int t) -> float2 {
        const int re = rowe[q], ro = rowo[q];
        const int tt = t < N ? t : P - 1 - t;
        const float2 e = re >= 0 ? Fin[(size_t)re * N + tt] : make_float2(0.f, 0.f);
        const float2 o = ro >= 0 ? Fin[(size_t)ro * N + tt] : make_float2(0.f, 0.f);
        return t < N ? make_float2(e.x + o.x, e.y + o.y) : make_float2(e.x - o.x, e.y - o.y);
    };
    constexpr int NP = mr_factors(P).n;
    if constexpr (NP >= 2) {
        // the junctions between the four transforms as fused passes (three fewer
        // round trips through shared memory)
        mr_run_range<P, 0, NP - 2, false, false, CPB>(mr_buf, T.tw, ext, sm, 0);
        mr_pass_dif_last_dit_first<P, CPB>(mr_buf, T.shm);          // K: phases
        mr_run_range<P, NP - 2, 1, true, true, CPB>(mr_buf, T.tw, sm, sm, NP - 2);
        mr_pass_dit_last_dif_first<P, CPB>(mr_buf, T.tw, T.ve);     // (1/P in ve) weights
        mr_run_range<P, 1, NP - 2, false, false, CPB>(mr_buf, T.tw, sm, sm, 1);
        mr_pass_dif_last_dit_first<P, CPB>(mr_buf, T.shp);          // K^T: phases (with 1/P)
        mr_run_range<P, NP - 2, 0, true, true, CPB>(mr_buf, T.tw, sm, sm, NP - 2);
    } else {
        mr_fft_dif<P, false, CPB>(mr_buf, T.tw, ext, [&](int q, int pos, float2 v) {
            mr_buf[q * P + pos] = mr_twiddle<false>(v, __ldg(T.shm + pos));
        });
        // (its 1/P is in ve) times the weights of the shifted points
        mr_fft_dit<P, true, CPB>(mr_buf, T.tw, sm, [&](int q, int t, float2 v) {
            const float w = __ldg(T.ve + t);
            mr_buf[q * P + t] = make_float2(v.x * w, v.y * w);
        });
        // K^T: DFT, conjugate phases (with 1/P), inverse DFT
        mr_fft_dif<P, false, CPB>(mr_buf, T.tw, sm, [&](int q, int pos, float2 v) {
            mr_buf[q * P + pos] = mr_twiddle<false>(v, __ldg(T.shp + pos));
        });
        mr_fft_dit<P, true, CPB>(mr_buf, T.tw, sm, sm);
    }
    // split by the reflection, fold, pole-ring terms and the odd-point term
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = 0; q < CPB; ++q) {
        const int re = rowe[q], ro = rowo[q];
        float2 acc = make_float2(0.f, 0.f);
        if (re >= 0 || ro >= 0) {
            const float2 d = ro >= 0 ? Fin[(size_t)ro * N + N - 1] : make_float2(0.f, 0.f);
            for (int t = threadIdx.x; t < N; t += blockDim.x) {
                const float2 w = mr_buf[q * P + t];
                const float vf = __ldg(T.vfold + t), qd = __ldg(T.qd + t);
                if (t < N - 1) {
                    const float2 h = mr_buf[q * P + P - 1 - t];
                    if (re >= 0) {
                        const float2 e = Fin[(size_t)re * N + t];
                        Gout[(size_t)re * N + t] = make_float2(fmaf(vf, e.x, fmaf(-2.f * qd, d.x, w.x + h.x)),
                                                               fmaf(vf, e.y, fmaf(-2.f * qd, d.y, w.y + h.y)));
                    }
                    if (ro >= 0) {
                        const float2 o = Fin[(size_t)ro * N + t];
                        const float qa = __ldg(T.qa + t);
                        Gout[(size_t)ro * N + t] = make_float2(fmaf(vf, o.x, fmaf(qa, d.x, w.x - h.x)),
                                                               fmaf(vf, o.y, fmaf(qa, d.y, w.y - h.y)));
                        acc.x = fmaf(qa, o.x, acc.x);
                        acc.y = fmaf(qa, o.y, acc.y);
                    }
                } else if (re >= 0) {
                    const float2 e = Fin[(size_t)re * N + t];
                    Gout[(size_t)re * N + t] = make_float2(fmaf(vf, e.x, fmaf(-qd, d.x, w.x)),
                                                           fmaf(vf, e.y, fmaf(-qd, d.y, w.y)));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) red[q][warp] = acc;
    }
    __syncthreads();
    // the pole ring of each parity -1 column: warp partial sums in a fixed order
    if (threadIdx.x < CPB && rowo[threadIdx.x] >= 0) {
        const int q = threadIdx.x, ro = rowo[q];
        float2 s = red[q][0];
        for (int i = 1; i < NW; ++i) {
            s.x += red[q][i].x;
            s.y += red[q][i].y;
        }
        const float2 d = Fin[(size_t)ro * N + N - 1];
        const float c = __ldg(T.qd + N - 1) + __ldg(T.vfold + N - 1);
        Gout[(size_t)ro * N + N - 1] = make_float2(fmaf(c, d.x, s.x), fmaf(c, d.y, s.y));
    }
}

}  // namespace s2g
