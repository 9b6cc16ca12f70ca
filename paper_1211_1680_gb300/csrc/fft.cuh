// Ring DFTs (length P = 2N-1, any N) and the MW theta-quadrature, built on
// one shared-memory power-of-two FFT and Bluestein's chirp-z identity
// (Bluestein 1970):  nk = (n^2 + k^2 - (k-n)^2)/2, so a length-P DFT is a
// circular convolution of length M >= 2P-1 with the chirp c_n = e^{i pi n^2/P}.
//
// Tables per band-limit N (all precomputed on the host in FP64):
//   chirp[n]  = e^{i pi n^2 / P},               n < P
//   bhat[k]   = FFT_M(b), b_j = chirp_|j| for |j| < P (indices mod M), stored bit-reversed
//   what[k]   = FFT_M(v), v_s = w(s) = int_0^pi e^{i s theta} sin theta dtheta, |s| <= 2N-2,
//               stored bit-reversed
//   tw        per-stage twiddles, stacked: tw[M - 2h + k] = e^{-2 pi i k/(2h)}, k < h,
//             for h = M/2, M/4, ..., 1 (M - 1 entries), so that the threads of a
//             stage read consecutive (or equal) entries
//   phase[k+N-1] = e^{i pi k / P},              |k| <= N-1
// M = next power of two >= max(4N-3, 2) serves both the Bluestein DFTs and
// the w-convolution (|a+b| <= 2N-2 for |a|, |b| <= N-1 needs M >= 4N-3).
#pragma once
#include "common.cuh"

namespace s2g {

// Shared-memory index with one padding element after every 16, which breaks
// the power-of-two strides of the late FFT stages across the banks.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int M) { return M + (M >> 4); }

template <typename C> struct FftTab {
    const C *chirp;
    const C *bhat;
    const C *bhat_g;   // bhat in the order of the fused middle pass: bhat_g[q (M/R) + j] = bhat[R j + q]
    const C *what;
    const C *tw;
    const C *phase;
    int N, P, M, logM;
};

// In-place radix-2 FFTs of length M in shared memory, without a permutation
// pass: the forward transform is decimation in frequency (natural-order input,
// bit-reversed output), the inverse is decimation in time (bit-reversed input,
// natural-order output), and the pointwise product between them uses kernel
// tables stored in bit-reversed order.  Unnormalised.
// Stages are fused RB at a time (RB <= 3): a thread loads the 2^RB elements one
// butterfly group of the fused stages touches, runs the RB radix-2 stages in
// registers and stores them back, so shared memory is read and written once per
// three stages.  The arithmetic and the output order are those of the plain
// radix-2 algorithms.
// Twiddles.  Stage half-size `half` multiplies by tw[M - 2 half + (pos mod
// half)] = e^{-2 pi i (pos mod half) / (2 half)}.  Within a radix-8 group
// (elements base + q sub, base = k mod sub) the twelve twiddles of its three
// stages are three table entries times eighth roots of unity, so a group loads
// three values and forms the rest with a multiplication by (1 - i)/sqrt(2) or
// exact multiplications by -i.
template <typename C> __device__ __forceinline__ C mul_mi(C w) { return mk(w.y, -w.x); }       // -i w
template <typename C> __device__ __forceinline__ C mul_w8(C w)                                // e^{-i pi/4} w
{
    using R = decltype(w.x);
    const R h = (R)0.70710678118654752440;
    return mk((w.x + w.y) * h, (w.y - w.x) * h);
}
// e^{-2 pi i e / 16}, e = 0..7 (constants: cos and sin of multiples of pi/8)
template <typename C> __device__ __forceinline__ C w16(int e)
{
    using R = decltype(C().x);
    const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, r2 = (R)0.70710678118654752440;
    switch (e) {
    case 0: return mk((R)1, (R)0);
    case 1: return mk(c1, -s1);
    case 2: return mk(r2, -r2);
    case 3: return mk(s1, -c1);
    case 4: return mk((R)0, (R)-1);
    case 5: return mk(-s1, -c1);
    case 6: return mk(-r2, -r2);
    default: return mk(-c1, -s1);
    }
}

// RB DIF stages on a group x[q] = a[base + q sub], first half-size h (sub = h / 2^(RB-1)).
template <typename C, int RB>
__device__ __forceinline__ void dif_group(C (&x)[1 << RB], int M, int h, int base, int sub, const C *__restrict__ tw)
{
    constexpr int R = 1 << RB;
    if constexpr (RB == 3) {
        const int k = base & (sub - 1);
        const C W = tw[M - 2 * h + k], W2 = tw[M - h + k], W4 = tw[M - h / 2 + k];
        const C w0[4] = {W, mul_w8(W), mul_mi(W), mul_mi(mul_w8(W))};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const C u = x[q], v = x[q + 4];
            x[q] = cadd(u, v);
            x[q + 4] = cmul(csub(u, v), w0[q]);
        }
        const C w1[2] = {W2, mul_mi(W2)};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q & 2) continue;
            const C u = x[q], v = x[q + 2];
            x[q] = cadd(u, v);
            x[q + 2] = cmul(csub(u, v), w1[q & 1]);
        }
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            const C u = x[q], v = x[q + 1];
            x[q] = cadd(u, v);
            x[q + 1] = cmul(csub(u, v), W4);
        }
    } else {
#pragma unroll
        for (int t = 0; t < RB; ++t) {
            const int half = h >> t;
            const int span = R >> (t + 1);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (q & span) continue;
                const int pos = base + q * sub;
                const C u = x[q], v = x[q + span];
                x[q] = cadd(u, v);
                x[q + span] = cmul(csub(u, v), tw[M - 2 * half + (pos & (half - 1))]);
            }
        }
    }
}

// RB DIT stages on a group x[q] = a[base + q sub], first half-size sub.
template <typename C, int RB>
__device__ __forceinline__ void dit_group(C (&x)[1 << RB], int M, int base, int sub, const C *__restrict__ tw)
{
    constexpr int R = 1 << RB;
    if constexpr (RB == 3) {
        const int k = base & (sub - 1);
        const C T1 = tw[M - 2 * sub + k], T2 = tw[M - 4 * sub + k], T4 = tw[M - 8 * sub + k];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            const C u = x[q], v = cmulc(x[q + 1], T1);
            x[q] = cadd(u, v);
            x[q + 1] = csub(u, v);
        }
        const C w1[2] = {T2, mul_mi(T2)};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q & 2) continue;
            const C u = x[q], v = cmulc(x[q + 2], w1[q & 1]);
            x[q] = cadd(u, v);
            x[q + 2] = csub(u, v);
        }
        const C w2[4] = {T4, mul_w8(T4), mul_mi(T4), mul_mi(mul_w8(T4))};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const C u = x[q], v = cmulc(x[q + 4], w2[q]);
            x[q] = cadd(u, v);
            x[q + 4] = csub(u, v);
        }
    } else {
#pragma unroll
        for (int t = 0; t < RB; ++t) {
            const int half = sub << t;
            const int span = 1 << t;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (q & span) continue;
                const int pos = base + q * sub;
                const C u = x[q];
                const C v = cmulc(x[q + span], tw[M - 2 * half + (pos & (half - 1))]);
                x[q] = cadd(u, v);
                x[q + span] = csub(u, v);
            }
        }
    }
}

// DIF pass over stages s .. s+RB-1 (first half h = 2^(logM-s)).
template <typename C, int RB>
__device__ __forceinline__ void dif_pass(C *a, int M, int logM, int s, const C *__restrict__ tw)
{
    constexpr int R = 1 << RB;
    const int h = 1 << (logM - s);
    const int sub = h >> (RB - 1);            // distance between the group's elements
    for (int j = threadIdx.x; j < M / R; j += blockDim.x) {
        const int g = j / sub, k = j - g * sub;
        const int base = g * 2 * h + k;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = a[pad16(base + q * sub)];
        dif_group<C, RB>(x, M, h, base, sub, tw);
#pragma unroll
        for (int q = 0; q < R; ++q) a[pad16(base + q * sub)] = x[q];
    }
    __syncthreads();
}

// DIT pass over stages s .. s+RB-1 (first half 2^(s-1)).
template <typename C, int RB>
__device__ __forceinline__ void dit_pass(C *a, int M, int logM, int s, const C *__restrict__ tw)
{
    constexpr int R = 1 << RB;
    const int sub = 1 << (s - 1);             // distance between the group's elements
    const int block = sub * R;
    for (int j = threadIdx.x; j < M / R; j += blockDim.x) {
        const int g = j / sub, k = j - g * sub;
        const int base = g * block + k;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = a[pad16(base + q * sub)];
        dit_group<C, RB>(x, M, base, sub, tw);
#pragma unroll
        for (int q = 0; q < R; ++q) a[pad16(base + q * sub)] = x[q];
    }
    __syncthreads();
}

// fft_dif: b_k = sum_j a_j e^{-2 pi i jk/M}, stored at position bitrev(k).
template <typename C>
__device__ void fft_dif(C *a, int M, int logM, const C *__restrict__ tw)
{
    int s = 1;
    for (; s + 2 <= logM; s += 3) dif_pass<C, 3>(a, M, logM, s, tw);
    if (s + 1 <= logM) {
        dif_pass<C, 2>(a, M, logM, s, tw);
        s += 2;
    }
    if (s <= logM) dif_pass<C, 1>(a, M, logM, s, tw);
}

// ifft_dit: a_j = sum_k b_k e^{+2 pi i jk/M} from b stored in bit-reversed order.
template <typename C>
__device__ void ifft_dit(C *a, int M, int logM, const C *__restrict__ tw)
{
    int s = 1;
    for (; s + 2 <= logM; s += 3) dit_pass<C, 3>(a, M, logM, s, tw);
    if (s + 1 <= logM) {
        dit_pass<C, 2>(a, M, logM, s, tw);
        s += 2;
    }
    if (s <= logM) dit_pass<C, 1>(a, M, logM, s, tw);
}

// buf := IFFT_M( FFT_M(buf) * K ), K = khat or conj(khat) (khat stored bit-reversed); unnormalised.
template <typename C, bool CONJ_K>
__device__ void conv_core(C *buf, const FftTab<C> &T, const C *__restrict__ khat)
{
    __syncthreads();
    fft_dif<C>(buf, T.M, T.logM, T.tw);
    for (int i = threadIdx.x; i < T.M; i += blockDim.x) {
        C k = khat[i];
        const int pi = pad16(i);
        buf[pi] = CONJ_K ? cmulc(buf[pi], k) : cmul(buf[pi], k);
    }
    __syncthreads();
    ifft_dit<C>(buf, T.M, T.logM, T.tw);
}

// ---------------------------------------------------------------- fused convolution
// The same convolution with fewer passes over shared memory (used by the ring
// DFTs): the first DIF pass takes its elements from load(pos) (zero padding
// included) instead of shared memory, the last RBF DIF stages, the pointwise
// product with the kernel table and the first RBF DIT stages run in one pass
// (both act on contiguous groups of 2^RBF in the bit-reversed order), and the
// last DIT pass hands its results to store(pos, value) instead of shared
// memory.  For M = 2^logM with logM >= RBF + 1.
template <typename C, int RB, typename LoadF>
__device__ __forceinline__ void dif_pass_load(C *a, int M, int logM, const C *__restrict__ tw, LoadF load)
{
    constexpr int R = 1 << RB;
    const int h = M >> 1;
    const int sub = h >> (RB - 1);
    for (int j = threadIdx.x; j < M / R; j += blockDim.x) {
        const int g = j / sub, k = j - g * sub;
        const int base = g * 2 * h + k;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = load(base + q * sub);
        dif_group<C, RB>(x, M, h, base, sub, tw);
#pragma unroll
        for (int q = 0; q < R; ++q) a[pad16(base + q * sub)] = x[q];
    }
    __syncthreads();
}

// last RB DIF stages, product with the kernel table (bit-reversed positions,
// stored group-major: entry q of group j at khat[q (M / 2^RB) + j]), first RB DIT
// stages.  The group starts at a multiple of 2^RB, so its twiddles are the
// 2^RB-th roots of unity e^{-2 pi i (q mod half)/(2 half)} = w16((q mod half) 8 / half).
template <typename C, int RB, bool CONJ_K>
__device__ __forceinline__ void mid_pass(C *a, int M, const C *__restrict__ khat)
{
    constexpr int R = 1 << RB;
    static_assert(RB <= 4, "sixteenth roots of unity only");
    for (int j = threadIdx.x; j < M / R; j += blockDim.x) {
        const int base = j * R;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = a[pad16(base + q)];
#pragma unroll
        for (int t = 0; t < RB; ++t) {            // DIF, half = R/2 ... 1
            const int half = R >> (t + 1);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (q & half) continue;
                const C u = x[q], v = x[q + half];
                x[q] = cadd(u, v);
                const C d = csub(u, v);
                const int e = (q & (half - 1)) * (8 / half);
                x[q + half] = e == 0 ? d : (e == 4 ? mul_mi(d) : cmul(d, w16<C>(e)));
            }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const C k = khat[q * (M / R) + j];           // group-major table: coalesced over j
            x[q] = CONJ_K ? cmulc(x[q], k) : cmul(x[q], k);
        }
#pragma unroll
        for (int t = 0; t < RB; ++t) {            // DIT, half = 1 ... R/2
            const int half = 1 << t;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (q & half) continue;
                const int e = (q & (half - 1)) * (8 / half);
                const C u = x[q];
                const C v = e == 0 ? x[q + half] : cmulc(x[q + half], w16<C>(e));
                x[q] = cadd(u, v);
                x[q + half] = csub(u, v);
            }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) a[pad16(base + q)] = x[q];
    }
    __syncthreads();
}

// DIT pass over stages s .. logM (RB = logM - s + 1) handing results to store(pos, value)
template <typename C, int RB, typename StoreF>
__device__ __forceinline__ void dit_pass_store(const C *a, int M, int logM, const C *__restrict__ tw, StoreF store)
{
    constexpr int R = 1 << RB;
    const int sub = M >> RB;
    for (int j = threadIdx.x; j < sub; j += blockDim.x) {
        const int base = j;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = a[pad16(base + q * sub)];
        dit_group<C, RB>(x, M, base, sub, tw);
#pragma unroll
        for (int q = 0; q < R; ++q) store(base + q * sub, x[q]);
    }
}

template <typename C, int RB, typename LoadF>
__device__ __forceinline__ void dif_first(C *a, int M, int logM, const C *tw, LoadF load, int rb)
{
    if (rb == 3) dif_pass_load<C, 3>(a, M, logM, tw, load);
    else if (rb == 2) dif_pass_load<C, 2>(a, M, logM, tw, load);
    else dif_pass_load<C, 1>(a, M, logM, tw, load);
}

// out(pos, v) receives IFFT_M( FFT_M(x) * K ) at every position pos < M, where
// x_pos = load(pos); K = khat or conj(khat) (bit-reversed).  Unnormalised.
// The middle pass runs FFT_RBF stages each way (radix 16) in single precision,
// three (radix 8) in double precision, where registers are twice as wide.
constexpr int FFT_RBF = 4;
template <typename C> constexpr int fft_rbf() { return sizeof(C) == 16 ? 3 : FFT_RBF; }
template <typename C, bool CONJ_K, typename LoadF, typename StoreF>
__device__ void conv_fused(C *buf, const FftTab<C> &T, const C *__restrict__ khat, LoadF load, StoreF store)
{
    constexpr int RBF = fft_rbf<C>();
    const int M = T.M, logM = T.logM;
    const int D = logM - RBF;                     // DIF (and DIT) stages outside the middle pass, >= 1
    const int rb1 = (D - 1) % 3 + 1;              // first DIF pass: 1..3 stages, then passes of 3
    dif_first<C, 3>(buf, M, logM, T.tw, load, rb1);
    for (int s = 1 + rb1; s <= D; s += 3) dif_pass<C, 3>(buf, M, logM, s, T.tw);
    mid_pass<C, RBF, CONJ_K>(buf, M, khat);
    const int rbl = (D - 1) % 3 + 1;              // last DIT pass: 1..3 stages, before it passes of 3
    for (int s = RBF + 1; s <= logM - rbl; s += 3) dit_pass<C, 3>(buf, M, logM, s, T.tw);
    if (rbl == 3) dit_pass_store<C, 3>(buf, M, logM, T.tw, store);
    else if (rbl == 2) dit_pass_store<C, 2>(buf, M, logM, T.tw, store);
    else dit_pass_store<C, 1>(buf, M, logM, T.tw, store);
}

template <typename R> __device__ __forceinline__ R inv_m(int M) { return (R)1 / (R)M; }

// Ring-DFT blocks have at most FFT_MAX_THREADS threads (M/16 for M <= 8192);
// single-precision kernels are built for two resident blocks per SM.
constexpr int FFT_MAX_THREADS = 512;

// ---------------------------------------------------------------- spectrum transposes
// The ring DFTs work on one ring (or two) per block, so they read and write
// spectra ring-major, Ft[b][t][mi] (orders contiguous); the theta quadrature and
// the Legendre stages use order-major spectra, F[b][mi][t] (rings contiguous).
// out[b][c][r] = in[b][r][c] for rows x cols matrices, through 32 x 32 tiles
// in shared memory (block 32 x 8 threads; grid (cols/32, rows/32, batch)).
template <typename C>
__global__ void __launch_bounds__(256) k_transpose(const C *__restrict__ in, C *__restrict__ out, int rows, int cols)
{
    __shared__ C tile[32][33];
    const size_t mat = (size_t)rows * cols;
    const C *src = in + blockIdx.z * mat;
    C *dst = out + blockIdx.z * mat;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
        const int r = r0 + ty + i, c = c0 + tx;
        if (r < rows && c < cols) tile[ty + i][tx] = src[(size_t)r * cols + c];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
        const int c = c0 + ty + i, r = r0 + tx;
        if (r < rows && c < cols) dst[(size_t)c * rows + r] = tile[tx][ty + i];
    }
}

// ---------------------------------------------------------------- S1: ring DFT
// F_m(theta_t) = scale * sum_p f(theta_t, phi_p) e^{-i m phi_p}, phi_p = 2 pi p / P.
// Real maps: two rings per block packed as one complex sequence, m = 0..N-1,
// written to Ft[b][t][m].  Complex maps: one ring per block, m = -(N-1)..N-1,
// written to Ft[b][t][m + N - 1].
template <typename R>
__global__ void __launch_bounds__(FFT_MAX_THREADS, sizeof(R) == 4 ? 2 : 1) k_ring_fwd_real(const R *__restrict__ f, cplx_t<R> *__restrict__ F, R scale,
                                FftTab<cplx_t<R>> T)
{
    using C = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int N = T.N, P = T.P, M = T.M;
    const int b = blockIdx.y;
    const int t0 = 2 * blockIdx.x, t1 = t0 + 1;
    const bool has1 = t1 < N;
    const R *r0 = f + ((size_t)b * N + t0) * P;
    const R *r1 = f + ((size_t)b * N + (has1 ? t1 : t0)) * P;
    auto load = [&](int n) -> C {
        return n < P ? cmulc(mk(r0[n], has1 ? r1[n] : (R)0), T.chirp[n]) : mk((R)0, (R)0);
    };
    if (T.logM > fft_rbf<C>()) {
        // the transform is read back at positions < P only
        conv_fused<C, false>(buf, T, T.bhat_g, load, [&](int pos, C v) {
            if (pos < P) buf[pad16(pos)] = v;
        });
    } else {
        for (int n = threadIdx.x; n < M; n += blockDim.x) buf[pad16(n)] = load(n);
        __syncthreads();
        conv_core<C, false>(buf, T, T.bhat);
    }
    __syncthreads();
    const R s = scale * inv_m<R>(M) * (R)0.5;
    C *out0 = F + ((size_t)b * N + t0) * N;
    C *out1 = F + ((size_t)b * N + t1) * N;
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        const int mp = (m == 0) ? 0 : P - m;
        C zk = cmulc(buf[pad16(m)], T.chirp[m]);    // conj(c_k) * buf[k]
        C zp = cmulc(buf[pad16(mp)], T.chirp[mp]);
        // X0 = (Zk + conj(Zp)) / 2, X1 = (Zk - conj(Zp)) / (2i)
        out0[m] = mk((zk.x + zp.x) * s, (zk.y - zp.y) * s);
        if (has1) out1[m] = mk((zk.y + zp.y) * s, (zp.x - zk.x) * s);
    }
}

template <typename R>
__global__ void __launch_bounds__(FFT_MAX_THREADS, sizeof(R) == 4 ? 2 : 1) k_ring_fwd_cplx(const cplx_t<R> *__restrict__ f, cplx_t<R> *__restrict__ F, R scale,
                                FftTab<cplx_t<R>> T)
{
    using C = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int N = T.N, P = T.P, M = T.M;
    const int b = blockIdx.y, t = blockIdx.x;
    const C *row = f + ((size_t)b * N + t) * P;
    const R s = scale * inv_m<R>(M);
    const int nm = 2 * N - 1;
    C *out = F + ((size_t)b * N + t) * nm;
    auto load = [&](int n) -> C { return n < P ? cmulc(row[n], T.chirp[n]) : mk((R)0, (R)0); };
    // position k < P holds order m = k (k < N) or m = k - P (k > P - N)
    auto store = [&](int k, C v) {
        if (k >= P || (k >= N && k <= P - N)) return;
        const int mi = (k < N ? k : k - P) + N - 1;
        out[mi] = cscale(cmulc(v, T.chirp[k]), s);
    };
    if (T.logM > fft_rbf<C>()) {
        conv_fused<C, false>(buf, T, T.bhat_g, load, store);
    } else {
        for (int n = threadIdx.x; n < M; n += blockDim.x) buf[pad16(n)] = load(n);
        __syncthreads();
        conv_core<C, false>(buf, T, T.bhat);
        for (int k = threadIdx.x; k < M; k += blockDim.x) store(k, buf[pad16(k)]);
    }
}

// ---------------------------------------------------------------- S6: inverse ring DFT
// f(theta_t, phi_p) = scale * sum_m F_m(theta_t) e^{i m phi_p} from ring-major
// spectra Ft[b][t][mi].  Real maps use F_{-m} = conj(F_m) and pack two rings
// per block.
template <typename R>
__global__ void __launch_bounds__(FFT_MAX_THREADS, sizeof(R) == 4 ? 2 : 1) k_ring_inv_real(const cplx_t<R> *__restrict__ F, R *__restrict__ f, R scale,
                                FftTab<cplx_t<R>> T)
{
    using C = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int N = T.N, P = T.P, M = T.M;
    const int b = blockIdx.y;
    const int t0 = 2 * blockIdx.x, t1 = t0 + 1;
    const bool has1 = t1 < N;
    const C *in0 = F + ((size_t)b * N + t0) * N;
    const C *in1 = F + ((size_t)b * N + (has1 ? t1 : t0)) * N;
    auto load = [&](int k) -> C {
        if (k >= P) return mk((R)0, (R)0);
        const bool neg = k >= N;
        const int m = neg ? P - k : k;
        C a = in0[m];
        C c = has1 ? in1[m] : mk((R)0, (R)0);
        if (neg) {
            a = cconj(a);
            c = cconj(c);
        }
        return cmul(mk(a.x - c.y, a.y + c.x), T.chirp[k]);   // (a + i c) chirp_k
    };
    const R s = scale * inv_m<R>(M);
    R *o0 = f + ((size_t)b * N + t0) * P;
    R *o1 = f + ((size_t)b * N + t1) * P;
    auto store = [&](int p, C v) {
        if (p >= P) return;
        v = cmul(v, T.chirp[p]);
        o0[p] = v.x * s;
        if (has1) o1[p] = v.y * s;
    };
    if (T.logM > fft_rbf<C>()) {
        conv_fused<C, true>(buf, T, T.bhat_g, load, store);
    } else {
        for (int k = threadIdx.x; k < M; k += blockDim.x) buf[pad16(k)] = load(k);
        __syncthreads();
        conv_core<C, true>(buf, T, T.bhat);
        for (int p = threadIdx.x; p < M; p += blockDim.x) store(p, buf[pad16(p)]);
    }
}

template <typename R>
__global__ void __launch_bounds__(FFT_MAX_THREADS, sizeof(R) == 4 ? 2 : 1) k_ring_inv_cplx(const cplx_t<R> *__restrict__ F, cplx_t<R> *__restrict__ f, R scale,
                                FftTab<cplx_t<R>> T)
{
    using C = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int N = T.N, P = T.P, M = T.M;
    const int b = blockIdx.y, t = blockIdx.x;
    const int nm = 2 * N - 1;
    const C *in = F + ((size_t)b * N + t) * nm;
    auto load = [&](int k) -> C {
        if (k >= P) return mk((R)0, (R)0);
        const int m = k < N ? k : k - P;
        return cmul(in[m + N - 1], T.chirp[k]);
    };
    const R s = scale * inv_m<R>(M);
    C *o = f + ((size_t)b * N + t) * P;
    auto store = [&](int p, C v) {
        if (p < P) o[p] = cscale(cmul(v, T.chirp[p]), s);
    };
    if (T.logM > fft_rbf<C>()) {
        conv_fused<C, true>(buf, T, T.bhat_g, load, store);
    } else {
        for (int k = threadIdx.x; k < M; k += blockDim.x) buf[pad16(k)] = load(k);
        __syncthreads();
        conv_core<C, true>(buf, T, T.bhat);
        for (int p = threadIdx.x; p < M; p += blockDim.x) store(p, buf[pad16(p)]);
    }
}

// ---------------------------------------------------------------- S2: theta quadrature
// For one order m and one map: x_t = F_m(theta_t), t < N, parity sigma = (-1)^m.
//  (a) extend to the circle: x~_t = x_t (t < N), x~_t = sigma x_{P-1-t} (N <= t < P)
//  (b) X_a = (1/P) sum_t x~_t e^{-i a theta_t},  theta_t = pi (2t+1)/P, |a| <= N-1
//  (c) H_b = sum_a X_a w(a+b),                    |b| <= N-1
//  (d) h_t = sum_b H_b e^{-i b theta_t},          t < P
//  (e) G_t = qscale (h_t + sigma h_{P-1-t}) for t < N-1, G_{N-1} = qscale h_{N-1}
// e^{-i a theta_t} = e^{-i pi a/P} e^{-2 pi i a t/P}: (b) and (d) are length-P
// DFTs (Bluestein) with a phase; (c) is a circular convolution of length M.
// The linear map x -> G is real and symmetric, so the same kernel also applies
// its transpose.  Q is the compute type (FP64 by default), R the storage type.
// parity < 0: sigma from m = mi - m_offset; parity 0 / 1: sigma = +1 / -1 for every row.
// gbuf: the block's transform buffer in global memory (padded_len(M) values per
// block) instead of shared memory, for lengths whose buffer exceeds it (the
// plan-time FP64 quadrature matrices at N > 2048); VPT >= M / blockDim.x.
template <typename Q, typename R, int VPT>
__global__ void k_theta_quad(const cplx_t<R> *__restrict__ Fin, cplx_t<R> *__restrict__ Gout,
                             int nmi, int m_offset, Q qscale, FftTab<cplx_t<Q>> T, int parity,
                             cplx_t<Q> *gbuf = nullptr)
{
    using C = cplx_t<Q>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = gbuf ? gbuf + (size_t)blockIdx.x * padded_len(T.M) : reinterpret_cast<C *>(smem_raw);
    const int N = T.N, P = T.P, M = T.M;
    const int mi = blockIdx.x, b = blockIdx.y;
    const int m = mi - m_offset;
    const Q sigma = (parity < 0 ? (m & 1) : parity) ? (Q)-1 : (Q)1;
    const cplx_t<R> *x = Fin + ((size_t)b * nmi + mi) * N;
    cplx_t<R> *g = Gout + ((size_t)b * nmi + mi) * N;
    const Q invM = (Q)1 / (Q)M;

    // (a) + pre-chirp of (b)
    for (int n = threadIdx.x; n < M; n += blockDim.x) {
        C v = mk((Q)0, (Q)0);
        if (n < N) {
            v = ccast<C>(x[n]);
        } else if (n < P) {
            v = cscale(ccast<C>(x[P - 1 - n]), sigma);
        }
        if (n < P) v = cmulc(v, T.chirp[n]);
        buf[pad16(n)] = v;
    }
    __syncthreads();
    conv_core<C, false>(buf, T, T.bhat);
    // (b) Y_k = conj(c_k) buf_k / M;  X_a = (1/P) e^{-i pi a/P} Y_{a mod P}
    // (c) input U_k = X_{-k} = (1/P) e^{i pi k/P} Y_{(-k) mod P} at k mod M, |k| <= N-1
    C hold[VPT];
    {
        const Q s = invM / (Q)P;
        int r = 0;
        for (int j = threadIdx.x; j < M; j += blockDim.x, ++r) {
            int k;
            bool ok = true;
            if (j <= N - 1) k = j;
            else if (j >= M - (N - 1)) k = j - M;
            else { k = 0; ok = false; }
            C v = mk((Q)0, (Q)0);
            if (ok) {
                int src = (-k) % P;
                if (src < 0) src += P;
                v = cmul(cmulc(buf[pad16(src)], T.chirp[src]), T.phase[k + N - 1]);
                v = cscale(v, s);
            }
            hold[r] = v;
        }
        __syncthreads();
        r = 0;
        for (int j = threadIdx.x; j < M; j += blockDim.x, ++r) buf[pad16(j)] = hold[r];
        __syncthreads();
    }
    conv_core<C, false>(buf, T, T.what);
    // H_b = buf[b mod M] / M;  (d) pre-chirp: z_n = H_b e^{-i pi b/P} conj(c_n), n = b mod P
    {
        int r = 0;
        for (int n = threadIdx.x; n < M; n += blockDim.x, ++r) {
            C v = mk((Q)0, (Q)0);
            if (n < P) {
                const int bb = (n <= N - 1) ? n : n - P;
                const int src = bb >= 0 ? bb : bb + M;
                v = cmulc(cscale(buf[pad16(src)], invM), T.phase[bb + N - 1]);   // H_b e^{-i pi b/P}
                v = cmulc(v, T.chirp[n]);
            }
            hold[r] = v;
        }
        __syncthreads();
        r = 0;
        for (int n = threadIdx.x; n < M; n += blockDim.x, ++r) buf[pad16(n)] = hold[r];
        __syncthreads();
    }
    conv_core<C, false>(buf, T, T.bhat);
    // h_t = conj(c_t) buf_t / M; (e) fold
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        C h = cscale(cmulc(buf[pad16(t)], T.chirp[t]), invM);
        if (t < N - 1) {
            const int u = P - 1 - t;
            C h2 = cscale(cmulc(buf[pad16(u)], T.chirp[u]), invM);
            h = cadd(h, cscale(h2, sigma));
        }
        h = cscale(h, qscale);
        g[t] = ccast<cplx_t<R>>(h);
    }
}

}  // namespace s2g
