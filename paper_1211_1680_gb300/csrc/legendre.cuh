// Legendre stages of the MW spherical harmonic transforms:
//   seeds     lambda_mm(theta_t) with a separate exponent, then the scaled
//             recurrence up to the first degree l_s(m, t) where
//             |lambda_lm(theta_t)| >= 2^-SEED_EXP; (l_s, lambda_{l_s-1}, lambda_{l_s})
//             are kept (FP64).  Smaller values are below 2^-100 and are dropped.
//   synthesis F_m(theta_t) = scale * sum_{l} c_l f_lm lambda_lm(theta_t)  (Eq. harmonicssynthesis)
//   analysis  f_lm = scale * c_l * sum_t lambda_lm(theta_t) G_m(theta_t)  (MW quadrature, last step)
// Normalised associated Legendre recurrence (Condon-Shortley phase):
//   lambda_lm = a_lm (x lambda_{l-1,m} - b_lm lambda_{l-2,m}),  x = cos(theta),
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)), b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
// FP64 path: x lambda is evaluated as sgn (lambda - y lambda), y = 1 - |x|,
// which keeps the rounding of each step small near the poles.
// FP32 path: the recurrence runs in float-float (FP32 pairs, about 48 bits),
// because a plain FP32 recurrence loses ~1e-3 relative accuracy at L = 2048
// for small m near the poles; the value used in the sum is the rounded FP32.
#pragma once
#include "common.cuh"

namespace s2g {

constexpr int SEED_EXP = 100;

struct RingD {           // per ring, FP64 path
    double sgn, y;       // cos(theta) = sgn (1 - y)
};
struct RingF {           // per ring, FP32 path: cos(theta) as float-float
    float xh, xl;
};

template <typename R> struct RecT;
template <> struct RecT<double> {
    using Ring = RingD;
    using Coef = double2;  // (a_lm, a_lm b_lm)
    double p0, p1, sg, y;
    __device__ __forceinline__ void ring(const RingD &r) { sg = r.sgn; y = r.y; }
    __device__ __forceinline__ void seed(double2 s) { p0 = s.x; p1 = s.y; }
    __device__ __forceinline__ double value() const { return p1; }
    __device__ __forceinline__ double step(const double2 c)
    {
        double p2 = c.x * (sg * (p1 - y * p1)) - c.y * p0;
        p0 = p1;
        p1 = p2;
        return p2;
    }
};
template <> struct RecT<float> {
    using Ring = RingF;
    using Coef = float4;   // (a hi, a lo, a b hi, a b lo)
    ff p0, p1, x;
    __device__ __forceinline__ void ring(const RingF &r) { x.h = r.xh; x.l = r.xl; }
    __device__ __forceinline__ void seed(double2 s)
    {
        p0.h = (float)s.x;
        p0.l = (float)(s.x - (double)p0.h);
        p1.h = (float)s.y;
        p1.l = (float)(s.y - (double)p1.h);
    }
    __device__ __forceinline__ float value() const { return p1.h; }
    __device__ __forceinline__ float step(const float4 c)
    {
        ff a;
        a.h = c.x;
        a.l = c.y;
        ff ab;
        ab.h = c.z;
        ab.l = c.w;
        ff ax = ff_mul(a, x);
        ff pa = ff_mul(ax, p1);
        ff pb = ff_mul(ab, p0);
        ff p2 = ff_sub(pa, pb);
        p0 = p1;
        p1 = p2;
        return p2.h;
    }
};

// ---------------------------------------------------------------- seeds (FP64)
// Sectoral values lambda_mm(theta_t) = -sqrt((2m+1)/(2m)) sin(theta) lambda_{m-1,m-1},
// lambda_00 = 1/sqrt(4 pi), kept as mantissa * 2^exponent.  One thread per ring.
static __global__ void k_sectoral(int N, const double *__restrict__ sinth, double *__restrict__ mant,
                           int *__restrict__ expo)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const double s = sinth[t];
    int e = 0;
    double f = frexp(0.28209479177387814347403972578039, &e);   // 1/sqrt(4 pi)
    mant[t] = f;
    expo[t] = e;
    for (int m = 1; m < N; ++m) {
        f *= -sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
        int k = 0;
        if (f != 0.0) {
            f = frexp(f, &k);
            e += k;
        }
        mant[(size_t)m * N + t] = f;
        expo[(size_t)m * N + t] = e;
    }
}

// First degree l_s >= m with |lambda_lm(theta_t)| >= 2^-SEED_EXP, and the pair
// (lambda_{l_s-1}, lambda_{l_s}); l_s = N when there is none.  One thread per (m, t).
static __global__ void k_seed_start(int N, const double *__restrict__ mant, const int *__restrict__ expo,
                             const RingD *__restrict__ ring, const double2 *__restrict__ coef, int ldc,
                             int *__restrict__ ls, double2 *__restrict__ seed)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N * N) return;
    const int m = (int)(idx / N), t = (int)(idx % N);
    const RingD r = ring[t];
    double p1 = mant[idx], p0 = 0.0;
    int e = expo[idx];
    int found = N;
    double2 s = make_double2(0.0, 0.0);
    if (p1 != 0.0 && ilogb(p1) + e >= -SEED_EXP) {
        found = m;
        s = make_double2(0.0, ldexp(p1, e));
    } else if (p1 != 0.0) {
        const double2 *cm = coef + (size_t)m * ldc;
        for (int l = m + 1; l < N; ++l) {
            const double2 c = cm[l];
            const double p2 = c.x * (r.sgn * (p1 - r.y * p1)) - c.y * p0;
            p0 = p1;
            p1 = p2;
            if (fabs(p1) > 0x1p+600) {
                p0 = ldexp(p0, -600);
                p1 = ldexp(p1, -600);
                e += 600;
            }
            if (p1 != 0.0 && ilogb(p1) + e >= -SEED_EXP) {
                found = l;
                s = make_double2(ldexp(p0, e), ldexp(p1, e));
                break;
            }
        }
    }
    ls[idx] = found;
    seed[idx] = s;
}

// Legendre tables for one band-limit N, read by the transform kernels.
template <typename R> struct LegTab {
    const int *ls;                              // [m][t], N x N
    const double2 *seed;                        // [m][t]
    const typename RecT<R>::Ring *ring;         // [t]
    const typename RecT<R>::Coef *coef;         // [m][l], row stride ldc (tables for the largest L)
    int ldc;
};

// ---------------------------------------------------------------- synthesis (S5)
// dst[b][mi(m)][t] = scale * sum_{l=|m|}^{N-1} kfac[l] src[b][mi_src(m)][l] lambda_{l|m|}(theta_t)
// src rows have stride lds (>= N); mi(m) = m for real maps, m + n - 1 for complex
// maps of band-limit n.  Complex maps: one block serves m and -m
// (lambda_{l,-m} = (-1)^m lambda_lm).  Grid: (N |m| values, ring tiles, batch tiles).
template <typename R, int BT, bool CPLX, int TT>
__global__ void __launch_bounds__(TT) k_leg_synth(const cplx_t<R> *__restrict__ src, int lds, int nmi_src,
                                                  int Lsrc, const R *__restrict__ kfac, R scale,
                                                  cplx_t<R> *__restrict__ dst, int N, int B, LegTab<R> tab)
{
    using C = cplx_t<R>;
    using Rec = RecT<R>;
    constexpr int LCH = 32;
    constexpr int NS = CPLX ? 2 : 1;
    __shared__ C sa[NS][LCH][BT];
    __shared__ typename Rec::Coef sc[LCH];
    __shared__ int smin[TT / 32];

    const int m = blockIdx.x;
    const int t = blockIdx.y * TT + threadIdx.x;
    const int b0 = blockIdx.z * BT;
    const bool active = t < N;
    const int nmi_dst = CPLX ? 2 * N - 1 : N;
    const int mi_dst_p = CPLX ? m + N - 1 : m;
    const int mi_dst_n = CPLX ? -m + N - 1 : m;
    const int mi_src_p = CPLX ? m + Lsrc - 1 : m;
    const int mi_src_n = CPLX ? -m + Lsrc - 1 : m;
    const bool two = CPLX && m > 0;

    int myls = active ? tab.ls[(size_t)m * N + t] : N;
    Rec rec;
    if (active) rec.ring(tab.ring[t]);
    // block minimum of l_s: degrees below it contribute nothing
    int v = myls;
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = v;
    __syncthreads();
    int lstart = smin[0];
    for (int w = 1; w < TT / 32; ++w) lstart = min(lstart, smin[w]);

    R acc[NS][BT][2];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int i = 0; i < BT; ++i) acc[s][i][0] = acc[s][i][1] = (R)0;

    for (int l0 = lstart; l0 < N; l0 += LCH) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < NS * LCH * BT; idx += TT) {
            const int s = idx / (LCH * BT);
            const int lc = (idx / BT) % LCH;
            const int bb = idx % BT;
            const int l = l0 + lc;
            C val = mk((R)0, (R)0);
            if (l < N && b0 + bb < B && (s == 0 || two)) {
                const int mi = s == 0 ? mi_src_p : mi_src_n;
                val = src[((size_t)(b0 + bb) * nmi_src + mi) * lds + l];
                if (kfac) val = cscale(val, kfac[l]);
            }
            sa[s][lc][bb] = val;
        }
        for (int lc = threadIdx.x; lc < LCH; lc += TT) {
            const int l = l0 + lc;
            if (l < N) sc[lc] = tab.coef[(size_t)m * tab.ldc + l];
        }
        __syncthreads();
        const int nl = min(LCH, N - l0);
        for (int lc = 0; lc < nl; ++lc) {
            const int l = l0 + lc;
            R lam;
            if (l < myls) {
                lam = (R)0;
            } else if (l == myls) {
                rec.seed(tab.seed[(size_t)m * N + t]);
                lam = rec.value();
            } else {
                lam = rec.step(sc[lc]);
            }
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int i = 0; i < BT; ++i) {
                    const C a = sa[s][lc][i];
                    acc[s][i][0] += lam * a.x;
                    acc[s][i][1] += lam * a.y;
                }
        }
    }
    if (!active) return;
    const R sgn_m = (m & 1) ? (R)-1 : (R)1;
#pragma unroll
    for (int i = 0; i < BT; ++i) {
        if (b0 + i >= B) break;
        C *row = dst + (size_t)(b0 + i) * nmi_dst * N;
        row[(size_t)mi_dst_p * N + t] = mk(acc[0][i][0] * scale, acc[0][i][1] * scale);
        if (two) row[(size_t)mi_dst_n * N + t] = mk(acc[NS - 1][i][0] * scale * sgn_m,
                                                     acc[NS - 1][i][1] * scale * sgn_m);
    }
}

// ---------------------------------------------------------------- analysis (S3)
// out_l = scale * kfac[l] * sum_t lambda_{l|m|}(theta_t) G[b][mi(m)][t], written
// (or added, when accumulate) to dst[b][mi_dst(m)][l], l = |m|..N-1.  One block
// holds every ring of one order (RPT rings per thread) and one batch tile.
// Degrees are processed in chunks of LCH; each lane accumulates V = LCH x
// (values per degree) partial sums over its rings, then a transposed butterfly
// (each shuffle step halves the values a lane holds) sums them over the warp
// with V - V/32 shuffles, and the warps' totals are added in shared memory.
template <typename R, int BT, bool CPLX, int RPT, int TPB, int V>
__global__ void __launch_bounds__(TPB) k_leg_anal(const cplx_t<R> *__restrict__ G, int N,
                                                  const R *__restrict__ kfac, R scale, int accumulate,
                                                  cplx_t<R> *__restrict__ dst, int ldd, int nmi_dst,
                                                  int Ldst, int B, LegTab<R> tab)
{
    using C = cplx_t<R>;
    using Rec = RecT<R>;
    constexpr int NS = CPLX ? 2 : 1;
    constexpr int PER_L = NS * BT * 2;
    constexpr int LCH = V / PER_L;
    static_assert(V % 32 == 0 && LCH >= 1 && LCH * PER_L == V, "chunk shape");
    constexpr int NW = TPB / 32;
    constexpr int VPL = V / 32;
    __shared__ R red[NW][V];
    __shared__ typename Rec::Coef sc[LCH];

    const int m = blockIdx.x;
    const int b0 = blockIdx.y * BT;
    const int nmi_src = CPLX ? 2 * N - 1 : N;
    const int mi_src_p = CPLX ? m + N - 1 : m;
    const int mi_src_n = CPLX ? -m + N - 1 : m;
    const int mi_dst_p = CPLX ? m + Ldst - 1 : m;
    const int mi_dst_n = CPLX ? -m + Ldst - 1 : m;
    const bool two = CPLX && m > 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    Rec rec[RPT];
    int myls[RPT];
    R g[RPT][NS][BT][2];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int t = threadIdx.x + k * TPB;
        const bool act = t < N;
        myls[k] = act ? tab.ls[(size_t)m * N + t] : N;
        if (act) rec[k].ring(tab.ring[t]);
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int i = 0; i < BT; ++i) {
                C v = mk((R)0, (R)0);
                if (act && b0 + i < B && (s == 0 || two)) {
                    const int mi = s == 0 ? mi_src_p : mi_src_n;
                    v = G[((size_t)(b0 + i) * nmi_src + mi) * N + t];
                }
                g[k][s][i][0] = v.x;
                g[k][s][i][1] = v.y;
            }
    }

    for (int l0 = m; l0 < N; l0 += LCH) {
        __syncthreads();
        for (int lc = threadIdx.x; lc < LCH; lc += TPB)
            if (l0 + lc < N) sc[lc] = tab.coef[(size_t)m * tab.ldc + l0 + lc];
        __syncthreads();
        const int nl = min(LCH, N - l0);
        R part[V];
#pragma unroll
        for (int v = 0; v < V; ++v) part[v] = (R)0;
#pragma unroll
        for (int lc = 0; lc < LCH; ++lc) {
            if (lc < nl) {
                const int l = l0 + lc;
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    R lam;
                    if (l < myls[k]) {
                        lam = (R)0;
                    } else if (l == myls[k]) {
                        rec[k].seed(tab.seed[(size_t)m * N + threadIdx.x + k * TPB]);
                        lam = rec[k].value();
                    } else {
                        lam = rec[k].step(sc[lc]);
                    }
#pragma unroll
                    for (int s = 0; s < NS; ++s)
#pragma unroll
                        for (int i = 0; i < BT; ++i) {
                            part[((lc * NS + s) * BT + i) * 2 + 0] += lam * g[k][s][i][0];
                            part[((lc * NS + s) * BT + i) * 2 + 1] += lam * g[k][s][i][1];
                        }
                }
            }
        }
        // transposed butterfly: after the step with offset o a lane keeps the
        // half selected by (lane & o); at the end lane L holds values [L*VPL, L*VPL+VPL)
#pragma unroll
        for (int st = 0; st < 5; ++st) {
            const int o = 16 >> st;
            const int h = V >> (st + 1);
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const R send = up ? part[i] : part[i + h];
                const R keep = up ? part[i + h] : part[i];
                part[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
#pragma unroll
        for (int j = 0; j < VPL; ++j) red[warp][lane * VPL + j] = part[j];
        __syncthreads();
        for (int q = threadIdx.x; q < nl * NS * BT; q += TPB) {
            const int lc = q / (NS * BT);
            const int s = (q / BT) % NS;
            const int i = q % BT;
            if (b0 + i >= B || (s == 1 && !two)) continue;
            R sx = 0, sy = 0;
            for (int w = 0; w < NW; ++w) {
                sx += red[w][2 * q];
                sy += red[w][2 * q + 1];
            }
            const int l = l0 + lc;
            R f = scale * (kfac ? kfac[l] : (R)1);
            if (s == 1) f *= (m & 1) ? (R)-1 : (R)1;
            const int mi = s == 0 ? mi_dst_p : mi_dst_n;
            C *o = dst + ((size_t)(b0 + i) * nmi_dst + mi) * ldd + l;
            C val = mk(sx * f, sy * f);
            if (accumulate) val = cadd(*o, val);
            *o = val;
        }
    }
}

}  // namespace s2g
