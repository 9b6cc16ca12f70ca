// FP32 contraction kernels of the FP32 path, organised as register-blocked
// shared-memory GEMMs over all maps of a batch tile at once:
//   k_quad_gemm      G_m = Q_sigma F_m          MW theta quadrature as a dense product
//   k_leg_anal_gemm  f_lm = sum_t lambda_lm(theta_t) G_m(theta_t)
//   k_leg_synth_gemm F_m(theta_t) = sum_l lambda_lm(theta_t) c_l f_lm
// In the Legendre kernels the recurrence (float-float, see legendre.cuh) runs
// once per (m, ring, degree) and writes lambda tiles to shared memory; every
// map of the tile reuses them, so the recurrence is amortised over 2 x maps
// real columns (re and im of each map, and of -m for complex maps).
#pragma once
#include "common.cuh"
#include "legendre.cuh"

namespace s2g {

// ---------------------------------------------------------------- quadrature GEMM
// Q (N x N, row-major, symmetric) built once per band-limit from the FP64
// quadrature; G[b][mi][t] = sum_t' Q_sigma[t][t'] F[b][mi][t'] for the orders mi
// = mi0, mi0 + 2, ... (one parity), re and im parts as separate columns.
// Tiles: 128 rows (t) x 128 columns (64 (b, mi) pairs x re/im) x 16 (t').
constexpr int QG_BM = 128, QG_BN = 128, QG_BK = 16;

static __global__ void __launch_bounds__(256, 2) k_quad_gemm(const float *__restrict__ Q, const float2 *__restrict__ F,
                                                   float2 *__restrict__ G, int N, int nmi, int mi0, int nj,
                                                   int npairs)
{
    __shared__ __align__(16) float As[2][QG_BK][QG_BM];
    __shared__ __align__(16) float Bs[2][QG_BK][QG_BN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.x * QG_BM;
    const int pair0 = blockIdx.y * (QG_BN / 2);

    // global -> register staging
    float4 ra[2];
    float2 rb[4];
    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * 256;      // 512 float4 = 16 x 128 floats
            const int k = idx >> 5, c4 = (idx & 31) * 4;
            const int kk = k0 + k, rr = row0 + c4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kk < N) {
                const float *q = Q + (size_t)kk * N + rr;   // Q symmetric: Q[k][row] = Q[row][k]
                if (rr + 3 < N && ((N & 3) == 0)) {
                    v = *reinterpret_cast<const float4 *>(q);
                } else {
                    v.x = rr < N ? q[0] : 0.f;
                    v.y = rr + 1 < N ? q[1] : 0.f;
                    v.z = rr + 2 < N ? q[2] : 0.f;
                    v.w = rr + 3 < N ? q[3] : 0.f;
                }
            }
            ra[r] = v;
        }
        {                                       // 64 pairs x 4 groups of 4 k: one per thread
            const int p = tid & 63, k4 = tid >> 6;
            const int pp = pair0 + p;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int kk = k0 + k4 * 4 + r;
                float2 v = make_float2(0.f, 0.f);
                if (pp < npairs && kk < N) {
                    const int b = pp / nj, j = pp % nj;
                    v = F[((size_t)b * nmi + mi0 + 2 * j) * N + kk];
                }
                rb[r] = v;
            }
        }
    };
    auto store = [&](int s) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * 256;
            const int k = idx >> 5, c4 = (idx & 31) * 4;
            *reinterpret_cast<float4 *>(&As[s][k][c4]) = ra[r];
        }
        {
            const int p = tid & 63, k4 = tid >> 6;
#pragma unroll
            for (int r = 0; r < 4; ++r)
                *reinterpret_cast<float2 *>(&Bs[s][k4 * 4 + r][2 * p]) = rb[r];
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int nk = (N + QG_BK - 1) / QG_BK;
    load(0);
    store(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt & 1;
        if (kt + 1 < nk) load((kt + 1) * QG_BK);
#pragma unroll
        for (int k = 0; k < QG_BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[s][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[s][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[s][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[s][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        if (kt + 1 < nk) store(s ^ 1);
        __syncthreads();
    }
    // rows ty*4 + {0..3} and 64 + ty*4 + {0..3}; columns tx*4 + {0..3} and 64 + tx*4 + {0..3}
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {            // column pairs (re, im) of one (b, mi)
        const int cl = (jj < 2) ? tx * 4 + 2 * jj : 64 + tx * 4 + 2 * (jj - 2);
        const int pp = pair0 + cl / 2;
        if (pp >= npairs) continue;
        const int b = pp / nj, j = pp % nj;
        float2 *out = G + ((size_t)b * nmi + mi0 + 2 * j) * N;
        const int jc = (jj < 2) ? 2 * jj : 4 + 2 * (jj - 2);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = row0 + ((i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (r < N) out[r] = make_float2(acc[i][jc], acc[i][jc + 1]);
        }
    }
}

// ---------------------------------------------------------------- Legendre GEMMs
// Shared layout: NS sign sets (m, and -m for complex maps) x BT maps x (re, im)
// = 128 columns.  Column c = (s * BT + b) * 2 + part.
template <bool CPLX> struct LegCols {
    static constexpr int NS = CPLX ? 2 : 1;
    static constexpr int BT = 64 / NS;
    static constexpr int NC = 128;
};

// Analysis.  One block per (order m, batch tile).  Recurrence states of all N
// rings live in shared memory; degrees are processed in tiles of LT = 128 and,
// within a tile, rings in groups of RG = 128: each of the first RG threads
// advances one ring LT steps writing lambda[l][t] to shared memory, then all 256
// threads accumulate acc[l][c] += lambda[l][t] G[t][c] (8 x 8 per thread).
constexpr int LA_LT = 128, LA_RG = 128;

template <bool CPLX>
__global__ void __launch_bounds__(256) k_leg_anal_gemm(const float2 *__restrict__ Gin, int N,
                                                       const float *__restrict__ kfac, float scale, int accumulate,
                                                       float2 *__restrict__ dst, int Ldst, int B, LegTab<float> tab)
{
    using Cols = LegCols<CPLX>;
    constexpr int NS = Cols::NS, BT = Cols::BT, NC = Cols::NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *lam = reinterpret_cast<float *>(smem_raw);                 // [LT][RG]
    float *gs = lam + LA_LT * LA_RG;                                   // [RG][NC]
    float4 *st = reinterpret_cast<float4 *>(gs + LA_RG * NC);          // [N] (p0.h, p0.l, p1.h, p1.l)
    int *sls = reinterpret_cast<int *>(st + N);                        // [N]
    __shared__ float4 sc[LA_LT];
    __shared__ int gmin[64];

    const int m = blockIdx.x;
    const int b0 = blockIdx.y * BT;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int nmi_src = CPLX ? 2 * N - 1 : N;
    const int nmi_dst = CPLX ? 2 * Ldst - 1 : Ldst;
    const bool two = CPLX && m > 0;
    const int ngroups = (N + LA_RG - 1) / LA_RG;

    // load l_s and mark states as not yet seeded
    for (int t = tid; t < N; t += 256) sls[t] = tab.ls[(size_t)m * N + t];
    __syncthreads();
    for (int g = tid; g < ngroups; g += 256) {
        int mn = N;
        for (int t = g * LA_RG; t < min(N, (g + 1) * LA_RG); ++t) mn = min(mn, sls[t]);
        gmin[g] = mn;
    }
    __syncthreads();

    for (int l0 = m; l0 < N; l0 += LA_LT) {
        const int nl = min(LA_LT, N - l0);
        for (int i = tid; i < nl; i += 256) sc[i] = tab.coef[(size_t)m * tab.ldc + l0 + i];
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        __syncthreads();
        for (int g = 0; g < ngroups; ++g) {
            if (gmin[g] >= l0 + nl) continue;                          // every lambda in the tile is zero
            const int tg0 = g * LA_RG;
            const int nt = min(LA_RG, N - tg0);
            // recurrence: thread tid < RG owns ring tg0 + tid
            if (tid < LA_RG) {
                const int t = tg0 + tid;
                float *col = lam + tid;
                if (tid < nt) {
                    RecT<float> rec;
                    rec.ring(tab.ring[t]);
                    const int ls = sls[t];
                    if (l0 > ls) {
                        const float4 s4 = st[t];
                        rec.p0.h = s4.x; rec.p0.l = s4.y; rec.p1.h = s4.z; rec.p1.l = s4.w;
                    }
                    for (int i = 0; i < nl; ++i) {
                        const int l = l0 + i;
                        float v;
                        if (l < ls) v = 0.f;
                        else if (l == ls) { rec.seed(tab.seed[(size_t)m * N + t]); v = rec.value(); }
                        else v = rec.step(sc[i]);
                        col[i * LA_RG] = v;
                    }
                    for (int i = nl; i < LA_LT; ++i) col[i * LA_RG] = 0.f;
                    if (l0 + nl - 1 >= ls) st[t] = make_float4(rec.p0.h, rec.p0.l, rec.p1.h, rec.p1.l);
                } else {
                    for (int i = 0; i < LA_LT; ++i) col[i * LA_RG] = 0.f;
                }
            }
            // G tile gs[t][c]: each thread moves 4 consecutive rings of one column pair
            for (int idx = tid; idx < (LA_RG / 4) * NS * BT; idx += 256) {
                const int sb = idx % (NS * BT);          // s * BT + b
                const int t4 = idx / (NS * BT);
                const int s = sb / BT, b = sb % BT;
                const bool ok = b0 + b < B && (s == 0 || two);
                const int mi = s == 0 ? (CPLX ? m + N - 1 : m) : (-m + N - 1);
                const float2 *row = Gin + ((size_t)(b0 + b) * nmi_src + mi) * N + tg0;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int tt = t4 * 4 + r;
                    const float2 v = (ok && tt < nt) ? row[tt] : make_float2(0.f, 0.f);
                    *reinterpret_cast<float2 *>(&gs[tt * NC + 2 * sb]) = v;
                }
            }
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < LA_RG; ++k) {
                float a[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    a[i] = lam[(ty * 4 + i) * LA_RG + k];
                    a[4 + i] = lam[(64 + ty * 4 + i) * LA_RG + k];
                }
                const float4 g0 = *reinterpret_cast<const float4 *>(&gs[k * NC + tx * 4]);
                const float4 g1 = *reinterpret_cast<const float4 *>(&gs[k * NC + 64 + tx * 4]);
                const float bb[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
            }
            __syncthreads();
        }
        // epilogue: rows l, columns (s, b, part)
        const float sgn_m = (m & 1) ? -1.f : 1.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int li = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
            if (li >= nl) continue;
            const int l = l0 + li;
            const float f = scale * (kfac ? kfac[l] : 1.f);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int c = (jj < 2) ? tx * 4 + 2 * jj : 64 + tx * 4 + 2 * (jj - 2);
                const int jc = (jj < 2) ? 2 * jj : 4 + 2 * (jj - 2);
                const int sb = c / 2, s = sb / BT, b = sb % BT;
                if (b0 + b >= B || (s == 1 && !two)) continue;
                const float fs = s == 1 ? f * sgn_m : f;
                const int mi = s == 0 ? (CPLX ? m + Ldst - 1 : m) : (-m + Ldst - 1);
                float2 *o = dst + ((size_t)(b0 + b) * nmi_dst + mi) * Ldst + l;
                float2 v = make_float2(acc[i][jc] * fs, acc[i][jc + 1] * fs);
                if (accumulate) {
                    const float2 w = *o;
                    v.x += w.x;
                    v.y += w.y;
                }
                *o = v;
            }
        }
        __syncthreads();
    }
}

// Synthesis.  One block per (tile of RT = 128 rings, order m, batch tile); the
// ring tiles of one order are adjacent in the grid so they share its
// coefficient rows in L2.
// Degrees in chunks of LK = 32: each of the first RT threads advances its ring
// LK steps writing lambda[l][t]; coefficient tile a[l][c] = c_l f_lm staged from
// the source; all 256 threads accumulate acc[t][c] += lambda[l][t] a[l][c].
constexpr int LS_RT = 128, LS_LK = 32;

template <bool CPLX>
__global__ void __launch_bounds__(256) k_leg_synth_gemm(const float2 *__restrict__ src, int Lsrc,
                                                        const float *__restrict__ kfac, float scale,
                                                        float2 *__restrict__ dst, int N, int B, LegTab<float> tab)
{
    using Cols = LegCols<CPLX>;
    constexpr int NS = Cols::NS, BT = Cols::BT, NC = Cols::NC;
    __shared__ __align__(16) float lam[LS_LK][LS_RT];
    __shared__ __align__(16) float as[LS_LK][NC];
    __shared__ float4 sc[LS_LK];
    __shared__ int smin[8];

    const int m = blockIdx.y;
    const int t0 = blockIdx.x * LS_RT;
    const int b0 = blockIdx.z * BT;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int nmi_src = CPLX ? 2 * Lsrc - 1 : Lsrc;
    const int nmi_dst = CPLX ? 2 * N - 1 : N;
    const bool two = CPLX && m > 0;

    const int t = t0 + tid;
    const bool owner = tid < LS_RT && t < N;
    int ls = owner ? tab.ls[(size_t)m * N + t] : N;
    RecT<float> rec;
    if (owner) rec.ring(tab.ring[t]);
    int v = ls;
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((tid & 31) == 0) smin[tid >> 5] = v;
    __syncthreads();
    int lstart = smin[0];
    for (int w = 1; w < 8; ++w) lstart = min(lstart, smin[w]);

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int l0 = lstart; l0 < N; l0 += LS_LK) {
        const int nl = min(LS_LK, N - l0);
        __syncthreads();
        for (int i = tid; i < nl; i += 256) sc[i] = tab.coef[(size_t)m * tab.ldc + l0 + i];
        // coefficient tile as[l][c]: each thread moves 4 consecutive degrees of one column pair
        for (int idx = tid; idx < (LS_LK / 4) * NS * BT; idx += 256) {
            const int sb = idx % (NS * BT);
            const int l4 = idx / (NS * BT);
            const int s = sb / BT, b = sb % BT;
            const bool ok = b0 + b < B && (s == 0 || two);
            const int mi = s == 0 ? (CPLX ? m + Lsrc - 1 : m) : (-m + Lsrc - 1);
            const float2 *row = src + ((size_t)(b0 + b) * nmi_src + mi) * Lsrc + l0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int li = l4 * 4 + r;
                float2 c = make_float2(0.f, 0.f);
                if (ok && li < nl) {
                    c = row[li];
                    if (kfac) {
                        const float k = kfac[l0 + li];
                        c.x *= k;
                        c.y *= k;
                    }
                }
                *reinterpret_cast<float2 *>(&as[li][2 * sb]) = c;
            }
        }
        __syncthreads();
        if (tid < LS_RT) {
            for (int i = 0; i < LS_LK; ++i) {
                const int l = l0 + i;
                float x = 0.f;
                if (owner && i < nl) {
                    if (l < ls) x = 0.f;
                    else if (l == ls) { rec.seed(tab.seed[(size_t)m * N + t]); x = rec.value(); }
                    else x = rec.step(sc[i]);
                }
                lam[i][tid] = x;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < LS_LK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&lam[k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&lam[k][64 + ty * 4]);
            const float4 c0 = *reinterpret_cast<const float4 *>(&as[k][tx * 4]);
            const float4 c1 = *reinterpret_cast<const float4 *>(&as[k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bb[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
    }
    const float sgn_m = (m & 1) ? -1.f : 1.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int ti = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
        const int tt = t0 + ti;
        if (tt >= N) continue;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int c = (jj < 2) ? tx * 4 + 2 * jj : 64 + tx * 4 + 2 * (jj - 2);
            const int jc = (jj < 2) ? 2 * jj : 4 + 2 * (jj - 2);
            const int sb = c / 2, s = sb / BT, b = sb % BT;
            if (b0 + b >= B || (s == 1 && !two)) continue;
            const float f = s == 1 ? scale * sgn_m : scale;
            const int mi = s == 0 ? (CPLX ? m + N - 1 : m) : (-m + N - 1);
            dst[((size_t)(b0 + b) * nmi_dst + mi) * N + tt] = make_float2(acc[i][jc] * f, acc[i][jc + 1] * f);
        }
    }
}

}  // namespace s2g
