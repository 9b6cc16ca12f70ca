// Legendre contractions of the split tensor-core plans on precomputed tables,
// FP16 hi/lo operands on tcgen05 (kind::f16, FP32 accumulation):
//   k_leg_h16<ANAL = true>   f_lm = scale c_l sum_t lambda_lm(theta_t) G_m(theta_t)  (last step of the MW quadrature)
//   k_leg_h16<ANAL = false>  F_m(theta_t) = scale sum_l lambda_lm(theta_t) c_l f_lm  (Eq. harmonicssynthesis)
//
// Split.  A value x is carried as hi + lo, hi = fp16(x), lo = fp16(x - hi), both
// rounded to nearest (11 significant bits each, 2^-22 relative), and a product as
// hi*hi + hi*lo + lo*hi.  FP16 has a narrow exponent range, so both operands
// are scaled by powers of two that the epilogue divides out exactly:
//   table   lambda_lm(theta_t) * 2^9: |lambda_lm| <= sqrt((2l+1)/(4 pi)) (the
//           addition theorem), below 2^5 for l < 4096, so |hi| < 2^14;
//   data    per column (map, order), 2^(12 - e) with 2^e <= max |x| < 2^(e+1) over
//           the K range the launch reads (k_h16_colscale), so |hi| < 2^13.
// A value below the scaled range keeps an absolute error of at most 2^-25 of
// the scale unit, i.e. 2^-37 of its column's largest value.
//
// Tables.  Two copies of the values of every stored 32 x 32 block (the block
// structure of legendre_img.cuh: i0, off, block 0 = zeros): `ta`, rows = degrees
// m + 32 i + r, K = 32 rings; `ts`, rows = rings 32 k + r, K = 32 degrees.  A row
// is 128 bytes, [32 hi | 32 lo] halves, its 16-byte pieces XOR-swizzled by
// r & 7, so four blocks stacked in shared memory are a 128 x 64 K-major
// SWIZZLE_128B operand: hi at byte 0 of the row, lo at byte 64, and the k-step
// of 16 at byte 32 ks.  Both directions read A straight from shared memory.
//
// Block roles (320 threads):
//   warps 0-7  operand B: asynchronous copies of a chunk of G (analysis) or f_lm
//              (synthesis) into a ring of LH_NRAW chunks, then scale (c_l in the
//              synthesis), split, store; drain the accumulators; epilogue
//   warp 8     bulk copies of the four table blocks of each chunk (A ring)
//   warp 9     TMEM allocation and the MMAs (one thread)
// Every wait is bounded; a wait that runs out sets the block's abort flag, all
// roles then run to the end without waiting, and the plan's error word is set.
#pragma once
#include <cuda_fp16.h>
#include "legendre_img.cuh"

namespace s2g {

constexpr float LH_TSCALE = 512.f;                   // table scale 2^9
constexpr int LH_NA = 6, LH_NB = 3, LH_NRAW = 4, LH_NR = 16, LH_NACC = 4, LH_D = 4;
constexpr int LH_BWARPS = 8, LH_COPY_WARP = 8, LH_MMA_WARP = 9, LH_THREADS = 320;
constexpr int LH_STAGE = 16384;                      // 128 rows x 128 bytes
constexpr int LH_B_OFF = LH_NA * LH_STAGE;
constexpr int LH_RAW_OFF = LH_B_OFF + LH_NB * LH_STAGE;    // operand B as read: FP32, LH_NRAW chunks
constexpr int LH_LIST_OFF = LH_RAW_OFF + LH_NRAW * LH_STAGE;
constexpr int LH_BLKS_OFF = LH_LIST_OFF + LI_MAXK * 4;      // table blocks of every chunk [c][4]
constexpr int LH_EPI_OFF = LH_BLKS_OFF + LI_MAXK * 16;      // per column pair: epilogue factor, output row
constexpr int LH_KF_OFF = LH_EPI_OFF + 64 * 12;             // synthesis: c_l of degrees m .. N - 1
constexpr int LH_MAXN = 2048;                                 // largest band-limit of the tables
constexpr int LH_SYNC_OFF = LH_KF_OFF + LH_MAXN * 4;
struct LhSync {
    uint64_t afull[LH_NA], bfull[LH_NB], done[LH_NR], tempty[LH_NACC], fin, mfull;
    uint32_t tslot;
    int abort, nk, ibase;
};
constexpr int LH_SYNC_BYTES = 512;
static_assert(sizeof(LhSync) <= LH_SYNC_BYTES, "sync block");
// a waiter for chunk c lags the MMAs by at most LH_NA (copies), LH_NB (operand B)
// or LH_D (LH_NACC - 1) (drains) chunks: fewer than the LH_NR phases of the ring
static_assert(LH_NA < LH_NR && LH_NB < LH_NR && LH_D * (LH_NACC - 1) < LH_NR, "barrier ring");
static_assert(128 * LH_NACC <= LT_TMEM_COLS, "tensor memory");
__host__ __device__ constexpr size_t leg_h16_smem() { return (size_t)LH_SYNC_OFF + LH_SYNC_BYTES + 1024; }
static_assert(leg_h16_smem() <= 227 * 1024, "shared memory");

// byte offset of byte `byte` (0..127) of row r in a tile of 128-byte rows with
// the 128-byte swizzle (8-row atoms of 1024 bytes, tile base 1024-aligned)
__host__ __device__ __forceinline__ uint32_t lh_sw(int r, int byte)
{
    return (uint32_t)(r * 128 + ((((byte >> 4) ^ r) & 7) << 4) + (byte & 15));
}

// Instruction descriptor, kind::f16: D FP32, A and B FP16, both K-major, dense.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16, issued by one thread.
__device__ __forceinline__ void mma_f16_ss(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// power-of-two column scale for a largest magnitude mx: mx * s in [2^12, 2^13)
__device__ __forceinline__ float lh_colscale(float mx)
{
    if (!(mx > 0.f) || !(mx <= 3.4e38f)) return 1.f;
    int e = (int)((__float_as_uint(mx) >> 23) & 255u) - 127;   // floor(log2 mx) for normal mx
    e = min(126, max(-126, 12 - e));
    return __uint_as_float((uint32_t)(e + 127) << 23);
}

// Column scales of one launch: one warp per source row (map b, order row mi).
//   analysis   rows of G [b][mi][t], t < N (mi over 2N - 1 orders, or N for real maps)
//   synthesis  rows of src [b][mi][l] (rectangle Lsrc), |m| <= l < N, times |kfac[l]|
template <bool ANAL>
static __global__ void k_h16_colscale(const float2 *__restrict__ src, int Lsrc, const float *__restrict__ kfac, int N,
                                      int B, int cplx, float *__restrict__ csc)
{
    const int nmi = ANAL ? (cplx ? 2 * N - 1 : N) : (cplx ? 2 * Lsrc - 1 : Lsrc);
    const int lds = ANAL ? N : Lsrc;
    const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (size_t)B * nmi) return;
    const int mi = (int)(gw % nmi);
    int k0 = 0;
    if (!ANAL) {
        const int m = cplx ? mi - (Lsrc - 1) : mi;
        k0 = m < 0 ? -m : m;
    }
    const float2 *row = src + gw * lds;
    float mx = 0.f;
#pragma unroll 4
    for (int k = k0 + lane; k < N; k += 32) {
        const float2 v = row[k];
        float x = fmaxf(fabsf(v.x), fabsf(v.y));
        if (!ANAL && kfac) x *= fabsf(kfac[k]);
        mx = fmaxf(mx, x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) csc[gw] = lh_colscale(mx);
}

// The stored blocks of both tables: one warp per (m, ring block k), lane = ring.
// Each lane runs the FP64 three-term recurrence of its ring from its seed
// (zero below the start degree l_s), the recurrence of the FP64 kernels
// (legendre.cuh); each value is scaled by 2^9 and split into FP16 hi and lo (lo
// from the FP64 remainder), and written to row r of the `ta` block and to
// column r of the `ts` block.  `ta` holds the blocks of (m, k) in degree order
// (off[m][k] + i - i0[m][k]); `ts` holds those of (m, i) in ring-block order,
// soff[m][i] + k - klo[m][i], so that the ring blocks of one degree block are
// adjacent (klo: the first ring block with a stored block i; rows [m][i] of
// stride ceil(N / 32)).
static __global__ void k_h16_fill(int N, const int *__restrict__ ls, const double2 *__restrict__ seed,
                                  const RingD *__restrict__ ring, const double2 *__restrict__ coef, int ldc,
                                  const int *__restrict__ i0, const int *__restrict__ off,
                                  const int *__restrict__ soff, const int *__restrict__ klo,
                                  unsigned char *__restrict__ ta, unsigned char *__restrict__ ts)
{
    const int nkr = (N + 31) / 32;
    const int gw = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (gw >= N * nkr) return;
    const int m = gw / nkr, k = gw % nkr, t = 32 * k + lane;
    const int nib = li_nib(N, m), ib = i0[gw];
    if (ib >= nib) return;
    const bool own = t < N;
    const int lsv = own ? ls[(size_t)m * N + t] : N;
    RecT<double> rec;
    rec.p0 = rec.p1 = 0.0;
    rec.sg = rec.y = 0.0;
    double2 sd = make_double2(0.0, 0.0);
    if (own) {
        rec.ring(ring[t]);
        sd = seed[(size_t)m * N + t];
    }
    const double2 *cm = coef + (size_t)m * ldc;
    size_t blk = (size_t)off[gw] * LI_BLK;
    for (int i = ib; i < nib; ++i, blk += LI_BLK) {
        const size_t tblk = (size_t)(soff[m * nkr + i] + k - klo[m * nkr + i]) * LI_BLK;
        for (int r = 0; r < 32; ++r) {
            const int l = m + 32 * i + r;
            double v = 0.0;
            if (l < N && l >= lsv) {
                if (l == lsv) rec.seed(sd);
                else rec.step(cm[l]);
                v = rec.value();
            }
            const double x = v * (double)LH_TSCALE;
            const __half h = __float2half_rn((float)x);
            const __half lo = __float2half_rn((float)(x - (double)__half2float(h)));
            *reinterpret_cast<__half *>(ta + blk + lh_sw(r, 2 * lane)) = h;
            *reinterpret_cast<__half *>(ta + blk + lh_sw(r, 64 + 2 * lane)) = lo;
            *reinterpret_cast<__half *>(ts + tblk + lh_sw(lane, 2 * r)) = h;
            *reinterpret_cast<__half *>(ts + tblk + lh_sw(lane, 64 + 2 * r)) = lo;
        }
    }
}

struct LegH16Args {
    const float2 *src;       // analysis: G [b][mi][t] (band-limit N); synthesis: f [b][mi][l] (rectangle Lsrc)
    int Lsrc;                // synthesis: rectangle of src
    const float *kfac;       // per-degree factor or nullptr
    float scale;
    int accumulate;          // analysis: add to dst
    float2 *dst;             // analysis: f [b][mi][l] (rectangle Ldst); synthesis: F [b][mi][t] (band-limit N)
    int Ldst;
    int N, B;
    LegImg T;                // block index (i0, off, adt, nkr)
    const unsigned char *tab;   // ta (analysis) or ts (synthesis)
    const float *csc;        // column scales [b][mi] of src (k_h16_colscale)
    int *err;
};

// split 8 scaled values into packed FP16 hi and lo words
__device__ __forceinline__ void lh_split8(const float (&x)[8], uint4 &hi, uint4 &lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __half2 hv = __floats2half2_rn(x[2 * q], x[2 * q + 1]);
        const float2 hf = __half22float2(hv);
        const __half2 lv = __floats2half2_rn(x[2 * q] - hf.x, x[2 * q + 1] - hf.y);
        h[q] = *reinterpret_cast<const uint32_t *>(&hv);
        l[q] = *reinterpret_cast<const uint32_t *>(&lv);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

template <bool ANAL, bool CPLX>
static __global__ void __launch_bounds__(LH_THREADS, 1) k_leg_h16(LegH16Args a)
{
    using Cols = LegCols<CPLX>;
    constexpr int BT = Cols::BT;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    LhSync &sy = *reinterpret_cast<LhSync *>(smem + LH_SYNC_OFF);
    int *klist = reinterpret_cast<int *>(smem + LH_LIST_OFF);
    int4 *blks = reinterpret_cast<int4 *>(smem + LH_BLKS_OFF);
    long long *epi_row = reinterpret_cast<long long *>(smem + LH_EPI_OFF);
    float *epi_f = reinterpret_cast<float *>(smem + LH_EPI_OFF + 64 * 8);
    float *kf_s = reinterpret_cast<float *>(smem + LH_KF_OFF);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.N;
    int m, tile, b0;
    if constexpr (ANAL) {
        const int2 md = a.T.adt[blockIdx.x];
        m = md.x;
        tile = md.y;
        b0 = blockIdx.y * BT;
    } else {
        tile = blockIdx.x;
        m = blockIdx.y;
        b0 = blockIdx.z * BT;
    }
    const int nib = li_nib(N, m);
    const bool two = CPLX && m > 0;
    volatile int *abort = &sy.abort;
    auto par = [](int c, int n) -> uint32_t { return (uint32_t)((c / n) & 1); };

    if (warp == LH_MMA_WARP) {
        tc::tmem_alloc(&sy.tslot, LT_TMEM_COLS);
    } else if (warp == LH_COPY_WARP && lane == 0) {
        // barriers, then the item's chunk list (built at plan creation) by bulk copies,
        // so that the first table copies can go out as soon as it lands
#pragma unroll
        for (int i = 0; i < LH_NA; ++i) tc::mbar_init(&sy.afull[i], 1);
#pragma unroll
        for (int i = 0; i < LH_NB; ++i) tc::mbar_init(&sy.bfull[i], LH_BWARPS);
#pragma unroll
        for (int i = 0; i < LH_NR; ++i) tc::mbar_init(&sy.done[i], 1);
#pragma unroll
        for (int i = 0; i < LH_NACC; ++i) tc::mbar_init(&sy.tempty[i], LH_BWARPS);
        tc::mbar_init(&sy.fin, 1);
        tc::mbar_init(&sy.mfull, 1);
        sy.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const int4 md = ANAL ? a.T.ameta[blockIdx.x] : a.T.smeta[(size_t)m * ((N + 127) / 128) + tile];
        sy.nk = md.y;
        sy.ibase = ANAL ? 0 : md.z;
        const uint32_t nb = (uint32_t)md.y * 16u, nl = ANAL ? (uint32_t)((md.y + 3) & ~3) * 4u : 0u;
        tc::mbar_arrive_expect_tx(&sy.mfull, nb + nl);
        if (md.y > 0) {
            tc::bulk_g2s(blks, (ANAL ? a.T.ablk : a.T.sblk) + md.x, nb, &sy.mfull);
            if (ANAL) tc::bulk_g2s(klist, a.T.ack + md.z, nl, &sy.mfull);
        }
    }
    if (!ANAL && a.kfac && warp < LH_BWARPS)
        for (int l = m + tid; l < N; l += 32 * LH_BWARPS) kf_s[l - m] = a.kfac[l];
    if (warp < LH_BWARPS && (lane & 0x14) == 0) {
        // per column pair p (one thread each): the factor that undoes the scales and
        // the offset of its output row (-1: absent pair)
        const int p = 8 * warp + (lane & 3) + 4 * ((lane >> 3) & 1);
        const int sg = p / BT, b = p % BT;
        const bool live = b0 + b < a.B && (sg == 0 || two);
        const int nmi_src = ANAL ? (CPLX ? 2 * N - 1 : N) : (CPLX ? 2 * a.Lsrc - 1 : a.Lsrc);
        const int moff = ANAL ? N - 1 : a.Lsrc - 1;
        const int mi = sg == 0 ? (CPLX ? m + moff : m) : (-m + moff);
        const int Lo = ANAL ? a.Ldst : N;                 // output rectangle
        const int nmi_dst = CPLX ? 2 * Lo - 1 : Lo;
        const int mid = sg == 0 ? (CPLX ? m + Lo - 1 : m) : (-m + Lo - 1);
        const float sgn = (sg == 1 && (m & 1)) ? -1.f : 1.f;
        epi_f[p] = live ? sgn * a.scale * (1.f / LH_TSCALE) / a.csc[(size_t)(b0 + b) * nmi_src + mi] : 0.f;
        epi_row[p] = live ? ((long long)(b0 + b) * nmi_dst + mid) * Lo : -1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sy.tslot;
    const int nk = sy.nk, ibase = sy.ibase;
    const int ng = (nk + LH_D - 1) / LH_D;
    const int nmi_src = ANAL ? (CPLX ? 2 * N - 1 : N) : (CPLX ? 2 * a.Lsrc - 1 : a.Lsrc);
    const int moff = ANAL ? N - 1 : a.Lsrc - 1, lds = ANAL ? N : a.Lsrc;
    // source row of column pair p (sign sg, map b); -1: absent pair
    auto src_row = [&](int p) -> long long {
        const int sg = p / BT, b = p % BT;
        if (b0 + b >= a.B || (sg == 1 && !two)) return -1;
        const int mi = sg == 0 ? (CPLX ? m + moff : m) : (-m + moff);
        return (long long)(b0 + b) * nmi_src + mi;
    };
    auto kstart = [&](int c) -> int { return ANAL ? 32 * klist[c] : m + 32 * (ibase + c); };

    if (warp < LH_BWARPS) {
        // ------------------------------------------------ operand B, drains, epilogue
        // unit of this thread in every chunk: column pair p, K values 8 kq .. 8 kq + 7
        const int p = 8 * warp + (lane & 3) + 4 * ((lane >> 3) & 1);
        const int kq = ((lane >> 2) & 1) + 2 * (lane >> 4);
        const long long rp = src_row(p);
        const float2 *row = rp >= 0 ? a.src + rp * lds : nullptr;
        const float cs = rp >= 0 ? a.csc[rp] : 0.f;
        const float *fac = (ANAL || !a.kfac) ? nullptr : kf_s - m;   // c_l by degree, from shared memory
        // the parity of the first K of every chunk is that of kstart(0), so
        // whether the thread's 64 source bytes are 16-byte aligned is fixed
        const bool al16 = row && ((reinterpret_cast<uintptr_t>(row + (ANAL ? 0 : m) + 8 * kq) & 15) == 0);
        float sum[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) sum[i] = 0.f;
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        const int h = warp >> 2;
        auto drain = [&](int g) {                     // accumulator g % LH_NACC into sum
            const int cl = min(LH_D * g + LH_D - 1, nk - 1);   // the group's last chunk
            lt_spin(&sy.done[cl % LH_NR], par(cl, LH_NR), abort);
            tc::fence_after();
            const uint32_t acc = tmem + lane_addr + (uint32_t)(128 * (g % LH_NACC) + 64 * h);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tc::tmem_ld16(acc + 16 * q, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[16 * q + i] += v[i];
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.tempty[g % LH_NACC]);
        };
        // raw slot of chunk c: the thread's q-th 16 bytes at (256 q + tid) 16
        auto raw = [&](int c, int q) -> unsigned char * {
            return smem + LH_RAW_OFF + (c % LH_NRAW) * LH_STAGE + (256 * q + tid) * 16;
        };
        // asynchronous copies of the thread's 8 values of chunk c (zeros past N and
        // for absent pairs), one commit group per chunk, empty past the last chunk
        auto issue = [&](int c) {
            if (c < nk) {
                const int k = kstart(c) + 8 * kq, kv = row ? N - k : 0;
                if (al16) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int nb = min(16, max(0, 8 * (kv - 2 * q)));
                        tc::cp_async16(tc::smem_addr(raw(c, q)), nb ? (const void *)(row + k + 2 * q) : a.src, nb);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const bool in = q < kv;
                        tc::cp_async8(tc::smem_addr(raw(c, q >> 1) + 8 * (q & 1)), in ? (const void *)(row + k + q) : a.src,
                                      in ? 8 : 0);
                    }
                }
            }
            tc::cp_async_commit();
        };
        auto store = [&](int c) {
            unsigned char *Bst = smem + LH_B_OFF + (c % LH_NB) * LH_STAGE;
            float xr[8], xi[8];
            const int k = kstart(c) + 8 * kq;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 x = *reinterpret_cast<const float4 *>(raw(c, q));
                float f0 = cs, f1 = cs;
                if (fac) {
                    if (k + 2 * q < N) f0 *= fac[k + 2 * q];
                    if (k + 2 * q + 1 < N) f1 *= fac[k + 2 * q + 1];
                }
                xr[2 * q] = x.x * f0;
                xi[2 * q] = x.y * f0;
                xr[2 * q + 1] = x.z * f1;
                xi[2 * q + 1] = x.w * f1;
            }
            uint4 hr, lr, hi, li;
            lh_split8(xr, hr, lr);
            lh_split8(xi, hi, li);
            const int n0 = 2 * p, n1 = 2 * p + 1;
            *reinterpret_cast<uint4 *>(Bst + lh_sw(n0, 16 * kq)) = hr;
            *reinterpret_cast<uint4 *>(Bst + lh_sw(n0, 64 + 16 * kq)) = lr;
            *reinterpret_cast<uint4 *>(Bst + lh_sw(n1, 16 * kq)) = hi;
            *reinterpret_cast<uint4 *>(Bst + lh_sw(n1, 64 + 16 * kq)) = li;
        };
        int drained = 0;
        if (ANAL) lt_spin(&sy.mfull, 0, abort);       // the chunks' ring blocks (klist) have landed
        for (int c = 0; c < LH_NRAW - 1; ++c) issue(c);
        // output index of this thread in the epilogue (TMEM lane = degree or ring)
        const int oidx = ANAL ? m + 128 * tile + 32 * (warp & 3) + lane : 128 * tile + 32 * (warp & 3) + lane;
        for (int c = 0; c < nk; ++c) {
            if (c == (nk > 8 ? nk - 8 : 0) && oidx < N) {
                // bring the output lines (and their address translations) close before the epilogue
#pragma unroll 4
                for (int j = 0; j < 32; ++j) {
                    const long long ro = epi_row[32 * h + j];
                    if (ro >= 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.dst + ro + oidx));
                }
            }
            issue(c + LH_NRAW - 1);                   // its slot held chunk c - 1, already stored
            // the accumulator of group c / LH_D - LH_NACC must be drained before chunk c's MMAs
            while (drained <= c / LH_D - LH_NACC) drain(drained++);
            if (c >= LH_NB) lt_spin(&sy.done[(c - LH_NB) % LH_NR], par(c - LH_NB, LH_NR), abort);
            tc::cp_async_wait<LH_NRAW - 1>();         // chunk c's copies have landed
            store(c);
            lt_warp_arrive(&sy.bfull[c % LH_NB], lane);
        }
        tc::cp_async_wait<0>();
        while (drained < ng) drain(drained++);
        if (!sy.abort && oidx < N) {
            // epilogue: TMEM lane = output index (degree or ring), accumulator column
            // pair = (map, sign of m); eight pairs per batch of loads and stores
            const float fo = (ANAL && a.kfac) ? a.kfac[oidx] : 1.f;
#pragma unroll
            for (int jb = 0; jb < 32; jb += 8) {
                float2 w[8];
                if (ANAL && a.accumulate) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const long long ro = epi_row[32 * h + jb + j];
                        w[j] = ro >= 0 ? a.dst[ro + oidx] : make_float2(0.f, 0.f);
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int pp = 32 * h + jb + j;
                    const long long ro = epi_row[pp];
                    if (ro >= 0) {
                        const float fs = epi_f[pp] * fo;
                        float2 v = make_float2(sum[2 * (jb + j)] * fs, sum[2 * (jb + j) + 1] * fs);
                        if (ANAL && a.accumulate) {
                            v.x += w[j].x;
                            v.y += w[j].y;
                        }
                        a.dst[ro + oidx] = v;
                    }
                }
            }
        }
    } else if (warp == LH_COPY_WARP) {
        // ------------------------------------------------ operand A: four table blocks per chunk
        if (lane == 0) {
            int issued = 0;
            lt_spin(&sy.mfull, 0, abort);              // the chunks' table blocks (blks) have landed
            for (int c = 0; c < nk; ++c) {
                if (c >= LH_NA && !lt_spin(&sy.done[(c - LH_NA) % LH_NR], par(c - LH_NA, LH_NR), abort)) break;
                if (*abort) break;
                const int s = c % LH_NA;
                unsigned char *dstA = smem + s * LH_STAGE;
                const int4 bl = blks[c];
                tc::mbar_arrive_expect_tx(&sy.afull[s], LH_STAGE);
                if (bl.y == bl.x + 1 && bl.z == bl.x + 2 && bl.w == bl.x + 3) {
                    // four adjacent blocks: one copy
                    tc::bulk_g2s(dstA, a.tab + (size_t)bl.x * LI_BLK, LH_STAGE, &sy.afull[s]);
                } else {
                    tc::bulk_g2s(dstA, a.tab + (size_t)bl.x * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + LI_BLK, a.tab + (size_t)bl.y * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + 2 * LI_BLK, a.tab + (size_t)bl.z * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + 3 * LI_BLK, a.tab + (size_t)bl.w * LI_BLK, LI_BLK, &sy.afull[s]);
                }
                issued = c + 1;
            }
            // no copy in flight when the block ends (only possible after an abort)
            tc::mbar_wait(&sy.mfull, 0, 1u << 22);
            for (int c = issued - LH_NA > 0 ? issued - LH_NA : 0; c < issued; ++c)
                tc::mbar_wait(&sy.afull[c % LH_NA], par(c, LH_NA), 1u << 22);
        }
    } else if (lane == 0) {
        // ------------------------------------------------ MMA issue: A and B from shared memory
        constexpr uint32_t IDESC = idesc_f16(128, 128);
        for (int c = 0; c < nk; ++c) {
            const int g = c / LH_D;
            const bool first = c % LH_D == 0;           // first chunk of group g
            bool ok = lt_spin(&sy.afull[c % LH_NA], par(c, LH_NA), abort);
            ok = lt_spin(&sy.bfull[c % LH_NB], par(c, LH_NB), abort) && ok;
            if (first && g >= LH_NACC) ok = lt_spin(&sy.tempty[g % LH_NACC], ((g / LH_NACC) - 1) & 1, abort) && ok;
            tc::fence_after();
            if (ok) {
                const uint32_t abase = tc::smem_addr(smem + (c % LH_NA) * LH_STAGE);
                const uint32_t bbase = tc::smem_addr(smem + LH_B_OFF + (c % LH_NB) * LH_STAGE);
                const uint32_t acc = tmem + (uint32_t)(128 * (g % LH_NACC));
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t ah = tc::smem_desc_sw128(abase + 32 * ks);
                    const uint64_t al = tc::smem_desc_sw128(abase + 64 + 32 * ks);
                    const uint64_t bh = tc::smem_desc_sw128(bbase + 32 * ks);
                    const uint64_t bl = tc::smem_desc_sw128(bbase + 64 + 32 * ks);
                    mma_f16_ss(acc, ah, bh, IDESC, (ks > 0 || !first) ? 1u : 0u);
                    mma_f16_ss(acc, ah, bl, IDESC, 1u);
                    mma_f16_ss(acc, al, bh, IDESC, 1u);
                }
            }
            tc::mma_commit(&sy.done[c % LH_NR]);
        }
        tc::mma_commit(&sy.fin);
        tc::mbar_wait(&sy.fin, 0, 1u << 22);   // no MMA in flight when TMEM is released
    }
    tc::fence_before();
    __syncthreads();
    if (warp == LH_MMA_WARP) tc::tmem_free(tmem, LT_TMEM_COLS);
    if (tid == 0 && sy.abort) atomicExch(a.err, 1);
}

}  // namespace s2g

namespace s2g {

// ---------------------------------------------------------------- two kernel sets
// k_leg_h16s2: the synthesis of two maps that share the band-limit N and the
// coefficients f_lm and differ in the kernel factors (two wavelet scales whose
// band-limits are both capped at L):
//   F^s_m(theta_t) = scale sum_l lambda_lm(theta_t) c^s_l f_lm,  s = 0, 1.
// One stream of the table feeds both: per chunk the four table blocks are
// copied once and the MMAs run for each set against its own operand B (the
// same raw f_lm rows, scaled by c^s_l and the set's column scale).  Tensor
// memory holds, per set, one accumulator (four K chunks) and the running sum
// (columns 256 s and 256 s + 128): the drain warps add the accumulator into the
// running sum with FP32 adds (the same sums the single-set kernel keeps in
// registers, for which two sets leave too few registers).
constexpr int LH2_NA = 5, LH2_NB = 2, LH2_NRAW = 3;
constexpr int LH2_B_OFF = LH2_NA * LH_STAGE;                   // stage s: set 0, set 1 (16 KB each)
constexpr int LH2_RAW_OFF = LH2_B_OFF + LH2_NB * 2 * LH_STAGE;
constexpr int LH2_BLKS_OFF = LH2_RAW_OFF + LH2_NRAW * LH_STAGE;
constexpr int LH2_EPI_OFF = LH2_BLKS_OFF + LI_MAXK * 16;       // output row [64], factors [2][64]
constexpr int LH2_KF_OFF = LH2_EPI_OFF + 64 * 8 + 2 * 64 * 4;  // c^s_l of degrees m .. N - 1 [2][LH_MAXN]
constexpr int LH2_SYNC_OFF = LH2_KF_OFF + 2 * LH_MAXN * 4;
struct Lh2Sync {
    uint64_t afull[LH2_NA], bfull[LH2_NB], done[LH_NR], tempty, fin, mfull;
    uint32_t tslot;
    int abort, nk, ibase;
};
static_assert(sizeof(Lh2Sync) <= LH_SYNC_BYTES, "sync block");
static_assert(LH2_NA < LH_NR && LH2_NB < LH_D, "barrier ring: a drain follows its group's last chunk");
__host__ __device__ constexpr size_t leg_h16s2_smem() { return (size_t)LH2_SYNC_OFF + LH_SYNC_BYTES + 1024; }
static_assert(leg_h16s2_smem() <= 227 * 1024, "shared memory");

struct LegH16Args2 {
    const float2 *src;       // f [b][mi][l] (rectangle Lsrc)
    int Lsrc;
    const float *kfac[2];    // per-degree factors of the two sets
    float scale;
    float2 *dst[2];          // F^s [b][mi][t] (band-limit N)
    int N, B;
    LegImg T;
    const unsigned char *tab;   // ts
    const float *csc[2];     // column scales of c^s_l f_lm [b][mi]
    int *err;
};

// 16 consecutive 32-bit columns of this thread's TMEM lane (two x8 stores)
__device__ __forceinline__ void lh_tmem_st16(uint32_t taddr, const float (&v)[16])
{
    tc::tmem_st8(taddr, *reinterpret_cast<const float(*)[8]>(v));
    tc::tmem_st8(taddr + 8, *reinterpret_cast<const float(*)[8]>(v + 8));
}

template <bool CPLX>
static __global__ void __launch_bounds__(LH_THREADS, 1) k_leg_h16s2(LegH16Args2 a)
{
    using Cols = LegCols<CPLX>;
    constexpr int BT = Cols::BT;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    Lh2Sync &sy = *reinterpret_cast<Lh2Sync *>(smem + LH2_SYNC_OFF);
    int4 *blks = reinterpret_cast<int4 *>(smem + LH2_BLKS_OFF);
    long long *epi_row = reinterpret_cast<long long *>(smem + LH2_EPI_OFF);
    float *epi_f = reinterpret_cast<float *>(smem + LH2_EPI_OFF + 64 * 8);       // [2][64]
    float *kf_s = reinterpret_cast<float *>(smem + LH2_KF_OFF);                  // [2][LH_MAXN]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.N;
    const int tile = blockIdx.x, m = blockIdx.y, b0 = blockIdx.z * BT;
    const bool two = CPLX && m > 0;
    volatile int *abort = &sy.abort;
    auto par = [](int c, int n) -> uint32_t { return (uint32_t)((c / n) & 1); };

    if (warp == LH_MMA_WARP) {
        tc::tmem_alloc(&sy.tslot, LT_TMEM_COLS);
    } else if (warp == LH_COPY_WARP && lane == 0) {
#pragma unroll
        for (int i = 0; i < LH2_NA; ++i) tc::mbar_init(&sy.afull[i], 1);
#pragma unroll
        for (int i = 0; i < LH2_NB; ++i) tc::mbar_init(&sy.bfull[i], LH_BWARPS);
#pragma unroll
        for (int i = 0; i < LH_NR; ++i) tc::mbar_init(&sy.done[i], 1);
        tc::mbar_init(&sy.tempty, LH_BWARPS);
        tc::mbar_init(&sy.fin, 1);
        tc::mbar_init(&sy.mfull, 1);
        sy.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const int4 md = a.T.smeta[(size_t)m * ((N + 127) / 128) + tile];
        sy.nk = md.y;
        sy.ibase = md.z;
        const uint32_t nb = (uint32_t)md.y * 16u;
        tc::mbar_arrive_expect_tx(&sy.mfull, nb);
        if (md.y > 0) tc::bulk_g2s(blks, a.T.sblk + md.x, nb, &sy.mfull);
    }
    if (warp < LH_BWARPS)
        for (int l = m + tid; l < N; l += 32 * LH_BWARPS) {
            kf_s[l - m] = a.kfac[0] ? a.kfac[0][l] : 1.f;
            kf_s[LH_MAXN + l - m] = a.kfac[1] ? a.kfac[1][l] : 1.f;
        }
    const int nmi_src = CPLX ? 2 * a.Lsrc - 1 : a.Lsrc;
    const int moff = a.Lsrc - 1;
    if (warp < LH_BWARPS && (lane & 0x14) == 0) {
        const int p = 8 * warp + (lane & 3) + 4 * ((lane >> 3) & 1);
        const int sg = p / BT, b = p % BT;
        const bool live = b0 + b < a.B && (sg == 0 || two);
        const int mi = sg == 0 ? (CPLX ? m + moff : m) : (-m + moff);
        const int nmi_dst = CPLX ? 2 * N - 1 : N;
        const int mid = sg == 0 ? (CPLX ? m + N - 1 : m) : (-m + N - 1);
        const float sgn = (sg == 1 && (m & 1)) ? -1.f : 1.f;
        const size_t rs = (size_t)(b0 + b) * nmi_src + mi;
#pragma unroll
        for (int s = 0; s < 2; ++s)
            epi_f[64 * s + p] = live ? sgn * a.scale * (1.f / LH_TSCALE) / a.csc[s][rs] : 0.f;
        epi_row[p] = live ? ((long long)(b0 + b) * nmi_dst + mid) * N : -1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sy.tslot;
    const int nk = sy.nk, ibase = sy.ibase;
    const int ng = (nk + LH_D - 1) / LH_D;
    auto kstart = [&](int c) -> int { return m + 32 * (ibase + c); };

    if (warp < LH_BWARPS) {
        // ------------------------------------------------ operand B of both sets, drains, epilogue
        const int p = 8 * warp + (lane & 3) + 4 * ((lane >> 3) & 1);
        const int kq = ((lane >> 2) & 1) + 2 * (lane >> 4);
        const int sg = p / BT, b = p % BT;
        const bool live = b0 + b < a.B && (sg == 0 || two);
        const long long rp = live ? (long long)(b0 + b) * nmi_src + (sg == 0 ? (CPLX ? m + moff : m) : (-m + moff)) : -1;
        const float2 *row = live ? a.src + rp * a.Lsrc : nullptr;
        const float cs0 = live ? a.csc[0][rp] : 0.f, cs1 = live ? a.csc[1][rp] : 0.f;
        const bool al16 = row && ((reinterpret_cast<uintptr_t>(row + m + 8 * kq) & 15) == 0);
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        const int h = warp >> 2;
        // the accumulators of group g into the running sums (both sets)
        auto drain = [&](int g) {
            const int cl = min(LH_D * g + LH_D - 1, nk - 1);
            lt_spin(&sy.done[cl % LH_NR], par(cl, LH_NR), abort);
            tc::fence_after();
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint32_t acc = tmem + lane_addr + (uint32_t)(256 * s + 64 * h);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v[16];
                    tc::tmem_ld16(acc + 16 * q, v);
                    if (g > 0) {
                        float w[16];
                        tc::tmem_ld16(acc + 128 + 16 * q, w);
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] += w[i];
                    }
                    lh_tmem_st16(acc + 128 + 16 * q, v);
                }
            }
            tc::tmem_wait_st();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.tempty);
        };
        auto raw = [&](int c, int q) -> unsigned char * {
            return smem + LH2_RAW_OFF + (c % LH2_NRAW) * LH_STAGE + (256 * q + tid) * 16;
        };
        auto issue = [&](int c) {
            if (c < nk) {
                const int k = kstart(c) + 8 * kq, kv = row ? N - k : 0;
                if (al16) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int nb = min(16, max(0, 8 * (kv - 2 * q)));
                        tc::cp_async16(tc::smem_addr(raw(c, q)), nb ? (const void *)(row + k + 2 * q) : a.src, nb);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const bool in = q < kv;
                        tc::cp_async8(tc::smem_addr(raw(c, q >> 1) + 8 * (q & 1)), in ? (const void *)(row + k + q) : a.src,
                                      in ? 8 : 0);
                    }
                }
            }
            tc::cp_async_commit();
        };
        auto store = [&](int c) {
            unsigned char *Bst = smem + LH2_B_OFF + (c % LH2_NB) * 2 * LH_STAGE;
            const int k = kstart(c) + 8 * kq;
            float2 x[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = *reinterpret_cast<const float4 *>(raw(c, q));
                x[2 * q] = make_float2(v.x, v.y);
                x[2 * q + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                float xr[8], xi[8];
                const float *kf = kf_s + LH_MAXN * s - m;
                const float cs = s ? cs1 : cs0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float f = (k + q < N) ? cs * kf[k + q] : 0.f;
                    xr[q] = x[q].x * f;
                    xi[q] = x[q].y * f;
                }
                uint4 hr, lr, hi, li;
                lh_split8(xr, hr, lr);
                lh_split8(xi, hi, li);
                unsigned char *Bs = Bst + s * LH_STAGE;
                const int n0 = 2 * p, n1 = 2 * p + 1;
                *reinterpret_cast<uint4 *>(Bs + lh_sw(n0, 16 * kq)) = hr;
                *reinterpret_cast<uint4 *>(Bs + lh_sw(n0, 64 + 16 * kq)) = lr;
                *reinterpret_cast<uint4 *>(Bs + lh_sw(n1, 16 * kq)) = hi;
                *reinterpret_cast<uint4 *>(Bs + lh_sw(n1, 64 + 16 * kq)) = li;
            }
        };
        const int oidx = 128 * tile + 32 * (warp & 3) + lane;   // output ring (TMEM lane)
        int drained = 0;
        for (int c = 0; c < LH2_NRAW - 1; ++c) issue(c);
        for (int c = 0; c < nk; ++c) {
            if (c == (nk > 8 ? nk - 8 : 0) && oidx < N) {
#pragma unroll 4
                for (int j = 0; j < 32; ++j) {
                    const long long ro = epi_row[32 * h + j];
                    if (ro >= 0) {
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.dst[0] + ro + oidx));
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.dst[1] + ro + oidx));
                    }
                }
            }
            issue(c + LH2_NRAW - 1);
            if (c >= LH2_NB) {
                // stage c % LH2_NB is free once chunk c - LH2_NB is done; if that chunk
                // closed a group, its accumulators go into the running sums now (the
                // MMAs of the next group wait for it)
                lt_spin(&sy.done[(c - LH2_NB) % LH_NR], par(c - LH2_NB, LH_NR), abort);
                if ((c - LH2_NB) % LH_D == LH_D - 1) drain(drained++);
            }
            tc::cp_async_wait<LH2_NRAW - 1>();
            store(c);
            lt_warp_arrive(&sy.bfull[c % LH2_NB], lane);
        }
        tc::cp_async_wait<0>();
        while (drained < ng) drain(drained++);
        // the TMEM loads are warp-collective: the whole warp takes them (the abort
        // flag read once per warp), and only the lanes of rings below N store
        if (!__shfl_sync(0xffffffffu, sy.abort, 0)) {
            // epilogue: TMEM lane = ring; columns 64 h .. of each set's running sum
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint32_t tot = tmem + lane_addr + (uint32_t)(256 * s + 128 + 64 * h);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v[16];
                    if (nk > 0) {
                        tc::tmem_ld16(tot + 16 * q, v);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int pp = 32 * h + 8 * q + i;
                        const long long ro = epi_row[pp];
                        if (ro >= 0 && oidx < N) {
                            const float f = epi_f[64 * s + pp];
                            a.dst[s][ro + oidx] = make_float2(v[2 * i] * f, v[2 * i + 1] * f);
                        }
                    }
                }
            }
        }
    } else if (warp == LH_COPY_WARP) {
        // ------------------------------------------------ the table blocks of each chunk, once for both sets
        if (lane == 0) {
            int issued = 0;
            lt_spin(&sy.mfull, 0, abort);
            for (int c = 0; c < nk; ++c) {
                if (c >= LH2_NA && !lt_spin(&sy.done[(c - LH2_NA) % LH_NR], par(c - LH2_NA, LH_NR), abort)) break;
                if (*abort) break;
                const int s = c % LH2_NA;
                unsigned char *dstA = smem + s * LH_STAGE;
                const int4 bl = blks[c];
                tc::mbar_arrive_expect_tx(&sy.afull[s], LH_STAGE);
                if (bl.y == bl.x + 1 && bl.z == bl.x + 2 && bl.w == bl.x + 3) {
                    tc::bulk_g2s(dstA, a.tab + (size_t)bl.x * LI_BLK, LH_STAGE, &sy.afull[s]);
                } else {
                    tc::bulk_g2s(dstA, a.tab + (size_t)bl.x * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + LI_BLK, a.tab + (size_t)bl.y * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + 2 * LI_BLK, a.tab + (size_t)bl.z * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + 3 * LI_BLK, a.tab + (size_t)bl.w * LI_BLK, LI_BLK, &sy.afull[s]);
                }
                issued = c + 1;
            }
            tc::mbar_wait(&sy.mfull, 0, 1u << 22);
            for (int c = issued - LH2_NA > 0 ? issued - LH2_NA : 0; c < issued; ++c)
                tc::mbar_wait(&sy.afull[c % LH2_NA], par(c, LH2_NA), 1u << 22);
        }
    } else if (lane == 0) {
        // ------------------------------------------------ MMAs: both sets per chunk
        constexpr uint32_t IDESC = idesc_f16(128, 128);
        for (int c = 0; c < nk; ++c) {
            const int g = c / LH_D;
            const bool first = c % LH_D == 0;
            bool ok = lt_spin(&sy.afull[c % LH2_NA], par(c, LH2_NA), abort);
            ok = lt_spin(&sy.bfull[c % LH2_NB], par(c, LH2_NB), abort) && ok;
            if (first && g >= 1) ok = lt_spin(&sy.tempty, (uint32_t)((g - 1) & 1), abort) && ok;
            tc::fence_after();
            if (ok) {
                const uint32_t abase = tc::smem_addr(smem + (c % LH2_NA) * LH_STAGE);
                const uint32_t bst = tc::smem_addr(smem + LH2_B_OFF + (c % LH2_NB) * 2 * LH_STAGE);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const uint32_t acc = tmem + (uint32_t)(256 * s);
                    const uint32_t bbase = bst + s * LH_STAGE;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ah = tc::smem_desc_sw128(abase + 32 * ks);
                        const uint64_t al = tc::smem_desc_sw128(abase + 64 + 32 * ks);
                        const uint64_t bh = tc::smem_desc_sw128(bbase + 32 * ks);
                        const uint64_t bl = tc::smem_desc_sw128(bbase + 64 + 32 * ks);
                        mma_f16_ss(acc, ah, bh, IDESC, (ks > 0 || !first) ? 1u : 0u);
                        mma_f16_ss(acc, ah, bl, IDESC, 1u);
                        mma_f16_ss(acc, al, bh, IDESC, 1u);
                    }
                }
            }
            tc::mma_commit(&sy.done[c % LH_NR]);
        }
        tc::mma_commit(&sy.fin);
        tc::mbar_wait(&sy.fin, 0, 1u << 22);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == LH_MMA_WARP) tc::tmem_free(tmem, LT_TMEM_COLS);
    if (tid == 0 && sy.abort) atomicExch(a.err, 1);
}

}  // namespace s2g

namespace s2g {

// k_leg_h16a2: the analysis of two maps at one band-limit N (two wavelet scales
// whose band-limits are both capped at L) into one set of coefficients:
//   f_lm (+)= scale (c^0_l sum_t lambda_lm(theta_t) G^0_m(theta_t) + c^1_l sum_t lambda_lm(theta_t) G^1_m(theta_t)).
// One stream of the table feeds both contractions, as in k_leg_h16s2; each set
// has its own source rows (copied by cp.async into its own ring, two chunks
// deep, with L2 prefetches four chunks ahead) and column scales.
constexpr int LH3_NA = 5, LH3_NB = 2, LH3_NRAW = 2;
constexpr int LH3_B_OFF = LH3_NA * LH_STAGE;                   // stage s: set 0, set 1
constexpr int LH3_RAW_OFF = LH3_B_OFF + LH3_NB * 2 * LH_STAGE; // slot r: set 0, set 1
constexpr int LH3_LIST_OFF = LH3_RAW_OFF + LH3_NRAW * 2 * LH_STAGE;
constexpr int LH3_BLKS_OFF = LH3_LIST_OFF + LI_MAXK * 4;
constexpr int LH3_EPI_OFF = LH3_BLKS_OFF + LI_MAXK * 16;       // output row [64], factors [2][64]
constexpr int LH3_SYNC_OFF = LH3_EPI_OFF + 64 * 8 + 2 * 64 * 4;
struct Lh3Sync {
    uint64_t afull[LH3_NA], bfull[LH3_NB], done[LH_NR], tempty, fin, mfull;
    uint32_t tslot;
    int abort, nk, ibase;
};
static_assert(sizeof(Lh3Sync) <= LH_SYNC_BYTES, "sync block");
static_assert(LH3_NA < LH_NR && LH3_NB < LH_D, "barrier ring: a drain follows its group's last chunk");
__host__ __device__ constexpr size_t leg_h16a2_smem() { return (size_t)LH3_SYNC_OFF + LH_SYNC_BYTES + 1024; }
static_assert(leg_h16a2_smem() <= 227 * 1024, "shared memory");

struct LegH16ArgsA2 {
    const float2 *src[2];    // G^s [b][mi][t] (band-limit N)
    const float *kfac[2];    // per-degree factors of the two sets (nullptr: 1)
    float scale;
    int accumulate;          // add to dst
    float2 *dst;             // f [b][mi][l] (rectangle Ldst)
    int Ldst;
    int N, B;
    LegImg T;
    const unsigned char *tab;   // ta
    const float *csc[2];     // column scales of G^s [b][mi]
    int *err;
};

template <bool CPLX>
static __global__ void __launch_bounds__(LH_THREADS, 1) k_leg_h16a2(LegH16ArgsA2 a)
{
    using Cols = LegCols<CPLX>;
    constexpr int BT = Cols::BT;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    Lh3Sync &sy = *reinterpret_cast<Lh3Sync *>(smem + LH3_SYNC_OFF);
    int *klist = reinterpret_cast<int *>(smem + LH3_LIST_OFF);
    int4 *blks = reinterpret_cast<int4 *>(smem + LH3_BLKS_OFF);
    long long *epi_row = reinterpret_cast<long long *>(smem + LH3_EPI_OFF);
    float *epi_f = reinterpret_cast<float *>(smem + LH3_EPI_OFF + 64 * 8);       // [2][64]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.N;
    const int2 md0 = a.T.adt[blockIdx.x];
    const int m = md0.x, tile = md0.y, b0 = blockIdx.y * BT;
    const bool two = CPLX && m > 0;
    volatile int *abort = &sy.abort;
    auto par = [](int c, int n) -> uint32_t { return (uint32_t)((c / n) & 1); };

    if (warp == LH_MMA_WARP) {
        tc::tmem_alloc(&sy.tslot, LT_TMEM_COLS);
    } else if (warp == LH_COPY_WARP && lane == 0) {
#pragma unroll
        for (int i = 0; i < LH3_NA; ++i) tc::mbar_init(&sy.afull[i], 1);
#pragma unroll
        for (int i = 0; i < LH3_NB; ++i) tc::mbar_init(&sy.bfull[i], LH_BWARPS);
#pragma unroll
        for (int i = 0; i < LH_NR; ++i) tc::mbar_init(&sy.done[i], 1);
        tc::mbar_init(&sy.tempty, LH_BWARPS);
        tc::mbar_init(&sy.fin, 1);
        tc::mbar_init(&sy.mfull, 1);
        sy.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const int4 md = a.T.ameta[blockIdx.x];
        sy.nk = md.y;
        sy.ibase = 0;
        const uint32_t nb = (uint32_t)md.y * 16u, nl = (uint32_t)((md.y + 3) & ~3) * 4u;
        tc::mbar_arrive_expect_tx(&sy.mfull, nb + nl);
        if (md.y > 0) {
            tc::bulk_g2s(blks, a.T.ablk + md.x, nb, &sy.mfull);
            tc::bulk_g2s(klist, a.T.ack + md.z, nl, &sy.mfull);
        }
    }
    const int nmi_src = CPLX ? 2 * N - 1 : N;
    const int moff = N - 1;
    if (warp < LH_BWARPS && (lane & 0x14) == 0) {
        const int p = 8 * warp + (lane & 3) + 4 * ((lane >> 3) & 1);
        const int sg = p / BT, b = p % BT;
        const bool live = b0 + b < a.B && (sg == 0 || two);
        const int mi = sg == 0 ? (CPLX ? m + moff : m) : (-m + moff);
        const int nmi_dst = CPLX ? 2 * a.Ldst - 1 : a.Ldst;
        const int mid = sg == 0 ? (CPLX ? m + a.Ldst - 1 : m) : (-m + a.Ldst - 1);
        const float sgn = (sg == 1 && (m & 1)) ? -1.f : 1.f;
        const size_t rs = (size_t)(b0 + b) * nmi_src + mi;
#pragma unroll
        for (int s = 0; s < 2; ++s)
            epi_f[64 * s + p] = live ? sgn * a.scale * (1.f / LH_TSCALE) / a.csc[s][rs] : 0.f;
        epi_row[p] = live ? ((long long)(b0 + b) * nmi_dst + mid) * a.Ldst : -1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sy.tslot;
    const int nk = sy.nk;
    const int ng = (nk + LH_D - 1) / LH_D;
    auto kstart = [&](int c) -> int { return 32 * klist[c]; };

    if (warp < LH_BWARPS) {
        // ------------------------------------------------ operand B of both sets, drains, epilogue
        const int p = 8 * warp + (lane & 3) + 4 * ((lane >> 3) & 1);
        const int kq = ((lane >> 2) & 1) + 2 * (lane >> 4);
        const int sg = p / BT, b = p % BT;
        const bool live = b0 + b < a.B && (sg == 0 || two);
        const long long rp = live ? (long long)(b0 + b) * nmi_src + (sg == 0 ? (CPLX ? m + moff : m) : (-m + moff)) : -1;
        const float2 *row0 = live ? a.src[0] + rp * N : nullptr;
        const float2 *row1 = live ? a.src[1] + rp * N : nullptr;
        const float cs0 = live ? a.csc[0][rp] : 0.f, cs1 = live ? a.csc[1][rp] : 0.f;
        // the first K of every chunk is a multiple of 32, so alignment is the row's
        const bool al0 = row0 && ((reinterpret_cast<uintptr_t>(row0 + 8 * kq) & 15) == 0);
        const bool al1 = row1 && ((reinterpret_cast<uintptr_t>(row1 + 8 * kq) & 15) == 0);
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        const int h = warp >> 2;
        auto drain = [&](int g) {
            const int cl = min(LH_D * g + LH_D - 1, nk - 1);
            lt_spin(&sy.done[cl % LH_NR], par(cl, LH_NR), abort);
            tc::fence_after();
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint32_t acc = tmem + lane_addr + (uint32_t)(256 * s + 64 * h);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v[16];
                    tc::tmem_ld16(acc + 16 * q, v);
                    if (g > 0) {
                        float w[16];
                        tc::tmem_ld16(acc + 128 + 16 * q, w);
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] += w[i];
                    }
                    lh_tmem_st16(acc + 128 + 16 * q, v);
                }
            }
            tc::tmem_wait_st();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.tempty);
        };
        auto raw = [&](int c, int s, int q) -> unsigned char * {
            return smem + LH3_RAW_OFF + ((c % LH3_NRAW) * 2 + s) * LH_STAGE + (256 * q + tid) * 16;
        };
        auto issue_set = [&](int c, int s, const float2 *row, bool al) {
            const int k = kstart(c) + 8 * kq, kv = row ? N - k : 0;
            if (al) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int nb = min(16, max(0, 8 * (kv - 2 * q)));
                    tc::cp_async16(tc::smem_addr(raw(c, s, q)), nb ? (const void *)(row + k + 2 * q) : (const void *)a.src[0],
                                   nb);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const bool in = q < kv;
                    tc::cp_async8(tc::smem_addr(raw(c, s, q >> 1) + 8 * (q & 1)),
                                  in ? (const void *)(row + k + q) : (const void *)a.src[0], in ? 8 : 0);
                }
            }
        };
        auto issue = [&](int c) {
            if (c < nk) {
                issue_set(c, 0, row0, al0);
                issue_set(c, 1, row1, al1);
            }
            tc::cp_async_commit();
            // the rows of chunk c + 4 into L2, so that its copies find them there
            if (c + 4 < nk) {
                const int k = kstart(c + 4) + 8 * kq;
                if (k < N) {
                    if (row0) asm volatile("prefetch.global.L2 [%0];" ::"l"(row0 + k));
                    if (row1) asm volatile("prefetch.global.L2 [%0];" ::"l"(row1 + k));
                }
            }
        };
        auto store = [&](int c) {
            unsigned char *Bst = smem + LH3_B_OFF + (c % LH3_NB) * 2 * LH_STAGE;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                float xr[8], xi[8];
                const float cs = s ? cs1 : cs0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 v = *reinterpret_cast<const float4 *>(raw(c, s, q));
                    xr[2 * q] = v.x * cs;
                    xi[2 * q] = v.y * cs;
                    xr[2 * q + 1] = v.z * cs;
                    xi[2 * q + 1] = v.w * cs;
                }
                uint4 hr, lr, hi, li;
                lh_split8(xr, hr, lr);
                lh_split8(xi, hi, li);
                unsigned char *Bs = Bst + s * LH_STAGE;
                const int n0 = 2 * p, n1 = 2 * p + 1;
                *reinterpret_cast<uint4 *>(Bs + lh_sw(n0, 16 * kq)) = hr;
                *reinterpret_cast<uint4 *>(Bs + lh_sw(n0, 64 + 16 * kq)) = lr;
                *reinterpret_cast<uint4 *>(Bs + lh_sw(n1, 16 * kq)) = hi;
                *reinterpret_cast<uint4 *>(Bs + lh_sw(n1, 64 + 16 * kq)) = li;
            }
        };
        const int oidx = m + 128 * tile + 32 * (warp & 3) + lane;   // output degree (TMEM lane)
        int drained = 0;
        lt_spin(&sy.mfull, 0, abort);                  // the chunks' ring blocks (klist) have landed
        for (int c = 0; c < LH3_NRAW - 1; ++c) issue(c);
        for (int c = 0; c < nk; ++c) {
            if (c == (nk > 8 ? nk - 8 : 0) && oidx < N) {
#pragma unroll 4
                for (int j = 0; j < 32; ++j) {
                    const long long ro = epi_row[32 * h + j];
                    if (ro >= 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.dst + ro + oidx));
                }
            }
            issue(c + LH3_NRAW - 1);
            if (c >= LH3_NB) {
                lt_spin(&sy.done[(c - LH3_NB) % LH_NR], par(c - LH3_NB, LH_NR), abort);
                if ((c - LH3_NB) % LH_D == LH_D - 1) drain(drained++);
            }
            tc::cp_async_wait<LH3_NRAW - 1>();
            store(c);
            lt_warp_arrive(&sy.bfull[c % LH3_NB], lane);
        }
        tc::cp_async_wait<0>();
        while (drained < ng) drain(drained++);
        // the TMEM loads are warp-collective: the whole warp takes them, only the
        // lanes of degrees below N load and store the coefficients
        if (!__shfl_sync(0xffffffffu, sy.abort, 0)) {
            const bool in = oidx < N;
            const float k0 = (in && a.kfac[0]) ? a.kfac[0][oidx] : 1.f;
            const float k1 = (in && a.kfac[1]) ? a.kfac[1][oidx] : 1.f;
            const uint32_t tot = tmem + lane_addr + (uint32_t)(128 + 64 * h);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v0[16], v1[16];
                if (nk > 0) {
                    tc::tmem_ld16(tot + 16 * q, v0);
                    tc::tmem_ld16(tot + 256 + 16 * q, v1);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v0[i] = v1[i] = 0.f;
                }
                float2 w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const long long ro = epi_row[32 * h + 8 * q + i];
                    w[i] = (a.accumulate && in && ro >= 0) ? a.dst[ro + oidx] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int pp = 32 * h + 8 * q + i;
                    const long long ro = epi_row[pp];
                    if (in && ro >= 0) {
                        const float f0 = epi_f[pp] * k0, f1 = epi_f[64 + pp] * k1;
                        a.dst[ro + oidx] = make_float2(w[i].x + v0[2 * i] * f0 + v1[2 * i] * f1,
                                                       w[i].y + v0[2 * i + 1] * f0 + v1[2 * i + 1] * f1);
                    }
                }
            }
        }
    } else if (warp == LH_COPY_WARP) {
        if (lane == 0) {
            int issued = 0;
            lt_spin(&sy.mfull, 0, abort);
            for (int c = 0; c < nk; ++c) {
                if (c >= LH3_NA && !lt_spin(&sy.done[(c - LH3_NA) % LH_NR], par(c - LH3_NA, LH_NR), abort)) break;
                if (*abort) break;
                const int s = c % LH3_NA;
                unsigned char *dstA = smem + s * LH_STAGE;
                const int4 bl = blks[c];
                tc::mbar_arrive_expect_tx(&sy.afull[s], LH_STAGE);
                if (bl.y == bl.x + 1 && bl.z == bl.x + 2 && bl.w == bl.x + 3) {
                    tc::bulk_g2s(dstA, a.tab + (size_t)bl.x * LI_BLK, LH_STAGE, &sy.afull[s]);
                } else {
                    tc::bulk_g2s(dstA, a.tab + (size_t)bl.x * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + LI_BLK, a.tab + (size_t)bl.y * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + 2 * LI_BLK, a.tab + (size_t)bl.z * LI_BLK, LI_BLK, &sy.afull[s]);
                    tc::bulk_g2s(dstA + 3 * LI_BLK, a.tab + (size_t)bl.w * LI_BLK, LI_BLK, &sy.afull[s]);
                }
                issued = c + 1;
            }
            tc::mbar_wait(&sy.mfull, 0, 1u << 22);
            for (int c = issued - LH3_NA > 0 ? issued - LH3_NA : 0; c < issued; ++c)
                tc::mbar_wait(&sy.afull[c % LH3_NA], par(c, LH3_NA), 1u << 22);
        }
    } else if (lane == 0) {
        constexpr uint32_t IDESC = idesc_f16(128, 128);
        for (int c = 0; c < nk; ++c) {
            const int g = c / LH_D;
            const bool first = c % LH_D == 0;
            bool ok = lt_spin(&sy.afull[c % LH3_NA], par(c, LH3_NA), abort);
            ok = lt_spin(&sy.bfull[c % LH3_NB], par(c, LH3_NB), abort) && ok;
            if (first && g >= 1) ok = lt_spin(&sy.tempty, (uint32_t)((g - 1) & 1), abort) && ok;
            tc::fence_after();
            if (ok) {
                const uint32_t abase = tc::smem_addr(smem + (c % LH3_NA) * LH_STAGE);
                const uint32_t bst = tc::smem_addr(smem + LH3_B_OFF + (c % LH3_NB) * 2 * LH_STAGE);
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const uint32_t acc = tmem + (uint32_t)(256 * s);
                    const uint32_t bbase = bst + s * LH_STAGE;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ah = tc::smem_desc_sw128(abase + 32 * ks);
                        const uint64_t al = tc::smem_desc_sw128(abase + 64 + 32 * ks);
                        const uint64_t bh = tc::smem_desc_sw128(bbase + 32 * ks);
                        const uint64_t bl = tc::smem_desc_sw128(bbase + 64 + 32 * ks);
                        mma_f16_ss(acc, ah, bh, IDESC, (ks > 0 || !first) ? 1u : 0u);
                        mma_f16_ss(acc, ah, bl, IDESC, 1u);
                        mma_f16_ss(acc, al, bh, IDESC, 1u);
                    }
                }
            }
            tc::mma_commit(&sy.done[c % LH_NR]);
        }
        tc::mma_commit(&sy.fin);
        tc::mbar_wait(&sy.fin, 0, 1u << 22);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == LH_MMA_WARP) tc::tmem_free(tmem, LT_TMEM_COLS);
    if (tid == 0 && sy.abort) atomicExch(a.err, 1);
}

}  // namespace s2g
