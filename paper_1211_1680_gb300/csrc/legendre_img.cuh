// Precomputed Legendre values of the TF32X3 plans ("tables") and the
// tensor-core Legendre contractions that stream them:
//   k_leg_img<ANAL = true>   f_lm = scale c_l sum_t lambda_lm(theta_t) G_m(theta_t)  (last step of the MW quadrature)
//   k_leg_img<ANAL = false>  F_m(theta_t) = scale sum_l lambda_lm(theta_t) c_l f_lm  (Eq. harmonicssynthesis)
// The values lambda_lm(theta_t) are computed once per plan by the FP64
// recurrence of the FP64 kernels (legendre.cuh) from the same seeds and rounded
// to FP32, the value the recurrence kernels of these plans contract too.  So a
// launch reads each value once from HBM instead of running the float-float
// recurrence for every batch of maps.
//
// Table layout.  Blocks of 32 degrees x 32 rings, 4 KB each, row = degree
// (m + 32 i + r), 32 rings per 128-byte row, the 16-byte pieces of row r XOR-
// swizzled by r & 7: a quarter of a 128 x 32 K-major operand image.  The
// analysis (A = lambda[degree][ring], K = rings) reads a block's rows, the
// synthesis (A = lambda[ring][degree], K = degrees) its columns; both read
// shared memory without bank conflicts.  For order m and ring block k only the
// degree blocks i >= i0[m][k], the first holding a value >= 2^-SEED_EXP, are
// stored (at block off[m][k] + i - i0[m][k]); block 0 holds zeros and stands for
// every block not stored.
//
// The contraction kernel is the pipeline of the tensor-core quadrature
// (quad_tc.cuh) with the image of each chunk gathered from four table blocks:
// producer warp w copies its block (one bulk copy, a ring of LI_NRAW slots),
// splits its row or column into TF32 hi and lo and writes TMEM lane quadrant w;
// warps 4-11 load, split and store operand B and drain the accumulators; warp
// 12 issues the MMAs.
//   analysis   block = (order m, degree tile dt of 128, batch tile); TMEM lane =
//              degree; K = the ring chunks k whose blocks 4 dt .. 4 dt + 3 are not
//              all zero (a list built per block); B = G rows, rings 32 k ...
//   synthesis  block = (ring tile rt of 128, order m, batch tile); TMEM lane =
//              ring; K = the degree blocks from the smallest i0 of the tile's
//              four ring blocks; B = c_l f_lm rows, degrees m + 32 i ...
#pragma once
#include "gemm_fp32.cuh"
#include "legendre.cuh"
#include "tc_pipe.cuh"

namespace s2g {

constexpr int LI_BLK = 4096;                        // bytes of one 32 x 32 block
struct LegImg {
    const unsigned char *img;                       // blocks; block 0 zeros
    const int *i0;                                  // [m][k] first stored degree block (nib(m) if none)
    const int *off;                                 // [m][k] block index of degree block i0
    const int2 *adt;                                // analysis blocks: (m, degree tile)
    int nkr;                                        // ring blocks: ceil(N / 32)
};
__host__ __device__ constexpr int li_nib(int N, int m) { return (N - m + 31) / 32; }

// table block of degree block i and ring block k of order m (0: zeros)
__device__ __forceinline__ int li_block(const LegImg &T, int nib, int m, int i, int k)
{
    if (k >= T.nkr || i >= nib) return 0;
    const int b = T.i0[m * T.nkr + k];
    return i >= b ? T.off[m * T.nkr + k] + (i - b) : 0;
}

// i0[m][k] from the start degrees l_s(m, t): one thread per (m, k).
static __global__ void k_img_i0(int N, const int *__restrict__ ls, int *__restrict__ i0)
{
    const int nkr = (N + 31) / 32;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * nkr) return;
    const int m = idx / nkr, k = idx % nkr;
    int mn = N;
    for (int t = 32 * k; t < min(N, 32 * k + 32); ++t) mn = min(mn, ls[(size_t)m * N + t]);
    i0[idx] = mn < N ? (mn - m) / 32 : li_nib(N, m);
}

// The stored blocks: one warp per (m, ring block k), lane = ring.  Each lane runs
// the FP64 recurrence of its ring from its seed (zero below l_s) and writes one
// value of every row of the blocks, the warp a whole 128-byte row per degree.
static __global__ void k_img_fill(int N, const int *__restrict__ ls, const double2 *__restrict__ seed,
                                  const RingD *__restrict__ ring, const double2 *__restrict__ coef, int ldc,
                                  const int *__restrict__ i0, const int *__restrict__ off,
                                  unsigned char *__restrict__ img)
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
    unsigned char *blk = img + (size_t)off[gw] * LI_BLK;
    for (int i = ib; i < nib; ++i, blk += LI_BLK) {
        for (int r = 0; r < 32; ++r) {
            const int l = m + 32 * i + r;
            double v = 0.0;
            if (l < N && l >= lsv) {
                if (l == lsv) rec.seed(sd);
                else rec.step(cm[l]);
                v = rec.value();
            }
            *reinterpret_cast<float *>(blk + tc::sw128_off(r, lane)) = (float)v;
        }
    }
}

// ---------------------------------------------------------------- contraction
constexpr int LI_NA = 2, LI_NACC = 3, LI_NB = 4, LI_NR = 12, LI_NRAW = 4, LI_D = 4;
constexpr int LI_ACOL = 128 * LI_NACC;               // TMEM: accumulators, then the operand-A stages
static_assert(LI_ACOL + 64 * LI_NA <= LT_TMEM_COLS, "tensor memory");
constexpr int LI_RAW = 4 * LI_BLK;                  // one chunk: the four producer warps' blocks
constexpr int LI_BSTAGE = 2 * LT_PLANE;             // operand B hi, lo
constexpr int LI_MAXK = 128;                        // ring chunks of the analysis list (N <= 4096)
constexpr int LI_RAW_OFF = LI_NB * LI_BSTAGE;
constexpr int LI_LIST_OFF = LI_RAW_OFF + LI_NRAW * LI_RAW;
constexpr int LI_SYNC_OFF = LI_LIST_OFF + LI_MAXK * 4;
struct LiSync {
    uint64_t full[LI_NR], done[LI_NR], tempty[LI_NACC], raw[LI_NRAW][LT_REC_WARPS], fin;
    uint32_t tslot;
    int abort, nk, ibase;
};
constexpr int LI_SYNC_BYTES = 512;
static_assert(sizeof(LiSync) <= LI_SYNC_BYTES, "sync block");
static_assert(LI_NR % LI_NA == 0 && LI_NR % LI_NB == 0 && 2 * LI_D < LI_NR, "barrier ring");
__host__ __device__ constexpr size_t leg_img_smem() { return (size_t)LI_SYNC_OFF + LI_SYNC_BYTES + 1024; }
static_assert(leg_img_smem() <= 227 * 1024, "shared memory");

struct LegImgArgs {
    const float2 *src;       // analysis: G [b][mi][t] (band-limit N); synthesis: f [b][mi][l] (rectangle Lsrc)
    int Lsrc;                // synthesis: rectangle of src
    const float *kfac;       // per-degree factor or nullptr
    float scale;
    int accumulate;          // analysis: add to dst
    float2 *dst;             // analysis: f [b][mi][l] (rectangle Ldst); synthesis: F [b][mi][t] (band-limit N)
    int Ldst;
    int N, B;
    LegImg T;
    int *err;
};

template <bool ANAL, bool CPLX>
static __global__ void __launch_bounds__(LT_THREADS, 1) k_leg_img(LegImgArgs a)
{
    using Cols = LegCols<CPLX>;
    constexpr int BT = Cols::BT;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    LiSync &sy = *reinterpret_cast<LiSync *>(smem + LI_SYNC_OFF);
    int *klist = reinterpret_cast<int *>(smem + LI_LIST_OFF);
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
    auto par = [](int c) -> uint32_t { return (uint32_t)((c / LI_NR) & 1); };

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < LI_NR; ++i) {
            tc::mbar_init(&sy.full[i], LT_REC_WARPS + LT_OPB_WARPS);
            tc::mbar_init(&sy.done[i], 1);
        }
#pragma unroll
        for (int i = 0; i < LI_NACC; ++i) tc::mbar_init(&sy.tempty[i], LT_OPB_WARPS);
#pragma unroll
        for (int s = 0; s < LI_NRAW; ++s)
#pragma unroll
            for (int w = 0; w < LT_REC_WARPS; ++w) tc::mbar_init(&sy.raw[s][w], 1);
        tc::mbar_init(&sy.fin, 1);
        sy.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == LT_MMA_WARP) {
        tc::tmem_alloc(&sy.tslot, LT_TMEM_COLS);
    } else if (warp == LT_MMA_WARP - 1) {
        // the chunk sequence, the same for every role
        if constexpr (ANAL) {
            // ring chunks with a stored block among degree blocks 4 tile .. 4 tile + 3
            int n = 0;
            for (int k0 = 0; k0 < a.T.nkr; k0 += 32) {
                const int k = k0 + lane;
                const bool act = k < a.T.nkr && a.T.i0[m * a.T.nkr + k] <= 4 * tile + 3;
                const unsigned bal = __ballot_sync(0xffffffffu, act);
                if (act) klist[n + __popc(bal & ((1u << lane) - 1u))] = k;
                n += __popc(bal);
            }
            if (lane == 0) {
                sy.nk = n;
                sy.ibase = 0;
            }
        } else {
            // degree blocks from the smallest i0 of the tile's ring blocks
            int v = nib;
            if (lane < 4 && 4 * tile + lane < a.T.nkr) v = a.T.i0[m * a.T.nkr + 4 * tile + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) {
                sy.ibase = v;
                sy.nk = nib - v;
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sy.tslot;
    const int nk = sy.nk, ibase = sy.ibase;
    const int ng = (nk + LI_D - 1) / LI_D;

    if (warp < LT_REC_WARPS) {
        // ------------------------------------------------ operand A: table block -> split -> TMEM
        auto blk = [&](int c) -> int {
            return ANAL ? li_block(a.T, nib, m, 4 * tile + warp, klist[c])
                        : li_block(a.T, nib, m, ibase + c, 4 * tile + warp);
        };
        unsigned char *raw = smem + LI_RAW_OFF + warp * LI_BLK;
        if (lane == 0) {
            for (int c = 0; c < nk && c < LI_NRAW; ++c) {
                tc::mbar_arrive_expect_tx(&sy.raw[c][warp], LI_BLK);
                tc::bulk_g2s(raw + c * LI_RAW, a.T.img + (size_t)blk(c) * LI_BLK, LI_BLK, &sy.raw[c][warp]);
            }
        }
        const uint32_t lane_addr = (uint32_t)(32 * warp) << 16;
        for (int c = 0; c < nk; ++c) {
            const int s = c % LI_NRAW;
            lt_wait(&sy.raw[s][warp], (uint32_t)((c / LI_NRAW) & 1), abort);
            const unsigned char *bp = raw + s * LI_RAW;
            float hi[32], lo[32];
            if constexpr (ANAL) {
                // row `lane` of the block: this degree's 32 rings
                const unsigned char *rowp = bp + lane * 128;
#pragma unroll
                for (int kg = 0; kg < 8; ++kg) {
                    const float4 x = *reinterpret_cast<const float4 *>(rowp + (((kg ^ lane) & 7) << 4));
                    tc::split_tf32(x.x, hi[4 * kg + 0], lo[4 * kg + 0]);
                    tc::split_tf32(x.y, hi[4 * kg + 1], lo[4 * kg + 1]);
                    tc::split_tf32(x.z, hi[4 * kg + 2], lo[4 * kg + 2]);
                    tc::split_tf32(x.w, hi[4 * kg + 3], lo[4 * kg + 3]);
                }
            } else {
                // column `lane` of the block: this ring's 32 degrees
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    tc::split_tf32(*reinterpret_cast<const float *>(bp + tc::sw128_off(r, lane)), hi[r], lo[r]);
            }
            // the slot's values are in registers: refill it with chunk c + LI_NRAW
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0 && c + LI_NRAW < nk) {
                tc::mbar_arrive_expect_tx(&sy.raw[s][warp], LI_BLK);
                tc::bulk_g2s(raw + s * LI_RAW, a.T.img + (size_t)blk(c + LI_NRAW) * LI_BLK, LI_BLK, &sy.raw[s][warp]);
            }
            if (c >= LI_NA) lt_wait(&sy.done[(c - LI_NA) % LI_NR], par(c - LI_NA), abort);
            tc::fence_after();
            const uint32_t ahi = tmem + lane_addr + (uint32_t)(LI_ACOL + 64 * (c % LI_NA)), alo = ahi + 32;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                tc::tmem_st8(ahi + 8 * g, *reinterpret_cast<const float(*)[8]>(hi + 8 * g));
                tc::tmem_st8(alo + 8 * g, *reinterpret_cast<const float(*)[8]>(lo + 8 * g));
            }
            tc::tmem_wait_st();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.full[c % LI_NR]);
        }
        // no copy of this warp still in flight when the block ends (only possible
        // after an abort): wait, bounded, for the last copy into each slot
        if (lane == 0)
            for (int c = nk - LI_NRAW > 0 ? nk - LI_NRAW : 0; c < nk; ++c)
                tc::mbar_wait(&sy.raw[c % LI_NRAW][warp], (uint32_t)((c / LI_NRAW) & 1), 1u << 22);
    } else if (warp < LT_MMA_WARP) {
        // ------------------------------------------------ operand B and drains
        const int u = tid - 32 * LT_REC_WARPS;
        float sum[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) sum[i] = 0.f;
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        const int h = (warp - LT_REC_WARPS) >> 2;
        auto drain = [&](int g) {                     // accumulator g % LI_NACC into sum
            const int cl = min(LI_D * g + LI_D - 1, nk - 1);   // the group's last chunk
            lt_spin(&sy.done[cl % LI_NR], par(cl), abort);
            tc::fence_after();
            const uint32_t acc = tmem + lane_addr + (uint32_t)(128 * (g % LI_NACC) + 64 * h);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tc::tmem_ld16(acc + 16 * q, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[16 * q + i] += v[i];
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.tempty[g % LI_NACC]);
        };
        // source row of column pair p, at the chunk's first K (nullptr: absent pair)
        const int nmi_src = ANAL ? (CPLX ? 2 * N - 1 : N) : (CPLX ? 2 * a.Lsrc - 1 : a.Lsrc);
        const int moff = ANAL ? N - 1 : a.Lsrc - 1, lds = ANAL ? N : a.Lsrc;
        auto load = [&](LtB &bv, int c) {
            const int k0 = ANAL ? 32 * klist[c] : m + 32 * (ibase + c);
            bv.load<ANAL>(u, [&](int p) -> const float2 * {
                const int sg = p / BT, b = p % BT;
                if (b0 + b >= a.B || (sg == 1 && !two)) return nullptr;
                const int mi = sg == 0 ? (CPLX ? m + moff : m) : (-m + moff);
                return a.src + ((size_t)(b0 + b) * nmi_src + mi) * lds + k0;
            }, N - k0, (!ANAL && a.kfac) ? a.kfac + k0 : nullptr);
        };
        int drained = 0;
        auto body = [&](int c, LtB &cur, LtB &next) {
            if (c >= nk) return;
            if (c + 1 < nk) load(next, c + 1);
            // the accumulator of group c / LI_D - LI_NACC must be drained before chunk c's MMAs
            while (drained <= c / LI_D - LI_NACC) drain(drained++);
            if (c >= LI_NB) lt_spin(&sy.done[(c - LI_NB) % LI_NR], par(c - LI_NB), abort);
            cur.store(smem + (c % LI_NB) * LI_BSTAGE, u);
            lt_warp_arrive(&sy.full[c % LI_NR], lane);
        };
        LtB bb0, bb1;
        if (nk > 0) load(bb0, 0);
        for (int c = 0; c < nk; c += 2) {
            body(c, bb0, bb1);
            body(c + 1, bb1, bb0);
        }
        while (drained < ng) drain(drained++);
        if (!sy.abort) {
            if constexpr (ANAL) {
                // epilogue: TMEM lane = degree
                const int l0 = m + 128 * tile, l = l0 + 32 * (warp & 3) + lane;
                if (l < N) {
                    const int nmi_dst = CPLX ? 2 * a.Ldst - 1 : a.Ldst;
                    const float sgn_m = (m & 1) ? -1.f : 1.f;
                    const float f = a.scale * (a.kfac ? a.kfac[l] : 1.f);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int p = 32 * h + j;
                        const int sg = p / BT, b = p % BT;
                        if (b0 + b < a.B && (sg == 0 || two)) {
                            const float fs = sg == 1 ? f * sgn_m : f;
                            const int mi = sg == 0 ? (CPLX ? m + a.Ldst - 1 : m) : (-m + a.Ldst - 1);
                            float2 *o = a.dst + ((size_t)(b0 + b) * nmi_dst + mi) * a.Ldst + l;
                            float2 v = make_float2(sum[2 * j] * fs, sum[2 * j + 1] * fs);
                            if (a.accumulate) {
                                const float2 w = *o;
                                v.x += w.x;
                                v.y += w.y;
                            }
                            *o = v;
                        }
                        if ((j & 7) == 7) asm volatile("" ::: "memory");   // keep the loads of later pairs below
                    }
                }
            } else {
                // epilogue: TMEM lane = ring
                const int t = 128 * tile + 32 * (warp & 3) + lane;
                if (t < N) {
                    const int nmi_dst = CPLX ? 2 * N - 1 : N;
                    const float sgn_m = (m & 1) ? -1.f : 1.f;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int p = 32 * h + j;
                        const int sg = p / BT, b = p % BT;
                        if (b0 + b >= a.B || (sg == 1 && !two)) continue;
                        const float f = sg == 1 ? a.scale * sgn_m : a.scale;
                        const int mi = sg == 0 ? (CPLX ? m + N - 1 : m) : (-m + N - 1);
                        a.dst[((size_t)(b0 + b) * nmi_dst + mi) * N + t] =
                            make_float2(sum[2 * j] * f, sum[2 * j + 1] * f);
                    }
                }
            }
        }
    } else if (lane == 0) {
        // ------------------------------------------------ MMA issue: A from TMEM, B from shared memory
        constexpr uint32_t IDESC = tc::idesc_tf32(128, 128);
        for (int c = 0; c < nk; ++c) {
            const int g = c / LI_D;
            const bool first = c % LI_D == 0;           // first chunk of group g
            bool ok = lt_spin(&sy.full[c % LI_NR], par(c), abort);
            if (first && g >= LI_NACC) ok = lt_spin(&sy.tempty[g % LI_NACC], ((g / LI_NACC) - 1) & 1, abort) && ok;
            tc::fence_after();
            if (ok) {
                const uint32_t bbase = tc::smem_addr(smem + (c % LI_NB) * LI_BSTAGE);
                const uint32_t acc = tmem + (uint32_t)(128 * (g % LI_NACC));
                const uint32_t ahi = tmem + (uint32_t)(LI_ACOL + 64 * (c % LI_NA)), alo = ahi + 32;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t b0d = tc::smem_desc_sw128(bbase + ks * 32);
                    const uint64_t b1d = tc::smem_desc_sw128(bbase + LT_PLANE + ks * 32);
                    tc::mma_tf32_ts(acc, ahi + 8 * ks, b1d, IDESC, (ks > 0 || !first) ? 1u : 0u);
                    tc::mma_tf32_ts(acc, alo + 8 * ks, b0d, IDESC, 1u);
                    tc::mma_tf32_ts(acc, ahi + 8 * ks, b0d, IDESC, 1u);
                }
            }
            tc::mma_commit(&sy.done[c % LI_NR]);
        }
        tc::mma_commit(&sy.fin);
        tc::mbar_wait(&sy.fin, 0, 1u << 22);   // no MMA in flight when TMEM is released
    }
    tc::fence_before();
    __syncthreads();
    if (warp == LT_MMA_WARP) tc::tmem_free(tmem, LT_TMEM_COLS);
    if (tid == 0 && sy.abort) atomicExch(a.err, 1);
}

}  // namespace s2g
