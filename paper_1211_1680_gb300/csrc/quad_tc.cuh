// MW theta quadrature of the TF32X3 plans as a pipelined tensor-core product:
//   G[b][mi][t] = sum_t' Q_sigma[t][t'] F[b][mi][t']
// for the orders mi = mi0, mi0 + 2, ... of one parity sigma.
// Block: (tile of 128 rows t, tile of 64 (b, mi) pairs); K = t' in chunks of 32.
//   operand A  Q_sigma, stored once per plan in FP32 as the shared-memory image
//              of each (row tile, K chunk): 128 x 32 values in the swizzled
//              layout, 16 KB, zeros outside N x N.  Producer warp w (< 4) owns
//              rows 32 w .. 32 w + 31, which are its TMEM lane quadrant and a
//              contiguous 4 KB quarter of each image.  It keeps QT_NRAW chunks of
//              its quarter in flight with bulk copies (TMA engine; one mbarrier
//              per warp and slot), reads its row of a chunk, splits it into TF32
//              hi and lo and writes both to TMEM (tcgen05.st); the MMAs read A
//              from TMEM.  The copies depend only on the slot being read, not on
//              the MMAs, so their latency is off the MMA critical path.
//   operand B  64 pairs x re/im of F, split while stored (LtB) by warps 4-11,
//              which also drain the accumulators into FP32 registers and write G.
//              The F values of a chunk arrive by asynchronous copies in a ring
//              of QT_NF slots (see FRAW below).
// The tensor core accumulates QT_D chunks (K = 32 QT_D) in one TMEM buffer;
// the sums of these groups are added in FP32 registers.  Its accumulation error
// grows with the number of products summed in TMEM, so this bounds it (measured
// 2e-7 relative per chunk) while the drains cost 1 / QT_D of one per chunk.
// Rings of chunk c (group g = c / QT_D):
//   operand A in TMEM        c % QT_NA    columns 384 + 64 (c % QT_NA) (hi), + 32 (lo)
//   accumulator in TMEM      g % QT_NACC  columns 128 (g % QT_NACC)
//   operand B in shared mem  c % QT_NB
//   raw A image in shared    c % QT_NRAW
//   raw F rows in shared     c % QT_NF
// Barriers: full[c % QT_NR] (4 producer + 8 operand-B warps arrive), done[c %
// QT_NR] (one commit: the chunk's MMAs completed, so its A and B slots are free,
// and after a group's last chunk its accumulator can be drained), tempty[g %
// QT_NACC] (drained), raw[slot][warp] (a quarter image landed).  QT_NR is a
// common multiple of the operand ring depths, and no waiter runs QT_NR chunks
// behind (a drain waits at most 2 QT_D chunks behind the MMAs).
#pragma once
#include "tc_pipe.cuh"

namespace s2g {

constexpr int QT_NA = 2, QT_NACC = 3, QT_NB = 4, QT_NR = 12, QT_NRAW = 4, QT_NF = 2, QT_D = 4;
constexpr int QT_RAW = LT_PLANE;                   // bytes of one (row tile, K chunk) image
constexpr int QT_QUARTER = QT_RAW / LT_REC_WARPS;  // one producer warp's rows of an image
constexpr int QT_BSTAGE = 2 * LT_PLANE;            // operand B hi, lo
constexpr int QT_FROW = 32 * 8;                    // bytes of one F row of a chunk (32 float2)
constexpr int QT_FSLOT = 64 * QT_FROW;             // F rows of the block's 64 pairs
constexpr int QT_RAW_OFF = QT_NB * QT_BSTAGE;
constexpr int QT_FRAW_OFF = QT_RAW_OFF + QT_NRAW * QT_RAW;
constexpr int QT_SYNC_OFF = QT_FRAW_OFF + QT_NF * QT_FSLOT;
struct QtSync {
    uint64_t full[QT_NR], done[QT_NR], tempty[QT_NACC], raw[QT_NRAW][LT_REC_WARPS], fin;
    uint32_t tslot;
    int abort;
};
constexpr int QT_SYNC_BYTES = 512;
static_assert(sizeof(QtSync) <= QT_SYNC_BYTES, "sync block");
static_assert(QT_NR % QT_NA == 0 && QT_NR % QT_NB == 0 && 2 * QT_D < QT_NR, "barrier ring");
__host__ __device__ constexpr size_t quad_tc_smem() { return (size_t)QT_SYNC_OFF + QT_SYNC_BYTES + 1024; }
static_assert(quad_tc_smem() <= 227 * 1024, "shared memory");

// FRAW: F values reach shared memory by 16-byte asynchronous copies (a ring of
// QT_NF chunks; each operand-B warp copies the rows it splits), so the split
// reads shared memory and never waits on global loads.  Needs 16-byte
// aligned rows (N even, F 16-byte aligned); otherwise (FRAW false) each thread
// loads its units from global memory one chunk ahead into registers.
template <bool FRAW>
static __global__ void __launch_bounds__(LT_THREADS, 1)
    k_quad_tcp(const unsigned char *__restrict__ Qimg, const float2 *__restrict__ F, float2 *__restrict__ G, int N,
               int nmi, int mi0, int nj, int npairs, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    QtSync &sy = *reinterpret_cast<QtSync *>(smem + QT_SYNC_OFF);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * 128, pair0 = blockIdx.y * 64;
    const int nk = (N + 31) / 32, ng = (nk + QT_D - 1) / QT_D;
    volatile int *abort = &sy.abort;
    // phase parity of the completion / readiness of chunk c
    auto par = [](int c) -> uint32_t { return (uint32_t)((c / QT_NR) & 1); };

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < QT_NR; ++i) {
            tc::mbar_init(&sy.full[i], LT_REC_WARPS + LT_OPB_WARPS);
            tc::mbar_init(&sy.done[i], 1);
        }
#pragma unroll
        for (int i = 0; i < QT_NACC; ++i) tc::mbar_init(&sy.tempty[i], LT_OPB_WARPS);
#pragma unroll
        for (int s = 0; s < QT_NRAW; ++s)
#pragma unroll
            for (int w = 0; w < LT_REC_WARPS; ++w) tc::mbar_init(&sy.raw[s][w], 1);
        tc::mbar_init(&sy.fin, 1);
        sy.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == LT_MMA_WARP) tc::tmem_alloc(&sy.tslot, LT_TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sy.tslot;

    if (warp < LT_REC_WARPS) {
        // ------------------------------------------------ operand A: raw ring -> split -> TMEM
        const unsigned char *img = Qimg + (size_t)blockIdx.x * nk * QT_RAW + warp * QT_QUARTER;
        unsigned char *raw = smem + QT_RAW_OFF + warp * QT_QUARTER;
        if (lane == 0) {
            for (int c = 0; c < nk && c < QT_NRAW; ++c) {
                tc::mbar_arrive_expect_tx(&sy.raw[c][warp], QT_QUARTER);
                tc::bulk_g2s(raw + c * QT_RAW, img + (size_t)c * QT_RAW, QT_QUARTER, &sy.raw[c][warp]);
            }
        }
        const int r = 32 * warp + lane;               // row of the tile = TMEM lane
        const uint32_t lane_addr = (uint32_t)(32 * warp) << 16;
        for (int c = 0; c < nk; ++c) {
            const int s = c % QT_NRAW;
            lt_wait(&sy.raw[s][warp], (uint32_t)((c / QT_NRAW) & 1), abort);
            const unsigned char *rowp = smem + QT_RAW_OFF + s * QT_RAW + r * 128;
            float hi[32], lo[32];
#pragma unroll
            for (int kg = 0; kg < 8; ++kg) {
                const float4 x = *reinterpret_cast<const float4 *>(rowp + (((kg ^ r) & 7) << 4));
                tc::split_tf32(x.x, hi[4 * kg + 0], lo[4 * kg + 0]);
                tc::split_tf32(x.y, hi[4 * kg + 1], lo[4 * kg + 1]);
                tc::split_tf32(x.z, hi[4 * kg + 2], lo[4 * kg + 2]);
                tc::split_tf32(x.w, hi[4 * kg + 3], lo[4 * kg + 3]);
            }
            // the slot's values are in registers: refill it with chunk c + QT_NRAW
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0 && c + QT_NRAW < nk) {
                tc::mbar_arrive_expect_tx(&sy.raw[s][warp], QT_QUARTER);
                tc::bulk_g2s(raw + s * QT_RAW, img + (size_t)(c + QT_NRAW) * QT_RAW, QT_QUARTER, &sy.raw[s][warp]);
            }
            if (c >= QT_NA) lt_wait(&sy.done[(c - QT_NA) % QT_NR], par(c - QT_NA), abort);
            tc::fence_after();
            const uint32_t ahi = tmem + lane_addr + (uint32_t)(384 + 64 * (c % QT_NA)), alo = ahi + 32;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                tc::tmem_st8(ahi + 8 * g, *reinterpret_cast<const float(*)[8]>(hi + 8 * g));
                tc::tmem_st8(alo + 8 * g, *reinterpret_cast<const float(*)[8]>(lo + 8 * g));
            }
            tc::tmem_wait_st();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.full[c % QT_NR]);
        }
        // no copy of this warp still in flight when the block ends (only possible
        // after an abort): wait, bounded, for the last copy into each slot
        if (lane == 0)
            for (int c = nk - QT_NRAW > 0 ? nk - QT_NRAW : 0; c < nk; ++c)
                tc::mbar_wait(&sy.raw[c % QT_NRAW][warp], (uint32_t)((c / QT_NRAW) & 1), 1u << 22);
    } else if (warp < LT_MMA_WARP) {
        // ------------------------------------------------ operand B (F) and drains
        const int u = tid - 32 * LT_REC_WARPS;
        float sum[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) sum[i] = 0.f;
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        const int h = (warp - LT_REC_WARPS) >> 2;
        auto drain = [&](int g) {                     // accumulator g % QT_NACC into sum
            const int cl = min(QT_D * g + QT_D - 1, nk - 1);   // the group's last chunk
            lt_spin(&sy.done[cl % QT_NR], par(cl), abort);
            tc::fence_after();
            const uint32_t acc = tmem + lane_addr + (uint32_t)(128 * (g % QT_NACC) + 64 * h);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tc::tmem_ld16(acc + 16 * q, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[16 * q + i] += v[i];
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.tempty[g % QT_NACC]);
        };
        int drained = 0;
        if constexpr (FRAW) {
            // Operand-B warp wb splits the units of pairs 4 wb .. 4 wb + 3 and 32 + 4 wb ..
            // 32 + 4 wb + 3: it stages exactly these 8 rows (256 bytes of a chunk each)
            // with 16-byte asynchronous copies, QT_NF chunks ahead.  Lane l copies
            // piece l & 15 of rows 2 r + (l >> 4), r = 0..3, so each copy instruction
            // covers two whole rows; values past N and rows of absent pairs are zero-
            // filled.  After its own copies land (wait_group), a warp barrier makes
            // the warp's rows visible to all its lanes.
            const int wb = warp - LT_REC_WARPS;
            unsigned char *fraw = smem + QT_FRAW_OFF;
            const int q = lane & 15;
            const float2 *srow[4];
            uint32_t drow[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int j = 2 * r + (lane >> 4);
                const int p = j < 4 ? 4 * wb + j : 32 + 4 * wb + (j - 4), pp = pair0 + p;
                srow[r] = nullptr;
                if (pp < npairs) {
                    const int b = pp / nj, jj = pp % nj;
                    srow[r] = F + ((size_t)b * nmi + mi0 + 2 * jj) * N + 2 * q;
                }
                drow[r] = tc::smem_addr(fraw + p * QT_FROW + 16 * q);
            }
            auto issue = [&](int c) {                 // the warp's rows of chunk c, slot c % QT_NF
                const int k0 = 32 * c, nv = max(0, min(2, N - k0 - 2 * q));
                const uint32_t so = (uint32_t)((c % QT_NF) * QT_FSLOT);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t n = srow[r] ? (uint32_t)nv : 0u;
                    tc::cp_async16(drow[r] + so, n ? srow[r] + k0 : F, n * 8);
                }
            };
#pragma unroll 1
            for (int c = 0; c < QT_NF; ++c) {
                if (c < nk) issue(c);
                tc::cp_async_commit();
            }
            // this thread's unit i: pair (u + 256 i) >> 3, values k = 4 kg .. 4 kg + 3 as
            // pieces 2 kg and 2 kg + 1 of the row; lanes with kg >= 4 read the second
            // piece first, so that the eight lanes of a phase hit distinct banks
            const int kg = u & 7, sw = (kg >> 2) & 1;
            for (int c = 0; c < nk; ++c) {
                tc::cp_async_wait<QT_NF - 1>();       // this thread's copies of chunk c landed
                __syncwarp();                         // ... and those of the warp's other lanes
                const float4 *slot = reinterpret_cast<const float4 *>(fraw + (c % QT_NF) * QT_FSLOT);
                LtB bv;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float4 *pc = slot + ((u + 256 * i) >> 3) * (QT_FROW / 16) + 2 * kg;
                    const float4 x = pc[sw], y = pc[sw ^ 1];
                    const float4 a = sw ? y : x, b = sw ? x : y;
                    bv.v[i][0] = make_float2(a.x, a.y);
                    bv.v[i][1] = make_float2(a.z, a.w);
                    bv.v[i][2] = make_float2(b.x, b.y);
                    bv.v[i][3] = make_float2(b.z, b.w);
                }
                // the accumulator of group c / QT_D - QT_NACC must be drained before chunk c's MMAs
                while (drained <= c / QT_D - QT_NACC) drain(drained++);
                if (c >= QT_NB) lt_spin(&sy.done[(c - QT_NB) % QT_NR], par(c - QT_NB), abort);
                bv.store(smem + (c % QT_NB) * QT_BSTAGE, u);
                // (the warp barrier in the arrival also orders every lane's reads of
                // the slot before its refill below)
                lt_warp_arrive(&sy.full[c % QT_NR], lane);
                if (c + QT_NF < nk) issue(c + QT_NF);
                tc::cp_async_commit();
            }
            tc::cp_async_wait<0>();
        } else {
            // F rows of this thread's two pairs, loaded one chunk ahead (two register
            // sets, the loop unrolled by two so that they stay registers)
            const float2 *frow[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int pp = pair0 + ((u + 256 * i) >> 3);
                frow[i] = nullptr;
                if (pp < npairs) {
                    const int b = pp / nj, j = pp % nj;
                    frow[i] = F + ((size_t)b * nmi + mi0 + 2 * j) * N;
                }
            }
            auto load = [&](LtB &bv, int c) {
                const int k0 = 32 * c;
                bv.load(u, [&](int p) -> const float2 * {
                    const float2 *rr = frow[p >= 32];
                    return rr ? rr + k0 : nullptr;
                }, N - k0, nullptr);
            };
            auto body = [&](int c, LtB &cur, LtB &next) {
                if (c >= nk) return;
                if (c + 1 < nk) load(next, c + 1);
                while (drained <= c / QT_D - QT_NACC) drain(drained++);
                if (c >= QT_NB) lt_spin(&sy.done[(c - QT_NB) % QT_NR], par(c - QT_NB), abort);
                cur.store(smem + (c % QT_NB) * QT_BSTAGE, u);
                lt_warp_arrive(&sy.full[c % QT_NR], lane);
            };
            LtB b0, b1;
            if (nk > 0) load(b0, 0);
            for (int c = 0; c < nk; c += 2) {
                body(c, b0, b1);
                body(c + 1, b1, b0);
            }
        }
        while (drained < ng) drain(drained++);
        // epilogue: TMEM lane = row t
        const int t = row0 + 32 * (warp & 3) + lane;
        if (t < N && !sy.abort) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int pp = pair0 + 32 * h + j;
                if (pp < npairs) {
                    const int b = pp / nj, jj = pp % nj;
                    G[((size_t)b * nmi + mi0 + 2 * jj) * N + t] = make_float2(sum[2 * j], sum[2 * j + 1]);
                }
            }
        }
    } else if (lane == 0) {
        // ------------------------------------------------ MMA issue: A from TMEM, B from shared memory
        constexpr uint32_t IDESC = tc::idesc_tf32(128, 128);
        for (int c = 0; c < nk; ++c) {
            const int g = c / QT_D;
            const bool first = c % QT_D == 0;           // first chunk of group g
            bool ok = lt_spin(&sy.full[c % QT_NR], par(c), abort);
            if (first && g >= QT_NACC) ok = lt_spin(&sy.tempty[g % QT_NACC], ((g / QT_NACC) - 1) & 1, abort) && ok;
            tc::fence_after();
            if (ok) {
                const uint32_t bbase = tc::smem_addr(smem + (c % QT_NB) * QT_BSTAGE);
                const uint32_t acc = tmem + (uint32_t)(128 * (g % QT_NACC));
                const uint32_t ahi = tmem + (uint32_t)(384 + 64 * (c % QT_NA)), alo = ahi + 32;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t b0d = tc::smem_desc_sw128(bbase + ks * 32);
                    const uint64_t b1d = tc::smem_desc_sw128(bbase + LT_PLANE + ks * 32);
                    tc::mma_tf32_ts(acc, ahi + 8 * ks, b1d, IDESC, (ks > 0 || !first) ? 1u : 0u);
                    tc::mma_tf32_ts(acc, alo + 8 * ks, b0d, IDESC, 1u);
                    tc::mma_tf32_ts(acc, ahi + 8 * ks, b0d, IDESC, 1u);
                }
            }
            tc::mma_commit(&sy.done[c % QT_NR]);
        }
        tc::mma_commit(&sy.fin);
        tc::mbar_wait(&sy.fin, 0, 1u << 22);   // no MMA in flight when TMEM is released
    }
    tc::fence_before();
    __syncthreads();
    if (warp == LT_MMA_WARP) tc::tmem_free(tmem, LT_TMEM_COLS);
    if (tid == 0 && sy.abort) atomicExch(err, 1);
}

// Q (FP32, N x N) -> shared-memory images of operand A: for row tile rt and K
// chunk c, Q[128 rt + r][32 c + k] at byte sw128_off(r, k) of the chunk's 16 KB
// image; zeros outside N x N.  One thread per 16-byte piece (4 values of k).
static __global__ void k_quad_images(const float *__restrict__ Q, unsigned char *__restrict__ img, int N)
{
    const int nk = (N + 31) / 32, nrt = (N + 127) / 128;
    const size_t npieces = (size_t)nrt * nk * 128 * 8;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npieces) return;
    const int kg = (int)(i & 7), r = (int)((i >> 3) & 127);
    const size_t tile = i >> 10;                      // rt * nk + c
    const int c = (int)(tile % nk), rt = (int)(tile / nk);
    const int row = 128 * rt + r;
    float x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 32 * c + 4 * kg + q;
        x[q] = (row < N && k < N) ? Q[(size_t)row * N + k] : 0.f;
    }
    *reinterpret_cast<float4 *>(img + tile * QT_RAW + tc::sw128_off(r, 4 * kg)) = make_float4(x[0], x[1], x[2], x[3]);
}

__host__ __device__ inline size_t quad_image_bytes(int N)
{
    return (size_t)((N + 127) / 128) * ((N + 31) / 32) * QT_RAW;
}

}  // namespace s2g
