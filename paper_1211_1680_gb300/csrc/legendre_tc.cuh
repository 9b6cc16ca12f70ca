// Legendre contractions of the TF32X3 plans on the tensor cores (tcgen05):
//   k_leg_synth_tc  F_m(theta_t) = scale sum_l lambda_lm(theta_t) c_l f_lm     (Eq. harmonicssynthesis)
//   k_leg_anal_tc   f_lm = scale c_l sum_t lambda_lm(theta_t) G_m(theta_t)    (last step of the MW quadrature)
// for one order m and a tile of 128 columns (64 maps x re/im for real maps;
// 32 maps x {m, -m} x re/im for complex maps, the layout of LegCols), on the
// pipeline of tc_pipe.cuh with recurrence warps as the operand-A producers.
//
// The associated Legendre values come from the float-float recurrence of
// legendre.cuh, are rounded to FP32 and split into TF32 hi + lo parts; so are
// the FP32 operands of the other side.
#pragma once
#include "common.cuh"
#include "gemm_fp32.cuh"
#include "legendre.cuh"
#include "tc_pipe.cuh"

namespace s2g {

// analysis: recurrence warps 0-3 (one per operand-A stage, each issuing its
// chunks' MMAs), warps 4-11 as in synthesis; twelve warps leave 168 registers
// per thread instead of 128
constexpr int LT_ANAL_THREADS = 32 * (LT_REC_WARPS + LT_OPB_WARPS);
constexpr int LT_ANAL_REC = LT_REC_WARPS;

// Branch-free float-float recurrence of one ring (the step of RecT<float>):
// the state is zero before l_s, so the recurrence yields zeros there; at
// l = l_s the seed pair is selected in; coefficients past the band-limit are
// zero, and so are the values.  A ring outside the map has x = 0, no seed.
struct LtRec {
    ff p0, p1, x, s0, s1;
    int ls;
    __device__ __forceinline__ void init(bool own, const RingF *ring, const double2 *seed, const int *lsp)
    {
        p0.h = p0.l = p1.h = p1.l = 0.f;
        x.h = x.l = 0.f;
        s0 = p0;
        s1 = p0;
        ls = 1 << 30;
        if (own) {
            const RingF r = *ring;
            x.h = r.xh;
            x.l = r.xl;
            ls = *lsp;
            const double2 sd = *seed;
            s0.h = (float)sd.x;
            s0.l = (float)(sd.x - (double)s0.h);
            s1.h = (float)sd.y;
            s1.l = (float)(sd.y - (double)s1.h);
        }
    }
    // step without the seed selection, for degrees l != l_s (after l_s, or before
    // it where the state is zero)
    __device__ __forceinline__ float step_plain(const float4 c)
    {
        ff a, ab;
        a.h = c.x;
        a.l = c.y;
        ab.h = c.z;
        ab.l = c.w;
        const ff p2 = ff_sub(ff_mul(ff_mul(a, x), p1), ff_mul(ab, p0));
        p0 = p1;
        p1 = p2;
        return p1.h;
    }
    // does the chain start in degrees [l0, l0 + n)?
    __device__ __forceinline__ bool starts_in(int l0, int n) const { return ls >= l0 && ls < l0 + n; }
    // value of degree l given the coefficient (a hi, a lo, a b hi, a b lo) of l
    __device__ __forceinline__ float step(const float4 c, int l)
    {
        ff a, ab;
        a.h = c.x;
        a.l = c.y;
        ab.h = c.z;
        ab.l = c.w;
        const ff ax = ff_mul(a, x);
        const ff pa = ff_mul(ax, p1);
        const ff pb = ff_mul(ab, p0);
        const ff p2 = ff_sub(pa, pb);
        const bool at = l == ls;
        p0.h = at ? s0.h : p1.h;
        p0.l = at ? s0.l : p1.l;
        p1.h = at ? s1.h : p2.h;
        p1.l = at ? s1.l : p2.l;
        return p1.h;
    }
};

// Recurrence coefficient of degree l0 + j held by lane j of the warp (cf),
// broadcast to every lane; all lanes must call it.
__device__ __forceinline__ float4 lt_coef(const float4 &cf, int j)
{
    return make_float4(__shfl_sync(0xffffffffu, cf.x, j), __shfl_sync(0xffffffffu, cf.y, j),
                       __shfl_sync(0xffffffffu, cf.z, j), __shfl_sync(0xffffffffu, cf.w, j));
}

// coefficient (a_lm, a_lm b_lm) of degree l as read by lane l - l0 (zero past the end)
__device__ __forceinline__ float4 lt_coef_load(const float4 *cm, int l, int N)
{
    return l < N ? __ldg(cm + l) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------- synthesis
// Block: (tile of 128 rings, order m, batch tile).  MMA rows = rings, K =
// degrees in chunks of 32 from the tile's smallest l_s, columns = coefficient
// columns.  Recurrence thread r owns ring t0 + r, which is row r of A and lane
// r of tensor memory: it writes its split lambda values straight into TMEM
// (tcgen05.st) and the MMAs read operand A from there, so the tensor core's
// shared-memory traffic is operand B only and does not throttle the recurrence.
// Rings of different depth for chunk c:
//   operand A in TMEM        stage c % LS_NA    columns 384 + 64 (c % LS_NA) (hi), + 32 (lo)
//   accumulator in TMEM      buffer c % LS_NACC columns 128 (c % LS_NACC)
//   operand B in shared mem  stage c % LS_NB
// Barriers: full[c % LS_NR] (4 recurrence + 8 operand-B warps arrive), done[c %
// LS_NR] (one commit: the chunk's MMAs completed, so its A and B stages are free
// and its accumulator can be drained), tempty[c % LS_NACC] (drained).  LS_NR is
// a common multiple of the ring depths, and no waiter runs LS_NR chunks behind,
// so one commit per chunk serves every ring.  More accumulators than operand-A
// stages: a chunk's MMAs wait for the drain three chunks back, which hides the
// commit-to-drain round trip behind the recurrence.
// Each recurrence warp stages its chunk's 32 recurrence coefficients in shared
// memory and every lane reads them with broadcast loads.  Waits poll without
// suspending (lt_spin): measured faster here than suspending waits.
constexpr int LS_NA = 2, LS_NACC = 3, LS_NB = 4, LS_NR = 12;
constexpr int LS_STAGE = 2 * LT_PLANE;                 // operand B hi, lo
struct LsSync {
    uint64_t full[LS_NR], done[LS_NR], tempty[LS_NACC], fin;
    uint32_t tslot;
    int abort, lmin;
};
constexpr int LS_COEF_OFF = LS_NB * LS_STAGE;          // 4 warps x 32 float4
constexpr int LS_SYNC_OFF = LS_COEF_OFF + LT_REC_WARPS * 32 * 16;
__host__ __device__ constexpr size_t ls_synth_smem() { return (size_t)LS_SYNC_OFF + 256 + 1024; }
static_assert(sizeof(LsSync) <= 256, "sync block");
static_assert(LS_NR % LS_NA == 0 && LS_NR % LS_NACC == 0 && LS_NR % LS_NB == 0, "barrier ring");

template <bool CPLX>
static __global__ void __launch_bounds__(LT_THREADS, 1)
    k_leg_synth_tc(const float2 *__restrict__ src, int Lsrc, const float *__restrict__ kfac, float scale,
                   float2 *__restrict__ dst, int N, int B, LegTab<float> tab, int *err)
{
    using Cols = LegCols<CPLX>;
    constexpr int BT = Cols::BT;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    LsSync &sy = *reinterpret_cast<LsSync *>(smem + LS_SYNC_OFF);
    float4 *coefs = reinterpret_cast<float4 *>(smem + LS_COEF_OFF);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t0 = blockIdx.x * 128, m = blockIdx.y, b0 = blockIdx.z * BT;
    const bool two = CPLX && m > 0;
    volatile int *abort = &sy.abort;
    // phase parity of the completion / readiness of chunk c
    auto par = [](int c) -> uint32_t { return (uint32_t)((c / LS_NR) & 1); };

    int ls = N;
    if (warp < LT_REC_WARPS && t0 + tid < N) ls = tab.ls[(size_t)m * N + t0 + tid];
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < LS_NR; ++i) {
            tc::mbar_init(&sy.full[i], LT_REC_WARPS + LT_OPB_WARPS);
            tc::mbar_init(&sy.done[i], 1);
        }
#pragma unroll
        for (int i = 0; i < LS_NACC; ++i) tc::mbar_init(&sy.tempty[i], LT_OPB_WARPS);
        tc::mbar_init(&sy.fin, 1);
        sy.abort = 0;
        sy.lmin = N;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == LT_MMA_WARP) tc::tmem_alloc(&sy.tslot, LT_TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp < LT_REC_WARPS) {
        int v = ls;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) atomicMin(&sy.lmin, v);
    }
    __syncthreads();
    const int lstart = sy.lmin;
    const int nk = lstart < N ? (N - lstart + 31) / 32 : 0;
    const uint32_t tmem = sy.tslot;

    if (warp < LT_REC_WARPS) {
        // ------------------------------------------------ recurrence (A = lambda[ring][degree] in TMEM)
        const int t = t0 + tid;
        const bool own = t < N;
        LtRec rec;
        rec.init(own, tab.ring + t, tab.seed + (size_t)m * N + t, tab.ls + (size_t)m * N + t);
        const float4 *cm = tab.coef + (size_t)m * tab.ldc;
        float4 *wc = coefs + 32 * warp;
        const uint32_t lane_addr = (uint32_t)(32 * warp) << 16;
        float4 cf_next = lt_coef_load(cm, lstart + lane, N);
        for (int c = 0; c < nk; ++c) {
            const int q = c % LS_NA;
            __syncwarp();
            wc[lane] = cf_next;                       // this chunk's coefficients, lane j: degree l0 + j
            __syncwarp();
            cf_next = lt_coef_load(cm, lstart + 32 * (c + 1) + lane, N);
            if (c >= LS_NA) lt_spin(&sy.done[(c - LS_NA) % LS_NR], par(c - LS_NA), abort);
            tc::fence_after();
            const uint32_t ahi = tmem + lane_addr + (uint32_t)(384 + 64 * q), alo = ahi + 32;
            const int l0 = lstart + 32 * c;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float hi[8], lo[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) tc::split_tf32(rec.step(wc[8 * g + j], l0 + 8 * g + j), hi[j], lo[j]);
                tc::tmem_st8(ahi + 8 * g, hi);
                tc::tmem_st8(alo + 8 * g, lo);
            }
            tc::tmem_wait_st();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.full[c % LS_NR]);
        }
    } else if (warp < LT_MMA_WARP) {
        // ------------------------------------------------ operand B (c_l f_lm) and drains
        const int u = tid - 32 * LT_REC_WARPS;
        const int nmi_src = CPLX ? 2 * Lsrc - 1 : Lsrc;
        float sum[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) sum[i] = 0.f;
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        const int h = (warp - LT_REC_WARPS) >> 2;
        auto drain = [&](int c) {                     // accumulator c % LS_NACC into sum
            lt_spin(&sy.done[c % LS_NR], par(c), abort);
            tc::fence_after();
            const uint32_t acc = tmem + lane_addr + (uint32_t)(128 * (c % LS_NACC) + 64 * h);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float v[16];
                tc::tmem_ld16(acc + 16 * g, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[16 * g + i] += v[i];
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.tempty[c % LS_NACC]);
        };
        int drained = 0;
        for (int c = 0; c < nk; ++c) {
            const int q = c % LS_NB;
            const int l0 = lstart + 32 * c;
            auto row = [&](int p) -> const float2 * {
                const int sg = p / BT, b = p % BT;
                if (b0 + b >= B || (sg == 1 && !two)) return nullptr;
                const int mi = sg == 0 ? (CPLX ? m + Lsrc - 1 : m) : (-m + Lsrc - 1);
                return src + ((size_t)(b0 + b) * nmi_src + mi) * Lsrc + l0;
            };
            LtB bv;
            bv.load(u, row, N - l0, kfac ? kfac + l0 : nullptr);
            // the accumulator of chunk c - LS_NACC must be drained before chunk c's MMAs;
            // draining no earlier keeps operand B LS_NACC chunks ahead of the MMAs
            while (drained <= c - LS_NACC) drain(drained++);
            if (c >= LS_NB) lt_spin(&sy.done[(c - LS_NB) % LS_NR], par(c - LS_NB), abort);
            bv.store(smem + q * LS_STAGE, u);
            lt_warp_arrive(&sy.full[c % LS_NR], lane);
        }
        while (drained < nk) drain(drained++);
        // epilogue: TMEM lane = ring
        const int t = t0 + 32 * (warp & 3) + lane;
        if (t < N && !sy.abort) {
            const int nmi_dst = CPLX ? 2 * N - 1 : N;
            const float sgn_m = (m & 1) ? -1.f : 1.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int p = 32 * h + j;
                const int sg = p / BT, b = p % BT;
                if (b0 + b >= B || (sg == 1 && !two)) continue;
                const float f = sg == 1 ? scale * sgn_m : scale;
                const int mi = sg == 0 ? (CPLX ? m + N - 1 : m) : (-m + N - 1);
                dst[((size_t)(b0 + b) * nmi_dst + mi) * N + t] = make_float2(sum[2 * j] * f, sum[2 * j + 1] * f);
            }
        }
    } else if (lane == 0) {
        // ------------------------------------------------ MMA issue: A from TMEM, B from shared memory
        constexpr uint32_t IDESC = tc::idesc_tf32(128, 128);
        for (int c = 0; c < nk; ++c) {
            bool ok = lt_spin(&sy.full[c % LS_NR], par(c), abort);
            if (c >= LS_NACC) ok = lt_spin(&sy.tempty[c % LS_NACC], ((c / LS_NACC) - 1) & 1, abort) && ok;
            tc::fence_after();
            if (ok) {
                const uint32_t bbase = tc::smem_addr(smem + (c % LS_NB) * LS_STAGE);
                const uint32_t acc = tmem + (uint32_t)(128 * (c % LS_NACC));
                const uint32_t ahi = tmem + (uint32_t)(384 + 64 * (c % LS_NA)), alo = ahi + 32;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t b0d = tc::smem_desc_sw128(bbase + ks * 32);
                    const uint64_t b1d = tc::smem_desc_sw128(bbase + LT_PLANE + ks * 32);
                    tc::mma_tf32_ts(acc, ahi + 8 * ks, b1d, IDESC, ks > 0 ? 1u : 0u);
                    tc::mma_tf32_ts(acc, alo + 8 * ks, b0d, IDESC, 1u);
                    tc::mma_tf32_ts(acc, ahi + 8 * ks, b0d, IDESC, 1u);
                }
            }
            tc::mma_commit(&sy.done[c % LS_NR]);
        }
        tc::mma_commit(&sy.fin);
        tc::mbar_wait(&sy.fin, 0, 1u << 22);   // no MMA in flight when TMEM is released
    }
    tc::fence_before();
    __syncthreads();
    if (warp == LT_MMA_WARP) tc::tmem_free(tmem, LT_TMEM_COLS);
    if (tid == 0 && sy.abort) atomicExch(err, 1);
}

// ---------------------------------------------------------------- analysis
// Block: (order m, batch tile).  Degree tiles of 128 from l = m (MMA rows),
// K = rings in chunks of 32 (chunks whose rings all have l_s beyond the degree
// tile are skipped), columns = G columns.  Twelve warps:
//   recurrence warps 0-3  warp w computes the chunks c = w mod 4 of the sequence
//                         into its own operand-A stage (lane i owns ring 32 k + i
//                         and writes column i of A: one 4-byte store per degree
//                         and plane, conflict-free in the swizzled layout), then
//                         one of its threads issues and commits the chunk's MMAs
//                         once operand B is in place.  There is no MMA warp, so a
//                         fourth recurrence warp fits in twelve warps (168
//                         registers per thread; thirteen would leave 128)
//   warps 4-11            operand B (G) in a ring of two stages, and the drains
//                         of the accumulators (three TMEM buffers) into FP32
//                         registers; epilogue per degree tile
// Barriers per chunk c: full[c % LA_NR] (the eight operand-B warps), done[c %
// LA_NR] (the MMAs completed: A stage c % 4 and B stage c % 2 are free, the
// accumulator can be drained), tempty[c % 3] (drained).  MMAs of different
// chunks may be issued out of order (by different warps); every wait names its
// chunk, and no waiter can fall LA_NR chunks behind a barrier.  The recurrence
// warps poll their waits without suspending (lt_spin): measured faster here.
// Recurrence states of all rings stay in shared memory between degree tiles;
// the recurrence warps meet at a named barrier at the end of each degree tile
// before the states are read again.
constexpr int LA_NA = LT_ANAL_REC, LA_NB = 2, LA_NACC = 3, LA_NR = 12;
constexpr int LA_STAGE = 2 * LT_PLANE;                // one operand: hi, lo
constexpr int LA_B_OFF = LA_NA * LA_STAGE;
constexpr int LA_SYNC_OFF = LA_B_OFF + LA_NB * LA_STAGE;
struct LaSync {
    uint64_t full[LA_NR], done[LA_NR], tempty[LA_NACC];
    uint32_t tslot;
    int abort;
};
constexpr int LA_SYNC_BYTES = 256;
static_assert(sizeof(LaSync) <= LA_SYNC_BYTES, "sync block");
static_assert(LA_NR % LA_NA == 0 && LA_NR % LA_NB == 0 && LA_NR % LA_NACC == 0, "barrier ring");
// The recurrence states of all rings stay in shared memory up to this
// band-limit (226 KB in all at 2048); above it they live in a global buffer of
// N float4 per block (st_g), read and written at each degree tile like the
// shared copy.
constexpr int LA_ST_SMEM_MAX = 2048;
__host__ __device__ constexpr size_t la_anal_smem(int N)
{
    return (size_t)LA_SYNC_OFF + LA_SYNC_BYTES + (size_t)(N <= LA_ST_SMEM_MAX ? N : 0) * sizeof(float4) +
           (size_t)((N + 31) / 32) * sizeof(int) + 1024;
}

template <bool CPLX>
static __global__ void __launch_bounds__(LT_ANAL_THREADS, 1)
    k_leg_anal_tc(const float2 *__restrict__ Gin, int N, const float *__restrict__ kfac, float scale, int accumulate,
                  float2 *__restrict__ dst, int Ldst, int B, LegTab<float> tab, int *err, float4 *st_g)
{
    using Cols = LegCols<CPLX>;
    constexpr int BT = Cols::BT;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    LaSync &sy = *reinterpret_cast<LaSync *>(smem + LA_SYNC_OFF);
    float4 *sts = reinterpret_cast<float4 *>(smem + LA_SYNC_OFF + LA_SYNC_BYTES);
    const bool st_shared = N <= LA_ST_SMEM_MAX;
    float4 *st = st_shared ? sts : st_g + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * N;
    int *gmin = reinterpret_cast<int *>(st_shared ? sts + N : sts);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = blockIdx.x, b0 = blockIdx.y * BT;
    const bool two = CPLX && m > 0;
    const int nkr = (N + 31) / 32;
    const int ndt = (N - m + 127) / 128;
    volatile int *abort = &sy.abort;
    auto par = [](int c) -> uint32_t { return (uint32_t)((c / LA_NR) & 1); };

    for (int k = warp; k < nkr; k += LT_ANAL_THREADS / 32) {
        const int t = 32 * k + lane;
        int v = t < N ? tab.ls[(size_t)m * N + t] : N;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) gmin[k] = v;
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < LA_NR; ++i) {
            tc::mbar_init(&sy.full[i], LT_OPB_WARPS);
            tc::mbar_init(&sy.done[i], 1);
        }
#pragma unroll
        for (int i = 0; i < LA_NACC; ++i) tc::mbar_init(&sy.tempty[i], LT_OPB_WARPS);
        sy.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&sy.tslot, LT_TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sy.tslot;

    if (warp < LA_NA) {
        // ------------------------------------------------ recurrence (A = lambda[degree][ring]) and MMA issue
        constexpr uint32_t IDESC = tc::idesc_tf32(128, 128);
        const float4 *cm = tab.coef + (size_t)m * tab.ldc;
        unsigned char *A = smem + warp * LA_STAGE;
        const uint32_t abase = tc::smem_addr(A);
        int c = 0, last = -1;
        for (int dt = 0; dt < ndt; ++dt) {
            const int l0 = m + 128 * dt;
            const int lend = min(N, l0 + 128);
            // lane j holds the coefficients of degrees l0 + 32 i + j, i = 0..3
            const float4 cf0 = lt_coef_load(cm, l0 + lane, lend), cf1 = lt_coef_load(cm, l0 + 32 + lane, lend);
            const float4 cf2 = lt_coef_load(cm, l0 + 64 + lane, lend), cf3 = lt_coef_load(cm, l0 + 96 + lane, lend);
            for (int k = 0; k < nkr; ++k) {
                if (gmin[k] >= lend) continue;
                const int cc = c++;
                if (cc % LA_NA != warp) continue;
                // the ring's tables are loaded before the wait for the stage, so that
                // their latency overlaps it
                const int t = 32 * k + lane;
                const bool own = t < N;
                LtRec rec;
                rec.init(own, tab.ring + t, tab.seed + (size_t)m * N + t, tab.ls + (size_t)m * N + t);
                if (cc >= LA_NA) lt_spin(&sy.done[(cc - LA_NA) % LA_NR], par(cc - LA_NA), abort);
                if (own && l0 > rec.ls) {
                    const float4 q = st[t];
                    rec.p0.h = q.x;
                    rec.p0.l = q.y;
                    rec.p1.h = q.z;
                    rec.p1.l = q.w;
                }
#pragma unroll 1
                for (int i = 0; i < 4; ++i) {
                    const float4 cf = i == 0 ? cf0 : i == 1 ? cf1 : i == 2 ? cf2 : cf3;
                    const int lb = l0 + 32 * i;
                    if (__any_sync(0xffffffffu, rec.starts_in(lb, 32))) {   // a chain of this warp starts here
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            float hi, lo;
                            tc::split_tf32(rec.step(lt_coef(cf, j), lb + j), hi, lo);
                            const uint32_t o = tc::sw128_off(32 * i + j, lane);
                            *reinterpret_cast<float *>(A + o) = hi;
                            *reinterpret_cast<float *>(A + LT_PLANE + o) = lo;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            float hi, lo;
                            tc::split_tf32(rec.step_plain(lt_coef(cf, j)), hi, lo);
                            const uint32_t o = tc::sw128_off(32 * i + j, lane);
                            *reinterpret_cast<float *>(A + o) = hi;
                            *reinterpret_cast<float *>(A + LT_PLANE + o) = lo;
                        }
                    }
                }
                if (own && lend - 1 >= rec.ls) st[t] = make_float4(rec.p0.h, rec.p0.l, rec.p1.h, rec.p1.l);
                // operand A written and visible to the tensor core; one thread issues
                // the chunk's MMAs once operand B is stored and the accumulator drained
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    bool ok = lt_spin(&sy.full[cc % LA_NR], par(cc), abort);
                    if (cc >= LA_NACC)
                        ok = lt_spin(&sy.tempty[cc % LA_NACC], ((cc / LA_NACC) - 1) & 1, abort) && ok;
                    tc::fence_after();
                    if (ok) {
                        const uint32_t bbase = tc::smem_addr(smem + LA_B_OFF + (cc % LA_NB) * LA_STAGE);
                        const uint32_t acc = tmem + (uint32_t)(128 * (cc % LA_NACC));
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint32_t ko = ks * 32;
                            const uint64_t a0 = tc::smem_desc_sw128(abase + ko);
                            const uint64_t a1 = tc::smem_desc_sw128(abase + LT_PLANE + ko);
                            const uint64_t b0d = tc::smem_desc_sw128(bbase + ko);
                            const uint64_t b1d = tc::smem_desc_sw128(bbase + LT_PLANE + ko);
                            tc::mma_tf32(acc, a0, b1d, IDESC, ks > 0 ? 1u : 0u);
                            tc::mma_tf32(acc, a1, b0d, IDESC, 1u);
                            tc::mma_tf32(acc, a0, b0d, IDESC, 1u);
                        }
                    }
                    tc::mma_commit(&sy.done[cc % LA_NR]);
                }
                __syncwarp();
                last = cc;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * LA_NA) : "memory");
        }
        // no MMA of this warp in flight when the block ends (its last commit
        // covers all of them; bounded)
        if (lane == 0 && last >= 0) tc::mbar_wait(&sy.done[last % LA_NR], par(last), 1u << 22);
    } else {
        // ------------------------------------------------ operand B (G) and drains
        const int u = tid - 32 * LT_REC_WARPS;
        const int nmi_src = CPLX ? 2 * N - 1 : N;
        const int nmi_dst = CPLX ? 2 * Ldst - 1 : Ldst;
        const float sgn_m = (m & 1) ? -1.f : 1.f;
        float sum[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) sum[i] = 0.f;
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        const int h = (warp - LT_REC_WARPS) >> 2;
        auto drain = [&](int c) {                     // accumulator c % LA_NACC into sum
            lt_wait(&sy.done[c % LA_NR], par(c), abort);
            tc::fence_after();
            const uint32_t acc = tmem + lane_addr + (uint32_t)(128 * (c % LA_NACC) + 64 * h);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tc::tmem_ld16(acc + 16 * q, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) sum[16 * q + i] += v[i];
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sy.tempty[c % LA_NACC]);
        };
        int c = 0, drained = 0;
        for (int dt = 0; dt < ndt; ++dt) {
            const int l0 = m + 128 * dt;
            const int lend = min(N, l0 + 128);
            for (int k = 0; k < nkr; ++k) {
                if (gmin[k] >= lend) continue;
                const int cc = c++;
                const int t0 = 32 * k;
                auto row = [&](int p) -> const float2 * {
                    const int sg = p / BT, b = p % BT;
                    if (b0 + b >= B || (sg == 1 && !two)) return nullptr;
                    const int mi = sg == 0 ? (CPLX ? m + N - 1 : m) : (-m + N - 1);
                    return Gin + ((size_t)(b0 + b) * nmi_src + mi) * N + t0;
                };
                LtB bv;
                bv.load<true>(u, row, N - t0, nullptr);
                // the next ring chunk's values of this thread into L2, so that its loads
                // (issued only one drain ahead of their use) find them there (the
                // chunk after k is usually k + 1; a skipped one costs a wasted prefetch)
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int unit = u + 256 * i, kk = t0 + 32 + 4 * (unit & 7);
                    const float2 *r = row(unit >> 3);
                    if (r && kk < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(r + 32 + 4 * (unit & 7)));
                }
                while (drained <= cc - LA_NACC) drain(drained++);
                if (cc >= LA_NB) lt_wait(&sy.done[(cc - LA_NB) % LA_NR], par(cc - LA_NB), abort);
                bv.store(smem + LA_B_OFF + (cc % LA_NB) * LA_STAGE, u);
                lt_warp_arrive(&sy.full[cc % LA_NR], lane);
            }
            while (drained < c) drain(drained++);
            // epilogue of the degree tile: TMEM lane = degree
            const int l = l0 + 32 * (warp & 3) + lane;
            if (l < lend && !sy.abort) {
                const float f = scale * (kfac ? kfac[l] : 1.f);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int p = 32 * h + j;
                    const int sg = p / BT, b = p % BT;
                    if (b0 + b < B && (sg == 0 || two)) {
                        const float fs = sg == 1 ? f * sgn_m : f;
                        const int mi = sg == 0 ? (CPLX ? m + Ldst - 1 : m) : (-m + Ldst - 1);
                        float2 *o = dst + ((size_t)(b0 + b) * nmi_dst + mi) * Ldst + l;
                        float2 v = make_float2(sum[2 * j] * fs, sum[2 * j + 1] * fs);
                        if (accumulate) {
                            const float2 w = *o;
                            v.x += w.x;
                            v.y += w.y;
                        }
                        *o = v;
                    }
                    if ((j & 7) == 7) asm volatile("" ::: "memory");   // keep the loads of later pairs below
                }
            }
#pragma unroll
            for (int i = 0; i < 64; ++i) sum[i] = 0.f;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, LT_TMEM_COLS);
    if (tid == 0 && sy.abort) atomicExch(err, 1);
}

}  // namespace s2g
