// Warp-specialised tcgen05 pipeline shared by the tensor-core contraction
// kernels (split-TF32 products, see tc_kernels.cuh for the split scheme).
// Each 128 x 128 x 32 chunk is the sum of the MMAs hi*lo + lo*hi + hi*hi
// accumulated in its own TMEM buffer, then added into FP32 registers.
//
// Warp roles, synchronised by mbarriers over LT_NS shared-memory stages:
//   producer warps  write operand A of a stage (recurrence values, or copies
//                   of a pre-split matrix)
//   warps 4-11      operand B (the data side) of a stage, and drain the TMEM
//                   accumulator of each finished chunk into registers; epilogue
//   MMA warp        one thread issues the MMAs and commits them
// Per stage: A hi, A lo, B hi, B lo, each a 128 x 32 FP32 tile in the K-major
// 128-byte-swizzled layout (16 KB).  Barriers per stage s:
//   full[s]   operands written: one arrival per writing warp (the producer
//             warps that wrote A and the eight operand-B warps), after each
//             lane's proxy fence and a warp barrier
//   empty[s]  the chunk's MMAs have completed (tcgen05.commit): stage s free and
//             TMEM buffer s holds the chunk's sum
//   tempty[s] TMEM buffer s drained (one arrival per operand-B warp)
// Every wait is bounded; a wait that runs out sets a shared abort flag, after
// which all roles run to the end without waiting and the error word is set.
#pragma once
#include "common.cuh"
#include "tc_kernels.cuh"
#include "tc_sm100.cuh"

namespace s2g {

constexpr int LT_REC_WARPS = 4, LT_OPB_WARPS = 8, LT_MMA_WARP = LT_REC_WARPS + LT_OPB_WARPS;
constexpr int LT_THREADS = 32 * (LT_MMA_WARP + 1);
constexpr int LT_NS = 3;
constexpr int LT_PLANE = TQ_TILE;                  // 128 x 32 FP32
constexpr int LT_STAGE = 4 * LT_PLANE;
constexpr int LT_TMEM_COLS = 512;                  // LT_NS accumulators of 128 columns

struct LtSync {
    uint64_t full[LT_NS], empty[LT_NS], tempty[LT_NS], done;
    uint32_t tslot;
    int abort;
    int lmin;
    int nchunks;
};
constexpr int LT_SYNC_BYTES = 128;
static_assert(sizeof(LtSync) <= LT_SYNC_BYTES, "sync block");

// dynamic shared memory: stages, sync block, 1024-byte alignment slack, and
// (analysis) recurrence states and per-ring-chunk minima of l_s for N rings
__host__ __device__ constexpr size_t lt_synth_smem() { return (size_t)LT_NS * LT_STAGE + LT_SYNC_BYTES + 1024; }
__host__ __device__ constexpr size_t lt_anal_smem(int N)
{
    return lt_synth_smem() + (size_t)N * sizeof(float4) + (size_t)((N + 31) / 32) * sizeof(int);
}

__device__ __forceinline__ bool lt_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        if (tc::mbar_try_wait_hint(bar, parity, 1000)) return true;
        if (*abort) return false;
    }
    *abort = 1;
    return false;
}

// As lt_wait, polling with the non-blocking test_wait instead of a suspending
// try_wait (for waits on the critical path of a block whose other warps have
// issue slots to spare).
__device__ __forceinline__ bool lt_spin(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    for (uint32_t i = 0; i < (1u << 26); ++i) {
        uint32_t ok;
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(ok)
            : "r"(tc::smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255) == 255 && *abort) return false;
    }
    *abort = 1;
    return false;
}

// The calling warp's shared-memory writes are complete and visible to the
// tensor core: every lane fences the async proxy, then one arrival for the warp.
__device__ __forceinline__ void lt_warp_arrive(uint64_t *bar, int lane)
{
    tc::fence_proxy_async();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(bar);
}

__device__ __forceinline__ unsigned char *lt_align(unsigned char *p)
{
    return p + ((1024 - (tc::smem_addr(p) & 1023)) & 1023);
}

// Barrier set-up (thread 0) and TMEM allocation (MMA warp); ends with a CTA
// barrier.  full_arrivals: arrivals on full[] per chunk (one per warp that
// writes an operand, one per bulk-copy issue); the eight drain warps arrive on
// tempty[].
__device__ __forceinline__ void lt_setup(LtSync &sy, int warp, int tid, int full_arrivals, int mma_warp)
{
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < LT_NS; ++i) {
            tc::mbar_init(&sy.full[i], full_arrivals);
            tc::mbar_init(&sy.empty[i], 1);
            tc::mbar_init(&sy.tempty[i], LT_OPB_WARPS);
        }
        tc::mbar_init(&sy.done, 1);
        sy.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == mma_warp) tc::tmem_alloc(&sy.tslot, LT_TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// MMA issue loop (one thread): chunk c uses stage and TMEM buffer c % LT_NS.
__device__ __forceinline__ void lt_issue(LtSync &sy, unsigned char *smem, uint32_t tmem, int nchunks)
{
    constexpr uint32_t IDESC = tc::idesc_tf32(128, 128);
    volatile int *abort = &sy.abort;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c % LT_NS;
        bool ok = lt_wait(&sy.full[s], (c / LT_NS) & 1, abort);
        if (c >= LT_NS) ok = lt_wait(&sy.tempty[s], ((c / LT_NS) - 1) & 1, abort) && ok;
        tc::fence_after();
        if (ok) {
            const uint32_t base = tc::smem_addr(smem + s * LT_STAGE);
            const uint32_t acc = tmem + (uint32_t)(s * 128);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t ko = ks * 32;
                const uint64_t a0 = tc::smem_desc_sw128(base + ko), a1 = tc::smem_desc_sw128(base + LT_PLANE + ko);
                const uint64_t b0 = tc::smem_desc_sw128(base + 2 * LT_PLANE + ko);
                const uint64_t b1 = tc::smem_desc_sw128(base + 3 * LT_PLANE + ko);
                tc::mma_tf32(acc, a0, b1, IDESC, ks > 0 ? 1u : 0u);
                tc::mma_tf32(acc, a1, b0, IDESC, 1u);
                tc::mma_tf32(acc, a0, b0, IDESC, 1u);
            }
        }
        tc::mma_commit(&sy.empty[s]);
    }
    tc::mma_commit(&sy.done);
    tc::mbar_wait(&sy.done, 0, 1u << 22);   // no MMA in flight when TMEM is released
}

// Operand-B / drain thread state: TMEM lane quadrant q = warp % 4, column half h.
struct LtDrain {
    float sum[64];
    uint32_t lane_addr;
    int h;
    __device__ __forceinline__ void init(int warp)
    {
        lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        h = (warp - LT_REC_WARPS) >> 2;
#pragma unroll
        for (int i = 0; i < 64; ++i) sum[i] = 0.f;
    }
    // add chunk c's accumulator (64 columns of this thread's lane) into sum; NS
    // stages (TMEM buffer c % NS at column 128 (c % NS))
    template <int NS = LT_NS> __device__ __forceinline__ void drain(LtSync &sy, uint32_t tmem, int c)
    {
        const int s = c % NS;
        lt_wait(&sy.empty[s], (c / NS) & 1, &sy.abort);
        tc::fence_after();
        const uint32_t acc = tmem + lane_addr + (uint32_t)(s * 128 + 64 * h);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float v[16];
            tc::tmem_ld16(acc + 16 * g, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) sum[16 * g + i] += v[i];
        }
        tc::fence_before();
        __syncwarp();
        if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&sy.tempty[s]);
    }
};

// Operand B of a chunk: 64 column pairs (sign s, map b) x 32 K values read
// from float2 rows (re, im), times an optional per-K factor, split into TF32
// hi and lo planes.  Two halves, so that the global loads of a chunk can be in
// flight while the thread waits for an accumulator to drain:
//   load:  u = operand-B thread index (0..255); row(p) returns the source row
//          of pair p shifted to the chunk's first K (nullptr: zero pair);
//          kmax = number of valid K values; fac = per-K factors (or nullptr)
//   store: split and write the swizzled planes of stage Bst
struct LtB {
    float2 v[2][4];
    // VEC: two 16-byte loads per unit where the row allows (measured faster in the
    // analysis, slightly slower in the quadrature and the synthesis)
    template <bool VEC = false, typename RowF>
    __device__ __forceinline__ void load(int u, RowF row, int kmax, const float *fac)
    {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int unit = u + 256 * i;
            const int kg = unit & 7, p = unit >> 3;
            const float2 *r = row(p);
            const int k = 4 * kg;
            if (VEC && r && k + 3 < kmax && ((reinterpret_cast<uintptr_t>(r + k) & 15) == 0)) {
                // two 16-byte loads cover the unit's four values
                const float4 a = *reinterpret_cast<const float4 *>(r + k);
                const float4 b = *reinterpret_cast<const float4 *>(r + k + 2);
                v[i][0] = make_float2(a.x, a.y);
                v[i][1] = make_float2(a.z, a.w);
                v[i][2] = make_float2(b.x, b.y);
                v[i][3] = make_float2(b.z, b.w);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[i][q] = (r && k + q < kmax) ? r[k + q] : make_float2(0.f, 0.f);
            }
            if (fac) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float f = (k + q < kmax) ? fac[k + q] : 0.f;
                    v[i][q].x *= f;
                    v[i][q].y *= f;
                }
            }
        }
    }
    __device__ __forceinline__ void store(unsigned char *Bst, int u) const
    {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int unit = u + 256 * i;
            const int kg = unit & 7, p = unit >> 3;
            float rh[4], rl[4], ih[4], il[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                tc::split_tf32(v[i][q].x, rh[q], rl[q]);
                tc::split_tf32(v[i][q].y, ih[q], il[q]);
            }
            const uint32_t o0 = tc::sw128_off(2 * p, 4 * kg), o1 = tc::sw128_off(2 * p + 1, 4 * kg);
            *reinterpret_cast<float4 *>(Bst + o0) = make_float4(rh[0], rh[1], rh[2], rh[3]);
            *reinterpret_cast<float4 *>(Bst + o1) = make_float4(ih[0], ih[1], ih[2], ih[3]);
            *reinterpret_cast<float4 *>(Bst + LT_PLANE + o0) = make_float4(rl[0], rl[1], rl[2], rl[3]);
            *reinterpret_cast<float4 *>(Bst + LT_PLANE + o1) = make_float4(il[0], il[1], il[2], il[3]);
        }
    }
};

__device__ __forceinline__ void lt_teardown(LtSync &sy, int warp, int tid, uint32_t tmem, int *err, int mma_warp)
{
    tc::fence_before();
    __syncthreads();
    if (warp == mma_warp) tc::tmem_free(tmem, LT_TMEM_COLS);
    if (tid == 0 && sy.abort) atomicExch(err, 1);
}

}  // namespace s2g
