// Pieces shared by the warp-specialised tcgen05 kernels (split-TF32 products,
// see tc_kernels.cuh for the split scheme): block shape constants, bounded
// mbarrier waits, the warp arrival after operand stores, and the operand-B
// loader/splitter.  Each 128 x 128 x 32 chunk of those kernels is the sum of
// the MMAs hi*lo + lo*hi + hi*hi; operands are 128 x 32 FP32 tiles in the
// K-major 128-byte-swizzled layout (16 KB per plane).
// Every wait is bounded; a wait that runs out sets a shared abort flag, after
// which all roles run to the end without waiting and the error word is set.
#pragma once
#include "common.cuh"
#include "tc_kernels.cuh"
#include "tc_sm100.cuh"

namespace s2g {

// producer warps 0-3 (one per TMEM lane quadrant), operand-B / drain warps 4-11,
// and (in the kernels that have one) an MMA warp 12
constexpr int LT_REC_WARPS = 4, LT_OPB_WARPS = 8, LT_MMA_WARP = LT_REC_WARPS + LT_OPB_WARPS;
constexpr int LT_THREADS = 32 * (LT_MMA_WARP + 1);
constexpr int LT_PLANE = TQ_TILE;                  // 128 x 32 FP32
constexpr int LT_TMEM_COLS = 512;                  // TMEM columns per block

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

}  // namespace s2g
