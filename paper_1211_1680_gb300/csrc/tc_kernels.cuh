// Tensor-core (tcgen05, split TF32) contraction kernels of the TF32X3 plans.
//
// Each FP32 operand x is split into TF32 parts (top 10 explicit mantissa bits
// each, by truncation, the remainders exact in FP32) and a product is taken as
// a sum of MMAs of the parts with FP32 accumulation in tensor memory (the split
// scheme of Ootomo & Yokota), then partial sums are added in FP32 registers.
#pragma once
#include "common.cuh"
#include "tc_sm100.cuh"

namespace s2g {

// ---------------------------------------------------------------- quadrature product
// G[b][mi][t] = sum_t' Q[t][t'] F[b][mi][t'] for the orders mi = mi0, mi0 + 2, ...
// Operands split three ways, x = x1 + x2 + x3 (each TF32), products kept down to
// 2^-22 relative: x1 y1 + x1 y2 + x2 y1 + x1 y3 + x2 y2 + x3 y1 (6 MMAs per K step).
// Q arrives pre-split (Q3 = three N x N planes, built once per plan); F is split
// while it is stored to shared memory.
// Block: 256 threads; tile 128 rows (t) x 128 columns (64 (b, mi) pairs x re/im);
// K (t') in chunks of 32, two shared-memory stages: while the tensor core works
// on one chunk the threads fill the next.
constexpr int TQ_M = 128, TQ_N = 128, TQ_K = 32, TQ_THREADS = 256;
constexpr int TQ_TILE = TQ_M * TQ_K * 4;          // bytes of one operand plane tile (16 KB)
constexpr int TQ_STAGE = 6 * TQ_TILE;             // A1 A2 A3 B1 B2 B3
constexpr int TQ_SMEM = 2 * TQ_STAGE + 64 + 1024; // + two mbarriers, the TMEM address, 1024-byte alignment

__device__ __forceinline__ void split3(float x, float &a, float &b, float &c)
{
    float r;
    tc::split_tf32(x, a, r);
    tc::split_tf32(r, b, c);
}

// Accumulation: the tensor core accumulates one K chunk (32 values, 24 MMAs) into
// a fresh TMEM buffer (two buffers of 128 columns alternate); after the chunk
// completes, every thread adds its 64 accumulator values of the chunk into FP32
// registers.  Accumulating all of K in TMEM left a ~1.4e-5 relative error at
// N = 2048; per-chunk partial sums added with IEEE FP32 adds do not.
static __global__ void __launch_bounds__(TQ_THREADS, 1) k_quad_tc(const float *__restrict__ Q3,
                                                                  const float2 *__restrict__ F,
                                                                  float2 *__restrict__ G, int N, int nmi, int mi0,
                                                                  int nj, int npairs, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    // operand tiles need 1024-byte alignment for the 128-byte swizzle
    unsigned char *smem = smem_dyn + ((1024 - (tc::smem_addr(smem_dyn) & 1023)) & 1023);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * TQ_STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 2 * TQ_STAGE + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * TQ_M;
    const int pair0 = blockIdx.y * (TQ_N / 2);
    const size_t plane = (size_t)N * N;
    constexpr uint32_t IDESC = tc::idesc_tf32(TQ_M, TQ_N);

    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(tslot, 2 * TQ_N);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    // this thread's accumulator slice: TMEM lane 32 (w % 4) + lane, columns 64 (w / 4) + [0, 64)
    const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
    const int cbase = (warp >> 2) * 64;
    float sum[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) sum[i] = 0.f;
    bool ok = true;
    auto drain = [&](int q) {            // add chunk q's accumulator into sum
        if (!tc::mbar_wait(&bar[q & 1], (q >> 1) & 1)) ok = false;
        tc::fence_after();
        const uint32_t acc = tmem + lane_addr + (uint32_t)((q & 1) * TQ_N + cbase);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float v[16];
            tc::tmem_ld16(acc + g * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) sum[g * 16 + i] += v[i];
        }
    };

    const int nk = (N + TQ_K - 1) / TQ_K;
    const bool vec = (N & 3) == 0;
    for (int c = 0; c < nk; ++c) {
        const int s = c & 1;
        unsigned char *st = smem + s * TQ_STAGE;
        if (c >= 2) drain(c - 2);        // frees shared stage s and TMEM buffer s
        const int k0 = c * TQ_K;
        // all global loads of this chunk first (8 consecutive threads read 128 or
        // 256 contiguous bytes), then the split and the swizzled stores, which
        // are conflict-free for the same 8 threads
        constexpr int NA = 3 * TQ_M * (TQ_K / 4) / TQ_THREADS;       // 12 float4 of Q3 per thread
        constexpr int NB = (TQ_N / 2) * (TQ_K / 4) / TQ_THREADS;     // 2 (pair, group of 4 K) per thread
        float4 av[NA];
        float2 bv[NB][4];
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int u = tid + i * TQ_THREADS;
            const int kg = u & 7, r = (u >> 3) & (TQ_M - 1), pl = u >> 10;
            const int rr = row0 + r, kk = k0 + kg * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rr < N) {
                const float *q = Q3 + pl * plane + (size_t)rr * N + kk;
                if (vec && kk + 3 < N) {
                    v = __ldg(reinterpret_cast<const float4 *>(q));
                } else {
                    v.x = kk < N ? q[0] : 0.f;
                    v.y = kk + 1 < N ? q[1] : 0.f;
                    v.z = kk + 2 < N ? q[2] : 0.f;
                    v.w = kk + 3 < N ? q[3] : 0.f;
                }
            }
            av[i] = v;
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int u = tid + i * TQ_THREADS;
            const int kg = u & 7, p = u >> 3;
            const int pp = pair0 + p, kk = k0 + kg * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[i][q] = make_float2(0.f, 0.f);
            if (pp < npairs) {
                const int b = pp / nj, j = pp % nj;
                const float2 *row = F + ((size_t)b * nmi + mi0 + 2 * j) * N + kk;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (kk + q < N) bv[i][q] = row[q];
            }
        }
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int u = tid + i * TQ_THREADS;
            const int kg = u & 7, r = (u >> 3) & (TQ_M - 1), pl = u >> 10;
            *reinterpret_cast<float4 *>(st + pl * TQ_TILE + tc::sw128_off(r, kg * 4)) = av[i];
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int u = tid + i * TQ_THREADS;
            const int kg = u & 7, p = u >> 3;
            float4 r1, r2, r3, i1, i2, i3;
            split3(bv[i][0].x, r1.x, r2.x, r3.x);
            split3(bv[i][1].x, r1.y, r2.y, r3.y);
            split3(bv[i][2].x, r1.z, r2.z, r3.z);
            split3(bv[i][3].x, r1.w, r2.w, r3.w);
            split3(bv[i][0].y, i1.x, i2.x, i3.x);
            split3(bv[i][1].y, i1.y, i2.y, i3.y);
            split3(bv[i][2].y, i1.z, i2.z, i3.z);
            split3(bv[i][3].y, i1.w, i2.w, i3.w);
            const uint32_t o0 = tc::sw128_off(2 * p, kg * 4), o1 = tc::sw128_off(2 * p + 1, kg * 4);
            *reinterpret_cast<float4 *>(st + 3 * TQ_TILE + o0) = r1;
            *reinterpret_cast<float4 *>(st + 4 * TQ_TILE + o0) = r2;
            *reinterpret_cast<float4 *>(st + 5 * TQ_TILE + o0) = r3;
            *reinterpret_cast<float4 *>(st + 3 * TQ_TILE + o1) = i1;
            *reinterpret_cast<float4 *>(st + 4 * TQ_TILE + o1) = i2;
            *reinterpret_cast<float4 *>(st + 5 * TQ_TILE + o1) = i3;
        }
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            const uint32_t base = tc::smem_addr(st);
            const uint32_t acc = tmem + (uint32_t)(s * TQ_N);
#pragma unroll
            for (int ks = 0; ks < TQ_K / 8; ++ks) {
                const uint32_t ko = ks * 32;               // K = 8 FP32 per MMA = 32 bytes of the 128-byte row
                uint64_t a[3], bb[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    a[i] = tc::smem_desc_sw128(base + i * TQ_TILE + ko);
                    bb[i] = tc::smem_desc_sw128(base + (3 + i) * TQ_TILE + ko);
                }
                // smallest terms first
                tc::mma_tf32(acc, a[0], bb[2], IDESC, ks > 0 ? 1u : 0u);
                tc::mma_tf32(acc, a[1], bb[1], IDESC, 1u);
                tc::mma_tf32(acc, a[2], bb[0], IDESC, 1u);
                tc::mma_tf32(acc, a[0], bb[1], IDESC, 1u);
                tc::mma_tf32(acc, a[1], bb[0], IDESC, 1u);
                tc::mma_tf32(acc, a[0], bb[0], IDESC, 1u);
            }
            tc::mma_commit(&bar[s]);
        }
    }
    if (nk >= 2) drain(nk - 2);
    drain(nk - 1);
    // epilogue: rows t, columns (pair, re/im) from the register sums
    const int t_out = row0 + 32 * (warp & 3) + lane;
    if (ok && t_out < N) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int pp = pair0 + cbase / 2 + j;
            if (pp < npairs) {
                const int b = pp / nj, jj = pp % nj;
                G[((size_t)b * nmi + mi0 + 2 * jj) * N + t_out] = make_float2(sum[2 * j], sum[2 * j + 1]);
            }
        }
    }
    if (!ok && lane == 0) atomicExch(err, 1);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 2 * TQ_N);
}

// Q (FP32, N x N) -> three TF32 planes x1, x2, x3 with x = x1 + x2 + x3.
static __global__ void k_split3_planes(const float *__restrict__ Q, float *__restrict__ Q3, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a, b, c;
    split3(Q[i], a, b, c);
    Q3[i] = a;
    Q3[n + i] = b;
    Q3[2 * n + i] = c;
}

}  // namespace s2g
