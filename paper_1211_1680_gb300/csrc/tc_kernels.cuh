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
// Operands split into S TF32 parts (x = x1 + x2 [+ x3]); the MMAs keep the
// products down to 2^-11 (S = 2: x1 y1, x1 y2, x2 y1) or 2^-22 relative
// (S = 3: the six products with i + j <= 4).  Q arrives pre-split (three N x N
// planes, built once per plan); F is split while it is stored to shared memory.
// Block: 256 threads; tile 128 rows (t) x 128 columns (64 (b, mi) pairs x re/im);
// K (t') in chunks of 32 over NS shared-memory stages: while the tensor core
// works on one chunk the threads fill the next ones.
// Accumulation: each K chunk accumulates into its own TMEM buffer (NS buffers of
// 128 columns); once a chunk completes, every thread adds its 64 accumulator
// values into FP32 registers.  Accumulating all of K in TMEM left a ~1.4e-5
// relative error at N = 2048; per-chunk sums added with IEEE FP32 adds do not.
constexpr int TQ_M = 128, TQ_N = 128, TQ_K = 32, TQ_THREADS = 256;
constexpr int TQ_TILE = TQ_M * TQ_K * 4;          // bytes of one operand plane tile (16 KB)
template <int S, int NS> struct TqShape {
    static constexpr int STAGE = 2 * S * TQ_TILE;
    static constexpr int SMEM = NS * STAGE + 64 + 1024;   // + mbarriers, TMEM address, alignment
    static constexpr int TMEM_COLS = NS * TQ_N <= 256 ? (NS * TQ_N <= 128 ? 128 : 256) : 512;
};

__device__ __forceinline__ void split3(float x, float &a, float &b, float &c)
{
    float r;
    tc::split_tf32(x, a, r);
    tc::split_tf32(r, b, c);
}

template <int S, int NS>
static __global__ void __launch_bounds__(TQ_THREADS, 1) k_quad_tc(const float *__restrict__ Q3,
                                                                  const float2 *__restrict__ F,
                                                                  float2 *__restrict__ G, int N, int nmi, int mi0,
                                                                  int nj, int npairs, int *err)
{
    using Sh = TqShape<S, NS>;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    // operand tiles need 1024-byte alignment for the 128-byte swizzle
    unsigned char *smem = smem_dyn + ((1024 - (tc::smem_addr(smem_dyn) & 1023)) & 1023);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + NS * Sh::STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + NS * Sh::STAGE + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * TQ_M;
    const int pair0 = blockIdx.y * (TQ_N / 2);
    const size_t plane = (size_t)N * N;
    constexpr uint32_t IDESC = tc::idesc_tf32(TQ_M, TQ_N);

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) tc::mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(tslot, Sh::TMEM_COLS);
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
        if (!tc::mbar_wait(&bar[q % NS], (q / NS) & 1)) ok = false;
        tc::fence_after();
        const uint32_t acc = tmem + lane_addr + (uint32_t)((q % NS) * TQ_N + cbase);
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
        const int s = c % NS;
        unsigned char *st = smem + s * Sh::STAGE;
        if (c >= NS) drain(c - NS);      // frees shared stage s and TMEM buffer s
        const int k0 = c * TQ_K;
        // all global loads of this chunk first (8 consecutive threads read 128 or
        // 256 contiguous bytes), then the split and the swizzled stores, which
        // are conflict-free for the same 8 threads
        constexpr int NA = S * TQ_M * (TQ_K / 4) / TQ_THREADS;       // float4 of Q planes per thread
        constexpr int NB = (TQ_N / 2) * (TQ_K / 4) / TQ_THREADS;     // (pair, group of 4 K) per thread
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
            float4 rp[3], ip[3];
            float *rr = reinterpret_cast<float *>(rp), *ii = reinterpret_cast<float *>(ip);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (S == 3) {
                    split3(bv[i][q].x, rr[q], rr[4 + q], rr[8 + q]);
                    split3(bv[i][q].y, ii[q], ii[4 + q], ii[8 + q]);
                } else {
                    tc::split_tf32(bv[i][q].x, rr[q], rr[4 + q]);
                    tc::split_tf32(bv[i][q].y, ii[q], ii[4 + q]);
                }
            }
            const uint32_t o0 = tc::sw128_off(2 * p, kg * 4), o1 = tc::sw128_off(2 * p + 1, kg * 4);
#pragma unroll
            for (int pl = 0; pl < S; ++pl) {
                *reinterpret_cast<float4 *>(st + (S + pl) * TQ_TILE + o0) = rp[pl];
                *reinterpret_cast<float4 *>(st + (S + pl) * TQ_TILE + o1) = ip[pl];
            }
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
                uint64_t a[S], bb[S];
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    a[i] = tc::smem_desc_sw128(base + i * TQ_TILE + ko);
                    bb[i] = tc::smem_desc_sw128(base + (S + i) * TQ_TILE + ko);
                }
                // smallest terms first
                if (S == 3) {
                    tc::mma_tf32(acc, a[0], bb[S - 1], IDESC, ks > 0 ? 1u : 0u);
                    tc::mma_tf32(acc, a[1], bb[1], IDESC, 1u);
                    tc::mma_tf32(acc, a[S - 1], bb[0], IDESC, 1u);
                    tc::mma_tf32(acc, a[0], bb[1], IDESC, 1u);
                } else {
                    tc::mma_tf32(acc, a[0], bb[1], IDESC, ks > 0 ? 1u : 0u);
                }
                tc::mma_tf32(acc, a[1], bb[0], IDESC, 1u);
                tc::mma_tf32(acc, a[0], bb[0], IDESC, 1u);
            }
            tc::mma_commit(&bar[s]);
        }
    }
    for (int q = nk > NS ? nk - NS : 0; q < nk; ++q) drain(q);
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
    if (warp == 0) tc::tmem_free(tmem, Sh::TMEM_COLS);
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
