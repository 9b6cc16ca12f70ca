// MW theta quadrature of the TF32X3 plans as a pipelined tensor-core product
// (tc_pipe.cuh):  G[b][mi][t] = sum_t' Q_sigma[t][t'] F[b][mi][t']  for the
// orders mi = mi0, mi0 + 2, ... of one parity sigma.
//   operand A  rows t of Q_sigma, pre-split into two TF32 planes (hi, and the
//              TF32 part of the remainder) with a zero-padded row stride ldq
//              (a multiple of 4 floats, so every row starts on 16 bytes); warps
//              0-3 copy them into the swizzled stage layout with cp.async,
//              two chunks in flight
//   operand B  64 (b, mi) pairs x re/im of F, split while stored (LtB)
// Block: (tile of 128 rows t, tile of 64 pairs).
#pragma once
#include "tc_pipe.cuh"

namespace s2g {

constexpr int QP_LOAD_WARPS = 4;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(tc::smem_addr(smem_dst)), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

static __global__ void __launch_bounds__(LT_THREADS, 1)
    k_quad_tcp(const float *__restrict__ Qp, int ldq, const float2 *__restrict__ F, float2 *__restrict__ G, int N,
               int nmi, int mi0, int nj, int npairs, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    LtSync &sy = *reinterpret_cast<LtSync *>(smem + LT_NS * LT_STAGE);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * 128, pair0 = blockIdx.y * 64;
    const int nk = (N + 31) / 32;
    lt_setup(sy, warp, tid, QP_LOAD_WARPS, LT_MMA_WARP);
    const uint32_t tmem = sy.tslot;

    if (warp < QP_LOAD_WARPS) {
        // ------------------------------------------------ operand A: Q planes by cp.async
        const size_t plane = (size_t)N * ldq;
        for (int c = 0; c < nk; ++c) {
            const int s = c % LT_NS;
            if (c >= LT_NS) lt_wait(&sy.empty[s], ((c / LT_NS) - 1) & 1, &sy.abort);
            unsigned char *A = smem + s * LT_STAGE;
            const int k0 = 32 * c;
#pragma unroll
            for (int i = 0; i < 16; ++i) {   // 2 planes x 128 rows x 8 pieces of 16 bytes
                const int u = tid + 128 * i;
                const int kg = u & 7, r = (u >> 3) & 127, pl = u >> 10;
                const int rr = row0 + r, kk = k0 + 4 * kg;
                const bool ok = rr < N && kk < ldq;
                const float *src = Qp + pl * plane + (ok ? (size_t)rr * ldq + kk : 0);
                cp_async16(A + pl * LT_PLANE + tc::sw128_off(r, 4 * kg), src, ok ? 16 : 0);
            }
            cp_async_commit();
            if (c > 0) {
                cp_async_wait<1>();          // this thread's copies of chunk c - 1 have landed
                lt_warp_arrive(&sy.full[(c - 1) % LT_NS], lane);
            }
        }
        if (nk > 0) {
            cp_async_wait<0>();
            lt_warp_arrive(&sy.full[(nk - 1) % LT_NS], lane);
        }
    } else if (warp < LT_MMA_WARP) {
        // ------------------------------------------------ operand B (F) and drains
        const int u = tid - 32 * LT_REC_WARPS;
        LtDrain d;
        d.init(warp);
        int drained = 0;
        for (int c = 0; c < nk; ++c) {
            const int s = c % LT_NS;
            const int k0 = 32 * c;
            auto row = [&](int p) -> const float2 * {
                const int pp = pair0 + p;
                if (pp >= npairs) return nullptr;
                const int b = pp / nj, j = pp % nj;
                return F + ((size_t)b * nmi + mi0 + 2 * j) * N + k0;
            };
            LtB bv;
            bv.load(u, row, N - k0, nullptr);
            while (drained <= c - LT_NS) d.drain(sy, tmem, drained++);
            bv.store(smem + s * LT_STAGE + 2 * LT_PLANE, u);
            lt_warp_arrive(&sy.full[s], lane);
        }
        while (drained < nk) d.drain(sy, tmem, drained++);
        // epilogue: TMEM lane = row t
        const int t = row0 + 32 * (warp & 3) + lane;
        if (t < N && !sy.abort) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int pp = pair0 + 32 * d.h + j;
                if (pp < npairs) {
                    const int b = pp / nj, jj = pp % nj;
                    G[((size_t)b * nmi + mi0 + 2 * jj) * N + t] = make_float2(d.sum[2 * j], d.sum[2 * j + 1]);
                }
            }
        }
    } else if (lane == 0) {
        lt_issue(sy, smem, tmem, nk);
    }
    lt_teardown(sy, warp, tid, tmem, err, LT_MMA_WARP);
}

// Q (FP32, N x N) -> planes hi, lo with row stride ldq >= N (zero padding):
// hi = the TF32 truncation of x, lo = the TF32 truncation of x - hi.
static __global__ void k_split2_padded(const float *__restrict__ Q, float *__restrict__ Qp, int N, int ldq)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = (size_t)N * ldq;
    if (i >= n) return;
    const int r = (int)(i / ldq), k = (int)(i % ldq);
    const float x = k < N ? Q[(size_t)r * N + k] : 0.f;
    float hi, rem, lo, drop;
    tc::split_tf32(x, hi, rem);
    tc::split_tf32(rem, lo, drop);
    Qp[i] = hi;
    Qp[n + i] = lo;
}

}  // namespace s2g
