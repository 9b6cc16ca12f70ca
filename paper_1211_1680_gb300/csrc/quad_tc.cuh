// MW theta quadrature of the TF32X3 plans as a pipelined tensor-core product
// (tc_pipe.cuh):  G[b][mi][t] = sum_t' Q_sigma[t][t'] F[b][mi][t']  for the
// orders mi = mi0, mi0 + 2, ... of one parity sigma.
//   operand A  Q_sigma, split into two TF32 planes (hi, and the TF32 part of
//              the remainder) and stored once per plan as the exact shared-
//              memory image of each (row tile, K chunk): two 128 x 32 tiles in
//              the swizzled layout, 32 KB contiguous, zeros outside N x N.  One
//              thread moves a chunk with a single bulk copy (TMA engine) whose
//              completion is counted on the stage's full barrier
//   operand B  64 (b, mi) pairs x re/im of F, split while stored (LtB) by
//              warps 4-11, which also drain the accumulators and write G
// Block: (tile of 128 rows t, tile of 64 pairs).
#pragma once
#include "tc_pipe.cuh"

namespace s2g {

constexpr int QP_IMG_CHUNK = 2 * LT_PLANE;   // bytes of one (row tile, K chunk) image
static __global__ void __launch_bounds__(LT_THREADS, 1)
    k_quad_tcp(const unsigned char *__restrict__ Qimg, const float2 *__restrict__ F, float2 *__restrict__ G, int N,
               int nmi, int mi0, int nj, int npairs, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *smem = lt_align(smem_dyn);
    LtSync &sy = *reinterpret_cast<LtSync *>(smem + LT_NS * LT_STAGE);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * 128, pair0 = blockIdx.y * 64;
    const int nk = (N + 31) / 32;
    lt_setup(sy, warp, tid, 1 + LT_OPB_WARPS, LT_MMA_WARP);
    const uint32_t tmem = sy.tslot;

    if (warp < LT_REC_WARPS) {
        // ------------------------------------------------ operand A: one bulk copy per chunk
        if (tid == 0) {
            const unsigned char *img = Qimg + (size_t)blockIdx.x * nk * QP_IMG_CHUNK;
            for (int c = 0; c < nk; ++c) {
                const int s = c % LT_NS;
                if (c >= LT_NS) lt_wait(&sy.empty[s], ((c / LT_NS) - 1) & 1, &sy.abort);
                tc::mbar_arrive_expect_tx(&sy.full[s], QP_IMG_CHUNK);
                tc::bulk_g2s(smem + s * LT_STAGE, img + (size_t)c * QP_IMG_CHUNK, QP_IMG_CHUNK, &sy.full[s]);
            }
        }
    } else if (warp < LT_MMA_WARP) {
        // ------------------------------------------------ operand B (F) and drains
        const int u = tid - 32 * LT_REC_WARPS;
        LtDrain d;
        d.init(warp);
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
                const float2 *r = frow[p >= 32];
                return r ? r + k0 : nullptr;
            }, N - k0, nullptr);
        };
        int drained = 0;
        auto body = [&](int c, LtB &cur, LtB &next) {
            if (c >= nk) return;
            if (c + 1 < nk) load(next, c + 1);
            while (drained <= c - LT_NS) d.drain(sy, tmem, drained++);
            cur.store(smem + (c % LT_NS) * LT_STAGE + 2 * LT_PLANE, u);
            lt_warp_arrive(&sy.full[c % LT_NS], lane);
        };
        LtB b0, b1;
        if (nk > 0) load(b0, 0);
        for (int c = 0; c < nk; c += 2) {
            body(c, b0, b1);
            body(c + 1, b1, b0);
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

// Q (FP32, N x N) -> shared-memory images of operand A: for row tile rt and K
// chunk c, plane 0 holds the TF32 truncation hi of Q[128 rt + r][32 c + k] and
// plane 1 the TF32 truncation of the remainder, at byte sw128_off(r, k) of the
// plane; zeros outside N x N.  One thread per 16-byte piece (4 values of k).
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
    float hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = 32 * c + 4 * kg + q;
        const float x = (row < N && k < N) ? Q[(size_t)row * N + k] : 0.f;
        float rem, drop;
        tc::split_tf32(x, hi[q], rem);
        tc::split_tf32(rem, lo[q], drop);
    }
    unsigned char *base = img + tile * QP_IMG_CHUNK + tc::sw128_off(r, 4 * kg);
    *reinterpret_cast<float4 *>(base) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<float4 *>(base + LT_PLANE) = make_float4(lo[0], lo[1], lo[2], lo[3]);
}

__host__ __device__ inline size_t quad_image_bytes(int N)
{
    return (size_t)((N + 127) / 128) * ((N + 31) / 32) * QP_IMG_CHUNK;
}

}  // namespace s2g
