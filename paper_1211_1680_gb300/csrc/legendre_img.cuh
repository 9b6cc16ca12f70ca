// Block structure of the Legendre tables of the split tensor-core plans (the
// values themselves, their FP16 hi/lo format and the contraction kernels that
// stream them are in legendre_h16.cuh).
//
// The values lambda_lm(theta_t) of band-limit N are cut into blocks of 32
// degrees x 32 rings (4 KB each in the FP16 hi/lo format): degree block i =
// degrees m + 32 i .. m + 32 i + 31 of order m, ring block k = rings 32 k ..
// 32 k + 31.  For order m and ring block k only the degree blocks i >= i0[m][k]
// are stored, the first holding a value >= 2^-SEED_EXP (the recurrence starts
// at l_s(m, t) on each ring; below it the values are left out as zero): in the
// analysis copy at block index off[m][k] + i - i0[m][k] (the degree blocks of a
// ring block adjacent), in the synthesis copy in ring-block order per degree
// block (legendre_h16.cuh, k_h16_fill); block 0 holds zeros and stands for
// every block not stored.  The analysis walks, per (order, degree tile of 128),
// the ring blocks with a stored block among its four degree blocks (adt lists
// these (m, tile) items); the synthesis walks, per (ring tile of 128, order),
// the degree blocks from the smallest i0 of its four ring blocks.
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
    // chunk lists of every item, built once per plan:
    //   ameta[adt item] = (first chunk, chunks, first entry of ack, 0), ablk[chunk] = the
    //   four blocks (degree blocks 4 tile .. 4 tile + 3 of ring block ack[chunk]);
    //   smeta[m * ceil(N / 128) + ring tile] = (first chunk, chunks, first degree block
    //   ibase, 0), sblk[chunk] = the four blocks (ring blocks 4 tile .. 4 tile + 3 of
    //   degree block ibase + chunk)
    const int4 *ameta, *ablk, *smeta, *sblk;
    const int *ack;                                 // each item's list starts at a multiple of 4
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

constexpr int LI_MAXK = 128;                        // ring chunks of the analysis list (N <= 4096)

}  // namespace s2g
