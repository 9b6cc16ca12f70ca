// Plan, dispatch and C ABI of the S2LET GPU library (see include/s2let_gpu.h).
//
// Data path of one forward transform at band-limit N (batch B):
//   S1 ring DFT      f[b][t][p]      -> F[b][m][t]     (fft.cuh)
//   S2 quadrature    F[b][m][t]      -> G[b][m][t]     (fft.cuh, FP64 by default)
//   S3 Legendre sum  G[b][m][t]      -> flm[b][m][l]   (legendre.cuh)
// and of one inverse transform:
//   S5 Legendre sum  flm[b][m][l]    -> F[b][m][t]
//   S6 ring DFT      F[b][m][t]      -> f[b][t][p]
// The kernel products of Eqs. wav2/wav4/waveletsynthesis are applied inside
// S3 (epilogue, with accumulation over scales) and S5 (coefficient staging).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/s2let_gpu.h"
#include "fft.cuh"
#include "fft_mr.cuh"
#include "gemm_fp32.cuh"
#include "tc_kernels.cuh"
#include "legendre_tc.cuh"
#include "legendre_img.cuh"
#include "legendre_h16.cuh"
#include "quad_tc.cuh"
#include "host_tables.h"
#include "legendre.cuh"

using namespace s2g;

namespace {

constexpr int kMaxL = 4096;
constexpr int kMaxM = 16384;  // FFT length for kMaxL (next power of two >= 4 kMaxL - 3)
constexpr int kMaxL64 = 2048; // FP64 plans: their shared-memory FFTs of length M hold 16 M bytes

int fft_threads(int M) { return std::max(32, std::min(FFT_MAX_THREADS, M / 16)); }

// Device memory of plans: cudaMalloc / cudaFree, or the caller's hook
// (s2let_set_allocator).  A plan keeps the hook it was created with.
struct DevAlloc {
    s2let_alloc_fn alloc = nullptr;
    s2let_free_fn release = nullptr;
    void *ctx = nullptr;
};
DevAlloc g_alloc;
std::mutex g_alloc_mu;

template <typename T> cudaError_t dm_alloc(const DevAlloc &a, T **p, size_t bytes)
{
    if (!a.alloc) return cudaMalloc(p, bytes);
    void *q = a.alloc(bytes, a.ctx);
    if (q && (reinterpret_cast<uintptr_t>(q) & 255)) {   // the kernels rely on cudaMalloc's alignment
        a.release(q, a.ctx);
        q = nullptr;
    }
    *p = static_cast<T *>(q);
    return q ? cudaSuccess : cudaErrorMemoryAllocation;
}
void dm_free(const DevAlloc &a, void *p)
{
    if (!p) return;
    if (a.release) a.release(p, a.ctx);
    else cudaFree(p);
}

template <typename K> void allow_smem_p(K kernel, size_t bytes)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
T *dev_upload(const DevAlloc &mem, const std::vector<T> &h, std::vector<void *> &owned, int &err)
{
    if (h.empty()) return nullptr;
    void *p = nullptr;
    if (dm_alloc(mem, &p, h.size() * sizeof(T)) != cudaSuccess) {
        err = S2LET_ERR_ALLOC;
        return nullptr;
    }
    owned.push_back(p);
    if (cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) err = S2LET_ERR_CUDA;
    return static_cast<T *>(p);
}

template <typename C> std::vector<C> to_c(const std::vector<s2h::cd> &v)
{
    std::vector<C> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        o[i].x = v[i].real();
        o[i].y = v[i].imag();
    }
    return o;
}

// Device tables for one band-limit.
struct BandDev {
    int N = 0, P = 0, M = 0, logM = 0;
    FftTab<double2> fd{};
    FftTab<float2> ff{};
    int *ls = nullptr;
    double2 *seed = nullptr;
    RingD *ringd = nullptr;
    RingF *ringf = nullptr;
    float *Qe = nullptr, *Qo = nullptr;     // FP32 plans: quadrature matrices, even / odd m
    float *Qe3 = nullptr, *Qo3 = nullptr;   // TF32X3 plans with three-part split: three TF32 planes
    unsigned char *Qei = nullptr, *Qoi = nullptr;   // TF32X3 plans: operand-A images of the two-part split
    // kernel choices (s2let_plan_autotune): tensor-core or CUDA-core kernels per
    // stage in TF32X3 plans, and the ring-DFT block size (0: M/16)
    bool tc_quad = true, tc_anal = true, tc_synth = true;
    int fft_th = 0;
    // FP32 / TF32X3 plans, P = 2N - 1 with a mixed-radix kernel (fft_mr.cuh): ring
    // DFTs of real maps on the P samples, and the theta quadrature in its FFT form
    // (mr_quad; else the dense product)
    bool has_mr = false, mr_quad = true;
    MrTab mr{};
    // TF32X3 plans: precomputed Legendre tables (legendre_img.cuh, legendre_h16.cuh) when they fit
    // the plan's budget, used by the tensor-core contractions (img_*; else the
    // recurrence kernels)
    bool has_img = false, img_anal = true, img_synth = true;
    LegImg img{};                           // block index; img.img = the analysis copy (rows = degrees)
    unsigned char *img_t = nullptr;         // the synthesis copy (rows = rings)
    int n_adt = 0;                          // analysis blocks (m, degree tile)
    size_t img_bytes = 0;
};

}  // namespace

struct s2let_plan {
    int L = 0, B = 0, J0 = 0, J = 0, flags = 0, batch = 0;
    bool cplx = false, multires = false, fp64 = true, quad64 = true;
    int n_scal = 0;
    std::vector<int> n_wav;                 // band-limit of scale J0 + i
    std::vector<int64_t> wav_off;           // element offsets in f_wav
    int64_t wav_elems = 0, scal_elems = 0;
    std::map<int, BandDev> bands;
    double2 *coefd = nullptr;               // [m][l] (a, a b), FP64
    float4 *coeff = nullptr;                // [m][l] float-float
    std::vector<void *> kfac;               // per map: scaling first, then scales J0..J (R[L])
    std::vector<double> noise_ratio;        // per map (same order): sqrt(sum_l |Psi_l0|^2), Eq. noisemodel
    int nsm = 0;                            // SMs of the plan's device
    void *F = nullptr, *flm = nullptr, *G = nullptr;   // workspace
    void *Ft = nullptr;                                // ring-major spectra of the ring DFTs
    float4 *anal_st = nullptr;                         // TF32X3, L > 2048: recurrence states of k_leg_anal_tc
    size_t img_budget = 0, img_used = 0;               // TF32X3: bytes allowed / held by Legendre tables
    float *csc = nullptr;                              // TF32X3: column scales of the table contractions [b][mi]
    float *csc2 = nullptr;                             // TF32X3: the second set's column scales (k_leg_h16s2)
    void *G2 = nullptr;                                // TF32X3 with tables: the second set's spectra
    bool quad_gemm = false;                 // FP32 plans: theta quadrature as a dense FP32 product
    bool tc = false;                        // TF32X3 plans: dense products on the tensor cores
    int tc_split = 2;                       // TF32 parts per operand in the tensor-core products
    int *d_err = nullptr;                   // device error word (bounded waits)
    std::vector<void *> owned;
    DevAlloc mem;                           // allocator of everything in `owned`
    // instrumentation
    struct Rec {
        int stage;
        cudaEvent_t a, b;
        double flops, bytes;
    };
    mutable bool prof = false;
    mutable std::vector<Rec> recs;
    mutable std::vector<cudaEvent_t> evpool;
    mutable size_t evnext = 0;
    mutable int64_t launches[S2LET_N_STAGES] = {0, 0, 0, 0, 0, 0};
    ~s2let_plan()
    {
        for (cudaEvent_t e : evpool) cudaEventDestroy(e);
        // cudaFree waits for the device; a hook's release may not, and kernels of
        // this plan may still be running
        if (mem.alloc) cudaDeviceSynchronize();
        for (void *q : owned) dm_free(mem, q);
    }
};

namespace {

int elem_size(const s2let_plan *p) { return p->fp64 ? 8 : 4; }
int nmi(const s2let_plan *p, int N) { return p->cplx ? 2 * N - 1 : N; }
int64_t map_elems(const s2let_plan *p, int N) { return (int64_t)N * (2 * N - 1) * (p->cplx ? 2 : 1); }

#define S2_LAUNCH_CHECK()                                      \
    do {                                                       \
        if (cudaGetLastError() != cudaSuccess) return S2LET_ERR_CUDA; \
    } while (0)

// Counts the kernel launches of one run of `stage` (nk kernels) and, when
// profiling, brackets the run with an event pair.
struct StageScope {
    const s2let_plan *p;
    cudaStream_t st;
    long slot = -1;
    StageScope(const s2let_plan *p_, int stage, cudaStream_t st_, double flops, double bytes, int nk = 1)
        : p(p_), st(st_)
    {
        p->launches[stage] += nk;
        if (p->prof && p->evnext + 2 <= p->evpool.size()) {
            s2let_plan::Rec r{stage, p->evpool[p->evnext], p->evpool[p->evnext + 1], flops, bytes};
            p->evnext += 2;
            slot = (long)p->recs.size();
            p->recs.push_back(r);
            cudaEventRecord(r.a, st);
        }
    }
    ~StageScope()
    {
        if (slot >= 0) cudaEventRecord(p->recs[slot].b, st);
    }
};

// Algorithmic work of one Legendre stage at band-limit N: 4 flops per
// (l, m, ring, map) product (real lambda times complex value); the recurrence
// that produces lambda is not counted here.
double legendre_flops(const s2let_plan *p, int N)
{
    const double pairs = p->cplx ? (double)N * N : 0.5 * (double)N * (N + 1);
    return 4.0 * pairs * N * p->batch;
}
double spectrum_bytes(const s2let_plan *p, int N) { return (double)p->batch * nmi(p, N) * N * 2 * elem_size(p); }
double map_bytes(const s2let_plan *p, int N) { return (double)p->batch * map_elems(p, N) * elem_size(p); }

template <typename R> const FftTab<cplx_t<R>> &fft_tab(const BandDev &b);
template <> const FftTab<double2> &fft_tab<double>(const BandDev &b) { return b.fd; }
template <> const FftTab<float2> &fft_tab<float>(const BandDev &b) { return b.ff; }

template <typename R> LegTab<R> leg_tab(const s2let_plan *p, const BandDev &b);
template <> LegTab<double> leg_tab<double>(const s2let_plan *p, const BandDev &b)
{
    LegTab<double> t;
    t.ls = b.ls;
    t.seed = b.seed;
    t.ring = b.ringd;
    t.coef = p->coefd;
    t.ldc = p->L;
    return t;
}
template <> LegTab<float> leg_tab<float>(const s2let_plan *p, const BandDev &b)
{
    LegTab<float> t;
    t.ls = b.ls;
    t.seed = b.seed;
    t.ring = b.ringf;
    t.coef = p->coeff;
    t.ldc = p->L;
    return t;
}

// ------------------------------------------------------------ mixed-radix kernels
// Launches KERNEL<P> for the P of the band (one of S2G_MR_LENGTHS).
#define S2G_MR_CASE(P_)                                                        \
    case P_:                                                                   \
        S2G_MR_LAUNCH(P_);                                                     \
        break;
#define S2G_MR_SWITCH(P) \
    switch (P) { S2G_MR_LENGTHS(S2G_MR_CASE) default: break; }

template <int P> void mr_set_smem()
{
    allow_smem_p(k_ring_fwd_real_mr<P>, mr_ring_smem<P>());
    allow_smem_p(k_ring_inv_real_mr<P>, mr_ring_smem<P>());
    allow_smem_p(k_quad_mr<P>, mr_quad_smem<P>());
}

// Position of X_k after the forward passes (mixed-radix digit reversal):
// pos(k) = (P / R1) (k mod R1) + pos'(k div R1) over the remaining radices.
int mr_pos(int k, int P, const MrFactors &f, int i)
{
    if (i >= f.n) return 0;
    const int R = f.r[i], M = P / R;
    return M * (k % R) + mr_pos(k / R, M, f, i + 1);
}

// Tables of fft_mr.cuh for band-limit N, in FP64 rounded to FP32.
int build_mr_tables(s2let_plan *p, int N, BandDev &bd)
{
    const int P = 2 * N - 1;
    const MrFactors f = mr_factors(P);
    std::vector<float2> tw(std::max(1, mr_tw_off(P, f.n))), shm(P), shp(P);
    std::vector<int> rev(P);
    for (int i = 0; i < f.n; ++i) {
        const int R = f.r[i], S = mr_sub(P, i), M = S / R, off = mr_tw_off(P, i);
        for (int s = 1; s < R; ++s)
            for (int j = 0; j < M; ++j) {
                double sn, cs;
                s2h::sincospi_rat(2 * (int64_t)j * s, S, &sn, &cs);   // 2 pi j s / S
                tw[off + (s - 1) * M + j] = make_float2((float)cs, (float)-sn);
            }
    }
    for (int k = 0; k < P; ++k) rev[k] = mr_pos(k, P, f, 0);
    for (int k = 0; k < P; ++k) {
        const int a = k < N ? k : k - P;
        double sn, cs;
        s2h::sincospi_rat(a, P, &sn, &cs);                        // a pi / P
        shm[rev[k]] = make_float2((float)cs, (float)-sn);
        shp[rev[k]] = make_float2((float)(cs / P), (float)(sn / P));
    }
    // weights on phi_u = pi u / P, u < 2P: v_u = (1/2) sum_{|c| <= P-1} w(c) e^{-i c phi_u}
    //   = 1 + sum_{c = 2, 4, .., P-1} 2 cos(c phi_u) / (1 - c^2) + (pi/2) sin(phi_u),
    // so that sum_u v_u g(phi_u) = P int_0^pi g(theta) sin(theta) dtheta for every
    // trigonometric polynomial g of degree <= P - 1 (the scale of the dense Q)
    std::vector<double> v(2 * P);
    for (int u = 0; u < 2 * P; ++u) {
        double s1, c1, s2, c2;
        s2h::sincospi_rat(u, P, &s1, &c1);                        // phi_u
        s2h::sincospi_rat(2 * (int64_t)u, P, &s2, &c2);           // 2 phi_u
        // e^{i c phi} by rotation with e^{2 i phi}; error grows like c eps
        double re = c2, im = s2, acc = 1.0;
        for (int c = 2; c <= P - 1; c += 2) {
            acc += 2.0 * re / (1.0 - (double)c * c);
            const double nr = re * c2 - im * s2, ni = re * s2 + im * c2;
            re = nr;
            im = ni;
        }
        v[u] = acc + 0.5 * M_PI * s1;
    }
    // The shifted-grid products keep only the even part of v (without the sin term),
    // which commutes with the reflection t -> P - 1 - t; the sin term reaches the
    // folded result only through the pole ring t = N - 1, by the two columns of
    // K^T diag(.) K at t = N - 1 below.  With K[u][t] = D(2u - 2t - 1),
    // D(s) = (1/P) sum_{|a| <= N-1} e^{i pi a s / P} = (-1)^((s-1)/2) / (P sin(pi s / 2P)), s odd:
    //   qd_t = sum_u K[u][t] v_even(u) K[u][N-1],  qa_t = 2 sum_u K[u][t] (pi/2) sin(phi_2u) K[u][N-1]
    std::vector<double> dk(2 * P + 2 * N);                    // D(s) at dk[s + 2N - 1], s odd
    for (int s = -(2 * N - 1); s < 2 * P; s += 2) {
        double sn, cs;
        s2h::sincospi_rat(s, 2 * P, &sn, &cs);
        dk[s + 2 * N - 1] = ((((s - 1) / 2) & 1) ? -1.0 : 1.0) / (P * sn);
    }
    auto Dk = [&](int s) { return dk[s + 2 * N - 1]; };
    std::vector<double> vs(P), va(P), kd(P);
    for (int u = 0; u < P; ++u) {
        double s1, c1;
        s2h::sincospi_rat(2 * u, P, &s1, &c1);
        va[u] = 0.5 * M_PI * s1;
        vs[u] = v[2 * u] - va[u];
        kd[u] = Dk(2 * u - P);
    }
    std::vector<float> ve(P), vfold(N), qd(N), qa(N);
    for (int t = 0; t < P; ++t) ve[t] = (float)(vs[t] / P);
    for (int t = 0; t < N; ++t) vfold[t] = (float)(t < N - 1 ? v[2 * t + 1] + v[2 * (P - 1 - t) + 1] : v[2 * t + 1]);
    for (int t = 0; t < N; ++t) {
        double sd = 0.0, sa = 0.0;
        for (int u = 0; u < P; ++u) {
            const double k = Dk(2 * u - 2 * t - 1) * kd[u];
            sd += k * vs[u];
            sa += k * va[u];
        }
        qd[t] = (float)sd;
        qa[t] = (float)(2.0 * sa);
    }
    int err = S2LET_OK;
    auto &o = p->owned;
    bd.mr.tw = dev_upload(p->mem, tw, o, err);
    bd.mr.rev = dev_upload(p->mem, rev, o, err);
    bd.mr.shm = dev_upload(p->mem, shm, o, err);
    bd.mr.shp = dev_upload(p->mem, shp, o, err);
    bd.mr.ve = dev_upload(p->mem, ve, o, err);
    bd.mr.vfold = dev_upload(p->mem, vfold, o, err);
    bd.mr.qd = dev_upload(p->mem, qd, o, err);
    bd.mr.qa = dev_upload(p->mem, qa, o, err);
    if (!err) bd.has_mr = true;
    return err;
}

// ------------------------------------------------------------ stage launchers
template <typename R>
int run_ring_fwd(const s2let_plan *p, const BandDev &bd, const void *f, void *F, double scale, cudaStream_t st)
{
    const auto &T = fft_tab<R>(bd);
    const size_t sm = (size_t)padded_len(bd.M) * sizeof(cplx_t<R>);
    const int th = bd.fft_th ? bd.fft_th : fft_threads(bd.M);
    if (std::is_same<R, float>::value && !p->cplx && bd.has_mr) {
        // samples -> order-major spectrum in one kernel
        StageScope sc(p, S2LET_STAGE_RING_FWD, st, 0.0, map_bytes(p, bd.N) + spectrum_bytes(p, bd.N), 1);
        const dim3 grid((bd.N + MR_RINGS - 1) / MR_RINGS, p->batch);
#define S2G_MR_LAUNCH(P_)                                                                                        \
    k_ring_fwd_real_mr<P_><<<grid, MR_THREADS, mr_ring_smem<P_>(), st>>>((const float *)f, (float2 *)F, (float)scale, \
                                                                         bd.mr)
        S2G_MR_SWITCH(bd.P)
#undef S2G_MR_LAUNCH
        S2_LAUNCH_CHECK();
        return S2LET_OK;
    }
    StageScope sc(p, S2LET_STAGE_RING_FWD, st, 0.0, map_bytes(p, bd.N) + spectrum_bytes(p, bd.N), 2);
    if (p->cplx) {
        k_ring_fwd_cplx<R><<<dim3(bd.N, p->batch), th, sm, st>>>((const cplx_t<R> *)f, (cplx_t<R> *)p->Ft, (R)scale,
                                                                  T);
    } else {
        k_ring_fwd_real<R><<<dim3((bd.N + 1) / 2, p->batch), th, sm, st>>>((const R *)f, (cplx_t<R> *)p->Ft,
                                                                           (R)scale, T);
    }
    // Ft[b][t][mi] -> F[b][mi][t]
    const int n = nmi(p, bd.N);
    k_transpose<cplx_t<R>><<<dim3((n + 31) / 32, (bd.N + 31) / 32, p->batch), dim3(32, 8), 0, st>>>(
        (const cplx_t<R> *)p->Ft, (cplx_t<R> *)F, bd.N, n);
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

template <typename R>
int run_ring_inv(const s2let_plan *p, const BandDev &bd, const void *F, void *f, double scale, cudaStream_t st)
{
    const auto &T = fft_tab<R>(bd);
    const size_t sm = (size_t)padded_len(bd.M) * sizeof(cplx_t<R>);
    const int th = bd.fft_th ? bd.fft_th : fft_threads(bd.M);
    if (std::is_same<R, float>::value && !p->cplx && bd.has_mr) {
        StageScope sc(p, S2LET_STAGE_RING_INV, st, 0.0, map_bytes(p, bd.N) + spectrum_bytes(p, bd.N), 1);
        const dim3 grid((bd.N + MR_RINGS - 1) / MR_RINGS, p->batch);
#define S2G_MR_LAUNCH(P_)                                                                                        \
    k_ring_inv_real_mr<P_><<<grid, MR_THREADS, mr_ring_smem<P_>(), st>>>((const float2 *)F, (float *)f, (float)scale, \
                                                                         bd.mr)
        S2G_MR_SWITCH(bd.P)
#undef S2G_MR_LAUNCH
        S2_LAUNCH_CHECK();
        return S2LET_OK;
    }
    StageScope sc(p, S2LET_STAGE_RING_INV, st, 0.0, map_bytes(p, bd.N) + spectrum_bytes(p, bd.N), 2);
    // F[b][mi][t] -> Ft[b][t][mi]
    const int n = nmi(p, bd.N);
    k_transpose<cplx_t<R>><<<dim3((bd.N + 31) / 32, (n + 31) / 32, p->batch), dim3(32, 8), 0, st>>>(
        (const cplx_t<R> *)F, (cplx_t<R> *)p->Ft, n, bd.N);
    if (p->cplx) {
        k_ring_inv_cplx<R><<<dim3(bd.N, p->batch), th, sm, st>>>((const cplx_t<R> *)p->Ft, (cplx_t<R> *)f, (R)scale,
                                                                  T);
    } else {
        k_ring_inv_real<R><<<dim3((bd.N + 1) / 2, p->batch), th, sm, st>>>((const cplx_t<R> *)p->Ft, (R *)f,
                                                                           (R)scale, T);
    }
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

// S2.  Returns the buffer that holds G: F itself (in-place FFT quadrature) or
// the plan's G buffer (dense-matrix quadrature of FP32 plans).
template <typename R>
void *run_theta_quad(const s2let_plan *p, const BandDev &bd, void *F, cudaStream_t st, int *err, void *Gout = nullptr)
{
    // Gout: where the dense-matrix quadrature writes G (default the plan's G buffer)
    void *const Gb = Gout ? Gout : p->G;
    const int n = nmi(p, bd.N);
    const int off = p->cplx ? bd.N - 1 : 0;
    *err = S2LET_OK;
    if (std::is_same<R, float>::value && p->quad_gemm) {
        // Dense products G = Q_sigma F, one per parity of m, over all orders, or
        // with the FFT form over |m| > MR_QUAD_DENSE_M only (see fft_mr.cuh)
        const bool fft = bd.has_mr && bd.mr_quad && bd.N - 1 > MR_QUAD_DENSE_M;
        const int mcut = fft ? MR_QUAD_DENSE_M : bd.N;
        const int lo = p->cplx ? std::max(0, bd.N - 1 - mcut) : 0;
        const int hi = p->cplx ? std::min(n - 1, bd.N - 1 + mcut) : std::min(n - 1, mcut);
        StageScope sc(p, S2LET_STAGE_THETA_QUAD, st, 0.0, 2.0 * spectrum_bytes(p, bd.N), (fft ? 1 : 0) + 2);
        for (int par = 0; par < 2; ++par) {
            // first row at or after lo whose order has parity par
            const int want = p->cplx ? (((bd.N - 1) & 1) ^ par) : par;
            const int mi0 = lo + ((want - lo) & 1);
            if (mi0 > hi) continue;
            const int nj = (hi - mi0) / 2 + 1;
            const int npairs = nj * p->batch;
            dim3 grid((bd.N + QG_BM - 1) / QG_BM, (npairs + QG_BN / 2 - 1) / (QG_BN / 2));
            if (p->tc && bd.tc_quad && p->tc_split == 2) {
                // F rows by bulk copies where every row starts on a 16-byte boundary
                const bool fraw = bd.N % 2 == 0 && (reinterpret_cast<uintptr_t>(F) & 15) == 0;
                (fraw ? k_quad_tcp<true> : k_quad_tcp<false>)<<<grid, LT_THREADS, quad_tc_smem(), st>>>(
                    par ? bd.Qoi : bd.Qei, (const float2 *)F, (float2 *)Gb, bd.N, n, mi0, nj, npairs, p->d_err);
            }
            else if (p->tc && bd.tc_quad)
                k_quad_tc<3, 2><<<grid, TQ_THREADS, TqShape<3, 2>::SMEM, st>>>(
                    par ? bd.Qo3 : bd.Qe3, (const float2 *)F, (float2 *)Gb, bd.N, n, mi0, nj, npairs, p->d_err);
            else
                k_quad_gemm<<<grid, 256, 0, st>>>(par ? bd.Qo : bd.Qe, (const float2 *)F, (float2 *)Gb, bd.N, n,
                                                  mi0, nj, npairs);
        }
        if (fft) {
            MrCols C;
            C.nmi = n;
            C.m_offset = off;
            if (p->cplx) {
                C.mstart = 0;
                C.seg0 = bd.N - 1 - mcut;
                C.gap = 2 * mcut + 1;
                C.K = 2 * C.seg0;
            } else {
                C.mstart = mcut + 1;
                C.K = n - mcut - 1;
                C.seg0 = C.K;
                C.gap = 0;
            }
            C.useg = (C.seg0 + 1) / 2;
            C.upm = C.useg + (C.K - C.seg0 + 1) / 2;
            C.nunits = C.upm * p->batch;
#define S2G_MR_LAUNCH(P_)                                                                                           \
    k_quad_mr<P_><<<(C.nunits + mr_quad_cpb<P_>() - 1) / mr_quad_cpb<P_>(), MR_THREADS, mr_quad_smem<P_>(), st>>>( \
        (const float2 *)F, (float2 *)Gb, C, bd.mr)
            S2G_MR_SWITCH(bd.P)
#undef S2G_MR_LAUNCH
        }
        if (cudaGetLastError() != cudaSuccess) *err = S2LET_ERR_CUDA;
        return Gb;
    }
    const int th = fft_threads(bd.M);
    StageScope sc(p, S2LET_STAGE_THETA_QUAD, st, 0.0, 2.0 * spectrum_bytes(p, bd.N));
    if (p->quad64) {
        const size_t sm = (size_t)padded_len(bd.M) * sizeof(double2);
        k_theta_quad<double, R, 16><<<dim3(n, p->batch), th, sm, st>>>((const cplx_t<R> *)F, (cplx_t<R> *)F, n, off,
                                                                       1.0, bd.fd, -1);
    } else {
        const size_t sm = (size_t)padded_len(bd.M) * sizeof(float2);
        k_theta_quad<float, R, 16><<<dim3(n, p->batch), th, sm, st>>>((const cplx_t<R> *)F, (cplx_t<R> *)F, n, off,
                                                                      1.0f, bd.ff, -1);
    }
    if (cudaGetLastError() != cudaSuccess) *err = S2LET_ERR_CUDA;
    return F;
}

template <typename R, int BT, bool CPLX>
void launch_synth(const s2let_plan *p, const BandDev &bd, const void *src, const void *kfac, double scale, void *dst,
                  cudaStream_t st)
{
    constexpr int TT = 128;
    dim3 grid(bd.N, (bd.N + TT - 1) / TT, (p->batch + BT - 1) / BT);
    k_leg_synth<R, BT, CPLX, TT><<<grid, TT, 0, st>>>((const cplx_t<R> *)src, p->L, nmi(p, p->L), p->L,
                                                      (const R *)kfac, (R)scale, (cplx_t<R> *)dst, bd.N, p->batch,
                                                      leg_tab<R>(p, bd));
}

// S5: dst (band-limit N rectangle) from the plan's L-rectangle src.
template <typename R>
int run_synth(const s2let_plan *p, const BandDev &bd, const void *src, const void *kfac, double scale, void *dst,
              cudaStream_t st)
{
    constexpr int BT = std::is_same<R, double>::value ? 4 : 8;
    StageScope sc(p, S2LET_STAGE_LEG_SYNTH, st, legendre_flops(p, bd.N), 0.0);
    if (std::is_same<R, float>::value) {
        const int bt = p->cplx ? LegCols<true>::BT : LegCols<false>::BT;
        dim3 grid((bd.N + LS_RT - 1) / LS_RT, bd.N, (p->batch + bt - 1) / bt);
        const LegTab<float> tab = leg_tab<float>(p, bd);
        if (p->tc && bd.tc_synth && bd.has_img && bd.img_synth) {
            const size_t rows = (size_t)p->batch * nmi(p, p->L);
            p->launches[S2LET_STAGE_LEG_SYNTH] += 1;           // the column scales
            k_h16_colscale<false><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
                (const float2 *)src, p->L, (const float *)kfac, bd.N, p->batch, p->cplx, p->csc);
            const LegH16Args a{(const float2 *)src, p->L, (const float *)kfac, (float)scale, 0, (float2 *)dst, 0,
                               bd.N, p->batch, bd.img, bd.img_t, p->csc, p->d_err};
            const dim3 g((bd.N + 127) / 128, bd.N, (p->batch + bt - 1) / bt);
            if (p->cplx) k_leg_h16<false, true><<<g, LH_THREADS, leg_h16_smem(), st>>>(a);
            else k_leg_h16<false, false><<<g, LH_THREADS, leg_h16_smem(), st>>>(a);
        } else if (p->tc && bd.tc_synth && p->cplx)
            k_leg_synth_tc<true><<<grid, LT_THREADS, ls_synth_smem(), st>>>(
                (const float2 *)src, p->L, (const float *)kfac, (float)scale, (float2 *)dst, bd.N, p->batch, tab,
                p->d_err);
        else if (p->tc && bd.tc_synth)
            k_leg_synth_tc<false><<<grid, LT_THREADS, ls_synth_smem(), st>>>(
                (const float2 *)src, p->L, (const float *)kfac, (float)scale, (float2 *)dst, bd.N, p->batch, tab,
                p->d_err);
        else if (p->cplx)
            k_leg_synth_gemm<true><<<grid, 256, 0, st>>>((const float2 *)src, p->L, (const float *)kfac, (float)scale,
                                                         (float2 *)dst, bd.N, p->batch, tab);
        else
            k_leg_synth_gemm<false><<<grid, 256, 0, st>>>((const float2 *)src, p->L, (const float *)kfac, (float)scale,
                                                          (float2 *)dst, bd.N, p->batch, tab);
    } else if (p->cplx) {
        launch_synth<R, BT, true>(p, bd, src, kfac, scale, dst, st);
    } else {
        launch_synth<R, BT, false>(p, bd, src, kfac, scale, dst, st);
    }
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

// S5 of two kernel sets that share the band-limit and f_lm: dst0, dst1 from the
// plan's L-rectangle src with factors kfac0, kfac1, one table stream (table
// kernels only: the caller checks synth2_ok).
bool synth2_ok(const s2let_plan *p, const BandDev &bd)
{
    return p->tc && p->G2 && p->csc2 && bd.tc_synth && bd.has_img && bd.img_synth;
}

int run_synth2(const s2let_plan *p, const BandDev &bd, const void *src, const void *kfac0, const void *kfac1,
               double scale, void *dst0, void *dst1, cudaStream_t st)
{
    StageScope sc(p, S2LET_STAGE_LEG_SYNTH, st, 2.0 * legendre_flops(p, bd.N), 0.0, 3);
    const size_t rows = (size_t)p->batch * nmi(p, p->L);
    k_h16_colscale<false><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>((const float2 *)src, p->L, (const float *)kfac0,
                                                                      bd.N, p->batch, p->cplx, p->csc);
    k_h16_colscale<false><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>((const float2 *)src, p->L, (const float *)kfac1,
                                                                      bd.N, p->batch, p->cplx, p->csc2);
    LegH16Args2 a{};
    a.src = (const float2 *)src;
    a.Lsrc = p->L;
    a.kfac[0] = (const float *)kfac0;
    a.kfac[1] = (const float *)kfac1;
    a.scale = (float)scale;
    a.dst[0] = (float2 *)dst0;
    a.dst[1] = (float2 *)dst1;
    a.N = bd.N;
    a.B = p->batch;
    a.T = bd.img;
    a.tab = bd.img_t;
    a.csc[0] = p->csc;
    a.csc[1] = p->csc2;
    a.err = p->d_err;
    const int bt = p->cplx ? LegCols<true>::BT : LegCols<false>::BT;
    const dim3 g((bd.N + 127) / 128, bd.N, (p->batch + bt - 1) / bt);
    if (p->cplx) k_leg_h16s2<true><<<g, LH_THREADS, leg_h16s2_smem(), st>>>(a);
    else k_leg_h16s2<false><<<g, LH_THREADS, leg_h16s2_smem(), st>>>(a);
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

// S3 of two maps at one band-limit into one set of coefficients: dst (+)=
// c^0 A(G0) + c^1 A(G1), one table stream (table kernels only: anal2_ok).
bool anal2_ok(const s2let_plan *p, const BandDev &bd)
{
    return p->tc && p->G2 && p->csc2 && p->quad_gemm && bd.tc_anal && bd.has_img && bd.img_anal;
}

int run_anal2(const s2let_plan *p, const BandDev &bd, const void *G0, const void *G1, const void *kfac0,
              const void *kfac1, double scale, int acc, void *dst, cudaStream_t st)
{
    StageScope sc(p, S2LET_STAGE_LEG_ANAL, st, 2.0 * legendre_flops(p, bd.N), 0.0, 3);
    const size_t rows = (size_t)p->batch * nmi(p, bd.N);
    k_h16_colscale<true><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>((const float2 *)G0, 0, nullptr, bd.N, p->batch,
                                                                     p->cplx, p->csc);
    k_h16_colscale<true><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>((const float2 *)G1, 0, nullptr, bd.N, p->batch,
                                                                     p->cplx, p->csc2);
    LegH16ArgsA2 a{};
    a.src[0] = (const float2 *)G0;
    a.src[1] = (const float2 *)G1;
    a.kfac[0] = (const float *)kfac0;
    a.kfac[1] = (const float *)kfac1;
    a.scale = (float)scale;
    a.accumulate = acc;
    a.dst = (float2 *)dst;
    a.Ldst = p->L;
    a.N = bd.N;
    a.B = p->batch;
    a.T = bd.img;
    a.tab = bd.img.img;
    a.csc[0] = p->csc;
    a.csc[1] = p->csc2;
    a.err = p->d_err;
    const int bt = p->cplx ? LegCols<true>::BT : LegCols<false>::BT;
    const dim3 g(bd.n_adt, (p->batch + bt - 1) / bt);
    if (p->cplx) k_leg_h16a2<true><<<g, LH_THREADS, leg_h16a2_smem(), st>>>(a);
    else k_leg_h16a2<false><<<g, LH_THREADS, leg_h16a2_smem(), st>>>(a);
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

size_t anal_gemm_smem(int N)
{
    return (size_t)(LA_LT * LA_RG + LA_RG * 128) * sizeof(float) + (size_t)N * (sizeof(float4) + sizeof(int));
}

template <typename R, int BT, bool CPLX, int RPT>
void launch_anal(const s2let_plan *p, const BandDev &bd, const void *G, const void *kfac, double scale, int acc,
                 void *dst, cudaStream_t st)
{
    constexpr int TPB = 256;
    constexpr int V = std::is_same<R, double>::value ? 32 : 64;
    dim3 grid(bd.N, (p->batch + BT - 1) / BT);
    k_leg_anal<R, BT, CPLX, RPT, TPB, V><<<grid, TPB, 0, st>>>((const cplx_t<R> *)G, bd.N, (const R *)kfac, (R)scale,
                                                            acc, (cplx_t<R> *)dst, p->L, nmi(p, p->L), p->L,
                                                            p->batch, leg_tab<R>(p, bd));
}

template <typename R, int BT, bool CPLX>
void launch_anal_rpt(const s2let_plan *p, const BandDev &bd, const void *G, const void *kfac, double scale, int acc,
                     void *dst, cudaStream_t st)
{
    if (bd.N <= 256) launch_anal<R, BT, CPLX, 1>(p, bd, G, kfac, scale, acc, dst, st);
    else if (bd.N <= 512) launch_anal<R, BT, CPLX, 2>(p, bd, G, kfac, scale, acc, dst, st);
    else if (bd.N <= 1024) launch_anal<R, BT, CPLX, 4>(p, bd, G, kfac, scale, acc, dst, st);
    else launch_anal<R, BT, CPLX, 8>(p, bd, G, kfac, scale, acc, dst, st);
}

// S3: dst (the plan's L-rectangle) from G at band-limit N.
template <typename R>
int run_anal(const s2let_plan *p, const BandDev &bd, const void *G, const void *kfac, double scale, int acc,
             void *dst, cudaStream_t st)
{
    constexpr int BT = std::is_same<R, double>::value ? 2 : 4;
    StageScope sc(p, S2LET_STAGE_LEG_ANAL, st, legendre_flops(p, bd.N), 0.0);
    if (std::is_same<R, float>::value) {
        const int bt = p->cplx ? LegCols<true>::BT : LegCols<false>::BT;
        dim3 grid(bd.N, (p->batch + bt - 1) / bt);
        const size_t sm = anal_gemm_smem(bd.N);
        const LegTab<float> tab = leg_tab<float>(p, bd);
        if (p->tc && bd.tc_anal && bd.has_img && bd.img_anal) {
            const size_t rows = (size_t)p->batch * nmi(p, bd.N);
            p->launches[S2LET_STAGE_LEG_ANAL] += 1;            // the column scales
            k_h16_colscale<true><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>((const float2 *)G, 0, nullptr, bd.N,
                                                                             p->batch, p->cplx, p->csc);
            const LegH16Args a{(const float2 *)G, 0, (const float *)kfac, (float)scale, acc, (float2 *)dst, p->L,
                               bd.N, p->batch, bd.img, bd.img.img, p->csc, p->d_err};
            const dim3 g(bd.n_adt, (p->batch + bt - 1) / bt);
            if (p->cplx) k_leg_h16<true, true><<<g, LH_THREADS, leg_h16_smem(), st>>>(a);
            else k_leg_h16<true, false><<<g, LH_THREADS, leg_h16_smem(), st>>>(a);
        } else if (p->tc && bd.tc_anal && p->cplx)
            k_leg_anal_tc<true><<<grid, LT_ANAL_THREADS, la_anal_smem(bd.N), st>>>(
                (const float2 *)G, bd.N, (const float *)kfac, (float)scale, acc, (float2 *)dst, p->L, p->batch, tab,
                p->d_err, p->anal_st);
        else if (p->tc && bd.tc_anal)
            k_leg_anal_tc<false><<<grid, LT_ANAL_THREADS, la_anal_smem(bd.N), st>>>(
                (const float2 *)G, bd.N, (const float *)kfac, (float)scale, acc, (float2 *)dst, p->L, p->batch, tab,
                p->d_err, p->anal_st);
        else if (p->cplx)
            k_leg_anal_gemm<true><<<grid, 256, sm, st>>>((const float2 *)G, bd.N, (const float *)kfac, (float)scale,
                                                         acc, (float2 *)dst, p->L, p->batch, tab);
        else
            k_leg_anal_gemm<false><<<grid, 256, sm, st>>>((const float2 *)G, bd.N, (const float *)kfac, (float)scale,
                                                          acc, (float2 *)dst, p->L, p->batch, tab);
    } else if (p->cplx) {
        launch_anal_rpt<R, BT, true>(p, bd, G, kfac, scale, acc, dst, st);
    } else {
        launch_anal_rpt<R, BT, false>(p, bd, G, kfac, scale, acc, dst, st);
    }
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

// ------------------------------------------------------------ pack / unpack f_lm
template <typename R>
__global__ void k_pack(const cplx_t<R> *__restrict__ rect, cplx_t<R> *__restrict__ out, int L, int cplx, int B)
{
    const size_t n = (size_t)L * L;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * B) return;
    const int b = (int)(i / n);
    const int idx = (int)(i % n);
    const int l = (int)sqrtf((float)idx);
    int ll = l;
    while ((ll + 1) * (ll + 1) <= idx) ++ll;
    while (ll * ll > idx) --ll;
    const int m = idx - ll * ll - ll;
    const int nm = cplx ? 2 * L - 1 : L;
    cplx_t<R> v;
    if (cplx) {
        v = rect[((size_t)b * nm + (m + L - 1)) * L + ll];
    } else if (m >= 0) {
        v = rect[((size_t)b * nm + m) * L + ll];
    } else {
        v = cconj(rect[((size_t)b * nm + (-m)) * L + ll]);
        if ((-m) & 1) {
            v.x = -v.x;
            v.y = -v.y;
        }
    }
    out[i] = v;
}

// out[i] += the packed value of k_pack (for gradients accumulated over scales)
template <typename R>
__global__ void k_pack_add(const cplx_t<R> *__restrict__ rect, cplx_t<R> *__restrict__ out, int L, int cplx, int B)
{
    const size_t n = (size_t)L * L;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * B) return;
    const int b = (int)(i / n);
    const int idx = (int)(i % n);
    int ll = (int)sqrtf((float)idx);
    while ((ll + 1) * (ll + 1) <= idx) ++ll;
    while (ll * ll > idx) --ll;
    const int m = idx - ll * ll - ll;
    const int nm = cplx ? 2 * L - 1 : L;
    cplx_t<R> v;
    if (cplx) {
        v = rect[((size_t)b * nm + (m + L - 1)) * L + ll];
    } else if (m >= 0) {
        v = rect[((size_t)b * nm + m) * L + ll];
    } else {
        v = cconj(rect[((size_t)b * nm + (-m)) * L + ll]);
        if ((-m) & 1) {
            v.x = -v.x;
            v.y = -v.y;
        }
    }
    out[i] = cadd(out[i], v);
}

template <typename R>
__global__ void k_unpack(const cplx_t<R> *__restrict__ in, cplx_t<R> *__restrict__ rect, int L, int cplx, int B)
{
    const int nm = cplx ? 2 * L - 1 : L;
    const size_t total = (size_t)B * nm * L;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int l = (int)(i % L);
    const int mi = (int)((i / L) % nm);
    const int b = (int)(i / ((size_t)L * nm));
    const int m = cplx ? mi - (L - 1) : mi;
    cplx_t<R> v = mk((R)0, (R)0);
    if (l >= (m < 0 ? -m : m)) v = in[(size_t)b * L * L + (size_t)l * l + l + m];
    rect[i] = v;
}

// ------------------------------------------------------------ transforms
template <typename R> int sht_fwd_to_rect(s2let_plan *p, const void *f, cudaStream_t st)
{
    const BandDev &bd = p->bands.at(p->L);
    int e;
    if ((e = run_ring_fwd<R>(p, bd, f, p->F, 1.0 / bd.P, st))) return e;
    void *G = run_theta_quad<R>(p, bd, p->F, st, &e);
    if (e) return e;
    return run_anal<R>(p, bd, G, nullptr, 2.0 * M_PI / bd.P, 0, p->flm, st);
}

template <typename R> int sht_forward_t(s2let_plan *p, const void *f, void *flm, cudaStream_t st)
{
    int e = sht_fwd_to_rect<R>(p, f, st);
    if (e) return e;
    const size_t n = (size_t)p->batch * p->L * p->L;
    StageScope sc(p, S2LET_STAGE_PACK, st, 0.0, 0.0);
    k_pack<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const cplx_t<R> *)p->flm, (cplx_t<R> *)flm, p->L,
                                                           p->cplx, p->batch);
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

template <typename R> int sht_inverse_t(s2let_plan *p, const void *flm, void *f, cudaStream_t st)
{
    const BandDev &bd = p->bands.at(p->L);
    const size_t n = (size_t)p->batch * nmi(p, p->L) * p->L;
    {
    StageScope sc(p, S2LET_STAGE_PACK, st, 0.0, 0.0);
    k_unpack<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const cplx_t<R> *)flm, (cplx_t<R> *)p->flm, p->L,
                                                             p->cplx, p->batch);
    }
    S2_LAUNCH_CHECK();
    int e;
    if ((e = run_synth<R>(p, bd, p->flm, nullptr, 1.0, p->F, st))) return e;
    return run_ring_inv<R>(p, bd, p->F, f, 1.0, st);
}

// Maps of a wavelet transform, in processing order: index into kfac, band-limit,
// pointer offset (elements) of the map block; scale J (band-limit L) first.
struct MapRef {
    int k;
    int N;
    int64_t off;
    bool scal;
};

std::vector<MapRef> map_order(const s2let_plan *p)
{
    std::vector<MapRef> v;
    const int ns = (int)p->n_wav.size();
    for (int i = ns - 1; i >= 0; --i) v.push_back({1 + i, p->n_wav[i], p->wav_off[i], false});
    v.push_back({0, p->n_scal, 0, true});
    return v;
}

// Scale k of the plan: 0 = scaling map, 1 + i = wavelet scale J0 + i.
MapRef map_ref(const s2let_plan *p, int k)
{
    if (k == 0) return {0, p->n_scal, 0, true};
    return {k, p->n_wav[k - 1], p->wav_off[k - 1], false};
}

template <typename R> int analysis_t(s2let_plan *p, const void *f, void *fw, void *fs, cudaStream_t st)
{
    int e = sht_fwd_to_rect<R>(p, f, st);
    if (e) return e;
    const int es = elem_size(p);
    const std::vector<MapRef> maps = map_order(p);
    for (size_t i = 0; i < maps.size(); ++i) {
        const MapRef &mr = maps[i];
        const BandDev &bd = p->bands.at(mr.N);
        char *out = mr.scal ? (char *)fs : (char *)fw + mr.off * es;
        if (std::is_same<R, float>::value && i + 1 < maps.size() && maps[i + 1].N == mr.N && synth2_ok(p, bd)) {
            // two maps at one band-limit: one table stream for both syntheses
            const MapRef &m2 = maps[i + 1];
            char *out2 = m2.scal ? (char *)fs : (char *)fw + m2.off * es;
            if ((e = run_synth2(p, bd, p->flm, p->kfac[mr.k], p->kfac[m2.k], 1.0, p->F, p->G2, st))) return e;
            if ((e = run_ring_inv<R>(p, bd, p->F, out, 1.0, st))) return e;
            if ((e = run_ring_inv<R>(p, bd, p->G2, out2, 1.0, st))) return e;
            ++i;
            continue;
        }
        if ((e = run_synth<R>(p, bd, p->flm, p->kfac[mr.k], 1.0, p->F, st))) return e;
        if ((e = run_ring_inv<R>(p, bd, p->F, out, 1.0, st))) return e;
    }
    return S2LET_OK;
}

template <typename R> int synthesis_t(s2let_plan *p, const void *fw, const void *fs, void *f, cudaStream_t st)
{
    const int es = elem_size(p);
    int e, first = 1;
    const std::vector<MapRef> maps = map_order(p);
    for (size_t i = 0; i < maps.size(); ++i) {
        const MapRef &mr = maps[i];
        const BandDev &bd = p->bands.at(mr.N);
        const char *in = mr.scal ? (const char *)fs : (const char *)fw + mr.off * es;
        if (std::is_same<R, float>::value && i + 1 < maps.size() && maps[i + 1].N == mr.N && anal2_ok(p, bd)) {
            // two maps at one band-limit: their spectra in G and G2, one table stream for both
            const MapRef &m2 = maps[i + 1];
            const char *in2 = m2.scal ? (const char *)fs : (const char *)fw + m2.off * es;
            if ((e = run_ring_fwd<R>(p, bd, in, p->F, 1.0 / bd.P, st))) return e;
            void *G = run_theta_quad<R>(p, bd, p->F, st, &e);
            if (e) return e;
            if ((e = run_ring_fwd<R>(p, bd, in2, p->F, 1.0 / bd.P, st))) return e;
            void *G2 = run_theta_quad<R>(p, bd, p->F, st, &e, p->G2);
            if (e) return e;
            if ((e = run_anal2(p, bd, G, G2, p->kfac[mr.k], p->kfac[m2.k], 2.0 * M_PI / bd.P, first ? 0 : 1, p->flm,
                               st)))
                return e;
            first = 0;
            ++i;
            continue;
        }
        if ((e = run_ring_fwd<R>(p, bd, in, p->F, 1.0 / bd.P, st))) return e;
        void *G = run_theta_quad<R>(p, bd, p->F, st, &e);
        if (e) return e;
        if ((e = run_anal<R>(p, bd, G, p->kfac[mr.k], 2.0 * M_PI / bd.P, first ? 0 : 1, p->flm, st))) return e;
        first = 0;
    }
    const BandDev &bl = p->bands.at(p->L);
    if ((e = run_synth<R>(p, bl, p->flm, nullptr, 1.0, p->F, st))) return e;
    return run_ring_inv<R>(p, bl, p->F, f, 1.0, st);
}

template <typename R> int adjoint_t(s2let_plan *p, const void *gw, const void *gs, void *gf, cudaStream_t st)
{
    const int es = elem_size(p);
    int e, first = 1;
    for (const MapRef &mr : map_order(p)) {
        const BandDev &bd = p->bands.at(mr.N);
        const char *in = mr.scal ? (const char *)gs : (const char *)gw + mr.off * es;
        // inverse-transform adjoint: unnormalised ring DFT, unweighted Legendre sum
        if ((e = run_ring_fwd<R>(p, bd, in, p->F, 1.0, st))) return e;
        if ((e = run_anal<R>(p, bd, p->F, p->kfac[mr.k], 1.0, first ? 0 : 1, p->flm, st))) return e;
        first = 0;
    }
    // forward-transform adjoint: Legendre sum (2 pi / P), quadrature (symmetric), ring DFT (1/P)
    const BandDev &bl = p->bands.at(p->L);
    if ((e = run_synth<R>(p, bl, p->flm, nullptr, 2.0 * M_PI / bl.P, p->F, st))) return e;
    void *G = run_theta_quad<R>(p, bl, p->F, st, &e);
    if (e) return e;
    return run_ring_inv<R>(p, bl, G, gf, 1.0 / bl.P, st);
}

// Pieces of the analysis for gradients with per-scale recomputation.
// The map of scale k (k = 0: scaling, k = 1 + j - J0: wavelet scale j) from
// harmonic coefficients in the public layout: W = Inv_{N_k}(c_k f_lm).
template <typename R> int wav_scale_t(s2let_plan *p, int k, const void *flm, void *w, cudaStream_t st)
{
    const MapRef mr = map_ref(p, k);
    const size_t n = (size_t)p->batch * nmi(p, p->L) * p->L;
    {
        StageScope sc(p, S2LET_STAGE_PACK, st, 0.0, 0.0);
        k_unpack<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const cplx_t<R> *)flm, (cplx_t<R> *)p->flm,
                                                                 p->L, p->cplx, p->batch);
    }
    S2_LAUNCH_CHECK();
    const BandDev &bd = p->bands.at(mr.N);
    int e;
    if ((e = run_synth<R>(p, bd, p->flm, p->kfac[mr.k], 1.0, p->F, st))) return e;
    return run_ring_inv<R>(p, bd, p->F, w, 1.0, st);
}

// glm (public layout) += c_k Inv_{N_k}^T(g): the transpose of wav_scale_t.
template <typename R> int wav_scale_adjoint_t(s2let_plan *p, int k, const void *g, void *glm, cudaStream_t st)
{
    const MapRef mr = map_ref(p, k);
    const BandDev &bd = p->bands.at(mr.N);
    const size_t rect = (size_t)p->batch * nmi(p, p->L) * p->L * 2 * elem_size(p);
    if (cudaMemsetAsync(p->flm, 0, rect, st) != cudaSuccess) return S2LET_ERR_CUDA;   // degrees >= N_k
    int e;
    if ((e = run_ring_fwd<R>(p, bd, g, p->F, 1.0, st))) return e;
    if ((e = run_anal<R>(p, bd, p->F, p->kfac[mr.k], 1.0, 0, p->flm, st))) return e;
    const size_t n = (size_t)p->batch * p->L * p->L;
    StageScope sc(p, S2LET_STAGE_PACK, st, 0.0, 0.0);
    k_pack_add<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const cplx_t<R> *)p->flm, (cplx_t<R> *)glm, p->L,
                                                               p->cplx, p->batch);
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

// gf = Fwd_L^T(glm): the transpose of the forward transform (the last part of adjoint_t).
template <typename R> int sht_forward_adjoint_t(s2let_plan *p, const void *glm, void *gf, cudaStream_t st)
{
    const size_t n = (size_t)p->batch * nmi(p, p->L) * p->L;
    {
        StageScope sc(p, S2LET_STAGE_PACK, st, 0.0, 0.0);
        k_unpack<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const cplx_t<R> *)glm, (cplx_t<R> *)p->flm,
                                                                 p->L, p->cplx, p->batch);
    }
    S2_LAUNCH_CHECK();
    const BandDev &bl = p->bands.at(p->L);
    int e;
    if ((e = run_synth<R>(p, bl, p->flm, nullptr, 2.0 * M_PI / bl.P, p->F, st))) return e;
    void *G = run_theta_quad<R>(p, bl, p->F, st, &e);
    if (e) return e;
    return run_ring_inv<R>(p, bl, G, gf, 1.0 / bl.P, st);
}

// ------------------------------------------------------------ plan construction
template <typename K> void allow_smem(K kernel, size_t bytes)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// FP32 kernels up to kMaxM, FP64 kernels (and the plan-time FP64 quadrature in
// shared memory) up to the FFT length of kMaxL64
void set_smem_limits(int Mmax)
{
    const size_t d = (size_t)padded_len(std::min(Mmax, kMaxM / 2)) * sizeof(double2),
                 f = (size_t)padded_len(Mmax) * sizeof(float2);
    allow_smem(k_ring_fwd_real<double>, d);
    allow_smem(k_ring_fwd_cplx<double>, d);
    allow_smem(k_ring_inv_real<double>, d);
    allow_smem(k_ring_inv_cplx<double>, d);
    allow_smem(k_ring_fwd_real<float>, f);
    allow_smem(k_ring_fwd_cplx<float>, f);
    allow_smem(k_ring_inv_real<float>, f);
    allow_smem(k_ring_inv_cplx<float>, f);
    allow_smem(k_quad_tcp<true>, quad_tc_smem());
    allow_smem(k_quad_tcp<false>, quad_tc_smem());
    allow_smem(k_quad_tc<3, 2>, TqShape<3, 2>::SMEM);
    allow_smem(k_leg_synth_tc<false>, ls_synth_smem());
    allow_smem(k_leg_synth_tc<true>, ls_synth_smem());
    allow_smem(k_leg_anal_tc<false>, la_anal_smem(LA_ST_SMEM_MAX));
    allow_smem(k_leg_anal_tc<true>, la_anal_smem(LA_ST_SMEM_MAX));
    allow_smem(k_leg_h16<true, false>, leg_h16_smem());
    allow_smem(k_leg_h16<true, true>, leg_h16_smem());
    allow_smem(k_leg_h16<false, false>, leg_h16_smem());
    allow_smem(k_leg_h16<false, true>, leg_h16_smem());
    allow_smem(k_leg_h16s2<false>, leg_h16s2_smem());
    allow_smem(k_leg_h16s2<true>, leg_h16s2_smem());
    allow_smem(k_leg_h16a2<false>, leg_h16a2_smem());
    allow_smem(k_leg_h16a2<true>, leg_h16a2_smem());
    allow_smem(k_leg_anal_gemm<false>, anal_gemm_smem(kMaxL));
    allow_smem(k_leg_anal_gemm<true>, anal_gemm_smem(kMaxL));
    allow_smem(k_theta_quad<double, double, 16>, d);
    allow_smem(k_theta_quad<double, float, 16>, d);
    allow_smem(k_theta_quad<float, float, 16>, f);
#define S2G_MR_SMEM(P_) mr_set_smem<P_>();
    S2G_MR_LENGTHS(S2G_MR_SMEM)
#undef S2G_MR_SMEM
}

__global__ void k_unit_rows(double2 *X, int N)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)N * N) return;
    const int r = (int)(i / N), c = (int)(i % N);
    X[i] = make_double2(r == c ? 1.0 : 0.0, 0.0);
}

__global__ void k_real_to_float(const double2 *X, float *Q, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) Q[i] = (float)X[i].x;
}

// Q_sigma (N x N, symmetric) by the FP64 theta quadrature applied to unit vectors:
// row i of the output is Q_sigma e_i.
int build_quad_matrices(s2let_plan *p, BandDev &bd)
{
    const int N = bd.N;
    const size_t nn = (size_t)N * N;
    double2 *X = nullptr;
    if (dm_alloc(p->mem, &X, nn * sizeof(double2)) != cudaSuccess) return S2LET_ERR_ALLOC;
    if (bd.M <= kMaxM / 2)   // above, the transform buffer is in global memory (no shared-memory attribute)
        cudaFuncSetAttribute(k_theta_quad<double, double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(padded_len(bd.M) * sizeof(double2)));
    int err = S2LET_OK;
    for (int par = 0; par < 2 && !err; ++par) {
        float *Q = nullptr;
        if (dm_alloc(p->mem, &Q, nn * sizeof(float)) != cudaSuccess) {
            err = S2LET_ERR_ALLOC;
            break;
        }
        p->owned.push_back(Q);
        (par ? bd.Qo : bd.Qe) = Q;
        k_unit_rows<<<(unsigned)((nn + 255) / 256), 256>>>(X, N);
        if (bd.M <= kMaxM / 2) {
            k_theta_quad<double, double, 16><<<dim3(N, 1), fft_threads(bd.M), padded_len(bd.M) * sizeof(double2)>>>(
                X, X, N, 0, 1.0, bd.fd, par);
        } else {
            // the FP64 transform buffer exceeds shared memory: global scratch for
            // QB columns at a time (fft_threads(M) = 512 threads, M / 512 <= 32 values each)
            constexpr int QB = 512;
            double2 *scratch = nullptr;
            if (dm_alloc(p->mem, &scratch, (size_t)QB * padded_len(bd.M) * sizeof(double2)) != cudaSuccess) {
                err = S2LET_ERR_ALLOC;
                break;
            }
            for (int c0 = 0; c0 < N; c0 += QB) {
                const int nb = std::min(QB, N - c0);
                k_theta_quad<double, double, 32><<<dim3(nb, 1), fft_threads(bd.M), 0>>>(
                    X + (size_t)c0 * N, X + (size_t)c0 * N, nb, 0, 1.0, bd.fd, par, scratch);
            }
            cudaDeviceSynchronize();
            dm_free(p->mem, scratch);
        }
        k_real_to_float<<<(unsigned)((nn + 255) / 256), 256>>>(X, Q, nn);
        if (p->tc && p->tc_split == 3) {
            float *Q3 = nullptr;
            if (dm_alloc(p->mem, &Q3, 3 * nn * sizeof(float)) != cudaSuccess) {
                err = S2LET_ERR_ALLOC;
                break;
            }
            p->owned.push_back(Q3);
            (par ? bd.Qo3 : bd.Qe3) = Q3;
            k_split3_planes<<<(unsigned)((nn + 255) / 256), 256>>>(Q, Q3, nn);
        } else if (p->tc) {
            unsigned char *img = nullptr;
            if (dm_alloc(p->mem, &img, quad_image_bytes(N)) != cudaSuccess) {
                err = S2LET_ERR_ALLOC;
                break;
            }
            p->owned.push_back(img);
            (par ? bd.Qoi : bd.Qei) = img;
            const size_t npieces = quad_image_bytes(N) / 16;
            k_quad_images<<<(unsigned)((npieces + 255) / 256), 256>>>(Q, img, N);
        }
        if (cudaGetLastError() != cudaSuccess) err = S2LET_ERR_CUDA;
    }
    // also on failure: kernels of the first parity may still read X
    if (cudaDeviceSynchronize() != cudaSuccess && !err) err = S2LET_ERR_CUDA;
    dm_free(p->mem, X);
    return err;
}

// v[R j + q] -> out[q (n / R) + j]: the order in which the fused middle FFT pass reads its table
std::vector<s2h::cd> group_major(const std::vector<s2h::cd> &v, int R)
{
    const size_t n = v.size(), ng = n / R;
    std::vector<s2h::cd> out(n);
    for (size_t j = 0; j < ng; ++j)
        for (int q = 0; q < R; ++q) out[(size_t)q * ng + j] = v[(size_t)R * j + q];
    return out;
}

// Legendre tables of band-limit N (TF32X3 plans), after the seeds: kept when
// they fit the plan's remaining budget, else the band uses the recurrence kernels.
int build_leg_img(s2let_plan *p, BandDev &bd)
{
    const int N = bd.N, nkr = (N + 31) / 32;
    const size_t nmk = (size_t)N * nkr;
    int *i0 = nullptr, *off_d = nullptr;
    int2 *adt_d = nullptr;
    unsigned char *img = nullptr;
    if (dm_alloc(p->mem, &i0, nmk * sizeof(int)) != cudaSuccess) return S2LET_ERR_ALLOC;
    k_img_i0<<<(unsigned)((nmk + 255) / 256), 256>>>(N, bd.ls, i0);
    std::vector<int> h(nmk), off(nmk);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(h.data(), i0, nmk * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        dm_free(p->mem, i0);
        return S2LET_ERR_CUDA;
    }
    int64_t nblk = 1;                                   // block 0: zeros
    for (int m = 0; m < N; ++m)
        for (int k = 0; k < nkr; ++k) {
            off[(size_t)m * nkr + k] = (int)std::min<int64_t>(nblk, INT32_MAX);
            nblk += li_nib(N, m) - h[(size_t)m * nkr + k];
        }
    // the synthesis copy: for each (m, degree block i), the ring blocks klo .. khi of
    // the blocks stored at i, adjacent (a gap, if the stored ring blocks of i were
    // not contiguous, holds zeros)
    std::vector<int> soff((size_t)N * nkr, 0), klo((size_t)N * nkr, 0);
    int64_t nblk_s = 1;                                 // block 0: zeros
    for (int m = 0; m < N; ++m)
        for (int i = 0; i < li_nib(N, m); ++i) {
            int lo = nkr, hi = -1;
            for (int k = 0; k < nkr; ++k)
                if (h[(size_t)m * nkr + k] <= i) {
                    lo = std::min(lo, k);
                    hi = k;
                }
            soff[(size_t)m * nkr + i] = (int)std::min<int64_t>(nblk_s, INT32_MAX);
            klo[(size_t)m * nkr + i] = lo;
            if (hi >= lo) nblk_s += hi - lo + 1;
        }
    // two copies of the blocks: rows = degrees (analysis), rows = rings (synthesis)
    const size_t bytes = ((size_t)nblk + (size_t)nblk_s) * LI_BLK;
    if (N > LH_MAXN || nblk > INT32_MAX || nblk_s > INT32_MAX || p->img_used + bytes > p->img_budget) {
        dm_free(p->mem, i0);
        return S2LET_OK;                                // no tables for this band-limit
    }
    std::vector<int2> adt;
    for (int m = 0; m < N; ++m)
        for (int dt = 0; dt < (N - m + 127) / 128; ++dt) adt.push_back(make_int2(m, dt));
    // the chunk list of every item: the four table blocks of each chunk and, for the
    // analysis, its ring block (each item's ring blocks start at a multiple of 4 entries)
    auto blk_of = [&](int m, int i, int k) -> int {
        if (k >= nkr || i >= li_nib(N, m)) return 0;
        const int b = h[(size_t)m * nkr + k];
        return i >= b ? off[(size_t)m * nkr + k] + (i - b) : 0;
    };
    std::vector<int4> ameta, ablk, smeta, sblk;
    std::vector<int> ack;
    for (const int2 &md : adt) {
        const int m = md.x, t4 = 4 * md.y;
        while (ack.size() % 4) ack.push_back(0);
        const int o = (int)ablk.size(), oc = (int)ack.size();
        for (int k = 0; k < nkr; ++k)
            if (h[(size_t)m * nkr + k] <= t4 + 3) {
                ack.push_back(k);
                ablk.push_back(make_int4(blk_of(m, t4, k), blk_of(m, t4 + 1, k), blk_of(m, t4 + 2, k),
                                         blk_of(m, t4 + 3, k)));
            }
        ameta.push_back(make_int4(o, (int)ablk.size() - o, oc, 0));
    }
    for (int q = 0; q < 4; ++q) ack.push_back(0);      // a list's copy rounds up to 4 entries
    const int nrt = (N + 127) / 128;
    for (int m = 0; m < N; ++m)
        for (int rt = 0; rt < nrt; ++rt) {
            const int nib = li_nib(N, m);
            int v = nib;
            for (int w = 0; w < 4; ++w)
                if (4 * rt + w < nkr) v = std::min(v, h[(size_t)m * nkr + 4 * rt + w]);
            const int o = (int)sblk.size();
            for (int i = v; i < nib; ++i) {
                int b[4];
                for (int w = 0; w < 4; ++w) {
                    const int k = 4 * rt + w;
                    const bool st = k < nkr && h[(size_t)m * nkr + k] <= i;
                    b[w] = st ? soff[(size_t)m * nkr + i] + k - klo[(size_t)m * nkr + i] : 0;
                }
                sblk.push_back(make_int4(b[0], b[1], b[2], b[3]));
            }
            smeta.push_back(make_int4(o, nib - v, v, 0));
        }
    if (dm_alloc(p->mem, &img, bytes) != cudaSuccess) {
        cudaGetLastError();
        dm_free(p->mem, i0);
        return S2LET_OK;                                // no room after all: the recurrence kernels
    }
    p->owned.push_back(i0);
    p->owned.push_back(img);
    int err = S2LET_OK;
    off_d = dev_upload(p->mem, off, p->owned, err);
    adt_d = dev_upload(p->mem, adt, p->owned, err);
    const int4 *ameta_d = dev_upload(p->mem, ameta, p->owned, err), *ablk_d = dev_upload(p->mem, ablk, p->owned, err);
    const int4 *smeta_d = dev_upload(p->mem, smeta, p->owned, err), *sblk_d = dev_upload(p->mem, sblk, p->owned, err);
    const int *ack_d = dev_upload(p->mem, ack, p->owned, err);
    const int *soff_d = dev_upload(p->mem, soff, p->owned, err), *klo_d = dev_upload(p->mem, klo, p->owned, err);
    if (err) return err;
    unsigned char *img_t = img + (size_t)nblk * LI_BLK;
    if (cudaMemset(img, 0, LI_BLK) != cudaSuccess || cudaMemset(img_t, 0, (size_t)nblk_s * LI_BLK) != cudaSuccess)
        return S2LET_ERR_CUDA;
    const size_t nthr = nmk * 32;
    k_h16_fill<<<(unsigned)((nthr + 127) / 128), 128>>>(N, bd.ls, bd.seed, bd.ringd, p->coefd, p->L, i0, off_d,
                                                        soff_d, klo_d, img, img_t);
    if (cudaGetLastError() != cudaSuccess) return S2LET_ERR_CUDA;
    bd.img = LegImg{img, i0, off_d, adt_d, nkr, ameta_d, ablk_d, smeta_d, sblk_d, ack_d};
    bd.img_t = img_t;
    bd.n_adt = (int)adt.size();
    bd.img_bytes = bytes;
    bd.has_img = true;
    p->img_used += bytes;
    return S2LET_OK;
}

int build_band_dev(s2let_plan *p, int N, BandDev &bd)
{
    s2h::Band h;
    s2h::build_band(N, h);
    int err = S2LET_OK;
    bd.N = h.N;
    bd.P = h.P;
    bd.M = h.M;
    bd.logM = h.logM;
    auto &o = p->owned;
    bd.fd.chirp = dev_upload(p->mem, to_c<double2>(h.chirp), o, err);
    bd.fd.bhat = dev_upload(p->mem, to_c<double2>(h.bhat), o, err);
    bd.fd.bhat_g = dev_upload(p->mem, to_c<double2>(group_major(h.bhat, 1 << fft_rbf<double2>())), o, err);
    bd.fd.what = dev_upload(p->mem, to_c<double2>(h.what), o, err);
    bd.fd.tw = dev_upload(p->mem, to_c<double2>(h.tw), o, err);
    bd.fd.phase = dev_upload(p->mem, to_c<double2>(h.phase), o, err);
    bd.ff.chirp = dev_upload(p->mem, to_c<float2>(h.chirp), o, err);
    bd.ff.bhat = dev_upload(p->mem, to_c<float2>(h.bhat), o, err);
    bd.ff.bhat_g = dev_upload(p->mem, to_c<float2>(group_major(h.bhat, 1 << fft_rbf<float2>())), o, err);
    bd.ff.what = dev_upload(p->mem, to_c<float2>(h.what), o, err);
    bd.ff.tw = dev_upload(p->mem, to_c<float2>(h.tw), o, err);
    bd.ff.phase = dev_upload(p->mem, to_c<float2>(h.phase), o, err);
    bd.fd.N = h.N;
    bd.fd.P = h.P;
    bd.fd.M = h.M;
    bd.fd.logM = h.logM;
    bd.ff.N = h.N;
    bd.ff.P = h.P;
    bd.ff.M = h.M;
    bd.ff.logM = h.logM;
    std::vector<RingD> rd(N);
    std::vector<RingF> rf(N);
    for (int t = 0; t < N; ++t) {
        rd[t].sgn = h.sgn[t];
        rd[t].y = h.y[t];
        rf[t].xh = h.xh[t];
        rf[t].xl = h.xl[t];
    }
    bd.ringd = dev_upload(p->mem, rd, o, err);
    bd.ringf = dev_upload(p->mem, rf, o, err);
    double *sinth = dev_upload(p->mem, h.sinth, o, err);
    if (err) return err;
    // seeds: sectoral values, then the first significant degree per (m, t)
    const size_t nn = (size_t)N * N;
    double *mant = nullptr;
    int *expo = nullptr;
    if (dm_alloc(p->mem, &mant, nn * sizeof(double)) != cudaSuccess) return S2LET_ERR_ALLOC;
    if (dm_alloc(p->mem, &expo, nn * sizeof(int)) != cudaSuccess) {
        dm_free(p->mem, mant);
        return S2LET_ERR_ALLOC;
    }
    void *ls = nullptr, *seed = nullptr;
    if (dm_alloc(p->mem, &ls, nn * sizeof(int)) != cudaSuccess || dm_alloc(p->mem, &seed, nn * sizeof(double2)) != cudaSuccess) {
        dm_free(p->mem, mant);
        dm_free(p->mem, expo);
        if (ls) dm_free(p->mem, ls);
        return S2LET_ERR_ALLOC;
    }
    o.push_back(ls);
    o.push_back(seed);
    bd.ls = (int *)ls;
    bd.seed = (double2 *)seed;
    if (!p->fp64 && mr_supported(bd.P)) {
        bd.mr_quad = !(p->flags & S2LET_QUAD_DENSE);
        if ((err = build_mr_tables(p, N, bd))) {
            dm_free(p->mem, mant);
            dm_free(p->mem, expo);
            return err;
        }
    }
    if (p->quad_gemm) {
        if ((err = build_quad_matrices(p, bd))) {
            dm_free(p->mem, mant);
            dm_free(p->mem, expo);
            return err;
        }
    }
    k_sectoral<<<(N + 127) / 128, 128>>>(N, sinth, mant, expo);
    k_seed_start<<<(unsigned)((nn + 127) / 128), 128>>>(N, mant, expo, bd.ringd, p->coefd, p->L, bd.ls, bd.seed);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    dm_free(p->mem, mant);
    dm_free(p->mem, expo);
    if (ce != cudaSuccess) return S2LET_ERR_CUDA;
    if (p->tc && p->img_budget > 0) {
        if ((err = build_leg_img(p, bd))) return err;
        if (cudaDeviceSynchronize() != cudaSuccess) return S2LET_ERR_CUDA;
    }
    return S2LET_OK;
}

int plan_create(s2let_plan **out, int L, int B, int J0, int flags, int batch)
{
    *out = nullptr;
    if (L < 3 || L > kMaxL || B < 2 || batch < 1) return S2LET_ERR_ARG;
    const int J = s2h::jmax(L, B);
    if (J0 < 0 || J0 >= J) return S2LET_ERR_ARG;
    const int prec = flags & S2LET_PREC_MASK;
    if (prec != S2LET_PREC_FP64 && prec != S2LET_PREC_FP32 && prec != S2LET_PREC_TF32X3) return S2LET_ERR_ARG;
    if (flags & ~(S2LET_COMPLEX | S2LET_MULTIRES | S2LET_PREC_MASK | S2LET_QUAD_FFT64 | S2LET_TC_SPLIT3 |
                  S2LET_KERNEL_BSPLINE | S2LET_QUAD_DENSE | S2LET_LEG_RECURRENCE))
        return S2LET_ERR_ARG;
    if ((flags & S2LET_TC_SPLIT3) && prec != S2LET_PREC_TF32X3) return S2LET_ERR_ARG;
    if ((flags & S2LET_LEG_RECURRENCE) && prec != S2LET_PREC_TF32X3) return S2LET_ERR_ARG;
    if ((flags & S2LET_QUAD_FFT64) && prec == S2LET_PREC_FP64) return S2LET_ERR_ARG;
    if (L > kMaxL64 && (prec == S2LET_PREC_FP64 || (flags & S2LET_QUAD_FFT64))) return S2LET_ERR_UNSUPPORTED;
    if ((flags & S2LET_QUAD_DENSE) && (prec == S2LET_PREC_FP64 || (flags & S2LET_QUAD_FFT64))) return S2LET_ERR_ARG;

    std::unique_ptr<s2let_plan> p(new (std::nothrow) s2let_plan());
    if (!p) return S2LET_ERR_ALLOC;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        p->mem = g_alloc;
    }
    p->L = L;
    p->B = B;
    p->J0 = J0;
    p->J = J;
    p->flags = flags;
    p->batch = batch;
    p->cplx = flags & S2LET_COMPLEX;
    p->multires = flags & S2LET_MULTIRES;
    p->fp64 = prec == S2LET_PREC_FP64;
    p->quad64 = true;
    p->tc = prec == S2LET_PREC_TF32X3;
    p->tc_split = (flags & S2LET_TC_SPLIT3) ? 3 : 2;
    p->quad_gemm = (prec == S2LET_PREC_FP32 || p->tc) && !(flags & S2LET_QUAD_FFT64);
    // band-limits (Sect. 3.1)
    const bool bspline = (flags & S2LET_KERNEL_BSPLINE) != 0;
    s2h::wav_bandlimits(L, B, J0, J, p->multires, bspline, &p->n_scal, p->n_wav);
    int64_t off = 0;
    for (int N : p->n_wav) {
        p->wav_off.push_back(off);
        off += map_elems(p.get(), N) * batch;
    }
    p->wav_elems = off;
    p->scal_elems = map_elems(p.get(), p->n_scal) * batch;

    int err = S2LET_OK;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return S2LET_ERR_CUDA;
    }
    if (p->tc && !(flags & S2LET_LEG_RECURRENCE)) {
        // Legendre tables: at most half the free device memory, and S2LET_LEG_TABLE_MAX_BYTES
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return S2LET_ERR_CUDA;
        p->img_budget = std::min<size_t>(fr / 2, (size_t)S2LET_LEG_TABLE_MAX_BYTES);
    }
    if (dm_alloc(p->mem, &p->d_err, sizeof(int)) != cudaSuccess) return S2LET_ERR_ALLOC;
    p->owned.push_back(p->d_err);
    if (cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) return S2LET_ERR_CUDA;
    // recurrence coefficients for degrees and orders < L
    std::vector<double> a, ab;
    s2h::legendre_coefs(L, a, ab);
    std::vector<double2> cd(a.size());
    std::vector<float4> cf(a.size());
    for (size_t i = 0; i < a.size(); ++i) {
        cd[i] = make_double2(a[i], ab[i]);
        const float ah = (float)a[i], bh = (float)ab[i];
        cf[i] = make_float4(ah, (float)(a[i] - (double)ah), bh, (float)(ab[i] - (double)bh));
    }
    p->coefd = dev_upload(p->mem, cd, p->owned, err);
    p->coeff = dev_upload(p->mem, cf, p->owned, err);
    if (err) return err;
    // kernel factors sqrt(4 pi/(2l+1)) Phi_l0 = eta(l / B^J0), sqrt(4 pi/(2l+1)) Psi^j_l0 = kappa(l / B^j)
    for (int k = 0; k <= J - J0 + 1; ++k) {
        std::vector<double> fac;
        s2h::wav_kernel(L, B, J0, J, bspline, k, fac);
        // white noise of unit harmonic variance has, in this map, the per-sample
        // variance sum_l |Psi_l0|^2 = sum_l (2l+1)/(4 pi) fac_l^2 (Eq. noisemodel)
        double v = 0.0;
        for (int l = 0; l < L; ++l) v += (2.0 * l + 1.0) / (4.0 * M_PI) * fac[l] * fac[l];
        p->noise_ratio.push_back(std::sqrt(v));
        if (p->fp64) {
            p->kfac.push_back(dev_upload(p->mem, fac, p->owned, err));
        } else {
            std::vector<float> ff(fac.begin(), fac.end());
            p->kfac.push_back(dev_upload(p->mem, ff, p->owned, err));
        }
        if (err) return err;
    }
    // per band-limit tables
    std::vector<int> Ns = p->n_wav;
    Ns.push_back(p->n_scal);
    Ns.push_back(L);
    std::sort(Ns.begin(), Ns.end());
    Ns.erase(std::unique(Ns.begin(), Ns.end()), Ns.end());
    int Mmax = 2;
    for (int N : Ns) {
        BandDev bd;
        if ((err = build_band_dev(p.get(), N, bd))) return err;
        Mmax = std::max(Mmax, bd.M);
        p->bands[N] = bd;
    }
    // kernel attributes are process-wide: set them for the largest supported
    // transform, so that a later, smaller plan cannot lower them under an earlier one
    (void)Mmax;
    set_smem_limits(kMaxM);
    // workspace: two L-rectangles of complex values per map
    const size_t ws = (size_t)batch * nmi(p.get(), L) * L * 2 * elem_size(p.get());
    if (dm_alloc(p->mem, &p->F, ws) != cudaSuccess) return S2LET_ERR_ALLOC;
    p->owned.push_back(p->F);
    if (dm_alloc(p->mem, &p->flm, ws) != cudaSuccess) return S2LET_ERR_ALLOC;
    p->owned.push_back(p->flm);
    if (dm_alloc(p->mem, &p->Ft, ws) != cudaSuccess) return S2LET_ERR_ALLOC;
    p->owned.push_back(p->Ft);
    if (p->quad_gemm) {
        if (dm_alloc(p->mem, &p->G, ws) != cudaSuccess) return S2LET_ERR_ALLOC;
        p->owned.push_back(p->G);
    }
    if (p->tc) {
        // column scales of the table contractions: one per (map, order row) of an L-rectangle
        if (dm_alloc(p->mem, &p->csc, (size_t)batch * nmi(p.get(), L) * sizeof(float)) != cudaSuccess)
            return S2LET_ERR_ALLOC;
        p->owned.push_back(p->csc);
        if (p->img_used > 0) {
            // two wavelet scales at one band-limit share one table stream (k_leg_h16s2)
            if (dm_alloc(p->mem, &p->csc2, (size_t)batch * nmi(p.get(), L) * sizeof(float)) != cudaSuccess)
                return S2LET_ERR_ALLOC;
            p->owned.push_back(p->csc2);
            if (dm_alloc(p->mem, &p->G2, ws) != cudaSuccess) return S2LET_ERR_ALLOC;
            p->owned.push_back(p->G2);
        }
    }
    if (p->tc && L > LA_ST_SMEM_MAX) {
        // one block per (order, batch tile) of the analysis at band-limit L, N float4 each
        const int bt = p->cplx ? LegCols<true>::BT : LegCols<false>::BT;
        const size_t nst = (size_t)L * ((batch + bt - 1) / bt) * L;
        if (dm_alloc(p->mem, &p->anal_st, nst * sizeof(float4)) != cudaSuccess) return S2LET_ERR_ALLOC;
        p->owned.push_back(p->anal_st);
    }
    if (cudaGetLastError() != cudaSuccess) return S2LET_ERR_CUDA;
    *out = p.release();
    return S2LET_OK;
}

}  // namespace

// ------------------------------------------------------------ C ABI
// ------------------------------------------------------------ autotuning
namespace {

// Median-free best-of timing of fn on the stream (ms); warm-up run first.
template <typename Fn> float time_best(cudaStream_t st, Fn fn, int reps = 3)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    fn();
    float best = 1e30f;
    for (int i = 0; i < reps; ++i) {
        cudaEventRecord(a, st);
        fn();
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

template <typename R> int autotune_t(s2let_plan *p, cudaStream_t st)
{
    // workspace as scratch operands: their contents do not change the timings
    const size_t ws = (size_t)p->batch * nmi(p, p->L) * p->L * 2 * elem_size(p);
    if (cudaMemsetAsync(p->F, 0, ws, st) != cudaSuccess || cudaMemsetAsync(p->flm, 0, ws, st) != cudaSuccess)
        return S2LET_ERR_CUDA;
    if (p->G && cudaMemsetAsync(p->G, 0, ws, st) != cudaSuccess) return S2LET_ERR_CUDA;
    const bool prof = p->prof;
    int64_t launches[S2LET_N_STAGES];
    std::copy(p->launches, p->launches + S2LET_N_STAGES, launches);
    p->prof = false;
    int e = S2LET_OK;
    for (auto &kv : p->bands) {
        BandDev &bd = kv.second;
        // ring DFTs: block of M/8, M/16, M/32 or M/64 threads (32 .. FFT_MAX_THREADS)
        std::vector<int> ths;
        for (int d : {8, 16, 32, 64}) {
            const int th = std::max(32, std::min(FFT_MAX_THREADS, bd.M / d));
            if (std::find(ths.begin(), ths.end(), th) == ths.end()) ths.push_back(th);
        }
        float best = 1e30f;
        int best_th = 0;
        for (int th : ths) {
            bd.fft_th = th;
            const float ms = time_best(st, [&] {
                run_ring_fwd<R>(p, bd, p->flm, p->F, 1.0, st);
                run_ring_inv<R>(p, bd, p->F, p->flm, 1.0, st);
            });
            if (ms < best) {
                best = ms;
                best_th = th;
            }
        }
        bd.fft_th = best_th;
        if (p->tc) {
            // each contraction stage: tensor-core kernel or CUDA-core GEMM kernel
            bd.mr_quad = false;
            bd.tc_quad = true;
            const float q1 = time_best(st, [&] { run_theta_quad<R>(p, bd, p->F, st, &e); });
            bd.tc_quad = false;
            const float q0 = time_best(st, [&] { run_theta_quad<R>(p, bd, p->F, st, &e); });
            bd.tc_quad = q1 <= q0;
            if (bd.has_mr && !(p->flags & S2LET_QUAD_DENSE)) {
                bd.mr_quad = true;
                const float q2 = time_best(st, [&] { run_theta_quad<R>(p, bd, p->F, st, &e); });
                bd.mr_quad = q2 <= std::min(q0, q1);
            }
            // Legendre stages: tensor-core kernel on the tables (where the plan holds
            // them), tensor-core kernel with the recurrence, CUDA-core kernel
            auto synth = [&] { run_synth<R>(p, bd, p->flm, nullptr, 1.0, p->F, st); };
            auto anal = [&] { run_anal<R>(p, bd, p->F, nullptr, 1.0, 0, p->flm, st); };
            bd.tc_synth = true;
            bd.img_synth = false;
            const float s1 = time_best(st, synth);
            float s2 = 1e30f;
            if (bd.has_img) {
                bd.img_synth = true;
                s2 = time_best(st, synth);
            }
            bd.tc_synth = false;
            const float s0 = time_best(st, synth);
            bd.tc_synth = std::min(s1, s2) <= s0;
            bd.img_synth = s2 <= s1;
            bd.tc_anal = true;
            bd.img_anal = false;
            const float a1 = time_best(st, anal);
            float a2 = 1e30f;
            if (bd.has_img) {
                bd.img_anal = true;
                a2 = time_best(st, anal);
            }
            bd.tc_anal = false;
            const float a0 = time_best(st, anal);
            bd.tc_anal = std::min(a1, a2) <= a0;
            bd.img_anal = a2 <= a1;
        }
        if (cudaGetLastError() != cudaSuccess) e = S2LET_ERR_CUDA;
        if (e) break;
    }
    p->prof = prof;
    std::copy(launches, launches + S2LET_N_STAGES, p->launches);
    if (!e && cudaStreamSynchronize(st) != cudaSuccess) e = S2LET_ERR_CUDA;
    return e;
}

}  // namespace

namespace {

// ---------------------------------------------------------------- hard thresholding (Sect. 4.3)
// The samples of scale s (R values of a real map, (re, im) pairs of a complex
// map) are [begin[s], begin[s+1]) of the wavelet buffer; each is set to zero
// where its modulus is below thr[s] (Eq. threshold).  Complex samples compare
// the squared modulus with thr^2, every product and the sum rounded on its own,
// so that the decision is the one the same-precision host arithmetic takes.
// Every thread walks all scales, a grid-stride pass per scale with U samples in
// flight, so no sample searches for its scale.
constexpr int kThrMaxScales = 32;
template <typename R> struct ThrTab {
    int n;
    int64_t begin[kThrMaxScales + 1];
    R thr[kThrMaxScales];
};
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

template <typename R, bool CPLX>
__global__ void __launch_bounds__(256) k_wav_threshold(R *__restrict__ w, ThrTab<R> tab)
{
    using C = cplx_t<R>;
    constexpr int U = 4;                          // samples in flight per thread
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int s = 0; s < tab.n; ++s) {
        const int64_t end = tab.begin[s + 1];
        const R t = tab.thr[s];
        const R t2 = mul_rn(t, t);
        for (int64_t i0 = tab.begin[s] + t0; i0 < end; i0 += U * stride) {
            C v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + u * stride;
                if (i < end) v[u] = CPLX ? reinterpret_cast<const C *>(w)[i] : C{w[i], R(0)};
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + u * stride;
                if (i >= end) continue;
                if (CPLX) {
                    if (add_rn(mul_rn(v[u].x, v[u].x), mul_rn(v[u].y, v[u].y)) < t2)
                        reinterpret_cast<C *>(w)[i] = C{R(0), R(0)};
                } else if (fabs(v[u].x) < t) {
                    w[i] = R(0);
                }
            }
        }
    }
}

template <typename R>
int run_threshold(const s2let_plan *p, void *f_wav, double sigma, double nsigma, cudaStream_t st)
{
    const int per = p->cplx ? 2 : 1;                 // R values per sample
    ThrTab<R> tab;
    tab.n = (int)p->n_wav.size();
    for (int s = 0; s < tab.n; ++s) {
        tab.begin[s] = p->wav_off[s] / per;
        tab.thr[s] = (R)(nsigma * sigma * p->noise_ratio[s + 1]);
    }
    tab.begin[tab.n] = p->wav_elems / per;
    const int64_t n = p->wav_elems / per;
    if (n == 0) return S2LET_OK;
    const int64_t want = (n + 256 * 4 - 1) / (256 * 4);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)p->nsm * 8));
    if (p->cplx)
        k_wav_threshold<R, true><<<blocks, 256, 0, st>>>((R *)f_wav, tab);
    else
        k_wav_threshold<R, false><<<blocks, 256, 0, st>>>((R *)f_wav, tab);
    S2_LAUNCH_CHECK();
    return S2LET_OK;
}

}  // namespace

// Failure-path check (s2let_plan_test_timeout): the two kinds of bounded wait
// of the tensor-core kernels, each on an mbarrier that nothing arrives at.
// Warp 0 waits with suspending try_wait polls (lt_wait), warp 1 with test_wait
// polls (lt_spin); whichever runs out first raises the shared abort flag, the
// other sees it and gives up too, and the error word is set as the tensor-core
// kernels set it.  No copy or MMA is issued, so nothing is in flight at exit.
__global__ void k_expire_waits(int *err)
{
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int *abort = &abort_flag;
    if (lane == 0) {
        // phase 0 of a fresh barrier never completes without an arrival
        if (warp == 0) lt_wait(&bar[0], 0, abort);
        else lt_spin(&bar[1], 0, abort);
    }
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) atomicExch(err, 1);
}

extern "C" {

int s2let_jmax(int L, int B)
{
    if (L < 2 || B < 2) return S2LET_ERR_ARG;
    return s2h::jmax(L, B);
}

int s2let_plan_create(s2let_plan **plan, int L, int B, int J_min, int flags, int batch)
{
    if (!plan) return S2LET_ERR_ARG;
    return plan_create(plan, L, B, J_min, flags, batch);
}

int s2let_plan_destroy(s2let_plan *plan)
{
    delete plan;
    return S2LET_OK;
}

int s2let_plan_info(const s2let_plan *p, int *J, int *n_scales, int64_t *wav_elems, int64_t *scal_elems, int *N_scal)
{
    if (!p) return S2LET_ERR_ARG;
    if (J) *J = p->J;
    if (n_scales) *n_scales = (int)p->n_wav.size();
    if (wav_elems) *wav_elems = p->wav_elems;
    if (scal_elems) *scal_elems = p->scal_elems;
    if (N_scal) *N_scal = p->n_scal;
    return S2LET_OK;
}

int s2let_wav_layout(const s2let_plan *p, int j, int *N_j, int64_t *offset, int64_t *elems)
{
    if (!p) return S2LET_ERR_ARG;
    if (j == -1) {
        if (N_j) *N_j = p->n_scal;
        if (offset) *offset = 0;
        if (elems) *elems = p->scal_elems;
        return S2LET_OK;
    }
    if (j < p->J0 || j > p->J) return S2LET_ERR_ARG;
    const int i = j - p->J0;
    if (N_j) *N_j = p->n_wav[i];
    if (offset) *offset = p->wav_off[i];
    if (elems) *elems = map_elems(p, p->n_wav[i]) * p->batch;
    return S2LET_OK;
}

#define S2_DISPATCH(fn, ...) (p->fp64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

int s2let_analysis(s2let_plan *p, const void *f, void *f_wav, void *f_scal, void *stream)
{
    if (!p || !f || !f_wav || !f_scal) return S2LET_ERR_ARG;
    return S2_DISPATCH(analysis_t, p, f, f_wav, f_scal, (cudaStream_t)stream);
}

int s2let_synthesis(s2let_plan *p, const void *f_wav, const void *f_scal, void *f, void *stream)
{
    if (!p || !f || !f_wav || !f_scal) return S2LET_ERR_ARG;
    return S2_DISPATCH(synthesis_t, p, f_wav, f_scal, f, (cudaStream_t)stream);
}

int s2let_adjoint(s2let_plan *p, const void *g_wav, const void *g_scal, void *g_f, void *stream)
{
    if (!p || !g_wav || !g_scal || !g_f) return S2LET_ERR_ARG;
    return S2_DISPATCH(adjoint_t, p, g_wav, g_scal, g_f, (cudaStream_t)stream);
}

static int scale_index(const s2let_plan *p, int j)
{
    if (j == -1) return 0;
    if (j < p->J0 || j > p->J) return -1;
    return 1 + j - p->J0;
}

int s2let_wav_scale(s2let_plan *p, int j, const void *flm, void *w, void *stream)
{
    if (!p || !flm || !w) return S2LET_ERR_ARG;
    const int k = scale_index(p, j);
    if (k < 0) return S2LET_ERR_ARG;
    return S2_DISPATCH(wav_scale_t, p, k, flm, w, (cudaStream_t)stream);
}

int s2let_wav_scale_adjoint(s2let_plan *p, int j, const void *g, void *glm, void *stream)
{
    if (!p || !g || !glm) return S2LET_ERR_ARG;
    const int k = scale_index(p, j);
    if (k < 0) return S2LET_ERR_ARG;
    return S2_DISPATCH(wav_scale_adjoint_t, p, k, g, glm, (cudaStream_t)stream);
}

int s2let_sht_forward_adjoint(s2let_plan *p, const void *glm, void *gf, void *stream)
{
    if (!p || !glm || !gf) return S2LET_ERR_ARG;
    return S2_DISPATCH(sht_forward_adjoint_t, p, glm, gf, (cudaStream_t)stream);
}

int s2let_sht_forward(s2let_plan *p, const void *f, void *flm, void *stream)
{
    if (!p || !f || !flm) return S2LET_ERR_ARG;
    return S2_DISPATCH(sht_forward_t, p, f, flm, (cudaStream_t)stream);
}

int s2let_sht_inverse(s2let_plan *p, const void *flm, void *f, void *stream)
{
    if (!p || !f || !flm) return S2LET_ERR_ARG;
    return S2_DISPATCH(sht_inverse_t, p, flm, f, (cudaStream_t)stream);
}


int s2let_plan_autotune(s2let_plan *p, void *stream)
{
    if (!p) return S2LET_ERR_ARG;
    return S2_DISPATCH(autotune_t, p, (cudaStream_t)stream);
}

int s2let_plan_leg_table_bytes(const s2let_plan *p, int N, size_t *bytes)
{
    if (!p || !bytes) return S2LET_ERR_ARG;
    if (N == 0) {
        *bytes = p->img_used;
        return S2LET_OK;
    }
    auto it = p->bands.find(N);
    if (it == p->bands.end()) return S2LET_ERR_ARG;
    *bytes = it->second.has_img ? it->second.img_bytes : 0;
    return S2LET_OK;
}

int s2let_plan_tuning(const s2let_plan *p, int N, int *tc_quad, int *tc_anal, int *tc_synth, int *fft_threads_out)
{
    if (!p) return S2LET_ERR_ARG;
    auto it = p->bands.find(N);
    if (it == p->bands.end()) return S2LET_ERR_ARG;
    const BandDev &bd = it->second;
    if (tc_quad)
        *tc_quad = (!p->fp64 && p->quad_gemm && bd.has_mr && bd.mr_quad && bd.N - 1 > MR_QUAD_DENSE_M)
                       ? 2
                       : (p->tc && bd.tc_quad);
    if (tc_anal) *tc_anal = (p->tc && bd.tc_anal) ? (bd.has_img && bd.img_anal ? 2 : 1) : 0;
    if (tc_synth) *tc_synth = (p->tc && bd.tc_synth) ? (bd.has_img && bd.img_synth ? 2 : 1) : 0;
    if (fft_threads_out) *fft_threads_out = bd.fft_th ? bd.fft_th : fft_threads(bd.M);
    return S2LET_OK;
}

int s2let_wav_bandlimits(int L, int B, int J_min, int flags, int *N_scal, int *N_wav, int n_wav_cap)
{
    if (L < 2 || B < 2 || (flags & ~(S2LET_COMPLEX | S2LET_MULTIRES | S2LET_PREC_MASK | S2LET_QUAD_FFT64 |
                                     S2LET_TC_SPLIT3 | S2LET_KERNEL_BSPLINE)))
        return S2LET_ERR_ARG;
    const int J = s2h::jmax(L, B);
    if (J_min < 0 || J_min >= J) return S2LET_ERR_ARG;
    const int ns = J - J_min + 1;
    if (N_wav && n_wav_cap < ns) return S2LET_ERR_ARG;
    int nsc = 0;
    std::vector<int> nw;
    s2h::wav_bandlimits(L, B, J_min, J, (flags & S2LET_MULTIRES) != 0, (flags & S2LET_KERNEL_BSPLINE) != 0, &nsc,
                        nw);
    if (N_scal) *N_scal = nsc;
    if (N_wav)
        for (int i = 0; i < ns; ++i) N_wav[i] = nw[i];
    return ns;
}

int s2let_wav_kernel(int L, int B, int J_min, int flags, int j, double *fac)
{
    if (L < 2 || L > (1 << 16) || B < 2 || !fac || (flags & ~(S2LET_COMPLEX | S2LET_MULTIRES | S2LET_PREC_MASK |
                                                             S2LET_QUAD_FFT64 | S2LET_TC_SPLIT3 |
                                                             S2LET_KERNEL_BSPLINE)))
        return S2LET_ERR_ARG;
    const int J = s2h::jmax(L, B);
    if (J_min < 0 || J_min >= J || (j != -1 && (j < J_min || j > J))) return S2LET_ERR_ARG;
    std::vector<double> f;
    s2h::wav_kernel(L, B, J_min, J, (flags & S2LET_KERNEL_BSPLINE) != 0, j == -1 ? 0 : j - J_min + 1, f);
    std::copy(f.begin(), f.end(), fac);
    return S2LET_OK;
}

int s2let_wav_noise_std(const s2let_plan *p, int j, double *ratio)
{
    if (!p || !ratio) return S2LET_ERR_ARG;
    if (j == -1) {
        *ratio = p->noise_ratio[0];
        return S2LET_OK;
    }
    if (j < p->J0 || j > p->J) return S2LET_ERR_ARG;
    *ratio = p->noise_ratio[j - p->J0 + 1];
    return S2LET_OK;
}

int s2let_wav_threshold(s2let_plan *p, void *f_wav, double sigma, double nsigma, void *stream)
{
    if (!p || !f_wav || !(sigma >= 0.0) || !(nsigma >= 0.0) || !std::isfinite(sigma * nsigma))
        return S2LET_ERR_ARG;
    if ((int)p->n_wav.size() > kThrMaxScales) return S2LET_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    return S2_DISPATCH(run_threshold, p, f_wav, sigma, nsigma, st);
}

int s2let_set_allocator(s2let_alloc_fn alloc, s2let_free_fn release, void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr)) return S2LET_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return S2LET_OK;
}

int s2let_plan_test_timeout(s2let_plan *p, void *stream)
{
    if (!p) return S2LET_ERR_ARG;
    k_expire_waits<<<1, 64, 0, (cudaStream_t)stream>>>(p->d_err);
    return cudaGetLastError() == cudaSuccess ? S2LET_OK : S2LET_ERR_CUDA;
}

int s2let_plan_status(s2let_plan *p)
{
    if (!p) return S2LET_ERR_ARG;
    int h = 0;
    if (cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return S2LET_ERR_CUDA;
    return h ? S2LET_ERR_TIMEOUT : S2LET_OK;
}

int s2let_plan_profile(s2let_plan *p, int enable)
{
    if (!p) return S2LET_ERR_ARG;
    if (enable) {
        const size_t want = 2 * 8192;
        while (p->evpool.size() < want) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return S2LET_ERR_CUDA;
            p->evpool.push_back(e);
        }
        p->recs.clear();
        p->evnext = 0;
        for (int i = 0; i < S2LET_N_STAGES; ++i) p->launches[i] = 0;
    }
    p->prof = enable != 0;
    return S2LET_OK;
}

int s2let_plan_stage_stats(s2let_plan *p, int stage, int64_t *launches, int64_t *timed, double *ms, double *flops,
                           double *bytes)
{
    if (!p || stage < 0 || stage >= S2LET_N_STAGES) return S2LET_ERR_ARG;
    double t = 0.0, f = 0.0, b = 0.0;
    int64_t n = 0;
    for (const auto &r : p->recs) {
        if (r.stage != stage) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return S2LET_ERR_CUDA;
        float x = 0.0f;
        if (cudaEventElapsedTime(&x, r.a, r.b) != cudaSuccess) return S2LET_ERR_CUDA;
        t += x;
        f += r.flops;
        b += r.bytes;
        ++n;
    }
    if (launches) *launches = p->launches[stage];
    if (timed) *timed = n;
    if (ms) *ms = t;
    if (flops) *flops = f;
    if (bytes) *bytes = b;
    return S2LET_OK;
}

const char *s2let_strerror(int s)
{
    switch (s) {
    case S2LET_OK: return "ok";
    case S2LET_ERR_ARG: return "invalid argument";
    case S2LET_ERR_ALLOC: return "allocation failed";
    case S2LET_ERR_CUDA: return "CUDA error";
    case S2LET_ERR_TIMEOUT: return "device wait timed out";
    case S2LET_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

}  // extern "C"
