// Allocation-free inverse spherical harmonic transform (see
// s2let_sht_inverse_noalloc in include/s2let_gpu.h).
//
// Everything this entry point needs on the device -- its tables (FFT chirps and
// twiddles, Legendre seeds and recurrence coefficients) and its two work
// buffers -- lives in one file-scope __device__ array, so it never calls
// cudaMalloc or cudaFree.  The kernels are the same templates the plans use.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/s2let_gpu.h"
#include "fft.cuh"
#include "gemm_fp32.cuh"
#include "host_tables.h"
#include "legendre.cuh"

using namespace s2g;

namespace {

constexpr size_t kScratchBytes = S2LET_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch array.  In host code its name is only a stand-in for the symbol;
// its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Layout {
    size_t rect, F, Ft, chirp, bhat, bhat_g, tw, phase, ls, seed, ringf, coeff, ringd, coefd, sinth, mant, expo, total;
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(int N, int nm, int batch, int M)
{
    Layout o;
    size_t p = 0;
    auto take = [&](size_t bytes) {
        const size_t at = p;
        p = up256(p + bytes);
        return at;
    };
    const size_t nn = (size_t)N * N;
    o.rect = take((size_t)batch * nm * N * sizeof(float2));
    o.F = take((size_t)batch * nm * N * sizeof(float2));
    o.Ft = take((size_t)batch * nm * N * sizeof(float2));
    o.chirp = take((size_t)(2 * N - 1) * sizeof(float2));
    o.bhat = take((size_t)M * sizeof(float2));
    o.bhat_g = take((size_t)M * sizeof(float2));
    o.tw = take((size_t)M * sizeof(float2));
    o.phase = take((size_t)(2 * N - 1) * sizeof(float2));
    o.ls = take(nn * sizeof(int));
    o.seed = take(nn * sizeof(double2));
    o.ringf = take((size_t)N * sizeof(RingF));
    o.coeff = take(nn * sizeof(float4));
    o.ringd = take((size_t)N * sizeof(RingD));
    o.coefd = take(nn * sizeof(double2));
    o.sinth = take((size_t)N * sizeof(double));
    o.mant = take(nn * sizeof(double));
    o.expo = take(nn * sizeof(int));
    o.total = p;
    return o;
}

struct DevState {
    unsigned char *base = nullptr;   // device address of g_scratch on this device
    int L = 0, batch = 0, cplx = -1; // tables currently held
    int M = 0, logM = 0;
};
std::mutex g_mu;
DevState g_dev[kMaxDevices];

__global__ void k_unpack_na(const float2 *__restrict__ in, float2 *__restrict__ rect, int L, int cplx, int B)
{
    const int nm = cplx ? 2 * L - 1 : L;
    const size_t total = (size_t)B * nm * L;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int l = (int)(i % L);
    const int mi = (int)((i / L) % nm);
    const int b = (int)(i / ((size_t)L * nm));
    const int m = cplx ? mi - (L - 1) : mi;
    float2 v = make_float2(0.f, 0.f);
    if (l >= (m < 0 ? -m : m)) v = in[(size_t)b * L * L + (size_t)l * l + l + m];
    rect[i] = v;
}

template <typename T> int put(unsigned char *dst, const std::vector<T> &h)
{
    if (h.empty()) return S2LET_OK;
    return cudaMemcpy(dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess ? S2LET_OK
                                                                                                : S2LET_ERR_CUDA;
}

// Fill the tables for band-limit L into the scratch of the current device.
// Earlier calls may still have kernels in flight that read the old tables (on
// any stream, including a non-blocking one that the copies below would not
// wait for), so the whole device is drained first.
int setup(DevState &d, int L, int batch, int cplx)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return S2LET_ERR_CUDA;
    if (!d.base) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return S2LET_ERR_CUDA;
        d.base = static_cast<unsigned char *>(ptr);
    }
    s2h::Band h;
    s2h::build_band(L, h);
    const int nm = cplx ? 2 * L - 1 : L;
    const Layout o = layout(L, nm, batch, h.M);
    if (o.total > kScratchBytes) return S2LET_ERR_UNSUPPORTED;
    int e = S2LET_OK;
    std::vector<float2> c(h.chirp.size()), bh(h.bhat.size()), tw(h.tw.size()), ph(h.phase.size());
    for (size_t i = 0; i < c.size(); ++i) c[i] = make_float2((float)h.chirp[i].real(), (float)h.chirp[i].imag());
    for (size_t i = 0; i < bh.size(); ++i) bh[i] = make_float2((float)h.bhat[i].real(), (float)h.bhat[i].imag());
    // group-major copy for the fused middle FFT pass (groups of R = 2^fft_rbf)
    std::vector<float2> bg(bh.size());
    {
        const size_t R = (size_t)1 << fft_rbf<float2>(), ng = bh.size() / R;
        for (size_t j = 0; j < ng; ++j)
            for (size_t q = 0; q < R; ++q) bg[q * ng + j] = bh[R * j + q];
    }
    for (size_t i = 0; i < tw.size(); ++i) tw[i] = make_float2((float)h.tw[i].real(), (float)h.tw[i].imag());
    for (size_t i = 0; i < ph.size(); ++i) ph[i] = make_float2((float)h.phase[i].real(), (float)h.phase[i].imag());
    std::vector<RingD> rd(L);
    std::vector<RingF> rf(L);
    for (int t = 0; t < L; ++t) {
        rd[t].sgn = h.sgn[t];
        rd[t].y = h.y[t];
        rf[t].xh = h.xh[t];
        rf[t].xl = h.xl[t];
    }
    std::vector<double> a, ab;
    s2h::legendre_coefs(L, a, ab);
    std::vector<double2> cd(a.size());
    std::vector<float4> cf(a.size());
    for (size_t i = 0; i < a.size(); ++i) {
        cd[i] = make_double2(a[i], ab[i]);
        const float ah = (float)a[i], bhh = (float)ab[i];
        cf[i] = make_float4(ah, (float)(a[i] - (double)ah), bhh, (float)(ab[i] - (double)bhh));
    }
    unsigned char *b = d.base;
    if (!e) e = put(b + o.chirp, c);
    if (!e) e = put(b + o.bhat, bh);
    if (!e) e = put(b + o.bhat_g, bg);
    if (!e) e = put(b + o.tw, tw);
    if (!e) e = put(b + o.phase, ph);
    if (!e) e = put(b + o.ringd, rd);
    if (!e) e = put(b + o.ringf, rf);
    if (!e) e = put(b + o.coefd, cd);
    if (!e) e = put(b + o.coeff, cf);
    if (!e) e = put(b + o.sinth, h.sinth);
    if (e) return e;
    const size_t nn = (size_t)L * L;
    k_sectoral<<<(L + 127) / 128, 128>>>(L, (const double *)(b + o.sinth), (double *)(b + o.mant),
                                         (int *)(b + o.expo));
    k_seed_start<<<(unsigned)((nn + 127) / 128), 128>>>(L, (const double *)(b + o.mant), (const int *)(b + o.expo),
                                                         (const RingD *)(b + o.ringd), (const double2 *)(b + o.coefd),
                                                         L, (int *)(b + o.ls), (double2 *)(b + o.seed));
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return S2LET_ERR_CUDA;
    d.L = L;
    d.batch = batch;
    d.cplx = cplx;
    d.M = h.M;
    d.logM = h.logM;
    return S2LET_OK;
}

}  // namespace

extern "C" int s2let_sht_inverse_noalloc(int L, int batch, int flags, const void *flm, void *f, void *stream)
{
    if (L < 2 || L > S2LET_NOALLOC_MAX_L || batch < 1 || batch > S2LET_NOALLOC_MAX_BATCH || !flm || !f)
        return S2LET_ERR_ARG;
    if ((flags & S2LET_PREC_MASK) != S2LET_PREC_FP32) return S2LET_ERR_ARG;
    if (flags & ~(S2LET_COMPLEX | S2LET_PREC_MASK)) return S2LET_ERR_ARG;
    const int cplx = (flags & S2LET_COMPLEX) ? 1 : 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return S2LET_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;

    std::lock_guard<std::mutex> lock(g_mu);
    DevState &d = g_dev[dev];
    if (d.L != L || d.batch != batch || d.cplx != cplx) {
        // the set-up copies and synchronises, which a stream capture does not allow
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
            return S2LET_ERR_UNSUPPORTED;
        const int e = setup(d, L, batch, cplx);
        if (e) {
            d.L = 0;
            return e;
        }
    }
    const int nm = cplx ? 2 * L - 1 : L;
    const Layout o = layout(L, nm, batch, d.M);
    unsigned char *b = d.base;
    float2 *rect = (float2 *)(b + o.rect);
    float2 *F = (float2 *)(b + o.F);

    // coefficients -> [b][m][l] rectangle (entries l < |m| cleared)
    const size_t n = (size_t)batch * nm * L;
    k_unpack_na<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float2 *)flm, rect, L, cplx, batch);
    // Legendre sums over degrees
    LegTab<float> tab;
    tab.ls = (const int *)(b + o.ls);
    tab.seed = (const double2 *)(b + o.seed);
    tab.ring = (const RingF *)(b + o.ringf);
    tab.coef = (const float4 *)(b + o.coeff);
    tab.ldc = L;
    const int bt = cplx ? LegCols<true>::BT : LegCols<false>::BT;
    dim3 grid((L + LS_RT - 1) / LS_RT, L, (batch + bt - 1) / bt);
    if (cplx)
        k_leg_synth_gemm<true><<<grid, 256, 0, st>>>(rect, L, nullptr, 1.0f, F, L, batch, tab);
    else
        k_leg_synth_gemm<false><<<grid, 256, 0, st>>>(rect, L, nullptr, 1.0f, F, L, batch, tab);
    // ring DFTs, on ring-major spectra
    float2 *Ft = (float2 *)(b + o.Ft);
    k_transpose<float2><<<dim3((L + 31) / 32, (nm + 31) / 32, batch), dim3(32, 8), 0, st>>>(F, Ft, nm, L);
    FftTab<float2> T;
    T.chirp = (const float2 *)(b + o.chirp);
    T.bhat = (const float2 *)(b + o.bhat);
    T.bhat_g = (const float2 *)(b + o.bhat_g);
    T.what = nullptr;
    T.tw = (const float2 *)(b + o.tw);
    T.phase = (const float2 *)(b + o.phase);
    T.N = L;
    T.P = 2 * L - 1;
    T.M = d.M;
    T.logM = d.logM;
    const int th = std::max(32, std::min(FFT_MAX_THREADS, d.M / 16));
    const size_t sm = (size_t)padded_len(d.M) * sizeof(float2);
    if (cplx)
        k_ring_inv_cplx<float><<<dim3(L, batch), th, sm, st>>>(Ft, (float2 *)f, 1.0f, T);
    else
        k_ring_inv_real<float><<<dim3((L + 1) / 2, batch), th, sm, st>>>(Ft, (float *)f, 1.0f, T);
    return cudaGetLastError() == cudaSuccess ? S2LET_OK : S2LET_ERR_CUDA;
}
