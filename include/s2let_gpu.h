/*
 * s2let_gpu.h — C ABI of a GB300 (sm_103a) library for the axisymmetric
 * scale-discretised wavelet transform on the sphere with McEwen-Wiaux (MW)
 * equiangular sampling (Leistedt, McEwen, Vandergheynst & Wiaux, "S2LET: A
 * code to perform fast wavelet analysis on the sphere", A&A 2013).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Sampling (Sect. 2.1, MW sampling theorem): a map of band-limit N has N
 *   rings theta_t = pi (2t+1)/(2N-1), t = 0..N-1 (t = N-1 is the south pole),
 *   and P = 2N-1 longitudes phi_p = 2 pi p / P.  It is stored row-major as
 *   N x P samples; the pole ring is stored in full (P copies).
 * Batches: every buffer holds `batch` maps (or coefficient sets) back to back.
 * Element type: FP64 plans use double, other plans float.  Real maps hold one
 *   value per sample; complex maps (S2LET_COMPLEX) hold interleaved (re, im).
 * Harmonic coefficients (s2let_sht_*): complex interleaved, index l*l + l + m,
 *   l < L, |m| <= l, L*L per map.  Real plans return the m < 0 half from the
 *   symmetry f_{l,-m} = (-1)^m conj(f_lm) and read only m >= 0.
 * Wavelet maps: `f_wav` is the concatenation over scales j = J_min..J of one
 *   block per scale, each block `batch` maps at that scale's band-limit N_j
 *   (s2let_wav_layout gives offsets); `f_scal` holds `batch` scaling maps.
 *   Multiresolution (S2LET_MULTIRES, Sect. 3.1): N_j = min(L, B^(j+1)) and the
 *   scaling band-limit is min(L, B^J_min); otherwise every map is at L.
 * Memory: every data pointer is a DEVICE pointer owned by the caller; the
 *   library never frees it.  The plan owns its tables and its workspace, which
 *   are allocated in s2let_plan_create; transform calls allocate nothing.
 * Streams: calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *   default stream).  Calls on one plan share its workspace and must not run
 *   concurrently; distinct plans are independent.
 * Errors: every function returns an int status.  Argument errors are detected
 *   on the host before anything is launched.  Launch failures return
 *   S2LET_ERR_CUDA.  The library never traps, asserts or exits on the device.
 */
#ifndef S2LET_GPU_H
#define S2LET_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define S2LET_OK 0
#define S2LET_ERR_ARG (-1)         /* invalid argument (size, flag, pointer)      */
#define S2LET_ERR_ALLOC (-2)       /* device or host allocation failed            */
#define S2LET_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define S2LET_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up          */
#define S2LET_ERR_UNSUPPORTED (-5) /* valid request the library does not support   */

/* plan flags (bitwise or) */
#define S2LET_REAL 0x0           /* real maps (default)                        */
#define S2LET_COMPLEX 0x1        /* complex maps                               */
#define S2LET_MULTIRES 0x2       /* multiresolution band-limits, Sect. 3.1     */
#define S2LET_PREC_FP64 0x00     /* every stage in FP64                        */
#define S2LET_PREC_FP32 0x10     /* FP32 storage and sums, float-float Legendre
                                    recurrence, FP64 seeds; theta quadrature as a
                                    dense FP32 product with its matrix built in
                                    FP64                                       */
#define S2LET_PREC_TF32X3 0x20   /* as FP32, with the dense quadrature product and
                                    the Legendre contractions on the tensor cores
                                    (tcgen05): operands split in hi + lo parts, 3
                                    MMAs per product, TMEM partial sums over at
                                    most 128 K values added in FP32; the parts
                                    are TF32 in the quadrature and the
                                    recurrence kernels, FP16 (with exact power-
                                    of-two scales) on the Legendre tables      */
#define S2LET_PREC_MASK 0xf0
#define S2LET_QUAD_FFT64 0x100   /* FP32 plans only: theta quadrature by FP64 FFTs
                                    instead of the dense FP32 product          */
#define S2LET_TC_SPLIT3 0x200    /* TF32X3 plans only: split operands in three
                                    TF32 parts (6 MMAs per product) instead of
                                    two (3 MMAs)                               */
#define S2LET_QUAD_DENSE 0x800   /* FP32 / TF32X3 plans: the dense quadrature
                                    product at every band-limit, also where the
                                    FFT form (mixed-radix ring length) exists  */
#define S2LET_LEG_RECURRENCE 0x1000 /* TF32X3 plans only: no Legendre tables;
                                    every Legendre contraction runs the float-
                                    float recurrence (see s2let_plan_create) */
#define S2LET_KERNEL_BSPLINE 0x400 /* B-spline generating functions (footnote of
                                    Sect. 2.2) instead of the smooth scale-
                                    discretised ones: k(t) = 3/2 B_3(2 t B^(J-1)
                                    / L), wavelet j the square root of
                                    k(l/B^(j+1)) - k(l/B^j), the finest scale J
                                    sqrt(1 - k(l/B^J)) (so that the tiling is
                                    admissible), scaling sqrt(k(l/B^J_min)).
                                    Multiresolution band-limits (Sect. 3.1):
                                    min(L, ceil(L / B^(J-j-2))) for scale j and
                                    min(L, ceil(L / B^(J-J_min-1))) for the
                                    scaling map                                */

typedef struct s2let_plan s2let_plan;

/* J = ceil(log_B(L-1)), the largest wavelet scale (Sect. 2.2), computed in
 * integers as the smallest J >= 0 with B^J >= L-1.  Returns J, or
 * S2LET_ERR_ARG if L < 2 or B < 2. */
int s2let_jmax(int L, int B);

/* Create a plan for `batch` maps of band-limit L with dilation B (the paper's
 * lambda, an integer >= 2 here) and lowest wavelet scale J_min, 0 <= J_min < J
 * (Sect. 2.2).  Builds the kernel tables Phi_l0, Psi^j_l0 (Sect. 2.2), the
 * Legendre seeds and the FFT tables on the current device and allocates the
 * workspace.  Limits: 3 <= L <= 4096, 1 <= batch (else S2LET_ERR_ARG); FP64
 * plans and S2LET_QUAD_FFT64 only up to L = 2048 (their shared-memory FFTs of
 * length M >= 4L - 3 would exceed the SM's shared memory; S2LET_ERR_UNSUPPORTED).
 * The MW sampling theorem is stable to such band-limits (Sect. 2.1).
 * TF32X3 plans without S2LET_LEG_RECURRENCE also store the associated Legendre
 * values lambda_lm(theta_t) of each band-limit N <= 2048 (the FP64 recurrence
 * from the FP64 seeds, scaled by 2^9 and split into FP16 hi + lo; about N^3 / 2
 * values less those below 2^-100, 4 bytes each, in two copies: one laid out for
 * the analysis, one for the synthesis), so that the Legendre stages stream them
 * instead of recomputing them for every batch.  Band-limits are stored from the
 * smallest up while the total stays within S2LET_LEG_TABLE_MAX_BYTES and half
 * the device memory free at creation; the others use the recurrence.  Such
 * plans also hold a second spectrum rectangle, so that two maps of a wavelet
 * transform at one band-limit share a table stream.  s2let_plan_leg_table_bytes
 * reports the sizes.  On error *plan is NULL. */
#define S2LET_LEG_TABLE_MAX_BYTES (64ull << 30)
int s2let_plan_create(s2let_plan **plan, int L, int B, int J_min, int flags, int batch);

/* Free a plan and everything it owns (NULL is accepted). */
int s2let_plan_destroy(s2let_plan *plan);

/* Plan geometry: J, the number of wavelet scales J-J_min+1, the element
 * count of f_wav and f_scal (per batch, in real numbers: complex maps count
 * 2 per sample) and the band-limit of the scaling map.  Any output pointer
 * may be NULL. */
int s2let_plan_info(const s2let_plan *plan, int *J, int *n_scales, int64_t *wav_elems,
                    int64_t *scal_elems, int *N_scal);

/* Layout of scale j (J_min <= j <= J) inside f_wav: its band-limit N_j, the
 * offset of its block and the block size, both in real numbers (elements of
 * the plan's type).  j = -1 describes f_scal (offset 0). */
int s2let_wav_layout(const s2let_plan *plan, int j, int *N_j, int64_t *offset, int64_t *elems);

/* Wavelet analysis (Eqs. wav2 and wav4, Sect. 2.2; multiresolution of
 * Sect. 3.1): forward MW transform of each map f at L, products with
 * Psi^j_l0 and Phi_l0 in harmonic space, inverse transform of each scale at
 * its band-limit.  In: f (batch maps at L).  Out: f_wav, f_scal. */
int s2let_analysis(s2let_plan *plan, const void *f, void *f_wav, void *f_scal, void *stream);

/* Wavelet synthesis (Eq. waveletsynthesis, Sect. 2.2): forward transform of
 * every wavelet and scaling map at its band-limit, harmonic-space sum with
 * Psi^j_l0 and Phi_l0, inverse transform at L.  In: f_wav, f_scal.  Out: f.
 * Exact inverse of s2let_analysis for band-limited maps (Eq. identity). */
int s2let_synthesis(s2let_plan *plan, const void *f_wav, const void *f_scal, void *f, void *stream);

/* Adjoint of s2let_analysis: the transpose of the analysis operator under the
 * Euclidean inner product of the stored samples (pole copies counted), i.e.
 * the conjugate transpose for complex maps.  The paper does not state it; it
 * is the transpose of Eqs. wav2/wav4 and of each transform step.  Used for
 * gradients.  In: g_wav, g_scal (shaped like f_wav, f_scal).  Out: g_f. */
int s2let_adjoint(s2let_plan *plan, const void *g_wav, const void *g_scal, void *g_f, void *stream);

/* Forward MW spherical harmonic transform at L (Eq. harmonicsanalysis made a
 * finite sum by the sampling theorem of Sect. 2.1).  In: f.  Out: flm. */
int s2let_sht_forward(s2let_plan *plan, const void *f, void *flm, void *stream);

/* Inverse MW spherical harmonic transform at L (Eq. harmonicssynthesis,
 * Sect. 2.1).  In: flm.  Out: f. */
int s2let_sht_inverse(s2let_plan *plan, const void *flm, void *f, void *stream);

/* ---- batches of maps of uneven band-limit and dilation ------------------
 * (no counterpart in the paper: its transforms take one map at a time)
 * A batch groups its maps by (L, B) into plans (same J_min and flags for all).
 * The buffers f, f_wav, f_scal, f_out of a batch are the concatenation of the
 * groups' buffers, group by group; s2let_batch_map_layout tells where map i
 * (in the caller's order) lives.  Limits as for s2let_plan_create. */
typedef struct s2let_batch s2let_batch;

int s2let_batch_create(s2let_batch **batch, int n_maps, const int *L, const int *B, int J_min, int flags);
int s2let_batch_destroy(s2let_batch *batch);

/* Total element counts (in real numbers of the plans' type) of f (= f_out),
 * f_wav and f_scal, and the number of (L, B) groups.  Outputs may be NULL. */
int s2let_batch_sizes(const s2let_batch *batch, int64_t *f_elems, int64_t *wav_elems, int64_t *scal_elems,
                      int *n_groups);

/* Where map i lives: element offsets of its samples in f, of its scaling map in
 * f_scal, its group index and its index inside the group; inside f_wav a
 * group's block holds, scale by scale, `group size` maps (see
 * s2let_wav_layout of the group's plan, returned by s2let_batch_group_plan). */
int s2let_batch_map_layout(const s2let_batch *batch, int i, int64_t *f_off, int64_t *scal_off, int *group,
                           int *index_in_group);

/* The plan of group g and the element offsets of its blocks in f, f_wav, f_scal. */
int s2let_batch_group_plan(const s2let_batch *batch, int g, s2let_plan **plan, int64_t *f_off, int64_t *wav_off,
                           int64_t *scal_off);

/* Autotunes every group's plan (s2let_plan_autotune) on `stream` and drops the
 * graphs captured so far, so that the next round trip captures the chosen
 * kernels.  Synchronises the stream. */
int s2let_batch_autotune(s2let_batch *batch, void *stream);

/* Analysis then synthesis of every map (f -> f_wav, f_scal -> f_out).  The
 * first call for a given set of pointers and stream captures the work of all
 * groups, each group on its own forked stream, into one CUDA graph; later
 * calls with the same pointers replay it with a single cudaGraphLaunch on
 * `stream`.  Graphs for up to 8 pointer sets are kept. */
int s2let_batch_round_trip(s2let_batch *batch, const void *f, void *f_wav, void *f_scal, void *f_out,
                           void *stream);

/* ---- instrumentation (no counterpart in the paper) ----------------------
 * Stages of the data path; every kernel launch belongs to one of them. */
#define S2LET_STAGE_RING_FWD 0   /* ring DFT, samples -> F_m(theta_t)           */
#define S2LET_STAGE_THETA_QUAD 1 /* MW theta quadrature, F_m -> G_m             */
#define S2LET_STAGE_LEG_ANAL 2   /* Legendre sum over rings (forward transform) */
#define S2LET_STAGE_LEG_SYNTH 3  /* Legendre sum over degrees (inverse)         */
#define S2LET_STAGE_RING_INV 4   /* inverse ring DFT, F_m(theta_t) -> samples   */
#define S2LET_STAGE_PACK 5       /* f_lm layout conversion                     */
#define S2LET_N_STAGES 6

/* enable = 1: clear the per-stage counters and, until called with enable = 0,
 * record a CUDA event pair on the call's stream around every kernel launch
 * (at most 8192 launches are timed; later ones are only counted).
 * Launch counts are kept whether or not timing is enabled. */
int s2let_plan_profile(s2let_plan *plan, int enable);

/* Totals for one stage since the last s2let_plan_profile(plan, 1): kernel
 * launches, device time in ms of the timed launches (this call synchronizes
 * their events), and the algorithmic work those timed launches stand for,
 * independent of how the kernels do it: Legendre stages count 4 flops per
 * (l, m, ring, map) product (the recurrence that yields lambda_lm is not
 * counted) and no bytes; ring-DFT stages count the bytes of the map and of
 * its order-major spectrum (Sect. 3.2: ring FFTs); the theta quadrature counts
 * the bytes of its input and output spectra and no flops.  Any output pointer
 * may be NULL. */
int s2let_plan_stage_stats(s2let_plan *plan, int stage, int64_t *launches, int64_t *timed, double *ms,
                           double *flops, double *bytes);

/* Pieces of the analysis for gradients that recompute one scale at a time
 * (the analysis is W^j = Inv_{N_j}(sqrt(4 pi/(2l+1)) Psi^j*_l0 f_lm), f_lm =
 * Fwd_L(f), Eqs. wav2 and wav4; the transposes are under the Euclidean inner
 * product of the stored arrays, as for s2let_adjoint):
 * s2let_wav_scale: the maps w of scale j (j = -1: the scaling maps) of the
 *   plan's batch from harmonic coefficients flm (device, batch x L*L complex,
 *   index l*l + l + m; real maps: the coefficients of a real map).  w is
 *   batch maps at that scale's band-limit (the layout of one block of f_wav).
 * s2let_wav_scale_adjoint: glm += the transpose of s2let_wav_scale applied to
 *   the maps g (same layouts; glm accumulates, so the caller zeroes it first).
 * s2let_sht_forward_adjoint: gf = the transpose of s2let_sht_forward applied to
 *   glm.  So the gradient of a loss of the wavelet maps is
 *   s2let_sht_forward_adjoint(sum_j s2let_wav_scale_adjoint(dloss/dW^j)), with
 *   each W^j recomputed from f_lm when it is needed.
 * All use the plan's workspace (a call must not overlap another call of the same
 * plan) and run asynchronously on `stream`; S2LET_ERR_ARG for a j outside
 * {-1, J_min..J} or a NULL pointer. */
int s2let_wav_scale(s2let_plan *plan, int j, const void *flm, void *w, void *stream);
int s2let_wav_scale_adjoint(s2let_plan *plan, int j, const void *g, void *glm, void *stream);
int s2let_sht_forward_adjoint(s2let_plan *plan, const void *glm, void *gf, void *stream);

/* Autotuner.  For every band-limit of the plan, times the candidate kernels of
 * each stage on the plan's own workspace (contents ignored) with the plan's
 * batch, and keeps the fastest: the ring-DFT block size (M/8, M/16, M/32 or
 * M/64 threads, 32..512) for all plans, and for TF32X3 plans, per contraction stage
 * (quadrature: dense tensor-core, dense CUDA-core or FFT form; Legendre
 * analysis and synthesis: the tensor-core kernel on the plan's Legendre tables
 * where it holds them, the tensor-core kernel with the float-float recurrence,
 * or the CUDA-core FP32 kernel; all meet the TF32X3 accuracy).  Runs on
 * `stream` and synchronises it; overwrites the workspace; the choices persist
 * for the plan.  Without this call the plan uses the tensor-core kernels (on
 * the tables where held) and M/16 threads. */
int s2let_plan_autotune(s2let_plan *plan, void *stream);

/* Bytes of device memory that hold the Legendre tables of band-limit N of the
 * plan (0: no tables there), or of all its band-limits for N = 0.  A band-limit
 * the plan does not have: S2LET_ERR_ARG. */
int s2let_plan_leg_table_bytes(const s2let_plan *plan, int N, size_t *bytes);

/* The choices in force for band-limit N of the plan: 1 = tensor-core kernel,
 * 0 = CUDA-core kernel; *tc_quad = 2: the theta quadrature runs in its FFT form
 * (mixed-radix, FP32) instead of a dense product; *tc_anal, *tc_synth = 2: the
 * tensor-core Legendre kernel reads the plan's Legendre tables (1: it runs the
 * recurrence). */
int s2let_plan_tuning(const s2let_plan *plan, int N, int *tc_quad, int *tc_anal, int *tc_synth,
                      int *fft_threads);

/* ---- allocation-free inverse transform (no counterpart in the paper) -----
 * For callers that cannot allocate device memory: applications whose device
 * memory is handed out once by a framework or a fixed budget (a cudaMalloc of
 * their own would fail or break that accounting), plug-ins that run inside a
 * host program which owns the allocator, and real-time or embedded hosts that
 * forbid allocation after start-up.  It computes the same inverse MW transform
 * as s2let_sht_inverse of an FP32 plan, without a plan and without calling
 * cudaMalloc, cudaFree or any allocating library routine: its tables and work
 * buffers live in one statically sized device array inside the library
 * (S2LET_NOALLOC_SCRATCH_BYTES), which every GPU that loads the library holds
 * until the process exits.
 *   L:      band-limit, 2 <= L <= S2LET_NOALLOC_MAX_L (else S2LET_ERR_ARG)
 *   batch:  number of maps, 1 <= batch <= S2LET_NOALLOC_MAX_BATCH (else S2LET_ERR_ARG)
 *   flags:  S2LET_PREC_FP32, optionally | S2LET_COMPLEX (any other bit: S2LET_ERR_ARG)
 *   flm:    device, batch x L*L complex float (index l*l + l + m), read only
 *   f:      device, batch maps of L x (2L-1) float (complex: interleaved), written
 * Set-up: the first call on a device, and every call whose (L, batch, complex)
 * differs from the previous call on that device, first waits for all work
 * already queued on the device (cudaDeviceSynchronize: kernels of earlier
 * calls, on any stream, still read the tables), then looks up the array's
 * device address (cudaGetSymbolAddress), copies tables into it and computes
 * Legendre seeds, synchronising the device again.  Make that first call before
 * any stream capture; a call that needs the set-up while `stream` is being
 * captured returns S2LET_ERR_UNSUPPORTED and does nothing.  The other calls
 * only launch kernels on `stream`.
 * The array is shared by every call on a device and keeps the last call's
 * contents; calls whose kernels overlap on the GPU (different streams, no
 * ordering) race on it and must be serialised by the caller. */
#define S2LET_NOALLOC_MAX_L 128
#define S2LET_NOALLOC_MAX_BATCH 8
#define S2LET_NOALLOC_SCRATCH_BYTES (8u << 20)
int s2let_sht_inverse_noalloc(int L, int batch, int flags, const void *flm, void *f, void *stream);

/* Host-only queries (no plan, no GPU), the tables a plan with these arguments uses:
 * s2let_wav_bandlimits: *N_scal and N_wav[0 .. J-J_min] (N_wav may be NULL,
 *   else it must hold n_wav_cap >= J - J_min + 1 entries) are the band-limits of
 *   the scaling map and of scales J_min..J under `flags` (S2LET_MULTIRES,
 *   S2LET_KERNEL_BSPLINE; Sect. 3.1).  Returns the number of scales J - J_min + 1,
 *   or S2LET_ERR_ARG (L < 2, B < 2, J_min outside [0, J), unknown flag bits, a
 *   too short N_wav).
 * s2let_wav_kernel: fac[l], l < L, the kernel factor sqrt(4 pi/(2l+1)) Psi^j_l0
 *   of scale j (J_min <= j <= J) or sqrt(4 pi/(2l+1)) Phi_l0 (j = -1) of the
 *   family `flags` selects (Sect. 2.2); fac holds L doubles (caller-owned).
 *   S2LET_ERR_ARG as above, for L > 65536, or for j outside {-1, J_min..J}. */
int s2let_wav_bandlimits(int L, int B, int J_min, int flags, int *N_scal, int *N_wav, int n_wav_cap);
int s2let_wav_kernel(int L, int B, int J_min, int flags, int j, double *fac);

/* Wavelet denoising by hard thresholding (Sect. 4.3).
 *
 * s2let_wav_noise_std: *ratio = sigma^j / sigma = sqrt(sum_l |Psi^j_l0|^2), the
 *   standard deviation in scale j (j = -1: the scaling function Phi) of zero-mean
 *   white noise whose harmonic coefficients have variance sigma^2 (Eqs. noisevar,
 *   noisemodel), from the plan's kernel tables.  Host only.  S2LET_ERR_ARG for a
 *   j outside {-1, J_min..J}.
 * s2let_wav_threshold: Eq. (threshold) in place on the wavelet maps `f_wav` (the
 *   plan's wavelet layout, device pointer, caller-owned): every sample of scale
 *   j whose modulus (absolute value of a real sample, |re + i im| of a complex
 *   one) is below T^j = nsigma * sigma^j is set to zero, the others are kept; the
 *   scaling maps are not thresholded (the paper keeps the scaling coefficients).
 *   The paper's T^j = 3 sigma^j is nsigma = 3.  The test is made in the plan's
 *   precision on T^j rounded to it (complex: re*re + im*im < T*T, each operation
 *   rounded to nearest).  One kernel launch on `stream`; S2LET_ERR_ARG for a
 *   negative or non-finite sigma or nsigma or a NULL pointer.
 * Denoising (Sect. 4.3) is s2let_analysis, s2let_wav_threshold on f_wav, then
 * s2let_synthesis with the unchanged f_scal. */
int s2let_wav_noise_std(const s2let_plan *plan, int j, double *ratio);
int s2let_wav_threshold(s2let_plan *plan, void *f_wav, double sigma, double nsigma, void *stream);

/* Device memory of plans.  By default plans (and the group plans of a batch)
 * take their tables and workspace from cudaMalloc and return them with
 * cudaFree.  s2let_set_allocator installs a process-wide hook instead:
 * alloc(bytes, ctx) returns device memory of the current device aligned to
 * 256 bytes, or NULL on failure; release(ptr, ctx) takes back what alloc
 * returned.  Plans created while a hook is installed use it for every
 * allocation, including the temporary ones of plan creation, and keep it until
 * they are destroyed.  A failed (NULL) or misaligned allocation makes the plan
 * creation return S2LET_ERR_ALLOC after releasing everything it allocated.
 * alloc = release = NULL restores cudaMalloc / cudaFree; exactly one of them
 * NULL is S2LET_ERR_ARG.  Transform calls never allocate.  Not part of the
 * paper: it lets a host framework own the memory (e.g. a caching allocator)
 * and lets tests simulate allocation failures. */
typedef void *(*s2let_alloc_fn)(size_t bytes, void *ctx);
typedef void (*s2let_free_fn)(void *ptr, void *ctx);
int s2let_set_allocator(s2let_alloc_fn alloc, s2let_free_fn release, void *ctx);

/* Failure-path check, not part of the paper: launches on `stream` one small
 * kernel whose two bounded waits -- the suspending and the polling kind that
 * the tensor-core kernels use -- wait on barriers that nothing arrives at.
 * They give up after their iteration limits (seconds), and the kernel sets the
 * plan's error word as a tensor-core kernel does when a wait runs out, so that
 * s2let_plan_status(plan) then returns S2LET_ERR_TIMEOUT for good.  The
 * kernel issues no copy and no MMA; the plan's transforms are unaffected. */
int s2let_plan_test_timeout(s2let_plan *plan, void *stream);

/* Device-side status of a plan: S2LET_ERR_TIMEOUT if a bounded wait inside a
 * tensor-core kernel gave up since the plan was created (its results are then
 * not valid), else S2LET_OK.  Synchronises the device. */
int s2let_plan_status(s2let_plan *plan);

/* Short text for a status code. */
const char *s2let_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* S2LET_GPU_H */
