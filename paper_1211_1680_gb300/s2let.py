"""Python face of the C ABI: a Plan object whose methods take torch CUDA
tensors and pass their device pointers and the current CUDA stream to
libs2let_gpu.so.  Every step of the transforms runs in the library's kernels;
this module only checks shapes and dtypes and marshals arguments."""
import ctypes

import torch

from . import _lib
from ._lib import (S2LET_COMPLEX, S2LET_MULTIRES, S2LET_PREC_FP32, S2LET_PREC_FP64,  # noqa: F401
                   S2LET_KERNEL_BSPLINE, S2LET_LEG_RECURRENCE, S2LET_PREC_TF32X3, S2LET_QUAD_DENSE,
                   S2LET_QUAD_FFT64, S2LET_TC_SPLIT3, check)

PRECISIONS = {"fp64": S2LET_PREC_FP64, "fp32": S2LET_PREC_FP32, "tf32x3": S2LET_PREC_TF32X3}


def jmax(L, B):
    r = _lib.lib().s2let_jmax(L, B)
    if r < 0:
        raise _lib.S2letError("s2let_jmax", r)
    return r


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _kernel_flag(kernel):
    if kernel not in ("sd", "bspline"):
        raise ValueError("kernel must be 'sd' or 'bspline'")
    return S2LET_KERNEL_BSPLINE if kernel == "bspline" else 0


_hook = None     # the installed allocator callbacks (kept alive while plans may use them)


def set_allocator(alloc=None, release=None):
    """Install a device-memory hook for plans created from now on
    (s2let_set_allocator): alloc(nbytes) -> device address (int, 0 on failure),
    release(address).  With no arguments, plans use cudaMalloc / cudaFree again.
    The callbacks stay referenced here, so that plans created with them can free
    their memory after the hook is replaced."""
    global _hook
    lib = _lib.lib()
    if alloc is None and release is None:
        check("s2let_set_allocator", lib.s2let_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None))
        return
    a = _lib.ALLOC_FN(lambda n, ctx: alloc(int(n)) or None)
    r = _lib.FREE_FN(lambda ptr, ctx: release(int(ptr)))
    check("s2let_set_allocator", lib.s2let_set_allocator(a, r, None))
    _keep.append((a, r))
    _hook = (a, r)


_keep = []


def use_torch_allocator(device=None):
    """Let PyTorch's caching allocator own the memory of plans created from now on."""
    dev = torch.cuda.current_device() if device is None else device

    def alloc(n):
        return torch.cuda.caching_allocator_alloc(n, dev)

    set_allocator(alloc, torch.cuda.caching_allocator_delete)


class Plan:
    """A batched transform plan: `batch` maps of band-limit L, dilation B,
    lowest scale J_min (Sect. 2.2), real or complex, multiresolution or not,
    precision "fp64", "fp32" or "tf32x3", generating functions `kernel` "sd"
    (smooth scale-discretised) or "bspline" (footnote of Sect. 2.2).  TF32X3
    plans (split tensor-core contractions) store the Legendre values of each
    band-limit up to 2048 that fits the table budget, as FP16 hi/lo parts in two
    copies, unless leg_recurrence is set (see table_bytes())."""

    def __init__(self, L, B, J_min, batch=1, real=True, multires=True, precision="fp64",
                 quad_fft64=False, tc_split3=False, device=None, kernel="sd", quad_dense=False,
                 leg_recurrence=False):
        flags = (0 if real else S2LET_COMPLEX) | (S2LET_MULTIRES if multires else 0) | PRECISIONS[precision]
        flags |= _kernel_flag(kernel)
        if quad_fft64:
            flags |= S2LET_QUAD_FFT64
        if tc_split3:
            flags |= S2LET_TC_SPLIT3
        if quad_dense:
            flags |= S2LET_QUAD_DENSE
        if leg_recurrence:
            flags |= S2LET_LEG_RECURRENCE
        self.L, self.B, self.J_min, self.batch = L, B, J_min, batch
        self.real, self.multires, self.precision, self.kernel = real, multires, precision, kernel
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self._h = ctypes.c_void_p()
        lib = _lib.lib()
        with torch.cuda.device(self.device):
            check("s2let_plan_create", lib.s2let_plan_create(ctypes.byref(self._h), L, B, J_min, flags, batch))
        J = ctypes.c_int()
        ns = ctypes.c_int()
        we = ctypes.c_int64()
        se = ctypes.c_int64()
        nsc = ctypes.c_int()
        check("s2let_plan_info", lib.s2let_plan_info(self._h, ctypes.byref(J), ctypes.byref(ns), ctypes.byref(we),
                                                     ctypes.byref(se), ctypes.byref(nsc)))
        self.J, self.n_scales = J.value, ns.value
        self.wav_elems, self.scal_elems, self.N_scal = we.value, se.value, nsc.value
        self.scales = []
        for j in range(J_min, self.J + 1):
            n = ctypes.c_int()
            off = ctypes.c_int64()
            cnt = ctypes.c_int64()
            check("s2let_wav_layout", lib.s2let_wav_layout(self._h, j, ctypes.byref(n), ctypes.byref(off),
                                                           ctypes.byref(cnt)))
            self.scales.append((j, n.value, off.value, cnt.value))

    def autotune(self, stream=None):
        """Time the candidate kernels of every stage and band-limit and keep the
        fastest (s2let_plan_autotune); returns the choices (see tuning())."""
        check("s2let_plan_autotune", _lib.lib().s2let_plan_autotune(self._h, _stream_handle(stream)))
        return self.tuning()

    def tuning(self):
        """{band-limit: {"tc_quad", "fft_quad", "tc_anal", "tc_synth", "table_anal", "table_synth": bool,
        "fft_threads": int}} (table_*: the tensor-core Legendre kernel reads the plan's tables)."""
        out = {}
        for n in sorted({self.L, self.N_scal} | {s[1] for s in self.scales}):
            v = [ctypes.c_int() for _ in range(4)]
            check("s2let_plan_tuning", _lib.lib().s2let_plan_tuning(self._h, n, *[ctypes.byref(x) for x in v]))
            out[n] = {"tc_quad": v[0].value == 1, "fft_quad": v[0].value == 2, "tc_anal": bool(v[1].value),
                      "tc_synth": bool(v[2].value), "table_anal": v[1].value == 2, "table_synth": v[2].value == 2,
                      "fft_threads": v[3].value}
        return out

    def table_bytes(self, N=0):
        """Device bytes of the plan's Legendre tables at band-limit N, or of all of
        them for N = 0 (s2let_plan_leg_table_bytes)."""
        b = ctypes.c_size_t()
        check("s2let_plan_leg_table_bytes", _lib.lib().s2let_plan_leg_table_bytes(self._h, N, ctypes.byref(b)))
        return b.value

    def status(self):
        """S2LET_OK, or S2LET_ERR_TIMEOUT if a bounded device wait gave up (synchronises)."""
        return _lib.lib().s2let_plan_status(self._h)

    def test_timeout(self, stream=None):
        """Failure-path check (s2let_plan_test_timeout): one kernel whose bounded
        waits run out; status() reports S2LET_ERR_TIMEOUT afterwards."""
        check("s2let_plan_test_timeout", _lib.lib().s2let_plan_test_timeout(self._h, _stream_handle(stream)))

    def close(self):
        if self._h:
            _lib.lib().s2let_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- instrumentation
    def profile(self, enable=True):
        """Start (clearing counters) or stop per-stage event timing."""
        check("s2let_plan_profile", _lib.lib().s2let_plan_profile(self._h, 1 if enable else 0))

    def stage_stats(self):
        """{stage: dict(launches, timed, ms, flops, bytes)} since profile(True)."""
        out = {}
        for i, name in enumerate(_lib.STAGES):
            n = ctypes.c_int64()
            tm = ctypes.c_int64()
            ms = ctypes.c_double()
            fl = ctypes.c_double()
            by = ctypes.c_double()
            check("s2let_plan_stage_stats", _lib.lib().s2let_plan_stage_stats(
                self._h, i, ctypes.byref(n), ctypes.byref(tm), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by)))
            out[name] = dict(launches=n.value, timed=tm.value, ms=ms.value, flops=fl.value, bytes=by.value)
        return out

    # ---------------------------------------------------------------- shapes
    def map_shape(self, N):
        s = (self.batch, N, 2 * N - 1)
        return s if self.real else s + (2,)

    def empty_map(self, N=None):
        return torch.empty(self.map_shape(self.L if N is None else N), dtype=self.dtype, device=self.device)

    def empty_wavelets(self):
        """(f_wav flat buffer, f_scal) as the library lays them out."""
        fw = torch.empty(self.wav_elems, dtype=self.dtype, device=self.device)
        fs = torch.empty(self.map_shape(self.N_scal), dtype=self.dtype, device=self.device)
        return fw, fs

    def wavelet_views(self, fw):
        """Views of each scale's block of the flat f_wav buffer, scale J_min first."""
        return [fw[off:off + cnt].view(self.map_shape(n)) for (_, n, off, cnt) in self.scales]

    def flm_shape(self):
        return (self.batch, self.L * self.L, 2)

    def _chk(self, t, numel, name):
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and t.numel() == numel):
            raise ValueError("%s: need a contiguous %s CUDA tensor with %d elements" % (name, self.dtype, numel))
        return ctypes.c_void_p(t.data_ptr())

    def _map_numel(self, N):
        n = self.batch * N * (2 * N - 1)
        return n if self.real else 2 * n

    # ---------------------------------------------------------------- transforms
    def analysis(self, f, f_wav=None, f_scal=None, stream=None):
        if f_wav is None:
            f_wav, f_scal = self.empty_wavelets()
        a = self._chk(f, self._map_numel(self.L), "f")
        w = self._chk(f_wav, self.wav_elems, "f_wav")
        s = self._chk(f_scal, self.scal_elems, "f_scal")
        check("s2let_analysis", _lib.lib().s2let_analysis(self._h, a, w, s, _stream_handle(stream)))
        return f_wav, f_scal

    def synthesis(self, f_wav, f_scal, f=None, stream=None):
        if f is None:
            f = self.empty_map()
        w = self._chk(f_wav, self.wav_elems, "f_wav")
        s = self._chk(f_scal, self.scal_elems, "f_scal")
        o = self._chk(f, self._map_numel(self.L), "f")
        check("s2let_synthesis", _lib.lib().s2let_synthesis(self._h, w, s, o, _stream_handle(stream)))
        return f

    def adjoint(self, g_wav, g_scal, g_f=None, stream=None):
        if g_f is None:
            g_f = self.empty_map()
        w = self._chk(g_wav, self.wav_elems, "g_wav")
        s = self._chk(g_scal, self.scal_elems, "g_scal")
        o = self._chk(g_f, self._map_numel(self.L), "g_f")
        check("s2let_adjoint", _lib.lib().s2let_adjoint(self._h, w, s, o, _stream_handle(stream)))
        return g_f

    def sht_forward(self, f, flm=None, stream=None):
        if flm is None:
            flm = torch.empty(self.flm_shape(), dtype=self.dtype, device=self.device)
        a = self._chk(f, self._map_numel(self.L), "f")
        o = self._chk(flm, self.batch * self.L * self.L * 2, "flm")
        check("s2let_sht_forward", _lib.lib().s2let_sht_forward(self._h, a, o, _stream_handle(stream)))
        return flm

    def sht_inverse(self, flm, f=None, stream=None):
        if f is None:
            f = self.empty_map()
        a = self._chk(flm, self.batch * self.L * self.L * 2, "flm")
        o = self._chk(f, self._map_numel(self.L), "f")
        check("s2let_sht_inverse", _lib.lib().s2let_sht_inverse(self._h, a, o, _stream_handle(stream)))
        return f

    # ---------------------------------------------------------------- per-scale pieces (gradients)
    def scale_bandlimit(self, j):
        """Band-limit of scale j's maps (j = -1: the scaling maps)."""
        if j == -1:
            return self.N_scal
        for (jj, n, _, _) in self.scales:
            if jj == j:
                return n
        raise ValueError("no scale %r" % (j,))

    def wav_scale(self, j, flm, w=None, stream=None):
        """The maps of scale j (j = -1: scaling) from harmonic coefficients flm."""
        n = self.scale_bandlimit(j)
        if w is None:
            w = self.empty_map(n)
        a = self._chk(flm, self.batch * self.L * self.L * 2, "flm")
        o = self._chk(w, self._map_numel(n), "w")
        check("s2let_wav_scale", _lib.lib().s2let_wav_scale(self._h, j, a, o, _stream_handle(stream)))
        return w

    def wav_scale_adjoint(self, j, g, glm, stream=None):
        """glm += the transpose of wav_scale(j) applied to the maps g."""
        n = self.scale_bandlimit(j)
        a = self._chk(g, self._map_numel(n), "g")
        o = self._chk(glm, self.batch * self.L * self.L * 2, "glm")
        check("s2let_wav_scale_adjoint", _lib.lib().s2let_wav_scale_adjoint(self._h, j, a, o, _stream_handle(stream)))
        return glm

    def sht_forward_adjoint(self, glm, gf=None, stream=None):
        """gf = the transpose of sht_forward applied to glm."""
        if gf is None:
            gf = self.empty_map()
        a = self._chk(glm, self.batch * self.L * self.L * 2, "glm")
        o = self._chk(gf, self._map_numel(self.L), "gf")
        check("s2let_sht_forward_adjoint", _lib.lib().s2let_sht_forward_adjoint(self._h, a, o, _stream_handle(stream)))
        return gf

    # ---------------------------------------------------------------- denoising (Sect. 4.3)
    def noise_std(self, j):
        """sigma^j / sigma for scale j (j = -1: the scaling function)."""
        r = ctypes.c_double()
        check("s2let_wav_noise_std", _lib.lib().s2let_wav_noise_std(self._h, j, ctypes.byref(r)))
        return r.value

    def threshold(self, f_wav, sigma, nsigma=3.0, stream=None):
        """Hard thresholding of the wavelet maps in place: |W^j| < nsigma sigma^j -> 0."""
        w = self._chk(f_wav, self.wav_elems, "f_wav")
        check("s2let_wav_threshold", _lib.lib().s2let_wav_threshold(self._h, w, float(sigma), float(nsigma),
                                                                     _stream_handle(stream)))
        return f_wav

    def denoise(self, y, sigma, nsigma=3.0, out=None, stream=None):
        """Analysis, hard thresholding of the wavelet maps (the scaling maps are
        kept), synthesis: the denoising of Sect. 4.3."""
        f_wav, f_scal = self.analysis(y, stream=stream)
        self.threshold(f_wav, sigma, nsigma, stream=stream)
        return self.synthesis(f_wav, f_scal, out, stream=stream)


class HostPipeline:
    """Streams batches of maps between pinned host memory and a plan's transforms
    with the copies overlapped: while step k computes on the caller's stream,
    step k+1's inputs are copied in (host -> device) on one copy stream and step
    k-1's results out (device -> host) on another.  Device buffers are kept in
    `depth` slots; CUDA events order each slot's copy-in, compute and copy-out,
    so no slot is overwritten while it is still read.  Only data movement and
    ordering live here: the transforms are whatever `compute` launches."""

    def __init__(self, in_like, out_like, depth=2):
        if depth < 2:
            raise ValueError("depth must be at least 2")
        self.depth = depth
        self.din = [torch.empty_like(in_like) for _ in range(depth)]
        self.dout = [torch.empty_like(out_like) for _ in range(depth)]
        self.h2d = torch.cuda.Stream(device=in_like.device)
        self.d2h = torch.cuda.Stream(device=in_like.device)
        self.in_ready = [torch.cuda.Event() for _ in range(depth)]
        self.computed = [torch.cuda.Event() for _ in range(depth)]
        self.out_free = [torch.cuda.Event() for _ in range(depth)]

    def run(self, n_steps, host_in, host_out, compute):
        """For k < n_steps: copy host_in(k) in, compute(din, dout) on the current
        stream, copy dout to host_out(k).  host_in / host_out return pinned host
        tensors shaped like the device buffers.  Returns when every copy-out has
        been queued; the caller synchronises."""
        cs = torch.cuda.current_stream()
        for k in range(n_steps):
            s = k % self.depth
            with torch.cuda.stream(self.h2d):
                if k >= self.depth:
                    self.h2d.wait_event(self.computed[s])       # step k - depth has read din[s]
                self.din[s].copy_(host_in(k), non_blocking=True)
                self.in_ready[s].record(self.h2d)
            cs.wait_event(self.in_ready[s])
            if k >= self.depth:
                cs.wait_event(self.out_free[s])                  # step k - depth's result has left dout[s]
            compute(self.din[s], self.dout[s])
            self.computed[s].record(cs)
            with torch.cuda.stream(self.d2h):
                self.d2h.wait_event(self.computed[s])
                host_out(k).copy_(self.dout[s], non_blocking=True)
                self.out_free[s].record(self.d2h)


class BatchPlan:
    """Maps of uneven band-limit L_i and dilation B_i (same J_min, real/complex and
    precision), transformed together: one plan per (L, B) group, and one CUDA
    graph (captured on the first call for a set of buffers) replays the round
    trip of every group with a single launch."""

    def __init__(self, Ls, Bs, J_min, real=True, multires=True, precision="fp32", device=None, kernel="sd"):
        Ls = [int(x) for x in Ls]
        Bs = [int(x) for x in Bs]
        if len(Ls) != len(Bs) or not Ls:
            raise ValueError("need equally long, non-empty L and B lists")
        flags = (0 if real else S2LET_COMPLEX) | (S2LET_MULTIRES if multires else 0) | PRECISIONS[precision]
        flags |= _kernel_flag(kernel)
        self.Ls, self.Bs, self.J_min, self.real = Ls, Bs, J_min, real
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self._h = ctypes.c_void_p()
        lib = _lib.lib()
        arrL = (ctypes.c_int * len(Ls))(*Ls)
        arrB = (ctypes.c_int * len(Bs))(*Bs)
        with torch.cuda.device(self.device):
            check("s2let_batch_create", lib.s2let_batch_create(ctypes.byref(self._h), len(Ls), arrL, arrB, J_min,
                                                               flags))
        fe, we, se, ng = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        check("s2let_batch_sizes", lib.s2let_batch_sizes(self._h, ctypes.byref(fe), ctypes.byref(we),
                                                         ctypes.byref(se), ctypes.byref(ng)))
        self.f_elems, self.wav_elems, self.scal_elems, self.n_groups = fe.value, we.value, se.value, ng.value
        self.layout = []
        for i in range(len(Ls)):
            fo, so, g, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
            check("s2let_batch_map_layout", lib.s2let_batch_map_layout(self._h, i, ctypes.byref(fo), ctypes.byref(so),
                                                                       ctypes.byref(g), ctypes.byref(k)))
            self.layout.append((fo.value, so.value, g.value, k.value))
        self.groups = []
        for g in range(self.n_groups):
            ph, fo, wo, so = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
            check("s2let_batch_group_plan", lib.s2let_batch_group_plan(self._h, g, ctypes.byref(ph), ctypes.byref(fo),
                                                                       ctypes.byref(wo), ctypes.byref(so)))
            self.groups.append((ph.value, fo.value, wo.value, so.value))

    def autotune(self, stream=None):
        """Autotune every group's plan (kernel choice per stage and band-limit,
        ring-DFT block size); later round trips capture the chosen kernels."""
        check("s2let_batch_autotune", _lib.lib().s2let_batch_autotune(self._h, _stream_handle(stream)))

    def close(self):
        if self._h:
            _lib.lib().s2let_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def map_numel(self, L):
        n = L * (2 * L - 1)
        return n if self.real else 2 * n

    def buffers(self):
        """Flat (f, f_wav, f_scal, f_out) device buffers in the batch layout."""
        mk = lambda n: torch.empty(n, dtype=self.dtype, device=self.device)  # noqa: E731
        return mk(self.f_elems), mk(self.wav_elems), mk(self.scal_elems), mk(self.f_elems)

    def map_view(self, flat, i):
        """Map i of a flat f / f_out buffer, shaped (L, 2L-1[, 2])."""
        L = self.Ls[i]
        off = self.layout[i][0]
        shape = (L, 2 * L - 1) if self.real else (L, 2 * L - 1, 2)
        return flat[off:off + self.map_numel(L)].view(shape)

    def round_trip(self, f, f_wav, f_scal, f_out, stream=None):
        """Analysis then synthesis of every map, as one graph launch."""
        for t, n, name in ((f, self.f_elems, "f"), (f_wav, self.wav_elems, "f_wav"), (f_scal, self.scal_elems, "f_scal"),
                           (f_out, self.f_elems, "f_out")):
            if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and t.numel() == n):
                raise ValueError("%s: need a contiguous %s CUDA tensor with %d elements" % (name, self.dtype, n))
        s = stream if stream is not None else torch.cuda.current_stream()
        if s == torch.cuda.default_stream(self.device):
            raise ValueError("round_trip needs a non-default stream (the work is captured into a CUDA graph)")
        check("s2let_batch_round_trip", _lib.lib().s2let_batch_round_trip(
            self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f_wav.data_ptr()),
            ctypes.c_void_p(f_scal.data_ptr()), ctypes.c_void_p(f_out.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
        return f_out
