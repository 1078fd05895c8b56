"""Python binding of the mr1l CUDA library (multiple rank-1 lattice sparse FFT).

Argument marshalling only: every step of the transforms runs in the CUDA
kernels of ``libmr1l.so`` (built in-tree by ``build.py``).  PyTorch provides
device memory and streams.  There is no CPU fallback: importing the binding
raises when the library has not been built.

Names follow the paper (Kaemmerer, Potts, Volkmer): ``plan`` builds a
multiple rank-1 lattice for a frequency set I (given lattices, or Algorithm 1
with ``plan_search``), ``Plan.reconstruct`` is Algorithm 2, ``Plan.evaluate``
the lattice evaluation and its adjoint, and ``sfft_dimincr`` Algorithm 3.
"""

from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmr1l.so")

MR1L_OK = 0
MR1L_E_INVAL = 1
MR1L_E_NOMEM = 2
MR1L_E_CUDA = 3
MR1L_E_NOT_RECONSTRUCTING = 4
MR1L_E_SAMPLER = 5
MR1L_E_TIMEOUT = 6
MR1L_STRICT = 1
MR1L_FFT_DF = 2
MR1L_REDRAW = 4
MR1L_EVAL = 0
MR1L_ADJOINT = 1
SFFT_THETA_ABS = 0
SFFT_THETA_REL = 1
SFFT_REQ_LINE = 0
SFFT_REQ_LATTICE = 1
SFFT_MAX_STEPS = 256

EXPORTS = [
    "mr1l_last_error", "mr1l_version", "mr1l_plan", "mr1l_plan_search", "mr1l_plan_info",
    "mr1l_plan_masks", "mr1l_destroy", "mr1l_reconstruct", "mr1l_evaluate", "sfft_dimincr",
    "sfft_free", "sfft_dimincr_batch", "mr1l_reconstruct_noalloc", "mr1l_lattice_noise", "mr1l_prof_enable", "mr1l_prof_reset", "mr1l_prof_launches", "mr1l_prof_read",
    "mr1l_tune_enable", "mr1l_tune_reset", "mr1l_tune_read", "sfft_theorem_params",
    "mr1l_reconstruct_batch", "mr1l_evaluate_batch", "mr1l_pool_stats", "mr1l_inject_alloc_failure",
    "sfft_select",
]


class Mr1lError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mr1l error {code}: {msg}")
        self.code = code


class sfft_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("t", C.c_int), ("rep", C.c_int), ("d", C.c_int),
                ("anchors", C.POINTER(C.c_double)), ("K", C.c_int), ("L", C.c_int),
                ("M", C.POINTER(C.c_int64)), ("z", C.POINTER(C.c_int64)), ("sum_M", C.c_int64)]


SAMPLE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(sfft_request), C.c_void_p, C.c_void_p)


class sfft_sampler(C.Structure):
    _fields_ = [("fn", SAMPLE_FN), ("user", C.c_void_p), ("freqs", C.POINTER(C.c_int32)),
                ("coeffs", C.POINTER(C.c_double)), ("s", C.c_int64), ("sigma", C.c_double),
                ("noise_seed", C.c_uint64), ("device_arrays", C.c_int), ("kind", C.c_int),
                ("n_groups", C.c_int), ("group_of", C.POINTER(C.c_int)), ("orders", C.POINTER(C.c_int))]


SFFT_SAMPLER_PLANTED, SFFT_SAMPLER_BSPLINE = 0, 1


def _bspline_sampler(d: int, function, keep: list) -> sfft_sampler:
    """The built-in Section 5.3 sampler for a description with .groups (lists
    of 0-based dimensions) and .orders (B-spline order per group)."""
    group_of = np.full(d, -1, dtype=np.int32)
    for g, dims in enumerate(function.groups):
        group_of[list(dims)] = g
    orders = np.ascontiguousarray(np.asarray(function.orders, dtype=np.int32))
    keep += [group_of, orders]
    return sfft_sampler(SAMPLE_FN(), None, None, None, 0, 0.0, 0, 0, SFFT_SAMPLER_BSPLINE, len(function.orders),
                        group_of.ctypes.data_as(C.POINTER(C.c_int)), orders.ctypes.data_as(C.POINTER(C.c_int)))


class sfft_params(C.Structure):
    _fields_ = [("d", C.c_int), ("N", C.c_int), ("s", C.c_int64), ("s_local", C.c_int64),
                ("r", C.c_int), ("b", C.c_int), ("theta", C.c_double), ("theta_mode", C.c_int),
                ("seed", C.c_uint64), ("batch_reps", C.c_int), ("fft_arith", C.c_int), ("t_stop", C.c_int),
                ("zero_anchors", C.c_int), ("redraw", C.c_int)]


class sfft_step_stats(C.Structure):
    _fields_ = [("t", C.c_int), ("n_line", C.c_int), ("n_cand", C.c_int64), ("L", C.c_int),
                ("attempts", C.c_int), ("covered", C.c_int), ("sum_M", C.c_int64),
                ("samples", C.c_int64), ("n_detected", C.c_int64)]


class sfft_stats(C.Structure):
    _fields_ = [("n_steps", C.c_int), ("samples", C.c_int64), ("ms_total", C.c_double),
                ("ms_sampling", C.c_double), ("steps", sfft_step_stats * SFFT_MAX_STEPS)]


class sfft_result(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int), ("freqs", C.POINTER(C.c_int32)),
                ("coeffs", C.POINTER(C.c_double)), ("stats", sfft_stats)]


_lib = None


def lib() -> C.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmr1l.so not built ({LIB_PATH}); run paper_1711_05152_gb300/build.py")
    L = C.CDLL(LIB_PATH)
    vp, i32p, i64p = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    L.mr1l_last_error.argtypes = [C.c_char_p, C.c_size_t]
    L.mr1l_version.argtypes = []
    L.mr1l_plan.argtypes = [i32p, C.c_int64, C.c_int, C.c_int, i64p, i64p, C.c_int, vp, C.POINTER(vp)]
    L.mr1l_plan_search.argtypes = [i32p, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_int, C.c_uint64,
                                   C.c_int, vp, C.POINTER(vp)]
    L.mr1l_plan_info.argtypes = [vp, C.POINTER(C.c_int), i64p, i64p, i64p, i64p, i64p]
    L.mr1l_plan_masks.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]
    L.mr1l_destroy.argtypes = [vp]
    L.mr1l_destroy.restype = None
    L.mr1l_reconstruct.argtypes = [vp, vp, C.c_int, vp, vp]
    L.mr1l_evaluate.argtypes = [vp, vp, C.c_int, vp, C.c_int, vp]
    L.mr1l_reconstruct_noalloc.argtypes = [vp, vp, C.c_int, vp, vp]
    L.mr1l_lattice_noise.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, i64p, C.c_double, vp, vp]
    L.sfft_dimincr.argtypes = [C.POINTER(sfft_params), C.POINTER(sfft_sampler), vp,
                               C.POINTER(C.POINTER(sfft_result))]
    L.sfft_free.argtypes = [C.POINTER(sfft_result)]
    L.sfft_free.restype = None
    L.sfft_dimincr_batch.argtypes = [C.POINTER(sfft_params), C.POINTER(sfft_sampler), C.c_int, C.c_int,
                                     C.POINTER(C.POINTER(sfft_result)), C.POINTER(C.c_int)]
    L.mr1l_prof_enable.argtypes = [C.c_int]
    L.mr1l_prof_reset.argtypes = []
    L.mr1l_prof_launches.argtypes = []
    L.mr1l_prof_launches.restype = C.c_longlong
    L.mr1l_prof_read.argtypes = [C.c_char_p, C.c_size_t]
    L.mr1l_reconstruct_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(C.c_int), C.POINTER(vp),
                                         vp]
    L.mr1l_evaluate_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(C.c_int), C.POINTER(vp),
                                      C.c_int, vp]
    L.sfft_theorem_params.argtypes = [C.c_int, C.c_int64, C.c_double, C.POINTER(C.c_int64), C.POINTER(C.c_int)]
    L.mr1l_tune_enable.argtypes = [C.c_int]
    L.mr1l_tune_reset.argtypes = []
    L.mr1l_tune_read.argtypes = [C.c_char_p, C.c_size_t]
    L.mr1l_pool_stats.argtypes = [C.c_int, i64p, i64p, i64p]
    L.mr1l_inject_alloc_failure.argtypes = [C.c_int64]
    L.sfft_select.argtypes = [vp, C.c_int64, C.c_int, vp, C.c_int64, C.c_double, C.c_int, vp, vp]
    _lib = L
    return L


def _check(rc: int):
    if rc != MR1L_OK:
        buf = C.create_string_buffer(1024)
        lib().mr1l_last_error(buf, 1024)
        raise Mr1lError(rc, buf.value.decode(errors="replace"))


def _stream(stream=None) -> int:
    """cudaStream_t of a torch stream (default: the current one); a plain int
    is taken as the raw handle (0 = legacy default stream)."""
    if isinstance(stream, int):
        return stream
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int64)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def check_out(out, shape, device, name: str = "out"):
    """An output tensor the library will write through a raw pointer: it must
    be a contiguous complex128 tensor of exactly `shape` on `device` (the
    input's device), or the kernels would write out of bounds or to another
    device's memory."""
    import torch
    if out.dtype != torch.complex128 or not out.is_contiguous():
        raise TypeError(f"{name} must be a contiguous complex128 tensor")
    if tuple(out.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(out.shape)}, expected {tuple(shape)}")
    if out.device != device:
        raise ValueError(f"{name} is on {out.device}, expected {device}")


class Plan:
    """A multiple rank-1 lattice planned for a frequency set I (rows of Z^t)."""

    def __init__(self, handle: int, nI: int, t: int):
        self._h = C.c_void_p(handle)
        self.nI = nI
        self.t = t
        info = self.info()
        self.L = info["L"]
        self.M = info["M"]
        self.z = info["z"]
        self.sum_M = info["sum_M"]
        self.nodes = info["nodes"]
        self.n_uncovered = info["n_uncovered"]

    def info(self) -> dict:
        L = C.c_int()
        M = np.zeros(64, dtype=np.int64)
        nodes, sum_M, unc = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().mr1l_plan_info(self._h, C.byref(L), _ptr(M, C.c_int64), None, C.byref(nodes),
                                    C.byref(sum_M), C.byref(unc)))
        z = np.zeros(L.value * self.t, dtype=np.int64)
        _check(lib().mr1l_plan_info(self._h, None, None, _ptr(z, C.c_int64), None, None, None))
        return dict(L=L.value, M=M[:L.value].copy(), z=z.reshape(L.value, self.t), nodes=nodes.value,
                    sum_M=sum_M.value, n_uncovered=unc.value)

    def masks(self):
        """(bitmask of lattices where each k is collision-free, residues [L][nI])."""
        m = np.zeros(self.nI, dtype=np.uint64)
        r = np.zeros((self.L, self.nI), dtype=np.uint32)
        _check(lib().mr1l_plan_masks(self._h, _ptr(m, C.c_uint64), _ptr(r, C.c_uint32)))
        return m, r

    def reconstruct(self, y, out=None, stream=None):
        """Algorithm 2: y complex128 [nrhs, sum_M] (or [sum_M]) on the GPU -> c [nrhs, nI]."""
        import torch
        squeeze = y.dim() == 1
        y2 = y.reshape(-1, self.sum_M)
        if y2.dtype != torch.complex128 or not y2.is_cuda or not y2.is_contiguous():
            raise TypeError("y must be a contiguous complex128 CUDA tensor")
        nrhs = y2.shape[0]
        if out is None:
            out = torch.empty((nrhs, self.nI), dtype=torch.complex128, device=y.device)
        else:
            if squeeze and out.dim() == 1:
                out = out.unsqueeze(0)
            check_out(out, (nrhs, self.nI), y.device)
        _check(lib().mr1l_reconstruct(self._h, C.c_void_p(y2.data_ptr()), nrhs, C.c_void_p(out.data_ptr()),
                                      C.c_void_p(_stream(stream))))
        return out[0] if squeeze else out

    def reconstruct_noalloc(self, y, out, stream=None):
        """Algorithm 2 like reconstruct, for callers that cannot allocate device
        memory: the output tensor is required and the library's intermediate
        data lives in its fixed scratch array (concurrent calls race)."""
        import torch
        y2 = y.reshape(-1, self.sum_M)
        if y2.dtype != torch.complex128 or not y2.is_cuda or not y2.is_contiguous():
            raise TypeError("y must be a contiguous complex128 CUDA tensor")
        check_out(out, (y2.shape[0], self.nI), y.device)
        _check(lib().mr1l_reconstruct_noalloc(self._h, C.c_void_p(y2.data_ptr()), y2.shape[0],
                                              C.c_void_p(out.data_ptr()), C.c_void_p(_stream(stream))))
        return out

    def evaluate(self, c, mode: int = MR1L_EVAL, out=None, stream=None):
        """Lattice evaluation (mode MR1L_EVAL) or the adjoint of Algorithm 2
        (MR1L_ADJOINT): c complex128 [nrhs, nI] -> y [nrhs, sum_M]."""
        import torch
        squeeze = c.dim() == 1
        c2 = c.reshape(-1, self.nI)
        if c2.dtype != torch.complex128 or not c2.is_cuda or not c2.is_contiguous():
            raise TypeError("c must be a contiguous complex128 CUDA tensor")
        nrhs = c2.shape[0]
        if out is None:
            out = torch.empty((nrhs, self.sum_M), dtype=torch.complex128, device=c.device)
        else:
            if squeeze and out.dim() == 1:
                out = out.unsqueeze(0)
            check_out(out, (nrhs, self.sum_M), c.device)
        _check(lib().mr1l_evaluate(self._h, C.c_void_p(c2.data_ptr()), nrhs, C.c_void_p(out.data_ptr()),
                                   mode, C.c_void_p(_stream(stream))))
        return out[0] if squeeze else out

    def close(self):
        if self._h and self._h.value:
            lib().mr1l_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _flags(strict: bool, fft: str, redraw: bool = False) -> int:
    if fft not in ("f64", "df"):
        raise ValueError('fft must be "f64" or "df"')
    return (MR1L_STRICT if strict else 0) | (MR1L_FFT_DF if fft == "df" else 0) | (MR1L_REDRAW if redraw else 0)


def plan(I, M, z, strict: bool = False, fft: str = "f64", stream=None) -> Plan:
    """Plan on given lattices (sizes M [L], generating vectors z [L, t]).
    fft="df" runs the Bluestein butterflies in double-float arithmetic."""
    I = _i32(I)
    if I.ndim == 1:
        I = I.reshape(-1, 1)
    n, t = I.shape
    M = _i64(M).reshape(-1)
    z = _i64(z).reshape(M.shape[0], t)
    h = C.c_void_p()
    _check(lib().mr1l_plan(_ptr(I, C.c_int32), n, t, M.shape[0], _ptr(M, C.c_int64), _ptr(z, C.c_int64),
                           _flags(strict, fft), C.c_void_p(_stream(stream)), C.byref(h)))
    return Plan(h.value, n, t)


def plan_search(I, seed: int, c: float = 2.0, gamma: float = 0.5, b: int = 10, strict: bool = False,
                fft: str = "f64", redraw: bool = False, stream=None) -> Plan:
    """Plan on a lattice built by Algorithm 1 (up to b searches); redraw:
    the redraw rule of the remark after Algorithm 1 (MR1L_REDRAW)."""
    I = _i32(I)
    if I.ndim == 1:
        I = I.reshape(-1, 1)
    n, t = I.shape
    h = C.c_void_p()
    _check(lib().mr1l_plan_search(_ptr(I, C.c_int32), n, t, c, gamma, b, seed, _flags(strict, fft, redraw),
                                  C.c_void_p(_stream(stream)), C.byref(h)))
    return Plan(h.value, n, t)


@dataclasses.dataclass
class SfftOutput:
    freqs: np.ndarray          # int64 [n, d]
    coeffs: np.ndarray         # complex128 [n]
    samples: int
    ms_total: float
    ms_sampling: float
    steps: list


def sfft_dimincr(d: int, N: int, s: int, r: int, theta: float, theta_mode: str = "rel", seed: int = 0,
                 s_local: int | None = None, b: int = 10, freqs=None, coeffs=None, sigma: float = 0.0,
                 noise_seed: int | None = None, sampler=None, batch_reps: bool = False,
                 t_stop: int | None = None, fft: str = "f64", zero_anchors: bool = False,
                 function=None, redraw: bool = False, stream=None) -> SfftOutput:
    """Algorithm 3.  Either a planted polynomial (freqs [s, d], coeffs [s],
    sigma) evaluated by the library, the Section 5.3 B-spline function
    (``function`` with .groups and .orders, evaluated by the library), or
    ``sampler(req, y_ptr, stream_ptr)``, a Python callable that fills the
    device buffer y_ptr for a request.
    zero_anchors: the deterministic variant (anchors 0, see sfft_params).
    redraw: Algorithm 1 with the redraw rule of the remark after it."""
    p = sfft_params(d=d, N=N, s=s, s_local=s if s_local is None else s_local, r=r, b=b, theta=theta,
                    theta_mode=SFFT_THETA_REL if theta_mode == "rel" else SFFT_THETA_ABS, seed=seed,
                    batch_reps=1 if batch_reps else 0, fft_arith=1 if fft == "df" else 0, t_stop=t_stop or 0,
                    zero_anchors=1 if zero_anchors else 0, redraw=1 if redraw else 0)
    keep = []
    nseed = seed if noise_seed is None else noise_seed
    if function is not None:
        samp = _bspline_sampler(d, function, keep)
    elif sampler is None and getattr(freqs, "is_cuda", False):
        # planted signal already resident on the device (int32 [s, d], complex128 [s])
        import torch
        if freqs.dtype != torch.int32 or coeffs.dtype != torch.complex128 or not (
                freqs.is_contiguous() and coeffs.is_contiguous()):
            raise TypeError("device planted arrays must be contiguous int32 / complex128")
        keep += [freqs, coeffs]
        samp = sfft_sampler(SAMPLE_FN(), None, C.cast(C.c_void_p(freqs.data_ptr()), C.POINTER(C.c_int32)),
                            C.cast(C.c_void_p(coeffs.data_ptr()), C.POINTER(C.c_double)), freqs.shape[0], sigma,
                            nseed, 1)
    elif sampler is None:
        f = _i32(freqs).reshape(-1, d)
        c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.complex128)).view(np.float64)
        keep += [f, c]
        samp = sfft_sampler(SAMPLE_FN(), None, _ptr(f, C.c_int32), _ptr(c, C.c_double), f.shape[0], sigma,
                            nseed, 0)
    else:
        def _cb(user, req, y, stream_ptr):
            try:
                return int(sampler(req.contents, y, stream_ptr) or 0)
            except Exception:  # reported as a sampler failure
                import traceback
                traceback.print_exc()
                return 1
        fn = SAMPLE_FN(_cb)
        keep.append(fn)
        samp = sfft_sampler(fn, None, None, None, 0, 0.0, 0, 0)
    out = C.POINTER(sfft_result)()
    _check(lib().sfft_dimincr(C.byref(p), C.byref(samp), C.c_void_p(_stream(stream)), C.byref(out)))
    try:
        return _convert(out.contents)
    finally:
        lib().sfft_free(out)


def _convert(res: sfft_result) -> SfftOutput:
    n, d = res.n, res.d
    fr = np.ctypeslib.as_array(res.freqs, shape=(max(n, 1) * d,))[: n * d].astype(np.int64).reshape(n, d)
    cf = np.ctypeslib.as_array(res.coeffs, shape=(max(n, 1) * 2,))[: 2 * n].copy().view(np.complex128)
    st = res.stats
    steps = []
    for i in range(st.n_steps):
        x = st.steps[i]
        steps.append(dict(t=x.t, n_line=x.n_line, n_cand=x.n_cand, L=x.L, attempts=x.attempts,
                          covered=bool(x.covered), sum_M=x.sum_M, samples=x.samples, n_detected=x.n_detected))
    return SfftOutput(fr, cf, st.samples, st.ms_total, st.ms_sampling, steps)


def sfft_dimincr_batch(problems: list[dict], concurrency: int = 16) -> list[SfftOutput]:
    """Algorithm 3 on many independent problems at once.  Each problem is a
    dict with d, N, s, r, theta, theta_mode, seed and either freqs, coeffs
    (a planted polynomial: host arrays, or contiguous int32 / complex128 CUDA
    tensors) or function (the Section 5.3 B-spline function, see
    sfft_dimincr), and optionally sigma, s_local, b, noise_seed, batch_reps,
    fft, zero_anchors, redraw."""
    n = len(problems)
    params = (sfft_params * max(n, 1))()
    samps = (sfft_sampler * max(n, 1))()
    keep = []
    for i, q in enumerate(problems):
        d = q["d"]
        params[i] = sfft_params(d=d, N=q["N"], s=q["s"], s_local=q.get("s_local", q["s"]), r=q["r"],
                                b=q.get("b", 10), theta=q["theta"],
                                theta_mode=SFFT_THETA_REL if q.get("theta_mode", "rel") == "rel" else SFFT_THETA_ABS,
                                seed=q["seed"], batch_reps=1 if q.get("batch_reps", True) else 0,
                                fft_arith=1 if q.get("fft", "f64") == "df" else 0,
                                zero_anchors=1 if q.get("zero_anchors", False) else 0,
                                redraw=1 if q.get("redraw", False) else 0)
        if q.get("function") is not None:
            samps[i] = _bspline_sampler(d, q["function"], keep)
            continue
        if getattr(q["freqs"], "is_cuda", False):
            f, c = q["freqs"], q["coeffs"]
            keep += [f, c]
            samps[i] = sfft_sampler(SAMPLE_FN(), None, C.cast(C.c_void_p(f.data_ptr()), C.POINTER(C.c_int32)),
                                    C.cast(C.c_void_p(c.data_ptr()), C.POINTER(C.c_double)), f.shape[0],
                                    q.get("sigma", 0.0), q.get("noise_seed", q["seed"]), 1)
            continue
        f = _i32(q["freqs"]).reshape(-1, d)
        c = np.ascontiguousarray(np.asarray(q["coeffs"], dtype=np.complex128)).view(np.float64)
        keep += [f, c]
        samps[i] = sfft_sampler(SAMPLE_FN(), None, _ptr(f, C.c_int32), _ptr(c, C.c_double), f.shape[0],
                                q.get("sigma", 0.0), q.get("noise_seed", q["seed"]), 0)
    outs = (C.POINTER(sfft_result) * max(n, 1))()
    status = (C.c_int * max(n, 1))()
    rc = lib().sfft_dimincr_batch(params, samps, n, concurrency, outs, status)
    try:
        _check(rc)
        return [_convert(outs[i].contents) for i in range(n)]
    finally:
        for i in range(n):
            if outs[i]:
                lib().sfft_free(outs[i])

def lattice_noise(seed: int, t: int, rep: int, M, sigma: float, stream=None):
    """The planted sampler's noise for lattice sizes M (complex128 CUDA tensor [sum M])."""
    import torch
    M = _i64(M).reshape(-1)
    y = torch.empty(int(M.sum()), dtype=torch.complex128, device="cuda")
    _check(lib().mr1l_lattice_noise(seed, t, rep, M.shape[0], _ptr(M, C.c_int64), sigma,
                                    C.c_void_p(y.data_ptr()), C.c_void_p(_stream(stream))))
    return y


def select(p, cap: int, theta: float, theta_mode: str = "rel", eligible=None, flags=None, stream=None):
    """sfft_select: the thresholded "(up to) cap largest" selection of
    Algorithm 3 over the rows of p (complex128 CUDA [nrhs, n]); returns the
    uint8 flags [n] (1 where some row selects the index; OR-ed into `flags`
    when given)."""
    import torch
    p2 = p.reshape(-1, p.shape[-1]) if p.dim() > 0 else p
    if p2.dtype != torch.complex128 or not p2.is_cuda or not p2.is_contiguous():
        raise TypeError("p must be a contiguous complex128 CUDA tensor")
    n = p2.shape[1]
    if flags is None:
        flags = torch.zeros(n, dtype=torch.uint8, device=p.device)
    elif flags.dtype != torch.uint8 or tuple(flags.shape) != (n,) or flags.device != p.device or \
            not flags.is_contiguous():
        raise ValueError(f"flags must be a contiguous uint8 tensor of shape ({n},) on {p.device}")
    el = None
    if eligible is not None:
        if eligible.dtype != torch.uint8 or tuple(eligible.shape) != (n,) or eligible.device != p.device or \
                not eligible.is_contiguous():
            raise ValueError(f"eligible must be a contiguous uint8 tensor of shape ({n},) on {p.device}")
        el = C.c_void_p(eligible.data_ptr())
    _check(lib().sfft_select(C.c_void_p(p2.data_ptr()), n, p2.shape[0], el, cap, theta,
                             SFFT_THETA_REL if theta_mode == "rel" else SFFT_THETA_ABS, C.c_void_p(flags.data_ptr()),
                             C.c_void_p(_stream(stream))))
    return flags


def pool_stats(device: int = 0) -> dict:
    """The library's device block cache on `device`: {"outstanding", "cached",
    "mallocs"} (see mr1l_pool_stats)."""
    o, c, m = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().mr1l_pool_stats(device, C.byref(o), C.byref(c), C.byref(m)))
    return {"outstanding": o.value, "cached": c.value, "mallocs": m.value}


def inject_alloc_failure(after: int) -> None:
    """Test aid: the library's device allocation request `after` requests from
    now fails with MR1L_E_NOMEM (-1 cancels; see mr1l_inject_alloc_failure)."""
    _check(lib().mr1l_inject_alloc_failure(after))


def prof_enable(on: bool = True) -> None:
    """Bracket every library kernel launch with CUDA events (see mr1l_prof_read)."""
    _check(lib().mr1l_prof_enable(1 if on else 0))


def prof_reset() -> None:
    _check(lib().mr1l_prof_reset())


def prof_launches() -> int:
    """Kernel launches of the library since the last reset."""
    return int(lib().mr1l_prof_launches())


def prof_read() -> dict:
    """Per-kernel totals {name: {launches, ms, flops, bytes}} since the last reset."""
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(lib().mr1l_prof_read(buf, 1 << 16))
    return json.loads(buf.value.decode())


def tune_enable(on: bool = True) -> None:
    """Allow (or forbid) the tiling trials of the tile tuner (see mr1l_tune_enable)."""
    _check(lib().mr1l_tune_enable(1 if on else 0))


def tune_reset() -> None:
    """Forget every cached tile choice."""
    _check(lib().mr1l_tune_reset())


def tune_read() -> list:
    """The cached tile choices [{device, P, mode, df, col_tile, row_tile, col_ms, row_ms}, ...]."""
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(lib().mr1l_tune_read(buf, 1 << 16))
    return json.loads(buf.value.decode())


def theorem_params(d: int, supp: int, eps: float) -> tuple[int, int]:
    """(r, b) of the Section 4 theorem for failure probability eps (see sfft_theorem_params)."""
    r, b = C.c_int64(), C.c_int()
    _check(lib().sfft_theorem_params(d, supp, eps, C.byref(r), C.byref(b)))
    return int(r.value), int(b.value)


def _batch_arrays(plans, xs, width):
    import torch
    n = len(plans)
    hs = (C.c_void_p * max(n, 1))(*[p._h.value for p in plans])
    ins, outs, nr, keep = (C.c_void_p * max(n, 1))(), (C.c_void_p * max(n, 1))(), (C.c_int * max(n, 1))(), []
    for i, (p, x) in enumerate(zip(plans, xs)):
        x2 = x.reshape(-1, width(p, True))
        if x2.dtype != torch.complex128 or not x2.is_cuda or not x2.is_contiguous():
            raise TypeError("inputs must be contiguous complex128 CUDA tensors")
        o = torch.empty((x2.shape[0], width(p, False)), dtype=torch.complex128, device=x2.device)
        keep += [x2, o]
        ins[i], outs[i], nr[i] = x2.data_ptr(), o.data_ptr(), x2.shape[0]
    return hs, ins, outs, nr, keep


def reconstruct_batch(plans, ys, stream=None) -> list:
    """mr1l_reconstruct_batch: Algorithm 2 for each (plan, y) pair in one call."""
    hs, ins, outs, nr, keep = _batch_arrays(plans, ys, lambda p, inp: p.sum_M if inp else p.nI)
    _check(lib().mr1l_reconstruct_batch(hs, len(plans), ins, nr, outs, C.c_void_p(_stream(stream))))
    return keep[1::2]


def evaluate_batch(plans, cs, mode: int = MR1L_EVAL, stream=None) -> list:
    """mr1l_evaluate_batch: lattice evaluation (or the adjoint) for each (plan, c) pair in one call."""
    hs, ins, outs, nr, keep = _batch_arrays(plans, cs, lambda p, inp: p.nI if inp else p.sum_M)
    _check(lib().mr1l_evaluate_batch(hs, len(plans), ins, nr, outs, mode, C.c_void_p(_stream(stream))))
    return keep[1::2]

