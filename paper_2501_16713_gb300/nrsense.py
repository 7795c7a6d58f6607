"""Thin ctypes binding of libnrsense (include/nrsense.h).

Argument marshalling only: every step of the operator runs in the library's
CUDA kernels and cuFFT.  PyTorch provides device memory and streams.  If the
library is missing this module raises at load time: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnrsense.so")

OK = 0
ERR_ARG = -1
ERR_CUDA = -4
STATUS = {
    0: "ok", -1: "invalid argument", -2: "out of memory", -3: "cuFFT failure",
    -4: "CUDA runtime failure", -5: "CG breakdown", -6: "CG not converged",
    -7: "device wait timed out", -9: "call not valid for this plan",
}
FP32 = 0
BF16_STORE = 1
FP32_COMPENSATED = 2
IDENTITY_WARP = 1


class NrsenseError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {STATUS.get(code, 'unknown')} ({code})")
        self.code = code


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("osf", ctypes.c_int32),
                ("kb_width", ctypes.c_int32), ("kb_beta", ctypes.c_double),
                ("n_phases", ctypes.c_int32), ("n_coils", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("phase_chunk", ctypes.c_int32), ("grid", ctypes.c_int32 * 3)]


class Tuning(ctypes.Structure):
    _fields_ = [("spread_variant", ctypes.c_int32), ("interp_coils", ctypes.c_int32),
                ("interp_tma", ctypes.c_int32),
                ("spread_ms", ctypes.c_double * 3), ("interp_ms", ctypes.c_double * 2),
                ("interp_tma_ms", ctypes.c_double * 2),
                ("spread_image_warp", ctypes.c_int32),
                ("spread_image_ms", ctypes.c_double * 3),
                ("fft_pruned", ctypes.c_int32), ("fft_ms", ctypes.c_double * 2),
                ("spread_mma_ms", ctypes.c_double), ("spread_mma_wpc", ctypes.c_int32),
                ("spread_mma_cube", ctypes.c_int32), ("spread_mma_geo_ms", ctypes.c_double * 2),
                ("interp_tma2_ms", ctypes.c_double), ("spread_max_item", ctypes.c_int32),
                ("spread_item_ms", ctypes.c_double * 3),
                ("interp_image_home", ctypes.c_int32), ("interp_image_ms", ctypes.c_double * 2),
                ("image_fft_pruned", ctypes.c_int32), ("image_fft_ms", ctypes.c_double * 2)]


class Info(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32 * 3), ("kb_beta", ctypes.c_double),
                ("kernel_poly_err", ctypes.c_double), ("total_samples", ctypes.c_int64),
                ("tile", ctypes.c_int32 * 3), ("n_tiles", ctypes.c_int64),
                ("occupied_fraction", ctypes.c_double), ("spread_items", ctypes.c_int64),
                ("split_tiles", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("phase_chunk", ctypes.c_int32), ("union_fraction", ctypes.c_double),
                ("union_columns", ctypes.c_double)]


_VP = ctypes.c_void_p
_SIGS = {
    "nrsense_plan_create": [ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_int64), _VP, _VP, _VP,
                            _VP, ctypes.POINTER(_VP)],
    "nrsense_plan_destroy": [_VP],
    "nrsense_plan_info": [_VP, ctypes.POINTER(Info)],
    "nrsense_apply_forward": [_VP, _VP, _VP, _VP],
    "nrsense_apply_adjoint": [_VP, _VP, _VP, _VP],
    "nrsense_apply_normal": [_VP, _VP, ctypes.c_double, _VP, _VP],
    "nrsense_warp_forward": [_VP, _VP, _VP, _VP],
    "nrsense_warp_adjoint": [_VP, _VP, _VP, _VP],
    "nrsense_kspace_forward": [_VP, ctypes.c_int32, _VP, _VP, _VP],
    "nrsense_kspace_adjoint": [_VP, ctypes.c_int32, _VP, _VP, _VP],
    "nrsense_device_status": [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _VP],
    "nrsense_status_string": [ctypes.c_int32],
    "nrsense_profile_start": [_VP, ctypes.c_int32],
    "nrsense_profile_stop": [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_int64)],
    "nrsense_stage_name": [ctypes.c_int32],
    "nrsense_dot_noalloc": [_VP, _VP, ctypes.c_int64, _VP, _VP],
    "nrsense_solve_cg": [_VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                         ctypes.c_uint32, _VP, ctypes.POINTER(ctypes.c_int32),
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _VP],
    "nrsense_solve_cg_record": [_VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                ctypes.c_uint32, _VP, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                _VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _VP],
    "nrsense_solve_fcg": [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                          ctypes.c_uint32, _VP, ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_int32), _VP],
    "nrsense_plan_autotune": [_VP, ctypes.c_int32, ctypes.POINTER(Tuning), _VP],
    "nrsense_plan_set_tuning": [_VP, ctypes.POINTER(Tuning)],
    "nrsense_cnn_create": [ctypes.POINTER(ctypes.c_int32), ctypes.c_uint32, _VP,
                           ctypes.POINTER(_VP)],
    "nrsense_cnn_destroy": [_VP],
    "nrsense_cnn_num_params": [],
    "nrsense_cnn_init_params": [_VP, ctypes.c_uint64, _VP],
    "nrsense_cnn_set_params": [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int64, _VP],
    "nrsense_cnn_get_params": [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int64, _VP],
    "nrsense_cnn_apply": [_VP, _VP, _VP, _VP],
    "nrsense_cnn_gradients": [_VP, _VP, ctypes.c_double, _VP, _VP, ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_double), _VP],
    "nrsense_cnn_get_grads": [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int64, _VP],
    "nrsense_cnn_adam_step": [_VP, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_uint32, _VP],
    "nrsense_cnn_launches": [_VP, ctypes.POINTER(ctypes.c_int64)],
    "nrsense_wavelet_forward": [_VP, _VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, _VP],
    "nrsense_wavelet_inverse": [_VP, _VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, _VP],
    "nrsense_wavelet_shrink": [_VP, _VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                               ctypes.c_double, _VP],
    "nrsense_normal_max_eig": [_VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _VP],
    "nrsense_fista_lipschitz": [_VP, _VP, ctypes.c_int32, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_double), _VP],
    "nrsense_dcf": [_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP],
    "nrsense_set_circulant": [_VP, ctypes.c_double, ctypes.c_int32, _VP],
    "nrsense_apply_circulant": [_VP, _VP, _VP, _VP],
    "nrsense_apply_adjoint_weighted": [_VP, _VP, _VP, _VP, _VP],
    "nrsense_translation_xcorr": [_VP, _VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_double), _VP],
    "nrsense_phase_ramp": [_VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double), _VP],
    "nrsense_kmeans": [ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int32,
                       ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "nrsense_solve_fista": [_VP, _VP, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                            ctypes.c_int32, ctypes.c_uint32, _VP, ctypes.POINTER(ctypes.c_double),
                            _VP],
    "nrsense_plan_set_reduce": [_VP, _VP, _VP],
    "nrsense_copy_c64": [_VP, _VP, ctypes.c_int64, _VP],
    "nrsense_cnn_set_conv": [_VP, ctypes.c_int32],
    "nrsense_cnn_device_status": [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _VP],
    "nrsense_set_deflation": [_VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _VP],
    "nrsense_deflation_from_solve": [_VP, _VP, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int32), _VP],
    "nrsense_symmetric_eigen": [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
}
# nrsense_reduce_fn: (user, image_dev, n, stream) -> status
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_void_p)
CG_X0 = 1
CG_GRAPH = 2
CG_CIRCULANT = 4
CG_DEFLATE = 8
DEFLATE_LARGEST = 16
NUM_STAGES = 16
_STRING_RESULT = ("nrsense_status_string", "nrsense_stage_name")
_INT64_RESULT = ("nrsense_cnn_num_params",)
CNN_CHANNELS = (2, 16, 16, 16, 16, 2)
CNN_FREEZE_BIAS = 1
CNN_SYMMETRIC = 1

_lib = None


def load(path: str | None = None):
    """Load libnrsense.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libnrsense.so not built ({p}); run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = (ctypes.c_char_p if name in _STRING_RESULT else
                      ctypes.c_int64 if name in _INT64_RESULT else ctypes.c_int32)
    if path is None:
        _lib = lib
    return lib


def exported_symbols():
    return sorted(_SIGS)


def _check(code, where):
    if code != OK:
        raise NrsenseError(code, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


DOT_NOALLOC_MAX_N = 16384 * 4096


def dot_noalloc(x, y, out=None, stream=None):
    """<x, y> in FP64 through nrsense_dot_noalloc (no plan, no allocation by
    the library).  x, y: contiguous complex64 CUDA tensors of equal size on
    one device; out: a float64 CUDA tensor of 2 elements on that device
    (allocated here if omitted -- the library call itself allocates nothing).
    The call runs with x's device current (on that device's current stream
    unless `stream` is given).  Returns out."""
    import torch
    lib = load()
    _need(x, torch.complex64, None, "x")
    _need(y, torch.complex64, tuple(x.shape), "y")
    if y.device != x.device:
        raise ValueError(f"y is on {y.device}, x on {x.device}")
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=x.device)
    _need(out, torch.float64, (2,), "out")
    if out.device != x.device:
        raise ValueError(f"out is on {out.device}, x on {x.device}")
    with torch.cuda.device(x.device):
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        _check(lib.nrsense_dot_noalloc(_ptr(x), _ptr(y), int(x.numel()), _ptr(out),
                                       _stream(stream)),
               "nrsense_dot_noalloc")
    return out



def _wavelet(fn, where, a, levels, out, tau=None, stream=None):
    import torch
    lib = load()
    _need(a, torch.complex64, None, "input")
    if a.dim() != 3:
        raise ValueError("input must be a 3D image")
    if out is None:
        out = torch.empty_like(a)
    _need(out, torch.complex64, tuple(a.shape), "out")
    n = (ctypes.c_int32 * 3)(*a.shape)
    args = [_ptr(a), _ptr(out), n, int(levels)] + ([float(tau)] if tau is not None else [])
    _check(getattr(lib, fn)(*args, _stream(stream)), where)
    return out


def wavelet_forward(x, levels, out=None, stream=None):
    """W x: orthonormal 3D Haar pyramid with `levels` levels, Mallat layout."""
    return _wavelet("nrsense_wavelet_forward", "nrsense_wavelet_forward", x, levels, out,
                    stream=stream)


def wavelet_inverse(c, levels, out=None, stream=None):
    """W^H c for Mallat-layout coefficients c."""
    return _wavelet("nrsense_wavelet_inverse", "nrsense_wavelet_inverse", c, levels, out,
                    stream=stream)


def wavelet_shrink(v, tau, levels, out=None, stream=None):
    """W^H soft(W v, tau): the proximal map of tau ||W .||_1 (out may be v)."""
    return _wavelet("nrsense_wavelet_shrink", "nrsense_wavelet_shrink", v, levels, out, tau,
                    stream=stream)



def translation_xcorr(ref, imgs, stream=None):
    """Translations of each image against ref by magnitude cross-correlation
    (nrsense_translation_xcorr).  ref: (n0, n1, n2), imgs: (count, n0, n1, n2)
    complex64 CUDA tensors.  Returns a (count, 3) float64 numpy array."""
    import torch
    lib = load()
    _need(ref, torch.complex64, None, "ref")
    if ref.dim() != 3:
        raise ValueError("ref must be a 3D image")
    _need(imgs, torch.complex64, None, "imgs")
    if imgs.dim() != 4 or tuple(imgs.shape[1:]) != tuple(ref.shape):
        raise ValueError("imgs must be (count,) + ref.shape")
    count = int(imgs.shape[0])
    out = np.zeros((count, 3), dtype=np.float64)
    n = (ctypes.c_int32 * 3)(*ref.shape)
    _check(lib.nrsense_translation_xcorr(
        _ptr(ref), _ptr(imgs), n, count,
        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)),
        "nrsense_translation_xcorr")
    return out


def phase_ramp(coords, y, seg_off, shifts, stream=None):
    """In place: y[r] *= exp(+i omega_r . t_s) for the rows of segment s
    (nrsense_phase_ramp).  coords: (rows, 3) float32, y: (rows, C) complex64
    CUDA tensors; seg_off: nseg + 1 row offsets; shifts: (nseg, 3) voxels."""
    import torch
    lib = load()
    _need(coords, torch.float32, None, "coords")
    _need(y, torch.complex64, None, "y")
    if y.dim() != 2 or coords.dim() != 2 or coords.shape[1] != 3 or coords.shape[0] != y.shape[0]:
        raise ValueError("coords must be (rows, 3) and y (rows, C)")
    off = np.ascontiguousarray(np.asarray(seg_off, dtype=np.int64))
    sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64).reshape(-1, 3))
    if off.size != sh.shape[0] + 1 or off[-1] > y.shape[0]:
        raise ValueError("seg_off must hold nseg + 1 offsets within the rows")
    _check(lib.nrsense_phase_ramp(
        _ptr(coords), _ptr(y), int(y.shape[0]), int(y.shape[1]), int(sh.shape[0]),
        off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)),
        "nrsense_phase_ramp")
    return y


def kmeans(points, k, max_iter=100):
    """k-means of (n, 3) points (nrsense_kmeans, host).  Returns (labels,
    centres, inertia, iterations, reference cluster)."""
    lib = load()
    p = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    n = p.shape[0]
    labels = np.zeros(n, dtype=np.int32)
    centres = np.zeros((max(int(k), 1), 3), dtype=np.float64)
    inertia, iters, ref = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.nrsense_kmeans(p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, int(k),
                              int(max_iter), labels.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              centres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              ctypes.byref(inertia), ctypes.byref(iters), ctypes.byref(ref)),
           "nrsense_kmeans")
    return labels, centres, inertia.value, iters.value, ref.value

def symmetric_eigen(a):
    """Eigenvalues (ascending) and eigenvectors (columns) of a real symmetric
    matrix by the library's host Jacobi solver (nrsense_symmetric_eigen)."""
    lib = load()
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    m = a.shape[0]
    vals = np.zeros(m, dtype=np.float64)
    vecs = np.zeros((m, m), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.nrsense_symmetric_eigen(int(m), a.ctypes.data_as(dp), vals.ctypes.data_as(dp),
                                       vecs.ctypes.data_as(dp)), "nrsense_symmetric_eigen")
    return vals, vecs


class Plan:
    """Nonrigid SENSE operator A_j = G_j S T_j over P motion states.

    shape   image size (n0, n1, n2), each even
    disp    (P, 3, n0, n1, n2) float32 CUDA tensor (voxels), or None with
            identity_warp=True
    coords  list of P (M_j, 3) float32 CUDA tensors (radians), or None (no coils)
    smaps   (C, n0, n1, n2) complex64 CUDA tensor, or None (image-space only)
    """

    def __init__(self, shape, disp=None, coords=None, smaps=None, n_phases=None, osf=2,
                 width=4, beta=0.0, identity_warp=False, stream=None, phase_chunk=0,
                 precision=FP32):
        import torch
        self.lib = load()
        self.shape = tuple(int(s) for s in shape)
        if smaps is not None:
            _need(smaps, torch.complex64, None, "smaps")
            self.n_coils = int(smaps.shape[0])
        else:
            self.n_coils = 0
        if n_phases is None:
            n_phases = int(disp.shape[0]) if disp is not None else len(coords)
        self.n_phases = int(n_phases)
        if disp is not None:
            _need(disp, torch.float32, (self.n_phases, 3) + self.shape, "disp")
        d = Desc()
        d.n[:] = self.shape
        # sigma: an integer (G = osf n), or rational with G = osf n whole on every axis
        if float(osf).is_integer():
            d.osf = int(osf)
            self.osf = int(osf)
        else:
            g = [float(osf) * n for n in self.shape]
            if any(abs(v - round(v)) > 1e-9 for v in g):
                raise ValueError("osf * n must be an integer on every axis")
            d.osf = 0
            d.grid[:] = [int(round(v)) for v in g]
            self.osf = float(osf)
        d.kb_width, d.kb_beta = int(width), float(beta)
        d.n_phases, d.n_coils = self.n_phases, self.n_coils
        d.precision = int(precision)
        self.width, self.precision = int(width), int(precision)
        d.flags = IDENTITY_WARP if identity_warp else 0
        d.phase_chunk = int(phase_chunk)
        self.counts = [0] * self.n_phases
        cat = None
        if self.n_coils > 0:
            if coords is None or len(coords) != self.n_phases:
                raise ValueError("coords must list one (M_j, 3) tensor per phase")
            for c in coords:
                _need(c, torch.float32, None, "coords[j]")
            self.counts = [int(c.shape[0]) for c in coords]
            cat = torch.cat([c.reshape(-1, 3) for c in coords]).contiguous()
        self.offsets = np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)
        counts = (ctypes.c_int64 * self.n_phases)(*self.counts)
        h = ctypes.c_void_p()
        st = self.lib.nrsense_plan_create(ctypes.byref(d), counts, _ptr(cat), _ptr(disp),
                                          _ptr(smaps), _stream(stream), ctypes.byref(h))
        _check(st, "nrsense_plan_create")
        self._h = h
        self.total_samples = int(self.offsets[-1])

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self.lib.nrsense_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        inf = Info()
        _check(self.lib.nrsense_plan_info(self._h, ctypes.byref(inf)), "nrsense_plan_info")
        return {f: (list(getattr(inf, f)) if f in ("grid", "tile") else getattr(inf, f))
                for f, _ in Info._fields_}

    # -- operators -------------------------------------------------------
    def _img(self):
        import torch
        return torch.empty(self.shape, dtype=torch.complex64, device="cuda")

    def forward_shape(self):
        if self.n_coils == 0:
            return (self.n_phases,) + self.shape
        return (self.total_samples, self.n_coils)

    def forward(self, x, out=None, stream=None):
        import torch
        _need(x, torch.complex64, self.shape, "x")
        if out is None:
            out = torch.empty(self.forward_shape(), dtype=torch.complex64, device="cuda")
        _need(out, torch.complex64, self.forward_shape(), "out")
        _check(self.lib.nrsense_apply_forward(self._h, _ptr(x), _ptr(out), _stream(stream)),
               "nrsense_apply_forward")
        return out

    def adjoint(self, y, out=None, stream=None):
        import torch
        _need(y, torch.complex64, self.forward_shape(), "y")
        out = self._img() if out is None else out
        _need(out, torch.complex64, self.shape, "out")
        _check(self.lib.nrsense_apply_adjoint(self._h, _ptr(y), _ptr(out), _stream(stream)),
               "nrsense_apply_adjoint")
        return out

    def normal(self, x, lam=0.0, out=None, stream=None):
        import torch
        _need(x, torch.complex64, self.shape, "x")
        out = self._img() if out is None else out
        _need(out, torch.complex64, self.shape, "out")
        _check(self.lib.nrsense_apply_normal(self._h, _ptr(x), float(lam), _ptr(out),
                                             _stream(stream)), "nrsense_apply_normal")
        return out

    def warp_forward(self, x, out=None, stream=None):
        import torch
        _need(x, torch.complex64, self.shape, "x")
        if out is None:
            out = torch.empty((self.n_phases,) + self.shape, dtype=torch.complex64, device="cuda")
        _check(self.lib.nrsense_warp_forward(self._h, _ptr(x), _ptr(out), _stream(stream)),
               "nrsense_warp_forward")
        return out

    def warp_adjoint(self, m, out=None, stream=None):
        import torch
        _need(m, torch.complex64, (self.n_phases,) + self.shape, "m")
        out = self._img() if out is None else out
        _check(self.lib.nrsense_warp_adjoint(self._h, _ptr(m), _ptr(out), _stream(stream)),
               "nrsense_warp_adjoint")
        return out

    def kspace_forward(self, phase, v, out=None, stream=None):
        import torch
        _need(v, torch.complex64, (self.n_coils,) + self.shape, "v")
        if out is None:
            out = torch.empty((self.counts[phase], self.n_coils), dtype=torch.complex64,
                              device="cuda")
        _check(self.lib.nrsense_kspace_forward(self._h, int(phase), _ptr(v), _ptr(out),
                                               _stream(stream)), "nrsense_kspace_forward")
        return out

    def kspace_adjoint(self, phase, y, out=None, stream=None):
        import torch
        _need(y, torch.complex64, (self.counts[phase], self.n_coils), "y")
        if out is None:
            out = torch.empty((self.n_coils,) + self.shape, dtype=torch.complex64, device="cuda")
        _check(self.lib.nrsense_kspace_adjoint(self._h, int(phase), _ptr(y), _ptr(out),
                                               _stream(stream)), "nrsense_kspace_adjoint")
        return out

    def device_status(self, clear=True, stream=None):
        v = ctypes.c_int32()
        _check(self.lib.nrsense_device_status(self._h, int(bool(clear)), ctypes.byref(v),
                                              _stream(stream)), "nrsense_device_status")
        return v.value

    def profile_start(self, max_launches=65536):
        _check(self.lib.nrsense_profile_start(self._h, int(max_launches)), "nrsense_profile_start")

    def profile_stop(self):
        """Synchronise and return ({stage: (ms, launches)}, own kernel launches)."""
        ms = (ctypes.c_double * NUM_STAGES)()
        cnt = (ctypes.c_int64 * NUM_STAGES)()
        own = ctypes.c_int64()
        _check(self.lib.nrsense_profile_stop(self._h, ms, cnt, ctypes.byref(own)),
               "nrsense_profile_stop")
        names = [self.lib.nrsense_stage_name(i).decode() for i in range(NUM_STAGES)]
        return {n: (ms[i], cnt[i]) for i, n in enumerate(names)}, own.value

    def solve_cg(self, y, lam, tol=1e-4, maxit=100, x0=None, graph=False, stream=None,
                 check=True, out=None):
        """CG on (sum_j A_j^H A_j + lam I) x = sum_j A_j^H y_j.

        Returns (x, iterations, residual history, true relative residual,
        status code).  With check=True a breakdown raises; not reaching tol
        does not."""
        import torch
        _need(y, torch.complex64, self.forward_shape(), "y")
        if x0 is not None:
            _need(x0, torch.complex64, self.shape, "x0")
            if out is not None and out.data_ptr() != x0.data_ptr():
                out.copy_(x0)
                x = out
            else:
                x = x0
        else:
            x = self._img() if out is None else _need(out, torch.complex64, self.shape, "out")
        it = ctypes.c_int32()
        hist = (ctypes.c_double * (int(maxit) + 1))()
        tres = ctypes.c_double()
        flags = (CG_X0 if x0 is not None else 0) | (CG_GRAPH if graph else 0)
        code = self.lib.nrsense_solve_cg(self._h, _ptr(y), float(lam), float(tol), int(maxit),
                                         flags, _ptr(x), ctypes.byref(it), hist,
                                         ctypes.byref(tres), _stream(stream))
        if check and code not in (OK, -6):
            _check(code, "nrsense_solve_cg")
        return x, it.value, list(hist[: it.value + 1]), tres.value, code

    def _x_for(self, x0, out):
        import torch
        if x0 is not None:
            _need(x0, torch.complex64, self.shape, "x0")
            if out is not None and out.data_ptr() != x0.data_ptr():
                out.copy_(x0)
                return out
            return x0
        return self._img() if out is None else _need(out, torch.complex64, self.shape, "out")

    def solve_cg_record(self, y, lam, capacity, tol=1e-4, maxit=100, x0=None, stream=None,
                        check=True):
        """Plain CG that records training pairs of the preconditioner: for
        k < capacity, r_k (recursive residual) and e_k = x_final - x_k.

        Returns (x, iterations, residual history, true relative residual,
        status code, r (K, *shape), e (K, *shape)) with K pairs recorded."""
        import torch
        _need(y, torch.complex64, self.forward_shape(), "y")
        x = self._x_for(x0, None)
        cap = int(capacity)
        rec_r = torch.empty((max(cap, 1),) + self.shape, dtype=torch.complex64, device=y.device)
        rec_e = torch.empty_like(rec_r)
        it, cnt = ctypes.c_int32(), ctypes.c_int32()
        hist = (ctypes.c_double * (int(maxit) + 1))()
        tres = ctypes.c_double()
        flags = CG_X0 if x0 is not None else 0
        code = self.lib.nrsense_solve_cg_record(
            self._h, _ptr(y), float(lam), float(tol), int(maxit), flags, _ptr(x),
            ctypes.byref(it), hist, ctypes.byref(tres), _ptr(rec_r), _ptr(rec_e), cap,
            ctypes.byref(cnt), _stream(stream))
        if check and code not in (OK, -6):
            _check(code, "nrsense_solve_cg_record")
        k = cnt.value
        return (x, it.value, list(hist[: it.value + 1]), tres.value, code, rec_r[:k], rec_e[:k])

    def set_circulant(self, lam, enable=True, stream=None):
        """Build (or switch off) the circulant preconditioner for lambda
        (nrsense_set_circulant): one normal-operator application."""
        _check(self.lib.nrsense_set_circulant(self._h, float(lam), int(bool(enable)),
                                              _stream(stream)), "nrsense_set_circulant")

    def apply_circulant(self, r, out=None, stream=None):
        """z = M_c r with the circulant preconditioner (nrsense_apply_circulant)."""
        import torch
        _need(r, torch.complex64, self.shape, "r")
        out = self._img() if out is None else _need(out, torch.complex64, self.shape, "out")
        _check(self.lib.nrsense_apply_circulant(self._h, _ptr(r), _ptr(out), _stream(stream)),
               "nrsense_apply_circulant")
        return out

    def set_deflation(self, w, stream=None):
        """Deflation basis (nrsense_set_deflation): w a (k,) + shape complex64
        CUDA tensor, or None to switch deflation off.  Returns the number of
        basis vectors kept after orthonormalisation."""
        import torch
        kept = ctypes.c_int32()
        if w is None:
            _check(self.lib.nrsense_set_deflation(self._h, None, 0, ctypes.byref(kept),
                                                  _stream(stream)), "nrsense_set_deflation")
            return 0
        if not isinstance(w, torch.Tensor) or w.dim() != 4 or tuple(w.shape[1:]) != self.shape:
            raise ValueError(f"w must be (k,) + {self.shape}")
        _need(w, torch.complex64, tuple(w.shape), "w")
        _check(self.lib.nrsense_set_deflation(self._h, _ptr(w), int(w.shape[0]),
                                              ctypes.byref(kept), _stream(stream)),
               "nrsense_set_deflation")
        return kept.value

    def deflation_from_solve(self, y, lam, steps=60, k=16, circulant=True, largest=False,
                             stream=None):
        """Deflation basis from the k smallest (largest=True: largest) Ritz
        pairs of `steps` iterations of (circulant-preconditioned) CG on the
        data y (nrsense_deflation_from_solve).  Returns (Ritz values, number
        of basis vectors kept)."""
        import torch
        _need(y, torch.complex64, self.forward_shape(), "y")
        ritz = (ctypes.c_double * int(k))()
        kept = ctypes.c_int32()
        flags = (CG_CIRCULANT if circulant else 0) | (DEFLATE_LARGEST if largest else 0)
        _check(self.lib.nrsense_deflation_from_solve(
            self._h, _ptr(y), float(lam), int(steps), int(k), flags, ritz, ctypes.byref(kept),
            _stream(stream)), "nrsense_deflation_from_solve")
        return np.array(ritz[:]), kept.value

    def solve_fcg(self, y, lam, net=None, tol=1e-4, maxit=100, x0=None, graph=False, stream=None,
                  check=True, out=None, circulant=False, deflate=False):
        """Flexible CG preconditioned by the network `net` (a Cnn, or None)
        and, with circulant=True, by the circulant preconditioner first
        (set_circulant must have been called); deflate=True projects out the
        plan's deflation space (set_deflation / deflation_from_solve).

        Returns (x, iterations, residual history, true relative residual,
        status code, fallbacks)."""
        import torch
        _need(y, torch.complex64, self.forward_shape(), "y")
        x = self._x_for(x0, out)
        it, fb = ctypes.c_int32(), ctypes.c_int32()
        hist = (ctypes.c_double * (int(maxit) + 1))()
        tres = ctypes.c_double()
        flags = ((CG_X0 if x0 is not None else 0) | (CG_GRAPH if graph else 0)
                 | (CG_CIRCULANT if circulant else 0) | (CG_DEFLATE if deflate else 0))
        code = self.lib.nrsense_solve_fcg(
            self._h, None if net is None else net._h, _ptr(y), float(lam), float(tol), int(maxit),
            flags, _ptr(x), ctypes.byref(it), hist, ctypes.byref(tres), ctypes.byref(fb),
            _stream(stream))
        if check and code not in (OK, -6):
            _check(code, "nrsense_solve_fcg")
        return x, it.value, list(hist[: it.value + 1]), tres.value, code, fb.value

    def tuning_key(self):
        """Key of the autotuning cache: geometry, sizes, precision, device."""
        import torch
        i = self.info()
        dev = torch.cuda.get_device_name(torch.cuda.current_device())
        return (f"{self.shape}|C{self.n_coils}|P{self.n_phases}|W{self.width}|osf{self.osf}|"
                f"prec{self.precision}|M{self.total_samples}|chunk{i['phase_chunk']}|{dev}")

    def autotune(self, reps=3, cache=None, stream=None):
        """Pick the faster k-space spreading and interpolation launch choices
        (nrsense_plan_autotune).  cache: path of a JSON file of earlier
        choices keyed by tuning_key(); read if it has this key, else tuned
        here and written back.  Returns the choices (and times when tuned)."""
        import json
        key = self.tuning_key()
        store = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                store = json.load(f)
        if key in store:
            t = Tuning()
            t.spread_variant = int(store[key]["spread_variant"])
            t.interp_coils = int(store[key]["interp_coils"])
            t.interp_tma = int(store[key].get("interp_tma", 0))
            t.spread_image_warp = int(store[key].get("spread_image_warp", 0))
            t.fft_pruned = int(store[key].get("fft_pruned", 0))
            t.spread_mma_wpc = int(store[key].get("spread_mma_wpc", 1))
            t.spread_mma_cube = int(store[key].get("spread_mma_cube", 0))
            t.spread_max_item = int(store[key].get("spread_max_item", 0))
            t.interp_image_home = int(store[key].get("interp_image_home", 0))
            t.image_fft_pruned = int(store[key].get("image_fft_pruned", 0))
            _check(self.lib.nrsense_plan_set_tuning(self._h, ctypes.byref(t)),
                   "nrsense_plan_set_tuning")
            return dict(store[key], cached=True)
        t = Tuning()
        _check(self.lib.nrsense_plan_autotune(self._h, int(reps), ctypes.byref(t), _stream(stream)),
               "nrsense_plan_autotune")
        res = {"spread_variant": t.spread_variant, "interp_coils": t.interp_coils,
               "interp_tma": t.interp_tma, "spread_ms": list(t.spread_ms),
               "interp_ms": list(t.interp_ms), "interp_tma_ms": list(t.interp_tma_ms),
               "spread_image_warp": t.spread_image_warp,
               "spread_image_ms": list(t.spread_image_ms),
               "fft_pruned": t.fft_pruned, "fft_ms": list(t.fft_ms),
               "spread_mma_ms": t.spread_mma_ms, "spread_mma_wpc": t.spread_mma_wpc,
               "spread_mma_cube": t.spread_mma_cube,
               "spread_mma_geo_ms": list(t.spread_mma_geo_ms),
               "interp_tma2_ms": t.interp_tma2_ms, "spread_max_item": t.spread_max_item,
               "spread_item_ms": list(t.spread_item_ms),
               "interp_image_home": t.interp_image_home,
               "interp_image_ms": list(t.interp_image_ms),
               "image_fft_pruned": t.image_fft_pruned, "image_fft_ms": list(t.image_fft_ms)}
        if cache:
            store[key] = res
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(store, f, indent=1)
            os.replace(tmp, cache)
        return dict(res, cached=False)

    def dcf(self, phase, iters=10, out=None, stream=None):
        """Pipe-Menon density compensation weights of one phase's samples
        (nrsense_dcf).  Returns a float32 CUDA tensor of M_phase values."""
        import torch
        m = int(self.counts[phase])
        if out is None:
            out = torch.empty(m, dtype=torch.float32, device="cuda")
        _need(out, torch.float32, (m,), "out")
        _check(self.lib.nrsense_dcf(self._h, int(phase), int(iters), _ptr(out), _stream(stream)),
               "nrsense_dcf")
        return out

    def adjoint_weighted(self, y, w, out=None, stream=None):
        """sum_j A_j^H (w . y_j) with one weight per sample (rows of y)."""
        import torch
        _need(y, torch.complex64, self.forward_shape(), "y")
        _need(w, torch.float32, (int(y.shape[0]),), "w")
        out = self._img() if out is None else _need(out, torch.complex64, self.shape, "out")
        _check(self.lib.nrsense_apply_adjoint_weighted(self._h, _ptr(y), _ptr(w), _ptr(out),
                                                       _stream(stream)),
               "nrsense_apply_adjoint_weighted")
        return out

    def set_reduce(self, fn):
        """Register the reduction of this plan's phase sums over ranks
        (nrsense_plan_set_reduce).  fn(buf, stream) must replace the complex64
        image tensor `buf` by the sum of every rank's image, in stream order on
        `stream` (a torch.cuda.ExternalStream of the library's stream); the
        image is staged in `buf` and copied back by the library's own copy.
        fn = None removes the hook."""
        import torch
        if fn is None:
            _check(self.lib.nrsense_plan_set_reduce(self._h, None, None), "nrsense_plan_set_reduce")
            self._reduce = None
            return
        buf = torch.empty(self.shape, dtype=torch.complex64, device="cuda")
        lib = self.lib

        def tramp(user, ptr, n, stream):
            try:
                if n != buf.numel():
                    return ERR_ARG
                s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                sp = ctypes.c_void_p(stream)
                if lib.nrsense_copy_c64(_ptr(buf), ctypes.c_void_p(ptr), n, sp) != OK:
                    return ERR_CUDA
                with torch.cuda.stream(s):
                    fn(buf, s)
                return lib.nrsense_copy_c64(ctypes.c_void_p(ptr), _ptr(buf), n, sp)
            except Exception:  # noqa: BLE001 - a failure must reach the C caller as a status
                return ERR_CUDA

        cb = REDUCE_FN(tramp)
        _check(self.lib.nrsense_plan_set_reduce(self._h, ctypes.cast(cb, ctypes.c_void_p), None),
               "nrsense_plan_set_reduce")
        self._reduce = (cb, buf)  # kept alive while registered

    def max_eig(self, v0, iters=30, stream=None):
        """Power iteration on sum_j A_j^H A_j from v0 (overwritten with the
        last normalised iterate).  Returns (Rayleigh quotient, v)."""
        import torch
        _need(v0, torch.complex64, self.shape, "v0")
        e = ctypes.c_double()
        _check(self.lib.nrsense_normal_max_eig(self._h, _ptr(v0), int(iters), ctypes.byref(e),
                                               _stream(stream)), "nrsense_normal_max_eig")
        return e.value, v0

    def lipschitz(self, iters=30, seed=0, margin=1.02, stream=None):
        """The FISTA step bound L = 2 margin lambda_max(sum_j A_j^H A_j)
        (nrsense_fista_lipschitz), power iteration from a seeded random start."""
        import torch
        g = torch.Generator(device="cuda").manual_seed(int(seed))
        v = torch.randn(self.shape, dtype=torch.complex64, device="cuda", generator=g)
        L = ctypes.c_double()
        _check(self.lib.nrsense_fista_lipschitz(self._h, _ptr(v), int(iters), float(margin),
                                                ctypes.byref(L), _stream(stream)),
               "nrsense_fista_lipschitz")
        return L.value

    def solve_fista(self, y, lam, levels=3, L=None, maxit=400, x0=None, graph=True, stream=None,
                    out=None):
        """Wavelet-FISTA on ||y - A x||^2 + lam ||W x||_1 (W: orthonormal 3D
        Haar with `levels` levels).  L: step bound (>= 2 lambda_max of the
        normal operator; estimated with lipschitz() when omitted).
        Returns (x, history of ||x_k - x_{k-1}|| / ||x_k||, L)."""
        import torch
        _need(y, torch.complex64, self.forward_shape(), "y")
        x = self._x_for(x0, out)
        if L is None:
            L = self.lipschitz(stream=stream)
        hist = (ctypes.c_double * max(int(maxit), 1))()
        flags = (CG_X0 if x0 is not None else 0) | (CG_GRAPH if graph else 0)
        _check(self.lib.nrsense_solve_fista(self._h, _ptr(y), float(lam), int(levels), float(L),
                                            int(maxit), flags, _ptr(x), hist, _stream(stream)),
               "nrsense_solve_fista")
        return x, list(hist[: int(maxit)]), float(L)

    def phase_slice(self, y, j):
        """Rows of phase j in a stacked (sum M_j, C) k-space array."""
        return y[int(self.offsets[j]):int(self.offsets[j + 1])]


class Cnn:
    """Preconditioner network M of flexible CG (include/nrsense.h,
    nrsense_cnn_*): 3x3x3 convolutions 2 -> 16 -> 16 -> 16 -> 16 -> 2 with
    ReLU between, residual output, BF16 tensor-core kernels.  symmetric=True
    (the default) selects z = u0 + N4^T (I + W5^T W5) N4 u0 (symmetric
    positive definite for fixed ReLU masks, biases unused); False the plain
    z = u0 + N(u0)."""

    def __init__(self, shape, seed=None, symmetric=True, stream=None):
        self.lib = load()
        self.shape = tuple(int(v) for v in shape)
        self.symmetric = bool(symmetric)
        n = (ctypes.c_int32 * 3)(*self.shape)
        h = ctypes.c_void_p()
        _check(self.lib.nrsense_cnn_create(n, CNN_SYMMETRIC if symmetric else 0, _stream(stream),
                                           ctypes.byref(h)),
               "nrsense_cnn_create")
        self._h = h
        self.n_params = int(self.lib.nrsense_cnn_num_params())
        if seed is not None:
            self.init(seed, stream)

    def close(self):
        if getattr(self, "_h", None):
            self.lib.nrsense_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, seed, stream=None):
        _check(self.lib.nrsense_cnn_init_params(self._h, int(seed), _stream(stream)),
               "nrsense_cnn_init_params")

    @staticmethod
    def flatten(params):
        """[(W (cout, cin, 3, 3, 3), b (cout)), ...] -> flat float32 array."""
        return np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(),
                                               np.asarray(b, np.float32).ravel()])
                               for w, b in params])

    @staticmethod
    def unflatten(flat):
        out, k = [], 0
        for cin, cout in zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:]):
            nw = cout * cin * 27
            out.append((flat[k:k + nw].reshape(cout, cin, 3, 3, 3).copy(),
                        flat[k + nw:k + nw + cout].copy()))
            k += nw + cout
        return out

    def set_params(self, params, stream=None):
        flat = np.ascontiguousarray(self.flatten(params) if not isinstance(params, np.ndarray)
                                    else params, dtype=np.float32)
        if flat.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {flat.size}")
        fp = flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        _check(self.lib.nrsense_cnn_set_params(self._h, fp, flat.size, _stream(stream)),
               "nrsense_cnn_set_params")

    def _download(self, fn, where, stream):
        flat = np.empty(self.n_params, np.float32)
        fp = flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        _check(fn(self._h, fp, flat.size, _stream(stream)), where)
        return flat

    def get_params(self, stream=None):
        return self.unflatten(self._download(self.lib.nrsense_cnn_get_params,
                                             "nrsense_cnn_get_params", stream))

    def get_grads(self, stream=None):
        return self.unflatten(self._download(self.lib.nrsense_cnn_get_grads,
                                             "nrsense_cnn_get_grads", stream))

    def apply(self, r, out=None, stream=None):
        import torch
        _need(r, torch.complex64, self.shape, "r")
        z = torch.empty_like(r) if out is None else _need(out, torch.complex64, self.shape, "out")
        _check(self.lib.nrsense_cnn_apply(self._h, _ptr(r), _ptr(z), _stream(stream)),
               "nrsense_cnn_apply")
        return z

    def gradients(self, r, e, accumulate=False, want_loss=True, plan=None, lam=0.0, stream=None):
        """Forward + backward for one pair; returns the loss (or None).
        plan=None: cosine loss; a Plan: energy loss with E = normal(., lam)."""
        import torch
        _need(r, torch.complex64, self.shape, "r")
        _need(e, torch.complex64, self.shape, "e")
        loss = ctypes.c_double()
        _check(self.lib.nrsense_cnn_gradients(self._h, None if plan is None else plan._h,
                                              float(lam), _ptr(r), _ptr(e),
                                              1 if accumulate else 0,
                                              ctypes.byref(loss) if want_loss else None,
                                              _stream(stream)),
               "nrsense_cnn_gradients")
        return loss.value if want_loss else None

    def adam_step(self, lr, grad_scale=1.0, beta1=0.9, beta2=0.999, eps=1e-8, freeze_bias=False,
                  stream=None):
        _check(self.lib.nrsense_cnn_adam_step(self._h, float(lr), float(grad_scale), float(beta1),
                                              float(beta2), float(eps),
                                              CNN_FREEZE_BIAS if freeze_bias else 0,
                                              _stream(stream)),
               "nrsense_cnn_adam_step")

    def launches(self):
        v = ctypes.c_int64()
        _check(self.lib.nrsense_cnn_launches(self._h, ctypes.byref(v)), "nrsense_cnn_launches")
        return v.value

    def set_conv(self, tcgen05):
        """Convolutions on the tcgen05 tensor cores (True) or mma.sync (False)
        (nrsense_cnn_set_conv)."""
        _check(self.lib.nrsense_cnn_set_conv(self._h, 1 if tcgen05 else 0), "nrsense_cnn_set_conv")

    def device_status(self, clear=True, stream=None):
        """The network's device status word (nrsense_cnn_device_status)."""
        v = ctypes.c_int32()
        _check(self.lib.nrsense_cnn_device_status(self._h, int(bool(clear)), ctypes.byref(v),
                                                  _stream(stream)), "nrsense_cnn_device_status")
        return v.value
