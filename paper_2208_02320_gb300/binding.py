"""ctypes binding of libhh (include/hh.h): argument marshalling only.

Every computation runs in the CUDA library. If libhh.so has not been built,
or no CUDA device is present, the calls raise; there is no CPU fallback.
Arrays may be numpy arrays (host) or CUDA torch tensors (passed by device
pointer on the context's stream).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhh.so")

HH_OK = 0
HH_WARN_NOT_CONVERGED = 1
HH_WARN_TARGET_UNMET = 2
HH_ERR_ARG = -1
HH_ERR_OOM = -2
HH_ERR_CUDA = -3
HH_ERR_NONFINITE = -4
HH_ERR_DEVICE_TIMEOUT = -5
HH_ERR_BAD_STIFFNESS = -6
HH_ERR_UNSUPPORTED = -7
HH_FP32, HH_FP64 = 0, 1
HH_CG, HH_BASIC, HH_EYRE_MILTON = 0, 1, 2
HH_NYQ_ZERO_COMPONENT, HH_NYQ_ZERO_MODE = 0, 1


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("nyquist", ctypes.c_int),
        ("fixed_iters", ctypes.c_int),
        ("ref_lambda", ctypes.c_double),
        ("ref_mu", ctypes.c_double),
        ("workspace_bytes", ctypes.c_int64),
        ("use_graphs", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("replace", ctypes.c_int),
        ("max_restarts", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("plane_smem_limit", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("wave_boxes", ctypes.c_int),
        ("fused", ctypes.c_int),
        ("shape_kernels", ctypes.c_int),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("C", ctypes.c_double * 36),
        ("C_sym", ctypes.c_double * 36),
        ("K", ctypes.c_double),
        ("G", ctypes.c_double),
        ("K_reuss", ctypes.c_double),
        ("G_reuss", ctypes.c_double),
        ("K_am", ctypes.c_double),
        ("G_am", ctypes.c_double),
        ("iters_max", ctypes.c_int),
        ("n_subimages", ctypes.c_int),
        ("n_surrogate_accepted", ctypes.c_int),
        ("n_clipped", ctypes.c_int),
        ("resid_max", ctypes.c_double),
        ("voxel_iters", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
        ("device_ms", ctypes.c_double),
        ("status", ctypes.c_int),
        ("n_fused", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        return dict(C=np.array(self.C).reshape(6, 6), C_sym=np.array(self.C_sym).reshape(6, 6),
                    K=self.K, G=self.G, K_reuss=self.K_reuss, G_reuss=self.G_reuss,
                    K_am=self.K_am, G_am=self.G_am, iters_max=self.iters_max,
                    n_subimages=self.n_subimages, n_surrogate_accepted=self.n_surrogate_accepted,
                    n_clipped=self.n_clipped, resid_max=self.resid_max,
                    voxel_iters=self.voxel_iters, kernel_launches=self.kernel_launches,
                    device_ms=self.device_ms, status=self.status, n_fused=self.n_fused)


class KernelStat(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("launches", ctypes.c_longlong),
        ("sampled", ctypes.c_longlong),
        ("sampled_ms", ctypes.c_double),
        ("sampled_bytes", ctypes.c_double),
    ]


class Phase(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double), ("G", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGNATURES = {
    "hh_version": (ctypes.c_char_p, []),
    "hh_status_string": (ctypes.c_char_p, [_I]),
    "hh_last_error": (ctypes.c_char_p, [_P]),
    "hh_options_default": (_I, [_P]),
    "hh_create": (_I, [_P, _I, _P]),
    "hh_destroy": (None, [_P]),
    "hh_homogenize_direct": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _P, _P]),
    "hh_homogenize_hierarchical": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _I, _I, _P, _P, _P, _P]),
    "hh_homogenize_partition": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _P, _I, _I, _P, _P, _P, _P]),
    "hh_solve_subimages": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P, _P, _P]),
    "hh_homogenize_aniso": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "hh_apply_operator": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _P]),
    "hh_extract_subimages": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _P, ctypes.c_int64]),
    "hh_extrapolate": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _P, _I, _I, _P, _P, _P, _P, _P, _P]),
    "hh_fit_inverse_n": (_I, [_P, _P, _P, _I, _P, _P]),
    "hh_profile_read": (_I, [_P, _P, _I, _P]),
    "hh_profile_reset": (_I, [_P]),
    "hh_apply_operator_noalloc": (_I, [_P, _P, _I, _I, _I, _I, _P, _P, _I, _P]),
    "hh_cnn_num_params": (ctypes.c_int64, []),
    "hh_cnn_init_params": (_I, [ctypes.c_uint64, _P]),
    "hh_cnn_forward": (_I, [_P, _P, _I, _P, _P, _P]),
    "hh_cnn_loss_grad": (_I, [_P, _P, _I, _P, _P, _P, _P, _P]),
    "hh_surrogate_train": (_I, [_P, _P, _I, _P, _P, _P, _I, _I, _D, ctypes.c_uint64, _P, _P]),
    "hh_surrogate_predict": (_I, [_P, _P, _I, _P, _P, _I, _D, _P]),
    "hh_surrogate_gate": (_I, [_P, _P, _I, _P, _P, _I, _P, _I, _D, _P, _P]),
    "hh_surrogate_save": (_I, [ctypes.c_char_p, _P, _I, _D]),
    "hh_surrogate_load": (_I, [ctypes.c_char_p, _P, ctypes.c_int64, _P, _P]),
    "hh_correlation": (_I, [_P, _P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P]),
    "hh_plan_partition": (_I, [_I, _I, _I, _I, _P, _P, _I, _D, _D, _P, _P, _P, _P]),
    "hh_set_memory_limit": (_I, [_P, ctypes.c_int64]),
    "hh_homogenize_multilevel": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _P, _P, _I, _P, _P]),
    "hh_homogenize_partition_surrogate": (_I, [_P, _P, _I, _I, _I, _I, _P, _I, _P, _I, _I, _P, _I, _D, _D, _D,
                                               ctypes.c_uint64, _P, _P, _P, _P, _P]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libhh.so (built by paper_2208_02320_gb300._build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhh.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def options(**kw) -> Options:
    o = Options()
    load().hh_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp32": HH_FP32, "fp64": HH_FP64}[v]
        if k == "scheme" and isinstance(v, str):
            v = {"cg": HH_CG, "basic": HH_BASIC, "em": HH_EYRE_MILTON}[v]
        if k == "nyquist" and isinstance(v, str):
            v = {"component": HH_NYQ_ZERO_COMPONENT, "mode": HH_NYQ_ZERO_MODE}[v]
        setattr(o, k, v)
    return o


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _u8(img):
    """(pointer, on_device, keepalive) for a uint8 image [z][y][x]."""
    if _is_torch_cuda(img):
        import torch
        t = img.contiguous()
        if t.dtype != torch.uint8:
            raise TypeError("image must be uint8")
        return ctypes.c_void_p(t.data_ptr()), 1, t
    a = np.ascontiguousarray(img, dtype=np.uint8)
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


def _phases(phases):
    ph = np.asarray(phases, dtype=np.float64).reshape(-1, 2)
    arr = (Phase * len(ph))(*[Phase(float(k), float(g)) for k, g in ph])
    return arr, len(ph)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def cnn_init_params(seed: int) -> np.ndarray:
    """He-uniform initial network parameters from the SplitMix64 draws of
    `seed` (hh_cnn_init_params; no GPU needed)."""
    lib = load()
    th = np.zeros(lib.hh_cnn_num_params(), dtype=np.float32)
    s = lib.hh_cnn_init_params(int(seed) & (2**64 - 1), _ptr(th))
    if s != HH_OK:
        raise HHError(s, lib.hh_last_error(None).decode())
    return th


def plan_partition(shape, n_min: int, bs, c_rel, a: float = 3.66, eps: float = 0.01) -> dict:
    """Subimage edge n and buffer b of least predicted cost whose predicted
    relative error c_rel[i] / n is at most eps (hh_plan_partition; no GPU
    needed). shape = (nz, ny, nx) of the image; c_rel[i] = |C_b| / M_inf
    fitted at buffer bs[i]. `met` is False when no candidate meets eps (the
    least-error candidate is returned)."""
    lib = load()
    nz, ny, nx = (int(v) for v in shape)
    b_arr = np.ascontiguousarray(bs, dtype=np.int32)
    c_arr = np.ascontiguousarray(c_rel, dtype=np.float64)
    if b_arr.size != c_arr.size:
        raise ValueError("bs and c_rel must have the same length")
    n, b, err, cost = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    s = lib.hh_plan_partition(nx, ny, nz, int(n_min), _ptr(b_arr), _ptr(c_arr), int(b_arr.size), float(a),
                              float(eps), ctypes.byref(n), ctypes.byref(b), ctypes.byref(err), ctypes.byref(cost))
    if s < 0:
        raise HHError(s, lib.hh_last_error(None).decode())
    return dict(n=n.value, b=b.value, err=err.value, cost=cost.value, met=s == HH_OK)


def surrogate_save(path: str, params_ensemble, scale: float) -> None:
    """Write an ensemble (params[ensemble][n_params] FP32) and its output
    scale to an ensemble file (hh_surrogate_save; no GPU needed)."""
    lib = load()
    th = np.ascontiguousarray(params_ensemble, dtype=np.float32)
    ens = th.shape[0] if th.ndim == 2 else 1
    if th.size != ens * lib.hh_cnn_num_params():
        raise ValueError("params_ensemble must hold ensemble x hh_cnn_num_params() values")
    s = lib.hh_surrogate_save(os.fsencode(path), _ptr(th), ens, float(scale))
    if s != HH_OK:
        raise HHError(s, lib.hh_last_error(None).decode())


def surrogate_load(path: str):
    """(params[ensemble][n_params] FP32, scale) from an ensemble file."""
    lib = load()
    ens, sc = ctypes.c_int(), ctypes.c_double()
    s = lib.hh_surrogate_load(os.fsencode(path), None, 0, ctypes.byref(ens), ctypes.byref(sc))
    if s == HH_OK:
        th = np.zeros((ens.value, lib.hh_cnn_num_params()), dtype=np.float32)
        s = lib.hh_surrogate_load(os.fsencode(path), _ptr(th), th.size, ctypes.byref(ens), ctypes.byref(sc))
    if s != HH_OK:
        raise HHError(s, lib.hh_last_error(None).decode())
    return th, sc.value


class Context:
    """A libhh context on one CUDA device (optionally bound to a CUDA stream)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self._lib = load()
        self._h = ctypes.c_void_p()
        s = self._lib.hh_create(ctypes.byref(self._h), int(device), ctypes.c_void_p(stream or 0))
        if s != HH_OK:
            raise HHError(s, "hh_create: " + self._lib.hh_last_error(None).decode())

    def set_memory_limit(self, nbytes: int):
        """Cap the context's device workspace (hh_set_memory_limit; 0 = none)."""
        self._check(self._lib.hh_set_memory_limit(self._h, int(nbytes)), "hh_set_memory_limit", allow_warn=False)

    def close(self):
        if self._h:
            self._lib.hh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s: int, what: str, allow_warn: bool = True):
        if s < 0 or (s > 0 and not allow_warn):
            raise HHError(s, f"{what}: {self._lib.hh_last_error(self._h).decode()}")
        return s

    # -------------------------------------------------------------- solves
    def homogenize_direct(self, img, phases, **opt) -> dict:
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        ph, nph = _phases(phases)
        o = options(**opt)
        r = Result()
        s = self._lib.hh_homogenize_direct(self._h, p, nx, ny, nz, dev, ph, nph, ctypes.byref(o), ctypes.byref(r))
        self._check(s, "hh_homogenize_direct")
        return r.as_dict()

    def homogenize_hierarchical(self, img, phases, n: int, b: int = 0, **opt) -> dict:
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        ph, nph = _phases(phases)
        o = options(**opt)
        nbox = (nx // n) * (ny // n) * (nz // n) if n > 0 and nx % n == 0 and ny % n == 0 and nz % n == 0 else 0
        Cb = np.zeros((max(nbox, 1), 6, 6))
        It = np.zeros((max(nbox, 1), 6), dtype=np.int32)
        r = Result()
        s = self._lib.hh_homogenize_hierarchical(self._h, p, nx, ny, nz, dev, ph, nph, int(n), int(b),
                                                 ctypes.byref(o), ctypes.byref(r), _ptr(Cb), _ptr(It))
        self._check(s, "hh_homogenize_hierarchical")
        d = r.as_dict()
        d.update(C_boxes=Cb[:nbox], iters_boxes=It[:nbox])
        return d

    def homogenize_partition(self, img, phases, boxes, unit: int = 0, **opt) -> dict:
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        ph, nph = _phases(phases)
        bx = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 7)
        o = options(**opt)
        Cb = np.zeros((len(bx), 6, 6))
        It = np.zeros((len(bx), 6), dtype=np.int32)
        r = Result()
        s = self._lib.hh_homogenize_partition(self._h, p, nx, ny, nz, dev, ph, nph, _ptr(bx), len(bx), int(unit),
                                              ctypes.byref(o), ctypes.byref(r), _ptr(Cb), _ptr(It))
        self._check(s, "hh_homogenize_partition")
        d = r.as_dict()
        d.update(C_boxes=Cb, iters_boxes=It)
        return d

    def solve_subimages(self, img, phases, boxes, **opt) -> dict:
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        ph, nph = _phases(phases)
        bx = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 7)
        o = options(**opt)
        nb = len(bx)
        C = np.zeros((nb, 6, 6))
        S = np.zeros((nb, 6, 6))
        E = np.zeros((nb, 6, 6))
        It = np.zeros((nb, 6), dtype=np.int32)
        Rs = np.zeros((nb, 6))
        s = self._lib.hh_solve_subimages(self._h, p, nx, ny, nz, dev, ph, nph, _ptr(bx), nb, ctypes.byref(o),
                                         _ptr(C), _ptr(S), _ptr(E), _ptr(It), _ptr(Rs))
        st = self._check(s, "hh_solve_subimages")
        return dict(C=C, Sigma=S, Eps=E, iters=It, resid=Rs, status=st)

    def homogenize_aniso(self, C21, **opt) -> dict:
        if _is_torch_cuda(C21):
            t = C21.contiguous()
            ptr, dev, keep = ctypes.c_void_p(t.data_ptr()), 1, t
            shape = tuple(t.shape)
        else:
            keep = np.ascontiguousarray(C21, dtype=np.float64)
            ptr, dev, shape = _ptr(keep), 0, keep.shape
        assert shape[0] == 21
        nz, ny, nx = shape[1:]
        o = options(**opt)
        r = Result()
        s = self._lib.hh_homogenize_aniso(self._h, ptr, nx, ny, nz, dev, ctypes.byref(o), ctypes.byref(r))
        self._check(s, "hh_homogenize_aniso")
        return r.as_dict()

    def apply_operator(self, p_field, labels=None, phases=None, C21=None, **opt) -> np.ndarray:
        pf = np.ascontiguousarray(p_field, dtype=np.float64)
        nz, ny, nx = pf.shape[1:]
        q = np.zeros_like(pf)
        o = options(**opt)
        if C21 is not None:
            c = np.ascontiguousarray(C21, dtype=np.float64)
            s = self._lib.hh_apply_operator(self._h, None, None, 0, _ptr(c), nx, ny, nz, _ptr(pf), _ptr(q),
                                            ctypes.byref(o))
        else:
            lab = np.ascontiguousarray(labels, dtype=np.uint8)
            ph, nph = _phases(phases)
            s = self._lib.hh_apply_operator(self._h, _ptr(lab), ph, nph, None, nx, ny, nz, _ptr(pf), _ptr(q),
                                            ctypes.byref(o))
        self._check(s, "hh_apply_operator", allow_warn=False)
        return q

    def extract_subimages(self, img, boxes) -> list:
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        bx = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 7)
        dims = [(int(r[5]) + 2 * int(r[6]), int(r[4]) + 2 * int(r[6]), int(r[3]) + 2 * int(r[6])) for r in bx]
        tot = sum(a * b * c for a, b, c in dims)
        out = np.zeros(max(tot, 1), dtype=np.uint8)
        s = self._lib.hh_extract_subimages(self._h, p, nx, ny, nz, dev, _ptr(bx), len(bx), _ptr(out), out.size)
        self._check(s, "hh_extract_subimages", allow_warn=False)
        res, o = [], 0
        for d in dims:
            n = d[0] * d[1] * d[2]
            res.append(out[o:o + n].reshape(d))
            o += n
        return res

    def extrapolate(self, img, phases, ns, b: int = 0, **opt) -> dict:
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        ph, nph = _phases(phases)
        nsa = np.ascontiguousarray(ns, dtype=np.int32)
        o = options(**opt)
        per = (Result * len(nsa))()
        out = [ctypes.c_double() for _ in range(4)]
        s = self._lib.hh_extrapolate(self._h, p, nx, ny, nz, dev, ph, nph, _ptr(nsa), len(nsa), int(b),
                                     ctypes.byref(o), *[ctypes.byref(v) for v in out], per)
        self._check(s, "hh_extrapolate")
        return dict(K_inf=out[0].value, C_K=out[1].value, G_inf=out[2].value, C_G=out[3].value,
                    per_n=[r.as_dict() for r in per])

    def fit_inverse_n(self, ns, M):
        nsa = np.ascontiguousarray(ns, dtype=np.int32)
        Ma = np.ascontiguousarray(M, dtype=np.float64)
        mi, c = ctypes.c_double(), ctypes.c_double()
        s = self._lib.hh_fit_inverse_n(self._h, _ptr(nsa), _ptr(Ma), len(nsa), ctypes.byref(mi), ctypes.byref(c))
        self._check(s, "hh_fit_inverse_n", allow_warn=False)
        return mi.value, c.value

    # ----- subimage surrogate (3D CNN, BF16 tensor cores) -----
    def cnn_num_params(self) -> int:
        return int(self._lib.hh_cnn_num_params())

    @staticmethod
    def _subs(labels, cores=None):
        """(concatenated labels, boxes[count][9] int32, count) of subimages given
        as a 4-D array [count][nz][ny][nx] or a list of 3-D arrays, with cores
        (ox, oy, oz, cnx, cny, cnz) per subimage (None: the whole box)."""
        subs = [np.ascontiguousarray(l, dtype=np.uint8) for l in (labels if isinstance(labels, (list, tuple))
                                                                  else np.asarray(labels).reshape(
                                                                      (-1,) + np.asarray(labels).shape[-3:]))]
        rows = []
        for i, l in enumerate(subs):
            nz, ny, nx = l.shape
            c = (0, 0, 0, nx, ny, nz) if cores is None or cores[i] is None else tuple(int(v) for v in cores[i])
            rows.append((nx, ny, nz) + c)
        return (np.concatenate([l.ravel() for l in subs]), np.ascontiguousarray(rows, dtype=np.int32).reshape(-1, 9),
                len(subs))

    def cnn_forward(self, labels, params, cores=None):
        lab, bx, n = self._subs(labels, cores)
        th = np.ascontiguousarray(params, dtype=np.float32)
        out = np.zeros((n, 21), dtype=np.float32)
        self._check(self._lib.hh_cnn_forward(self._h, _ptr(lab), n, _ptr(bx), _ptr(th), _ptr(out)), "hh_cnn_forward",
                    allow_warn=False)
        return out

    def cnn_loss_grad(self, labels, params, targets, cores=None):
        lab, bx, n = self._subs(labels, cores)
        th = np.ascontiguousarray(params, dtype=np.float32)
        tg = np.ascontiguousarray(targets, dtype=np.float32).reshape(n, 21)
        loss = ctypes.c_double()
        grad = np.zeros(th.size, dtype=np.float32)
        self._check(self._lib.hh_cnn_loss_grad(self._h, _ptr(lab), n, _ptr(bx), _ptr(th), _ptr(tg), ctypes.byref(loss),
                                               _ptr(grad)), "hh_cnn_loss_grad", allow_warn=False)
        return loss.value, grad

    def surrogate_train(self, labels, targets, init, epochs=10, batch=32, lr=1e-3, seed=0, cores=None):
        lab, bx, n = self._subs(labels, cores)
        tg = np.ascontiguousarray(targets, dtype=np.float32).reshape(n, 21)
        th0 = np.ascontiguousarray(init, dtype=np.float32)
        out = np.zeros(th0.size, dtype=np.float32)
        hist = np.zeros(epochs)
        self._check(self._lib.hh_surrogate_train(self._h, _ptr(lab), n, _ptr(bx), _ptr(tg), _ptr(th0), int(epochs),
                                                 int(batch), float(lr), int(seed), _ptr(out), _ptr(hist)),
                    "hh_surrogate_train", allow_warn=False)
        return out, hist

    def surrogate_predict(self, labels, params_ensemble, scale, cores=None):
        lab, bx, n = self._subs(labels, cores)
        th = np.ascontiguousarray(params_ensemble, dtype=np.float32)
        ens = th.shape[0] if th.ndim == 2 else 1
        out = np.zeros((n, ens, 21), dtype=np.float32)
        self._check(self._lib.hh_surrogate_predict(self._h, _ptr(lab), n, _ptr(bx), _ptr(th), ens, float(scale),
                                                   _ptr(out)), "hh_surrogate_predict", allow_warn=False)
        return out

    def surrogate_gate(self, labels, phases, members, spread=0.01, cores=None):
        lab, bx, n = self._subs(labels, cores)
        ph, nph = _phases(phases)
        mem = np.ascontiguousarray(members, dtype=np.float32)
        ens = mem.shape[1]
        acc = np.zeros(n, dtype=np.int32)
        c21 = np.zeros((n, 21))
        self._check(self._lib.hh_surrogate_gate(self._h, _ptr(lab), n, _ptr(bx), ph, nph, _ptr(mem), ens, float(spread),
                                                _ptr(acc), _ptr(c21)), "hh_surrogate_gate", allow_warn=False)
        return acc.astype(bool), c21

    def correlation(self, img, pore_label: int, lmax: int) -> dict:
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        counts = np.zeros((3, lmax + 1), dtype=np.int64)
        corr = np.zeros((3, lmax + 1))
        xi = np.zeros(3)
        n_min = ctypes.c_int()
        self._check(self._lib.hh_correlation(self._h, p, nx, ny, nz, dev, int(pore_label), int(lmax), _ptr(counts),
                                             _ptr(corr), _ptr(xi), ctypes.byref(n_min)), "hh_correlation",
                    allow_warn=False)
        return dict(counts=counts, corr=corr, xi=xi, n_min=n_min.value)

    def homogenize_multilevel(self, img, phases, levels, **opt) -> dict:
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        ph, nph = _phases(phases)
        ns = np.ascontiguousarray([lv[0] for lv in levels], dtype=np.int32)
        bs = np.ascontiguousarray([lv[1] for lv in levels], dtype=np.int32)
        o = options(**opt)
        r = Result()
        s = self._lib.hh_homogenize_multilevel(self._h, p, nx, ny, nz, dev, ph, nph, _ptr(ns), _ptr(bs), len(ns),
                                               ctypes.byref(o), ctypes.byref(r))
        self._check(s, "hh_homogenize_multilevel")
        return r.as_dict()

    def homogenize_partition_surrogate(self, img, phases, boxes, params_ensemble, unit=None, scale=100.0,
                                       spread=0.01, audit=0.0, audit_seed=0, **opt) -> dict:
        """accepted: the gate's decisions; audited: the accepted subimages the
        FFT solver also solved (fraction `audit`, SplitMix64 draws seeded with
        `audit_seed`); audit_err: the prediction's relative K/G error there
        (NaN elsewhere)."""
        p, dev, keep = _u8(img)
        nz, ny, nx = img.shape
        ph, nph = _phases(phases)
        bx = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 7)
        th = np.ascontiguousarray(params_ensemble, dtype=np.float32)
        ens = th.shape[0] if th.ndim == 2 else 1
        if unit is None:
            unit = 0  # the library derives the coarse unit from the partition
        o = options(**opt)
        r = Result()
        nb = len(bx)
        Cb = np.zeros((nb, 6, 6))
        acc = np.zeros(nb, dtype=np.int32)
        err = np.zeros(nb)
        s = self._lib.hh_homogenize_partition_surrogate(self._h, p, nx, ny, nz, dev, ph, nph, _ptr(bx), nb, int(unit),
                                                        _ptr(th), ens, float(scale), float(spread), float(audit),
                                                        int(audit_seed) & (2**64 - 1), ctypes.byref(o),
                                                        ctypes.byref(r), _ptr(Cb), _ptr(acc), _ptr(err))
        self._check(s, "hh_homogenize_partition_surrogate")
        d = r.as_dict()
        d.update(C_boxes=Cb, accepted=acc > 0, audited=acc == 2, audit_err=np.where(acc == 2, err, np.nan))
        return d

    def profile(self) -> dict:
        arr = (KernelStat * 64)()
        n = ctypes.c_int()
        self._check(self._lib.hh_profile_read(self._h, arr, 64, ctypes.byref(n)), "hh_profile_read")
        return {arr[i].name.decode(): dict(launches=arr[i].launches, sampled=arr[i].sampled,
                                           sampled_ms=arr[i].sampled_ms, sampled_bytes=arr[i].sampled_bytes)
                for i in range(min(n.value, 64))}

    def profile_reset(self):
        self._check(self._lib.hh_profile_reset(self._h), "hh_profile_reset")

    # raw status calls (tests of the error paths)
    def raw(self):
        return self._lib, self._h
