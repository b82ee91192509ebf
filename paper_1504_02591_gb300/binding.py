"""Thin ctypes binding of the C ABI in include/recon.h (argument marshalling only).

Every step of the reconstruction runs in the CUDA kernels of librecon_gb300.so.  There is no CPU
path: if the library is missing, or no CUDA device is present, the calls raise.  PyTorch supplies
device memory (the workspace and output tensors) and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librecon_gb300.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_STATE, ERR_TIMEOUT, \
    ERR_UNSUPPORTED = range(9)
LOS_RADIAL, LOS_FIXED = 0, 1
MEAN_RANDOMS, MEAN_UNIFORM = 0, 1
F64, F32 = 0, 1
START_PLAIN, START_APPROX1, START_FFTA = 0, 1, 2
FIELD_RHO_G, FIELD_RHO_R, FIELD_DELTA, FIELD_DELTA_K, FIELD_PSI = range(5)

# every symbol include/recon.h declares
ABI_SYMBOLS = (
    "recon_workspace_bytes", "recon_create", "recon_deposit", "recon_smooth", "recon_iterate",
    "recon_get_trace", "recon_shift", "recon_get_psi", "recon_get_field", "recon_get_scalars",
    "recon_fft_r2c", "recon_fft_c2r", "recon_destroy", "recon_status_str", "recon_last_error",
    "recon_set_timing", "recon_get_timing", "recon_reset_timing", "recon_cic_deposit_noalloc",
    "recon_set_option", "recon_reconfigure", "recon_batch_run", "recon_batch_plan",
    "recon_unet_param_count", "recon_unet_create", "recon_unet_set_params", "recon_unet_get_params",
    "recon_unet_get_grads", "recon_unet_forward", "recon_unet_backward", "recon_unet_adamw",
    "recon_unet_destroy", "recon_unet_last_error", "recon_unet_set_option", "recon_unet_get_layer",
    "recon_unet_launch_count",
    "recon_iterate_from", "recon_start_features",
    "recon_get_radial", "recon_radial_ratio", "recon_ratio_stats", "recon_helmholtz_x",
    "recon_radial_nbar", "recon_fkp_weights", "recon_fd_solve", "recon_start_coefficient",
)
OPT_DEPOSIT_PATH, OPT_SHIFT_PATH, OPT_GRAPH, OPT_LINE_TILE, OPT_KSPACE_GENERIC, OPT_REUSE_SORT = 0, 1, 2, 3, 4, 5
OPT_PLANE_BATCH, OPT_ASSIGN, OPT_KITER_TMA, OPT_FFT_RADIX = 6, 7, 8, 9
ASSIGN_CIC, ASSIGN_NGP = 0, 1
UNET_OPT_TENSOR_CORES = 0
PATH_DIRECT, PATH_SORTED = 0, 1
BATCH_TUNE, BATCH_ONE_GRAPH = 1, 2
KERNEL_KINDS = ("deposit", "z_fwd", "z_inv", "z_delta", "z_proj", "z_final", "line_fwd", "line_inv",
                "conv", "k_delta", "k_iter", "shift", "other", "sort")


class ReconParams(C.Structure):
    _fields_ = [("nmesh", C.c_int * 3), ("box", C.c_double * 3), ("b", C.c_double), ("f", C.c_double),
                ("smooth_R", C.c_double), ("los_mode", C.c_int), ("observer", C.c_double * 3),
                ("periodic", C.c_int), ("mask_frac", C.c_double), ("lognormal", C.c_int),
                ("mean_density_mode", C.c_int)]


class ReconCatalog(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("w", C.c_void_p), ("n", C.c_int64), ("dtype", C.c_int),
                ("on_device", C.c_int)]


class ReconBatchItem(C.Structure):
    _fields_ = [("params", ReconParams), ("gal", ReconCatalog), ("ran", ReconCatalog), ("start", C.c_int),
                ("tol", C.c_double), ("max_iter", C.c_int), ("shift_gal", C.c_void_p), ("shift_ran", C.c_void_p),
                ("out_on_device", C.c_int), ("n_iter", C.c_int), ("rel", C.c_double), ("status", C.c_int),
                ("ms", C.c_float)]


class ReconError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load librecon_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    P, VP, I, D = C.POINTER, C.c_void_p, C.c_int, C.c_double
    lib.recon_workspace_bytes.argtypes = [P(ReconParams), P(C.c_size_t)]
    lib.recon_create.argtypes = [P(ReconParams), VP, VP, C.c_size_t, P(VP)]
    lib.recon_deposit.argtypes = [VP, P(ReconCatalog), P(ReconCatalog)]
    lib.recon_smooth.argtypes = [VP]
    lib.recon_iterate.argtypes = [VP, I, D, I, P(I), P(D)]
    lib.recon_get_trace.argtypes = [VP, P(D), I, P(I)]
    lib.recon_shift.argtypes = [VP, P(ReconCatalog), I, VP, VP, I]
    lib.recon_get_psi.argtypes = [VP, VP, I]
    lib.recon_get_field.argtypes = [VP, I, VP, I]
    lib.recon_get_scalars.argtypes = [VP, P(D)]
    lib.recon_fft_r2c.argtypes = [VP, VP, VP]
    lib.recon_fft_c2r.argtypes = [VP, VP, VP]
    lib.recon_destroy.argtypes = [VP]
    lib.recon_set_timing.argtypes = [VP, I]
    lib.recon_get_timing.argtypes = [VP, I, P(D), P(C.c_int64), P(D)]
    lib.recon_reset_timing.argtypes = [VP]
    lib.recon_set_option.argtypes = [VP, I, I]
    lib.recon_reconfigure.argtypes = [VP, P(ReconParams)]
    lib.recon_batch_run.argtypes = [P(ReconBatchItem), I, VP, I]
    lib.recon_batch_plan.argtypes = [I, P(I), P(I), P(I), P(I)]
    lib.recon_iterate_from.argtypes = [VP, VP, I, D, I, P(I), P(D)]
    lib.recon_start_features.argtypes = [VP, I, I, VP]
    lib.recon_get_radial.argtypes = [VP, I, VP]
    lib.recon_unet_param_count.argtypes = [I, P(C.c_size_t)]
    lib.recon_unet_create.argtypes = [I, I, VP, P(VP)]
    lib.recon_unet_set_params.argtypes = [VP, VP, C.c_size_t]
    lib.recon_unet_get_params.argtypes = [VP, VP, C.c_size_t]
    lib.recon_unet_get_grads.argtypes = [VP, VP, C.c_size_t]
    lib.recon_unet_forward.argtypes = [VP, VP, I, VP]
    lib.recon_unet_backward.argtypes = [VP, VP, VP, I, P(D)]
    lib.recon_unet_adamw.argtypes = [VP, C.c_float, C.c_float]
    lib.recon_unet_destroy.argtypes = [VP]
    lib.recon_unet_set_option.argtypes = [VP, C.c_int, C.c_int]
    lib.recon_unet_get_layer.argtypes = [VP, C.c_int, VP, C.c_size_t]
    lib.recon_unet_launch_count.argtypes = [VP, C.POINTER(C.c_longlong)]
    lib.recon_unet_last_error.argtypes = [VP]
    lib.recon_unet_last_error.restype = C.c_char_p
    lib.recon_fd_solve.argtypes = [VP, D, I, P(I), P(D), VP]
    lib.recon_start_coefficient.argtypes = [I, D, P(D)]
    lib.recon_radial_nbar.argtypes = [VP, P(ReconCatalog), I, D, D, D, P(D)]
    lib.recon_fkp_weights.argtypes = [VP, P(ReconCatalog), I, D, D, P(D), D, VP]
    lib.recon_radial_ratio.argtypes = [VP, VP, VP, P(ReconCatalog), D, D, P(D)]
    lib.recon_ratio_stats.argtypes = [VP, VP, VP, C.c_int64, D, D, P(D)]
    lib.recon_helmholtz_x.argtypes = [VP, VP, VP, VP]
    lib.recon_cic_deposit_noalloc.argtypes = [VP, I, VP, C.c_int64, I, D, VP, VP, VP]
    lib.recon_status_str.argtypes = [I]
    lib.recon_status_str.restype = C.c_char_p
    lib.recon_last_error.argtypes = [VP]
    lib.recon_last_error.restype = C.c_char_p
    for name in ABI_SYMBOLS:
        if name not in ("recon_status_str", "recon_last_error", "recon_unet_last_error"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def make_params(n, L, b, f, R, observer, los_mode=LOS_RADIAL, periodic=False, mask_frac=0.01,
                lognormal=False, uniform=False) -> ReconParams:
    p = ReconParams()
    p.nmesh[:] = (int(n),) * 3
    p.box[:] = (float(L),) * 3
    p.b, p.f, p.smooth_R = float(b), float(f), float(R)
    p.los_mode = int(los_mode)
    p.observer[:] = tuple(float(v) for v in observer)
    p.periodic = int(bool(periodic))
    p.mask_frac = float(mask_frac)
    p.lognormal = int(bool(lognormal))
    p.mean_density_mode = MEAN_UNIFORM if uniform else MEAN_RANDOMS
    return p


def start_coefficient(start: int, beta: float) -> float:
    """recon_start_coefficient: the coefficient c of a start for beta = f / b."""
    lib = load()
    c = C.c_double()
    st = lib.recon_start_coefficient(start, beta, C.byref(c))
    if st != OK:
        raise ReconError(st, "recon_start_coefficient: " + lib.recon_status_str(st).decode())
    return c.value


def workspace_bytes(params: ReconParams) -> int:
    lib = load()
    out = C.c_size_t(0)
    st = lib.recon_workspace_bytes(C.byref(params), C.byref(out))
    if st != OK:
        raise ReconError(st, "recon_workspace_bytes: " + lib.recon_status_str(st).decode())
    return out.value


def _catalog(pos, w, keep):
    """Build a recon_catalog from a torch tensor (CUDA or CPU) or a numpy array."""
    import torch
    cat = ReconCatalog()
    if pos is None:
        return None
    if isinstance(pos, np.ndarray):
        pos = np.ascontiguousarray(pos)
        if pos.dtype not in (np.float64, np.float32) or pos.ndim != 2 or pos.shape[1] != 3:
            raise ValueError("positions must be (n, 3) float64 or float32")
        keep.append(pos)
        cat.pos = pos.ctypes.data if len(pos) else None
        cat.n = len(pos)
        cat.dtype = F64 if pos.dtype == np.float64 else F32
        cat.on_device = 0
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float32)
            keep.append(w)
            cat.w = w.ctypes.data
        return cat
    if not isinstance(pos, torch.Tensor):
        raise TypeError("positions must be a torch.Tensor or numpy.ndarray")
    pos = pos.contiguous()
    if pos.dtype not in (torch.float64, torch.float32) or pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError("positions must be (n, 3) float64 or float32")
    keep.append(pos)
    cat.pos = pos.data_ptr() if pos.numel() else None
    cat.n = pos.shape[0]
    cat.dtype = F64 if pos.dtype == torch.float64 else F32
    cat.on_device = int(pos.is_cuda)
    if w is not None:
        w = w.to(device=pos.device, dtype=torch.float32).contiguous()
        keep.append(w)
        cat.w = w.data_ptr()
    return cat


def _host_ptr(x):
    """Address of a host numpy array or CPU torch tensor (pinned or not)."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Recon:
    """One reconstruction context (a recon_handle) on the current CUDA device and stream."""

    def __init__(self, n, L, b, f, R, observer, los_mode=LOS_RADIAL, periodic=False, mask_frac=0.01,
                 lognormal=False, uniform=False, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the reconstruction runs only on the GPU")
        self.lib = load()
        self.params = make_params(n, L, b, f, R, observer, los_mode, periodic, mask_frac, lognormal,
                                  uniform)
        self.n = int(n)
        self.uniform = bool(uniform)
        self.ws_bytes = workspace_bytes(self.params)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = self.lib.recon_create(C.byref(self.params), C.c_void_p(self.stream.cuda_stream),
                                   C.c_void_p(self.workspace.data_ptr()), self.ws_bytes, C.byref(h))
        self._check(st, "recon_create", handle=False)
        self.h = h

    @classmethod
    def from_mock(cls, mock, **over):
        p = mock.params(**over)
        return cls(p["n"], p["L"], p["b"], p["f"], p["R"], p["observer"], p["los_mode"],
                   p["periodic"], p["mask_frac"], p["lognormal"], p["uniform"])

    def _check(self, st, what, handle=True, allow=()):
        if st == OK or st in allow:
            return st
        msg = f"{what}: {self.lib.recon_status_str(st).decode()}"
        if handle and getattr(self, "h", None):
            extra = self.lib.recon_last_error(self.h).decode()
            if extra:
                msg += f" ({extra})"
        raise ReconError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.recon_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- pipeline --------------------------------------------------------------------------------
    def deposit(self, gal_pos, gal_w=None, ran_pos=None, ran_w=None):
        keep = []
        g = _catalog(gal_pos, gal_w, keep)
        r = _catalog(ran_pos, ran_w, keep)
        st = self.lib.recon_deposit(self.h, C.byref(g), C.byref(r) if r is not None else None)
        self._check(st, "recon_deposit")

    def smooth(self):
        self._check(self.lib.recon_smooth(self.h), "recon_smooth")

    def iterate(self, start=START_PLAIN, tol=0.0, max_iter=6):
        """Returns (n_iter, rel, status); status is OK or ERR_NOT_CONVERGED."""
        n = C.c_int(0)
        rel = C.c_double(0)
        st = self.lib.recon_iterate(self.h, int(start), float(tol), int(max_iter), C.byref(n), C.byref(rel))
        self._check(st, "recon_iterate", allow=(ERR_NOT_CONVERGED,))
        return n.value, rel.value, st

    def iterate_from(self, u0, tol=0.0, max_iter=6, level=0):
        """Iterate from a supplied radial displacement (CUDA tensor): level 0 on the mesh, level 1/2
        a prediction of the block means after start_features(level); (n_iter, rel, status)."""
        import torch
        u0 = u0.to(device="cuda", dtype=torch.float32).contiguous()
        n = C.c_int(0)
        rel = C.c_double(0)
        st = self.lib.recon_iterate_from(self.h, C.c_void_p(u0.data_ptr()), int(level), float(tol), int(max_iter),
                                         C.byref(n), C.byref(rel))
        self._check(st, "recon_iterate_from", allow=(ERR_NOT_CONVERGED,))
        return n.value, rel.value, st

    def start_features(self, start=START_FFTA, level=0):
        """(M, M, M, 5) CUDA tensor of network inputs (delta, r, u_s) block means, M = N >> level."""
        import torch
        m = self.n >> level
        feat = torch.empty((m, m, m, 5), dtype=torch.float32, device="cuda")
        self._check(self.lib.recon_start_features(self.h, int(start), int(level), C.c_void_p(feat.data_ptr())),
                    "recon_start_features")
        return feat

    def get_radial(self, level=0):
        import torch
        m = self.n >> level
        u = torch.empty((m, m, m), dtype=torch.float32, device="cuda")
        self._check(self.lib.recon_get_radial(self.h, int(level), C.c_void_p(u.data_ptr())), "recon_get_radial")
        return u

    def trace(self):
        buf = (C.c_double * 4096)()
        n = C.c_int(0)
        self._check(self.lib.recon_get_trace(self.h, buf, 4096, C.byref(n)), "recon_get_trace")
        return [buf[i] for i in range(min(n.value, 4096))]

    def shift(self, pos, is_galaxy, want_pos=False, out=None, pos_out=None):
        """Shift vectors (n, 3) float32 (and shifted positions (n, 3) float64 if want_pos).
        Outputs live where the positions live (CUDA tensors for CUDA input, numpy for host)."""
        import torch
        keep = []
        cat = _catalog(pos, None, keep)
        n = cat.n
        on_dev = bool(cat.on_device)
        if on_dev:
            sh = out if out is not None else torch.empty((n, 3), dtype=torch.float32, device="cuda")
            po = (pos_out if pos_out is not None else torch.empty((n, 3), dtype=torch.float64, device="cuda")) \
                if want_pos else None
            sp, pp = sh.data_ptr(), (po.data_ptr() if po is not None else None)
        else:
            sh = out if out is not None else np.empty((n, 3), dtype=np.float32)
            po = (pos_out if pos_out is not None else np.empty((n, 3), dtype=np.float64)) if want_pos else None
            sp, pp = _host_ptr(sh), (_host_ptr(po) if po is not None else None)
        st = self.lib.recon_shift(self.h, C.byref(cat), int(bool(is_galaxy)), C.c_void_p(sp),
                                  C.c_void_p(pp) if pp else None, int(on_dev))
        self._check(st, "recon_shift")
        return (sh, po) if want_pos else sh

    # -- the finite-difference method (Sec. 2.1) ------------------------------------------------
    def fd_solve(self, tol=1e-6, max_iter=200):
        """Eq. mainpot by finite differences after smooth(): (Psi (3, N, N, N) CUDA, iterations,
        true relative residual, status)."""
        import torch
        psi = torch.empty((3, self.n, self.n, self.n), dtype=torch.float32, device="cuda")
        it = C.c_int(0)
        res = C.c_double(0)
        st = self.lib.recon_fd_solve(self.h, float(tol), int(max_iter), C.byref(it), C.byref(res),
                                     C.c_void_p(psi.data_ptr()))
        self._check(st, "recon_fd_solve", allow=(ERR_NOT_CONVERGED,))
        return psi, it.value, res.value, st

    # -- the paper's front end: n(r) and FKP weights ---------------------------------------------
    def radial_nbar(self, pos, nbins, rmin, rmax, sky_area):
        """n(r) (numpy, nbins) of the particles pos (CUDA (n, 3)) about the handle's observer."""
        keep = []
        cat = _catalog(pos, None, keep)
        out = (C.c_double * int(nbins))()
        self._check(self.lib.recon_radial_nbar(self.h, C.byref(cat), int(nbins), float(rmin), float(rmax),
                                               float(sky_area), out), "recon_radial_nbar")
        return np.array(out[:], dtype=np.float64)

    def fkp_weights(self, pos, nbar, rmin, rmax, P0=20000.0):
        """FKP weights (CUDA float32 (n,)) of the particles pos for the shells' nbar."""
        import torch
        keep = []
        cat = _catalog(pos, None, keep)
        nb = np.ascontiguousarray(nbar, dtype=np.float64)
        w = torch.empty(cat.n, dtype=torch.float32, device="cuda")
        self._check(self.lib.recon_fkp_weights(self.h, C.byref(cat), len(nb), float(rmin), float(rmax),
                                               nb.ctypes.data_as(C.POINTER(C.c_double)), float(P0),
                                               C.c_void_p(w.data_ptr())), "recon_fkp_weights")
        return w

    # -- the paper's diagnostics -----------------------------------------------------------------
    def radial_ratio(self, psi_num, psi_den, pos, lo=-1.0, hi=3.0):
        """Eq. ratio at the particles pos (CUDA (n, 3)): (mean, std, outlier fraction, kept)."""
        keep = []
        cat = _catalog(pos, None, keep)
        a = psi_num.contiguous()
        b = psi_den.contiguous()
        out = (C.c_double * 4)()
        self._check(self.lib.recon_radial_ratio(self.h, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                                C.byref(cat), float(lo), float(hi), out), "recon_radial_ratio")
        return out[0], out[1], out[2], int(out[3])

    def ratio_stats(self, num, den, lo=-1.0, hi=3.0):
        """Ratio statistics of two CUDA float32 arrays: (mean, std, outlier fraction, kept)."""
        a = num.contiguous()
        b = den.contiguous()
        out = (C.c_double * 4)()
        self._check(self.lib.recon_ratio_stats(self.h, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                               a.numel(), float(lo), float(hi), out), "recon_ratio_stats")
        return out[0], out[1], out[2], int(out[3])

    def helmholtz_x(self, psi_x):
        """Sec. 4.1 split of (Psi.x) x: (grad_A, curl_B), each a (3, N, N, N) CUDA tensor."""
        import torch
        x = psi_x.to(device="cuda", dtype=torch.float32).contiguous()
        ga = torch.empty((3, self.n, self.n, self.n), dtype=torch.float32, device="cuda")
        cb = torch.empty_like(ga)
        self._check(self.lib.recon_helmholtz_x(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(ga.data_ptr()),
                                               C.c_void_p(cb.data_ptr())), "recon_helmholtz_x")
        return ga, cb

    # -- accessors -------------------------------------------------------------------------------
    def get_psi(self):
        import torch
        out = torch.empty((3, self.n, self.n, self.n), dtype=torch.float32, device="cuda")
        self._check(self.lib.recon_get_psi(self.h, C.c_void_p(out.data_ptr()), 1), "recon_get_psi")
        return out

    def get_field(self, which):
        import torch
        n = self.n
        if which == FIELD_DELTA_K:
            out = torch.empty((n, n, n // 2 + 1, 2), dtype=torch.float32, device="cuda")
        elif which == FIELD_PSI:
            out = torch.empty((3, n, n, n), dtype=torch.float32, device="cuda")
        else:
            out = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        self._check(self.lib.recon_get_field(self.h, int(which), C.c_void_p(out.data_ptr()), 1),
                    "recon_get_field")
        if which == FIELD_DELTA_K:
            return torch.view_as_complex(out)
        return out

    def scalars(self):
        buf = (C.c_double * 8)()
        self._check(self.lib.recon_get_scalars(self.h, buf), "recon_get_scalars")
        keys = ("sum_wg", "sum_wr", "alpha", "threshold", "lognormal_C", "n_mask", "norm_d2", "norm_s2")
        return dict(zip(keys, list(buf)))

    def set_option(self, option, value):
        self._check(self.lib.recon_set_option(self.h, int(option), int(value)), "recon_set_option")

    def set_timing(self, enable: bool):
        self._check(self.lib.recon_set_timing(self.h, int(bool(enable))), "recon_set_timing")

    def reset_timing(self):
        self._check(self.lib.recon_reset_timing(self.h), "recon_reset_timing")

    def timing(self):
        """{kind: (launches, total_ms, algorithmic_bytes)} for every kernel kind."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            ms = C.c_double(0)
            cnt = C.c_int64(0)
            by = C.c_double(0)
            self._check(self.lib.recon_get_timing(self.h, k, C.byref(ms), C.byref(cnt), C.byref(by)),
                        "recon_get_timing")
            out[name] = (cnt.value, ms.value, by.value)
        return out

    def fft_r2c(self, x):
        import torch
        x = x.to(device="cuda", dtype=torch.float32).contiguous()
        n = self.n
        out = torch.empty((n, n, n // 2 + 1, 2), dtype=torch.float32, device="cuda")
        self._check(self.lib.recon_fft_r2c(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr())),
                    "recon_fft_r2c")
        return torch.view_as_complex(out)

    def fft_c2r(self, X):
        import torch
        X = torch.view_as_real(X.to(device="cuda", dtype=torch.complex64).contiguous()).contiguous()
        n = self.n
        out = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        self._check(self.lib.recon_fft_c2r(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(out.data_ptr())),
                    "recon_fft_c2r")
        return out

    def run(self, gal_pos, ran_pos=None, start=START_PLAIN, tol=0.0, max_iter=6, gal_w=None, ran_w=None):
        """deposit -> smooth -> iterate; returns (n_iter, rel, status)."""
        self.deposit(gal_pos, gal_w, ran_pos, ran_w)
        self.smooth()
        return self.iterate(start, tol, max_iter)


def batch_run(mocks, start=START_FFTA, tol=1e-6, max_iter=80, autotune=True, stream=None, one_graph=False,
              out=None, **over):
    """Reconstruct a list of mocks in one recon_batch_run call (one_graph: the whole batch as one
    CUDA graph with the size classes side by side, RECON_BATCH_ONE_GRAPH).

    Each entry is a mocks.Mock (numpy catalogues, moved to the GPU first) or a dict with "params"
    (as Mock.params()), "gal" and "ran" (CUDA float64 (n, 3) tensors, "ran" None for uniform mean
    density).  out, if given, holds per mock the (galaxy, random) shift tensors to write into
    (float32 CUDA (n, 3), contiguous; None for a mock without randoms), e.g. those of an earlier
    call; otherwise they are allocated.  Returns the batch status and, per mock, a dict with n_iter,
    rel, status, ms and the galaxy / random shift tensors."""
    import torch
    lib = load()
    items = (ReconBatchItem * len(mocks))()
    keep, outs = [], []
    for i, m in enumerate(mocks):
        if isinstance(m, dict):
            p = dict(m["params"], **over)
            g, r = m["gal"], m["ran"]
        else:
            p = m.params(**over)
            g = torch.from_numpy(m.galaxies.pos).cuda()
            r = torch.from_numpy(m.randoms.pos).cuda() if m.randoms is not None and not p["uniform"] else None
        items[i].params = make_params(p["n"], p["L"], p["b"], p["f"], p["R"], p["observer"], p["los_mode"],
                                      p["periodic"], p["mask_frac"], p["lognormal"], p["uniform"])
        items[i].gal = _catalog(g, None, keep)
        has_ran = r is not None and not p["uniform"]
        if out is not None:
            sg, sr = out[i]
            for t, src in ((sg, g), (sr, r if has_ran else None)):
                if src is None:
                    continue
                if (t is None or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous()
                        or tuple(t.shape) != (len(src), 3)):
                    raise ValueError(f"batch_run: out[{i}] must hold float32 CUDA (n, 3) tensors")
        else:
            sg = torch.empty((len(g), 3), dtype=torch.float32, device="cuda")
            sr = torch.empty((len(r), 3), dtype=torch.float32, device="cuda") if has_ran else None
        items[i].shift_gal = sg.data_ptr()
        if has_ran:
            items[i].ran = _catalog(r, None, keep)
            items[i].shift_ran = sr.data_ptr()
        else:
            sr = None
        keep += [g, r, sg, sr]
        items[i].start, items[i].tol, items[i].max_iter, items[i].out_on_device = int(start), float(tol), int(max_iter), 1
        outs.append((sg, sr))
    st = (stream or torch.cuda.current_stream()).cuda_stream
    flags = (BATCH_TUNE if autotune else 0) | (BATCH_ONE_GRAPH if one_graph else 0)
    status = lib.recon_batch_run(items, len(mocks), C.c_void_p(st), flags)
    torch.cuda.synchronize()
    res = []
    for i in range(len(mocks)):
        res.append(dict(n_iter=items[i].n_iter, rel=items[i].rel, status=items[i].status, ms=items[i].ms,
                        shift_gal=outs[i][0], shift_ran=outs[i][1]))
    return status, res


def batch_plan(nmesh):
    lib = load()
    a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    st = lib.recon_batch_plan(int(nmesh), C.byref(a), C.byref(b), C.byref(c), C.byref(d))
    return None if st != OK else dict(line_tile=a.value, deposit_path=b.value, shift_path=c.value,
                                      fft_radix=d.value)


class UNet:
    """The warm-start network (recon_unet_*): parameters live on the device."""

    def __init__(self, c1=16, bf16=True, stream=None):
        import torch
        self.lib = load()
        self.c1 = int(c1)
        cnt = C.c_size_t(0)
        st = self.lib.recon_unet_param_count(self.c1, C.byref(cnt))
        if st != OK:
            raise ReconError(st, "recon_unet_param_count")
        self.count = cnt.value
        h = C.c_void_p()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        st = self.lib.recon_unet_create(self.c1, int(bool(bf16)), C.c_void_p(s), C.byref(h))
        if st != OK:
            raise ReconError(st, "recon_unet_create: " + self.lib.recon_status_str(st).decode())
        self.h = h

    def _check(self, st, what):
        if st != OK:
            raise ReconError(st, f"{what}: {self.lib.recon_status_str(st).decode()} "
                                 f"({self.lib.recon_unet_last_error(self.h).decode()})")

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self.lib.recon_unet_set_params(self.h, flat.ctypes.data, flat.size), "recon_unet_set_params")

    def get_params(self):
        out = np.empty(self.count, dtype=np.float32)
        self._check(self.lib.recon_unet_get_params(self.h, out.ctypes.data, out.size), "recon_unet_get_params")
        return out

    def get_grads(self):
        out = np.empty(self.count, dtype=np.float32)
        self._check(self.lib.recon_unet_get_grads(self.h, out.ctypes.data, out.size), "recon_unet_get_grads")
        return out

    def forward(self, x):
        import torch
        n = x.shape[0]
        x = x.to(device="cuda", dtype=torch.float32).contiguous()
        y = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        self._check(self.lib.recon_unet_forward(self.h, C.c_void_p(x.data_ptr()), n, C.c_void_p(y.data_ptr())),
                    "recon_unet_forward")
        return y

    def backward(self, x, target):
        import torch
        n = x.shape[0]
        x = x.to(device="cuda", dtype=torch.float32).contiguous()
        t = target.to(device="cuda", dtype=torch.float32).contiguous()
        loss = C.c_double(0)
        self._check(self.lib.recon_unet_backward(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), n,
                                                 C.byref(loss)), "recon_unet_backward")
        return loss.value

    def adamw(self, lr, wd=1e-4):
        self._check(self.lib.recon_unet_adamw(self.h, float(lr), float(wd)), "recon_unet_adamw")

    def set_option(self, option, value):
        self._check(self.lib.recon_unet_set_option(self.h, int(option), int(value)), "recon_unet_set_option")

    def launch_count(self):
        c = C.c_longlong(0)
        self._check(self.lib.recon_unet_launch_count(self.h, C.byref(c)), "recon_unet_launch_count")
        return c.value

    def get_layer(self, layer, n, cout):
        """Output of convolution layer `layer` of the last forward, (n, n, n, cout) host float32."""
        out = np.empty((n, n, n, cout), dtype=np.float32)
        self._check(self.lib.recon_unet_get_layer(self.h, int(layer), out.ctypes.data, out.size),
                    "recon_unet_get_layer")
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.recon_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def flat_params(params, specs):
    """Flatten {name: (w, b)} in the layer order of the ABI (host float32)."""
    parts = []
    for name, _, _ in specs:
        w, b = params[name]
        parts += [np.asarray(w, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()]
    return np.concatenate(parts).astype(np.float32)


def unflat_params(flat, specs):
    out, o = {}, 0
    for name, ci, co in specs:
        nt = 1 if name == "head" else 27
        w = flat[o:o + nt * ci * co].reshape(nt, ci, co)
        o += nt * ci * co
        b = flat[o:o + co]
        o += co
        out[name] = (w, b)
    return out
