"""ctypes binding of libamber (include/amber.h): argument marshalling only.

Every step of the path runs in the CUDA library; this module only converts
torch tensors to raw device pointers, fills the parameter structs and turns
non-zero status codes into exceptions.  There is no fallback: if the shared
library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libamber.so")

AMBER_OK = 0
AMBER_ERR_INVALID_ARG = 1
AMBER_ERR_NO_SOLUTION = 2
AMBER_ERR_NONFINITE = 4
AMBER_ERR_OOM = 8
AMBER_ERR_DEVICE_TIMEOUT = 16
AMBER_ERR_CUDA = 32
AMBER_ERR_INVALID_MASS = 64
AMBER_ERR_CAPACITY = 128

EXPORTED = [
    "amber_history_default", "amber_history_coeffs", "amber_history_table", "amber_create", "amber_destroy",
    "amber_workspace_bytes", "amber_radiation_field", "amber_radiation_field_f64", "amber_rank",
    "amber_rank_f64", "amber_assign_zre", "amber_solve", "amber_solve_f64", "amber_sync_status",
    "amber_status_string", "amber_profile_enable", "amber_profile_reset", "amber_profile_kinds",
    "amber_profile_read", "amber_sort_passes", "amber_test_wait_timeout", "amber_source_field",
    "amber_solve_ex", "amber_assign_zre_ranked", "amber_batch_create", "amber_batch_launch", "amber_batch_destroy",
    "amber_delta_z", "amber_epsilon_z_pdf", "amber_power_bins", "amber_power_spectrum",
    "amber_lpt_displacement", "amber_mesh_density", "amber_esf_fcoll", "amber_sigma2_tophat",
    "amber_solve_tomographic", "amber_autotune", "amber_set_tuning", "amber_get_tuning",
    "amber_rank_noalloc", "amber_power_derived", "amber_spectrum_bytes", "amber_source_spectrum",
    "amber_solve_spectrum", "amber_batch_kernel_nodes", "amber_solve_host", "amber_struct_layout",
]


AMBER_WEIGHT_MASS = 0
AMBER_WEIGHT_MASS_GROWTH = 1
AMBER_WEIGHT_VOLUME = 2


class amber_history_t(C.Structure):
    _fields_ = [("z_mid", C.c_double), ("dz", C.c_double), ("Az", C.c_double),
                ("x_ear", C.c_double), ("x_mid", C.c_double), ("x_lat", C.c_double),
                ("z_lo", C.c_double), ("z_hi", C.c_double), ("n_table", C.c_int),
                ("weighting", C.c_int), ("omega_m", C.c_double)]


class amber_params_t(C.Structure):
    _fields_ = [("n", C.c_int), ("box", C.c_double), ("l_mfp", C.c_double),
                ("hist", amber_history_t), ("precision", C.c_int)]


class amber_tuning_t(C.Structure):
    _fields_ = [("n", C.c_int), ("fft_variant", C.c_int), ("sort_digit_bits", C.c_int), ("sort_match", C.c_int),
                ("tuned", C.c_int), ("fft_ms", C.c_double * 2), ("sort_ms", C.c_double * 4),
                ("fuse_histogram", C.c_int), ("zpass_tma", C.c_int), ("fft_tma_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {"n": self.n, "fft_variant": self.fft_variant, "sort_digit_bits": self.sort_digit_bits,
                "sort_match": self.sort_match, "tuned": self.tuned, "fft_ms": list(self.fft_ms),
                "sort_ms": list(self.sort_ms), "fuse_histogram": self.fuse_histogram,
                "zpass_tma": self.zpass_tma, "fft_tma_ms": self.fft_tma_ms}


class amber_batch_item(C.Structure):
    _fields_ = [("d_src", C.c_void_p), ("d_mass", C.c_void_p), ("params", amber_params_t), ("d_zre", C.c_void_p)]


class AmberError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: amber status {code} ({status_string(code)})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libamber.so not built at {LIB_PATH}; run __graft_entry__.build() first")
    lib = C.CDLL(LIB_PATH)
    vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
    H = C.POINTER(amber_history_t)
    sig = {
        "amber_history_default": (i32, [H, dbl, dbl, dbl]),
        "amber_history_coeffs": (i32, [H, C.POINTER(dbl)]),
        "amber_history_table": (i32, [H, C.POINTER(dbl), C.POINTER(dbl)]),
        "amber_create": (i32, [C.POINTER(vp), i32, i64]),
        "amber_destroy": (i32, [vp]),
        "amber_workspace_bytes": (i32, [i64, C.POINTER(C.c_size_t)]),
        "amber_radiation_field": (i32, [vp, vp, i32, dbl, dbl, vp, vp]),
        "amber_radiation_field_f64": (i32, [vp, vp, i32, dbl, dbl, vp, vp]),
        "amber_rank": (i32, [vp, vp, i64, vp, vp]),
        "amber_rank_f64": (i32, [vp, vp, i64, vp, vp]),
        "amber_assign_zre": (i32, [vp, vp, vp, i64, H, vp, vp, vp]),
        "amber_solve": (i32, [vp, vp, vp, C.POINTER(amber_params_t), vp, vp, vp]),
        "amber_solve_f64": (i32, [vp, vp, vp, C.POINTER(amber_params_t), vp, vp, vp]),
        "amber_sync_status": (i32, [vp, vp]),
        "amber_status_string": (C.c_char_p, [i32]),
        "amber_profile_enable": (i32, [vp, i32]),
        "amber_profile_reset": (i32, [vp]),
        "amber_profile_kinds": (i32, []),
        "amber_struct_layout": (i32, [i32, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), i32, C.POINTER(i32)]),
        "amber_profile_read": (i32, [vp, i32, C.POINTER(C.c_char_p), C.POINTER(dbl), C.POINTER(i64)]),
        "amber_sort_passes": (i32, [vp, C.POINTER(i32)]),
        "amber_source_field": (i32, [vp, vp, i64, dbl, dbl, vp, vp, vp]),
        "amber_solve_ex": (i32, [vp, vp, vp, C.POINTER(amber_params_t), vp, vp, vp, vp, vp]),
        "amber_assign_zre_ranked": (i32, [vp, vp, vp, i64, H, vp, vp, vp]),
        "amber_batch_create": (i32, [C.POINTER(vp), C.POINTER(vp), i32, C.POINTER(amber_batch_item), i32]),
        "amber_batch_launch": (i32, [vp, vp]),
        "amber_batch_destroy": (i32, [vp]),
        "amber_batch_kernel_nodes": (i32, [vp, C.POINTER(i32)]),
        "amber_solve_host": (i32, [vp, vp, vp, C.POINTER(amber_params_t), vp, vp]),
        "amber_delta_z": (i32, [vp, vp, i64, vp, vp, vp]),
        "amber_epsilon_z_pdf": (i32, [vp, vp, vp, i64, dbl, dbl, i32, vp, vp, vp]),
        "amber_power_bins": (i32, [i32, C.POINTER(i32)]),
        "amber_power_spectrum": (i32, [vp, vp, vp, i32, dbl, vp, vp, vp, vp, vp, vp]),
        "amber_lpt_displacement": (i32, [vp, vp, i32, dbl, dbl, dbl, vp, vp, vp, vp]),
        "amber_mesh_density": (i32, [vp, vp, vp, vp, vp, i32, dbl, i32, i32, vp, vp]),
        "amber_esf_fcoll": (i32, [vp, vp, i32, dbl, dbl, i32, dbl, dbl, vp, vp]),
        "amber_sigma2_tophat": (i32, [C.POINTER(dbl), C.POINTER(dbl), i32, dbl, C.POINTER(dbl)]),
        "amber_solve_tomographic": (i32, [vp, C.POINTER(vp), i32, C.POINTER(dbl), vp, C.POINTER(amber_params_t), vp,
                                          vp]),
        "amber_autotune": (i32, [vp, vp, vp, i32, dbl, dbl, C.POINTER(amber_tuning_t), vp]),
        "amber_set_tuning": (i32, [vp, C.POINTER(amber_tuning_t)]),
        "amber_get_tuning": (i32, [vp, i32, C.POINTER(amber_tuning_t)]),
        "amber_rank_noalloc": (i32, [vp, i64, vp, vp, vp]),
        "amber_power_derived": (i32, [vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp]),
        "amber_spectrum_bytes": (i32, [i32, C.POINTER(C.c_size_t)]),
        "amber_source_spectrum": (i32, [vp, vp, i32, vp, vp]),
        "amber_solve_spectrum": (i32, [vp, vp, vp, C.POINTER(amber_params_t), vp, vp, vp, vp, vp]),
        "amber_test_wait_timeout": (i32, [vp, C.c_uint, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def status_string(code: int) -> str:
    return lib.amber_status_string(int(code)).decode()


def _check(code: int, what: str):
    if code != AMBER_OK:
        raise AmberError(code, what)


def history(z_mid: float, dz: float, Az: float, x_points=(0.05, 0.5, 0.95), z_lo: float = 5.0,
            z_hi: float = 20.0, n_table: int = 2000, weighting: int = AMBER_WEIGHT_MASS,
            omega_m: float = 0.3) -> amber_history_t:
    h = amber_history_t()
    _check(lib.amber_history_default(C.byref(h), z_mid, dz, Az), "amber_history_default")
    h.x_ear, h.x_mid, h.x_lat = x_points
    h.z_lo, h.z_hi, h.n_table = z_lo, z_hi, n_table
    h.weighting, h.omega_m = weighting, omega_m
    return h


def sigma2_tophat(k, Delta2, R: float) -> float:
    """Eq. variance by the trapezoid rule in ln k (host)."""
    import numpy as np
    k = np.ascontiguousarray(k, dtype=np.float64)
    d = np.ascontiguousarray(Delta2, dtype=np.float64)
    out = C.c_double()
    _check(lib.amber_sigma2_tophat(k.ctypes.data_as(C.POINTER(C.c_double)), d.ctypes.data_as(C.POINTER(C.c_double)),
                                   len(k), R, C.byref(out)), "amber_sigma2_tophat")
    return out.value


def power_bins(n: int) -> int:
    out = C.c_int()
    _check(lib.amber_power_bins(n, C.byref(out)), "amber_power_bins")
    return out.value


def history_coeffs(h: amber_history_t):
    out = (C.c_double * 3)()
    _check(lib.amber_history_coeffs(C.byref(h), out), "amber_history_coeffs")
    return tuple(out)


def history_table(h: amber_history_t):
    import numpy as np
    z = np.zeros(h.n_table)
    x = np.zeros(h.n_table)
    _check(lib.amber_history_table(C.byref(h), z.ctypes.data_as(C.POINTER(C.c_double)),
                                   x.ctypes.data_as(C.POINTER(C.c_double))), "amber_history_table")
    return z, x


def spectrum_bytes(n: int) -> int:
    out = C.c_size_t()
    _check(lib.amber_spectrum_bytes(n, C.byref(out)), "amber_spectrum_bytes")
    return out.value


def workspace_bytes(max_cells: int) -> int:
    out = C.c_size_t()
    _check(lib.amber_workspace_bytes(max_cells, C.byref(out)), "amber_workspace_bytes")
    return out.value


def _ptr(t):
    """Raw data pointer of a tensor the library reads or writes as a flat array."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("libamber takes contiguous arrays; pass .contiguous()")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def params(n: int, box: float, l_mfp: float, h: amber_history_t, precision: int = 32) -> amber_params_t:
    p = amber_params_t()
    p.n, p.box, p.l_mfp, p.hist, p.precision = n, box, l_mfp, h, precision
    return p


class Batch:
    """Many solves in one captured CUDA graph of one launch per stage (see amber_batch_create)."""

    def __init__(self, ctxs, items):
        """items: (S, mass, box, l_mfp, history, z_out) tuples of device tensors."""
        self._keep = (list(ctxs), list(items))
        arr = (amber_batch_item * len(items))()
        for i, (S, m, box, l, h, z) in enumerate(items):
            arr[i].d_src, arr[i].d_mass, arr[i].d_zre = _ptr(S).value, _ptr(m).value, _ptr(z).value
            arr[i].params = params(S.shape[0], box, l, h)
        hs = (C.c_void_p * len(ctxs))(*[c._h.value for c in ctxs])
        self._h = C.c_void_p()
        _check(lib.amber_batch_create(C.byref(self._h), hs, len(ctxs), arr, len(items)), "amber_batch_create")

    def launch(self, stream=None):
        _check(lib.amber_batch_launch(self._h, _stream(stream)), "amber_batch_launch")

    def kernel_nodes(self) -> int:
        out = C.c_int()
        _check(lib.amber_batch_kernel_nodes(self._h, C.byref(out)), "amber_batch_kernel_nodes")
        return out.value

    def close(self):
        if self._h:
            lib.amber_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """An amber_ctx: one device, a workspace sized for max_cells cells."""

    def __init__(self, max_cells: int, device: int = 0):
        self._h = C.c_void_p()
        self.device = device
        self.max_cells = max_cells
        _check(lib.amber_create(C.byref(self._h), device, max_cells), "amber_create")

    def close(self):
        if self._h:
            lib.amber_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- the path -----------------------------------------------------------
    def radiation_field(self, S, box: float, l_mfp: float, out=None, stream=None):
        import torch
        n = S.shape[0]
        f64 = S.dtype == torch.float64
        if out is None:
            out = torch.empty_like(S)
        fn = lib.amber_radiation_field_f64 if f64 else lib.amber_radiation_field
        _check(fn(self._h, _ptr(S), n, box, l_mfp, _ptr(out), _stream(stream)), "amber_radiation_field")
        return out

    def rank(self, J, out=None, stream=None):
        import torch
        n = J.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=J.device)
        fn = lib.amber_rank_f64 if J.dtype == torch.float64 else lib.amber_rank
        _check(fn(self._h, _ptr(J), n, _ptr(out), _stream(stream)), "amber_rank")
        return out

    def assign_zre(self, order, mass, h: amber_history_t, out=None, F=None, stream=None):
        import torch
        n = order.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=order.device)
        _check(lib.amber_assign_zre(self._h, _ptr(order), _ptr(mass), n, C.byref(h), _ptr(out), _ptr(F),
                                    _stream(stream)), "amber_assign_zre")
        return out

    def source_field(self, delta, delta_c: float = 1.686, sigma_f: float = 0.7, out=None, mass_out=None,
                     stream=None):
        import torch
        if out is None:
            out = torch.empty_like(delta)
        _check(lib.amber_source_field(self._h, _ptr(delta), delta.numel(), delta_c, sigma_f, _ptr(out),
                                      _ptr(mass_out), _stream(stream)), "amber_source_field")
        return out

    def solve(self, S, mass, box: float, l_mfp: float, h: amber_history_t, out=None, J_out=None, stream=None):
        import torch
        n = S.shape[0]
        p = amber_params_t()
        p.n, p.box, p.l_mfp, p.hist = n, box, l_mfp, h
        f64 = S.dtype == torch.float64
        p.precision = 64 if f64 else 32
        if out is None:
            out = torch.empty(S.shape, dtype=torch.float32, device=S.device)
        fn = lib.amber_solve_f64 if f64 else lib.amber_solve
        _check(fn(self._h, _ptr(S), _ptr(mass), C.byref(p), _ptr(out), _ptr(J_out), _stream(stream)), "amber_solve")
        return out

    def solve_host(self, S, mass, box: float, l_mfp: float, h: amber_history_t, out, stream=None):
        """The whole path from host tensors (S, mass; pinned for full speed) into
        the host tensor out, enqueued on the stream (synchronise before reading out)."""
        p = params(S.shape[0], box, l_mfp, h)
        _check(lib.amber_solve_host(self._h, _ptr(S), _ptr(mass), C.byref(p), _ptr(out), _stream(stream)),
               "amber_solve_host")
        return out

    def solve_ex(self, S, mass, box: float, l_mfp: float, h: amber_history_t, out, order_out, mass_rank_out,
                 J_out=None, stream=None):
        """Solve and keep the rank order and rank-order masses (for history-only reruns)."""
        p = params(S.shape[0], box, l_mfp, h)
        _check(lib.amber_solve_ex(self._h, _ptr(S), _ptr(mass), C.byref(p), _ptr(out), _ptr(J_out), _ptr(order_out),
                                  _ptr(mass_rank_out), _stream(stream)), "amber_solve_ex")
        return out

    def source_spectrum(self, S, out=None, stream=None):
        """The x- and y-transformed source field (a flat uint8 device tensor of
        amber_spectrum_bytes(n) bytes) that solve_spectrum starts from."""
        import torch
        n = S.shape[0]
        if out is None:
            out = torch.empty(spectrum_bytes(n), dtype=torch.uint8, device=S.device)
        _check(lib.amber_source_spectrum(self._h, _ptr(S), n, _ptr(out), _stream(stream)), "amber_source_spectrum")
        return out

    def solve_spectrum(self, spec, mass, box: float, l_mfp: float, h: amber_history_t, out, order_out=None,
                       mass_rank_out=None, J_out=None, stream=None):
        """solve_ex from a kept source spectrum (l_mfp and history free to change)."""
        p = params(mass.shape[0], box, l_mfp, h)
        _check(lib.amber_solve_spectrum(self._h, _ptr(spec), _ptr(mass), C.byref(p), _ptr(out), _ptr(J_out),
                                        _ptr(order_out), _ptr(mass_rank_out), _stream(stream)),
               "amber_solve_spectrum")
        return out

    def assign_zre_ranked(self, order, mass_rank, h: amber_history_t, out, F=None, stream=None):
        _check(lib.amber_assign_zre_ranked(self._h, _ptr(order), _ptr(mass_rank), order.numel(), C.byref(h),
                                           _ptr(out), _ptr(F), _stream(stream)), "amber_assign_zre_ranked")
        return out

    def sync_status(self, stream=None) -> int:
        return lib.amber_sync_status(self._h, _stream(stream))

    # --- profiling ----------------------------------------------------------
    def profile(self, on: bool = True):
        _check(lib.amber_profile_enable(self._h, 1 if on else 0), "amber_profile_enable")

    def profile_reset(self):
        _check(lib.amber_profile_reset(self._h), "amber_profile_reset")

    def profile_read(self) -> dict:
        out = {}
        for k in range(lib.amber_profile_kinds()):
            name, ms, cnt = C.c_char_p(), C.c_double(), C.c_int64()
            _check(lib.amber_profile_read(self._h, k, C.byref(name), C.byref(ms), C.byref(cnt)), "amber_profile_read")
            out[name.value.decode()] = (ms.value, cnt.value)
        return out

    def sort_passes(self) -> int:
        out = C.c_int()
        _check(lib.amber_sort_passes(self._h, C.byref(out)), "amber_sort_passes")
        return out.value

    def test_wait_timeout(self, spin_limit: int, stream=None):
        _check(lib.amber_test_wait_timeout(self._h, spin_limit, _stream(stream)), "amber_test_wait_timeout")

    # --- autotuning of the FP32 solve path per grid size ----------------------
    def autotune(self, S, mass, box: float, l_mfp: float, stream=None) -> dict:
        """Time every FFT variant and ranking choice on these inputs; keep the fastest for S's size."""
        t = amber_tuning_t()
        _check(lib.amber_autotune(self._h, _ptr(S), _ptr(mass), S.shape[0], box, l_mfp, C.byref(t), _stream(stream)),
               "amber_autotune")
        return t.as_dict()

    def set_tuning(self, n: int, fft_variant=None, sort_digit_bits=None, sort_match=None, fuse_histogram=None,
                   zpass_tma=None):
        """Set the choices for size n; a choice left as None keeps its current value."""
        cur = self.get_tuning(n)
        t = amber_tuning_t(n, cur["fft_variant"] if fft_variant is None else fft_variant,
                           cur["sort_digit_bits"] if sort_digit_bits is None else sort_digit_bits,
                           cur["sort_match"] if sort_match is None else sort_match, 0)
        t.fuse_histogram = cur["fuse_histogram"] if fuse_histogram is None else fuse_histogram
        t.zpass_tma = cur["zpass_tma"] if zpass_tma is None else zpass_tma
        _check(lib.amber_set_tuning(self._h, C.byref(t)), "amber_set_tuning")

    def get_tuning(self, n: int) -> dict:
        t = amber_tuning_t()
        _check(lib.amber_get_tuning(self._h, n, C.byref(t)), "amber_get_tuning")
        return t.as_dict()

    def solve_tomographic(self, sources, z_bounds, mass, box: float, l_mfp: float, h: amber_history_t, out=None,
                          stream=None):
        """z_re from one source field per redshift interval (intervals from z_bounds, decreasing)."""
        import torch
        S0 = sources[0]
        n = S0.shape[0]
        if out is None:
            out = torch.empty(S0.shape, dtype=torch.float32, device=S0.device)
        srcs = (C.c_void_p * len(sources))(*[_ptr(x) for x in sources])
        zb = (C.c_double * len(z_bounds))(*z_bounds)
        p = params(n, box, l_mfp, h)
        _check(lib.amber_solve_tomographic(self._h, srcs, len(sources), zb, _ptr(mass), C.byref(p), _ptr(out),
                                           _stream(stream)), "amber_solve_tomographic")
        return out

    # --- source-field pipeline (Sec. 3.2, 3.2.1, 3.3) -------------------------
    def lpt_displacement(self, delta_lin, box: float, D1: float, D2: float, stream=None):
        """(psi_x, psi_y, psi_z) of the second-order displacement (Eq. xlpt), box units."""
        import torch
        n = delta_lin.shape[0]
        psi = tuple(torch.empty_like(delta_lin) for _ in range(3))
        _check(lib.amber_lpt_displacement(self._h, _ptr(delta_lin), n, box, D1, D2, _ptr(psi[0]), _ptr(psi[1]),
                                          _ptr(psi[2]), _stream(stream)), "amber_lpt_displacement")
        return psi

    def mesh_density(self, psi, box: float, order: int = 3, interlace: bool = True, mass=None, out=None,
                     stream=None):
        """rho / <rho> from displaced lattice particles (Sec. 3.2.1, Eqs. interlace, Wofk)."""
        import torch
        n = psi[0].shape[0]
        if out is None:
            out = torch.empty_like(psi[0])
        _check(lib.amber_mesh_density(self._h, _ptr(psi[0]), _ptr(psi[1]), _ptr(psi[2]), _ptr(mass), n, box, order,
                                      1 if interlace else 0, _ptr(out), _stream(stream)), "amber_mesh_density")
        return out

    def esf_fcoll(self, delta_lin, box: float, R: float, delta_c: float, dsigma2: float, filter: str = "sharpk",
                  out=None, stream=None):
        """Collapsed fraction of the filtered linear field (Eq. fcoll)."""
        import torch
        n = delta_lin.shape[0]
        if out is None:
            out = torch.empty_like(delta_lin)
        _check(lib.amber_esf_fcoll(self._h, _ptr(delta_lin), n, box, R, 0 if filter == "sharpk" else 1, delta_c,
                                   dsigma2, _ptr(out), _stream(stream)), "amber_esf_fcoll")
        return out

    # --- analysis of z_re fields (Sec. 2.3) ----------------------------------
    def delta_z(self, z, out=None, stream=None):
        """(delta_z field, zbar tensor) of a float field (Eq. deltaz)."""
        import torch
        if out is None:
            out = torch.empty_like(z)
        zbar = torch.empty(1, dtype=torch.float64, device=z.device)
        _check(lib.amber_delta_z(self._h, _ptr(z), z.numel(), _ptr(out), _ptr(zbar), _stream(stream)),
               "amber_delta_z")
        return out, zbar

    def epsilon_z_pdf(self, z, z_ref, lo: float, hi: float, nbins: int, stream=None):
        """(counts [nbins + 2] with under/overflow at the ends, [sum eps, sum eps^2]) (Eq. epsz)."""
        import torch
        counts = torch.empty(nbins + 2, dtype=torch.int64, device=z.device)
        mom = torch.empty(2, dtype=torch.float64, device=z.device)
        _check(lib.amber_epsilon_z_pdf(self._h, _ptr(z), _ptr(z_ref), z.numel(), lo, hi, nbins, _ptr(counts),
                                       _ptr(mom), _stream(stream)), "amber_epsilon_z_pdf")
        return counts, mom

    def derived_spectra(self, s: dict, stream=None) -> dict:
        """Delta^2 (Eq. Dk), bias (Eq. bias) and cross-correlation r (Eq. rcc) per
        shell from power_spectrum's output, formed on the device (device tensors)."""
        import torch
        nb = s["k"].numel()
        out = {key: torch.empty(nb, dtype=torch.float64, device=s["k"].device)
               for key in ("Delta2_aa", "Delta2_bb", "bias", "r")}
        _check(lib.amber_power_derived(self._h, _ptr(s["k"]), _ptr(s["Paa"]), _ptr(s["Pbb"]), _ptr(s["Pab"]), nb,
                                       _ptr(out["Delta2_aa"]), _ptr(out["Delta2_bb"]), _ptr(out["bias"]),
                                       _ptr(out["r"]), _stream(stream)), "amber_power_derived")
        out["k"] = s["k"]
        return out

    def power_spectrum(self, a, b=None, box: float = 1.0, stream=None):
        """Shell spectra (Eqs. Pk, Dk, bias, rcc) of n^3 float fields: dict of
        device tensors k, Paa, Pbb, Pab, modes (per shell)."""
        import torch
        n = a.shape[0]
        nb = power_bins(n)
        out = {key: torch.empty(nb, dtype=torch.float64, device=a.device) for key in ("k", "Paa", "Pbb", "Pab", "modes")}
        _check(lib.amber_power_spectrum(self._h, _ptr(a), _ptr(b), n, box, _ptr(out["k"]), _ptr(out["Paa"]),
                                        _ptr(out["Pbb"]), _ptr(out["Pab"]), _ptr(out["modes"]), _stream(stream)),
               "amber_power_spectrum")
        return out
