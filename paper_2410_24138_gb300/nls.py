"""Python binding of the C-ABI library ``libnls.so`` (include/nls.h): argument marshalling only.

Every computation runs in the library's sm_103a kernels.  Host arrays are numpy arrays;
device arrays are torch CUDA tensors (their ``data_ptr()`` is passed through).  Loading
fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build
from .inputs import LAMBDA_PLANE_STRESS, LAMBDA_PRINTED, LAW_DIFFUSION, LAW_NEOHOOKE, Problem

P1_TRI, Q1_QUAD = 1, 2
COUPLING = {"one": 0, "add": 1, "hybrid": 2}
PREC_FP64, PREC_FP32_IR = 0, 1
COARSE_FACTOR_AUTO, COARSE_FACTOR_BAND, COARSE_FACTOR_TILES = 0, 1, 2
COARSE_NONE, COARSE_RGDSW = 0, 1

STATUS = {0: "ok", -1: "E_ARG", -2: "E_CUDA", -3: "E_NOMEM", -4: "E_UNSUPPORTED", -5: "E_LOCAL_NEWTON",
          -6: "E_PIVOT", -7: "E_GMRES", -8: "E_DIVERGED", -9: "E_DEVICE_TIMEOUT", 1: "W_NOT_CONVERGED"}


class Options(ctypes.Structure):
    _fields_ = [("coupling", ctypes.c_int32), ("local_precision", ctypes.c_int32),
                ("coarse_precision", ctypes.c_int32), ("load_steps", ctypes.c_int32),
                ("outer_atol", ctypes.c_double), ("outer_maxit", ctypes.c_int32),
                ("inner_rtol", ctypes.c_double), ("inner_atol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int32), ("ls_trials", ctypes.c_int32), ("armijo", ctypes.c_double),
                ("gmres_rtol", ctypes.c_double), ("gmres_restart", ctypes.c_int32), ("gmres_maxit", ctypes.c_int32),
                ("ir_rtol", ctypes.c_double), ("ir_max_sweeps", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("verbose", ctypes.c_int32),
                ("profile_kernels", ctypes.c_int32), ("cuda_graphs", ctypes.c_int32),
                ("coarse_reuse", ctypes.c_int32), ("local_reuse", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("l2_prefetch", ctypes.c_int32), ("outer_backtrack", ctypes.c_int32),
                ("coarse_rebuild", ctypes.c_int32), ("coarse_factor", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("gmres_iterations", ctypes.c_int32), ("subdomain_newton_steps", ctypes.c_int64),
                ("coarse_newton_steps", ctypes.c_int32), ("local_failures", ctypes.c_int32),
                ("first_failed_subdomain", ctypes.c_int32), ("final_residual", ctypes.c_double),
                ("time_total_s", ctypes.c_double), ("time_inner_s", ctypes.c_double),
                ("time_coarse_s", ctypes.c_double), ("time_gmres_s", ctypes.c_double),
                ("time_other_s", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("local_chord_steps", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Sizes(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_dofs", ctypes.c_int64), ("n_elems", ctypes.c_int64),
                ("ndof", ctypes.c_int32), ("n_sub", ctypes.c_int32), ("n_coarse_nodes", ctypes.c_int32),
                ("n_coarse_dofs", ctypes.c_int32), ("total_local_dofs", ctypes.c_int64),
                ("total_overlap_elems", ctypes.c_int64), ("max_local_dofs", ctypes.c_int32),
                ("max_half_band", ctypes.c_int32), ("coarse_half_band", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("total_factor_entries", ctypes.c_int64),
                ("total_local_nnz", ctypes.c_int64), ("total_table_dofs", ctypes.c_int64),
                ("factor_bytes", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("total_solve_entries", ctypes.c_int64), ("lu_flops", ctypes.c_double),
                ("solve_flops", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("newton_threads", ctypes.c_int32), ("apply_threads", ctypes.c_int32),
                ("newton_tuned", ctypes.c_int32), ("apply_tuned", ctypes.c_int32),
                ("newton_ms", ctypes.c_double * 2), ("graphs_captured", ctypes.c_int32),
                ("coarse_threads", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"newton_threads": self.newton_threads, "apply_threads": self.apply_threads,
                "newton_tuned": bool(self.newton_tuned), "apply_tuned": bool(self.apply_tuned),
                "newton_ms": list(self.newton_ms), "graphs_captured": self.graphs_captured,
                "coarse_threads": self.coarse_threads}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


EXPORTS = ["nls_options_default", "nls_create", "nls_destroy", "nls_strerror", "nls_last_error", "nls_set_mesh",
           "nls_set_dirichlet", "nls_set_traction", "nls_set_material", "nls_set_partition", "nls_set_coarse",
           "nls_set_options", "nls_get_options", "nls_setup", "nls_setup_host", "nls_solve", "nls_get_sizes", "nls_get_local_dofs",
           "nls_get_overlap_elems", "nls_get_owners", "nls_get_coarse_nodes", "nls_get_coarse_basis", "nls_eval_F",
           "nls_eval_Fx", "nls_apply_tangent", "nls_get_local_states", "nls_get_kernel_stats",
           "nls_reset_kernel_stats", "nls_local_corrections_noalloc", "nls_guess_create", "nls_guess_destroy",
           "nls_guess_attach", "nls_guess_train", "nls_guess_pairs", "nls_guess_get_params", "nls_guess_set_params",
           "nls_guess_get_normalisation", "nls_guess_set_normalisation", "nls_guess_gradient", "nls_guess_forward",
           "nls_guess_counts", "nls_get_tuning", "nls_guess_set_smoothing", "nls_set_coefficients",
           "nls_set_volume_force", "nls_set_lambda_mode", "nls_get_coarse_matrix", "nls_band_solve",
           "nls_guess_features", "nls_guess_decode", "nls_guess_smooth", "nls_guess_create_kind", "nls_guess_dims"]

_LIB = None
_P = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libnls.so (built in-tree by ``paper_2410_24138_gb300.build.build()``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the sm_103a library first (paper_2410_24138_gb300.build.build())")
    lib = ctypes.CDLL(path)
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "nls_options_default": (None, [ctypes.POINTER(Options)]),
        "nls_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
        "nls_destroy": (None, [_P]),
        "nls_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "nls_last_error": (ctypes.c_char_p, [_P]),
        "nls_set_mesh": (ctypes.c_int, [_P, ctypes.c_int, i64, _P, i64, _P]),
        "nls_set_dirichlet": (ctypes.c_int, [_P, i64, _P, _P]),
        "nls_set_traction": (ctypes.c_int, [_P, i64, _P, _P]),
        "nls_set_material": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
        "nls_set_volume_force": (ctypes.c_int, [_P, _P]),
        "nls_set_lambda_mode": (ctypes.c_int, [_P, ctypes.c_int]),
        "nls_set_partition": (ctypes.c_int, [_P, i32, _P, i32]),
        "nls_set_coarse": (ctypes.c_int, [_P, ctypes.c_int]),
        "nls_set_options": (ctypes.c_int, [_P, ctypes.POINTER(Options)]),
        "nls_get_options": (ctypes.c_int, [_P, ctypes.POINTER(Options)]),
        "nls_setup": (ctypes.c_int, [_P]),
        "nls_setup_host": (ctypes.c_int, [_P]),
        "nls_solve": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(Report)]),
        "nls_get_sizes": (ctypes.c_int, [_P, ctypes.POINTER(Sizes)]),
        "nls_get_local_dofs": (ctypes.c_int, [_P, i32, i64, _P, _P, ctypes.POINTER(i64)]),
        "nls_get_overlap_elems": (ctypes.c_int, [_P, i32, i64, _P, ctypes.POINTER(i64)]),
        "nls_get_owners": (ctypes.c_int, [_P, _P]),
        "nls_get_coarse_nodes": (ctypes.c_int, [_P, _P]),
        "nls_get_coarse_basis": (ctypes.c_int, [_P, _P]),
        "nls_get_coarse_matrix": (ctypes.c_int, [_P, _P]),
        "nls_guess_features": (ctypes.c_int, [_P, _P, dbl, _P]),
        "nls_guess_decode": (ctypes.c_int, [_P, _P, dbl, _P, _P]),
        "nls_guess_smooth": (ctypes.c_int, [_P, _P, dbl, _P, _P]),
        "nls_band_solve": (ctypes.c_int, [ctypes.c_int, i32, i32, _P, _P, _P, i32, i32, _P]),
        "nls_eval_F": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, dbl]),
        "nls_eval_Fx": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, dbl, _P, _P]),
        "nls_apply_tangent": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
        "nls_get_local_states": (ctypes.c_int, [_P, _P, ctypes.c_int]),
        "nls_get_kernel_stats": (ctypes.c_int, [_P, i32, ctypes.POINTER(KernelStat), ctypes.POINTER(i32)]),
        "nls_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
        "nls_reset_kernel_stats": (ctypes.c_int, [_P]),
        "nls_local_corrections_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, dbl]),
        "nls_guess_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, i32, i32, ctypes.c_uint64, i64]),
        "nls_guess_create_kind": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, i32, i32, i32, ctypes.c_uint64,
                                                 i64]),
        "nls_guess_dims": (ctypes.c_int, [_P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "nls_guess_destroy": (None, [_P]),
        "nls_guess_attach": (ctypes.c_int, [_P, _P, i32]),
        "nls_guess_train": (ctypes.c_int, [_P, i32, i32, dbl, ctypes.c_uint64, _P]),
        "nls_guess_pairs": (ctypes.c_int, [_P, ctypes.POINTER(i64)]),
        "nls_guess_get_params": (ctypes.c_int, [_P, _P, ctypes.POINTER(i64)]),
        "nls_guess_set_params": (ctypes.c_int, [_P, _P, i64]),
        "nls_guess_get_normalisation": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_float)]),
        "nls_guess_set_normalisation": (ctypes.c_int, [_P, _P, _P, ctypes.c_float]),
        "nls_guess_gradient": (ctypes.c_int, [_P, i32, _P, _P, i32, _P, ctypes.POINTER(ctypes.c_float)]),
        "nls_guess_forward": (ctypes.c_int, [_P, i32, _P, _P]),
        "nls_guess_counts": (ctypes.c_int, [_P, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "nls_guess_set_smoothing": (ctypes.c_int, [_P, i32, ctypes.c_double]),
        "nls_set_coefficients": (ctypes.c_int, [_P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    return int(a.data_ptr())  # torch tensor


def _is_device(a) -> int:
    return 0 if isinstance(a, np.ndarray) else int(getattr(a, "is_cuda", False))


class NLSError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")
        self.status = status


def default_options() -> Options:
    o = Options()
    load().nls_options_default(ctypes.byref(o))
    return o


class Solver:
    """One solver context: mesh + law + partition + coarse space -> solution of F(u) = 0."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self.lib = load()
        self.h = _P()
        self._check(self.lib.nls_create(ctypes.byref(self.h), device, stream), "nls_create")
        self.device = device
        self.ndof = 1
        self.n_nodes = 0
        self.n_sub = 0

    def _check(self, st: int, where: str) -> int:
        if st < 0:
            raise NLSError(st, where, self.lib.nls_last_error(self.h).decode() if self.h else "")
        return st

    def close(self):
        if self.h:
            self.lib.nls_destroy(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- problem description --------------------------------------------------------------
    def set_problem(self, p: Problem):
        xy = np.ascontiguousarray(p.xy, dtype=np.float64)
        conn = np.ascontiguousarray(p.conn, dtype=np.int32)
        self._check(self.lib.nls_set_mesh(self.h, p.elem_type, xy.shape[0], _ptr(xy), conn.shape[0], _ptr(conn)),
                    "nls_set_mesh")
        law = p.law
        self.ndof = p.ndof
        self.n_nodes = xy.shape[0]
        if law == LAW_DIFFUSION:
            k = None if p.k_elem is None else np.ascontiguousarray(p.k_elem, dtype=np.float64)
            f = None if p.f_elem is None else np.ascontiguousarray(p.f_elem, dtype=np.float64)
            self._check(self.lib.nls_set_material(self.h, law, None, _ptr(k), _ptr(f)), "nls_set_material")
        else:
            params = np.array([p.young, p.poisson], dtype=np.float64)
            self._check(self.lib.nls_set_material(self.h, law, _ptr(params), None, None), "nls_set_material")
            if p.lambda_mode != LAMBDA_PRINTED:
                self.set_lambda_mode(p.lambda_mode)
            if p.f_vol is not None:
                self.set_volume_force(p.f_vol)
        dofs = np.ascontiguousarray(p.dirichlet_dofs(), dtype=np.int64)
        vals = np.zeros(dofs.shape[0])
        self._check(self.lib.nls_set_dirichlet(self.h, dofs.shape[0], _ptr(dofs), _ptr(vals)), "nls_set_dirichlet")
        if p.traction_edges is not None:
            e = np.ascontiguousarray(p.traction_edges, dtype=np.int32)
            t = np.ascontiguousarray(p.traction, dtype=np.float64)
            self._check(self.lib.nls_set_traction(self.h, e.shape[0], _ptr(e), _ptr(t)), "nls_set_traction")
        e2s = np.ascontiguousarray(p.elem_to_sub, dtype=np.int32)
        self._check(self.lib.nls_set_partition(self.h, p.n_sub, _ptr(e2s), p.overlap), "nls_set_partition")
        self.n_sub = p.n_sub

    def set_coarse(self, kind: int):
        self._check(self.lib.nls_set_coarse(self.h, kind), "nls_set_coarse")

    def set_options(self, **kw) -> Options:
        o = Options()
        self._check(self.lib.nls_get_options(self.h, ctypes.byref(o)), "nls_get_options")
        for k, v in kw.items():
            if k == "coupling" and isinstance(v, str):
                v = COUPLING[v]
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        self._check(self.lib.nls_set_options(self.h, ctypes.byref(o)), "nls_set_options")
        return o

    def setup(self):
        self._check(self.lib.nls_setup(self.h), "nls_setup")

    def setup_host(self):
        """Integer maps only (no GPU needed)."""
        self._check(self.lib.nls_setup_host(self.h), "nls_setup_host")

    # -- solve ----------------------------------------------------------------------------
    def solve(self, u=None):
        """Solve F(u) = 0; u (numpy host array or torch CUDA tensor) is overwritten."""
        if u is None:
            u = np.zeros(self.n_nodes * self.ndof)
        rep = Report()
        st = self.lib.nls_solve(self.h, _ptr(u), _is_device(u), ctypes.byref(rep))
        self._check(st, "nls_solve")
        return u, rep

    # -- inspection / parity hooks --------------------------------------------------------
    def sizes(self) -> Sizes:
        s = Sizes()
        self._check(self.lib.nls_get_sizes(self.h, ctypes.byref(s)), "nls_get_sizes")
        return s

    def local_dofs(self, sub: int):
        n = ctypes.c_int64()
        self._check(self.lib.nls_get_local_dofs(self.h, sub, 0, None, None, ctypes.byref(n)), "nls_get_local_dofs")
        dofs = np.zeros(n.value, dtype=np.int64)
        owned = np.zeros(n.value, dtype=np.uint8)
        self._check(self.lib.nls_get_local_dofs(self.h, sub, n.value, _ptr(dofs), _ptr(owned), ctypes.byref(n)),
                    "nls_get_local_dofs")
        return dofs, owned.astype(bool)

    def overlap_elems(self, sub: int) -> np.ndarray:
        n = ctypes.c_int64()
        self._check(self.lib.nls_get_overlap_elems(self.h, sub, 0, None, ctypes.byref(n)), "nls_get_overlap_elems")
        out = np.zeros(n.value, dtype=np.int32)
        self._check(self.lib.nls_get_overlap_elems(self.h, sub, n.value, _ptr(out), ctypes.byref(n)),
                    "nls_get_overlap_elems")
        return out

    def owners(self) -> np.ndarray:
        out = np.zeros(self.n_nodes, dtype=np.int32)
        self._check(self.lib.nls_get_owners(self.h, _ptr(out)), "nls_get_owners")
        return out

    def coarse_nodes(self) -> np.ndarray:
        out = np.zeros(self.sizes().n_coarse_nodes, dtype=np.int32)
        self._check(self.lib.nls_get_coarse_nodes(self.h, _ptr(out)), "nls_get_coarse_nodes")
        return out

    def coarse_basis(self) -> np.ndarray:
        s = self.sizes()
        out = np.zeros((s.n_coarse_dofs, s.n_dofs), dtype=np.float64)  # column-major N x N0
        self._check(self.lib.nls_get_coarse_basis(self.h, _ptr(out)), "nls_get_coarse_basis")
        return out.T

    def coarse_matrix(self) -> np.ndarray:
        """A_0 of the last tangent phase in band storage [n_coarse_dofs, 2 b0 + 1] (FP64)."""
        s = self.sizes()
        out = np.zeros((s.n_coarse_dofs, 2 * s.coarse_half_band + 1), dtype=np.float64)
        self._check(self.lib.nls_get_coarse_matrix(self.h, _ptr(out)), "nls_get_coarse_matrix")
        return out

    def eval_F(self, u, load: float = 1.0):
        F = np.zeros_like(u) if isinstance(u, np.ndarray) else u.new_zeros(u.shape)
        self._check(self.lib.nls_eval_F(self.h, _ptr(u), _ptr(F), _is_device(u), load), "nls_eval_F")
        return F

    def eval_Fx(self, u, load: float = 1.0):
        Fx = np.zeros_like(u) if isinstance(u, np.ndarray) else u.new_zeros(u.shape)
        its = np.zeros(self.n_sub, dtype=np.int32)
        st = np.zeros(self.n_sub, dtype=np.int32)
        self._check(self.lib.nls_eval_Fx(self.h, _ptr(u), _ptr(Fx), _is_device(u), load, _ptr(its), _ptr(st)),
                    "nls_eval_Fx")
        return Fx, its, st

    def apply_tangent(self, v):
        y = np.zeros_like(v) if isinstance(v, np.ndarray) else v.new_zeros(v.shape)
        self._check(self.lib.nls_apply_tangent(self.h, _ptr(v), _ptr(y), _is_device(v)), "nls_apply_tangent")
        return y

    def kernel_stats(self) -> dict:
        """{kernel: (launches, total ms)} accumulated while the profile_kernels option is set."""
        cap = 64
        arr = (KernelStat * cap)()
        n = ctypes.c_int32()
        self._check(self.lib.nls_get_kernel_stats(self.h, cap, arr, ctypes.byref(n)), "nls_get_kernel_stats")
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}

    def set_volume_force(self, f_vol=None):
        """Neo-Hooke volume force per element [n_elems, 2] at load factor 1 (None removes it)."""
        f = None if f_vol is None else np.ascontiguousarray(f_vol, dtype=np.float64).reshape(-1)
        self._check(self.lib.nls_set_volume_force(self.h, _ptr(f)), "nls_set_volume_force")

    def set_lambda_mode(self, mode: int):
        """Lame lambda of Eq. 2: LAMBDA_PRINTED or LAMBDA_PLANE_STRESS (before setup)."""
        self._check(self.lib.nls_set_lambda_mode(self.h, int(mode)), "nls_set_lambda_mode")

    def set_coefficients(self, k_elem=None, f_elem=None):
        """New per-element k and f (diffusion), keeping the maps of the current setup."""
        k = None if k_elem is None else np.ascontiguousarray(k_elem, dtype=np.float64)
        f = None if f_elem is None else np.ascontiguousarray(f_elem, dtype=np.float64)
        self._check(self.lib.nls_set_coefficients(self.h, _ptr(k), _ptr(f)), "nls_set_coefficients")

    def tuning(self) -> dict:
        """CTA sizes in use (autotuned or fixed) and the number of captured GMRES iteration graphs."""
        t = Tuning()
        self._check(self.lib.nls_get_tuning(self.h, ctypes.byref(t)), "nls_get_tuning")
        return t.as_dict()

    def reset_kernel_stats(self):
        self._check(self.lib.nls_reset_kernel_stats(self.h), "nls_reset_kernel_stats")

    def _device_tensor(self, t, name: str, dtype_name: str, numel: int, optional: bool = False):
        """Check that t is a contiguous CUDA tensor on this context's device with the given dtype
        and length: the allocation-free call hands raw device pointers to the kernel, so a host
        array, a short tensor or a wrong element type must be refused here, before any launch."""
        if t is None:
            if optional:
                return
            raise ValueError(f"{name} is required")
        if isinstance(t, np.ndarray) or not getattr(t, "is_cuda", False):
            raise ValueError(f"{name} must be a CUDA torch tensor (got {type(t).__name__})")
        if t.device.index != self.device:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{self.device}")
        if str(t.dtype) != "torch." + dtype_name:
            raise ValueError(f"{name} must be {dtype_name} (got {t.dtype})")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() != numel:
            raise ValueError(f"{name} must have {numel} entries (got {t.numel()})")

    def local_corrections_noalloc(self, x, Fx, its=None, status=None, load: float = 1.0):
        """One-level corrections into the caller's device tensor Fx, using no allocation (see nls.h).
        x, Fx: float64 CUDA tensors of n_dofs entries; its, status (optional): int32 CUDA tensors of
        n_sub entries, all on the context's device; ValueError otherwise (nothing is launched)."""
        n = self.n_nodes * self.ndof
        self._device_tensor(x, "x", "float64", n)
        self._device_tensor(Fx, "Fx", "float64", n)
        self._device_tensor(its, "its", "int32", self.n_sub, optional=True)
        self._device_tensor(status, "status", "int32", self.n_sub, optional=True)
        self._check(self.lib.nls_local_corrections_noalloc(self.h, _ptr(x), _ptr(Fx), _ptr(its), _ptr(status), load),
                    "nls_local_corrections_noalloc")
        return Fx

    def local_states(self) -> np.ndarray:
        out = np.zeros(self.sizes().total_local_dofs)
        self._check(self.lib.nls_get_local_states(self.h, _ptr(out), 0), "nls_get_local_states")
        return out


GUESS_USE, GUESS_HARVEST, GUESS_FIRST_OUTER = 1, 2, 4
GUESS_FEATURES, GUESS_OUTPUTS = 391, 1024              # scalar kind (Eq. 1)
GUESS_FEATURES_DISP, GUESS_OUTPUTS_DISP = 267, 2048    # displacement kind (Eq. 2)
GUESS_KIND_SCALAR, GUESS_KIND_DISPLACEMENT = 0, 1


class GuessNet:
    """The learned-initial-guess network (include/nls.h); host arrays are numpy float32."""

    def __init__(self, h1: int = 512, h2: int = 512, seed: int = 1, capacity: int = 0, device: int = 0,
                 kind: int = GUESS_KIND_SCALAR):
        self.lib = load()
        self.h = _P()
        st = self.lib.nls_guess_create_kind(ctypes.byref(self.h), device, kind, h1, h2, seed, capacity)
        if st < 0:
            raise NLSError(st, "nls_guess_create_kind", "")
        self.h1, self.h2 = h1, h2
        k, ni, no = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.nls_guess_dims(self.h, ctypes.byref(k), ctypes.byref(ni), ctypes.byref(no)),
                    "nls_guess_dims")
        self.kind, self.n_in, self.n_out = k.value, ni.value, no.value

    def close(self):
        if self.h:
            self.lib.nls_guess_destroy(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where):
        if st < 0:
            raise NLSError(st, where, "")

    def pairs(self) -> int:
        n = ctypes.c_int64()
        self._check(self.lib.nls_guess_pairs(self.h, ctypes.byref(n)), "nls_guess_pairs")
        return n.value

    def params(self) -> np.ndarray:
        n = ctypes.c_int64()
        self._check(self.lib.nls_guess_get_params(self.h, None, ctypes.byref(n)), "nls_guess_get_params")
        out = np.zeros(n.value, dtype=np.float32)
        self._check(self.lib.nls_guess_get_params(self.h, _ptr(out), ctypes.byref(n)), "nls_guess_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.nls_guess_set_params(self.h, _ptr(p), p.shape[0]), "nls_guess_set_params")

    def normalisation(self):
        mean = np.zeros(self.n_in, dtype=np.float32)
        scale = np.zeros(self.n_in, dtype=np.float32)
        ts = ctypes.c_float()
        self._check(self.lib.nls_guess_get_normalisation(self.h, _ptr(mean), _ptr(scale), ctypes.byref(ts)),
                    "nls_guess_get_normalisation")
        return mean, scale, ts.value

    def set_normalisation(self, mean, scale, tscale: float):
        mean = np.ascontiguousarray(mean, dtype=np.float32)
        scale = np.ascontiguousarray(scale, dtype=np.float32)
        if mean.shape != (self.n_in,) or scale.shape != (self.n_in,):
            raise ValueError(f"mean and scale need {self.n_in} entries")
        self._check(self.lib.nls_guess_set_normalisation(self.h, _ptr(mean), _ptr(scale), tscale),
                    "nls_guess_set_normalisation")

    def gradient(self, X: np.ndarray, T: np.ndarray, bf16: bool = False):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != self.n_in or T.shape != (X.shape[0], self.n_out):
            raise ValueError(f"X must be [B, {self.n_in}] and T [B, {self.n_out}]")
        g = np.zeros(self.params().shape[0], dtype=np.float32)
        L = ctypes.c_float()
        self._check(self.lib.nls_guess_gradient(self.h, X.shape[0], _ptr(X), _ptr(T), 1 if bf16 else 0, _ptr(g),
                                                ctypes.byref(L)), "nls_guess_gradient")
        return g, L.value

    def forward(self, X: np.ndarray) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != self.n_in:
            raise ValueError(f"X must be [B, {self.n_in}]")
        Y = np.zeros((X.shape[0], self.n_out), dtype=np.float32)
        self._check(self.lib.nls_guess_forward(self.h, X.shape[0], _ptr(X), _ptr(Y)), "nls_guess_forward")
        return Y

    def train(self, steps: int, batch: int = 256, lr: float = 1e-3, seed: int = 7) -> np.ndarray:
        losses = np.zeros(steps, dtype=np.float32)
        self._check(self.lib.nls_guess_train(self.h, steps, batch, lr, seed, _ptr(losses)), "nls_guess_train")
        return losses

    def split(self, flat: np.ndarray):
        """[(W, b)] of the three layers from a flat parameter array."""
        sizes = [self.n_in, self.h1, self.h2, self.n_out]
        out, o = [], 0
        for fi, fo in zip(sizes[:-1], sizes[1:]):
            W = flat[o:o + fo * fi].reshape(fo, fi)
            o += fo * fi
            b = flat[o:o + fo]
            o += fo
            out.append((W, b))
        return out


def attach_guess(solver: "Solver", net: "GuessNet", mode: int):
    solver._check(solver.lib.nls_guess_attach(solver.h, net.h if net else None, mode), "nls_guess_attach")
    solver._guess_dims = (net.n_in, net.n_out) if (net and mode) else None


def _attached_dims(solver: "Solver"):
    dims = getattr(solver, "_guess_dims", None)
    if dims is None:
        raise ValueError("the learned-guess hooks need an attached network")
    return dims


def set_guess_smoothing(solver: "Solver", sweeps: int, omega: float = 0.8):
    solver._check(solver.lib.nls_guess_set_smoothing(solver.h, sweeps, omega), "nls_guess_set_smoothing")


def guess_features(solver: "Solver", x: np.ndarray, load: float = 1.0) -> np.ndarray:
    """Raw inputs [n_sub, n_in] of every subdomain at x (test hook; needs an attached network)."""
    n_in, _ = _attached_dims(solver)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = solver.n_nodes * solver.ndof
    if x.shape != (n,):
        raise ValueError(f"x must have {n} entries")
    out = np.zeros((solver.n_sub, n_in), dtype=np.float32)
    solver._check(solver.lib.nls_guess_features(solver.h, _ptr(x), load, _ptr(out)), "nls_guess_features")
    return out


def guess_decode(solver: "Solver", x: np.ndarray, Y: np.ndarray, load: float = 1.0) -> np.ndarray:
    """Proposal (concatenated local unknowns) decoded from network outputs Y [n_sub, n_out] at x."""
    _, n_out = _attached_dims(solver)
    x = np.ascontiguousarray(x, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    n = solver.n_nodes * solver.ndof
    if x.shape != (n,) or Y.shape != (solver.n_sub, n_out):
        raise ValueError(f"x must have {n} entries and Y be [{solver.n_sub}, {n_out}]")
    out = np.zeros(solver.sizes().total_local_dofs)
    solver._check(solver.lib.nls_guess_decode(solver.h, _ptr(x), load, _ptr(Y), _ptr(out)), "nls_guess_decode")
    return out


def guess_smooth(solver: "Solver", x: np.ndarray, w: np.ndarray, load: float = 1.0) -> np.ndarray:
    """The smoothing of given starts w (concatenated local unknowns) at x."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n, nt = solver.n_nodes * solver.ndof, solver.sizes().total_local_dofs
    if x.shape != (n,) or w.shape != (nt,):
        raise ValueError(f"x must have {n} entries and w {nt}")
    out = np.zeros_like(w)
    solver._check(solver.lib.nls_guess_smooth(solver.h, _ptr(x), load, _ptr(w), _ptr(out)), "nls_guess_smooth")
    return out


def guess_counts(solver: "Solver"):
    p, a = ctypes.c_int64(), ctypes.c_int64()
    solver._check(solver.lib.nls_guess_counts(solver.h, ctypes.byref(p), ctypes.byref(a)), "nls_guess_counts")
    return p.value, a.value


def band_solve(band: np.ndarray, rhs: np.ndarray, precision: int = PREC_FP32_IR, method: int = COARSE_FACTOR_TILES,
               device: int = 0, want_factors: bool = False):
    """Factor the band matrix band [n, 2b + 1] with the coarse factorization and solve band x = rhs
    (include/nls.h nls_band_solve); returns x, or (x, factors in the same band layout)."""
    lib = load()
    band = np.ascontiguousarray(band, dtype=np.float64)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    n, w = band.shape
    x = np.zeros(n)
    fac = np.zeros_like(band) if want_factors else None
    st = lib.nls_band_solve(device, n, (w - 1) // 2, _ptr(band), _ptr(rhs), _ptr(x), precision, method, _ptr(fac))
    if st < 0:
        raise NLSError(st, "nls_band_solve", "")
    return (x, fac) if want_factors else x


def make_solver(p: Problem, coupling: str = "hybrid", precision: str = "fp32", coarse: Optional[bool] = None,
                device: int = 0, setup: bool = True, **opts) -> Solver:
    """Context for a problem from ``paper_2410_24138_gb300.inputs`` with the given options."""
    s = Solver(device)
    s.set_problem(p)
    use_coarse = (coupling != "one") if coarse is None else coarse
    s.set_coarse(COARSE_RGDSW if use_coarse else COARSE_NONE)
    prec = PREC_FP32_IR if precision == "fp32" else PREC_FP64
    kw = dict(coupling=COUPLING[coupling], local_precision=prec, coarse_precision=prec, load_steps=p.load_steps)
    kw.update(opts)
    s.set_options(**kw)
    if setup == "host":
        s.setup_host()
    elif setup:
        s.setup()
    return s
