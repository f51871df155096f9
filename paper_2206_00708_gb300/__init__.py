"""Thin Python binding of libbem.so, the GB300 library for acoustic transmission
through a penetrable object with nonconforming grids (arXiv 2206.00708).

Argument marshalling only: every numerical step runs in the CUDA library behind
the C ABI of `include/bem.h`.  The functions keep the C names.  Host arrays are
NumPy arrays; device arrays are CUDA torch tensors (PyTorch provides device
memory and streams, nothing else).  A missing library raises at import time:
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libbem.so")

BEM_OK = 0
BEM_E_INVALID_ARG = -1
BEM_E_OOM = -2
BEM_E_NOT_CONVERGED = -3
BEM_E_NONFINITE = -4
BEM_E_TIMEOUT = -5
BEM_E_ADMISSION_REFUSED = -6
BEM_E_BUSY = -7
BEM_E_CUDA = -8
BEM_E_INTERNAL = -9
BEM_E_CANCELLED = -10

BEM_OP_V, BEM_OP_K, BEM_OP_T, BEM_OP_D = 0, 1, 2, 3
BEM_PREC_FP64 = 0
BEM_PREC_MIXED = 1
BEM_MTF_DERIVED, BEM_MTF_PRINTED = 0, 1
BEM_FORM_MTF, BEM_FORM_PMCHWT, BEM_FORM_MULLER, BEM_FORM_PMCHWT_INT, BEM_FORM_MULLER_INT = 0, 1, 2, 3, 4
BEM_FORM_HC_EXT_NEU, BEM_FORM_HC_EXT_DIR, BEM_FORM_HC_INT_NEU, BEM_FORM_HC_INT_DIR = 5, 6, 7, 8


class BemError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"bem status {status}: {message}")
        self.status = status


class bem_c128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class bem_incident(C.Structure):
    _fields_ = [("n_rhs", C.c_int32), ("dirs", C.POINTER(C.c_double)), ("amps", C.POINTER(bem_c128)),
                ("kind", C.c_int32), ("sources", C.POINTER(C.c_double)), ("f", C.POINTER(bem_c128)),
                ("g", C.POINTER(bem_c128))]


BEM_INC_PLANE_WAVE, BEM_INC_POINT_SOURCE, BEM_INC_USER_TRACES = 0, 1, 2


def _incident(dirs=None, amps=None, sources=None, traces=None, on_device=False):
    """bem_incident for plane waves (dirs [n, 3]), point sources (sources [n, 3]) or the
    caller's weak-form data (traces = (f, g), each [n, N_ext]; f may be None for a
    screen; NumPy arrays, or CUDA tensors with on_device).  Returns (struct, n_rhs,
    arrays kept alive for the call)."""
    inc = bem_incident()
    keep = []
    given = [x is not None for x in (dirs, sources, traces)]
    if sum(given) != 1:
        raise ValueError("give exactly one of dirs, sources, traces")
    if traces is not None:
        f, g = traces
        inc.kind = BEM_INC_USER_TRACES
        n_rhs = None
        for name, a in (("f", f), ("g", g)):
            if a is None:
                continue
            if isinstance(a, np.ndarray):
                if on_device:
                    raise ValueError("traces must be CUDA tensors when on_device is set")
                a = np.ascontiguousarray(np.atleast_2d(a), dtype=np.complex128)
            elif not on_device:
                raise ValueError("traces must be NumPy arrays unless on_device is set")
            keep.append(a)
            n_rhs = int(a.shape[0]) if a.ndim == 2 else 1
            setattr(inc, name, C.cast(_ptr(a)[0], C.POINTER(bem_c128)))
        if n_rhs is None:
            raise ValueError("traces need g")
        inc.n_rhs = n_rhs
        return inc, n_rhs, keep
    pos = np.ascontiguousarray(np.atleast_2d(dirs if dirs is not None else sources), dtype=np.float64)
    keep.append(pos)
    n_rhs = pos.shape[0]
    inc.n_rhs = n_rhs
    if dirs is not None:
        inc.kind = BEM_INC_PLANE_WAVE
        inc.dirs = pos.ctypes.data_as(C.POINTER(C.c_double))
    else:
        inc.kind = BEM_INC_POINT_SOURCE
        inc.sources = pos.ctypes.data_as(C.POINTER(C.c_double))
    if amps is not None:
        amp_arr = (bem_c128 * n_rhs)(*[_c128(a) for a in np.atleast_1d(amps)])
        keep.append(amp_arr)
        inc.amps = C.cast(amp_arr, C.POINTER(bem_c128))
    return inc, n_rhs, keep


class bem_solve_opts(C.Structure):
    _fields_ = [
        ("gmres_tol", C.c_double),
        ("gmres_maxiter", C.c_int32),
        ("precision", C.c_int32),
        ("n_singular", C.c_int32),
        ("mtf_variant", C.c_int32),
        ("center", C.c_double * 3),
        ("ir_inner_tol", C.c_double),
        ("batch_columns", C.c_int32),
        ("tensor_cores", C.c_int32),
        ("formulation", C.c_int32),
        ("dd_switch", C.c_double),
        ("cuda_graphs", C.c_int32),
    ]


class bem_instance(C.Structure):
    _fields_ = [
        ("ext", C.c_void_p),
        ("intr", C.c_void_p),
        ("k_ext", bem_c128),
        ("k_int", bem_c128),
        ("rho_int_over_rho_ext", C.c_double),
        ("dir", C.c_double * 3),
        ("amp", bem_c128),
        ("v_ext", C.c_void_p),
        ("w_ext", C.c_void_p),
        ("v_int", C.c_void_p),
        ("w_int", C.c_void_p),
    ]


class bem_solve_report(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32),
        ("converged", C.c_int32),
        ("residual", C.c_double),
        ("t_assembly_ms", C.c_double),
        ("t_mortar_ms", C.c_double),
        ("t_solve_ms", C.c_double),
        ("mtf_variant", C.c_int32),
        ("outer_iterations", C.c_int32),
    ]


class bem_server_opts(C.Structure):
    _fields_ = [
        ("device", C.c_int32),
        ("max_inflight", C.c_int32),
        ("hbm_budget_bytes", C.c_int64),
        ("precision", C.c_int32),
        ("gmres_maxiter", C.c_int32),
        ("gmres_tol", C.c_double),
        ("dry_run", C.c_int32),
        ("group_max", C.c_int32),
        ("dry_run_us_per_unknown", C.c_double),
    ]


class bem_request(C.Structure):
    _fields_ = [
        ("xyz_ext", C.c_void_p), ("nv_ext", C.c_int64), ("tri_ext", C.c_void_p), ("nt_ext", C.c_int64),
        ("xyz_int", C.c_void_p), ("nv_int", C.c_int64), ("tri_int", C.c_void_p), ("nt_int", C.c_int64),
        ("k_ext", bem_c128), ("k_int", bem_c128),
        ("rho_int_over_rho_ext", C.c_double),
        ("n_rhs", C.c_int32),
        ("precision", C.c_int32),
        ("dirs", C.c_void_p),
        ("amps", C.c_void_p),
        ("timeout_ms", C.c_double),
    ]


class bem_result(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iterations", C.c_int32), ("residual", C.c_double),
        ("queue_ms", C.c_double), ("run_ms", C.c_double), ("total_ms", C.c_double),
        ("nv_ext", C.c_int64), ("nv_int", C.c_int64), ("n_rhs", C.c_int32), ("precision", C.c_int32),
        ("bytes_reserved", C.c_int64),
        ("group_size", C.c_int32), ("group_waves", C.c_int32),
    ]


class bem_serve_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("submitted", "completed", "refused", "cancelled", "timed_out", "failed",
                                         "queued", "running", "hbm_budget_bytes", "hbm_reserved_bytes",
                                         "hbm_high_water_bytes", "groups", "grouped")]


_VP = C.c_void_p
_PVP = C.POINTER(C.c_void_p)
_I64 = C.c_int64
_PI64 = C.POINTER(C.c_int64)

_SIGNATURES = {
    "bem_last_error": (C.c_char_p, []),
    "bem_version": (C.c_char_p, []),
    "bem_launch_count": (C.c_uint64, []),
    "bem_selftest": (C.c_int32, [_VP, C.c_int, C.POINTER(C.c_double)]),
    "bem_profile_enable": (None, [C.c_int]),
    "bem_profile_select": (None, [C.c_char_p]),
    "bem_profile_reset": (None, []),
    "bem_autotune": (C.c_int32, [_VP, _VP, _VP, C.c_int32]),
    "bem_context_set_exclusive": (C.c_int32, [_VP, C.c_int]),
    "bem_solve_screen": (C.c_int32, [_VP, _VP, _VP, bem_c128, _VP, _VP, C.c_int32, _VP, C.c_int, _VP]),
    "bem_tune_get": (C.c_int32, [C.c_char_p, C.c_int32, _I64, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double)]),
    "bem_tune_count": (C.c_int32, []),
    "bem_tune_clear": (None, []),
    "bem_tune_save": (C.c_int32, [C.c_char_p]),
    "bem_tune_load": (C.c_int32, [C.c_char_p]),
    "bem_profile_count": (C.c_int, []),
    "bem_profile_get": (C.c_int32, [C.c_int, C.c_char_p, C.c_int, C.POINTER(C.c_double), _PI64]),
    "bem_context_create": (C.c_int32, [C.c_int, _VP, _PVP]),
    "bem_context_destroy": (C.c_int32, [_VP]),
    "bem_context_synchronize": (C.c_int32, [_VP]),
    "bem_grid_create": (C.c_int32, [_VP, _VP, _I64, _VP, _I64, C.c_int, _PVP]),
    "bem_grid_destroy": (C.c_int32, [_VP]),
    "bem_grid_num_vertices": (C.c_int64, [_VP]),
    "bem_grid_num_triangles": (C.c_int64, [_VP]),
    "bem_assemble": (C.c_int32, [_VP, C.c_int, bem_c128, _VP, _VP, C.c_int, C.c_int, _PVP]),
    "bem_matrix_destroy": (C.c_int32, [_VP]),
    "bem_matrix_copy_out": (C.c_int32, [_VP, _VP, _VP, _I64, C.c_int]),
    "bem_matrix_entry_bytes": (C.c_int, [_VP]),
    "bem_matrix_shape": (C.c_int32, [_VP, _PI64, _PI64]),
    "bem_mass": (C.c_int32, [_VP, _VP, _PVP]),
    "bem_projection": (C.c_int32, [_VP, _VP, _VP, C.POINTER(C.c_double), _PVP]),
    "bem_projection_noalloc": (C.c_int32, [_VP, _VP, _VP, C.POINTER(C.c_double), _VP, _VP, _VP, _I64, _PI64]),
    "bem_sparse_destroy": (C.c_int32, [_VP]),
    "bem_sparse_info": (C.c_int32, [_VP, _PI64, _PI64, _PI64]),
    "bem_sparse_copy_out": (C.c_int32, [_VP, _VP, _VP, _VP, _VP, _I64]),
    "bem_solve_opts_default": (None, [C.POINTER(bem_solve_opts)]),
    "bem_serve_opts_default": (None, [C.POINTER(bem_server_opts)]),
    "bem_serve_create": (C.c_int32, [C.POINTER(bem_server_opts), _PVP]),
    "bem_serve_destroy": (C.c_int32, [_VP]),
    "bem_serve_submit": (C.c_int32, [_VP, C.POINTER(bem_request), C.POINTER(C.c_uint64)]),
    "bem_serve_poll": (C.c_int32, [_VP, C.c_uint64, C.POINTER(bem_result), _VP, _VP, _VP, _VP]),
    "bem_serve_wait": (C.c_int32, [_VP, C.c_uint64, C.c_double]),
    "bem_serve_cancel": (C.c_int32, [_VP, C.c_uint64]),
    "bem_serve_get_stats": (C.c_int32, [_VP, C.POINTER(bem_serve_stats)]),
    "bem_solve_many": (C.c_int32, [_VP, C.c_int32, _VP, _VP, C.c_int, _VP]),
    "bem_field": (C.c_int32, [_VP, _VP, bem_c128, _VP, _VP, _VP, _I64, _VP, C.c_int]),
    "bem_solve_transmission": (C.c_int32, [_VP, _VP, _VP, bem_c128, bem_c128, C.c_double,
                                           C.POINTER(bem_incident), C.POINTER(bem_solve_opts),
                                           _VP, _VP, _VP, _VP, C.c_int, C.POINTER(bem_solve_report)]),
}


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(the GB300 path has no CPU fallback)")
    lib = C.CDLL(_LIB_PATH, mode=C.RTLD_GLOBAL)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def library():
    """The loaded ctypes library (for tests that check the exported symbols)."""
    return _lib


def library_path():
    return _LIB_PATH


def _check(status):
    if status != BEM_OK:
        raise BemError(status, _lib.bem_last_error().decode())
    return status


def _c128(z):
    z = complex(z)
    return bem_c128(z.real, z.imag)


def _ptr(a):
    """Data pointer of a NumPy array (host) or a torch tensor (device)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return C.c_void_p(a.ctypes.data), False
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), bool(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


# ------------------------------------------------------------------ context / grids
def bem_version():
    return _lib.bem_version().decode()


def bem_launch_count():
    return int(_lib.bem_launch_count())


def bem_selftest(ctx, which=0):
    r = C.c_double()
    _check(_lib.bem_selftest(ctx, int(which), C.byref(r)))
    return r.value


def bem_profile_enable(on=True):
    _lib.bem_profile_enable(int(bool(on)))


def bem_profile_select(prefixes=None):
    """Time only kernels whose names start with one of `prefixes` (list of str); None: all."""
    _lib.bem_profile_select(",".join(prefixes).encode() if prefixes else None)


def bem_profile_reset():
    _lib.bem_profile_reset()


BEM_SCREEN_MASS, BEM_SCREEN_OO = 0, 1


def bem_solve_screen(ctx, screen, k, dirs=None, coarse=None, precond=BEM_SCREEN_MASS, amps=None, opts=None, out=None,
                     on_device=False, sources=None, traces=None):
    """Neumann screen D phi = gamma_N u_inc (mass or opposite-order preconditioning), for
    plane waves (dirs), point sources (sources) or the caller's data (traces = (None, g)).

    Returns (phi [n_rhs, N] complex128 (zero on the screen's boundary), report dict);
    raises BemError on failure (BEM_E_NOT_CONVERGED with .outputs and .report)."""
    inc, n_rhs, _keep = _incident(dirs, amps, sources, traces, on_device)
    o = _opts(opts)
    N = bem_grid_num_vertices(screen)
    if out is None:
        if on_device:
            raise ValueError("device outputs must be preallocated")
        out = np.zeros((n_rhs, N), dtype=np.complex128)
    rep = bem_solve_report()
    st = _lib.bem_solve_screen(ctx, screen, coarse, _c128(k), C.byref(inc), C.byref(o), int(precond), _ptr(out)[0],
                               int(bool(on_device)), C.byref(rep))
    report = {f: getattr(rep, f) for f, _ in bem_solve_report._fields_}
    if st != BEM_OK:
        err = BemError(st, _lib.bem_last_error().decode())
        err.outputs, err.report = out, report
        raise err
    return out, report


def bem_autotune(ctx, ext, intr, n_rhs=1):
    """Time the candidate launch shapes for these grids' sizes and keep the fastest."""
    _check(_lib.bem_autotune(ctx, ext, intr, int(n_rhs)))


def bem_tune_get(kernel, width, rows):
    """(block, variant, ms) chosen for (kernel, width, rows); block 0: no entry."""
    b, v, ms = C.c_int32(), C.c_int32(), C.c_double()
    _check(_lib.bem_tune_get(kernel.encode(), int(width), int(rows), C.byref(b), C.byref(v), C.byref(ms)))
    return b.value, v.value, ms.value


def bem_tune_count():
    return int(_lib.bem_tune_count())


def bem_tune_clear():
    _lib.bem_tune_clear()


def bem_tune_save(path):
    _check(_lib.bem_tune_save(os.fsencode(path)))


def bem_tune_load(path):
    _check(_lib.bem_tune_load(os.fsencode(path)))


def bem_profile_count():
    return int(_lib.bem_profile_count())


def bem_profile_get(index):
    """(kernel name, total device ms, launches) of the index-th profiled kernel."""
    buf = C.create_string_buffer(256)
    ms, n = C.c_double(), C.c_int64()
    _check(_lib.bem_profile_get(int(index), buf, 256, C.byref(ms), C.byref(n)))
    return buf.value.decode(), ms.value, n.value


def bem_profile_table():
    """All profiled kernels as a list of (name, total ms, launches), longest first."""
    rows = [bem_profile_get(i) for i in range(bem_profile_count())]
    return sorted(rows, key=lambda r: -r[1])


def bem_context_create(device=0, stream=None):
    """stream: a torch.cuda.Stream, an integer cudaStream_t, or None (own stream)."""
    h = C.c_void_p()
    s = None
    if stream is not None:
        s = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(_lib.bem_context_create(int(device), s, C.byref(h)))
    _CTX_DEVICE[h.value] = int(device)
    return h


_CTX_DEVICE = {}  # context handle -> CUDA device index it was created on


def bem_context_device(ctx):
    """The CUDA device index of a context created by this binding (None if unknown)."""
    return _CTX_DEVICE.get(ctx.value if hasattr(ctx, "value") else ctx)


def bem_context_set_exclusive(ctx, exclusive=True):
    """True only if this context's solves never overlap with others on the device: the
    mass inverses then run as one cooperative launch each (default False: step launches
    replayed as CUDA graphs)."""
    _check(_lib.bem_context_set_exclusive(ctx, int(bool(exclusive))))


def bem_context_destroy(ctx):
    _check(_lib.bem_context_destroy(ctx))
    _CTX_DEVICE.pop(ctx.value if hasattr(ctx, "value") else ctx, None)


def bem_context_synchronize(ctx):
    _check(_lib.bem_context_synchronize(ctx))


def bem_grid_create(ctx, xyz, tri):
    """xyz float64 [N,3], tri int32 [T,3]: both NumPy (host) or both CUDA tensors."""
    if isinstance(xyz, np.ndarray):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
    px, dx = _ptr(xyz)
    pt, dt = _ptr(tri)
    if dx != dt:
        raise ValueError("xyz and tri must both be on the host or both on the device")
    h = C.c_void_p()
    _check(_lib.bem_grid_create(ctx, px, int(xyz.shape[0]), pt, int(tri.shape[0]), int(dx), C.byref(h)))
    return h


def bem_grid_destroy(g):
    _check(_lib.bem_grid_destroy(g))


def bem_grid_num_vertices(g):
    return int(_lib.bem_grid_num_vertices(g))


def bem_grid_num_triangles(g):
    return int(_lib.bem_grid_num_triangles(g))


# ------------------------------------------------------------------ operators
def bem_assemble(ctx, op, k, test, trial=None, precision=BEM_PREC_FP64, n_singular=4):
    h = C.c_void_p()
    _check(_lib.bem_assemble(ctx, int(op), _c128(k), test, trial if trial is not None else test,
                             int(precision), int(n_singular), C.byref(h)))
    return h


def bem_matrix_destroy(m):
    _check(_lib.bem_matrix_destroy(m))


def bem_matrix_shape(m):
    r, c = C.c_int64(), C.c_int64()
    _check(_lib.bem_matrix_shape(m, C.byref(r), C.byref(c)))
    return r.value, c.value


def bem_matrix_entry_bytes(m):
    return int(_lib.bem_matrix_entry_bytes(m))


def bem_matrix_copy_out(ctx, m, out=None):
    """Copy into `out` (complex128 NumPy array or CUDA tensor); allocates a NumPy
    array when out is None.  Returns out."""
    rows, cols = bem_matrix_shape(m)
    if out is None:
        dt = np.complex128 if bem_matrix_entry_bytes(m) == 16 else np.complex64
        out = np.empty((rows, cols), dtype=dt)
    p, dev = _ptr(out)
    nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
    _check(_lib.bem_matrix_copy_out(ctx, m, p, int(nbytes), int(dev)))
    return out


def bem_mass(ctx, g):
    h = C.c_void_p()
    _check(_lib.bem_mass(ctx, g, C.byref(h)))
    return h


def bem_projection(ctx, a, b, center=None):
    h = C.c_void_p()
    c = None
    if center is not None:
        c = (C.c_double * 3)(*[float(x) for x in center])
    _check(_lib.bem_projection(ctx, a, b, c, C.byref(h)))
    return h


def bem_projection_noalloc(ctx, a, b, row, col, val, center=None):
    """Mortar matrix into caller-owned device arrays (CUDA tensors int32, int32,
    float64 of equal length) without any device allocation by the library; for
    callers whose device memory comes from their own budgeted pool or whose loop
    cannot pay for an allocation.  Returns the number of COO entries written.  The
    library's fixed scratch array is shared by all calls: serialise calls."""
    import torch
    for name, t, dt in (("row", row, torch.int32), ("col", col, torch.int32), ("val", val, torch.float64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must have dtype {dt} (got {t.dtype})")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        dev = bem_context_device(ctx)
        if dev is not None and t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{dev}")
    c = None
    if center is not None:
        c = (C.c_double * 3)(*[float(x) for x in center])
    cap = min(int(row.numel()), int(col.numel()), int(val.numel()))
    n = C.c_int64()
    _check(_lib.bem_projection_noalloc(ctx, a, b, c, C.c_void_p(row.data_ptr()), C.c_void_p(col.data_ptr()),
                                       C.c_void_p(val.data_ptr()), cap, C.byref(n)))
    return n.value


def bem_sparse_destroy(s):
    _check(_lib.bem_sparse_destroy(s))


def bem_sparse_info(s):
    r, c, n = C.c_int64(), C.c_int64(), C.c_int64()
    _check(_lib.bem_sparse_info(s, C.byref(r), C.byref(c), C.byref(n)))
    return r.value, c.value, n.value


def bem_sparse_copy_out(ctx, s):
    """COO triplets (row int32, col int32, val float64); repeated entries add up."""
    _, _, nnz = bem_sparse_info(s)
    row = np.empty(nnz, dtype=np.int32)
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    _check(_lib.bem_sparse_copy_out(ctx, s, row.ctypes.data, col.ctypes.data, val.ctypes.data, nnz))
    return row, col, val


# ------------------------------------------------------------------ solve
def bem_solve_opts_default():
    o = bem_solve_opts()
    _lib.bem_solve_opts_default(C.byref(o))
    return o


def bem_solve_transmission(ctx, ext, intr, k_int, k_ext, rho_int_over_rho_ext, dirs=None, amps=None, opts=None,
                           out=None, on_device=False, sources=None, traces=None):
    """Solve the mass-preconditioned MTF (or opts["formulation"]) for plane waves
    `dirs` [n_rhs, 3], point sources `sources` [n_rhs, 3] (with amplitudes `amps`), or
    the caller's weak-form data `traces` = (f, g), each [n_rhs, N_ext].

    out: optional dict of preallocated outputs v_ext, w_ext [n_rhs, N_ext] and
    v_int, w_int [n_rhs, N_int] (complex128 NumPy arrays, or CUDA tensors with
    on_device=True).  Returns (outputs dict, report dict); raises BemError on
    failure (BEM_E_NOT_CONVERGED included, with the outputs attached as .outputs).
    """
    inc, n_rhs, _keep = _incident(dirs, amps, sources, traces, on_device)
    if opts is None:
        opts = bem_solve_opts_default()
    elif isinstance(opts, dict):
        o = bem_solve_opts_default()
        for key, val in opts.items():
            if key == "center":
                o.center = (C.c_double * 3)(*val)
            else:
                setattr(o, key, val)
        opts = o
    Ne, Ni = bem_grid_num_vertices(ext), bem_grid_num_vertices(intr)
    if out is None:
        if on_device:
            raise ValueError("device outputs must be preallocated")
        out = {k: np.zeros((n_rhs, n), dtype=np.complex128) for k, n in
               (("v_ext", Ne), ("w_ext", Ne), ("v_int", Ni), ("w_int", Ni))}
    ptrs = [_ptr(out[k])[0] for k in ("v_ext", "w_ext", "v_int", "w_int")]
    rep = bem_solve_report()
    st = _lib.bem_solve_transmission(ctx, ext, intr, _c128(k_int), _c128(k_ext), float(rho_int_over_rho_ext),
                                     C.byref(inc), C.byref(opts), *ptrs, int(bool(on_device)), C.byref(rep))
    report = {f: getattr(rep, f) for f, _ in bem_solve_report._fields_}
    if st != BEM_OK:
        err = BemError(st, _lib.bem_last_error().decode())
        err.outputs, err.report = out, report
        raise err
    return out, report


def bem_field(ctx, grid, k, points, phi=None, psi=None):
    """u [M] = V[psi] - K[phi] at points [M, 3] (host NumPy arrays); phi, psi: [N] or None."""
    pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    u = np.zeros(len(pts), dtype=np.complex128)
    ph = None if phi is None else np.ascontiguousarray(phi, dtype=np.complex128)
    ps = None if psi is None else np.ascontiguousarray(psi, dtype=np.complex128)
    _check(_lib.bem_field(ctx, grid, _c128(k), None if ph is None else ph.ctypes.data,
                          None if ps is None else ps.ctypes.data, pts.ctypes.data, len(pts), u.ctypes.data, 0))
    return u


def _opts(opts):
    if opts is None:
        return bem_solve_opts_default()
    if isinstance(opts, dict):
        o = bem_solve_opts_default()
        for key, val in opts.items():
            if key == "center":
                o.center = (C.c_double * 3)(*val)
            else:
                setattr(o, key, val)
        return o
    return opts


def bem_solve_many(ctx, problems, opts=None):
    """Solve many independent transmission problems together (mixed precision).

    problems: list of dicts with keys ext, intr (grid handles), k_ext, k_int, rho
    (rho_int / rho_ext), dir (3 floats, unit) and optional amp (default 1).
    Returns (list of output dicts v_ext, w_ext, v_int, w_int, list of report dicts);
    raises BemError on failure (with .outputs and .reports attached).
    """
    if opts is None or isinstance(opts, dict):
        opts = {"precision": BEM_PREC_MIXED, **(opts or {})}
    o = _opts(opts)
    n = len(problems)
    arr = (bem_instance * n)()
    outs = []
    for i, p in enumerate(problems):
        Ne, Ni = bem_grid_num_vertices(p["ext"]), bem_grid_num_vertices(p["intr"])
        out = {k: np.zeros(m, dtype=np.complex128) for k, m in
               (("v_ext", Ne), ("w_ext", Ne), ("v_int", Ni), ("w_int", Ni))}
        outs.append(out)
        q = arr[i]
        q.ext, q.intr = p["ext"], p["intr"]
        q.k_ext, q.k_int = _c128(p["k_ext"]), _c128(p["k_int"])
        q.rho_int_over_rho_ext = float(p["rho"])
        q.dir = (C.c_double * 3)(*[float(v) for v in p["dir"]])
        q.amp = _c128(p.get("amp", 1.0))
        q.v_ext, q.w_ext, q.v_int, q.w_int = [out[k].ctypes.data for k in ("v_ext", "w_ext", "v_int", "w_int")]
    reps = (bem_solve_report * n)()
    st = _lib.bem_solve_many(ctx, n, C.cast(arr, C.c_void_p), C.byref(o), 0, C.cast(reps, C.c_void_p))
    reports = [{f: getattr(r, f) for f, _ in bem_solve_report._fields_} for r in reps]
    if st != BEM_OK:
        err = BemError(st, _lib.bem_last_error().decode())
        err.outputs, err.reports = outs, reports
        raise err
    return outs, reports


# ------------------------------------------------------------------ serving
def bem_serve_opts_default():
    o = bem_server_opts()
    _lib.bem_serve_opts_default(C.byref(o))
    return o


def bem_serve_create(**kw):
    """Create a request server; keyword arguments override bem_server_opts fields."""
    o = bem_serve_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    h = C.c_void_p()
    _check(_lib.bem_serve_create(C.byref(o), C.byref(h)))
    return h


def bem_serve_destroy(srv):
    _check(_lib.bem_serve_destroy(srv))


def bem_serve_submit(srv, xyz_ext, tri_ext, xyz_int, tri_int, k_ext, k_int, rho_int_over_rho_ext, dirs,
                     amps=None, precision=-1, timeout_ms=0.0):
    """Queue one request (host arrays are copied); returns the ticket."""
    xe = np.ascontiguousarray(xyz_ext, dtype=np.float64)
    te = np.ascontiguousarray(tri_ext, dtype=np.int32)
    xi = np.ascontiguousarray(xyz_int, dtype=np.float64)
    ti = np.ascontiguousarray(tri_int, dtype=np.int32)
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    q = bem_request()
    q.xyz_ext, q.nv_ext, q.tri_ext, q.nt_ext = xe.ctypes.data, len(xe), te.ctypes.data, len(te)
    q.xyz_int, q.nv_int, q.tri_int, q.nt_int = xi.ctypes.data, len(xi), ti.ctypes.data, len(ti)
    q.k_ext, q.k_int = _c128(k_ext), _c128(k_int)
    q.rho_int_over_rho_ext = float(rho_int_over_rho_ext)
    q.n_rhs = d.shape[0]
    q.precision = int(precision)
    q.dirs = d.ctypes.data
    amp_arr = None
    if amps is not None:
        amp_arr = (bem_c128 * d.shape[0])(*[_c128(a) for a in np.atleast_1d(amps)])
        q.amps = C.cast(amp_arr, C.c_void_p)
    q.timeout_ms = float(timeout_ms)
    t = C.c_uint64()
    _check(_lib.bem_serve_submit(srv, C.byref(q), C.byref(t)))
    return t.value


def bem_serve_poll(srv, ticket):
    """None while the request is queued or running; otherwise its info dict (the
    request is released without copying traces; see bem_serve_take)."""
    info = bem_result()
    st = _lib.bem_serve_poll(srv, C.c_uint64(ticket), C.byref(info), None, None, None, None)
    if st == BEM_E_BUSY:
        return None
    _check(st)
    return {f: getattr(info, f) for f, _ in bem_result._fields_}


def bem_serve_take(srv, ticket, n_rhs, nv_ext, nv_int):
    """Like bem_serve_poll, copying the traces into new arrays of the given sizes."""
    info = bem_result()
    out = {"v_ext": np.zeros((n_rhs, nv_ext), dtype=np.complex128),
           "w_ext": np.zeros((n_rhs, nv_ext), dtype=np.complex128),
           "v_int": np.zeros((n_rhs, nv_int), dtype=np.complex128),
           "w_int": np.zeros((n_rhs, nv_int), dtype=np.complex128)}
    st = _lib.bem_serve_poll(srv, C.c_uint64(ticket), C.byref(info), out["v_ext"].ctypes.data,
                             out["w_ext"].ctypes.data, out["v_int"].ctypes.data, out["w_int"].ctypes.data)
    if st == BEM_E_BUSY:
        return None
    _check(st)
    return out, {f: getattr(info, f) for f, _ in bem_result._fields_}


def bem_serve_wait(srv, ticket, timeout_ms=0.0):
    """True once the request has finished, False on timeout."""
    st = _lib.bem_serve_wait(srv, C.c_uint64(ticket), float(timeout_ms))
    if st == BEM_E_BUSY:
        return False
    _check(st)
    return True


def bem_serve_cancel(srv, ticket):
    _check(_lib.bem_serve_cancel(srv, C.c_uint64(ticket)))


def bem_serve_get_stats(srv):
    st = bem_serve_stats()
    _check(_lib.bem_serve_get_stats(srv, C.byref(st)))
    return {f: getattr(st, f) for f, _ in bem_serve_stats._fields_}
