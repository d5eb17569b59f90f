"""Python binding of libnmg (include/nmg.h): argument marshalling only.

Every function has the name and the arguments of its C counterpart.  Pointer
arguments accept a torch tensor (device or host), a numpy array (host) or a
raw integer address.  Status codes are returned unchanged; ``check`` turns a
negative status into an :class:`NmgError` carrying nmg_last_error().  All
compute runs inside libnmg's CUDA kernels: there is no Python or CPU fallback,
and importing this module fails if the library has not been built.
"""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnmg.so")

NMG_OK = 0
NMG_PENDING = 1
NMG_ERR_INVALID = -1
NMG_ERR_OOM = -2
NMG_ERR_SINGULAR_PATCH = -3
NMG_ERR_NOT_CONVERGED = -4
NMG_ERR_NONFINITE = -5
NMG_ERR_TIMEOUT = -6
NMG_ERR_CUDA = -7

NMG_PREC_FP64 = 0
NMG_PREC_FP32 = 1
NMG_PREC_BF16 = 2

NMG_WEIGHT_AVERAGE = 0
NMG_WEIGHT_SUM = 1

NMG_ENGINE_AUTO = 0
NMG_ENGINE_KERNELS = 1
NMG_ENGINE_PERSISTENT = 2
NMG_ENGINE_FUSED = 3


class nmg_mesh_desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n", C.c_int * 3),
        ("levels", C.c_int),
        ("ncomp", C.c_int),
        ("patch_cells", C.c_int),
        ("dirichlet_mask", C.c_void_p),
        ("precisions", C.c_int),
        ("mem_budget_bytes", C.c_size_t),
        ("stream", C.c_void_p),
    ]


class nmg_solve_opts(C.Structure):
    _fields_ = [
        ("rtol", C.c_double),
        ("restart", C.c_int),
        ("maxit", C.c_int),
        ("nu1", C.c_int),
        ("nu2", C.c_int),
        ("omega", C.c_double),
        ("precision", C.c_int),
        ("weighting", C.c_int),
        ("use_graph", C.c_int),
        ("engine", C.c_int),
        ("tail_patches", C.c_int),
        ("tile_patches", C.c_int),
    ]


class nmg_solve_info(C.Structure):
    _fields_ = [
        ("iterations", C.c_int),
        ("restarts", C.c_int),
        ("rel_residual", C.c_double),
        ("ms_total", C.c_double),
        ("status", C.c_int),
        ("launches", C.c_int64),
        ("engine", C.c_int),
        ("device_loop", C.c_int),
    ]


class nmg_jacobian_reuse(C.Structure):
    _fields_ = [
        ("gamma", C.c_double),
        ("last", C.c_double),
        ("rate", C.c_double),
        ("have_last", C.c_int),
        ("have_jacobian", C.c_int),
        ("steps", C.c_int64),
        ("assemblies", C.c_int64),
    ]


class NmgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"nmg status {status}: {message}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libnmg.so is not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = C.CDLL(LIB_PATH)

_P = C.c_void_p
_H = C.c_void_p
_SIGS = {
    "nmg_default_opts": [C.POINTER(nmg_solve_opts)],
    "nmg_create_hierarchy": [C.POINTER(nmg_mesh_desc), C.POINTER(_H)],
    "nmg_set_jacobian": [_H, C.c_int, C.c_int64, C.c_int64, _P, _P, _P, C.c_int],
    "nmg_solve": [_H, _P, _P, C.POINTER(nmg_solve_opts), C.POINTER(nmg_solve_info)],
    "nmg_matvec": [_H, C.c_int, C.c_int, _P, _P],
    "nmg_residual": [_H, C.c_int, C.c_int, _P, _P, _P],
    "nmg_smooth": [_H, C.c_int, C.c_int, _P, _P, C.c_int, C.c_int, C.c_double, C.c_int],
    "nmg_restrict": [_H, C.c_int, C.c_int, _P, _P],
    "nmg_prolongate_add": [_H, C.c_int, C.c_int, _P, _P],
    "nmg_coarse_solve": [_H, C.c_int, _P, _P],
    "nmg_vcycle": [_H, C.POINTER(nmg_solve_opts), _P, _P],
    "nmg_vcycle_many": [_H, C.POINTER(nmg_solve_opts), C.c_int, _P, _P],
    "nmg_solve_many": [_H, C.c_int, _P, _P, C.POINTER(nmg_solve_opts), _P],
    "nmg_get_patch_inverses": [_H, C.c_int, C.c_int, C.c_int64, C.c_int64, _P],
    "nmg_hierarchy_bytes": [_H, C.POINTER(C.c_size_t)],
    "nmg_destroy_hierarchy": [_H],
    "nmg_profile_enable": [_H, C.c_int],
    "nmg_profile_read": [_H, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double)],
    "nmg_autotune_report": [_H, C.c_char_p, C.c_size_t],
    "nmg_server_create": [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)],
    "nmg_submit": [C.c_void_p, _H, _P, _P, C.POINTER(nmg_solve_opts), C.POINTER(C.c_uint64)],
    "nmg_poll": [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(nmg_solve_info)],
    "nmg_server_destroy": [C.c_void_p],
    "nmg_server_set_workspaces": [C.c_void_p, C.c_int],
    "nmg_server_set_batching": [C.c_void_p, C.c_int],
    "nmg_server_memory": [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)],
    "nmg_set_wait_limit": [_H, C.c_int],
    "nmg_set_lifting_operator": [_H, C.c_int64, C.c_int64, _P, _P, _P, C.c_int],
    "nmg_set_large_patches": [_H, _P],
    "nmg_patch_layout": [_H, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                         C.POINTER(C.c_int)],
    "nmg_deformation_update": [_H, _P, _P, C.c_double, _P, _P],
    "nmg_extension_rhs": [_H, _P, _P, _P],
    "nmg_newton_substeps": [_H, _H, _P, _P, C.c_double, _P, _P, _P, _P, C.POINTER(nmg_solve_opts),
                            C.POINTER(nmg_solve_opts), C.POINTER(nmg_solve_info), C.POINTER(nmg_solve_info)],
    "nmg_jacobian_reuse_init": [C.POINTER(nmg_jacobian_reuse), C.c_double],
    "nmg_jacobian_reuse_time_step": [C.POINTER(nmg_jacobian_reuse)],
    "nmg_jacobian_reuse_decide": [C.POINTER(nmg_jacobian_reuse), C.c_double, C.POINTER(C.c_int)],
    "nmg_vanka_correct_noalloc": [C.c_int, C.POINTER(C.c_int), C.c_int, _P, C.c_int64, _P, _P, C.c_double,
                                  C.c_int, C.c_int, _P],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.nmg_last_error.argtypes = []
_lib.nmg_last_error.restype = C.c_char_p

EXPORTED = sorted(list(_SIGS) + ["nmg_last_error"])


def ptr(a) -> int:
    """Address of a torch tensor, numpy array or integer."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


def nmg_last_error() -> str:
    return _lib.nmg_last_error().decode()


def check(status: int) -> int:
    if status < 0:
        raise NmgError(status, nmg_last_error())
    return status


def nmg_default_opts(opts: nmg_solve_opts) -> int:
    return _lib.nmg_default_opts(C.byref(opts))


def nmg_create_hierarchy(desc: nmg_mesh_desc, out: C.c_void_p) -> int:
    return _lib.nmg_create_hierarchy(C.byref(desc), C.byref(out))


def nmg_set_jacobian(h, level, nrows_blk, nnzb, row_ptr, col_idx, vals, ptr_location) -> int:
    return _lib.nmg_set_jacobian(h, level, nrows_blk, nnzb, ptr(row_ptr), ptr(col_idx), ptr(vals), ptr_location)


def nmg_solve(h, b, x, opts: nmg_solve_opts, info: nmg_solve_info) -> int:
    return _lib.nmg_solve(h, ptr(b), ptr(x), C.byref(opts), C.byref(info) if info is not None else None)


def nmg_matvec(h, level, precision, x, y) -> int:
    return _lib.nmg_matvec(h, level, precision, ptr(x), ptr(y))


def nmg_residual(h, level, precision, b, x, r) -> int:
    return _lib.nmg_residual(h, level, precision, ptr(b), ptr(x), ptr(r))


def nmg_smooth(h, level, precision, b, x, steps, x_is_zero, omega, weighting) -> int:
    return _lib.nmg_smooth(h, level, precision, ptr(b), ptr(x), steps, x_is_zero, omega, weighting)


def nmg_restrict(h, level, precision, r_fine, r_coarse) -> int:
    return _lib.nmg_restrict(h, level, precision, ptr(r_fine), ptr(r_coarse))


def nmg_prolongate_add(h, level, precision, e_coarse, x_fine) -> int:
    return _lib.nmg_prolongate_add(h, level, precision, ptr(e_coarse), ptr(x_fine))


def nmg_coarse_solve(h, precision, b, x) -> int:
    return _lib.nmg_coarse_solve(h, precision, ptr(b), ptr(x))


def nmg_vcycle(h, opts: nmg_solve_opts, r, z) -> int:
    return _lib.nmg_vcycle(h, C.byref(opts), ptr(r), ptr(z))


def nmg_vcycle_many(h, opts: nmg_solve_opts, nrhs, r, z) -> int:
    return _lib.nmg_vcycle_many(h, C.byref(opts), nrhs, ptr(r), ptr(z))


def nmg_solve_many(h, nrhs, b, x, opts: nmg_solve_opts, info=None) -> int:
    """info: None or a ctypes array of nrhs nmg_solve_info records."""
    return _lib.nmg_solve_many(h, nrhs, ptr(b), ptr(x), C.byref(opts), C.cast(info, C.c_void_p) if info is not None else None)


def nmg_get_patch_inverses(h, level, precision, first, count, out) -> int:
    return _lib.nmg_get_patch_inverses(h, level, precision, first, count, ptr(out))


def nmg_hierarchy_bytes(h, out: C.c_size_t) -> int:
    return _lib.nmg_hierarchy_bytes(h, C.byref(out))


def nmg_destroy_hierarchy(h) -> int:
    return _lib.nmg_destroy_hierarchy(h)


def nmg_profile_enable(h, enable) -> int:
    return _lib.nmg_profile_enable(h, enable)


def nmg_profile_read(h, ms: C.c_double, launches: C.c_int64, bytes_per_launch: C.c_double) -> int:
    ref = lambda v: None if v is None else C.byref(v)
    return _lib.nmg_profile_read(h, ref(ms), ref(launches), ref(bytes_per_launch))


def nmg_vanka_correct_noalloc(dim, cells, precision, inv, inv_stride, d, x, omega, weighting, x_is_zero,
                              stream=None) -> int:
    c = (C.c_int * 3)(*(list(cells) + [0] * (3 - len(cells))))
    return _lib.nmg_vanka_correct_noalloc(dim, c, precision, ptr(inv), inv_stride, ptr(d), ptr(x), omega,
                                          weighting, x_is_zero, stream)


def nmg_server_create(mem_budget_bytes, max_slots, out: C.c_void_p) -> int:
    return _lib.nmg_server_create(mem_budget_bytes, max_slots, C.byref(out))


def nmg_submit(server, h, b, x, opts: nmg_solve_opts, ticket: C.c_uint64) -> int:
    return _lib.nmg_submit(server, h, ptr(b), ptr(x), C.byref(opts), C.byref(ticket))


def nmg_poll(server, ticket, timeout_ms, info: nmg_solve_info) -> int:
    return _lib.nmg_poll(server, ticket, timeout_ms, C.byref(info) if info is not None else None)


def nmg_server_destroy(server) -> int:
    return _lib.nmg_server_destroy(server)


def nmg_server_set_workspaces(server, extra_per_hierarchy) -> int:
    return _lib.nmg_server_set_workspaces(server, extra_per_hierarchy)


def nmg_server_set_batching(server, max_columns) -> int:
    return _lib.nmg_server_set_batching(server, max_columns)


def nmg_autotune_report(h, buf, length) -> int:
    return _lib.nmg_autotune_report(h, buf, length)


def nmg_server_memory(server, resident: C.c_size_t, peak: C.c_size_t) -> int:
    ref = lambda v: None if v is None else C.byref(v)
    return _lib.nmg_server_memory(server, ref(resident), ref(peak))


def nmg_set_wait_limit(h, spins) -> int:
    return _lib.nmg_set_wait_limit(h, spins)


def nmg_set_lifting_operator(h, nrows_blk, nnzb, row_ptr, col_idx, vals, ptr_location) -> int:
    return _lib.nmg_set_lifting_operator(h, nrows_blk, nnzb, ptr(row_ptr), ptr(col_idx), ptr(vals), ptr_location)


def nmg_deformation_update(h, r, dv, k_theta, update_nodes, du) -> int:
    return _lib.nmg_deformation_update(h, ptr(r), ptr(dv), k_theta, ptr(update_nodes), ptr(du))


def nmg_extension_rhs(h, b5, g, rhs) -> int:
    return _lib.nmg_extension_rhs(h, ptr(b5), ptr(g), ptr(rhs))


def nmg_newton_substeps(h1, h3, b1, r, k_theta, update_nodes, b5, dw, du, opts1: nmg_solve_opts,
                        opts3: nmg_solve_opts, info1=None, info3=None) -> int:
    ref = lambda v: None if v is None else C.byref(v)
    return _lib.nmg_newton_substeps(h1, h3, ptr(b1), ptr(r), k_theta, ptr(update_nodes), ptr(b5), ptr(dw), ptr(du),
                                    C.byref(opts1), C.byref(opts3), ref(info1), ref(info3))


def nmg_jacobian_reuse_init(m: nmg_jacobian_reuse, gamma) -> int:
    return _lib.nmg_jacobian_reuse_init(C.byref(m) if m is not None else None, gamma)


def nmg_jacobian_reuse_time_step(m: nmg_jacobian_reuse) -> int:
    return _lib.nmg_jacobian_reuse_time_step(C.byref(m) if m is not None else None)


def nmg_jacobian_reuse_decide(m: nmg_jacobian_reuse, residual_inf, assemble: C.c_int) -> int:
    return _lib.nmg_jacobian_reuse_decide(C.byref(m) if m is not None else None, residual_inf,
                                          C.byref(assemble) if assemble is not None else None)


def nmg_set_large_patches(h, cell_mask) -> int:
    return _lib.nmg_set_large_patches(h, ptr(cell_mask))


def nmg_patch_layout(h, level, nsmall, nlarge, np_small, np_large) -> int:
    ref = lambda v: None if v is None else C.byref(v)
    return _lib.nmg_patch_layout(h, level, ref(nsmall), ref(nlarge), ref(np_small), ref(np_large))
