"""Python binding of libfem (include/fem.h): argument marshalling only.

Every function keeps the C-ABI name and forwards to the compiled library; tensors are CUDA tensors whose
data pointers are passed as device pointers, and the current torch stream is passed as the CUDA stream.
There is no fallback: if libfem.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfem.so")

FEM_OK = 0
FEM_ERR_ARG, FEM_ERR_OOM, FEM_ERR_CUDA = -1, -2, -3
FEM_ERR_NOT_CONVERGED, FEM_ERR_BREAKDOWN, FEM_ERR_NONFINITE, FEM_ERR_TIMEOUT, FEM_ERR_STATE = -4, -5, -6, -7, -8
FEM_FP64, FEM_FP32_INNER = 0, 1
FEM_PRED_AB4, FEM_PRED_DD = 0, 1
FEM_INNER_FP32, FEM_INNER_TC = 0, 1
FEM_FIELD_U, FEM_FIELD_V, FEM_FIELD_A, FEM_FIELD_DU, FEM_FIELD_B, FEM_FIELD_GUESS = range(6)

# every symbol include/fem.h declares
EXPORTS = ("fem_opts_default", "fem_mesh_create", "fem_mesh_create_tet10", "fem_mesh_destroy", "fem_mesh_tune", "fem_mesh_autotune",
           "fem_mesh_info", "fem_mesh_split_product",
           "fem_mesh_set_regions", "fem_ebe_apply",
           "fem_ebe_apply_noalloc", "fem_mesh10_create", "fem_mesh10_destroy", "fem_ebe10_apply", "pcg10_solve",
           "pcg_solve", "fem_batch_create", "fem_batch_destroy", "fem_case_add", "fem_step", "predictor_fit",
           "predictor_predict", "predictor_coefficients", "fem_case_get", "fem_batch_set_loads", "fem_batch_get_field", "fem_batch_get_field_async",
           "fem_batch_sync", "fem_step_async", "fem_batch_profile",
           "fem_case_stats", "fem_batch_steps", "fem_mlp_create", "fem_mlp_destroy", "fem_mlp_get_params",
           "fem_mlp_forward", "fem_mlp_loss_grad", "fem_mlp_train", "fem_batch_set_mlp", "fem_batch_collect",
           "fem_batch_collected", "fem_batch_proposal_counts", "fem_last_error", "fem_mlp_loss_grad_residual",
           "fem_mlp_train_residual", "fem_batch_collect_residual", "fem_mesh_set_absorbing", "fem_case_add_impulses",
           "fem_batch_predictor_balance")
FEM_MLP_N_PARAMS, FEM_MLP_IN, FEM_MLP_OUT, FEM_MLP_RES = 90656, 64, 32, 560


class FemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libfem status {status}: {msg}")
        self.status = status


class fem_time_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("a0", ctypes.c_double), ("a1", ctypes.c_double)]


class fem_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("predictor", ctypes.c_int), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("s_max", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("tau", ctypes.c_double), ("snapshot_format", ctypes.c_int), ("check_every", ctypes.c_int),
                ("refresh_every", ctypes.c_int), ("cert_df", ctypes.c_int), ("fuse_meshes", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("wait_budget", ctypes.c_int),
                ("cpu_predictor", ctypes.c_int), ("inner_margin", ctypes.c_double),
                ("inner_product", ctypes.c_int), ("pred_guard", ctypes.c_int)]


class fem_profile(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("kernel_launches", ctypes.c_longlong),
                ("ebe32_launches", ctypes.c_longlong), ("ebe32_ms", ctypes.c_double),
                ("ebe64_launches", ctypes.c_longlong), ("ebe64_ms", ctypes.c_double),
                ("cg_vec_launches", ctypes.c_longlong), ("cg_vec_ms", ctypes.c_double),
                ("predict_ms", ctypes.c_double), ("rhs_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("update_ms", ctypes.c_double), ("ebe16_launches", ctypes.c_longlong), ("ebe16_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fem_case_stats_t(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("iters", ctypes.c_int), ("outer", ctypes.c_int), ("status", ctypes.c_int),
                ("init_relres", ctypes.c_double), ("relres", ctypes.c_double), ("guess", ctypes.c_int),
                ("fallbacks", ctypes.c_int)]


_lib = None


def lib():
    """Loads libfem.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2409_20380_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "fem_opts_default": (None, [ctypes.POINTER(fem_opts)]),
        "fem_mesh_create": (I, [I64, P, I64, P, P, I, P, P, ctypes.POINTER(fem_time_params), P, ctypes.POINTER(P)]),
        "fem_mesh_create_tet10": (I, [I64, P, I64, P, P, I, P, P, ctypes.POINTER(fem_time_params), P,
                                      ctypes.POINTER(P)]),
        "fem_mesh_destroy": (I, [P]),
        "fem_mesh_tune": (I, [P, I, I]),
        "fem_mesh_split_product": (I, [P, I, P, P, P, I, P]),
        "fem_mesh_autotune": (I, [P, I, I, P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
        "fem_mesh_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "fem_mesh_set_regions": (I, [P, P]),
        "fem_ebe_apply": (I, [P, I, P, P, I, D, D, P, P]),
        "fem_ebe_apply_noalloc": (I, [P, I, P, P, I, D, D, P, P]),
        "fem_mesh10_create": (I, [I64, P, I64, P, P, I, P, P, P, ctypes.POINTER(P)]),
        "fem_mesh10_destroy": (I, [P]),
        "fem_ebe10_apply": (I, [P, I, P, P, I, D, D, P, P]),
        "pcg10_solve": (I, [P, I, P, P, I, D, D, D, I, P, P, P]),
        "pcg_solve": (I, [P, P, P, I, ctypes.POINTER(fem_opts), P, P, P]),
        "fem_batch_create": (I, [ctypes.POINTER(fem_opts), P, ctypes.POINTER(P)]),
        "fem_batch_destroy": (I, [P]),
        "fem_case_add": (I, [P, P, ctypes.c_int32, P, D, D, D, ctypes.POINTER(I)]),
        "fem_step": (I, [P, I, P, P]),
        "predictor_fit": (I, [P, I]),
        "predictor_predict": (I, [P, I, P]),
        "predictor_coefficients": (I, [P, I, P, ctypes.POINTER(I)]),
        "fem_case_get": (I, [P, I, I, P, I]),
        "fem_batch_set_loads": (I, [P, P]),
        "fem_batch_get_field": (I, [P, I, P, I]),
        "fem_batch_get_field_async": (I, [P, I, P]),
        "fem_batch_sync": (I, [P]),
        "fem_step_async": (I, [P, I]),
        "fem_batch_profile": (I, [P, I, ctypes.POINTER(fem_profile)]),
        "fem_case_stats": (I, [P, I, ctypes.POINTER(fem_case_stats_t)]),
        "fem_batch_steps": (I, [P, ctypes.POINTER(I)]),
        "fem_mlp_create": (I, [P, P, ctypes.POINTER(P)]),
        "fem_mlp_destroy": (I, [P]),
        "fem_mlp_get_params": (I, [P, P]),
        "fem_mlp_forward": (I, [P, P, I64, P]),
        "fem_mlp_loss_grad": (I, [P, P, P, I64, P, ctypes.POINTER(D)]),
        "fem_mlp_train": (I, [P, P, P, I64, P, I, I, D, P]),
        "fem_batch_set_mlp": (I, [P, P]),
        "fem_batch_collect": (I, [P, P, P, I64]),
        "fem_batch_collect_residual": (I, [P, P, P, I64]),
        "fem_mesh_set_absorbing": (I, [P, I64, P, P]),
        "fem_batch_predictor_balance": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D),
                                            ctypes.POINTER(D), ctypes.POINTER(D)]),
        "fem_case_add_impulses": (I, [P, P, I64, P, P, P, ctypes.POINTER(I)]),
        "fem_mlp_loss_grad_residual": (I, [P, P, P, I64, P, ctypes.POINTER(D)]),
        "fem_mlp_train_residual": (I, [P, P, P, I64, P, I, I, D, P]),
        "fem_batch_collected": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I)]),
        "fem_batch_proposal_counts": (I, [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "fem_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st):
    if st != FEM_OK:
        raise FemError(st, lib().fem_last_error().decode())
    return st


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype=None):
    if t is None:
        return None
    import torch
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    if dtype is not None:
        assert t.dtype == dtype, f"expected {dtype}, got {t.dtype}"
    return ctypes.c_void_p(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def fem_opts_default(**overrides) -> fem_opts:
    o = fem_opts()
    lib().fem_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _mesh_create(fn, mesh, tp, stream):
    xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    mat = np.ascontiguousarray(mesh.mat_id, dtype=np.int32)
    lmr = np.ascontiguousarray(mesh.lam_mu_rho, dtype=np.float64)
    fixed = np.ascontiguousarray(mesh.fixed_dof, dtype=np.uint8)
    t = fem_time_params(tp.dt, tp.beta, tp.gamma, tp.a0, tp.a1)
    h = ctypes.c_void_p()
    _check(fn(xyz.shape[0], _np_ptr(xyz), conn.shape[0], _np_ptr(conn), _np_ptr(mat), lmr.shape[0], _np_ptr(lmr),
              _np_ptr(fixed), ctypes.byref(t), _stream(stream), ctypes.byref(h)))
    return h


def fem_mesh_create(mesh, tp, stream=None):
    """mesh: workload.Mesh (host arrays); tp: workload.TimeParams.  Returns an opaque handle."""
    assert mesh.conn.shape[1] == 4, "linear tets: conn [E][4] (fem_mesh_create_tet10 takes quadratic tets)"
    return _mesh_create(lib().fem_mesh_create, mesh, tp, stream)


def fem_mesh_create_tet10(mesh10, tp, stream=None):
    """mesh10: workload.Mesh10 (conn [E][10]); the same handle type as fem_mesh_create's."""
    assert mesh10.conn.shape[1] == 10, "quadratic tets: conn [E][10]"
    return _mesh_create(lib().fem_mesh_create_tet10, mesh10, tp, stream)


def fem_mesh_destroy(h):
    _check(lib().fem_mesh_destroy(h))


def fem_mesh_tune(h, ebe_variant=0, hex_per_tile=0):
    _check(lib().fem_mesh_tune(h, ebe_variant, hex_per_tile))


def fem_mesh_autotune(h, precision, n_rhs, stream=None):
    """Returns (ebe_variant, hex_per_tile, ms per product) of the fastest EBE implementation, now in use."""
    v, t, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().fem_mesh_autotune(h, precision, n_rhs, _stream(stream), ctypes.byref(v), ctypes.byref(t),
                                   ctypes.byref(ms)))
    return v.value, t.value, ms.value


def fem_mesh_split_product(h, mode, p, qM, qK, n_rhs, stream=None):
    """qM = M p, qK = K p (FP64 CUDA tensors, [node][3][n_rhs]); mode 0..3 as in include/fem.h."""
    import torch
    _check(lib().fem_mesh_split_product(h, mode, _ptr(p, torch.float64), _ptr(qM, torch.float64),
                                        _ptr(qK, torch.float64), n_rhs, _stream(stream)))


def fem_mesh_info(h):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().fem_mesh_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"has_hex_patches": a.value, "ebe_variant": b.value, "hex_per_tile": c.value}


def fem_mesh_set_regions(h, region_of_node):
    reg = np.ascontiguousarray(region_of_node, dtype=np.int32)
    _check(lib().fem_mesh_set_regions(h, _np_ptr(reg)))


def fem_ebe_apply(h, p, q, n_rhs, alpha_M, alpha_K, ptq=None, precision=None, stream=None):
    import torch
    if precision is None:
        precision = FEM_FP64 if p.dtype == torch.float64 else FEM_FP32_INNER
    dt = torch.float64 if precision == FEM_FP64 else torch.float32
    _check(lib().fem_ebe_apply(h, precision, _ptr(p, dt), _ptr(q, dt), n_rhs, float(alpha_M), float(alpha_K),
                               _ptr(ptq, torch.float64), _stream(stream)))


def fem_ebe_apply_noalloc(h, p, q, n_rhs, alpha_M, alpha_K, ptq=None, precision=None, stream=None):
    """Like fem_ebe_apply, but the library allocates no device memory (fixed internal scratch)."""
    import torch
    if precision is None:
        precision = FEM_FP64 if p.dtype == torch.float64 else FEM_FP32_INNER
    dt = torch.float64 if precision == FEM_FP64 else torch.float32
    _check(lib().fem_ebe_apply_noalloc(h, precision, _ptr(p, dt), _ptr(q, dt), n_rhs, float(alpha_M),
                                       float(alpha_K), _ptr(ptq, torch.float64), _stream(stream)))


def fem_mesh10_create(mesh10, stream=None):
    """mesh10: workload.Mesh10 (host arrays, corners then edge midpoints).  Returns an opaque handle."""
    xyz = np.ascontiguousarray(mesh10.xyz, dtype=np.float64)
    conn = np.ascontiguousarray(mesh10.conn, dtype=np.int32)
    mat = np.ascontiguousarray(mesh10.mat_id, dtype=np.int32)
    lmr = np.ascontiguousarray(mesh10.lam_mu_rho, dtype=np.float64)
    fixed = np.ascontiguousarray(mesh10.fixed_dof, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(lib().fem_mesh10_create(xyz.shape[0], _np_ptr(xyz), conn.shape[0], _np_ptr(conn), _np_ptr(mat),
                                   lmr.shape[0], _np_ptr(lmr), _np_ptr(fixed), _stream(stream), ctypes.byref(h)))
    return h


def fem_mesh10_destroy(h):
    _check(lib().fem_mesh10_destroy(h))


def fem_ebe10_apply(h, p, q, n_rhs, alpha_M, alpha_K, ptq=None, precision=None, stream=None):
    import torch
    if precision is None:
        precision = FEM_FP64 if p.dtype == torch.float64 else FEM_FP32_INNER
    dt = torch.float64 if precision == FEM_FP64 else torch.float32
    _check(lib().fem_ebe10_apply(h, precision, _ptr(p, dt), _ptr(q, dt), n_rhs, float(alpha_M), float(alpha_K),
                                 _ptr(ptq, torch.float64), _stream(stream)))


def pcg10_solve(h, b, x, n_rhs, alpha_M, alpha_K, tol=1e-8, maxit=5000, precision=None, stream=None):
    """PCG on the tet10 system (FEM_FP64 plain, FEM_FP32_INNER refined); returns (iters, relres) [n_rhs]."""
    import torch
    precision = FEM_FP64 if precision is None else precision
    iters = np.zeros(n_rhs, dtype=np.int32)
    relres = np.zeros(n_rhs, dtype=np.float64)
    _check(lib().pcg10_solve(h, precision, _ptr(b, torch.float64), _ptr(x, torch.float64), n_rhs, float(alpha_M),
                             float(alpha_K), float(tol), int(maxit), _stream(stream), _np_ptr(iters),
                             _np_ptr(relres)))
    return iters, relres


def pcg_solve(h, b, x, n_rhs, opts, stream=None, raise_on_error=True):
    """Returns (status, iters [n_rhs], relres [n_rhs])."""
    import torch
    iters = np.zeros(n_rhs, dtype=np.int32)
    relres = np.zeros(n_rhs, dtype=np.float64)
    st = lib().pcg_solve(h, _ptr(b, torch.float64), _ptr(x, torch.float64), n_rhs, ctypes.byref(opts),
                         _stream(stream), _np_ptr(iters), _np_ptr(relres))
    if raise_on_error and st not in (FEM_OK,):
        _check(st)
    return st, iters, relres


def fem_batch_create(opts, stream=None):
    h = ctypes.c_void_p()
    _check(lib().fem_batch_create(ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
    return h


def fem_batch_destroy(h):
    _check(lib().fem_batch_destroy(h))


def fem_case_add(batch, mesh_h, src):
    """src: workload.Source.  Returns the case id."""
    d = np.ascontiguousarray(src.direction, dtype=np.float64)
    cid = ctypes.c_int()
    _check(lib().fem_case_add(batch, mesh_h, int(src.node), _np_ptr(d), float(src.f0), float(src.t0),
                              float(src.amp), ctypes.byref(cid)))
    return cid.value


def fem_step(batch, n_steps, n_cases, raise_on_error=True):
    """Returns (status, iters [n_cases] summed over the steps, max relres [n_cases])."""
    iters = np.zeros(n_cases, dtype=np.int32)
    relres = np.zeros(n_cases, dtype=np.float64)
    st = lib().fem_step(batch, n_steps, _np_ptr(iters), _np_ptr(relres))
    if raise_on_error:
        _check(st)
    return st, iters, relres


def predictor_fit(batch, case_id):
    _check(lib().predictor_fit(batch, case_id))


def predictor_predict(batch, case_id, x_guess):
    import torch
    _check(lib().predictor_predict(batch, case_id, _ptr(x_guess, torch.float64)))


def predictor_coefficients(batch, case_id, n_regions, s_max):
    """Returns (coefficients [n_regions][s_max], pairs used) of the last step's data-driven correction."""
    coef = np.zeros((n_regions, s_max), dtype=np.float64)
    n = ctypes.c_int(0)
    _check(lib().predictor_coefficients(batch, case_id, _np_ptr(coef), ctypes.byref(n)))
    return coef, n.value


def fem_mesh_set_absorbing(h, faces, stream=None):
    """faces: [n][3] node triples of the absorbing boundary faces (None or empty: remove the dashpots)."""
    f = np.ascontiguousarray(faces if faces is not None else np.zeros((0, 3)), dtype=np.int32).reshape(-1, 3)
    _check(lib().fem_mesh_set_absorbing(h, f.shape[0], _np_ptr(f) if f.size else None, _stream(stream)))


def fem_case_add_impulses(batch, h, imp):
    """imp: workload.Impulses (nodes, steps, forces).  Returns the case id."""
    nodes = np.ascontiguousarray(imp.nodes, dtype=np.int32)
    steps = np.ascontiguousarray(imp.steps, dtype=np.int32)
    forces = np.ascontiguousarray(imp.forces, dtype=np.float64).reshape(-1, 3)
    cid = ctypes.c_int(-1)
    _check(lib().fem_case_add_impulses(batch, h, nodes.size, _np_ptr(nodes), _np_ptr(steps), _np_ptr(forces),
                                       ctypes.byref(cid)))
    return cid.value


def fem_batch_predictor_balance(batch, case_id):
    """Heterogeneous scheme: dict(s, predict_ms, solve_ms, predict_total_ms, wait_total_ms) of a case's set."""
    sc = ctypes.c_int()
    v = [ctypes.c_double() for _ in range(4)]
    _check(lib().fem_batch_predictor_balance(batch, case_id, ctypes.byref(sc), *[ctypes.byref(x) for x in v]))
    return dict(s=sc.value, predict_ms=v[0].value, solve_ms=v[1].value, predict_total_ms=v[2].value,
                wait_total_ms=v[3].value)


def fem_case_get(batch, case_id, what, n_nodes, out=None):
    """Returns field `what` of a case as a host numpy array [n_nodes*3] (or fills the CUDA tensor `out`)."""
    import torch
    if out is not None:
        _check(lib().fem_case_get(batch, case_id, what, _ptr(out, torch.float64), 1))
        return out
    a = np.zeros(3 * n_nodes, dtype=np.float64)
    _check(lib().fem_case_get(batch, case_id, what, _np_ptr(a), 0))
    return a


def fem_batch_set_loads(batch, loads):
    """loads: host array [n_cases][3] (numpy; pinned torch CPU tensors are passed by pointer too)."""
    if hasattr(loads, "data_ptr"):
        ptr = ctypes.c_void_p(loads.data_ptr())
    else:
        loads = np.ascontiguousarray(loads, dtype=np.float64)
        ptr = _np_ptr(loads)
    _check(lib().fem_batch_set_loads(batch, ptr))


def fem_batch_get_field(batch, what, out):
    """out: host numpy array or CUDA/CPU torch tensor [n_cases*n_nodes*3] (float64), filled in place."""
    if hasattr(out, "data_ptr"):
        _check(lib().fem_batch_get_field(batch, what, ctypes.c_void_p(out.data_ptr()), 1 if out.is_cuda else 0))
    else:
        assert out.dtype == np.float64 and out.flags.c_contiguous
        _check(lib().fem_batch_get_field(batch, what, _np_ptr(out), 0))
    return out


def fem_batch_get_field_async(batch, what, out):
    """out: page-locked host torch tensor [n_cases*n_nodes*3] (float64); filled after fem_batch_sync (the copy
    overlaps the steps queued next)."""
    assert not out.is_cuda and out.dtype.itemsize == 8 and out.is_contiguous()
    _check(lib().fem_batch_get_field_async(batch, what, ctypes.c_void_p(out.data_ptr())))
    return out


def fem_batch_sync(batch, raise_on_error=True):
    """Waits for the batch (steps and field copies); returns the worst status of fem_step_async's steps."""
    st = lib().fem_batch_sync(batch)
    if raise_on_error:
        _check(st)
    return st


def fem_step_async(batch, n_steps):
    """Queues n_steps without waiting; fem_batch_sync reports their status."""
    _check(lib().fem_step_async(batch, n_steps))


def fem_batch_profile(batch, enable=-1):
    p = fem_profile()
    _check(lib().fem_batch_profile(batch, enable, ctypes.byref(p)))
    return p.as_dict()


def fem_case_stats(batch, case_id):
    st = fem_case_stats_t()
    _check(lib().fem_case_stats(batch, case_id, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in st._fields_}


def fem_batch_steps(batch):
    s = ctypes.c_int()
    _check(lib().fem_batch_steps(batch, ctypes.byref(s)))
    return s.value


def fem_mlp_create(params, stream=None):
    """params: FP32 array [90656] (host, copied)."""
    import numpy as np
    a = np.ascontiguousarray(params, dtype=np.float32)
    assert a.shape == (FEM_MLP_N_PARAMS,)
    h = ctypes.c_void_p()
    _check(lib().fem_mlp_create(_np_ptr(a), _stream(stream), ctypes.byref(h)))
    return h


def fem_mlp_destroy(h):
    _check(lib().fem_mlp_destroy(h))


def fem_mlp_get_params(h):
    import numpy as np
    out = np.empty(FEM_MLP_N_PARAMS, dtype=np.float32)
    _check(lib().fem_mlp_get_params(h, _np_ptr(out)))
    return out


def fem_mlp_forward(h, x, out):
    import torch
    assert x.shape[-1] == FEM_MLP_IN and out.shape[-1] == FEM_MLP_OUT and x.shape[0] == out.shape[0]
    _check(lib().fem_mlp_forward(h, _ptr(x, torch.float32), x.shape[0], _ptr(out, torch.float32)))


def fem_mlp_loss_grad(h, x, t, grad=None):
    import torch
    loss = ctypes.c_double()
    _check(lib().fem_mlp_loss_grad(h, _ptr(x, torch.float32), _ptr(t, torch.float32), x.shape[0],
                                   _ptr(grad, torch.float32), ctypes.byref(loss)))
    return loss.value


def fem_mlp_train(h, x, t, order, lr=1e-3, with_loss=True):
    """order: int32 CUDA tensor [n_updates][batch] of sample rows.  Returns the losses (numpy) or None."""
    import numpy as np
    import torch
    n_up, batch = order.shape
    losses = np.zeros(n_up) if with_loss else None
    _check(lib().fem_mlp_train(h, _ptr(x, torch.float32), _ptr(t, torch.float32), x.shape[0],
                               _ptr(order, torch.int32), n_up, batch, lr,
                               _np_ptr(losses) if with_loss else None))
    return losses


def fem_mlp_loss_grad_residual(h, x, s, grad=None):
    """Residual-space loss (s: CUDA tensor [B][FEM_MLP_RES]) and, optionally, its gradient into grad."""
    import torch
    loss = ctypes.c_double()
    _check(lib().fem_mlp_loss_grad_residual(h, _ptr(x, torch.float32), _ptr(s, torch.float32), x.shape[0],
                                            _ptr(grad, torch.float32), ctypes.byref(loss)))
    return loss.value


def fem_mlp_train_residual(h, x, s, order, lr=1e-3, with_loss=True):
    """Adam on the residual-space loss; order: int32 CUDA tensor [n_updates][batch].  Returns the losses."""
    import numpy as np
    import torch
    n_up, batch = order.shape
    losses = np.zeros(n_up) if with_loss else None
    _check(lib().fem_mlp_train_residual(h, _ptr(x, torch.float32), _ptr(s, torch.float32), x.shape[0],
                                        _ptr(order, torch.int32), n_up, batch, lr,
                                        _np_ptr(losses) if with_loss else None))
    return losses


def fem_batch_collect_residual(batch, x, s):
    """Collect residual-space samples into CUDA tensors x [cap][64], s [cap][FEM_MLP_RES] (x = None stops)."""
    import torch
    if x is None:
        _check(lib().fem_batch_collect_residual(batch, None, None, 0))
        return
    assert x.shape[1] == FEM_MLP_IN and s.shape[1] == FEM_MLP_RES and x.shape[0] == s.shape[0]
    _check(lib().fem_batch_collect_residual(batch, _ptr(x, torch.float32), _ptr(s, torch.float32), x.shape[0]))


def fem_batch_set_mlp(batch, net):
    _check(lib().fem_batch_set_mlp(batch, net))


def fem_batch_collect(batch, x, t):
    """Collect training samples into CUDA tensors x [cap][64], t [cap][32] (x = None stops)."""
    import torch
    if x is None:
        _check(lib().fem_batch_collect(batch, None, None, 0))
        return
    assert x.shape[1] == FEM_MLP_IN and t.shape[1] == FEM_MLP_OUT and x.shape[0] == t.shape[0]
    _check(lib().fem_batch_collect(batch, _ptr(x, torch.float32), _ptr(t, torch.float32), x.shape[0]))


def fem_batch_collected(batch):
    rows, full = ctypes.c_int64(), ctypes.c_int()
    _check(lib().fem_batch_collected(batch, ctypes.byref(rows), ctypes.byref(full)))
    return rows.value, bool(full.value)


def fem_batch_proposal_counts(batch):
    t, r = ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib().fem_batch_proposal_counts(batch, ctypes.byref(t), ctypes.byref(r)))
    return t.value, r.value


def fem_last_error():
    return lib().fem_last_error().decode()
