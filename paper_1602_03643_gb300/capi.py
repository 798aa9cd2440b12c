"""ctypes binding of liboasis (include/oasis.h), argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the scheme: all work runs in the CUDA kernels of liboasis.so.
If the library is missing, loading fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboasis.so")

OASIS_OK = 0
OASIS_EINVAL = -1
OASIS_ECUDA = -2
OASIS_EMESH = -3
OASIS_ENOTCONV = -4
OASIS_EBREAKDOWN = -5
OASIS_ENAN = -6
OASIS_ENOMEM = -7
OASIS_EWAIT = -8
OASIS_FP64 = 0
OASIS_MIXED = 1
OASIS_GUESS_ZERO = 0
OASIS_GUESS_PREV_PHI = 1
OASIS_GUESS_LEARNED = 2
OASIS_PC_JACOBI = 0
OASIS_PC_AMG = 1
OASIS_CONV_ABCN = 0
OASIS_CONV_ABE = 1
OASIS_UPDATE_LUMPED = 0
OASIS_UPDATE_CONSISTENT = 1
OASIS_MAX_SCALARS = 8
OASIS_MAT_M, OASIS_MAT_K, OASIS_MAT_G0, OASIS_MAT_G1, OASIS_MAT_G2, OASIS_MAT_A = range(6)

ERROR_NAMES = {0: "OK", -1: "EINVAL", -2: "ECUDA", -3: "EMESH", -4: "ENOTCONV", -5: "EBREAKDOWN",
               -6: "ENAN", -7: "ENOMEM", -8: "EWAIT"}


class oasis_params(C.Structure):
    _fields_ = [("nu", C.c_double), ("dt", C.c_double), ("f", C.c_double * 3),
                ("rtol_u", C.c_double), ("rtol_p", C.c_double),
                ("max_it_u", C.c_int32), ("max_it_p", C.c_int32), ("precision", C.c_int32),
                ("inner_rtol", C.c_double), ("batch_rhs", C.c_int32), ("use_graph", C.c_int32),
                ("guess", C.c_int32), ("spmv_variant", C.c_int32), ("pressure_pc", C.c_int32),
                ("inner_iters", C.c_int32), ("convection", C.c_int32),
                ("velocity_update", C.c_int32), ("bicg_variant", C.c_int32)]


class oasis_amg_info(C.Structure):
    _fields_ = [("levels", C.c_int32), ("rows", C.c_int64 * 16), ("nnz", C.c_int64 * 16),
                ("setup_s", C.c_double), ("p_nnz", C.c_int64 * 16), ("packed", C.c_int32 * 16)]


class oasis_tuning(C.Structure):
    _fields_ = [("n_variants", C.c_int32), ("chosen", C.c_int32), ("chunk", C.c_int32 * 16),
                ("min_blocks", C.c_int32 * 16), ("prefetch", C.c_int32 * 16), ("col16", C.c_int32 * 16),
                ("streamed", C.c_int32 * 16), ("warps_per_block", C.c_int32 * 16), ("us", C.c_double * 16),
                ("bicg_n_variants", C.c_int32), ("bicg_chosen", C.c_int32), ("bicg_lanes", C.c_int32 * 8),
                ("bicg_rows", C.c_int32 * 8), ("bicg_min_blocks", C.c_int32 * 8), ("bicg_us", C.c_double * 8),
                ("bicg_col16", C.c_int32 * 8)]

    def as_dict(self):
        n = self.n_variants
        return {"chosen": self.chosen,
                "candidates": [{"chunk": self.chunk[k], "min_blocks": self.min_blocks[k],
                                "prefetch": self.prefetch[k], "col16": self.col16[k],
                                "streamed": self.streamed[k], "warps_per_block": self.warps_per_block[k],
                                "us": self.us[k]}
                               for k in range(n)],
                "bicg_chosen": self.bicg_chosen,
                "bicg_candidates": [{"lanes": self.bicg_lanes[k], "rows": self.bicg_rows[k],
                                     "min_blocks": self.bicg_min_blocks[k], "col16": self.bicg_col16[k],
                                     "us": self.bicg_us[k]}
                                    for k in range(self.bicg_n_variants)]}


class oasis_step_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("it_u", C.c_int32 * 3), ("sweeps_u", C.c_int32),
                ("it_p", C.c_int32), ("sweeps_p", C.c_int32), ("guess_used", C.c_int32),
                ("res_u", C.c_double * 3), ("res_p", C.c_double), ("t", C.c_double),
                ("guess_res", C.c_double * 2), ("res_m", C.c_double * 3), ("it_m", C.c_int32),
                ("it_c", C.c_int32), ("res_c", C.c_double)]

    def as_dict(self):
        return {"status": self.status, "it_u": list(self.it_u), "sweeps_u": self.sweeps_u,
                "it_p": self.it_p, "sweeps_p": self.sweeps_p, "guess_used": self.guess_used,
                "res_u": list(self.res_u), "res_p": self.res_p, "t": self.t,
                "guess_res": list(self.guess_res), "res_m": list(self.res_m), "it_m": self.it_m,
                "it_c": self.it_c, "res_c": self.res_c}


class OasisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None

P = C.c_void_p
PP = C.POINTER(C.c_void_p)
I32 = C.c_int32
I64 = C.c_int64
DPTR = C.c_void_p

# name -> (restype, argtypes); the exported surface of include/oasis.h
SIGNATURES = {
    "oasis_version": (C.c_int, []),
    "oasis_last_error": (C.c_char_p, []),
    "oasis_mesh_create": (C.c_int, [I32, I64, DPTR, I64, DPTR, DPTR, I64, DPTR, PP]),
    "oasis_mesh_info": (C.c_int, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
    "oasis_assemble_constant": (C.c_int, [P, P]),
    "oasis_mesh_get_pattern": (C.c_int, [P, DPTR, DPTR]),
    "oasis_mesh_get_matrix": (C.c_int, [P, I32, DPTR]),
    "oasis_spmv_f64": (C.c_int, [P, I32, DPTR, DPTR, I32, P]),
    "oasis_spmv_f32": (C.c_int, [P, I32, DPTR, DPTR, I32, P]),
    "oasis_spmv_dot_f64": (C.c_int, [P, I32, DPTR, DPTR, DPTR, P]),
    "oasis_spmv_dot_f64_noalloc": (C.c_int, [P, I32, DPTR, DPTR, DPTR, P]),
    "oasis_solver_create": (C.c_int, [P, C.POINTER(oasis_params), I64, DPTR, P, PP]),
    "oasis_set_fields": (C.c_int, [P, DPTR, DPTR, DPTR, C.c_double, I32, P]),
    "oasis_set_dirichlet": (C.c_int, [P, DPTR, I32, P]),
    "oasis_step": (C.c_int, [P, P, C.POINTER(oasis_step_stats)]),
    "oasis_last_stats": (C.c_int, [P, C.POINTER(oasis_step_stats)]),
    "oasis_get_fields": (C.c_int, [P, DPTR, DPTR, DPTR, I32, P]),
    "oasis_solver_set_scalars": (C.c_int, [P, I32, DPTR, DPTR, I64, DPTR]),
    "oasis_set_scalar_fields": (C.c_int, [P, DPTR, I32, P]),
    "oasis_get_scalar_fields": (C.c_int, [P, DPTR, I32, P]),
    "oasis_set_scalar_dirichlet": (C.c_int, [P, DPTR, I32, P]),
    "oasis_get_tentative_system": (C.c_int, [P, DPTR, DPTR, P]),
    "oasis_profile": (C.c_int, [P, I32]),
    "oasis_profile_read": (C.c_int, [P, I32, C.POINTER(I64), C.POINTER(C.c_double)]),
    "oasis_net_create": (C.c_int, [P, PP]),
    "oasis_net_set_params": (C.c_int, [P, DPTR]),
    "oasis_net_get_params": (C.c_int, [P, DPTR]),
    "oasis_net_forward": (C.c_int, [P, DPTR, DPTR, P]),
    "oasis_net_backward": (C.c_int, [P, DPTR, DPTR, DPTR, DPTR, P]),
    "oasis_net_adam": (C.c_int, [P, DPTR, C.c_float, C.c_float, C.c_float, C.c_float, I32, P]),
    "oasis_net_destroy": (None, [P]),
    "oasis_solver_set_guess_net": (C.c_int, [P, P]),
    "oasis_solver_record_guess": (C.c_int, [P, I32]),
    "oasis_get_guess_sample": (C.c_int, [P, DPTR, DPTR, P]),
    "oasis_get_tuning": (C.c_int, [P, C.POINTER(oasis_tuning)]),
    "oasis_get_amg_info": (C.c_int, [P, C.POINTER(oasis_amg_info)]),
    "oasis_amg_apply": (C.c_int, [P, DPTR, DPTR, P]),
    "oasis_solver_destroy": (None, [P]),
    "oasis_mesh_destroy": (None, [P]),
}


def lib():
    """Load liboasis.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1602_03643_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH, mode=C.RTLD_GLOBAL)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != OASIS_OK:
        raise OasisError(rc, lib().oasis_last_error().decode())
    return rc


def _ptr(a):
    """Host numpy array or torch tensor (host or device) -> address."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()      # torch.Tensor


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream     # torch.cuda.Stream


def oasis_version():
    return lib().oasis_version()


def oasis_mesh_create(dim, coords, cells, dof_of_vertex=None, n_dofs=None, perm=None):
    """perm: optional dof renumbering, perm[d] = the library's internal index of dof d."""
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    dov = None if dof_of_vertex is None else np.ascontiguousarray(dof_of_vertex, dtype=np.int32)
    prm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    if n_dofs is None:
        n_dofs = coords.shape[0] if dov is None else int(dov.max()) + 1
    out = C.c_void_p()
    check(lib().oasis_mesh_create(dim, coords.shape[0], _ptr(coords), cells.shape[0], _ptr(cells),
                                  _ptr(dov), int(n_dofs), _ptr(prm), C.byref(out)))
    return out


def oasis_mesh_info(mesh):
    n, t, z = I64(), I64(), I64()
    check(lib().oasis_mesh_info(mesh, C.byref(n), C.byref(t), C.byref(z)))
    return n.value, t.value, z.value


def oasis_assemble_constant(mesh, stream=None):
    check(lib().oasis_assemble_constant(mesh, _stream(stream)))


def oasis_mesh_get_pattern(mesh):
    n, _, nnz = oasis_mesh_info(mesh)
    rp = np.empty(n + 1, np.int32)
    col = np.empty(nnz, np.int32)
    check(lib().oasis_mesh_get_pattern(mesh, _ptr(rp), _ptr(col)))
    return rp, col


def oasis_mesh_get_matrix(mesh, which):
    n, _, nnz = oasis_mesh_info(mesh)
    out = np.empty(n if which == -1 else nnz, np.float64)
    check(lib().oasis_mesh_get_matrix(mesh, which, _ptr(out)))
    return out


def oasis_spmv_f64(mesh, which, x, y, lanes=0, stream=None):
    check(lib().oasis_spmv_f64(mesh, which, _ptr(x), _ptr(y), lanes, _stream(stream)))


def oasis_spmv_f32(mesh, which, x, y, lanes=0, stream=None):
    check(lib().oasis_spmv_f32(mesh, which, _ptr(x), _ptr(y), lanes, _stream(stream)))


def oasis_spmv_dot_f64(mesh, which, x, y, xy, stream=None):
    check(lib().oasis_spmv_dot_f64(mesh, which, _ptr(x), _ptr(y), _ptr(xy), _stream(stream)))


def oasis_spmv_dot_f64_noalloc(mesh, which, x, y, xy, stream=None):
    check(lib().oasis_spmv_dot_f64_noalloc(mesh, which, _ptr(x), _ptr(y), _ptr(xy), _stream(stream)))


def make_params(nu, dt, f=(0.0, 0.0, 0.0), rtol_u=1e-8, rtol_p=1e-8, max_it_u=1000, max_it_p=20000,
                precision=OASIS_FP64, inner_rtol=1e-4, batch_rhs=1, use_graph=0, guess=OASIS_GUESS_ZERO,
                spmv_variant=0, pressure_pc=0, inner_iters=1,
                convection=0, velocity_update=0, bicg_variant=0):
    p = oasis_params()
    p.nu, p.dt = nu, dt
    ff = list(f) + [0.0] * (3 - len(f))
    for k in range(3):
        p.f[k] = ff[k]
    p.rtol_u, p.rtol_p = rtol_u, rtol_p
    p.max_it_u, p.max_it_p = max_it_u, max_it_p
    p.precision, p.inner_rtol = precision, inner_rtol
    p.batch_rhs, p.use_graph, p.guess, p.spmv_variant = batch_rhs, use_graph, guess, spmv_variant
    p.pressure_pc = pressure_pc
    p.inner_iters = inner_iters
    p.convection = convection
    p.velocity_update = velocity_update
    p.bicg_variant = bicg_variant
    return p


def oasis_solver_create(mesh, params, dirichlet_dofs, stream=None):
    d = np.ascontiguousarray(dirichlet_dofs, dtype=np.int32)
    out = C.c_void_p()
    check(lib().oasis_solver_create(mesh, C.byref(params), d.size, _ptr(d) if d.size else None,
                                    _stream(stream), C.byref(out)))
    return out


def oasis_set_fields(solver, u_nm1, u_nm2, p, t, on_device=False, stream=None):
    if not on_device:
        u_nm1 = np.ascontiguousarray(u_nm1, dtype=np.float64)
        u_nm2 = np.ascontiguousarray(u_nm2, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
    check(lib().oasis_set_fields(solver, _ptr(u_nm1), _ptr(u_nm2), _ptr(p), float(t), int(on_device),
                                 _stream(stream)))


def oasis_set_dirichlet(solver, g, on_device=False, stream=None):
    if not on_device:
        g = np.ascontiguousarray(g, dtype=np.float64)
    check(lib().oasis_set_dirichlet(solver, _ptr(g), int(on_device), _stream(stream)))


def oasis_step(solver, stream=None, want_stats=True):
    if want_stats:
        st = oasis_step_stats()
        check(lib().oasis_step(solver, _stream(stream), C.byref(st)))
        return st
    check(lib().oasis_step(solver, _stream(stream), None))
    return None


def oasis_last_stats(solver):
    st = oasis_step_stats()
    check(lib().oasis_last_stats(solver, C.byref(st)))
    return st


def oasis_get_fields(solver, dim, n, on_device=False, u=None, p=None, phi=None, stream=None):
    if not on_device:
        u = np.empty((dim, n)) if u is None else u
        p = np.empty(n) if p is None else p
        phi = np.empty(n) if phi is None else phi
    check(lib().oasis_get_fields(solver, _ptr(u), _ptr(p), _ptr(phi), int(on_device), _stream(stream)))
    return u, p, phi


def oasis_solver_set_scalars(solver, diffusivity, source, dirichlet_dofs):
    dif = np.ascontiguousarray(diffusivity, dtype=np.float64).reshape(-1)
    src = np.ascontiguousarray(source, dtype=np.float64).reshape(-1)
    d = np.ascontiguousarray(dirichlet_dofs, dtype=np.int32).reshape(-1)
    check(lib().oasis_solver_set_scalars(solver, int(dif.size), _ptr(dif) if dif.size else None,
                                         _ptr(src) if src.size else None, int(d.size),
                                         _ptr(d) if d.size else None))


def oasis_set_scalar_fields(solver, c, on_device=False, stream=None):
    if not on_device:
        c = np.ascontiguousarray(c, dtype=np.float64)
    check(lib().oasis_set_scalar_fields(solver, _ptr(c), int(on_device), _stream(stream)))


def oasis_get_scalar_fields(solver, ns, n, on_device=False, c=None, stream=None):
    if not on_device:
        c = np.empty((ns, n)) if c is None else c
    check(lib().oasis_get_scalar_fields(solver, _ptr(c), int(on_device), _stream(stream)))
    return c


def oasis_set_scalar_dirichlet(solver, g, on_device=False, stream=None):
    if not on_device:
        g = np.ascontiguousarray(g, dtype=np.float64)
    check(lib().oasis_set_scalar_dirichlet(solver, _ptr(g), int(on_device), _stream(stream)))


def oasis_get_tentative_system(solver, dim, n, nnz, stream=None):
    A = np.empty(nnz)
    r0 = np.empty((dim, n))
    check(lib().oasis_get_tentative_system(solver, _ptr(A), _ptr(r0), _stream(stream)))
    return A, r0


PROF_FAMILIES = {"pcg_spmv": 0, "bicg_spmm": 1, "assemble": 2, "pcg_update": 3, "update": 4,
                 "pressure_rhs": 5, "guess": 6, "amg": 7, "mass": 8, "amg_fine": 9, "amg_transfer": 10,
                 "amg_coarse": 11, "bicg_vec": 12, "outer": 13}


def oasis_profile(solver, enable=True):
    check(lib().oasis_profile(solver, int(enable)))


def oasis_profile_read(solver, family):
    n, ms = I64(), C.c_double()
    check(lib().oasis_profile_read(solver, PROF_FAMILIES.get(family, family), C.byref(n), C.byref(ms)))
    return n.value, ms.value


OASIS_NET_PARAMS = 2339


def oasis_net_create(mesh):
    out = C.c_void_p()
    check(lib().oasis_net_create(mesh, C.byref(out)))
    return out


def oasis_net_set_params(net, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == OASIS_NET_PARAMS
    check(lib().oasis_net_set_params(net, _ptr(p)))


def oasis_net_get_params(net):
    p = np.empty(OASIS_NET_PARAMS, np.float32)
    check(lib().oasis_net_get_params(net, _ptr(p)))
    return p


def oasis_net_forward(net, features, y, stream=None):
    check(lib().oasis_net_forward(net, _ptr(features), _ptr(y), _stream(stream)))


def oasis_net_backward(net, features, target, grad=None, loss=None, stream=None):
    check(lib().oasis_net_backward(net, _ptr(features), _ptr(target), _ptr(grad), _ptr(loss), _stream(stream)))


def oasis_net_adam(net, grad=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, step=1, stream=None):
    check(lib().oasis_net_adam(net, _ptr(grad), lr, beta1, beta2, eps, int(step), _stream(stream)))


def oasis_net_destroy(net):
    lib().oasis_net_destroy(net)


def oasis_solver_set_guess_net(solver, net):
    check(lib().oasis_solver_set_guess_net(solver, net))


def oasis_solver_record_guess(solver, on=True):
    check(lib().oasis_solver_record_guess(solver, int(on)))


def oasis_get_guess_sample(solver, features, target, stream=None):
    check(lib().oasis_get_guess_sample(solver, _ptr(features), _ptr(target), _stream(stream)))


def oasis_get_tuning(solver):
    t = oasis_tuning()
    check(lib().oasis_get_tuning(solver, C.byref(t)))
    return t.as_dict()


def oasis_get_amg_info(solver):
    t = oasis_amg_info()
    check(lib().oasis_get_amg_info(solver, C.byref(t)))
    return {"levels": t.levels, "rows": list(t.rows[:t.levels]), "nnz": list(t.nnz[:t.levels]),
            "setup_s": t.setup_s, "p_nnz": list(t.p_nnz[:max(0, t.levels - 1)]),
            "packed": list(t.packed[:max(0, t.levels - 1)])}


def oasis_amg_apply(solver, r, u, stream=None):
    check(lib().oasis_amg_apply(solver, _ptr(r), _ptr(u), _stream(stream)))


def oasis_solver_destroy(solver):
    lib().oasis_solver_destroy(solver)


def oasis_mesh_destroy(mesh):
    lib().oasis_mesh_destroy(mesh)
