"""ctypes binding of include/hf.h.  Argument marshalling only: every step of
the Newton iteration runs in the CUDA library.  Importing fails loudly if the
shared library cannot be built or loaded; there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HF_OK = 0
HF_PREC_FP64 = 0
HF_PREC_MIXED = 1
HF_SCHEME_COUPLED = 0
HF_SCHEME_STAGGERED = 1
STATUS = {0: "HF_OK", -1: "HF_ERR_INVALID_ARG", -2: "HF_ERR_OOM", -3: "HF_ERR_CUDA",
          -4: "HF_ERR_NOT_CONVERGED", -5: "HF_ERR_NONFINITE", -6: "HF_ERR_TIMEOUT",
          -7: "HF_ERR_DEVICE_ASSERT", -8: "HF_ERR_STATE"}

_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_i8p = C.POINTER(C.c_int8)


class hf_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("order", C.c_int), ("n_nodes", C.c_int64), ("xyz", _dp),
                ("n_elems", C.c_int64), ("elem_nodes", _i32p), ("n_faces", C.c_int64),
                ("face_elems", _i32p), ("face_local", _i8p), ("face_crackable", _i8p),
                ("n_dirichlet", C.c_int64), ("dir_dof", _i64p), ("dir_val", _dp),
                ("n_neumann", C.c_int64), ("neu_face", _i32p), ("neu_traction", _dp)]


class hf_solver_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("restart", C.c_int), ("max_iters", C.c_int),
                ("rtol", C.c_double), ("inner_rtol", C.c_double), ("jacobi_block", C.c_int),
                ("fluid_scaling", C.c_int), ("newton_tol", C.c_double), ("use_graphs", C.c_int),
                ("coarse", C.c_int), ("coarse_max", C.c_int), ("reorth", C.c_int), ("scheme", C.c_int)]


class hf_newton_report(C.Structure):
    _fields_ = [("du_rel", C.c_double), ("dp_rel", C.c_double), ("res_norm", C.c_double),
                ("lin_res", C.c_double), ("gmres_iters", C.c_int), ("refinements", C.c_int),
                ("converged", C.c_int), ("lin_converged", C.c_int), ("fp64_fallback", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hf_step_opts(C.Structure):
    _fields_ = [("newton_max", C.c_int), ("criterion_rounds", C.c_int), ("max_cutbacks", C.c_int),
                ("max_new_facets", C.c_int)]


class hf_step_report(C.Structure):
    _fields_ = [("newton_iters", C.c_int64), ("gmres_iters", C.c_int64), ("substeps", C.c_int64),
                ("cutbacks", C.c_int64), ("new_alpha", C.c_int64), ("new_beta", C.c_int64),
                ("t", C.c_double), ("du_rel", C.c_double), ("dp_rel", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hf_runtime_opts(C.Structure):
    _fields_ = [("slots", C.c_int), ("hbm_budget_bytes", C.c_int64), ("max_bypass", C.c_int), ("device", C.c_int)]


class hf_request(C.Structure):
    _fields_ = [("mesh", C.POINTER(hf_mesh_desc)),
                ("E", C.c_double), ("nu", C.c_double), ("sigma_c", C.c_double), ("delta_c", C.c_double),
                ("b_stab", C.c_double), ("mu", C.c_double), ("Q0", C.c_double),
                ("n_inj", C.c_int64), ("inj_dofs", _i64p), ("inj_weights", _dp),
                ("delta_f", C.c_double), ("dt", C.c_double), ("p_vapor", C.c_double),
                ("cutoff_on", C.c_int), ("L_ref", C.c_double),
                ("solver", hf_solver_opts), ("step", hf_step_opts), ("n_steps", C.c_int),
                ("U0", _dp), ("P0", _dp), ("alpha0", _i8p), ("beta0", _i8p), ("t0", C.c_double)]


class hf_result(C.Structure):
    _fields_ = [("status", C.c_int), ("n_u", C.c_int64), ("n_p", C.c_int64), ("n_faces", C.c_int64),
                ("steps_done", C.c_int64), ("newton_iters", C.c_int64), ("gmres_iters", C.c_int64),
                ("cutbacks", C.c_int64), ("device_bytes", C.c_int64), ("estimate_bytes", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("t_final", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_H = C.c_void_p
SIGNATURES = {
    "hf_default_solver_opts": (None, [C.POINTER(hf_solver_opts)]),
    "hf_mesh_create": (C.c_int, [C.POINTER(hf_mesh_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "hf_mesh_destroy": (C.c_int, [_H]),
    "hf_set_material": (C.c_int, [_H, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]),
    "hf_set_injection": (C.c_int, [_H, C.c_double, C.c_double, C.c_int64, _i64p, _dp, C.c_double,
                                   C.c_double, C.c_double, C.c_int, C.c_double]),
    "hf_set_solver": (C.c_int, [_H, C.POINTER(hf_solver_opts)]),
    "hf_set_fixed_pressure": (C.c_int, [_H, C.c_int64, _i64p, _dp]),
    "hf_set_wait_limit": (C.c_int, [_H, C.c_int64]),
    "hf_get_subdomains": (C.c_int, [_H, _i32p, _i32p]),
    "hf_check_wait_timeout": (C.c_int, [_H]),
    "hf_set_state": (C.c_int, [_H, _dp, _dp, _i8p, _i8p, _dp, C.c_double]),
    "hf_get_state": (C.c_int, [_H, _dp, _dp, _i8p, _i8p, _dp, _dp]),
    "hf_newton_step": (C.c_int, [_H, C.POINTER(hf_newton_report)]),
    "hf_check_fracture_criterion": (C.c_int, [_H, _i64p]),
    "hf_accept_step": (C.c_int, [_H, _i64p]),
    "hf_get_opening_pressure": (C.c_int, [_H, _dp, _dp, _i8p, _i8p]),
    "hf_get_sizes": (C.c_int, [_H, _i64p, _i64p, _i64p]),
    "hf_eval_residual": (C.c_int, [_H, _dp]),
    "hf_apply_jacobian": (C.c_int, [_H, _dp, _dp]),
    "hf_get_criterion_traction": (C.c_int, [_H, _dp]),
    "hf_apply_preconditioner": (C.c_int, [_H, _dp, _dp]),
    "hf_solve_linear": (C.c_int, [_H, _dp, _dp, C.POINTER(hf_newton_report)]),
    "hf_set_profiling": (C.c_int, [_H, C.c_int]),
    "hf_get_kernel_times": (C.c_int, [_H, _dp, _i64p]),
    "hf_get_stats": (C.c_int, [_H, _i64p]),
    "hf_last_error": (C.c_char_p, [_H]),
    "hf_increment_norms_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                             C.c_void_p, C.c_char_p, C.c_int64]),
    "hf_default_step_opts": (None, [C.POINTER(hf_step_opts)]),
    "hf_advance_step": (C.c_int, [_H, C.POINTER(hf_step_opts), C.POINTER(hf_step_report)]),
    "hf_mesh_sizes": (C.c_int, [C.POINTER(hf_mesh_desc), _i64p, _i64p]),
    "hf_get_aggregates": (C.c_int, [_H, _i32p]),
    "hf_get_coarse_operator": (C.c_int, [_H, _i64p, _dp, _dp, _dp]),
    "hf_estimate_device_bytes": (C.c_int, [C.POINTER(hf_mesh_desc), C.POINTER(hf_solver_opts), _i64p]),
    "hf_runtime_create": (C.c_int, [C.POINTER(hf_runtime_opts), C.POINTER(C.c_void_p)]),
    "hf_runtime_destroy": (C.c_int, [C.c_void_p]),
    "hf_runtime_submit": (C.c_int, [C.c_void_p, C.POINTER(hf_request), _i64p]),
    "hf_runtime_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.POINTER(hf_result)]),
    "hf_runtime_fetch": (C.c_int, [C.c_void_p, C.c_int64, _dp, _dp, _i8p, _i8p]),
    "hf_runtime_stats": (C.c_int, [C.c_void_p, _i64p]),
    "hf_runtime_now": (C.c_double, [C.c_void_p]),
}
KERNEL_CLASSES = ["spmv", "precond", "orth", "factor", "assembly", "spmv64", "update", "precond_aux", "gmres_cycles"]

_lib = None


def load(build_if_missing: bool = True):
    """Load libhfgb300.so (building it in-tree first when absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{path} is missing; run __graft_entry__.build()")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


class HFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def make_desc(dim, xyz, elem_nodes, face_elems, face_local, face_crackable, dir_dof, dir_val,
              neu_face=None, neu_traction=None):
    """hf_mesh_desc over contiguous copies of the arrays; returns (desc, keep),
    where keep owns the memory the descriptor points into."""
    keep = [np.ascontiguousarray(xyz, dtype=np.float64),
            np.ascontiguousarray(elem_nodes, dtype=np.int32),
            np.ascontiguousarray(face_elems, dtype=np.int32),
            np.ascontiguousarray(face_local, dtype=np.int8),
            np.ascontiguousarray(face_crackable, dtype=np.int8),
            np.ascontiguousarray(dir_dof, dtype=np.int64),
            np.ascontiguousarray(dir_val, dtype=np.float64),
            np.ascontiguousarray(neu_face if neu_face is not None else np.zeros(0), dtype=np.int32),
            np.ascontiguousarray(neu_traction if neu_traction is not None else np.zeros(0), dtype=np.float64)]
    x, en, fe, fl, fc, dd, dv, nf_, nt = keep
    d = hf_mesh_desc(dim, 2, x.shape[0], _ptr(x, C.c_double), en.shape[0], _ptr(en, C.c_int32),
                     fe.shape[0], _ptr(fe, C.c_int32), _ptr(fl, C.c_int8), _ptr(fc, C.c_int8),
                     dd.shape[0], _ptr(dd, C.c_int64), _ptr(dv, C.c_double),
                     nf_.shape[0], _ptr(nf_, C.c_int32), _ptr(nt, C.c_double))
    return d, keep


def desc_of(m):
    """make_desc for an object with the mesh attributes (dim, xyz, elem_nodes,
    face_elems, face_local, face_crackable, dir_dof, dir_val)."""
    return make_desc(m.dim, m.xyz, m.elem_nodes, m.face_elems, m.face_local, m.face_crackable, m.dir_dof,
                     m.dir_val)


def hf_mesh_sizes(m):
    d, keep = desc_of(m)
    nu, np_ = C.c_int64(), C.c_int64()
    st = load().hf_mesh_sizes(C.byref(d), C.byref(nu), C.byref(np_))
    if st != HF_OK:
        raise HFError(st, "hf_mesh_sizes")
    return nu.value, np_.value


def hf_estimate_device_bytes(m, **solver):
    """Device-memory bound of a handle for mesh m with these solver options
    (keyword arguments of hf_set_solver; the defaults otherwise)."""
    d, keep = desc_of(m)
    b = C.c_int64()
    o = solver_opts(**solver)
    st = load().hf_estimate_device_bytes(C.byref(d), C.byref(o), C.byref(b))
    if st != HF_OK:
        raise HFError(st, "hf_estimate_device_bytes")
    return b.value


def solver_opts(**kw):
    o = hf_solver_opts()
    load().hf_default_solver_opts(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = HF_PREC_MIXED if v == "mixed" else HF_PREC_FP64
        if k == "scheme" and isinstance(v, str):
            v = {"coupled": HF_SCHEME_COUPLED, "staggered": HF_SCHEME_STAGGERED}[v]
        setattr(o, k, v)
    return o


def step_opts(**kw):
    o = hf_step_opts()
    load().hf_default_step_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class HFMesh:
    """One discretised problem on the GPU (an hf_mesh handle)."""

    def __init__(self, dim, xyz, elem_nodes, face_elems, face_local, face_crackable, dir_dof, dir_val,
                 neu_face=None, neu_traction=None, stream=None):
        self.lib = load()
        d, self._keep = make_desc(dim, xyz, elem_nodes, face_elems, face_local, face_crackable, dir_dof, dir_val,
                                  neu_face, neu_traction)
        fe = self._keep[2]
        h = C.c_void_p()
        st = self.lib.hf_mesh_create(C.byref(d), C.c_void_p(stream) if stream else None, C.byref(h))
        if st != HF_OK:
            raise HFError(st, "hf_mesh_create failed")
        self.h = h
        self.dim = dim
        self.n_faces = fe.shape[0]
        nu, np_, nfn = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.hf_get_sizes(h, C.byref(nu), C.byref(np_), C.byref(nfn)))
        self.n_u, self.n_p, self.nfn = nu.value, np_.value, nfn.value
        self.N = self.n_u + self.n_p

    @classmethod
    def from_mesh(cls, m, **kw):
        return cls(m.dim, m.xyz, m.elem_nodes, m.face_elems, m.face_local, m.face_crackable,
                   m.dir_dof, m.dir_val, **kw)

    def _check(self, st):
        if st != HF_OK:
            raise HFError(st, self.lib.hf_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.hf_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up
    def hf_set_material(self, E, nu, sigma_c, delta_c, b_stab=10.0):
        self._check(self.lib.hf_set_material(self.h, E, nu, sigma_c, delta_c, b_stab))

    def hf_set_injection(self, mu, Q0, p_dofs, weights, delta_f, dt, p_vapor=0.0, cutoff_on=False, L_ref=1.0):
        pd = np.ascontiguousarray(p_dofs, dtype=np.int64)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        self._check(self.lib.hf_set_injection(self.h, mu, Q0, pd.shape[0], _ptr(pd, C.c_int64),
                                              _ptr(w, C.c_double), delta_f, dt, p_vapor,
                                              int(bool(cutoff_on)), L_ref))

    def default_opts(self):
        o = hf_solver_opts()
        self.lib.hf_default_solver_opts(C.byref(o))
        return o

    def hf_get_subdomains(self):
        ne = self._keep[1].shape[0]
        sd = np.zeros(ne, np.int32)
        order = np.zeros(ne, np.int32)
        self._check(self.lib.hf_get_subdomains(self.h, _ptr(sd, C.c_int32), _ptr(order, C.c_int32)))
        return sd, order

    def hf_set_wait_limit(self, polls):
        self._check(self.lib.hf_set_wait_limit(self.h, int(polls)))

    def hf_check_wait_timeout(self):
        self._check(self.lib.hf_check_wait_timeout(self.h))

    def hf_set_fixed_pressure(self, p_dofs, values):
        d = np.ascontiguousarray(p_dofs, dtype=np.int64)
        v = np.ascontiguousarray(values, dtype=np.float64)
        self._check(self.lib.hf_set_fixed_pressure(self.h, int(d.size), _ptr(d, C.c_int64), _ptr(v, C.c_double)))

    def hf_set_solver(self, **kw):
        o = solver_opts(**kw)
        self._check(self.lib.hf_set_solver(self.h, C.byref(o)))
        return o

    def hf_advance_step(self, **kw):
        """One time step (Newton, criterion, end of step, cutbacks); returns the
        step report as a dict."""
        o = step_opts(**kw)
        r = hf_step_report()
        self._check(self.lib.hf_advance_step(self.h, C.byref(o), C.byref(r)))
        return r.as_dict()

    def hf_set_state(self, U, P, alpha, beta, w_old=None, t=0.0):
        U = np.ascontiguousarray(U, dtype=np.float64)
        P = np.ascontiguousarray(P, dtype=np.float64)
        a = np.ascontiguousarray(alpha, dtype=np.int8)
        b = np.ascontiguousarray(beta, dtype=np.int8)
        wo = None if w_old is None else np.ascontiguousarray(w_old, dtype=np.float64)
        self._check(self.lib.hf_set_state(self.h, _ptr(U, C.c_double), _ptr(P, C.c_double), _ptr(a, C.c_int8),
                                          _ptr(b, C.c_int8), _ptr(wo, C.c_double), float(t)))

    def hf_get_state(self):
        U = np.zeros(self.n_u)
        P = np.zeros(max(self.n_p, 1))
        a = np.zeros(self.n_faces, np.int8)
        b = np.zeros(self.n_faces, np.int8)
        wo = np.zeros(self.n_faces * self.nfn)
        t = C.c_double()
        self._check(self.lib.hf_get_state(self.h, _ptr(U, C.c_double), _ptr(P, C.c_double), _ptr(a, C.c_int8),
                                          _ptr(b, C.c_int8), _ptr(wo, C.c_double), C.byref(t)))
        return U, P[: self.n_p], a, b, wo.reshape(self.n_faces, self.nfn), t.value

    # -- the Newton step and its companions
    def hf_newton_step(self):
        r = hf_newton_report()
        self._check(self.lib.hf_newton_step(self.h, C.byref(r)))
        return r.as_dict()

    def hf_check_fracture_criterion(self):
        n = C.c_int64()
        self._check(self.lib.hf_check_fracture_criterion(self.h, C.byref(n)))
        return n.value

    def hf_accept_step(self):
        n = C.c_int64()
        self._check(self.lib.hf_accept_step(self.h, C.byref(n)))
        return n.value

    def hf_get_opening_pressure(self):
        w = np.zeros(self.n_faces * self.nfn)
        p = np.zeros(max(self.n_p, 1))
        a = np.zeros(self.n_faces, np.int8)
        b = np.zeros(self.n_faces, np.int8)
        self._check(self.lib.hf_get_opening_pressure(self.h, _ptr(w, C.c_double), _ptr(p, C.c_double),
                                                     _ptr(a, C.c_int8), _ptr(b, C.c_int8)))
        return w.reshape(self.n_faces, self.nfn), p[: self.n_p], a, b

    # -- diagnostics
    def hf_eval_residual(self):
        R = np.zeros(self.N)
        self._check(self.lib.hf_eval_residual(self.h, _ptr(R, C.c_double)))
        return R

    def hf_apply_jacobian(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.N)
        self._check(self.lib.hf_apply_jacobian(self.h, _ptr(x, C.c_double), _ptr(y, C.c_double)))
        return y

    def hf_get_criterion_traction(self):
        t = np.zeros(self.n_faces)
        self._check(self.lib.hf_get_criterion_traction(self.h, _ptr(t, C.c_double)))
        return t

    def hf_apply_preconditioner(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        z = np.zeros(self.N)
        self._check(self.lib.hf_apply_preconditioner(self.h, _ptr(x, C.c_double), _ptr(z, C.c_double)))
        return z

    def hf_get_aggregates(self):
        a = np.zeros(self._keep[1].shape[0], np.int32)
        self._check(self.lib.hf_get_aggregates(self.h, _ptr(a, C.c_int32)))
        return a

    def hf_get_coarse_operator(self):
        """(A0, A0^-1, geo) of the coarse level: geo[g] = centre (3) and size."""
        nc = C.c_int64()
        self._check(self.lib.hf_get_coarse_operator(self.h, C.byref(nc), None, None, None))
        n = nc.value
        A0 = np.zeros((n, n))
        inv = np.zeros((n, n))
        nagg = n // (3 if self.dim == 2 else 6)
        geo = np.zeros((nagg, 4))
        self._check(self.lib.hf_get_coarse_operator(self.h, C.byref(nc), _ptr(A0, C.c_double), _ptr(inv, C.c_double),
                                                    _ptr(geo, C.c_double)))
        return A0, inv, geo

    def hf_set_profiling(self, on=True):
        """on: False/0 off, True/1 every kernel class, 2 whole GMRES cycles."""
        self._check(self.lib.hf_set_profiling(self.h, int(on)))

    def hf_get_kernel_times(self):
        ms = np.zeros(len(KERNEL_CLASSES))
        n = np.zeros(len(KERNEL_CLASSES), np.int64)
        self._check(self.lib.hf_get_kernel_times(self.h, _ptr(ms, C.c_double), _ptr(n, C.c_int64)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def hf_get_stats(self):
        st = np.zeros(16, np.int64)
        self._check(self.lib.hf_get_stats(self.h, _ptr(st, C.c_int64)))
        keys = ["elements", "interior_slots", "subdomain_slots", "levels_max", "subdomains", "nl_faces",
                "n_p", "faces", "kernel_launches", "graph_timing_error", "device_bytes", "coarse_unknowns",
                "aggregate_size", "gs_reorths", "gs_cols", "gs_reorth_cols"]
        return dict(zip(keys, (int(x) for x in st)))

    def hf_solve_linear(self, rhs):
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        d = np.zeros(self.N)
        r = hf_newton_report()
        self._check(self.lib.hf_solve_linear(self.h, _ptr(rhs, C.c_double), _ptr(d, C.c_double), C.byref(r)))
        return d, r.as_dict()


class HFRuntime:
    """The request loop of include/hf.h (hf_runtime_*): admission by free slot
    and device-memory budget, requests overlapping on the GPU."""

    def __init__(self, slots=8, hbm_budget_bytes=200 << 30, max_bypass=8, device=0):
        self.lib = load()
        o = hf_runtime_opts(int(slots), int(hbm_budget_bytes), int(max_bypass), int(device))
        h = C.c_void_p()
        st = self.lib.hf_runtime_create(C.byref(o), C.byref(h))
        if st != HF_OK:
            raise HFError(st, "hf_runtime_create")
        self.h = h

    def submit(self, mesh, *, E, nu, sigma_c, delta_c, mu, Q0, inj_dofs, inj_weights, delta_f, dt, n_steps,
               b_stab=10.0, p_vapor=0.0, cutoff_on=True, L_ref=1.0, solver=None, step=None, U0=None, P0=None,
               alpha0=None, beta0=None, t0=0.0):
        """Queue one request (mesh: an object with the mesh attributes); the
        runtime copies every array before this returns.  Returns its id."""
        d, keep = desc_of(mesh)
        inj = np.ascontiguousarray(inj_dofs, dtype=np.int64)
        wts = np.ascontiguousarray(inj_weights, dtype=np.float64)
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=t)
                for a, t in ((U0, np.float64), (P0, np.float64), (alpha0, np.int8), (beta0, np.int8))]
        r = hf_request(C.pointer(d), E, nu, sigma_c, delta_c, b_stab, mu, Q0, inj.shape[0], _ptr(inj, C.c_int64),
                       _ptr(wts, C.c_double), delta_f, dt, p_vapor, int(bool(cutoff_on)), L_ref,
                       solver_opts(**(solver or {})), step_opts(**(step or {})), int(n_steps),
                       _ptr(arrs[0], C.c_double), _ptr(arrs[1], C.c_double), _ptr(arrs[2], C.c_int8),
                       _ptr(arrs[3], C.c_int8), float(t0))
        i = C.c_int64()
        st = self.lib.hf_runtime_submit(self.h, C.byref(r), C.byref(i))
        if st != HF_OK:
            raise HFError(st, "hf_runtime_submit")
        return i.value

    def wait(self, rid, timeout=-1.0):
        """The request's hf_result as a dict, or None if it has not finished
        within timeout seconds."""
        res = hf_result()
        st = self.lib.hf_runtime_wait(self.h, int(rid), float(timeout), C.byref(res))
        if st == -6:
            return None
        if st != HF_OK:
            raise HFError(st, "hf_runtime_wait")
        return res.as_dict()

    def fetch(self, rid, res):
        """Final state (U, P, alpha, beta) of a finished request; forgets it."""
        U = np.zeros(max(res["n_u"], 1))
        P = np.zeros(max(res["n_p"], 1))
        a = np.zeros(max(res["n_faces"], 1), np.int8)
        b = np.zeros(max(res["n_faces"], 1), np.int8)
        st = self.lib.hf_runtime_fetch(self.h, int(rid), _ptr(U, C.c_double), _ptr(P, C.c_double), _ptr(a, C.c_int8),
                                       _ptr(b, C.c_int8))
        if st != HF_OK:
            raise HFError(st, "hf_runtime_fetch")
        return U[: res["n_u"]], P[: res["n_p"]], a[: res["n_faces"]], b[: res["n_faces"]]

    def stats(self):
        st = np.zeros(8, np.int64)
        self.lib.hf_runtime_stats(self.h, _ptr(st, C.c_int64))
        keys = ["queued", "running", "unfetched", "admitted_bytes", "peak_bytes", "peak_running", "completed",
                "failed"]
        return dict(zip(keys, (int(x) for x in st)))

    def now(self):
        return float(self.lib.hf_runtime_now(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.hf_runtime_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
