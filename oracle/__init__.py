"""TEST INFRASTRUCTURE ONLY: ctypes binding of the plain FP64 CPU oracle.

The oracle (``orc.cpp``) restates arXiv 2303.10785 step by step on the CPU in
FP64.  It is imported only by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; the product path never touches it.  It shares
no code with the CUDA library.  The only module both sides use is
``paper_2303_10785_b300.inputs`` (seeded grids and initial states).

Parity unpinned: the face state of the eigenvectors, the MP-limiter constants, the
value of the jet's Sutherland constant S/T_ref and the jet boundary/sponge forms.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle, lib_path


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("periodic", ctypes.c_int * 3),
        ("ghost_nodes", ctypes.c_int),
        ("bc", (ctypes.c_int * 2) * 3),
        ("metric_scheme", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("prandtl", ctypes.c_double),
        ("reynolds", ctypes.c_double),
        ("sutherland_s", ctypes.c_double),
        ("t_ref", ctypes.c_double),
        ("alpha_damping", ctypes.c_double),
        ("mp_alpha", ctypes.c_double),
        ("mp_beta", ctypes.c_double),
        ("mp_eps", ctypes.c_double),
        ("gradient_scheme", ctypes.c_int),
    ]


_LIBS = {}
_P = ctypes.POINTER(ctypes.c_double)


def _lib(counting=False):
    key = bool(counting)
    if key in _LIBS:
        return _LIBS[key]
    path = lib_path(counting)
    src = os.path.join(os.path.dirname(path), "orc.cpp")
    if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
        build_oracle()
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.orc_create.argtypes = [ctypes.POINTER(OrcParams), _P, _P, ctypes.POINTER(vp)]
    lib.orc_set_nodes.argtypes = [vp, _P, _P]
    lib.orc_set_centroids.argtypes = [vp, _P, _P]
    lib.orc_destroy.argtypes = [vp]
    lib.orc_last_error.restype = ctypes.c_char_p
    lib.orc_get_cell_metrics.argtypes = [vp, _P, _P]
    lib.orc_get_cell_time_metrics.argtypes = [vp, _P]
    lib.orc_get_face_metrics.argtypes = [vp, ctypes.c_int, _P, _P, _P]
    lib.orc_get_gcl.argtypes = [vp, _P]
    lib.orc_set_inflow.argtypes = [vp, _P]
    lib.orc_set_sponge.argtypes = [vp, _P, _P]
    lib.orc_rhs.argtypes = [vp, _P, _P]
    lib.orc_residual.argtypes = [vp, _P, _P]
    lib.orc_face_flux.argtypes = [vp, _P, ctypes.c_int, _P]
    lib.orc_primitives.argtypes = [vp, _P, _P]
    lib.orc_dt.argtypes = [vp, _P, ctypes.c_double]
    lib.orc_dt.restype = ctypes.c_double
    lib.orc_viscosity.argtypes = [vp, ctypes.c_double]
    lib.orc_viscosity.restype = ctypes.c_double
    lib.orc_rk3.argtypes = [vp, _P, ctypes.c_double, ctypes.POINTER(_P), ctypes.POINTER(_P)]
    lib.orc_op1d.argtypes = [ctypes.c_int, ctypes.c_int, _P, _P]
    lib.orc_eigen.argtypes = [ctypes.c_int, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P]
    lib.orc_hllc.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_double, ctypes.c_double, _P]
    lib.orc_mp_limit.argtypes = [ctypes.c_double] * 10
    lib.orc_mp_limit.restype = ctypes.c_double
    lib.orc_count_get.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)] * 4
    lib.orc_count_get_phase.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_ulonglong)] * 4
    _LIBS[key] = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_params(case):
    p = OrcParams()
    nd = int(case["ndim"])
    p.ndim = nd
    n = list(case["n"]) + [1] * (3 - len(case["n"]))
    per = list(case.get("periodic", (1, 1, 1))) + [1] * 3
    for d in range(3):
        p.n[d] = int(n[d]) if d < nd else 1
        p.periodic[d] = int(per[d])
    p.ghost_nodes = int(case.get("ghost_nodes", 10))
    bc = case.get("bc", ((1, 1), (1, 1), (1, 1)))
    for d in range(3):
        for s in range(2):
            p.bc[d][s] = int(bc[d][s])
    p.metric_scheme = int(case.get("metric_scheme", 0))
    for key in ("gamma", "prandtl", "reynolds", "sutherland_s", "t_ref", "alpha_damping", "mp_alpha", "mp_beta",
                "mp_eps"):
        setattr(p, key, float(case[key]))
    p.gradient_scheme = {"meg6": 0, "mig4": 1}[case.get("gradient_scheme", "meg6")]
    return p


class Oracle:
    """One grid of the oracle.  ``case`` is a dict from ``inputs.case_params``."""

    def __init__(self, case, nodes=None, node_vel=None, counting=False):
        self.lib = _lib(counting)
        self.case = dict(case)
        self.nd = int(case["ndim"])
        self.nv = self.nd + 2
        self.n = tuple(int(v) for v in case["n"][: self.nd])
        self.params = make_params(case)
        self.h = ctypes.c_void_p()
        nodes = _f64(nodes)
        node_vel = _f64(node_vel)
        rc = self.lib.orc_create(ctypes.byref(self.params), _ptr(nodes), _ptr(node_vel), ctypes.byref(self.h))
        if rc:
            raise ValueError(self.lib.orc_last_error().decode())

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.orc_destroy(self.h)
            self.h = ctypes.c_void_p()

    @property
    def cell_shape(self):
        return tuple(reversed(self.n))

    def face_shape(self, d):
        n = list(self.n)
        n[d] += 1
        return tuple(reversed(n))

    # ---- geometry
    def set_nodes(self, nodes, node_vel=None):
        nodes = _f64(nodes)
        node_vel = _f64(node_vel)
        if self.lib.orc_set_nodes(self.h, _ptr(nodes), _ptr(node_vel)):
            raise ValueError(self.lib.orc_last_error().decode())

    def set_centroids(self, xc_ext, vc_ext=None):
        xc_ext = _f64(xc_ext)
        vc_ext = _f64(vc_ext)
        if self.lib.orc_set_centroids(self.h, _ptr(xc_ext), _ptr(vc_ext)):
            raise ValueError(self.lib.orc_last_error().decode())

    def cell_metrics(self):
        nd = self.nd
        mh = np.zeros((nd, nd) + self.cell_shape)
        det = np.zeros(self.cell_shape)
        self.lib.orc_get_cell_metrics(self.h, _ptr(mh), _ptr(det))
        return mh, det

    def cell_time_metrics(self):
        mt = np.zeros((self.nd,) + self.cell_shape)
        self.lib.orc_get_cell_time_metrics(self.h, _ptr(mt))
        return mt

    def face_metrics(self, d):
        nd = self.nd
        fs = self.face_shape(d)
        fh = np.zeros((nd,) + fs)
        fu = np.zeros((nd, nd) + fs)
        ft = np.zeros(fs)
        self.lib.orc_get_face_metrics(self.h, d, _ptr(fh), _ptr(fu), _ptr(ft))
        return fh, fu, ft

    def gcl(self):
        g = np.zeros(self.cell_shape)
        self.lib.orc_get_gcl(self.h, _ptr(g))
        return g

    def set_inflow(self, prim):
        prim = _f64(prim)
        self.lib.orc_set_inflow(self.h, _ptr(prim))

    def set_sponge(self, sigma, q_amb):
        self._sponge = (_f64(sigma), _f64(q_amb))
        self.lib.orc_set_sponge(self.h, _ptr(self._sponge[0]), _ptr(self._sponge[1]))

    # ---- right-hand side
    def _state(self, q):
        q = _f64(q)
        assert q.shape == (self.nv,) + self.cell_shape, q.shape
        return q

    def rhs(self, q):
        q = self._state(q)
        out = np.zeros_like(q)
        self.lib.orc_rhs(self.h, _ptr(q), _ptr(out))
        return out

    def residual(self, q):
        q = self._state(q)
        out = np.zeros_like(q)
        self.lib.orc_residual(self.h, _ptr(q), _ptr(out))
        return out

    def face_flux(self, q, d):
        q = self._state(q)
        out = np.zeros((self.nv,) + self.face_shape(d))
        self.lib.orc_face_flux(self.h, _ptr(q), d, _ptr(out))
        return out

    def primitives(self, q):
        q = self._state(q)
        out = np.zeros_like(q)
        self.lib.orc_primitives(self.h, _ptr(q), _ptr(out))
        return out

    def dt(self, q, cfl):
        q = self._state(q)
        return float(self.lib.orc_dt(self.h, _ptr(q), float(cfl)))

    def viscosity(self, T):
        """Dynamic viscosity mu(T) (Sec. 2) of this grid's parameters."""
        return float(self.lib.orc_viscosity(self.h, float(T)))

    def rk3(self, q, dt, stage_nodes=None, stage_vel=None):
        q = self._state(q).copy()
        sn = sv = None
        keep = []
        if stage_nodes is not None:
            arrs = [_f64(a) for a in stage_nodes]
            keep += arrs
            sn = (_P * 3)(*[_ptr(a) for a in arrs])
            if stage_vel is not None:
                varrs = [_f64(a) for a in stage_vel]
                keep += varrs
                sv = (_P * 3)(*[_ptr(a) for a in varrs])
        rc = self.lib.orc_rk3(self.h, _ptr(q), float(dt), sn, sv)
        if rc:
            raise ValueError(self.lib.orc_last_error().decode())
        return q


def op1d(kind, f, counting=False):
    """Line operators: 'e6', 'second', 'face', 'D', 'e4', 'ig4' on a periodic line; 'ig4_open':
    IG4 on an open line whose three end points at each side take the explicit end rows; 'D_walls':
    the metric derivative D on a line bounded by walls (App. C)
    (counting=True: run in the operation-counting build, for flop_counts)."""
    k = {"e6": 0, "second": 1, "face": 2, "D": 3, "e4": 4, "ig4": 5, "ig4_open": 6, "D_walls": 7}[kind]
    f = _f64(f)
    out = np.zeros_like(f)
    _lib(counting).orc_op1d(k, f.size, _ptr(f), _ptr(out))
    return out


def eigen(nd, nh, rho, p, gamma=1.4):
    nv = nd + 2
    R = np.zeros((nv, nv))
    L = np.zeros((nv, nv))
    nh3 = np.zeros(3)
    v = np.asarray(nh, dtype=np.float64).reshape(-1)
    nh3[: min(3, v.size)] = v[:3]
    _lib().orc_eigen(nd, _ptr(nh3), float(rho), float(p), float(gamma), _ptr(R), _ptr(L))
    return R, L


def hllc(nd, PL, PR, nh, nt=0.0, gamma=1.4):
    nv = nd + 2
    F = np.zeros(nv)
    nh3 = np.zeros(3)
    nh3[:nd] = np.asarray(nh, dtype=np.float64)[:nd]
    _lib().orc_hllc(nd, _ptr(_f64(PL)), _ptr(_f64(PR)), _ptr(nh3), float(nt), float(gamma), _ptr(F))
    return F


def mp_limit(wface, w_up, w_base, w_down, d_up, d_base, d_down, alpha=4.0, beta=4.0, eps=1e-20):
    return float(_lib().orc_mp_limit(wface, w_up, w_base, w_down, d_up, d_base, d_down, alpha, beta, eps))


PHASES = {"misc": 0, "prim": 1, "grad": 2, "face": 3, "res": 4, "geom": 5}


def flop_counts(fn):
    """Run ``fn()`` (which must use ``Oracle(..., counting=True)``) and return the operation
    tallies per phase of the method (add/sub, mul, div, sqrt; flops = their sum)."""
    lib = _lib(True)
    lib.orc_count_reset()
    fn()
    out = {}
    for name, ph in list(PHASES.items()) + [("all", -1)]:
        vals = [ctypes.c_ulonglong() for _ in range(4)]
        lib.orc_count_get_phase(ph, *[ctypes.byref(v) for v in vals])
        add, mul, div, sq = (v.value for v in vals)
        out[name] = {"add": add, "mul": mul, "div": div, "sqrt": sq, "flops": add + mul + div + sq}
    return out


def threads():
    return int(_lib().orc_threads())


def set_threads(n):
    """Threads the oracle's loops use from now on (timing at one thread and at all cores)."""
    _lib().orc_set_threads(int(n))
