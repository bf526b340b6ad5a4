"""Thin ctypes binding of the C ABI in include/gbr.h (argument marshalling only).

Every step of the right-hand side runs in the in-tree CUDA library
``libgbr.so`` (sm_103a).  PyTorch supplies device memory (the workspace and
state tensors) and the CUDA stream; it does no arithmetic of the method.
Importing this module without the built library raises immediately: there is
no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbr.so")

GBR_OK, GBR_EINVAL, GBR_ENOMEM, GBR_ECUDA, GBR_ENONFINITE, GBR_ETIMEOUT, GBR_ESTATE = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENONFINITE", "ETIMEOUT", "ESTATE"]
(GBR_FIELD_CELL_METRICS, GBR_FIELD_CELL_DET, GBR_FIELD_CELL_TIME, GBR_FIELD_FACE_HAT, GBR_FIELD_FACE_UNHAT,
 GBR_FIELD_FACE_TIME, GBR_FIELD_GCL, GBR_FIELD_FACE_FLUX) = range(8)
GBR_PREC_FP64, GBR_PREC_MIXED = 0, 1
GBR_BC_ZEROGRAD, GBR_BC_INFLOW, GBR_BC_WALL = 1, 2, 3
GBR_GRAD_MEG6, GBR_GRAD_MIG4 = 0, 1


class gbr_params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("periodic", ctypes.c_int * 3),
        ("ghost_nodes", ctypes.c_int),
        ("bc", (ctypes.c_int * 2) * 3),
        ("gamma", ctypes.c_double),
        ("prandtl", ctypes.c_double),
        ("reynolds", ctypes.c_double),
        ("sutherland_s", ctypes.c_double),
        ("t_ref", ctypes.c_double),
        ("alpha_damping", ctypes.c_double),
        ("mp_alpha", ctypes.c_double),
        ("mp_beta", ctypes.c_double),
        ("mp_eps", ctypes.c_double),
        ("moving", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("gradient_scheme", ctypes.c_int),
    ]


class gbr_motion(ctypes.Structure):
    _fields_ = [
        ("origin", ctypes.c_double * 3),
        ("h", ctypes.c_double * 3),
        ("amp", ctypes.c_double * 3),
        ("omega", ctypes.c_double),
        ("k", (ctypes.c_double * 3) * 3),
    ]


class GbrError(RuntimeError):
    def __init__(self, status, msg, member=-1):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status
        self.member = member  # Batch.sync: index of the first member with a bad state (else -1)


_lib = None
_P = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is not built (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    L.gbr_workspace_bytes.argtypes = [ctypes.POINTER(gbr_params)]
    L.gbr_workspace_bytes.restype = ctypes.c_size_t
    L.gbr_create.argtypes = [ctypes.POINTER(gbr_params), _P, _P, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]
    L.gbr_compute_metrics.argtypes = [_vp]
    L.gbr_move_mesh.argtypes = [_vp, _P, _P]
    L.gbr_set_motion.argtypes = [_vp, ctypes.POINTER(gbr_motion), ctypes.c_double]
    L.gbr_set_state.argtypes = [_vp, _vp, ctypes.c_int]
    L.gbr_get_state.argtypes = [_vp, _vp, ctypes.c_int]
    L.gbr_set_inflow.argtypes = [_vp, _vp, ctypes.c_int]
    L.gbr_set_sponge.argtypes = [_vp, _P, _P]
    L.gbr_rhs.argtypes = [_vp, _vp]
    L.gbr_compute_dt.argtypes = [_vp, ctypes.c_double, _P]
    L.gbr_rk_step.argtypes = [_vp, ctypes.c_double]
    L.gbr_sync.argtypes = [_vp, ctypes.c_double]
    L.gbr_get_time.argtypes = [_vp, _P, _P]
    L.gbr_get_field.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _P]
    L.gbr_profile.argtypes = [_vp, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    L.gbr_check_bounded_wait.argtypes = [_vp, ctypes.c_int]
    L.gbr_alu_peak.argtypes = [ctypes.c_int, _vp, _P, _P]
    L.gbr_alu_peak.restype = ctypes.c_int
    L.gbr_check_rcp.argtypes = [ctypes.c_longlong, ctypes.c_ulonglong, _vp, ctypes.POINTER(ctypes.c_longlong)]
    L.gbr_check_rcp.restype = ctypes.c_int
    L.gbr_set_state_async.argtypes = [_vp, _vp, _vp]
    L.gbr_get_state_async.argtypes = [_vp, _vp, _vp]
    L.gbr_profile.restype = ctypes.c_int
    L.gbr_rhs_static.argtypes = [ctypes.POINTER(gbr_params), _P, _P, _vp, _vp, _vp, ctypes.c_char_p, ctypes.c_size_t]
    L.gbr_rhs_static.restype = ctypes.c_int
    _ll = ctypes.c_longlong
    _ip = ctypes.POINTER(ctypes.c_int)
    L.gbr_batch_workspace_bytes.argtypes = [ctypes.c_int]
    L.gbr_batch_workspace_bytes.restype = ctypes.c_size_t
    L.gbr_batch_create.argtypes = [ctypes.c_int, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]
    L.gbr_batch_set_options.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.gbr_batch_add.argtypes = [_vp, _vp, ctypes.c_double]
    L.gbr_batch_remove.argtypes = [_vp, _vp]
    L.gbr_batch_step.argtypes = [_vp, ctypes.c_int]
    L.gbr_batch_sync.argtypes = [_vp, ctypes.c_double, _ip]
    L.gbr_batch_info.argtypes = [_vp, _ip, _ip, ctypes.POINTER(_ll), ctypes.POINTER(_ll)]
    L.gbr_batch_tuning.argtypes = [_vp, ctypes.c_int, _ip, _ip, _ip, _ip, _ip, _ip]
    L.gbr_batch_check_barrier.argtypes = [_vp, ctypes.c_int]
    L.gbr_batch_check_barrier.restype = ctypes.c_int
    L.gbr_batch_last_error.argtypes = [_vp]
    L.gbr_batch_last_error.restype = ctypes.c_char_p
    L.gbr_batch_destroy.argtypes = [_vp]
    L.gbr_arena_create.argtypes = [_vp, ctypes.c_size_t, ctypes.POINTER(_vp)]
    L.gbr_arena_alloc.argtypes = [_vp, ctypes.c_size_t, ctypes.POINTER(_vp)]
    L.gbr_arena_free.argtypes = [_vp, _vp]
    L.gbr_arena_stats.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_size_t)] * 3 + [_ip]
    L.gbr_arena_destroy.argtypes = [_vp]
    for name in ("gbr_batch_create", "gbr_batch_set_options", "gbr_batch_add", "gbr_batch_remove", "gbr_batch_step",
                 "gbr_batch_sync", "gbr_batch_info", "gbr_batch_tuning", "gbr_arena_create", "gbr_arena_alloc",
                 "gbr_arena_free", "gbr_arena_stats"):
        getattr(L, name).restype = ctypes.c_int
    L.gbr_last_error.argtypes = [_vp]
    L.gbr_last_error.restype = ctypes.c_char_p
    L.gbr_last_global_error.restype = ctypes.c_char_p
    L.gbr_destroy.argtypes = [_vp]
    for name in ("gbr_create", "gbr_compute_metrics", "gbr_move_mesh", "gbr_set_motion", "gbr_set_state",
                 "gbr_get_state", "gbr_set_inflow", "gbr_set_sponge", "gbr_rhs", "gbr_compute_dt", "gbr_rk_step",
                 "gbr_sync", "gbr_get_time", "gbr_get_field"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/gbr.h that the library must export."""
    return ["gbr_workspace_bytes", "gbr_create", "gbr_compute_metrics", "gbr_move_mesh", "gbr_set_motion",
            "gbr_set_state", "gbr_get_state", "gbr_set_inflow", "gbr_set_sponge", "gbr_rhs", "gbr_compute_dt",
            "gbr_set_state_async", "gbr_get_state_async", "gbr_rk_step", "gbr_sync", "gbr_get_time", "gbr_get_field",
            "gbr_profile", "gbr_check_bounded_wait", "gbr_alu_peak", "gbr_check_rcp",
            "gbr_rhs_static",
            "gbr_batch_workspace_bytes", "gbr_batch_create", "gbr_batch_set_options", "gbr_batch_add",
            "gbr_batch_remove", "gbr_batch_step", "gbr_batch_sync", "gbr_batch_info", "gbr_batch_tuning",
            "gbr_batch_check_barrier", "gbr_batch_last_error", "gbr_batch_destroy", "gbr_arena_create", "gbr_arena_alloc", "gbr_arena_free",
            "gbr_arena_stats", "gbr_arena_destroy", "gbr_last_error", "gbr_last_global_error", "gbr_destroy"]


def alu_peak(precision="fp64", stream=None):
    """Measured FMA throughput of the current device: (TFLOP/s, ms of the timed launch)."""
    L = lib()
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    st = None if stream is None else _vp(stream.cuda_stream)
    rc = L.gbr_alu_peak({"fp64": GBR_PREC_FP64, "mixed": GBR_PREC_MIXED}[precision], st, ctypes.byref(tf),
                        ctypes.byref(ms))
    if rc:
        raise GbrError(rc, L.gbr_last_global_error().decode())
    return tf.value, ms.value


def check_rcp(n, seed=0, stream=None):
    """Largest ulp distance between the kernels' FP64 reciprocal and the division over n random x."""
    L = lib()
    out = ctypes.c_longlong()
    st = None if stream is None else _vp(stream.cuda_stream)
    rc = L.gbr_check_rcp(int(n), int(seed), st, ctypes.byref(out))
    if rc:
        raise GbrError(rc, L.gbr_last_global_error().decode())
    return out.value


def make_params(case):
    p = gbr_params()
    nd = int(case["ndim"])
    p.ndim = nd
    n = list(case["n"]) + [1] * 3
    per = list(case.get("periodic", (1, 1, 1))) + [1] * 3
    for d in range(3):
        p.n[d] = int(n[d]) if d < nd else 1
        p.periodic[d] = int(per[d])
    p.ghost_nodes = int(case.get("ghost_nodes", 10))
    bc = case.get("bc", ((1, 1), (1, 1), (1, 1)))
    for d in range(3):
        for s in range(2):
            p.bc[d][s] = int(bc[d][s])
    for key in ("gamma", "prandtl", "reynolds", "sutherland_s", "t_ref", "alpha_damping", "mp_alpha", "mp_beta",
                "mp_eps"):
        setattr(p, key, float(case[key]))
    p.moving = int(case.get("moving", 0))
    p.precision = {"fp64": GBR_PREC_FP64, "mixed": GBR_PREC_MIXED}[case.get("precision", "fp64")]
    p.gradient_scheme = {"meg6": GBR_GRAD_MEG6, "mig4": GBR_GRAD_MIG4}[case.get("gradient_scheme", "meg6")]
    return p


def make_motion(m):
    """gbr_motion from an ``inputs.SinusoidalMotion``."""
    g = gbr_motion()
    for a in range(m.nd):
        g.origin[a] = m.origin[a]
        g.h[a] = m.h[a]
        g.amp[a] = m.amp[a]
        for b in range(m.nd):
            g.k[a][b] = m.k[a][b]
    g.omega = m.omega
    return g


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


class Solver:
    """One grid on one GPU.  ``case`` is a dict from ``inputs.case_params``."""

    def __init__(self, case, nodes, node_vel=None, device="cuda", stream=None, moving=None, workspace=None):
        """workspace: optional (device pointer, bytes) owned by the caller (e.g. from an ``Arena``);
        by default a torch tensor of ``workspace_bytes`` is allocated."""
        import torch

        self.torch = torch
        self.L = lib()
        self.case = dict(case)
        if moving is not None:
            self.case["moving"] = int(moving)
        elif node_vel is not None:
            self.case["moving"] = 1
        self.nd = int(case["ndim"])
        self.nv = self.nd + 2
        self.n = tuple(int(v) for v in case["n"][: self.nd])
        self.params = make_params(self.case)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = self.L.gbr_workspace_bytes(ctypes.byref(self.params))
        if nbytes == 0:
            raise GbrError(GBR_EINVAL, self.L.gbr_last_global_error().decode())
        self.workspace_bytes = int(nbytes)
        if workspace is None:
            self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) & ~255
        else:
            aligned, avail = int(workspace[0]), int(workspace[1])
            if avail < self.workspace_bytes:
                raise GbrError(GBR_ENOMEM, "external workspace smaller than gbr_workspace_bytes")
            self.workspace = None
        self.h = _vp()
        nodes = _f64(nodes)
        node_vel = _f64(node_vel)
        rc = self.L.gbr_create(ctypes.byref(self.params), _ptr(nodes), _ptr(node_vel), _vp(aligned),
                               ctypes.c_size_t(self.workspace_bytes), _vp(self.stream.cuda_stream), ctypes.byref(self.h))
        if rc:
            raise GbrError(rc, self.L.gbr_last_global_error().decode())
        self._check(self.L.gbr_compute_metrics(self.h))

    def _check(self, rc):
        if rc:
            raise GbrError(rc, self.L.gbr_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.gbr_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        self.close()

    @property
    def cell_shape(self):
        return tuple(reversed(self.n))

    def face_shape(self, d):
        n = list(self.n)
        n[d] += 1
        return tuple(reversed(n))

    # ---- state
    def set_state(self, q):
        t = self.torch
        if isinstance(q, t.Tensor) and q.is_cuda:
            q = q.contiguous().to(t.float64)
            self._check(self.L.gbr_set_state(self.h, _vp(q.data_ptr()), 1))
            self.stream.synchronize()
        else:
            q = _f64(q)
            assert q.shape == (self.nv,) + self.cell_shape, q.shape
            self._check(self.L.gbr_set_state(self.h, _vp(q.ctypes.data), 0))

    def get_state(self):
        out = np.empty((self.nv,) + self.cell_shape)
        self._check(self.L.gbr_get_state(self.h, _vp(out.ctypes.data), 0))
        return out

    def state_into(self, tensor):
        self._check(self.L.gbr_get_state(self.h, _vp(tensor.data_ptr()), 1))

    def _stage(self, which):
        # device staging buffers of the pipelined transfers ("in", "out"), allocated on first use
        stages = self.__dict__.setdefault("_stages", {})
        if which not in stages:
            stages[which] = self.torch.empty((self.nv,) + self.cell_shape, dtype=self.torch.float64,
                                             device=self.device)
        return stages[which]

    def set_state_async(self, host):
        """Upload a pinned host tensor [nv][cells] (float64) on a copy stream; it becomes the state
        at this point of the stream order.  Keep it unchanged until sync()."""
        assert host.is_pinned() and host.dtype == self.torch.float64 and host.is_contiguous()
        self._check(self.L.gbr_set_state_async(self.h, _vp(host.data_ptr()), _vp(self._stage("in").data_ptr())))

    def get_state_async(self, host):
        """Download the state at this point of the stream order into a pinned host tensor on a copy
        stream; valid after sync()."""
        assert host.is_pinned() and host.dtype == self.torch.float64 and host.is_contiguous()
        self._check(self.L.gbr_get_state_async(self.h, _vp(host.data_ptr()), _vp(self._stage("out").data_ptr())))

    # ---- method
    def rhs(self, out=None):
        t = self.torch
        if out is None:
            out = t.empty((self.nv,) + self.cell_shape, dtype=t.float64, device=self.device)
        self._check(self.L.gbr_rhs(self.h, _vp(out.data_ptr())))
        return out

    def dt(self, cfl):
        v = ctypes.c_double()
        self._check(self.L.gbr_compute_dt(self.h, float(cfl), ctypes.byref(v)))
        return v.value

    def rk_step(self, cfl_or_neg_dt):
        self._check(self.L.gbr_rk_step(self.h, float(cfl_or_neg_dt)))

    def sync(self, timeout=60.0):
        self._check(self.L.gbr_sync(self.h, float(timeout)))

    def check_bounded_wait(self, polls=64):
        """Run the kernels' bounded-wait timeout path on purpose (a wait nothing completes): the
        next sync raises GbrError with status GBR_ETIMEOUT."""
        self._check(self.L.gbr_check_bounded_wait(self.h, int(polls)))

    def time(self):
        t = ctypes.c_double()
        dt = ctypes.c_double()
        self._check(self.L.gbr_get_time(self.h, ctypes.byref(t), ctypes.byref(dt)))
        return t.value, dt.value

    def move_mesh(self, nodes, node_vel=None):
        nodes = _f64(nodes)
        node_vel = _f64(node_vel)
        self._check(self.L.gbr_move_mesh(self.h, _ptr(nodes), _ptr(node_vel)))

    def set_motion(self, motion, t0=0.0):
        self._motion = make_motion(motion)
        self._check(self.L.gbr_set_motion(self.h, ctypes.byref(self._motion), float(t0)))

    def set_inflow(self, prim):
        """x-low inflow primitives [nv][nk][nj]: a host array, or a CUDA tensor copied in stream order."""
        t = self.torch
        if isinstance(prim, t.Tensor) and prim.is_cuda:
            assert prim.dtype == t.float64 and prim.is_contiguous()
            self._check(self.L.gbr_set_inflow(self.h, _vp(prim.data_ptr()), 1))
        else:
            prim = _f64(prim)
            self._check(self.L.gbr_set_inflow(self.h, _vp(prim.ctypes.data), 0))

    def set_sponge(self, sigma, q_amb):
        sigma = _f64(sigma)
        q_amb = _f64(q_amb)
        self._check(self.L.gbr_set_sponge(self.h, _ptr(sigma), _ptr(q_amb)))

    def profile(self, enable=True):
        """(face-kernel ms, face launches, kernel launches) since the last call; then (re)arms recording."""
        ms = ctypes.c_double()
        nf = ctypes.c_longlong()
        nl = ctypes.c_longlong()
        self._check(self.L.gbr_profile(self.h, int(enable), ctypes.byref(ms), ctypes.byref(nf), ctypes.byref(nl)))
        return ms.value, nf.value, nl.value

    # ---- read-back for tests
    def field(self, which, d=0):
        nd = self.nd
        shapes = {
            GBR_FIELD_CELL_METRICS: (nd, nd) + self.cell_shape,
            GBR_FIELD_CELL_DET: self.cell_shape,
            GBR_FIELD_CELL_TIME: (nd,) + self.cell_shape,
            GBR_FIELD_FACE_HAT: (nd,) + self.face_shape(d),
            GBR_FIELD_FACE_UNHAT: (nd, nd) + self.face_shape(d),
            GBR_FIELD_FACE_TIME: self.face_shape(d),
            GBR_FIELD_GCL: self.cell_shape,
            GBR_FIELD_FACE_FLUX: (self.nv,) + self.face_shape(d),
        }
        out = np.empty(shapes[which])
        self._check(self.L.gbr_get_field(self.h, which, d, _ptr(out)))
        return out


class Batch:
    """Many static-mesh ``Solver``s advanced together (one launch per phase and kind, one CUDA graph
    per step).  Members must use the batch's stream."""

    def __init__(self, max_members, device="cuda", stream=None, use_graph=True, autotune=True):
        import torch

        self.L = lib()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = int(self.L.gbr_batch_workspace_bytes(int(max_members)))
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) & ~255
        self.h = _vp()
        rc = self.L.gbr_batch_create(int(max_members), _vp(aligned), ctypes.c_size_t(nbytes),
                                     _vp(self.stream.cuda_stream), ctypes.byref(self.h))
        if rc:
            raise GbrError(rc, self.L.gbr_last_global_error().decode())
        self._check(self.L.gbr_batch_set_options(self.h, int(use_graph), int(autotune)))
        self.members = []

    def _check(self, rc):
        if rc:
            raise GbrError(rc, self.L.gbr_batch_last_error(self.h).decode())

    def add(self, solver, cfl_or_neg_dt):
        self._check(self.L.gbr_batch_add(self.h, solver.h, float(cfl_or_neg_dt)))
        self.members.append(solver)

    def remove(self, solver):
        self._check(self.L.gbr_batch_remove(self.h, solver.h))
        self.members.remove(solver)

    def step(self, n=1):
        self._check(self.L.gbr_batch_step(self.h, int(n)))

    def sync(self, timeout=60.0):
        """Drain the stream; GbrError (ENONFINITE) names the first member whose state went bad in
        .member (the others are unaffected: members share launches, not data)."""
        bad = ctypes.c_int(-1)
        rc = self.L.gbr_batch_sync(self.h, float(timeout), ctypes.byref(bad))
        if rc:
            raise GbrError(rc, self.L.gbr_batch_last_error(self.h).decode(), bad.value)

    def info(self):
        m, k = ctypes.c_int(), ctypes.c_int()
        lps, lt = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self.L.gbr_batch_info(self.h, ctypes.byref(m), ctypes.byref(k), ctypes.byref(lps),
                                          ctypes.byref(lt)))
        return {"members": m.value, "kinds": k.value, "launches_per_step": lps.value, "launches": lt.value}

    def check_barrier(self, polls=1000):
        """Run the fused stage kernel's barrier timeout path on purpose (the next sync raises ETIMEOUT)."""
        self._check(self.L.gbr_batch_check_barrier(self.h, int(polls)))

    def tuning(self):
        out = []
        for kind in range(self.info()["kinds"]):
            v = [ctypes.c_int() for _ in range(6)]
            self._check(self.L.gbr_batch_tuning(self.h, kind, *[ctypes.byref(x) for x in v]))
            out.append(dict(zip(("ndim", "viscous", "mixed", "face_block", "fused_grad", "fused_stage"),
                                (x.value for x in v))))
        return out

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.gbr_batch_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        self.close()


class Arena:
    """First-fit bookkeeping of one device range (``gbr_arena_*``): jobs are admitted when their
    workspace fits."""

    def __init__(self, base, nbytes):
        self.L = lib()
        self.h = _vp()
        rc = self.L.gbr_arena_create(_vp(int(base)), ctypes.c_size_t(int(nbytes)), ctypes.byref(self.h))
        if rc:
            raise GbrError(rc, self.L.gbr_last_global_error().decode())
        self.capacity = int(nbytes) & ~255

    def alloc(self, nbytes):
        """Device pointer, or None when no free range fits."""
        p = _vp()
        rc = self.L.gbr_arena_alloc(self.h, ctypes.c_size_t(int(nbytes)), ctypes.byref(p))
        if rc == GBR_ENOMEM:
            return None
        if rc:
            raise GbrError(rc, self.L.gbr_last_global_error().decode())
        return p.value

    def free(self, ptr):
        rc = self.L.gbr_arena_free(self.h, _vp(int(ptr)))
        if rc:
            raise GbrError(rc, self.L.gbr_last_global_error().decode())

    def stats(self):
        v = [ctypes.c_size_t() for _ in range(3)]
        nb = ctypes.c_int()
        self.L.gbr_arena_stats(self.h, *[ctypes.byref(x) for x in v], ctypes.byref(nb))
        return {"used": v[0].value, "free": v[1].value, "largest_free": v[2].value, "blocks": nb.value}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.gbr_arena_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        self.close()
