"""gbr_rhs_static: the right-hand side for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc or own a workspace (code inside another
framework's memory pool, under a fixed device-memory budget, or forbidden to
allocate after start-up).  gbr_rhs_static keeps all of its scratch in one
fixed-size array compiled into the library, so such callers pass only their
inputs and outputs.  This test calls it through the C ABI twice in a row (the
scratch keeps the previous call's contents) and checks both results against the
regular workspace path (gbr_create + gbr_compute_metrics + gbr_rhs), within the
tolerance of the other right-hand-side tests: 1e-12 of the cancellation scale.
It is collected last so that a run that stops at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2303_10785_b300 import gbr
from paper_2303_10785_b300 import inputs as I
from _util import cancellation_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _static_rhs(case, nodes, q_dev, out_dev, vel=None):
    import torch

    lib = gbr.lib()
    p = gbr.make_params(dict(case, moving=1 if vel is not None else 0))
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
    msg = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream()
    rc = lib.gbr_rhs_static(ctypes.byref(p), nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            None if vel is None else vel.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            ctypes.c_void_p(q_dev.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()),
                            ctypes.c_void_p(stream.cuda_stream), msg, ctypes.c_size_t(256))
    stream.synchronize()
    return rc, msg.value.decode()


def _workspace_rhs(case, nodes, q, vel=None):
    s = gbr.Solver(case, nodes, vel, moving=1 if vel is not None else 0)
    s.set_state(q)
    L = s.rhs().cpu().numpy()
    s.close()
    return L


def _err(a, b, scale):
    return (np.abs(a - b).reshape(a.shape[0], -1).max(axis=1) / scale).max()


def test_static_scratch_rhs_matches_workspace_rhs_twice_in_a_row():
    import torch

    n = (21, 18, 16)
    case = I.case_params(3, n, reynolds=1600.0)
    nodes = I.nodes_random(n, (2 * np.pi,) * 3, frac=0.15)
    xc = I.centroids(nodes, n, (1, 1, 1))
    q1 = I.prim_to_cons(I.tgv_prim(*xc), 1.4)
    q2 = I.prim_to_cons(I.tgv_prim(xc[0] + 0.3, xc[1] - 0.2, xc[2] + 0.1, mach=0.3), 1.4)
    scale1 = cancellation_scale(O.Oracle(case, nodes), q1)
    scale2 = cancellation_scale(O.Oracle(case, nodes), q2)
    out = torch.empty(q1.shape, dtype=torch.float64, device="cuda")
    for q, scale in ((q1, scale1), (q2, scale2)):
        ref = _workspace_rhs(case, nodes, q)
        qd = torch.from_numpy(q).cuda()
        rc, msg = _static_rhs(case, nodes, qd, out)
        assert rc == gbr.GBR_OK, msg
        assert _err(out.cpu().numpy(), ref, scale) < 1e-12


def test_static_scratch_rhs_moving_2d_after_3d():
    import torch

    m = I.motion_dynamic_2d(n=40, L=10.0, amp=0.3)
    case = I.case_params(2, (40, 40))
    nodes, vel = m.nodes(0.21), m.velocity(0.21)
    xc = I.centroids(nodes, (40, 40), (1, 1))
    q = I.prim_to_cons(I.vortex_prim(xc[0], xc[1]), 1.4)
    ref = _workspace_rhs(case, nodes, q, vel)
    scale = cancellation_scale(O.Oracle(case, nodes, vel), q)
    out = torch.empty(q.shape, dtype=torch.float64, device="cuda")
    rc, msg = _static_rhs(case, nodes, torch.from_numpy(q).cuda(), out, vel)
    assert rc == gbr.GBR_OK, msg
    assert _err(out.cpu().numpy(), ref, scale) < 1e-12


def test_static_scratch_rejects_oversize_grid():
    import torch

    n = (128, 128, 128)
    case = I.case_params(3, n, reynolds=1600.0)
    nodes = I.nodes_uniform(n, (1.0, 1.0, 1.0))
    q = torch.zeros((5, 2), dtype=torch.float64, device="cuda")
    rc, msg = _static_rhs(case, nodes, q, q)
    assert rc == gbr.GBR_EINVAL
    assert "too large" in msg


def test_static_scratch_rhs_open_axis_with_ghost_nodes():
    """A non-periodic x axis with zero-gradient sides and 10 ghost node layers: exercises the ghost-node
    offset of the node extension and the zero-gradient primitive ghosts of the allocation-free path."""
    import torch

    n = (26, 14, 12)
    L = (3.0, 2.0, 2.0)
    h = [Lx / m for Lx, m in zip(L, n)]

    def f(i, j, k):
        x, y, z = i * h[0], j * h[1], k * h[2]
        s = 0.04 * np.sin(2 * np.pi * x / 3.0) * np.sin(2 * np.pi * y / 2.0) * np.sin(2 * np.pi * z / 2.0)
        return x + s, y + 0.5 * s, z - s

    nodes = I.nodes_from_functions(n, (0, 1, 1), 10, f)
    case = I.case_params(3, n, periodic=(0, 1, 1), reynolds=400.0, ghost_nodes=10)
    xc = I.centroids(nodes, n, (0, 1, 1))
    P = I.tgv_prim(2 * np.pi * xc[0] / 3.0, np.pi * xc[1], np.pi * xc[2], mach=0.3)
    P[0] = P[0] * (1.0 + 0.1 * np.tanh(4.0 * (xc[0] - 1.5)))  # a density ramp across the open axis
    q = I.prim_to_cons(P, 1.4)
    ref = _workspace_rhs(case, nodes, q)
    scale = cancellation_scale(O.Oracle(case, nodes), q)
    out = torch.empty(q.shape, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        rc, msg = _static_rhs(case, nodes, torch.from_numpy(q).cuda(), out)
        assert rc == gbr.GBR_OK, msg
        assert _err(out.cpu().numpy(), ref, scale) < 1e-12
