"""GPU: batched stepping (gbr_batch_*) against each member stepped alone with gbr_rk_step.

The batch runs the same kernel bodies on the same data in the same order as the
per-context path (the primitives and ghost layers in one pass instead of
interior + axis-by-axis copies, which copy the same values), and the time step
is an exact minimum, so every member's state and time must be bitwise equal to
those of the member stepped alone -- whatever the batch composition, membership
changes, graph replay or tuning.
"""
import numpy as np
import pytest

from paper_2303_10785_b300 import gbr
from paper_2303_10785_b300 import inputs as I
from test_gpu_parity import GAMMA, case_2d_viscous_random, case_2d_vortex, case_3d_inviscid_ragged, case_jet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def tgv(n, precision="fp64"):
    case = I.case_params(3, (n, n, n), reynolds=1600.0, precision=precision)
    nodes = I.nodes_tgv_3d(n, 0.1)
    xc = I.centroids(nodes, (n, n, n), (1, 1, 1))
    return case, nodes, I.prim_to_cons(I.tgv_prim(*xc, mach=0.1), GAMMA)


def sod(precision="fp64"):
    n = (40, 32)
    case = I.case_params(2, n, precision=precision)
    nodes = I.nodes_skewed_2d(n, (1.25, 1.0), skew_deg=25.0, jitter=0.1, seed=5)
    xc = I.centroids(nodes, n, (1, 1))
    rho, p = I.sod_slab_prim(xc[1], L=1.0)
    P = np.stack([rho, np.zeros_like(rho), np.zeros_like(rho), p])
    return case, nodes, I.prim_to_cons(P, GAMMA)


def jobs():
    """(case, nodes, q, cfl_or_neg_dt, extra): every kind the batch groups, CFL and fixed steps."""
    out = []
    c, n, _, q = case_2d_vortex(48)
    out.append((c, n, q, 0.4, None))
    out.append((dict(c, precision="mixed"), n, q, 0.4, None))
    c, n, _, q = case_2d_viscous_random()
    out.append((c, n, q, 0.3, None))
    c, n, q = tgv(20)
    out.append((c, n, q, 0.2, None))
    c, n, q = tgv(24, "mixed")
    out.append((c, n, q, 0.2, None))
    c, n, _, q = case_3d_inviscid_ragged()
    out.append((dict(c, precision="mixed"), n, q, -2e-3, None))
    c, n, q = sod()
    out.append((c, n, q, 0.3, None))
    c, n, _, q, extra = case_jet()
    out.append((c, n, q, -2e-3, extra))
    return out


def make(job):
    case, nodes, q, _, extra = job
    s = gbr.Solver(case, nodes)
    if extra:
        s.set_inflow(extra["inflow"])
        s.set_sponge(extra["sigma"], extra["qamb"])
    s.set_state(q)
    return s


def alone(job, steps):
    s = make(job)
    for _ in range(steps):
        s.rk_step(job[3])
    s.sync()
    out = s.get_state(), s.time()
    s.close()
    return out


@pytest.mark.parametrize("use_graph,autotune", [(True, True), (False, False)])
def test_batch_results_bitwise_equal_to_members_alone(use_graph, autotune):
    js = jobs()
    steps = 4
    refs = [alone(j, steps) for j in js]
    b = gbr.Batch(len(js), use_graph=use_graph, autotune=autotune)
    members = [make(j) for j in js]
    for s, j in zip(members, js):
        b.add(s, j[3])
    b.step(steps)
    b.sync()
    info = b.info()
    assert info["members"] == len(js) and info["kinds"] == 6
    assert info["launches"] == steps * info["launches_per_step"]
    for s, (qref, tref) in zip(members, refs):
        assert np.array_equal(s.get_state(), qref)
        assert s.time() == tref
    for t in b.tuning():
        assert t["face_block"] in (64, 128, 256) and t["fused_grad"] in (0, 1)
    b.close()
    for s in members:
        s.close()


def test_batch_membership_changes_between_steps():
    js = jobs()[:5]
    b = gbr.Batch(8)
    s = [make(j) for j in js]
    b.add(s[0], js[0][3])
    b.add(s[3], js[3][3])
    b.step(2)
    b.add(s[1], js[1][3])   # joins after two steps
    b.add(s[4], js[4][3])
    b.step(1)
    b.remove(s[0])           # leaves after three steps
    b.add(s[2], js[2][3])
    b.step(3)
    b.sync()
    done = {0: 3, 1: 4, 2: 3, 3: 6, 4: 4}
    for m, steps in done.items():
        qref, tref = alone(js[m], steps)
        assert np.array_equal(s[m].get_state(), qref), m
        assert s[m].time() == tref
    b.close()
    for x in s:
        x.close()


def test_batch_rejects_a_foreign_stream_and_duplicates():
    import torch

    b = gbr.Batch(2)
    c, n, _, q = case_2d_vortex(32)
    other = gbr.Solver(c, n, stream=torch.cuda.Stream())
    with pytest.raises(gbr.GbrError):
        b.add(other, 0.4)
    mine = gbr.Solver(c, n)
    b.add(mine, 0.4)
    with pytest.raises(gbr.GbrError):
        b.add(mine, 0.4)
    b.close()
    mine.close()
    other.close()


def test_batch_reports_the_member_with_a_bad_state():
    js = jobs()[:2]
    b = gbr.Batch(2)
    s = [make(j) for j in js]
    q = js[1][2].copy()
    q[0, 0, 0] = -1.0  # negative density in one cell of the second member
    s[1].set_state(q)
    for x, j in zip(s, js):
        b.add(x, -1e-3)
    b.step(1)
    with pytest.raises(gbr.GbrError) as e:
        b.sync()
    assert e.value.status == gbr.GBR_ENONFINITE and "member 1" in str(e.value)
    b.close()
    for x in s:
        x.close()


def _oracle_steps(job, steps):
    """The member's states after `steps` SSP-RK3 steps on the oracle (own CFL time step, or fixed)."""
    import oracle as O

    case, nodes, q, cfl, extra = job
    orc = O.Oracle(dict(case, precision="fp64"), nodes)
    if extra:
        orc.set_inflow(extra["inflow"])
        orc.set_sponge(extra["sigma"], extra["qamb"])
    qo = q.copy()
    for _ in range(steps):
        qo = orc.rk3(qo, orc.dt(qo, cfl) if cfl > 0 else -cfl)
    _, det = orc.cell_metrics()
    return qo, det


def test_batch_members_match_the_oracle():
    """Every kind the batch groups, after 10 batched steps, against the FP64 oracle: FP64 members
    within 1e-10 of max |Q| (L1 <= 1e-8 where the limiter is active: the Sod slab and the jet's
    inflow edge); mixed members within 1e-5 (L-infinity, against the FP64 oracle)."""
    from test_gpu_parity import rel_state

    js = jobs()
    smooth = {0, 2, 3}  # the FP64 vortex, viscous random-mesh vortex and Taylor-Green members of jobs()
    steps = 10
    b = gbr.Batch(len(js))
    members = [make(j) for j in js]
    for s, j in zip(members, js):
        b.add(s, j[3])
    b.step(steps)
    b.sync()
    for m, (s, j) in enumerate(zip(members, js)):
        qo, det = _oracle_steps(j, steps)
        qg = s.get_state()
        nv = qg.shape[0]
        if j[0].get("precision", "fp64") == "mixed":
            assert rel_state(qg, qo) < 1e-5, m
            continue
        l1 = (np.abs(qg - qo) * det).reshape(nv, -1).sum(axis=1) / (np.abs(qo) * det).reshape(nv, -1).sum(axis=1)
        assert l1.max() < 1e-8, m
        if m in smooth:
            assert rel_state(qg, qo) < 1e-10, m
    b.close()
    for s in members:
        s.close()


def moving_and_mig4_jobs():
    """Members with per-member work: prescribed motion (2D FP64, 3D viscous mixed), MIG4 (3D viscous
    FP64, 2D mixed), a moving MIG4 member, and a static MEG6 member beside them."""
    out = []
    m2 = I.motion_dynamic_2d(n=40, L=10.0, amp=0.3)
    c2 = I.case_params(2, (40, 40), moving=1)
    xc = I.centroids(m2.nodes(0.0), (40, 40), (1, 1))
    q2 = I.prim_to_cons(I.vortex_prim(xc[0], xc[1]), GAMMA)
    out.append((c2, m2, q2, 0.4))
    m3 = I.motion_deforming_3d(n=16, L=12.0)
    c3 = I.case_params(3, (16, 16, 16), moving=1, reynolds=500.0, precision="mixed")
    xc3 = I.centroids(m3.nodes(0.0), (16, 16, 16), (1, 1, 1))
    s = 2 * np.pi / 12.0
    q3 = I.prim_to_cons(I.tgv_prim(xc3[0] * s, xc3[1] * s, xc3[2] * s, mach=0.3), GAMMA)
    out.append((c3, m3, q3, -0.01))
    c, n, q = tgv(20)
    out.append((dict(c, gradient_scheme="mig4"), n, q, 0.2))
    c, n, _, q = case_2d_vortex(48)
    out.append((dict(c, gradient_scheme="mig4", precision="mixed"), n, q, 0.4))
    out.append((dict(c2, gradient_scheme="mig4"), m2, q2, -0.01))
    out.append((c, n, q, 0.4))
    return out


def make_mv(job):
    case, geo, q, _ = job
    if isinstance(geo, np.ndarray):
        s = gbr.Solver(case, geo)
    else:
        s = gbr.Solver(case, geo.nodes(0.0), geo.velocity(0.0))
        s.set_motion(geo, 0.0)
    s.set_state(q)
    return s


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_moving_mesh_and_mig4_members_bitwise_equal_alone(use_graph):
    """Members with prescribed motion recompute their geometry at every stage time inside the batched
    step, MIG4 members solve their own gradient lines there; every member's state and time are bitwise
    those of gbr_rk_step on it alone."""
    js = moving_and_mig4_jobs()
    steps = 4
    refs = []
    for j in js:
        s = make_mv(j)
        for _ in range(steps):
            s.rk_step(j[3])
        s.sync()
        refs.append((s.get_state(), s.time()))
        s.close()
    b = gbr.Batch(len(js), use_graph=use_graph, autotune=False)
    members = [make_mv(j) for j in js]
    for s, j in zip(members, js):
        b.add(s, j[3])
    b.step(steps)
    b.sync()
    info = b.info()
    assert info["members"] == len(js) and info["kinds"] == 6
    assert info["launches_per_step"] > 0 and info["launches"] == steps * info["launches_per_step"]
    for m, (s, (qref, tref)) in enumerate(zip(members, refs)):
        assert np.array_equal(s.get_state(), qref), m
        assert s.time() == tref, m
    b.close()
    for s in members:
        s.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_fused_stage_kernel_bitwise_equal_to_members_alone(use_graph):
    """The fused stage kernel (every phase of a stage in one persistent cooperative launch, grid-wide
    barriers between the phases) on every kind of jobs(): each member's state and time bitwise those of
    gbr_rk_step alone, as for the phase kernels."""
    js = jobs()
    steps = 3
    refs = [alone(j, steps) for j in js]
    b = gbr.Batch(len(js), use_graph=use_graph, autotune=2)
    members = [make(j) for j in js]
    for s, j in zip(members, js):
        b.add(s, j[3])
    b.step(steps)
    b.sync()
    info = b.info()
    assert info["launches"] == steps * info["launches_per_step"]
    assert all(t["fused_stage"] == 1 and t["face_block"] == 128 for t in b.tuning())
    for s, (qref, tref) in zip(members, refs):
        assert np.array_equal(s.get_state(), qref)
        assert s.time() == tref
    b.close()
    for s in members:
        s.close()
    # fewer launches per step than the phase kernels
    b0 = gbr.Batch(len(js), use_graph=use_graph, autotune=0)
    m0 = [make(j) for j in js]
    for s, j in zip(m0, js):
        b0.add(s, j[3])
    assert b0.info()["launches_per_step"] > info["launches_per_step"]
    b0.close()
    for s in m0:
        s.close()


def test_fused_stage_barrier_timeout_is_reported():
    """The grid barrier of the fused stage kernel waits a bounded number of polls: its timeout path,
    run on purpose (a barrier no arrival completes, no fault), sets the batch's sticky flag and
    gbr_batch_sync reports GBR_ETIMEOUT; the members' states are left as they were."""
    js = jobs()[:2]
    b = gbr.Batch(2, autotune=2)
    members = [make(j) for j in js]
    for s, j in zip(members, js):
        b.add(s, j[3])
    b.step(1)
    b.sync()
    before = [s.get_state() for s in members]
    b.check_barrier(2000)
    with pytest.raises(gbr.GbrError) as e:
        b.sync()
    assert e.value.status == gbr.GBR_ETIMEOUT
    for s, q in zip(members, before):
        assert np.array_equal(s.get_state(), q)
    b.close()
    for s in members:
        s.close()
