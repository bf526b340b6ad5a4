"""GPU: pipelined host transfers (gbr_set_state_async / gbr_get_state_async) against the
synchronous gbr_set_state / gbr_get_state: the same states bit for bit, step after step, while the
uploads and downloads run on copy streams beside the steps."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2303_10785_b300 import gbr
from test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pipelined_transfers_equal_synchronous(precision):
    case, nodes, vel, q = CASES["3d_tgv"]()
    case = dict(case, precision=precision)
    K = 4
    # one problem per step: the state scaled by 1 + k/100 (same velocity, pressure scaled)
    states = [q * (1.0 + 0.01 * k) for k in range(K)]
    s = gbr.Solver(case, nodes, vel)
    ref = []
    for k in range(K):
        s.set_state(states[k])
        s.rk_step(0.3)
        ref.append(s.get_state())
    s.close()

    s = gbr.Solver(case, nodes, vel)
    h_in = [torch.from_numpy(x.copy()).pin_memory() for x in states]
    h_out = [torch.empty(q.shape, dtype=torch.float64).pin_memory() for _ in range(K)]
    for k in range(K):
        s.set_state_async(h_in[k])
        s.rk_step(0.3)
        s.get_state_async(h_out[k])
    s.sync()
    for k in range(K):
        assert np.array_equal(h_out[k].numpy(), ref[k]), k
    assert not np.array_equal(ref[0], ref[1])
    # pageable host memory is refused (the copy engines would stage it synchronously)
    pageable = np.ascontiguousarray(states[0])
    stage = s._stage("in")
    assert s.L.gbr_set_state_async(s.h, ctypes.c_void_p(pageable.ctypes.data), ctypes.c_void_p(stage.data_ptr())) == gbr.GBR_EINVAL
    s.close()
