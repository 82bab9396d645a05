"""Device status words reach the caller: a bounded wait that gave up is QNEP_ERR_TIMEOUT.

No device wait is made to run out: a test hook ORs the timeout bit into the status
word of the last call from the host (as a kernel that gave up would), and the status
calls of the single-structure model and of the batch must both return
QNEP_ERR_TIMEOUT; a clean call before and after returns QNEP_OK.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_single_structure_timeout_bit_is_reported(dev):
    from paper_2601_19034_gb300 import _lib
    from paper_2601_19034_gb300.qnep import QNEP

    sysm, hp, params, elec = wl.config_water_small()
    model = QNEP(hp, params, elec)
    pos = torch.tensor(sysm.positions, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    model.compute(pos, typ, sysm.box)
    assert model.sync_status() == _lib.QNEP_OK
    assert model.lib.qnep_debug_set_status(model.handle, 2) == _lib.QNEP_OK
    assert model.sync_status() == _lib.QNEP_ERR_TIMEOUT
    assert b"wait gave up" in model.lib.qnep_last_error(model.handle)
    # the next call starts from a clean word
    out = model.compute(pos, typ, sysm.box)
    assert model.sync_status() == _lib.QNEP_OK
    assert torch.isfinite(out["forces"]).all()
    model.close()


def test_batch_timeout_bit_is_reported(dev):
    from paper_2601_19034_gb300 import _lib
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures

    base = wl.llzo_base_cell()
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(5), n_candidates=32)
    pos, typ, off, boxes = stack_structures([base])
    b = QNEPBatch(hp, params, wl.Elec(mode=1, kind="ewald"))
    pt, tt = torch.tensor(pos, device=dev), torch.tensor(typ, device=dev)
    b.compute(pt, tt, off, boxes)
    assert b.sync_status() == _lib.QNEP_OK
    assert b.lib.qnep_batch_debug_set_status(b.handle, 2) == _lib.QNEP_OK
    assert b.sync_status() == _lib.QNEP_ERR_TIMEOUT
    # overflow takes precedence over a timeout in the same word
    assert b.lib.qnep_batch_debug_set_status(b.handle, 1) == _lib.QNEP_OK
    assert b.sync_status() == _lib.QNEP_ERR_NBR_OVERFLOW
    out = b.compute(pt, tt, off, boxes)
    assert b.sync_status() == _lib.QNEP_OK
    assert torch.isfinite(out["energy"]).all()
    b.close()
