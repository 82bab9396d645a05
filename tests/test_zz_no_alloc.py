"""qnep_ewald_kspace_noalloc against the reciprocal-space part of qnep_compute.

The entry point serves callers that must not allocate device memory (a host
program that owns all GPU memory through its own pool, or a time-critical loop
where cudaMalloc would synchronise the device).  This test calls it through the
C ABI twice in a row on the charges and positions of a mode-2 Ewald force call
(mode 2 has no real-space or self term, so the existing entry point's potential
is exactly the reciprocal-space potential) and compares potential and energy
with it, and potential, energy, forces and the 3x3 static virial element by
element with the FP64 oracle's reciprocal-space Ewald sum of the same charges,
with the tolerances of the parity tests.  The file is named so that pytest
collects it last; it also runs alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


def _entry(lib):
    return lib.qnep_ewald_kspace_noalloc   # argument types declared by the binding


def test_noalloc_matches_qnep_compute_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    from paper_2601_19034_gb300.qnep import QNEP, parse_scalars

    lib = _lib.load()
    fn = _entry(lib)
    dev = torch.device("cuda:0")
    sysm, hp, params, _ = wl.config_water_small()
    elec = wl.Elec(mode=2, kind="ewald")
    model = QNEP(hp, params, elec)
    pos = torch.tensor(sysm.positions, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    ref = model.compute(pos, typ, sysm.box, potential=True)
    torch.cuda.synchronize()
    ref_sc = parse_scalars(ref["scalars"])
    n = sysm.n_atoms
    # the oracle's reciprocal-space sum (mode 2: U^k only) of the same charges and positions
    from oracle import ewald as oewald
    q64 = ref["charges"].double().cpu().numpy()
    ora = oewald.ewald_static(sysm.positions.astype(np.float64), np.asarray(sysm.box, np.float64), q64, None, elec,
                              with_kspace=True)
    box = (ctypes.c_double * 9)(*np.asarray(sysm.box, np.float64).ravel())
    err = ctypes.create_string_buffer(256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        phi = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
        force = torch.full((n, 3), float("nan"), dtype=torch.float32, device=dev)
        ev = torch.full((10,), float("nan"), dtype=torch.float64, device=dev)
        st = fn(n, pos.data_ptr(), ref["charges"].data_ptr(), box, elec.alpha, elec.kmax, phi.data_ptr(),
                force.data_ptr(), ev.data_ptr(), stream, err, len(err))
        assert st == 0, err.value.decode()
        torch.cuda.synchronize()
        assert abs(ev[0].item() - ref_sc["e_kspace"]) / n <= 1e-6
        assert (phi - ref["potential"]).abs().max().item() <= 2e-5
        evh = ev.cpu().numpy()
        assert abs(evh[0] - ora["e_kspace"]) / n <= 1e-6
        phih = phi.double().cpu().numpy()
        assert np.abs(phih - ora["phi"]).max() <= 1e-5 * np.abs(ora["phi"]).max()
        assert np.abs(force.double().cpu().numpy() - ora["force"]).max() <= 1e-4
        assert np.abs(evh[1:10].reshape(3, 3) - ora["virial"]).max() / n <= 1e-5
    # sizes beyond the fixed array are refused before any GPU work, with a message
    big = torch.zeros((8193, 3), dtype=torch.float32, device=dev)
    q = torch.zeros(8193, dtype=torch.float32, device=dev)
    st = fn(8193, big.data_ptr(), q.data_ptr(), box, elec.alpha, elec.kmax, None, None, None, stream, err, len(err))
    assert st == _lib.QNEP_ERR_UNSUPPORTED and b"QNEP_NOALLOC_MAX_ATOMS" in err.value
    model.close()
