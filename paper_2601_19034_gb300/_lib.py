"""ctypes view of the C ABI in include/qnep.h (argument marshalling only).

``load()`` opens the in-tree ``libqnep.so``; it raises if the library has not
been built, so nothing silently falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqnep.so")

QNEP_OK = 0
QNEP_ERR_ARG = 1
QNEP_ERR_CUDA = 2
QNEP_ERR_NBR_OVERFLOW = 3
QNEP_ERR_UNSUPPORTED = 4
QNEP_ERR_TIMEOUT = 5
QNEP_ERR_OOM = 6
QNEP_BATCH_CONTRACT_FP32 = 0
QNEP_BATCH_CONTRACT_BF16X3 = 1
QNEP_BATCH_CONTRACT_BF16 = 2
QNEP_EWALD = 0
QNEP_PPPM = 1
QNEP_PREC_FP32 = 0
QNEP_PREC_MLP_BF16 = 1
QNEP_PREC_MLP_TF32 = 2
QNEP_NSCALARS = 20
QNEP_NSTAGES = 10
QNEP_BATCH_ORDER_LARGEST_FIRST, QNEP_BATCH_ORDER_STRUCTURE = 0, 1
QNEP_PATH_AUTO = 0
QNEP_PATH_WARP = 1
QNEP_PATH_THREAD = 2
SCALAR_NAMES = {
    "energy": 0, "e_nep": 1, "e_real": 2, "e_kspace": 3, "e_self": 4,
    "virial": slice(5, 14), "polarization": slice(14, 17), "qtilde_sum": 17, "phi_mean": 18, "status": 19,
}


class HParamsC(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int), ("rc_radial", ctypes.c_float), ("rc_angular", ctypes.c_float),
                ("n_radial", ctypes.c_int), ("n_angular", ctypes.c_int), ("basis_radial", ctypes.c_int),
                ("basis_angular", ctypes.c_int), ("l_max", ctypes.c_int), ("use_4body", ctypes.c_int),
                ("n_neurons", ctypes.c_int)]


class ElecC(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("kind", ctypes.c_int), ("alpha", ctypes.c_double),
                ("rc_real", ctypes.c_double), ("kmax", ctypes.c_double), ("mesh", ctypes.c_int * 3),
                ("order", ctypes.c_int), ("q_total", ctypes.c_double)]


class OutputsC(ctypes.Structure):
    _fields_ = [("scalars", ctypes.c_void_p), ("forces", ctypes.c_void_p), ("charges", ctypes.c_void_p),
                ("bec", ctypes.c_void_p), ("site_energy", ctypes.c_void_p), ("potential", ctypes.c_void_p),
                ("descriptor", ctypes.c_void_p), ("want_virial", ctypes.c_int), ("atom_virial", ctypes.c_void_p)]


class VjpC(ctypes.Structure):
    _fields_ = [("energy_weight", ctypes.c_double), ("charge_weight", ctypes.c_void_p),
                ("polar_weight", ctypes.c_double * 3), ("grad", ctypes.c_void_p)]


class BatchOutputsC(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_void_p), ("forces", ctypes.c_void_p), ("charges", ctypes.c_void_p),
                ("virial", ctypes.c_void_p), ("bec", ctypes.c_void_p), ("total_charge", ctypes.c_void_p),
                ("polarization", ctypes.c_void_p)]


class LossInputsC(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_void_p), ("forces", ctypes.c_void_p), ("virial", ctypes.c_void_p),
                ("bec", ctypes.c_void_p), ("total_charge", ctypes.c_void_p)]


class LossWeightsFullC(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("force", ctypes.c_double), ("virial", ctypes.c_double),
                ("bec", ctypes.c_double), ("charge", ctypes.c_double), ("l1", ctypes.c_double),
                ("l2", ctypes.c_double)]


class LossWeightsVC(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("force", ctypes.c_double), ("virial", ctypes.c_double),
                ("l1", ctypes.c_double), ("l2", ctypes.c_double)]


class LossWeightsC(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("force", ctypes.c_double), ("l1", ctypes.c_double),
                ("l2", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def _declare(lib):
    p = ctypes.c_void_p
    i = ctypes.c_int
    lib.qnep_param_count.argtypes = [ctypes.POINTER(HParamsC)]
    lib.qnep_param_count.restype = ctypes.c_size_t
    lib.qnep_create.argtypes = [ctypes.POINTER(p), ctypes.POINTER(HParamsC), p, ctypes.c_size_t, i,
                                ctypes.POINTER(ElecC), i]
    lib.qnep_create.restype = i
    lib.qnep_reserve.argtypes = [p, i, p]
    lib.qnep_reserve.restype = i
    lib.qnep_compute.argtypes = [p, i, p, p, p, p, ctypes.POINTER(OutputsC)]
    lib.qnep_compute.restype = i
    lib.qnep_compute_vjp.argtypes = [p, i, p, p, p, p, ctypes.POINTER(OutputsC), ctypes.POINTER(VjpC)]
    lib.qnep_compute_vjp.restype = i
    lib.qnep_compute_host.argtypes = [p, i, p, p, p, p, ctypes.POINTER(OutputsC)]
    lib.qnep_compute_host.restype = i
    lib.qnep_sync_status.argtypes = [p, p]
    lib.qnep_sync_status.restype = i
    lib.qnep_status_from_device_bits.argtypes = [ctypes.c_uint]
    lib.qnep_status_from_device_bits.restype = i
    lib.qnep_debug_set_status.argtypes = [p, ctypes.c_uint]
    lib.qnep_debug_set_status.restype = i
    lib.qnep_batch_debug_set_status.argtypes = [p, ctypes.c_uint]
    lib.qnep_batch_debug_set_status.restype = i
    lib.qnep_set_path.argtypes = [p, i]
    lib.qnep_set_path.restype = i
    lib.qnep_set_capacity.argtypes = [p, i, i]
    lib.qnep_set_capacity.restype = i
    lib.qnep_set_skin.argtypes = [p, ctypes.c_double]
    lib.qnep_set_skin.restype = i
    lib.qnep_skin_rebuilds.argtypes = [p, ctypes.POINTER(ctypes.c_uint)]
    lib.qnep_skin_rebuilds.restype = i
    lib.qnep_destroy.argtypes = [p]
    lib.qnep_destroy.restype = None
    lib.qnep_status_string.argtypes = [i]
    lib.qnep_status_string.restype = ctypes.c_char_p
    lib.qnep_last_error.argtypes = [p]
    lib.qnep_last_error.restype = ctypes.c_char_p
    lib.qnep_set_profiling.argtypes = [p, i]
    lib.qnep_set_profiling.restype = i
    lib.qnep_stage_times.argtypes = [p, ctypes.POINTER(ctypes.c_float), i, ctypes.POINTER(i)]
    lib.qnep_stage_times.restype = i
    lib.qnep_stage_name.argtypes = [i]
    lib.qnep_stage_name.restype = ctypes.c_char_p
    lib.qnep_nve_run.argtypes = [p, i, p, p, p, p, p, ctypes.c_double, i, p, p, p]
    lib.qnep_nve_run.restype = i
    lib.qnep_nve_run_field.argtypes = [p, i, p, p, p, p, p, ctypes.c_double, i, p, p, p, p, p, p]
    lib.qnep_nve_run_field.restype = i
    lib.qnep_field_response.argtypes = [i, p, p, p, p, i, p, p]
    lib.qnep_field_response.restype = i
    lib.qnep_ewald_kspace_noalloc.argtypes = [i, p, p, p, ctypes.c_double, ctypes.c_double, p, p, p, p,
                                              ctypes.c_char_p, ctypes.c_size_t]
    lib.qnep_ewald_kspace_noalloc.restype = i
    # batched evaluation
    lib.qnep_batch_create.argtypes = [ctypes.POINTER(p), ctypes.POINTER(HParamsC), p, ctypes.c_size_t, i,
                                      ctypes.POINTER(ElecC)]
    lib.qnep_batch_create.restype = i
    lib.qnep_batch_compute.argtypes = [p, i, p, p, p, p, p, p, p, p]
    lib.qnep_batch_compute.restype = i
    lib.qnep_batch_compute_outputs.argtypes = [p, i, p, p, p, p, p, ctypes.POINTER(BatchOutputsC)]
    lib.qnep_batch_compute_outputs.restype = i
    lib.qnep_batch_compute_host.argtypes = [p, i, p, p, p, p, p, ctypes.POINTER(BatchOutputsC)]
    lib.qnep_batch_compute_host.restype = i
    lib.qnep_batch_loss_v.argtypes = [i, i, p, i, p, p, p, p, p, p, p, i, ctypes.POINTER(LossWeightsVC), p, p, p]
    lib.qnep_batch_loss_v.restype = i
    lib.qnep_batch_loss_full.argtypes = [i, i, p, i, ctypes.POINTER(LossInputsC), ctypes.POINTER(LossInputsC), p, p,
                                         i, ctypes.POINTER(LossWeightsFullC), p, p, p]
    lib.qnep_batch_loss_full.restype = i
    lib.qnep_batch_set_static_geometry.argtypes = [p, i]
    lib.qnep_batch_set_static_geometry.restype = i
    lib.qnep_batch_geometry_changed.argtypes = [p]
    lib.qnep_batch_geometry_changed.restype = i
    lib.qnep_batch_set_contraction.argtypes = [p, i]
    lib.qnep_batch_set_contraction.restype = i
    lib.qnep_batch_get_contraction.argtypes = [p, ctypes.POINTER(i)]
    lib.qnep_batch_get_contraction.restype = i
    lib.qnep_batch_sync_status.argtypes = [p]
    lib.qnep_batch_sync_status.restype = i
    lib.qnep_batch_set_capacity.argtypes = [p, i, i]
    lib.qnep_batch_set_capacity.restype = i
    lib.qnep_batch_capacity.argtypes = [p, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.qnep_batch_capacity.restype = i
    lib.qnep_batch_set_config.argtypes = [p, i, i]
    lib.qnep_batch_set_config.restype = i
    lib.qnep_batch_get_config.argtypes = [p, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.qnep_batch_get_config.restype = i
    lib.qnep_batch_autotune.argtypes = [p, i, p, p, p, p, p, p, p, p, i, ctypes.POINTER(ctypes.c_double)]
    lib.qnep_batch_autotune.restype = i
    lib.qnep_batch_set_profiling.argtypes = [p, i]
    lib.qnep_batch_set_profiling.restype = i
    lib.qnep_batch_stage_times.argtypes = [p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i)]
    lib.qnep_batch_stage_times.restype = i
    lib.qnep_batch_last_error.argtypes = [p]
    lib.qnep_batch_last_error.restype = ctypes.c_char_p
    lib.qnep_batch_set_params.argtypes = [p, p, p]
    lib.qnep_batch_set_params.restype = i
    lib.qnep_snes_sample.argtypes = [i, i, p, p, p, p, p]
    lib.qnep_snes_sample.restype = i
    lib.qnep_batch_loss.argtypes = [i, i, p, i, p, p, p, p, p, i, ctypes.POINTER(LossWeightsC), p, p, p]
    lib.qnep_batch_loss.restype = i
    lib.qnep_snes_update.argtypes = [i, i, p, p, p, p, ctypes.c_double, ctypes.c_double, p]
    lib.qnep_snes_update.restype = i
    lib.qnep_batch_destroy.argtypes = [p]
    lib.qnep_batch_destroy.restype = None
    return lib


def load(path: str = LIB_PATH):
    """Open libqnep.so (built by ``paper_2601_19034_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libqnep.so not built ({path}); run __graft_entry__.build()")
            _lib = _declare(ctypes.CDLL(path))
        return _lib


class QnepError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        lib = load()
        super().__init__(f"{lib.qnep_status_string(status).decode()} ({status}): {detail}")
        self.status = status


def check(status: int, model=None, batch=None):
    if status != QNEP_OK:
        lib = load()
        if batch:
            detail = lib.qnep_batch_last_error(batch).decode()
        else:
            detail = lib.qnep_last_error(model).decode() if model else ""
        raise QnepError(status, detail)
