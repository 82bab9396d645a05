"""The C-ABI library loads and exports every entry point declared in include/qnep.h.

CPU only: no call touches a GPU (qnep_param_count and qnep_status_string are
pure host functions).
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2601_19034_gb300 import _lib
from paper_2601_19034_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "qnep.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qnep_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert "qnep_compute" in names and "qnep_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_param_count_matches_documented_layout(lib):
    for s in (1, 2, 3, 4):
        hp = wl.HParams(n_species=s)
        c = _lib.HParamsC(hp.n_species, hp.rc_radial, hp.rc_angular, hp.n_radial, hp.n_angular,
                          hp.basis_radial, hp.basis_angular, hp.l_max, hp.use_4body, hp.n_neurons)
        assert lib.qnep_param_count(ctypes.byref(c)) == hp.n_params


def test_status_strings(lib):
    for code in range(7):
        assert lib.qnep_status_string(code)
    assert lib.qnep_status_string(_lib.QNEP_ERR_NBR_OVERFLOW).decode() == "neighbour list overflow"


def test_struct_layouts_match_header():
    # qnep_elec: int, int, double x3, int[3], int, double -> 56 bytes with natural alignment
    assert ctypes.sizeof(_lib.ElecC) == 56
    assert ctypes.sizeof(_lib.HParamsC) == 40
    assert ctypes.sizeof(_lib.OutputsC) == 72
    assert ctypes.sizeof(_lib.BatchOutputsC) == 56      # seven pointers
    assert ctypes.sizeof(_lib.LossInputsC) == 40        # five pointers
    assert ctypes.sizeof(_lib.LossWeightsFullC) == 56   # seven doubles


def test_full_loss_rejects_unpaired_buffers_before_any_gpu_work(lib):
    """qnep_batch_loss_full: each output comes with its reference, BEC with its structure mask."""
    dummy = ctypes.c_void_p(0x1000)       # never dereferenced: every call below returns before using it
    fn = lib.qnep_batch_loss_full
    w = _lib.LossWeightsFullC(1, 1, 1, 1, 1, 0, 0)
    full = _lib.LossInputsC(dummy, dummy, dummy, dummy, dummy)
    for k in ("forces", "virial", "bec", "total_charge"):
        half = _lib.LossInputsC(dummy, dummy, dummy, dummy, dummy)
        setattr(half, k, None)
        assert fn(2, 1, dummy, 4, full, half, dummy, None, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG, k
        assert fn(2, 1, dummy, 4, half, full, dummy, None, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG, k
    assert fn(2, 1, dummy, 4, full, full, None, None, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG   # no mask
    no_energy = _lib.LossInputsC(None, dummy, dummy, dummy, dummy)
    assert fn(2, 1, dummy, 4, no_energy, full, dummy, None, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    bad = _lib.LossWeightsFullC(1, 1, 1, float("nan"), 1, 0, 0)
    assert fn(2, 1, dummy, 4, full, full, dummy, None, 0, bad, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    assert fn(0, 1, dummy, 4, full, full, dummy, None, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    assert fn(2, 1, dummy, 4, None, full, dummy, None, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG


def test_static_geometry_switch_rejects_bad_arguments(lib):
    """qnep_batch_set_static_geometry / qnep_batch_geometry_changed refuse a NULL batch (host-only
    checks, no CUDA call; the enable flag's range needs a batch, so a device)."""
    assert lib.qnep_batch_set_static_geometry(None, 1) == _lib.QNEP_ERR_ARG
    assert lib.qnep_batch_geometry_changed(None) == _lib.QNEP_ERR_ARG


def test_new_entry_points_reject_bad_arguments_before_any_gpu_work(lib):
    """Host-side checks of the field-response and training entry points (no CUDA call is reached)."""
    dummy = ctypes.c_void_p(0x1000)       # never dereferenced: every call below returns before using it
    e = (ctypes.c_double * 3)(0.1, 0.0, 0.0)
    nan_e = (ctypes.c_double * 3)(float("nan"), 0.0, 0.0)
    fr = lib.qnep_field_response
    assert fr(-1, dummy, e, dummy, dummy, 0, dummy, None) == _lib.QNEP_ERR_ARG
    assert fr(4, dummy, None, None, dummy, 0, None, None) == _lib.QNEP_ERR_ARG       # forces without a field
    assert fr(4, dummy, e, None, None, 0, dummy, None) == _lib.QNEP_ERR_ARG          # Pdot without velocities
    assert fr(4, None, e, None, dummy, 0, None, None) == _lib.QNEP_ERR_ARG           # no Z
    assert fr(4, dummy, nan_e, None, dummy, 0, None, None) == _lib.QNEP_ERR_ARG      # non-finite field
    assert fr(4, ctypes.c_void_p(0x1002), e, None, dummy, 0, None, None) == _lib.QNEP_ERR_ARG   # misaligned
    assert fr(4, dummy, e, None, dummy, 3, None, None) == _lib.QNEP_ERR_ARG          # accumulate flag
    assert fr(4, dummy, None, None, None, 0, None, None) == _lib.QNEP_OK             # nothing asked: no work
    assert lib.qnep_snes_sample(0, 5, dummy, dummy, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    assert lib.qnep_snes_sample(3, 5, None, dummy, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    assert lib.qnep_snes_update(1025, 5, dummy, dummy, dummy, dummy, -1.0, -1.0, None) == _lib.QNEP_ERR_ARG
    assert lib.qnep_snes_update(4, 5, dummy, dummy, dummy, dummy, float("inf"), -1.0, None) == _lib.QNEP_ERR_ARG
    w = _lib.LossWeightsC(1.0, 1.0, 0.0, 0.0)
    bad = _lib.LossWeightsC(1.0, float("nan"), 0.0, 0.0)
    bl = lib.qnep_batch_loss
    assert bl(0, 1, dummy, 4, dummy, dummy, dummy, dummy, None, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    assert bl(2, 1, dummy, 4, dummy, dummy, dummy, None, None, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    assert bl(2, 1, dummy, 4, dummy, None, dummy, None, dummy, 0, w, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    assert bl(2, 1, dummy, 4, dummy, None, dummy, None, None, 0, bad, dummy, dummy, None) == _lib.QNEP_ERR_ARG
    assert lib.qnep_batch_set_params(None, dummy, None) == _lib.QNEP_ERR_ARG
    assert lib.qnep_nve_run_field(None, 4, dummy, dummy, dummy, dummy, dummy, 0.5, 1, e, None, dummy, dummy,
                                  dummy, dummy) == _lib.QNEP_ERR_ARG


def test_device_status_bits_decode(lib):
    """The status word the kernels write maps to the documented codes (bit 1: a bounded wait gave up)."""
    f = lib.qnep_status_from_device_bits        # argument types declared by the binding
    assert f(0) == _lib.QNEP_OK
    assert f(1) == _lib.QNEP_ERR_NBR_OVERFLOW
    assert f(2) == _lib.QNEP_ERR_TIMEOUT
    assert f(4) == _lib.QNEP_ERR_ARG
    assert f(3) == _lib.QNEP_ERR_NBR_OVERFLOW     # precedence: species, overflow, timeout
    assert f(6) == _lib.QNEP_ERR_ARG
    assert f(8) == _lib.QNEP_OK                    # undefined bits are ignored


def test_noalloc_refuses_oversized_k_set_before_any_gpu_work(lib):
    """A huge k_max * L is refused from the arguments alone (no enumeration, no CUDA call)."""
    fn = lib.qnep_ewald_kspace_noalloc    # argument types declared by the binding
    dummy = ctypes.c_void_p(0x1000)       # never dereferenced: every call below returns before using it
    box = (ctypes.c_double * 9)(10.0, 0, 0, 0, 10.0, 0, 0, 0, 10.0)
    err = ctypes.create_string_buffer(256)
    for kmax in (1e3, 1e12, 1e300):
        assert fn(16, dummy, dummy, box, 0.3, kmax, None, None, None, None, err, len(err)) == _lib.QNEP_ERR_UNSUPPORTED
        assert b"QNEP_NOALLOC_MAX_PHASE" in err.value
    # n_max = 40 per axis: 41 + 81 + 88 = 210 phase factors > 128
    assert fn(16, dummy, dummy, box, 0.3, 2 * np.pi * 40.5 / 10.0, None, None, None, None, err,
              len(err)) == _lib.QNEP_ERR_UNSUPPORTED
    assert fn(16, dummy, dummy, box, 0.3, float("inf"), None, None, None, None, err, len(err)) == _lib.QNEP_ERR_ARG
    assert fn(8193, dummy, dummy, box, 0.3, 2.0, None, None, None, None, err, len(err)) == _lib.QNEP_ERR_UNSUPPORTED


def _header_constants():
    """Every integer constant the header defines: enum entries and #defines (comments removed)."""
    text = open(os.path.join(ROOT, "include", "qnep.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    vals = {k: int(v) for k, v in re.findall(r"\b(QNEP_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    vals.update({k: int(v) for k, v in re.findall(r"#define\s+(QNEP_[A-Z0-9_]+)\s+(\d+)\s*$", text, flags=re.M)})
    return vals


def test_binding_constants_match_the_header():
    """The status codes, option codes and sizes the Python binding passes are the header's values, and
    the named scalars it reads back sit at the header's indices."""
    hc = _header_constants()
    names = [n for n in dir(_lib) if n.startswith("QNEP_")]
    assert len(names) >= 20
    for n in names:
        assert n in hc, n
        assert getattr(_lib, n) == hc[n], n
    s = _lib.SCALAR_NAMES
    assert s["energy"] == hc["QNEP_S_ENERGY"] and s["e_nep"] == hc["QNEP_S_E_NEP"]
    assert s["e_real"] == hc["QNEP_S_E_REAL"] and s["e_kspace"] == hc["QNEP_S_E_KSPACE"]
    assert s["e_self"] == hc["QNEP_S_E_SELF"] and s["qtilde_sum"] == hc["QNEP_S_QTILDE_SUM"]
    assert s["phi_mean"] == hc["QNEP_S_PHI_MEAN"] and s["status"] == hc["QNEP_S_STATUS"]
    assert s["virial"] == slice(hc["QNEP_S_VIRIAL"], hc["QNEP_S_VIRIAL"] + 9)
    assert s["polarization"] == slice(hc["QNEP_S_POLARIZATION"], hc["QNEP_S_POLARIZATION"] + 3)
    assert hc["QNEP_NSCALARS"] == hc["QNEP_S_STATUS"] + 1


def test_parse_scalars_and_stack_structures_on_the_host():
    """Host helpers of the binding: the scalar vector split into named values (virial row-major),
    and ragged structures (an empty one among them) stacked with their offsets and boxes."""
    from paper_2601_19034_gb300.qnep import parse_scalars, stack_structures
    v = np.arange(_lib.QNEP_NSCALARS, dtype=np.float64) * 0.5
    sc = parse_scalars(v)
    assert sc["energy"] == 0.0 and sc["e_kspace"] == 1.5 and sc["status"] == 9.5
    np.testing.assert_array_equal(sc["virial"], (np.arange(5, 14) * 0.5).reshape(3, 3))
    np.testing.assert_array_equal(sc["polarization"], np.arange(14, 17) * 0.5)
    rng = np.random.default_rng(3)
    systems = []
    for n, edge in ((5, 9.0), (0, 10.0), (3, 11.0)):
        box = np.diag([edge, edge + 1.0, edge + 2.0])
        box[1, 0] = 0.5
        systems.append(wl.System(rng.uniform(0, edge, (n, 3)).astype(np.float32),
                                 rng.integers(0, 2, n).astype(np.int32), box, ("H", "O")))
    pos, typ, off, boxes = stack_structures(systems)
    assert off.tolist() == [0, 5, 5, 8] and off.dtype == np.int32
    assert pos.shape == (8, 3) and pos.dtype == np.float32 and typ.dtype == np.int32
    np.testing.assert_array_equal(pos[5:], systems[2].positions)
    np.testing.assert_array_equal(typ[:5], systems[0].types)
    assert boxes.shape == (3, 3, 3) and boxes.dtype == np.float64
    np.testing.assert_array_equal(boxes[1], systems[1].box)


def _prototypes():
    """name -> (return type, [parameter declarations]) of every function the header declares."""
    text = open(os.path.join(ROOT, "include", "qnep.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"#[^\n]*", "", text)
    out = {}
    for m in re.finditer(r"([A-Za-z_][A-Za-z0-9_ \*]*?)\b(qnep_[a-z_]+)\s*\(([^()]*)\)\s*;", text):
        ret, name, params = " ".join(m.group(1).split()), m.group(2), " ".join(m.group(3).split())
        plist = [] if params in ("", "void") else [x.strip() for x in params.split(",")]
        out[name] = (ret.split("}")[-1].strip(), plist)
    return out


def _kind_of_c(decl):
    if "*" in decl or "[" in decl:
        return "ptr"
    words = decl.replace("const ", "").split()
    t = " ".join(words[:-1]) if len(words) > 1 else words[0]
    return {"int": "int", "unsigned int": "uint", "size_t": "size", "double": "double", "float": "float",
            "qnep_status": "int"}[t]


def _kind_of_ctypes(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_uint: "uint", ctypes.c_size_t: "size", ctypes.c_double: "double",
            ctypes.c_float: "float"}[t]


def test_binding_signatures_match_the_header(lib):
    """Every entry point the header declares has ctypes argument types in the binding (without them a
    device pointer would be passed as a 32-bit int), with the header's count of arguments, and each
    argument and the result of the header's kind: pointer, int, unsigned, size_t, double or float."""
    protos = _prototypes()
    assert set(protos) == set(_declared_symbols())
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, f"{name}: no argtypes"
        assert len(fn.argtypes) == len(params), name
        for k, (decl, t) in enumerate(zip(params, fn.argtypes)):
            assert _kind_of_ctypes(t) == _kind_of_c(decl), f"{name} argument {k}: {decl}"
        want = "void" if ret == "void" else ("ptr" if "*" in ret else _kind_of_c(ret + " r"))
        assert _kind_of_ctypes(fn.restype) == want, f"{name} result: {ret}"


STRUCTS = {"qnep_hparams": "HParamsC", "qnep_elec": "ElecC", "qnep_outputs": "OutputsC", "qnep_vjp": "VjpC",
           "qnep_batch_outputs": "BatchOutputsC", "qnep_loss_weights": "LossWeightsC",
           "qnep_loss_weights_v": "LossWeightsVC", "qnep_loss_inputs": "LossInputsC",
           "qnep_loss_weights_full": "LossWeightsFullC"}


def test_struct_fields_match_the_compiled_header(tmp_path):
    """Every struct the header declares, compiled by the C compiler: the binding's ctypes structure
    has the same fields (a missing name does not compile) at the same offsets with the same sizes,
    and the same total size."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    text = open(os.path.join(ROOT, "include", "qnep.h")).read()
    assert set(re.findall(r"\}\s*(qnep_[a-z_]+)\s*;", text)) - {"qnep_status"} == set(STRUCTS)
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qnep.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in getattr(_lib, pyname)._fields_:
            lines.append(f'    printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f'sizeof((({cname}*)0)->{fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    rows = [ln.split() for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                                                text=True).stdout.splitlines()]
    c = {}
    for r in rows:
        if r[1] == "size":
            c[(r[0], None)] = (int(r[2]),)
        else:
            c[(r[0], r[1])] = (int(r[2]), int(r[3]))
    for cname, pyname in STRUCTS.items():
        cls = getattr(_lib, pyname)
        assert ctypes.sizeof(cls) == c[(cname, None)][0], cname
        for fname, _ in cls._fields_:
            f = getattr(cls, fname)
            assert (f.offset, f.size) == c[(cname, fname)], f"{cname}.{fname}"


def test_missing_library_fails_loudly_and_the_package_never_imports_the_oracle():
    """The product path has no fallback: opening a library that is not there raises (in a fresh
    interpreter, as the binding caches the open library), and no module of the package imports the
    FP64 oracle."""
    import subprocess
    import sys
    code = ("from paper_2601_19034_gb300 import _lib\n"
            "try:\n"
            "    _lib.load('/nonexistent/libqnep.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "raised: libqnep.so not built" in r.stdout, r.stdout + r.stderr
    pkg = os.path.join(ROOT, "paper_2601_19034_gb300")
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, name)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, flags=re.M), name
