"""Host logic of the Ewald path on the CPU: the half-space k-set the kernels use (csrc/kset_host.h).

The header is compiled into a small host program (g++; CUDA headers only for the vector
types) that prints every real wave vector of the set with its G(k).  Against the oracle's
full-sphere enumeration (oracle/ewald.py, written separately): the set is exactly one of
each +-k pair with 0 < |k| < k_max, every G(k) = (2 pi / V) exp(-k^2 / 4 alpha^2) / k^2 to
FP32 rounding, the padding entries carry G = 0, and the columns hold contiguous n3 runs.
"""
import math
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import ewald

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include "kset_host.h"
int main(int argc, char** argv) {
    double L[3] = {atof(argv[1]), atof(argv[2]), atof(argv[3])};
    qnep::KSet ks = qnep::build_kset(L, atof(argv[4]), atof(argv[5]));
    int ncol = (int)ks.cols.size() - 1;
    printf("%d %d %d %zu %zu\n", ncol, (int)ks.chunk_col.size(), (int)ks.cols[ncol].w, ks.kg.size(), ks.chunk_col.size());
    for (int c = 0; c < ncol; ++c) {
        int4 col = ks.cols[c];
        int len = ks.cols[c + 1].w - col.w;
        for (int t = 0; t < len; ++t) printf("%d %d %d %d %.9e\n", c, col.x, col.y, col.z + t, ks.kg[col.w + t]);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are not available")
    d = tmp_path_factory.mktemp("kset")
    src = d / "kset_main.cpp"
    src.write_text(HARNESS)
    exe = d / "kset_main"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2601_19034_gb300", "csrc"),
                    "-I", CUDA_INC, str(src), "-o", str(exe)], check=True, capture_output=True)
    return str(exe)


def _run(exe, lengths, kmax, alpha):
    out = subprocess.run([exe, *[repr(float(x)) for x in lengths], repr(kmax), repr(alpha)], check=True,
                         capture_output=True, text=True).stdout.split("\n")
    head = [int(x) for x in out[0].split()]
    rows = np.array([[float(x) for x in ln.split()] for ln in out[1:] if ln.strip()])
    return head, rows


@pytest.mark.parametrize("lengths", [(12.42, 12.42, 12.42), (40.0, 40.0, 40.0), (12.97, 25.94, 12.97),
                                     (20.3, 31.7, 100.5), (8.0, 8.0, 8.0)])
def test_half_space_kset_matches_the_oracle(harness, lengths):
    alpha = 0.3
    kmax = 2.0 * alpha * math.sqrt(math.log(1e6))
    head, rows = _run(harness, lengths, kmax, alpha)
    ncol, nchunk, nk_padded = head[0], head[1], head[2]
    assert nk_padded == 8 * nchunk and len(rows) == nk_padded
    real = rows[rows[:, 4] > 0]
    n = real[:, 1:4].astype(np.int64)
    full = ewald.kspace_integers(np.diag(lengths), kmax)
    # exactly one of each +-k pair
    assert 2 * len(n) == len(full)
    half = {tuple(v) for v in n}
    assert len(half) == len(n)
    for v in map(tuple, full):
        assert (v in half) != (tuple(-x for x in v) in half)
    # G(k) to FP32 rounding
    k = 2 * math.pi * n / np.asarray(lengths)
    k2 = (k * k).sum(1)
    g = (2 * math.pi / np.prod(lengths)) * np.exp(-k2 / (4 * alpha * alpha)) / k2
    np.testing.assert_allclose(real[:, 4], g, rtol=2e-7)
    # padding carries G = 0 and lies outside the sphere or past the column's run
    pad = rows[rows[:, 4] == 0]
    kp = 2 * math.pi * pad[:, 1:4] / np.asarray(lengths)
    inside = ((kp * kp).sum(1) < kmax * kmax) & ((kp * kp).sum(1) > 0)
    for (c, n1, n2, n3, _), ins in zip(pad, inside):
        if ins:   # a padded slot inside the sphere must be past the column's last real n3
            col = real[real[:, 0] == c]
            assert n3 > col[:, 3].max()
    # each column's real entries are one contiguous run of n3
    for c in range(ncol):
        col = real[real[:, 0] == c][:, 3]
        assert len(col) and np.array_equal(col, np.arange(col.min(), col.max() + 1))


HARNESS_BOX = r"""
#include <cstdio>
#include <cstdlib>
#include "kset_host.h"
int main(int argc, char** argv) {
    double box[9];
    for (int k = 0; k < 9; ++k) box[k] = atof(argv[1 + k]);
    qnep::KSet ks = qnep::build_kset_box(box, atof(argv[10]), atof(argv[11]));
    int ncol = (int)ks.cols.size() - 1;
    printf("%d %d %d %zu %zu\n", ncol, (int)ks.chunk_col.size(), (int)ks.cols[ncol].w, ks.kg.size(), ks.chunk_col.size());
    for (int c = 0; c < ncol; ++c) {
        int4 col = ks.cols[c];
        int len = ks.cols[c + 1].w - col.w;
        for (int t = 0; t < len; ++t) printf("%d %d %d %d %.9e\n", c, col.x, col.y, col.z + t, ks.kg[col.w + t]);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness_box(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are not available")
    d = tmp_path_factory.mktemp("kset_box")
    src = d / "kset_box.cpp"
    src.write_text(HARNESS_BOX)
    exe = d / "kset_box"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2601_19034_gb300", "csrc"),
                    "-I", CUDA_INC, str(src), "-o", str(exe)], check=True, capture_output=True)
    return str(exe)


@pytest.mark.parametrize("box", [
    [[12.42, 0.62, -0.5], [2.48, 12.42, 0.75], [-1.24, 1.86, 12.42]],     # every off-diagonal non-zero
    [[12.97, 0.0, 0.0], [1.556, 12.97, 0.0], [-1.038, 1.297, 12.97]],     # the restricted form
    [[0.0, 2.82, 2.82], [2.82, 0.0, 2.82], [2.82, 2.82, 0.0]],           # fcc primitive cell
])
def test_half_space_kset_of_a_general_cell_matches_the_oracle(harness_box, box):
    """The k-set of a general cell (k = 2 pi H^-1 n, the tables of the sheared-cell Ewald paths)
    against the oracle's full-sphere enumeration: one of each +-k pair, G(k) with V = |det H| to
    FP32 rounding, padding with G = 0, contiguous n3 runs per column."""
    box = np.asarray(box, dtype=np.float64)
    alpha = 0.3
    kmax = 2.0 * alpha * math.sqrt(math.log(1e6))
    out = subprocess.run([harness_box, *[repr(float(x)) for x in box.ravel()], repr(kmax), repr(alpha)], check=True,
                         capture_output=True, text=True).stdout.split("\n")
    head = [int(x) for x in out[0].split()]
    rows = np.array([[float(x) for x in ln.split()] for ln in out[1:] if ln.strip()])
    ncol, nchunk, nk_padded = head[0], head[1], head[2]
    assert nk_padded == 8 * nchunk and len(rows) == nk_padded
    real = rows[rows[:, 4] > 0]
    n = real[:, 1:4].astype(np.int64)
    full = ewald.kspace_integers(box, kmax)
    assert 2 * len(n) == len(full)
    half = {tuple(v) for v in n}
    assert len(half) == len(n)
    for v in map(tuple, full):
        assert (v in half) != (tuple(-x for x in v) in half)
    k = 2 * math.pi * n @ np.linalg.inv(box).T
    k2 = (k * k).sum(1)
    g = (2 * math.pi / abs(np.linalg.det(box))) * np.exp(-k2 / (4 * alpha * alpha)) / k2
    np.testing.assert_allclose(real[:, 4], g, rtol=2e-7)
    for c in range(ncol):
        col = real[real[:, 0] == c][:, 3]
        assert len(col) and np.array_equal(col, np.arange(col.min(), col.max() + 1))


HARNESS_ROT = r"""
#include <cstdio>
#include <cstdlib>
#include "kset_host.h"
int main(int argc, char** argv) {
    double box[9], R[9], out[9];
    for (int k = 0; k < 9; ++k) box[k] = atof(argv[1 + k]);
    if (!qnep::rotate_to_restricted(box, R, out)) { printf("degenerate\n"); return 0; }
    for (int k = 0; k < 9; ++k) printf("%.17g ", R[k]);
    printf("\n");
    for (int k = 0; k < 9; ++k) printf("%.17g ", out[k]);
    printf("\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness_rot(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are not available")
    d = tmp_path_factory.mktemp("rot")
    src = d / "rot.cpp"
    src.write_text(HARNESS_ROT)
    exe = d / "rot"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2601_19034_gb300", "csrc"),
                    "-I", CUDA_INC, str(src), "-o", str(exe)], check=True, capture_output=True)
    return str(exe)


def _rotate(exe, box):
    out = subprocess.run([exe, *[repr(float(x)) for x in np.asarray(box).ravel()]], check=True,
                         capture_output=True, text=True).stdout.split("\n")
    if out[0].strip() == "degenerate":
        return None, None
    return (np.array([float(x) for x in out[0].split()]).reshape(3, 3),
            np.array([float(x) for x in out[1].split()]).reshape(3, 3))


def test_general_cell_rotation_into_the_restricted_form(harness_rot):
    """The batched call's turn of a general cell into the restricted form: R is a rotation
    (orthonormal, det +1), the turned rows are R a, R b, R c with a' along x and b' in the xy plane,
    so lengths, angles and the volume are kept; a left-handed cell comes out with c'_z < 0, and a
    cell with a parallel to b is reported as degenerate."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        box = np.diag(rng.uniform(8.0, 30.0, 3)) + rng.normal(0.0, 2.0, (3, 3))
        if np.linalg.det(box) < 0:
            box[2] = -box[2]
        r, turned = _rotate(harness_rot, box)
        np.testing.assert_allclose(r @ r.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(r) - 1.0) < 1e-13
        np.testing.assert_allclose(turned, box @ r.T, atol=1e-12 * np.abs(box).max())
        assert turned[0, 1] == 0.0 and turned[0, 2] == 0.0 and turned[1, 2] == 0.0
        assert turned[0, 0] > 0 and turned[1, 1] > 0 and turned[2, 2] > 0
        np.testing.assert_allclose(turned @ turned.T, box @ box.T, rtol=1e-12, atol=1e-10)
        assert abs(np.linalg.det(turned) - np.linalg.det(box)) < 1e-10 * abs(np.linalg.det(box))
    left = np.array([[20.0, 0.3, 0.2], [1.0, 20.0, 0.5], [0.4, 2.0, -20.0]])
    _, turned = _rotate(harness_rot, left)
    assert turned[2, 2] < 0
    r, turned = _rotate(harness_rot, np.array([[10.0, 1.0, 0.0], [20.0, 2.0, 0.0], [0.0, 0.0, 10.0]]))
    assert r is None


HARNESS_COUNT = r"""
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include "kset_host.h"
// argv: 9 box entries, k_max, alpha, build (1: also enumerate the set and count from its n_max)
int main(int argc, char** argv) {
    double box[9];
    for (int k = 0; k < 9; ++k) box[k] = atof(argv[1 + k]);
    const double kmax = atof(argv[10]), alpha = atof(argv[11]);
    const bool tri = box[1] != 0 || box[2] != 0 || box[3] != 0 || box[5] != 0 || box[6] != 0 || box[7] != 0;
    double len[3];
    for (int d = 0; d < 3; ++d) {
        const double* a = box + 3 * d;
        len[d] = tri ? std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) : box[4 * d];
    }
    const double pre = qnep::kset_phase_count(len, kmax);
    printf("%.17g\n", pre);
    if (atoi(argv[12])) {
        qnep::KSet ks = tri ? qnep::build_kset_box(box, kmax, alpha) : qnep::build_kset(len, kmax, alpha);
        printf("%d\n", (ks.nmax[0] + 1) + (2 * ks.nmax[1] + 1) + (2 * ks.nmax[2] + 8));
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness_count(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are not available")
    d = tmp_path_factory.mktemp("kset_count")
    src = d / "kset_count.cpp"
    src.write_text(HARNESS_COUNT)
    exe = d / "kset_count"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2601_19034_gb300", "csrc"),
                    "-I", CUDA_INC, str(src), "-o", str(exe)], check=True, capture_output=True)
    return str(exe)


def _count(exe, box, kmax, build):
    out = subprocess.run([exe, *[repr(float(x)) for x in np.asarray(box, dtype=np.float64).ravel()], repr(kmax),
                          "0.3", "1" if build else "0"], check=True, capture_output=True, text=True,
                         timeout=30).stdout.split()
    return float(out[0]), (int(out[1]) if build else None)


def test_phase_count_is_known_before_the_enumeration(harness_count):
    """The phase-factor count per atom that both force calls check against their shared-memory
    limits before they enumerate a k-set: equal to the count from the n_max the builders find, for
    orthorhombic and general cells, and over every limit (without an int overflow or a long loop)
    when k_max times an edge is huge or not finite."""
    alpha = 0.3
    kmax = 2.0 * alpha * math.sqrt(math.log(1e6))
    boxes = [np.diag([12.42, 12.42, 12.42]), np.diag([12.97, 25.94, 40.0]),
             [[12.42, 0.62, -0.5], [2.48, 12.42, 0.75], [-1.24, 1.86, 12.42]],
             [[12.97, 0.0, 0.0], [1.556, 12.97, 0.0], [-1.038, 1.297, 12.97]],
             [[0.0, 2.82, 2.82], [2.82, 0.0, 2.82], [2.82, 2.82, 0.0]]]
    for box in boxes:
        pre, built = _count(harness_count, box, kmax, True)
        assert pre == built
        # by hand: n_d = floor(k_max |a_d| / 2 pi)
        nd = [math.floor(kmax * np.linalg.norm(row) / (2 * math.pi)) for row in np.asarray(box, dtype=np.float64)]
        assert built == (nd[0] + 1) + (2 * nd[1] + 1) + (2 * nd[2] + 8)
    for kbig in (1e3, 1e12, 1e300, float("inf")):
        pre, _ = _count(harness_count, np.diag([10.0, 10.0, 10.0]), kbig, False)
        assert pre > 1e3


def test_documented_phase_limits_match_the_kernels():
    """The limits the C header states for the two Ewald force calls are the constants the host code
    checks against."""
    with open(os.path.join(ROOT, "include", "qnep.h")) as f:
        header = " ".join(" ".join(ln.strip().lstrip("*") for ln in f).split())   # comment text, one line
    csrc = os.path.join(ROOT, "paper_2601_19034_gb300", "csrc")
    with open(os.path.join(csrc, "batch_internal.cuh")) as f:
        batch = f.read()
    with open(os.path.join(csrc, "qnep_internal.cuh")) as f:
        single = f.read()
    nb = int(re.search(r"constexpr int BATCH_MAX_NPH = (\d+);", batch).group(1))
    ns = int(re.search(r"constexpr int EWALD_MAX_NPH = (\d+);", single).group(1))
    assert f"at most {nb} Ewald phase factors per atom" in header
    assert f"Ewald: at most {ns} phase factors per atom" in header
    assert ns % 2 == 1   # the single-structure rows are rounded up to an odd length
