"""Pins of the oracle's velocity-Verlet integrator (oracle/md.py), independent of the GPU path.

* One atom in an isotropic harmonic well U = k |x|^2 / 2: the velocity-Verlet map is linear and
  has the closed-form solution x_n = x_0 cos(n theta) + D sin(n theta), cos theta = 1 - (omega h)^2
  / 2, D = h v_0 / sin theta, with v_n = (x_{n+1} - x_{n-1}) / 2h.  At omega h = 1.2 the phase per
  step theta = 1.287 differs from omega h by 7 %, so any other update (a dropped 1/2, the old
  forces in the velocity half-step, symplectic Euler) leaves the closed form at once.
* Time reversibility on a Morse cluster: n steps forward, the velocities reversed, n steps more
  give back the start to rounding.
* Second order: the total-energy error of the Morse cluster over the same time falls by ~4 when h
  is halved.
* Units: the (eV/A)/amu -> A/fs^2 and amu A^2/fs^2 -> eV conversions are inverse to each other
  (energy = force x length), an atom of 1 amu with 1 eV of kinetic energy moves at 13.89 km/s,
  and the CUDA integrator's own FP32 constant equals the SI-derived one to FP32 rounding.
"""
import math
import os
import re

import numpy as np
import pytest

from oracle import md

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _well(k):
    def forces_of(x):
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        return 0.5 * k * float((x * x).sum()), -k * x
    return forces_of


@pytest.mark.parametrize("omega_h", [0.05, 1.2])
def test_harmonic_well_follows_the_closed_form_of_the_map(omega_h):
    k, m = 2.5, np.array([12.0])                    # eV/A^2, amu
    omega = math.sqrt(k * md.ACC_UNIT / m[0])       # 1/fs
    h = omega_h / omega
    rng = np.random.default_rng(1)
    x0, v0 = rng.normal(0.0, 0.3, (1, 3)), rng.normal(0.0, 0.01, (1, 3))
    theta = math.acos(1.0 - 0.5 * omega_h ** 2)
    d = h * v0 / math.sin(theta)
    forces_of = _well(k)
    x, v = x0.copy(), v0.copy()
    _, f = forces_of(x)
    scale = float(np.abs(x0).max() + np.abs(d).max())
    for n in range(1, 301):
        x, v, f, _ = md.step(x, v, f, m, h, forces_of)
        xn = x0 * math.cos(n * theta) + d * math.sin(n * theta)
        vn = (math.sin(theta) / h) * (d * math.cos(n * theta) - x0 * math.sin(n * theta))
        np.testing.assert_allclose(x, xn, atol=1e-11 * scale * n)
        np.testing.assert_allclose(v, vn, atol=1e-11 * scale * n * math.sin(theta) / h)


def test_run_records_the_initial_state_and_every_step():
    k, m, h = 2.5, np.array([12.0]), 0.5
    forces_of = _well(k)
    x0, v0 = np.array([[0.2, -0.1, 0.05]]), np.array([[0.001, 0.002, -0.003]])
    x, v, f, e = md.run(x0, v0, m, h, 7, forces_of)
    assert e.shape == (8, 2)
    assert e[0, 0] == pytest.approx(0.5 * k * (x0 ** 2).sum(), rel=1e-15)
    assert e[0, 1] == pytest.approx(md.kinetic_energy(v0, m), rel=1e-15)
    xs, vs = x0, v0
    _, fs = forces_of(xs)
    for _ in range(7):
        xs, vs, fs, us = md.step(xs, vs, fs, m, h, forces_of)
    np.testing.assert_array_equal(x, xs)
    np.testing.assert_array_equal(v, vs)
    assert e[7, 0] == us and e[7, 1] == md.kinetic_energy(vs, m)


def _morse_cluster(n=8, seed=3):
    rng = np.random.default_rng(seed)
    grid = np.stack(np.meshgrid(*[np.arange(2)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n] * 2.6
    x0 = grid + rng.normal(0.0, 0.05, grid.shape)
    masses = rng.uniform(1.0, 16.0, n)
    v0 = rng.normal(0.0, 0.01, (n, 3))
    de, a, r0 = 0.4, 1.3, 2.5                        # eV, 1/A, A

    def forces_of(x):
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        d = x[:, None, :] - x[None, :, :]
        r = np.sqrt((d * d).sum(-1) + np.eye(len(x)))
        e = np.exp(-a * (r - r0))
        u = de * (1.0 - e) ** 2 - de
        np.fill_diagonal(u, 0.0)
        dudr = 2.0 * de * a * e * (1.0 - e)
        np.fill_diagonal(dudr, 0.0)
        f = -((dudr / r)[:, :, None] * d).sum(1)
        return 0.5 * float(u.sum()), f
    return x0, v0, masses, forces_of


def test_reversing_the_velocities_retraces_the_trajectory():
    x0, v0, m, forces_of = _morse_cluster()
    x, v, _, _ = md.run(x0, v0, m, 1.0, 200, forces_of)
    assert np.abs(x - x0).max() > 0.1                # the cluster has moved
    xb, vb, _, _ = md.run(x, -v, m, 1.0, 200, forces_of)
    np.testing.assert_allclose(xb, x0, atol=1e-9)
    np.testing.assert_allclose(-vb, v0, atol=1e-11)


def test_energy_error_is_second_order_in_the_step():
    x0, v0, m, forces_of = _morse_cluster()
    errs = []
    for h in (1.0, 0.5, 0.25):
        _, _, _, e = md.run(x0, v0, m, h, int(round(100.0 / h)), forces_of)
        etot = e.sum(1)
        errs.append(np.abs(etot - etot[0]).max())
    for coarse, fine in zip(errs, errs[1:]):
        assert 3.3 < coarse / fine < 4.7, errs


def test_unit_conversions():
    assert md.ACC_UNIT * md.KE_UNIT == pytest.approx(1.0, rel=1e-15)
    # 1 eV of kinetic energy on 1 amu: v = sqrt(2 x 1.602176634e-19 J / 1.66053906660e-27 kg) = 13.891 km/s
    v = math.sqrt(2.0 / md.KE_UNIT)                  # A/fs
    assert v * 1e5 == pytest.approx(13891.0, rel=1e-4)
    assert md.kinetic_energy(np.array([[v, 0.0, 0.0]]), np.array([1.0])) == pytest.approx(1.0, rel=1e-14)


def test_cuda_integrator_constant_equals_the_si_value():
    """The CUDA integrator writes its conversion as an FP32 literal; it is the SI-derived value to
    FP32 rounding (the two are written separately, neither reads the other)."""
    src = open(os.path.join(ROOT, "paper_2601_19034_gb300", "csrc", "md.cu")).read()
    lit = float(re.search(r"constexpr float ACC_UNIT = ([0-9.eE+-]+)f;", src).group(1))
    assert lit == pytest.approx(md.ACC_UNIT, rel=2e-7)
