"""The nested RK form with a source, as the library's sweeps run it, against Algorithms rk2 / rk4
as printed (Section 5.3; the oracle's rk2_step / rk4_step), on a linear system U' = B U + f(t)
with f(t) = Re(J e^{i w t}) (Eq. ode_system), no GPU.

The library evaluates every sweep in nested form, v_s = U + dt/s (B U + g_s) and v_k = U + dt/k
(B v_{k+1} + g_k) for k = s - 1, ..., 1, with the source combined per nested stage from its
values at t_m, t_m + dt/2, t_m + dt:

  RK4: g_4 = f1, g_3 = (f1 + f2) / 2, g_2 = (f1 + 2 f2) / 3, g_1 = (f1 + 4 f2 + f4) / 6
  RK2: g_2 = f1, g_1 = f2

For a linear system this is the printed RK polynomial exactly, so one step of either form
agrees to rounding, and the first nested stage evaluates Phi(t_m, U_m) = K_1 (what the Hermite
filter accumulates).  A wrong weight, offset or stage order fails these checks.
"""
import math

import numpy as np

from oracle.timestep import rk2_step, rk4_step

W4 = [(1.0, 0.0, 0.0), (0.5, 0.5, 0.0), (1.0 / 3.0, 2.0 / 3.0, 0.0), (1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0)]
W2 = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0)]
OFFSETS = (0.0, 0.5, 1.0)


def _system(seed, n=7):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(n, n)) - 2.0 * np.eye(n)
    J = rng.normal(size=n) + 1j * rng.normal(size=n)
    w = float(rng.uniform(1.0, 9.0))
    U = rng.normal(size=n)
    return B, J, w, U


def _nested_step(B, f, t, U, dt, s):
    W = W4 if s == 4 else W2
    v = U
    first = None
    for r in range(s):  # launch r is nested stage k = s - r
        g = sum(wj * f(t + oj * dt) for wj, oj in zip(W[r], OFFSETS) if wj != 0.0)
        phi = B @ v + g
        if r == 0:
            first = phi
        v = U + dt / (s - r) * phi
    return v, first


def test_nested_source_step_is_the_printed_rk_step():
    for seed in range(6):
        B, J, w, U = _system(seed)
        f = lambda t: np.real(J * np.exp(1j * w * t))
        phi = lambda t, X: B @ X + f(t)
        for s, step in ((4, rk4_step), (2, rk2_step)):
            for dt in (0.01, 0.05, 0.13):
                t = 0.37 * seed
                ref, K1 = step(phi, t, U, dt)
                got, first = _nested_step(B, f, t, U, dt, s)
                assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), (seed, s, dt)
                assert np.allclose(first, K1, rtol=0, atol=1e-13 * np.linalg.norm(K1))


def test_source_only_step_is_the_quadrature_of_the_printed_form():
    # B = 0: one RK4 step integrates f exactly like Simpson's rule, RK2 like the midpoint rule.
    rng = np.random.default_rng(9)
    J = rng.normal(size=3) + 1j * rng.normal(size=3)
    w, t, dt = 3.0, 0.2, 0.1
    f = lambda x: np.real(J * np.exp(1j * w * x))
    B = np.zeros((3, 3))
    U = np.zeros(3)
    got4, _ = _nested_step(B, f, t, U, dt, 4)
    simpson = dt / 6 * (f(t) + 4 * f(t + dt / 2) + f(t + dt))
    assert np.allclose(got4, simpson, rtol=0, atol=1e-15)
    got2, _ = _nested_step(B, f, t, U, dt, 2)
    assert np.allclose(got2, dt * f(t + dt / 2), rtol=0, atol=1e-15)


def test_a_wrong_weight_is_detected():
    B, J, w, U = _system(3)
    f = lambda t: np.real(J * np.exp(1j * w * t))
    phi = lambda t, X: B @ X + f(t)
    ref, _ = rk4_step(phi, 0.1, U, 0.1)
    global W4
    saved = W4
    try:
        W4 = [(1.0, 0.0, 0.0), (0.5, 0.5, 0.0), (0.5, 0.5, 0.0), (1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0)]
        bad, _ = _nested_step(B, f, 0.1, U, 0.1, 4)
    finally:
        W4 = saved
    assert np.linalg.norm(bad - ref) > 1e-8 * np.linalg.norm(ref)
    assert math.isfinite(float(np.linalg.norm(bad)))
