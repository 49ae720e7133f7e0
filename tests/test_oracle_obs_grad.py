"""Pins for observables and gradients: closed forms on product states and the
agreement of two independent derivative rules."""
import math

import numpy as np
import pytest

import circuits as C
from oracle import gradients as GR
from oracle import observables as O
from oracle import statevector as S


def test_tfim_on_basis_and_plus_states():
    n = 6
    obs = C.tfim(n)
    assert abs(O.expval(C.zero_state(n), obs) - (n - 1)) < 1e-14
    plus = np.full(1 << n, 1 / math.sqrt(1 << n), dtype=complex)
    assert abs(O.expval(plus, obs) - 0.7 * n) < 1e-13


def _product_layer(n, ty, tz):
    gates = [C.Gate("RY", (q,), q) for q in range(n)] + [C.Gate("RZ", (q,), n + q) for q in range(n)]
    return C.Circuit(n, gates, 2 * n)


def test_product_state_closed_forms():
    n = 4
    rng = np.random.default_rng(1)
    ty, tz = rng.uniform(-3, 3, n), rng.uniform(-3, 3, n)
    c = _product_layer(n, ty, tz)
    params = np.concatenate([ty, tz])
    psi = S.simulate(c, params)
    for q in range(n):
        z = ["I"] * n
        z[q] = "Z"
        x = ["I"] * n
        x[q] = "X"
        assert abs(O.expval(psi, C.Observable(n, [(1.0, "".join(z))])) - math.cos(ty[q])) < 1e-13
        assert abs(O.expval(psi, C.Observable(n, [(1.0, "".join(x))])) - math.sin(ty[q]) * math.cos(tz[q])) < 1e-13
    # <sum X_q>: analytic gradient
    obs = C.Observable(n, [(1.0, "".join("X" if k == q else "I" for k in range(n))) for q in range(n)])
    g_ana = np.concatenate([np.cos(ty) * np.cos(tz), -np.sin(ty) * np.sin(tz)])
    g_ps = GR.parameter_shift(c, params, obs)
    g_fd = GR.finite_difference(c, params, obs)
    assert np.abs(g_ps - g_ana).max() < 1e-12
    assert np.abs(g_fd - g_ana).max() < 1e-8


def test_shift_and_fd_agree_on_hea():
    c = C.hea(4, 2)
    p = C.hea_params(c.n_params, 7)
    obs = C.tfim(4)
    g_ps = GR.parameter_shift(c, p, obs)
    g_fd = GR.finite_difference(c, p, obs)
    assert np.linalg.norm(g_ps - g_fd) <= 1e-8 * np.linalg.norm(g_ps)


def test_pauli_y_and_mixed_terms():
    # <Y> on RX(t)|0> = -sin t ; <Z Z> on a Bell state = 1 ; <X X> on a Bell state = 1
    t = 0.9
    c = C.Circuit(1, [C.Gate("RX", (0,), -1, (t,))])
    psi = S.simulate(c)
    assert abs(O.expval(psi, C.Observable(1, [(1.0, "Y")])) + math.sin(t)) < 1e-14
    bell = S.simulate(C.ghz(2))
    assert abs(O.expval(bell, C.Observable(2, [(1.0, "ZZ")])) - 1) < 1e-14
    assert abs(O.expval(bell, C.Observable(2, [(1.0, "XX")])) - 1) < 1e-14
    assert abs(O.expval(bell, C.Observable(2, [(1.0, "YY")])) + 1) < 1e-14
