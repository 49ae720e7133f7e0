"""Reference gradients of f(theta) = <psi(theta)|H|psi(theta)>.

* central finite differences, step h = 1e-5;
* the parameter-shift rule [f(theta + pi/2) - f(theta - pi/2)] / 2, exact for
  RX/RY/RZ rotations exp(-i theta P / 2) whose parameter feeds one gate.
"""
import math

import numpy as np

from .observables import expval
from .statevector import simulate


def energy(circuit, params, obs, psi0=None):
    return expval(simulate(circuit, params, psi0), obs)


def finite_difference(circuit, params, obs, h=1e-5, psi0=None):
    params = np.asarray(params, dtype=np.float64)
    g = np.zeros_like(params)
    for k in range(len(params)):
        p = params.copy()
        p[k] += h
        fp = energy(circuit, p, obs, psi0)
        p[k] -= 2 * h
        fm = energy(circuit, p, obs, psi0)
        g[k] = (fp - fm) / (2 * h)
    return g


def parameter_shift(circuit, params, obs, psi0=None):
    params = np.asarray(params, dtype=np.float64)
    users = {}
    for gt in circuit.gates:
        if gt.param >= 0:
            users.setdefault(gt.param, []).append(gt.kind)
    for k, kinds in users.items():
        if len(kinds) != 1 or kinds[0] not in ("RX", "RY", "RZ"):
            raise ValueError("parameter shift needs one RX/RY/RZ gate per parameter")
    g = np.zeros_like(params)
    for k in range(len(params)):
        p = params.copy()
        p[k] += math.pi / 2
        fp = energy(circuit, p, obs, psi0)
        p[k] -= math.pi
        fm = energy(circuit, p, obs, psi0)
        g[k] = 0.5 * (fp - fm)
    return g
