"""GPU parity of the batched form (sv_batch_create / sv_run_batch / sv_autotune):
many circuits of uneven width, E = <psi|O|psi> and the adjoint gradient in one
persistent launch replayed from a captured CUDA graph.

References: the CPU oracle (E from the gate-by-gate simulation; gradients by
parameter shift, exact for RX / RY / RZ) on small circuits, and the single-circuit
CUDA path (sv_grad, itself pinned to the oracle) on wide ones.  Tolerances: E within
1e-6 relative (max(|E|, 1)); gradients within 1e-4 relative (2-norm).
"""
import numpy as np
import pytest

import circuits as C
from oracle import gradients as GR
from oracle import observables as O
from oracle import statevector as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as ge
    ge.build()
    import paper_2509_14098_gb300 as pkg
    return pkg


def e_tol(e_ref):
    return 1e-6 * max(abs(e_ref), 1.0)


def grad_ok(g, g_ref):
    return np.linalg.norm(g - g_ref) <= 1e-4 * max(np.linalg.norm(g_ref), 1e-12)


def plain_grad(sv, circ, params, obs, L=10):
    plan = sv.Plan(circ, min(L, circ.n_qubits))
    st = sv.StateVector(circ.n_qubits)
    e, g = st.grad(plan, params, obs)
    st.close()
    return e, g


def mixed_circuit(n, seed):
    """Parametric RX / RY / RZ layers with fixed H, T, CZ, CP, SWAP, U3 in between."""
    rng = np.random.default_rng(seed)
    gates = []
    slot = 0
    for layer in range(3):
        for q in range(n):
            gates.append(C.Gate(["RX", "RY"][rng.integers(2)], (q,), slot))
            slot += 1
        for q in range(0, n - 1, 2):
            gates.append(C.Gate("CZ", (q, q + 1)))
        gates.append(C.Gate("H", (int(rng.integers(n)),)))
        gates.append(C.Gate("T", (int(rng.integers(n)),)))
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        gates.append(C.Gate("CP", (a, b), -1, (float(rng.uniform(-3, 3)),)))
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        gates.append(C.Gate("SWAP", (a, b)))
        gates.append(C.Gate("U3", (int(rng.integers(n)),), -1, tuple(float(x) for x in rng.uniform(-3, 3, 3))))
        for q in range(n):
            gates.append(C.Gate("RZ", (q,), slot))
            slot += 1
        for q in range(n - 1):
            gates.append(C.Gate("CX", (q, q + 1)))
    return C.Circuit(n, gates, slot)


def test_small_batch_vs_oracle(sv):
    """Whole-in-shared-memory circuits (n <= 13): E vs the oracle, gradients vs
    parameter shift on the oracle."""
    spec = C.batch_spec(12, seed=11, n_lo=7, n_hi=10, layers=3)
    circs = [c for c, _ in spec]
    obs = [C.zz_chain(c.n_qubits) for c in circs]
    params = np.concatenate([p for _, p in spec])
    b = sv.Batch(circs, obs)
    info = b.info()
    assert info["graph"] == 1 and info["n_resident"] == len(circs) and info["workspace_bytes"] == 0
    e, g = b.run(params)
    off = 0
    for i, (c, p) in enumerate(spec):
        psi = S.simulate(c, p)
        e_ref = O.expval(psi, obs[i])
        assert abs(e[i] - e_ref) <= e_tol(e_ref), (i, e[i], e_ref)
        gi = g[off: off + c.n_params]
        if i < 4:
            g_ref = GR.parameter_shift(c, p, obs[i])
            assert grad_ok(gi, g_ref), (i, np.linalg.norm(gi - g_ref), np.linalg.norm(g_ref))
        off += c.n_params


def test_structures_and_swaps_vs_oracle(sv):
    """Fixed gates between the parametric layers, SWAP relabels, several widths and
    tile widths (single- and multi-stage): E vs the oracle, gradient vs sv_grad."""
    circs = [mixed_circuit(n, 100 + n) for n in (7, 9, 11, 12, 14)]
    obs = [C.Observable(c.n_qubits, [(1.0, "Z" * 2 + "I" * (c.n_qubits - 2)),
                                      (0.5, "I" * (c.n_qubits - 1) + "Z"),
                                      (-0.25, "Z" + "I" * (c.n_qubits - 3) + "ZZ")]) for c in circs]
    rng = np.random.default_rng(5)
    ps = [rng.uniform(-np.pi, np.pi, c.n_params) for c in circs]
    for tune in (None, {11: (8, 2), 12: (9, 3), 14: (10, 4)}):
        b = sv.Batch(circs, obs, tune=tune)
        e, g = b.run(np.concatenate(ps))
        off = 0
        for i, c in enumerate(circs):
            e_ref = O.expval(S.simulate(c, ps[i]), obs[i])
            assert abs(e[i] - e_ref) <= e_tol(e_ref), (tune, i, e[i], e_ref)
            _, g_ref = plain_grad(sv, c, ps[i], obs[i])
            assert grad_ok(g[off: off + c.n_params], g_ref), (tune, i)
            off += c.n_params
        b.close()


def test_tiled_circuits_vs_plain_path(sv):
    """Wide circuits swept through HBM (several stages and tiles, fused last stage)."""
    spec = C.batch_spec(6, seed=12, n_lo=14, n_hi=17, layers=6)
    circs = [c for c, _ in spec]
    obs = [C.zz_chain(c.n_qubits) for c in circs]
    params = np.concatenate([p for _, p in spec])
    for tune in ({n: (10, 3) for n in range(14, 18)}, {n: (12, 4) for n in range(14, 18)}):
        b = sv.Batch(circs, obs, tune=tune)
        info = b.info()
        assert info["n_resident"] == 0 and info["workspace_bytes"] > 0   # wide groups or HBM-tiled circuits
        e, g = b.run(params)
        off = 0
        for i, (c, p) in enumerate(spec):
            e_ref, g_ref = plain_grad(sv, c, p, obs[i])
            assert abs(e[i] - e_ref) <= e_tol(e_ref), (i, e[i], e_ref)
            assert grad_ok(g[off: off + c.n_params], g_ref), i
            off += c.n_params
        b.close()
    # the widest oracle check: E at n = 14
    c, p = next((c, p) for c, p in spec if c.n_qubits == min(x.n_qubits for x in circs))
    e_ref = O.expval(S.simulate(c, p), C.zz_chain(c.n_qubits))
    b = sv.Batch([c], [C.zz_chain(c.n_qubits)], tune={c.n_qubits: (10, 3)})
    e, _ = b.run(p)
    assert abs(e[0] - e_ref) <= e_tol(e_ref)


def test_wide_groups_vs_oracle(sv):
    """Circuits of 14 and 15 qubits run as wide groups: every circuit of one structure
    sweeps each stage together in one generated kernel, each with its own parameters;
    mixed rotation kinds, fixed gates and SWAP relabels; a small circuit beside them in
    the persistent kernel.  E against the oracle, gradients against the oracle's
    parameter shift, on two replays with different parameters."""
    circs = [mixed_circuit(14, 41), mixed_circuit(14, 41), mixed_circuit(15, 42), mixed_circuit(14, 41),
             mixed_circuit(9, 43)]
    obs = [C.Observable(c.n_qubits, [(1.0, "Z" * 2 + "I" * (c.n_qubits - 2)),
                                      (0.5, "I" * (c.n_qubits - 1) + "Z"),
                                      (-0.25, "Z" + "I" * (c.n_qubits - 3) + "ZZ")]) for c in circs]
    b = sv.Batch(circs, obs)
    info = b.info()
    assert info["n_programs"] == 3          # two wide structures and the small circuit's
    rng = np.random.default_rng(8)
    for rep in range(2):
        ps = [rng.uniform(-np.pi, np.pi, c.n_params) for c in circs]
        e, g = b.run(np.concatenate(ps))
        off = 0
        for i, c in enumerate(circs):
            e_ref = O.expval(S.simulate(c, ps[i]), obs[i])
            assert abs(e[i] - e_ref) <= e_tol(e_ref), (rep, i, e[i], e_ref)
            if i in (1, 2, 4):
                g_ref = GR.parameter_shift(c, ps[i], obs[i])
                assert grad_ok(g[off: off + c.n_params], g_ref), (rep, i)
            off += c.n_params
    b.close()


def test_replay_and_autotune(sv):
    """The captured graph replays with new parameters; the autotuner returns a valid
    table and the rebuilt batch gives the same results."""
    spec = C.batch_spec(10, seed=13, n_lo=9, n_hi=15, layers=2)
    circs = [c for c, _ in spec]
    obs = [C.zz_chain(c.n_qubits) for c in circs]
    p1 = np.concatenate([p for _, p in spec])
    p2 = np.random.default_rng(3).uniform(-np.pi, np.pi, p1.size)
    b = sv.Batch(circs, obs)
    e1, g1 = b.run(p1)
    e2, g2 = b.run(p2)
    e1b, g1b = b.run(p1)
    assert np.array_equal(e1, e1b) and np.array_equal(g1, g1b)   # deterministic
    assert not np.allclose(e1, e2)
    table = b.autotune(p1)
    # circuits of 14 or more qubits run as wide groups (tile width 12, register width 4):
    # only the persistent kernel's widths are tuned
    widths = sorted({c.n_qubits for c in circs if c.n_qubits < 14})
    assert sorted(table) == widths
    for n, (L, k) in table.items():
        assert 2 <= k <= 4 and (L == n if n <= 13 else 11 <= L <= 13)
    e3, g3 = b.run(p2)
    off = 0
    for i, c in enumerate(circs):
        assert abs(e3[i] - e2[i]) <= e_tol(e2[i])
        assert grad_ok(g3[off: off + c.n_params], g2[off: off + c.n_params])
        off += c.n_params


def test_batch_errors(sv):
    c = C.hea(8, 1)
    with pytest.raises(sv.SvError) as ei:
        sv.Batch([c], [C.tfim(8, 0.7)])   # X terms: not a Z-string sum
    assert ei.value.status == 5
    with pytest.raises(sv.SvError) as ei:
        sv.Batch([C.hea(6, 1)], [C.zz_chain(6)])   # below the minimum width
    assert ei.value.status == 1
    pc = C.Circuit(8, [C.Gate("P", (0,), 0), C.Gate("H", (1,))], 1)
    with pytest.raises(sv.SvError) as ei:
        sv.Batch([pc], [C.zz_chain(8)])
    assert ei.value.status == 5
    b = sv.Batch([c], [C.zz_chain(8)])
    with pytest.raises(ValueError):
        b.run(np.zeros(3))


def test_full_size_batch_sampled(sv):
    """The 2048-circuit workload (n uniform in [10, 20], 6 layers, sum ZZ): sampled
    circuits against sv_grad and, for the narrow ones, against the oracle; every E
    within [-(n-1), n-1] and every gradient finite."""
    spec = C.batch_spec(2048, seed=5, n_lo=10, n_hi=20, layers=6)
    circs = [c for c, _ in spec]
    obs = [C.zz_chain(c.n_qubits) for c in circs]
    params = np.concatenate([p for _, p in spec])
    b = sv.Batch(circs, obs)
    e, g = b.run(params)
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(g))
    assert all(abs(e[i]) <= circs[i].n_qubits - 1 + 1e-5 for i in range(len(circs)))
    offs = np.concatenate([[0], np.cumsum([c.n_params for c in circs])])
    rng = np.random.default_rng(0)
    by_n = {}
    for i, c in enumerate(circs):
        by_n.setdefault(c.n_qubits, []).append(i)
    sample = [int(rng.choice(by_n[n])) for n in sorted(by_n)]
    for i in sample:
        c, p = spec[i]
        e_ref, g_ref = plain_grad(sv, c, p, obs[i], L=12)
        assert abs(e[i] - e_ref) <= e_tol(e_ref), (i, c.n_qubits)
        assert grad_ok(g[offs[i]: offs[i + 1]], g_ref), (i, c.n_qubits)
        if c.n_qubits <= 12:
            e_or = O.expval(S.simulate(c, p), obs[i])
            assert abs(e[i] - e_or) <= e_tol(e_or)


def test_autograd_functions(sv):
    """torch.autograd through the adjoint path: the plain form against parameter shift
    on the oracle, the batched form against the plain form."""
    import torch
    from paper_2509_14098_gb300 import autograd as AG
    c = C.hea(8, 2)
    obs = C.tfim(8, 0.7)
    p0 = C.hea_params(c.n_params, 21)
    plan = sv.Plan(c, 6)
    st = sv.StateVector(8)
    theta = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    e = AG.expval(st, plan, theta, obs)
    (g,) = torch.autograd.grad(3.0 * e, theta)
    e_ref = O.expval(S.simulate(c, p0), obs)
    g_ref = GR.parameter_shift(c, p0, obs)
    assert abs(e.item() - e_ref) <= e_tol(e_ref)
    assert grad_ok(g.numpy() / 3.0, g_ref)
    with torch.no_grad():
        assert abs(AG.expval(st, plan, theta.detach(), obs).item() - e_ref) <= e_tol(e_ref)
    # batched: weighted sum of the circuits' energies
    spec = C.batch_spec(5, seed=23, n_lo=8, n_hi=11, layers=2)
    circs = [x for x, _ in spec]
    zz = [C.zz_chain(x.n_qubits) for x in circs]
    b = sv.Batch(circs, zz)
    th = torch.tensor(np.concatenate([p for _, p in spec]), requires_grad=True)
    w = torch.arange(1.0, 6.0, dtype=torch.float64)
    es = AG.batch_expval(b, th)
    (gb,) = torch.autograd.grad((w * es).sum(), th)
    off = 0
    for i, (x, p) in enumerate(spec):
        e_i, g_i = plain_grad(sv, x, p, zz[i])
        assert abs(es[i].item() - e_i) <= e_tol(e_i)
        assert grad_ok(gb[off: off + x.n_params].numpy() / w[i].item(), g_i)
        off += x.n_params
