"""Pins for the oracle partitioner: the paper's worked example, brute-force closeness
on tiny DAGs, NetworkX's closeness, validator invariants, execution equivalence."""
import inspect
import itertools
import json
import os
import types
from fractions import Fraction

import numpy as np
import pytest

import circuits as C
from oracle import partition as P
from oracle import statevector as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_ghz3_paper_example():
    gold = json.load(open(os.path.join(GOLD, "ghz3_example.json")))
    c = C.Circuit(3, [C.Gate(k, tuple(q)) for k, q in gold["qasm_gates"]])
    _, _, level = P.build_dag(c)
    assert level[0] == gold["printed_levels"]["H"]
    assert level[1] == gold["printed_levels"]["first CX"]
    stages, final = P.partition(c, gold["local_qubits"])
    assert final == [0, 1, 2]
    assert len(stages) == len(gold["partition_tree"])
    for (local, ids), node in zip(stages, gold["partition_tree"]):
        assert sorted(local) == node["local"]
        assert sorted(set(range(3)) - set(local)) == node["global"]
        assert ids == node["gates"]
    psi = S.simulate(c)
    for k, v in gold["final_amplitudes"].items():
        assert abs(psi[int(k)] - v) < 1e-15
    cc, size, dist, _ = P.closeness(c)
    d = gold["derived_not_printed"]
    assert size == d["reach_size"] and dist == d["dist"]
    assert cc == [Fraction(a, b) for a, b in d["cc_numerator_denominator"]]


def _cc_cases():
    return json.load(open(os.path.join(GOLD, "cc_choice.json")))["cases"]


def _cc_circuit(case):
    return C.Circuit(case["n_qubits"], [C.Gate(k, tuple(q)) for k, q in case["gates"]])


def _stages_match(partition_fn, case):
    stages, _ = partition_fn(_cc_circuit(case), case["L"])
    return [(sorted(loc), ids) for loc, ids in stages] == [(s["local"], s["gates"]) for s in case["stages"]]


@pytest.mark.parametrize("case", _cc_cases(), ids=lambda c: c["name"])
def test_closeness_choice_golden(case):
    """Hand-derived cases in which the highest-closeness choice (Sec. 4.2, step 3)
    decides the partitions: levels, reachable sets, distance sums, exact closeness
    and the stage lists."""
    c = _cc_circuit(case)
    _, succs, level = P.build_dag(c)
    rn, dist = P.reach_and_dist(succs, level)
    assert level == case["levels"]
    assert [sorted(i for i in range(len(level)) if (r >> i) & 1) for r in rn] == case["reach"]
    assert dist == case["dist"]
    cc, _, _, _ = P.closeness(c)
    assert cc == [Fraction(a, b) for a, b in case["cc"]]
    assert _stages_match(P.partition, case)
    assert P.validate(c, P.partition(c, case["L"])[0], case["L"])[0]


def test_closeness_choice_golden_catches_planted_mistakes():
    """The golden cases fail an oracle whose choice takes the lowest closeness first,
    or breaks ties towards the higher gate index (mutations planted in a copy of the
    oracle's source, on the CPU)."""
    src = inspect.getsource(P)
    assert src.count("cc[i] > cc[best]") == 1
    cases = _cc_cases()
    for mutated in ("cc[i] < cc[best]", "cc[i] >= cc[best]"):
        mod = types.ModuleType("mutated_partition")
        exec(compile(src.replace("cc[i] > cc[best]", mutated), "mutated_partition", "exec"), mod.__dict__)
        assert not all(_stages_match(mod.partition, case) for case in cases), mutated


def _brute_force_closeness(circuit):
    """All-pairs downstream shortest paths with edge weight |l_a - l_b| (Floyd-Warshall)."""
    preds, succs, level = P.build_dag(circuit)
    G = len(level)
    INF = float("inf")
    d = [[INF] * G for _ in range(G)]
    for v in range(G):
        d[v][v] = 0
        for w in succs[v]:
            d[v][w] = abs(level[v] - level[w])
    for k in range(G):
        for i in range(G):
            if d[i][k] == INF:
                continue
            for j in range(G):
                if d[i][k] + d[k][j] < d[i][j]:
                    d[i][j] = d[i][k] + d[k][j]
    out = []
    for v in range(G):
        reach = [x for x in range(G) if x != v and d[v][x] < INF]
        tot = sum(d[v][x] for x in reach)
        out.append((len(reach), tot))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_closeness_brute_force(seed):
    c = C.random_circuit(5, 25, seed)
    cc, size, dist, _ = P.closeness(c)
    bf = _brute_force_closeness(c)
    N = len(c.gates)
    for v, (r, tot) in enumerate(bf):
        assert size[v] == r and dist[v] == tot
        assert cc[v] == (Fraction(0) if r == 0 else Fraction(r * r, tot * N))


def test_closeness_matches_networkx():
    nx = pytest.importorskip("networkx")
    c = C.random_circuit(6, 40, 11)
    preds, succs, level = P.build_dag(c)
    g = nx.DiGraph()
    g.add_nodes_from(range(len(level)))
    for v, ws in enumerate(succs):
        for w in ws:
            g.add_edge(v, w, w_=abs(level[v] - level[w]))
    # networkx measures distances *to* a node; reverse to get downstream reach
    ref = nx.closeness_centrality(g.reverse(), distance="w_", wf_improved=True)
    cc, _, _, _ = P.closeness(c)
    N = len(level)
    for v in range(N):
        # networkx normalises by N-1, the paper's factor by N
        assert abs(float(cc[v]) * N - ref[v] * (N - 1)) < 1e-12


@pytest.mark.parametrize("L,fixed", [(2, ()), (3, ()), (3, (0,)), (4, (0, 1)), (5, (0, 1, 2, 3))])
@pytest.mark.parametrize("seed", range(5))
def test_partition_valid_and_equivalent(L, fixed, seed):
    n = 6
    c = C.random_circuit(n, 50, seed)
    stages, final = P.partition(c, L, fixed)
    ok, why = P.validate(c, stages, L, fixed)
    assert ok, why
    for local, _ in stages:
        assert len(local) == min(L, n)
    # execution equivalence: stage order (SWAPs applied as real gates) == original order
    order = [i for _, ids in stages for i in ids]
    psi0 = C.random_state(n, seed)
    reordered = C.Circuit(n, [c.gates[i] for i in order])
    assert np.abs(S.simulate(reordered, None, psi0) - S.simulate(c, None, psi0)).max() < 1e-12


def test_exemptions():
    # Sec. 4.2: a diagonal gate and a controlled gate with a non-local control are
    # absorbed into a partition whose local set holds only the target.
    n = 4
    g = [C.Gate("H", (0,)), C.Gate("CP", (3, 0), -1, (0.3,)), C.Gate("CZ", (2, 3)),
         C.Gate("RZ", (2,), -1, (0.1,)), C.Gate("CX", (3, 0)), C.Gate("CX", (0, 3))]
    c = C.Circuit(n, g)
    stages, _ = P.partition(c, 1)
    assert stages[0][1] == [0, 1, 2, 3, 4]          # H, CP, CZ, RZ, CX(3->0) all in the first partition
    assert stages[0][0] == frozenset({0})
    assert stages[1][1] == [5]                       # CX with a non-local *target* is not


def test_swap_is_relabel():
    c = C.Circuit(3, [C.Gate("SWAP", (0, 2)), C.Gate("H", (0,))])
    phys, final = P.physical_qubits(c)
    assert phys[1] == (2,) and final == [2, 1, 0]
    stages, _ = P.partition(c, 1)
    assert len(stages) == 1 and stages[0][0] == frozenset({2})


def test_validator_catches_a_planted_mistake():
    c = C.ghz(4)
    stages, _ = P.partition(c, 2)
    bad = [(stages[0][0], list(reversed(stages[0][1])))] + stages[1:]
    assert not P.validate(c, bad, 2)[0]
    bad = [(frozenset({0}), stages[0][1])] + stages[1:]
    assert not P.validate(c, bad, 2)[0]


def test_exhaustive_tiny():
    kinds = ["H", "CX", "CZ", "SWAP"]
    n = 3
    pairs = [(0, 1), (1, 2), (2, 0), (1, 0)]
    count = 0
    for seq in itertools.product(range(len(kinds) * 4), repeat=3):
        gates = []
        for s in seq:
            k = kinds[s // 4]
            gates.append(C.Gate(k, (s % 3,)) if k == "H" else C.Gate(k, pairs[s % 4]))
        c = C.Circuit(n, gates)
        for L in (1, 2, 3):
            try:
                stages, _ = P.partition(c, L)
            except P.PartitionError:
                assert L == 1
                continue
            assert P.validate(c, stages, L)[0]
            count += 1
    assert count > 3000


def test_config_partitions_are_valid():
    for name in ("brick16", "qft30", "hea28"):
        c, _, L = C.workload(name)
        stages, _ = P.partition(c, L, range(4))
        assert P.validate(c, stages, L, range(4))[0]
