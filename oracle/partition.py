"""Closeness-centrality partitioner written plainly from Sec. 4.1-4.2 (oracle twin).

Step A (Sec. 4.1): every gate is a tensor node; edges are qubit dimensions.  A gate
depends on the previous gate on each of its qubits.  Each node carries the length of
its critical path to the state tensor psi: l_psi = 0 and l_g = 1 + max over the
gate's predecessors (the paper's example: l_H = 1, l_CX = 2 for GHZ-3).  Gates are
kept in their original flat order; nothing is reordered or replaced.

Step B (Sec. 4.2, Eqs. for CC, RN and dist): a backward traversal builds, for every
node v, its reachable set RN(v) = union over downstream neighbours w of {w} u RN(w)
(downstream neighbours = immediate successors, the next gate on each qubit), and the
distance sum dist(v) = sum over x in RN(v) of d(v, x), where d accumulates
|l_a - l_b| along a downstream path.  Levels strictly increase along every path, so
that sum telescopes to l_x - l_v for every path and dist is exact without the
paper's overlap threshold heuristic (which only approximates the union).  Closeness
is |RN|/dist times the Wasserman-Faust factor |RN|/N, N = number of gates; CC = 0
when RN is empty.  Ranking compares CC exactly (rationals).

Step B, forward pass (Sec. 4.2, step 3): starting from the frontier of ready gates,
the partition repeatedly (i) absorbs, scanning in original order to a fixed point,
every ready gate whose required dimensions are already local, then (ii) makes local
the qubits of the highest-centrality ready gate (ties: lowest gate index) that still
fits the budget of L local qubits; when no ready gate fits, the partition is cut and
the frontier starts a fresh local set.  Required dimensions follow the two exemptions
of Sec. 4.2: a diagonal gate needs none of its qubits, and a controlled gate needs
only its target (a non-local control is allowed).  SWAP needs none: it is executed as
a relabelling of which physical bit holds which circuit qubit (it is still a node of
the DAG and still counted).  The partitioner therefore works on physical bit
positions obtained by replaying the SWAP relabellings in circuit order.

``fixed`` lists physical bits that are local in every partition (the bits a tile
must always contain, e.g. the low bits that make memory accesses contiguous); they
count toward the budget L.

After a cut the local set is filled up to min(L, n) bits: first with the other
physical bits the partition's gates touch (controls, diagonal partners), ascending,
then with the lowest remaining bits.  In the GHZ-3 example with two local qubits
this gives the paper's partition tree (Sec. 4.3): L0 keeps {0, 1} local and R0 keeps
{1, 2} local.  Filling cannot enable another absorption: any ready gate whose
required bits fit in the filled set would have fitted the budget in step (ii).
"""
from fractions import Fraction

DIAGONAL = {"Z", "S", "SDG", "T", "TDG", "RZ", "P", "CZ", "CP"}
CONTROLLED = {"CX", "CY"}


def build_dag(circuit):
    """Predecessor / successor lists (deduplicated, ascending) and critical-path levels."""
    n = circuit.n_qubits
    G = len(circuit.gates)
    last = [-1] * n
    preds = [[] for _ in range(G)]
    succs = [[] for _ in range(G)]
    level = [0] * G
    for i, g in enumerate(circuit.gates):
        ps = sorted({last[q] for q in g.qubits if last[q] >= 0})
        preds[i] = ps
        for p in ps:
            succs[p].append(i)
        level[i] = 1 + max((level[p] for p in ps), default=0)
        for q in g.qubits:
            last[q] = i
    return preds, succs, level


def reach_and_dist(succs, level):
    """Backward traversal (reverse original order = reverse topological order).
    RN as Python-int bitsets; dist(v) = sum_{x in RN(v)} (l_x - l_v)."""
    G = len(level)
    rn = [0] * G
    dist = [0] * G
    for v in range(G - 1, -1, -1):
        s = 0
        for w in succs[v]:
            s |= (1 << w) | rn[w]
        rn[v] = s
        total = 0
        x = s
        while x:
            low = x & -x
            idx = low.bit_length() - 1
            total += level[idx] - level[v]
            x ^= low
        dist[v] = total
    return rn, dist


def closeness(circuit):
    """Exact closeness centrality per gate as Fractions, plus |RN| and dist."""
    _, succs, level = build_dag(circuit)
    rn, dist = reach_and_dist(succs, level)
    N = len(level)
    cc, size = [], []
    for v in range(N):
        r = bin(rn[v]).count("1")
        size.append(r)
        cc.append(Fraction(0) if r == 0 else Fraction(r, dist[v]) * Fraction(r, N))
    return cc, size, dist, level


def physical_qubits(circuit):
    """Physical bit positions of each gate's qubits after replaying SWAP relabels in
    circuit order, and the final map circuit-qubit -> physical bit."""
    where = list(range(circuit.n_qubits))
    out = []
    for g in circuit.gates:
        out.append(tuple(where[q] for q in g.qubits))
        if g.kind == "SWAP":
            a, b = g.qubits
            where[a], where[b] = where[b], where[a]
    return out, where


def need(gate, phys, strict=False):
    """Physical bits a gate requires to be local (Sec. 4.2 exemptions).  strict: no
    exemptions (every qubit of a gate local, SWAP still a relabel) — used when each
    partition must be one fixed dense unitary on its local qubits."""
    if gate.kind == "SWAP":
        return frozenset()
    if strict:
        return frozenset(phys)
    if gate.kind in DIAGONAL:
        return frozenset()
    if gate.kind in CONTROLLED:
        return frozenset((phys[1],))
    return frozenset(phys)


class PartitionError(Exception):
    pass


def partition(circuit, L, fixed=(), strict=False):
    """Forward frontier pass.  Returns a list of stages (local_bits frozenset, [gate ids in
    execution order]) and the final circuit-qubit -> physical-bit map."""
    gates = circuit.gates
    G = len(gates)
    preds, _, _ = build_dag(circuit)
    cc, _, _, _ = closeness(circuit)
    phys, final_map = physical_qubits(circuit)
    needs = [need(g, p, strict) for g, p in zip(gates, phys)]
    fixed = frozenset(fixed)
    if len(fixed) > L:
        raise PartitionError("fixed bits exceed the budget")
    done = [False] * G
    n_done = 0
    stages = []
    while n_done < G:
        local = set(fixed)
        stage = []
        while True:
            changed = True
            while changed:                                    # (i) absorb to a fixed point
                changed = False
                for i in range(G):
                    if not done[i] and all(done[p] for p in preds[i]) and needs[i] <= local:
                        done[i] = True
                        n_done += 1
                        stage.append(i)
                        changed = True
            best = -1                                          # (ii) highest-CC ready gate that fits
            for i in range(G):
                if done[i] or not all(done[p] for p in preds[i]):
                    continue
                if len(local | needs[i]) > L:
                    continue
                if best < 0 or cc[i] > cc[best]:
                    best = i
            if best < 0:
                break
            local |= needs[best]
        if not stage:                                          # (iii) cut
            raise PartitionError("a ready gate needs more than L local qubits")
        width = min(L, circuit.n_qubits)
        for q in sorted({b for i in stage for b in phys[i]}):  # fill: touched bits first
            if len(local) >= width:
                break
            local.add(q)
        q = 0
        while len(local) < width:                              # then the lowest free bits
            local.add(q)
            q += 1
        stages.append((frozenset(local), stage))
    return stages, final_map


def validate(circuit, stages, L, fixed=(), strict=False):
    """Invariants: every gate exactly once; the concatenated order respects every
    dependency; each stage's gates need only its local bits; |local| <= L; fixed bits local."""
    preds, _, _ = build_dag(circuit)
    phys, _ = physical_qubits(circuit)
    seen = {}
    pos = 0
    for local, ids in stages:
        if len(local) > L:
            return False, "stage exceeds L"
        if not frozenset(fixed) <= local:
            return False, "fixed bit not local"
        for i in ids:
            if i in seen:
                return False, f"gate {i} twice"
            if not need(circuit.gates[i], phys[i], strict) <= local:
                return False, f"gate {i} needs a non-local bit"
            for p in preds[i]:
                if p not in seen:
                    return False, f"gate {i} before its predecessor {p}"
            seen[i] = pos
            pos += 1
    if len(seen) != len(circuit.gates):
        return False, "missing gates"
    return True, "ok"
