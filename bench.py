#!/usr/bin/env python
"""Benchmark: 30-qubit QFT followed by its inverse (960 gates, partition budget
L = 11) on a random normalised complex64 state, on one GB300 per rank.

One step = partition the circuit on the host (C++ closeness-centrality
partitioner), run every stage sweep on the GPU, and reduce the state norm in FP64
(the step's device->host result).  Reported: time per circuit, the live roofline
of the stage-sweep kernel, the HBM passes, the adjoint-gradient / forward ratio
on the 28-qubit hardware-efficient ansatz, an end-to-end number through the C ABI
with host buffers, and the CPU oracle timed on a bounded sample.

Multi-GPU: the path does not shard (one full state per GPU), so N ranks run N
independent replicas (weak scaling) with a barrier and max-over-ranks timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "30-qubit circuit time & achieved HBM GB/s vs peak; adjoint-grad/forward ratio"
N_QUBITS, L_BUDGET = 30, 11


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=L_BUDGET)
    ap.add_argument("--n", type=int, default=N_QUBITS)
    ap.add_argument("--grad-n", type=int, default=28)
    ap.add_argument("--grad-L", type=int, default=11)
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, grad ratio, batch and CPU baseline")
    ap.add_argument("--part", default="all", choices=["all", "batch", "gemm", "aux", "grad"],
                    help="batch / gemm / aux: only that section (for profiling)")
    ap.add_argument("--aux-n", type=int, default=N_QUBITS, help="state width of the aux section")
    ap.add_argument("--gemm-n", type=int, default=32)
    ap.add_argument("--gemm-k", default="5,6,7")
    ap.add_argument("--gemm-prec", default="1,2", help="1 = TF32x3, 2 = BF16x3")
    ap.add_argument("--no-c128", action="store_true", help="gemm section without the complex128 reference")
    ap.add_argument("--gemm-hier", default="2:5,2:6,1:5",
                    help="hierarchical tensor-core runs, prec:k pairs ('' for none)")
    ap.add_argument("--batch-count", type=int, default=2048)
    ap.add_argument("--no-autotune", action="store_true", help="batch section with the default (L, k) table")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--sample-seconds", type=float, default=12.0, help=argparse.SUPPRESS)
    ap.add_argument("--full-n", type=int, default=20, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle sample (runs in a child process with one BLAS / OpenMP thread)
# ---------------------------------------------------------------------------
def cpu_sample(seconds, full_n=20):
    """Two oracle timings on one core: (1) a bounded prefix of the QFT24 roundtrip,
    extrapolated to the QFT30 roundtrip by amplitudes and gates (an estimate: the
    oracle cannot hold 2^30 amplitudes for minutes per gate); (2) a complete
    QFT(full_n) roundtrip, every gate, measured end to end."""
    import numpy as np

    import circuits as C
    from oracle import statevector as S
    n_s = 24
    circ = C.qft_roundtrip(n_s)
    psi = C.random_state(n_s, 2)
    t0 = time.perf_counter()
    k = 0
    while k < len(circ.gates) and time.perf_counter() - t0 < seconds:
        g = circ.gates[k]
        psi = S.apply_gate(psi, n_s, g, circ.angles_of(g, None))
        k += 1
    dt = time.perf_counter() - t0
    full_gates = len(C.qft_roundtrip(N_QUBITS).gates)
    per_gate_amp = dt / (k * (1 << n_s))
    est_ms = per_gate_amp * full_gates * (1 << N_QUBITS) * 1e3
    rec = {"ms_per_circuit": est_ms, "seconds": dt, "gates": k, "n_sample": n_s,
           "full_gates": full_gates, "norm": float(np.vdot(psi, psi).real)}
    if full_n:
        fc = C.qft_roundtrip(full_n)
        x = C.random_state(full_n, 2)
        t0 = time.perf_counter()
        y = S.simulate(fc, None, x)
        rec["full_run"] = {"workload": f"qft{full_n}_roundtrip", "gates": len(fc.gates),
                           "ms": (time.perf_counter() - t0) * 1e3,
                           "error_l2_vs_input": float(np.linalg.norm(y - x))}
    print(json.dumps(rec))


def run_cpu_sample(seconds, full_n=20):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", "--sample-seconds", str(seconds),
                        "--full-n", str(full_n)], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    scale = (2.0 ** N_QUBITS / 2.0 ** d["n_sample"]) * (d["full_gates"] / d["gates"])
    out = {
        "value": d["ms_per_circuit"], "unit": "ms", "cores": 1, "kind": "oracle",
        "extrapolated": True, "measured_gates": d["gates"], "measured_n": d["n_sample"],
        "measured_s": d["seconds"], "scale": scale,
        "sample": (f"ESTIMATE: first {d['gates']} gates of the QFT{d['n_sample']} roundtrip (complex128 gate-by-gate "
                   f"oracle) on a 2^{d['n_sample']} state took {d['seconds']:.1f} s; value = that time x {scale:.4g} "
                   f"(2^{N_QUBITS}/2^{d['n_sample']} amplitudes x {d['full_gates']}/{d['gates']} gates); "
                   f"1 thread of {os.cpu_count()} host cores"),
    }
    if "full_run" in d:
        out["measured_full_run"] = dict(d["full_run"], cores=1, extrapolated=False)
    return out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def sampling(self):
        """True once the sampler has written its first row (or cannot run)."""
        if self.proc is None:
            return True
        self.f.flush()
        return os.path.getsize(self.f.name) > 0

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("jit.cpp", "jit_prelude.cuh", "program.h", "lower.cpp"):
        h.update(open(os.path.join(ROOT, "paper_2509_14098_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch():
    """DRAM bytes per stage-sweep launch from the committed ncu summary, if it was
    taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "stage_fwd_qft30.json")
    try:
        d = json.load(open(p))
    except OSError:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def main_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    samples, measured = [], []
    per = max(2.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    full = None
    for i in range(args.warmup + args.steps):
        # one complete (not extrapolated) oracle run, on the last step only
        cb = run_cpu_sample(per, full_n=20 if i == args.warmup + args.steps - 1 else 0)
        if cb is None:
            print(json.dumps({"impl": "reference", "unavailable": "oracle sample failed"}))
            return
        if i >= args.warmup:
            samples.append(cb["value"])
            measured.append(cb["measured_s"])
        full = cb.get("measured_full_run", full)
    v = statistics.median(samples)
    cb["value"] = v
    cb["measured_s"] = sum(measured)
    if full:
        cb["measured_full_run"] = full
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "qft30_roundtrip", "n_qubits": N_QUBITS, "L": args.L, "gates": 960},
        "extrapolated": True,
        "estimate": (f"value and ms_per_step are extrapolated from {args.steps} bounded oracle samples "
                     f"({cb['measured_s']:.1f} s of measured CPU time in all); see cpu_baseline"),
        "cpu_baseline": cb, "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def grad_ratio(args, gn):
    """Adjoint gradient against the forward pass on the hardware-efficient ansatz
    (10 layers, TFIM): wall time of sv_grad and sv_run (3 each after a warm-up that
    also compiles the stage kernels) and the per-kernel-class device times."""
    import torch

    import circuits as C
    import paper_2509_14098_gb300 as sv
    hc = C.hea(gn, 10)
    hp = C.hea_params(hc.n_params, 4)
    hplan = sv.Plan(hc, args.grad_L)
    g = sv.StateVector(gn)
    obs = C.tfim(gn)

    def grad():
        g.reset()
        return g.grad(hplan, hp, obs)

    g.reset(); g.run(hplan, hp); g.expval(obs); grad()
    torch.cuda.synchronize()
    g.timing(True); g.timing(reset=True)
    t0 = time.perf_counter(); [g.run(hplan, hp) for _ in range(3)]; torch.cuda.synchronize()
    t_fwd = (time.perf_counter() - t0) / 3
    tf = g.timing(reset=True)
    t0 = time.perf_counter(); [grad() for _ in range(3)]; torch.cuda.synchronize()
    t_grad = (time.perf_counter() - t0) / 3
    tg = g.timing(reset=True)
    g.timing(False)
    g.close()
    torch.cuda.empty_cache()
    return {
        "workload": f"hea{gn}x10 ({hc.n_params} params), TFIM open chain, L={args.grad_L}",
        "ratio": (t_grad - t_fwd) / t_fwd, "grad_over_forward": t_grad / t_fwd,
        "forward_ms": t_fwd * 1e3, "grad_ms": t_grad * 1e3,
        "kernel_ms": {"forward_stages": tf["stage_ms"] / 3, "grad_forward_stages": tg["stage_ms"] / 3,
                      "backward_stages": tg["backward_ms"] / 3, "lambda_and_expval": tg["observable_ms"] / 3},
        "definition": "(time(sv_grad) - time(sv_run)) / time(sv_run): lambda formation + backward over forward",
    }



def batch_section(args, steps):
    """Batched form: count HEA circuits (n uniform in [10, 20], 6 layers, 12 n
    parameters each, sum ZZ open chain), E and the adjoint gradient of every circuit
    per evaluation (one graph launch), after the autotuner; against looping the plain
    path (sv_grad per circuit, partitions cached) over the same batch."""
    import numpy as np
    import torch

    import circuits as C
    import paper_2509_14098_gb300 as sv
    spec = C.batch_spec(args.batch_count, seed=5, n_lo=10, n_hi=20, layers=6)
    circs = [c for c, _ in spec]
    obs = [C.zz_chain(c.n_qubits) for c in circs]
    params = np.concatenate([p for _, p in spec])
    t0 = time.perf_counter()
    b = sv.Batch(circs, obs)
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    table = {} if args.no_autotune else b.autotune(params)
    tune_s = time.perf_counter() - t0
    for _ in range(2):
        e, g = b.run(params)
    dev_ms, wall_ms = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        e, g = b.run(params)
        wall_ms.append((time.perf_counter() - t0) * 1e3)
        dev_ms.append(b.info()["last_ms"])
    info = b.info()
    out = {"workload": f"{len(circs)} HEA circuits, n ~ U[10, 20], 6 layers, sum ZZ, seed 5",
           "circuits_per_s": len(circs) / (statistics.median(wall_ms) * 1e-3),
           "ms_per_batch_device": statistics.median(dev_ms), "ms_per_batch_wall": statistics.median(wall_ms),
           "build_s": build_s, "autotune_s": tune_s,
           "tune": {str(k): list(v) for k, v in sorted(table.items())},
           "programs": info["n_programs"], "resident_circuits": info["n_resident"],
           "workspace_gb": info["workspace_bytes"] / 1e9, "smem_bytes": info["smem_bytes"], "grid": info["grid"],
           "graph": bool(info["graph"]), "graph_launches_per_batch": 1,
           "wide_threshold": int(os.environ.get("SVGB_BATCH_WIDE", "14")),
           "fusion_width_k": "register-group width (amplitudes per thread 2^k) of the persistent kernel; "
                             "circuits at or above wide_threshold qubits run as wide groups (one generated "
                             "kernel per stage over all circuits of a structure, L = 12, k = 4)"}
    b.close()
    if args.part == "all":
        plans = [sv.Plan(c, min(12, c.n_qubits)) for c in circs]
        offs = np.concatenate([[0], np.cumsum([c.n_params for c in circs])])
        sts = {}
        seen = set()
        for i in range(len(circs)):   # warm-up: one handle and one run (kernel compile) per width
            if circs[i].n_qubits in seen:
                continue
            seen.add(circs[i].n_qubits)
            st = sts.setdefault(circs[i].n_qubits, sv.StateVector(circs[i].n_qubits))
            st.reset()
            st.grad(plans[i], params[offs[i]:offs[i + 1]], obs[i])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_loop = np.zeros(len(circs))
        for i, c in enumerate(circs):
            st = sts.get(c.n_qubits)
            if st is None:
                st = sts[c.n_qubits] = sv.StateVector(c.n_qubits)
            st.reset()
            e_loop[i], _ = st.grad(plans[i], params[offs[i]:offs[i + 1]], obs[i])
        torch.cuda.synchronize()
        loop_s = time.perf_counter() - t0
        for st in sts.values():
            st.close()
        out["loop_circuits_per_s"] = len(circs) / loop_s
        out["speedup_vs_loop"] = out["circuits_per_s"] / out["loop_circuits_per_s"]
        out["max_abs_dE_vs_loop"] = float(np.max(np.abs(e_loop - e)))
    return out


def gemm_section(args):
    """Precision / tensor-core stages: brickwork of depth 24 (U3 with uniform angles
    plus CZ, seed 3) on gemm_n qubits from a random complex64 state; each (k, precision)
    runs the partition without exemptions as tcgen05 GEMM stages.  Reported: time per
    circuit, stages (= HBM passes), per-stage time and algorithmic GB/s, and the error
    against the complex128 CUDA-core run of the same circuit and input."""
    import torch

    import circuits as C
    import paper_2509_14098_gb300 as sv
    n = args.gemm_n
    circ = C.brickwork(n, 24, 3)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    psi0 = torch.randn(1 << n, dtype=torch.complex64, device="cuda", generator=gen)
    psi0 /= torch.linalg.vector_norm(psi0)
    ref = None
    if not args.no_c128:
        r = psi0.to(torch.complex128)
        st = sv.StateVector(n, sv.SV_C128, tensor=r)
        st.run(sv.Plan(circ, 11))
        st.synchronize()
        st.close()
        ref = r.to(torch.complex64)   # rounding to complex64 adds <= 6e-8 relative per amplitude
        del r
        torch.cuda.empty_cache()
    psi = torch.empty_like(psi0)
    st = sv.StateVector(n, tensor=psi)
    bytes_pass = 2.0 * (1 << n) * 8
    rows = []
    for k, prec, hier in gemm_configs(args):
        plan = sv.Plan(circ, k, gemm=(prec != 0 and not hier), hier=hier)
        psi.copy_(psi0)
        # warm-up: the raw split-precision result (no norm restoration), compared below
        st.run(plan, None, prec | (sv.SV_PREC_NO_RENORM if prec else 0))
        st.synchronize()
        err_raw = float(torch.linalg.vector_norm(psi - ref).item()) if ref is not None else None
        psi.copy_(psi0)
        st.timing(True)
        st.timing(reset=True)
        t0 = time.perf_counter()
        st.run(plan, None, prec)
        st.synchronize()
        wall = (time.perf_counter() - t0) * 1e3
        tm = st.timing(reset=True)
        st.timing(False)
        err = float(torch.linalg.vector_norm(psi - ref).item()) if ref is not None else None
        per = tm["stage_ms"] / max(1, tm["stage_launches"])
        row = {"k": k, "prec": prec_name(prec, hier), "stages": tm["stage_launches"], "ms_circuit": wall,
               "ms_per_stage": per, "gbs_per_stage": bytes_pass / (per * 1e-3) / 1e9, "err_l2_vs_c128": err}
        if prec:
            row["err_l2_vs_c128_raw"] = err_raw   # without the norm restoration
        if hier:
            row["sub_partitions"] = plan.hier_info(prec)[1]
        rows.append(row)
    st.close()
    out = {"workload": f"brickwork n={n}, depth 24, seed 3, random complex64 input", "runs": rows,
           "reference": "complex128 CUDA-core run (L=11)" if ref is not None else None,
           "target_err_l2": 2e-5}
    del psi, psi0, ref
    torch.cuda.empty_cache()
    o26 = gemm_oracle26(args)
    if o26:
        out["oracle_26q"] = o26
    return out


def gemm_configs(args):
    """(k, prec, hierarchical) runs of the tensor-core sections: flat stages per --gemm-k x
    --gemm-prec, hierarchical ones per --gemm-hier, and the CUDA-core L = 11 plan."""
    cfgs = [(int(k), int(p), False) for p in args.gemm_prec.split(",") for k in args.gemm_k.split(",")]
    cfgs += [(int(pk.split(":")[1]), int(pk.split(":")[0]), True) for pk in args.gemm_hier.split(",") if pk]
    return cfgs + [(11, 0, False)]


def prec_name(prec, hier):
    return {0: "cudacore_c64_L11", 1: "tf32x3", 2: "bf16x3"}[prec] + ("_hier" if hier else "")


def gemm_eps(K, prec):
    """Per split-precision GEMM on a norm-1 state: FP32 accumulation 3 (K / 8) 2^-23 plus
    the state operand's split u = 2^-16 (BF16x3) / 2^-22 (TF32x3)."""
    return 3 * (K / 8) * 2.0 ** -23 + (2.0 ** -16 if prec == 2 else 2.0 ** -22)


def derived_gemm_bound(plan, prec):
    """gemm_eps summed over the fused stages (K = 2^(k_eff + 1), k_eff = max(k, 6))."""
    return sum(gemm_eps(2 ** (max(6, bin(m).count("1")) + 1), prec) for m, _ in plan.stages())


def gemm_oracle26(args):
    """The precision workload at 26 qubits against the FP64 oracle's stored values
    (tests/golden/brick26_oracle.json): the complex128 CUDA-core run against the
    oracle's sampled amplitudes and <Z_q>, then every (k, precision) against the
    complex128 run (whole vector) and the oracle's samples."""
    import numpy as np
    import torch

    import circuits as C
    import paper_2509_14098_gb300 as sv
    p = os.path.join(ROOT, "tests", "golden", "brick26_oracle.json")
    if not os.path.exists(p):
        return None
    gold = json.load(open(p))
    n = gold["n_qubits"]
    circ = C.brickwork(n, gold["depth"], gold["circuit_seed"])
    x64 = C.random_state(n, gold["circuit_seed"]).astype(np.complex64)
    idx = torch.tensor(gold["indices"], device="cuda")
    amp = torch.tensor([complex(a, b) for a, b in gold["amplitudes"]], dtype=torch.complex128, device="cuda")
    r = torch.from_numpy(x64.astype(np.complex128)).to("cuda")
    st = sv.StateVector(n, sv.SV_C128, tensor=r)
    st.run(sv.Plan(circ, 11))
    st.synchronize()
    st.close()
    c128_sample_err = float((r[idx] - amp).abs().max().item())
    x = torch.from_numpy(x64).to("cuda")
    psi = torch.empty_like(x)
    st = sv.StateVector(n, tensor=psi)
    rows = []
    for k, prec, hier in gemm_configs(args):
        plan = sv.Plan(circ, k, gemm=(prec != 0 and not hier), hier=hier)
        err_raw = None
        if prec:
            psi.copy_(x)
            st.run(plan, None, prec | sv.SV_PREC_NO_RENORM)
            st.synchronize()
            err_raw = float(torch.linalg.vector_norm(psi.to(torch.complex128) - r).item())
        psi.copy_(x)
        st.run(plan, None, prec)
        st.synchronize()
        err = float(torch.linalg.vector_norm(psi.to(torch.complex128) - r).item())
        samp = float((psi[idx].to(torch.complex128) - amp).abs().max().item())
        if hier:
            bound = plan.hier_info(prec)[1] * gemm_eps(2 ** (k + 1), prec)
        else:
            bound = derived_gemm_bound(plan, prec) if prec else 2e-5
        row = {"k": k, "prec": prec_name(prec, hier), "stages": len(plan.stages()), "err_l2_vs_c128": err,
               "max_err_vs_oracle_samples": samp, "derived_bound": bound, "meets_target_2e-5": err <= 2e-5}
        if prec:
            row["err_l2_vs_c128_raw"] = err_raw   # without the norm restoration
        rows.append(row)
    st.close()
    del r, x, psi
    torch.cuda.empty_cache()
    return {"workload": f"brickwork n={n}, depth {gold['depth']}, seed {gold['circuit_seed']}, "
                        f"input random_state({n}, {gold['circuit_seed']}) rounded to complex64",
            "oracle": "tests/golden/brick26_oracle.json (complex128 gate-by-gate oracle: 64 sampled amplitudes, <Z_q>)",
            "c128_max_err_vs_oracle_samples": c128_sample_err, "runs": rows}


def partition_section(widths=(30, 34, 37), L=11, reps=3):
    """Host partitioner (C++, exact closeness, Sec. 4.1-4.2) on the paper's benchmark
    families at its 30-37 qubit widths: best-of-reps wall time per circuit, with
    gate and stage counts.  The paper's own figures (Python + NetworkX) are context."""
    import circuits as C
    import paper_2509_14098_gb300 as sv
    rows = []
    for name in sorted(C.FAMILIES):
        for n in widths:
            c = C.FAMILIES[name](n)
            best = float("inf")
            for _ in range(reps):
                t0 = time.perf_counter()
                plan = sv.Plan(c, L)
                best = min(best, time.perf_counter() - t0)
            rows.append({"family": name, "n_qubits": n, "gates": len(c.gates), "stages": len(plan.stages()),
                         "partition_ms": best * 1e3})
    return {"L": L, "n_fixed": 4, "runs": rows,
            "paper_context": "Sec. 5.2: under 1 s for most circuits, about 4-5 s for qnn and vqc "
                             "(Python + NetworkX, 30-37 qubits, three-level hierarchy; other hardware)"}


def aux_section(n, reps=3):
    """Permutation sweep (bit reversal of n qubits: out-of-place, then copied back) and the
    FP64 reductions (norm; TFIM expectation by Pauli sweeps) on a 2^n complex64 state:
    device time per call (CUDA events via the library's timing record where it has one)
    and algorithmic GB/s."""
    import torch

    import circuits as C
    import paper_2509_14098_gb300 as sv
    psi = torch.randn(1 << n, dtype=torch.complex64, device="cuda")
    psi /= torch.linalg.vector_norm(psi)
    st = sv.StateVector(n, tensor=psi)
    rev = [n - 1 - q for q in range(n)]
    st.permute(rev)
    st.norm()
    st.expval(C.tfim(n))
    st.timing(True)
    st.timing(reset=True)
    for _ in range(reps):
        st.permute(rev)
    st.synchronize()
    tm = st.timing(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st.stream)
    for _ in range(reps):
        st.norm()
    e1.record(st.stream)
    torch.cuda.synchronize()
    norm_ms = e0.elapsed_time(e1) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        st.expval(C.tfim(n))
    ev_ms = (time.perf_counter() - t0) * 1e3 / reps
    # the QFT alone ends in the bit reversal: its last stage writes through the map
    qft = C.qft(n)
    st.run(sv.Plan(qft, L_BUDGET))
    st.synchronize()
    st.timing(reset=True)
    e0.record(st.stream)
    for _ in range(reps):
        st.run(sv.Plan(qft, L_BUDGET))
    e1.record(st.stream)
    torch.cuda.synchronize()
    qft_ms = e0.elapsed_time(e1) / reps
    tq = st.timing(reset=True)
    qinfo = st.run_info()
    st.timing(False)
    st.close()
    nb = (1 << n) * 8
    perm_ms = tm["permute_ms"] / max(1, tm["permute_launches"])
    qft_rec = {"what": f"QFT{n} alone (the SWAPs leave the bit reversal; the last stage writes through it "
                       "out of place, then a copy into the caller's buffer)",
               "ms": qft_ms, "stage_sweeps": qinfo["stage_sweeps"],
               "permutation_sweeps": qinfo["permutation_sweeps"],
               "stage_ms": tq["stage_ms"] / reps}
    return {"n_qubits": n,
            "permutation": {"what": "bit reversal, one out-of-place sweep (kernel time; sv_permute then copies the result back into the caller's buffer)", "ms_per_sweep": perm_ms,
                            "gbs": 2 * nb / (perm_ms * 1e-3) / 1e9, "launches": tm["permute_launches"] / reps},
            "norm": {"what": "||psi||^2 in FP64 (host result)", "ms": norm_ms, "gbs": nb / (norm_ms * 1e-3) / 1e9},
            "expval_tfim": {"what": "<psi| sum ZZ + 0.7 sum X |psi> (Pauli sweeps, FP64, host result)", "ms": ev_ms},
            "qft_alone": qft_rec}


def main_ours(args):
    import ctypes

    import numpy as np
    import torch

    import circuits as C
    import __graft_entry__ as ge
    ge.build()
    import paper_2509_14098_gb300 as sv
    from paper_2509_14098_gb300 import _native as N

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.part == "batch":
        r = batch_section(args, args.steps)
        if rank == 0:
            print(json.dumps({"part": "batch", "batch": r}))
        return
    if args.part == "gemm":
        r = gemm_section(args)
        if rank == 0:
            print(json.dumps({"part": "gemm", "gemm": r}))
        return
    if args.part == "grad":
        r = {"grad_forward_ratio": grad_ratio(args, args.grad_n)}
        if rank == 0:
            print(json.dumps({"part": "grad", "grad": r}))
        return
    if args.part == "aux":
        r = aux_section(args.aux_n)
        if rank == 0:
            print(json.dumps({"part": "aux", "aux": r}))
        return
    n, L = args.n, args.L
    circ = C.qft_roundtrip(n)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2 + rank)
    psi = torch.randn(1 << n, dtype=torch.complex64, device=dev, generator=gen)
    psi /= torch.linalg.vector_norm(psi)
    ref_copy = psi.clone() if rank == 0 else None
    st = sv.StateVector(n, tensor=psi)
    stream = st.stream

    t0 = time.perf_counter()
    plan0 = sv.Plan(circ, L)
    partition_ms = (time.perf_counter() - t0) * 1e3
    stages = plan0.stages()

    # ||psi||^2 of each step goes to its own device double (sv_norm_noalloc, enqueued
    # without a host wait), so the host partitions and lowers step k + 1 while the GPU
    # still runs step k; every result is read back once the timed steps are done
    dnorm = torch.zeros(max(1, args.steps), dtype=torch.float64, device=dev)
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def step(i=0):
        plan = sv.Plan(circ, L)
        st.run(plan)
        N.check(N.lib.sv_norm_noalloc(ctypes.c_void_p(psi.data_ptr()), n, sv.SV_C64, sptr,
                                      ctypes.c_void_p(dnorm.data_ptr() + 8 * i)))

    for _ in range(args.warmup):
        step()
    st.synchronize()
    info = st.run_info()
    launches_per_step = info["kernel_launches"] + 2           # + norm and its reduction
    passes = info["stage_sweeps"] + info["permutation_sweeps"]
    torch.cuda.synchronize()
    barrier(pg)
    clocks = Clocks(local)
    clocks.start()
    t_wait = time.perf_counter()
    while not clocks.sampling() and time.perf_counter() - t_wait < 5.0:   # untimed: the sampler starts under load
        step()
    torch.cuda.synchronize()
    barrier(pg)
    st.timing(True)
    st.timing(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    st.synchronize()                                  # reports a stage wait that gave up
    norms = dnorm.cpu().tolist()
    ms_total = e0.elapsed_time(e1)
    tm = st.timing(reset=True)
    st.timing(False)
    ck = clocks.stop()
    barrier(pg)
    ms_total = max_over_ranks(pg, ms_total)
    ms_step = ms_total / args.steps
    value = ms_step / world                                       # ms per circuit, whole job

    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    bytes_per_launch = 2.0 * (1 << n) * 8
    avg_stage_ms = tm["stage_ms"] / max(1, tm["stage_launches"])
    achieved = bytes_per_launch / (avg_stage_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic_per_launch(),
                "kernel": "svj_fwd_* (generated sweep of one partition, complex64)",
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback",
                "avg_launch_ms": avg_stage_ms, "launches": tm["stage_launches"]}
    whole_gbs = passes * bytes_per_launch / (ms_step * 1e-3) / 1e9

    extras = {}
    if rank == 0 and not args.no_extras:
        # parity check: one QFT then inverse QFT (the identity) from a fresh copy of the input
        psi.copy_(ref_copy)
        st.run(sv.Plan(circ, L))
        st.synchronize()
        err = float(torch.linalg.vector_norm(psi - ref_copy).item())
        extras["roundtrip_error_l2"] = err
        extras["roundtrip_error_tolerance"] = 2e-5
        del ref_copy
        # end to end through the C ABI with host buffers (pinned)
        host_in = torch.empty(1 << n, dtype=torch.complex64, pin_memory=True)
        host_in.copy_(psi)
        host_out = torch.empty_like(host_in, pin_memory=True)
        h = st.handle

        def e2e_step():
            N.check(N.lib.sv_set_state_host(h, ctypes.c_void_p(host_in.data_ptr())))
            plan = sv.Plan(circ, L)
            st.run(plan)
            nrm = st.norm()
            N.check(N.lib.sv_get_state_host(h, ctypes.c_void_p(host_out.data_ptr())))
            return nrm

        e2e_step()
        t0 = time.perf_counter()
        ne = 2
        for _ in range(ne):
            e2e_step()
        seq_ms = (time.perf_counter() - t0) * 1e3 / ne
        # the same steps streamed through two handles on two CUDA streams: a step's input
        # copy and stage sweeps are issued before the previous step's result is read back,
        # so the two copy directions overlap; every step still copies its whole input in
        # and its whole result (and the norm) out
        st2_psi = torch.empty_like(psi)
        st2 = sv.StateVector(n, tensor=st2_psi, stream=torch.cuda.Stream(device=dev))
        hosts = [(host_in, host_out), (torch.empty_like(host_in, pin_memory=True), torch.empty_like(host_in, pin_memory=True))]
        hosts[1][0].copy_(host_in)
        sts = [st, st2]

        def issue(i):
            s_, (hin, _) = sts[i & 1], hosts[i & 1]
            N.check(N.lib.sv_set_state_host(s_.handle, ctypes.c_void_p(hin.data_ptr())))
            s_.run(sv.Plan(circ, L))

        def finish(i):
            s_, (_, hout) = sts[i & 1], hosts[i & 1]
            nrm = s_.norm()
            N.check(N.lib.sv_get_state_host(s_.handle, ctypes.c_void_p(hout.data_ptr())))
            return nrm

        issue(0)
        issue(1)
        finish(0)
        finish(1)
        ne2 = 4
        t0 = time.perf_counter()
        issue(0)
        for i in range(ne2):
            if i + 1 < ne2:
                issue(i + 1)
            finish(i)
        pipe_ms = (time.perf_counter() - t0) * 1e3 / ne2
        extras["e2e"] = {"value": pipe_ms, "unit": "ms", "h2d_bytes_per_step": (1 << n) * 8,
                         "d2h_bytes_per_step": (1 << n) * 8 + 8,
                         "mode": "steps streamed through two handles on two CUDA streams (sv_set_state_host, sv_run, "
                                 "sv_norm, sv_get_state_host per step; a step's input copy and sweeps overlap the "
                                 "previous step's result copy)",
                         "sequential_ms": seq_ms, "steps": ne2}
        st2.close()
        del st2, st2_psi, hosts
        del host_in, host_out
        # adjoint gradient / forward ratio on the hardware-efficient ansatz (the
        # differentiation workload's width, and 30 qubits)
        st.close()
        del st, psi
        torch.cuda.empty_cache()

        extras["grad_forward_ratio"] = grad_ratio(args, args.grad_n)
        if args.grad_n != N_QUBITS:
            extras["grad_forward_ratio_30q"] = grad_ratio(args, N_QUBITS)
        extras["batch"] = batch_section(args, 3)
        torch.cuda.empty_cache()
        extras["tensor_core_stages"] = gemm_section(args)
        torch.cuda.empty_cache()
        extras["permutation_and_reductions"] = aux_section(n)
        extras["partitioner"] = partition_section()
    cpu = None
    if rank == 0 and world == 1 and not args.no_extras:
        cpu = run_cpu_sample(args.sample_seconds)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "qft30_roundtrip", "n_qubits": n, "L": L, "gates": len(circ.gates),
                       "state": "complex64, i.i.d. N(0,1) re/im (seeded torch Philox), normalised",
                       "l2": f"inputs larger than L2 ({(1 << n) * 8 / 2**30:g} GiB state)", "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "hbm_passes": passes, "stages": len(stages), "achieved_gbs_whole_circuit": whole_gbs,
            "partition_ms": partition_ms, "norm_last_step": norms[-1],
            "gpu_launches": launches_per_step * args.steps,
            "clocks": ck,
        }
        if cpu:
            out["cpu_baseline"] = cpu
        out.update(extras)
        print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.cpu_sample:
        cpu_sample(a.sample_seconds, a.full_n)
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_ours(a)
