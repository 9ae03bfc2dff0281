"""Benchmark: energy + adjoint-gradient (+ 1-RDM) evaluations per second at 30 qubits.

One step = one pass of the whole hot path over one synthetic problem: prepare the
Jordan-Wigner HF reference, apply the 200-operator ADAPT-style ansatz, evaluate
E = <psi|H|psi> and lambda = (H - c) psi, run the adjoint sweep for dE/dtheta,
restore psi(theta) and take the spin-resolved 1-RDM.  Workload: 30 qubits
(15 spatial orbitals, 10 electrons), seeded synthetic integrals shaped like the
paper's molecules (config 5 of the workload list).

Headline: the dense 2^30-amplitude complex64 state (8 GiB per vector, float64
reductions), the state-vector method the metric is defined on; complex128 beside
it.  Also timed: the same step in sector storage (only the C(15,5)^2 = 9,018,009
amplitudes of the (5, 5) sector, 72 MB, a separate row with its own roofline), with
real float32 amplitudes (the real-angle ansatz keeps psi real), and the batched
small-instance launch (config 4).  L2 is flushed (a 256 MB write)
before every timed step, outside its events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica (the path does not shard in this build: "replicas only"); value is the
evaluations of all ranks divided by the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "energy+adjoint-grad evals/s at 30 qubits, FP32-state vs FP64; % of HBM peak"
UNIT = "evals/s"
CONFIG_ID = 5
# DRAM bytes (read + write) of one sector-storage expectation per expectation form, from
# the ncu captures summarised in profiles/sigma_products_n30_sector_c64.md (form 4:
# k_phase_planar, k_transpose_pieces, k_same_tc, k_sigma_ab, k_sigma_comb; form 5: the
# same with k_ab_tc for k_sigma_ab and the gathering k_sigma_comb); None once a kernel
# changes.
SIGMA_TRAFFIC_BYTES = {4: 1555.6e6, 5: 12283.4e6}
SIGMA_KERNELS = {
    3: "expectation: k_sigma_ab + k_sigma_same (two launches)",
    4: "expectation: k_phase_planar + k_transpose_pieces + k_same_tc (same-spin products, tcgen05 bf16x3) "
       "+ k_sigma_ab + k_sigma_comb",
    5: "expectation: k_phase_planar + k_transpose_pieces + k_same_tc (same-spin products) + k_ab_tc "
       "(alpha-beta products; both tcgen05 bf16x3) + k_sigma_comb (gathers the alpha-beta planes)"}
# DRAM bytes per k_adjoint launch of the dense headline: the 28-qubit capture's
# traffic / algorithmic ratio (1.115, profiles/k_adjoint_dram_n28_dense_c64.md) times
# the 30-qubit algorithmic bytes per launch; None once the kernel changes.
ADJOINT_TRAFFIC_BYTES = 4.93e9


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def touched_bytes(ops, n, amp_bytes):
    """Algorithmic bytes of one rotation per op: read + write of the 2 * 2^(n - nbits) touched amplitudes."""
    kind = np.asarray(ops)[:, 0]
    nbits = np.where((kind == 1) | (kind == 3), 2, 4)
    return (4.0 * (2.0 ** (n - nbits)) * amp_bytes)


def sector_touched_bytes(ops, n_orb, na, nb, amp_bytes):
    """Algorithmic bytes of one rotation per op on sector storage: read + write of the
    2 * C(N - k_a, na - f_a) C(N - k_b, nb - f_b) amplitudes it pairs, where k_a (f_a) is
    the number of alpha spin-orbitals in the op's mask (among its occupied ones)."""
    from math import comb
    out = []
    for kind, i, j, a, b in np.asarray(ops):
        occ = [i] if kind in (1, 3) else [i, j]
        vir = [a] if kind in (1, 3) else [a, b]
        ka = sum(1 for q in occ + vir if q % 2 == 0)
        fa = sum(1 for q in occ if q % 2 == 0)
        kb, fb = len(occ) + len(vir) - ka, len(occ) - fa
        cnt = comb(n_orb - ka, na - fa) * comb(n_orb - kb, nb - fb) if na >= fa and nb >= fb else 0
        out.append(4.0 * cnt * amp_bytes)
    return np.array(out)


# ---------------------------------------------------------------- ranks

def reduce_max(values):
    """Element-wise maximum over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def throughput(world, steps, max_ms):
    """Evaluations of all ranks per second of the slowest rank: each rank runs `steps` of its own replica."""
    return world * steps / (max_ms / 1000.0)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)

def oracle_eval_sample(p, sector=None, sigma_rows=6000, ops_sample=4):
    """Time the CPU oracle on a bounded sample of one evaluation and scale to a full one.

    Sample: `ops_sample` rotations and generator applications over the full sector,
    sigma = H psi on `sigma_rows` evenly spaced determinants (scaled by D / rows),
    the full 1-RDM.  One evaluation = L forward rotations + sigma + L reverse
    steps (two rotations and one generator application each) + 1-RDM.
    """
    import oracle
    from oracle import route_a as A
    sec = sector or oracle.Sector(p["n_qubits"], p["na"], p["nb"])
    psi = A.hf_state(sec, p["occ"])
    ops, theta, L = p["ops"], p["theta"], len(p["ops"])
    t0 = time.perf_counter()
    for k in range(ops_sample):
        psi = A.rotate(sec, ops[k], theta[k], psi)
    t_rot = (time.perf_counter() - t0) / ops_sample
    t0 = time.perf_counter()
    for k in range(ops_sample):
        A.generator_apply(sec, ops[k], psi)
    t_gen = (time.perf_counter() - t0) / ops_sample
    rows = np.linspace(0, sec.D - 1, min(sigma_rows, sec.D)).astype(np.int64)
    t0 = time.perf_counter()
    A.hamiltonian_apply(sec, p["h"], p["eri"], p["e_nuc"], psi, rows=rows)
    t_sig = (time.perf_counter() - t0) * sec.D / len(rows)
    t0 = time.perf_counter()
    A.rdm1(sec, psi)
    t_rdm = time.perf_counter() - t0
    t_eval = L * t_rot + t_sig + L * (2 * t_rot + t_gen) + t_rdm
    t_energy = L * t_rot + t_sig  # energy only: the ansatz and one sigma
    sample = ("%d of %d rotations and generator applications over the full %d-determinant sector, "
              "H psi on %d of %d determinants (scaled), full 1-RDM; scaled to one eval"
              % (ops_sample, L, sec.D, len(rows), sec.D))
    oracle_eval_sample.last = {"energy_only_evals_per_s": 1.0 / t_energy, "energy_grad_rdm_evals_per_s": 1.0 / t_eval,
                               "seconds": {"rotation": t_rot, "generator": t_gen, "sigma": t_sig, "rdm1": t_rdm}}
    return 1.0 / t_eval, sample, sec


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2405_11567_gb300 import inputs
    import oracle
    p = inputs.config_problem(CONFIG_ID)
    sec = None
    for _ in range(args.warmup):
        _, _, sec = oracle_eval_sample(p, sec, sigma_rows=1500, ops_sample=1)
    vals = []
    sample = ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, sample, sec = oracle_eval_sample(p, sec)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(statistics.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(p),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample, "wall_s": wall,
                         "energy_only_evals_per_s": oracle_eval_sample.last["energy_only_evals_per_s"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def problem(args):
    from paper_2405_11567_gb300 import inputs
    if args.qubits:
        ne = 2 * max(1, round(args.qubits / 6))
        return inputs.make_problem(args.qubits, ne, 200, 1000 + CONFIG_ID)
    return inputs.config_problem(CONFIG_ID)


def workload_config(p):
    return {"workload": "n%d_ne%d_adapt%d_synthetic" % (p["n_qubits"], p["n_elec"], len(p["ops"])),
            "n_qubits": p["n_qubits"], "n_electrons": p["n_elec"],
            "n_ops": int(len(p["ops"])), "seed": p["seed"],
            "step": "prepare_hf + energy_grad (forward, sigma, adjoint) + rdm1",
            "storage": "dense 2^30 amplitudes (8 GiB per vector, complex64); sector storage timed beside it",
            "l2": "flushed before every timed step (256 MB write outside the step's events)"}


# ---------------------------------------------------------------- our arm

def sigma_terms(p):
    """Hamiltonian connections applied by one sigma = (H - c) psi on the (na, nb) sector:
    every determinant has the same count (diagonal, singles and doubles of each spin,
    alpha-beta doubles)."""
    from math import comb
    N, na, nb = p["n_orb"], p["na"], p["nb"]
    D = comb(N, na) * comb(N, nb)
    sa, sb = na * (N - na), nb * (N - nb)
    per = 1 + sa + sb + comb(na, 2) * comb(N - na, 2) + comb(nb, 2) * comb(N - nb, 2) + sa * sb
    return D, per


def pool_pairs(pool, n_orb, na, nb):
    """Determinant pairs an operator screening visits: per fermionic operator (kind, i, j, a, b;
    i, j annihilated, a, b created) the alpha strings matching its alpha pattern times the beta
    strings matching its beta pattern, C(N - |touched|, n_sigma - |annihilated|) per spin."""
    from math import comb

    total = 0
    for op in pool:
        ann = [int(op[1])] + ([int(op[2])] if op[0] == 2 else [])
        cre = [int(op[3])] + ([int(op[4])] if op[0] == 2 else [])
        cnt = 1
        for spin, ne in ((0, na), (1, nb)):
            touched = len({j // 2 for j in ann + cre if j % 2 == spin})
            k = ne - sum(j % 2 == spin for j in ann)
            cnt *= comb(n_orb - touched, k) if 0 <= k <= n_orb - touched else 0
        total += cnt
    return total


def fp32_peak_tflops(sm_mhz):
    """Plain (non-tensor) FP32 FMA peak: 152 SMs x 128 lanes x 2 flops x the SM clock."""
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2405_11567_gb300 import build as libbuild
    from paper_2405_11567_gb300 import inputs, sv

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    p = problem(args)
    n, L = p["n_qubits"], len(p["ops"])
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    stream = torch.cuda.Stream()
    peak, peak_kind = measured_peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # 256 MB > 126 MB of L2

    def timed(dtype, sector):
        st = sv.StateVector(n, dtype, stream, sector=(p["na"], p["nb"]) if sector else None)
        st.set_option(sv.SV_OPT_PROFILE, 1)
        if args.expect_variant is not None:  # a fixed expectation form (profiling; with --no-autotune)
            st.set_option(sv.SV_OPT_EXPECT_VARIANT, args.expect_variant)
        outs = {}
        tuned = None
        if not args.no_autotune:  # launch choices timed on this problem, before any timed step
            st.prepare_hf(p["occ"])
            tuned = st.autotune(ham, p["ops"], p["theta"])

        def step():
            st.prepare_hf(p["occ"])
            E, g = st.energy_grad(ham, p["ops"], p["theta"])
            rdm = st.rdm1()  # host-synchronising reads: energy, gradient, 1-RDM
            outs["E"], outs["g"], outs["rdm"] = E, g, rdm
            return st.phase_times()

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = ClockSampler(local_rank)
        clocks.start()
        launches0 = st.launches
        phases, evs, t_host = [], [], 0.0
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # L2 flush between timed steps, outside the timed region
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t0 = time.perf_counter()
            phases.append(step())
            t_host += time.perf_counter() - t0
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        launches = st.launches - launches0
        clk = clocks.stop()
        if dist:
            dist.barrier()
        ms, t_host = reduce_max([ms, t_host])
        avg = {k: statistics.mean(ph[k] for ph in phases) for k in phases[0]}
        st.close()
        return dict(ms=ms, t_host=t_host, phases=avg, clocks=clk, launches=launches, out=outs, tuned=tuned)

    def timed_batch():
        """Config 4: 512 instances (10-20 qubits, 40 operators each), one graph launch per step."""
        probs = inputs.batch_problems(512)
        b = sv.Batch(probs, "c64", stream)
        theta = np.concatenate([q["theta"] for q in probs])
        grid = None if args.no_autotune else b.autotune(theta)
        for _ in range(args.warmup):
            b.energy_grad(theta)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = b.launches
        ev0.record(stream)
        for _ in range(args.steps):
            b.energy_grad(theta)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        out = {"workload": "512 instances, 10-20 qubits, 40-operator ADAPT-style ansatz each, complex64",
               "ms_per_batch": ms, "instance_evals_per_s": 512 / (ms / 1000.0),
               "gpu_launches_per_batch": (b.launches - l0) // args.steps, "autotuned_grid": grid}
        b.close()
        return out

    def timed_pool(dtype, sector, variant):
        """ADAPT operator screening: the gradient of every operator of the UCCSD pool from the HF
        reference (config 5: 3,500 operators) at the ansatz state, one sv_pool_gradients call."""
        pool = inputs.uccsd_pool(n, p["na"] + p["nb"])
        st = sv.StateVector(n, dtype, stream, sector=(p["na"], p["nb"]) if sector else None)
        st.set_option(sv.SV_OPT_POOL_VARIANT, variant)
        st.prepare_hf(p["occ"])
        st.apply_ansatz(p["ops"], p["theta"])
        for _ in range(args.warmup):
            E, g = st.pool_gradients(ham, pool)
        torch.cuda.synchronize()
        evs = []
        l0 = st.launches
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E, g = st.pool_gradients(ham, pool)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        out = {"ms_per_screening": ms, "operators": len(pool), "operators_per_s": len(pool) / (ms / 1000.0),
               "gpu_launches_per_screening": (st.launches - l0) // args.steps, "E": E,
               "max_abs_grad": float(np.max(np.abs(g)))}
        st.close()
        return out, g

    def pool_rows():
        rows = {}
        ref_g = None
        for label, dtype, sector, variant in (("dense_c64_lists", "c64", False, 2), ("sector_c64_lists", "c64", True, 2),
                                              ("sector_c64_scan", "c64", True, 1),
                                              ("sector_c128_lists", "c128", True, 2)):
            if (args.no_c128 and dtype == "c128") or (args.pool_storage == "sector" and not sector):
                continue
            r, g = timed_pool(dtype, sector, variant)
            if ref_g is None:
                ref_g, ref_label = g, label
            else:
                r["max_abs_dg_vs_" + ref_label] = float(np.max(np.abs(g - ref_g)))
            rows[label] = r
        pairs = pool_pairs(inputs.uccsd_pool(n, p["na"] + p["nb"]), p["n_orb"], p["na"], p["nb"])
        rows["pairs_per_screening"] = int(pairs)
        rows["workload"] = "UCCSD pool of %d operators from the HF reference, %d qubits, %d electrons" % (
            len(inputs.uccsd_pool(n, p["na"] + p["nb"])), n, p["na"] + p["nb"])
        return rows

    if args.pool_only:  # profiling runs: only the operator screening
        pr = pool_rows()
        if rank == 0:
            print(json.dumps({"profile": "pool-only (not the bench line)", "pool_screening": pr}), flush=True)
        return 0
    if args.batch_only:  # profiling runs: only the batched launch (config 4)
        rb = timed_batch()
        if rank == 0:
            print(json.dumps({"profile": "batch-only (not the bench line)", "batch_config4": rb}), flush=True)
        return 0
    if args.sector_only:  # profiling runs: only the sector-storage complex64 step, a few GB on the device
        so = timed("c64", sector=True)
        if rank == 0:
            print(json.dumps({"profile": "sector-only (not the bench line)", "ms_per_step": so["ms"] / args.steps,
                              "phases_ms": so["phases"], "tuned": so["tuned"]}), flush=True)
        return 0
    head = timed("c64", sector=False)
    head128 = None if args.no_c128 else timed("c128", sector=False)
    s64 = None if args.no_sector else timed("c64", sector=True)
    s128 = None if (args.no_sector or args.no_c128) else timed("c128", sector=True)
    r32d = None if args.no_real else timed("r32", sector=False)
    r32s = None if (args.no_real or args.no_sector) else timed("r32", sector=True)
    rbatch = None if (args.qubits or args.no_batch) else timed_batch()
    rpool = None if args.no_pool else pool_rows()
    if rank != 0:
        return 0
    K = args.steps
    value = throughput(world, K, head["ms"])
    e2e = throughput(world, K, 1000.0 * head["t_host"])
    # roofline of the dominant kernel (by phase time): algorithmic bytes per launch / mean launch time
    rot_bytes = touched_bytes(p["ops"], n, 8)
    kernels = {
        "adjoint_step": dict(phase="reverse", mult=2.0,
                             desc="fused adjoint step (k_adjoint): psi and lambda pairs, read + write"),
        "rotation": dict(phase="forward", mult=1.0, desc="excitation rotation (k_rotate): touched pairs, read + write"),
    }
    rows = {}
    for name, kd in kernels.items():
        t_launch = head["phases"][kd["phase"]] / L / 1000.0
        per_launch = kd["mult"] * rot_bytes.sum() / L
        a = per_launch / t_launch / 1e9
        rows[name] = {"achieved_gbs": a, "frac": a / peak, "mean_launch_ms": t_launch * 1e3,
                      "bytes_per_launch": per_launch, "launches_per_step": L, "desc": kd["desc"]}
    dom = max(kernels, key=lambda k: head["phases"][kernels[k]["phase"]])
    roof = {"bound": "hbm", "kernel": dom, "achieved": rows[dom]["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": rows[dom]["frac"], "traffic": ADJOINT_TRAFFIC_BYTES if dom == "adjoint_step" else None,
            "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": head["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "precision": "complex64 state, float64 reductions", "data": "synthetic",
        "config": workload_config(p),
        "roofline": roof,
        "kernels": rows,
        "phases_ms": head["phases"],
        "clocks": head["clocks"],
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(L * (20 + 8) + len(p["occ"]) * 4),
                "d2h_bytes_per_step": int((1 + L) * 8 + 2 * 2 * p["n_orb"] ** 2 * 8)},
        "gpu_launches": int(head["launches"]),
        "autotune": head["tuned"],
    }
    if head128 is not None:
        v128 = throughput(world, K, head128["ms"])
        line["fp64_state"] = {"value": v128, "ms_per_step": head128["ms"] / K, "phases_ms": head128["phases"],
                              "clocks": head128["clocks"]}
        line["speedup_fp32_over_fp64"] = value / v128
        line["fp32_vs_fp64"] = {
            "abs_dE": abs(head["out"]["E"] - head128["out"]["E"]),
            "max_abs_dg": float(np.max(np.abs(head["out"]["g"] - head128["out"]["g"]))),
            "max_abs_drdm": float(np.max(np.abs(head["out"]["rdm"] - head128["out"]["rdm"]))),
            "E_fp64": head128["out"]["E"]}
    if s64 is not None:
        # sector storage: a separate row (the state is 0.84% of 2^30 amplitudes and L2-resident), with the
        # expectation's two kernels against the plain FP32 FMA peak
        D, per = sigma_terms(p)
        flops = 4.0 * D * per  # complex amplitude x real matrix element = 2 FMA per connection
        t_sig = s64["phases"]["expectation"] / 1000.0
        sm_mhz = s64["clocks"].get("sm_mhz")
        fpeak = fp32_peak_tflops(sm_mhz)
        ach = flops / t_sig / 1e12
        sb = sector_touched_bytes(p["ops"], p["n_orb"], p["na"], p["nb"], 8)
        sv_form = int((s64["tuned"] or {}).get("expect_variant", s64.get("variant", 5)))
        t_rot = s64["phases"]["forward"] / L / 1000.0
        t_adj = s64["phases"]["reverse"] / L / 1000.0
        sect = {"storage": "sector: C(15,5)^2 = 9,018,009 amplitudes (72 MB complex64), L2-resident",
                "value": throughput(world, K, s64["ms"]), "unit": UNIT, "ms_per_step": s64["ms"] / K,
                "phases_ms": s64["phases"], "clocks": s64["clocks"], "gpu_launches": int(s64["launches"]),
                "roofline": {"bound": "alu", "kernel": SIGMA_KERNELS.get(sv_form, "expectation form %d" % sv_form),
                             "achieved": ach, "peak": fpeak, "unit": "TFLOP/s", "frac": ach / fpeak,
                             "traffic": SIGMA_TRAFFIC_BYTES.get(sv_form),
                             "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flops x %.0f MHz"
                                          % (sm_mhz or 2070.0),
                             "algorithmic": "%d determinants x %d connections x 4 flops = %.1f GFLOP"
                                            % (D, per, flops / 1e9)},
                "kernels": {"rotation_l": {"algorithmic_gbs": sb.sum() / L / t_rot / 1e9,
                                           "mean_launch_ms": t_rot * 1e3},
                            "adjoint_l": {"algorithmic_gbs": 2.0 * sb.sum() / L / t_adj / 1e9,
                                          "mean_launch_ms": t_adj * 1e3}},
                "autotune": s64["tuned"],
                "abs_dE_vs_dense_c64": abs(s64["out"]["E"] - head["out"]["E"]),
                "max_abs_dg_vs_dense_c64": float(np.max(np.abs(s64["out"]["g"] - head["out"]["g"])))}
        if s128 is not None:
            sect["fp64_state"] = {"value": throughput(world, K, s128["ms"]), "ms_per_step": s128["ms"] / K,
                                  "phases_ms": s128["phases"]}
            if head128 is not None:
                sect["abs_dE_vs_dense_c128"] = abs(s128["out"]["E"] - head128["out"]["E"])
        line["sector_storage"] = sect
    if r32d is not None:
        # real-amplitude float32 state (the real-angle ansatz keeps psi real): half the bytes per amplitude
        rb4 = touched_bytes(p["ops"], n, 4)
        t_adj = r32d["phases"]["reverse"] / L / 1000.0
        a = 2.0 * rb4.sum() / L / t_adj / 1e9
        real = {"state": "real float32 amplitudes, float64 reductions",
                "dense": {"value": throughput(world, K, r32d["ms"]), "ms_per_step": r32d["ms"] / K,
                          "phases_ms": r32d["phases"], "adjoint_step_gbs": a, "adjoint_step_frac": a / peak,
                          "abs_dE_vs_c64": abs(r32d["out"]["E"] - head["out"]["E"]),
                          "max_abs_dg_vs_c64": float(np.max(np.abs(r32d["out"]["g"] - head["out"]["g"])))}}
        if r32s is not None:
            real["sector"] = {"value": throughput(world, K, r32s["ms"]), "ms_per_step": r32s["ms"] / K,
                              "phases_ms": r32s["phases"]}
        line["real_state"] = real
    if rbatch is not None:
        line["batch_config4"] = rbatch
    if rpool is not None:
        line["pool_screening"] = rpool
    if world == 1 and not args.no_cpu_baseline and not args.qubits:
        import oracle
        v, sample, _ = oracle_eval_sample(p)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": sample,
                                "energy_only_evals_per_s": oracle_eval_sample.last["energy_only_evals_per_s"]}
    print(json.dumps(line), flush=True)
    return 0


def op_profile(args):
    """Per-operator rotation timing (CUDA events per launch) grouped by the operator's lowest
    address bit in the automatic storage layout: the cost of short contiguous runs."""
    import torch
    from paper_2405_11567_gb300 import build as libbuild
    from paper_2405_11567_gb300 import sv
    libbuild.build()
    p = problem(args)
    n = p["n_qubits"]
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    stream = torch.cuda.Stream()
    peak, _ = measured_peaks()
    out = {}
    for dtype in ("c64", "c128"):
        st = sv.StateVector(n, dtype, stream)
        st.prepare_hf(p["occ"])
        st.energy_grad(ham, p["ops"], p["theta"])          # picks the automatic layout
        lay = st.layout()
        st.set_option(sv.SV_OPT_LAYOUT_AUTO, 0)
        st.prepare_hf(p["occ"])
        groups = {}
        for k, op in enumerate(p["ops"]):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st.apply_ansatz(op[None, :], p["theta"][k:k + 1])
            e1.record(stream)
            torch.cuda.synchronize()
            kind = int(op[0])
            qs = [op[1], op[3]] if kind in (1, 3) else list(op[1:5])
            low = min(int(min(lay[q] for q in qs)), 5)
            b = touched_bytes(op[None, :], n, 8 if dtype == "c64" else 16)[0]
            groups.setdefault("%s, lowest address bit %s" % ("single" if kind in (1, 3) else "double",
                                                             ">=5" if low == 5 else low), []).append(
                b / (e0.elapsed_time(e1) / 1e3) / 1e9)
        out[dtype] = {k: {"ops": len(v), "median_gbs": float(np.median(v)), "frac_of_peak": float(np.median(v)) / peak}
                      for k, v in sorted(groups.items())}
        st.close()
    print(json.dumps({"op_profile": out, "workload": workload_config(p)["workload"], "peak_gbs": peak}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-c128", action="store_true", help="skip the complex128 comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (config 4) timing")
    ap.add_argument("--no-sector", action="store_true", help="skip the sector-storage timing")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch choices")
    ap.add_argument("--no-real", action="store_true", help="skip the real-amplitude (float32) timing")
    ap.add_argument("--no-pool", action="store_true", help="skip the operator-screening timing")
    ap.add_argument("--expect-variant", type=int, default=None, choices=[0, 1, 2, 3, 4, 5],
                    help="profiling: force an expectation form (SV_OPT_EXPECT_VARIANT); use with --no-autotune")
    ap.add_argument("--pool-only", action="store_true",
                    help="profiling: time only the operator screening (no bench line)")
    ap.add_argument("--pool-storage", choices=["all", "sector"], default="all",
                    help="operator screening rows: every storage, or sector storage only (no 2^n vector)")
    ap.add_argument("--batch-only", action="store_true",
                    help="profiling only: time just the batched launch (prints no bench line)")
    ap.add_argument("--sector-only", action="store_true",
                    help="profiling only: time just the sector-storage complex64 step (prints no bench line)")
    ap.add_argument("--op-profile", action="store_true",
                    help="per-operator rotation bandwidth by lowest address bit (diagnostic, not the bench line)")
    ap.add_argument("--qubits", type=int, default=0,
                    help="profiling only: a smaller register (same generator, n/3 rounded to even electrons, "
                         "200 operators); the bench line is then not the headline workload")
    args = ap.parse_args()
    rank, world, local_rank = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.op_profile:
        return op_profile(args)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group(backend="nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
