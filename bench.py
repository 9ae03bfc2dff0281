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
SIGMA_KERNELS = {
    3: "expectation: k_sigma_ab + k_sigma_same (two launches)",
    4: "expectation: k_phase_planar + k_transpose_pieces + k_same_tc (same-spin products, tcgen05 bf16x3) "
       "+ k_sigma_ab + k_sigma_comb",
    5: "expectation: k_phase_planar + k_transpose_pieces + k_same_tc (same-spin products) + k_ab_tc "
       "(alpha-beta products; both tcgen05 bf16x3) + k_sigma_comb (gathers the alpha-beta planes)"}
# Measured DRAM traffic lives in a small committed record written from ncu captures
# (--record-traffic), keyed by a hash of the sources of the kernels it measured: a
# record whose sources changed since is stale and the bench line reports null.
TRAFFIC_RECORDS = os.path.join(ROOT, "profiles", "traffic.json")
CSRC = "paper_2405_11567_gb300/csrc/"
TRAFFIC_SOURCES = {
    "dense_adjoint_c64": [CSRC + "k_state.cu", CSRC + "sv_device.cuh"],
    "sector_sigma_c64": [CSRC + "k_rows.cu", CSRC + "k_tcgemm.cu", CSRC + "k_abtc.cu", CSRC + "sv_sigma.cuh",
                         CSRC + "sv_device.cuh"],
}
GOLDEN = os.path.join(ROOT, "tests", "golden", "config5_oracle.json")
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 rate, nominal


def sources_sha256(paths):
    import hashlib
    h = hashlib.sha256()
    for rel in sorted(paths):
        h.update(rel.encode())
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_record(name):
    """The committed traffic record `name` if its kernel sources are unchanged, else None."""
    if not os.path.exists(TRAFFIC_RECORDS):
        return None
    with open(TRAFFIC_RECORDS) as f:
        rec = json.load(f).get(name)
    if rec is None or rec.get("sources_sha256") != sources_sha256(TRAFFIC_SOURCES[name]):
        return None
    return rec


def lowest_bit_class(b):
    return str(b) if b < 3 else "3+"


def op_qubits(op):
    kind = int(op[0])
    return [int(op[1]), int(op[3])] if kind in (1, 3) else [int(x) for x in op[1:5]]


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
    # one full evaluation takes the oracle tens of minutes at 30 qubits: each step times a bounded
    # sample of it (ms_per_step is that sample's measured wall time) and `value` is projected from it
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(p),
        "projected": {"value": value, "from": sample,
                      "projected_ms_per_eval": 1000.0 / value,
                      "note": "value is projected to one full evaluation; ms_per_step is the sample's wall time"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample, "wall_s": wall, "projected": True,
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
        layout = None if sector else [int(x) for x in st.layout()]
        variant = st.option(sv.SV_OPT_EXPECT_VARIANT)
        st.close()
        return dict(ms=ms, t_host=t_host, phases=avg, clocks=clk, launches=launches, out=outs, tuned=tuned,
                    layout=layout, variant=variant)

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
    if args.sector_only:  # profiling runs: only the sector-storage step, a few GB on the device
        so = timed(args.sector_dtype, sector=True)
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
                             desc="fused adjoint step (k_adjoint_i: psi and lambda interleaved in one buffer): "
                                  "psi and lambda pairs, read + write"),
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
    traffic, traffic_note = None, "no ncu record for the current kernel sources"
    rec = traffic_record("dense_adjoint_c64")
    if dom == "adjoint_step" and rec is not None and head["layout"] is not None:
        # the record's DRAM / algorithmic ratio of each lowest-address-bit class, weighted by this ansatz's ops
        ratio = rec["ratio_by_lowest_bit"]
        tb = 2.0 * rot_bytes
        cls = [lowest_bit_class(min(head["layout"][q] for q in op_qubits(op))) for op in p["ops"]]
        traffic = float(sum(t * ratio[c] for t, c in zip(tb, cls)) / L)
        traffic_note = "ncu DRAM bytes per launch by lowest-address-bit class (%s), weighted by this ansatz" % rec[
            "capture"]
    roof = {"bound": "hbm", "kernel": dom, "achieved": rows[dom]["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": rows[dom]["frac"], "traffic": traffic, "traffic_note": traffic_note,
            "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s"}
    golden = load_golden()
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
        "step_lower_bound": step_lower_bound(rot_bytes, n, 8, head["ms"] / K, peak),
    }
    if golden is not None:
        line["vs_oracle"] = vs_golden(head["out"], golden)
    if head128 is not None:
        v128 = throughput(world, K, head128["ms"])
        fp64 = fp64_peak(torch)
        line["fp64_state"] = {"value": v128, "ms_per_step": head128["ms"] / K, "phases_ms": head128["phases"],
                              "clocks": head128["clocks"],
                              "bound": fp64_rooflines(p, head128["phases"], fp64, peak, head128["variant"]),
                              "expectation_form": head128["variant"],
                              "vs_oracle": vs_golden(head128["out"], golden) if golden is not None else None}
        line["speedup_fp32_over_fp64"] = value / v128
        line["speedup_bounds"] = {
            "complex64": "HBM: the sweeps move their bytes at %.2f (reverse) / %.2f (forward) of the copy peak"
                         % (rows["adjoint_step"]["frac"], rows["rotation"]["frac"]),
            "complex128": "the sweeps on the FP64 pipe (fp64_state.bound: FP64 flops / time against the "
                          "measured FP64 rate), the expectation in float-float arithmetic on the FP32 pipe; the "
                          "byte ratio alone would give 2x"}
        line["fp32_vs_fp64"] = {
            "abs_dE": abs(head["out"]["E"] - head128["out"]["E"]),
            "max_abs_dg": float(np.max(np.abs(head["out"]["g"] - head128["out"]["g"]))),
            "max_abs_drdm": float(np.max(np.abs(head["out"]["rdm"] - head128["out"]["rdm"]))),
            "E_fp64": head128["out"]["E"]}
    if s64 is not None:
        line["sector_storage"] = sector_row(p, s64, s128, head, head128, world, K, L, golden)
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
        if not args.no_per_config:
            # configs 1-4 (their GPU rows are latency-bound: timed before the 30-qubit oracle sample below,
            # whose host work and memory would otherwise sit beside them)
            pc_clocks = ClockSampler(local_rank)
            pc_clocks.start()
            line["per_config"] = per_config_rows(args, stream, peak, rbatch)
            line["per_config"]["clocks"] = pc_clocks.stop()
        t0 = time.perf_counter()
        v, sample, _ = oracle_eval_sample(p)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": sample, "projected": True, "sample_wall_s": time.perf_counter() - t0,
                                "energy_only_evals_per_s": oracle_eval_sample.last["energy_only_evals_per_s"]}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- bench-line helpers

def load_golden():
    """The oracle's 30-qubit energy, gradient and 1-RDM (tests/golden, written by the oracle alone)."""
    if not os.path.exists(GOLDEN):
        return None
    with open(GOLDEN) as f:
        return json.load(f)


def vs_golden(out, golden):
    rdm = np.array(golden["rdm1_re"]) + 1j * np.array(golden["rdm1_im"])
    return {"abs_dE": abs(out["E"] - golden["energy"]),
            "max_abs_dg": float(np.max(np.abs(np.asarray(out["g"]) - np.array(golden["gradient"])))),
            "max_abs_drdm": float(np.max(np.abs(np.asarray(out["rdm"]) - rdm))),
            "oracle": "tests/golden/config5_oracle.json (route A, complex128, %d threads, %.0f s)"
                      % (golden["oracle_threads"], golden["seconds"])}


def fp64_peak(torch):
    """FP64 throughput measured in this run: a 4096^3 float64 matrix product (cuBLAS) on the GPU, best of 3."""
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    best = None
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return 2.0 * 4096 ** 3 / (best / 1e3) / 1e12


def fp64_rooflines(p, phases, fp64_tflops, hbm_peak, variant=None):
    """complex128 sweeps against the FP64 pipe and HBM: FP64 flops per amplitude pair = 12 in the rotation
    (three shears of the real and imaginary parts, six FMAs) and 32 in the adjoint step (two rotations plus
    four FMAs of the gradient term).  The expectation: 4 flops of float64 work per Hamiltonian connection
    (complex amplitude x real element, two FMAs) -- on the FP64 pipe (form 3), or in float-float arithmetic
    on the FP32 pipe (form 6, about 12 FP32 operations per float64 multiply-add)."""
    n, L = p["n_qubits"], len(p["ops"])
    kind = np.asarray(p["ops"])[:, 0]
    pairs = np.where((kind == 1) | (kind == 3), 2.0 ** (n - 2), 2.0 ** (n - 4)).sum()
    D, per = sigma_terms(p)
    out = {"fp64_peak_tflops": fp64_tflops,
           "fp64_peak_kind": "measured in this run: 4096^3 float64 matmul (cuBLAS), best of 4; nominal %.2f"
                             % FP64_NOMINAL_TFLOPS}
    tb = touched_bytes(p["ops"], n, 16).sum()
    for name, phase, flops_per_pair, mult in (("rotation", "forward", 12.0, 1.0),
                                              ("adjoint_step", "reverse", 32.0, 2.0)):
        t = phases[phase] / 1000.0
        tf = flops_per_pair * pairs / t / 1e12
        gbs = mult * tb / t / 1e9
        out[name] = {"bound": "fp64", "achieved_tflops": tf, "frac_fp64": tf / fp64_tflops,
                     "hbm_gbs": gbs, "frac_hbm": gbs / hbm_peak, "flops_per_pair": flops_per_pair,
                     "pairs_per_sweep": pairs, "mean_launch_ms": phases[phase] / L}
    t = phases["expectation"] / 1000.0
    tf = 4.0 * D * per / t / 1e12
    if variant == 6:
        ops = 2.0 * D * per * 12.0  # float-float multiply-adds, ~12 FP32 operations each
        fp32 = fp32_ops_peak()
        out["expectation"] = {
            "form": "float-float split (variant 6): float64 values as two float32 words, FP32 pipe",
            "bound": "shared memory (staged partner rows, 16 bytes per complex amplitude)",
            "fp64_work_tflops": tf, "fp64_work_frac_of_fp64_peak": tf / fp64_tflops,
            "fp32_ops_per_s": ops / t / 1e12, "fp32_ops_frac": ops / t / 1e12 / fp32,
            "algorithmic": "%d determinants x %d connections x 4 flops of float64 work" % (D, per)}
    else:
        out["expectation"] = {"form": "float64 split (variant %s)" % variant, "bound": "fp64",
                              "achieved_tflops": tf, "frac_fp64": tf / fp64_tflops,
                              "algorithmic": "%d determinants x %d connections x 4 flops" % (D, per)}
    return out


def fp32_ops_peak(sm_mhz=2070.0):
    """FP32 pipe issue rate in tera-operations per second (an FMA counts once): 152 SMs x 128 lanes x clock."""
    return 152 * 128 * sm_mhz * 1e6 / 1e12


def mma_flops(p, planes=2):
    """bf16 tensor-core flops the two tcgen05 kernels issue per sigma: k_same_tc, tiles of 128 x 256 over
    K blocks of 32 (both products, six piece products); k_ab_tc, units of 128 alpha strings x one partner beta
    string, N = 64 columns over K blocks of 16 (six piece products per plane)."""
    from math import comb
    N, na, nb = p["n_orb"], p["na"], p["nb"]
    Da, Db = comb(N, na), comb(N, nb)
    cdiv = lambda a, b: (a + b - 1) // b  # noqa: E731
    same = cdiv(Db, 256) * cdiv(Da, 128) * planes * (cdiv(Da, 32) + cdiv(Db, 32)) * 6 * 2.0 * 128 * 256 * 32
    units = cdiv(Da, 128) * Db
    ab = units * planes * cdiv(N * (N + 1) // 2, 16) * 6 * 2.0 * 128 * 64 * 16
    return same, ab


def sector_row(p, s64, s128, head, head128, world, K, L, golden):
    """Sector storage (the state is 0.84% of 2^30 amplitudes and L2-resident): its own row, with the
    tensor-core expectation kernels against the tensor pipe's measured bf16 peak."""
    D, per = sigma_terms(p)
    useful = 4.0 * D * per  # complex amplitude x real matrix element = 2 FMA per connection
    ph = s64["phases"]
    peaks = measured_tensor_peaks()
    same, ab = mma_flops(p)
    kern = {}
    if ph.get("same_products", 0) > 0:
        kern["k_same_tc"] = {"mma_tflop": same / 1e12, "ms": ph["same_products"],
                             "achieved_tflops": same / (ph["same_products"] / 1e3) / 1e12,
                             "note": "includes k_transpose_pieces"}
    if ph.get("ab_products", 0) > 0:
        kern["k_ab_tc"] = {"mma_tflop": ab / 1e12, "ms": ph["ab_products"],
                           "achieved_tflops": ab / (ph["ab_products"] / 1e3) / 1e12}
    roof = None
    if kern:
        dom = max(kern, key=lambda k: kern[k]["ms"])
        rec = traffic_record("sector_sigma_c64")
        roof = {"bound": "tensor", "kernel": dom, "achieved": kern[dom]["achieved_tflops"],
                "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": kern[dom]["achieved_tflops"] /
                peaks["bf16_tflops"], "peak_kind": peaks["kind"],
                "traffic": (rec["bytes_per_launch"].get(dom) if rec else None),
                "traffic_note": ("ncu DRAM bytes of one launch (%s)" % rec["capture"]) if rec else
                "no ncu record for the current kernel sources",
                "algorithmic": "bf16 MMA flops issued per launch (six bf16 piece products per float32 product)"}
    t_sig = ph["expectation"] / 1000.0
    sb = sector_touched_bytes(p["ops"], p["n_orb"], p["na"], p["nb"], 8)
    t_rot = ph["forward"] / L / 1000.0
    t_adj = ph["reverse"] / L / 1000.0
    rec = traffic_record("sector_sigma_c64")
    sect = {"storage": "sector: C(15,5)^2 = 9,018,009 amplitudes (72 MB complex64), L2-resident",
            "value": throughput(world, K, s64["ms"]), "unit": UNIT, "ms_per_step": s64["ms"] / K,
            "phases_ms": ph, "clocks": s64["clocks"], "gpu_launches": int(s64["launches"]),
            "expectation_form": SIGMA_KERNELS.get(s64["variant"], "expectation form %d" % s64["variant"]),
            "roofline": roof, "tensor_kernels": kern,
            "useful": {"tflops": useful / t_sig / 1e12, "gflop": useful / 1e9,
                       "algorithmic": "%d determinants x %d connections x 4 flops of sparse work per sigma"
                                      % (D, per)},
            "sigma_traffic_bytes": rec["bytes_per_sigma"] if rec else None,
            "kernels": {"rotation_l": {"algorithmic_gbs": sb.sum() / L / t_rot / 1e9, "mean_launch_ms": t_rot * 1e3},
                        "adjoint_l": {"algorithmic_gbs": 2.0 * sb.sum() / L / t_adj / 1e9,
                                      "mean_launch_ms": t_adj * 1e3}},
            "autotune": s64["tuned"],
            "abs_dE_vs_dense_c64": abs(s64["out"]["E"] - head["out"]["E"]),
            "max_abs_dg_vs_dense_c64": float(np.max(np.abs(s64["out"]["g"] - head["out"]["g"])))}
    if golden is not None:
        sect["vs_oracle"] = vs_golden(s64["out"], golden)
    if s128 is not None:
        sect["fp64_state"] = {"value": throughput(world, K, s128["ms"]), "ms_per_step": s128["ms"] / K,
                              "phases_ms": s128["phases"],
                              "vs_oracle": vs_golden(s128["out"], golden) if golden is not None else None}
        if head128 is not None:
            sect["abs_dE_vs_dense_c128"] = abs(s128["out"]["E"] - head128["out"]["E"])
    return sect


def measured_tensor_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"bf16_tflops": float(d["bf16_tflops"]), "kind": "measured burst (MEASURED_PEAKS.json bf16_tflops)"}
    return {"bf16_tflops": 1900.0, "kind": "fallback 1.9 PFLOP/s bf16 burst"}


def step_lower_bound(rot_bytes, n, amp_bytes, ms_step, peak):
    """The whole evaluation against its algorithmic lower bound: the forward sweep's touched bytes, twice that for
    the adjoint sweep (psi and lambda), two reads of the state and one write (energy, sigma) -- the bytes the dense
    method must move -- at the measured copy peak, against the measured step time."""
    state = float(2 ** n * amp_bytes)
    fwd = float(rot_bytes.sum())
    total = fwd + 2.0 * fwd + 3.0 * state
    t_lb = total / (peak * 1e9) * 1e3
    return {"bytes": total, "ms_at_peak": t_lb, "ms_measured": ms_step, "frac": t_lb / ms_step,
            "terms": "forward touched bytes + 2 x forward (adjoint on psi and lambda) + 2 state reads + 1 state write"}


def oracle_seconds(fn, budget_s=2.0):
    """Wall seconds of one oracle call: where a call takes under a quarter of the budget, the median of up to
    five calls after a first (warm-up) call; else the first call itself.  Returns (seconds, result, calls timed)."""
    t0 = time.perf_counter()
    res = fn()
    t1 = time.perf_counter() - t0
    if t1 >= budget_s / 4:
        return t1, res, 1
    reps = int(max(1, min(5, budget_s / max(t1, 1e-6))))
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        res = fn()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts)), res, reps


def per_config_rows(args, stream, peak, rbatch):
    """Configs 1-4 beside the headline: GPU evaluations per second (dense storage, the workload's own
    dtype; CUDA events, after warm-up) with the roof that binds them, and the CPU oracle timed on full
    evaluations -- energy only and energy + gradient (+ 1-RDM for config 3) separately, after a warm-up call
    where a call is short (oracle_seconds) -- with the GPU results' deviation from it.  Config 4: the oracle over all 512 instances (energy + gradient)."""
    import torch
    import oracle
    from oracle import route_a as A
    from paper_2405_11567_gb300 import inputs, sv
    out = {"cores": oracle.num_threads()}
    roofs = {1: "launch latency: 4 KiB state, 15 one-launch operators (microseconds each)",
             2: "launch latency / L2: 1 MiB state, 198 operators",
             3: "L2 / HBM: 128 MiB (complex64) and 256 MiB (complex128) vectors against a 126 MB L2"}
    for cid, dtypes in ((1, ("c128",)), (2, ("c128",)), (3, ("c64", "c128"))):
        p = inputs.config_problem(cid)
        n, L = p["n_qubits"], len(p["ops"])
        with_grad, with_rdm = cid >= 2, cid == 3
        sec = oracle.Sector(n, p["na"], p["nb"])
        psi0 = A.hf_state(sec, p["occ"])
        def o_energy():
            ps = A.apply_ansatz(sec, p["ops"], p["theta"], psi0)
            return ps, A.energy(sec, p["h"], p["eri"], p["e_nuc"], ps)

        t_e, (psi, E_o), n_e = oracle_seconds(o_energy)
        row = {"workload": "n%d_ne%d_%s_%s" % (n, p["n_elec"], "uccsd" if cid < 3 else "adapt%d" % L,
                                               "/".join(dtypes)),
               "oracle": {"energy_only_s": t_e, "energy_only_evals_per_s": 1.0 / t_e, "energy_only_calls": n_e},
               "gpu": {}, "binding_roof": roofs[cid]}
        g_o = rdm_o = None
        if with_grad:
            def o_grad():
                _, gg = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], psi0)
                return gg, (A.rdm1(sec, psi) if with_rdm else None)

            t_g, (g_o, rdm_o), n_g = oracle_seconds(o_grad)
            row["oracle"].update({"energy_grad_s": t_g, "energy_grad_evals_per_s": 1.0 / t_g,
                                  "energy_grad_calls": n_g, "includes_rdm1": with_rdm})
        ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
        for dtype in dtypes:
            st = sv.StateVector(n, dtype, stream)
            res = {}

            def energy_only():
                st.prepare_hf(p["occ"])
                st.apply_ansatz(p["ops"], p["theta"])
                return st.energy(ham)

            def full():
                st.prepare_hf(p["occ"])
                E, g = st.energy_grad(ham, p["ops"], p["theta"])
                r = st.rdm1() if with_rdm else None
                return E, g, r

            for name, fn in (("energy_only", energy_only),) + ((("energy_grad", full),) if with_grad else ()):
                for _ in range(3):
                    fn()
                torch.cuda.synchronize()
                k = 20 if cid < 3 else 5
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(k):
                    r = fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / k
                res[name] = {"ms": ms, "evals_per_s": 1000.0 / ms}
                if name == "energy_only":
                    res[name]["abs_dE_vs_oracle"] = abs(r - E_o)
                    # its two parts, timed the same way: preparation + ansatz, then the expectation alone
                    e0.record(stream)
                    for _ in range(k):
                        st.prepare_hf(p["occ"])
                        st.apply_ansatz(p["ops"], p["theta"])
                    e1.record(stream)
                    torch.cuda.synchronize()
                    res[name]["prepare_ansatz_ms"] = e0.elapsed_time(e1) / k
                    e0.record(stream)
                    for _ in range(k):
                        st.energy(ham)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    res[name]["expectation_ms"] = e0.elapsed_time(e1) / k
                else:
                    res[name]["abs_dE_vs_oracle"] = abs(r[0] - E_o)
                    res[name]["max_abs_dg_vs_oracle"] = float(np.max(np.abs(r[1] - g_o)))
                    if with_rdm:
                        res[name]["max_abs_drdm_vs_oracle"] = float(np.max(np.abs(r[2] - rdm_o)))
            if cid == 3 and "energy_grad" in res:
                tb = touched_bytes(p["ops"], n, 8 if dtype == "c64" else 16).sum()
                res["sweeps_algorithmic_gbs"] = 3.0 * tb / (res["energy_grad"]["ms"] / 1e3) / 1e9
                res["sweeps_frac_of_hbm_peak"] = res["sweeps_algorithmic_gbs"] / peak
            row["gpu"][dtype] = res
            st.close()
        ham.close()
        if cid < 3:
            # the same evaluation (energy and gradient) as one instance of the persistent batched engine:
            # one graph launch per call, the state in shared memory
            b = sv.Batch([p], "c128", stream)
            for _ in range(3):
                b.energy_grad(p["theta"])
            torch.cuda.synchronize()
            k = 50
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                E_b, g_b = b.energy_grad(p["theta"])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            rb = {"ms": ms, "evals_per_s": 1000.0 / ms, "abs_dE_vs_oracle": abs(float(E_b[0]) - E_o),
                  "note": "energy + gradient of this one instance through sv_batch_energy_grad"}
            if g_o is not None:
                rb["max_abs_dg_vs_oracle"] = float(np.max(np.abs(g_b[0] - g_o)))
            row["gpu"]["c128_batched_engine"] = rb
            b.close()
        out["config%d" % cid] = row
    # config 4: the oracle over every instance of the batch
    probs = inputs.batch_problems(512)
    t0 = time.perf_counter()
    for q in probs:
        sec = oracle.Sector(q["n_qubits"], q["na"], q["nb"])
        A.energy_grad(sec, q["h"], q["eri"], q["e_nuc"], q["ops"], q["theta"], A.hf_state(sec, q["occ"]))
    t_b = time.perf_counter() - t0
    row = {"oracle": {"energy_grad_s_all_512": t_b, "instance_evals_per_s": 512 / t_b},
           "binding_roof": "shared memory and barriers inside one block per instance (persistent launch)"}
    if rbatch is not None:
        row["gpu"] = {"ms_per_batch": rbatch["ms_per_batch"], "instance_evals_per_s": rbatch["instance_evals_per_s"]}
    out["config4"] = row
    return out


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


def traffic_probe(args):
    """One dense complex64 energy + gradient evaluation (no autotuning, no warm-up) at --qubits: the
    reverse sweep's k_adjoint_i launches are the op list backwards.  Writes, per launch, the op, its lowest
    address bit in the automatic layout and its algorithmic bytes, plus up to two launches of each
    lowest-bit class to capture (ncu -k regex:k_adjoint_i -s <launch> -c 1)."""
    import torch
    from paper_2405_11567_gb300 import build as libbuild
    from paper_2405_11567_gb300 import sv
    libbuild.build()
    if not args.qubits:
        args.qubits = 26
    p = problem(args)
    n, L = p["n_qubits"], len(p["ops"])
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = sv.StateVector(n, "c64")
    st.prepare_hf(p["occ"])
    st.energy_grad(ham, p["ops"], p["theta"])
    torch.cuda.synchronize()
    lay = [int(x) for x in st.layout()]
    tb = 2.0 * touched_bytes(p["ops"], n, 8)
    launches, pick = [], {}
    for j in range(L):
        k = L - 1 - j
        b = min(lay[q] for q in op_qubits(p["ops"][k]))
        launches.append({"launch": j, "op": k, "lowest_bit": b, "alg_bytes": float(tb[k]),
                         "kind": int(p["ops"][k][0])})
        c = lowest_bit_class(b)
        if int(p["ops"][k][0]) in (2, 4) and len(pick.setdefault(c, [])) < 2:
            pick[c].append(j)
    out = {"workload": workload_config(p)["workload"], "layout": lay, "launches": launches,
           "capture": sorted(j for v in pick.values() for j in v)}
    with open(args.traffic_probe, "w") as f:
        json.dump(out, f)
    print(" ".join(str(j) for j in out["capture"]))
    return 0


def _ncu_rows(path):
    """(kernel name, metric name -> value in base units) per captured launch of an ncu --csv log."""
    import csv
    rows = {}
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        key = (r["ID"], r["Kernel Name"])
        v = r["Metric Value"].replace(",", "")
        try:
            rows.setdefault(key, {})[r["Metric Name"]] = float(v)
        except ValueError:
            pass
    return rows


def record_traffic(argv):
    """Write one record of profiles/traffic.json from ncu captures (--metrics dram__bytes_read.sum,
    dram__bytes_write.sum,gpu__time_duration.sum --print-units base --csv), keyed by the current hash of the
    measured kernels' sources."""
    import re
    what, files = argv[0], argv[1:]
    recs = {}
    if os.path.exists(TRAFFIC_RECORDS):
        with open(TRAFFIC_RECORDS) as f:
            recs = json.load(f)
    if what == "dense":
        with open(files[0]) as f:
            probe = json.load(f)
        # DRAM reads / the algorithmic reads of the launch, per lowest-address-bit class.  The kernel
        # writes back exactly the sectors it read; a capture of a few-GB problem undercounts the writes
        # (lines still dirty in L2 when the kernel ends), so traffic = 2 x reads is recorded.
        per, wr = {}, {}
        for path in files[1:]:
            j = int(re.search(r"_(\d+)\.csv$", path).group(1))
            (key, m), = _ncu_rows(path).items()
            ln = probe["launches"][j]
            c = lowest_bit_class(ln["lowest_bit"])
            per.setdefault(c, []).append(2.0 * m["dram__bytes_read.sum"] / ln["alg_bytes"])
            wr.setdefault(c, []).append(2.0 * m["dram__bytes_write.sum"] / ln["alg_bytes"])
        ratio = {c: float(np.mean(v)) for c, v in per.items()}
        recs["dense_adjoint_c64"] = {
            "kernel": "k_adjoint_i (complex64)", "ratio_by_lowest_bit": ratio,
            "write_ratio_by_lowest_bit_as_captured": {c: float(np.mean(v)) for c, v in wr.items()},
            "launches_per_class": {c: len(v) for c, v in per.items()},
            "capture": "%s, %d launches" % (probe["workload"], sum(len(v) for v in per.values())),
            "ratio": "2 x DRAM read bytes / algorithmic bytes (reads and write-backs move the same sectors)",
            "sources_sha256": sources_sha256(TRAFFIC_SOURCES["dense_adjoint_c64"])}
    elif what == "sector":
        rows = _ncu_rows(files[0])
        by = {}
        for (rid, name), m in rows.items():
            nm = name.replace("<unnamed>::", "").replace("(anonymous namespace)::", "")
            base = re.sub(r"<.*", "", nm.split("(")[0]).strip().split()[-1].split("::")[-1]
            by[base] = by.get(base, 0.0) + m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"]
        recs["sector_sigma_c64"] = {
            "kernels": sorted(by), "bytes_per_launch": by, "bytes_per_sigma": float(sum(by.values())),
            "capture": "30 qubits, sector storage, complex64, one launch of each expectation kernel",
            "sources_sha256": sources_sha256(TRAFFIC_SOURCES["sector_sigma_c64"])}
    else:
        raise SystemExit("--record-traffic dense PROBE CSV... | sector CSV")
    with open(TRAFFIC_RECORDS, "w") as f:
        json.dump(recs, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(recs, indent=1))
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
    ap.add_argument("--sector-dtype", choices=["c64", "c128"], default="c64",
                    help="state type of --sector-only (profiling)")
    ap.add_argument("--op-profile", action="store_true",
                    help="per-operator rotation bandwidth by lowest address bit (diagnostic, not the bench line)")
    ap.add_argument("--no-per-config", action="store_true",
                    help="skip the per-config block (configs 1-4 on the GPU and the oracle timed on full evaluations)")
    ap.add_argument("--traffic-probe", metavar="OUT_JSON", default=None,
                    help="profiling only: one dense complex64 energy_grad at --qubits (default 26), no autotuning; "
                         "writes the reverse sweep's launches (op, lowest address bit, algorithmic bytes) to OUT_JSON")
    ap.add_argument("--record-traffic", nargs="+", metavar="FILE", default=None,
                    help="write the traffic record of profiles/traffic.json from ncu CSV captures: "
                         "'dense PROBE_JSON CSV...' (one k_adjoint_i launch per CSV, named ..._<launch>.csv) or "
                         "'sector CSV' (one launch of each expectation kernel)")
    ap.add_argument("--qubits", type=int, default=0,
                    help="profiling only: a smaller register (same generator, n/3 rounded to even electrons, "
                         "200 operators); the bench line is then not the headline workload")
    args = ap.parse_args()
    rank, world, local_rank = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.record_traffic:
        return record_traffic(args.record_traffic)
    if args.traffic_probe:
        return traffic_probe(args)
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
