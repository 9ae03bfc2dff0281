"""Write the oracle's values for the full-size parity test (30 qubits, config 5).

Calls only the CPU oracle (route A) on the seeded inputs of
``paper_2405_11567_gb300.inputs``; nothing here comes from the CUDA path.  The
output, ``config5_oracle.json``, holds the energy, the 200 gradient entries, the
1-RDM, the amplitudes of psi(theta) at 4096 seeded sample determinants and a
fingerprint of the inputs (so a test can tell whether the generator still draws
the same numbers on its machine).  Takes tens of minutes on 8 cores.

    python tests/golden/make_golden.py [--config 5]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import route_a as A  # noqa: E402
from paper_2405_11567_gb300 import inputs  # noqa: E402


def fingerprint(p) -> dict:
    """Input checks: operators and angles are drawn directly (exact on any machine); the
    two-electron integrals are an einsum whose last bits depend on the platform's
    summation order, so only their checksums are kept (compared to 1e-12 relative)."""
    def sha(a):
        return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
    eri = np.asarray(p["eri"], dtype=np.float64)
    return {"ops_sha256": sha(np.asarray(p["ops"], dtype=np.int32)),
            "theta_sha256": sha(np.asarray(p["theta"], dtype=np.float64)),
            "h_sha256": sha(np.asarray(p["h"], dtype=np.float64)),
            "eri_sum": float(eri.sum()), "eri_abs_sum": float(np.abs(eri).sum()),
            "eri_sq_sum": float((eri * eri).sum())}


def same_inputs(fp_here: dict, fp_gold: dict) -> bool:
    exact = all(fp_here[k] == fp_gold[k] for k in ("ops_sha256", "theta_sha256", "h_sha256"))
    close = all(abs(fp_here[k] - fp_gold[k]) <= 1e-12 * max(1.0, abs(fp_gold[k]))
                for k in ("eri_sum", "eri_abs_sum", "eri_sq_sum"))
    return exact and close


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--refingerprint", action="store_true",
                    help="only rewrite the input fingerprint of an existing file (no oracle run)")
    args = ap.parse_args()
    p = inputs.config_problem(args.config)
    path = os.path.join(HERE, "config%d_oracle.json" % args.config)
    if args.refingerprint:
        with open(path) as f:
            out = json.load(f)
        out["fingerprint"] = fingerprint(p)
        with open(path, "w") as f:
            json.dump(out, f)
        print(path, "fingerprint rewritten")
        return
    t0 = time.time()
    sec = oracle.Sector(p["n_qubits"], p["na"], p["nb"])
    psi0 = A.hf_state(sec, p["occ"])
    psi = A.apply_ansatz(sec, p["ops"], p["theta"], psi0)
    E, g = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], psi0)
    rdm = A.rdm1(sec, psi)
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(sec.D, size=min(4096, sec.D), replace=False))
    # the largest-weight determinants as well (where complex64 rounding matters most)
    top = np.argsort(-np.abs(psi))[:256]
    idx = np.unique(np.concatenate([idx, top]))
    out = {
        "what": "CPU oracle (route A) on config %d; written by tests/golden/make_golden.py" % args.config,
        "config": args.config, "n_qubits": p["n_qubits"], "n_elec": p["n_elec"], "n_ops": int(len(p["ops"])),
        "fingerprint": fingerprint(p),
        "energy": E, "gradient": list(map(float, g)),
        "rdm1_re": np.asarray(rdm.real).tolist(), "rdm1_im": np.asarray(rdm.imag).tolist(),
        "sample_x": [int(sec.dets[i]) for i in idx],
        "sample_re": [float(psi[i].real) for i in idx], "sample_im": [float(psi[i].imag) for i in idx],
        "oracle_threads": oracle.num_threads(), "seconds": time.time() - t0,
    }
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, "E = %.12f" % E, "%.0f s" % out["seconds"])


if __name__ == "__main__":
    main()
