"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own replica
("replicas only": the path does not shard), rank 0 reporting the evaluations of all
ranks over the slowest rank's time.  The reference arm runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, host = bench.reduce_max([100.0 * (rank + 1), 2.0 - rank])   # rank 1 is the slow device, rank 0 the slow host
    value = bench.throughput(world, 5, ms)
    # the reference arm: only rank 0 works, the others return at once
    import argparse
    other = bench.run_reference(argparse.Namespace(steps=1, warmup=0, gpus=world), rank, world) if rank else None
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, host, value, other))


def test_two_gloo_ranks_take_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, host, value, other in out:
        assert ms == 200.0 and host == 2.0                 # max over ranks, on every rank
        assert abs(value - 2 * 5 / 0.2) < 1e-9             # all ranks' evaluations over the slowest time
    assert out[1][4] == 0                                  # reference arm: rank 1 exits without work


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3.0, 4.0]) == [3.0, 4.0]
    assert bench.throughput(1, 4, 2000.0) == 2.0


def test_sigma_connection_count_brute_force():
    """bench.sigma_terms (the algorithmic FLOP count of one expectation) against a brute-force
    count of the sector determinants within two excitations of each determinant."""
    sys.path.insert(0, ROOT)
    import itertools
    import bench
    for N, na, nb in [(5, 2, 1), (4, 2, 2), (6, 3, 2), (3, 0, 2)]:
        sa = [sum(1 << (2 * q) for q in c) for c in itertools.combinations(range(N), na)]
        sb = [sum(1 << (2 * q + 1) for q in c) for c in itertools.combinations(range(N), nb)]
        dets = [a | b for a in sa for b in sb]
        counts = {sum(1 for y in dets if bin(x ^ y).count("1") <= 4) for x in dets}
        D, per = bench.sigma_terms({"n_orb": N, "na": na, "nb": nb})
        assert D == len(dets) and counts == {per}
    assert bench.sigma_terms({"n_orb": 15, "na": 5, "nb": 5}) == (9018009, 3501)


def test_pool_pair_count_brute_force():
    """bench.pool_pairs (the pairs one operator screening visits) against a count of the sector
    determinants on which each pool operator's excitation does not vanish."""
    sys.path.insert(0, ROOT)
    import itertools
    import bench
    from paper_2405_11567_gb300 import inputs
    for N, na, nb, ne_pool in [(5, 2, 1, 3), (4, 2, 2, 4), (6, 3, 2, 4), (5, 1, 3, 4)]:
        sa = [sum(1 << (2 * q) for q in c) for c in itertools.combinations(range(N), na)]
        sb = [sum(1 << (2 * q + 1) for q in c) for c in itertools.combinations(range(N), nb)]
        dets = [a | b for a in sa for b in sb]
        pool = inputs.uccsd_pool(2 * N, ne_pool)
        want = 0
        for op in pool:
            ann = [int(op[1])] + ([int(op[2])] if op[0] == 2 else [])
            cre = [int(op[3])] + ([int(op[4])] if op[0] == 2 else [])
            want += sum(1 for x in dets if all(x >> j & 1 for j in ann) and not any(x >> j & 1 for j in cre))
        assert bench.pool_pairs(pool, N, na, nb) == want


def _pattern_count(xs, op):
    """Amplitudes an excitation rotates among the basis indices xs: those holding its
    annihilated spin-orbitals and not its created ones, and their partners."""
    ann = [int(op[1])] + ([int(op[2])] if op[0] in (2, 4) else [])
    cre = [int(op[3])] + ([int(op[4])] if op[0] in (2, 4) else [])
    fwd = sum(1 for x in xs if all(x >> j & 1 for j in ann) and not any(x >> j & 1 for j in cre))
    bwd = sum(1 for x in xs if all(x >> j & 1 for j in cre) and not any(x >> j & 1 for j in ann))
    return fwd + bwd


def test_touched_bytes_brute_force():
    """bench.touched_bytes (the algorithmic bytes of the headline's rotation and adjoint
    kernels: read + write of every amplitude a rotation pairs) against a count over all
    2^n basis indices, for fermionic and qubit singles and doubles."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    n = 8
    xs = range(1 << n)
    ops = np.array([[1, 0, 0, 4, 0], [1, 3, 0, 7, 0], [2, 0, 2, 4, 6], [2, 1, 3, 5, 7], [2, 0, 1, 2, 3],
                    [3, 2, 0, 6, 0], [4, 0, 1, 6, 7]], dtype=np.int32)
    got = bench.touched_bytes(ops, n, 8)
    want = [2 * _pattern_count(xs, op) * 8 for op in ops]
    assert list(got) == want


def test_sector_touched_bytes_brute_force():
    """bench.sector_touched_bytes (the algorithmic bytes of the sector-storage rotation and
    adjoint kernels) against a count over the sector's determinants."""
    sys.path.insert(0, ROOT)
    import itertools
    import numpy as np
    import bench
    from paper_2405_11567_gb300 import inputs
    for N, na, nb, ne_pool in [(5, 2, 1, 3), (4, 2, 2, 4), (6, 3, 2, 4), (5, 1, 3, 4)]:
        sa = [sum(1 << (2 * q) for q in c) for c in itertools.combinations(range(N), na)]
        sb = [sum(1 << (2 * q + 1) for q in c) for c in itertools.combinations(range(N), nb)]
        dets = [a | b for a in sa for b in sb]
        pool = inputs.uccsd_pool(2 * N, ne_pool)
        got = bench.sector_touched_bytes(pool, N, na, nb, 8)
        want = [2 * _pattern_count(dets, op) * 8 for op in pool]
        assert list(got) == want
