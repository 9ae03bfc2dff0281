"""GPU parity of the batched persistent launch (config 4: 512 instances of 10-20
qubits, 40 operators each) against the CPU oracle, instance by instance."""
import numpy as np
import pytest

import oracle
from oracle import route_a as A
from paper_2405_11567_gb300 import inputs, sv

pytestmark = pytest.mark.gpu

TOL = {"c128": (1e-10, 1e-9), "c64": (1e-5, 1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2405_11567_gb300 import build
    build.build()
    sv.lib()


def _oracle(p):
    sec = oracle.Sector(p["n_qubits"], p["na"], p["nb"])
    return A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], A.hf_state(sec, p["occ"]))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_matches_oracle_mixed_sizes(dtype):
    probs = inputs.batch_problems(24)
    assert len({p["n_qubits"] for p in probs}) >= 4
    b = sv.Batch(probs, dtype)
    theta = np.concatenate([p["theta"] for p in probs])
    E, g = b.energy_grad(theta)
    tE, tg = TOL[dtype]
    for k, p in enumerate(probs):
        Er, gr = _oracle(p)
        assert abs(E[k] - Er) <= tE, (k, p["n_qubits"], E[k], Er)
        assert np.max(np.abs(g[k] - gr)) <= tg, (k, p["n_qubits"])
    assert b.launches == 2  # the angles' cosines and sines, then the batched kernel


def test_batch_full_config4_sampled():
    """All 512 instances in one launch (complex64); instances of every size checked against the oracle."""
    probs = inputs.batch_problems(512)
    b = sv.Batch(probs, "c64")
    theta = np.concatenate([p["theta"] for p in probs])
    E, g = b.energy_grad(theta)
    assert np.all(np.isfinite(E))
    picked = {}
    for k, p in enumerate(probs):
        picked.setdefault(p["n_qubits"], []).append(k)
    for n, ks in sorted(picked.items()):
        for k in ks[:2]:
            Er, gr = _oracle(probs[k])
            assert abs(E[k] - Er) <= 1e-5, (n, k)
            assert np.max(np.abs(g[k] - gr)) <= 1e-5, (n, k)
    # a second launch with other angles gives other numbers, replayed from the same graph
    E2, _ = b.energy_grad(theta * 0.5)
    assert not np.allclose(E, E2)
    assert b.launches == 4


def test_batch_deterministic_and_same_as_single_handles():
    probs = inputs.batch_problems(10, first=100)
    b = sv.Batch(probs, "c128")
    theta = np.concatenate([p["theta"] for p in probs])
    E1, g1 = b.energy_grad(theta)
    E2, g2 = b.energy_grad(theta)
    assert np.array_equal(E1, E2) and all(np.array_equal(x, y) for x, y in zip(g1, g2))
    for k, p in enumerate(probs[:4]):
        ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
        st = sv.StateVector(p["n_qubits"], "c128")
        st.prepare_hf(p["occ"])
        E, g = st.energy_grad(ham, p["ops"], p["theta"])
        assert abs(E - E1[k]) <= 1e-11 and np.max(np.abs(g - g1[k])) <= 1e-10


def test_batch_time_limit_reports_timeout_and_recovers():
    probs = inputs.batch_problems(64)
    b = sv.Batch(probs, "c64")
    theta = np.concatenate([p["theta"] for p in probs])
    b.set_time_limit(1e-6)          # 1 ns: every block stops before taking a second instance
    with pytest.raises(sv.SvError) as e:
        b.energy_grad(theta)
    assert e.value.status == 4
    b.set_time_limit(0)
    E, g = b.energy_grad(theta)
    assert np.all(np.isfinite(E))


def test_batch_edges_and_errors():
    p = inputs.make_problem(8, 2, "uccsd", 5)
    empty = dict(p, ops=p["ops"][:0], theta=np.zeros(0))
    vac = dict(p, occ=[])
    b = sv.Batch([p, empty, vac], "c128")
    E, g = b.energy_grad(np.concatenate([p["theta"], [], p["theta"]]))
    Er, gr = _oracle(p)
    assert abs(E[0] - Er) <= 1e-10 and np.max(np.abs(g[0] - gr)) <= 1e-9
    sec = oracle.Sector(8, 1, 1)
    assert abs(E[1] - A.energy(sec, p["h"], p["eri"], p["e_nuc"], A.hf_state(sec, p["occ"]))) <= 1e-12
    assert len(g[1]) == 0
    assert abs(E[2] - p["e_nuc"]) <= 1e-12 and np.max(np.abs(g[2])) == 0.0
    bad = dict(p, ops=np.array([(2, 0, 1, 2, 2)], np.int32), theta=np.zeros(1))
    with pytest.raises(sv.SvError) as e:
        sv.Batch([bad], "c64")
    assert e.value.status == 1
    with pytest.raises(sv.SvError):
        b.energy_grad(np.full(2 * len(p["ops"]), np.nan))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_generic_path_for_large_string_spaces(dtype):
    """An instance with more than 512 alpha strings (24 qubits, 5 alpha + 1 beta electrons:
    792 x 12 determinants) takes the generic per-element sigma and filtered sweeps; batched
    beside instances that take the string-blocked path, every instance matches the oracle."""
    big = inputs.make_problem(24, 6, 12, seed=4242)
    big["occ"] = np.array([0, 2, 4, 6, 8, 1], dtype=np.int32)   # alpha orbitals 0-4, beta orbital 0
    big["na"], big["nb"] = 5, 1
    probs = [big] + inputs.batch_problems(3, first=7)
    b = sv.Batch(probs, dtype)
    theta = np.concatenate([p["theta"] for p in probs]) * 4
    E, g = b.energy_grad(theta)
    tE, tg = TOL[dtype]
    off = 0
    for k, p in enumerate(probs):
        q = dict(p, theta=theta[off:off + len(p["ops"])])
        off += len(p["ops"])
        Er, gr = _oracle(q)
        assert abs(E[k] - Er) <= tE, (k, E[k], Er)
        assert np.max(np.abs(g[k] - gr)) <= tg, k
