"""Host-side checks that need no GPU: the C-ABI library builds for sm_103a, loads,
exports every symbol include/sv.h declares, and validates its host-only inputs;
the input generators produce the operator pools and sector sizes the workloads
specify."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2405_11567_gb300 import build as libbuild
from paper_2405_11567_gb300 import inputs
from paper_2405_11567_gb300 import sv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cabi():
    libbuild.build()
    return sv.lib()


def test_header_declares_exactly_the_exports():
    text = open(os.path.join(ROOT, "include", "sv.h")).read()
    declared = set(re.findall(r"^\s*(?:sv_status|const char \*|uint64_t|uint32_t)\s*\*?\s*(sv_\w+)\s*\(", text, re.M))
    assert declared == set(sv.EXPORTS)


def test_library_exports_every_declared_symbol(cabi):
    for name in sv.EXPORTS:
        assert hasattr(cabi, name), name
    assert "sm_103a" in sv.sv_version()


def test_checked_build_exports_the_same_symbols_and_default_reports_nothing(cabi):
    """The checked build (every source with SV_CHECK=1: kernels record out-of-range table
    indices instead of faulting) compiles and exports the same C ABI; in the default build
    sv_check_status is 0 (no GPU call)."""
    path = libbuild.build(check=True)
    assert path == libbuild.LIB_CHECK and os.path.exists(path)
    checked = ctypes.CDLL(path)
    for name in sv.EXPORTS:
        assert hasattr(checked, name), name
    assert sv.sv_check_status() == 0


def test_library_built_for_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(libbuild.ARCH)


def test_library_needs_no_blas(cabi):
    """Every product on the path is the library's own kernel: the shared library's
    dynamic section names no cuBLAS / cuBLASLt dependency."""
    import shutil
    import subprocess
    readelf = shutil.which("readelf")
    if readelf is None:
        pytest.skip("readelf not available")
    out = subprocess.run([readelf, "-d", libbuild.LIB], capture_output=True, text=True, check=True).stdout
    needed = re.findall(r"\(NEEDED\)\s+Shared library: \[([^\]]+)\]", out)
    assert needed, out
    assert not [x for x in needed if "blas" in x.lower()], needed


def test_ham_create_validates_on_host(cabi):
    N = 3
    rng = np.random.default_rng(0)
    h, eri, e_nuc = inputs.synthetic_integrals(N, rng)
    ham = sv.sv_ham_create(h, eri, e_nuc)
    sv.sv_ham_destroy(ham)
    bad = eri.copy()
    bad[0, 1, 2, 0] += 1e-6                      # breaks (pq|rs) = (qp|rs)
    with pytest.raises(sv.SvError) as e:
        sv.sv_ham_create(h, bad, e_nuc)
    assert e.value.status == 1
    hb = h.copy()
    hb[0, 1] += 1e-3
    with pytest.raises(sv.SvError):
        sv.sv_ham_create(hb, eri, e_nuc)
    with pytest.raises(sv.SvError):
        sv.sv_ham_create(h, eri, float("nan"))


def test_null_and_bad_arguments_rejected_without_device(cabi):
    out = ctypes.c_void_p()
    assert cabi.sv_create(7, 0, None, ctypes.byref(out)) == 1      # odd qubit count
    assert cabi.sv_create(34, 0, None, ctypes.byref(out)) == 1     # beyond 32 qubits
    assert cabi.sv_create(8, 5, None, ctypes.byref(out)) == 1      # bad dtype
    assert cabi.sv_create(8, 0, None, None) == 1
    assert cabi.sv_create_sector(8, 5, 1, 0, None, ctypes.byref(out)) == 1   # more electrons than orbitals
    assert cabi.sv_create_sector(8, 1, -1, 0, None, ctypes.byref(out)) == 1  # negative count
    assert cabi.sv_create_sector(9, 1, 1, 0, None, ctypes.byref(out)) == 1   # odd qubit count
    assert cabi.sv_create_sector(8, 1, 1, 7, None, ctypes.byref(out)) == 1   # bad dtype
    v = ctypes.c_int64()
    assert cabi.sv_get_option(None, 1, ctypes.byref(v)) == 1
    assert cabi.sv_autotune(None, None, None, 0, None) == 1
    assert cabi.sv_batch_autotune(None, None, None) == 1
    assert cabi.sv_destroy(None) == 0
    assert cabi.sv_energy(None, None, None) == 1
    assert b"NULL" in cabi.sv_last_error(None)


@pytest.mark.parametrize("n,ne,expect", [(8, 2, (6, 9)), (10, 2, (8, 16)), (12, 4, (16, 76)), (16, 4, (24, 174)),
                                         (20, 6, (42, 567)), (24, 8, (64, 1360)), (30, 10, (100, 3400))])
def test_uccsd_pool_sizes(n, ne, expect):
    pool = inputs.uccsd_pool(n, ne)
    assert (int(np.sum(pool[:, 0] == 1)), int(np.sum(pool[:, 0] == 2))) == expect
    # every operator conserves S_z and excites from occupied to virtual
    for k, i, j, a, b in pool:
        occ = [i] if k == 1 else [i, j]
        vir = [a] if k == 1 else [a, b]
        assert all(o < ne for o in occ) and all(v >= ne for v in vir)
        assert sorted(o % 2 for o in occ) == sorted(v % 2 for v in vir)


def test_configs_are_seeded_and_shaped():
    p = inputs.config_problem(5)
    assert p["n_qubits"] == 30 and p["n_elec"] == 10 and len(p["ops"]) == 200 and p["eri"].shape == (15,) * 4
    q = inputs.config_problem(5)
    assert np.array_equal(p["ops"], q["ops"]) and np.array_equal(p["eri"], q["eri"])
    # (pp|pp) in [0.3, 0.8] exactly by construction, 8-fold symmetry, PSD supermatrix
    d = np.einsum("pppp->p", p["eri"])
    assert np.all(d >= 0.3) and np.all(d <= 0.8)
    e = p["eri"]
    assert np.allclose(e, e.transpose(1, 0, 2, 3)) and np.allclose(e, e.transpose(2, 3, 0, 1))
    assert np.linalg.eigvalsh(e.reshape(225, 225)).min() > -1e-10
    assert len(inputs.config_problem(3)["ops"]) == 120 and len(inputs.config_problem(2)["ops"]) == 198
    b = inputs.batch_problems(6)
    assert all(x["n_qubits"] in (10, 12, 14, 16, 18, 20) and len(x["ops"]) == 40 for x in b)
    assert [inputs.batch_electrons(q) for q in (10, 12, 14, 16, 18, 20)] == [2, 4, 4, 4, 4, 6]
