"""Thin ctypes binding of the C-ABI declared in include/sv.h.

Functions carry the C names and do argument marshalling only: every step of
the path runs in the library's CUDA kernels.  The shared library is loaded on
first use; if it has not been built (``paper_2405_11567_gb300.build.build()``)
or no GPU is present, calls raise -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SV_C64, SV_C128, SV_R32, SV_R64 = 0, 1, 2, 3
# numpy element type of each state dtype (host views of a handle's amplitudes)
NP_DTYPE = {SV_C64: np.complex64, SV_C128: np.complex128, SV_R32: np.float32, SV_R64: np.float64}
_DTYPE_NAMES = {"c64": SV_C64, "c128": SV_C128, "r32": SV_R32, "r64": SV_R64,
                np.complex64: SV_C64, np.complex128: SV_C128, np.float32: SV_R32, np.float64: SV_R64}


def dtype_code(dtype) -> int:
    """SV_* code of a dtype given as "c64" / "c128" / "r32" / "r64", a numpy type or a code."""
    if isinstance(dtype, int) and dtype in NP_DTYPE:
        return dtype
    if dtype in _DTYPE_NAMES:
        return _DTYPE_NAMES[dtype]
    raise ValueError("unknown state dtype %r" % (dtype,))
SV_OPT_CHECKPOINT_INTERVAL, SV_OPT_MAX_BYTES, SV_OPT_EXPECT_VARIANT, SV_OPT_RDM_VARIANT = 1, 2, 3, 4
SV_OPT_PROFILE = 5
SV_OPT_LAYOUT_AUTO = 6
SV_OPT_AB_CHUNK = 7
SV_OPT_ROT_BLOCKS_PER_SM, SV_OPT_SECT_BLOCKS_PER_SM, SV_OPT_RDM_BLOCKS_PER_SM = 8, 9, 10
SV_OPT_POOL_VARIANT = 11
SV_OPT_L2_FETCH = 12
SV_OPT_REVERSE_INTERLEAVED = 14
SV_OPT_WAIT_POLLS = 15
SV_OPT_TEST_STALL = 16
SV_OPT_SECTOR_SWEEP = 17
SV_OPT_SWEEP_BLOCKS_PER_SM = 18
SV_PHASES = 8
PHASE_NAMES = ("reference", "forward", "expectation", "reverse", "restore", "rdm1", "same_products", "ab_products")
STATUS = {0: "SV_OK", 1: "SV_ERR_ARG", 2: "SV_ERR_OOM", 3: "SV_ERR_CUDA", 4: "SV_ERR_TIMEOUT", 5: "SV_ERR_STATE"}

# every symbol include/sv.h declares
EXPORTS = (
    "sv_create", "sv_create_sector", "sv_create_with_buffers", "sv_destroy", "sv_prepare_hf", "sv_prepare_state",
    "sv_get_state", "sv_get_amplitudes", "sv_state_device_ptr", "sv_set_layout", "sv_get_layout", "sv_ham_create", "sv_ham_destroy", "sv_apply_ansatz",
    "sv_energy", "sv_energy_grad", "sv_pool_gradients", "sv_rdm1", "sv_set_option", "sv_phase_times", "sv_last_error",
    "sv_launch_count", "sv_version", "sv_batch_create", "sv_batch_energy_grad", "sv_batch_set_time_limit",
    "sv_batch_launch_count", "sv_batch_destroy", "sv_rdm1_noalloc", "sv_autotune", "sv_get_option",
    "sv_batch_autotune", "sv_check_status",
)


class SvError(RuntimeError):
    def __init__(self, status, message):
        self.status = int(status)
        super().__init__("%s: %s" % (STATUS.get(self.status, str(status)), message))


class sv_excitation(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("occ", ctypes.c_int32 * 2), ("vir", ctypes.c_int32 * 2)]


class sv_instance(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("occ", ctypes.c_void_p), ("n_occ", ctypes.c_int32),
                ("h", ctypes.c_void_p), ("eri", ctypes.c_void_p), ("e_nuc", ctypes.c_double),
                ("ops", ctypes.c_void_p), ("n_ops", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    """The C-ABI library: the default build, or the checked build (SV_CHECK) when the
    environment variable SV_GB300_CHECKED is 1."""
    return _build.LIB_CHECK if os.environ.get("SV_GB300_CHECKED") == "1" else _build.LIB


def lib():
    """The loaded C-ABI library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing: build it with paper_2405_11567_gb300.build.build()"
                               % path)
        L = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "sv_create": (i32, [i32, i32, vp, pp]),
            "sv_create_sector": (i32, [i32, i32, i32, i32, vp, pp]),
            "sv_create_with_buffers": (i32, [i32, i32, vp, vp, vp, pp]),
            "sv_destroy": (i32, [vp]),
            "sv_prepare_hf": (i32, [vp, vp, i32]),
            "sv_prepare_state": (i32, [vp, vp, i32, i32]),
            "sv_get_state": (i32, [vp, vp]),
            "sv_get_amplitudes": (i32, [vp, vp, i32, vp]),
            "sv_state_device_ptr": (i32, [vp, pp]),
            "sv_set_layout": (i32, [vp, vp]),
            "sv_get_layout": (i32, [vp, vp]),
            "sv_ham_create": (i32, [i32, vp, vp, dbl, pp]),
            "sv_ham_destroy": (i32, [vp]),
            "sv_apply_ansatz": (i32, [vp, vp, i32, vp]),
            "sv_energy": (i32, [vp, vp, vp]),
            "sv_energy_grad": (i32, [vp, vp, vp, i32, vp, vp, vp]),
            "sv_rdm1": (i32, [vp, vp, vp]),
            "sv_pool_gradients": (i32, [vp, vp, vp, i32, vp, vp]),
            "sv_set_option": (i32, [vp, i32, i64]),
            "sv_phase_times": (i32, [vp, vp, i32]),
            "sv_last_error": (ctypes.c_char_p, [vp]),
            "sv_launch_count": (ctypes.c_uint64, [vp]),
            "sv_version": (ctypes.c_char_p, []),
            "sv_check_status": (ctypes.c_uint32, []),
            "sv_batch_create": (i32, [i32, vp, i32, vp, pp]),
            "sv_batch_energy_grad": (i32, [vp, vp, vp, vp]),
            "sv_batch_set_time_limit": (i32, [vp, dbl]),
            "sv_batch_launch_count": (ctypes.c_uint64, [vp]),
            "sv_batch_destroy": (i32, [vp]),
            "sv_rdm1_noalloc": (i32, [vp, i32, i32, i32, i32, vp, vp, vp]),
            "sv_autotune": (i32, [vp, vp, vp, i32, vp]),
            "sv_get_option": (i32, [vp, i32, vp]),
            "sv_batch_autotune": (i32, [vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ck(status, handle=None):
    if status != 0:
        msg = lib().sv_last_error(handle)
        raise SvError(status, msg.decode() if msg else "")


def _ops_array(ops):
    a = np.ascontiguousarray(np.asarray(ops, dtype=np.int32).reshape(-1, 5))
    return a


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---------------------------------------------------------------- C names

def sv_version() -> str:
    return lib().sv_version().decode()


def sv_check_status() -> int:
    """Checked build: the kinds of out-of-range table index its kernels skipped since the
    last call (then cleared); 0 in the default build."""
    return int(lib().sv_check_status())


def sv_last_error(handle=None) -> str:
    return lib().sv_last_error(handle).decode()


def sv_create(n_qubits: int, dtype: int, stream=None):
    h = ctypes.c_void_p()
    _ck(lib().sv_create(int(n_qubits), int(dtype), _stream_ptr(stream), ctypes.byref(h)))
    return h


def sv_create_sector(n_qubits: int, n_alpha: int, n_beta: int, dtype: int, stream=None):
    h = ctypes.c_void_p()
    _ck(lib().sv_create_sector(int(n_qubits), int(n_alpha), int(n_beta), int(dtype), _stream_ptr(stream),
                               ctypes.byref(h)))
    return h


def sv_create_with_buffers(n_qubits: int, dtype: int, stream, psi_dev: int, lam_dev=None):
    h = ctypes.c_void_p()
    _ck(lib().sv_create_with_buffers(int(n_qubits), int(dtype), _stream_ptr(stream), ctypes.c_void_p(psi_dev),
                                     ctypes.c_void_p(lam_dev) if lam_dev else None, ctypes.byref(h)))
    return h


def sv_destroy(h):
    _ck(lib().sv_destroy(h))


def sv_prepare_hf(h, occ):
    occ = np.ascontiguousarray(np.asarray(occ, dtype=np.int32).reshape(-1))
    _ck(lib().sv_prepare_hf(h, _ptr(occ), len(occ)), h)


def sv_prepare_state(h, amplitudes, n_alpha: int, n_beta: int, dtype=None):
    """Amplitudes in the handle's dtype (converted when `dtype` is given; a complex array for a
    real handle must have zero imaginary parts)."""
    a = np.asarray(amplitudes)
    if dtype is not None:
        want = NP_DTYPE[dtype_code(dtype)]
        if np.issubdtype(want, np.floating) and np.iscomplexobj(a):
            if np.any(a.imag != 0):
                raise ValueError("a real-amplitude handle needs a real state")
            a = a.real
        a = a.astype(want)
    a = np.ascontiguousarray(a)
    if a.dtype.type not in (np.complex64, np.complex128, np.float32, np.float64):
        raise TypeError("amplitudes must be complex64, complex128, float32 or float64 (the handle's dtype)")
    _ck(lib().sv_prepare_state(h, _ptr(a), int(n_alpha), int(n_beta)), h)


def sv_get_state(h, n_qubits: int, dtype: int) -> np.ndarray:
    out = np.empty(1 << n_qubits, dtype=NP_DTYPE[dtype_code(dtype)])
    _ck(lib().sv_get_state(h, _ptr(out)), h)
    return out


def sv_get_amplitudes(h, basis, dtype: int) -> np.ndarray:
    idx = np.ascontiguousarray(np.asarray(basis, dtype=np.uint64).reshape(-1))
    out = np.empty(len(idx), dtype=NP_DTYPE[dtype_code(dtype)])
    _ck(lib().sv_get_amplitudes(h, _ptr(idx), len(idx), _ptr(out)), h)
    return out


def sv_state_device_ptr(h) -> int:
    p = ctypes.c_void_p()
    _ck(lib().sv_state_device_ptr(h, ctypes.byref(p)), h)
    return p.value


def sv_set_layout(h, storage_of_qubit):
    a = np.ascontiguousarray(np.asarray(storage_of_qubit, dtype=np.int32).reshape(-1))
    _ck(lib().sv_set_layout(h, _ptr(a)), h)


def sv_get_layout(h, n_qubits: int) -> np.ndarray:
    out = np.zeros(n_qubits, dtype=np.int32)
    _ck(lib().sv_get_layout(h, _ptr(out)), h)
    return out


def sv_ham_create(h_mat, eri, e_nuc: float):
    hm = np.ascontiguousarray(np.asarray(h_mat, dtype=np.float64))
    N = hm.shape[0]
    er = np.ascontiguousarray(np.asarray(eri, dtype=np.float64).reshape(N, N, N, N))
    out = ctypes.c_void_p()
    _ck(lib().sv_ham_create(N, _ptr(hm), _ptr(er), float(e_nuc), ctypes.byref(out)))
    return out


def sv_ham_destroy(ham):
    _ck(lib().sv_ham_destroy(ham))


def sv_apply_ansatz(h, ops, theta):
    o = _ops_array(ops)
    t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
    if len(t) != len(o):
        raise ValueError("one angle per excitation")
    _ck(lib().sv_apply_ansatz(h, _ptr(o), len(o), _ptr(t)), h)


def sv_energy(h, ham) -> float:
    e = np.zeros(1)
    _ck(lib().sv_energy(h, ham, _ptr(e)), h)
    return float(e[0])


def sv_energy_grad(h, ham, ops, theta):
    o = _ops_array(ops)
    t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
    if len(t) != len(o):
        raise ValueError("one angle per excitation")
    e = np.zeros(1)
    g = np.zeros(max(len(o), 1))
    _ck(lib().sv_energy_grad(h, ham, _ptr(o), len(o), _ptr(t), _ptr(e), _ptr(g)), h)
    return float(e[0]), g[:len(o)]


def sv_pool_gradients(h, ham, pool):
    o = _ops_array(pool)
    e = np.zeros(1)
    g = np.zeros(max(len(o), 1))
    _ck(lib().sv_pool_gradients(h, ham, _ptr(o), len(o), _ptr(e), _ptr(g)), h)
    return float(e[0]), g[:len(o)]


def sv_rdm1(h, n_orb: int) -> np.ndarray:
    re = np.zeros((2, n_orb, n_orb))
    im = np.zeros((2, n_orb, n_orb))
    _ck(lib().sv_rdm1(h, _ptr(re), _ptr(im)), h)
    return re + 1j * im


def sv_rdm1_noalloc(psi_dev: int, n_qubits: int, dtype: int, n_alpha: int, n_beta: int, stream=None) -> np.ndarray:
    """1-RDM of a device-resident state in qubit order, using only the library's fixed scratch array.

    ``stream`` must be the stream that wrote ``psi_dev`` or one ordered after it (None is the
    legacy default stream, which is not ordered after non-blocking streams such as torch's):
    ``StateVector.rdm1_noalloc`` passes its handle's stream."""
    N = n_qubits // 2
    re = np.zeros((2, N, N))
    im = np.zeros((2, N, N))
    _ck(lib().sv_rdm1_noalloc(ctypes.c_void_p(psi_dev), int(n_qubits), int(dtype), int(n_alpha), int(n_beta),
                              _stream_ptr(stream), _ptr(re), _ptr(im)))
    return re + 1j * im


def sv_set_option(h, opt: int, value: int):
    _ck(lib().sv_set_option(h, int(opt), int(value)), h)


def sv_get_option(h, opt: int) -> int:
    v = ctypes.c_int64()
    _ck(lib().sv_get_option(h, int(opt), ctypes.byref(v)), h)
    return int(v.value)


def sv_autotune(h, ham, ops, theta):
    o = _ops_array(ops)
    t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
    if len(t) != len(o):
        raise ValueError("one angle per excitation")
    _ck(lib().sv_autotune(h, ham, _ptr(o), len(o), _ptr(t)), h)


def sv_phase_times(h) -> dict:
    ms = np.zeros(SV_PHASES)
    _ck(lib().sv_phase_times(h, _ptr(ms), SV_PHASES), h)
    return dict(zip(PHASE_NAMES, ms.tolist()))


def sv_launch_count(h) -> int:
    return int(lib().sv_launch_count(h))


def sv_batch_create(problems, dtype: int, stream=None):
    """problems: dicts with n_qubits, occ, h, eri, e_nuc, ops (the inputs module's format)."""
    keep = []
    arr = (sv_instance * len(problems))()
    for k, p in enumerate(problems):
        occ = np.ascontiguousarray(np.asarray(p["occ"], dtype=np.int32).reshape(-1))
        hm = np.ascontiguousarray(np.asarray(p["h"], dtype=np.float64))
        er = np.ascontiguousarray(np.asarray(p["eri"], dtype=np.float64))
        ops = _ops_array(p["ops"])
        keep += [occ, hm, er, ops]
        arr[k] = sv_instance(int(p["n_qubits"]), occ.ctypes.data, len(occ), hm.ctypes.data, er.ctypes.data,
                             float(p["e_nuc"]), ops.ctypes.data, len(ops))
    out = ctypes.c_void_p()
    _ck(lib().sv_batch_create(len(problems), ctypes.cast(arr, ctypes.c_void_p), int(dtype), _stream_ptr(stream),
                              ctypes.byref(out)))
    return out


def sv_batch_energy_grad(b, theta_concat, n_inst: int, total_ops: int):
    t = np.ascontiguousarray(np.asarray(theta_concat, dtype=np.float64).reshape(-1))
    if len(t) != total_ops:
        raise ValueError("theta must hold every instance's angles, concatenated")
    e = np.zeros(n_inst)
    g = np.zeros(max(total_ops, 1))
    _ck(lib().sv_batch_energy_grad(b, _ptr(t), _ptr(e), _ptr(g)))
    return e, g[:total_ops]


def sv_batch_autotune(b, theta_concat, total_ops: int) -> int:
    t = np.ascontiguousarray(np.asarray(theta_concat, dtype=np.float64).reshape(-1))
    if len(t) != total_ops:
        raise ValueError("theta must hold every instance's angles, concatenated")
    grid = ctypes.c_int()
    _ck(lib().sv_batch_autotune(b, _ptr(t), ctypes.byref(grid)))
    return int(grid.value)


def sv_batch_set_time_limit(b, ms: float):
    _ck(lib().sv_batch_set_time_limit(b, float(ms)))


def sv_batch_launch_count(b) -> int:
    return int(lib().sv_batch_launch_count(b))


def sv_batch_destroy(b):
    _ck(lib().sv_batch_destroy(b))


# ---------------------------------------------------------------- convenience objects

class Batch:
    """Owns an ``sv_batch_handle``: many independent problems in one persistent launch."""

    def __init__(self, problems, dtype="c64", stream=None):
        self.dtype = dtype_code(dtype)
        self.sizes = [len(p["ops"]) for p in problems]
        self.n_inst = len(problems)
        self.total_ops = int(sum(self.sizes))
        self.handle = sv_batch_create(problems, self.dtype, stream)

    def energy_grad(self, theta_concat):
        """(E per instance, list of gradient arrays per instance)."""
        e, g = sv_batch_energy_grad(self.handle, theta_concat, self.n_inst, self.total_ops)
        return e, np.split(g, np.cumsum(self.sizes)[:-1])

    def set_time_limit(self, ms):
        sv_batch_set_time_limit(self.handle, ms)

    def autotune(self, theta_concat) -> int:
        """Time the batched launch at 1-4 blocks per SM and keep the fastest grid (returned)."""
        return sv_batch_autotune(self.handle, theta_concat, self.total_ops)

    @property
    def launches(self) -> int:
        return sv_batch_launch_count(self.handle)

    def close(self):
        if self.handle is not None:
            sv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

class Hamiltonian:
    """Owns an ``sv_ham_handle`` built from (h, eri, e_nuc)."""

    def __init__(self, h_mat, eri, e_nuc):
        self.n_orb = int(np.asarray(h_mat).shape[0])
        self.handle = sv_ham_create(h_mat, eri, e_nuc)

    def close(self):
        if self.handle is not None:
            sv_ham_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StateVector:
    """Owns an ``sv_handle``: an n-qubit state on the current CUDA device.

    ``sector=(n_alpha, n_beta)`` keeps only that particle-number sector's
    amplitudes on the device (``sv_create_sector``); the default is the dense
    2^n vector.
    """

    def __init__(self, n_qubits: int, dtype="c64", stream=None, sector=None):
        self.n = int(n_qubits)
        self.dtype = dtype_code(dtype)
        self.sector = None if sector is None else (int(sector[0]), int(sector[1]))
        self.stream = stream
        self.handle = None
        if self.sector is None:
            self.handle = sv_create(self.n, self.dtype, stream)
        else:
            self.handle = sv_create_sector(self.n, self.sector[0], self.sector[1], self.dtype, stream)

    def close(self):
        if self.handle is not None:
            sv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prepare_hf(self, occ):
        sv_prepare_hf(self.handle, occ)

    def prepare_state(self, amplitudes, n_alpha, n_beta):
        """Any dense 2^n amplitude array of the (n_alpha, n_beta) sector, converted to the handle's dtype."""
        sv_prepare_state(self.handle, amplitudes, n_alpha, n_beta, dtype=self.dtype)

    def state(self) -> np.ndarray:
        return sv_get_state(self.handle, self.n, self.dtype)

    def amplitudes(self, basis) -> np.ndarray:
        return sv_get_amplitudes(self.handle, basis, self.dtype)

    def apply_ansatz(self, ops, theta):
        sv_apply_ansatz(self.handle, ops, theta)

    def energy(self, ham: Hamiltonian) -> float:
        return sv_energy(self.handle, ham.handle)

    def energy_grad(self, ham: Hamiltonian, ops, theta):
        return sv_energy_grad(self.handle, ham.handle, ops, theta)

    def rdm1(self) -> np.ndarray:
        return sv_rdm1(self.handle, self.n // 2)

    def rdm1_noalloc(self, n_alpha: int, n_beta: int) -> np.ndarray:
        """The 1-RDM through sv_rdm1_noalloc (no device allocation) on this handle's stream, so
        that it is ordered after the handle's queued work.  Dense storage in qubit order only."""
        if self.sector is not None:
            raise ValueError("sv_rdm1_noalloc reads a dense 2^n state")
        if not np.array_equal(self.layout(), np.arange(self.n)):
            raise ValueError("sv_rdm1_noalloc reads the state in qubit order: set_layout(range(n)) first")
        return sv_rdm1_noalloc(sv_state_device_ptr(self.handle), self.n, self.dtype, n_alpha, n_beta,
                               stream=self.stream)

    def pool_gradients(self, ham: Hamiltonian, pool):
        """(E, gradients of appending each pool operator at angle 0) for the current state."""
        return sv_pool_gradients(self.handle, ham.handle, pool)

    def set_option(self, opt, value):
        sv_set_option(self.handle, opt, value)

    def option(self, opt) -> int:
        return sv_get_option(self.handle, opt)

    def autotune(self, ham: Hamiltonian, ops, theta) -> dict:
        """Time the candidate launch choices on this problem and keep the fastest (sv_autotune)."""
        sv_autotune(self.handle, ham.handle, ops, theta)
        return {name: self.option(opt) for name, opt in (
            ("expect_variant", SV_OPT_EXPECT_VARIANT), ("ab_chunk", SV_OPT_AB_CHUNK),
            ("rot_blocks_per_sm", SV_OPT_ROT_BLOCKS_PER_SM), ("sect_blocks_per_sm", SV_OPT_SECT_BLOCKS_PER_SM),
            ("rdm_blocks_per_sm", SV_OPT_RDM_BLOCKS_PER_SM), ("sweep_blocks_per_sm", SV_OPT_SWEEP_BLOCKS_PER_SM))}

    def set_layout(self, storage_of_qubit):
        sv_set_layout(self.handle, storage_of_qubit)

    def layout(self) -> np.ndarray:
        return sv_get_layout(self.handle, self.n)

    def phase_times(self) -> dict:
        return sv_phase_times(self.handle)

    @property
    def launches(self) -> int:
        return sv_launch_count(self.handle)
