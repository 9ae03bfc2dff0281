"""Build the C-ABI shared library (hand-written CUDA for sm_103a) in-tree.

``python -m paper_2405_11567_gb300.build`` or ``build()``: compiles every source
under ``csrc/`` with nvcc for ``sm_103a`` in parallel and links
``_build/libsv_gb300.so`` (git-ignored).  Rebuilds only when a source or header
is newer than the library.  ``build(check=True)`` builds the checked library
``_build/libsv_gb300_check.so`` (SV_CHECK: kernels record out-of-range table
indices instead of faulting); the binding loads it when SV_GB300_CHECKED=1.
"""
import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsv_gb300.so")
LIB_CHECK = os.path.join(OUT_DIR, "libsv_gb300_check.so")  # the checked build (SV_CHECK)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile and link the library if needed; return its path.  check=True builds the
    checked library (LIB_CHECK: every source compiled with SV_CHECK=1, objects apart)."""
    lib = LIB_CHECK if check else LIB
    if not force and not _stale(lib):
        return lib
    obj_dir = os.path.join(OUT_DIR, "check") if check else OUT_DIR
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = CFLAGS + (["-DSV_CHECK=1"] if check else [])
    objs = []
    cmds = []
    for src in sources():
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        cmds.append([nvcc] + ARCH + flags + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return r

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        list(ex.map(run, cmds))
    tmp = lib + ".tmp.%d" % os.getpid()
    run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
