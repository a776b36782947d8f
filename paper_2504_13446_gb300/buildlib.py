"""Compile the CUDA library in-tree for sm_103a (GB300).

Each ``csrc/*.cu`` file is compiled to an object in parallel with nvcc, then
linked into a shared library next to this file.  A rebuild happens only when a
source or header is newer than the library.

Two builds exist, with the same entry points and the same results bit for bit:

* ``single_gpu`` (``librkr.so``, the default): row-owned tensor-core screens run
  as CTA pairs that share B tiles through TMA loads multicast within a cluster
  (``csrc/tc_pair.cuh``, compiled only here, with ``RKR_CLUSTER_MULTICAST``).
* ``replica`` (``librkr_replica.so``): no cluster multicast in any kernel; every
  screen runs on the single-CTA kernel.  A process that is one rank of a
  multi-GPU job loads this build (``RKR_LIB_VARIANT=replica``).
"""

from __future__ import annotations

import concurrent.futures as cf
import contextlib
import fcntl
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

VARIANTS = {
    "single_gpu": {"lib": "librkr.so", "objdir": "_build", "defines": ["-DRKR_CLUSTER_MULTICAST"]},
    "replica": {"lib": "librkr_replica.so", "objdir": "_build_replica", "defines": []},
}
LIB = os.path.join(PKG, VARIANTS["single_gpu"]["lib"])
OBJDIR = os.path.join(PKG, VARIANTS["single_gpu"]["objdir"])


def lib_path(variant: str = "single_gpu") -> str:
    return os.path.join(PKG, VARIANTS[variant]["lib"])


def selected_variant() -> str:
    """The build this process loads: RKR_LIB_VARIANT, else single_gpu."""
    v = os.environ.get("RKR_LIB_VARIANT", "single_gpu")
    if v not in VARIANTS:
        raise RuntimeError(f"RKR_LIB_VARIANT={v!r}: expected one of {sorted(VARIANTS)}")
    return v


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librkr.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def flags(variant: str = "single_gpu", verbose: bool = False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    f += VARIANTS[variant]["defines"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def up_to_date(variant: str = "single_gpu") -> bool:
    lib = lib_path(variant)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


@contextlib.contextmanager
def _build_lock(objdir):
    # one build at a time per variant (several ranks of a job may ask at once)
    os.makedirs(objdir, exist_ok=True)
    with open(os.path.join(objdir, ".lock"), "w") as f:
        fcntl.flock(f, fcntl.LOCK_EX)
        try:
            yield
        finally:
            fcntl.flock(f, fcntl.LOCK_UN)


def build(force: bool = False, verbose: bool = False, variant: str = "single_gpu") -> str:
    lib = lib_path(variant)
    objdir = os.path.join(PKG, VARIANTS[variant]["objdir"])
    if not force and up_to_date(variant):
        return lib
    with _build_lock(objdir):
        if not force and up_to_date(variant):
            return lib
        nvcc = _nvcc()
        fl = flags(variant, verbose)

        def compile_one(src):
            obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
            r = subprocess.run([nvcc, "-c", src, "-o", obj] + fl, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
            return obj, r.stderr

        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            results = list(ex.map(compile_one, _sources()))
        if verbose:
            for _, log in results:
                print(log)
        objs = [o for o, _ in results]
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc, "-shared", "-o", tmp] + ARCH + objs, capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


def included_headers(src: str, variant: str = "single_gpu"):
    """Headers of this package that one translation unit includes in a build."""
    r = subprocess.run([_nvcc(), "-M", src] + flags(variant), capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc -M failed on {src}:\n{r.stderr}")
    deps = r.stdout.replace("\\\n", " ").split()
    return sorted({os.path.basename(p) for p in deps if os.path.dirname(os.path.abspath(p)) == CSRC})


if __name__ == "__main__":
    import sys
    var = "replica" if "--replica" in sys.argv else "single_gpu"
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, variant=var))
