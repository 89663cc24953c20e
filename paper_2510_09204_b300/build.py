"""Build the SF solver's shared library (``libsf.so``) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libsf.so")
# the same sources with the device-side bounds checks compiled in (SF_BOUNDS_CHECK): a
# test build that reports SF_EBOUNDS per instance instead of touching memory out of bounds
LIB_CHECK = os.path.join(PKG, "libsf_check.so")
CHECK_FLAGS = ("-DSF_BOUNDS_CHECK",)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def source_digest() -> str:
    """SHA-256 over the kernel sources (csrc/ and include/, names and contents): a profile
    summary records it, and its counters apply only while the sources are unchanged."""
    import hashlib
    h = hashlib.sha256()
    for f in sources() + headers():
        h.update(os.path.relpath(f, ROOT).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def stale(out: str = LIB) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in sources() + headers())


def _run(cmd):
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False, verbose: bool = False, out: str = LIB, extra=()) -> str:
    """Compile every .cu under csrc/ (one object per file, in parallel) and link them into
    one shared library; returns its path."""
    if not force and not stale(out):
        return out
    objdir = os.path.join(PKG, "_build" if not extra else "_build_" + os.path.splitext(os.path.basename(out))[0])
    os.makedirs(objdir, exist_ok=True)
    flags = [NVCC, "-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC, *extra]
    if verbose:
        flags += ["-Xptxas", "-v"]
    objs, cmds = [], []
    for src in sources():
        obj = os.path.join(objdir, os.path.splitext(os.path.basename(src))[0] + ".o")
        objs.append(obj)
        cmds.append(flags + ["-c", src, "-o", obj])
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
        results = list(ex.map(_run, cmds))
    for r in results:
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed building %s" % out)
        if verbose:
            sys.stderr.write(r.stderr)
    r = _run([NVCC, *ARCH, "-shared", "-o", out, *objs])
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking %s" % out)
    return out


def build_check(force: bool = False) -> str:
    """The bounds-checked library (libsf_check.so)."""
    return build(force=force, out=LIB_CHECK, extra=CHECK_FLAGS)


def build_all(force: bool = False) -> tuple:
    """Both libraries at once: their longest translation units compile side by side
    instead of one build after the other."""
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build, force)
        b = ex.submit(build_check, force)
        return a.result(), b.result()


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
    if "--check" in sys.argv:
        print(build_check(force=True))
