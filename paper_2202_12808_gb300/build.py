"""In-tree build of libcofem.so for GB300 (sm_103a) with nvcc.

Each .cu under csrc/ is compiled to an object in parallel, then linked into
paper_2202_12808_gb300/libcofem.so against the shared CUDA runtime.  An
object is rebuilt unless a stamp beside it records the SHA-1 of exactly the
same compiler command, source and headers (file times are not trusted: a
copied tree keeps them); the library is relinked unless its stamp records the
same objects' hashes and link command.
"""
import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcofem.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")] + ARCH


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "cofem.h"))
    return hs


def _digest(parts, files):
    h = hashlib.sha1()
    for p in parts:
        h.update(p.encode())
        h.update(b"\0")
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _fresh(target, digest):
    """target exists and its stamp records `digest`."""
    stamp = target + ".sha1"
    if not (os.path.exists(target) and os.path.exists(stamp)):
        return False
    with open(stamp) as fh:
        return fh.read().strip() == digest


def _stamp(target, digest):
    with open(target + ".sha1", "w") as fh:
        fh.write(digest + "\n")


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [_nvcc()] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
    digest = _digest(cmd, [src] + sorted(_headers()))
    if not _fresh(obj, digest):
        if os.path.exists(obj + ".sha1"):
            os.remove(obj + ".sha1")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if r.stderr.strip():
            sys.stderr.write(r.stderr)
        _stamp(obj, digest)
    return obj


def build(verbose=False, extra=()):
    """Compile csrc/*.cu and link libcofem.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(extra)), srcs))
    cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB] + objs + [
        "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    digest = _digest(cmd, objs)
    if not _fresh(LIB, digest):
        if os.path.exists(LIB + ".sha1"):
            os.remove(LIB + ".sha1")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        _stamp(LIB, digest)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
