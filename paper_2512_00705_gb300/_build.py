"""Build the CUDA library (libflexiwalk.so) for sm_103a with nvcc, in-tree.

Translation units are compiled in parallel and linked into one shared
library that exports the C ABI of include/flexiwalk.h.  The CUDA runtime is
linked statically, so the library needs only the driver at run time.
"""
from __future__ import annotations

import glob
import hashlib
import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libflexiwalk.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-fmad=true",
              "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs_digest() -> str:
    h = hashlib.sha256()
    files = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")))
    files.append(os.path.join(ROOT, "include", "flexiwalk.h"))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    # the flags name the include directory by absolute path: hash them with the
    # repository root factored out, so a checkout elsewhere has the same digest
    h.update(" ".join(ARCH + NVCC_FLAGS).replace(ROOT, "<root>").encode())
    return h.hexdigest()


# The files that define the walk kernel and the device data it reads (records,
# filters, label-grouped view): profiles of the kernel are keyed to their digest.
WALK_KERNEL_FILES = ["fw_device.cuh", "fw_walk.cuh", "fw_kernels.cu", "fw_walk_mixed.cu", "fw_internal.h", "fw_api.cu"]


def _code_only(text: str) -> str:
    """C/C++ source without comments and with runs of whitespace collapsed
    (the sources hold no string literals with comment markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def walk_kernel_digest() -> str:
    """Digest of the walk kernel's code (comments and layout ignored), the
    public header and the nvcc flags (repository root factored out): a
    recorded profile of the walk kernel applies while this is unchanged."""
    h = hashlib.sha256()
    paths = [os.path.join(CSRC, f) for f in WALK_KERNEL_FILES] + [os.path.join(ROOT, "include", "flexiwalk.h")]
    for path in paths:
        h.update(os.path.basename(path).encode())
        with open(path, encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    h.update(" ".join(ARCH + NVCC_FLAGS).replace(ROOT, "<root>").encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ and link libflexiwalk.so; returns its path.
    Skips the work when the sources are unchanged since the last build."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "libflexiwalk.stamp")
    digest = _inputs_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == digest:
        return LIB
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
