"""Build the CUDA library libpf.so in-tree with nvcc for sm_103a.

The translation units are compiled in parallel and linked into
``paper_2302_13612_gb300/_lib/libpf.so``; a rebuild happens only when a
source, a header or the flags changed.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libpf.so")

SOURCES = ["pf_k_xfwd.cu", "pf_k_xinv.cu", "pf_k_yz.cu", "pf_xfix.cu", "pf_xfix_pfa.cu", "pf_yzfix.cu", "pf_yzfix_pfa.cu", "pf_ytc.cu", "pf_kernels.cu", "pf_api.cu", "pf_static.cu", "pf_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpf.so")


def headers():
    """Every header under csrc/ (sorted), so that a new or edited header
    always changes the fingerprint."""
    return sorted(n for n in os.listdir(CSRC) if n.endswith((".h", ".cuh", ".hpp")))


def _fingerprint(extra) -> str:
    h = hashlib.sha256()
    for name in SOURCES + headers():
        h.update(name.encode())
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(INCLUDE, "pf.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).encode())
    return h.hexdigest()


LIB_CHECK = os.path.join(LIBDIR, "libpf_check.so")


def build_library(force: bool = False, extra_flags=(), verbose: bool = False, check: bool = False) -> str:
    """Compile (if needed) and return the path of libpf.so; check=True builds
    the PF_CHECK variant (kernels verify their shared-memory layout and tile
    coordinates and report PF_ECHECK) as libpf_check.so beside it."""
    os.makedirs(LIBDIR, exist_ok=True)
    lib = LIB_CHECK if check else LIB
    tag = "_check" if check else ""
    if check:
        extra_flags = tuple(extra_flags) + ("-DPF_CHECK",)
    stamp = os.path.join(LIBDIR, f"libpf{tag}.stamp")
    fp = _fingerprint(extra_flags)
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == fp:
                return lib
    cc = nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(LIBDIR, src.replace(".cu", f"{tag}.o"))
        objs.append(obj)
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + out.decode(errors="replace"))
        if verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    tmp = lib + ".tmp"
    link = [cc, *ARCH, "-shared", *objs, "-o", tmp]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    with open(stamp, "w") as fh:
        fh.write(fp)
    return lib


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))
