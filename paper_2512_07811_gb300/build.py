"""Builds the in-tree shared library libqtt.so for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel (one -gencode, no
cmake) and the objects are linked into paper_2512_07811_gb300/libqtt.so.
Objects go to paper_2512_07811_gb300/_build/ (git-ignored).

Whether an object (or the library) is current is decided by content, not by
file times: every object carries a stamp file with the SHA-256 of its source,
of every header it can include, of the compiler flags and of the machine
architecture; the library's stamp hashes the objects' stamps.  A copied tree
whose times say "newer" but whose stamps do not match is rebuilt.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqtt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]


def nvcc() -> str:
    for cand in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the QTT library needs the CUDA toolkit to build")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    hs.append(os.path.join(os.path.dirname(HERE), "include", "qtt.h"))
    return hs


def _digest(paths, extra) -> str:
    h = hashlib.sha256()
    for p in paths:
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    for e in extra:
        h.update(e.encode())
    return h.hexdigest()


def _stamp_ok(stamp: str, target: str, digest: str) -> bool:
    if not (os.path.exists(target) and os.path.exists(stamp)):
        return False
    with open(stamp) as f:
        return f.read().strip() == digest


def _write_stamp(stamp: str, digest: str) -> None:
    with open(stamp, "w") as f:
        f.write(digest + "\n")


def _compile(src: str) -> tuple[str, str]:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    stamp = obj + ".sha256"
    digest = _digest([src] + _headers(), ARCH + FLAGS + [platform.machine()])
    if _stamp_ok(stamp, obj, digest):
        return obj, digest
    if os.path.exists(stamp):
        os.remove(stamp)
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    _write_stamp(stamp, digest)
    return obj, digest


def build(verbose: bool = True) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        done = list(ex.map(_compile, srcs))
    objs = [o for o, _ in done]
    lib_digest = hashlib.sha256("".join(d for _, d in done).encode()).hexdigest()
    lib_stamp = os.path.join(BUILD, "libqtt.so.sha256")
    if _stamp_ok(lib_stamp, LIB, lib_digest):
        return LIB
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    _write_stamp(lib_stamp, lib_digest)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build()
