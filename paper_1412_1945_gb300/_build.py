"""In-tree build of ``libocq.so`` (the CUDA library) with nvcc for sm_103a.

Each ``csrc/*.cu`` file is compiled to an object in parallel, then linked
into one shared library next to this file.  Rebuilds only what changed.
"""
from __future__ import annotations

import glob
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "libocq.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I", INCLUDE, "-I", CSRC] + ARCH


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _digest(paths, extra=""):
    h = hashlib.sha256(extra.encode())
    for p in paths:
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def build(verbose: bool = False, extra_flags=()) -> str:
    """Compile and link ``libocq.so``; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = _headers()
    flags = CFLAGS + list(extra_flags)
    objs, jobs = [], []
    for src in sources:
        tag = _digest([src] + hdr, " ".join(flags))
        obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + "." + tag + ".o")
        objs.append(obj)
        if not os.path.exists(obj):
            cmd = [NVCC] + flags + ["-c", src, "-o", obj]
            jobs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, cmd, p in jobs:
        out, _ = p.communicate()
        if verbose and out:
            print(out.decode(errors="replace"))
        if p.returncode != 0:
            errors.append(f"{os.path.basename(src)}:\n{out.decode(errors='replace')}")
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    link_tag = _digest(objs)
    stamp = SO + ".stamp"
    if jobs or not os.path.exists(SO) or not os.path.exists(stamp) or open(stamp).read() != link_tag:
        tmp = SO + ".tmp"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, SO)
        with open(stamp, "w") as f:
            f.write(link_tag)
    # drop stale objects
    keep = set(objs)
    for o in glob.glob(os.path.join(BUILD, "*.o")):
        if o not in keep:
            os.remove(o)
    return SO


if __name__ == "__main__":
    print(build(verbose=True))
