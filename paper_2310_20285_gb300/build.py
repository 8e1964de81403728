"""Build libitergp.so and libitergp_probe.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under ``csrc/`` is compiled in parallel, then linked into
``paper_2310_20285_gb300/libitergp.so`` (the product library, git-ignored); the
throughput probes under ``csrc_probe/`` (bench tooling) go into ``libitergp_probe.so``.
A unit is rebuilt when its source or any header under ``csrc/`` or ``include/`` is newer
than its object.

    python -m paper_2310_20285_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
CSRC_PROBE = os.path.join(PKG, "csrc_probe")
OBJ = os.path.join(ROOT, "_build", "obj")
LIB = os.path.join(PKG, "libitergp.so")
LIB_PROBE = os.path.join(PKG, "libitergp_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA 13 toolkit required)")


def _sources(d=CSRC):
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    inc = os.path.join(ROOT, "include")
    hs += [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]
    return hs


def _compile(nvcc, src, obj, verbose):
    cmd = [nvcc, *ARCH, *CFLAGS, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, r.returncode, r.stdout + r.stderr


def _link(nvcc, objs, lib, rebuilt):
    if rebuilt or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-Xlinker", "--no-undefined", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}{r.stderr}")
        os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    hdr_time = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    todo = []
    targets = {LIB: [], LIB_PROBE: []}
    for lib, srcdir in ((LIB, CSRC), (LIB_PROBE, CSRC_PROBE)):
        for src in _sources(srcdir):
            obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
            targets[lib].append(obj)
            if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_time):
                todo.append((src, obj))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for src, rc, out in ex.map(lambda a: _compile(nvcc, a[0], a[1], verbose), todo):
                if rc != 0:
                    raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{out}")
                if verbose and out.strip():
                    print(out)
    done = {o for _, o in todo}
    for lib, objs in targets.items():
        _link(nvcc, objs, lib, any(o in done for o in objs))
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose))
    sys.exit(0)
