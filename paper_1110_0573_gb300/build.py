"""Builds libqt.so in-tree (paper_1110_0573_gb300/_build/) with nvcc for
sm_103a.  Translation units compile in parallel.  A unit is rebuilt when the
SHA-256 of its inputs (its source, every header in csrc/ and include/, the
compiler's version line and the flags) differs from the one recorded beside
its object, or when the object is missing; file times play no part, so objects
copied from another machine are reused only when they were built from the
same sources by the same compiler.  Every build writes
_build/build_record.json: the input hash of each object and whether this run
compiled it.

    python -m paper_1110_0573_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import json
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libqt.so")
RECORD = os.path.join(BUILD, "build_record.json")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          f"-I{os.path.join(ROOT, 'include')}"]


def nvcc() -> str:
    cand = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"),
            shutil.which("nvcc") or ""]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqt")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def _digest(paths, extra):
    h = hashlib.sha256()
    for p in paths:
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    for e in extra:
        h.update(e.encode())
    return h.hexdigest()


def _compiler_id(cc):
    r = subprocess.run([cc, "--version"], capture_output=True, text=True)
    return (r.stdout.strip().splitlines() or [""])[-1] + " " + platform.machine()


def _cmd(cc, src, out, verbose):
    cmd = [cc, *COMMON, *ARCH, "-c", src, "-o", out]
    if src.endswith(".cpp"):
        cmd[1:1] = ["-x", "cu"]
    if verbose:
        cmd.append("-Xptxas=-v")
    return cmd


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    comp = _compiler_id(cc)
    headers = _headers()
    try:
        with open(RECORD) as f:
            old = json.load(f).get("objects", {})
    except (OSError, ValueError):
        old = {}
    jobs, objs, record = [], [], {}
    for src in _sources():
        name = os.path.basename(src) + ".o"
        obj = os.path.join(BUILD, name)
        objs.append(obj)
        # the flags without this checkout's absolute paths, so that the same
        # sources reached through another path (a symlink) keep their objects
        flags = " ".join(_cmd(cc, src, "", False)).replace(ROOT, "<root>")
        key = _digest([src, *headers], [comp, flags])
        fresh = not force and os.path.exists(obj) and old.get(name, {}).get("inputs") == key
        record[name] = {"inputs": key, "compiled": not fresh}
        if not fresh:
            jobs.append((_cmd(cc, src, obj + ".tmp", verbose), obj))

    def run(job):
        cmd, obj = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{r.stdout}\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for out in ex.map(run, jobs):
                if verbose and out:
                    sys.stderr.write(out)
    lib_key = _digest(objs, [comp])
    try:
        with open(RECORD) as f:
            old_lib = json.load(f).get("library", {}).get("inputs")
    except (OSError, ValueError):
        old_lib = None
    relink = force or bool(jobs) or not os.path.exists(LIB) or old_lib != lib_key
    if relink:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc, "-shared", *ARCH, "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    with open(RECORD + ".tmp", "w") as f:
        json.dump({"compiler": comp, "objects": record,
                   "library": {"inputs": lib_key, "linked": relink}}, f, indent=1)
    os.replace(RECORD + ".tmp", RECORD)
    rebuilt = [n for n, r in record.items() if r["compiled"]]
    if rebuilt:
        sys.stderr.write(f"libqt: compiled {len(rebuilt)} of {len(record)} units: "
                         f"{', '.join(sorted(rebuilt))}\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
