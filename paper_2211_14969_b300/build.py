"""Build libhps.so (the CUDA library behind include/hps.h) in-tree for sm_103a.

Usage: python -m paper_2211_14969_b300.build  (or build() from Python).
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libhps.so")
SOURCES = ["hps_api.cu", "condense.cu", "merge.cu", "merge_split.cu", "noalloc.cu", "slab.cu", "ozaki.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


OBJ = os.path.join(HERE, "_build")


def _deps(path, seen=None):
    """The file and every header it includes with #include "...", recursively
    (looked up beside it, then in include/)."""
    seen = set() if seen is None else seen
    if path in seen or not os.path.exists(path):
        return seen
    seen.add(path)
    with open(path) as fh:
        for line in fh:
            t = line.strip()
            if t.startswith("#include") and '"' in t:
                name = t.split('"')[1]
                for d in (os.path.dirname(path), os.path.join(ROOT, "include")):
                    cand = os.path.join(d, name)
                    if os.path.exists(cand):
                        _deps(cand, seen)
                        break
    return seen


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _stale():
    srcs = [os.path.join(CSRC, f) for f in SOURCES]
    deps = set().union(*(_deps(f) for f in srcs)) | {os.path.abspath(__file__)}
    return _newer(LIB, deps)


def build(force=False, verbose=False):
    """Compile the sources whose object is out of date (in parallel, objects
    kept in _build/), then link libhps.so."""
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    common = [*ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        common.insert(0, "-Xptxas=-v")
    if os.environ.get("HPS_SPLIT_COMPILE") == "1":   # faster rebuilds while iterating
        common.append("--split-compile=0")
    os.makedirs(OBJ, exist_ok=True)
    objs, cmds = [], []
    for f in SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OBJ, f[:-3] + ".o")
        objs.append(obj)
        if force or verbose or _newer(obj, _deps(src) | {os.path.abspath(__file__)}):
            cmds.append([nvcc, *common, "-c", src, "-o", obj + ".tmp"])
    if verbose:
        for c in cmds:
            print(" ".join(c))
    if cmds:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c), cmds))
        for c, r in zip(cmds, results):
            if r.returncode != 0:
                raise subprocess.CalledProcessError(r.returncode, r.args)
            os.replace(c[-1], c[-1][:-4])
    subprocess.run([nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs], check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
