"""Build libbats (the CUDA library behind include/bats.h) in-tree for sm_103a.

    python -m paper_2501_06717_gb300.build [--verbose]

Compiles each CUDA translation unit in parallel with nvcc and links
``_build/libbats.so`` next to this file (CUDA runtime linked statically).
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbats.so")
# the checked build: every kernel index range-tested (tests only)
OUT_CHECKED = os.path.join(HERE, "_build_checked")
SOURCES = ["bats_stage.cu", "bats_stage_flux.cu", "bats_host.cu", "bats_noalloc.cu", "bats_mlp.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "bats_internal.h"), os.path.join(CSRC, "bats_tc.h"),
            os.path.join(CSRC, "bats_stage_kernel.h"), os.path.join(ROOT, "include", "bats.h")]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(verbose=False, force=False, checked=False):
    out = OUT_CHECKED if checked else OUT
    lib = os.path.join(out, "libbats.so")
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(out, s.replace(".cu", ".o"))
        if force or _stale(obj, src):
            cmd = [nvcc, *ARCH, *FLAGS, *(["-DBATS_CHECKED"] if checked else []), "-c", src, "-o", obj]
            if verbose:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for c, r in zip(jobs, res):
        if verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError("nvcc failed: %s" % " ".join(c))
    objs = [os.path.join(out, s.replace(".cu", ".o")) for s in SOURCES]
    if jobs or not os.path.exists(lib):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv, force="--force" in sys.argv, checked="--checked" in sys.argv))
