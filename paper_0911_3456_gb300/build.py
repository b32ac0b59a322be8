"""Build libfbcorr.so in-tree with nvcc for sm_103a.

Steps: embed the NVRTC kernel templates (rtcg_direct.cuh, rtcg_ptx.cuh,
rtcg_tc.cuh, rtcg_nn.cuh and their parameter headers) as strings, compile
every csrc/*.cu translation unit in parallel, link one shared library that
statically links the CUDA runtime and dynamically links NVRTC.  Usage:
``python -m paper_0911_3456_gb300.build`` or ``build()`` from Python.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "fbcorr")
LIB = os.path.join(PKG, "libfbcorr.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _embed():
    out = os.path.join(CSRC, "_embedded_src.inc")
    body = "// generated by build.py from the NVRTC kernel sources -- do not edit\n"
    for fname, var in (("rtcg_direct.cuh", "kRtcgDirectSrc"), ("tc_params.h", "kRtcgTcParamsSrc"),
                       ("rtcg_ptx.cuh", "kRtcgPtxSrc"), ("rtcg_tc.cuh", "kRtcgTcSrc"),
                       ("nn_params.h", "kRtcgNnParamsSrc"), ("rtcg_nn.cuh", "kRtcgNnSrc")):
        text = open(os.path.join(CSRC, fname)).read()
        assert ')FBCSRC"' not in text
        body += "static const char " + var + '[] = R"FBCSRC(' + text + ')FBCSRC";\n'
    if not os.path.exists(out) or open(out).read() != body:
        with open(out, "w") as f:
            f.write(body)


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-Wall", "-I", INCLUDE, "-I", CSRC, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    nvcc = _nvcc()
    cuda = _cuda_home(nvcc)
    os.makedirs(BUILD, exist_ok=True)
    _embed()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = srcs + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.inc")) + [os.path.join(INCLUDE, "fbcorr.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    objs = []
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        futs = {}
        for s in srcs:
            o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
            objs.append(o)
            futs[ex.submit(_compile, nvcc, s, o, extra)] = s
        for f in cf.as_completed(futs):
            msg = f.result()
            if verbose and msg:
                print(f"== {os.path.basename(futs[f])}\n{msg}", file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    libdir = os.path.join(cuda, "lib64")
    if not os.path.isdir(libdir):
        libdir = os.path.join(cuda, "lib")
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-L", libdir, "-lnvrtc",
           "-Xlinker", "-rpath," + libdir, "-Xlinker", "--no-undefined"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
