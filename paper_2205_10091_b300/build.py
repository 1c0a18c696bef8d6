"""Build libtc_b300.so in-tree with nvcc for sm_103a (no JIT, no torch extension).

Usage: python -m paper_2205_10091_b300.build [--force] [--debug]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libtc_b300.so")

SOURCES = ["sv_kernels.cu", "planner.cpp", "abi.cpp", "jit.cpp", "noalloc.cu", "tn.cpp", "tn_kernels.cu", "tn_tc.cu", "qgt.cu", "server.cpp", "dm.cpp",
           "dm_kernels.cu", "small.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", os.path.join(ROOT, "include"),
          "-I", BUILD]


# device headers compiled again at run time by the specialised pass kernels
JIT_HEADERS = ["plan.h", "sv_args.h", "sv_core.cuh"]
JIT_INC = os.path.join(BUILD, "jit_headers.inc")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "tc.h"))
    return hs


def _write_jit_headers():
    """Embed the device headers as string literals (jit.cpp hands them to NVRTC)."""
    names, srcs = [], []
    for h in JIT_HEADERS:
        with open(os.path.join(CSRC, h)) as f:
            text = f.read()
        assert ")TCJIT\"" not in text
        names.append(h)
        srcs.append(text)
    body = "static const int kJitHeaderCount = %d;\n" % len(names)
    body += "static const char* const kJitHeaderNames[] = {%s};\n" % ", ".join('"%s"' % n for n in names)
    body += "static const char* const kJitHeaderSrcs[] = {\n"
    body += ",\n".join('R"TCJIT(%s)TCJIT"' % t for t in srcs)
    body += "};\n"
    old = open(JIT_INC).read() if os.path.exists(JIT_INC) else None
    if old != body:
        with open(JIT_INC, "w") as f:
            f.write(body)


def _compile(src: str, debug: bool, verbose: bool) -> str:
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    newest = max([os.path.getmtime(path)] + [os.path.getmtime(h) for h in _headers() + [JIT_INC]])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    cmd = [NVCC] + ARCH + COMMON + (["-DTC_DEBUG=1"] if debug else [])
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"] if verbose else []
        cmd += ["-x", "cu"]
    cmd += ["-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, debug: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    _write_jit_headers()
    if force:
        for f in os.listdir(BUILD):
            if f.endswith(".o"):
                os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, debug, verbose), SOURCES))
    if not os.path.exists(LIB) or max(os.path.getmtime(o) for o in objs) > os.path.getmtime(LIB) or force:
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart", "-lnvrtc"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, debug="--debug" in sys.argv, verbose="-v" in sys.argv))
