"""Build libtwofold.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit compiles in its own nvcc process (in parallel), then
one link step writes ``libtwofold.so`` next to this file.  Device code is
compiled with -fmad=false so no multiply-add is ever contracted.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libtwofold.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-fmad=false", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
              "-Xptxas", "-v"]
SOURCES = ["tf_abi.cu", "tf_ew.cu", "tf_reduce.cu", "tf_reduce32.cu", "tf_horner.cu", "tf_batch.cu", "tf_serve.cu",
           "tf_jit.cu", "tf_probe.cu"]
# device headers the runtime compiler of tf_jit.cu gets as text (embedded at build time)
JIT_HEADERS = ["tf_soft.cuh", "tf_device.cuh", "tf_device_f32.cuh"]
CUDA_LIB = "/usr/local/cuda/lib64"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtwofold.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _jit_sources(path: str) -> None:
    """Write the JIT's device headers as C string literals (only when changed)."""
    parts = ["// generated by build.py from csrc/" + ", csrc/".join(JIT_HEADERS) + "\n",
             f"static const int kJitHeaderCount = {len(JIT_HEADERS)};\n",
             "static const char *const kJitHeaderNames[] = {" + ", ".join(f'"{h}"' for h in JIT_HEADERS) + "};\n",
             "static const char *const kJitHeaders[] = {\n"]
    for h in JIT_HEADERS:
        text = open(os.path.join(CSRC, h)).read()
        assert ")TFJITSRC" not in text
        parts.append('R"TFJITSRC(' + text + ')TFJITSRC",\n')
    parts.append("};\n")
    body = "".join(parts)
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as f:
            f.write(body)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    _jit_sources(os.path.join(BUILD, "tf_jit_sources.inc"))
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "twofold.h"))
    headers.append(os.path.join(BUILD, "tf_jit_sources.inc"))
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *NVCC_FLAGS, "-I", BUILD, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with ThreadPoolExecutor(max(1, len(jobs))) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        for log in logs:
            sys.stderr.write(log)
    if force or jobs or _stale(OUT, objs):
        tmp = OUT + f".tmp{os.getpid()}"
        run([nvcc(), *ARCH, "-shared", *objs, "-o", tmp, "-lcudart", "-lnvrtc", "-L", CUDA_LIB,
             "-Xlinker", "-rpath", "-Xlinker", CUDA_LIB])
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
