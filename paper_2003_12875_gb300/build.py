"""Build librfgpu.so in-tree for sm_103a (GB300).

Every translation unit in csrc/ is compiled by nvcc in parallel with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3``; ptxas register
and spill reports go to _build/ptxas.log.  The library links the CUDA runtime
dynamically, so that once torch has loaded ``libcudart.so.13`` the library
shares that runtime instance (streams and allocations interoperate).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librfgpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_lib_dir(nvcc: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return os.path.join(root, "lib64")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    deps.append(os.path.join(HERE, "..", "include", "rf.h"))
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


# the device headers NVRTC compiles per graph (jit.cpp): every kernel gets the
# first list; toy kernels also get the second
PRELUDE_HEADERS = ["rf_internal.h", "rf_device.cuh", "rf_kernels.cuh"]
TOY_PRELUDE_HEADERS = ["rf_toys.cuh"]
FORMULA_PRELUDE_HEADERS = ["rf_expr.cuh"]


def _raw(name: str, headers: list[str]) -> str:
    parts = []
    for h in headers:
        with open(os.path.join(CSRC, h)) as f:
            for line in f:
                t = line.strip()
                if t == "#pragma once" or (t.startswith('#include "') and t.endswith('"')):
                    continue
                parts.append(line)
    body = "".join(parts)
    assert ")RFJIT\"" not in body
    return f'static const char {name}[] = R"RFJIT(\n' + body + '\n)RFJIT";\n'


def write_prelude() -> str:
    """Embed the device headers as C++ raw strings (rf_jit_prelude.inc)."""
    out = os.path.join(BUILD, "rf_jit_prelude.inc")
    text = (_raw("kRfJitPrelude", PRELUDE_HEADERS) + _raw("kRfJitToysPrelude", TOY_PRELUDE_HEADERS)
            + _raw("kRfJitFormulaPrelude", FORMULA_PRELUDE_HEADERS))
    if not os.path.exists(out) or open(out).read() != text:
        with open(out, "w") as f:
            f.write(text)
    return out


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    write_prelude()
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC,
              "-I", BUILD, "-I", os.path.join(HERE, "..", "include")]
    objs, cmds = [], []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        extra = ARCH + ["-Xptxas", "-v"] if src.endswith(".cu") else []
        cmds.append([nvcc, *common, *extra, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    jobs = jobs or min(len(cmds), os.cpu_count() or 4)
    log = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for cmd, r in ex.map(run, cmds):
            log.append(f"$ {' '.join(cmd)}\n{r.stdout}{r.stderr}")
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        f.write("\n".join(log))
    tmp = LIB + f".tmp{os.getpid()}"
    libdir = _cuda_lib_dir(nvcc)
    link = [nvcc, "-shared", *ARCH, "-cudart", "shared", "-o", tmp, *objs,
            "-L", libdir, "-lnvrtc", "-lpthread", "-Xlinker", f"-rpath,{libdir}"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
