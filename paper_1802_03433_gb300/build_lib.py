"""Build libfea.so (the CUDA library behind include/fea.h) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by its own nvcc process (in
parallel), then linked into paper_1802_03433_gb300/libfea.so against the
shared CUDA runtime.  Objects go to paper_1802_03433_gb300/_build/.

build(checked=True) builds the same sources with -DFEA_CHECKED into
libfea_checked.so (objects in _build_checked/): every vertex gather of the
element kernels and every shared-memory slot and CSR position of the
scatters is bounds-checked, a failed check latching DEV_ERR_INDEX
(fea_mesh_check returns FEA_ERR_INDEX) instead of touching memory.  The
binding loads it when FEA_CHECKED=1 is set in the environment.
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
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfea.so")
OUT_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libfea_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def cuda_lib_dir() -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for d in (os.path.join(root, "lib64"), os.path.join(root, "lib")):
        if os.path.exists(os.path.join(d, "libnvrtc.so")):
            return d
    raise RuntimeError(f"libnvrtc.so not found under {root}")


# Headers the runtime-compiled kernels include (NVRTC has no file system view
# of csrc/, so jit.cu carries their text).
JIT_HEADERS = ["devcommon.cuh", "element.cuh", "vecmem.cuh", "elem_user.cuh"]


def gen_jit_headers(out_dir: str = OUT) -> str:
    out = os.path.join(out_dir, "jit_headers.inc")
    texts = []
    for h in JIT_HEADERS:
        with open(os.path.join(CSRC, h)) as f:
            t = f.read()
        if ')FEAJIT"' in t:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        texts.append(t)
    body = ["// Generated by build_lib.py: the headers the runtime-compiled kernels include.",
            f"static const int JIT_HEADER_COUNT = {len(JIT_HEADERS)};",
            "static const char* const JIT_HEADER_NAMES[] = {" + ", ".join(f'"{h}"' for h in JIT_HEADERS) + "};",
            "static const char* const JIT_HEADER_SOURCES[] = {"]
    body.append(",\n".join(f'R"FEAJIT({t})FEAJIT"' for t in texts))
    body.append("};\n")
    new = "\n".join(body)
    if not os.path.exists(out) or open(out).read() != new:
        with open(out, "w") as f:
            f.write(new)
    return out


def _stale(srcs, target) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> str:
    out_dir, lib = (OUT_CHECKED, LIB_CHECKED) if checked else (OUT, LIB)
    os.makedirs(out_dir, exist_ok=True)
    cus = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(os.path.dirname(HERE), "include", "fea.h")]
    if not force and not _stale(cus + hdrs + [__file__], lib):
        return lib
    cc = nvcc()
    gen_jit_headers(out_dir)
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DFEA_CHECKED"] if checked else [])

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        if force or _stale([src] + hdrs + [__file__], obj):
            cmd = [cc, *ARCH, *FLAGS, *extra, "-I", out_dir, "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
            if verbose or ptxas_info:
                sys.stderr.write(r.stderr)
        return obj

    workers = min(len(cus), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, cus))
    tmp = lib + f".tmp{os.getpid()}"
    libdir = cuda_lib_dir()
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-L", libdir, "-lnvrtc",
           "-Xlinker", f"-rpath={libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
