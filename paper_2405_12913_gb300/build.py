"""Builds the in-tree CUDA library ``_build/libhrt.so`` for sm_103a with nvcc (no cmake, parallel TUs)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhrt.so")
SOURCES = ["api.cu", "mesh_kernels.cu", "ray_kernels.cu", "cosmo.cpp", "noalloc.cu", "adjoint_kernels.cu", "mlp_kernels.cu", "xpass_kernels.cu", "raymesh.cu", "tape.cu", "sort_kernels.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *COMMON, "-x", "cu" if src.endswith(".cu") else "c++", "-c", os.path.join(CSRC, src),
           "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def _callback_blob() -> str:
    """LTO fatbin of the k-space load callback (linked into cuFFT kernels at plan time), embedded as bytes."""
    fatbin = os.path.join(OUT, "kspace_callback.fatbin")
    # compute_100 LTO IR with C++ linkage: the form cuFFT's JIT link accepts (it resolves the plain C++ name
    # and links the IR into its own kernels for the device's sm_103)
    cmd = [nvcc(), "-gencode", "arch=compute_100,code=lto_100", "-dc", "-fatbin", "-O3", "-std=c++17",
           os.path.join(CSRC, "kspace_callback.cu"), "-o", fatbin]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for the callback:\n{r.stdout}\n{r.stderr}")
    data = open(fatbin, "rb").read()
    src = os.path.join(OUT, "kspace_callback_blob.c")
    with open(src, "w") as f:
        f.write("#include <stddef.h>\n")
        f.write("const unsigned char hrt_kspace_callback_fatbin[] __attribute__((aligned(16))) = {\n")
        for i in range(0, len(data), 24):
            f.write(",".join(str(x) for x in data[i:i + 24]) + ",\n")
        f.write("};\n")
        f.write(f"const size_t hrt_kspace_callback_fatbin_size = {len(data)};\n")
    obj = src + ".o"
    r = subprocess.run(["gcc", "-c", "-fPIC", "-O1", src, "-o", obj], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed for the callback blob:\n{r.stderr}")
    return obj


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES + ["kspace_callback.cu"]]
    srcs += [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    srcs.append(os.path.join(os.path.dirname(HERE), "include", "hrt.h"))
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in srcs):
        return LIB
    with cf.ThreadPoolExecutor(len(SOURCES) + 1) as ex:
        blob = ex.submit(_callback_blob)
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
        objs.append(blob.result())
    cmd = [nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lcufft", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
