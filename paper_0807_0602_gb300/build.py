"""In-tree build of the CUDA library (sm_103a) behind include/lbm.h.

nvcc compiles each translation unit in parallel, then links one shared
library ``_build/libshanchen_gb300.so``.  The FP64 kernels are compiled with
``--fmad=false`` (no multiply-add contraction), so they evaluate the step in
the documented order with every operation rounded on its own.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libshanchen_gb300.so")
# the checked build (-DLBM_CHECKED): every step kernel validates its tile and
# its run's layout first and reports LBM_EBOUNDS instead of accessing memory
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libshanchen_gb300_checked.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
UNITS = {
    "kernels_f64.cu": ["--fmad=false"],
    "kernels_gen_f64.cu": ["--fmad=false"],
    "kernels_f32.cu": [],
    "kernels_gen_f32.cu": [],
    "kernels_f16.cu": [],
    "kernels_gen_f16.cu": [],
    "lbm_capi.cu": [],
    "mlp.cu": [],
    "lbm_noalloc.cu": [],
    "lbm_selftest.cu": [],
    "lbm_jit.cu": [],
}
# headers that the run-time compiled step kernel includes (embedded into the
# library by write_jit_sources, in this order)
JIT_HEADERS = [os.path.join(INCLUDE, "lbm.h"), os.path.join(CSRC, "lbm_device.h"), os.path.join(CSRC, "lbm_kernels.cuh")]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return p


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + [
        os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def write_jit_sources(build_dir: str, nvcc: str) -> None:
    """Writes lbm_jit_sources.h: the step kernel's headers as string literals
    and the toolkit's include directory (for cuda_fp16.h), for NVRTC."""
    inc = os.path.realpath(os.path.join(os.path.dirname(os.path.realpath(nvcc)), "..", "include"))
    lines = ["// Written by build.py: the headers of the run-time compiled step kernel.", "#pragma once",
             f'#define LBM_CUDA_INCLUDE "{inc}"', f"static const int kJitHeaderCount = {len(JIT_HEADERS)};",
             "static const char* const kJitHeaderNames[] = {" +
             ", ".join(f'"{os.path.basename(h)}"' for h in JIT_HEADERS) + "};",
             "static const char* const kJitHeaders[] = {"]
    for h in JIT_HEADERS:
        with open(h) as fh:
            text = fh.read()
        if ")LBMJIT\"" in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        lines.append('R"LBMJIT(' + text + ')LBMJIT",')
    lines.append("};")
    path = os.path.join(build_dir, "lbm_jit_sources.h")
    new = "\n".join(lines) + "\n"
    if not os.path.exists(path) or open(path).read() != new:
        with open(path, "w") as fh:
            fh.write(new)


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in _sources() + [__file__])


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds the library (the checked variant with checked=True) unless it
    is newer than every source; returns its path."""
    lib_path, build_dir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    defines = ["-DLBM_CHECKED"] if checked else []
    if not force and up_to_date(lib_path):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    write_jit_sources(build_dir, nvcc)
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        src = os.path.join(CSRC, unit)
        if not os.path.exists(src):
            continue
        obj = os.path.join(build_dir, unit.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, "-I" + build_dir, *defines, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    errors = []
    for unit, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{unit}:\n{out.decode(errors='replace')}")
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib_path + f".tmp{os.getpid()}"
    libdir = os.path.realpath(os.path.join(os.path.dirname(os.path.realpath(nvcc)), "..", "lib64"))
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lnvrtc", "-Xlinker", "-rpath", "-Xlinker", libdir]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
