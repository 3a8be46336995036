"""The step kernel's headers compile under NVRTC, as LBM_KERNEL_BIDIR_JIT
compiles them at run time, for every storage precision, strip width and
species model, with a grid's sizes as constants.  No GPU is needed: this
checks the compile step only (tests/test_gpu_jit.py runs the kernels)."""
import ctypes
import ctypes.util
import glob
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", "lbm.h"),
           os.path.join(ROOT, "paper_0807_0602_gb300", "csrc", "lbm_device.h"),
           os.path.join(ROOT, "paper_0807_0602_gb300", "csrc", "lbm_kernels.cuh")]


def _toolkit():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.realpath(os.path.join(os.path.dirname(os.path.realpath(nvcc)), ".."))


def _nvrtc():
    cands = glob.glob(os.path.join(_toolkit(), "lib64", "libnvrtc.so*")) + [ctypes.util.find_library("nvrtc") or ""]
    for c in cands:
        if c and "builtins" not in c and "alt" not in c:
            try:
                return ctypes.CDLL(c)
            except OSError:
                continue
    pytest.skip("libnvrtc not found")


@pytest.mark.parametrize("ty,W,gen", [("float", 64, "false"), ("float", 128, "true"), ("__half", 64, "false"),
                                      ("__half", 128, "false"), ("double", 64, "false"), ("double", 64, "true")])
def test_bidirectional_march_compiles_for_one_grid(ty, W, gen):
    lib = _nvrtc()
    texts = [open(h, "rb").read() for h in HEADERS]
    names = [os.path.basename(h).encode() for h in HEADERS]
    prog = ctypes.c_void_p()
    hs = (ctypes.c_char_p * 3)(*texts)
    hn = (ctypes.c_char_p * 3)(*names)
    assert lib.nvrtcCreateProgram(ctypes.byref(prog), b'#include "lbm_kernels.cuh"\n', b"jit.cu", 3, hs, hn) == 0
    expr = f"sc::k_step_bidir<{ty}, {W}, {gen}>".encode()
    assert lib.nvrtcAddNameExpression(prog, expr) == 0
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17", b"-default-device",
            b"-I" + os.path.join(_toolkit(), "include").encode(), b"-DLBM_JIT_GRID=1", b"-DLBM_JIT_NX=300",
            b"-DLBM_JIT_NY=41", b"-DLBM_JIT_PITCH=320", b"-DLBM_JIT_PLANE=13120u",
            b"--fmad=false" if ty == "double" else b"--fmad=true"]
    rc = lib.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    n = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(n.value + 1)
    lib.nvrtcGetProgramLog(prog, log)
    assert rc == 0, log.value.decode(errors="replace")[-2000:]
    low = ctypes.c_char_p()
    assert lib.nvrtcGetLoweredName(prog, expr, ctypes.byref(low)) == 0 and low.value.startswith(b"_ZN2sc12k_step_bidir")
    size = ctypes.c_size_t()
    assert lib.nvrtcGetCUBINSize(prog, ctypes.byref(size)) == 0 and size.value > 1000
    lib.nvrtcDestroyProgram(ctypes.byref(prog))


def test_build_embeds_the_headers_verbatim(tmp_path):
    """The library compiles the grid-specific kernel from header text embedded
    at build time: write_jit_sources writes each header as one raw string
    literal, in the order NVRTC is given their names, with the toolkit's
    include directory."""
    from paper_0807_0602_gb300 import build as B
    B.write_jit_sources(str(tmp_path), shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc")
    text = (tmp_path / "lbm_jit_sources.h").read_text()
    assert "kJitHeaderCount = 3" in text
    assert '"lbm.h", "lbm_device.h", "lbm_kernels.cuh"' in text
    inc = text.split('#define LBM_CUDA_INCLUDE "', 1)[1].split('"', 1)[0]
    assert os.path.exists(os.path.join(inc, "cuda_fp16.h"))
    bodies = text.split('R"LBMJIT(')[1:]
    assert len(bodies) == 3
    for h, body in zip(HEADERS, bodies):
        assert body.split(')LBMJIT"', 1)[0] == open(h).read()
