// Run-time compilation of the bidirectional march for one grid
// (LBM_KERNEL_BIDIR_JIT).  The kernel is the same source as k_step_bidir,
// compiled by NVRTC with the run's nx, ny, pitch and plane as constants:
// every load and store of the 18 population planes then addresses its plane
// and row by an immediate offset instead of integer arithmetic (on the
// 8192x160 capillary: 18.3 instead of 20.8 warp instructions per node).
// The arithmetic is the same code with the same floating-point options, so
// the populations equal those of every other step kernel bit for bit.
//
// Compiled kernels are cached for the life of the process, keyed by storage
// precision, strip width, species model, build flavour and grid; the
// libraries are loaded with cudaLibraryLoadData (context-independent) and
// launched with cudaLaunchKernel.  Header sources are embedded at build time
// (lbm_jit_sources.h, written by build.py), so the library needs only NVRTC
// and the toolkit's own headers at run time.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "lbm.h"
#include "lbm_jit.h"
#include "lbm_jit_sources.h"

namespace sc {
namespace {

using Key = std::tuple<int, int, int, int, int, int, int, long long>;
std::mutex g_mu;
std::map<Key, const void*> g_cache;
std::string g_last_log;

const char* type_name(int precision) {
    switch (precision) {
        case LBM_F64: return "double";
        case LBM_F32: return "float";
        case LBM_F16S: return "__half";
        default: return nullptr;
    }
}

#ifdef LBM_CHECKED
constexpr int kChecked = 1;
#else
constexpr int kChecked = 0;
#endif

}  // namespace

int jit_bidir(int precision, int W, bool gen, int nx, int ny, int pitch, long long plane, const void** fn) {
    if (!fn) return LBM_EINVAL;
    *fn = nullptr;
    const char* tn = type_name(precision);
    if (!tn || (W != 64 && W != 128) || (precision == LBM_F64 && W != 64) || nx < 1 || ny < 1 ||
        plane != (long long)ny * pitch || plane * 18 >= (1LL << 31))
        return LBM_EINVAL;
    const Key key{precision, W, gen ? 1 : 0, kChecked, nx, ny, pitch, plane};
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *fn = it->second;
        return LBM_OK;
    }
    char name[96];
    std::snprintf(name, sizeof(name), "sc::k_step_bidir<%s, %d, %s>", tn, W, gen ? "true" : "false");
    std::string src = "#include \"lbm_kernels.cuh\"\n";
    nvrtcProgram prog = nullptr;
    if (nvrtcCreateProgram(&prog, src.c_str(), "lbm_bidir_jit.cu", kJitHeaderCount, kJitHeaders, kJitHeaderNames) !=
        NVRTC_SUCCESS)
        return LBM_ECUDA;
    nvrtcAddNameExpression(prog, name);
    char dnx[48], dny[48], dpitch[48], dplane[64];
    std::snprintf(dnx, sizeof(dnx), "-DLBM_JIT_NX=%d", nx);
    std::snprintf(dny, sizeof(dny), "-DLBM_JIT_NY=%d", ny);
    std::snprintf(dpitch, sizeof(dpitch), "-DLBM_JIT_PITCH=%d", pitch);
    std::snprintf(dplane, sizeof(dplane), "-DLBM_JIT_PLANE=%lluu", (unsigned long long)plane);
    std::vector<const char*> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device",
                                     "-I" LBM_CUDA_INCLUDE, "-DLBM_JIT_GRID=1", dnx, dny, dpitch, dplane,
                                     // the FP64 units are compiled without contraction, the others with
                                     precision == LBM_F64 ? "--fmad=false" : "--fmad=true"};
    if (kChecked) opts.push_back("-DLBM_CHECKED");
    const nvrtcResult cr = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
    size_t logn = 0;
    nvrtcGetProgramLogSize(prog, &logn);
    g_last_log.assign(logn, '\0');
    if (logn) nvrtcGetProgramLog(prog, &g_last_log[0]);
    int rc = LBM_OK;
    std::vector<char> cubin;
    std::string lowered;
    if (cr != NVRTC_SUCCESS) {
        rc = LBM_ECUDA;
    } else {
        const char* low = nullptr;
        size_t n = 0;
        if (nvrtcGetLoweredName(prog, name, &low) != NVRTC_SUCCESS || !low ||
            nvrtcGetCUBINSize(prog, &n) != NVRTC_SUCCESS || n == 0) {
            rc = LBM_ECUDA;
        } else {
            lowered = low;
            cubin.resize(n);
            if (nvrtcGetCUBIN(prog, cubin.data()) != NVRTC_SUCCESS) rc = LBM_ECUDA;
        }
    }
    nvrtcDestroyProgram(&prog);
    if (rc) return rc;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
        cudaLibraryGetKernel(&kern, lib, lowered.c_str()) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    g_cache[key] = reinterpret_cast<const void*>(kern);
    *fn = reinterpret_cast<const void*>(kern);
    return LBM_OK;
}

const char* jit_last_log() { return g_last_log.c_str(); }

}  // namespace sc
