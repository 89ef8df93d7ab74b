// NVRTC compilation of expression integrands.  libnvrtc is opened on first
// use (dlopen), so the library loads and runs registry integrands on hosts
// without it; an expression then fails with ZMC_ERR_COMPILE.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "jit.h"
#include "zmc_layout.h"

// kJitHeaderNames / kJitHeaders / kJitNumHeaders: the device headers as
// strings, generated from csrc/ by the package build step.
#include "jit_sources.inc"

namespace zmc {

namespace {

struct Nvrtc {
    bool tried = false, ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*,
                          const char* const*) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char* const*) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t*) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char*) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t*) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char*) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram*) = nullptr;
    const char* (*err)(nvrtcResult) = nullptr;
};

Nvrtc g_nvrtc;
std::mutex g_mu;
std::map<std::string, const void*> g_cache;

template <class T>
bool sym(void* lib, const char* name, T& out) {
    out = reinterpret_cast<T>(dlsym(lib, name));
    return out != nullptr;
}

bool load_nvrtc() {
    if (g_nvrtc.tried) return g_nvrtc.ok;
    g_nvrtc.tried = true;
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void* lib = nullptr;
    for (const char* n : names)
        if ((lib = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
    if (!lib) {
        g_nvrtc.why = "libnvrtc could not be opened";
        return false;
    }
    Nvrtc& N = g_nvrtc;
    N.ok = sym(lib, "nvrtcCreateProgram", N.create) && sym(lib, "nvrtcCompileProgram", N.compile) &&
           sym(lib, "nvrtcGetProgramLogSize", N.log_size) && sym(lib, "nvrtcGetProgramLog", N.log) &&
           sym(lib, "nvrtcGetCUBINSize", N.cubin_size) && sym(lib, "nvrtcGetCUBIN", N.cubin) &&
           sym(lib, "nvrtcDestroyProgram", N.destroy) && sym(lib, "nvrtcGetErrorString", N.err);
    if (!N.ok) N.why = "libnvrtc lacks an expected entry point";
    return N.ok;
}

bool ident_char(char c) {
    return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9') || c == '_';
}

// Keep FP32 expressions in FP32: give unsuffixed floating literals an 'f'.
std::string float_literals(const std::string& e) {
    std::string out;
    size_t i = 0;
    while (i < e.size()) {
        const char c = e[i];
        const bool starts = (c >= '0' && c <= '9') ||
                            (c == '.' && i + 1 < e.size() && e[i + 1] >= '0' && e[i + 1] <= '9');
        if (!starts || (i > 0 && ident_char(e[i - 1]))) {
            out += c;
            ++i;
            continue;
        }
        if (c == '0' && i + 1 < e.size() && (e[i + 1] == 'x' || e[i + 1] == 'X')) {
            while (i < e.size() && ident_char(e[i])) out += e[i++];
            continue;
        }
        size_t j = i;
        bool is_float = false;
        while (j < e.size() && e[j] >= '0' && e[j] <= '9') ++j;
        if (j < e.size() && e[j] == '.') {
            is_float = true;
            ++j;
            while (j < e.size() && e[j] >= '0' && e[j] <= '9') ++j;
        }
        if (j < e.size() && (e[j] == 'e' || e[j] == 'E')) {
            size_t k = j + 1;
            if (k < e.size() && (e[k] == '+' || e[k] == '-')) ++k;
            if (k < e.size() && e[k] >= '0' && e[k] <= '9') {
                is_float = true;
                j = k;
                while (j < e.size() && e[j] >= '0' && e[j] <= '9') ++j;
            }
        }
        out.append(e, i, j - i);
        const bool suffixed = j < e.size() && (e[j] == 'f' || e[j] == 'F' || e[j] == 'l' || e[j] == 'L');
        if (is_float && !suffixed) out += 'f';
        i = j;
    }
    return out;
}


// The expression as pasted into the kernel: one C++ expression, FP32
// literals in the FP32 modes.  ZMC_OK or ZMC_ERR_ARG / ZMC_ERR_COMPILE.
int prepare_expression(const char* expr, int mode, std::string* e, std::string* log) {
    *e = expr ? expr : "";
    if (e->empty()) {
        *log = "empty expression";
        return ZMC_ERR_ARG;
    }
    for (size_t i = 0; i < e->size(); ++i) {
        const char c = (*e)[i];
        if (c == ';' || c == '{' || c == '}' || c == '#' || c == '"' || c == '\\' || c == '\'' ||
            (c == '/' && i + 1 < e->size() && ((*e)[i + 1] == '/' || (*e)[i + 1] == '*'))) {
            *log = "expression may not contain ; { } # quotes, backslashes or comments";
            return ZMC_ERR_COMPILE;
        }
    }
    if (mode != ZMC_FP64) *e = float_literals(*e);
    return ZMC_OK;
}

// NVRTC: the sampling kernel with expression `e` for compute capability
// major.minor, as a cubin.  Needs no device.
int nvrtc_cubin(const std::string& e, int dim, int mode, int major, int minor,
                std::vector<char>* cubin, std::string* log) {
    if (!load_nvrtc()) {
        *log = "expression integrands need NVRTC: " + g_nvrtc.why;
        return ZMC_ERR_COMPILE;
    }
    std::string src =
        "typedef unsigned int uint32_t;\ntypedef int int32_t;\n"
        "typedef long long int64_t;\ntypedef unsigned long long uint64_t;\n"
        "typedef unsigned long size_t;\n"
        "#include \"eval_kernel.cuh\"\n"
        "struct ZmcUserExpr {\n"
        "  template <typename R>\n"
        "  static __device__ __forceinline__ R eval(const R* x, const R* p) {\n"
        "    return (R)(" + e + ");\n  }\n};\n"
        "extern \"C\" __global__ void __launch_bounds__(zmc::kEvalMaxThreads, zmc::eval_min_blocks<" + std::to_string(mode) + ">())\n"
        "zmc_eval_expr(const zmc::Desc* __restrict__ desc, zmc::State* st,\n"
        "              const uint32_t* __restrict__ parents, double2* __restrict__ sums, int level,\n"
        "              const zmc::PhiloxKeys keys) {\n"
        "  zmc::eval_expr_body<" + std::to_string(mode) + ", " + std::to_string(dim) +
        ", ZmcUserExpr>(desc, st, parents, sums, level, keys);\n}\n";
    nvrtcProgram prog = nullptr;
    nvrtcResult r = g_nvrtc.create(&prog, src.c_str(), "zmc_expr.cu", kJitNumHeaders, kJitHeaders,
                                   kJitHeaderNames);
    if (r != NVRTC_SUCCESS) {
        *log = std::string("nvrtcCreateProgram: ") + g_nvrtc.err(r);
        return ZMC_ERR_COMPILE;
    }
    const std::string arch = "-arch=sm_" + std::to_string(major * 10 + minor) + (major >= 9 ? "a" : "");
#ifdef ZMC_CHECKED
    const char* opts[] = {arch.c_str(), "-std=c++17", "-default-device", "-lineinfo",
                          "-DZMC_CHECKED"};
#else
    const char* opts[] = {arch.c_str(), "-std=c++17", "-default-device", "-lineinfo"};
#endif
    r = g_nvrtc.compile(prog, (int)(sizeof opts / sizeof opts[0]), opts);
    size_t ls = 0;
    g_nvrtc.log_size(prog, &ls);
    std::string clog(ls, '\0');
    if (ls) g_nvrtc.log(prog, &clog[0]);
    if (r != NVRTC_SUCCESS) {
        *log = "expression failed to compile:\n" + clog;
        g_nvrtc.destroy(&prog);
        return ZMC_ERR_COMPILE;
    }
    size_t cs = 0;
    g_nvrtc.cubin_size(prog, &cs);
    cubin->assign(cs, 0);
    g_nvrtc.cubin(prog, cubin->data());
    g_nvrtc.destroy(&prog);
    return ZMC_OK;
}

}  // namespace

int jit_compile(const char* expr, int dim, int n_params, int mode, JitKernel* out,
                std::string* log) {
    std::string e;
    int rc = prepare_expression(expr, mode, &e, log);
    if (rc != ZMC_OK) return rc;
    const std::string key = std::to_string(dim) + "|" + std::to_string(n_params) + "|" +
                            std::to_string(mode) + "|" + e;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        out->kernel = it->second;
        return ZMC_OK;
    }
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    std::vector<char> cubin;
    rc = nvrtc_cubin(e, dim, mode, major, minor, &cubin, log);
    if (rc != ZMC_OK) return rc;
    cudaLibrary_t lib = nullptr;
    cudaError_t ce = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce != cudaSuccess) {
        *log = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(ce);
        return ZMC_ERR_CUDA;
    }
    cudaKernel_t k = nullptr;
    ce = cudaLibraryGetKernel(&k, lib, "zmc_eval_expr");
    if (ce != cudaSuccess) {
        *log = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(ce);
        return ZMC_ERR_CUDA;
    }
    g_cache[key] = (const void*)k;
    out->kernel = (const void*)k;
    return ZMC_OK;
}

int jit_check(const char* expr, int dim, int mode, int major, int minor, std::string* log) {
    std::string e;
    int rc = prepare_expression(expr, mode, &e, log);
    if (rc != ZMC_OK) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    std::vector<char> cubin;
    return nvrtc_cubin(e, dim, mode, major, minor, &cubin, log);
}

void jit_release(JitKernel* k) {
    // Compiled kernels stay in the process-wide cache until exit.
    if (k) k->kernel = nullptr;
}

}  // namespace zmc
