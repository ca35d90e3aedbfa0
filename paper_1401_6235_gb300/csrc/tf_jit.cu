// Runtime specialisation of elementwise programs.
//
// For large arrays twofold_ew / twofold_ew_f32 compile the program itself
// into a straight-line kernel: the operations, operand kinds and flag mode
// become compile-time constants, every input of the thread's elements is
// loaded before any arithmetic (two elements per thread for the
// bandwidth-bound binary32 basis), and no per-step dispatch remains; the
// plain twins are specialised the same way.  The
// source is generated here, compiled once per distinct program by NVRTC for
// sm_103a from the same device headers the library is built from (embedded
// at build time), loaded with cudaLibraryLoadData and cached.  The
// arithmetic is the library's own device code, so the bits are those of the
// generic kernels; any failure to build leaves the call on them.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include <nvrtc.h>

#include "tf_host.cuh"
#include "tf_device_f32.cuh"
#include "tf_jit.h"
#include "tf_jit_sources.inc"     // kJitHeaderNames / kJitHeaders: the device headers as text

namespace tfjit {
namespace {

constexpr int kThreads = 128;

// binary32 is bandwidth-bound: two elements per thread, all loads first
// (four consecutive ones in 16-byte accesses when the arrays allow: the
// twofold chain 1.80 -> 1.64 ms at 2^28, 90 -> 99 % of HBM, the plain twin
// 0.85 -> 0.79 ms); binary64 is bound by its arithmetic: one element per
// thread, more threads.
int elems_of(const Prog &p) { return p.vec4 ? 4 : (p.is_f32 ? 2 : 1); }

std::mutex g_mu;
std::unordered_map<std::string, cudaKernel_t> g_cache;     // nullptr: failed to build
int g_mode = -1;                                            // -1: read TWOFOLD_JIT once
int64_t g_built = 0, g_failed = 0;

int mode_locked() {
    if (g_mode < 0) {
        const char *e = std::getenv("TWOFOLD_JIT");
        g_mode = e && (e[0] == '0' || e[0] == '2') ? e[0] - '0' : 1;
    }
    return g_mode;
}

std::string key_of(const Prog &p) {
    std::string k(p.is_f32 ? "f" : "d");
    char buf[64];
    std::snprintf(buf, sizeof buf, "|%d|%d|%x|%d|%d|%d%d%d|", p.nprog, p.nin, p.dotted_mask, p.flags ? 1 : 0,
                  p.sticky ? 1 : 0, p.plain ? 1 : 0, p.plain_int ? 1 : 0, p.vec4 ? 1 : 0);
    k += buf;
    for (int s = 0; s < p.nprog; ++s) {
        std::snprintf(buf, sizeof buf, "%d,%d,%d,%d;", p.op[s], p.dst[s], p.a[s], p.b[s]);
        k += buf;
    }
    return k;
}

bool unary(int op) { return op == TF_SQRT || op == TF_PSQRT; }

// Register budget as CTAs of 128 per SM, measured on the sqrt((a*b+c)/d)
// chain over 2^28 elements.  binary64: a short program (the chain shape: up
// to 4 inputs, 8 instructions) runs at full occupancy, 16 CTAs (32
// registers, a little spill to L1: 3.6 % faster than 12); longer programs
// keep 12 (40 registers).  binary32 (two elements per thread): the twofold
// kernel at 8 (1.80 ms against 1.83 with the compiler's choice, 1.91 at
// 12), the plain twin at 16 (0.85 ms against 0.97); with four elements per
// thread the twofold kernel at 6 (1.641 ms against 1.647 at 8), the plain
// twin at 16 (0.793 ms against 0.799 at 12).
std::string min_blocks(const Prog &p) {
    if (p.vec4) return p.plain ? ", 16" : ", 6";
    if (p.is_f32) return p.plain ? ", 16" : ", 8";
    return p.nin <= 4 && p.nprog <= 8 ? ", 16" : ", 12";
}

// The binary32 twofold kernel with four consecutive elements per thread:
// each input's heads and tails as one 16-byte load, the results as 16-byte
// stores and the flags as one 4-byte store; the last partial group of the
// array through scalar accesses.
std::string source_vec4(const Prog &p, const bool *used, const bool *written, bool coupled) {
    std::string s = std::string("extern \"C\" __global__ void __launch_bounds__(128") + min_blocks(p) + ") " +
                    (p.plain ? "tf_jit_plain" : "tf_jit_ew") + "(const __grid_constant__ JArgs A) {\n";
    s += "  for (long long j = (long long)blockIdx.x * 128 + threadIdx.x; 4 * j < A.n; j += (long long)gridDim.x * 128) {\n";
    s += "    const long long i0 = 4 * j; const bool full = i0 + 3 < A.n;\n";
    char buf[1024];
    for (int k = 0; k < p.nin; ++k) {
        if (!used[k]) continue;
        const bool dotted = p.plain || ((p.dotted_mask >> k) & 1);
        std::snprintf(buf, sizeof buf,
                      "    float4 h%d, l%d = make_float4(0.f, 0.f, 0.f, 0.f);\n"
                      "    if (full) h%d = *reinterpret_cast<const float4 *>(A.hi[%d] + i0);\n"
                      "    else { h%d = make_float4(A.hi[%d][i0], i0 + 1 < A.n ? A.hi[%d][i0 + 1] : 1.f, "
                      "i0 + 2 < A.n ? A.hi[%d][i0 + 2] : 1.f, 1.f); }\n",
                      k, k, k, k, k, k, k, k);
        s += buf;
        if (!dotted) {
            std::snprintf(buf, sizeof buf,
                          "    if (full) l%d = *reinterpret_cast<const float4 *>(A.lo[%d] + i0);\n"
                          "    else { l%d = make_float4(A.lo[%d][i0], i0 + 1 < A.n ? A.lo[%d][i0 + 1] : 0.f, "
                          "i0 + 2 < A.n ? A.lo[%d][i0 + 2] : 0.f, 0.f); }\n",
                          k, k, k, k, k, k);
            s += buf;
        }
    }
    static const char *const comp[4] = {"x", "y", "z", "w"};
    const int last = p.dst[p.nprog - 1];
    s += "    float r0[4], r1[4];\n    unsigned char fo[4] = {0, 0, 0, 0};\n";
    for (int e = 0; e < 4; ++e) {
        s += "    {\n      unsigned char st = 0;\n";
        for (int k = 0; k < p.nin; ++k) {
            if (!used[k]) continue;
            std::snprintf(buf, sizeof buf, "      T e%dr%d_0 = h%d.%s, e%dr%d_1 = l%d.%s;\n", e, k, k, comp[e], e, k,
                          k, comp[e]);
            s += buf;
        }
        for (int r = p.nin; r < TF_EW_MAX_REGS; ++r)
            if (written[r]) {
                std::snprintf(buf, sizeof buf, "      T e%dr%d_0, e%dr%d_1;\n", e, r, e, r);
                s += buf;
            }
        for (int q = 0; q < p.nprog; ++q) {
            const int op = p.op[q], a = p.a[q], b = p.b[q], d = p.dst[q];
            if (p.plain) {                       // the plain twin: heads only
                std::snprintf(buf, sizeof buf, "      e%dr%d_0 = tf::apply_plain(%d, e%dr%d_0, %s);\n", e, d, op, e, a,
                              unary(op) ? "T(0)" : ("e" + std::to_string(e) + "r" + std::to_string(b) + "_0").c_str());
                s += buf;
                continue;
            }
            const bool xd = a < p.nin && ((p.dotted_mask >> a) & 1);
            const bool yd = unary(op) || (b < p.nin && ((p.dotted_mask >> b) & 1));
            std::string y0 = "T(0)", y1 = "T(0)";
            if (!unary(op)) {
                y0 = "e" + std::to_string(e) + "r" + std::to_string(b) + "_0";
                y1 = "e" + std::to_string(e) + "r" + std::to_string(b) + "_1";
            }
            std::snprintf(buf, sizeof buf,
                          "      { const tf::f2 z = tf::apply_any<%s>(%d, e%dr%d_0, e%dr%d_1, %s, %s, %s, %s); "
                          "e%dr%d_0 = z.z0; e%dr%d_1 = z.z1;%s }\n",
                          coupled ? "true" : "false", op, e, a, e, a, xd ? "true" : "false", y0.c_str(),
                          y1.c_str(), yd ? "true" : "false", e, d, e, d,
                          p.sticky ? " st |= tf::flag_of(z.z0, z.z1, A.fc);" : "");
            s += buf;
        }
        std::snprintf(buf, sizeof buf, "      r0[%d] = e%dr%d_0; r1[%d] = %s;\n", e, e, last, e,
                      p.plain ? "T(0)" : ("e" + std::to_string(e) + "r" + std::to_string(last) + "_1").c_str());
        s += buf;
        if (p.flags && !p.plain) {
            std::snprintf(buf, sizeof buf, "      fo[%d] = tf::flag_of(e%dr%d_0, e%dr%d_1, A.fc) | st;\n", e, e,
                          last, e, last);
            s += buf;
        }
        s += "      (void)st;\n    }\n";
    }
    const bool twofold = !p.plain, fl = p.flags && !p.plain;
    s += "    if (full) {\n"
         "      *reinterpret_cast<float4 *>(A.oh + i0) = make_float4(r0[0], r0[1], r0[2], r0[3]);\n";
    if (twofold) s += "      *reinterpret_cast<float4 *>(A.ol + i0) = make_float4(r1[0], r1[1], r1[2], r1[3]);\n";
    if (fl) s += "      *reinterpret_cast<uchar4 *>(A.fl + i0) = make_uchar4(fo[0], fo[1], fo[2], fo[3]);\n";
    s += "    } else {\n      for (int e = 0; e < 4 && i0 + e < A.n; ++e) {\n        A.oh[i0 + e] = r0[e];\n";
    if (twofold) s += "        A.ol[i0 + e] = r1[e];\n";
    if (fl) s += "        A.fl[i0 + e] = fo[e];\n";
    s += "      }\n    }\n  }\n}\n";
    return s;
}

// Source of the specialised kernel.
std::string source_of(const Prog &p) {
    bool coupled = false, used[TF_EW_MAX_REGS] = {}, written[TF_EW_MAX_REGS] = {};
    for (int s = 0; s < p.nprog; ++s) {
        coupled |= p.op[s] > TF_SQRT;
        used[p.a[s]] = true;
        if (!unary(p.op[s])) used[p.b[s]] = true;
        written[p.dst[s]] = true;
    }
    const char *T = p.is_f32 ? "float" : "double";
    const char *pair = p.is_f32 ? "tf::f2" : "tf::d2";
    std::string s =
        "typedef unsigned long long uint64_t; typedef long long int64_t; typedef unsigned int uint32_t;\n"
        "typedef int int32_t; typedef unsigned short uint16_t; typedef unsigned char uint8_t; typedef signed char int8_t;\n"
        "#include \"tf_device_f32.cuh\"\n";
    s += std::string("typedef ") + T + " T;\n";
    s += std::string("typedef ") + (p.is_f32 ? "tf::FlagCfg32" : "tf::FlagCfg") + " FC;\n";
    s += "struct JArgs { long long n; const T *hi[12]; const T *lo[12]; T *oh; T *ol; unsigned char *fl; FC fc; };\n";
    const int E = elems_of(p);
    if (p.vec4) return s + source_vec4(p, used, written, coupled);
    s += std::string("extern \"C\" __global__ void __launch_bounds__(128") + min_blocks(p) + ") " +
         (p.plain ? "tf_jit_plain" : "tf_jit_ew") + "(const __grid_constant__ JArgs A) {\n";
    s += "  for (long long i0 = (long long)blockIdx.x * " + std::to_string(128 * E) +
         " + threadIdx.x; i0 < A.n; i0 += (long long)gridDim.x * " + std::to_string(128 * E) + ") {\n";
    if (E == 2) s += "    const long long i1 = i0 + 128; const bool v1 = i1 < A.n;\n";
    char buf[512];
    // all loads first, every element of the thread
    for (int e = 0; e < E; ++e) {
        for (int k = 0; k < p.nin; ++k) {
            if (!used[k]) continue;
            const std::string r = "e" + std::to_string(e) + "r" + std::to_string(k), ks = std::to_string(k);
            const bool dotted = p.plain || ((p.dotted_mask >> k) & 1);
            if (e == 0) {
                s += "    T " + r + "_0 = A.hi[" + ks + "][i0];";
                s += " T " + r + "_1 = " + (dotted ? std::string("T(0)") : "A.lo[" + ks + "][i0]") + ";\n";
            } else {
                s += "    T " + r + "_0 = v1 ? A.hi[" + ks + "][i1] : T(1);";
                s += " T " + r + "_1 = " + (dotted ? std::string("T(0)") : "v1 ? A.lo[" + ks + "][i1] : T(0)") + ";\n";
            }
        }
    }
    for (int e = 0; e < E; ++e) {
        s += "    {\n      unsigned char st = 0;\n";
        for (int r = p.nin; r < TF_EW_MAX_REGS; ++r)
            if (written[r]) {
                std::snprintf(buf, sizeof buf, "      T e%dr%d_0, e%dr%d_1;\n", e, r, e, r);
                s += buf;
            }
        for (int q = 0; q < p.nprog; ++q) {
            const int op = p.op[q], a = p.a[q], b = p.b[q], d = p.dst[q];
            if (p.plain) {                       // the plain twin: heads only
                std::snprintf(buf, sizeof buf, "      e%dr%d_0 = tf::apply_plain%s(%d, e%dr%d_0, %s);\n", e, d,
                              p.plain_int ? "_int" : "", op, e, a,
                              unary(op) ? "T(0)" : ("e" + std::to_string(e) + "r" + std::to_string(b) + "_0").c_str());
                s += buf;
                continue;
            }
            const bool xd = a < p.nin && ((p.dotted_mask >> a) & 1);
            const bool yd = unary(op) || (b < p.nin && ((p.dotted_mask >> b) & 1));
            std::string y0 = "T(0)", y1 = "T(0)";
            if (!unary(op)) {
                y0 = "e" + std::to_string(e) + "r" + std::to_string(b) + "_0";
                y1 = "e" + std::to_string(e) + "r" + std::to_string(b) + "_1";
            }
            std::snprintf(buf, sizeof buf,
                          "      { const %s z = tf::apply_any<%s>(%d, e%dr%d_0, e%dr%d_1, %s, %s, %s, %s); "
                          "e%dr%d_0 = z.z0; e%dr%d_1 = z.z1;%s }\n",
                          pair, coupled ? "true" : "false", op, e, a, e, a, xd ? "true" : "false", y0.c_str(),
                          y1.c_str(), yd ? "true" : "false", e, d, e, d,
                          p.sticky ? " st |= tf::flag_of(z.z0, z.z1, A.fc);" : "");
            s += buf;
        }
        const int last = p.dst[p.nprog - 1];
        const char *idx = e == 0 ? "i0" : "i1";
        if (p.plain) std::snprintf(buf, sizeof buf, "      %sA.oh[%s] = e%dr%d_0;\n", e == 0 ? "" : "if (v1) ", idx, e, last);
        else std::snprintf(buf, sizeof buf, "      %s{ A.oh[%s] = e%dr%d_0; A.ol[%s] = e%dr%d_1; }\n",
                           e == 0 ? "" : "if (v1) ", idx, e, last, idx, e, last);
        s += buf;
        if (p.flags && !p.plain) {
            std::snprintf(buf, sizeof buf, "      %sA.fl[%s] = tf::flag_of(e%dr%d_0, e%dr%d_1, A.fc) | st;\n",
                          e == 0 ? "" : "if (v1) ", idx, e, last, e, last);
            s += buf;
        }
        s += "      (void)st;\n    }\n";
    }
    s += "  }\n}\n";
    return s;
}

cudaKernel_t build(const Prog &p) {
    const std::string src = source_of(p);
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "tf_jit_ew.cu", kJitHeaderCount, kJitHeaders, kJitHeaderNames) !=
        NVRTC_SUCCESS)
        return nullptr;
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "--fmad=false", "-default-device",
                          "--ftz=false", "--prec-div=true", "--prec-sqrt=true"};
    const nvrtcResult cr = nvrtcCompileProgram(prog, (int)(sizeof opts / sizeof opts[0]), opts);
    size_t n = 0;
    std::string cubin;
    if (cr == NVRTC_SUCCESS && nvrtcGetCUBINSize(prog, &n) == NVRTC_SUCCESS && n > 0) {
        cubin.resize(n);
        if (nvrtcGetCUBIN(prog, &cubin[0]) != NVRTC_SUCCESS) cubin.clear();
    } else if (std::getenv("TWOFOLD_JIT_LOG")) {
        size_t ln = 0;
        nvrtcGetProgramLogSize(prog, &ln);
        std::string log(ln, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        std::fprintf(stderr, "twofold JIT: compile failed\n%s\n%s\n", src.c_str(), log.c_str());
    }
    nvrtcDestroyProgram(&prog);
    if (cubin.empty()) return nullptr;
    cudaLibrary_t lib;
    const cudaError_t le = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (le != cudaSuccess) {
        if (std::getenv("TWOFOLD_JIT_LOG"))
            std::fprintf(stderr, "twofold JIT: %zu-byte cubin not loaded: %s\n", cubin.size(), cudaGetErrorString(le));
        (void)cudaGetLastError();
        return nullptr;
    }
    cudaKernel_t k;
    if (cudaLibraryGetKernel(&k, lib, p.plain ? "tf_jit_plain" : "tf_jit_ew") != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return k;
}

template <typename T, typename FC>
struct JArgs {
    long long n;
    const T *hi[12];
    const T *lo[12];
    T *oh, *ol;
    unsigned char *fl;
    FC fc;
};

template <typename T, typename FC>
bool launch_impl(const Prog &p_in, const T *const *hi, const T *const *lo, T *oh, T *ol, uint8_t *fl, const FC &fc,
                 int64_t n, cudaStream_t stream, int *status) {
    Prog p = p_in;
    p.vec4 = false;
    if (p.is_f32) {
        // four consecutive elements per thread when every array is 16-byte
        // aligned (the flags 4-byte aligned)
        uintptr_t m = reinterpret_cast<uintptr_t>(oh);
        if (!p.plain) m |= reinterpret_cast<uintptr_t>(ol);
        for (int i = 0; i < p.nin; ++i) {
            m |= reinterpret_cast<uintptr_t>(hi[i]);
            if (!p.plain && !((p.dotted_mask >> i) & 1)) m |= reinterpret_cast<uintptr_t>(lo[i]);
        }
        p.vec4 = (m & 15) == 0 && (p.plain || !p.flags || (reinterpret_cast<uintptr_t>(fl) & 3) == 0);
    }
    cudaKernel_t k;
    {
        std::lock_guard<std::mutex> g(g_mu);
        const int m = mode_locked();
        if (m == 0 || (m == 1 && n < kAutoMinElements)) return false;
        const std::string key = key_of(p);
        auto it = g_cache.find(key);
        if (it == g_cache.end()) {
            k = build(p);
            g_cache.emplace(key, k);
            if (k) ++g_built;
            else ++g_failed;
        } else {
            k = it->second;
        }
    }
    if (!k) return false;
    JArgs<T, FC> A{};
    A.n = n;
    for (int i = 0; i < p.nin; ++i) {
        A.hi[i] = hi[i];
        A.lo[i] = lo[i];
    }
    A.oh = oh;
    A.ol = ol;
    A.fl = fl;
    A.fc = fc;
    const int64_t want = (n + kThreads * elems_of(p) - 1) / (kThreads * elems_of(p));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k, kThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 8;
    }
    const int64_t cap = (int64_t)tfh::sm_count() * per_sm;
    void *args[] = {&A};
    const cudaError_t e =
        cudaLaunchKernel((const void *)k, dim3((unsigned)(want < cap ? want : cap)), dim3(kThreads), args, 0, stream);
    *status = e == cudaSuccess ? TF_OK : TF_ECUDA;
    return true;
}

}  // namespace

bool launch(const Prog &p, const double *const *hi, const double *const *lo, double *oh, double *ol, uint8_t *fl,
            const tf::FlagCfg &fc, int64_t n, cudaStream_t stream, int *status) {
    return launch_impl(p, hi, lo, oh, ol, fl, fc, n, stream, status);
}

bool launch(const Prog &p, const float *const *hi, const float *const *lo, float *oh, float *ol, uint8_t *fl,
            const tf::FlagCfg32 &fc, int64_t n, cudaStream_t stream, int *status) {
    return launch_impl(p, hi, lo, oh, ol, fl, fc, n, stream, status);
}

}  // namespace tfjit

extern "C" int twofold_ew_jit(int32_t mode, int64_t *built, int64_t *failed) {
    std::lock_guard<std::mutex> g(tfjit::g_mu);
    const int prev = tfjit::mode_locked();
    if (mode >= 0 && mode <= 2) tfjit::g_mode = mode;
    else if (mode != -1) return TF_EINVAL;
    if (built) *built = tfjit::g_built;
    if (failed) *failed = tfjit::g_failed;
    return prev;
}
