// Host-side helpers shared by the library's translation units: parameter
// defaults, argument checks, launch-error mapping.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstddef>

#include "../../include/twofold.h"
#include "tf_device.cuh"

namespace tfh {

constexpr double kDefaultTau = 0x1p-40;
constexpr float kDefaultTau32 = 0x1p-18f;     // binary32: the same share of the significand as 2^-40 of 53 bits
constexpr double kDefaultUlps = 4096.0;
constexpr int kDefaultLeaf = 256;

inline tf::FlagCfg flag_cfg(const tf_params *p) {
    tf::FlagCfg f;
    f.mode = p ? p->panic_mode : TF_PANIC_REL;
    f.tau = p ? p->panic_tau : kDefaultTau;
    f.m = p ? p->panic_ulps : kDefaultUlps;
    // tau = 2^k with -1074 <= k <= 0 and a normal power of two: integer scaling
    f.k = 1;
    int e = 0;
    if (f.tau > 0.0 && std::frexp(f.tau, &e) == 0.5 && e - 1 <= 0 && e - 1 >= -1022) f.k = e - 1;
    return f;
}

inline bool params_ok(const tf_params *p) {
    if (!p) return true;
    if ((p->panic_mode & ~TF_PANIC_STICKY) != TF_PANIC_REL && (p->panic_mode & ~TF_PANIC_STICKY) != TF_PANIC_ULP)
        return false;
    if (p->leaf < 1) return false;
    if (!(p->panic_tau >= 0.0) || !(p->panic_ulps >= 0.0)) return false;   // also rejects NaN
    return true;
}

// plain_arith: TF_PLAIN_INTEGER makes the plain binary64 twins use the
// integer-pipe routines of tf_soft.cuh where they are faster (same bits).
inline std::atomic<int> g_plain_mode{TF_PLAIN_NATIVE};
inline bool plain_integer() { return g_plain_mode.load(std::memory_order_relaxed) == TF_PLAIN_INTEGER; }

inline int leaf_of(const tf_params *p) { return p ? p->leaf : kDefaultLeaf; }

inline bool aligned8(const void *ptr) { return ((uintptr_t)ptr & 7u) == 0; }
inline bool dptr_ok(const void *ptr) { return ptr != nullptr && aligned8(ptr); }
inline bool optr_ok(const void *ptr) { return ptr == nullptr || aligned8(ptr); }

// Element pointers of either basis: non-null (or nullable) and aligned to the element.
template <typename T>
inline bool fptr_ok(const T *ptr) { return ptr != nullptr && ((uintptr_t)ptr % sizeof(T)) == 0; }
template <typename T>
inline bool foptr_ok(const T *ptr) { return ptr == nullptr || ((uintptr_t)ptr % sizeof(T)) == 0; }

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TF_OK : TF_ECUDA;
}

// Launch with programmatic stream serialization: the kernel may begin while
// its predecessor in the stream finishes, and must call griddepcontrol.wait
// before it touches memory that the predecessor may write or read.
template <typename Arg>
inline cudaError_t launch_pdl(void (*kernel)(Arg), int64_t grid, int block, size_t smem, cudaStream_t s,
                              const Arg &a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

inline int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 148;
    }
    return sms;
}

}  // namespace tfh
