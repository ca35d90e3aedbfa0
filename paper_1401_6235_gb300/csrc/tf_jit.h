// Runtime specialisation of elementwise programs (tf_jit.cu): the program in
// a fixed form, and the launch of its compiled kernel.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/twofold.h"
#include "tf_device_f32.cuh"

namespace tfjit {

// Below this many elements the generic kernels run (a compile costs ~1 s).
constexpr int64_t kAutoMinElements = int64_t(1) << 20;

struct Prog {
    int nprog, nin;
    int8_t op[TF_EW_MAX_PROG], dst[TF_EW_MAX_PROG], a[TF_EW_MAX_PROG], b[TF_EW_MAX_PROG];
    uint32_t dotted_mask;       // bit k: input k has no tail
    bool flags, sticky, is_f32;
    bool plain;                 // the plain twin: heads only, one output
    bool plain_int;             // plain twin: division and root on the integer pipes
    bool vec4;                  // binary32 twofold: four consecutive elements per thread in
                                // 16-byte accesses (set at launch when every array allows it)
};

// Launches the program's specialised kernel and returns true (status: the
// launch's), or returns false when the generic kernels must run (mode off,
// a small n in automatic mode, or no kernel could be built).
bool launch(const Prog &p, const double *const *hi, const double *const *lo, double *oh, double *ol, uint8_t *fl,
            const tf::FlagCfg &fc, int64_t n, cudaStream_t stream, int *status);
bool launch(const Prog &p, const float *const *hi, const float *const *lo, float *oh, float *ol, uint8_t *fl,
            const tf::FlagCfg32 &fc, int64_t n, cudaStream_t stream, int *status);

}  // namespace tfjit
