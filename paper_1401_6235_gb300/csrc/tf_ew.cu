// twofold_ew / plain_ew (binary64) and twofold_ew_f32 / plain_ew_f32
// (binary32): straight-line programs of twofold operations over arrays (the
// array functions vtadd2/vtadd1/vtadd... of the paper's C++ test code,
// generalised to a fused chain so intermediates never touch HBM).
//
// One thread evaluates one element at a time in a grid-stride loop.
// Inputs are read from global memory when an instruction first needs them;
// temporaries live in a per-thread column of shared memory (layout
// [temp][hi|lo][thread], so a warp touches consecutive words: no bank
// conflicts), or in registers for chain-shaped programs.  The program is
// warp-uniform, so its dispatch never diverges.  Kernels are instantiated
// per number type and with or without the coupled operations.
#include "tf_host.cuh"
#include "tf_device_f32.cuh"
#include "tf_jit.h"

namespace {

constexpr int kThreads = 128;

template <typename T> struct FlagOf;
template <> struct FlagOf<double> { using type = tf::FlagCfg; };
template <> struct FlagOf<float> { using type = tf::FlagCfg32; };

template <typename T>
struct EwArgs {
    int64_t n;
    int nprog, nin, ntemp, last;
    int8_t op[TF_EW_MAX_PROG], dst[TF_EW_MAX_PROG], a[TF_EW_MAX_PROG], b[TF_EW_MAX_PROG];
    const T *hi[TF_EW_MAX_INPUTS];
    const T *lo[TF_EW_MAX_INPUTS];
    T *out_hi, *out_lo;
    uint8_t *flags;
    typename FlagOf<T>::type fc;
};

template <typename T, bool P>
__global__ void __launch_bounds__(kThreads) ew_kernel(const __grid_constant__ EwArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *regs = reinterpret_cast<T *>(smem_raw);      // [ntemp][2][kThreads]
    const int t = threadIdx.x;
    const bool sticky_on = (A.fc.mode & TF_PANIC_STICKY) != 0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + t; i < A.n; i += (int64_t)gridDim.x * kThreads) {
        uint8_t sticky = 0;
        for (int s = 0; s < A.nprog; ++s) {
            const int op = A.op[s], ra = A.a[s], rb = A.b[s];
            T x0, x1 = T(0), y0 = T(0), y1 = T(0);
            bool xd = false, yd = true;
            if (ra < A.nin) {
                x0 = A.hi[ra][i];
                xd = A.lo[ra] == nullptr;
                if (!xd) x1 = A.lo[ra][i];
            } else {
                x0 = regs[((ra - A.nin) * 2 + 0) * kThreads + t];
                x1 = regs[((ra - A.nin) * 2 + 1) * kThreads + t];
            }
            if (!tf::unary(op)) {
                if (rb < A.nin) {
                    y0 = A.hi[rb][i];
                    yd = A.lo[rb] == nullptr;
                    if (!yd) y1 = A.lo[rb][i];
                } else {
                    y0 = regs[((rb - A.nin) * 2 + 0) * kThreads + t];
                    y1 = regs[((rb - A.nin) * 2 + 1) * kThreads + t];
                    yd = false;
                }
            }
            const auto z = tf::apply_any<P>(op, x0, x1, xd, y0, y1, yd);
            if (sticky_on) sticky |= tf::flag_of(z.z0, z.z1, A.fc);
            const int rd = A.dst[s] - A.nin;
            regs[(rd * 2 + 0) * kThreads + t] = z.z0;
            regs[(rd * 2 + 1) * kThreads + t] = z.z1;
        }
        const int rl = A.last - A.nin;
        const T z0 = regs[(rl * 2 + 0) * kThreads + t];
        const T z1 = regs[(rl * 2 + 1) * kThreads + t];
        A.out_hi[i] = z0;
        A.out_lo[i] = z1;
        if (A.flags) A.flags[i] = tf::flag_of(z0, z1, A.fc) | sticky;
    }
}

// Chain programs: every instruction after the first takes the previous
// result as its first operand and an input (or nothing, for SQRT) as its
// second.  The running twofold stays in registers; no shared memory.
template <typename T>
struct ChainArgs {
    int64_t n;
    int nsteps;
    int first;                                  // input register of the first operand
    int8_t op[TF_EW_MAX_PROG], in[TF_EW_MAX_PROG];   // second operand's input register
    const T *hi[TF_EW_MAX_INPUTS];
    const T *lo[TF_EW_MAX_INPUTS];
    T *out_hi, *out_lo;
    uint8_t *flags;
    typename FlagOf<T>::type fc;
};

template <typename T, bool P>
__global__ void __launch_bounds__(kThreads) chain_kernel(const __grid_constant__ ChainArgs<T> A) {
    const bool sticky_on = (A.fc.mode & TF_PANIC_STICKY) != 0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * kThreads) {
        T x0 = A.hi[A.first][i], x1 = T(0);
        bool xd = A.lo[A.first] == nullptr;
        if (!xd) x1 = A.lo[A.first][i];
        uint8_t sticky = 0;
        for (int s = 0; s < A.nsteps; ++s) {
            const int op = A.op[s];
            T y0 = T(0), y1 = T(0);
            bool yd = true;
            if (!tf::unary(op)) {
                const int k = A.in[s];
                y0 = A.hi[k][i];
                yd = A.lo[k] == nullptr;
                if (!yd) y1 = A.lo[k][i];
            }
            const auto z = tf::apply_any<P>(op, x0, x1, xd, y0, y1, yd);
            if (sticky_on) sticky |= tf::flag_of(z.z0, z.z1, A.fc);
            x0 = z.z0;
            x1 = z.z1;
            xd = false;
        }
        A.out_hi[i] = x0;
        A.out_lo[i] = x1;
        if (A.flags) A.flags[i] = tf::flag_of(x0, x1, A.fc) | sticky;
    }
}

// A validated program in chain form: fills op/in/first and returns true.
template <typename T>
bool as_chain(const int8_t *op, const int8_t *dst, const int8_t *a, const int8_t *b, int nprog, int nin,
              ChainArgs<T> &C) {
    if (a[0] >= nin) return false;
    C.first = a[0];
    for (int s = 0; s < nprog; ++s) {
        if (s > 0 && a[s] != dst[s - 1]) return false;
        const bool un = op[s] == TF_SQRT || op[s] == TF_PSQRT;
        if (!un && b[s] >= nin) return false;
        C.op[s] = op[s];
        C.in[s] = un ? 0 : b[s];
    }
    C.nsteps = nprog;
    return true;
}

template <typename T>
struct PlainArgs {
    int64_t n;
    int nprog, nin, ntemp, last;
    int8_t op[TF_EW_MAX_PROG], dst[TF_EW_MAX_PROG], a[TF_EW_MAX_PROG], b[TF_EW_MAX_PROG];
    const T *in[TF_EW_MAX_INPUTS];
    T *out;
};

// INT: binary64 division and square root on the integer pipes (plain_arith).
template <typename T, bool INT>
__global__ void __launch_bounds__(kThreads) plain_ew_kernel(const __grid_constant__ PlainArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *regs = reinterpret_cast<T *>(smem_raw);      // [ntemp][kThreads]
    const int t = threadIdx.x;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + t; i < A.n; i += (int64_t)gridDim.x * kThreads) {
        for (int s = 0; s < A.nprog; ++s) {
            const int op = A.op[s], ra = A.a[s], rb = A.b[s];
            const T x = ra < A.nin ? A.in[ra][i] : regs[(ra - A.nin) * kThreads + t];
            T y = T(0);
            if (!tf::unary(op)) y = rb < A.nin ? A.in[rb][i] : regs[(rb - A.nin) * kThreads + t];
            T r;
            if constexpr (INT) r = tf::apply_plain_int(op, x, y);
            else r = tf::apply_plain(op, x, y);
            regs[(A.dst[s] - A.nin) * kThreads + t] = r;
        }
        A.out[i] = regs[(A.last - A.nin) * kThreads + t];
    }
}

// Validate a program; returns the number of temporaries needed or -1.
int check_prog(const int32_t *prog, int nprog, int nin, int8_t *op, int8_t *dst, int8_t *a,
               int8_t *b, int *last) {
    if (!prog || nprog < 1 || nprog > TF_EW_MAX_PROG || nin < 1 || nin > TF_EW_MAX_INPUTS) return -1;
    bool defined[TF_EW_MAX_REGS] = {};
    for (int k = 0; k < nin; ++k) defined[k] = true;
    int maxreg = nin - 1;
    for (int s = 0; s < nprog; ++s) {
        const int32_t o = prog[4 * s], d = prog[4 * s + 1], ra = prog[4 * s + 2];
        int32_t rb = prog[4 * s + 3];
        if (o < TF_ADD || o > TF_PSQRT) return -1;
        if (d < nin || d >= TF_EW_MAX_REGS) return -1;
        if (ra < 0 || ra >= TF_EW_MAX_REGS || !defined[ra]) return -1;
        if (o == TF_SQRT || o == TF_PSQRT) rb = ra;
        if (rb < 0 || rb >= TF_EW_MAX_REGS || !defined[rb]) return -1;
        defined[d] = true;
        if (d > maxreg) maxreg = d;
        op[s] = (int8_t)o; dst[s] = (int8_t)d; a[s] = (int8_t)ra; b[s] = (int8_t)rb;
        *last = d;
    }
    return maxreg + 1 - nin;
}

int grid_for(int64_t n, size_t smem, const void *kernel) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t want = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)tfh::sm_count() * per_sm;
    return (int)(want < cap ? want : cap);
}

tf::FlagCfg flag_cfg_of(const tf_params *p, double) { return tfh::flag_cfg(p); }
tf::FlagCfg32 flag_cfg_of(const tf_params *p, float) {
    tf::FlagCfg32 f;
    f.mode = p ? p->panic_mode : TF_PANIC_REL;
    f.tau = p ? (float)p->panic_tau : tfh::kDefaultTau32;
    f.m = p ? (float)p->panic_ulps : (float)tfh::kDefaultUlps;
    return f;
}

template <typename T, typename In, typename Out>
int run_ew(const int32_t *prog, int32_t nprog, const In *in, int32_t nin, int64_t n, Out out,
           const tf_params *p, void *stream) {
    EwArgs<T> A{};
    if (n < 0 || !in || !tfh::params_ok(p)) return TF_EINVAL;
    A.ntemp = check_prog(prog, nprog, nin, A.op, A.dst, A.a, A.b, &A.last);
    if (A.ntemp < 1) return TF_EINVAL;
    if (n == 0) return TF_OK;     // nothing is dereferenced: pointers may be NULL
    if (!tfh::fptr_ok(out.hi) || !tfh::fptr_ok(out.lo)) return TF_EINVAL;
    for (int k = 0; k < nin; ++k) {
        if (!tfh::fptr_ok(in[k].hi) || !tfh::foptr_ok(in[k].lo)) return TF_EINVAL;
        A.hi[k] = in[k].hi;
        A.lo[k] = in[k].lo;
    }
    A.n = n; A.nprog = nprog; A.nin = nin;
    A.out_hi = out.hi; A.out_lo = out.lo; A.flags = out.flags;
    A.fc = flag_cfg_of(p, T(0));
    bool coupled = false;
    for (int q = 0; q < nprog; ++q) coupled |= A.op[q] > TF_SQRT;
    cudaStream_t st = tfh::as_stream(stream);
    // large arrays: the program's own straight-line kernel (compiled once)
    tfjit::Prog jp{};
    jp.nprog = nprog;
    jp.nin = nin;
    for (int q = 0; q < nprog; ++q) {
        jp.op[q] = A.op[q]; jp.dst[q] = A.dst[q]; jp.a[q] = A.a[q]; jp.b[q] = A.b[q];
    }
    for (int k = 0; k < nin; ++k)
        if (!A.lo[k]) jp.dotted_mask |= 1u << k;
    jp.flags = A.flags != nullptr;
    jp.sticky = (A.fc.mode & TF_PANIC_STICKY) != 0;
    jp.is_f32 = sizeof(T) == 4;
    int jst = TF_OK;
    if (tfjit::launch(jp, A.hi, A.lo, A.out_hi, A.out_lo, A.flags, A.fc, n, st, &jst)) return jst;
    ChainArgs<T> C{};
    if (as_chain(A.op, A.dst, A.a, A.b, nprog, nin, C)) {
        C.n = n;
        for (int k = 0; k < nin; ++k) { C.hi[k] = A.hi[k]; C.lo[k] = A.lo[k]; }
        C.out_hi = A.out_hi; C.out_lo = A.out_lo; C.flags = A.flags; C.fc = A.fc;
        if (coupled)
            chain_kernel<T, true><<<grid_for(n, 0, (const void *)chain_kernel<T, true>), kThreads, 0, st>>>(C);
        else
            chain_kernel<T, false><<<grid_for(n, 0, (const void *)chain_kernel<T, false>), kThreads, 0, st>>>(C);
        return tfh::launch_status();
    }
    const size_t smem = (size_t)A.ntemp * 2 * kThreads * sizeof(T);
    const void *kern = coupled ? (const void *)ew_kernel<T, true> : (const void *)ew_kernel<T, false>;
    if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                                cudaSuccess)
        return TF_ECUDA;
    const int grid = grid_for(n, smem, kern);
    if (coupled) ew_kernel<T, true><<<grid, kThreads, smem, st>>>(A);
    else ew_kernel<T, false><<<grid, kThreads, smem, st>>>(A);
    return tfh::launch_status();
}

template <typename T, bool INT>
int launch_plain_generic(const PlainArgs<T> &A, int64_t n, void *stream) {
    const size_t smem = (size_t)A.ntemp * kThreads * sizeof(T);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(plain_ew_kernel<T, INT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return TF_ECUDA;
    const int grid = grid_for(n, smem, (const void *)plain_ew_kernel<T, INT>);
    plain_ew_kernel<T, INT><<<grid, kThreads, smem, tfh::as_stream(stream)>>>(A);
    return tfh::launch_status();
}

template <typename T>
int run_plain(const int32_t *prog, int32_t nprog, const T *const *in, int32_t nin, int64_t n, T *out,
              void *stream) {
    PlainArgs<T> A{};
    if (n < 0 || !in) return TF_EINVAL;
    A.ntemp = check_prog(prog, nprog, nin, A.op, A.dst, A.a, A.b, &A.last);
    if (A.ntemp < 1) return TF_EINVAL;
    if (n == 0) return TF_OK;
    if (!tfh::fptr_ok(out)) return TF_EINVAL;
    for (int k = 0; k < nin; ++k) {
        if (!tfh::fptr_ok(in[k])) return TF_EINVAL;
        A.in[k] = in[k];
    }
    A.n = n; A.nprog = nprog; A.nin = nin; A.out = out;
    tfjit::Prog jp{};
    jp.nprog = nprog;
    jp.nin = nin;
    for (int q = 0; q < nprog; ++q) {
        jp.op[q] = A.op[q]; jp.dst[q] = A.dst[q]; jp.a[q] = A.a[q]; jp.b[q] = A.b[q];
    }
    jp.dotted_mask = (1u << nin) - 1;
    jp.is_f32 = sizeof(T) == 4;
    jp.plain = true;
    const bool use_int = sizeof(T) == 8 && tfh::plain_integer();
    jp.plain_int = use_int;
    const T *nolo[TF_EW_MAX_INPUTS] = {};
    typename FlagOf<T>::type fc{};
    int jst = TF_OK;
    if (tfjit::launch(jp, A.in, nolo, out, nullptr, nullptr, fc, n, tfh::as_stream(stream), &jst)) return jst;
    if constexpr (sizeof(T) == 8) {
        if (use_int) return launch_plain_generic<T, true>(A, n, stream);
    }
    return launch_plain_generic<T, false>(A, n, stream);
}

}  // namespace

extern "C" int twofold_ew(const int32_t *prog, int32_t nprog, const tf_in *in, int32_t nin,
                          int64_t n, tf_out out, const tf_params *p, void *stream) {
    return run_ew<double>(prog, nprog, in, nin, n, out, p, stream);
}

extern "C" int plain_ew(const int32_t *prog, int32_t nprog, const double *const *in, int32_t nin,
                        int64_t n, double *out, void *stream) {
    return run_plain<double>(prog, nprog, in, nin, n, out, stream);
}

extern "C" int plain_arith(int32_t mode) {
    if (mode == -1) return tfh::g_plain_mode.load();
    if (mode != TF_PLAIN_NATIVE && mode != TF_PLAIN_INTEGER) return TF_EINVAL;
    return tfh::g_plain_mode.exchange(mode);
}

extern "C" int twofold_ew_f32(const int32_t *prog, int32_t nprog, const tf_in_f32 *in, int32_t nin,
                              int64_t n, tf_out_f32 out, const tf_params *p, void *stream) {
    return run_ew<float>(prog, nprog, in, nin, n, out, p, stream);
}

extern "C" int plain_ew_f32(const int32_t *prog, int32_t nprog, const float *const *in, int32_t nin,
                            int64_t n, float *out, void *stream) {
    return run_plain<float>(prog, nprog, in, nin, n, out, stream);
}
