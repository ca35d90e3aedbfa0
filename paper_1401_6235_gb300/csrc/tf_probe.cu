// Issue-rate probes of the SM's execution pipes (measurement only; the paper
// has no counterpart).  The binary64 twofold kernels are bound by the FP64
// pipe and the integer pipes, not by HBM, so their roofline needs the rate
// at which one SM retires each kind of instruction.  Each probe runs long
// unrolled streams of one instruction over 8 independent register chains
// per thread; every CTA stamps its SM id and its start and end SM clocks
// (clock64, taken by thread 0 between barriers), and the host turns the
// stamps into lane operations per SM clock: per SM, the CTAs' operations
// over the span from the first start to the last end.  The result does not
// depend on the SM clock frequency.  The latency form runs the same number
// of instructions as ONE dependent chain per thread: with one warp per SM,
// 32 lanes over the measured rate is the latency of one instruction.
#include "tf_host.cuh"

namespace {

constexpr int kChains = 8;     // independent chains per thread
constexpr int kRepeat = 16;    // chain rounds per loop iteration (loop overhead below 2 %)

__device__ __forceinline__ unsigned smid() {
    unsigned s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

// One instruction of the probed kind on chain j.  Integer chains mix in a
// neighbour chain, so that no two steps fold into one instruction (chains
// of associative integer adds or logic ops are not used: the compiler
// merges them into three-input instructions).
template <int OP>
__device__ __forceinline__ void step(double (&d)[kChains], float (&f)[kChains], uint32_t (&u)[kChains],
                                     uint64_t (&w)[kChains], int j, double a, double b, float af, float bf,
                                     uint32_t m) {
    if constexpr (OP == TF_PROBE_DADD) {
        asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(d[j]) : "d"(a));
    } else if constexpr (OP == TF_PROBE_DMUL) {
        asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(d[j]) : "d"(a));
    } else if constexpr (OP == TF_PROBE_DFMA) {
        asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[j]) : "d"(a), "d"(b));
    } else if constexpr (OP == TF_PROBE_FFMA) {
        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[j]) : "f"(af), "f"(bf));
    } else if constexpr (OP == TF_PROBE_IMAD) {
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(u[j]) : "r"(m), "r"(u[(j + 1) & 7]));
    } else if constexpr (OP == TF_PROBE_SHF) {   // a funnel shift does not merge with its neighbours
        asm volatile("shf.l.wrap.b32 %0, %0, %1, 13;" : "+r"(u[j]) : "r"(u[(j + 1) & 7]));
    } else if constexpr (OP == TF_PROBE_MULHI64) {   // several instructions per operation
        asm volatile("mul.hi.u64 %0, %0, %1;" : "+l"(w[j]) : "l"(w[(j + 1) & 7]));
    } else if constexpr (OP == TF_PROBE_MUFU) {   // a chain of roots (a chain of reciprocals could cancel)
        asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
    } else {   // TF_PROBE_I2F: the converted bits feed the next conversion of the chain
        asm volatile("{\n\t.reg .f32 t;\n\tcvt.rn.f32.u32 t, %0;\n\tmov.b32 %0, t;\n\t}" : "+r"(u[j]));
    }
}

// The latency-critical loop of a short reduction: acc = (acc + e_i) + t_i,
// two dependent binary64 adds per element with the pair (e_i, t_i) from one
// 16-byte shared-memory load (TF_PROBE_CHAIN_LDS; one chain per thread).
__global__ void __launch_bounds__(1024) chain_lds_kernel(int64_t iters, long long *rec) {
    __shared__ __align__(16) double2 S[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) S[k] = make_double2(1e-20 * k, -1e-21 * k);
    __syncthreads();
    double acc = 0.0;
    const long long t0 = clock64();
    for (int64_t it = 0; it < iters; ++it) {
        for (int i = 0; i < 256; i += 8) {
            double2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[u].x), "=d"(v[u].y)
                             : "r"((unsigned)__cvta_generic_to_shared(&S[i + u])));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc) : "d"(v[u].x));
                asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc) : "d"(v[u].y));
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        rec[4 * blockIdx.x + 0] = smid();
        rec[4 * blockIdx.x + 1] = t0;
        rec[4 * blockIdx.x + 2] = t1;
        rec[4 * blockIdx.x + 3] = __double_as_longlong(acc);
    }
}

// The same loop in a fixed order (TF_PROBE_CHAIN_AHEAD): loads and adds as
// inline PTX, the next 8 elements' loads issued right after the first add
// of the 8 before (the order of the CTA-pair reduction's chains).
__global__ void __launch_bounds__(1024) chain_ahead_kernel(int64_t iters, long long *rec) {
    __shared__ __align__(16) double2 S[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) S[k] = make_double2(1e-20 * k, -1e-21 * k);
    __syncthreads();
    const unsigned base = (unsigned)__cvta_generic_to_shared(S);
    double acc = 0.0;
    double2 cur[8], nxt[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(cur[u].x), "=d"(cur[u].y) : "r"(base + 16 * u));
    const long long t0 = clock64();
    for (int64_t it = 0; it < iters; ++it) {
        for (int i = 0; i < 256; i += 8) {
            const unsigned na = base + 16 * ((i + 8) & 255);
            asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc) : "d"(cur[0].x));
#pragma unroll
            for (int u = 0; u < 8; ++u)
                asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(nxt[u].x), "=d"(nxt[u].y) : "r"(na + 16 * u));
            asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc) : "d"(cur[0].y));
#pragma unroll
            for (int u = 1; u < 8; ++u) {
                asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc) : "d"(cur[u].x));
                asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc) : "d"(cur[u].y));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) cur[u] = nxt[u];
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        rec[4 * blockIdx.x + 0] = smid();
        rec[4 * blockIdx.x + 1] = t0;
        rec[4 * blockIdx.x + 2] = t1;
        rec[4 * blockIdx.x + 3] = __double_as_longlong(acc);
    }
}

template <int OP, bool LAT>
__global__ void __launch_bounds__(1024) pipe_probe_kernel(int64_t iters, double a, double b, uint32_t m,
                                                          long long *rec) {
    double d[kChains];
    float f[kChains];
    uint32_t u[kChains];
    uint64_t w[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        d[j] = 1.0 + 0.125 * j;
        f[j] = 1.0f + 0.125f * (float)j;
        u[j] = threadIdx.x * 2654435761u + (uint32_t)j;
        w[j] = ((uint64_t)u[j] << 32) | 0x9E3779B9u;
    }
    const float af = (float)a, bf = (float)b;
    __syncthreads();
    const long long t0 = clock64();
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < kRepeat; ++r) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) step<OP>(d, f, u, w, LAT ? 0 : j, a, b, af, bf, m);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    // keep every chain live (the stamps' slot 3 receives a digest of them)
    uint64_t dig = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        dig ^= (uint64_t)__double_as_longlong(d[j]) ^ __float_as_uint(f[j]) ^ u[j] ^ w[j];
    if (threadIdx.x == 0) {
        rec[4 * blockIdx.x + 0] = smid();
        rec[4 * blockIdx.x + 1] = t0;
        rec[4 * blockIdx.x + 2] = t1;
        rec[4 * blockIdx.x + 3] = (long long)dig;
    }
}

template <int OP>
cudaError_t launch(bool lat, int64_t iters, int blocks, int threads, long long *rec, cudaStream_t s) {
    if (lat) pipe_probe_kernel<OP, true><<<blocks, threads, 0, s>>>(iters, 1.0, 0x1p-60, 0x9E3779B1u, rec);
    else pipe_probe_kernel<OP, false><<<blocks, threads, 0, s>>>(iters, 1.0, 0x1p-60, 0x9E3779B1u, rec);
    return cudaGetLastError();
}

}  // namespace

extern "C" int twofold_pipe_probe(int32_t op, int64_t iters, int32_t blocks, int32_t threads, int64_t *rec,
                                  void *stream) {
    if (iters < 0 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0) return TF_EINVAL;
    if (!tfh::dptr_ok(rec)) return TF_EINVAL;
    long long *r = reinterpret_cast<long long *>(rec);
    cudaStream_t s = tfh::as_stream(stream);
    if (op == (TF_PROBE_LATENCY | TF_PROBE_CHAIN_LDS)) {
        chain_lds_kernel<<<blocks, threads, 0, s>>>(iters, r);
        return cudaGetLastError() == cudaSuccess ? TF_OK : TF_ECUDA;
    }
    if (op == (TF_PROBE_LATENCY | TF_PROBE_CHAIN_AHEAD)) {
        chain_ahead_kernel<<<blocks, threads, 0, s>>>(iters, r);
        return cudaGetLastError() == cudaSuccess ? TF_OK : TF_ECUDA;
    }
    const bool lat = (op & TF_PROBE_LATENCY) != 0;
    if (lat && op != (TF_PROBE_LATENCY | TF_PROBE_DADD) && op != (TF_PROBE_LATENCY | TF_PROBE_DMUL) &&
        op != (TF_PROBE_LATENCY | TF_PROBE_DFMA) && op != (TF_PROBE_LATENCY | TF_PROBE_IMAD))
        return TF_EINVAL;
    cudaError_t e;
    switch (op & ~TF_PROBE_LATENCY) {
    case TF_PROBE_DADD: e = launch<TF_PROBE_DADD>(lat, iters, blocks, threads, r, s); break;
    case TF_PROBE_DMUL: e = launch<TF_PROBE_DMUL>(lat, iters, blocks, threads, r, s); break;
    case TF_PROBE_DFMA: e = launch<TF_PROBE_DFMA>(lat, iters, blocks, threads, r, s); break;
    case TF_PROBE_FFMA: e = launch<TF_PROBE_FFMA>(lat, iters, blocks, threads, r, s); break;
    case TF_PROBE_IMAD: e = launch<TF_PROBE_IMAD>(lat, iters, blocks, threads, r, s); break;
    case TF_PROBE_SHF: e = launch<TF_PROBE_SHF>(lat, iters, blocks, threads, r, s); break;
    case TF_PROBE_MULHI64: e = launch<TF_PROBE_MULHI64>(lat, iters, blocks, threads, r, s); break;
    case TF_PROBE_MUFU: e = launch<TF_PROBE_MUFU>(lat, iters, blocks, threads, r, s); break;
    case TF_PROBE_I2F: e = launch<TF_PROBE_I2F>(lat, iters, blocks, threads, r, s); break;
    default: return TF_EINVAL;
    }
    return e == cudaSuccess ? TF_OK : TF_ECUDA;
}
