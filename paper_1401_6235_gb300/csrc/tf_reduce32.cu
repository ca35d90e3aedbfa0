// Twofold sum and dot over binary32 twofolds (and their plain binary32
// twins) in the same fixed blocked-pairwise order as the binary64 ones:
// leaves of L consecutive elements accumulated left to right from (+0, +0)
// with ATF1 (ATF1.1 for a dotted sum; a dot adds the twofold product of the
// operand kinds), then the bottom-up pairwise ATF1 tree with the odd node
// carried.  An aligned block of B = 2^k leaves is a subtree: red32_blocks
// reduces one block per CTA (one leaf per thread, its elements staged
// through shared memory, then a strided tree in shared memory) and
// red32_final combines the block partials with the same tree, so the result
// does not depend on B or the grid.
//
// The binary32 operations run on the FP32 pipe (explicit round-to-nearest
// intrinsics, no contraction, subnormals kept), which on this GPU is wide:
// the kernels are bound by memory and latency, not by arithmetic.
#include "tf_host.cuh"
#include "tf_device_f32.cuh"

namespace {

constexpr int kThreads32 = 256;   // = maximum leaves per block

struct Red32Args {
    const float *xh, *xl, *yh, *yl;
    int64_t n, L;
    int B;                        // leaves per block (power of two <= kThreads32)
    int64_t nblk;
    float *part0, *part1;         // block partials (nblk > 1)
    float *out_hi, *out_lo;
    uint8_t *flags;
    tf::FlagCfg32 fc;
};

template <bool PLAIN>
__device__ __forceinline__ tf::f2 combine32(tf::f2 l, tf::f2 r) {
    if (PLAIN) return {__fadd_rn(l.z0, r.z0), 0.0f};
    return tf::atf1(l.z0, l.z1, r.z0, r.z1);
}

template <bool PLAIN>
__device__ __forceinline__ void write32(const Red32Args &A, tf::f2 r) {
    A.out_hi[0] = r.z0;
    if (!PLAIN) {
        A.out_lo[0] = r.z1;
        if (A.flags) A.flags[0] = tf::flag_of(r.z0, r.z1, A.fc);
    }
}

// The strided pairwise tree over s0/s1[0, cnt) in shared memory (cnt <= the
// CTA's threads); the root ends in s0[0], s1[0].
template <bool PLAIN>
__device__ __forceinline__ void smem_tree32(float *s0, float *s1, int cnt) {
    const int t = threadIdx.x;
    for (int s = 1; s < cnt; s <<= 1) {
        if ((t & (2 * s - 1)) == 0 && t + s < cnt) {
            const tf::f2 r = combine32<PLAIN>({s0[t], s1[t]}, {s0[t + s], s1[t + s]});
            s0[t] = r.z0;
            s1[t] = r.z1;
        }
        __syncthreads();
    }
}

// One CTA per aligned block of B leaves; thread t runs leaf b B + t.  The
// block's elements are staged through shared memory chunk by chunk
// (kChunk32 elements of every leaf per chunk), with asynchronous copies
// into two buffers so that the next chunk is in flight while the current
// one is walked; consecutive threads copy consecutive addresses, and rows
// are padded to kChunk32 + 1 words so that the leaf walks hit distinct
// banks.
// (measured, 2^28-element dotted dot: 16 -> 4.0 TB/s, 32 -> 4.4 TB/s)
constexpr int kChunk32 = 32;
static_assert(kChunk32 >= 1 && kChunk32 <= 32 && (kChunk32 & (kChunk32 - 1)) == 0,
              "a chunk must divide a warp's width (every CTA has at least 32 threads)");

__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit32() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev32() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// One element of a leaf: acc = ATF1(acc, term) (ATF1.1 for a dotted sum);
// XD / YD: dotted operands (no tails).
template <bool DOT, bool PLAIN, bool XD, bool YD>
__device__ __forceinline__ void step32(tf::f2 &acc, const float *row, int ox, int oxl, int oy, int oyl, int k) {
    const float x0 = row[ox + k];
    if (PLAIN) {
        acc.z0 = __fadd_rn(acc.z0, DOT ? __fmul_rn(x0, row[oy + k]) : x0);
    } else if (!DOT) {
        acc = XD ? tf::atf11(acc.z0, acc.z1, x0) : tf::atf1(acc.z0, acc.z1, x0, row[oxl + k]);
    } else {
        const tf::f2 q = tf::apply(tf::OP_MUL, x0, XD ? 0.0f : row[oxl + k], XD, row[oy + k], YD ? 0.0f : row[oyl + k], YD);
        acc = tf::atf1(acc.z0, acc.z1, q.z0, q.z1);
    }
}

template <bool DOT, bool PLAIN, bool XD, bool YD>
__global__ void __launch_bounds__(kThreads32) red32_blocks(const __grid_constant__ Red32Args A) {
    extern __shared__ float st32[];                   // [2][narr][B][kChunk32 + 1]
    __shared__ float s0[kThreads32], s1[kThreads32];
    const int t = threadIdx.x;
    const int64_t m = (A.n + A.L - 1) / A.L;
    const int64_t leaf0 = (int64_t)blockIdx.x * A.B;
    const int nl = (int)min((int64_t)A.B, m - leaf0);
    constexpr bool xd = XD, yd = YD;
    const int RS = kChunk32 + 1, TS = A.B * RS;       // row and array strides in a buffer
    const int ox = 0, oxl = TS, oy = oxl + (xd || PLAIN ? 0 : TS), oyl = oy + TS;
    const int BS = (1 + (!PLAIN && !xd) + (DOT ? 1 + (!PLAIN && !yd) : 0)) * TS;   // buffer stride
    const int64_t base = leaf0 * A.L;
    const int64_t my_len = t < nl ? min(A.L, A.n - (base + (int64_t)t * A.L)) : 0;
    const int64_t nchunk = (A.L + kChunk32 - 1) / kChunk32;

    // thread t copies column k = t mod kChunk32 of rows r0, r0 + rstep, ...
    const int k = t % kChunk32, r0 = t / kChunk32, rstep = (int)blockDim.x / kChunk32;
    auto issue = [&](int64_t c) {
        float *q = st32 + (c & 1) * BS + r0 * RS + k;
        const int64_t off = c * kChunk32 + k;         // element of each leaf
        if (off < A.L) {
            int64_t g = base + (int64_t)r0 * A.L + off;
#pragma unroll 4
            for (int r = r0; r < nl; r += rstep, g += (int64_t)rstep * A.L, q += rstep * RS) {
                if (g >= A.n) break;                  // rows are in element order: the rest lie past n too
                cp_async4(q + ox, A.xh + g);
                if (!PLAIN && !xd) cp_async4(q + oxl, A.xl + g);
                if (DOT) {
                    cp_async4(q + oy, A.yh + g);
                    if (!PLAIN && !yd) cp_async4(q + oyl, A.yl + g);
                }
            }
        }
        cp_commit32();
    };

    tf::f2 acc = {0.0f, 0.0f};
    issue(0);
    for (int64_t c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) issue(c + 1);
        else cp_commit32();                           // an empty group keeps the wait count uniform
        cp_wait_prev32();                             // this thread's copies of chunk c have landed
        __syncthreads();                              // ... and everyone's
        const float *row = st32 + (c & 1) * BS + t * RS;
        const int cnt = (int)max((int64_t)0, min((int64_t)kChunk32, my_len - c * kChunk32));
        if (cnt == kChunk32) {
#pragma unroll
            for (int k = 0; k < kChunk32; ++k) step32<DOT, PLAIN, XD, YD>(acc, row, ox, oxl, oy, oyl, k);
        } else {
            for (int k = 0; k < cnt; ++k) step32<DOT, PLAIN, XD, YD>(acc, row, ox, oxl, oy, oyl, k);
        }
        __syncthreads();                              // the buffer is free for chunk c + 2
    }
    if (t < nl) {
        s0[t] = acc.z0;
        s1[t] = acc.z1;
    }
    __syncthreads();
    smem_tree32<PLAIN>(s0, s1, nl);
    if (t == 0) {
        if (A.nblk == 1) write32<PLAIN>(A, {s0[0], s1[0]});
        else {
            A.part0[blockIdx.x] = s0[0];
            A.part1[blockIdx.x] = s1[0];
        }
    }
}

// The same block reduction for leaves of a multiple of 4 elements on
// 16-byte aligned arrays: the chunk copies move 16 bytes each (a partial
// last vector of the job copies only its valid bytes), and each leaf row of
// 32 elements is stored as 8 vectors of 4 with the vector index XORed by
// the row's low three bits, so that the 16-byte row reads of any 8
// consecutive threads (one shared-memory wavefront) hit distinct banks.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}

template <bool DOT, bool PLAIN, bool XD, bool YD>
__device__ __forceinline__ void vstep32(tf::f2 &acc, float x0, float x1, float y0, float y1) {
    if (PLAIN) {
        acc.z0 = __fadd_rn(acc.z0, DOT ? __fmul_rn(x0, y0) : x0);
    } else if (!DOT) {
        acc = XD ? tf::atf11(acc.z0, acc.z1, x0) : tf::atf1(acc.z0, acc.z1, x0, x1);
    } else {
        const tf::f2 q = tf::apply(tf::OP_MUL, x0, x1, XD, y0, y1, YD);
        acc = tf::atf1(acc.z0, acc.z1, q.z0, q.z1);
    }
}

template <bool DOT, bool PLAIN, bool XD, bool YD>
__global__ void __launch_bounds__(kThreads32) red32_blocks_v4(const __grid_constant__ Red32Args A) {
    extern __shared__ float4 sv4[];                   // [2][narr][B][8] vectors
    __shared__ float s0[kThreads32], s1[kThreads32];
    static_assert(kChunk32 == 32, "a row is 8 vectors of 4");
    const int t = threadIdx.x;
    const int64_t m = (A.n + A.L - 1) / A.L;
    const int64_t leaf0 = (int64_t)blockIdx.x * A.B;
    const int nl = (int)min((int64_t)A.B, m - leaf0);
    const int TS = A.B * 8;                           // vectors per array in a buffer
    const int ox = 0, oxl = TS, oy = oxl + (XD || PLAIN ? 0 : TS), oyl = oy + TS;
    const int BS = (1 + (!PLAIN && !XD) + (DOT ? 1 + (!PLAIN && !YD) : 0)) * TS;
    const int64_t base = leaf0 * A.L;
    const int64_t my_len = t < nl ? min(A.L, A.n - (base + (int64_t)t * A.L)) : 0;
    const int64_t nchunk = (A.L + kChunk32 - 1) / kChunk32;
    // thread t copies vector j = t mod 8 of rows r0, r0 + rstep, ...
    const int j = t & 7, r0 = t >> 3, rstep = (int)blockDim.x >> 3;
    auto issue = [&](int64_t c) {
        const int64_t off = c * kChunk32 + 4 * j;     // first element of the vector within each leaf
        if (off < A.L) {
            float4 *q = sv4 + (c & 1) * BS + r0 * 8 + (j ^ (r0 & 7));
            int64_t g = base + (int64_t)r0 * A.L + off;
            for (int r = r0; r < nl; r += rstep, g += (int64_t)rstep * A.L) {
                const int64_t rem = A.n - g;          // elements of the job from g on
                if (rem <= 0) break;                  // rows are in element order
                const int bytes = rem >= 4 ? 16 : (int)rem * 4;
                float4 *qr = q + (r - r0) * 8 + ((j ^ (r & 7)) - (j ^ (r0 & 7)));
                cp_async16(qr + ox, A.xh + g, bytes);
                if (!PLAIN && !XD) cp_async16(qr + oxl, A.xl + g, bytes);
                if (DOT) {
                    cp_async16(qr + oy, A.yh + g, bytes);
                    if (!PLAIN && !YD) cp_async16(qr + oyl, A.yl + g, bytes);
                }
            }
        }
        cp_commit32();
    };

    tf::f2 acc = {0.0f, 0.0f};
    const int sw = t & 7;
    issue(0);
    for (int64_t c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) issue(c + 1);
        else cp_commit32();
        cp_wait_prev32();
        __syncthreads();
        const float4 *row = sv4 + (c & 1) * BS + t * 8;
        const int cnt = (int)max((int64_t)0, min((int64_t)kChunk32, my_len - c * kChunk32));
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            if (4 * v >= cnt) break;
            const int pv = v ^ sw;
            const float4 X = row[ox + pv];
            const float4 XL = (!PLAIN && !XD) ? row[oxl + pv] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 Y = DOT ? row[oy + pv] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 YL = (DOT && !PLAIN && !YD) ? row[oyl + pv] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int left = cnt - 4 * v;
            vstep32<DOT, PLAIN, XD, YD>(acc, X.x, XL.x, Y.x, YL.x);
            if (left > 1) vstep32<DOT, PLAIN, XD, YD>(acc, X.y, XL.y, Y.y, YL.y);
            if (left > 2) vstep32<DOT, PLAIN, XD, YD>(acc, X.z, XL.z, Y.z, YL.z);
            if (left > 3) vstep32<DOT, PLAIN, XD, YD>(acc, X.w, XL.w, Y.w, YL.w);
        }
        __syncthreads();
    }
    if (t < nl) {
        s0[t] = acc.z0;
        s1[t] = acc.z1;
    }
    __syncthreads();
    smem_tree32<PLAIN>(s0, s1, nl);
    if (t == 0) {
        if (A.nblk == 1) write32<PLAIN>(A, {s0[0], s1[0]});
        else {
            A.part0[blockIdx.x] = s0[0];
            A.part1[blockIdx.x] = s1[0];
        }
    }
}

// One CTA of T threads: thread t first folds the aligned group of G
// partials [tG, (t+1)G) (G = 2^g, G T >= nblk), a subtree, then the CTA
// reduces the group roots.  Groups of up to 8 partials are loaded together
// (32 contiguous bytes per thread and array) and folded in registers;
// larger groups fold in place in the workspace.  T = 256 up to 2048
// partials, 1024 beyond.
constexpr int kFinal32 = 1024;

template <bool PLAIN, int T>
__global__ void __launch_bounds__(T) red32_final(const __grid_constant__ Red32Args A) {
    __shared__ float s0[T], s1[T];
    const int t = threadIdx.x;
    const int64_t nb = A.nblk;
    int64_t G = 1;
    while (G * T < nb) G <<= 1;
    const int ng = (int)((nb + G - 1) / G);
    if (t < ng) {
        float *q0 = A.part0 + (int64_t)t * G, *q1 = A.part1 + (int64_t)t * G;
        const int64_t cnt = min(G, nb - (int64_t)t * G);
        if (G <= 8) {
            float r0[8], r1[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < cnt) { r0[i] = q0[i]; r1[i] = q1[i]; }
#pragma unroll
            for (int st = 1; st < 8; st <<= 1)
#pragma unroll
                for (int i = 0; i + st < 8; i += 2 * st)
                    if (i + st < cnt) {
                        const tf::f2 r = combine32<PLAIN>({r0[i], r1[i]}, {r0[i + st], r1[i + st]});
                        r0[i] = r.z0;
                        r1[i] = r.z1;
                    }
            s0[t] = r0[0];
            s1[t] = r1[0];
        } else {
            for (int64_t st = 1; st < cnt; st <<= 1)
                for (int64_t i = 0; i + st < cnt; i += 2 * st) {
                    const tf::f2 r = combine32<PLAIN>({q0[i], q1[i]}, {q0[i + st], q1[i + st]});
                    q0[i] = r.z0;
                    q1[i] = r.z1;
                }
            s0[t] = q0[0];
            s1[t] = q1[0];
        }
    }
    __syncthreads();
    smem_tree32<PLAIN>(s0, s1, ng);
    if (t == 0) write32<PLAIN>(A, {s0[0], s1[0]});
}

__global__ void red32_zero(float *hi, float *lo, uint8_t *flags) {
    hi[0] = 0.0f;
    if (lo) lo[0] = 0.0f;
    if (flags) flags[0] = 0;
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

tf::FlagCfg32 flag_cfg32(const tf_params *p) {
    tf::FlagCfg32 f;
    f.mode = p ? p->panic_mode : TF_PANIC_REL;
    f.tau = p ? (float)p->panic_tau : tfh::kDefaultTau32;
    f.m = p ? (float)p->panic_ulps : (float)tfh::kDefaultUlps;
    return f;
}

template <bool DOT, bool PLAIN>
int run32(const float *xh, const float *xl, const float *yh, const float *yl, int64_t n, float *out_hi,
          float *out_lo, uint8_t *flags, const tf_params *p, void *ws, size_t ws_bytes, void *stream) {
    if (n < 0 || !tfh::params_ok(p)) return TF_EINVAL;
    if (!tfh::fptr_ok(out_hi) || (!PLAIN && !tfh::fptr_ok(out_lo)) || (!PLAIN && !tfh::foptr_ok(flags)))
        return TF_EINVAL;
    if (n > 0) {
        if (!tfh::fptr_ok(xh) || !tfh::foptr_ok(xl)) return TF_EINVAL;
        if (DOT && (!tfh::fptr_ok(yh) || !tfh::foptr_ok(yl))) return TF_EINVAL;
    }
    cudaStream_t s = tfh::as_stream(stream);
    if (n == 0) {
        red32_zero<<<1, 1, 0, s>>>(out_hi, PLAIN ? nullptr : out_lo, PLAIN ? nullptr : flags);
        return tfh::launch_status();
    }
    Red32Args A{};
    A.xh = xh; A.xl = xl; A.yh = yh; A.yl = yl;
    A.n = n;
    A.L = tfh::leaf_of(p);
    const int64_t M = (n + A.L - 1) / A.L;
    // staged arrays; leaves per block B: at most what leaves three CTAs'
    // double buffers of all arrays room in shared memory (more resident warps
    // hide the leaves' dependent chains: a 2^28-element dotted dot took
    // 0.355 ms at B = 128, three CTAs per SM, against 0.428 ms at B = 256,
    // one), and at least ~1024 blocks while B >= 1; then larger (up to one
    // CTA per SM) where the caller's workspace would not hold the partials
    const int narr = 1 + (!PLAIN && xl != nullptr) + (DOT ? 1 + (!PLAIN && yl != nullptr) : 0);
    auto tile_bytes = [&](int b) { return 2 * (size_t)narr * b * (kChunk32 + 1) * sizeof(float); };
    constexpr size_t kSmem = 227 * 1024;
    int Bfit = kThreads32, Bocc = kThreads32;
    while (Bfit > 1 && tile_bytes(Bfit) > kSmem) Bfit >>= 1;
    while (Bocc > 1 && 3 * tile_bytes(Bocc) > kSmem) Bocc >>= 1;
    int B = 1;
    while (B < Bocc && (int64_t)B * 2 * 1024 <= M) B <<= 1;
    auto ws_need = [&](int b) {
        const int64_t nb = (M + b - 1) / b;
        return nb > 1 ? 2 * al256(sizeof(float) * (size_t)nb) : (size_t)0;
    };
    while (B < Bfit && ws_need(B) > ws_bytes) B <<= 1;
    A.B = B;
    A.nblk = (M + B - 1) / B;
    if (A.nblk > 0x7FFFFFFFLL) return TF_EUNSUPPORTED;
    A.out_hi = out_hi; A.out_lo = out_lo; A.flags = PLAIN ? nullptr : flags;
    A.fc = flag_cfg32(p);
    if (A.nblk > 1) {
        const size_t need = 2 * al256(sizeof(float) * (size_t)A.nblk);
        if (!ws || ws_bytes < need || ((uintptr_t)ws % 8) != 0) return TF_ENOSPC;
        A.part0 = static_cast<float *>(ws);
        A.part1 = reinterpret_cast<float *>(static_cast<char *>(ws) + al256(sizeof(float) * (size_t)A.nblk));
    }
    const int threads = B < 32 ? 32 : B;
    // 16-byte copies when every leaf starts on a 16-byte boundary
    auto a16 = [](const float *q) { return q == nullptr || ((uintptr_t)q % 16) == 0; };
    const bool v4 = A.L % 4 == 0 && a16(xh) && a16(xl) && a16(yh) && a16(yl);
    const size_t smem = v4 ? 2 * (size_t)narr * B * kChunk32 * sizeof(float) : tile_bytes(B);
    auto kern = v4 ? (xl ? (yl ? red32_blocks_v4<DOT, PLAIN, false, false> : red32_blocks_v4<DOT, PLAIN, false, true>)
                         : (yl ? red32_blocks_v4<DOT, PLAIN, true, false> : red32_blocks_v4<DOT, PLAIN, true, true>))
                   : (xl ? (yl ? red32_blocks<DOT, PLAIN, false, false> : red32_blocks<DOT, PLAIN, false, true>)
                         : (yl ? red32_blocks<DOT, PLAIN, true, false> : red32_blocks<DOT, PLAIN, true, true>));
    if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                                cudaSuccess)
        return TF_ECUDA;
    kern<<<(unsigned)A.nblk, threads, smem, s>>>(A);
    if (A.nblk > 8 * kThreads32) red32_final<PLAIN, kFinal32><<<1, kFinal32, 0, s>>>(A);
    else if (A.nblk > 1) red32_final<PLAIN, kThreads32><<<1, kThreads32, 0, s>>>(A);
    return tfh::launch_status();
}

}  // namespace

extern "C" int twofold_sum_f32(tf_in_f32 x, int64_t n, tf_out_f32 out1, const tf_params *p, void *ws,
                               size_t ws_bytes, void *stream) {
    return run32<false, false>(x.hi, x.lo, nullptr, nullptr, n, out1.hi, out1.lo, out1.flags, p, ws, ws_bytes,
                               stream);
}

extern "C" int twofold_dot_f32(tf_in_f32 x, tf_in_f32 y, int64_t n, tf_out_f32 out1, const tf_params *p,
                               void *ws, size_t ws_bytes, void *stream) {
    return run32<true, false>(x.hi, x.lo, y.hi, y.lo, n, out1.hi, out1.lo, out1.flags, p, ws, ws_bytes, stream);
}

extern "C" int plain_sum_f32(const float *x, int64_t n, float *out1, const tf_params *p, void *ws,
                             size_t ws_bytes, void *stream) {
    return run32<false, true>(x, nullptr, nullptr, nullptr, n, out1, nullptr, nullptr, p, ws, ws_bytes, stream);
}

extern "C" int plain_dot_f32(const float *x, const float *y, int64_t n, float *out1, const tf_params *p,
                             void *ws, size_t ws_bytes, void *stream) {
    return run32<true, true>(x, nullptr, y, nullptr, n, out1, nullptr, nullptr, p, ws, ws_bytes, stream);
}
