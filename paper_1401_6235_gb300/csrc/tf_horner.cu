// Twofold Horner evaluation (single or batched) and its plain twin.
//
// p(x) = a_0 + a_1 x + ... + a_k x^k, dotted coefficients and points:
//   s = (a_k, +0);  for i = k-1 .. 0:  s = ATF1.1(MTF1.1(s, x), a_i)
// One thread evaluates one point at a time in a grid-stride loop over the
// concatenated points of all jobs, so jobs of different degree share the
// machine evenly.  A thread finds its job by binary search in the job table
// (warp-uniform except at job boundaries); coefficients are read through the
// read-only cache (every lane of a warp reads the same address).
#include <cstring>
#include <vector>

#include "tf_host.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kInlineJobs = 32;

struct HTab {
    const int64_t *xoff;     // device (njobs+1) or nullptr: inline copy
    const int32_t *coff;     // device (njobs)
    const int32_t *k;        // device (njobs)
    int64_t ixoff[kInlineJobs + 1];
    int32_t icoff[kInlineJobs];
    int32_t ik[kInlineJobs];
    __device__ __forceinline__ int64_t xo(int j) const { return xoff ? xoff[j] : ixoff[j]; }
    __device__ __forceinline__ int32_t co(int j) const { return coff ? coff[j] : icoff[j]; }
    __device__ __forceinline__ int32_t kk(int j) const { return k ? k[j] : ik[j]; }
};

struct HArgs {
    const double *coefs, *x;
    int njobs;
    int64_t n0, n1;            // points [n0, n1) of the concatenation
    HTab tab;
    double *out_hi, *out_lo, *out_plain;
    uint8_t *flags;
    tf::FlagCfg fc;
};

__device__ __forceinline__ int job_at(const HTab &T, int njobs, int64_t i) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (T.xo(mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// IMUL (plain twin only): the multiplication s * x on the integer pipes
// (correctly rounded, the same bits; plain_arith).
template <bool PLAIN, bool IMUL = false>
__global__ void __launch_bounds__(kThreads) horner_kernel(const __grid_constant__ HArgs A) {
    for (int64_t i = A.n0 + (int64_t)blockIdx.x * kThreads + threadIdx.x; i < A.n1;
         i += (int64_t)gridDim.x * kThreads) {
        const int j = job_at(A.tab, A.njobs, i);
        const double *a = A.coefs + A.tab.co(j);
        const int k = A.tab.kk(j);
        const double x = A.x[i];
        if (PLAIN) {
            double s = __ldg(a + k);
            for (int c = k - 1; c >= 0; --c) {
                double sx;
                if constexpr (IMUL) sx = tf::soft::mul_rn(s, x);
                else sx = __dmul_rn(s, x);
                s = __dadd_rn(sx, __ldg(a + c));
            }
            A.out_plain[i] = s;
        } else {
            tf::d2 s = {__ldg(a + k), 0.0};
            for (int c = k - 1; c >= 0; --c) {
                tf::d2 m = tf::mtf11(s.z0, s.z1, x);
                s = tf::atf11(m.z0, m.z1, __ldg(a + c));
            }
            A.out_hi[i] = s.z0;
            A.out_lo[i] = s.z1;
            if (A.flags) A.flags[i] = tf::flag_of(s.z0, s.z1, A.fc);
        }
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

template <bool PLAIN, bool IMUL>
int launch(const HArgs &A, int64_t npts, cudaStream_t s) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, horner_kernel<PLAIN, IMUL>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t want = (npts + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)tfh::sm_count() * per_sm;
    horner_kernel<PLAIN, IMUL><<<(unsigned)(want < cap ? want : cap), kThreads, 0, s>>>(A);
    return tfh::launch_status();
}

template <bool PLAIN>
int run(const double *coefs, const int32_t *coff, const int32_t *ks, int njobs, const double *x,
        const int64_t *xoff, double *hi, double *lo, double *plain, uint8_t *flags, const tf_params *p,
        void *ws, size_t ws_bytes, void *stream) {
    if (njobs < 0 || !tfh::params_ok(p)) return TF_EINVAL;
    if (njobs == 0) return TF_OK;
    if (!coff || !ks || !xoff || xoff[0] < 0) return TF_EINVAL;
    for (int j = 0; j < njobs; ++j) {
        if (xoff[j + 1] < xoff[j] || ks[j] < 0 || ks[j] > TF_HORNER_MAX_K || coff[j] < 0) return TF_EINVAL;
    }
    const int64_t n0 = xoff[0], n1 = xoff[njobs];
    if (n1 == n0) return TF_OK;
    if (!tfh::dptr_ok(coefs) || !tfh::dptr_ok(x)) return TF_EINVAL;
    if (PLAIN ? !tfh::dptr_ok(plain) : (!tfh::dptr_ok(hi) || !tfh::dptr_ok(lo))) return TF_EINVAL;
    HArgs A{};
    A.coefs = coefs; A.x = x; A.njobs = njobs; A.n0 = n0; A.n1 = n1;
    A.out_hi = hi; A.out_lo = lo; A.out_plain = plain; A.flags = PLAIN ? nullptr : flags;
    A.fc = tfh::flag_cfg(p);
    cudaStream_t s = tfh::as_stream(stream);
    if (njobs <= kInlineJobs) {
        for (int j = 0; j < njobs; ++j) {
            A.tab.ixoff[j] = xoff[j];
            A.tab.icoff[j] = coff[j];
            A.tab.ik[j] = ks[j];
        }
        A.tab.ixoff[njobs] = xoff[njobs];
    } else {
        const size_t b0 = align256(sizeof(int64_t) * (njobs + 1));
        const size_t b1 = align256(sizeof(int32_t) * njobs);
        if (!ws || ws_bytes < b0 + 2 * b1 || !tfh::aligned8(ws)) return TF_ENOSPC;
        std::vector<char> host(b0 + 2 * b1);
        memcpy(host.data(), xoff, sizeof(int64_t) * (njobs + 1));
        memcpy(host.data() + b0, coff, sizeof(int32_t) * njobs);
        memcpy(host.data() + b0 + b1, ks, sizeof(int32_t) * njobs);
        if (cudaMemcpyAsync(ws, host.data(), host.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return TF_ECUDA;
        char *w = static_cast<char *>(ws);
        A.tab.xoff = reinterpret_cast<const int64_t *>(w);
        A.tab.coff = reinterpret_cast<const int32_t *>(w + b0);
        A.tab.k = reinterpret_cast<const int32_t *>(w + b0 + b1);
    }
    if (PLAIN && tfh::plain_integer()) return launch<PLAIN, true>(A, n1 - n0, s);
    return launch<PLAIN, false>(A, n1 - n0, s);
}

}  // namespace

extern "C" size_t twofold_horner_workspace_bytes(int32_t njobs) {
    if (njobs < 1) return 0;
    return align256(sizeof(int64_t) * (njobs + 1)) + 2 * align256(sizeof(int32_t) * njobs);
}

extern "C" int twofold_horner(const double *coef, int32_t k, const double *x, int64_t n, tf_out out,
                              const tf_params *p, void *stream) {
    if (n < 0) return TF_EINVAL;
    const int32_t coff = 0;
    const int64_t xoff[2] = {0, n};
    return run<false>(coef, &coff, &k, 1, x, xoff, out.hi, out.lo, nullptr, out.flags, p, nullptr, 0,
                      stream);
}

extern "C" int twofold_horner_batched(const double *coefs, const int32_t *coef_offs, const int32_t *ks,
                                      int32_t njobs, const double *x, const int64_t *x_offs, tf_out out,
                                      const tf_params *p, void *ws, size_t ws_bytes, void *stream) {
    return run<false>(coefs, coef_offs, ks, njobs, x, x_offs, out.hi, out.lo, nullptr, out.flags, p, ws,
                      ws_bytes, stream);
}

extern "C" int plain_horner(const double *coef, int32_t k, const double *x, int64_t n, double *out,
                            void *stream) {
    if (n < 0) return TF_EINVAL;
    const int32_t coff = 0;
    const int64_t xoff[2] = {0, n};
    return run<true>(coef, &coff, &k, 1, x, xoff, nullptr, nullptr, out, nullptr, nullptr, nullptr, 0,
                     stream);
}

extern "C" int plain_horner_batched(const double *coefs, const int32_t *coef_offs, const int32_t *ks,
                                    int32_t njobs, const double *x, const int64_t *x_offs, double *out,
                                    void *ws, size_t ws_bytes, void *stream) {
    return run<true>(coefs, coef_offs, ks, njobs, x, x_offs, nullptr, nullptr, out, nullptr, nullptr, ws,
                     ws_bytes, stream);
}
