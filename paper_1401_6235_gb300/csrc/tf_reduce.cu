// Twofold sum and dot (and their plain binary64 twins) in the fixed
// blocked-pairwise order, single or batched.
//
// Order (also in twofold.h): leaves of L consecutive elements, each
// accumulated left to right into a twofold from (+0, +0) with ATF1 (the
// paper's twofold accumulator, "2x" section: adding a plain value is strict
// per step); leaf results combined by a bottom-up pairwise ATF1 tree with
// an odd last node carried up.  Node i of level j covers leaves
// [i 2^j, min((i+1) 2^j, m)), so an aligned block of B = 2^k leaves is a
// subtree: reduce_blocks handles one block per CTA (one leaf per thread,
// then an in-place strided tree in shared memory) and reduce_final
// combines the partials of each job with the same tree.  Results therefore
// do not depend on B, the grid or the device.
#include <algorithm>
#include <mutex>
#include <vector>

#include "tf_host.cuh"
#include "tf_leaf.cuh"

namespace {

constexpr int kThreads = 256;        // = maximum leaves per block
constexpr int kInlineJobs = 32;      // job tables up to this size travel in the launch params
constexpr int64_t kLatMaxLeaves = 2048;   // latency schedule: at most this many leaves in all
constexpr int64_t kLatMaxLeaf = 2048;     // ... each at most this long (one CTA holds B L <= 2048)

struct Tab {
    const int64_t *offs;   // device job table (njobs+1), or nullptr: use the inline copy
    const int64_t *blk0;
    int64_t ioffs[kInlineJobs + 1];
    int64_t iblk0[kInlineJobs + 1];
    __device__ __forceinline__ int64_t off(int j) const { return offs ? offs[j] : ioffs[j]; }
    __device__ __forceinline__ int64_t b0(int j) const { return blk0 ? blk0[j] : iblk0[j]; }
};

struct RedArgs {
    const double *xh, *xl, *yh, *yl;
    int njobs;
    int64_t L;
    int B;                     // leaves per block (power of two, <= kThreads)
    int C;                     // elements of each leaf staged per chunk (power of two)
    int narr;                  // staged arrays: x, [x tails], [y, [y tails]]
    Tab tab;
    double *part0, *part1;     // partial results, one per block
    double *out_hi, *out_lo;
    uint8_t *flags;
    tf::FlagCfg fc;
    int write_single;          // reduce_final writes jobs of one partial too (twofold_combine)
    int pair_drop;             // latency schedule, failure injection: the chunk whose tails are not sent (-1: none)
    long long pair_spin;       // latency schedule: polls of an mbarrier before a wait gives up
};

// Job of block b: the largest j with blk0[j] <= b (empty jobs own no block).
__device__ __forceinline__ int job_of(const Tab &T, int njobs, int64_t b) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (T.b0(mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while its predecessor in the
// stream finishes; griddep_wait() blocks until that predecessor has completed
// and its memory is visible (a no-op for an ordinary launch), and
// griddep_release() lets the successor start launching.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// One element of a leaf: acc = ATF1(acc, term) (ATF1.1 for a dotted sum);
// the plain twin adds the plain term (separate multiplication and addition).
template <bool DOT, bool PLAIN>
__device__ __forceinline__ void leaf_step(tf::d2 &acc, double x0, double x1, bool xd, double y0, double y1,
                                          bool yd) {
    if (PLAIN) {
        acc.z0 = __dadd_rn(acc.z0, DOT ? __dmul_rn(x0, y0) : x0);
    } else if (!DOT) {
        acc = xd ? tf::atf11(acc.z0, acc.z1, x0) : tf::atf1(acc.z0, acc.z1, x0, x1);
    } else {
        const tf::d2 p = tf::apply(tf::OP_MUL, x0, x1, xd, y0, y1, yd);
        acc = tf::atf1(acc.z0, acc.z1, p.z0, p.z1);
    }
}

template <bool PLAIN>
__device__ __forceinline__ tf::d2 combine(tf::d2 l, tf::d2 r) {
    if (PLAIN) return {__dadd_rn(l.z0, r.z0), 0.0};
    // the floating-point form of the Two-Sum tail (same bits): its latency,
    // which a tree level waits for, is the shorter one (a 64-node final tree
    // measured 2.8 against 3.1 us)
    return tf::atf1_fp(l.z0, l.z1, r.z0, r.z1);
}

template <bool PLAIN>
__device__ __forceinline__ void write_result(const RedArgs &A, int j, tf::d2 r) {
    A.out_hi[j] = r.z0;
    if (!PLAIN) {
        A.out_lo[j] = r.z1;
        if (A.flags) A.flags[j] = tf::flag_of(r.z0, r.z1, A.fc);
    }
}

// One CTA reduces an aligned block of B leaves, one leaf per thread, then
// an in-place strided tree in shared memory.  STAGED: the leaves' elements
// are staged chunk by chunk (C elements per leaf) into shared memory with
// cp.async, double buffered, rows padded to C+1 words, and thread t walks
// leaf t's row (used by the memory-bound plain twin); otherwise thread t
// reads its leaf straight from global memory through L1 (the twofold step
// is compute-bound and barrier-free this way).
// The twofold (not STAGED) kernel walks its leaves with tf::leaf_walk,
// specialised on the operand kinds KD (bit 0: x dotted, bit 1: y dotted or
// no y); with L even and aligned arrays every leaf of a CTA takes its
// 16-byte loads.
template <bool DOT, bool PLAIN, bool STAGED, int KD = 3>
__global__ void __launch_bounds__(kThreads) reduce_blocks(const __grid_constant__ RedArgs A) {
    extern __shared__ double stage[];                // [2][narr][B][C+1] when STAGED
    __shared__ double s0[kThreads], s1[kThreads];
    griddep_wait();
    griddep_release();
    const int t = threadIdx.x;
    const int64_t b = blockIdx.x;
    const int j = job_of(A.tab, A.njobs, b);
    const int64_t e0 = A.tab.off(j), len = A.tab.off(j + 1) - e0;
    const int64_t m = (len + A.L - 1) / A.L;
    const int64_t leaf0 = (b - A.tab.b0(j)) * A.B;
    const int nl = (int)min((int64_t)A.B, m - leaf0);
    const int64_t base = e0 + leaf0 * A.L;           // first element of the block
    const int64_t end = e0 + len;
    const int64_t lb = base + (int64_t)t * A.L;      // this thread's leaf
    const int64_t llen = t < nl ? min(A.L, end - lb) : 0;
    const bool xd = A.xl == nullptr, yd = A.yl == nullptr;
    tf::d2 acc = {0.0, 0.0};
    if constexpr (!STAGED) {
        static_assert(!PLAIN, "the plain twin stages its leaves");
        constexpr bool XD = (KD & 1) != 0, YD = (KD & 2) != 0;
        if (llen > 0)
            acc = tf::leaf_walk<DOT, XD, YD>(A.xh + lb, XD ? nullptr : A.xl + lb, DOT ? A.yh + lb : nullptr,
                                             (DOT && !YD) ? A.yl + lb : nullptr, llen);
    } else {
        const int B = A.B, C = A.C, S = C + 1, narr = A.narr;
        const double *src[4] = {nullptr, nullptr, nullptr, nullptr};
        int na = 0;
        src[na++] = A.xh;
        if (A.xl) src[na++] = A.xl;
        if (DOT) {
            src[na++] = A.yh;
            if (A.yl) src[na++] = A.yl;
        }
        const int lgC = __ffs(C) - 1;
        const int64_t nch = (A.L + C - 1) / C;       // chunks per (full) leaf
        auto load = [&](int64_t c, int buf) {
            double *dst = stage + (size_t)buf * narr * B * S;
            for (int idx = t; idx < nl * C; idx += kThreads) {
                const int row = idx >> lgC, k = idx & (C - 1);
                const int64_t off = c * C + k;
                const int64_t g = base + (int64_t)row * A.L + off;
                if (off < A.L && g < end) {
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        if (a < na) cp_async8(dst + ((size_t)a * B + row) * S + k, src[a] + g);
                }
            }
            cp_commit();
        };
        load(0, 0);
        for (int64_t c = 0; c < nch; ++c) {
            if (c + 1 < nch) { load(c + 1, (int)((c + 1) & 1)); cp_wait_one(); }
            else cp_wait_all();
            __syncthreads();
            const double *buf = stage + (size_t)(c & 1) * narr * B * S;
            const int cnt = (int)max((int64_t)0, min((int64_t)C, llen - c * C));
            if (cnt > 0) {
                int a = 0;
                const double *X = buf + ((size_t)(a++) * B + t) * S;
                const double *XL = xd ? nullptr : buf + ((size_t)(a++) * B + t) * S;
                const double *Y = DOT ? buf + ((size_t)(a++) * B + t) * S : nullptr;
                const double *YL = (DOT && !yd) ? buf + ((size_t)(a++) * B + t) * S : nullptr;
                for (int k = 0; k < cnt; ++k)
                    leaf_step<DOT, PLAIN>(acc, X[k], xd ? 0.0 : XL[k], xd, DOT ? Y[k] : 0.0,
                                          (DOT && !yd) ? YL[k] : 0.0, yd);
            }
            __syncthreads();
        }
    }
    if (t < nl) {
        s0[t] = acc.z0;
        s1[t] = acc.z1;
    }
    __syncthreads();
    for (int s = 1; s < nl; s <<= 1) {
        if ((t & (2 * s - 1)) == 0 && t + s < nl) {
            tf::d2 r = combine<PLAIN>({s0[t], s1[t]}, {s0[t + s], s1[t + s]});
            s0[t] = r.z0;
            s1[t] = r.z1;
        }
        __syncthreads();
    }
    if (t == 0) {
        const tf::d2 r = {s0[0], s1[0]};
        if (A.tab.b0(j + 1) - A.tab.b0(j) == 1) write_result<PLAIN>(A, j, r);
        else { A.part0[b] = r.z0; A.part1[b] = r.z1; }
    }
}

// Named barriers for the chunk hand-overs of reduce_lat (ids 1..2 kLatChunks;
// id 0 is __syncthreads).
constexpr int kLatChunks = 7;
__device__ __forceinline__ void bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_wait(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Latency schedule for jobs with few leaves.  A CTA takes an aligned block
// of B leaves (B L <= kLatElems; one warp lane per leaf) and splits each
// leaf's left-to-right accumulation acc = ATF1(acc, term_i) into its
// independent and its sequential parts:
//   terms (p_i, e_i) of all B leaves    - all threads (kLatPer loads each, in flight together)
//   z0 chain  s_i = s_{i-1} + p_i        - warp 0, lane l = leaf l; it keeps only
//                                          the checkpoints s_{8k+7}
//   tails     s_{8k..8k+7} again from the checkpoint s_{8k-1} (the same adds
//             in the same order, so the same bits) and
//             t_i = Two-Sum tail(s_{i-1}, p_i, s_i), in place of p_i
//                                        - warps 2.., one lane per 8 steps of a leaf
//   z1 chain  acc1 = (acc1 + e_i) + t_i  - warp 1, lane l (acc1 + t_i for ATF1.1)
// then the block's subtree of the pairwise tree by warp shuffles.  Every
// operation and operand is the one the sequential leaf uses, so the bits are
// the same.  On this GPU a dependent FP64 add costs ~64 cycles, a warp
// issues one FP64 instruction per ~64 cycles whatever its active lanes, and
// chains in different warps do not slow each other: so the B leaves share
// the cost of one chain, and the chain warps issue little besides their adds
// (a store behind each add would cost ~40 more cycles per step).  The three
// stages form a pipeline over chunks of the leaf (a short first chunk, then
// at most kLatChunks - 1 more): warp 0 hands a finished z0 chunk to the tail
// warps, they hand its tails to warp 1, each through a named barrier
// (bar.arrive / bar.sync; ids 1..kLatChunks and kLatChunks+1..2 kLatChunks,
// each used once; every participant walks the same chunk count, so every
// barrier completes).  The chains run in register blocks of 8 steps, and a
// lane past the end of its (short, last) leaf adds -0.0, which leaves every
// value unchanged.
constexpr int kLatThreads = 512;
constexpr int kLatPer = 4;                          // phase-1 elements per thread
constexpr int kLatElems = kLatPer * kLatThreads;    // elements per CTA at most
constexpr int kTailThreads = kLatThreads - 64;      // warps 2..
constexpr int kLatFirst = 16;                       // length of the first chunk

// Chunk c of a leaf of (rounded) length n8: [start, end), multiples of 8.
__device__ __forceinline__ int lat_chunk_start(int c, int n8) {
    if (c == 0) return 0;
    const int first = min(kLatFirst, n8);
    const int rest = n8 - first;
    const int per = (((rest + kLatChunks - 2) / (kLatChunks - 1)) + 7) & ~7;
    return min(n8, first + (c - 1) * per);
}

// Shared-memory rows of reduce_lat for leaves of length L (rows hold L8 =
// L rounded up to 8 entries plus padding, so that a chain reads whole
// blocks of 8 without bounds checks and 16-byte loads of different lanes
// fall in different banks):
//   PT [B][L8 + 2]  doubles   p_i (terms; x_i for a sum)
//   ET [B][L8 + 1]  double2   (e_i, t_i): term tails and Two-Sum tails
//   CK [B][L8/8 + 1] doubles  z0 checkpoints s_{8k+7}
// Entries past the end of a leaf hold -0.0, which leaves an accumulator
// unchanged.
struct LatRows {
    int L8, SP, SE, SC;
    __host__ __device__ explicit LatRows(int64_t L)
        : L8((int)((L + 7) & ~7)), SP(L8 + 2), SE(L8 + 1), SC(L8 / 8 + 1) {}
    __host__ __device__ size_t bytes(int B) const {
        return ((size_t)B * SP + 2 * (size_t)B * SE + (size_t)B * SC) * sizeof(double);
    }
};

template <bool DOT, bool PLAIN>
__global__ void __launch_bounds__(kLatThreads) reduce_lat(const __grid_constant__ RedArgs A) {
    extern __shared__ __align__(16) double lat[];
    __shared__ double r0[32];
    griddep_wait();
    griddep_release();
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int64_t b = blockIdx.x;
    const int j = job_of(A.tab, A.njobs, b);
    const int64_t e0 = A.tab.off(j), len = A.tab.off(j + 1) - e0;
    const int64_t m = (len + A.L - 1) / A.L;
    const int64_t leaf0 = (b - A.tab.b0(j)) * A.B;
    const int nl = (int)min((int64_t)A.B, m - leaf0);
    const int64_t base = e0 + leaf0 * A.L, end = e0 + len;
    const int L = (int)A.L;
    const LatRows R(A.L);
    const int nel = (int)min((int64_t)nl * L, end - base);   // elements of the block
    double *PT = lat;
    double2 *ET = reinterpret_cast<double2 *>(lat + (size_t)A.B * R.SP);
    double *CK = lat + (size_t)A.B * R.SP + 2 * (size_t)A.B * R.SE;
    const bool xd = A.xl == nullptr, yd = A.yl == nullptr;
    {
        // element k of the block is element k - r L of leaf r = k / L
        double xv[kLatPer], xlv[kLatPer], yv[kLatPer], ylv[kLatPer];
#pragma unroll
        for (int u = 0; u < kLatPer; ++u) {
            const int k = t + u * kLatThreads;
            xv[u] = xlv[u] = yv[u] = ylv[u] = 0.0;
            if (k < nel) {
                const int64_t g = base + k;
                xv[u] = A.xh[g];
                if (!xd) xlv[u] = A.xl[g];
                if (DOT) {
                    yv[u] = A.yh[g];
                    if (!yd) ylv[u] = A.yl[g];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kLatPer; ++u) {
            const int k = t + u * kLatThreads;
            if (k < nel) {
                const int r = k / L, i = k - r * L;
                if (PLAIN) {
                    PT[r * R.SP + i] = DOT ? __dmul_rn(xv[u], yv[u]) : xv[u];
                } else if (DOT) {
                    const tf::d2 q = tf::apply(tf::OP_MUL, xv[u], xlv[u], xd, yv[u], ylv[u], yd);
                    PT[r * R.SP + i] = q.z0;
                    ET[r * R.SE + i].x = q.z1;
                } else {
                    PT[r * R.SP + i] = xv[u];
                    if (!xd) ET[r * R.SE + i].x = xlv[u];
                }
            }
        }
        // -0.0 past the end of each leaf, up to L8
        for (int q = t; q < nl * R.L8; q += kLatThreads) {
            const int r = q / R.L8, i = q - r * R.L8;
            if (base + (int64_t)r * L + i >= end || i >= L) {
                PT[r * R.SP + i] = -0.0;
                if (!PLAIN) ET[r * R.SE + i] = make_double2(-0.0, -0.0);
            }
        }
    }
    __syncthreads();
    // this lane's leaf (lanes >= nl repeat the last leaf's chain; their
    // results are never used); leaf 0 is the longest
    const int row = min(lane, nl - 1);
    const int len0 = (int)min((int64_t)L, end - base);
    const int n8 = (len0 + 7) & ~7;
    const double2 *Pp = reinterpret_cast<const double2 *>(PT + row * R.SP);   // (p_i, p_i+1) pairs
    tf::d2 acc = {0.0, 0.0};
    if (PLAIN) {
        if (warp == 0) {
            for (int i = 0; i < n8; i += 8) {
                double2 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = Pp[(i >> 1) + u];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc.z0 = __dadd_rn(acc.z0, v[u].x);
                    acc.z0 = __dadd_rn(acc.z0, v[u].y);
                }
            }
        }
    } else {
        int nch = 1;
        while (nch < kLatChunks && lat_chunk_start(nch, n8) < n8) ++nch;
        if (warp == 0) {
            double *Cr = CK + lane * R.SC;
            for (int c = 0; c < nch; ++c) {
                const int i1 = lat_chunk_start(c + 1, n8);
                for (int i = lat_chunk_start(c, n8); i < i1; i += 8) {
                    double2 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = Pp[(i >> 1) + u];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        acc.z0 = __dadd_rn(acc.z0, v[u].x);
                        acc.z0 = __dadd_rn(acc.z0, v[u].y);
                    }
                    if (lane < nl) Cr[i >> 3] = acc.z0;          // s_{i+7}
                }
                __syncwarp();
                __threadfence_block();
                bar_arrive(1 + c, 32 + kTailThreads);
            }
            r0[lane] = acc.z0;
        } else if (warp >= 2) {
            for (int c = 0; c < nch; ++c) {
                bar_wait(1 + c, 32 + kTailThreads);
                const int k0 = lat_chunk_start(c, n8) >> 3, nk = (lat_chunk_start(c + 1, n8) >> 3) - k0;
                for (int task = t - 64; task < nl * nk; task += kTailThreads) {
                    const int r = task / nk, k = k0 + task - r * nk;
                    const int rl = (int)min((int64_t)L, end - (base + (int64_t)r * L));
                    const double *Pr = PT + r * R.SP;
                    double2 *Er = ET + r * R.SE;
                    double sv = k ? CK[r * R.SC + k - 1] : 0.0;
                    for (int i = 8 * k; i < min(8 * k + 8, rl); ++i) {
                        const double p = Pr[i];
                        const double sn = __dadd_rn(sv, p);
                        Er[i].y = tf::soft::sum_err(sv, p, sn);            // t_i
                        sv = sn;
                    }
                }
                __threadfence_block();
                bar_arrive(1 + kLatChunks + c, 32 + kTailThreads);
            }
        } else {   // warp 1
            const double2 *Q = ET + row * R.SE;
            for (int c = 0; c < nch; ++c) {
                bar_wait(1 + kLatChunks + c, 32 + kTailThreads);
                const int i1 = lat_chunk_start(c + 1, n8);
                for (int i = lat_chunk_start(c, n8); i < i1; i += 8) {
                    double2 v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = Q[i + u];
                    if (DOT || !xd) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) acc.z1 = __dadd_rn(__dadd_rn(acc.z1, v[u].x), v[u].y);
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) acc.z1 = __dadd_rn(acc.z1, v[u].y);
                    }
                }
            }
        }
        __syncthreads();
        if (warp == 1) acc.z0 = r0[lane];
    }
    // the block's subtree: node l of level k combines lanes l and l + 2^k
    const int tw = PLAIN ? 0 : 1;
    if (warp == tw) {
        for (int st = 1; st < nl; st <<= 1) {
            const double o0 = __shfl_down_sync(0xffffffffu, acc.z0, st);
            const double o1 = __shfl_down_sync(0xffffffffu, acc.z1, st);
            if ((lane & (2 * st - 1)) == 0 && lane + st < nl) acc = combine<PLAIN>(acc, {o0, o1});
        }
        if (lane == 0) {
            if (A.tab.b0(j + 1) - A.tab.b0(j) == 1) write_result<PLAIN>(A, j, acc);
            else { A.part0[b] = acc.z0; A.part1[b] = acc.z1; }
        }
    }
}

// Leaves per CTA of the latency schedule: the largest power of two <= 32
// with B L <= kLatElems that still leaves >= kLatTargetCtas CTAs for the M
// leaves (1 when L alone exceeds it).  Spreading the leaves over more SMs
// shortens the term phase (measured at n = 65536, L = 256: B = 2 -> 30.0 us
// per dot, B = 8 -> 31.0 us, B = 1 -> 32.0 us: 256 CTAs and a deeper tree).
constexpr int64_t kLatTargetCtas = 128;
int lat_group(int64_t L, int64_t M) {
    int B = 32;
    while (B > 1 && ((int64_t)B * L > kLatElems || (int64_t)B * kLatTargetCtas > M)) B >>= 1;
    return B;
}

size_t lat_smem(int B, int64_t L) { return LatRows(L).bytes(B); }

// ----------------------------------------------------------------------
// Latency schedule on a CTA pair: a thread-block cluster of two CTAs, one
// per SM.  The z1 chain (two dependent FP64 adds per element) is the
// longest path of a short dot, and it ran ~20 % slower per element when
// the z0 chain and the tail computation shared its SM (measured: ~174 SM
// clocks per element in the one-CTA kernel against ~143 alone).  So the
// producer CTA (rank 0) forms the products p_i, runs the z0 chains (every
// partial sum s_i kept in shared memory) and the Two-Sum tails
// t_i = err(s_{i-1} + p_i), one element per thread, written over p_i, and
// sends each chunk of tails into the consumer's shared memory with one bulk
// copy per leaf row, whose completion counts on a transaction mbarrier of
// the consumer; the consumer CTA (rank 1) forms the product tails e_i and
// runs only the z1 chains, then the block's subtree.  Every operation and
// operand is the one of reduce_lat (p_i = RN(x_i y_i) is Two-Product's
// head), so the bits are the same.  Waits are bounded (kPairSpin polls); a
// wait that runs out leaves NaN in the block's result and counts in
// g_pair_timeouts.  Both CTAs meet at a cluster barrier at the start (the
// consumer's mbarriers are initialised by then) and at the end (the
// consumer outlives every copy into its shared memory, the producer every
// copy out of its own).
constexpr int kPairChunks = 12;                 // hand-over chunks (named barriers 1..kPairChunks)
constexpr int kPairTail = kLatThreads - 32;     // producer warps 1.. compute tails
constexpr long long kPairSpin = 1ll << 24;      // polls of an mbarrier before giving up
constexpr long long kPairSpinInjected = 1ll << 12;   // ... while a failure is injected
constexpr int64_t kPairTargetClusters = 64;

__device__ unsigned long long g_pair_timeouts;

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The same meeting with a relaxed arrive (the wait keeps its default
// acquire): at the start of the pair kernel, after fence.mbarrier_init has
// released the mbarriers' initialisation, and at its end, where only the
// order of execution matters (the consumer arrives after its mbarriers
// completed, so no copy still reads the producer's shared memory; the
// partials reach the final tree through the grid's completion).  A release
// arrive waits for the CTA's earlier memory accesses: at the end the
// consumer's global stores (~0.5 us per call), at the start the terms'
// loads in flight.
__device__ __forceinline__ void cluster_sync_exec() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_init(uint32_t a, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t a, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// true once phase 0 of the mbarrier has completed; false after `spin` polls
__device__ __forceinline__ bool mbar_wait0(uint32_t a, long long spin) {
    for (long long it = 0; it < spin; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(a) : "memory");
        if (ok) return true;
    }
    return false;
}
// true if phase 0 of the mbarrier has completed (one non-blocking test)
__device__ __forceinline__ bool mbar_test0(uint32_t a) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(a) : "memory");
    return ok != 0;
}

// The dependent chains of the pair kernel are written as inline PTX in a
// fixed order: a batch's operands are loaded from shared memory one batch
// ahead, issued right after the first addition of the batch before.  On
// GB300 a binary64 add whose chain is interleaved with shared-memory loads
// otherwise ran ~14 clocks per load above its 64-clock latency (~142 clocks
// per z1 element against 128.5 with the operands in registers); in this
// order ~134 in the kernel.
__device__ __forceinline__ void lds2(double2 &v, uint32_t a) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
}
// the same load without a compiler memory barrier: volatile asm keeps its
// place after the (volatile) mbarrier waits, and nothing later depends on
// its order against other memory accesses
__device__ __forceinline__ void lds2v(double2 &v, uint32_t a) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
}
__device__ __forceinline__ void sts2(uint32_t a, double x, double y) {
    asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(x), "d"(y) : "memory");
}
__device__ __forceinline__ void dadd_to(double &acc, double v) {
    asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(acc) : "d"(v));
}

// `bytes` (a multiple of 16) from this CTA's shared memory at `src` into the
// peer's at `remote` (both 16-byte aligned), counted on the peer's mbarrier
__device__ __forceinline__ void bulk_to_peer(uint32_t remote, uint32_t src, unsigned bytes, uint32_t remote_mbar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(remote), "r"(src), "r"(bytes), "r"(remote_mbar) : "memory");
}
// 8 bytes into the peer's shared memory, counted on the peer's mbarrier
__device__ __forceinline__ void st_async8(uint32_t remote, double v, uint32_t remote_mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
                 ::"r"(remote), "l"(__double_as_longlong(v)), "r"(remote_mbar) : "memory");
}

// End of chunk c of a leaf of (rounded) length n8: 16, 32, 56, 96, 160,
// 264, ... elements (each end the largest multiple of 8 <= 8 + 13/8 of the
// one before).  The producer's z0 chain takes ~80 clocks per element and the
// consumer's z1 chain ~140, so a chunk of this size is complete when the
// consumer, started after the first chunk, reaches it.  (A first chunk of 8
// measured 0.2 us slower: the second chunk's hand-over then stalled the
// chain.)  The last possible chunk runs to the end of the leaf.  (A table:
// computing the recurrence on the device put ~1.5 us of dependent integer
// work in front of the terms.)
__constant__ int kPairEnd[kPairChunks] = {16, 32, 56, 96, 160, 264, 432, 704, 1152, 1880, 2048, 2048};
__device__ __forceinline__ int pair_chunk_end(int c, int n8) {
    return c >= kPairChunks - 1 ? n8 : min(kPairEnd[c], n8);
}

// Shared memory of reduce_lat_pair: two regions of [B][SP] doubles.  The
// producer keeps the products p_i in region 0 (overwritten by the tails t_i
// once a chunk's z0 chain is done) and the partial sums s_i in region 1; the
// consumer keeps e_i in region 0 and receives the t_i into region 1 (the
// same offset in both CTAs, so the producer maps its own address).  Rows
// padded with -0.0.
size_t pair_smem(int B, int64_t L) {
    const LatRows R(L);
    return 2 * (size_t)B * R.SP * sizeof(double);
}

// The consumer's z1 chain over one leaf row: e_i at shared address ea, t_i
// at ta (TWO: acc = (acc + e_i) + t_i; else acc = acc + t_i, a sum of
// binary64 values), chunk by chunk as the mbarriers at mb (8 bytes apart)
// complete.  One flat loop over batches of 8 elements: the next batch is
// loaded right after the batch's first add, and where it starts a new chunk
// the (bounded) wait for that chunk comes just before its loads.  (Nested
// per-chunk loops, or a non-blocking test of the next chunk in every batch,
// measured 10-15 clocks per element slower.)  False if a wait gave up.
template <bool TWO>
__device__ __forceinline__ void z1_load(double2 (&e)[4], double2 (&tt)[4], uint32_t ea, uint32_t ta, int i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (TWO) lds2v(e[u], ea + 8 * i + 16 * u);
        lds2v(tt[u], ta + 8 * i + 16 * u);
    }
}
template <bool TWO>
__device__ __forceinline__ bool z1_chain(uint32_t ea, uint32_t ta, uint32_t mb, int n8, int nch, long long spin,
                                         double &acc) {
    bool ok = mbar_wait0(mb, spin);
    double2 ce[4], ct[4], ne[4], nt[4];
    z1_load<TWO>(ce, ct, ea, ta, 0);
    int c = 0, cend = pair_chunk_end(0, n8);
    for (int i = 0; i < n8; i += 8) {
        const int in = i + 8 < n8 ? i + 8 : i;   // the last batch reloads itself (unused)
        dadd_to(acc, TWO ? ce[0].x : ct[0].x);
        if (in == cend) {
            ++c;
            cend = pair_chunk_end(c, n8);
            if (!mbar_test0(mb + 8 * c)) ok = mbar_wait0(mb + 8 * c, spin) && ok;
        }
        z1_load<TWO>(ne, nt, ea, ta, in);
        if (TWO) {
            dadd_to(acc, ct[0].x);
            dadd_to(acc, ce[0].y);
        }
        dadd_to(acc, ct[0].y);
#pragma unroll
        for (int u = 1; u < 4; ++u) {
            if (TWO) dadd_to(acc, ce[u].x);
            dadd_to(acc, ct[u].x);
            if (TWO) dadd_to(acc, ce[u].y);
            dadd_to(acc, ct[u].y);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            ce[u] = ne[u];
            ct[u] = nt[u];
        }
    }
    for (int k = c + 1; k < nch; ++k) ok = mbar_wait0(mb + 8 * k, spin) && ok;
    return ok;
}

template <bool DOT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kLatThreads) reduce_lat_pair(const __grid_constant__ RedArgs A) {
    extern __shared__ __align__(16) double lat[];
    __shared__ __align__(8) unsigned long long mbar[kPairChunks + 1];
    __shared__ double r0[32];                    // consumer: the leaves' z0 results
    griddep_wait();
    griddep_release();
    const unsigned rank = cluster_rank();
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int64_t b = blockIdx.x >> 1;           // the pair's block of B leaves
    const int j = job_of(A.tab, A.njobs, b);
    const int64_t e0 = A.tab.off(j), len = A.tab.off(j + 1) - e0;
    const int64_t m = (len + A.L - 1) / A.L;
    const int64_t leaf0 = (b - A.tab.b0(j)) * A.B;
    const int nl = (int)min((int64_t)A.B, m - leaf0);
    const int64_t base = e0 + leaf0 * A.L, end = e0 + len;
    const int L = (int)A.L;
    const LatRows R(A.L);
    const int nel = (int)min((int64_t)nl * L, end - base);
    double *PT = lat;                            // producer: p_i, then t_i; consumer: e_i
    double *SS = lat + (size_t)A.B * R.SP;       // producer: s_i; consumer: t_i (copied by the producer)
    const bool xd = A.xl == nullptr, yd = A.yl == nullptr;
    const int len0 = (int)min((int64_t)L, end - base);
    const int n8 = (len0 + 7) & ~7;
    int nch = 1;
    while (nch < kPairChunks && pair_chunk_end(nch - 1, n8) < n8) ++nch;
    // the terms' loads go out first (their latency covers the mbarrier
    // set-up and the cluster barrier): the producer needs x_i (and y_i), the
    // consumer x_i, y_i and the tails for a dot, xl_i for a sum
    double xv[kLatPer], xlv[kLatPer], yv[kLatPer], ylv[kLatPer];
#pragma unroll
    for (int u = 0; u < kLatPer; ++u) {
        const int k = t + u * kLatThreads;
        xv[u] = xlv[u] = yv[u] = ylv[u] = 0.0;
        if (k < nel) {
            const int64_t g = base + k;
            if (rank == 0 || DOT) xv[u] = A.xh[g];
            if (!xd && rank == 1) xlv[u] = A.xl[g];
            if (DOT) {
                yv[u] = A.yh[g];
                if (!yd && rank == 1) ylv[u] = A.yl[g];
            }
        }
    }
    if (rank == 1 && t <= nch) {
        // phase bytes: the tails of chunk t of every row (-0.0 past a leaf's
        // end); the z0 results (t = nch)
        unsigned bytes = 8u * (unsigned)nl;
        if (t < nch) bytes *= (unsigned)(pair_chunk_end(t, n8) - (t ? pair_chunk_end(t - 1, n8) : 0));
        mbar_init(smem_addr(&mbar[t]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect(smem_addr(&mbar[t]), bytes);
    }
    // the consumer's mbarriers are ready before any producer copy (their
    // initialisation is released by fence.mbarrier_init and acquired by the
    // cluster wait; the arrive is relaxed so that the terms' loads stay in
    // flight across the barrier); the terms follow in both CTAs
    cluster_sync_exec();
    const int row = min(lane, nl - 1);
    {
        // terms: the producer keeps p_i = RN(x_i y_i) (or x_i for a sum),
        // the consumer e_i (the product's z1: Two-Product's tail, or the
        // general product's; xl_i for a sum)
#pragma unroll
        for (int u = 0; u < kLatPer; ++u) {
            const int k = t + u * kLatThreads;
            if (k < nel) {
                const int r = k / L, i = k - r * L;
                if (rank == 0) PT[r * R.SP + i] = DOT ? __dmul_rn(xv[u], yv[u]) : xv[u];
                else if (DOT) PT[r * R.SP + i] = tf::apply(tf::OP_MUL, xv[u], xlv[u], xd, yv[u], ylv[u], yd).z1;
                else if (!xd) PT[r * R.SP + i] = xlv[u];
            }
        }
        // -0.0 past the end of each leaf, up to L8 (the tails there come from the producer)
        for (int q = t; q < nl * R.L8; q += kLatThreads) {
            const int r = q / R.L8, i = q - r * R.L8;
            if (base + (int64_t)r * L + i >= end || i >= L) PT[r * R.SP + i] = -0.0;
        }
    }
    __syncthreads();
    if (rank == 0) {
        if (warp == 0) {                         // z0 chains; every s_i kept, in 16-byte pairs
            const uint32_t pa = smem_addr(PT + row * R.SP), sa = smem_addr(SS + row * R.SP);
            double acc0 = 0.0;
            double2 cur[4], nxt[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) lds2(cur[u], pa + 16 * u);
            int c = 0, cend = pair_chunk_end(0, n8);
            for (int i = 0; i < n8; i += 8) {
                double sx, sy;
                dadd_to(acc0, cur[0].x);
                sx = acc0;
                if (i + 8 < n8) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) lds2(nxt[u], pa + 8 * (i + 8) + 16 * u);
                }
                dadd_to(acc0, cur[0].y);
                sy = acc0;
                if (lane < nl) sts2(sa + 8 * i, sx, sy);
#pragma unroll
                for (int u = 1; u < 4; ++u) {
                    dadd_to(acc0, cur[u].x);
                    sx = acc0;
                    dadd_to(acc0, cur[u].y);
                    sy = acc0;
                    if (lane < nl) sts2(sa + 8 * i + 16 * u, sx, sy);
                }
                if (i + 8 == cend) {
                    __syncwarp();
                    __threadfence_block();
                    bar_arrive(1 + c, kLatThreads);
                    ++c;
                    cend = pair_chunk_end(c, n8);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) cur[u] = nxt[u];
            }
            if (lane < nl) st_async8(peer_addr(smem_addr(&r0[lane]), 1), acc0, peer_addr(smem_addr(&mbar[nch]), 1));
        } else {
            // tails t_i of each chunk, one element per thread, written over
            // p_i (only this thread reads p_i once the chunk's z0 chain is
            // done; -0.0 past a leaf's end); then one bulk copy per row into
            // the consumer's t row
            for (int c = 0; c < nch; ++c) {
                bar_wait(1 + c, kLatThreads);
                const int i0 = c ? pair_chunk_end(c - 1, n8) : 0, w = pair_chunk_end(c, n8) - i0;
                for (int task = t - 32; task < nl * w; task += kPairTail) {
                    const int r = task / w, i = i0 + task - r * w;
                    const int rl = (int)min((int64_t)L, end - (base + (int64_t)r * L));
                    double tv = -0.0;
                    if (i < rl) {
                        const double sp = i ? SS[r * R.SP + i - 1] : 0.0;
                        tv = tf::soft::sum_err(sp, PT[r * R.SP + i], SS[r * R.SP + i]);
                    }
                    PT[r * R.SP + i] = tv;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_wait(kPairChunks + 1, kPairTail);
                if (t == 32 && c != A.pair_drop) {   // pair_drop: injected failure, this chunk never arrives
                    const uint32_t rmb = peer_addr(smem_addr(&mbar[c]), 1);
                    for (int r = 0; r < nl; ++r)
                        bulk_to_peer(peer_addr(smem_addr(SS + r * R.SP + i0), 1), smem_addr(PT + r * R.SP + i0),
                                     8u * (unsigned)w, rmb);
                }
            }
        }
    } else if (warp == 0) {                      // the z1 chains, then the block's subtree
        const uint32_t ea = smem_addr(PT + row * R.SP), ta = smem_addr(SS + row * R.SP), mb = smem_addr(&mbar[0]);
        tf::d2 acc = {0.0, 0.0};
        const bool ok = (DOT || !xd) ? z1_chain<true>(ea, ta, mb, n8, nch, A.pair_spin, acc.z1)
                                     : z1_chain<false>(ea, ta, mb, n8, nch, A.pair_spin, acc.z1);
        // every chunk was waited for (each wait bounded), so every copy the
        // producer sent has landed before this CTA leaves
        const bool ok_all = __all_sync(0xffffffffu, mbar_wait0(smem_addr(&mbar[nch]), A.pair_spin) && ok);
        acc.z0 = ok_all ? r0[row] : __longlong_as_double(0x7FF8000000000000ll);
        if (!ok_all) acc.z1 = acc.z0;
        for (int st = 1; st < nl; st <<= 1) {
            const double o0 = __shfl_down_sync(0xffffffffu, acc.z0, st);
            const double o1 = __shfl_down_sync(0xffffffffu, acc.z1, st);
            if ((lane & (2 * st - 1)) == 0 && lane + st < nl) acc = combine<false>(acc, {o0, o1});
        }
        if (lane == 0) {
            if (!ok_all) atomicAdd(&g_pair_timeouts, 1ull);
            if (A.tab.b0(j + 1) - A.tab.b0(j) == 1) write_result<false>(A, j, acc);
            else { A.part0[b] = acc.z0; A.part1[b] = acc.z1; }
        }
    }
    cluster_sync_exec();
}

// Leaves per pair: the largest power of two <= 32 with B L <= kLatElems that
// still leaves >= kPairTargetClusters pairs (two CTAs each) for the M leaves.
int pair_group(int64_t L, int64_t M) {
    int B = 32;
    while (B > 1 && ((int64_t)B * L > kLatElems || (int64_t)B * kPairTargetClusters > M)) B >>= 1;
    return B;
}

// One CTA of T threads per job with 0 or >= 2 blocks.  Thread t first
// reduces the aligned group of G partials [tG, (t+1)G) (G = 2^g,
// G T >= nb), which is a subtree, then the CTA reduces the group roots.
// Groups of up to 4 partials are loaded together and folded in registers;
// larger groups fold in place in the workspace (a dependent global load per
// step).  T = 256 up to 1024 partials per job, 1024 beyond (launch_final).
constexpr int kFinalThreads = 1024;

template <bool PLAIN, int T>
__global__ void __launch_bounds__(T) reduce_final(const __grid_constant__ RedArgs A) {
    __shared__ double s0[T], s1[T];
    griddep_wait();
    griddep_release();
    const int j = blockIdx.x, t = threadIdx.x;
    const int64_t p0 = A.tab.b0(j), nb = A.tab.b0(j + 1) - p0;
    if (nb == 1) {
        if (A.write_single && t == 0) write_result<PLAIN>(A, j, {A.part0[p0], A.part1[p0]});
        return;
    }
    if (nb == 0) {
        if (t == 0) write_result<PLAIN>(A, j, {0.0, 0.0});
        return;
    }
    if (nb <= 128) {
        // one warp: lane l folds the aligned group of partials [4l, 4l + 4) in
        // registers, then the group roots combine by shuffles (the same tree,
        // without a barrier per level)
        if (t >= 32) return;
        const int cnt = (int)max((int64_t)0, min((int64_t)4, nb - 4 * (int64_t)t));
        double q0[4] = {0.0, 0.0, 0.0, 0.0}, q1[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (i < cnt) { q0[i] = __ldcg(A.part0 + p0 + 4 * t + i); q1[i] = __ldcg(A.part1 + p0 + 4 * t + i); }
#pragma unroll
        for (int st = 1; st < 4; st <<= 1)
#pragma unroll
            for (int i = 0; i + st < 4; i += 2 * st)
                if (i + st < cnt) {
                    const tf::d2 r = combine<PLAIN>({q0[i], q1[i]}, {q0[i + st], q1[i + st]});
                    q0[i] = r.z0;
                    q1[i] = r.z1;
                }
        tf::d2 acc = {q0[0], q1[0]};
        const int ng = (int)((nb + 3) / 4);
        for (int st = 1; st < ng; st <<= 1) {
            const double o0 = __shfl_down_sync(0xffffffffu, acc.z0, st);
            const double o1 = __shfl_down_sync(0xffffffffu, acc.z1, st);
            if ((t & (2 * st - 1)) == 0 && t + st < ng) acc = combine<PLAIN>(acc, {o0, o1});
        }
        if (t == 0) write_result<PLAIN>(A, j, acc);
        return;
    }
    int64_t G = 1;
    while (G * T < nb) G <<= 1;
    const int ng = (int)((nb + G - 1) / G);
    if (t < ng) {
        double *q0 = A.part0 + p0 + (int64_t)t * G, *q1 = A.part1 + p0 + (int64_t)t * G;
        const int64_t cnt = min(G, nb - (int64_t)t * G);
        if (G <= 4) {
            double r0[4], r1[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < cnt) { r0[i] = q0[i]; r1[i] = q1[i]; }
#pragma unroll
            for (int st = 1; st < 4; st <<= 1)
#pragma unroll
                for (int i = 0; i + st < 4; i += 2 * st)
                    if (i + st < cnt) {
                        const tf::d2 r = combine<PLAIN>({r0[i], r1[i]}, {r0[i + st], r1[i + st]});
                        r0[i] = r.z0;
                        r1[i] = r.z1;
                    }
            s0[t] = r0[0];
            s1[t] = r1[0];
        } else {
            for (int64_t s = 1; s < cnt; s <<= 1)
                for (int64_t i = 0; i + s < cnt; i += 2 * s) {
                    tf::d2 r = combine<PLAIN>({q0[i], q1[i]}, {q0[i + s], q1[i + s]});
                    q0[i] = r.z0;
                    q1[i] = r.z1;
                }
            s0[t] = q0[0];
            s1[t] = q1[0];
        }
    }
    __syncthreads();
    for (int s = 1; s < ng; s <<= 1) {
        if ((t & (2 * s - 1)) == 0 && t + s < ng) {
            tf::d2 r = combine<PLAIN>({s0[t], s1[t]}, {s0[t + s], s1[t + s]});
            s0[t] = r.z0;
            s1[t] = r.z1;
        }
        __syncthreads();
    }
    if (t == 0) write_result<PLAIN>(A, j, {s0[0], s1[0]});
}

// Leaves per block: at least ~1024 blocks while that keeps blocks >= 1 leaf.
int leaves_per_block(int64_t M) {
    int B = 1;
    while (B < kThreads && (int64_t)B * 2 * 1024 <= M) B <<= 1;
    return B;
}

// Elements of each leaf staged per chunk: a power of two with both buffers
// of all staged arrays within ~96 KiB of shared memory, and no larger than
// the leaf rounded up to a power of two.
int chunk_of(int B, int narr, int64_t L) {
    const int64_t budget = 6144 / ((int64_t)narr * B);     // elements per row and buffer
    int C = 1;
    while ((int64_t)C * 2 <= budget) C <<= 1;
    int64_t lp = 1;
    while (lp < L) lp <<= 1;
    return (int)(C < lp ? C : lp);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// twofold_inject_pair_drop: the chunk the latency schedule's producers skip
// (-1: none); read at each launch.
std::atomic<int> g_pair_drop{-1};

// Workspace: [offs (njobs+1) | blk0 (njobs+1)] [part0 (nblk)] [part1 (nblk)].
size_t ws_need(int njobs, int64_t nblk) {
    return align256(sizeof(int64_t) * 2 * (size_t)(njobs + 1)) + 2 * align256(sizeof(double) * (size_t)nblk);
}

// The final tree's launch, its CTA size chosen by the most partials of a job.
template <bool PLAIN>
cudaError_t launch_final(int njobs, int64_t max_partials, cudaStream_t s, const RedArgs &A) {
    if (max_partials > 4 * kThreads)
        return tfh::launch_pdl(reduce_final<PLAIN, kFinalThreads>, njobs, kFinalThreads, 0, s, A);
    return tfh::launch_pdl(reduce_final<PLAIN, kThreads>, njobs, kThreads, 0, s, A);
}

template <bool DOT, bool PLAIN>
int run(const double *xh, const double *xl, const double *yh, const double *yl, const int64_t *offs,
        int njobs, double *out_hi, double *out_lo, uint8_t *flags, const tf_params *p, void *ws,
        size_t ws_bytes, void *stream) {
    if (njobs < 0 || !offs || !tfh::params_ok(p)) return TF_EINVAL;
    if (njobs == 0) return TF_OK;
    if (!tfh::dptr_ok(out_hi) || (!PLAIN && !tfh::dptr_ok(out_lo))) return TF_EINVAL;
    if (offs[0] < 0) return TF_EINVAL;
    for (int j = 0; j < njobs; ++j)
        if (offs[j + 1] < offs[j]) return TF_EINVAL;
    const int64_t ntot = offs[njobs];
    if (ntot > 0) {
        if (!tfh::dptr_ok(xh) || !tfh::optr_ok(xl)) return TF_EINVAL;
        if (DOT && (!tfh::dptr_ok(yh) || !tfh::optr_ok(yl))) return TF_EINVAL;
    }
    const int64_t L = tfh::leaf_of(p);
    std::vector<int64_t> tab(2 * (size_t)(njobs + 1));
    int64_t M = 0;
    for (int j = 0; j < njobs; ++j) M += (offs[j + 1] - offs[j] + L - 1) / L;
    // few leaves of moderate length: the latency schedule, one CTA per leaf
    const bool lat = M <= kLatMaxLeaves && L <= kLatMaxLeaf;
    // the twofold latency schedule runs on CTA pairs (reduce_lat_pair), the
    // plain twin on single CTAs (reduce_lat)
    const int B = lat ? (PLAIN ? lat_group(L, M) : pair_group(L, M)) : leaves_per_block(M);
    int64_t nblk = 0;
    bool need_final = false;
    for (int j = 0; j < njobs; ++j) {
        tab[j] = offs[j];
        tab[njobs + 1 + j] = nblk;
        const int64_t m = (offs[j + 1] - offs[j] + L - 1) / L;
        const int64_t nb = (m + B - 1) / B;
        need_final |= (nb != 1);
        nblk += nb;
    }
    tab[njobs] = offs[njobs];
    tab[2 * (size_t)njobs + 1] = nblk;
    if (nblk > 0x7FFFFFFFLL) return TF_EUNSUPPORTED;

    RedArgs A{};
    A.xh = xh; A.xl = xl; A.yh = yh; A.yl = yl;
    A.njobs = njobs; A.L = L; A.B = B;
    A.out_hi = out_hi; A.out_lo = out_lo; A.flags = PLAIN ? nullptr : flags;
    A.fc = tfh::flag_cfg(p);
    A.pair_drop = g_pair_drop.load(std::memory_order_relaxed);
    A.pair_spin = A.pair_drop >= 0 ? kPairSpinInjected : kPairSpin;
    cudaStream_t s = tfh::as_stream(stream);
    const bool inl = njobs <= kInlineJobs;
    size_t need = 0;
    if (!inl) need += align256(sizeof(int64_t) * tab.size());
    if (need_final && nblk > 0) need += 2 * align256(sizeof(double) * (size_t)nblk);
    if (need > 0 && (!ws || ws_bytes < need || !tfh::aligned8(ws))) return TF_ENOSPC;
    char *w = static_cast<char *>(ws);
    if (inl) {
        for (int j = 0; j <= njobs; ++j) {
            A.tab.ioffs[j] = tab[j];
            A.tab.iblk0[j] = tab[njobs + 1 + j];
        }
    } else {
        A.tab.offs = reinterpret_cast<int64_t *>(w);
        A.tab.blk0 = A.tab.offs + (njobs + 1);
        if (cudaMemcpyAsync(w, tab.data(), tab.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return TF_ECUDA;
        w += align256(sizeof(int64_t) * tab.size());
    }
    if (need_final && nblk > 0) {
        A.part0 = reinterpret_cast<double *>(w);
        A.part1 = reinterpret_cast<double *>(w + align256(sizeof(double) * (size_t)nblk));
    }
    A.narr = 1 + (xl != nullptr) + (DOT ? 1 + (yl != nullptr) : 0);
    A.C = chunk_of(B, A.narr, L);
    if (nblk > 0) {
        if (lat && !PLAIN) {
            const size_t smem = pair_smem(B, L);
            if (smem > 48 * 1024 && cudaFuncSetAttribute(reduce_lat_pair<DOT>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)smem) != cudaSuccess)
                return TF_ECUDA;
            if (tfh::launch_pdl(reduce_lat_pair<DOT>, 2 * nblk, kLatThreads, smem, s, A) != cudaSuccess)
                return TF_ECUDA;
        } else if (lat) {
            const size_t smem = lat_smem(B, L);
            if (smem > 48 * 1024 && cudaFuncSetAttribute(reduce_lat<DOT, PLAIN>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)smem) != cudaSuccess)
                return TF_ECUDA;
            if (tfh::launch_pdl(reduce_lat<DOT, PLAIN>, nblk, kLatThreads, smem, s, A) != cudaSuccess) return TF_ECUDA;
        } else if constexpr (PLAIN) {
            const size_t smem = (size_t)2 * A.narr * B * (A.C + 1) * sizeof(double);
            if (smem > 48 * 1024 && cudaFuncSetAttribute(reduce_blocks<DOT, PLAIN, true>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)smem) != cudaSuccess)
                return TF_ECUDA;
            if (tfh::launch_pdl(reduce_blocks<DOT, PLAIN, true>, nblk, kThreads, smem, s, A) != cudaSuccess)
                return TF_ECUDA;
        } else {
            // operand kinds: bit 0 x dotted, bit 1 y dotted (or a sum)
            const int kd = (xl == nullptr ? 1 : 0) | (!DOT || yl == nullptr ? 2 : 0);
            cudaError_t e;
            switch (kd) {
            case 0: e = tfh::launch_pdl(reduce_blocks<DOT, false, false, 0>, nblk, kThreads, 0, s, A); break;
            case 1: e = tfh::launch_pdl(reduce_blocks<DOT, false, false, 1>, nblk, kThreads, 0, s, A); break;
            case 2: e = tfh::launch_pdl(reduce_blocks<DOT, false, false, 2>, nblk, kThreads, 0, s, A); break;
            default: e = tfh::launch_pdl(reduce_blocks<DOT, false, false, 3>, nblk, kThreads, 0, s, A); break;
            }
            if (e != cudaSuccess) return TF_ECUDA;
        }
    }
    int64_t maxp = 0;                                 // the most partials of one job
    for (int j = 0; j < njobs; ++j) maxp = std::max(maxp, tab[njobs + 2 + j] - tab[njobs + 1 + j]);
    if (need_final && launch_final<PLAIN>(njobs, maxp, s, A) != cudaSuccess)
        return TF_ECUDA;
    return tfh::launch_status();
}

}  // namespace

extern "C" size_t twofold_workspace_bytes(int32_t kind, int64_t n_total, int32_t njobs,
                                          const tf_params *p) {
    (void)kind;
    if (n_total < 0 || njobs < 1) return 0;
    const int64_t L = p && p->leaf >= 1 ? p->leaf : tfh::kDefaultLeaf;
    const int64_t Mmax = n_total / L + njobs;            // >= sum of ceil(len_j / L)
    // blocks <= M/B + njobs with B = leaves_per_block(M): M/B < 2048 or B = 256
    int64_t per = Mmax / kThreads + 1;
    if (per < 2048) per = 2048;
    const int64_t nblk = per + njobs;
    return ws_need(njobs, nblk);
}

extern "C" int twofold_sum(tf_in x, int64_t n, tf_out out1, const tf_params *p, void *ws,
                           size_t ws_bytes, void *stream) {
    if (n < 0) return TF_EINVAL;
    const int64_t offs[2] = {0, n};
    return run<false, false>(x.hi, x.lo, nullptr, nullptr, offs, 1, out1.hi, out1.lo, out1.flags, p, ws,
                             ws_bytes, stream);
}

extern "C" int twofold_dot(tf_in x, tf_in y, int64_t n, tf_out out1, const tf_params *p, void *ws,
                           size_t ws_bytes, void *stream) {
    if (n < 0) return TF_EINVAL;
    const int64_t offs[2] = {0, n};
    return run<true, false>(x.hi, x.lo, y.hi, y.lo, offs, 1, out1.hi, out1.lo, out1.flags, p, ws, ws_bytes,
                            stream);
}

extern "C" int twofold_sum_batched(tf_in x, const int64_t *offs, int32_t njobs, tf_out out,
                                   const tf_params *p, void *ws, size_t ws_bytes, void *stream) {
    return run<false, false>(x.hi, x.lo, nullptr, nullptr, offs, njobs, out.hi, out.lo, out.flags, p, ws,
                             ws_bytes, stream);
}

extern "C" int twofold_dot_batched(tf_in x, tf_in y, const int64_t *offs, int32_t njobs, tf_out out,
                                   const tf_params *p, void *ws, size_t ws_bytes, void *stream) {
    return run<true, false>(x.hi, x.lo, y.hi, y.lo, offs, njobs, out.hi, out.lo, out.flags, p, ws,
                            ws_bytes, stream);
}

extern "C" int plain_sum(const double *x, int64_t n, double *out1, const tf_params *p, void *ws,
                         size_t ws_bytes, void *stream) {
    if (n < 0) return TF_EINVAL;
    const int64_t offs[2] = {0, n};
    return run<false, true>(x, nullptr, nullptr, nullptr, offs, 1, out1, nullptr, nullptr, p, ws, ws_bytes,
                            stream);
}

extern "C" int plain_dot(const double *x, const double *y, int64_t n, double *out1, const tf_params *p,
                         void *ws, size_t ws_bytes, void *stream) {
    if (n < 0) return TF_EINVAL;
    const int64_t offs[2] = {0, n};
    return run<true, true>(x, nullptr, y, nullptr, offs, 1, out1, nullptr, nullptr, p, ws, ws_bytes, stream);
}

extern "C" int plain_dot_batched(const double *x, const double *y, const int64_t *offs, int32_t njobs,
                                 double *out, const tf_params *p, void *ws, size_t ws_bytes, void *stream) {
    return run<true, true>(x, nullptr, y, nullptr, offs, njobs, out, nullptr, nullptr, p, ws, ws_bytes,
                           stream);
}

// ----------------------------------------------------------------------
// twofold_dot_noalloc: the dot product without a caller workspace.
//
// For callers that cannot allocate device memory at the point of the call:
// code that must not touch the allocator once it is running (a latency-
// critical loop with a fixed memory budget, a plug-in inside a host program
// that owns every device allocation), or that holds no spare buffer to lend
// as a workspace.  The partials of the reduction live in a static device
// array of this library, reserved on every GPU that loads it until the
// process exits.  The array's address comes from cudaGetSymbolAddress, once
// per device, on the first call made with that device current; make that
// first call before any stream capture.  The address is kept per device
// index for the life of the process, so it is the one of the primary
// context: a program that resets the device (cudaDeviceReset) or works
// under another driver context must not call this entry point on that
// device afterwards.  All calls share the one array, so
// calls whose kernels overlap on the GPU (different streams, no ordering)
// race; calls ordered on one stream do not.  Nothing here needs zeroing:
// every partial is written before it is read.

namespace {

constexpr size_t kNoAllocScratchBytes = 512 * 1024;   // 32768 partial blocks
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

int noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TF_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return TF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return TF_ECUDA;
        g_noalloc_addr[dev] = ptr;
    }
    *out = g_noalloc_addr[dev];
    return TF_OK;
}

}  // namespace

extern "C" int twofold_inject_pair_drop(int32_t chunk) {
    if (chunk < -1 || chunk >= kPairChunks) return TF_EINVAL;
    return g_pair_drop.exchange(chunk);
}

extern "C" int twofold_wait_timeouts(uint64_t *count) {
    if (!count) return TF_EINVAL;
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_pair_timeouts, sizeof v) != cudaSuccess) {
        (void)cudaGetLastError();
        return TF_ECUDA;
    }
    *count = v;
    return TF_OK;
}

extern "C" int twofold_dot_noalloc(tf_in x, tf_in y, int64_t n, tf_out out1, const tf_params *p,
                                   void *stream) {
    if (n < 0) return TF_EINVAL;
    void *scratch = nullptr;
    const int st = noalloc_scratch(&scratch);
    if (st != TF_OK) return st;
    const int64_t offs[2] = {0, n};
    const int r = run<true, false>(x.hi, x.lo, y.hi, y.lo, offs, 1, out1.hi, out1.lo, out1.flags, p, scratch,
                                   kNoAllocScratchBytes, stream);
    return r == TF_ENOSPC ? TF_EUNSUPPORTED : r;     // beyond the static scratch
}

// The upper levels of the blocked pairwise order over m partials given in
// device memory (the results of aligned 2^k-leaf blocks, e.g. one per
// shard): the pairwise tree with the odd node carried, then the flag.
extern "C" int twofold_combine(const double *z0, const double *z1, int64_t m, tf_out out1, const tf_params *p,
                               void *ws, size_t ws_bytes, void *stream) {
    if (m < 0 || !tfh::params_ok(p) || !tfh::dptr_ok(out1.hi) || !tfh::dptr_ok(out1.lo)) return TF_EINVAL;
    if (m > 0 && (!tfh::dptr_ok(z0) || !tfh::dptr_ok(z1))) return TF_EINVAL;
    const size_t need = 2 * align256(sizeof(double) * (size_t)m);
    if (m > 0 && (!ws || ws_bytes < need || !tfh::aligned8(ws))) return TF_ENOSPC;
    RedArgs A{};
    A.njobs = 1;
    A.tab.ioffs[0] = 0;
    A.tab.ioffs[1] = m;
    A.tab.iblk0[0] = 0;
    A.tab.iblk0[1] = m;
    A.out_hi = out1.hi;
    A.out_lo = out1.lo;
    A.flags = out1.flags;
    A.fc = tfh::flag_cfg(p);
    A.write_single = 1;
    cudaStream_t s = tfh::as_stream(stream);
    if (m > 0) {
        // the tree works in place: on a copy in the workspace
        A.part0 = static_cast<double *>(ws);
        A.part1 = reinterpret_cast<double *>(static_cast<char *>(ws) + align256(sizeof(double) * (size_t)m));
        if (cudaMemcpyAsync(A.part0, z0, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(A.part1, z1, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return TF_ECUDA;
    }
    if (launch_final<false>(1, m, s, A) != cudaSuccess) return TF_ECUDA;
    return tfh::launch_status();
}
