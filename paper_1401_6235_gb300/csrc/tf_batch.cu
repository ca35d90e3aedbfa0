// Mixed persistent batches: sum, dot and Horner jobs of any sizes in one
// launch.
//
// Work items are an aligned block of B leaves of a sum/dot job (B a power of
// two; by the blocked pairwise order an aligned block of 2^k leaves is a
// subtree, so a job split into several items combines their partials with
// the same tree as the single-job call) or a range of P points of a Horner
// job.  The host lists the items largest first; resident CTAs take them from
// an atomic counter, so uneven jobs spread over the GPU.  The CTA that
// completes the last item of a split job (an atomic count per job, after a
// memory fence) runs that job's tree over the partials: no CTA ever waits
// for another.  The last CTA to leave resets the item counter, and each
// job's finisher its job counter, so a prepared batch can be launched again
// (for instance from a captured CUDA graph) with no host work.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tf_host.cuh"
#include "tf_leaf.cuh"

namespace {

struct BJob {
    const double *xh, *xl, *yh, *yl, *coefs;
    double *oh, *ol;
    uint8_t *of;
    int64_t n, m;          // elements (points) and leaves
    int32_t kind, k;
    int32_t nitems;        // items of this job
    int32_t part;          // first partial of a split reduction job
};

struct BArgs {
    const BJob *jobs;
    const int2 *items;     // (job, index within the job)
    int nitems;
    double *p0, *p1;       // partials of split reduction jobs
    unsigned *ctr;         // [0] item counter, [1] CTAs done, [2 + j] items done of job j
    int64_t L;
    int B, P;
    tf::FlagCfg fc;
};

// The caller's plan (tf_batch_plan is its opaque storage).
struct Plan {
    BArgs a;
    int threads, grid;
    int64_t magic;
};
static_assert(sizeof(Plan) <= sizeof(tf_batch_plan), "plan storage too small");
constexpr int64_t kPlanMagic = 0x7466626174636831LL;

__device__ __forceinline__ void put(const BJob &J, int64_t i, tf::d2 r, const tf::FlagCfg &fc) {
    J.oh[i] = r.z0;
    J.ol[i] = r.z1;
    if (J.of) J.of[i] = tf::flag_of(r.z0, r.z1, fc);
}

template <int T>
__global__ void __launch_bounds__(T) batch_kernel(const __grid_constant__ BArgs A) {
    __shared__ double s0[T], s1[T];
    __shared__ int sh_item, sh_last;
    const int t = threadIdx.x;
    for (;;) {
        if (t == 0) sh_item = (int)atomicAdd(&A.ctr[0], 1u);
        __syncthreads();
        const int it = sh_item;
        __syncthreads();
        if (it >= A.nitems) break;
        const int2 w = A.items[it];
        const BJob J = A.jobs[w.x];
        if (J.kind == TF_JOB_HORNER) {
            // s = (a_k, +0); s = ATF1.1(MTF1.1(s, x), a_i) for i = k-1 .. 0
            const int64_t q0 = (int64_t)w.y * A.P, q1 = min(J.n, q0 + A.P);
            for (int64_t i = q0 + t; i < q1; i += T) {
                const double x = J.xh[i];
                tf::d2 s = {__ldg(J.coefs + J.k), 0.0};
                for (int c = J.k - 1; c >= 0; --c) {
                    const tf::d2 m = tf::mtf11(s.z0, s.z1, x);
                    s = tf::atf11(m.z0, m.z1, __ldg(J.coefs + c));
                }
                put(J, i, s, A.fc);
            }
            continue;
        }
        // reduction item: leaves [w.y B, w.y B + nl), one per thread, then the
        // block's subtree; dotted sums and dots walk their leaves with the
        // specialised tf::leaf_walk (16-byte loads), jobs with tails with the
        // general step (fewer registers for the whole kernel)
        const bool xd = J.xl == nullptr, yd = J.yl == nullptr;
        const int64_t leaf0 = (int64_t)w.y * A.B;
        const int nl = (int)max((int64_t)0, min((int64_t)A.B, J.m - leaf0));
        if (t < nl) {
            const int64_t lb = (leaf0 + t) * A.L, le = min(J.n, lb + A.L);
            tf::d2 acc = {0.0, 0.0};
            if (J.kind == TF_JOB_DOT && xd && yd) {
                acc = tf::leaf_walk<true, true, true>(J.xh + lb, nullptr, J.yh + lb, nullptr, le - lb);
            } else if (J.kind != TF_JOB_DOT && xd) {
                acc = tf::leaf_walk<false, true, true>(J.xh + lb, nullptr, nullptr, nullptr, le - lb);
            } else {
                for (int64_t i = lb; i < le; ++i) {
                    if (J.kind == TF_JOB_DOT) {
                        const tf::d2 p = tf::apply(tf::OP_MUL, J.xh[i], xd ? 0.0 : J.xl[i], xd, J.yh[i],
                                                   yd ? 0.0 : J.yl[i], yd);
                        acc = tf::atf1(acc.z0, acc.z1, p.z0, p.z1);
                    } else {
                        acc = tf::atf1(acc.z0, acc.z1, J.xh[i], J.xl[i]);
                    }
                }
            }
            s0[t] = acc.z0;
            s1[t] = acc.z1;
        }
        __syncthreads();
        for (int st = 1; st < nl; st <<= 1) {
            if ((t & (2 * st - 1)) == 0 && t + st < nl) {
                const tf::d2 r = tf::atf1(s0[t], s1[t], s0[t + st], s1[t + st]);
                s0[t] = r.z0;
                s1[t] = r.z1;
            }
            __syncthreads();
        }
        if (J.nitems == 1) {
            if (t == 0) put(J, 0, nl ? tf::d2{s0[0], s1[0]} : tf::d2{0.0, 0.0}, A.fc);
            __syncthreads();
            continue;
        }
        if (t == 0) {
            A.p0[J.part + w.y] = s0[0];
            A.p1[J.part + w.y] = s1[0];
            __threadfence();
            const unsigned done = atomicAdd(&A.ctr[2 + w.x], 1u);
            sh_last = done == (unsigned)J.nitems - 1;
        }
        __syncthreads();
        if (sh_last) {
            // this CTA finished the job's last item: the tree over its partials.
            // Thread t folds the aligned group [t G, (t+1) G) (a subtree), then
            // the CTA combines the group roots.
            __threadfence();
            const int nb = J.nitems;
            double *q0 = A.p0 + J.part, *q1 = A.p1 + J.part;
            int G = 1;
            while (G * T < nb) G <<= 1;
            const int ng = (nb + G - 1) / G;
            if (t < ng) {
                double *g0 = q0 + t * G, *g1 = q1 + t * G;
                const int cnt = min(G, nb - t * G);
                for (int st = 1; st < cnt; st <<= 1)
                    for (int i = 0; i + st < cnt; i += 2 * st) {
                        const tf::d2 r = tf::atf1(__ldcg(g0 + i), __ldcg(g1 + i), __ldcg(g0 + i + st),
                                                  __ldcg(g1 + i + st));
                        __stcg(g0 + i, r.z0);
                        __stcg(g1 + i, r.z1);
                    }
                s0[t] = __ldcg(g0);
                s1[t] = __ldcg(g1);
            }
            __syncthreads();
            for (int st = 1; st < ng; st <<= 1) {
                if ((t & (2 * st - 1)) == 0 && t + st < ng) {
                    const tf::d2 r = tf::atf1(s0[t], s1[t], s0[t + st], s1[t + st]);
                    s0[t] = r.z0;
                    s1[t] = r.z1;
                }
                __syncthreads();
            }
            if (t == 0) {
                put(J, 0, {s0[0], s1[0]}, A.fc);
                A.ctr[2 + w.x] = 0;              // ready for the next launch
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        __threadfence();
        const unsigned e = atomicAdd(&A.ctr[1], 1u);
        if (e == gridDim.x - 1) {                // every CTA has left the item loop
            A.ctr[0] = 0;
            A.ctr[1] = 0;
            __threadfence();
        }
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Cfg {
    int B, P, T, per_sm;
};

bool cfg_of(const tf_batch_config *c, Cfg &o) {
    o = {256, 16384, 256, 0};
    if (!c) return true;
    o = {c->leaves_per_item, c->points_per_item, c->threads, c->ctas_per_sm};
    if (o.T != 128 && o.T != 256 && o.T != 512) return false;
    if (o.B < 1 || o.B > o.T || (o.B & (o.B - 1))) return false;
    if (o.P < 1 || o.per_sm < 0) return false;
    return true;
}

// Items and partials of a job list (host arithmetic only); false on a bad job.
bool count_items(const tf_job *jobs, int njobs, int64_t L, const Cfg &c, int64_t &nitems, int64_t &nparts) {
    nitems = nparts = 0;
    for (int j = 0; j < njobs; ++j) {
        const tf_job &J = jobs[j];
        if (J.n < 0) return false;
        int64_t ni;
        if (J.kind == TF_JOB_HORNER) {
            ni = (J.n + c.P - 1) / c.P;
        } else if (J.kind == TF_JOB_SUM || J.kind == TF_JOB_DOT) {
            const int64_t m = (J.n + L - 1) / L;
            ni = m == 0 ? 1 : (m + c.B - 1) / c.B;
            if (ni > 1) nparts += ni;
        } else {
            return false;
        }
        nitems += ni;
    }
    return true;
}

size_t ws_bytes_for(int njobs, int64_t nitems, int64_t nparts) {
    return align256(sizeof(BJob) * (size_t)njobs) + align256(sizeof(int2) * (size_t)nitems) +
           align256(sizeof(unsigned) * (size_t)(njobs + 2)) + 2 * align256(sizeof(double) * (size_t)nparts);
}

bool job_ok(const tf_job &J) {
    if (J.kind == TF_JOB_HORNER) {
        if (J.k < 0 || J.k > TF_HORNER_MAX_K) return false;
        if (J.n == 0) return true;                   // nothing read or written
        return tfh::dptr_ok(J.x.hi) && J.x.lo == nullptr && tfh::dptr_ok(J.coefs) && tfh::dptr_ok(J.out.hi) &&
               tfh::dptr_ok(J.out.lo);
    }
    if (!tfh::dptr_ok(J.out.hi) || !tfh::dptr_ok(J.out.lo)) return false;
    if (J.n > 0) {
        if (!tfh::dptr_ok(J.x.hi) || !tfh::optr_ok(J.x.lo)) return false;
        if (J.kind == TF_JOB_DOT && (!tfh::dptr_ok(J.y.hi) || !tfh::optr_ok(J.y.lo))) return false;
    }
    return true;
}

template <int T>
int occupancy_grid(int per_sm) {
    int b = per_sm;
    if (b == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_kernel<T>, T, 0) != cudaSuccess || b < 1))
        b = 1;
    return b * tfh::sm_count();
}

}  // namespace

extern "C" size_t twofold_batch_workspace_bytes(const tf_job *jobs, int32_t njobs, const tf_params *p,
                                                const tf_batch_config *cfg) {
    Cfg c;
    int64_t ni, np;
    if (njobs < 0 || (njobs > 0 && !jobs) || !cfg_of(cfg, c) || !tfh::params_ok(p)) return 0;
    if (!count_items(jobs, njobs, tfh::leaf_of(p), c, ni, np)) return 0;
    return ws_bytes_for(njobs, ni, np);
}

extern "C" int twofold_batch_prepare(const tf_job *jobs, int32_t njobs, const tf_params *p,
                                     const tf_batch_config *cfg, void *ws, size_t ws_bytes,
                                     tf_batch_plan *plan, void *stream) {
    Cfg c;
    if (!plan || njobs < 0 || (njobs > 0 && !jobs) || !cfg_of(cfg, c) || !tfh::params_ok(p)) return TF_EINVAL;
    std::memset(plan, 0, sizeof(*plan));
    const int64_t L = tfh::leaf_of(p);
    int64_t nitems, nparts;
    if (!count_items(jobs, njobs, L, c, nitems, nparts)) return TF_EINVAL;
    for (int j = 0; j < njobs; ++j)
        if (!job_ok(jobs[j])) return TF_EINVAL;
    if (nitems > 0x7FFFFFFFLL || nparts > 0x7FFFFFFFLL) return TF_EUNSUPPORTED;
    const size_t need = ws_bytes_for(njobs, nitems, nparts);
    if (njobs > 0 && (!ws || ws_bytes < need || ((uintptr_t)ws & 255))) return TF_ENOSPC;

    // host image: job table, items (largest first), zeroed counters
    std::vector<BJob> J(njobs);
    struct It {
        int2 w;
        double cost;
    };
    std::vector<It> items;
    items.reserve((size_t)nitems);
    int64_t part = 0;
    for (int j = 0; j < njobs; ++j) {
        const tf_job &s = jobs[j];
        BJob &d = J[j];
        d.xh = s.x.hi; d.xl = s.x.lo; d.yh = s.y.hi; d.yl = s.y.lo; d.coefs = s.coefs;
        d.oh = s.out.hi; d.ol = s.out.lo; d.of = s.out.flags;
        d.n = s.n; d.kind = s.kind; d.k = s.k;
        if (s.kind == TF_JOB_HORNER) {
            d.m = 0;
            d.nitems = (int32_t)((s.n + c.P - 1) / c.P);
            for (int i = 0; i < d.nitems; ++i) {
                const int64_t pts = std::min<int64_t>(c.P, s.n - (int64_t)i * c.P);
                items.push_back({make_int2(j, i), 1.25 * (double)pts * std::max(1, s.k)});
            }
        } else {
            d.m = (s.n + L - 1) / L;
            d.nitems = (int32_t)(d.m == 0 ? 1 : (d.m + c.B - 1) / c.B);
            d.part = d.nitems > 1 ? (int32_t)part : 0;
            if (d.nitems > 1) part += d.nitems;
            for (int i = 0; i < d.nitems; ++i) {
                const int64_t el = std::min<int64_t>((int64_t)c.B * L, s.n - (int64_t)i * c.B * L);
                items.push_back({make_int2(j, i), (s.kind == TF_JOB_DOT ? 1.0 : 0.7) * (double)std::max<int64_t>(el, 1)});
            }
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const It &a, const It &b) { return a.cost > b.cost; });
    std::vector<int2> iw(items.size());
    for (size_t i = 0; i < items.size(); ++i) iw[i] = items[i].w;

    Plan P{};
    char *w = static_cast<char *>(ws);
    BArgs &A = P.a;
    A.jobs = reinterpret_cast<const BJob *>(w);
    w += align256(sizeof(BJob) * (size_t)njobs);
    A.items = reinterpret_cast<const int2 *>(w);
    w += align256(sizeof(int2) * (size_t)nitems);
    A.ctr = reinterpret_cast<unsigned *>(w);
    w += align256(sizeof(unsigned) * (size_t)(njobs + 2));
    A.p0 = reinterpret_cast<double *>(w);
    w += align256(sizeof(double) * (size_t)nparts);
    A.p1 = reinterpret_cast<double *>(w);
    A.nitems = (int)nitems;
    A.L = L;
    A.B = c.B;
    A.P = c.P;
    A.fc = tfh::flag_cfg(p);
    P.threads = c.T;
    P.grid = c.T == 128 ? occupancy_grid<128>(c.per_sm) : c.T == 256 ? occupancy_grid<256>(c.per_sm)
                                                                    : occupancy_grid<512>(c.per_sm);
    P.magic = kPlanMagic;
    cudaStream_t s = tfh::as_stream(stream);
    if (njobs > 0) {
        if (cudaMemcpyAsync((void *)A.jobs, J.data(), sizeof(BJob) * (size_t)njobs, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            (nitems > 0 && cudaMemcpyAsync((void *)A.items, iw.data(), sizeof(int2) * (size_t)nitems,
                                           cudaMemcpyHostToDevice, s) != cudaSuccess) ||
            cudaMemsetAsync(A.ctr, 0, sizeof(unsigned) * (size_t)(njobs + 2), s) != cudaSuccess)
            return TF_ECUDA;
    }
    std::memcpy(plan, &P, sizeof(P));
    return TF_OK;
}

extern "C" int twofold_batch_launch(const tf_batch_plan *plan, void *stream) {
    if (!plan) return TF_EINVAL;
    Plan P;
    std::memcpy(&P, plan, sizeof(P));
    if (P.magic != kPlanMagic) return TF_EINVAL;
    if (P.a.nitems == 0) return TF_OK;
    cudaStream_t s = tfh::as_stream(stream);
    switch (P.threads) {
    case 128: batch_kernel<128><<<P.grid, 128, 0, s>>>(P.a); break;
    case 256: batch_kernel<256><<<P.grid, 256, 0, s>>>(P.a); break;
    case 512: batch_kernel<512><<<P.grid, 512, 0, s>>>(P.a); break;
    default: return TF_EINVAL;
    }
    return tfh::launch_status();
}

extern "C" int twofold_batch(const tf_job *jobs, int32_t njobs, const tf_params *p, const tf_batch_config *cfg,
                             void *ws, size_t ws_bytes, void *stream) {
    tf_batch_plan plan;
    const int st = twofold_batch_prepare(jobs, njobs, p, cfg, ws, ws_bytes, &plan, stream);
    if (st != TF_OK) return st;
    return twofold_batch_launch(&plan, stream);
}
