// A serving loop for twofold jobs: requests with host buffers are admitted
// by device memory, batched continuously and run as mixed persistent
// batches (sum / dot / Horner) plus elementwise launches.
//
// One scheduler thread per server owns a device arena of the configured
// size.  Requests wait in FIFO order; whenever memory and a stream are free
// the scheduler admits the longest prefix of the queue that fits (inputs,
// outputs and the batch workspace) within a quarter of the arena (so that
// up to three batches share it and their copies pipeline even when the
// queue is long), copies the inputs in, runs the batch and
// copies the results out on a free stream of its pool, and records an event.
// Finished batches release their memory, and requests that arrived while
// others ran are admitted as memory frees up, so several batches are in
// flight at once and their copies and kernels overlap.  Every result is the
// one the single-job entry point returns for the same inputs: a request's
// result does not depend on what it is batched with.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tf_host.cuh"

namespace {

constexpr int kStreams = 4;          // stream pool; at most kStreams - 1 batches in flight
constexpr size_t kAlign = 256;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) with coalescing free blocks.
class Arena {
  public:
    void init(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, o = it->first + bytes;
                free_.erase(it);
                if (rest) free_[o] = rest;
                used_ += bytes;
                if (used_ > peak_) peak_ = used_;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = up(bytes ? bytes : 1);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t peak() const { return peak_; }

  private:
    size_t used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

enum { ST_PENDING = 1, ST_RUNNING = 2 };

struct Req {
    uint64_t id = 0;
    tf_request r{};
    std::vector<int32_t> prog;
    size_t off = 0, bytes = 0;           // arena block of inputs and outputs
    int status = ST_PENDING;             // then TF_OK or a negative tf_status
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    int batch_jobs = 0;
    // device addresses inside the block
    const double *din[8] = {};
    const double *dcoefs = nullptr;
    double *dhi = nullptr, *dlo = nullptr;
    uint8_t *dfl = nullptr;
};

int nin_of(const tf_request &r) {
    switch (r.kind) {
    case TF_JOB_SUM: return 2;
    case TF_JOB_DOT: return 4;
    case TF_JOB_HORNER: return 1;
    default: return 2 * r.nin;
    }
}

int64_t nout_of(const tf_request &r) { return (r.kind == TF_JOB_SUM || r.kind == TF_JOB_DOT) ? 1 : r.n; }

// Bytes of a request's block: its present inputs, coefficients and outputs.
size_t block_bytes(const tf_request &r) {
    size_t b = 0;
    const int ni = nin_of(r);
    for (int i = 0; i < ni; ++i)
        if (r.in[i]) b += up(sizeof(double) * (size_t)r.n);
    if (r.kind == TF_JOB_HORNER) b += up(sizeof(double) * (size_t)(r.k + 1));
    const size_t no = (size_t)nout_of(r);
    b += 2 * up(sizeof(double) * no) + up(no);
    return b;
}

void place(Req &q, char *base) {
    char *p = base + q.off;
    const int ni = nin_of(q.r);
    const size_t n = (size_t)q.r.n;
    for (int i = 0; i < ni; ++i) {
        if (q.r.in[i]) {
            q.din[i] = reinterpret_cast<const double *>(p);
            p += up(sizeof(double) * n);
        } else {
            q.din[i] = nullptr;
        }
    }
    if (q.r.kind == TF_JOB_HORNER) {
        q.dcoefs = reinterpret_cast<const double *>(p);
        p += up(sizeof(double) * (size_t)(q.r.k + 1));
    }
    const size_t no = (size_t)nout_of(q.r);
    q.dhi = reinterpret_cast<double *>(p);
    p += up(sizeof(double) * no);
    q.dlo = reinterpret_cast<double *>(p);
    p += up(sizeof(double) * no);
    q.dfl = reinterpret_cast<uint8_t *>(p);
}

struct Batch {
    std::vector<std::shared_ptr<Req>> reqs;
    int stream = -1;
    cudaEvent_t ev = nullptr;
    size_t ws_off = 0, ws_bytes = 0;
    int status = TF_OK;
};

}  // namespace

struct tf_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
    std::vector<std::unique_ptr<Batch>> inflight;
    Arena arena;
    char *base = nullptr;
    cudaStream_t streams[kStreams] = {};
    bool stream_busy[kStreams] = {};
    std::thread th;
    bool stop = false;
    int device = 0;
    int max_jobs = 4096;
    size_t batch_cap = 0;      // request bytes per batch (a larger single request runs alone)
    bool has_p = false, has_cfg = false;
    tf_params p{};
    tf_batch_config cfg{};
    uint64_t next_id = 1;
    tf_server_stats st{};
    int inject_every = 0;      // twofold_server_inject_failures: fail every n-th started batch
    int64_t started = 0;       // batches started since injection was set

    void run();
    bool admit(Batch &b);
    void start(Batch &b);
    void finish(Batch &b, int status);
};

// Forms a batch from the head of the queue (caller holds mu).  False when
// nothing could be admitted.
bool tf_server::admit(Batch &b) {
    const tf_params *pp = has_p ? &p : nullptr;
    const tf_batch_config *cp = has_cfg ? &cfg : nullptr;
    size_t bytes = 0;
    while (!pending.empty() && (int)b.reqs.size() < max_jobs) {
        auto q = pending.front();
        if (!b.reqs.empty() && bytes + q->bytes > batch_cap) break;
        size_t off;
        if (!arena.alloc(q->bytes, &off)) break;
        bytes += q->bytes;
        q->off = off;
        pending.pop_front();
        b.reqs.push_back(q);
    }
    // the batch workspace; give back the newest requests until it fits
    while (!b.reqs.empty()) {
        std::vector<tf_job> jobs;
        for (auto &q : b.reqs) {
            if (q->r.kind == TF_JOB_EW) continue;
            tf_job j{};
            j.kind = q->r.kind;
            j.k = q->r.k;
            j.n = q->r.n;
            j.x = {reinterpret_cast<const double *>(kAlign), nullptr};    // sizes only
            j.out = {reinterpret_cast<double *>(kAlign), reinterpret_cast<double *>(kAlign), nullptr};
            jobs.push_back(j);
        }
        b.ws_bytes = jobs.empty() ? 0 : twofold_batch_workspace_bytes(jobs.data(), (int32_t)jobs.size(), pp, cp);
        if (b.ws_bytes == 0 || arena.alloc(b.ws_bytes, &b.ws_off)) break;
        auto q = b.reqs.back();
        b.reqs.pop_back();
        arena.release(q->off, q->bytes);
        pending.push_front(q);
    }
    if (b.reqs.empty() && inflight.empty() && !pending.empty()) {
        // the head cannot fit even in an empty arena
        auto q = pending.front();
        pending.pop_front();
        q->status = TF_ENOSPC;
        q->t_done = now_ns();
        ++st.failed;
        cv_done.notify_all();
    }
    return !b.reqs.empty();
}

// Copies in, computes and copies out on the batch's stream (no lock held).
// The stream is idle when the batch starts (its previous batch finished), so
// the table upload of the batch plan does not wait for anything.
void tf_server::start(Batch &b) {
    cudaStream_t s = streams[b.stream];
    const tf_params *pp = has_p ? &p : nullptr;
    const tf_batch_config *cp = has_cfg ? &cfg : nullptr;
    int status = TF_OK;
    std::vector<tf_job> jobs;
    for (auto &qp : b.reqs) {
        Req &q = *qp;
        place(q, base);
        if (q.r.kind == TF_JOB_EW) continue;
        tf_job j{};
        j.kind = q.r.kind;
        j.k = q.r.k;
        j.n = q.r.n;
        if (q.r.kind == TF_JOB_HORNER) {
            j.x = {q.din[0], nullptr};
            j.coefs = q.dcoefs;
        } else {
            j.x = {q.din[0], q.din[1]};
            if (q.r.kind == TF_JOB_DOT) j.y = {q.din[2], q.din[3]};
        }
        j.out = {q.dhi, q.dlo, q.dfl};
        jobs.push_back(j);
    }
    tf_batch_plan plan;
    if (!jobs.empty())
        status = twofold_batch_prepare(jobs.data(), (int32_t)jobs.size(), pp, cp, base + b.ws_off, b.ws_bytes, &plan,
                                       s);
    for (auto &qp : b.reqs) {
        Req &q = *qp;
        const int ni = nin_of(q.r);
        for (int i = 0; i < ni && status == TF_OK; ++i)
            if (q.r.in[i] && q.r.n > 0 &&
                cudaMemcpyAsync((void *)q.din[i], q.r.in[i], sizeof(double) * (size_t)q.r.n,
                                cudaMemcpyHostToDevice, s) != cudaSuccess)
                status = TF_ECUDA;
        if (q.r.kind == TF_JOB_HORNER && status == TF_OK &&
            cudaMemcpyAsync((void *)q.dcoefs, q.r.coefs, sizeof(double) * (size_t)(q.r.k + 1),
                            cudaMemcpyHostToDevice, s) != cudaSuccess)
            status = TF_ECUDA;
    }
    if (status == TF_OK && !jobs.empty()) status = twofold_batch_launch(&plan, s);
    for (auto &qp : b.reqs) {
        Req &q = *qp;
        if (status != TF_OK) break;
        if (q.r.kind == TF_JOB_EW) {
            tf_in in[4];
            for (int i = 0; i < q.r.nin; ++i) in[i] = {q.din[2 * i], q.din[2 * i + 1]};
            status = twofold_ew(q.prog.data(), (int32_t)q.prog.size() / 4, in, q.r.nin, q.r.n,
                                tf_out{q.dhi, q.dlo, q.dfl}, pp, s);
        }
    }
    for (auto &qp : b.reqs) {
        Req &q = *qp;
        if (status != TF_OK) break;
        const size_t no = (size_t)nout_of(q.r);
        if (no == 0) continue;
        if (cudaMemcpyAsync(q.r.out_hi, q.dhi, sizeof(double) * no, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(q.r.out_lo, q.dlo, sizeof(double) * no, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (q.r.out_flags &&
             cudaMemcpyAsync(q.r.out_flags, q.dfl, no, cudaMemcpyDeviceToHost, s) != cudaSuccess))
            status = TF_ECUDA;
    }
    if (status == TF_OK && cudaEventRecord(b.ev, s) != cudaSuccess) status = TF_ECUDA;
    if (status != TF_OK) cudaStreamSynchronize(s);   // nothing of the batch may still run when it is released
    b.status = status;
}

void tf_server::finish(Batch &b, int status) {
    const int64_t t = now_ns();
    for (auto &q : b.reqs) {
        q->status = status;
        q->t_done = t;
        q->batch_jobs = (int)b.reqs.size();
        arena.release(q->off, q->bytes);
        if (status == TF_OK) ++st.completed;
        else ++st.failed;
    }
    if (b.ws_bytes) arena.release(b.ws_off, b.ws_bytes);
    stream_busy[b.stream] = false;
    ++st.batches;
    st.batched_jobs += (int64_t)b.reqs.size();
    cv_done.notify_all();
}

void tf_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // completions
        for (size_t i = 0; i < inflight.size();) {
            Batch &b = *inflight[i];
            const cudaError_t e = b.status == TF_OK ? cudaEventQuery(b.ev) : cudaSuccess;
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            if (e != cudaSuccess) (void)cudaGetLastError();
            finish(b, b.status != TF_OK ? b.status : (e == cudaSuccess ? TF_OK : TF_ECUDA));
            if (b.ev) cudaEventDestroy(b.ev);        // null when its creation failed
            inflight.erase(inflight.begin() + (long)i);
        }
        if (stop && pending.empty() && inflight.empty()) break;
        // admission onto a free stream
        int free_stream = -1;
        for (int k = 0; k < kStreams; ++k)
            if (!stream_busy[k]) { free_stream = k; break; }
        std::unique_ptr<Batch> nb;
        if (free_stream >= 0 && (int)inflight.size() < kStreams - 1 && !pending.empty()) {
            nb.reset(new Batch());
            if (!admit(*nb)) nb.reset();
        }
        if (nb) {
            nb->stream = free_stream;
            stream_busy[free_stream] = true;
            const int64_t t = now_ns();
            for (auto &q : nb->reqs) {
                q->status = ST_RUNNING;
                q->t_admit = t;
            }
            if (inflight.size() + 1 > (size_t)st.max_inflight) st.max_inflight = (int32_t)(inflight.size() + 1);
            st.peak_bytes = (int64_t)arena.peak();
            Batch *bp = nb.get();
            inflight.push_back(std::move(nb));
            const bool injected = inject_every > 0 && ++started % inject_every == 0;
            lk.unlock();
            if (cudaEventCreateWithFlags(&bp->ev, cudaEventDisableTiming) != cudaSuccess) bp->status = TF_ECUDA;
            else if (injected) bp->status = TF_ECUDA;    // an injected failure: nothing of the batch runs
            else start(*bp);
            lk.lock();
            continue;
        }
        if (!inflight.empty()) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            cv_work.wait(lk, [&] { return stop || !pending.empty(); });
        }
    }
}

extern "C" int twofold_server_create(size_t mem_cap_bytes, int32_t max_batch_jobs, const tf_params *p,
                                     const tf_batch_config *cfg, tf_server **out) {
    if (!out || mem_cap_bytes < 4096 || max_batch_jobs < 1 || !tfh::params_ok(p)) return TF_EINVAL;
    *out = nullptr;
    if (cfg) {
        tf_job dummy{};
        dummy.kind = TF_JOB_SUM;
        if (twofold_batch_workspace_bytes(&dummy, 1, p, cfg) == 0) return TF_EINVAL;
    }
    std::unique_ptr<tf_server> s(new tf_server());
    if (cudaGetDevice(&s->device) != cudaSuccess) return TF_ECUDA;
    if (cudaMalloc(&s->base, mem_cap_bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return TF_ECUDA;
    }
    s->arena.init(mem_cap_bytes);
    for (int k = 0; k < kStreams; ++k) {
        if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
            for (int i = 0; i < k; ++i) cudaStreamDestroy(s->streams[i]);
            cudaFree(s->base);
            return TF_ECUDA;
        }
    }
    s->max_jobs = max_batch_jobs;
    s->batch_cap = mem_cap_bytes / kStreams;
    if (p) { s->p = *p; s->has_p = true; }
    if (cfg) { s->cfg = *cfg; s->has_cfg = true; }
    s->st.arena_bytes = (int64_t)mem_cap_bytes;
    tf_server *raw = s.get();
    s->th = std::thread([raw] { raw->run(); });
    *out = s.release();
    return TF_OK;
}

extern "C" int twofold_server_submit(tf_server *s, const tf_request *r, uint64_t *ticket) {
    if (!s || !r || !ticket || r->n < 0) return TF_EINVAL;
    const bool red = r->kind == TF_JOB_SUM || r->kind == TF_JOB_DOT;
    if (!red && r->kind != TF_JOB_HORNER && r->kind != TF_JOB_EW) return TF_EINVAL;
    if (nout_of(*r) > 0 && (!r->out_hi || !r->out_lo)) return TF_EINVAL;
    auto q = std::make_shared<Req>();
    q->r = *r;
    if (r->n > 0) {
        if (!r->in[0]) return TF_EINVAL;
        if (r->kind == TF_JOB_DOT && !r->in[2]) return TF_EINVAL;
    }
    if (r->kind == TF_JOB_HORNER) {
        if (r->k < 0 || r->k > TF_HORNER_MAX_K || !r->coefs || r->in[1]) return TF_EINVAL;
    }
    if (r->kind == TF_JOB_EW) {
        if (r->nin < 1 || r->nin > 4 || !r->prog || r->nprog < 1 || r->nprog > TF_EW_MAX_PROG) return TF_EINVAL;
        for (int i = 0; i < r->nin; ++i)
            if (r->n > 0 && !r->in[2 * i]) return TF_EINVAL;
        q->prog.assign(r->prog, r->prog + 4 * r->nprog);
        q->r.prog = nullptr;
        // validate the program (n = 0: nothing is read, written or launched)
        tf_in in[4] = {};
        if (twofold_ew(q->prog.data(), r->nprog, in, r->nin, 0, tf_out{}, s->has_p ? &s->p : nullptr, nullptr) !=
            TF_OK)
            return TF_EINVAL;
    } else {
        q->r.nin = 0;
    }
    q->bytes = block_bytes(q->r);
    q->t_submit = now_ns();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) return TF_EINVAL;
        q->id = s->next_id++;
        s->reqs[q->id] = q;
        s->pending.push_back(q);
        *ticket = q->id;
    }
    s->cv_work.notify_one();
    return TF_OK;
}

extern "C" int twofold_server_wait(tf_server *s, uint64_t ticket, int32_t timeout_ms, tf_request_info *info) {
    if (!s) return TF_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return TF_EINVAL;
    auto q = it->second;
    auto done = [&] { return q->status != ST_PENDING && q->status != ST_RUNNING; };
    if (timeout_ms < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return TF_ETIMEOUT;
    if (info) {
        info->submitted_ns = q->t_submit;
        info->admitted_ns = q->t_admit;
        info->done_ns = q->t_done;
        info->status = q->status;
        info->batch_jobs = q->batch_jobs;
    }
    s->reqs.erase(it);
    return q->status;
}

extern "C" int twofold_server_stats(tf_server *s, tf_server_stats *out) {
    if (!s || !out) return TF_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    out->peak_bytes = (int64_t)s->arena.peak();
    out->pending = (int64_t)s->pending.size();
    out->inflight = (int32_t)s->inflight.size();
    return TF_OK;
}

extern "C" int twofold_server_inject_failures(tf_server *s, int32_t every) {
    if (!s || every < 0) return TF_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    s->inject_every = every;
    s->started = 0;
    return TF_OK;
}

extern "C" int twofold_server_destroy(tf_server *s) {
    if (!s) return TF_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (int k = 0; k < kStreams; ++k) cudaStreamDestroy(s->streams[k]);
    const cudaError_t e = cudaFree(s->base);
    delete s;
    return e == cudaSuccess ? TF_OK : TF_ECUDA;
}
