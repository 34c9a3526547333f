// Continuous-batching request server for overdensity profiles.
//
// Rapid scanning (many cosmologies, halo masses, relic masses and grids) means
// a stream of requests of very different sizes.  The server keeps the GPU busy
// with all of them at once: a worker thread admits queued requests first come,
// first served while the device budget (one arena, sub-allocated first fit)
// and the slot limit allow, and runs one persistent trajectory launch per
// iteration over every admitted request.  Each launch advances every request
// by a chunk of RK4 steps, with the trajectories' state kept in device memory
// between launches; a request that reaches its last step forms its quadrature
// in that launch and leaves, freeing its memory for the next ones.  Requests
// that arrive while others are on the GPU therefore join at the next launch
// and share it (iteration-level batching).  Because a request is integrated
// with the same operations and the same tiles whatever shares its launches,
// its result is bitwise the one it gets alone.
//
// A request whose last chunk runs in a launch is delivered as soon as its
// last radius is finished: the kernel raises a flag in host-mapped memory and
// the worker reads the result while the launch still runs the others.
//
// Every wait on the GPU is bounded (gpu_timeout_ms): a launch that does not
// complete in time fails the requests it carried with NU_ETIMEDOUT and the
// server stops admitting work.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <vector>

#include "nuprof_internal.h"

using namespace nuprof;

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// First-fit sub-allocator over one device block (offsets, 256-byte aligned).
class Arena {
public:
    void reset(void* base, size_t bytes)
    {
        base_ = static_cast<unsigned char*>(base);
        size_ = bytes;
        free_.clear();
        free_[0] = bytes;
        used_ = peak_ = 0;
    }
    void* alloc(size_t bytes)
    {
        bytes = up256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            sizes_[off] = bytes;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return base_ + off;
        }
        return nullptr;
    }
    void release(void* p)
    {
        if (!p) return;
        const size_t off = static_cast<unsigned char*>(p) - base_;
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t len = s->second;
        sizes_.erase(s);
        used_ -= len;
        size_t start = off;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first == off + len) {   // merge right
            len += next->second;
            free_.erase(next);
        }
        auto prev = free_.lower_bound(off);
        if (prev != free_.begin()) {                                // merge left
            --prev;
            if (prev->first + prev->second == off) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    unsigned char* base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;    // offset -> length
    std::map<size_t, size_t> sizes_;   // offset -> length of live blocks
};

void* arena_alloc_cb(size_t bytes, void* ctx) { return static_cast<Arena*>(ctx)->alloc(bytes); }
void arena_free_cb(void* p, size_t, void* ctx) { static_cast<Arena*>(ctx)->release(p); }

struct Pending {
    long long ticket;
    nu_cosmo cosmo;
    nu_halo halo;
    nu_relic relic;
    nu_pgrid grid;
    nu_opts opts;
    std::vector<double> radii;
    std::vector<double> masses;   // relic masses of a mass-reuse request (owned copy)
    std::vector<double> ftable;   // tabulated f (owned copy)
    Clock::time_point t_submit;
    void fix()
    {
        relic.masses_eV = masses.empty() ? nullptr : masses.data();
        relic.f_table = ftable.empty() ? nullptr : ftable.data();
    }
};

struct Active {
    long long ticket;
    nu_profile* h;
    void* state;
    int progress;
    int n_steps;
    bool cancelled;
    Clock::time_point t_submit;
    Clock::time_point t_ready;    // verified requests: when the mixed result was ready
};

struct Done {
    int rc;
    std::vector<double> out, err;
    double latency_ms;
};

}  // namespace

struct nu_server {
    nu_server_opts o;
    int device = 0;
    void* block = nullptr;                  // the arena's device memory
    Arena arena;
    cudaStream_t compute = nullptr, upload = nullptr;
    cudaStream_t verify = nullptr;          // FP64 runs of verified requests
    cudaEvent_t ev = nullptr;
    DevProblem* d_desc[2] = {nullptr, nullptr};   // per-iteration descriptors (double buffer)
    int* d_prefix[2] = {nullptr, nullptr};
    unsigned* d_ctrl = nullptr;
    size_t capacity = 0;                    // arena bytes left for requests

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> pending;
    std::map<long long, Done> done;
    std::set<long long> delivered;
    std::map<long long, bool> cancel_requests;
    std::vector<Active> active;             // on the GPU (the launch in flight)
    std::vector<Active> staged;             // admitted, join the next launch
    std::vector<Active> verifying;          // mixed result ready, FP64 run still going
    std::atomic<int> on_device{0};          // active + staged, for statistics
    long long next_ticket = 1;
    bool stop = false;
    int fatal = NU_OK;
    std::thread worker;

    // statistics (under mu)
    long long submitted = 0, admitted = 0, completed = 0, cancelled = 0, rejected = 0;
    long long iterations = 0, traj_steps = 0, early = 0;
    double busy_ms = 0.0;
    int max_active_seen = 0;
    std::vector<double> latencies;

    void run();
    bool admit_one();
    void deliver_verified();
    double staged_work() const
    {
        double w = 0.0;
        for (const Active& a : staged)
            w += (double)profile_n_traj(a.h) * (o.chunk_steps > 0 ? o.chunk_steps : a.n_steps);
        return w;
    }
    void finish(Active& a, int rc, std::vector<double>* out, std::vector<double>* err);
    void release(Active& a);                // memory back to the arena
    void record(Active& a, int rc, std::vector<double>* out, std::vector<double>* err);

    // early delivery: a request whose last chunk is in the launch signals its
    // last radius through host-mapped flags, and its result is read and
    // delivered while the launch still runs the others
    unsigned* h_flags = nullptr;            // page-locked, mapped: one per active slot
    unsigned* d_flags = nullptr;            // the same memory as the device sees it
    unsigned* d_counts = nullptr;           // radii finished, per active slot (arena)

    // resident launches: the work queue (page-locked, mapped) through which
    // requests admitted during a launch join it
    QueueCtl* h_q = nullptr;
    QueueCtl* d_q = nullptr;
    bool resident_running = false;          // a resident launch is waiting on the host
    bool defer_close = false;               // a request can only be admitted after it ends
    long long joined = 0, queue_expired = 0;   // statistics (under mu)
};

void nu_server::finish(Active& a, int rc, std::vector<double>* out, std::vector<double>* err)
{
    release(a);
    record(a, rc, out, err);
}

void nu_server::release(Active& a)
{
    nu_profile_destroy(a.h);                 // returns its memory to the arena
    arena.release(a.state);
    on_device.fetch_sub(1);
}

void nu_server::record(Active& a, int rc, std::vector<double>* out, std::vector<double>* err)
{
    Done d;
    d.rc = rc;
    if (out) d.out.swap(*out);
    if (err) d.err.swap(*err);
    d.latency_ms = ms_since(a.t_submit);
    std::lock_guard<std::mutex> g(mu);
    if (rc == NU_OK) {
        ++completed;
        latencies.push_back(d.latency_ms);
    } else if (rc == NU_ECANCELED) {
        ++cancelled;
    }
    done[a.ticket] = std::move(d);
}

// Admit the request at the head of the queue into `staged` if memory and
// slots allow.  Returns true if the queue head was consumed (admitted,
// refused or cancelled), false if it has to wait (or the queue is empty).
bool nu_server::admit_one()
{
    Pending p;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (pending.empty() || (int)(active.size() + staged.size()) >= o.max_active || fatal != NU_OK)
            return false;
        auto c = cancel_requests.find(pending.front().ticket);
        if (c != cancel_requests.end()) {
            done[pending.front().ticket] = Done{NU_ECANCELED, {}, {}, ms_since(pending.front().t_submit)};
            ++cancelled;
            cancel_requests.erase(c);
            pending.pop_front();
            return true;
        }
        p = pending.front();
    }
    p.fix();
    nu_plan_info info;
    int rc = nu_profile_plan(&p.cosmo, &p.halo, &p.relic, p.radii.data(), (int)p.radii.size(),
                             &p.grid, &p.opts, &info);
    const size_t sz = o.precision == NU_FP64 ? sizeof(double) : sizeof(float);
    const size_t state_bytes = (size_t)info.n_traj * 4 * sz;
    if (rc == NU_OK && up256((size_t)info.device_bytes) + up256(state_bytes) > capacity)
        rc = NU_ENOMEM;                       // can never fit: refuse
    // while a resident launch waits on this thread, nothing may synchronize the
    // device: a request whose upload would grow the page-locked staging buffer
    // waits for the launch to end
    if (rc == NU_OK && resident_running && (size_t)info.h2d_bytes > staging_capacity()) {
        defer_close = true;
        return false;
    }
    nu_profile* h = nullptr;
    void* state = nullptr;
    if (rc == NU_OK) {
        state = arena.alloc(state_bytes);
        if (state) rc = nu_profile_create(&p.cosmo, &p.halo, &p.relic, p.radii.data(),
                                          (int)p.radii.size(), &p.grid, &p.opts, &h);
        if (!state || rc == NU_ENOMEM) {
            arena.release(state);
            if (h) nu_profile_destroy(h);
            if (!active.empty() || !staged.empty()) {                // wait for room
                defer_close = resident_running;
                return false;
            }
            rc = NU_ENOMEM;                   // nothing to wait for: refuse
            state = nullptr;
            h = nullptr;
        }
    }
    if (rc == NU_OK && profile_twin(h)) {     // a verified request: its FP64 run starts now
        rc = profile_twin_run(h, verify);
        if (rc != NU_OK) {
            nu_profile_destroy(h);
            h = nullptr;
        }
    }
    std::lock_guard<std::mutex> g(mu);
    pending.pop_front();
    if (rc != NU_OK) {
        arena.release(state);
        done[p.ticket] = Done{rc, {}, {}, ms_since(p.t_submit)};
        ++rejected;
        return true;
    }
    staged.push_back(Active{p.ticket, h, state, 0, profile_n_steps(h), false, p.t_submit, {}});
    ++admitted;
    on_device.store((int)(active.size() + staged.size()));
    return true;
}

// Deliver verified requests whose FP64 run has finished (bounded: one that
// does not finish within gpu_timeout_ms of its mixed result fails with
// NU_ETIMEDOUT, and its memory is leaked rather than freed under a kernel).
void nu_server::deliver_verified()
{
    for (size_t i = 0; i < verifying.size();) {
        Active& a = verifying[i];
        const int q = profile_twin_query(a.h);
        if (q == NU_EAGAIN && ms_since(a.t_ready) <= o.gpu_timeout_ms) {
            ++i;
            continue;
        }
        if (q == NU_OK) {
            const int nr = profile_n_out(a.h);
            std::vector<double> out(nr), err(nr);
            const int r = profile_read(a.h, out.data(), err.data(), upload);
            finish(a, r, &out, &err);
        } else {
            record(a, q == NU_EAGAIN ? NU_ETIMEDOUT : q, nullptr, nullptr);
        }
        verifying.erase(verifying.begin() + i);
    }
}

void nu_server::run()
{
    cudaSetDevice(device);
    const int tpt = o.tpt;
    const int tile = o.block * traj_per_thread(tpt);
    const bool gtab = (o.flags & NU_FLAG_GTAB) != 0;
    int slot = 0;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) return;
            if (active.empty() && staged.empty() && pending.empty())
                cv.wait_for(lk, std::chrono::milliseconds(verifying.empty() ? 20 : 1));
            if (stop) return;
        }
        deliver_verified();
        // with nothing on the GPU, admit requests up to one launch's budget
        // before launching (the rest are admitted while it runs)
        if (active.empty()) {
            double work = 0.0;
            while (work < o.step_budget && admit_one())
                if (!staged.empty()) work = staged_work();
        }
        for (auto& a : staged) active.push_back(a);
        staged.clear();
        {
            std::lock_guard<std::mutex> g(mu);
            max_active_seen = std::max(max_active_seen, (int)active.size());
            for (auto& a : active) {
                auto c = cancel_requests.find(a.ticket);
                if (c != cancel_requests.end()) {
                    a.cancelled = true;
                    cancel_requests.erase(c);
                }
            }
        }
        // retire cancelled requests before the launch
        for (size_t i = 0; i < active.size();) {
            if (active[i].cancelled) {
                finish(active[i], NU_ECANCELED, nullptr, nullptr);
                active.erase(active.begin() + i);
            } else {
                ++i;
            }
        }
        if (active.empty()) continue;

        // ---- one launch: every active request advances by one chunk ----
        // chunk: chunk_steps, shrunk so that the launch stays within step_budget
        double traj_active = 0.0;
        for (const Active& a : active) traj_active += (double)profile_n_traj(a.h);
        int chunk = o.chunk_steps;
        if (chunk > 0 && traj_active * chunk > o.step_budget)
            chunk = std::max(1, (int)(o.step_budget / traj_active));
        std::vector<DevProblem> desc(active.size());
        std::vector<int> early_st(active.size(), 0);   // 1: signals this launch, 2: delivered
        std::vector<int> prefix(active.size() + 1, 0);
        long long steps_this = 0;
        size_t smem = 0;                          // the largest table staged this launch
        for (size_t i = 0; i < active.size(); ++i) {
            const Active& a = active[i];
            smem = std::max(smem, coef_smem_bytes(o.precision, a.n_steps, tpt));
            DevProblem d = profile_desc(a.h);
            const long long seg = (long long)d.n_q * d.n_mu;
            d.tile = tile;
            d.tiles_per_seg = (int)((seg + tile - 1) / tile);
            d.state = a.state;
            d.step_begin = a.progress;
            d.step_end = std::min(a.n_steps, a.progress + (chunk > 0 ? chunk : a.n_steps));
            d.done_count = nullptr;
            d.done_flag = nullptr;
            if (h_flags && d.step_end == a.n_steps && !profile_twin(a.h)) {
                h_flags[i] = 0u;
                d.done_count = d_counts + i;
                d.done_flag = d_flags + i;
                early_st[i] = 1;
            }
            desc[i] = d;
            prefix[i + 1] = prefix[i] + d.tiles_per_seg * d.n_radii;
            steps_this += profile_n_traj(a.h) * (d.step_end - d.step_begin);
        }
        const int n = (int)active.size();
        int rc = NU_OK;
        if (cudaMemcpyAsync(d_desc[slot], desc.data(), n * sizeof(DevProblem), cudaMemcpyHostToDevice,
                            compute) != cudaSuccess ||
            cudaMemcpyAsync(d_prefix[slot], prefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice,
                            compute) != cudaSuccess ||
            cudaMemsetAsync(d_ctrl, 0, 2 * sizeof(unsigned), compute) != cudaSuccess ||
            (h_flags && cudaMemsetAsync(d_counts, 0, n * sizeof(unsigned), compute) != cudaSuccess))
            rc = NU_ECUDA;
        int grid = 0, per_sm = 0, sms = 0;
        // a resident launch stages tables up to the largest a request may have
        // (requests join it later), so that its shared memory fits any of them
        const bool res = o.resident != 0;
        if (res) smem = std::max(smem, coef_smem_bytes(o.precision, NU_MAX_STEPS, tpt));
        if (rc == NU_OK) rc = max_ctas_per_sm(o.precision, tpt, o.block, smem, &per_sm, gtab);
        if (rc == NU_OK && (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
                            per_sm < 1))
            rc = NU_ECUDA;
        if (rc == NU_OK && res) {                // open the queue with this launch's requests
            h_q->n_probs = (unsigned)n;
            h_q->want_work = 0u;
            h_q->wait_limit_ns = (unsigned long long)(o.queue_wait_ms * 1e6);
            __atomic_store_n(&h_q->word, ((unsigned long long)kQueueOpen << 32) | (unsigned)prefix[n],
                             __ATOMIC_SEQ_CST);
        }
        if (rc == NU_OK) {
            // a resident launch keeps every CTA: the ones without work wait for
            // requests that join
            grid = res ? per_sm * sms : std::max(1, std::min(prefix[n], per_sm * sms));
            rc = launch_traj(o.precision, tpt, o.block, grid, smem, d_desc[slot], d_prefix[slot], n,
                             prefix[n], d_ctrl, compute, gtab, res ? d_q : nullptr);
        }
        const auto t_launch = Clock::now();
        auto t_publish = t_launch;               // resident: the last time work joined
        auto t_want = t_launch;                  // resident: when the queue was first seen dry
        bool queue_open = res && rc == NU_OK;
        bool want_seen = false;
        resident_running = queue_open;
        defer_close = false;
        // resident: no more joins; CTAs that run dry then leave the launch
        auto close_queue = [&]() {
            unsigned long long w = __atomic_load_n(&h_q->word, __ATOMIC_SEQ_CST);
            while ((unsigned)(w >> 32) == kQueueOpen) {
                const unsigned long long closed = ((unsigned long long)kQueueClosed << 32) | (unsigned)w;
                if (__atomic_compare_exchange_n(&h_q->word, &w, closed, false, __ATOMIC_SEQ_CST,
                                                __ATOMIC_SEQ_CST))
                    break;
            }
            queue_open = false;
        };
        // resident: append staged requests to the running launch and publish them
        auto join_staged = [&]() {
            static const unsigned zero = 0u;
            size_t k = 0;
            for (; k < staged.size() && active.size() < (size_t)o.max_active; ++k) {
                Active& a = staged[k];
                const int i = (int)active.size();
                DevProblem d = profile_desc(a.h);
                const long long seg = (long long)d.n_q * d.n_mu;
                d.tile = tile;
                d.tiles_per_seg = (int)((seg + tile - 1) / tile);
                d.state = a.state;
                d.step_begin = 0;
                d.step_end = a.n_steps;
                d.done_count = nullptr;
                d.done_flag = nullptr;
                const bool signal = !profile_twin(a.h);
                if (signal) {
                    h_flags[i] = 0u;
                    d.done_count = d_counts + i;
                    d.done_flag = d_flags + i;
                }
                const int next = prefix.back() + d.tiles_per_seg * d.n_radii;
                if (cudaMemcpyAsync(d_desc[slot] + i, &d, sizeof(DevProblem), cudaMemcpyHostToDevice,
                                    upload) != cudaSuccess ||
                    cudaMemcpyAsync(d_prefix[slot] + i + 1, &next, sizeof(int), cudaMemcpyHostToDevice,
                                    upload) != cudaSuccess ||
                    cudaMemcpyAsync(d_counts + i, &zero, sizeof(unsigned), cudaMemcpyHostToDevice,
                                    upload) != cudaSuccess ||
                    cudaStreamSynchronize(upload) != cudaSuccess) {
                    cudaGetLastError();
                    break;                       // it stays staged for the next launch
                }
                __atomic_store_n(&h_q->n_probs, (unsigned)(i + 1), __ATOMIC_SEQ_CST);
                unsigned long long expect = ((unsigned long long)kQueueOpen << 32) | (unsigned)prefix.back();
                const unsigned long long want = ((unsigned long long)kQueueOpen << 32) | (unsigned)next;
                if (!__atomic_compare_exchange_n(&h_q->word, &expect, want, false, __ATOMIC_SEQ_CST,
                                                 __ATOMIC_SEQ_CST)) {
                    queue_open = false;          // closed or expired meanwhile: next launch
                    break;
                }
                active.push_back(a);
                desc.push_back(d);
                prefix.push_back(next);
                early_st.push_back(signal ? 1 : 0);
                steps_this += profile_n_traj(a.h) * a.n_steps;
                t_publish = Clock::now();
                std::lock_guard<std::mutex> g(mu);
                ++joined;
                max_active_seen = std::max(max_active_seen, (int)active.size());
            }
            staged.erase(staged.begin(), staged.begin() + k);
        };
        if (rc == NU_OK && cudaEventRecord(ev, compute) != cudaSuccess) rc = NU_ECUDA;
        // bounded wait for the launch; requests that arrive meanwhile are
        // admitted now (their tables upload on a separate stream) and join
        // the next launch
        while (rc == NU_OK) {
            const cudaError_t q = cudaEventQuery(ev);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) {
                rc = NU_ECUDA;
                break;
            }
            if (ms_since(t_publish) > o.gpu_timeout_ms) {
                rc = NU_ETIMEDOUT;
                break;
            }
            // deliver requests that have finished inside the running launch
            for (size_t i = 0; i < active.size(); ++i) {
                if (early_st[i] != 1 || reinterpret_cast<volatile unsigned*>(h_flags)[i] != 1u) continue;
                const int nr = profile_n_out(active[i].h);
                std::vector<double> out(nr), err(nr);
                const int r = profile_read(active[i].h, out.data(), err.data(), upload);
                record(active[i], r, &out, &err);
                early_st[i] = 2;
                std::lock_guard<std::mutex> g(mu);
                ++early;
            }
            deliver_verified();
            const bool admitted_one = admit_one();
            if (queue_open) {
                if (!staged.empty()) join_staged();
                // close the queue (no more joins; the launch ends when its CTAs
                // have run dry) when it has run dry with nothing queued for
                // linger_ms, when its slots are used up while requests wait,
                // when a request can only be admitted after the launch, or
                // when the launch has lived a quarter of the GPU time limit
                if (!want_seen && __atomic_load_n(&h_q->want_work, __ATOMIC_ACQUIRE) != 0u) {
                    want_seen = true;
                    t_want = Clock::now();
                }
                bool waiting;
                {
                    std::lock_guard<std::mutex> g(mu);
                    waiting = !pending.empty();
                }
                const auto t_dry = std::max(t_want, t_publish);
                bool close = defer_close || ms_since(t_launch) > 0.25 * o.gpu_timeout_ms ||
                             (active.size() >= (size_t)o.max_active && (waiting || !staged.empty()));
                if (want_seen && !waiting && staged.empty() && ms_since(t_dry) >= o.linger_ms) close = true;
                if (close) close_queue();
            }
            // poll closely at first (short launches finish within a few ms and a
            // sleep would add its granularity to every chunk), then back off
            if (!admitted_one) {
                if (ms_since(t_launch) < 2.0) std::this_thread::yield();
                else std::this_thread::sleep_for(std::chrono::microseconds(50));
            }
        }
        if (queue_open) close_queue();           // an error ended the wait: no CTA waits on
        resident_running = false;
        if (res && rc == NU_OK &&
            (unsigned)(__atomic_load_n(&h_q->word, __ATOMIC_SEQ_CST) >> 32) == kQueueExpired) {
            std::lock_guard<std::mutex> g(mu);
            ++queue_expired;                     // a CTA's bounded wait ended the launch
        }
        const double launch_ms = ms_since(t_launch);
        slot ^= 1;
        if (rc != NU_OK) {
            cudaGetLastError();
            {
                // the server stops admitting: queued requests fail with the same status
                std::lock_guard<std::mutex> g(mu);
                fatal = rc;
                for (auto& p : pending) done[p.ticket] = Done{rc, {}, {}, ms_since(p.t_submit)};
                pending.clear();
            }
            if (rc == NU_ETIMEDOUT) {
                // the GPU may still be running the launch: fail the requests but
                // keep their memory (it may still be written)
                std::lock_guard<std::mutex> g(mu);
                for (size_t i = 0; i < active.size(); ++i)   // (those delivered early keep their result)
                    if (early_st[i] != 2) done[active[i].ticket] = Done{rc, {}, {}, ms_since(active[i].t_submit)};
                for (auto& a : staged) done[a.ticket] = Done{rc, {}, {}, ms_since(a.t_submit)};
                active.clear();
                staged.clear();
                return;
            }
            for (size_t i = 0; i < active.size(); ++i) {
                if (early_st[i] == 2) release(active[i]);
                else finish(active[i], rc, nullptr, nullptr);
            }
            active.clear();
            continue;
        }
        {
            std::lock_guard<std::mutex> g(mu);
            ++iterations;
            traj_steps += steps_this;
            busy_ms += launch_ms;
        }
        // ---- retire the requests that reached their last step ----
        // (desc[i] describes active[i] of this launch; build the survivors in a
        // new list so that the two stay paired while requests leave)
        std::vector<Active> keep;
        keep.reserve(active.size());
        for (size_t i = 0; i < active.size(); ++i) {
            Active a = active[i];
            a.progress = desc[i].step_end;
            if (a.progress < a.n_steps) {
                keep.push_back(a);
                continue;
            }
            if (early_st[i] == 2) {               // delivered during the launch
                release(a);
                continue;
            }
            if (profile_twin(a.h)) {              // delivered when its FP64 run is done
                a.t_ready = Clock::now();
                verifying.push_back(a);
                continue;
            }
            const int nr = profile_n_out(a.h);
            std::vector<double> out(nr), err(nr);
            const int r = profile_read(a.h, out.data(), err.data(), upload);
            finish(a, r, &out, &err);
        }
        active.swap(keep);
    }
}

extern "C" {

int nu_server_create(const nu_server_opts* opts, nu_server** out)
{
    if (!opts || !out) return NU_EINVAL;
    std::unique_ptr<nu_server> s(new (std::nothrow) nu_server());
    if (!s) return NU_ENOMEM;
    s->o = *opts;
    nu_server_opts& o = s->o;
    if (o.precision != NU_FP64 && o.precision != NU_MIXED) return NU_EINVAL;
    if (o.max_active <= 0) o.max_active = 64;
    if (o.max_active > 65536) return NU_EINVAL;
    if (o.block == 0) o.block = o.precision == NU_MIXED ? 128 : 256;
    if (o.tpt == 0) {
        o.tpt = o.precision == NU_MIXED ? kTptPacked : 1;
        if (o.precision == NU_MIXED && o.flags == 0) o.flags = NU_FLAG_GTAB;
    }
    if (o.block < 64 || o.block > 512 || o.block % 32 != 0) return NU_EINVAL;
    if (o.tpt != 1 && o.tpt != 2 && o.tpt != kTptPacked) return NU_EINVAL;
    if (o.tpt == kTptPacked && o.precision != NU_MIXED) return NU_EINVAL;
    if (o.chunk_steps < 0) return NU_EINVAL;
    if (o.gpu_timeout_ms <= 0.0) o.gpu_timeout_ms = 60000.0;
    if (o.resident && o.chunk_steps != 0) return NU_EINVAL;   // resident launches run whole requests
    if (o.linger_ms < 0.0) return NU_EINVAL;
    if (o.queue_wait_ms <= 0.0) o.queue_wait_ms = 1000.0;
    if (o.step_budget <= 0.0) o.step_budget = 4e9;
    if (o.device_bytes < ((size_t)1 << 20)) return NU_EINVAL;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    if (o.alloc) {
        s->block = o.alloc(o.device_bytes, o.alloc_ctx);
        if (!s->block) return NU_ENOMEM;
    } else if (cudaMalloc(&s->block, o.device_bytes) != cudaSuccess) {
        cudaGetLastError();
        return NU_ENOMEM;
    }
    s->arena.reset(s->block, o.device_bytes);
    for (int i = 0; i < 2; ++i) {
        s->d_desc[i] = static_cast<DevProblem*>(s->arena.alloc((size_t)o.max_active * sizeof(DevProblem)));
        s->d_prefix[i] = static_cast<int*>(s->arena.alloc((size_t)(o.max_active + 1) * sizeof(int)));
    }
    s->d_ctrl = static_cast<unsigned*>(s->arena.alloc(256));
    s->d_counts = static_cast<unsigned*>(s->arena.alloc((size_t)o.max_active * sizeof(unsigned)));
    s->capacity = s->arena.size() - s->arena.used();
    auto fail = [&](int rc) {
        if (s->compute) cudaStreamDestroy(s->compute);
        if (s->upload) cudaStreamDestroy(s->upload);
        if (s->verify) cudaStreamDestroy(s->verify);
        if (s->ev) cudaEventDestroy(s->ev);
        if (o.alloc) {
            if (o.free) o.free(s->block, o.device_bytes, o.alloc_ctx);
        } else {
            cudaFree(s->block);
        }
        return rc;
    };
    if (!s->d_desc[0] || !s->d_desc[1] || !s->d_prefix[0] || !s->d_prefix[1] || !s->d_ctrl ||
        !s->d_counts)
        return fail(NU_ENOMEM);
    // completion flags in page-locked memory the GPU writes directly; without
    // them results are delivered when their launch ends
    if (cudaHostAlloc(reinterpret_cast<void**>(&s->h_flags), (size_t)o.max_active * sizeof(unsigned),
                      cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_flags), s->h_flags, 0) != cudaSuccess) {
        cudaGetLastError();
        if (s->h_flags) cudaFreeHost(s->h_flags);
        s->h_flags = nullptr;
        s->d_flags = nullptr;
    }
    if (o.resident) {
        // the queue word is changed by compare-and-swap from the host and the GPU
        int native = 0;
        if (!s->h_flags ||
            cudaDeviceGetAttribute(&native, cudaDevAttrHostNativeAtomicSupported, s->device) != cudaSuccess ||
            !native) {
            cudaGetLastError();
            if (s->h_flags) cudaFreeHost(s->h_flags);
            return fail(NU_ENOTSUP);
        }
        if (cudaHostAlloc(reinterpret_cast<void**>(&s->h_q), sizeof(QueueCtl), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_q), s->h_q, 0) != cudaSuccess) {
            cudaGetLastError();
            if (s->h_q) cudaFreeHost(s->h_q);
            cudaFreeHost(s->h_flags);
            return fail(NU_ECUDA);
        }
        std::memset(s->h_q, 0, sizeof(QueueCtl));
        // room for typical uploads, so that admissions during a launch never
        // have to grow the staging buffer
        staging_reserve((size_t)16 << 20);
    }
    if (cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->verify, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (s->h_flags) cudaFreeHost(s->h_flags);
        if (s->h_q) cudaFreeHost(s->h_q);
        return fail(NU_ECUDA);
    }
    nu_server* raw = s.get();
    raw->worker = std::thread([raw] { raw->run(); });
    *out = s.release();
    return NU_OK;
}

int nu_server_submit(nu_server* s, const nu_cosmo* cosmo, const nu_halo* halo, const nu_relic* relic,
                     const double* radii, int n_radii, const nu_pgrid* p_grid, const nu_opts* opts,
                     long long* ticket)
{
    if (!s || !cosmo || !halo || !relic || !radii || n_radii < 1 || !p_grid || !ticket) return NU_EINVAL;
    Pending p;
    p.cosmo = *cosmo;
    p.halo = *halo;
    p.relic = *relic;
    p.grid = *p_grid;
    std::memset(&p.opts, 0, sizeof(p.opts));
    if (opts) {
        p.opts.n_steps = opts->n_steps;
        p.opts.z_end = opts->z_end;
        p.opts.radii_unit = opts->radii_unit;
        p.opts.flags = opts->flags & NU_FLAG_VERIFY;
    }
    p.opts.precision = s->o.precision;
    p.opts.block = s->o.block;
    p.opts.tpt = s->o.tpt;
    p.opts.alloc = arena_alloc_cb;
    p.opts.free = arena_free_cb;
    p.opts.alloc_ctx = &s->arena;
    p.opts.stream = s->upload;
    p.radii.assign(radii, radii + n_radii);
    if (relic->n_masses > 0 && relic->masses_eV)
        p.masses.assign(relic->masses_eV, relic->masses_eV + std::min(relic->n_masses, NU_MAX_MASSES));
    if (relic->f_kind == NU_F_TABLE && relic->f_table && relic->n_table > 0)
        p.ftable.assign(relic->f_table, relic->f_table + std::min(relic->n_table, NU_MAX_FTABLE));
    p.fix();
    nu_plan_info info;
    const int rc = nu_profile_plan(&p.cosmo, &p.halo, &p.relic, radii, n_radii, &p.grid, &p.opts, &info);
    if (rc != NU_OK) return rc;
    p.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->fatal != NU_OK) return s->fatal;
        p.ticket = s->next_ticket++;
        *ticket = p.ticket;
        s->pending.push_back(std::move(p));
        ++s->submitted;
    }
    s->cv.notify_one();
    return NU_OK;
}

int nu_server_poll(nu_server* s, long long ticket, double* n_over_nbar, double* err_est, int n_radii,
                   double* latency_ms)
{
    if (!s || !n_over_nbar) return NU_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        if (ticket < 1 || ticket >= s->next_ticket || s->delivered.count(ticket)) return NU_EINVAL;
        return NU_EAGAIN;
    }
    const Done& d = it->second;
    if (latency_ms) *latency_ms = d.latency_ms;
    const int rc = d.rc;
    if (rc == NU_OK) {
        if ((int)d.out.size() != n_radii) return NU_EINVAL;
        std::memcpy(n_over_nbar, d.out.data(), n_radii * sizeof(double));
        if (err_est) std::memcpy(err_est, d.err.data(), n_radii * sizeof(double));
    }
    s->done.erase(it);
    s->delivered.insert(ticket);
    return rc;
}

int nu_server_cancel(nu_server* s, long long ticket)
{
    if (!s) return NU_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (ticket < 1 || ticket >= s->next_ticket) return NU_EINVAL;
        if (s->done.count(ticket) || s->delivered.count(ticket)) return NU_EINVAL;   // finished
        s->cancel_requests[ticket] = true;
    }
    s->cv.notify_one();
    return NU_OK;
}

int nu_server_stats(nu_server* s, nu_serve_stats* out)
{
    if (!s || !out) return NU_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->cancelled = s->cancelled;
    out->rejected = s->rejected;
    out->iterations = s->iterations;
    out->traj_steps = s->traj_steps;
    out->busy_ms = s->busy_ms;
    out->pending = (int)s->pending.size();
    out->active = s->on_device.load();
    out->max_active_seen = s->max_active_seen;
    out->arena_bytes = (long long)s->arena.size();
    out->arena_peak = (long long)s->arena.peak();
    out->status = s->fatal;
    out->early = s->early;
    out->joined = s->joined;
    out->queue_expired = s->queue_expired;
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            const double pos = p * (l.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - i;
            return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double m = 0;
        for (double v : l) m += v;
        out->mean_ms = m / l.size();
    }
    return NU_OK;
}

void nu_server_destroy(nu_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    const bool gpu_ok = s->fatal != NU_ETIMEDOUT;
    if (gpu_ok) {
        cudaStreamSynchronize(s->compute);
        cudaStreamSynchronize(s->verify);
        for (auto* list : {&s->active, &s->staged, &s->verifying})
            for (auto& a : *list) {
                nu_profile_destroy(a.h);
                s->arena.release(a.state);
            }
    }
    // after a timeout the arena and the flags may still be in use by the GPU:
    // they are leaked rather than freed under a running kernel
    if (gpu_ok) {
        if (s->h_flags) cudaFreeHost(s->h_flags);
        if (s->h_q) cudaFreeHost(s->h_q);
        if (s->o.alloc) {
            if (s->o.free) s->o.free(s->block, s->o.device_bytes, s->o.alloc_ctx);
        } else {
            cudaFree(s->block);
        }
    }
    cudaStreamDestroy(s->compute);
    cudaStreamDestroy(s->upload);
    cudaStreamDestroy(s->verify);
    cudaEventDestroy(s->ev);
    delete s;
}

}  // extern "C"
