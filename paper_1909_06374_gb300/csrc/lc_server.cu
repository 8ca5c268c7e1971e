// lc_server.cu -- continuous-batching server of the C ABI (lc_server_create,
// lc_submit, lc_poll, lc_server_stats, lc_server_trace, lc_server_destroy).
//
// The server owns the large per-sample buffers (state, FFT, draws, sort keys
// and positions, amplitudes, TK spectrum) as planes of a fixed capacity of C
// samples, sized from the HBM budget when the server starts.  A buddy
// allocator hands every admitted job its own power-of-two slot of the
// planes; the slot returns to the allocator as soon as the job's result has
// been copied out, so memory frees up job by job, not cohort by cohort.
//
// A host thread admits waiting jobs whose slot can be allocated -- in arrival
// order, skipping a job that does not fit unless it has waited longer than
// kAgeLimit, after which nothing behind it is admitted until it fits -- as a
// cohort: a ragged plan whose curves live at their slots and whose small
// per-plan tables are allocated stream-ordered.  Every live cohort advances by
// a chunk of iterations per round on its own stream, so cohorts admitted at
// different times overlap on the device.  Kernels skip a curve once its
// iteration count is reached, so a retired job's slot can be reused by a new
// cohort while its old cohort keeps running.  Kernels are per-curve
// deterministic, so a job's result does not depend on its cohort or slot.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>

#include "lc_internal.h"

namespace lc {

using Clock = std::chrono::steady_clock;

struct Pending {
    lc_job job;
    lc_ticket ticket;
    Clock::time_point t_submit;
};

struct Finished {
    std::vector<char> data;
    uint64_t latency_ns;
    lc_status status;
    std::string error;
};

// Buddy allocator over [0, 2^max_log2) samples, blocks of 2^min_log2 ..
// 2^max_log2; a block of 2^l starts at a multiple of 2^l.
class Buddy {
public:
    void init(int min_log2, int max_log2)
    {
        lo_ = min_log2;
        hi_ = max_log2;
        free_.assign((size_t)hi_ + 1, {});
        free_[hi_].insert(0);
    }
    bool alloc(int log2n, uint64_t* off)
    {
        const int want = std::max(log2n, lo_);
        int l = want;
        while (l <= hi_ && free_[l].empty()) ++l;
        if (l > hi_) return false;
        uint64_t o = *free_[l].begin();
        free_[l].erase(free_[l].begin());
        while (l > want) {  // split: keep the low half, free the high half
            --l;
            free_[l].insert(o + (1ull << l));
        }
        *off = o;
        return true;
    }
    void release(uint64_t off, int log2n)
    {
        int l = std::max(log2n, lo_);
        while (l < hi_) {  // coalesce with a free buddy
            const uint64_t b = off ^ (1ull << l);
            auto it = free_[l].find(b);
            if (it == free_[l].end()) break;
            free_[l].erase(it);
            off = std::min(off, b);
            ++l;
        }
        free_[l].insert(off);
    }
    uint64_t free_samples() const
    {
        uint64_t n = 0;
        for (int l = lo_; l <= hi_; ++l) n += (uint64_t)free_[l].size() << l;
        return n;
    }

private:
    int lo_ = 4, hi_ = 4;
    std::vector<std::set<uint64_t>> free_;
};

struct Member {
    Pending p;
    uint64_t off;          // slot in the planes (samples)
    bool retired = false;   // result copy queued
    bool released = false;  // result delivered (or failed) and slot returned
    void* staging = nullptr;
};

struct Cohort {
    Plan* plan = nullptr;
    std::vector<Member> members;
    uint32_t done_iters = 0;
    uint32_t max_iters = 0;
    cudaEvent_t ev = nullptr;          // end of the last queued chunk
    cudaEvent_t t0 = nullptr, t1 = nullptr;  // device time of the last chunk
    std::vector<size_t> pending_copy;  // members copied in the last chunk
    bool in_flight = false;
};

constexpr size_t kMaxQueue = 1u << 20;
constexpr uint32_t kChunkIters = 8;
constexpr size_t kMaxCohortJobs = 4096;
constexpr size_t kMaxCohorts = 32;
constexpr auto kAgeLimit = std::chrono::milliseconds(1000);
constexpr size_t kMaxIntervals = 1u << 16;
constexpr int kMinSlotLog2 = 4;

}  // namespace lc

using namespace lc;

struct lc_server_s {
    int device = 0;
    lc_precision prec = LC_FP32;
    size_t budget = 0;
    uint64_t capacity = 0;  // samples of the planes
    void* planes_mem = nullptr;
    ExtPlanes planes{};
    Buddy buddy;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> queue;
    std::unordered_map<lc_ticket, Finished> done;
    std::unordered_map<lc_ticket, int> active;  // ticket -> 1 while admitted
    std::vector<std::unique_ptr<Cohort>> cohorts;
    std::map<int, std::vector<void*>> pinned_pool;  // staging buffers by log2n
    std::thread th;
    bool stop = false;
    bool retry_wait = false;  // a cohort start ran out of memory: wait for progress
    lc_ticket next_ticket = 1;
    uint64_t n_finished = 0;
    std::string fault;         // sticky: the CUDA context is unusable
    cudaEvent_t t_ref = nullptr;
    std::vector<std::pair<double, double>> iv;  // chunk intervals (ms after t_ref)
    std::vector<int> iv_cohort;
    int next_cohort_id = 0;
    std::unordered_map<Cohort*, int> cohort_id;
};

namespace lc {

static size_t elem_bytes(lc_precision p) { return p == LC_FP32 ? 4 : 8; }

static void* take_pinned(lc_server_s* s, int log2n)
{
    auto& v = s->pinned_pool[log2n];
    if (!v.empty()) {
        void* p = v.back();
        v.pop_back();
        return p;
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, ((size_t)1 << log2n) * elem_bytes(s->prec)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// A CUDA error after which the context cannot be used any more.
static bool context_lost(cudaError_t e)
{
    switch (e) {
    case cudaErrorIllegalAddress:
    case cudaErrorLaunchFailure:
    case cudaErrorIllegalInstruction:
    case cudaErrorMisalignedAddress:
    case cudaErrorInvalidAddressSpace:
    case cudaErrorInvalidPc:
    case cudaErrorHardwareStackError:
    case cudaErrorAssert:
    case cudaErrorLaunchTimeout:
    case cudaErrorECCUncorrectable:
        return true;
    default:
        return false;
    }
}

static void fail_tickets(lc_server_s* s, Cohort& c, lc_status st, const std::string& why)
{
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& m : c.members) {
        if (m.released) continue;
        m.released = true;
        Finished f{{}, 0, st, why};
        s->done.emplace(m.p.ticket, std::move(f));
        s->active.erase(m.p.ticket);
        s->buddy.release(m.off, (int)m.p.job.log2n);
    }
}

static void retire_copied(lc_server_s* s, Cohort& c)
{
    const size_t ts = elem_bytes(s->prec);
    auto now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t m : c.pending_copy) {
        Member& mb = c.members[m];
        const size_t n = (size_t)1 << mb.p.job.log2n;
        Finished f{{}, 0, LC_OK, {}};
        f.data.resize(n * ts);
        std::memcpy(f.data.data(), mb.staging, n * ts);
        f.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - mb.p.t_submit).count();
        s->done.emplace(mb.p.ticket, std::move(f));
        s->active.erase(mb.p.ticket);
        ++s->n_finished;
        // the slot is free for the next job: this cohort's kernels skip the curve
        s->buddy.release(mb.off, (int)mb.p.job.log2n);
        mb.released = true;
        s->pinned_pool[(int)mb.p.job.log2n].push_back(mb.staging);
        mb.staging = nullptr;
    }
    c.pending_copy.clear();
}

// Queue the next chunk of a cohort and the copies of the jobs it finishes.
static lc_status advance(lc_server_s* s, Cohort& c)
{
    const size_t ts = elem_bytes(s->prec);
    Plan& p = *c.plan;
    const uint32_t step = std::min(kChunkIters, c.max_iters - c.done_iters);
    uint64_t launches = 0;
    cudaEventRecord(c.t0, p.stream);
    if (step > 0) {
        lc_status st = plan_continue(p, step, p.stream, &launches);
        if (st != LC_OK) return st;
    }
    c.done_iters += step;
    for (size_t m = 0; m < c.members.size(); ++m) {
        Member& mb = c.members[m];
        if (mb.retired || mb.p.job.iters > c.done_iters) continue;
        const size_t n = (size_t)1 << mb.p.job.log2n;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            mb.staging = take_pinned(s, (int)mb.p.job.log2n);
        }
        if (!mb.staging) { set_error("pinned staging allocation failed"); return LC_ERR_NOMEM; }
        if (cudaMemcpyAsync(mb.staging, (char*)p.d_x + mb.off * ts, n * ts, cudaMemcpyDeviceToHost, p.stream) !=
            cudaSuccess) {
            set_error("result copy failed");
            return LC_ERR_CUDA;
        }
        mb.retired = true;
        c.pending_copy.push_back(m);
    }
    cudaEventRecord(c.t1, p.stream);
    cudaEventRecord(c.ev, p.stream);
    c.in_flight = true;
    return LC_OK;
}

static void record_interval(lc_server_s* s, Cohort& c)
{
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, s->t_ref, c.t0) != cudaSuccess ||
        cudaEventElapsedTime(&b, s->t_ref, c.t1) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->iv.size() >= kMaxIntervals) return;
    s->iv.emplace_back(a, b);
    s->iv_cohort.push_back(s->cohort_id[&c]);
}

static void destroy_cohort(lc_server_s* s, std::unique_ptr<Cohort>& c)
{
    if (c->plan) plan_free(c->plan);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->t0) cudaEventDestroy(c->t0);
    if (c->t1) cudaEventDestroy(c->t1);
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& m : c->members)
        if (m.staging) s->pinned_pool[(int)m.p.job.log2n].push_back(m.staging);
    s->cohort_id.erase(c.get());
}

static void server_loop(lc_server_s* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        // admission: arrival order; a job whose slot cannot be allocated is
        // skipped unless it has waited longer than kAgeLimit, in which case no
        // later job is admitted before it
        std::vector<Member> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            if (s->cohorts.size() < kMaxCohorts && !s->retry_wait && s->fault.empty()) {
                const auto now = Clock::now();
                for (auto it = s->queue.begin(); it != s->queue.end() && batch.size() < kMaxCohortJobs;) {
                    uint64_t off = 0;
                    if (s->buddy.alloc((int)it->job.log2n, &off)) {
                        batch.push_back(Member{*it, off});
                        s->active[it->ticket] = 1;
                        it = s->queue.erase(it);
                        continue;
                    }
                    if (now - it->t_submit > kAgeLimit) break;
                    ++it;
                }
            }
        }
        if (!batch.empty()) {
            std::vector<lc_job> jobs;
            std::vector<uint64_t> offs;
            for (auto& b : batch) {
                jobs.push_back(b.p.job);
                offs.push_back(b.off);
            }
            Plan* p = nullptr;
            lc_status st = plan_create_ext(jobs.data(), jobs.size(), s->prec, s->device, &s->planes, offs.data(), &p);
            auto c = std::make_unique<Cohort>();
            c->members = std::move(batch);
            if (st == LC_OK) {
                c->plan = p;
                for (auto& m : c->members) c->max_iters = std::max(c->max_iters, m.p.job.iters);
                cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
                cudaEventCreate(&c->t0);
                cudaEventCreate(&c->t1);
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->cohort_id[c.get()] = s->next_cohort_id++;
                }
                uint64_t l = 0;
                st = plan_setup(*p, nullptr, p->stream, &l);
                if (st == LC_OK) st = advance(s, *c);
            }
            if (st != LC_OK) {
                const cudaError_t e = cudaPeekAtLastError();
                const std::string why = std::string("cohort start failed: ") + last_error_text();
                if (context_lost(e)) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->fault = why;
                } else if (st == LC_ERR_NOMEM && !s->cohorts.empty()) {
                    // back to the front of the queue, in order; retry once
                    // another cohort has made progress
                    cudaGetLastError();
                    std::lock_guard<std::mutex> lk(s->mu);
                    for (auto it = c->members.rbegin(); it != c->members.rend(); ++it) {
                        s->buddy.release(it->off, (int)it->p.job.log2n);
                        s->active.erase(it->p.ticket);
                        s->queue.push_front(it->p);
                    }
                    s->retry_wait = true;
                    c->members.clear();
                } else {
                    cudaGetLastError();
                    fail_tickets(s, *c, st, why);
                }
                destroy_cohort(s, c);
                continue;
            }
            std::lock_guard<std::mutex> lk(s->mu);
            s->cohorts.push_back(std::move(c));
        }
        // progress: every cohort whose last chunk has finished
        bool progressed = false;
        for (size_t i = 0; i < s->cohorts.size();) {
            Cohort& c = *s->cohorts[i];
            if (c.in_flight) {
                const cudaError_t q = cudaEventQuery(c.ev);
                if (q == cudaErrorNotReady) { ++i; continue; }
                if (q != cudaSuccess) {
                    const std::string why = std::string("chunk failed: ") + cudaGetErrorString(q);
                    cudaGetLastError();
                    if (context_lost(q)) {
                        std::lock_guard<std::mutex> lk(s->mu);
                        s->fault = why;
                    }
                    fail_tickets(s, c, LC_ERR_CUDA, why);
                    destroy_cohort(s, s->cohorts[i]);
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->cohorts.erase(s->cohorts.begin() + (long)i);
                    continue;
                }
                record_interval(s, c);
            }
            c.in_flight = false;
            retire_copied(s, c);
            progressed = true;
            bool all = true;
            for (auto& m : c.members) all &= m.retired;
            if (all) {
                destroy_cohort(s, s->cohorts[i]);
                std::lock_guard<std::mutex> lk(s->mu);
                s->cohorts.erase(s->cohorts.begin() + (long)i);
                continue;
            }
            const lc_status st = advance(s, c);
            if (st != LC_OK) {
                const std::string why = std::string("chunk failed: ") + last_error_text();
                const cudaError_t e = cudaPeekAtLastError();
                cudaGetLastError();
                if (context_lost(e)) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->fault = why;
                }
                cudaStreamSynchronize(c.plan->stream);
                retire_copied(s, c);
                fail_tickets(s, c, st, why);
                destroy_cohort(s, s->cohorts[i]);
                std::lock_guard<std::mutex> lk(s->mu);
                s->cohorts.erase(s->cohorts.begin() + (long)i);
                continue;
            }
            ++i;
        }
        if (progressed) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->retry_wait = false;
        }
        if (!progressed && batch.empty()) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            s->cv.wait_for(lk, std::chrono::microseconds(200));
        }
    }
    // shutdown: drop everything
    for (auto& c : s->cohorts) {
        if (c->plan) cudaStreamSynchronize(c->plan->stream);
        destroy_cohort(s, c);
    }
    s->cohorts.clear();
}

}  // namespace lc

extern "C" {

lc_status lc_server_create(int device, size_t hbm_budget_bytes, lc_precision prec, lc_server* out)
{
    if (!out) { set_error("out is null"); return LC_ERR_INVALID; }
    *out = nullptr;
    if (prec != LC_FP32 && prec != LC_FP64) { set_error("bad precision"); return LC_ERR_INVALID; }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("no such CUDA device");
        return LC_ERR_INVALID;
    }
    DeviceGuard g(device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    auto* s = new (std::nothrow) lc_server_s();
    if (!s) return LC_ERR_NOMEM;
    s->device = device;
    s->prec = prec;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
    // planes of a power-of-two capacity: 7/8 of the budget (the rest holds
    // the cohorts' per-plan tables and twiddles)
    const size_t bps = ext_plane_bytes_per_sample(prec);
    const double fit = 0.875 * (double)s->budget / (double)bps;
    int cap_log2 = kMinSlotLog2;
    while (cap_log2 < 40 && (double)(1ull << (cap_log2 + 1)) <= fit) ++cap_log2;
    if ((double)(1ull << cap_log2) > fit) {
        delete s;
        set_error("HBM budget too small for any job");
        return LC_ERR_INVALID;
    }
    s->capacity = 1ull << cap_log2;
    const size_t C = (size_t)s->capacity, ts = elem_bytes(prec);
    const size_t nh = (size_t)ext_half_offset(C) + 1;
    const size_t bytes = 3 * C * ts + 2 * C * ts + 2 * C * 4 + nh * ts + nh * 16 + 6 * 256;
    if (cudaMalloc(&s->planes_mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        set_error("device allocation of the server planes (" + std::to_string(bytes) + " bytes) failed");
        return LC_ERR_NOMEM;
    }
    char* b = (char*)s->planes_mem;
    size_t at = 0;
    auto take = [&](size_t n) { void* q = b + at; at = (at + n + 255) / 256 * 256; return q; };
    s->planes.x = take(C * ts);
    s->planes.f = take(C * ts);
    s->planes.s = take(C * ts);
    s->planes.keysA = take(C * ts);
    s->planes.keysB = take(C * ts);
    s->planes.valsA = (uint32_t*)take(C * 4);
    s->planes.valsB = (uint32_t*)take(C * 4);
    s->planes.A = take(nh * ts);
    s->planes.spec = (double2*)take(nh * 16);
    s->buddy.init(kMinSlotLog2, cap_log2);
    cudaEventCreate(&s->t_ref);
    cudaEventRecord(s->t_ref, 0);
    cudaEventSynchronize(s->t_ref);
    try {
        s->th = std::thread(server_loop, s);
    } catch (...) {
        cudaFree(s->planes_mem);
        cudaEventDestroy(s->t_ref);
        delete s;
        set_error("could not start the server thread");
        return LC_ERR_NOMEM;
    }
    *out = s;
    return LC_OK;
}

lc_status lc_submit(lc_server server, const lc_job* job, lc_ticket* out)
{
    if (!server || !job || !out) { set_error("null argument"); return LC_ERR_INVALID; }
    lc_status st = validate_job(*job);
    if (st != LC_OK) return st;
    if (((uint64_t)1 << std::max<uint32_t>(job->log2n, (uint32_t)kMinSlotLog2)) > server->capacity) {
        set_error("job longer than the server's planes (HBM budget)");
        return LC_ERR_INVALID;
    }
    {
        std::lock_guard<std::mutex> lk(server->mu);
        if (!server->fault.empty()) { set_error(server->fault); return LC_ERR_CUDA; }
        if (server->queue.size() >= kMaxQueue) { set_error("admission queue full"); return LC_ERR_BUSY; }
        Pending p{*job, server->next_ticket++, Clock::now()};
        server->queue.push_back(p);
        *out = p.ticket;
    }
    server->cv.notify_one();
    return LC_OK;
}

lc_status lc_poll(lc_server server, lc_ticket ticket, void* out_host, uint64_t* latency_ns)
{
    if (!server) { set_error("null server"); return LC_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(server->mu);
    auto it = server->done.find(ticket);
    if (it != server->done.end()) {
        const lc_status st = it->second.status;
        if (st == LC_OK) {
            if (out_host) std::memcpy(out_host, it->second.data.data(), it->second.data.size());
            if (latency_ns) *latency_ns = it->second.latency_ns;
        } else {
            set_error(it->second.error);
        }
        server->done.erase(it);
        return st;
    }
    if (!server->fault.empty()) { set_error(server->fault); return LC_ERR_CUDA; }
    if (server->active.count(ticket)) return LC_PENDING;
    for (auto& p : server->queue)
        if (p.ticket == ticket) return LC_PENDING;
    set_error("unknown ticket");
    return LC_ERR_UNKNOWN_TICKET;
}

lc_status lc_server_stats(lc_server server, uint64_t* finished, uint64_t* active, uint64_t* waiting)
{
    if (!server) { set_error("null server"); return LC_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(server->mu);
    if (finished) *finished = server->n_finished;
    if (active) *active = server->active.size();
    if (waiting) *waiting = server->queue.size();
    return LC_OK;
}

lc_status lc_server_trace(lc_server server, double* busy_ms, double* overlap_ms, uint64_t* free_samples,
                          uint64_t* capacity)
{
    if (!server) { set_error("null server"); return LC_ERR_INVALID; }
    std::vector<std::pair<double, double>> iv;
    std::vector<int> who;
    {
        std::lock_guard<std::mutex> lk(server->mu);
        iv = server->iv;
        who = server->iv_cohort;
        if (free_samples) *free_samples = server->buddy.free_samples();
        if (capacity) *capacity = server->capacity;
    }
    // sweep over chunk start / end points: time with at least one chunk on
    // the device, and time with chunks of two or more cohorts at once
    std::vector<std::pair<double, int>> ev;  // (time, +cohort+1 start / -(cohort+1) end)
    for (size_t i = 0; i < iv.size(); ++i) {
        ev.emplace_back(iv[i].first, who[i] + 1);
        ev.emplace_back(iv[i].second, -(who[i] + 1));
    }
    std::sort(ev.begin(), ev.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
        return a.first < b.first || (a.first == b.first && a.second < b.second);
    });
    std::map<int, int> live;  // cohort -> chunks in flight
    double busy = 0.0, over = 0.0, last = 0.0;
    for (auto& e : ev) {
        const double dt = e.first - last;
        if (!live.empty()) busy += dt;
        if (live.size() >= 2) over += dt;
        last = e.first;
        const int c = std::abs(e.second) - 1;
        if (e.second > 0) ++live[c];
        else if (--live[c] == 0) live.erase(c);
    }
    if (busy_ms) *busy_ms = busy;
    if (overlap_ms) *overlap_ms = over;
    return LC_OK;
}

lc_status lc_server_destroy(lc_server server)
{
    if (!server) { set_error("null server"); return LC_ERR_INVALID; }
    {
        std::lock_guard<std::mutex> lk(server->mu);
        server->stop = true;
    }
    server->cv.notify_all();
    if (server->th.joinable()) server->th.join();
    {
        DeviceGuard g(server->device);
        cudaDeviceSynchronize();
        for (auto& kv : server->pinned_pool)
            for (void* p : kv.second) cudaFreeHost(p);
        cudaFree(server->planes_mem);
        cudaEventDestroy(server->t_ref);
    }
    delete server;
    return LC_OK;
}

lc_status lc_plan_footprint(const lc_job* jobs, size_t njobs, lc_precision prec, size_t* bytes)
{
    if (!bytes) { set_error("bytes is null"); return LC_ERR_INVALID; }
    return plan_arena_bytes(jobs, njobs, prec, false, bytes);
}

}  // extern "C"
