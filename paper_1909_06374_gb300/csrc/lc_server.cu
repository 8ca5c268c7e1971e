// lc_server.cu -- continuous-batching server of the C ABI (lc_server_create,
// lc_submit, lc_poll, lc_server_stats, lc_server_destroy).
//
// Jobs arrive at any time.  A host thread owned by the server admits waiting
// jobs in FIFO order as a new cohort (one ragged plan) whenever the cohort's
// device footprint fits in the HBM budget, runs the cohort's setup stage, and
// then advances every live cohort by a fixed chunk of iterations per round on
// the cohort's own stream, so cohorts admitted at different times overlap on
// the device.  After each chunk the jobs whose iteration count is reached are
// copied out (device to pinned host) and retired; a cohort's memory is freed
// when its last job has retired.  Kernels are per-curve deterministic, so a
// job's result does not depend on the cohort it ran in.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
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
};

struct Cohort {
    Plan* plan = nullptr;
    std::vector<Pending> members;
    std::vector<bool> retired;
    uint32_t done_iters = 0;
    uint32_t max_iters = 0;
    void* pinned = nullptr;           // staging for finished series
    cudaEvent_t ev = nullptr;         // end of the last queued chunk
    std::vector<size_t> pending_copy; // members copied in the last chunk
    bool in_flight = false;
    size_t bytes = 0;
};

constexpr size_t kMaxQueue = 1u << 20;
constexpr uint32_t kChunkIters = 8;
constexpr size_t kMaxCohortJobs = 4096;
constexpr size_t kMaxCohorts = 8;

}  // namespace lc

using namespace lc;

struct lc_server_s {
    int device = 0;
    lc_precision prec = LC_FP32;
    size_t budget = 0;
    size_t used = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> queue;
    std::unordered_map<lc_ticket, Finished> done;
    std::unordered_map<lc_ticket, int> active;  // ticket -> 1 while admitted
    std::vector<std::unique_ptr<Cohort>> cohorts;
    std::thread th;
    bool stop = false;
    lc_ticket next_ticket = 1;
    uint64_t n_finished = 0;
    std::string fault;
};

namespace lc {

// Device bytes of a one-job plan (the arena of plan_create), used for admission.
static size_t job_footprint(const lc_job& j, lc_precision prec)
{
    const size_t ts = prec == LC_FP32 ? 4 : 8;
    const size_t n = (size_t)1 << j.log2n;
    const size_t nh = n / 2 + 1;
    const size_t tiles = n >= (size_t)kSortTile ? n / kSortTile : 1;
    size_t b = 4 * n * ts;                                  // x, f, s, A (upper bound)
    b += std::max(2 * n * ts + 2 * n * 4, 16 * nh);         // sort buffers / FP64 spectrum
    b += tiles * 256 * 4 * 2 + n / 2 * 2 * ts + 64 * 1024;  // histograms, twiddles, descriptors
    if (j.erdf.kind != LC_ERDF_SHARP) b += sizeof(double) * (kErdfTable + 1);  // ERDF CDF table
    return b;
}

static size_t plan_footprint(const std::vector<Pending>& v, lc_precision prec)
{
    size_t b = 0;
    for (auto& p : v) b += job_footprint(p.job, prec);
    return b;
}

static void retire_copied(lc_server_s* s, Cohort& c)
{
    const size_t ts = s->prec == LC_FP32 ? 4 : 8;
    auto now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t m : c.pending_copy) {
        const Pending& p = c.members[m];
        const size_t n = (size_t)1 << p.job.log2n;
        Finished f;
        f.data.resize(n * ts);
        std::memcpy(f.data.data(), (char*)c.pinned + c.plan->h_curves[m].off * ts, n * ts);
        f.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - p.t_submit).count();
        s->done.emplace(p.ticket, std::move(f));
        s->active.erase(p.ticket);
        ++s->n_finished;
    }
    c.pending_copy.clear();
}

// Queue the next chunk of a cohort and the copies of the jobs it finishes.
static lc_status advance(lc_server_s* s, Cohort& c)
{
    const size_t ts = s->prec == LC_FP32 ? 4 : 8;
    Plan& p = *c.plan;
    const uint32_t step = std::min(kChunkIters, c.max_iters - c.done_iters);
    uint64_t launches = 0;
    if (step > 0) {
        lc_status st = plan_continue(p, step, p.stream, &launches);
        if (st != LC_OK) return st;
    }
    c.done_iters += step;
    for (size_t m = 0; m < c.members.size(); ++m) {
        if (c.retired[m] || c.members[m].job.iters > c.done_iters) continue;
        const CurveDev& cv = p.h_curves[m];
        const size_t n = (size_t)1 << cv.log2n;
        if (cudaMemcpyAsync((char*)c.pinned + cv.off * ts, (char*)p.d_x + cv.off * ts, n * ts,
                            cudaMemcpyDeviceToHost, p.stream) != cudaSuccess) {
            set_error("result copy failed");
            return LC_ERR_CUDA;
        }
        c.retired[m] = true;
        c.pending_copy.push_back(m);
    }
    cudaEventRecord(c.ev, p.stream);
    c.in_flight = true;
    return LC_OK;
}

static void fail_all(lc_server_s* s, const std::string& why)
{
    std::lock_guard<std::mutex> lk(s->mu);
    s->fault = why;
}

static void server_loop(lc_server_s* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        // admission: FIFO while the next job fits in the budget
        std::vector<Pending> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            size_t bytes = 0;
            if (s->cohorts.size() < kMaxCohorts) {
                while (!s->queue.empty() && batch.size() < kMaxCohortJobs) {
                    const size_t b = job_footprint(s->queue.front().job, s->prec);
                    if (s->used + bytes + b > s->budget) break;
                    bytes += b;
                    batch.push_back(s->queue.front());
                    s->active[s->queue.front().ticket] = 1;
                    s->queue.pop_front();
                }
            }
            if (!batch.empty()) s->used += bytes;
        }
        if (!batch.empty()) {
            std::vector<lc_job> jobs;
            for (auto& b : batch) jobs.push_back(b.job);
            Plan* p = nullptr;
            lc_status st = plan_create(jobs.data(), jobs.size(), s->prec, s->device, &p);
            auto c = std::make_unique<Cohort>();
            c->members = std::move(batch);
            c->bytes = plan_footprint(c->members, s->prec);
            if (st == LC_OK) {
                c->plan = p;
                c->retired.assign(c->members.size(), false);
                for (auto& m : c->members) c->max_iters = std::max(c->max_iters, m.job.iters);
                const size_t ts = s->prec == LC_FP32 ? 4 : 8;
                if (cudaMallocHost(&c->pinned, p->total * ts) != cudaSuccess) st = LC_ERR_NOMEM;
                cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
                uint64_t l = 0;
                if (st == LC_OK) st = plan_setup(*p, nullptr, p->stream, &l);
                if (st == LC_OK) st = advance(s, *c);
            }
            if (st != LC_OK) {
                fail_all(s, std::string("cohort start failed: ") + last_error_text());
                if (c->plan) plan_free(c->plan);
                if (c->pinned) cudaFreeHost(c->pinned);
                if (c->ev) cudaEventDestroy(c->ev);
                std::lock_guard<std::mutex> lk(s->mu);
                for (auto& m : c->members) s->active.erase(m.ticket);
                s->used -= c->bytes;
                continue;
            }
            std::lock_guard<std::mutex> lk(s->mu);
            s->cohorts.push_back(std::move(c));
        }
        // progress: every cohort whose last chunk has finished
        bool progressed = !batch.empty();
        for (size_t i = 0; i < s->cohorts.size();) {
            Cohort& c = *s->cohorts[i];
            if (c.in_flight && cudaEventQuery(c.ev) == cudaErrorNotReady) { ++i; continue; }
            c.in_flight = false;
            retire_copied(s, c);
            progressed = true;
            bool all = true;
            for (bool r : c.retired) all &= r;
            if (all) {
                plan_free(c.plan);
                cudaFreeHost(c.pinned);
                cudaEventDestroy(c.ev);
                std::lock_guard<std::mutex> lk(s->mu);
                s->used -= c.bytes;
                s->cohorts.erase(s->cohorts.begin() + (long)i);
                continue;
            }
            if (advance(s, c) != LC_OK) {
                fail_all(s, std::string("chunk failed: ") + last_error_text());
                c.in_flight = false;
            }
            ++i;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            s->cv.wait_for(lk, std::chrono::microseconds(200));
        }
    }
    // shutdown: drop everything
    for (auto& c : s->cohorts) {
        if (c->plan) plan_free(c->plan);
        if (c->pinned) cudaFreeHost(c->pinned);
        if (c->ev) cudaEventDestroy(c->ev);
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
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    cudaSetDevice(prev);
    auto* s = new (std::nothrow) lc_server_s();
    if (!s) return LC_ERR_NOMEM;
    s->device = device;
    s->prec = prec;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
    try {
        s->th = std::thread(server_loop, s);
    } catch (...) {
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
    if (job_footprint(*job, server->prec) > server->budget) {
        set_error("job footprint exceeds the server's HBM budget");
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
        if (out_host) std::memcpy(out_host, it->second.data.data(), it->second.data.size());
        if (latency_ns) *latency_ns = it->second.latency_ns;
        server->done.erase(it);
        return LC_OK;
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

lc_status lc_server_destroy(lc_server server)
{
    if (!server) { set_error("null server"); return LC_ERR_INVALID; }
    {
        std::lock_guard<std::mutex> lk(server->mu);
        server->stop = true;
    }
    server->cv.notify_all();
    if (server->th.joinable()) server->th.join();
    delete server;
    return LC_OK;
}

}  // extern "C"
