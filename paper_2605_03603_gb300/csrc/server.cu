// Serving counts: a request loop over resident graphs with continuous
// batching.
//
// Requests (graph, p, q) arrive at any time (sbc_server_submit, thread-safe)
// and are answered asynchronously (sbc_server_wait). A scheduler thread owns
// the queue and a set of device lanes (one CUDA stream and one worker thread
// each). Whenever a lane is free it forms the next job from the oldest
// waiting request:
//  * requests on small graphs are fused with the other waiting small-graph
//    requests of the same (p, q) into one batched count (the disjoint-union
//    count of sbc_count_batch); a graph asked for twice in one job is counted
//    once;
//  * requests on large graphs run alone.
// A job is admitted only while the device bytes of the jobs in flight plus
// its estimated footprint stay within the server's memory budget (a job that
// alone exceeds the budget waits until nothing else runs). Jobs on different
// lanes run concurrently on the device, so requests arriving while others
// are on the GPU are admitted as lanes and memory free up. Graphs stay
// resident (their oriented structures are built once and reused); results
// are never cached across requests.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sbc_internal.cuh"

namespace sbc {

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
}

struct Request {
    uint64_t ticket = 0;
    uint32_t gid = 0;
    int p = 0, q = 0;
    Clock::time_point submitted, done;
    int state = 0;  // 0 waiting, 1 running, 2 finished
    sbc_status status = SBC_OK;
    std::string error;
    sbc_u128 result{0, 0};
};

struct Job {
    std::vector<Request *> reqs;
    int p = 0, q = 0;
    uint64_t bytes = 0;
    bool batched = false;
};

struct Lane {
    cudaStream_t stream = nullptr;
    std::thread thread;
    Job *job = nullptr;
    std::condition_variable cv;
};

}  // namespace
}  // namespace sbc

struct sbc_server {
    sbc_server_opts opts;
    int device = 0;
    std::vector<const sbc_graph *> graphs;
    std::vector<uint64_t> footprint;  // estimated device bytes of one count per graph
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<sbc::Request *> waiting;
    std::unordered_map<uint64_t, sbc::Request *> requests;
    uint64_t next_ticket = 1;
    uint64_t in_flight_bytes = 0, peak_bytes = 0;
    int running_jobs = 0;
    bool stopping = false;
    std::vector<sbc::Lane *> lanes;
    std::thread scheduler;
    // statistics
    std::vector<double> latencies_ms;
    uint64_t submitted = 0, completed = 0, failed = 0, jobs = 0, fused = 0;
    sbc::Clock::time_point first_submit, last_done;
    bool any_submit = false;
};

namespace sbc {
namespace {

// Rough device footprint of one count: oriented structures are resident, a
// count allocates plan arrays per edge and anchor, candidate masks bounded by
// the wedges, and work items.
uint64_t estimate_bytes(const sbc_graph *g) {
    const uint64_t w = std::min(g->wedges_u, g->wedges_v);
    return 32ull * (uint64_t)g->nnz + 64ull * (uint64_t)std::max(g->n_u, g->n_v) + 4ull * w +
           (1ull << 20);
}

void lane_main(sbc_server *s, Lane *lane) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        lane->cv.wait(lock, [&] { return lane->job != nullptr || s->stopping; });
        if (!lane->job) return;
        Job *job = lane->job;
        lock.unlock();
        // distinct graphs of the job, in first-request order
        std::vector<uint32_t> gids;
        std::unordered_map<uint32_t, size_t> slot;
        for (Request *r : job->reqs)
            if (!slot.count(r->gid)) {
                slot[r->gid] = gids.size();
                gids.push_back(r->gid);
            }
        std::vector<sbc_u128> res(gids.size(), sbc_u128{0, 0});
        sbc_status st = SBC_OK;
        std::string err;
        try {
            if (job->batched && gids.size() > 1) {
                std::vector<const sbc_graph *> gs(gids.size());
                for (size_t i = 0; i < gids.size(); i++) gs[i] = s->graphs[gids[i]];
                std::unique_ptr<sbc_batch, void (*)(sbc_batch *)> b(
                    batch_create(gs.data(), gs.size(), job->p, job->q, false, nullptr, lane->stream),
                    batch_destroy);
                const sbc_u128 *first = batch_first(b.get());
                for (size_t i = 0; i < gids.size(); i++) res[i] = first[i];
            } else {
                for (size_t i = 0; i < gids.size(); i++) {
                    sbc_count_stats stt;
                    count_graph(s->graphs[gids[i]], job->p, job->q, nullptr, &stt, lane->stream);
                    res[i] = stt.count;
                }
            }
        } catch (const SbcError &e) {
            st = e.status;
            err = e.what();
        } catch (const std::exception &e) {
            st = SBC_E_CUDA;
            err = e.what();
        }
        const auto now = Clock::now();
        lock.lock();
        for (Request *r : job->reqs) {
            r->status = st;
            r->error = err;
            r->result = res[slot[r->gid]];
            r->done = now;
            r->state = 2;
            s->latencies_ms.push_back(1e3 * seconds_since(r->submitted, now));
            if (st == SBC_OK) s->completed++; else s->failed++;
        }
        s->last_done = now;
        s->in_flight_bytes -= job->bytes;
        s->running_jobs--;
        lane->job = nullptr;
        delete job;
        s->cv_done.notify_all();
        s->cv_sched.notify_all();
    }
}

void scheduler_main(sbc_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        s->cv_sched.wait(lock, [&] {
            if (s->stopping) return true;
            if (s->waiting.empty()) return false;
            for (Lane *l : s->lanes)
                if (!l->job) return true;
            return false;
        });
        if (s->stopping) return;
        Lane *free_lane = nullptr;
        for (Lane *l : s->lanes)
            if (!l->job) {
                free_lane = l;
                break;
            }
        if (!free_lane || s->waiting.empty()) continue;
        // next job from the oldest waiting request
        Request *head = s->waiting.front();
        const sbc_graph *hg = s->graphs[head->gid];
        const bool small = hg->nnz <= s->opts.small_edges;
        std::unique_ptr<Job> job(new Job());
        job->p = head->p;
        job->q = head->q;
        job->batched = small;
        uint64_t bytes = 0;
        std::vector<uint32_t> seen;
        for (auto it = s->waiting.begin(); it != s->waiting.end();) {
            Request *r = *it;
            const bool take_head = r == head;
            bool fit = false;
            if (take_head) {
                fit = true;
            } else if (small && (int)job->reqs.size() < s->opts.max_batch && r->p == head->p &&
                       r->q == head->q && s->graphs[r->gid]->nnz <= s->opts.small_edges) {
                fit = true;
            }
            if (fit) {
                uint64_t add = 0;
                if (std::find(seen.begin(), seen.end(), r->gid) == seen.end()) {
                    add = s->footprint[r->gid];
                    if (!take_head && bytes + add + s->in_flight_bytes > s->opts.mem_budget_bytes) {
                        ++it;
                        continue;
                    }
                    seen.push_back(r->gid);
                }
                bytes += add;
                job->reqs.push_back(r);
                it = s->waiting.erase(it);
            } else {
                ++it;
            }
        }
        // admission: the job must fit the budget next to the jobs in flight
        // (a job larger than the budget runs only when nothing else does)
        if (s->in_flight_bytes > 0 && s->in_flight_bytes + bytes > s->opts.mem_budget_bytes) {
            for (auto rit = job->reqs.rbegin(); rit != job->reqs.rend(); ++rit)
                s->waiting.push_front(*rit);
            // wait for a completion before trying again
            s->cv_sched.wait(lock, [&] { return s->stopping || s->running_jobs == 0 ||
                                                s->in_flight_bytes + bytes <= s->opts.mem_budget_bytes; });
            continue;
        }
        for (Request *r : job->reqs) r->state = 1;
        job->bytes = bytes;
        s->in_flight_bytes += bytes;
        s->peak_bytes = std::max(s->peak_bytes, s->in_flight_bytes);
        s->running_jobs++;
        s->jobs++;
        if (job->reqs.size() > 1) s->fused += job->reqs.size();
        free_lane->job = job.release();
        free_lane->cv.notify_one();
    }
}

}  // namespace

}  // namespace sbc

using namespace sbc;

#define SBC_SRV_TRY try {
#define SBC_SRV_END                           \
    }                                         \
    catch (const SbcError &e) {               \
        set_last_error(e.what());             \
        return e.status;                      \
    }                                         \
    catch (const std::exception &e) {         \
        set_last_error(e.what());             \
        return SBC_E_CUDA;                    \
    }                                         \
    return SBC_OK;

extern "C" {

sbc_status sbc_server_create(const sbc_server_opts *opts, sbc_server **out) {
    SBC_SRV_TRY
    if (!out) fail(SBC_E_INVAL, "out is NULL");
    *out = nullptr;
    std::unique_ptr<sbc_server> s(new sbc_server());
    SBC_CUDA(cudaGetDevice(&s->device));
    sbc_server_opts o{};
    if (opts) o = *opts;
    if (o.lanes <= 0) o.lanes = 4;
    if (o.lanes > 64) fail(SBC_E_INVAL, "at most 64 lanes");
    if (o.max_batch <= 0) o.max_batch = 64;
    if (o.small_edges <= 0) o.small_edges = 200000;
    if (o.mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        SBC_CUDA(cudaMemGetInfo(&fr, &tot));
        o.mem_budget_bytes = (uint64_t)(fr * 0.8);
    }
    s->opts = o;
    for (int i = 0; i < o.lanes; i++) {
        Lane *l = new Lane();
        s->lanes.push_back(l);
        SBC_CUDA(cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking));
    }
    sbc_server *raw = s.get();
    for (Lane *l : s->lanes) l->thread = std::thread(lane_main, raw, l);
    s->scheduler = std::thread(scheduler_main, raw);
    *out = s.release();
    SBC_SRV_END
}

sbc_status sbc_server_add_graph(sbc_server *s, const sbc_graph *g, uint32_t *gid) {
    SBC_SRV_TRY
    if (!s || !g || !gid) fail(SBC_E_INVAL, "NULL argument");
    if (g->device != s->device) fail(SBC_E_INVAL, "graph and server are on different devices");
    std::lock_guard<std::mutex> lock(s->mu);
    *gid = (uint32_t)s->graphs.size();
    s->graphs.push_back(g);
    s->footprint.push_back(estimate_bytes(g));
    SBC_SRV_END
}

sbc_status sbc_server_submit(sbc_server *s, uint32_t gid, int p, int q, uint64_t *ticket) {
    SBC_SRV_TRY
    if (!s || !ticket) fail(SBC_E_INVAL, "NULL argument");
    if (p < 2 || q < 2 || p > 8 || q > 8) fail(SBC_E_INVAL, "p and q must be in [2, 8]");
    std::lock_guard<std::mutex> lock(s->mu);
    if (gid >= s->graphs.size()) fail(SBC_E_INVAL, "unknown graph id %u", gid);
    if (s->stopping) fail(SBC_E_BUSY, "server is shutting down");
    Request *r = new Request();
    r->ticket = s->next_ticket++;
    r->gid = gid;
    r->p = p;
    r->q = q;
    r->submitted = Clock::now();
    if (!s->any_submit) {
        s->first_submit = r->submitted;
        s->any_submit = true;
    }
    s->submitted++;
    s->requests[r->ticket] = r;
    s->waiting.push_back(r);
    *ticket = r->ticket;
    s->cv_sched.notify_all();
    SBC_SRV_END
}

sbc_status sbc_server_wait(sbc_server *s, uint64_t ticket, int64_t timeout_us, sbc_u128 *out,
                           double *latency_s) {
    SBC_SRV_TRY
    if (!s) fail(SBC_E_INVAL, "server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) fail(SBC_E_INVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    auto ready = [&] { return r->state == 2; };
    if (timeout_us < 0) {
        s->cv_done.wait(lock, ready);
    } else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready)) {
        fail(SBC_E_TIMEOUT, "request %llu not finished within %lld us", (unsigned long long)ticket,
             (long long)timeout_us);
    }
    const sbc_status st = r->status;
    const std::string err = r->error;
    if (out) *out = r->result;
    if (latency_s) *latency_s = seconds_since(r->submitted, r->done);
    s->requests.erase(it);
    delete r;
    if (st != SBC_OK) fail(st, "%s", err.c_str());
    SBC_SRV_END
}

sbc_status sbc_server_stats(sbc_server *s, sbc_server_stats_t *out) {
    SBC_SRV_TRY
    if (!s || !out) fail(SBC_E_INVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->jobs = s->jobs;
    out->fused_requests = s->fused;
    out->peak_admitted_bytes = s->peak_bytes;
    out->mem_budget_bytes = s->opts.mem_budget_bytes;
    std::vector<double> v = s->latencies_ms;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double f) {
            size_t k = (size_t)std::ceil(f * v.size());
            if (k == 0) k = 1;
            return v[std::min(k, v.size()) - 1];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
        const double span = seconds_since(s->first_submit, s->last_done);
        out->throughput_rps = span > 0 ? (double)v.size() / span : 0;
    }
    SBC_SRV_END
}

sbc_status sbc_server_reset_stats(sbc_server *s) {
    SBC_SRV_TRY
    if (!s) fail(SBC_E_INVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    s->latencies_ms.clear();
    s->submitted = s->completed = s->failed = s->jobs = s->fused = 0;
    s->peak_bytes = s->in_flight_bytes;
    s->any_submit = false;
    SBC_SRV_END
}

sbc_status sbc_server_destroy(sbc_server *s) {
    SBC_SRV_TRY
    if (!s) return SBC_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
        for (Lane *l : s->lanes) l->cv.notify_all();
        s->cv_sched.notify_all();
    }
    if (s->scheduler.joinable()) s->scheduler.join();
    for (Lane *l : s->lanes) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            l->cv.notify_all();
        }
        if (l->thread.joinable()) l->thread.join();
        if (l->stream) cudaStreamDestroy(l->stream);
        delete l;
    }
    for (auto &kv : s->requests) delete kv.second;  // every request is in the map
    delete s;
    SBC_SRV_END
}

}  // extern "C"
