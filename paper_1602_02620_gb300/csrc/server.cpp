// server.cpp -- continuous-batching request server over one resident index.
//
// Requests (a block of queries with one radius each) are queued by any thread.
// A scheduler thread keeps up to `slots` device batches in flight, each on its
// own query context and stream: whenever a slot is free it packs the requests at
// the head of the queue into one batch (per-query radii, so requests of different
// radius share a launch), admits the batch only if the device has the memory it
// needs, copies it through pinned staging, and enqueues the whole batch with
// fclsh_query_async.  Finished slots are retired as soon as their event fires, so
// requests that arrive while others run are admitted as slots and memory free up,
// and batches on different slots overlap on the device.  Each query's answer is
// the same alone or in a batch: the kernels treat queries independently.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    std::vector<uint64_t> queries;
    uint64_t nq = 0;
    uint32_t radius = 0;
    Clock::time_point t_submit, t_done;
    std::vector<uint64_t> offs, coll, cand;
    std::vector<uint32_t> ids;
    bool done = false;
    fclsh_status status = FCLSH_OK;
    std::string error;
};

struct Slot {
    fclsh_qctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    uint64_t *h_q = nullptr, *d_q = nullptr;
    uint32_t *h_r = nullptr, *d_r = nullptr;
    uint64_t cap_q = 0;   // queries the staging holds
    std::vector<std::shared_ptr<Request>> reqs;
    uint64_t nq = 0;
    bool busy = false;
};

}  // namespace

struct fclsh_server {
    fclsh_index *idx = nullptr;
    fclsh_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> live;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    // statistics
    uint64_t done_requests = 0, done_queries = 0, batches = 0, batch_queries = 0, deferred_for_memory = 0;
    std::vector<double> latencies_ms;
    Clock::time_point t_first, t_last;
};

namespace {

fclsh_status slot_reserve(fclsh_server *srv, Slot &sl, uint64_t nq)
{
    if (nq <= sl.cap_q) return FCLSH_OK;
    const uint32_t words = srv->idx->words;
    uint64_t cap = std::max<uint64_t>(nq, sl.cap_q * 2);
    if (sl.h_q) cudaFreeHost(sl.h_q);
    if (sl.h_r) cudaFreeHost(sl.h_r);
    if (sl.d_q) cudaFree(sl.d_q);
    if (sl.d_r) cudaFree(sl.d_r);
    sl.h_q = sl.d_q = nullptr;
    sl.h_r = sl.d_r = nullptr;
    sl.cap_q = 0;
    FCLSH_CUDA(cudaMallocHost(&sl.h_q, cap * words * 8));
    FCLSH_CUDA(cudaMallocHost(&sl.h_r, cap * 4));
    FCLSH_CUDA(cudaMalloc(&sl.d_q, cap * words * 8));
    FCLSH_CUDA(cudaMalloc(&sl.d_r, cap * 4));
    sl.cap_q = cap;
    return FCLSH_OK;
}

// Device memory a batch of nq queries may need beyond what its slot already holds.
uint64_t batch_bytes(const fclsh_index *idx, uint64_t nq)
{
    return nq * ((uint64_t)idx->words * 8 + 4 + 8 * 4 + 64 * 8);
}

void finish_requests(fclsh_server *srv, Slot &sl, const fclsh_result *r, fclsh_status st, const char *err)
{
    std::lock_guard<std::mutex> g(srv->mu);
    const auto now = Clock::now();
    uint64_t q0 = 0;
    for (auto &rq : sl.reqs) {
        rq->status = st;
        if (st == FCLSH_OK) {
            const uint64_t base = r->offs[q0];
            rq->offs.resize(rq->nq + 1);
            for (uint64_t i = 0; i <= rq->nq; ++i) rq->offs[i] = r->offs[q0 + i] - base;
            rq->ids.assign(r->ids + base, r->ids + r->offs[q0 + rq->nq]);
            rq->coll.assign(r->collisions + q0, r->collisions + q0 + rq->nq);
            rq->cand.assign(r->candidates + q0, r->candidates + q0 + rq->nq);
        } else {
            rq->error = err ? err : "";
        }
        q0 += rq->nq;
        rq->t_done = now;
        rq->done = true;
        srv->done_requests++;
        srv->done_queries += rq->nq;
        srv->latencies_ms.push_back(std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count());
        srv->t_last = now;
    }
    sl.reqs.clear();
    sl.busy = false;
    srv->cv_done.notify_all();
}

void retire(fclsh_server *srv, Slot &sl)
{
    fclsh_result *r = nullptr;
    fclsh_status st = fclsh_qctx_fetch(sl.ctx, &r);
    finish_requests(srv, sl, r, st, st == FCLSH_OK ? nullptr : fclsh_last_error());
    if (r) fclsh_result_free(r);
}

fclsh_status launch(fclsh_server *srv, Slot &sl)
{
    const uint32_t words = srv->idx->words;
    fclsh_status st = slot_reserve(srv, sl, sl.nq);
    if (st != FCLSH_OK) return st;
    uint64_t at = 0;
    uint32_t rmax = 0;
    for (auto &rq : sl.reqs) {
        memcpy(sl.h_q + at * words, rq->queries.data(), rq->nq * words * 8);
        for (uint64_t i = 0; i < rq->nq; ++i) sl.h_r[at + i] = rq->radius;
        rmax = std::max(rmax, rq->radius);
        at += rq->nq;
    }
    FCLSH_CUDA(cudaMemcpyAsync(sl.d_q, sl.h_q, sl.nq * words * 8, cudaMemcpyHostToDevice, sl.stream));
    FCLSH_CUDA(cudaMemcpyAsync(sl.d_r, sl.h_r, sl.nq * 4, cudaMemcpyHostToDevice, sl.stream));
    st = fclsh_query_async(sl.ctx, sl.d_q, sl.nq, rmax, sl.d_r, sl.stream);
    if (st != FCLSH_OK) return st;
    FCLSH_CUDA(cudaEventRecord(sl.done_ev, sl.stream));
    return FCLSH_OK;
}

void worker_main(fclsh_server *srv)
{
    cudaSetDevice(srv->idx->device);
    for (;;) {
        bool did = false;
        // retire finished batches
        for (auto &sl : srv->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done_ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            retire(srv, sl);
            did = true;
        }
        // admit queued requests into free slots
        for (auto &sl : srv->slots) {
            if (sl.busy) continue;
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->pending.empty()) break;
            uint64_t nq = 0;
            std::vector<std::shared_ptr<Request>> batch;
            while (!srv->pending.empty()) {
                auto &rq = srv->pending.front();
                if (!batch.empty() && nq + rq->nq > srv->opts.max_batch_queries) break;
                nq += rq->nq;
                batch.push_back(rq);
                srv->pending.pop_front();
            }
            // admission by free device memory (keep opts.mem_reserve free)
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            bool any_busy = false;
            for (auto &o : srv->slots) any_busy |= o.busy;
            if (any_busy && free_b < batch_bytes(srv->idx, nq) + srv->opts.mem_reserve) {
                for (auto it = batch.rbegin(); it != batch.rend(); ++it) srv->pending.push_front(*it);
                srv->deferred_for_memory++;
                break;
            }
            lk.unlock();
            sl.reqs = std::move(batch);
            sl.nq = nq;
            sl.busy = true;
            fclsh_status st = launch(srv, sl);
            if (st != FCLSH_OK) {
                finish_requests(srv, sl, nullptr, st, fclsh_last_error());
            } else {
                std::lock_guard<std::mutex> g(srv->mu);
                srv->batches++;
                srv->batch_queries += nq;
            }
            did = true;
        }
        std::unique_lock<std::mutex> lk(srv->mu);
        bool busy = false;
        for (auto &sl : srv->slots) busy |= sl.busy;
        if (srv->stop && srv->pending.empty() && !busy) return;
        if (!did) {
            if (busy)
                srv->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(5),
                                      [&] { return srv->stop || !srv->pending.empty(); });
        }
    }
}

fclsh_status fail(fclsh_status st, const char *msg)
{
    fclsh::set_error("%s", msg);
    return st;
}

}  // namespace

extern "C" fclsh_status fclsh_server_create(fclsh_index *idx, const fclsh_server_opts *opts, fclsh_server **out)
{
    if (!idx || !out) return fail(FCLSH_EINVAL, "NULL argument");
    *out = nullptr;
    FCLSH_CUDA(cudaSetDevice(idx->device));
    auto srv = std::make_unique<fclsh_server>();
    srv->idx = idx;
    srv->opts = fclsh_server_opts{4, 16384, 1ULL << 30};
    if (opts) {
        if (opts->slots) srv->opts.slots = opts->slots;
        if (opts->max_batch_queries) srv->opts.max_batch_queries = opts->max_batch_queries;
        srv->opts.mem_reserve = opts->mem_reserve;
    }
    if (srv->opts.slots > 64) return fail(FCLSH_EINVAL, "at most 64 slots");
    srv->slots.resize(srv->opts.slots);
    for (auto &sl : srv->slots) {
        fclsh_status st = fclsh_qctx_create(idx, &sl.ctx);
        if (st == FCLSH_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
            st = fail(FCLSH_ECUDA, "cudaStreamCreate failed");
        if (st == FCLSH_OK && cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming) != cudaSuccess)
            st = fail(FCLSH_ECUDA, "cudaEventCreate failed");
        if (st != FCLSH_OK) {
            for (auto &o : srv->slots) {
                if (o.ctx) fclsh_qctx_free(o.ctx);
                if (o.stream) cudaStreamDestroy(o.stream);
                if (o.done_ev) cudaEventDestroy(o.done_ev);
            }
            return st;
        }
    }
    srv->worker = std::thread(worker_main, srv.get());
    *out = srv.release();
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_server_submit(fclsh_server *srv, const uint64_t *queries, uint64_t nq, uint32_t radius,
                                            uint64_t *ticket)
{
    if (!srv || !ticket || (!queries && nq)) return fail(FCLSH_EINVAL, "NULL argument");
    if (radius > srv->idx->r) {
        fclsh::set_error("radius %u exceeds the build radius %u", radius, srv->idx->r);
        return FCLSH_ERADIUS;
    }
    auto rq = std::make_shared<Request>();
    rq->queries.assign(queries, queries + nq * srv->idx->words);
    rq->nq = nq;
    rq->radius = radius;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        rq->ticket = srv->next_ticket++;
        rq->t_submit = Clock::now();
        if (srv->done_requests == 0 && srv->live.empty()) srv->t_first = rq->t_submit;
        if (nq == 0) {
            rq->offs.assign(1, 0);
            rq->done = true;
            rq->t_done = rq->t_submit;
        } else {
            srv->pending.push_back(rq);
        }
        srv->live[rq->ticket] = rq;
        *ticket = rq->ticket;
    }
    srv->cv_work.notify_one();
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_server_wait(fclsh_server *srv, uint64_t ticket, int timeout_ms, fclsh_result **out,
                                          double *latency_ms)
{
    if (!srv || !out) return fail(FCLSH_EINVAL, "NULL argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->live.find(ticket);
    if (it == srv->live.end()) return fail(FCLSH_EINVAL, "unknown ticket");
    auto rq = it->second;
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0x7fffffff : timeout_ms),
                                          [&] { return rq->done; });
    if (!ok) return fail(FCLSH_ETIMEOUT, "request not finished within the timeout");
    srv->live.erase(ticket);
    lk.unlock();
    if (rq->status != FCLSH_OK) return fail(rq->status, rq->error.c_str());
    fclsh_result *r = (fclsh_result *)calloc(1, sizeof(fclsh_result));
    if (!r) return fail(FCLSH_ENOMEM, "host allocation failed");
    r->nq = rq->nq;
    r->offs = (uint64_t *)malloc((rq->nq + 1) * 8);
    r->ids = (uint32_t *)malloc(std::max<size_t>(rq->ids.size(), 1) * 4);
    r->collisions = (uint64_t *)malloc(std::max<uint64_t>(rq->nq, 1) * 8);
    r->candidates = (uint64_t *)malloc(std::max<uint64_t>(rq->nq, 1) * 8);
    if (!r->offs || !r->ids || !r->collisions || !r->candidates) {
        fclsh_result_free(r);
        return fail(FCLSH_ENOMEM, "host allocation failed");
    }
    memcpy(r->offs, rq->offs.data(), (rq->nq + 1) * 8);
    if (!rq->ids.empty()) memcpy(r->ids, rq->ids.data(), rq->ids.size() * 4);
    if (rq->nq) {
        memcpy(r->collisions, rq->coll.data(), rq->nq * 8);
        memcpy(r->candidates, rq->cand.data(), rq->nq * 8);
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count();
    *out = r;
    return FCLSH_OK;
}

extern "C" fclsh_status fclsh_server_stats(fclsh_server *srv, fclsh_serve_stats *out, int reset)
{
    if (!srv || !out) return fail(FCLSH_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(srv->mu);
    memset(out, 0, sizeof *out);
    out->requests = srv->done_requests;
    out->queries = srv->done_queries;
    out->batches = srv->batches;
    out->deferred_for_memory = srv->deferred_for_memory;
    out->mean_batch_queries = srv->batches ? (double)srv->batch_queries / srv->batches : 0.0;
    if (!srv->latencies_ms.empty()) {
        std::vector<double> v = srv->latencies_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min<size_t>(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        const double span = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
        out->queries_per_s = span > 0 ? srv->done_queries / span : 0.0;
    }
    if (reset) {
        srv->done_requests = srv->done_queries = srv->batches = srv->batch_queries = srv->deferred_for_memory = 0;
        srv->latencies_ms.clear();
        srv->t_first = Clock::now();
    }
    return FCLSH_OK;
}

extern "C" void fclsh_server_free(fclsh_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->idx->device);
    for (auto &sl : srv->slots) {
        if (sl.ctx) fclsh_qctx_free(sl.ctx);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done_ev) cudaEventDestroy(sl.done_ev);
        if (sl.h_q) cudaFreeHost(sl.h_q);
        if (sl.h_r) cudaFreeHost(sl.h_r);
        if (sl.d_q) cudaFree(sl.d_q);
        if (sl.d_r) cudaFree(sl.d_r);
    }
    delete srv;
}
