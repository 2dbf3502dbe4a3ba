// server.cpp -- continuous-batching request server over one resident index.
//
// Requests (a block of queries with one radius each) are queued by any thread; the
// submitting thread copies the queries into pinned host memory from a pool, so the
// scheduler never touches query data on the host.  A scheduler thread keeps up to
// `slots` device batches in flight, each on its own query context and stream: whenever
// a slot is free it packs the requests at the head of the queue into one batch
// (per-query radii, so requests of different radius share a launch), admits the batch
// only if the device has the memory the batch would add, and enqueues the copies in,
// the whole batch (fclsh_query_async) and the copies of its result offsets and
// counters back into a pinned result block.  When those arrive the ids follow, sized
// by the result total; when they arrive the batch's requests are marked done and hold
// a reference to the block with their offset into it.  A waiting thread builds its
// own result from the block outside the server's lock, and the block returns to the
// pool when the last request of its batch has been collected.  Finished slots are
// retired as soon as their copies land (a host callback on the slot's stream wakes
// the scheduler), so requests that arrive while others run are admitted as slots and
// memory free up, and batches on different slots overlap on the device.  Each query's
// answer is the same alone or in a batch: the kernels treat queries independently.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// Pinned host buffers by power-of-two size class, reused across requests and batches.
class PinnedPool {
  public:
    ~PinnedPool()
    {
        for (auto &kv : free_)
            for (void *p : kv.second) cudaFreeHost(p);
    }
    // A buffer of at least `bytes` (its class size in *cls); nullptr if pinned memory ran out.
    void *get(size_t bytes, size_t *cls)
    {
        size_t c = 256;
        while (c < bytes) c <<= 1;
        *cls = c;
        {
            std::lock_guard<std::mutex> g(mu_);
            auto &v = free_[c];
            if (!v.empty()) {
                void *p = v.back();
                v.pop_back();
                return p;
            }
        }
        void *p = nullptr;
        if (cudaHostAlloc(&p, c, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void put(void *p, size_t cls)
    {
        if (!p) return;
        std::lock_guard<std::mutex> g(mu_);
        free_[cls].push_back(p);
    }

  private:
    std::mutex mu_;
    std::map<size_t, std::vector<void *>> free_;
};

// One batch's results on the host (pinned, from the pool): offsets [nq+1], counters [nq]
// each, the hit count, and the ids.
struct ResultBlock {
    PinnedPool *pool = nullptr;
    uint64_t *head = nullptr;   // offs [nq+1] | coll [nq] | cand [nq] | hits [1]
    size_t head_cls = 0;
    uint32_t *ids = nullptr;
    size_t ids_cls = 0;
    uint64_t nq = 0, total = 0;
    uint64_t *offs() const { return head; }
    uint64_t *coll() const { return head + nq + 1; }
    uint64_t *cand() const { return head + 2 * nq + 1; }
    unsigned long long *hits() const { return reinterpret_cast<unsigned long long *>(head + 3 * nq + 1); }
    ~ResultBlock()
    {
        if (pool) {
            pool->put(head, head_cls);
            pool->put(ids, ids_cls);
        }
    }
};

struct Request {
    uint64_t ticket = 0;
    uint64_t *h_q = nullptr;   // pinned copy of the queries (from the pool)
    size_t h_q_cls = 0;
    uint64_t nq = 0;
    uint32_t radius = 0;
    Clock::time_point t_submit, t_done;
    std::shared_ptr<ResultBlock> block;   // the batch's results, shared by its requests
    uint64_t q0 = 0;                      // this request's first query in the batch
    bool done = false;
    fclsh_status status = FCLSH_OK;
    std::string error;
};

enum SlotState { IDLE = 0, RUNNING = 1, DRAINING = 2 };

struct Slot {
    fclsh_qctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;    // the copies of the current stage have landed
    uint64_t *d_q = nullptr;
    uint32_t *d_r = nullptr, *h_r = nullptr;
    uint64_t cap_q = 0;          // queries d_q / d_r / h_r hold
    std::vector<std::shared_ptr<Request>> reqs;
    std::shared_ptr<ResultBlock> block;
    uint64_t nq = 0;
    SlotState state = IDLE;
};

}  // namespace

struct fclsh_server {
    fclsh_index *idx = nullptr;
    fclsh_server_opts opts{};
    PinnedPool pool;
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

fclsh_status fail(fclsh_status st, const char *msg)
{
    fclsh::set_error("%s", msg);
    return st;
}

void CUDART_CB wake_scheduler(void *p) { static_cast<fclsh_server *>(p)->cv_work.notify_one(); }

void release_queries(fclsh_server *srv, Request &rq)
{
    srv->pool.put(rq.h_q, rq.h_q_cls);
    rq.h_q = nullptr;
}

// Device and pinned buffers of a slot for nq queries (at creation; again only for a single
// request larger than max_batch_queries).
fclsh_status slot_reserve(fclsh_server *srv, Slot &sl, uint64_t nq)
{
    if (nq <= sl.cap_q) return FCLSH_OK;
    const uint32_t words = srv->idx->words;
    fclsh::dev_free(sl.d_q);
    fclsh::dev_free(sl.d_r);
    if (sl.h_r) cudaFreeHost(sl.h_r);
    sl.d_q = nullptr;
    sl.d_r = sl.h_r = nullptr;
    sl.cap_q = 0;
    FCLSH_CUDA(fclsh::dev_alloc((void **)&sl.d_q, nq * words * 8));
    FCLSH_CUDA(fclsh::dev_alloc((void **)&sl.d_r, nq * 4));
    FCLSH_CUDA(cudaHostAlloc((void **)&sl.h_r, nq * 4, cudaHostAllocPortable));
    sl.cap_q = nq;
    return FCLSH_OK;
}

// Mark the slot's requests done (sharing its result block) or failed, and free the slot.
void finish_requests(fclsh_server *srv, Slot &sl, fclsh_status st, const char *err)
{
    const auto now = Clock::now();
    for (auto &rq : sl.reqs) release_queries(srv, *rq);
    {
        std::lock_guard<std::mutex> g(srv->mu);
        uint64_t q0 = 0;
        for (auto &rq : sl.reqs) {
            rq->status = st;
            if (st == FCLSH_OK) {
                rq->block = sl.block;
                rq->q0 = q0;
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
    }
    sl.reqs.clear();
    sl.block.reset();
    sl.state = IDLE;
    srv->cv_done.notify_all();
}

// Stage 1: the queries in, the batch, and its result offsets and counters back.
fclsh_status launch(fclsh_server *srv, Slot &sl)
{
    const uint32_t words = srv->idx->words;
    fclsh_status st = slot_reserve(srv, sl, sl.nq);
    if (st != FCLSH_OK) return st;
    uint64_t at = 0;
    uint32_t rmax = 0;
    for (auto &rq : sl.reqs) {
        FCLSH_CUDA(cudaMemcpyAsync(sl.d_q + at * words, rq->h_q, rq->nq * words * 8, cudaMemcpyHostToDevice, sl.stream));
        for (uint64_t i = 0; i < rq->nq; ++i) sl.h_r[at + i] = rq->radius;
        rmax = std::max(rmax, rq->radius);
        at += rq->nq;
    }
    FCLSH_CUDA(cudaMemcpyAsync(sl.d_r, sl.h_r, sl.nq * 4, cudaMemcpyHostToDevice, sl.stream));
    st = fclsh_query_async(sl.ctx, sl.d_q, sl.nq, rmax, sl.d_r, sl.stream);
    if (st != FCLSH_OK) return st;
    auto blk = std::make_shared<ResultBlock>();
    blk->pool = &srv->pool;
    blk->nq = sl.nq;
    blk->head = static_cast<uint64_t *>(srv->pool.get((3 * sl.nq + 2) * 8, &blk->head_cls));
    if (!blk->head) return fail(FCLSH_ENOMEM, "pinned host memory for results");
    const uint64_t *offs, *coll, *cand;
    const uint32_t *ids;
    const unsigned long long *hits;
    uint64_t cap = 0;
    fclsh::qctx_result_ptrs(sl.ctx, &offs, &ids, &coll, &cand, &hits, &cap);
    FCLSH_CUDA(cudaMemcpyAsync(blk->offs(), offs, (sl.nq + 1) * 8, cudaMemcpyDeviceToHost, sl.stream));
    FCLSH_CUDA(cudaMemcpyAsync(blk->coll(), coll, sl.nq * 8, cudaMemcpyDeviceToHost, sl.stream));
    FCLSH_CUDA(cudaMemcpyAsync(blk->cand(), cand, sl.nq * 8, cudaMemcpyDeviceToHost, sl.stream));
    FCLSH_CUDA(cudaMemcpyAsync(blk->hits(), hits, 8, cudaMemcpyDeviceToHost, sl.stream));
    FCLSH_CUDA(cudaEventRecord(sl.ev, sl.stream));
    FCLSH_CUDA(cudaLaunchHostFunc(sl.stream, wake_scheduler, srv));
    sl.block = std::move(blk);
    sl.state = RUNNING;
    return FCLSH_OK;
}

// Stage 2: with the total known, the ids back.  A batch whose hits passed the context's
// result buffer is completed by fclsh_qctx_wait first (it reruns the overflowed queries).
fclsh_status fetch_ids(fclsh_server *srv, Slot &sl)
{
    ResultBlock &b = *sl.block;
    const uint64_t *offs, *coll, *cand;
    const uint32_t *ids;
    const unsigned long long *hits;
    uint64_t cap = 0;
    fclsh::qctx_result_ptrs(sl.ctx, &offs, &ids, &coll, &cand, &hits, &cap);
    if (*b.hits() > cap) {
        fclsh_status st = fclsh_qctx_wait(sl.ctx, nullptr);
        if (st != FCLSH_OK) return st;
        fclsh::qctx_result_ptrs(sl.ctx, &offs, &ids, &coll, &cand, &hits, &cap);
        FCLSH_CUDA(cudaMemcpy(b.offs(), offs, (b.nq + 1) * 8, cudaMemcpyDeviceToHost));
        FCLSH_CUDA(cudaMemcpy(b.coll(), coll, b.nq * 8, cudaMemcpyDeviceToHost));
        FCLSH_CUDA(cudaMemcpy(b.cand(), cand, b.nq * 8, cudaMemcpyDeviceToHost));
    }
    b.total = b.offs()[b.nq];
    b.ids = static_cast<uint32_t *>(srv->pool.get(std::max<uint64_t>(b.total, 1) * 4, &b.ids_cls));
    if (!b.ids) return fail(FCLSH_ENOMEM, "pinned host memory for result ids");
    if (b.total) FCLSH_CUDA(cudaMemcpyAsync(b.ids, ids, b.total * 4, cudaMemcpyDeviceToHost, sl.stream));
    FCLSH_CUDA(cudaEventRecord(sl.ev, sl.stream));
    FCLSH_CUDA(cudaLaunchHostFunc(sl.stream, wake_scheduler, srv));
    sl.state = DRAINING;
    return FCLSH_OK;
}

void worker_main(fclsh_server *srv)
{
    cudaSetDevice(srv->idx->device);
    for (;;) {
        bool did = false;
        // advance slots whose copies have landed
        for (auto &sl : srv->slots) {
            if (sl.state == IDLE) continue;
            cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            did = true;
            if (q != cudaSuccess) {
                cudaGetLastError();
                finish_requests(srv, sl, FCLSH_ECUDA, cudaGetErrorString(q));
                continue;
            }
            if (sl.state == RUNNING) {
                const fclsh_status st = fetch_ids(srv, sl);
                if (st != FCLSH_OK) finish_requests(srv, sl, st, fclsh_last_error());
            } else {
                finish_requests(srv, sl, FCLSH_OK, nullptr);
            }
        }
        // admit queued requests into free slots
        for (auto &sl : srv->slots) {
            if (sl.state != IDLE) continue;
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
            // admission by free device memory: what the batch would add to the slot's context
            // and buffers must leave opts.mem_reserve free (an idle server admits regardless)
            bool any_busy = false;
            for (auto &o : srv->slots) any_busy |= o.state != IDLE;
            if (any_busy) {
                size_t free_b = 0, total_b = 0;
                cudaMemGetInfo(&free_b, &total_b);
                uint64_t need = fclsh::qctx_grow_bytes(sl.ctx, nq);
                if (nq > sl.cap_q) need += nq * ((uint64_t)srv->idx->words * 8 + 4);
                if (free_b < need + srv->opts.mem_reserve) {
                    for (auto it = batch.rbegin(); it != batch.rend(); ++it) srv->pending.push_front(*it);
                    srv->deferred_for_memory++;
                    break;
                }
            }
            srv->batches++;
            srv->batch_queries += nq;
            lk.unlock();
            sl.reqs = std::move(batch);
            sl.nq = nq;
            const fclsh_status st = launch(srv, sl);
            if (st != FCLSH_OK) finish_requests(srv, sl, st, fclsh_last_error());
            did = true;
        }
        std::unique_lock<std::mutex> lk(srv->mu);
        bool busy = false;
        for (auto &sl : srv->slots) busy |= sl.state != IDLE;
        if (srv->stop && srv->pending.empty() && !busy) return;
        if (!did) {
            if (busy)   // woken by the slots' stream callbacks; the timeout only bounds a missed wake-up
                srv->cv_work.wait_for(lk, std::chrono::microseconds(200));
            else
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(5),
                                      [&] { return srv->stop || !srv->pending.empty(); });
        }
    }
}

void free_slot(Slot &sl)
{
    if (sl.ctx) fclsh_qctx_free(sl.ctx);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ev) cudaEventDestroy(sl.ev);
    fclsh::dev_free(sl.d_q);
    fclsh::dev_free(sl.d_r);
    if (sl.h_r) cudaFreeHost(sl.h_r);
    sl = Slot{};
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
    fclsh_status st = FCLSH_OK;
    for (auto &sl : srv->slots) {
        st = fclsh_qctx_create(idx, &sl.ctx);
        if (st == FCLSH_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
            st = fail(FCLSH_ECUDA, "cudaStreamCreate failed");
        if (st == FCLSH_OK && cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess)
            st = fail(FCLSH_ECUDA, "cudaEventCreate failed");
        if (st == FCLSH_OK) st = slot_reserve(srv.get(), sl, srv->opts.max_batch_queries);
        if (st != FCLSH_OK) break;
    }
    if (st != FCLSH_OK) {
        for (auto &sl : srv->slots) free_slot(sl);
        return st;
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
    rq->nq = nq;
    rq->radius = radius;
    if (nq) {   // staged into pinned memory here, by the submitting thread
        const size_t bytes = nq * srv->idx->words * 8;
        rq->h_q = static_cast<uint64_t *>(srv->pool.get(bytes, &rq->h_q_cls));
        if (!rq->h_q) return fail(FCLSH_ENOMEM, "pinned host memory for the request's queries");
        memcpy(rq->h_q, queries, bytes);
    }
    {
        std::lock_guard<std::mutex> g(srv->mu);
        rq->ticket = srv->next_ticket++;
        rq->t_submit = Clock::now();
        if (srv->done_requests == 0 && srv->live.empty()) srv->t_first = rq->t_submit;
        if (nq == 0) {
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
    // the result is built here, by the waiting thread, from the batch's pinned block
    if (rq->status != FCLSH_OK) return fail(rq->status, rq->error.c_str());
    const uint64_t nq = rq->nq;
    const ResultBlock *b = rq->block.get();
    const uint64_t base = b ? b->offs()[rq->q0] : 0, end = b ? b->offs()[rq->q0 + nq] : 0;
    fclsh_result *r = (fclsh_result *)calloc(1, sizeof(fclsh_result));
    if (!r) return fail(FCLSH_ENOMEM, "host allocation failed");
    r->nq = nq;
    r->offs = (uint64_t *)malloc((nq + 1) * 8);
    r->ids = (uint32_t *)malloc(std::max<uint64_t>(end - base, 1) * 4);
    r->collisions = (uint64_t *)malloc(std::max<uint64_t>(nq, 1) * 8);
    r->candidates = (uint64_t *)malloc(std::max<uint64_t>(nq, 1) * 8);
    if (!r->offs || !r->ids || !r->collisions || !r->candidates) {
        fclsh_result_free(r);
        return fail(FCLSH_ENOMEM, "host allocation failed");
    }
    r->offs[0] = 0;
    if (b) {
        for (uint64_t i = 0; i <= nq; ++i) r->offs[i] = b->offs()[rq->q0 + i] - base;
        if (end > base) memcpy(r->ids, b->ids + base, (end - base) * 4);
        memcpy(r->collisions, b->coll() + rq->q0, nq * 8);
        memcpy(r->candidates, b->cand() + rq->q0, nq * 8);
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count();
    rq->block.reset();   // the block returns to the pool with its batch's last request
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
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        free_slot(sl);
    }
    for (auto &kv : srv->live) release_queries(srv, *kv.second);
    delete srv;
}
