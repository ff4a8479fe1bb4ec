// serve.cu -- continuous-batching request server over one graph.
//
// Clients submit insert and query requests from any thread; one worker
// thread owns the graph and turns the queue into device steps:
//
//   form step t   take waiting requests in submission order while their
//                 points fit max_step_points (and, for inserts, the graph's
//                 capacity); pack them (queries first) into the pinned host
//                 staging of slot t % 2
//   launch t      host->device copy on the upload stream; the compute stream
//                 waits for it, queries the graph (per-query restart streams)
//                 and inserts the step's points; results go back on the
//                 download stream once the compute stream has them
//   finish t-1    wait for step t-1's download, hand its results to the
//                 waiting clients
//
// so step t's kernels overlap the upload of t+1 and the download of t-1.
// The queries of a step run before its inserts on one stream: every search
// of a step sees the graph of the previous step (its epoch), and a step's
// inserts become visible to the next step only.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "knn_graph.h"

using namespace knn;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t REQ_MAX_POINTS = 1 << 20;  // query ids: request * 2^20 + point

struct Request {
    uint64_t id = 0;
    int32_t kind = KNN_REQ_QUERY;
    int64_t m = 0;
    std::vector<float> vecs;       // [m][dim], owned until the step is packed
    std::vector<int64_t> ids;      // query: [m][k_out]; insert: [m]
    std::vector<float> sims;       // query: [m][k_out]
    knn_request_info info{};
    Clock::time_point t_submit, t_admit;
    bool done = false;
};

struct Slot {
    // pinned host staging
    float *h_vecs = nullptr;       // [P][dim]
    uint64_t *h_qids = nullptr;    // [P]
    int64_t *h_ids = nullptr;      // [P][k_out]  (query results, then insert ids)
    float *h_sims = nullptr;       // [P][k_out]
    // device
    float *d_vecs = nullptr;
    uint64_t *d_qids = nullptr;
    int64_t *d_qids_out = nullptr;  // [P][k_out]
    float *d_sims = nullptr;        // [P][k_out]
    int64_t *d_new = nullptr;       // [P]
    cudaEvent_t uploaded = nullptr, computed = nullptr, downloaded = nullptr, t0 = nullptr, t1 = nullptr;
    // the step in the slot
    std::vector<Request *> reqs;
    int64_t mq = 0, mi = 0, step = -1, epoch = 0;
    bool busy = false;
    knn_status st = KNN_OK;
};

}  // namespace

struct knn_server {
    knn_graph *g = nullptr;
    GraphShape shape{};
    int k_out = 0;
    int64_t P = 0;  // points per step
    int device = 0;
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    Slot slots[2];

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_id = 0;
    bool stopping = false;
    int64_t pending_inserts = 0;  // insert points admitted into the step being formed
    int64_t headroom = 0;         // bytes that must stay free when the graph grows (0: no growth)
    std::vector<int64_t> parts;   // query partitions at creation (empty: plain search)
    bool grow_failed = false;     // the last growth for the insert at the queue head failed
    knn_server_stats stats{};
    std::thread worker;

    void run();
    void finish(Slot &sl);
};

static knn_status server_fail(knn_status st, const char *msg) { return record_error(st, msg); }

void knn_server::finish(Slot &sl) {
    if (!sl.busy) return;
    cudaError_t e = cudaEventSynchronize(sl.downloaded);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, sl.t0, sl.t1);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    stats.busy_ms += ms;
    int64_t qoff = 0, ioff = 0;
    for (Request *r : sl.reqs) {
        r->info.status = sl.st != KNN_OK ? sl.st : (e == cudaSuccess ? KNN_OK : KNN_ERR_CUDA);
        r->info.epoch = sl.epoch;
        r->info.step = sl.step;
        r->info.queue_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
        r->info.latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
        if (r->kind == KNN_REQ_QUERY) {
            r->ids.assign(sl.h_ids + qoff * k_out, sl.h_ids + (qoff + r->m) * k_out);
            r->sims.assign(sl.h_sims + qoff * k_out, sl.h_sims + (qoff + r->m) * k_out);
            qoff += r->m;
        } else {
            const int64_t *base = sl.h_ids + sl.mq * k_out;  // insert ids follow the query results
            r->ids.assign(base + ioff, base + ioff + r->m);
            ioff += r->m;
        }
        r->done = true;
    }
    sl.reqs.clear();
    sl.busy = false;
    cv_done.notify_all();
}

void knn_server::run() {
    cudaSetDevice(device);
    int64_t step = 0, epoch = 0;
    for (;;) {
        Slot &sl = slots[step & 1];
        finish(sl);  // the slot's previous step (t - 2) is done before it is reused
        int64_t grow_to = 0;  // capacity an insert at the queue head needs
        {
            std::unique_lock<std::mutex> lk(mu);
            Slot &other = slots[(step + 1) & 1];
            while (queue.empty() && !stopping) {
                if (other.busy) break;  // finish step t-1 while waiting
                cv_work.wait(lk);
            }
            if (queue.empty()) {
                if (other.busy) {
                    lk.unlock();
                    finish(other);
                    continue;
                }
                if (stopping) break;
                continue;
            }
            // admission: submission order, while the points fit the slot and
            // the inserts fit the graph (or, with a headroom set, the graph
            // can be grown within free device memory)
            int64_t pts = 0;
            const auto now = Clock::now();
            while (!queue.empty()) {
                Request *r = queue.front();
                if (pts + r->m > P) break;
                if (r->kind == KNN_REQ_INSERT && shape.n + pending_inserts + r->m > shape.capacity) {
                    if (!sl.reqs.empty()) break;  // try again once this step has committed
                    if (headroom > 0 && !grow_failed) {
                        grow_to = shape.n + r->m;
                        break;  // grow outside the lock, then admit again
                    }
                    // can never fit: fail it
                    queue.pop_front();
                    r->info.status = headroom > 0 ? KNN_ERR_OOM : KNN_ERR_CAPACITY;
                    r->t_admit = now;
                    r->info.latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
                    r->done = true;
                    grow_failed = false;
                    cv_done.notify_all();
                    continue;
                }
                queue.pop_front();
                r->t_admit = now;
                sl.reqs.push_back(r);
                pts += r->m;
                if (r->kind == KNN_REQ_INSERT) pending_inserts += r->m;
            }
            if (sl.reqs.empty() && grow_to == 0) continue;
        }
        if (grow_to > 0) {
            // nothing may be in flight while the graph's arrays move; grow by
            // half the capacity, else just to what the insert needs
            finish(slots[0]);
            finish(slots[1]);
            const int64_t big = std::min<int64_t>(std::max<int64_t>(grow_to, shape.capacity + shape.capacity / 2),
                                                  (int64_t)INT32_MAX - 1);
            knn_status st = knn_graph_reserve(g, big, headroom, comp);
            if (st != KNN_OK && big > grow_to) st = knn_graph_reserve(g, grow_to, headroom, comp);
            std::lock_guard<std::mutex> lk(mu);
            if (st == KNN_OK) {
                shape = graph_shape(g);
                stats.grows += 1;
                stats.capacity = shape.capacity;
            } else {
                grow_failed = true;  // the insert at the head fails at the next admission
            }
            continue;
        }
        // pack: queries first, then inserts
        const int d = shape.dim;
        sl.mq = sl.mi = 0;
        for (Request *r : sl.reqs)
            if (r->kind == KNN_REQ_QUERY) {
                std::memcpy(sl.h_vecs + sl.mq * d, r->vecs.data(), (size_t)r->m * d * 4);
                for (int64_t i = 0; i < r->m; ++i) sl.h_qids[sl.mq + i] = (r->id << 20) + (uint64_t)i;
                sl.mq += r->m;
            }
        for (Request *r : sl.reqs)
            if (r->kind == KNN_REQ_INSERT) {
                std::memcpy(sl.h_vecs + (sl.mq + sl.mi) * d, r->vecs.data(), (size_t)r->m * d * 4);
                sl.mi += r->m;
            }
        for (Request *r : sl.reqs) std::vector<float>().swap(r->vecs);
        const int64_t m = sl.mq + sl.mi;
        sl.step = step;
        sl.epoch = epoch;
        sl.st = KNN_OK;
        sl.busy = true;
        auto launch = [&]() -> knn_status {
            if (cudaMemcpyAsync(sl.d_vecs, sl.h_vecs, (size_t)m * d * 4, cudaMemcpyHostToDevice, up) != cudaSuccess ||
                cudaMemcpyAsync(sl.d_qids, sl.h_qids, (size_t)sl.mq * 8, cudaMemcpyHostToDevice, up) != cudaSuccess ||
                cudaEventRecord(sl.uploaded, up) != cudaSuccess || cudaStreamWaitEvent(comp, sl.uploaded, 0) != cudaSuccess)
                return server_fail(KNN_ERR_CUDA, "server upload failed");
            cudaEventRecord(sl.t0, comp);
            if (sl.mq > 0) {
                knn_status st;
                if (parts.empty()) {
                    st = knn_graph_query_ids(g, sl.d_vecs, sl.mq, k_out, sl.d_qids, sl.d_qids_out, sl.d_sims, comp);
                } else {
                    // the parts at creation, the last one stretched over the
                    // nodes inserted since (the graph of this step's epoch)
                    std::vector<int64_t> off(parts);
                    off.back() = shape.n;
                    st = knn_graph_query_partitioned_ids(g, sl.d_vecs, sl.mq, k_out, sl.d_qids, off.data(),
                                                         (int32_t)off.size() - 1, sl.d_qids_out, sl.d_sims, comp);
                }
                if (st != KNN_OK) return st;
            }
            if (sl.mi > 0) {
                const knn_status st = knn_graph_insert_batch(g, sl.d_vecs + sl.mq * d, sl.mi, sl.d_new, nullptr, comp);
                if (st != KNN_OK) return st;
            }
            cudaEventRecord(sl.t1, comp);
            if (cudaEventRecord(sl.computed, comp) != cudaSuccess || cudaStreamWaitEvent(down, sl.computed, 0) != cudaSuccess ||
                cudaMemcpyAsync(sl.h_ids, sl.d_qids_out, (size_t)sl.mq * k_out * 8, cudaMemcpyDeviceToHost, down) != cudaSuccess ||
                cudaMemcpyAsync(sl.h_sims, sl.d_sims, (size_t)sl.mq * k_out * 4, cudaMemcpyDeviceToHost, down) != cudaSuccess ||
                cudaMemcpyAsync(sl.h_ids + sl.mq * k_out, sl.d_new, (size_t)sl.mi * 8, cudaMemcpyDeviceToHost, down) != cudaSuccess)
                return server_fail(KNN_ERR_CUDA, "server download failed");
            return KNN_OK;
        };
        sl.st = launch();
        cudaEventRecord(sl.downloaded, down);
        {
            std::lock_guard<std::mutex> lk(mu);
            stats.steps += 1;
            stats.points += m;
            stats.queries += sl.mq;
            stats.inserts += sl.mi;
            stats.requests += (int64_t)sl.reqs.size();
            pending_inserts -= sl.mi;  // committed (or failed): the graph's n now counts them
            if (sl.mi > 0 && sl.st == KNN_OK) {
                shape.n += sl.mi;
                epoch += 1;
                stats.epoch = epoch;
            }
        }
        ++step;
        // finish the step before this one while this one runs
        finish(slots[step & 1]);
    }
    finish(slots[0]);
    finish(slots[1]);
}

extern "C" {

KNN_API knn_status knn_server_create(knn_graph *g, const knn_server_params *p, knn_server **out) {
    if (!g || !p || !out) return server_fail(KNN_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    const GraphShape sh = graph_shape(g);
    if (p->k_out < 1 || p->k_out > sh.k) return server_fail(KNN_ERR_INVALID_ARG, "k_out outside 1..k");
    const int64_t P = p->max_step_points == 0 ? sh.max_batch : p->max_step_points;
    if (P < 1 || P > sh.max_batch) return server_fail(KNN_ERR_INVALID_ARG, "max_step_points outside 1..max_batch");
    std::unique_ptr<knn_server> s(new knn_server());
    s->g = g;
    s->shape = sh;
    s->k_out = p->k_out;
    s->P = P;
    if (p->grow_headroom_bytes < 0) return server_fail(KNN_ERR_INVALID_ARG, "grow_headroom_bytes must be >= 0");
    s->headroom = p->grow_headroom_bytes;
    if (p->query_parts > 1) {
        if (!p->part_offsets || p->query_parts > KNN_MAX_PARTS || p->query_parts > sh.max_batch)
            return server_fail(KNN_ERR_INVALID_ARG, "query_parts needs part_offsets and at most KNN_MAX_PARTS parts");
        s->parts.assign(p->part_offsets, p->part_offsets + p->query_parts + 1);
        if (s->parts.front() != 0 || s->parts.back() != sh.n)
            return server_fail(KNN_ERR_INVALID_ARG, "part_offsets must run from 0 to the graph's n");
        for (int q = 0; q < p->query_parts; ++q)
            if (s->parts[(size_t)q + 1] < s->parts[(size_t)q])
                return server_fail(KNN_ERR_INVALID_ARG, "part_offsets decrease");
    }
    s->stats.capacity = sh.capacity;
    if (cudaGetDevice(&s->device) != cudaSuccess) return server_fail(KNN_ERR_CUDA, "no CUDA device");
    bool ok = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->down, cudaStreamNonBlocking) == cudaSuccess;
    const size_t d = (size_t)sh.dim, K = (size_t)p->k_out;
    for (Slot &sl : s->slots) {
        if (!ok) break;
        ok = cudaMallocHost(&sl.h_vecs, (size_t)P * d * 4) == cudaSuccess &&
             cudaMallocHost(&sl.h_qids, (size_t)P * 8) == cudaSuccess &&
             cudaMallocHost(&sl.h_ids, (size_t)P * (K + 1) * 8) == cudaSuccess &&
             cudaMallocHost(&sl.h_sims, (size_t)P * K * 4) == cudaSuccess &&
             cudaMalloc(&sl.d_vecs, (size_t)P * d * 4) == cudaSuccess &&
             cudaMalloc(&sl.d_qids, (size_t)P * 8) == cudaSuccess &&
             cudaMalloc(&sl.d_qids_out, (size_t)P * K * 8) == cudaSuccess &&
             cudaMalloc(&sl.d_sims, (size_t)P * K * 4) == cudaSuccess &&
             cudaMalloc(&sl.d_new, (size_t)P * 8) == cudaSuccess;
        for (cudaEvent_t *ev : {&sl.uploaded, &sl.computed, &sl.downloaded})
            ok = ok && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) == cudaSuccess;
        for (cudaEvent_t *ev : {&sl.t0, &sl.t1}) ok = ok && cudaEventCreate(ev) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        knn_server_destroy(s.release());
        return server_fail(KNN_ERR_OOM, "server buffers could not be allocated");
    }
    s->worker = std::thread([srv = s.get()] { srv->run(); });
    *out = s.release();
    return KNN_OK;
}

KNN_API knn_status knn_server_submit(knn_server *s, int32_t kind, const float *vecs, int64_t m,
                                     uint64_t *request_id) {
    if (!s || !vecs) return server_fail(KNN_ERR_INVALID_ARG, "null argument");
    if (kind != KNN_REQ_INSERT && kind != KNN_REQ_QUERY) return server_fail(KNN_ERR_INVALID_ARG, "unknown kind");
    if (m < 1 || m > s->P || m > REQ_MAX_POINTS)
        return server_fail(KNN_ERR_INVALID_ARG, "request size outside 1..max_step_points");
    auto r = std::make_unique<Request>();
    r->kind = kind;
    r->m = m;
    r->vecs.assign(vecs, vecs + m * s->shape.dim);
    r->info.kind = kind;
    r->info.m = m;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return server_fail(KNN_ERR_INVALID_ARG, "server is stopping");
        r->id = s->next_id++;
        if (request_id) *request_id = r->id;
        s->queue.push_back(r.get());
        s->stats.max_queue = std::max<int64_t>(s->stats.max_queue, (int64_t)s->queue.size());
        s->reqs.emplace(r->id, std::move(r));
    }
    s->cv_work.notify_one();
    return KNN_OK;
}

KNN_API knn_status knn_server_wait(knn_server *s, uint64_t request_id, int64_t *out_ids, float *out_sims,
                                   knn_request_info *info) {
    if (!s) return server_fail(KNN_ERR_INVALID_ARG, "null argument");
    std::unique_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->reqs.find(request_id);
        if (it == s->reqs.end()) return server_fail(KNN_ERR_NOT_FOUND, "unknown or already taken request");
        Request *q = it->second.get();
        s->cv_done.wait(lk, [q] { return q->done; });
        r = std::move(it->second);
        s->reqs.erase(it);
    }
    if (out_ids) std::memcpy(out_ids, r->ids.data(), r->ids.size() * 8);
    if (out_sims && !r->sims.empty()) std::memcpy(out_sims, r->sims.data(), r->sims.size() * 4);
    if (info) *info = r->info;
    return r->info.status == KNN_OK ? KNN_OK : server_fail((knn_status)r->info.status, "request failed");
}

KNN_API knn_status knn_server_get_stats(knn_server *s, knn_server_stats *out) {
    if (!s || !out) return server_fail(KNN_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return KNN_OK;
}

KNN_API void knn_server_destroy(knn_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot &sl : s->slots) {
        for (void *p : {(void *)sl.h_vecs, (void *)sl.h_qids, (void *)sl.h_ids, (void *)sl.h_sims})
            if (p) cudaFreeHost(p);
        for (void *p : {(void *)sl.d_vecs, (void *)sl.d_qids, (void *)sl.d_qids_out, (void *)sl.d_sims, (void *)sl.d_new})
            if (p) cudaFree(p);
        for (cudaEvent_t ev : {sl.uploaded, sl.computed, sl.downloaded, sl.t0, sl.t1})
            if (ev) cudaEventDestroy(ev);
    }
    if (s->comp) graph_forget_stream(s->g, s->comp);
    for (cudaStream_t st : {s->up, s->comp, s->down})
        if (st) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
