// sfc_serve.cu - a request server over the library's entry points.
//
// Requests (a cloud from host memory, optionally a set of query centres, one radius or
// kNN search) arrive at any time through server_submit.  `slots` worker threads, each
// with its own CUDA stream, take them from one FIFO queue: a request is admitted when a
// slot is free and the device memory held by admitted, unreleased requests plus its own
// estimate stays within the budget (a request larger than the whole budget runs alone).
// A worker that admits an all-points request also takes the all-points requests queued
// right behind it (up to max_batch of them, batch_points points in all) and answers them
// with one batched pass (batch_search); other requests go through octree_build +
// radius_search / knn.  So requests that arrive while others are on the device start as
// soon as a slot and memory free up, and their work overlaps on the device.  Octrees and
// results stay resident until server_release; the neighbour arithmetic is the plain
// path's in both cases, so a request's result does not depend on what ran beside it.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sfc_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// device bytes held per point while a cloud is built and searched (input copy, sorted
// points, codes and indices in both sort buffers, node tables, hit-mask records), and
// per point once only the octree stays
constexpr int64_t kBuildBytesPerPoint = 160;
constexpr int64_t kTreeBytesPerPoint = 48;
constexpr int64_t kRadiusBytesPerRow = 8 + 4 * 64;  // row pointer + 64 neighbours (estimate)

// One device pass: a single request, or several all-points requests merged.
struct Pass {
    cudaStream_t stream = nullptr;
    sfc_batch batch = nullptr;  // merged requests
    ~Pass() {
        if (batch) batch_free(batch, stream);
    }
};

struct Request {
    int64_t id = 0;
    sfc_request req{};
    Clock::time_point arrival, admitted, done;
    int64_t reserve = 0;  // bytes counted against the budget
    sfc_status status = SFC_OK;
    bool finished = false;
    int32_t batched_with = 1;
    // results of a merged pass
    std::shared_ptr<Pass> pass;
    int32_t cloud = -1;
    // results of a single pass
    sfc_octree tree = nullptr;
    sfc_csr csr{};
    int32_t* knn_idx = nullptr;
    float* knn_d2 = nullptr;
    int64_t rows = 0;
    cudaStream_t stream = nullptr;  // where its results were made (frees go there)
};

int64_t estimate(const sfc_request& r) {
    const int64_t rows = r.queries_xyz ? r.n_queries : r.n_points;
    const int64_t out = r.search == SFC_SEARCH_KNN ? rows * r.k * 8 : rows * kRadiusBytesPerRow;
    return r.n_points * kBuildBytesPerPoint + rows * 12 + out;
}

int64_t held_bytes(const Request& q) {
    const int64_t out = q.req.search == SFC_SEARCH_KNN ? q.rows * q.req.k * 8 : 8 * (q.rows + 1) + 4 * q.csr.nnz;
    return q.req.n_points * kTreeBytesPerPoint + out;
}

bool mergeable(const sfc_request& r, int64_t batch_points) {
    return r.queries_xyz == nullptr && r.n_points > 0 && r.n_points <= batch_points;
}

}  // namespace

struct sfc_server_s {
    sfc_server_opts o{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t next_id = 1;
    int64_t reserved = 0;  // bytes of admitted, unreleased requests
    int64_t admitted_count = 0;
    bool stopping = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
};

namespace {

sfc_status run_single(sfc_server_s* S, Request& q, cudaStream_t s) {
    const sfc_request& r = q.req;
    sfc_build_opts o;
    sfc_build_opts_default(&o);
    o.leaf_capacity = S->o.leaf_capacity;
    float* dpts = nullptr;
    float* dq = nullptr;
    sfc::Scratch scratch(s);  // the device copies of the points and centres, freed in stream order on return
    SFC_TRY(scratch.alloc(&dpts, 3 * r.n_points));
    if (r.n_points > 0)
        SFC_CUDA(cudaMemcpyAsync(dpts, r.points_xyz, sizeof(float) * 3 * r.n_points, cudaMemcpyHostToDevice, s));
    sfc_status st = octree_build(dpts, r.n_points, S->o.enc, &o, s, &q.tree);  // copies what it keeps
    if (st != SFC_OK) return st;
    q.rows = r.queries_xyz ? r.n_queries : r.n_points;
    if (r.queries_xyz) {
        SFC_TRY(scratch.alloc(&dq, 3 * r.n_queries));
        if (r.n_queries > 0)
            SFC_CUDA(cudaMemcpyAsync(dq, r.queries_xyz, sizeof(float) * 3 * r.n_queries, cudaMemcpyHostToDevice, s));
    }
    if (r.search == SFC_SEARCH_RADIUS) {
        st = radius_search(q.tree, dq, r.queries_xyz ? r.n_queries : 0, r.r, static_cast<sfc_kernel>(r.kernel), s,
                           &q.csr);
    } else {
        st = sfc::dev_alloc(&q.knn_idx, q.rows * r.k, s);
        if (st == SFC_OK) st = sfc::dev_alloc(&q.knn_d2, q.rows * r.k, s);
        if (st == SFC_OK) st = knn(q.tree, dq, r.queries_xyz ? r.n_queries : 0, r.k, s, q.knn_idx, q.knn_d2);
    }
    if (st != SFC_OK) return st;
    SFC_CUDA(cudaStreamSynchronize(s));
    return SFC_OK;
}

sfc_status run_merged(sfc_server_s* S, std::vector<Request*>& group, cudaStream_t s, std::shared_ptr<Pass>& pass) {
    int64_t total = 0;
    std::vector<sfc_batch_cloud> clouds(group.size());
    for (size_t i = 0; i < group.size(); ++i) {
        const sfc_request& r = group[i]->req;
        sfc_batch_cloud& c = clouds[i];
        memset(&c, 0, sizeof c);
        c.n_points = r.n_points;
        c.search = r.search;
        c.kernel = r.kernel;
        c.r = r.r;
        c.k = r.k;
        total += r.n_points;
    }
    float* dpts = nullptr;
    sfc::Scratch scratch(s);  // the device copy of the clouds, freed in stream order on return
    SFC_TRY(scratch.alloc(&dpts, 3 * total));
    int64_t off = 0;
    for (Request* q : group) {
        if (q->req.n_points > 0)
            SFC_CUDA(cudaMemcpyAsync(dpts + 3 * off, q->req.points_xyz, sizeof(float) * 3 * q->req.n_points,
                                     cudaMemcpyHostToDevice, s));
        off += q->req.n_points;
    }
    sfc_build_opts o;
    sfc_build_opts_default(&o);
    o.leaf_capacity = S->o.leaf_capacity;
    pass = std::make_shared<Pass>();
    pass->stream = s;
    const sfc_status st = batch_search(dpts, clouds.data(), static_cast<int32_t>(clouds.size()), S->o.enc, &o, s,
                                       &pass->batch);
    if (st != SFC_OK) return st;
    for (size_t i = 0; i < group.size(); ++i) {
        Request& q = *group[i];
        q.pass = pass;
        q.cloud = static_cast<int32_t>(i);
        q.rows = q.req.n_points;
        if (q.req.search == SFC_SEARCH_RADIUS) {
            const int64_t* rp = nullptr;
            const int32_t* cols = nullptr;
            SFC_TRY(batch_cloud_result(pass->batch, q.cloud, &rp, &cols, &q.csr.nnz, nullptr, nullptr));
        }
    }
    SFC_CUDA(cudaStreamSynchronize(s));
    return SFC_OK;
}

void release_single(Request& q) {
    if (q.csr.row_ptr || q.csr.cols) sfc_csr_free(&q.csr, q.stream);
    sfc::dev_free(q.knn_idx, q.stream);
    sfc::dev_free(q.knn_d2, q.stream);
    if (q.tree) octree_free(q.tree, q.stream);
    q.tree = nullptr;
    q.knn_idx = nullptr;
    q.knn_d2 = nullptr;
    q.csr = sfc_csr{};
}

void worker(sfc_server_s* S, int slot) {
    cudaSetDevice(S->device);
    const cudaStream_t s = S->streams[slot];
    for (;;) {
        std::vector<Request*> group;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // the budget holds while the server stops too: queued requests still wait for
            // memory (finished requests release theirs once stopping, see below)
            S->cv_work.wait(lk, [&] {
                if (S->queue.empty()) return S->stopping;
                const int64_t e = S->queue.front()->reserve;
                return S->reserved + e <= S->o.hbm_budget || S->reserved == 0;
            });
            if (S->queue.empty()) {
                if (S->stopping) return;
                continue;
            }
            Request* head = S->queue.front();
            S->queue.pop_front();
            S->reserved += head->reserve;
            group.push_back(head);
            if (mergeable(head->req, S->o.batch_points)) {
                int64_t pts = head->req.n_points;
                while (!S->queue.empty() && static_cast<int32_t>(group.size()) < S->o.max_batch) {
                    Request* nx = S->queue.front();
                    if (!mergeable(nx->req, S->o.batch_points) || pts + nx->req.n_points > S->o.batch_points ||
                        S->reserved + nx->reserve > S->o.hbm_budget)
                        break;
                    S->queue.pop_front();
                    S->reserved += nx->reserve;
                    pts += nx->req.n_points;
                    group.push_back(nx);
                }
            }
            const Clock::time_point now = Clock::now();
            for (Request* q : group) {
                q->admitted = now;
                q->batched_with = static_cast<int32_t>(group.size());
                q->stream = s;
            }
            S->admitted_count += static_cast<int64_t>(group.size());
        }
        std::shared_ptr<Pass> pass;
        // alone (nothing queued to merge with, or query centres given): the single-cloud path
        std::vector<sfc_status> status(group.size(), SFC_OK);
        if (group.size() == 1) {
            status[0] = run_single(S, *group[0], s);
        } else if (run_merged(S, group, s, pass) != SFC_OK) {
            // one request of the merged pass failed (a non-finite cloud, say): answer each
            // alone, so that only the failing one reports the failure
            cudaStreamSynchronize(s);
            for (Request* q : group) {
                q->pass.reset();
                q->cloud = -1;
                q->batched_with = 1;
                q->csr = sfc_csr{};
            }
            pass.reset();
            for (size_t i = 0; i < group.size(); ++i) {
                status[i] = run_single(S, *group[i], s);
                if (status[i] != SFC_OK) cudaStreamSynchronize(s);
            }
        }
        if (group.size() == 1 && status[0] != SFC_OK) cudaStreamSynchronize(s);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const Clock::time_point now = Clock::now();
            for (size_t i = 0; i < group.size(); ++i) {
                Request* q = group[i];
                const sfc_status st = status[i];
                q->done = now;
                q->status = st;
                q->finished = true;
                if (st != SFC_OK || S->stopping) {
                    // failed, or the server is stopping (no one reads results after
                    // server_destroy): free its memory now so that queued requests fit
                    release_single(*q);
                    q->pass.reset();
                    S->reserved -= q->reserve;
                    q->reserve = 0;
                } else {
                    const int64_t held = held_bytes(*q);
                    S->reserved += held - q->reserve;  // from the estimate to what stays resident
                    q->reserve = held;
                }
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

sfc_status sfc_server_opts_default(sfc_server_opts* o) {
    if (!o) return SFC_ERR_INVALID;
    o->slots = 4;
    o->max_batch = 64;
    o->batch_points = 4000000;
    o->hbm_budget = 150LL << 30;
    o->enc = SFC_ENC_HILBERT;
    o->leaf_capacity = 64;
    return SFC_OK;
}

sfc_status server_create(const sfc_server_opts* opts, sfc_server* out) {
    if (!out) return SFC_ERR_INVALID;
    *out = nullptr;
    sfc_server_opts o;
    sfc_server_opts_default(&o);
    if (opts) o = *opts;
    if (o.slots < 1 || o.slots > 16 || o.max_batch < 1 || o.max_batch > sfc::kBatchMax || o.batch_points < 0 ||
        o.hbm_budget <= 0 || o.leaf_capacity < 1 || (o.enc != SFC_ENC_MORTON && o.enc != SFC_ENC_HILBERT))
        return SFC_ERR_INVALID;
    sfc_server_s* S = new (std::nothrow) sfc_server_s;
    if (!S) return SFC_ERR_OOM;
    S->o = o;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return SFC_ERR_CUDA;
    }
    if (sfc::ensure_pool(S->device) != SFC_OK) {
        delete S;
        return SFC_ERR_CUDA;
    }
    for (int i = 0; i < o.slots; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            delete S;
            return SFC_ERR_CUDA;
        }
        S->streams.push_back(st);
    }
    for (int i = 0; i < o.slots; ++i) S->workers.emplace_back(worker, S, i);
    *out = S;
    return SFC_OK;
}

sfc_status server_submit(sfc_server S, const sfc_request* r, int64_t* id) {
    if (!S || !r || !id) return SFC_ERR_INVALID;
    if (r->n_points < 0 || (r->n_points > 0 && !r->points_xyz) || (r->queries_xyz && r->n_queries < 0)) return SFC_ERR_INVALID;
    if (r->search == SFC_SEARCH_RADIUS) {
        if (r->kernel < 0 || r->kernel > 3 || r->r != r->r) return SFC_ERR_INVALID;
    } else if (r->search == SFC_SEARCH_KNN) {
        if (r->k < 1) return SFC_ERR_INVALID;
        if (r->k > sfc::kMaxK) return SFC_ERR_TOO_LARGE;
    } else {
        return SFC_ERR_INVALID;
    }
    std::unique_ptr<Request> q(new (std::nothrow) Request);
    if (!q) return SFC_ERR_OOM;
    q->req = *r;
    q->arrival = Clock::now();
    q->reserve = estimate(*r);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) return SFC_ERR_INVALID;
        q->id = S->next_id++;
        *id = q->id;
        S->queue.push_back(q.get());
        S->reqs.emplace(q->id, std::move(q));
    }
    S->cv_work.notify_one();
    return SFC_OK;
}

sfc_status server_wait(sfc_server S, int64_t id, int32_t timeout_ms, sfc_status* result) {
    if (!S) return SFC_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return SFC_ERR_INVALID;
    Request* q = it->second.get();
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, [&] { return q->finished; });
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return q->finished; })) {
        return SFC_ERR_TIMEOUT;
    }
    if (result) *result = q->status;
    return SFC_OK;
}

sfc_status server_result(sfc_server S, int64_t id, sfc_request_result* out) {
    if (!S || !out) return SFC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || !it->second->finished) return SFC_ERR_INVALID;
    const Request& q = *it->second;
    if (q.status != SFC_OK) return q.status;
    memset(out, 0, sizeof *out);
    out->n_rows = q.rows;
    out->batched_with = q.batched_with;
    out->queue_ms = std::chrono::duration<double, std::milli>(q.admitted - q.arrival).count();
    out->latency_ms = std::chrono::duration<double, std::milli>(q.done - q.arrival).count();
    if (q.pass) {
        const int64_t* rp = nullptr;
        const int32_t* cols = nullptr;
        const int32_t* ki = nullptr;
        const float* kd = nullptr;
        int64_t nnz = 0;
        SFC_TRY(batch_cloud_result(q.pass->batch, q.cloud, &rp, &cols, &nnz, &ki, &kd));
        out->row_ptr = rp;  // the batch hands out every cloud's rows starting at 0
        out->cols = cols;
        out->nnz = nnz;
        out->knn_idx = ki;
        out->knn_d2 = kd;
    } else if (q.req.search == SFC_SEARCH_RADIUS) {
        out->row_ptr = q.csr.row_ptr;
        out->cols = q.csr.cols;
        out->nnz = q.csr.nnz;
    } else {
        out->knn_idx = q.knn_idx;
        out->knn_d2 = q.knn_d2;
    }
    return SFC_OK;
}

sfc_status server_release(sfc_server S, int64_t id) {
    if (!S) return SFC_ERR_INVALID;
    std::unique_ptr<Request> q;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end() || !it->second->finished) return SFC_ERR_INVALID;
        q = std::move(it->second);
        S->reqs.erase(it);
        S->reserved -= q->reserve;
    }
    release_single(*q);
    q->pass.reset();  // the merged pass goes with its last request
    S->cv_work.notify_all();
    return SFC_OK;
}

sfc_status server_stats(sfc_server S, sfc_server_stats* out) {
    if (!S || !out) return SFC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof *out);
    out->queued = static_cast<int64_t>(S->queue.size());
    out->admitted = S->admitted_count;
    out->reserved_bytes = S->reserved;
    for (const auto& kv : S->reqs)
        if (!kv.second->finished && std::find(S->queue.begin(), S->queue.end(), kv.second.get()) == S->queue.end())
            ++out->running;
    return SFC_OK;
}

sfc_status server_destroy(sfc_server S) {
    if (!S) return SFC_ERR_INVALID;
    {
        // finished requests give their memory back first, so that the queued ones, which
        // still run, are admitted within the budget
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (auto& kv : S->reqs) {
            Request& q = *kv.second;
            if (!q.finished) continue;
            release_single(q);
            q.pass.reset();
            S->reserved -= q.reserve;
            q.reserve = 0;
        }
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto& kv : S->reqs) {
        release_single(*kv.second);
        kv.second->pass.reset();
    }
    S->reqs.clear();
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete S;
    return SFC_OK;
}

}  // extern "C"
