// Serving loop: continuous batching of slice requests over resident
// sequences and dictionaries (no counterpart in the paper, which matches one
// slice at a time).
//
// submit()  copies the request's fingerprints into library memory and queues it.
// A scheduler thread (one per context) repeatedly
//   - retires finished launches (event query), releasing their device memory;
//   - admits queued requests while a stream slot is free and the HBM budget
//     has room for the batch: requests with the same batch key (mode,
//     dictionary/sequence/grid, options) are concatenated, oldest first, up to
//     max_batch_voxels, into ONE matcher or ZOOM launch;
//   - launches the batch on its slot's stream: H2D copy, kernels, D2H copy of
//     each request's results, completion event.
// Requests that arrive while others run are admitted as slots and memory
// free up, so their copies and kernels overlap the running work. Every
// voxel's result is independent of its batch-mates (deterministic kernels),
// so a request gives the same result alone and in a mix.
// poll() waits on a condition variable with a deadline; it never blocks
// beyond the caller's timeout.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "mrf_internal.h"

namespace {

struct Req {
    uint64_t ticket = 0;
    int mode = 0;
    const mrf_dict *dict = nullptr;
    mrf_match_opts match{};
    const mrf_seq *seq = nullptr;
    mrf_grid_desc grid{};
    mrf_zoom_opts zoom{};
    int64_t V = 0;
    int n = 0;
    std::vector<float> fp;            // V x n complex64
    std::vector<mrf_result> result;   // filled at completion
    bool done = false;
    int status = MRF_OK;
    std::string error;
};

struct Launch {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<std::shared_ptr<Req>> reqs;
    void *dev = nullptr;
    size_t bytes = 0;
    mrf_result *host_out = nullptr;   // pinned staging for the batch's results
    size_t host_bytes = 0;
    bool busy = false;
};

bool same_key(const Req &a, const Req &b)
{
    if (a.mode != b.mode || a.n != b.n) return false;
    if (a.mode == MRF_MODE_BRUTE)
        return a.dict == b.dict && a.match.precision == b.match.precision && a.match.top_k == b.match.top_k &&
               a.match.rescore == b.match.rescore;
    return a.seq == b.seq && memcmp(&a.grid, &b.grid, sizeof a.grid) == 0 && memcmp(&a.zoom, &b.zoom, sizeof a.zoom) == 0;
}

// Device bytes a batch of V voxels needs beyond resident data: fingerprints,
// results, and the matcher's scratch (voxel operands, partial lists, candidates).
size_t batch_bytes(const mrf_ctx *ctx, const Req &r, int64_t V)
{
    size_t b = (size_t)V * r.n * 8 + (size_t)V * sizeof(mrf_result) + 4096;
    if (r.mode == MRF_MODE_BRUTE) {
        const int64_t blk = r.dict->dtype == MRF_F32 ? 64 : 128;   // voxels per matcher work unit
        const int64_t vp = (V + blk - 1) / blk * blk;
        const size_t eb = r.dict->dtype == MRF_FP8E4M3 ? 1 : 2;
        b += (size_t)(2 * vp) * r.dict->ld * eb * (r.dict->dtype == MRF_F32 ? 2 : 1);
        b += (size_t)V * ctx->sm_count * r.match.top_k * 8 + (size_t)V * r.match.top_k * 12 + 8 * 1024;
    } else {
        b += 64 * 1024 + (size_t)(r.grid.n_t1 + r.grid.n_t2 + r.grid.n_df) * 16;
    }
    return b;
}

}  // namespace

struct ServeState {
    mrf_ctx *ctx = nullptr;
    mrf_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work;   // scheduler wake-ups
    std::condition_variable cv_done;   // poll wake-ups
    std::deque<std::shared_ptr<Req>> queue;
    std::map<uint64_t, std::shared_ptr<Req>> tickets;
    std::vector<Launch> slots;
    std::thread thread;
    bool stopping = false;
    uint64_t next_ticket = 1;
    mrf_serve_stats stats{};
    size_t inflight_bytes = 0;
};

static void finish_slot(ServeState *S, Launch &L)
{
    // results are in pinned host memory; split them back to the requests
    int64_t off = 0;
    for (auto &r : L.reqs) {
        r->result.assign(L.host_out + off, L.host_out + off + r->V);
        off += r->V;
        r->done = true;
        S->stats.completed++;
    }
    S->stats.running_now -= L.reqs.size();
    S->inflight_bytes -= L.bytes;
    S->stats.request_bytes_in_use = S->inflight_bytes;
    L.reqs.clear();
    L.busy = false;
}

static void fail_slot(ServeState *S, Launch &L, int code, const std::string &msg)
{
    for (auto &r : L.reqs) {
        r->status = code;
        r->error = msg;
        r->done = true;
    }
    S->stats.running_now -= L.reqs.size();
    S->inflight_bytes -= L.bytes;
    S->stats.request_bytes_in_use = S->inflight_bytes;
    L.reqs.clear();
    L.busy = false;
}

// Launch one batch on slot L (called with the state mutex released).
static int launch_batch(ServeState *S, Launch &L, std::vector<std::shared_ptr<Req>> &batch, int64_t V)
{
    mrf_ctx *ctx = S->ctx;
    const Req &k = *batch[0];
    const size_t fp_bytes = (size_t)V * k.n * 8, out_bytes = (size_t)V * sizeof(mrf_result);
    const size_t dev_bytes = fp_bytes + 256 + out_bytes;
    int rc = budget_charge(ctx, dev_bytes);
    if (rc) return rc;
    uint8_t *dev = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&dev, dev_bytes, L.stream);
    if (e != cudaSuccess) { budget_release(ctx, dev_bytes); return cuda_fail(e, "serving buffers"); }
    float *fp = (float *)dev;
    mrf_result *out = (mrf_result *)(dev + ((fp_bytes + 255) & ~(size_t)255));
    if (L.host_bytes < out_bytes) {
        if (L.host_out) cudaFreeHost(L.host_out);
        L.host_out = nullptr;
        e = cudaMallocHost((void **)&L.host_out, out_bytes);
        if (e != cudaSuccess) {
            cudaFreeAsync(dev, L.stream);
            budget_release(ctx, dev_bytes);
            L.host_bytes = 0;
            return cuda_fail(e, "serving host staging");
        }
        L.host_bytes = out_bytes;
    }
    int64_t off = 0;
    for (auto &r : batch) {
        e = cudaMemcpyAsync(fp + off * k.n * 2, r->fp.data(), (size_t)r->V * k.n * 8, cudaMemcpyHostToDevice, L.stream);
        if (e != cudaSuccess) break;
        off += r->V;
    }
    if (e == cudaSuccess) {
        if (k.mode == MRF_MODE_BRUTE)
            rc = run_match(ctx, k.dict, fp, V, k.match.precision, k.match.top_k, k.match.rescore, out, nullptr,
                           nullptr, L.stream);
        else
            rc = run_zoom(ctx, k.seq, &k.grid, &k.zoom, fp, V, out, L.stream);
        if (rc == MRF_OK) e = cudaMemcpyAsync(L.host_out, out, out_bytes, cudaMemcpyDeviceToHost, L.stream);
    }
    cudaFreeAsync(dev, L.stream);
    budget_release(ctx, dev_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "serving copies");
    if (rc) return rc;
    e = cudaEventRecord(L.done, L.stream);
    if (e != cudaSuccess) return cuda_fail(e, "serving event");
    return MRF_OK;
}

static void scheduler(ServeState *S)
{
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // 1. retire finished launches
        bool progressed = false;
        for (auto &L : S->slots) {
            if (!L.busy) continue;
            cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaSuccess) {
                finish_slot(S, L);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                fail_slot(S, L, MRF_E_CUDA, cudaGetErrorString(q));
                progressed = true;
            }
        }
        if (progressed) S->cv_done.notify_all();

        // 2. admit and launch while a slot is free
        for (auto &L : S->slots) {
            if (L.busy || S->queue.empty()) continue;
            std::shared_ptr<Req> head = S->queue.front();
            std::vector<std::shared_ptr<Req>> batch;
            int64_t V = 0;
            for (auto it = S->queue.begin(); it != S->queue.end();) {
                if (same_key(**it, *head) &&
                    (batch.empty() || V + (*it)->V <= (int64_t)S->cfg.max_batch_voxels)) {
                    V += (*it)->V;
                    batch.push_back(*it);
                    it = S->queue.erase(it);
                } else {
                    ++it;
                }
            }
            const size_t need = batch_bytes(S->ctx, *head, V);
            const size_t used = S->ctx->used.load();
            const bool fits_now = used + need <= S->ctx->budget &&
                                  S->inflight_bytes + need <= S->cfg.request_bytes_budget;
            const bool alone = S->inflight_bytes == 0;
            if (!fits_now && !alone) {
                // put the batch back (front, original order) and wait for memory
                for (auto it = batch.rbegin(); it != batch.rend(); ++it) S->queue.push_front(*it);
                break;
            }
            L.busy = true;
            L.reqs = batch;
            L.bytes = need;
            S->inflight_bytes += need;
            S->stats.request_bytes_in_use = S->inflight_bytes;
            if (S->inflight_bytes > S->stats.request_bytes_peak) S->stats.request_bytes_peak = S->inflight_bytes;
            S->stats.admitted += batch.size();
            S->stats.queued_now -= batch.size();
            S->stats.running_now += batch.size();
            S->stats.launches++;
            lk.unlock();
            const int rc = launch_batch(S, L, batch, V);
            const std::string msg = rc ? mrf_last_error() : "";
            lk.lock();
            if (rc) {
                fail_slot(S, L, rc, msg);
                S->cv_done.notify_all();
            }
        }

        bool any_busy = false;
        for (auto &L : S->slots) any_busy |= L.busy;
        if (S->stopping && S->queue.empty() && !any_busy) break;
        // short sleep while kernels run; wake at once for new work
        S->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 200 : 20000));
    }
}

extern "C" int mrf_serve_start(mrf_ctx *ctx, const mrf_serve_config *cfg)
{
    if (!ctx || !cfg) return set_error(MRF_E_INVALID, "NULL argument");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 16 || cfg->max_batch_voxels < 1)
        return set_error(MRF_E_INVALID, "serve: max_inflight must be 1..16 and max_batch_voxels >= 1");
    if (ctx->serve) return set_error(MRF_E_INVALID, "serve: already started");
    cudaSetDevice(ctx->device);
    ServeState *S = new ServeState();
    S->ctx = ctx;
    S->cfg = *cfg;
    if (S->cfg.request_bytes_budget == 0) S->cfg.request_bytes_budget = ctx->budget;
    S->slots.resize(cfg->max_inflight);
    for (auto &L : S->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (auto &M : S->slots) {
                if (M.stream) cudaStreamDestroy(M.stream);
                if (M.done) cudaEventDestroy(M.done);
            }
            delete S;
            return cuda_fail(e, "serve streams");
        }
    }
    ctx->serve = S;
    S->thread = std::thread(scheduler, S);
    return MRF_OK;
}

extern "C" int mrf_serve_submit(mrf_ctx *ctx, const mrf_request *rq, uint64_t *ticket)
{
    if (!ctx || !rq || !ticket) return set_error(MRF_E_INVALID, "NULL argument");
    ServeState *S = ctx->serve;
    if (!S) return set_error(MRF_E_INVALID, "serve: not started");
    if (rq->V < 1 || !rq->fp_host) return set_error(MRF_E_INVALID, "serve: need V >= 1 and fingerprints");
    auto r = std::make_shared<Req>();
    r->mode = rq->mode;
    r->V = rq->V;
    if (rq->mode == MRF_MODE_BRUTE) {
        if (!rq->dict) return set_error(MRF_E_INVALID, "serve: brute-force request without a dictionary");
        const mrf_match_opts &o = rq->match;
        const int k = o.top_k;
        if (o.precision != rq->dict->dtype || !(k == 1 || k == 2 || k == 4 || k == 8 || k == 16 || k == 32) ||
            (o.rescore != 0 && o.rescore != 1))
            return set_error(MRF_E_INVALID, "serve: bad match options");
        r->dict = rq->dict;
        r->match = o;
        r->n = rq->dict->n;
    } else if (rq->mode == MRF_MODE_ZOOM) {
        if (!rq->seq || !rq->grid) return set_error(MRF_E_INVALID, "serve: ZOOM request needs a sequence and a grid");
        int rc = grid_validate(rq->grid);
        if (rc) return rc;
        r->seq = rq->seq;
        r->grid = *rq->grid;
        if (rq->zoom) r->zoom = *rq->zoom;
        else mrf_zoom_opts_default(&r->zoom);
        // requests are concatenated into shared launches: no slice geometry
        if (r->zoom.prior_chain != 0)
            return set_error(MRF_E_UNSUPPORTED, "serve: the spatial-neighbour prior needs mrf_zoom_search");
        r->n = rq->seq->n;
    } else {
        return set_error(MRF_E_INVALID, "serve: unknown mode");
    }
    const size_t need = batch_bytes(ctx, *r, r->V);
    if (need > S->cfg.request_bytes_budget || need > ctx->budget) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stats.rejected++;
        return set_error(MRF_E_BUDGET, "serve: request needs " + std::to_string(need) + " device bytes, more than the budget");
    }
    r->fp.resize((size_t)r->V * r->n * 2);
    memcpy(r->fp.data(), rq->fp_host, r->fp.size() * sizeof(float));
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return set_error(MRF_E_INVALID, "serve: stopping");
    r->ticket = S->next_ticket++;
    S->tickets[r->ticket] = r;
    S->queue.push_back(r);
    S->stats.submitted++;
    S->stats.queued_now++;
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return MRF_OK;
}

extern "C" int mrf_serve_poll(mrf_ctx *ctx, uint64_t ticket, int32_t timeout_ms, mrf_result *out)
{
    if (!ctx || !out) return set_error(MRF_E_INVALID, "NULL argument");
    ServeState *S = ctx->serve;
    if (!S) return set_error(MRF_E_INVALID, "serve: not started");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return set_error(MRF_E_NOTFOUND, "serve: unknown or retired ticket");
    std::shared_ptr<Req> r = it->second;
    if (!r->done && timeout_ms > 0) {
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
        S->cv_done.wait_until(lk, deadline, [&] { return r->done; });
    }
    if (!r->done) {
        if (timeout_ms <= 0) return MRF_PENDING;
        return set_error(MRF_E_TIMEOUT, "serve: request not finished within the timeout");
    }
    S->tickets.erase(ticket);
    if (r->status != MRF_OK) return set_error(r->status, "serve: " + r->error);
    memcpy(out, r->result.data(), sizeof(mrf_result) * r->V);
    return MRF_OK;
}

extern "C" int mrf_serve_cancel(mrf_ctx *ctx, uint64_t ticket)
{
    if (!ctx) return set_error(MRF_E_INVALID, "NULL argument");
    ServeState *S = ctx->serve;
    if (!S) return set_error(MRF_E_INVALID, "serve: not started");
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        if ((*it)->ticket == ticket) {
            S->queue.erase(it);
            S->tickets.erase(ticket);
            S->stats.cancelled++;
            S->stats.queued_now--;
            return MRF_OK;
        }
    }
    return set_error(MRF_E_NOTFOUND, "serve: ticket not queued (unknown, running or finished)");
}

extern "C" int mrf_serve_get_stats(mrf_ctx *ctx, mrf_serve_stats *out)
{
    if (!ctx || !out) return set_error(MRF_E_INVALID, "NULL argument");
    ServeState *S = ctx->serve;
    if (!S) return set_error(MRF_E_INVALID, "serve: not started");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return MRF_OK;
}

extern "C" int mrf_serve_stop(mrf_ctx *ctx)
{
    if (!ctx) return set_error(MRF_E_INVALID, "NULL argument");
    ServeState *S = ctx->serve;
    if (!S) return MRF_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    if (S->thread.joinable()) S->thread.join();
    for (auto &L : S->slots) {
        cudaStreamSynchronize(L.stream);
        cudaStreamDestroy(L.stream);
        cudaEventDestroy(L.done);
        if (L.host_out) cudaFreeHost(L.host_out);
    }
    S->cv_done.notify_all();
    ctx->serve = nullptr;
    delete S;
    return MRF_OK;
}
