// Continuous-batching decision server over many concurrent streams.
//
// Each stream (one video being encoded) keeps on the device, for as long as
// it is open: one co-located CTU time map per temporal layer (the estimator
// input of Sec. 2.1: the CTU times of the previously encoded frame of the
// same temporal layer, the co-TL frame; refreshed by
// trs_server_update_times_layer after each encoded frame) and
// kSlotsPerStream request slots (a luma plane buffer plus the statistics,
// tables and search scratch of one decision).  All of that memory is
// allocated when the stream is admitted; admission fails with TRS_EBUSY when
// it would exceed the server's memory budget.
//
// A worker thread forms device batches from pending requests, first come
// first served: whenever requests are waiting and one of max_inflight batch
// slots is free, it copies their planes in and launches the whole hot path
// for them on that slot's CUDA stream, so batches launched while others run
// overlap on the device.  A finished batch (its event) releases its request
// slots and its decisions become available to trs_server_poll.  Every wait
// is bounded; no device code waits on anything.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.h"

using namespace trs;

namespace {

constexpr int kSlotsPerStream = 2;
constexpr int kMaxLayers = TRS_MAX_TEMPORAL_LAYERS;

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

struct Slot {
    DevBuf mem;  // luma plane, statistics, tables, search scratch
    uint8_t *luma = nullptr;
    size_t dpitch = 0;
    uint8_t *stats = nullptr, *tables = nullptr, *scratch = nullptr;
    bool busy = false;
};

struct Stream {
    bool open = false;
    int W = 0, H = 0, bd = 0, n = 0;
    float lambda = 0.0f;
    PlanEntry *pe = nullptr;
    int layers = 1;
    DevBuf times;                 // layers x R*C resident co-located CTU time maps
    size_t tmap = 0;              // bytes of one map (256-aligned)
    bool have[kMaxLayers] = {};   // a map of that layer was given
    int last = -1;                // layer of the most recent map
    Slot slot[kSlotsPerStream];
    int inflight = 0;
    size_t bytes = 0;
};

struct Request {
    int stream = 0, slot = 0;
    const float *times = nullptr;  // the map this decision reads
    uint64_t ticket = 0, tag = 0;
    const void *luma = nullptr;
    size_t pitch = 0;
    double t_submit = 0.0;
};

struct Batch {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr, copied = nullptr;
    DevBuf dev;  // descriptor blob | flags | scal | partitions
    uint8_t *db = nullptr;
    uint32_t *flags = nullptr;
    uint64_t *scal = nullptr;
    trs_partition *out_dev = nullptr;
    void *host = nullptr;  // pinned: descriptor blob, then partitions
    uint8_t *hb = nullptr;
    trs_partition *out_host = nullptr;
    std::vector<Request> reqs;
    bool busy = false;
    int failed = TRS_OK;  // status of a launch that could not be enqueued
};

}  // namespace

struct trs_server {
    trs_server_opts o{};
    trs_ctx *ctx = nullptr;  // plans and kernel set-up
    std::vector<Stream> streams;
    std::vector<Batch> batches;
    std::deque<Request> pending;
    std::deque<trs_decision> done;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int worker_status = TRS_OK;
    size_t mem_used = 0;
    uint64_t next_ticket = 1;
    uint64_t n_batches = 0, n_frames = 0, n_done_total = 0;
};

namespace {

size_t slot_bytes(const Stream &st) {
    const size_t dpitch = (fmt_row_bytes(st.W, st.bd) + 15) & ~size_t(15);
    const int C = st.pe->host.C, R = st.pe->host.R;
    return align256(dpitch * st.H) + align256(stats_bytes(C, R)) + tables_offsets(C, R).bytes + st.pe->scr.bytes;
}

// Launches one batch on slot b (called by the worker without the lock).
int launch_batch(trs_server *srv, Batch &b) {
    TRS_GUARD_BEGIN
    const int nf = (int)b.reqs.size();
    std::vector<PlanEntry *> pe(nf);
    DevFrame *hf = (DevFrame *)b.hb;
    // frames ordered by shape, so that those sharing a plan are adjacent (the
    // column DP packs them into one warp); each keeps its own output slot
    std::vector<int> order(nf);
    for (int i = 0; i < nf; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const Stream &a = srv->streams[b.reqs[x].stream], &c = srv->streams[b.reqs[y].stream];
        return std::make_tuple(a.W, a.H, a.n) < std::make_tuple(c.W, c.H, c.n);
    });
    for (int j = 0; j < nf; ++j) {
        const int i = order[j];
        const Request &r = b.reqs[i];
        Stream &st = srv->streams[r.stream];
        Slot &sl = st.slot[r.slot];
        TRS_CK(copy_rows_h2d(sl.luma, sl.dpitch, r.luma, r.pitch, fmt_row_bytes(st.W, st.bd), st.H, b.s));
        const int C = st.pe->host.C, R = st.pe->host.R, cells = C * R;
        DevFrame f{};
        f.luma = sl.luma;
        f.pitch = sl.dpitch;
        f.W = st.W;
        f.H = st.H;
        f.bd = fmt_depth(st.bd);
        f.packed = st.bd == TRS_PACKED10;
        f.vec_ok = 1;
        f.times = r.times;
        f.s1 = (uint32_t *)sl.stats;
        f.cnt = (uint32_t *)(sl.stats + align256((size_t)cells * 4));
        f.vmax = (uint32_t *)(sl.stats + 2 * align256((size_t)cells * 4));
        f.s2 = (uint64_t *)(sl.stats + 3 * align256((size_t)cells * 4));
        f.flags = b.flags + j;
        f.tables = sl.tables;
        set_search_scratch(f, *st.pe, sl.scratch, st.n, st.lambda);
        f.scal = b.scal + 4 * j;
        f.out = b.out_dev + i;
        hf[j] = f;
        pe[j] = st.pe;
    }
    BatchLaunch bl;
    batch_describe(bl, b.hb, b.db, nf, pe.data(), b.flags, b.scal, SearchTune{});
    TRS_CK(batch_enqueue(bl, b.s, b.copied, nullptr));
    TRS_CK(cudaMemcpyAsync(b.out_host, b.out_dev, (size_t)nf * sizeof(trs_partition), cudaMemcpyDeviceToHost, b.s));
    TRS_CK(cudaEventRecord(b.done, b.s));
    return TRS_OK;
    TRS_GUARD_END
}

void worker_main(trs_server *srv) {
    cudaSetDevice(srv->o.device);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        // harvest finished batches
        bool any_busy = false;
        for (Batch &b : srv->batches) {
            if (!b.busy) continue;
            const cudaError_t q = b.failed != TRS_OK ? cudaSuccess : cudaEventQuery(b.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            const double t = now_us();
            for (size_t i = 0; i < b.reqs.size(); ++i) {
                const Request &r = b.reqs[i];
                trs_decision d{};
                d.ticket = r.ticket;
                d.tag = r.tag;
                d.stream_id = r.stream;
                d.status = b.failed != TRS_OK ? b.failed : (q == cudaSuccess ? b.out_host[i].status : TRS_ECUDA);
                d.latency_us = t - r.t_submit;
                d.partition = b.out_host[i];
                try {
                    srv->done.push_back(d);
                } catch (const std::bad_alloc &) {
                    srv->worker_status = TRS_ENOMEM;  // the decision is lost; callers see the status
                }
                Stream &st = srv->streams[r.stream];
                st.slot[r.slot].busy = false;
                st.inflight--;
            }
            srv->n_done_total += b.reqs.size();
            b.reqs.clear();
            b.busy = false;
            b.failed = TRS_OK;
            if (q != cudaSuccess) srv->worker_status = TRS_ECUDA;
            srv->cv_done.notify_all();
        }
        // launch while requests wait and a batch slot is free
        while (!srv->pending.empty()) {
            Batch *fb = nullptr;
            for (Batch &b : srv->batches)
                if (!b.busy) {
                    fb = &b;
                    break;
                }
            if (!fb) break;
            const int take = (int)std::min<size_t>(srv->pending.size(), (size_t)srv->o.max_batch);
            for (int i = 0; i < take; ++i) {
                fb->reqs.push_back(srv->pending.front());
                srv->pending.pop_front();
            }
            fb->busy = true;
            any_busy = true;
            srv->n_batches++;
            srv->n_frames += (uint64_t)take;
            lk.unlock();
            const int rc = launch_batch(srv, *fb);
            lk.lock();
            if (rc != TRS_OK) {
                fb->failed = rc;
                srv->worker_status = rc;
            }
        }
        if (srv->stop && srv->pending.empty() && !any_busy) break;
        // bounded wait: new work wakes us, in-flight batches are polled every 20 us
        srv->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 2000));
    }
}

void free_stream(trs_server *srv, Stream &st) {
    for (Slot &sl : st.slot) dev_free(sl.mem);
    dev_free(st.times);
    srv->mem_used -= st.bytes;
    st = Stream();
}

}  // namespace

extern "C" {

int trs_server_create(trs_server **out, const trs_server_opts *o) {
    if (!out || !o) return TRS_EINVAL;
    *out = nullptr;
    if (o->max_streams < 1 || o->max_batch < 1 || o->max_inflight < 1) return TRS_EINVAL;
    trs_opts co{o->max_width, o->max_height, o->max_regions, o->max_batch, o->k_area, o->device};
    trs_ctx *ctx = nullptr;
    TRS_TRY(trs_create(&ctx, &co));
    trs_server *srv = new (std::nothrow) trs_server();
    if (!srv) {
        trs_destroy(ctx);
        return TRS_ENOMEM;
    }
    srv->o = *o;
    srv->ctx = ctx;
    try {
        srv->streams.resize(o->max_streams);
        srv->batches.resize(o->max_inflight);
        for (Batch &b : srv->batches) b.reqs.reserve(o->max_batch);  // the worker never grows them
    } catch (const std::bad_alloc &) {
        trs_server_destroy(srv);
        return TRS_ENOMEM;
    }
    const size_t blob = batch_blob_bytes(o->max_batch);
    const size_t fl = align256((size_t)o->max_batch * 4), sc = align256((size_t)o->max_batch * 32);
    const size_t pb = align256((size_t)o->max_batch * sizeof(trs_partition));
    int rc = TRS_OK;
    for (Batch &b : srv->batches) {
        if (rc != TRS_OK) break;
        rc = dev_alloc(b.dev, blob + fl + sc + pb, &srv->mem_used);
        if (rc != TRS_OK) break;
        b.db = (uint8_t *)b.dev.p;
        b.flags = (uint32_t *)(b.db + blob);
        b.scal = (uint64_t *)(b.db + blob + fl);
        b.out_dev = (trs_partition *)(b.db + blob + fl + sc);
        if (cudaMallocHost(&b.host, blob + pb) != cudaSuccess) rc = TRS_ENOMEM;
        if (rc != TRS_OK) break;
        b.hb = (uint8_t *)b.host;
        b.out_host = (trs_partition *)(b.hb + blob);
        if (cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.copied, cudaEventDisableTiming) != cudaSuccess)
            rc = TRS_ECUDA;
    }
    if (rc == TRS_OK && o->mem_budget_bytes && srv->mem_used > o->mem_budget_bytes) rc = TRS_EBUSY;
    if (rc != TRS_OK) {
        trs_server_destroy(srv);
        return rc;
    }
    try {
        srv->worker = std::thread(worker_main, srv);
    } catch (const std::system_error &) {
        trs_server_destroy(srv);
        return TRS_ENOMEM;
    }
    *out = srv;
    return TRS_OK;
}

int trs_server_destroy(trs_server *srv) {
    if (!srv) return TRS_OK;
    if (srv->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->stop = true;
        }
        srv->cv_work.notify_all();
        srv->worker.join();
    }
    cudaDeviceSynchronize();
    for (Stream &st : srv->streams)
        if (st.open) free_stream(srv, st);
    for (Batch &b : srv->batches) {
        dev_free(b.dev);
        if (b.host) cudaFreeHost(b.host);
        if (b.s) cudaStreamDestroy(b.s);
        if (b.done) cudaEventDestroy(b.done);
        if (b.copied) cudaEventDestroy(b.copied);
    }
    trs_destroy(srv->ctx);
    delete srv;
    return TRS_OK;
}

int trs_server_open_stream(trs_server *srv, int width, int height, int bit_depth, int n_regions, float lambda,
                           int *stream_id) {
    return trs_server_open_stream_layers(srv, width, height, bit_depth, n_regions, lambda, 1, stream_id);
}

int trs_server_open_stream_layers(trs_server *srv, int width, int height, int bit_depth, int n_regions,
                                  float lambda, int n_layers, int *stream_id) {
    TRS_GUARD_BEGIN
    if (!srv || !stream_id || n_layers < 1 || n_layers > kMaxLayers) return TRS_EINVAL;
    TRS_TRY(check_frame(srv->ctx, width, height));
    if (!fmt_ok(bit_depth) || n_regions < 1 || n_regions > srv->o.max_regions) return TRS_EINVAL;
    if (!std::isfinite(lambda) || lambda < 0.0f || lambda > 1000.0f) return TRS_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    int id = -1;
    for (int i = 0; i < (int)srv->streams.size(); ++i)
        if (!srv->streams[i].open) {
            id = i;
            break;
        }
    if (id < 0) return TRS_EBUSY;
    Stream st;
    st.W = width;
    st.H = height;
    st.bd = bit_depth;
    st.n = n_regions;
    st.lambda = lambda;
    TRS_TRY(get_plan(srv->ctx, width, height, n_regions, &st.pe));
    const size_t per_slot = slot_bytes(st);
    st.layers = n_layers;
    st.tmap = align256((size_t)st.pe->host.C * st.pe->host.R * 4);
    const size_t need = st.tmap * n_layers + kSlotsPerStream * per_slot;
    if (srv->o.mem_budget_bytes && srv->mem_used + need > srv->o.mem_budget_bytes) return TRS_EBUSY;
    size_t used = 0;
    int rc = dev_alloc(st.times, st.tmap * n_layers, &used);
    const int C = st.pe->host.C, R = st.pe->host.R;
    for (Slot &sl : st.slot) {
        if (rc != TRS_OK) break;
        rc = dev_alloc(sl.mem, per_slot, &used);
        if (rc != TRS_OK) break;
        sl.dpitch = (fmt_row_bytes(width, bit_depth) + 15) & ~size_t(15);
        sl.luma = (uint8_t *)sl.mem.p;
        sl.stats = sl.luma + align256(sl.dpitch * height);
        sl.tables = sl.stats + align256(stats_bytes(C, R));
        sl.scratch = sl.tables + tables_offsets(C, R).bytes;
    }
    if (rc != TRS_OK) {
        for (Slot &sl : st.slot) dev_free(sl.mem);
        dev_free(st.times);
        return rc;
    }
    st.bytes = used;
    st.open = true;
    srv->mem_used += used;
    srv->streams[id] = st;
    *stream_id = id;
    return TRS_OK;
    TRS_GUARD_END
}

// Waits (bounded) until no request of the stream is on the device.
static int wait_stream_idle(trs_server *srv, std::unique_lock<std::mutex> &lk, Stream &st) {
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(10);
    while (st.inflight > 0) {
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && st.inflight > 0) return TRS_ETIMEOUT;
    }
    return TRS_OK;
}

int trs_server_close_stream(trs_server *srv, int id) {
    if (!srv) return TRS_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (id < 0 || id >= (int)srv->streams.size() || !srv->streams[id].open) return TRS_EINVAL;
    Stream &st = srv->streams[id];
    TRS_TRY(wait_stream_idle(srv, lk, st));
    free_stream(srv, st);
    return TRS_OK;
}

int trs_server_update_times(trs_server *srv, int id, const float *times_host) {
    return trs_server_update_times_layer(srv, id, 0, times_host);
}

int trs_server_update_times_layer(trs_server *srv, int id, int layer, const float *times_host) {
    if (!srv || !times_host) return TRS_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (id < 0 || id >= (int)srv->streams.size() || !srv->streams[id].open) return TRS_EINVAL;
    Stream &st = srv->streams[id];
    if (layer < 0 || layer >= st.layers) return TRS_EINVAL;
    TRS_TRY(wait_stream_idle(srv, lk, st));
    const size_t bytes = (size_t)st.pe->host.C * st.pe->host.R * sizeof(float);
    TRS_CK(cudaMemcpy((uint8_t *)st.times.p + st.tmap * layer, times_host, bytes, cudaMemcpyHostToDevice));
    st.have[layer] = true;
    st.last = layer;
    return TRS_OK;
}

int trs_server_submit(trs_server *srv, int id, const void *luma_host, size_t pitch_bytes, uint64_t tag,
                      uint64_t *ticket) {
    return trs_server_submit_layer(srv, id, 0, luma_host, pitch_bytes, tag, ticket);
}

int trs_server_submit_layer(trs_server *srv, int id, int layer, const void *luma_host, size_t pitch_bytes,
                            uint64_t tag, uint64_t *ticket) {
    TRS_GUARD_BEGIN
    if (!srv || !luma_host) return TRS_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (id < 0 || id >= (int)srv->streams.size() || !srv->streams[id].open) return TRS_EINVAL;
    if (srv->worker_status != TRS_OK) return srv->worker_status;
    Stream &st = srv->streams[id];
    if (layer < 0 || layer >= st.layers || st.last < 0) return TRS_EINVAL;
    // the co-TL map; before a layer's first encoded frame, the most recent map of any layer
    const int use = st.have[layer] ? layer : st.last;
    if (pitch_bytes < fmt_row_bytes(st.W, st.bd)) return TRS_EINVAL;
    int s = -1;
    for (int i = 0; i < kSlotsPerStream; ++i)
        if (!st.slot[i].busy) {
            s = i;
            break;
        }
    if (s < 0) return TRS_EBUSY;
    st.slot[s].busy = true;
    st.inflight++;
    Request r;
    r.stream = id;
    r.slot = s;
    r.times = (const float *)((const uint8_t *)st.times.p + st.tmap * use);
    r.ticket = srv->next_ticket++;
    r.tag = tag;
    r.luma = luma_host;
    r.pitch = pitch_bytes;
    r.t_submit = now_us();
    srv->pending.push_back(r);
    if (ticket) *ticket = r.ticket;
    srv->cv_work.notify_one();
    return TRS_OK;
    TRS_GUARD_END
}

int trs_server_poll(trs_server *srv, trs_decision *out, int max_out, int timeout_us, int *n_out) {
    if (!srv || !out || max_out < 1 || !n_out) return TRS_EINVAL;
    *n_out = 0;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->done.empty() && timeout_us > 0)
        srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !srv->done.empty(); });
    int k = 0;
    while (k < max_out && !srv->done.empty()) {
        out[k++] = srv->done.front();
        srv->done.pop_front();
    }
    *n_out = k;
    if (k == 0) return srv->worker_status != TRS_OK ? srv->worker_status : TRS_ETIMEOUT;
    return TRS_OK;
}

int trs_server_info(trs_server *srv, trs_server_stats *out) {
    if (!srv || !out) return TRS_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    out->batches = srv->n_batches;
    out->frames = srv->n_frames;
    out->decided = srv->n_done_total;
    out->mem_used_bytes = srv->mem_used + trs_ctx_bytes(srv->ctx);
    out->pending = (int)srv->pending.size();
    int open = 0, inflight = 0;
    for (const Stream &st : srv->streams) {
        open += st.open;
        inflight += st.inflight;
    }
    out->streams_open = open;
    out->inflight = inflight;
    out->status = srv->worker_status;
    return TRS_OK;
}

}  // extern "C"
