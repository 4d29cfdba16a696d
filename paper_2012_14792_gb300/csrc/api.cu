// The C ABI of include/trs.h: contexts, argument checks, buffers, plans and
// the launch sequences of the one-frame and batched paths.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "ctx.h"

using namespace trs;

namespace {
thread_local char g_err[512] = "";
}  // namespace

namespace trs {

int cuda_fail(cudaError_t e, const char *what) {
    std::snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
    return TRS_ECUDA;
}

int dev_alloc(DevBuf &b, size_t bytes, size_t *total) {
    if (b.n >= bytes && b.p) return TRS_OK;
    if (b.p) {
        cudaDeviceSynchronize();
        cudaFree(b.p);
        *total -= b.n;
        b.p = nullptr;
        b.n = 0;
    }
    if (bytes == 0) return TRS_OK;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cuda_fail(e, "cudaMalloc");
        b.p = nullptr;
        return TRS_ENOMEM;
    }
    b.n = bytes;
    *total += bytes;
    return TRS_OK;
}

void dev_free(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

uint32_t lambda_to_q(float lambda) { return (uint32_t)std::rint((double)lambda * 65536.0); }

int check_frame(const trs_ctx *ctx, int W, int H) {
    if (W <= 0 || H <= 0 || W > ctx->o.max_width || H > ctx->o.max_height) return TRS_EINVAL;
    return TRS_OK;
}

int get_plan(trs_ctx *ctx, int W, int H, int n, PlanEntry **out) {
    TRS_GUARD_BEGIN
    auto key = std::make_tuple(W, H, n, ctx->window_step);
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        *out = it->second;
        return TRS_OK;
    }
    PlanEntry *e = new PlanEntry();
    int s = build_plan(W, H, n, ctx->o.k_area, &e->host, ctx->window_step);
    if (s != TRS_OK) {
        delete e;
        return s;
    }
    std::vector<uint8_t> blob;
    s = dev_alloc(e->blob, plan_blob_bytes(e->host), &ctx->total);
    if (s != TRS_OK) {
        delete e;
        return s;
    }
    plan_serialize(e->host, (uint8_t *)e->blob.p, blob);
    cudaError_t ce = cudaMemcpy(e->blob.p, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        ctx->total -= e->blob.n;
        dev_free(e->blob);
        delete e;
        return cuda_fail(ce, "plan upload");
    }
    e->dev = (const DevPlan *)e->blob.p;
    e->scr = scratch_layout(e->host);
    ctx->plans[key] = e;
    *out = e;
    return TRS_OK;
    TRS_GUARD_END
}

size_t stats_bytes(int C, int R) {
    return align256((size_t)R * C * 4) * 3 + align256((size_t)R * C * 8) + 256;
}

void drop_graphs(trs_ctx *ctx) {
    for (auto &g : ctx->graphs)
        if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    ctx->graphs.clear();
}

}  // namespace trs

extern "C" {

int trs_version(void) { return TRS_ABI_VERSION; }

const char *trs_strerror(int status) {
    switch (status) {
        case TRS_OK: return "ok";
        case TRS_EINVAL: return "invalid argument";
        case TRS_ERANGE: return "sample or time out of range";
        case TRS_EINFEASIBLE: return "no partition satisfies the area rule";
        case TRS_ENOMEM: return "out of memory or beyond the context's limits";
        case TRS_EBUSY: return "admission refused";
        case TRS_ETIMEOUT: return "a bounded wait gave up";
        case TRS_ECUDA: return "CUDA runtime error";
        default: return "unknown status";
    }
}

const char *trs_last_error(void) { return g_err; }

size_t trs_sizeof(const char *name) {
    if (!name) return 0;
    if (!std::strcmp(name, "trs_opts")) return sizeof(trs_opts);
    if (!std::strcmp(name, "trs_ctu_stats")) return sizeof(trs_ctu_stats);
    if (!std::strcmp(name, "trs_tables_layout")) return sizeof(trs_tables_layout);
    if (!std::strcmp(name, "trs_partition")) return sizeof(trs_partition);
    if (!std::strcmp(name, "trs_frame_desc")) return sizeof(trs_frame_desc);
    if (!std::strcmp(name, "trs_server_opts")) return sizeof(trs_server_opts);
    if (!std::strcmp(name, "trs_decision")) return sizeof(trs_decision);
    if (!std::strcmp(name, "trs_server_stats")) return sizeof(trs_server_stats);
    if (!std::strcmp(name, "trs_tune_report")) return sizeof(trs_tune_report);
    if (!std::strcmp(name, "trs_mt_partition")) return sizeof(trs_mt_partition);
    return 0;
}

int trs_plan_work(int width, int height, int n, int k, double *row_relax, double *col_relax) {
    if (!row_relax || !col_relax) return TRS_EINVAL;
    HostPlan p;
    TRS_TRY(build_plan(width, height, n, k, &p));
    double rows = 0.0, cols = 0.0;
    for (const PlanItem &it : p.items) {
        const int dmin = std::max(1, (int)((it.hlo + kCtu - 1) / kCtu));
        const int dmax = std::min(p.R, (int)(it.hhi / kCtu) + 1);
        rows += (double)it.kmax * (dmax - dmin + 1) * p.R;
    }
    for (size_t w = 0; w < p.win_a.size(); ++w)
        for (int b = 0; b < p.nb; ++b) {
            const int32_t slot = p.slot_of[w * p.nb + b];
            if (slot < 0) continue;
            const int klo = std::max(1, (int)p.items[slot].kmin), khi = std::min((int)p.items[slot].kmax, p.n);
            for (int k = klo; k <= khi; ++k) cols += (double)(p.n - k + 1);  // m = k..n
        }
    *row_relax = rows;
    *col_relax = cols;
    return TRS_OK;
}

int trs_count_partitions(int width, int height, int n, int k, double *count) {
    if (!count) return TRS_EINVAL;
    long double c = 0.0L;
    TRS_TRY(count_partitions(width, height, n, k, &c));
    *count = (double)c;
    return TRS_OK;
}

int trs_plan_stats(int width, int height, int n, int k, int *n_windows, int *n_items) {
    if (!n_windows || !n_items) return TRS_EINVAL;
    HostPlan p;
    TRS_TRY(build_plan(width, height, n, k, &p));
    *n_windows = (int)p.win_a.size();
    *n_items = (int)p.items.size();
    return TRS_OK;
}

int trs_plan_coverage(int width, int height, int n, int k, int window_step, int *windows, int *short_windows,
                      double *in_windows) {
    return plan_coverage(width, height, n, k, window_step, windows, short_windows, in_windows);
}

int trs_create(trs_ctx **out, const trs_opts *o) {
    TRS_GUARD_BEGIN
    if (!out || !o) return TRS_EINVAL;
    *out = nullptr;
    if (o->max_width < 1 || o->max_width > kCtu * kMaxC || o->max_height < 1 || o->max_height > kCtu * kMaxR ||
        o->max_regions < 1 || o->max_regions > kMaxN || o->max_batch < 1 || o->k_area < 1)
        return TRS_EINVAL;
    TRS_CK(cudaSetDevice(o->device));
    TRS_CK((cudaError_t)prepare_tables_kernel());
    TRS_CK((cudaError_t)prepare_search_kernels());
    trs_ctx *c = new trs_ctx();
    c->o = *o;
    c->maxC = (o->max_width + kCtu - 1) / kCtu;
    c->maxR = (o->max_height + kCtu - 1) / kCtu;
    const size_t cells = (size_t)c->maxC * c->maxR;
    const int bps = 2;
    int s = TRS_OK;
    s = s ? s : dev_alloc(c->s1, cells * 4, &c->total);
    s = s ? s : dev_alloc(c->s2, cells * 8, &c->total);
    s = s ? s : dev_alloc(c->cnt, cells * 4, &c->total);
    s = s ? s : dev_alloc(c->vmax, cells * 4, &c->total);
    s = s ? s : dev_alloc(c->flags, 256, &c->total);
    s = s ? s : dev_alloc(c->tables, tables_offsets(c->maxC, c->maxR).bytes, &c->total);
    s = s ? s : dev_alloc(c->scal, 256, &c->total);
    s = s ? s : dev_alloc(c->part, sizeof(trs_partition), &c->total);
    s = s ? s : dev_alloc(c->luma_stage, (size_t)align256((size_t)o->max_width * bps) * o->max_height, &c->total);
    s = s ? s : dev_alloc(c->time_stage, cells * 4, &c->total);
    if (s == TRS_OK && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) s = TRS_ECUDA;
    if (s == TRS_OK && cudaEventCreateWithFlags(&c->copied, cudaEventDisableTiming) != cudaSuccess) s = TRS_ECUDA;
    if (s == TRS_OK && cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess) s = TRS_ECUDA;
    for (int i = 0; i < kMaxParts && s == TRS_OK; ++i)
        if (cudaEventCreateWithFlags(&c->tex_done[i], cudaEventDisableTiming) != cudaSuccess) s = TRS_ECUDA;
    if (s == TRS_OK && cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) s = TRS_ECUDA;
    for (int i = 0; i <= trs_ctx::kStages && s == TRS_OK; ++i)
        if (cudaEventCreate(&c->stage[i]) != cudaSuccess) s = TRS_ECUDA;
    if (s != TRS_OK) {
        trs_destroy(c);
        return s;
    }
    *out = c;
    return TRS_OK;
    TRS_GUARD_END
}

int trs_destroy(trs_ctx *c) {
    if (!c) return TRS_OK;
    cudaDeviceSynchronize();
    drop_graphs(c);
    for (auto &p : c->plans) {
        dev_free(p.second->blob);
        delete p.second;
    }
    for (auto &m : c->mt) mt_free(m.second);
    if (c->mt_cap) cudaStreamDestroy(c->mt_cap);
    DevBuf *bufs[] = {&c->s1, &c->s2, &c->cnt, &c->vmax, &c->flags, &c->tables, &c->scratch, &c->scal,
                      &c->part, &c->luma_stage, &c->time_stage, &c->arena, &c->desc,
                      &c->hb_luma, &c->hb_time, &c->hb_out};
    for (DevBuf *b : bufs) dev_free(*b);
    if (c->staging) cudaFreeHost(c->staging);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->copied) cudaEventDestroy(c->copied);
    if (c->cap2) cudaStreamDestroy(c->cap2);
    for (int i = 0; i < kMaxParts; ++i)
        if (c->tex_done[i]) cudaEventDestroy(c->tex_done[i]);
    if (c->join) cudaEventDestroy(c->join);
    for (int i = 0; i <= trs_ctx::kStages; ++i)
        if (c->stage[i]) cudaEventDestroy(c->stage[i]);
    delete c;
    return TRS_OK;
}

size_t trs_ctx_bytes(const trs_ctx *c) { return c ? c->total : 0; }

int trs_tables_layout_get(int width, int height, trs_tables_layout *out) {
    if (!out || width <= 0 || height <= 0) return TRS_EINVAL;
    const int C = (width + kCtu - 1) / kCtu, R = (height + kCtu - 1) / kCtu;
    if (C > kMaxC || R > kMaxR) return TRS_EINVAL;
    const TablesOffsets o = tables_offsets(C, R);
    out->width = width;
    out->height = height;
    out->cols = C;
    out->rows = R;
    out->bands = num_bands(C);
    out->reserved = 0;
    out->bytes = o.bytes;
    out->off_tq = o.tq;
    out->off_sat_s1 = o.sat_s1;
    out->off_sat_s2 = o.sat_s2;
    out->off_sat_t = o.sat_t;
    out->off_rect_t = o.rect_t;
    out->off_rect_q = o.rect_q;
    out->off_status = o.status;
    return TRS_OK;
}

int trs_texture_map(trs_ctx *ctx, const void *luma, int W, int H, size_t pitch, int bd, const trs_ctu_stats *st,
                    void *stream) {
    if (!ctx || !luma || !st || !st->s1 || !st->s2 || !st->count || !st->vmax || !st->flags) return TRS_EINVAL;
    TRS_TRY(check_frame(ctx, W, H));
    if (!fmt_ok(bd)) return TRS_EINVAL;
    if (pitch < fmt_row_bytes(W, bd)) return TRS_EINVAL;
    LaunchArgs a{};
    DevFrame &f = a.single;
    f.luma = (const uint8_t *)luma;
    f.pitch = pitch;
    f.W = W;
    f.H = H;
    f.bd = fmt_depth(bd);
    f.packed = bd == TRS_PACKED10;
    f.vec_ok = ((uintptr_t)luma % 16 == 0) && (pitch % 16 == 0);
    f.C = (W + kCtu - 1) / kCtu;
    f.R = (H + kCtu - 1) / kCtu;
    f.s1 = st->s1;
    f.s2 = st->s2;
    f.cnt = st->count;
    f.vmax = st->vmax;
    f.flags = st->flags;
    a.nframes = 1;
    a.single_ctus = f.C * f.R;
    TRS_CK(cudaMemsetAsync(st->flags, 0, sizeof(uint32_t), (cudaStream_t)stream));
    TRS_CK((cudaError_t)launch_texture(a, f.C * f.R, stream));
    return TRS_OK;
}

int trs_region_tables(trs_ctx *ctx, const trs_ctu_stats *st, const float *times, int W, int H, void *tables,
                      size_t tables_bytes, void *stream) {
    if (!ctx || !st || !st->s1 || !st->s2 || !st->flags || !times || !tables) return TRS_EINVAL;
    TRS_TRY(check_frame(ctx, W, H));
    const int C = (W + kCtu - 1) / kCtu, R = (H + kCtu - 1) / kCtu;
    const TablesOffsets o = tables_offsets(C, R);
    if (tables_bytes < o.bytes || (uintptr_t)tables % 256) return TRS_EINVAL;
    LaunchArgs a{};
    DevFrame &f = a.single;
    f.W = W;
    f.H = H;
    f.C = C;
    f.R = R;
    f.times = times;
    f.s1 = st->s1;
    f.s2 = st->s2;
    f.flags = st->flags;
    f.tables = (uint8_t *)tables;
    a.nframes = 1;
    const int groups = (num_bands(C) + kBandsPerBlock - 1) / kBandsPerBlock;
    a.single_bandgrp = groups;
    TRS_CK((cudaError_t)launch_tables(a, groups, C, R, stream));
    return TRS_OK;
}

static int search_one(trs_ctx *ctx, const void *tables, int W, int H, int n, float lambda, trs_partition *out,
                      void *stream) {
    if (!ctx || !tables || !out || (uintptr_t)tables % 256) return TRS_EINVAL;
    TRS_TRY(check_frame(ctx, W, H));
    if (n < 1 || n > ctx->o.max_regions) return TRS_EINVAL;
    if (!std::isfinite(lambda) || lambda < 0.0f || lambda > 1000.0f) return TRS_EINVAL;
    PlanEntry *pe;
    TRS_TRY(get_plan(ctx, W, H, n, &pe));
    TRS_TRY(dev_alloc(ctx->scratch, pe->scr.bytes, &ctx->total));
    LaunchArgs a{};
    DevFrame &f = a.single;
    uint8_t *scr = (uint8_t *)ctx->scratch.p;
    f.W = W;
    f.H = H;
    f.C = pe->host.C;
    f.R = pe->host.R;
    f.tables = (uint8_t *)tables;
    set_search_scratch(f, *pe, scr, n, lambda);
    f.scal = (uint64_t *)ctx->scal.p;
    f.out = out;
    a.nframes = 1;
    const int nitems = (int)pe->host.items.size(), nwin = (int)pe->host.win_a.size();
    a.single_items = nitems;
    a.single_windows = nwin;
    a.single_bands = pe->host.nb;
    const ColGeom cg = col_uniform(a, pe->host, 1, ctx->tune);
    TRS_CK((cudaError_t)launch_search(a, pe->host.nb, nwin, f.C, f.R, n, f.scal, 4, stream, cg, nullptr, &ctx->tune,
                                      3, pe->host.max_nd));
    return TRS_OK;
}

int trs_search_lambdas(trs_ctx *ctx, const void *tables, int W, int H, int n, const float *lambdas, int nl,
                       trs_partition *out, void *stream) {
    TRS_GUARD_BEGIN
    if (!ctx || !tables || !out || !lambdas || (uintptr_t)tables % 256) return TRS_EINVAL;
    if (nl < 1 || nl > TRS_MAX_LAMBDAS) return TRS_EINVAL;
    TRS_TRY(check_frame(ctx, W, H));
    if (n < 1 || n > ctx->o.max_regions) return TRS_EINVAL;
    for (int i = 0; i < nl; ++i)
        if (!std::isfinite(lambdas[i]) || lambdas[i] < 0.0f || lambdas[i] > 1000.0f) return TRS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PlanEntry *pe;
    TRS_TRY(get_plan(ctx, W, H, n, &pe));
    const size_t per = align256(pe->scr.bytes);
    TRS_TRY(dev_alloc(ctx->scratch, per * nl, &ctx->total));
    const size_t blob = batch_blob_bytes(nl);
    if (ctx->desc.n < blob) {  // captured batches hold the old descriptor address
        drop_graphs(ctx);
        TRS_TRY(dev_alloc(ctx->desc, blob * 2, &ctx->total));
    }
    if (ctx->staging_n < blob) {
        TRS_CK(cudaEventSynchronize(ctx->copied));
        if (ctx->staging) cudaFreeHost(ctx->staging);
        ctx->staging = nullptr;
        ctx->staging_n = 0;
        drop_graphs(ctx);
        TRS_CK(cudaMallocHost(&ctx->staging, blob * 2));
        ctx->staging_n = blob * 2;
    }
    TRS_CK(cudaEventSynchronize(ctx->copied));  // the staging blob is free again
    uint8_t *hb = (uint8_t *)ctx->staging;
    DevFrame *hf = (DevFrame *)hb;
    uint8_t *scr = (uint8_t *)ctx->scratch.p;
    uint64_t *scal = (uint64_t *)ctx->scal.p;  // 4 words per lambda
    for (int i = 0; i < nl; ++i) {
        DevFrame f{};
        f.W = W;
        f.H = H;
        f.tables = (uint8_t *)tables;
        set_search_scratch(f, *pe, scr + i * per, n, lambdas[i]);
        f.scal = scal + 4 * i;
        f.out = out + i;
        hf[i] = f;
    }
    for (int i = 1; i < nl; ++i) {  // step 1 is shared: every lambda reads the first one's results
        hf[i].V1 = hf[0].V1;
        hf[i].wres1 = hf[0].wres1;
    }
    std::vector<PlanEntry *> pes(nl, pe);
    BatchLaunch bl;
    batch_describe(bl, hb, (uint8_t *)ctx->desc.p, nl, pes.data(), nullptr, scal, ctx->tune);
    TRS_CK(cudaMemcpyAsync(bl.db, hb, bl.blob, cudaMemcpyHostToDevice, s));
    TRS_CK(cudaEventRecord(ctx->copied, s));
    TRS_CK(cudaMemsetAsync(scal, 0xff, (size_t)nl * 4 * sizeof(uint64_t), s));
    LaunchArgs one{};
    one.single = hf[0];
    one.nframes = 1;
    one.single_items = (int)pe->host.items.size();
    one.single_windows = (int)pe->host.win_a.size();
    one.single_bands = pe->host.nb;
    const ColGeom cg1 = col_uniform(one, pe->host, 1, ctx->tune);
    TRS_CK((cudaError_t)launch_search(one, pe->host.nb, one.single_windows, pe->host.C, pe->host.R, n, scal, 4, s,
                                      cg1, nullptr, &ctx->tune, 1, pe->host.max_nd));
    for (int i = 1; i < nl; ++i)  // T_min of step 1 for every lambda
        TRS_CK(cudaMemcpyAsync(scal + 4 * i, scal, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    LaunchArgs all{};
    all.frames = (const DevFrame *)bl.db;
    all.nframes = nl;
    all.pre.items = (const int32_t *)(bl.db + bl.fr_bytes + 2 * bl.pre_bytes);
    all.pre.windows = (const int32_t *)(bl.db + bl.fr_bytes + 3 * bl.pre_bytes);
    all.pre.bands = (const int32_t *)(bl.db + bl.fr_bytes + 4 * bl.pre_bytes);
    const ColGeom cg2 = col_uniform(all, pe->host, nl, ctx->tune);
    TRS_CK((cudaError_t)launch_search(all, bl.bands, bl.windows, pe->host.C, pe->host.R, n, scal, (size_t)nl * 4, s,
                                      cg2, nullptr, &ctx->tune, 2, pe->host.max_nd));
    return TRS_OK;
    TRS_GUARD_END
}

int trs_search(trs_ctx *ctx, const void *tables, int W, int H, int n, float lambda, trs_partition *out,
               void *stream) {
    return search_one(ctx, tables, W, H, n, lambda, out, stream);
}

int trs_decide(trs_ctx *ctx, const void *luma, int W, int H, size_t pitch, int bd, const float *times, int n,
               float lambda, trs_partition *out, void *stream) {
    if (!ctx) return TRS_EINVAL;
    trs_ctu_stats st{(uint32_t *)ctx->s1.p, (uint64_t *)ctx->s2.p, (uint32_t *)ctx->cnt.p, (uint32_t *)ctx->vmax.p,
                     (uint32_t *)ctx->flags.p};
    TRS_TRY(trs_texture_map(ctx, luma, W, H, pitch, bd, &st, stream));
    TRS_TRY(trs_region_tables(ctx, &st, times, W, H, ctx->tables.p, ctx->tables.n, stream));
    return search_one(ctx, ctx->tables.p, W, H, n, lambda, out, stream);
}

int trs_decide_host(trs_ctx *ctx, const void *luma_host, int W, int H, size_t pitch, int bd,
                    const float *times_host, int n, float lambda, trs_partition *out_host, void *stream) {
    if (!ctx || !luma_host || !times_host || !out_host) return TRS_EINVAL;
    TRS_TRY(check_frame(ctx, W, H));
    if (!fmt_ok(bd)) return TRS_EINVAL;
    const size_t rowb = fmt_row_bytes(W, bd);
    if (pitch < rowb) return TRS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t dpitch = (rowb + 15) & ~size_t(15);  // 16-byte rows: the vector path, and no padding to copy
    const int C = (W + kCtu - 1) / kCtu, R = (H + kCtu - 1) / kCtu;
    TRS_CK(copy_rows_h2d(ctx->luma_stage.p, dpitch, luma_host, pitch, rowb, H, s));
    TRS_CK(cudaMemcpyAsync(ctx->time_stage.p, times_host, (size_t)R * C * sizeof(float), cudaMemcpyHostToDevice, s));
    TRS_TRY(trs_decide(ctx, ctx->luma_stage.p, W, H, dpitch, bd, (const float *)ctx->time_stage.p, n, lambda,
                       (trs_partition *)ctx->part.p, stream));
    TRS_CK(cudaMemcpyAsync(out_host, ctx->part.p, sizeof(trs_partition), cudaMemcpyDeviceToHost, s));
    TRS_CK(cudaStreamSynchronize(s));
    return TRS_OK;
}

/* ---------------------------------------------------------------------- */
/* Batched path                                                           */

}  // extern "C"

namespace trs {

int batch_run(trs_ctx *ctx, const trs_frame_desc *fd, int nf, trs_partition *out, cudaStream_t stream,
              bool use_graph) {
    TRS_GUARD_BEGIN
    if (!ctx || !fd || !out || nf < 1 || nf > ctx->o.max_batch) return TRS_EINVAL;
    std::vector<PlanEntry *> pe(nf);
    std::vector<int64_t> key;
    key.reserve((size_t)nf * 5 + 1);
    key.push_back(nf);
    for (int i = 0; i < nf; ++i) {
        const trs_frame_desc &d = fd[i];
        if (!d.luma_dev || !d.ctu_time_dev) return TRS_EINVAL;
        TRS_TRY(check_frame(ctx, d.width, d.height));
        if (!fmt_ok(d.bit_depth)) return TRS_EINVAL;
        if (d.pitch_bytes < fmt_row_bytes(d.width, d.bit_depth)) return TRS_EINVAL;
        if (d.n_regions < 1 || d.n_regions > ctx->o.max_regions) return TRS_EINVAL;
        if (!std::isfinite(d.lambda) || d.lambda < 0.0f || d.lambda > 1000.0f) return TRS_EINVAL;
        TRS_TRY(get_plan(ctx, d.width, d.height, d.n_regions, &pe[i]));
        const int vec = ((uintptr_t)d.luma_dev % 16 == 0) && (d.pitch_bytes % 16 == 0);
        key.push_back(d.width);
        key.push_back(d.height);
        key.push_back(d.bit_depth);
        key.push_back(d.n_regions);
        key.push_back(vec);
    }
    // arena layout: flags [nf] | scal [nf][4] | per frame: stats, tables, search scratch
    size_t off = 0;
    const size_t flags_off = off;
    off = align256(off + (size_t)nf * 4);
    const size_t scal_off = off;
    off = align256(off + (size_t)nf * 4 * 8);
    std::vector<size_t> fo(nf);
    for (int i = 0; i < nf; ++i) {
        fo[i] = off;
        const HostPlan &hp = pe[i]->host;
        off += stats_bytes(hp.C, hp.R) + tables_offsets(hp.C, hp.R).bytes + pe[i]->scr.bytes;
    }
    if (ctx->arena.n < off) {
        drop_graphs(ctx);
        TRS_TRY(dev_alloc(ctx->arena, off + off / 4, &ctx->total));
    }
    // a graph batch in chunks keeps one descriptor blob per chunk; each adds
    // at most 6 x 256 bytes of alignment and one prefix entry per table
    const size_t blob = batch_blob_bytes(nf) + (size_t)kMaxParts * 1600;
    if (ctx->desc.n < blob) {
        drop_graphs(ctx);
        TRS_TRY(dev_alloc(ctx->desc, blob * 2, &ctx->total));
    }
    if (ctx->staging_n < blob) {
        TRS_CK(cudaEventSynchronize(ctx->copied));
        if (ctx->staging) cudaFreeHost(ctx->staging);
        ctx->staging = nullptr;
        ctx->staging_n = 0;
        drop_graphs(ctx);
        TRS_CK(cudaMallocHost(&ctx->staging, blob * 2));
        ctx->staging_n = blob * 2;
    }
    // Graph batches run as P chunks of at least kChunkMin frames each (see
    // below).  Inside each chunk the frames are ordered by shape so that
    // frames sharing a plan are adjacent (the column DP packs them into one
    // warp); every frame keeps its own output slot.
    const int parts = use_graph ? std::max(1, std::min(ctx->parts, nf / kChunkMin)) : 1;
    int first[kMaxParts + 1];
    first[0] = 0;
    for (int c = 0; c < parts; ++c) first[c + 1] = (int)((int64_t)nf * (c + 1) / parts);
    std::vector<int> order(nf);
    for (int i = 0; i < nf; ++i) order[i] = i;
    for (int c = 0; c < parts; ++c)
        std::stable_sort(order.begin() + first[c], order.begin() + first[c + 1], [&](int x, int y) {
            return std::make_tuple(fd[x].width, fd[x].height, fd[x].n_regions) <
                   std::make_tuple(fd[y].width, fd[y].height, fd[y].n_regions);
        });
    std::vector<PlanEntry *> pes(nf);
    for (int j = 0; j < nf; ++j) pes[j] = pe[order[j]];
    // the previous replay must have read the staging blob before it is rewritten
    TRS_CK(cudaEventSynchronize(ctx->copied));
    uint8_t *hb = (uint8_t *)ctx->staging;
    DevFrame *hf = (DevFrame *)hb;
    uint8_t *ab = (uint8_t *)ctx->arena.p;
    for (int j = 0; j < nf; ++j) {
        const int i = order[j];
        const trs_frame_desc &d = fd[i];
        const HostPlan &hp = pe[i]->host;
        DevFrame f{};
        const int C = hp.C, R = hp.R, cells = C * R;
        uint8_t *p = ab + fo[i];
        f.luma = (const uint8_t *)d.luma_dev;
        f.pitch = d.pitch_bytes;
        f.W = d.width;
        f.H = d.height;
        f.bd = fmt_depth(d.bit_depth);
        f.packed = d.bit_depth == TRS_PACKED10;
        f.vec_ok = ((uintptr_t)d.luma_dev % 16 == 0) && (d.pitch_bytes % 16 == 0);
        f.times = d.ctu_time_dev;
        f.s1 = (uint32_t *)p;
        f.cnt = (uint32_t *)(p + align256((size_t)cells * 4));
        f.vmax = (uint32_t *)(p + 2 * align256((size_t)cells * 4));
        f.s2 = (uint64_t *)(p + 3 * align256((size_t)cells * 4));
        p += stats_bytes(C, R);
        f.flags = (uint32_t *)(ab + flags_off) + j;
        f.tables = p;
        p += tables_offsets(C, R).bytes;
        set_search_scratch(f, *pe[i], p, d.n_regions, d.lambda);
        f.scal = (uint64_t *)(ab + scal_off) + 4 * j;
        f.out = out + i;
        hf[j] = f;
    }
    uint32_t *flags = (uint32_t *)(ab + flags_off);
    uint64_t *scal = (uint64_t *)(ab + scal_off);
    if (!use_graph) {
        BatchLaunch bl;
        batch_describe(bl, hb, (uint8_t *)ctx->desc.p, nf, pes.data(), flags, scal, ctx->tune);
        bl.tune = ctx->tune;
        cudaError_t e = batch_enqueue(bl, stream, ctx->copied, ctx->stage);
        if (e != cudaSuccess) return cuda_fail(e, "batch launch");
        ctx->stage_valid = true;
        ctx->stage_frames = nf;
        ctx->last_kernels = kKernelsPerBatch;
        return TRS_OK;
    }
    // Graph batches run as P chunks, software pipelined on two streams
    // (chunk c on stream c % 2): chunk c's texture kernel (bound by HBM)
    // starts once chunk c-1's has finished and runs beside chunk c-1's tables
    // and search (bound by the ALUs).  Stage events time chunk 0.
    key.push_back(parts);
    BatchLaunch bl[kMaxParts];
    size_t off_c[kMaxParts + 1];
    off_c[0] = 0;
    for (int c = 0; c < parts; ++c) off_c[c + 1] = off_c[c] + batch_blob_bytes(first[c + 1] - first[c]);
    // each chunk's descriptors at the start of its own blob; the last chunk
    // first, so that no move overwrites descriptors not yet moved
    for (int c = parts - 1; c > 0; --c)
        std::memmove(hb + off_c[c], hb + (size_t)first[c] * sizeof(DevFrame),
                     (size_t)(first[c + 1] - first[c]) * sizeof(DevFrame));
    for (int c = 0; c < parts; ++c) {
        batch_describe(bl[c], hb + off_c[c], (uint8_t *)ctx->desc.p + off_c[c], first[c + 1] - first[c],
                       pes.data() + first[c], flags + first[c], scal + 4 * first[c], ctx->tune);
        bl[c].tune = ctx->tune;
    }
    BatchGraph &g = ctx->graphs[key];
    if (!g.exec) {
        cudaStream_t cs = ctx->cap, st[2] = {ctx->cap, ctx->cap2};
        TRS_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemcpyAsync(bl[0].db, bl[0].hb, off_c[parts], cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = record_event(ctx->copied, cs);
        for (int c = 0; c < parts && e == cudaSuccess; ++c) {
            if (c > 0) e = cudaStreamWaitEvent(st[c % 2], ctx->tex_done[c - 1], 0);
            if (e == cudaSuccess)
                e = batch_enqueue_work(bl[c], st[c % 2], c == 0 ? ctx->stage : nullptr,
                                       c + 1 < parts ? ctx->tex_done[c] : nullptr);
        }
        if (parts > 1) {
            if (e == cudaSuccess) e = cudaEventRecord(ctx->join, ctx->cap2);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->join, 0);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ctx->graphs.erase(key);
            return cuda_fail(e, "batch graph capture");
        }
        g.staged_bytes = blob;
    }
    TRS_CK(cudaGraphLaunch(g.exec, stream));
    ctx->stage_valid = true;
    ctx->stage_frames = first[1];
    ctx->last_kernels = parts * kKernelsPerBatch;
    return TRS_OK;
    TRS_GUARD_END
}

size_t batch_blob_bytes(int nf) {
    return align256((size_t)nf * sizeof(DevFrame)) + 5 * align256((size_t)(nf + 1) * 4) +
           align256((size_t)nf * sizeof(ColChunk));
}

ColGeom col_uniform(LaunchArgs &a, const HostPlan &hp, int nf, const SearchTune &t) {
    const int fpw = nf == 1 ? 1 : col_fpw(hp.n, t);
    a.cchunks = nullptr;
    a.col_fpw = fpw;
    a.col_nchunks = (nf + fpw - 1) / fpw;
    ColGeom g;
    g.units = (int)hp.win_a.size() * a.col_nchunks;
    g.add(hp.C, hp.n, hp.max_edge_vals, fpw);
    return g;
}

void set_search_scratch(DevFrame &f, const PlanEntry &pe, uint8_t *p, int n, float lambda) {
    f.plan = pe.dev;
    f.C = pe.host.C;
    f.R = pe.host.R;
    f.n = n;
    f.lambda_q = lambda_to_q(lambda);
    f.V1 = (uint64_t *)(p + pe.scr.V1);
    f.V2 = (uint64_t *)(p + pe.scr.V2);
    f.wres1 = (uint64_t *)(p + pe.scr.w1);
    f.wres2 = (uint64_t *)(p + pe.scr.w2);
    f.H2 = (uint64_t *)(p + pe.scr.H2);
    f.codes = (WinCode *)(p + pe.scr.codes);
}

void batch_describe(BatchLaunch &bl, uint8_t *hb, uint8_t *db, int nf, PlanEntry *const *pe, uint32_t *flags_dev,
                    uint64_t *scal_dev, const SearchTune &tune) {
    bl.hb = hb;
    bl.db = db;
    bl.nf = nf;
    bl.fr_bytes = align256((size_t)nf * sizeof(DevFrame));
    bl.pre_bytes = align256((size_t)(nf + 1) * 4);
    bl.blob = batch_blob_bytes(nf);
    bl.flags_dev = flags_dev;
    bl.scal_dev = scal_dev;
    int32_t *pc = (int32_t *)(hb + bl.fr_bytes), *pg = (int32_t *)(hb + bl.fr_bytes + bl.pre_bytes);
    int32_t *pi = (int32_t *)(hb + bl.fr_bytes + 2 * bl.pre_bytes);
    int32_t *pw = (int32_t *)(hb + bl.fr_bytes + 3 * bl.pre_bytes);
    int32_t *pb = (int32_t *)(hb + bl.fr_bytes + 4 * bl.pre_bytes);
    pc[0] = pg[0] = pi[0] = pw[0] = pb[0] = 0;
    bl.maxC = bl.maxR = bl.maxN = 1;
    bl.maxND = 0;
    for (int i = 0; i < nf; ++i) {
        const HostPlan &hp = pe[i]->host;
        pc[i + 1] = pc[i] + hp.C * hp.R;
        pg[i + 1] = pg[i] + (num_bands(hp.C) + kBandsPerBlock - 1) / kBandsPerBlock;
        pi[i + 1] = pi[i] + (int)hp.items.size();
        pw[i + 1] = pw[i] + (int)hp.win_a.size();
        pb[i + 1] = pb[i] + hp.nb;
        bl.maxC = hp.C > bl.maxC ? hp.C : bl.maxC;
        bl.maxR = hp.R > bl.maxR ? hp.R : bl.maxR;
        bl.maxN = hp.n > bl.maxN ? hp.n : bl.maxN;
        bl.maxND = hp.max_nd > bl.maxND ? hp.max_nd : bl.maxND;
    }
    bl.ctus = pc[nf];
    bl.groups = pg[nf];
    bl.bands = pb[nf];
    bl.windows = pw[nf];
    bl.uniform = 1;
    for (int i = 1; i < nf && bl.uniform; ++i) bl.uniform = pe[i] == pe[0];
    if (nf > 0) {
        bl.u_ctus = pc[1];
        bl.u_groups = pg[1];
        bl.u_items = pi[1];
        bl.u_windows = pw[1];
        bl.u_bands = pb[1];
    }
    // column DP: runs of consecutive frames with one plan, cut into chunks
    // of as many frames as one warp takes
    bl.col = ColGeom{};
    bl.col_chunks_dev = nullptr;
    if (nf > 0 && bl.uniform) {
        LaunchArgs a{};
        a.nframes = nf;
        bl.col = col_uniform(a, pe[0]->host, nf, tune);
        bl.col_nchunks = a.col_nchunks;
        bl.col_fpw = a.col_fpw;
        return;
    }
    const size_t ch_off = bl.fr_bytes + 5 * bl.pre_bytes;
    ColChunk *ch = (ColChunk *)(hb + ch_off);
    int nch = 0, unit = 0;
    for (int i = 0; i < nf;) {
        const HostPlan &hp = pe[i]->host;
        const int fpw = col_fpw(hp.n, tune);
        int cnt = 1;
        while (cnt < fpw && i + cnt < nf && pe[i + cnt] == pe[i]) ++cnt;
        ch[nch] = ColChunk{i, cnt, fpw, unit};
        unit += (int)hp.win_a.size();
        bl.col.add(hp.C, hp.n, hp.max_edge_vals, fpw);
        ++nch;
        i += cnt;
    }
    bl.col.units = unit;
    bl.col_nchunks = nch;
    bl.col_fpw = 0;
    bl.col_chunks_dev = (const ColChunk *)(db + ch_off);
}

cudaError_t batch_enqueue_work(const BatchLaunch &bl, cudaStream_t cs, cudaEvent_t *stage, cudaEvent_t after_texture) {
    LaunchArgs a{};
    a.frames = (const DevFrame *)bl.db;
    a.nframes = bl.nf;
    a.pre.ctus = (const int32_t *)(bl.db + bl.fr_bytes);
    a.pre.bandgrp = (const int32_t *)(bl.db + bl.fr_bytes + bl.pre_bytes);
    a.pre.items = (const int32_t *)(bl.db + bl.fr_bytes + 2 * bl.pre_bytes);
    a.pre.windows = (const int32_t *)(bl.db + bl.fr_bytes + 3 * bl.pre_bytes);
    a.pre.bands = (const int32_t *)(bl.db + bl.fr_bytes + 4 * bl.pre_bytes);
    if (bl.uniform) {
        a.uniform = 1;
        a.single_ctus = bl.u_ctus;
        a.single_bandgrp = bl.u_groups;
        a.single_items = bl.u_items;
        a.single_windows = bl.u_windows;
        a.single_bands = bl.u_bands;
    }
    a.cchunks = bl.col_chunks_dev;
    a.col_nchunks = bl.col_nchunks;
    a.col_fpw = bl.col_fpw;
    const bool events = stage != nullptr;
    auto mark = [&](int i, cudaError_t e) {
        if (events && e == cudaSuccess) e = record_event(stage[i], cs);
        return e;
    };
    cudaError_t e = cudaMemsetAsync(bl.flags_dev, 0, (size_t)bl.nf * 4, cs);
    e = mark(0, e);
    if (e == cudaSuccess) e = (cudaError_t)launch_texture(a, bl.ctus, cs);
    e = mark(1, e);
    if (e == cudaSuccess && after_texture) e = cudaEventRecord(after_texture, cs);
    if (e == cudaSuccess) e = (cudaError_t)launch_tables(a, bl.groups, bl.maxC, bl.maxR, cs);
    e = mark(2, e);
    if (e == cudaSuccess)
        e = (cudaError_t)launch_search(a, bl.bands, bl.windows, bl.maxC, bl.maxR, bl.maxN, bl.scal_dev,
                                       (size_t)bl.nf * 4, cs, bl.col, events ? stage + 3 : nullptr, &bl.tune, 3,
                                       bl.maxND);
    return e;
}

cudaError_t batch_enqueue(const BatchLaunch &bl, cudaStream_t cs, cudaEvent_t copied, cudaEvent_t *stage) {
    cudaError_t e = cudaMemcpyAsync(bl.db, bl.hb, bl.blob, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && copied) e = record_event(copied, cs);
    if (e == cudaSuccess) e = batch_enqueue_work(bl, cs, stage, nullptr);
    return e;
}

}  // namespace trs

extern "C" {

int trs_batch_decide(trs_ctx *ctx, const trs_frame_desc *fd, int nf, trs_partition *out, void *stream) {
    return batch_run(ctx, fd, nf, out, (cudaStream_t)stream, true);
}

int trs_autotune(trs_ctx *ctx, const trs_frame_desc *fd, int nf, trs_tune_report *rep, void *stream) {
    TRS_GUARD_BEGIN
    if (!ctx || !fd || !rep || nf < 1 || nf > ctx->o.max_batch) return TRS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    TRS_TRY(dev_alloc(ctx->hb_out, (size_t)ctx->o.max_batch * sizeof(trs_partition), &ctx->total));
    static const int bws[3] = {2, 4, 8};
    static const int cws[3] = {1, 2, 4};
    static const int cbs[2] = {4, 8};
    const SearchTune keep = ctx->tune;
    SearchTune cand[6];
    for (int j = 0; j < 6; ++j) {
        cand[j].band_warps = bws[j % 3];
        cand[j].col_warps = cws[j / 2];
        cand[j].col_batch = cbs[j % 2];
    }
    float rows[6], cols[6];
    for (int j = 0; j < 6; ++j) rows[j] = cols[j] = 1e30f;
    // one warm-up round, then three timed rounds; the fastest time of each candidate counts
    for (int round = 0; round < 4; ++round)
        for (int j = 0; j < 6; ++j) {
            ctx->tune = cand[j];
            int rc = batch_run(ctx, fd, nf, (trs_partition *)ctx->hb_out.p, s, false);
            if (rc != TRS_OK) {
                ctx->tune = keep;
                return rc;
            }
            float ms[trs_ctx::kStages] = {};
            if (trs_batch_stage_ms(ctx, ms, trs_ctx::kStages) != trs_ctx::kStages) {
                ctx->tune = keep;
                return cuda_fail(cudaErrorUnknown, "autotune stage events");
            }
            if (round == 0) continue;
            rows[j] = std::fmin(rows[j], ms[2] + ms[4]);
            cols[j] = std::fmin(cols[j], ms[3] + ms[5]);
        }
    int jb = 0, jc = 0;
    for (int j = 1; j < 6; ++j) {
        if (rows[j] < rows[jb]) jb = j;
        if (cols[j] < cols[jc]) jc = j;
    }
    ctx->tune.band_warps = cand[jb].band_warps;
    ctx->tune.col_warps = cand[jc].col_warps;
    ctx->tune.col_batch = cand[jc].col_batch;
    drop_graphs(ctx);  // graphs are captured again with the chosen shapes
    rep->band_warps = ctx->tune.band_warps;
    rep->col_warps = ctx->tune.col_warps;
    rep->col_batch = ctx->tune.col_batch;
    rep->n_candidates = 6;
    for (int j = 0; j < 6; ++j) {
        rep->cand_band_warps[j] = cand[j].band_warps;
        rep->cand_col_warps[j] = cand[j].col_warps;
        rep->cand_col_batch[j] = cand[j].col_batch;
        rep->rows_ms[j] = rows[j];
        rep->cols_ms[j] = cols[j];
    }
    return TRS_OK;
    TRS_GUARD_END
}

int trs_set_window_step(trs_ctx *ctx, int step) {
    if (!ctx || step < 1 || step > 64) return TRS_EINVAL;
    ctx->window_step = step;
    drop_graphs(ctx);
    return TRS_OK;
}

int trs_set_tune(trs_ctx *ctx, int band_warps, int col_warps, int col_batch) {
    auto ok_w = [](int w) { return w == 2 || w == 4 || w == 8; };
    if (!ctx || !ok_w(band_warps) || !(col_warps == 1 || ok_w(col_warps)) || (col_batch != 4 && col_batch != 8))
        return TRS_EINVAL;
    ctx->tune.band_warps = band_warps;
    ctx->tune.col_warps = col_warps;
    ctx->tune.col_batch = col_batch;
    drop_graphs(ctx);
    return TRS_OK;
}

int trs_batch_stage_frames(const trs_ctx *ctx) { return ctx && ctx->stage_valid ? ctx->stage_frames : 0; }

int trs_batch_kernels(const trs_ctx *ctx) { return ctx && ctx->stage_valid ? ctx->last_kernels : 0; }

int trs_set_batch_parts(trs_ctx *ctx, int parts) {
    if (!ctx || parts < 1 || parts > kMaxParts) return TRS_EINVAL;
    ctx->parts = parts;
    return TRS_OK;
}

int trs_batch_stage_ms(trs_ctx *ctx, float *ms, int max_stages) {
    if (!ctx || !ms || max_stages < 1) return 0;
    if (!ctx->stage_valid) return 0;
    if (cudaEventSynchronize(ctx->stage[trs_ctx::kStages]) != cudaSuccess) return 0;
    int k = 0;
    for (; k < trs_ctx::kStages && k < max_stages; ++k) {
        float v = 0.0f;
        if (cudaEventElapsedTime(&v, ctx->stage[k], ctx->stage[k + 1]) != cudaSuccess) return k;
        ms[k] = v;
    }
    return k;
}

int trs_batch_decide_host(trs_ctx *ctx, const trs_frame_desc *fd, int nf, trs_partition *out_host, void *stream) {
    TRS_GUARD_BEGIN
    if (!ctx || !fd || !out_host || nf < 1 || nf > ctx->o.max_batch) return TRS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<size_t> lo(nf), to(nf), dp(nf);
    size_t lb = 0, tb = 0;
    for (int i = 0; i < nf; ++i) {
        const trs_frame_desc &d = fd[i];
        if (!d.luma_dev || !d.ctu_time_dev) return TRS_EINVAL;
        TRS_TRY(check_frame(ctx, d.width, d.height));
        if (!fmt_ok(d.bit_depth)) return TRS_EINVAL;
        if (d.pitch_bytes < fmt_row_bytes(d.width, d.bit_depth)) return TRS_EINVAL;
        dp[i] = (fmt_row_bytes(d.width, d.bit_depth) + 15) & ~size_t(15);  // the vector path needs 16-byte rows
        lo[i] = lb;
        lb += dp[i] * d.height;
        to[i] = tb;
        tb += align256((size_t)((d.width + kCtu - 1) / kCtu) * ((d.height + kCtu - 1) / kCtu) * 4);
    }
    TRS_TRY(dev_alloc(ctx->hb_luma, lb, &ctx->total));
    TRS_TRY(dev_alloc(ctx->hb_time, tb, &ctx->total));
    TRS_TRY(dev_alloc(ctx->hb_out, (size_t)ctx->o.max_batch * sizeof(trs_partition), &ctx->total));
    std::vector<trs_frame_desc> dd(fd, fd + nf);
    for (int i = 0; i < nf; ++i) {
        const trs_frame_desc &d = fd[i];
        uint8_t *dl = (uint8_t *)ctx->hb_luma.p + lo[i];
        uint8_t *dt = (uint8_t *)ctx->hb_time.p + to[i];
        const size_t cells = (size_t)((d.width + kCtu - 1) / kCtu) * ((d.height + kCtu - 1) / kCtu);
        TRS_CK(copy_rows_h2d(dl, dp[i], d.luma_dev, d.pitch_bytes, fmt_row_bytes(d.width, d.bit_depth), d.height, s));
        TRS_CK(cudaMemcpyAsync(dt, d.ctu_time_dev, cells * 4, cudaMemcpyHostToDevice, s));
        dd[i].luma_dev = dl;
        dd[i].pitch_bytes = dp[i];
        dd[i].ctu_time_dev = (const float *)dt;
    }
    TRS_TRY(batch_run(ctx, dd.data(), nf, (trs_partition *)ctx->hb_out.p, s, true));
    TRS_CK(cudaMemcpyAsync(out_host, ctx->hb_out.p, (size_t)nf * sizeof(trs_partition), cudaMemcpyDeviceToHost, s));
    TRS_CK(cudaStreamSynchronize(s));
    return TRS_OK;
    TRS_GUARD_END
}

}  // extern "C"
