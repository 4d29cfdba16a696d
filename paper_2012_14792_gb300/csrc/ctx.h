// Host-side state of a trs_ctx and the helpers shared by api.cu and
// server.cu.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <map>
#include <tuple>
#include <vector>

#include <new>
#include <system_error>

#include "plan.h"
#include "trs_internal.cuh"

#define TRS_CK(call)                                                  \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::trs::cuda_fail(e_, #call);    \
    } while (0)

// Host allocation or thread start-up failures end an entry point with
// TRS_ENOMEM instead of unwinding into its C caller.
#define TRS_GUARD_BEGIN try {
#define TRS_GUARD_END                                       \
    }                                                       \
    catch (const std::bad_alloc &) { return TRS_ENOMEM; }   \
    catch (const std::system_error &) { return TRS_ENOMEM; }

#define TRS_TRY(expr)                \
    do {                             \
        int s_ = (expr);             \
        if (s_ != TRS_OK) return s_; \
    } while (0)

namespace trs {

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
};

struct PlanEntry {
    HostPlan host;
    DevBuf blob;
    const DevPlan *dev = nullptr;
    SearchScratch scr{};
};

struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    size_t staged_bytes = 0;
};

constexpr int kKernelsPerBatch = 9;  // texture, tables, 2 x (rows, columns), rebuild walk, cut bits, finish
constexpr int kMaxParts = 4;         // most chunks a captured batch is pipelined in
constexpr int kChunkMin = 4;         // fewest frames in a chunk

}  // namespace trs

namespace trs {
// Per-call arguments of a multi-tile search, read by its kernels from device memory.
struct MtCall {
    const uint8_t *tables;
    trs_mt_partition *out;
    uint32_t lambda_q;
    uint32_t reserved;
};

// The multi-tile candidate list of one frame shape, on the device, and the
// captured graphs of its search: kMtSlots copies, each copying the per-call
// arguments from its own pinned block, used in turn so that a call waits
// only for the call kMtSlots before it to have read its block.
constexpr int kMtSlots = 4;
struct MtEntry {
    DevBuf cands;        // count * n words: slice i of set c at i * count + c, its rectangle-table entry
    int64_t count = 0;
    DevBuf work;         // MtCall, T_min, and the second pass's per-block (Q, set) minima
    MtCall *call_host = nullptr;  // pinned, kMtSlots blocks
    cudaGraphExec_t graph[kMtSlots] = {};
    cudaEvent_t copied[kMtSlots] = {};  // graph s has read call_host[s]
    int next = 0;
};
}  // namespace trs

struct trs_ctx {
    trs_opts o{};
    size_t total = 0;
    int maxC = 0, maxR = 0;
    // one-frame path
    trs::DevBuf s1, s2, cnt, vmax, flags, tables, scratch, scal, part, luma_stage, time_stage;
    // plans by (W, H, n, window step)
    std::map<std::tuple<int, int, int, int>, trs::PlanEntry *> plans;
    int window_step = 1;  // 1: exact search; > 1: every window_step-th area window (trs_set_window_step)
    // batched path
    trs::DevBuf arena, desc;
    void *staging = nullptr;  // pinned host copy of the descriptor blob
    size_t staging_n = 0;
    cudaStream_t cap = nullptr, cap2 = nullptr;  // capture streams (second: the batch's second half)
    cudaEvent_t copied = nullptr, join = nullptr;
    cudaEvent_t tex_done[trs::kMaxParts] = {};  // chunk c's texture kernel has run
    static constexpr int kStages = 8;
    cudaEvent_t stage[kStages + 1] = {};  // timing events recorded inside batch graphs
    bool stage_valid = false;
    int stage_frames = 0;  // frames the stage events covered
    int last_kernels = 0;  // kernels the most recent batched call launched
    int parts = 2;         // chunks of a captured batch (trs_set_batch_parts)
    // host-buffer batches: device staging of planes, times and partitions
    trs::DevBuf hb_luma, hb_time, hb_out;
    trs::SearchTune tune;  // launch shapes of the search kernels (trs_autotune)
    std::map<std::vector<int64_t>, trs::BatchGraph> graphs;
    // multi-tile search: candidate lists by (W, H, n), and its three result words
    std::map<std::tuple<int, int, int>, trs::MtEntry *> mt;
    cudaStream_t mt_cap = nullptr;  // capture stream of the multi-tile graphs
};

namespace trs {

// Records the CUDA error text for trs_last_error(); returns TRS_ECUDA.
int cuda_fail(cudaError_t e, const char *what);
// Grows a device buffer to at least `bytes` (synchronising the device first
// if it must free the old one); *total tracks the context's bytes.
int dev_alloc(DevBuf &b, size_t bytes, size_t *total);
void dev_free(DevBuf &b);
uint32_t lambda_to_q(float lambda);
int check_frame(const trs_ctx *ctx, int W, int H);
int get_plan(trs_ctx *ctx, int W, int H, int n, PlanEntry **out);
size_t stats_bytes(int C, int R);
void drop_graphs(trs_ctx *ctx);
// Launch geometry of one batch: the descriptor blob (DevFrame[nf] and the
// work prefix sums) written in pinned host memory hb, to be copied to db.
struct BatchLaunch {
    uint8_t *hb = nullptr, *db = nullptr;
    size_t blob = 0, fr_bytes = 0, pre_bytes = 0;
    int nf = 0, ctus = 0, groups = 0, bands = 0, windows = 0, maxC = 1, maxR = 1, maxN = 1, maxND = 0;
    // every frame has the same plan: the work units of one frame
    int uniform = 0, u_ctus = 0, u_groups = 0, u_items = 0, u_windows = 0, u_bands = 0;
    uint32_t *flags_dev = nullptr;  // nf words, zeroed by the launch
    uint64_t *scal_dev = nullptr;   // nf * 4 words, reset by the launch
    SearchTune tune;
    // column DP: chunks of frames that share a plan (device table in the blob unless uniform)
    ColGeom col;
    int col_nchunks = 0, col_fpw = 1;
    const ColChunk *col_chunks_dev = nullptr;
};
size_t batch_blob_bytes(int nf);
// Column-DP units of nf frames that all use plan hp (a's col_* fields are set).
ColGeom col_uniform(LaunchArgs &a, const HostPlan &hp, int nf, const SearchTune &t);
// Points a frame's search fields at the plan and at the scratch starting at p.
void set_search_scratch(DevFrame &f, const PlanEntry &pe, uint8_t *p, int n, float lambda);
// Writes the work prefix sums and the column-DP chunks after the DevFrame
// array already placed in hb (frames that share a plan are grouped into
// chunks when they are consecutive there).
void batch_describe(BatchLaunch &bl, uint8_t *hb, uint8_t *db, int nf, PlanEntry *const *pe, uint32_t *flags_dev,
                    uint64_t *scal_dev, const SearchTune &tune);
// Enqueues the descriptor copy (then records `copied`), the flag reset and
// every kernel of the hot path on cs; stage events (9) when stage != nullptr.
cudaError_t batch_enqueue(const BatchLaunch &bl, cudaStream_t cs, cudaEvent_t copied, cudaEvent_t *stage);
// The same without the descriptor copy; records after_texture (if given)
// once the texture kernel is enqueued.
cudaError_t batch_enqueue_work(const BatchLaunch &bl, cudaStream_t cs, cudaEvent_t *stage, cudaEvent_t after_texture);


// Host-to-device copy of `rows` rows of `width` bytes: one linear copy when
// both pitches equal the width (the driver's 2-D copy of rows that are not
// a multiple of its transfer size runs at half the link rate), else 2-D.
inline cudaError_t copy_rows_h2d(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width,
                                 size_t rows, cudaStream_t s) {
    if (dpitch == width && spitch == width)
        return cudaMemcpyAsync(dst, src, width * rows, cudaMemcpyHostToDevice, s);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyHostToDevice, s);
}

// Releases a multi-tile entry (device list, work area, pinned block, graph).
void mt_free(MtEntry *me);

// Decides nf frames described by device pointers in one launch of each
// kernel on `stream`, through a cached CUDA graph or by direct launches.
int batch_run(trs_ctx *ctx, const trs_frame_desc *fd, int nf, trs_partition *out, cudaStream_t stream,
              bool use_graph);

}  // namespace trs
