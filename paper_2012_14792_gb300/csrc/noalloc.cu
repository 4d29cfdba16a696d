// trs_search_noalloc: trs_search for callers that must not allocate memory.
//
// Some callers cannot call cudaMalloc: real-time loops where the implicit
// device synchronisation of cudaMalloc/cudaFree would stall the pipeline,
// and hosts that hand all device memory to their own pool allocator and
// forbid stray allocations.
// This entry point needs no context: its search plan and scratch live in
// one file-scope device array of fixed size, and it makes no cudaMalloc /
// cudaFree call and no call of an allocating library routine (host-side it
// uses static storage only).
//
// Limits and sharing:
//  * kNoAllocBytes (8 MiB) holds the plan and scratch of one frame; a frame
//    shape whose needs exceed it is rejected with TRS_ENOMEM.  A 3840x2160
//    frame with n = 16 needs about 2.5 MiB.
//  * Every GPU that loads the library keeps this array until the process
//    exits.
//  * All calls on a device share the array and it keeps the last call's
//    contents.  The words that must start at +infinity (T_min, Q*) are reset
//    by every call; everything else is written before it is read.  Calls
//    whose work overlaps on the GPU (other streams, or several host threads)
//    race on the array: serialise them.
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current).
//  * A call whose shape (W, H, n, k) differs from the one the array holds
//    (the first call included) writes the new plan over the old one: a
//    cudaMemcpyAsync on the call's stream from static, pageable host
//    storage.  The copy is ordered after earlier work on that stream only,
//    not on other streams, so the kernels of every earlier call with another
//    shape must have finished first.  Until the copy is enqueued the device
//    keeps no shape: a failed copy leaves the next call to copy its plan
//    again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "trs_internal.cuh"

using namespace trs;

namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// static host storage (no heap): the plan is laid out here, then copied
alignas(256) unsigned char g_host_plan[kNoAllocBytes];
uint64_t g_areas[4 * kMaxC * kMaxR];
std::mutex g_mu;

struct DeviceSlot {
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch on this device
    int W = -1, H = -1, n = -1, k = -1;  // shape whose plan the array holds
    size_t plan_bytes = 0;
    int nwin = 0, nitems = 0, nb = 0, C = 0, R = 0, max_edge_vals = 1;
};
DeviceSlot g_dev[kMaxDevices];

// Distinct pixel lengths of runs of whole CTUs [i, j) (last CTU clipped), sorted.
int extents(int cells, int total, uint32_t *out) {
    int m = 0;
    for (int i = 0; i < cells; ++i)
        for (int j = i + 1; j <= cells; ++j) out[m++] = line_px(j, total) - line_px(i, total);
    std::sort(out, out + m);
    return (int)(std::unique(out, out + m) - out);
}

// Lays the plan of (W, H, n, k) out in g_host_plan, addressed for a copy at
// dev_base.  It is the unpruned form of the context path's plan: the same
// area windows, but every tile column a window admits (no slice-count,
// tiling or reachability pruning), slice counts 1..min(n, R, H / hlo) for
// every item and no per-item staging bound.  The search then relaxes
// options no partition uses, at a cost in time, and returns the same
// result.  Returns TRS_ENOMEM if plan + scratch exceed kNoAllocBytes.
int layout_plan(int W, int H, int n, int k, unsigned char *dev_base, DeviceSlot *s) {
    const int C = (W + kCtu - 1) / kCtu, R = (H + kCtu - 1) / kCtu;
    static uint32_t ws[kMaxC * (kMaxC + 1) / 2], hs[kMaxR * (kMaxR + 1) / 2];
    const int nw = extents(C, W, ws), nh = extents(R, H, hs);
    const uint64_t A = (uint64_t)W * (uint64_t)H;
    int na = 0;
    for (int i = 0; i < nw; ++i)
        for (int j = 0; j < nh; ++j) {
            const uint64_t a = (uint64_t)ws[i] * hs[j];
            if (a * (uint64_t)n <= A && ((uint64_t)k * a - 1) * (uint64_t)n >= A) g_areas[na++] = a;
        }
    std::sort(g_areas, g_areas + na);
    const int nwin = (int)(std::unique(g_areas, g_areas + na) - g_areas);
    const int nb = num_bands(C);

    size_t off = align256(sizeof(DevPlan));
    const size_t off_win = off;
    off = align256(off + (size_t)nwin * 8 + 8);
    const size_t off_slot = off;
    off = align256(off + (size_t)nwin * nb * 4 + 4);
    const size_t off_x0 = off;
    off = align256(off + (size_t)nb * 2 + 2);
    const size_t off_x1 = off;
    off = align256(off + (size_t)nb * 2 + 2);
    const size_t off_bi = off;
    off = align256(off + (size_t)(nb + 1) * 4 + 4);
    const size_t off_items = off;
    if (off_items > kNoAllocBytes) return TRS_ENOMEM;

    std::memcpy(g_host_plan + off_win, g_areas, (size_t)nwin * 8);
    int32_t *slot = reinterpret_cast<int32_t *>(g_host_plan + off_slot);
    int16_t *bx0 = reinterpret_cast<int16_t *>(g_host_plan + off_x0);
    int16_t *bx1 = reinterpret_cast<int16_t *>(g_host_plan + off_x1);
    int32_t *bitems = reinterpret_cast<int32_t *>(g_host_plan + off_bi);
    PlanItem *items = reinterpret_cast<PlanItem *>(g_host_plan + off_items);
    const size_t item_cap = (kNoAllocBytes - off_items) / sizeof(PlanItem);
    for (size_t i = 0; i < (size_t)nwin * nb; ++i) slot[i] = -1;
    int nitems = 0;
    for (int x0 = 0; x0 < C; ++x0)
        for (int x1 = x0 + 1; x1 <= C; ++x1) {
            const int b = band_index(C, x0, x1);
            bx0[b] = (int16_t)x0;
            bx1[b] = (int16_t)x1;
        }
    for (int b = 0; b < nb; ++b) {
        bitems[b] = nitems;
        const uint64_t wb = line_px(bx1[b], W) - line_px(bx0[b], W);
        int prev_lo = -1, prev_hi = -1, prev_slot = -1;
        for (int wi = 0; wi < nwin; ++wi) {
            const uint64_t lo = g_areas[wi], hi = (uint64_t)k * lo - 1;
            int ilo = 0;
            while (ilo < nh && wb * hs[ilo] < lo) ++ilo;
            int ihi = nh - 1;
            while (ihi >= 0 && wb * hs[ihi] > hi) --ihi;
            if (ilo > ihi) continue;
            if (ilo != prev_lo || ihi != prev_hi) {
                if ((size_t)nitems >= item_cap) return TRS_ENOMEM;
                PlanItem &it = items[nitems];
                it.b = b;
                it.w_first = wi;
                it.hlo = hs[ilo];
                it.hhi = hs[ihi];
                it.kmax = std::min(std::min(n, R), (int)(H / it.hlo));
                it.kmin = 1;
                prev_lo = ilo;
                prev_hi = ihi;
                prev_slot = nitems++;
            }
            slot[(size_t)wi * nb + b] = prev_slot;
            items[prev_slot].w_last = wi;
        }
    }
    bitems[nb] = nitems;
    // the column DP's step entries of every (window, band), after the items
    const size_t off_sk = align256(off_items + (size_t)nitems * sizeof(PlanItem) + 16);
    if (off_sk + (size_t)nwin * nb * 8 + 8 > kNoAllocBytes) return TRS_ENOMEM;
    uint64_t *sk = reinterpret_cast<uint64_t *>(g_host_plan + off_sk);
    int max_edge_vals = 1;
    for (int wi = 0; wi < nwin; ++wi)
        for (int x = 0; x < C; ++x) {
            int vals = 0;
            for (int x1 = x + 1; x1 <= C; ++x1) {
                const int b = band_index(C, x, x1);
                const int sl = slot[(size_t)wi * nb + b];
                uint64_t e = 0;
                if (sl >= 0 && items[sl].kmax >= 1) {
                    e = pack_slot_k(sl, 1, items[sl].kmax);
                    vals += items[sl].kmax;
                }
                sk[(size_t)wi * nb + b] = e;
            }
            max_edge_vals = std::max(max_edge_vals, vals);
        }
    const size_t plan_bytes = align256(off_sk + (size_t)nwin * nb * 8 + 8);
    // scratch of the search after the plan
    const size_t v = (size_t)nitems * (n + 1) * 8;
    const size_t need = plan_bytes + 2 * align256(v + 8) + 2 * align256((size_t)nwin * 8 + 8) +
                        align256((size_t)nwin * (C + 1) * (n + 1) * 8 + 8) +
                        align256((size_t)nwin * sizeof(WinCode) + 8) + align256(4 * 8);
    if (need > kNoAllocBytes) return TRS_ENOMEM;

    DevPlan d;
    d.W = W;
    d.H = H;
    d.C = C;
    d.R = R;
    d.n = n;
    d.k = k;
    d.nb = nb;
    d.nwin = nwin;
    d.nitems = nitems;
    d.A = A;
    d.win_a = reinterpret_cast<const uint64_t *>(dev_base + off_win);
    d.items = reinterpret_cast<const PlanItem *>(dev_base + off_items);
    d.slot_of = reinterpret_cast<const int32_t *>(dev_base + off_slot);
    d.band_x0 = reinterpret_cast<const int16_t *>(dev_base + off_x0);
    d.band_x1 = reinterpret_cast<const int16_t *>(dev_base + off_x1);
    d.band_items = reinterpret_cast<const int32_t *>(dev_base + off_bi);
    d.slot_k = reinterpret_cast<const uint64_t *>(dev_base + off_sk);
    d.max_edge_vals = max_edge_vals;
    std::memcpy(g_host_plan, &d, sizeof(d));
    s->plan_bytes = plan_bytes;
    s->nwin = nwin;
    s->nitems = nitems;
    s->nb = nb;
    s->C = C;
    s->R = R;
    s->max_edge_vals = max_edge_vals;
    return TRS_OK;
}

}  // namespace

extern "C" int trs_search_noalloc(const void *tables, int W, int H, int n, int k_area, float lambda,
                                  trs_partition *out, void *stream) {
    if (!tables || !out || (uintptr_t)tables % 256) return TRS_EINVAL;
    if (W <= 0 || H <= 0 || W > kCtu * kMaxC || H > kCtu * kMaxR) return TRS_EINVAL;
    if (n < 1 || n > kMaxN || k_area < 1) return TRS_EINVAL;
    if (!std::isfinite(lambda) || lambda < 0.0f || lambda > 1000.0f) return TRS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TRS_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSlot &s = g_dev[dev];
    if (!s.base) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TRS_ECUDA;
        if (prepare_search_kernels() != (int)cudaSuccess) return TRS_ECUDA;
        s.base = (unsigned char *)p;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (s.W != W || s.H != H || s.n != n || s.k != k_area) {
        DeviceSlot t = s;
        const int rc = layout_plan(W, H, n, k_area, s.base, &t);
        if (rc != TRS_OK) return rc;
        // the old plan is overwritten from here on: the slot holds no shape
        // until the new plan's copy is enqueued
        s.W = s.H = s.n = s.k = -1;
        if (cudaMemcpyAsync(s.base, g_host_plan, t.plan_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return TRS_ECUDA;
        t.W = W;
        t.H = H;
        t.n = n;
        t.k = k_area;
        s = t;
    }
    unsigned char *p = s.base + s.plan_bytes;
    const size_t v = align256((size_t)s.nitems * (n + 1) * 8 + 8);
    const size_t w = align256((size_t)s.nwin * 8 + 8);
    LaunchArgs a{};
    DevFrame &f = a.single;
    f.W = W;
    f.H = H;
    f.C = s.C;
    f.R = s.R;
    f.n = n;
    f.tables = (uint8_t *)tables;
    f.plan = reinterpret_cast<const DevPlan *>(s.base);
    f.lambda_q = (uint32_t)std::rint((double)lambda * 65536.0);
    f.V1 = reinterpret_cast<uint64_t *>(p);
    f.V2 = reinterpret_cast<uint64_t *>(p + v);
    f.wres1 = reinterpret_cast<uint64_t *>(p + 2 * v);
    f.wres2 = reinterpret_cast<uint64_t *>(p + 2 * v + w);
    f.H2 = reinterpret_cast<uint64_t *>(p + 2 * v + 2 * w);
    const size_t h2 = align256((size_t)s.nwin * (s.C + 1) * (n + 1) * 8 + 8);
    f.codes = reinterpret_cast<WinCode *>(p + 2 * v + 2 * w + h2);
    f.scal = reinterpret_cast<uint64_t *>(p + 2 * v + 2 * w + h2 + align256((size_t)s.nwin * sizeof(WinCode) + 8));
    f.out = out;
    a.nframes = 1;
    a.single_items = s.nitems;
    a.single_windows = s.nwin;
    a.single_bands = s.nb;
    a.col_nchunks = 1;
    a.col_fpw = 1;
    ColGeom cg;
    cg.units = s.nwin;
    cg.add(s.C, n, s.max_edge_vals, 1);
    // launch_search resets T_min and Q* to +infinity before its kernels
    if (launch_search(a, s.nb, s.nwin, s.C, s.R, n, f.scal, 4, stream, cg) != (int)cudaSuccess) return TRS_ECUDA;
    return TRS_OK;
}
