// a3-a5: the two search steps of Sec. 2.3 and the decoding of the winner.
//
// The candidate space S(n) (exactly n slices, slices are runs of whole CTU
// rows inside a tile, tiles on a CTU grid, k*A_min > A_max) is searched
// exactly, through two facts:
//  (i)  a tile-row cut adds no geometry: cutting every tile column at the
//       same line as slice boundaries gives the same slices, with a smaller
//       canonical code.  The winner therefore has one tile row, and the
//       search runs over tile columns ("bands"), each cut into slices;
//  (ii) the area rule holds iff all slice areas lie in a window [a, k*a-1]
//       for some slice area a.  Inside one window Eq. 1's max and Eq. 2's
//       sum separate over bands and, inside a band, over slices.
// For each window the search is a DP over bands of a DP over slice rows.
// Windows that give a band the same admissible slice heights share one row
// DP ("item" of the shape's plan); the plan also bounds each item's slice
// count by what the rest of the frame can hold (necessary conditions).
//
//  band_kernel<STEP,S>  one warp per (frame, tile column), running all of
//                       the column's items (two at a time for frames of at
//                       most 17 CTU rows): lanes are the start row y of the
//                       remaining rows [y, R); for k = 1..kmax it relaxes
//                       every admissible slice height d, reading
//                       G_{k-1}[y+d] from shared memory.  Step 1 combines
//                       with max (Eq. 1), step 2 with + (Eq. 2) and drops
//                       slices whose time exceeds the Eq. 4 bound.
//  column_kernel<STEP>  one warp per (window, frames sharing the plan): DP
//                       over tile-column right edges with lanes over
//                       (slice count m, frame); the candidate steps and
//                       their V values of the next left edge are staged in
//                       shared memory while the current one relaxes.
//                       Step 1's window minima reduce into T_min (Eq. 3),
//                       step 2's into Q*.
//  rebuild_kernel       one warp per (frame, window): in a window that
//                       reaches Q*, walks the smallest canonical code's
//                       tile columns (smallest next edge first); a column
//                       whose optimum one slice count completes is left
//                       pending, otherwise its smallest cut bits are chosen
//                       here with warp ballots.
//  cuts_kernel          the pending columns of a frame's tied codes, one
//                       warp each: the column's row DP with every layer
//                       kept, then its smallest cut bits.
//  finish_kernel        one warp per frame: the smallest code over windows,
//                       decoded into trs_partition.
#include <cuda_runtime.h>

#include <algorithm>

#include "trs_internal.cuh"

namespace trs {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarps = 8;    // largest warps per block of band_kernel / column_kernel (tunable)
// Saturating infinity inside the DPs: sums of a value below 2^44 and kSoft
// stay below 2^63, so the relaxations need no infinity branches.
constexpr uint64_t kSoft = 1ull << 62;

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }
__device__ __forceinline__ uint64_t hard_inf(uint64_t v) { return v >= kSoft ? kInf : v; }

template <typename VT>
struct Soft;  // saturating infinity of a value type
template <>
struct Soft<uint64_t> {
    static constexpr uint64_t v = kSoft;
};
template <>
struct Soft<uint32_t> {
    static constexpr uint32_t v = 1u << 31;  // step-1 values of a frame whose total time is below 2^31
};

__device__ __forceinline__ bool frame_t32(const DevFrame &fr) {
    const TablesOffsets off = tables_offsets(fr.C, fr.R);
    return reinterpret_cast<const int32_t *>(fr.tables + off.status)[3] != 0;
}

__device__ __forceinline__ int32_t frame_status(const DevFrame &fr) {
    const TablesOffsets off = tables_offsets(fr.C, fr.R);
    return *reinterpret_cast<const int32_t *>(fr.tables + off.status);
}

// Suffix row DP of one item for one warp.  After iteration k, lane y holds
// G_k[y] = best value of rows [y, R) of the band cut into k admissible
// slices.  Each lane first stages, for every slice height d in the item's
// range, the slice's value (time for step 1, floor-SSE for step 2) in
// shared memory and an admissibility bit; the k loop then only shuffles
// G_{k-1}[y+d] from lane y+d and relaxes.  Writes V[k] = G_k[0] (k = 1..n,
// kInf where no split exists) and, when asked, every layer into
// layers[k*32 + y].
template <int STEP>
__device__ void item_dp(const DevFrame &fr, const PlanItem &it, uint64_t thr, int n, uint64_t *V,
                        uint64_t *layers, uint64_t *stage, uint32_t *vm_out = nullptr) {
    const int lane = threadIdx.x & 31;
    const int R = fr.R, H = fr.H;
    const TablesOffsets off = tables_offsets(fr.C, R);
    const size_t base = (size_t)it.b * R * R;
    const uint64_t *RT = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_t) + base;
    const uint64_t *RQ = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_q) + base;
    // slice row counts that can reach a pixel height in [hlo, hhi]
    const int dmin = max(1, (int)((it.hlo + kCtu - 1) / kCtu));
    const int dmax = min(R, (int)(it.hhi / kCtu) + 1);
    const int nd = dmax - dmin + 1;
    const uint32_t ytop = line_px(lane, H);
    uint32_t vmask = 0;
#pragma unroll 4
    for (int i = 0; i < nd; ++i) {
        const int d = dmin + i, y1 = lane + d;
        const bool in = lane < R && y1 <= R;
        const size_t e = in ? (size_t)(d - 1) * R + lane : 0;
        // both words are loaded unconditionally so the loads of all heights overlap
        const uint64_t tv = __ldg(RT + e);
        const uint64_t qv = STEP == 2 ? __ldg(RQ + e) : 0ull;
        const uint32_t h = line_px(y1, H) - ytop;
        const bool ok = in && h >= it.hlo && h <= it.hhi && (STEP == 1 || tv <= thr);
        stage[i * 32 + lane] = STEP == 1 ? tv : qv;
        vmask |= (ok ? 1u : 0u) << i;
    }
    if (vm_out) vm_out[lane] = vmask;
    __syncwarp();
    // G_0: only the empty remainder (y = R) holds zero slices
    uint64_t G = (lane == R) ? 0ull : kSoft;
    if (layers) layers[lane] = hard_inf(G);
    for (int k = 1; k <= it.kmax; ++k) {
        const uint64_t edge = (k == 1) ? 0ull : kSoft;  // G_{k-1}[R] when R == 32 (no lane 32)
        uint64_t best = kSoft;
        for (int i = 0; i < nd; ++i) {
            const int src = lane + dmin + i;
            uint64_t prev = __shfl_sync(kFull, G, src & 31);
            if (src >= 32) prev = edge;
            if ((vmask >> i) & 1u) {
                const uint64_t val = stage[i * 32 + lane];
                const uint64_t c = STEP == 1 ? umax64(prev, val) : prev + val;
                best = umin64(best, c);
            }
        }
        G = umin64(best, kSoft);
        if (layers) layers[k * 32 + lane] = hard_inf(G);
        if (V) {
            const uint64_t g0 = __shfl_sync(kFull, G, 0);
            if (lane == 0) V[k] = hard_inf(g0);
        }
    }
    if (V && lane == 0) {
        V[0] = kInf;
        for (int k = it.kmax + 1; k <= n; ++k) V[k] = kInf;
    }
    __syncwarp();
}

// k loop of one item (see band_kernel), on values of type VT.  sv[i*32 + y]
// holds the value of the slice [y, y+dmin+i) with the saturating infinity
// for heights the item does not admit; G (64 words) holds G_{k-1}[y] for
// y = 0..63, the saturating infinity past the frame except G_0[R] = 0.
// Lane y reads G[y+d] (consecutive words, no bank conflicts), so a step is
// two shared loads, a max (step 1) or add (step 2) and a min.  Returns, in
// lane k (lane 0 for k = 32), V[k] = G_k[0] with kInf where no split exists.
template <int STEP, typename VT>
__device__ __forceinline__ uint64_t item_rows(const VT *sv, VT *G, int nd, int dmin, int kmax, int R) {
    const int lane = threadIdx.x & 31;
    constexpr VT soft = Soft<VT>::v;
    __syncwarp();  // every lane is done with the previous item's G
    G[lane] = lane == R ? VT(0) : soft;
    G[lane + 32] = lane + 32 == R ? VT(0) : soft;
    __syncwarp();
    uint64_t vreg = kInf;
    const VT *gp = G + lane + dmin;
    const VT *sp = sv + lane;
    for (int k = 1; k <= kmax; ++k) {
        VT best = soft;
#pragma unroll 4
        for (int i = 0; i < nd; ++i) {
            const VT prev = gp[i], val = sp[i * 32];
            const VT c = STEP == 1 ? (prev > val ? prev : val) : VT(prev + val);
            best = c < best ? c : best;
        }
        __syncwarp();
        G[lane] = best < soft ? best : soft;  // lanes at or past R find no slice: soft
        if (lane == 0) G[32] = soft;          // G_k[32] of a 32-row frame (k >= 1)
        __syncwarp();
        const VT g0 = G[0];
        if (lane == (k & 31)) vreg = g0 >= soft ? kInf : (uint64_t)g0;
    }
    return vreg;
}

// k >= 2 of item_pair for ND admitted heights or fewer in each half (ND a
// compile-time bound): the half's full-height slice values live in
// registers and the loop over heights is unrolled, so a relaxation step is
// one shared load, a max (step 1) or add (step 2) and a min.  Ga holds G_1
// on entry (G_1[16] included), Gb the saturating infinity at 16 and above.
// Both halves compute every k up to kmm (a half past its kmax is never
// read); lane k - 1 keeps G_k[0], returned raw.
template <int STEP, typename VT, int S, int ND>
__device__ __forceinline__ VT pair_rows(const uint64_t *stage, int nd, int dlo, int kmm, VT *Ga, VT *Gb, VT g0) {
    const int lane = threadIdx.x & 31, l = lane & 15, y = l;
    constexpr VT soft = Soft<VT>::v;
    VT v[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) v[i] = i < nd ? (VT)stage[(dlo + i - 1) * S + y] : soft;
    const int goff = y + dlo;
    auto step = [&](const VT *gp, VT *out, int k) {
        VT b0 = soft, b1 = soft;  // two independent minimum chains
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            const VT p = gp[i];
            const VT c = STEP == 1 ? (p > v[i] ? p : v[i]) : VT(p + v[i]);
            if (i & 1)
                b1 = c < b1 ? c : b1;
            else
                b0 = c < b0 ? c : b0;
        }
        const VT best = b0 < b1 ? b0 : b1;
        // step 1 combines with max, so values never pass the saturating
        // infinity; step 2's sums can, and are clamped
        out[y] = STEP == 1 ? best : (best < soft ? best : soft);
        __syncwarp();
        if (l == k - 1) g0 = out[0];
    };
    if (kmm < 2) return g0;
    step(Ga + goff, Gb, 2);
    // G_1's buffer takes G_3 next: its row 16 (G_1[16]) becomes empty
    if (l == 0) Ga[16] = soft;
    for (int k = 3; k <= kmm; ++k) {
        VT *t = Ga;
        Ga = Gb;
        Gb = t;
        step(Ga + goff, Gb, k);
    }
    return g0;
}

// The same for any number of heights: the values come from the per-half
// table sv (sv[i*32 + lane], filled by the caller).
template <int STEP, typename VT>
__device__ __forceinline__ VT pair_rows_any(const VT *sv, int ndm, int dlo, int kmm, VT *Ga, VT *Gb, VT g0) {
    const int lane = threadIdx.x & 31, l = lane & 15, y = l;
    constexpr VT soft = Soft<VT>::v;
    const VT *sp = sv + lane;
    auto step = [&](const VT *gp, VT *out, int k) {
        VT b0 = soft, b1 = soft;
        int i = 0;
#pragma unroll 2
        for (; i + 1 < ndm; i += 2) {
            const VT p0 = gp[i], v0 = sp[i * 32], p1 = gp[i + 1], v1 = sp[(i + 1) * 32];
            const VT c0 = STEP == 1 ? (p0 > v0 ? p0 : v0) : VT(p0 + v0);
            const VT c1 = STEP == 1 ? (p1 > v1 ? p1 : v1) : VT(p1 + v1);
            b0 = c0 < b0 ? c0 : b0;
            b1 = c1 < b1 ? c1 : b1;
        }
        if (i < ndm) {
            const VT p0 = gp[i], v0 = sp[i * 32];
            const VT c0 = STEP == 1 ? (p0 > v0 ? p0 : v0) : VT(p0 + v0);
            b0 = c0 < b0 ? c0 : b0;
        }
        const VT best = b0 < b1 ? b0 : b1;
        out[y] = STEP == 1 ? best : (best < soft ? best : soft);
        __syncwarp();
        if (l == k - 1) g0 = out[0];
    };
    if (kmm < 2) return g0;
    step(Ga + y + dlo, Gb, 2);
    if (l == 0) Ga[16] = soft;
    for (int k = 3; k <= kmm; ++k) {
        VT *t = Ga;
        Ga = Gb;
        Gb = t;
        step(Ga + y + dlo, Gb, k);
    }
    return g0;
}

constexpr int kNdRegs = 12;  // most admitted heights the register form of the row DP takes

// Two items of one tile column per warp, for frames of at most 17 CTU rows
// and n <= 16 (every workload of the paper): half h = lane / 16 runs one
// item with its lane l on start row y = l.
//  * A slice [y, y+d) that ends above the frame's last row is d full CTU
//    rows high, so the item admits it iff d lies in [dlo, dhi] (its pixel
//    range over 128).  The slice ending on the last row (possibly clipped)
//    only starts a 1-slice remainder: G_{k-1}[R] is empty for k >= 2.  So
//    G_1[y] is that one slice (if admitted) and, for k >= 2, lane y relaxes
//    d = dlo..dhi only.
//  * Row 16, the last row of a 17-row frame, needs no lane: G_1[16] is its
//    one-row slice and G_k[16] (k >= 2) is empty.
//  * G_{k-1} and G_k alternate between two 64-word buffers per half, one
//    warp barrier per k.
// Loops run to the larger of the two items' bounds (extra heights hold the
// saturating infinity), so both halves stay in step.  The staged values
// already hold the saturating infinity for slices past Eq. 4's bound (step
// 2).  Each half runs its item mi (none if mi is negative), described by it.
template <int STEP, typename VT, int S>
__device__ void item_pair(const DevFrame &fr, const DevPlan &pl, int mi, const PlanItem &it, uint64_t *Vall,
                          const uint64_t *stage, VT *sv, VT *G) {
    const int lane = threadIdx.x & 31, h = lane >> 4, l = lane & 15, y = l;
    const int n = pl.n, R = fr.R, H = fr.H;
    constexpr VT soft = Soft<VT>::v;
    // G_{k-1} in Ga, G_k into Gb, then swapped; half 1's pair sits 16 words
    // further so that the halves' 32-bit reads fall in different banks
    VT *Ga = G + h * 144, *Gb = Ga + 64;
    const bool have = mi >= 0;
    const int kmax = have ? it.kmax : 0;
    const int dlo = max(1, (int)((it.hlo + kCtu - 1) / kCtu));
    const int nd = have ? (int)(it.hhi / kCtu) - dlo + 1 : 0;  // full-height slices admitted (may be <= 0)
    const int ndm = max(nd, __shfl_xor_sync(kFull, nd, 16));
    const int kmm = max(kmax, __shfl_xor_sync(kFull, kmax, 16));
    __syncwarp();  // every lane is done with the previous pair's tables
    if (ndm > kNdRegs)
        for (int i = 0; i < ndm; ++i) sv[i * 32 + lane] = i < nd ? (VT)stage[(dlo + i - 1) * S + y] : soft;
    // G_1: the single slice [y, R), for y = l and for row 16
    auto last_slice = [&](int yy) -> VT {
        const uint32_t hh = (uint32_t)H - line_px(yy, H);
        return have && yy < R && hh >= it.hlo && hh <= it.hhi ? (VT)stage[(R - yy - 1) * S + yy] : soft;
    };
    // G_1 into Gb (row 16 included); every other word of both tables holds
    // the saturating infinity (G_0 is never read: k = 1 is closed-form)
    const VT g16 = last_slice(16);
    const VT g1 = last_slice(y);
    Gb[y] = g1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e = l + 16 * q;
        Ga[e] = soft;
        if (q) Gb[e] = soft;
    }
    if (l == 0) Gb[16] = g16;
    __syncwarp();
    VT g0 = l == 0 ? g1 : soft;  // lane k - 1 collects G_k[0]
    // k >= 2 relaxes only full-height slices: with none admitted in either
    // half G_k is empty for every k >= 2
#define TRS_ND_CASE(K) \
    case K: g0 = pair_rows<STEP, VT, S, K>(stage, nd, dlo, kmm, Gb, Ga, g0); break;
    if (ndm >= 1) {
        if (sizeof(VT) == 8) {
            // 64-bit values: even bounds only (an odd count runs one height
            // of the saturating infinity more), half the code to cache
            switch ((ndm + 1) & ~1) {
                TRS_ND_CASE(2) TRS_ND_CASE(4) TRS_ND_CASE(6) TRS_ND_CASE(8) TRS_ND_CASE(10) TRS_ND_CASE(12)
                default: g0 = pair_rows_any<STEP, VT>(sv, ndm, dlo, kmm, Gb, Ga, g0);
            }
        } else {
            switch (ndm) {
                TRS_ND_CASE(1) TRS_ND_CASE(2) TRS_ND_CASE(3) TRS_ND_CASE(4) TRS_ND_CASE(5) TRS_ND_CASE(6)
                TRS_ND_CASE(7) TRS_ND_CASE(8) TRS_ND_CASE(9) TRS_ND_CASE(10) TRS_ND_CASE(11) TRS_ND_CASE(12)
                default: g0 = pair_rows_any<STEP, VT>(sv, ndm, dlo, kmm, Gb, Ga, g0);
            }
        }
    }
#undef TRS_ND_CASE
    if (have) {
        uint64_t *V = Vall + (size_t)mi * (n + 1);
        if (l == 0) V[0] = kInf;
        const int kmin = pl.items[mi].kmin;  // read here: nothing extra stays live through the k loop
        // counts outside [kmin, kmax] complete no partition; "none" is kSoft
        // in step 2 (the column DP adds it)
        const int k = l + 1;
        if (l < n) V[k] = k >= kmin && k <= kmax && g0 < soft ? (uint64_t)g0 : (STEP == 1 ? kInf : kSoft);
    }
}

// The items of one tile column two at a time (see item_pair), the next
// pair's descriptions loaded while the current pair runs.  Step 2 runs only
// the items with a window whose step-1 best time meets Eq. 4 (no other
// window is read again): the frame's windows that meet it are first marked
// in a bit mask, then the live items listed in order in `list` and paired.
// A column has at most 2 x (distinct slice heights) <= 4R items, so
// kListMax entries hold them for R <= 17.
constexpr int kListMax = 128;
constexpr int kMaskWindows = 1024;  // windows the step-2 bit mask covers (more: tested per item)
template <int STEP, typename VT, int S>
__device__ void items_paired(const DevFrame &fr, const DevPlan &pl, int i0, int i1, uint64_t *Vall,
                             const uint64_t *stage, VT *sv, VT *G, int16_t *list, uint32_t *wmask,
                             uint64_t thr) {
    const int lane = threadIdx.x & 31, h = lane >> 4;
    int cnt = i1 - i0;
    if (STEP == 2) {
        const int nwin = pl.nwin;
        const bool masked = nwin <= kMaskWindows;
        if (masked) {
            for (int w0 = 0; w0 < nwin; w0 += 32) {
                const bool ok = w0 + lane < nwin && fr.wres1[w0 + lane] <= thr;
                const unsigned m = __ballot_sync(kFull, ok);
                if (lane == 0) wmask[w0 >> 5] = m;
            }
            __syncwarp();
        }
        cnt = 0;
        for (int base = i0; base < i1; base += 32) {
            bool live = false;
            if (base + lane < i1) {
                const PlanItem it = pl.items[base + lane];
                if (masked) {
                    for (int w = it.w_first; w <= it.w_last && !live; w = (w | 31) + 1) {
                        const int hi = min(it.w_last, w | 31);
                        const uint32_t bits = wmask[w >> 5] >> (w & 31);
                        const int span = hi - w + 1;  // 1..32
                        live = (span == 32 ? bits : bits & ((1u << span) - 1u)) != 0u;
                    }
                } else {
                    for (int w = it.w_first; w <= it.w_last && !live; ++w) live = fr.wres1[w] <= thr;
                }
            }
            const unsigned m = __ballot_sync(kFull, live);
            if (live) list[cnt + __popc(m & ((1u << lane) - 1u))] = (int16_t)(base + lane - i0);
            cnt += __popc(m);
        }
        __syncwarp();
    }
    auto item_at = [&](int j) { return j < cnt ? i0 + (STEP == 1 ? j : (int)list[j]) : -1; };
    PlanItem nxt{0, 0, 1u, 0u, 0, -1, 1, 0};
    int mnext = item_at(h);
    if (mnext >= 0) nxt = pl.items[mnext];
    for (int p = 0; p < cnt; p += 2) {
        const PlanItem cur = nxt;
        const int mi = mnext;
        mnext = item_at(p + 2 + h);
        if (mnext >= 0) nxt = pl.items[mnext];
        item_pair<STEP, VT, S>(fr, pl, mi, cur, Vall, stage, sv, G);
    }
}

// Row DPs, one warp per (frame, tile column): the column's slice values
// for every height d are staged once in shared memory (stage[(d-1)*S + y],
// S = 17 when every frame of the launch has at most 17 CTU rows and n <= 16,
// else 32; step 2 stages the saturating infinity for slices past Eq. 4's
// bound), then the column's items run from there (items_paired, or one at a
// time through item_rows for taller frames or n > 16).  V[k] = G_k[0] is
// collected in lane k and stored with one coalesced write per item.
// per warp after the two staging areas: G tables (288 words), item list
// (kListMax 16-bit entries: 32 words), step-2 window mask (16)
constexpr int kBandTail = 336;
template <int STEP, int S>
__global__ void __launch_bounds__(kMaxWarps * 32) band_kernel(LaunchArgs args, int total, int stage_words,
                                                               int itm_words) {
    extern __shared__ uint64_t bsm[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    if (gw >= total) return;
    int b;
    const int f = locate(args, args.pre.bands, args.single_bands, gw, &b);
    const DevFrame &fr = frame_at(args, f);
    const DevPlan &pl = *fr.plan;
    const int n = pl.n, R = fr.R, H = fr.H;
    const int i0 = pl.band_items[b], i1 = pl.band_items[b + 1];
    if (i0 == i1) return;
    uint64_t *Vall = STEP == 1 ? fr.V1 : fr.V2;
    if (frame_status(fr) != TRS_OK) {
        for (int ii = i0; ii < i1; ++ii)
            for (int k = lane; k <= n; k += 32) Vall[(size_t)ii * (n + 1) + k] = STEP == 1 ? kInf : kSoft;
        return;
    }
    const uint64_t thr = STEP == 2 ? eq4_threshold(fr.scal[0], fr.lambda_q) : kInf;
    const bool t32 = STEP == 1 && frame_t32(fr);
    const TablesOffsets off = tables_offsets(fr.C, R);
    const size_t base = (size_t)b * R * R;
    const uint64_t *RT = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_t) + base;
    const uint64_t *RQ = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_q) + base;
    // per warp: the column's slice values by height, one item's admitted
    // values, and the G tables (288 words)
    uint64_t *stage = bsm + (size_t)wib * (stage_words + itm_words + kBandTail);
    uint64_t *itm = stage + stage_words;
    uint64_t *gbuf = itm + itm_words;
    int16_t *list = reinterpret_cast<int16_t *>(gbuf + 288);
    uint32_t *wmask = reinterpret_cast<uint32_t *>(gbuf + 320);
    uint32_t tok = 0;  // step 2: bit d-1 set if the slice [lane, lane+d) meets the Eq. 4 bound
#pragma unroll 8
    for (int d = 1; d <= R; ++d) {
        const bool in = lane < R && lane + d <= R;
        const size_t e = in ? (size_t)(d - 1) * R + lane : 0;
        const uint64_t tv = __ldg(RT + e);
        if (STEP == 2) {
            // slices past the Eq. 4 bound hold the saturating infinity
            const bool meets = in && tv <= thr;
            const uint64_t qv = __ldg(RQ + e);
            if (lane < S) stage[(d - 1) * S + lane] = meets ? qv : kSoft;
            tok |= (meets ? 1u : 0u) << (d - 1);
        } else {
            if (lane < S) stage[(d - 1) * S + lane] = tv;
        }
    }
    __syncwarp();
    // with S = 17 every column takes this path (R <= 17 admits at most 68 items)
    if (R <= 17 && n <= 16 && i1 - i0 <= kListMax) {
        if (STEP == 1 && t32)
            items_paired<1, uint32_t, S>(fr, pl, i0, i1, Vall, stage, reinterpret_cast<uint32_t *>(itm),
                                         reinterpret_cast<uint32_t *>(gbuf), list, wmask, thr);
        else
            items_paired<STEP, uint64_t, S>(fr, pl, i0, i1, Vall, stage, itm, gbuf, list, wmask, thr);
        return;
    }
    const uint32_t ytop = line_px(lane, H);
    for (int ii = i0; ii < i1; ++ii) {
        const PlanItem it = pl.items[ii];
        uint64_t *V = Vall + (size_t)ii * (n + 1);
        if (STEP == 2) {
            // an item only matters if one of its windows still meets Eq. 4
            bool need = false;
            for (int w = it.w_first + lane; w <= it.w_last; w += 32) need |= fr.wres1[w] <= thr;
            if (!__any_sync(kFull, need)) {
                for (int k = lane; k <= n; k += 32) V[k] = kSoft;
                continue;
            }
        }
        const int dmin = max(1, (int)((it.hlo + kCtu - 1) / kCtu));
        const int dmax = min(R, (int)(it.hhi / kCtu) + 1);
        const int nd = dmax - dmin + 1;
        // this item's slice values, the saturating infinity where a height is not admitted
        uint64_t vreg;
        if (STEP == 1 && t32) {
            uint32_t *sv = reinterpret_cast<uint32_t *>(itm);
            for (int i = 0; i < nd; ++i) {
                const int d = dmin + i, y1 = lane + d;
                const uint32_t h = line_px(y1, H) - ytop;
                const bool ok = lane < R && y1 <= R && h >= it.hlo && h <= it.hhi;
                sv[i * 32 + lane] = ok ? (uint32_t)stage[(d - 1) * S + lane] : Soft<uint32_t>::v;
            }
            vreg = item_rows<1, uint32_t>(sv, reinterpret_cast<uint32_t *>(gbuf), nd, dmin, it.kmax, R);
        } else {
            for (int i = 0; i < nd; ++i) {
                const int d = dmin + i, y1 = lane + d;
                const uint32_t h = line_px(y1, H) - ytop;
                const bool ok = lane < R && y1 <= R && h >= it.hlo && h <= it.hhi &&
                                (STEP == 1 || ((tok >> (d - 1)) & 1u));
                itm[i * 32 + lane] = ok ? stage[(d - 1) * S + lane] : kSoft;
            }
            vreg = item_rows<STEP, uint64_t>(itm, gbuf, nd, dmin, it.kmax, R);
        }
        // counts below kmin complete no partition; "none" is kSoft in step 2 (the column DP adds it)
        const uint64_t none = STEP == 1 ? kInf : kSoft;
        if (lane == 0) {
            V[0] = kInf;
            if (n == 32) V[32] = 32 >= it.kmin && vreg != kInf ? vreg : none;
        } else if (lane <= n) {
            V[lane] = lane >= it.kmin && vreg != kInf ? vreg : none;
        }
    }
}

// ---- column DP ---------------------------------------------------------
//
// For one window w, the suffix DP over tile-column edges
//   H[x][m] = min over x1 > x and k of  V[item(w, [x, x1))][k] (max | +) H[x1][m - k],
//   H[C][0] = 0,
// where k runs over the item's slice counts [klo, khi].  One warp runs one
// window for F frames that share the plan (the plan fixes which bands and
// slice counts each step relaxes, so the warp's control flow is the same
// for all of them): lane (m - 1) * F + f holds H[x][m] of frame f.  The H
// tables sit in the warp's shared memory, frames interleaved, so a step is
// three shared loads (the value's H offset and V, both broadcast to the
// frame's lanes, and H[x1][m - k], consecutive over the lanes), a max
// (Eq. 1) or add (Eq. 2) and a min, in one flat loop over the edge's
// (band, slice count) values with no per-lane branch.  The values of left
// edge x - 1 are staged while edge x relaxes: their list from the plan's
// per-window entries (loaded one edge further ahead) and the V values by
// asynchronous global-to-shared copies spread evenly over the lanes,
// double-buffered, so no global load latency sits on the chain of edges.
// No block barrier: the warps of a block are independent.

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// every committed group but the most recent one is complete
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// One warp's shared memory for the column DP.
struct ColSmem {
    const uint64_t **vptr;  // [8]: V array of each frame of the warp
    uint32_t *md;           // [2][v_words]: per staged value, its H offset and slice count (see col_stage)
    uint64_t *vb;           // [2][v_words]: the staged V values, frames interleaved
    void *hs;               // H tables, frames interleaved
    int v_words;
};

// Stages left edge x into buffer bsel.  The edge's values are the pairs
// (band [x, x1) with an item in the window, slice count k in the item's
// range [klo, khi]), in order of x1 then k; value i gets
//   md[i] = ((x1 * stride - k) * F) << 6 | k
// (so H[x1][m - k] of frame f sits at Hs[(md[i] >> 6) + m * F + f]) and its
// V[item][k] of each of the F frames at vb[i * F + f], copied
// asynchronously.  The lanes take the (value, frame) pairs in turn, each
// finding its value's band by a binary search over the candidates' prefix
// sums, so no lane runs a loop of its own length.  e0: the plan entries of
// the first 32 candidate right edges (lane j: x1 = x + 1 + j), loaded ahead.
// Returns the number of values.
__device__ int col_stage(const uint64_t *sk, int C, int x, uint64_t e0, int stride, int F, int lf,
                         const ColSmem &sm, int bsel) {
    const int lane = threadIdx.x & 31;
    uint32_t *md = sm.md + bsel * sm.v_words;
    uint64_t *vb = sm.vb + (size_t)bsel * sm.v_words;
    const int ncand = C - x;
    const int b0 = band_index(C, x, x + 1);  // bands [x, x+1), [x, x+2), ... are consecutive
    int vtot = 0;
    for (int j0 = 0; j0 < ncand; j0 += 32) {
        const int j = j0 + lane;
        const uint64_t e = j0 == 0 ? e0 : (j < ncand ? __ldg(sk + b0 + j) : 0ull);
        const int item = (int)(uint32_t)e - 1;
        const int klo = (int)(e >> 32) & 0xff, khi = (int)(e >> 40) & 0xff;
        const int len = item >= 0 ? khi - klo + 1 : 0;
        int incl = len;  // inclusive prefix sum of len over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const int excl = incl - len;
        const int cnt = __shfl_sync(kFull, incl, 31);
        for (int q0 = 0; q0 < cnt * F; q0 += 32) {
            const int q = q0 + lane, i = q >> lf, ff = q & (F - 1);
            // the value's candidate: the last lane whose values start at or before i
            int o = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int ex = __shfl_sync(kFull, excl, o + st);
                if (ex <= i) o += st;
            }
            const int it_o = __shfl_sync(kFull, item, o);
            const int k = __shfl_sync(kFull, klo, o) + (i - __shfl_sync(kFull, excl, o));
            if (q < cnt * F) {
                cp_async8(vb + (size_t)(vtot + i) * F + ff, sm.vptr[ff] + (size_t)it_o * stride + k);
                if (ff == 0) md[vtot + i] = (uint32_t)(((x + 1 + j0 + o) * stride - k) * F) << 6 | (uint32_t)k;
            }
        }
        vtot += cnt;
    }
    return vtot;
}

// The column DP of window w for the F frames of the warp (lane
// (m - 1) * F + f, F = 1 << lf), values of type VT; V values are read as
// stored (the missing ones are kInf for step 1, whose low word exceeds the
// 32-bit saturating infinity too, and kSoft for step 2).  Leaves the H
// tables in shared memory; returns H[0][n] of the lane's frame.
template <int STEP, typename VT>
__device__ VT col_frames(const DevPlan &pl, int C, int w, int F, int lf, int f, int mi, const ColSmem &sm) {
    const int lane = threadIdx.x & 31;
    const int n = pl.n, stride = n + 1;
    constexpr VT soft = Soft<VT>::v;
    VT *Hs = reinterpret_cast<VT *>(sm.hs);
    const int m = mi < n ? mi + 1 : n;  // lanes past n shadow m = n and never store
    const bool mlive = mi < n;
    const int mF = m * F + f;
    const int total = (C + 1) * stride * F, zero0 = C * stride * F;
    for (int i = lane; i < total; i += 32) Hs[i] = (i >= zero0 && i < zero0 + F) ? VT(0) : soft;  // H[C][0] = 0
    const uint64_t *sk = pl.slot_k + (size_t)w * pl.nb;
    auto entry = [&](int x) -> uint64_t {  // plan entries of the first 32 candidate right edges of left edge x
        return (x >= 0 && lane < C - x) ? __ldg(sk + band_index(C, x, x + 1) + lane) : 0ull;
    };
    __syncwarp();
    int nv = col_stage(sk, C, C - 1, entry(C - 1), stride, F, lf, sm, 0);
    cp_async_commit();
    uint64_t e_next = entry(C - 2);
    for (int x = C - 1; x >= 0; --x) {
        const int bsel = (C - 1 - x) & 1;
        int nv_next = 0;
        if (x > 0) {
            const uint64_t e_after = entry(x - 2);
            nv_next = col_stage(sk, C, x - 1, e_next, stride, F, lf, sm, bsel ^ 1);
            e_next = e_after;
        }
        cp_async_commit();
        cp_async_wait_prev();  // edge x's values have landed
        __syncwarp();
        const uint32_t *md = sm.md + bsel * sm.v_words;
        const uint64_t *vb = sm.vb + (size_t)bsel * sm.v_words + f;
        // two minimum chains; H[x1][m - k] is read for every lane (x1 >= 1
        // keeps the offset inside the table) and replaced by the saturating
        // infinity where k > m
        VT acc0 = soft, acc1 = soft;
        int i = 0;
#pragma unroll 2
        for (; i + 1 < nv; i += 2) {
            const uint32_t d0 = md[i], d1 = md[i + 1];
            const VT v0 = (VT)vb[(size_t)i * F], v1 = (VT)vb[(size_t)(i + 1) * F];
            const VT g0 = Hs[(d0 >> 6) + mF], g1 = Hs[(d1 >> 6) + mF];
            const VT h0 = (int)(d0 & 63) <= m ? g0 : soft, h1 = (int)(d1 & 63) <= m ? g1 : soft;
            const VT c0 = STEP == 1 ? (v0 > h0 ? v0 : h0) : VT(v0 + h0);
            const VT c1 = STEP == 1 ? (v1 > h1 ? v1 : h1) : VT(v1 + h1);
            acc0 = c0 < acc0 ? c0 : acc0;
            acc1 = c1 < acc1 ? c1 : acc1;
        }
        if (i < nv) {
            const uint32_t d0 = md[i];
            const VT v0 = (VT)vb[(size_t)i * F];
            const VT g0 = Hs[(d0 >> 6) + mF];
            const VT h0 = (int)(d0 & 63) <= m ? g0 : soft;
            const VT c0 = STEP == 1 ? (v0 > h0 ? v0 : h0) : VT(v0 + h0);
            acc0 = c0 < acc0 ? c0 : acc0;
        }
        const VT acc = acc0 < acc1 ? acc0 : acc1;
        if (mlive) Hs[(x * stride + m) * F + f] = acc;
        __syncwarp();
        nv = nv_next;
    }
    return Hs[n * F + f];
}

// Which frames and window column-DP warp u runs.
__device__ __forceinline__ void col_unit(const LaunchArgs &a, int u, int *first, int *count, int *F, int *w) {
    if (!a.cchunks) {
        const int nch = a.col_nchunks, fpw = a.col_fpw;
        const int ww = u / nch, c = u - ww * nch;
        *w = ww;
        *F = fpw;
        *first = c * fpw;
        *count = min(fpw, a.nframes - c * fpw);
        return;
    }
    int lo = 0, hi = a.col_nchunks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.cchunks[mid].unit0 <= u) lo = mid; else hi = mid - 1;
    }
    const ColChunk ch = a.cchunks[lo];
    *first = ch.first;
    *count = ch.count;
    *F = ch.fpw;
    *w = u - ch.unit0;
}

constexpr int kColHead = 64;  // the vptr table at the start of a warp's shared memory

// One warp per (window, frames sharing the plan): the column DP of Eq. 1
// (step 1, reduced into T_min, Eq. 3) or Eq. 2 (step 2, into Q*), see
// col_frames.  Step 2 runs only for frames whose step-1 window best meets
// Eq. 4 (every item of such a window was relaxed by step 2's row DP) and
// stores their H tables for the rebuild.
template <int STEP>
__global__ void __launch_bounds__(kMaxWarps * 32) column_kernel(LaunchArgs args, int total, int warp_bytes,
                                                                 int v_words) {
    extern __shared__ __align__(16) unsigned char colsm[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * (blockDim.x >> 5) + wib;
    if (u >= total) return;
    int first, count, F, w;
    col_unit(args, u, &first, &count, &F, &w);
    const int lf = __ffs(F) - 1;
    const int f = lane & (F - 1), mi = lane >> lf;
    const bool fvalid = f < count;
    const DevFrame &fr = frame_at(args, first + (fvalid ? f : 0));
    const DevPlan &pl = *fr.plan;
    const int C = fr.C, n = pl.n;
    unsigned char *base = colsm + (size_t)wib * warp_bytes;
    ColSmem sm;
    sm.vptr = reinterpret_cast<const uint64_t **>(base);
    sm.vb = reinterpret_cast<uint64_t *>(base + kColHead);
    sm.md = reinterpret_cast<uint32_t *>(base + kColHead + (size_t)2 * v_words * 8);
    sm.v_words = v_words;
    sm.hs = base + kColHead + (size_t)2 * v_words * 12;
    uint64_t *wres = STEP == 1 ? fr.wres1 : fr.wres2;
    const bool ok = fvalid && frame_status(fr) == TRS_OK;
    bool pass = ok;
    if (STEP == 2) pass = ok && fr.wres1[w] <= eq4_threshold(fr.scal[0], fr.lambda_q);
    if (!__any_sync(kFull, pass)) {  // no frame of the warp has a candidate here
        if (fvalid && mi == 0) wres[w] = kInf;
        return;
    }
    if (mi == 0) sm.vptr[f] = STEP == 1 ? fr.V1 : fr.V2;
    uint64_t res = kInf;
    if (STEP == 1) {
        if (__all_sync(kFull, !fvalid || frame_t32(fr))) {
            const uint32_t r = col_frames<1, uint32_t>(pl, C, w, F, lf, f, mi, sm);
            res = r >= Soft<uint32_t>::v ? kInf : r;
        } else {
            // 64-bit values: the frames one at a time, lanes over the slice count
            for (int g = 0; g < count; ++g) {
                ColSmem s1 = sm;
                s1.vptr = sm.vptr + g;
                const uint64_t r = col_frames<1, uint64_t>(pl, C, w, 1, 0, 0, lane, s1);
                if (f == g) res = r >= kSoft ? kInf : r;
                __syncwarp();
            }
        }
    } else {
        const uint64_t r = col_frames<2, uint64_t>(pl, C, w, F, lf, f, mi, sm);
        res = r >= kSoft ? kInf : r;
    }
    if (!pass) res = kInf;
    if (fvalid && mi == 0) {
        wres[w] = res;
        if (res != kInf) atomicMin(reinterpret_cast<unsigned long long *>(&fr.scal[STEP == 1 ? 0 : 1]), res);
    }
    if (STEP == 2 && pass) {
        // the frame's H table of this window, for the rebuild (lanes of frame f)
        const uint64_t *Hs = reinterpret_cast<const uint64_t *>(sm.hs);
        const int words = (C + 1) * (n + 1);
        uint64_t *H2 = fr.H2 + (size_t)w * words;
        for (int i = mi; i < words; i += 32 >> lf) H2[i] = hard_inf(Hs[i * F + f]);
    }
}

// '0' < '1' read from CTU line 1 downwards: compare bit-reversed words.
__device__ __forceinline__ bool bits_less(uint32_t a, uint32_t b) { return __brev(a) < __brev(b); }

// A code's cut word before cuts_kernel: bit 31 set, the band's item in
// bits 6..30 and its slice count in bits 0..5.  Cut bits themselves never
// set bit 31 (at most 31 CTU lines inside a frame of 32 rows).
constexpr uint32_t kCutPending = 1u << 31;

// Smallest cut bits of a k-slice split of the item's band that reaches
// layers[k][0], read greedily top-down: the largest next cut line first.
// Slice values and admissibility come from the shared-memory staging of
// item_dp (stage[i*32 + y] = floor-SSE of rows [y, y+dmin+i), bit i of
// vm[y] = admissible).
__device__ uint32_t lexmin_bits(const PlanItem &it, int R, const uint64_t *layers, const uint64_t *stage,
                                const uint32_t *vm, int k) {
    const int lane = threadIdx.x & 31;
    const int dmin = max(1, (int)((it.hlo + kCtu - 1) / kCtu));
    uint32_t bits = 0;
    int y = 0;
    for (int kk = k; kk > 1; --kk) {
        const int y1 = lane;  // candidate next cut line
        const int i = y1 - y - dmin;
        bool ok = false;
        if (y1 > y && y1 < R && i >= 0 && i < 32 && ((vm[y] >> i) & 1u)) {
            const uint64_t nxt = layers[(kk - 1) * 32 + y1];
            ok = nxt != kInf && nxt + stage[i * 32 + y] == layers[kk * 32 + y];
        }
        const unsigned m = __ballot_sync(kFull, ok);
        if (!m) return ~0u;  // unreachable when layers[kk][y] is finite
        const int cut = 31 - __clz(m);
        bits |= 1u << (cut - 1);
        y = cut;
    }
    return bits;
}

__device__ bool code_less_g(const WinCode &a, const WinCode &b) {
    const int c = a.c < b.c ? a.c : b.c;
    for (int i = 0; i < c; ++i) {
        if (a.xe[i + 1] != b.xe[i + 1]) return a.xe[i + 1] < b.xe[i + 1];
        if (a.cut[i] != b.cut[i]) return bits_less(a.cut[i], b.cut[i]);
    }
    return false;
}

// One warp per (frame, window): if the window reaches Q*, rebuild its
// smallest canonical code.  At each left edge x the warp walks the
// candidate right edges x1 in increasing order (their items fetched by the
// lanes at once) and, with lanes over the slice count k, keeps the first x1
// for which some k completes an optimal partition:
//   V2[item][k] + H2[x1][m-k] == H2[x][m].
// When one k does (every column of the benchmarked sequence), the column's
// cut word records the item and k with kCutPending set and cuts_kernel
// fills in the bits; when several do, the band's row DP is redone here with
// every layer kept in shared memory and the smallest cut bits among them
// win.
__global__ void __launch_bounds__(32) rebuild_kernel(LaunchArgs args, int total, int layer_words,
                                                      int stage_words) {
    extern __shared__ uint64_t rsm[];
    uint64_t *layers = rsm;
    uint64_t *stage = rsm + layer_words;
    __shared__ uint32_t vm[32];
    const int gw = blockIdx.x;
    if (gw >= total) return;
    int w;
    const int f = locate(args, args.pre.windows, args.single_windows, gw, &w);
    const DevFrame &fr = frame_at(args, f);
    const DevPlan &pl = *fr.plan;
    const int lane = threadIdx.x;
    const int C = fr.C, R = fr.R, n = pl.n, nb = pl.nb, stride = n + 1;
    WinCode &code = fr.codes[w];
    const uint64_t qstar = fr.scal[1];
    if (frame_status(fr) != TRS_OK || qstar == kInf || fr.wres2[w] != qstar) {
        if (lane == 0) code.c = -1;
        return;
    }
    const uint64_t thr = eq4_threshold(fr.scal[0], fr.lambda_q);
    const uint64_t *H2 = fr.H2 + (size_t)w * (C + 1) * stride;
    const int32_t *slot_row = pl.slot_of + (size_t)w * nb;
    int x = 0, m = n, c = 0;
    while (x < C) {
        const uint64_t target = H2[x * stride + m];
        int x1 = -1, slot = -1;
        unsigned kmask = 0;
        for (int base = 0; base < C - x && x1 < 0; base += 32) {
            const int cx = x + 1 + base + lane;
            const int sl = cx <= C ? slot_row[band_index(C, x, cx)] : -1;
            unsigned cand = __ballot_sync(kFull, sl >= 0);
            while (cand) {
                const int j = __ffs(cand) - 1;
                cand &= cand - 1;
                const int sj = __shfl_sync(kFull, sl, j);
                const int xj = x + 1 + base + j;
                const int k = lane + 1;
                bool ok = false;
                if (k <= m) {
                    const uint64_t v = fr.V2[(size_t)sj * stride + k], h = H2[xj * stride + m - k];
                    ok = v < kSoft && h != kInf && v + h == target;
                }
                const unsigned km = __ballot_sync(kFull, ok);
                if (km) {
                    x1 = xj;
                    slot = sj;
                    kmask = km;
                    break;
                }
            }
        }
        if (x1 < 0) {  // cannot happen when H2[x][m] is finite
            if (lane == 0) code.c = -1;
            return;
        }
        uint32_t bb;
        int bk;
        if (!(kmask & (kmask - 1)) && slot < (1 << 25)) {
            // one slice count completes the optimum: the column's cut bits
            // are left to cuts_kernel, which runs the row DPs of all the
            // code's tile columns in parallel
            bk = __ffs(kmask);
            bb = kCutPending | (uint32_t)slot << 6 | (uint32_t)bk;
        } else {
            // several do: the smallest cut bits among them decide here
            const PlanItem it = pl.items[slot];
            item_dp<2>(fr, it, thr, n, nullptr, layers, stage, vm);
            bb = 0;
            bk = -1;
            for (unsigned mm = kmask; mm; mm &= mm - 1) {
                const int kk = __ffs(mm);  // slice count kk = bit index + 1
                const uint32_t bits = lexmin_bits(it, R, layers, stage, vm, kk);
                if (bk < 0 || bits_less(bits, bb)) {
                    bb = bits;
                    bk = kk;
                }
            }
            __syncwarp();
        }
        if (lane == 0) {
            code.xe[c + 1] = (int16_t)x1;
            code.cut[c] = bb;
        }
        c++;
        m -= bk;
        x = x1;
    }
    if (lane == 0) {
        code.xe[0] = 0;
        code.c = c;
    }
}

// The cut bits of the tile columns the rebuild left pending.  Block (frame
// f, slot s) takes the windows of f that reached Q* (c > 0) whose rank among
// them is s modulo kCutSlots; its warps take their tile columns j = warp,
// warp + kCutWarps, ...: each redoes the column's row DP with every layer
// kept and reads the smallest cut bits of its slice count (lexmin_bits).
constexpr int kCutSlots = 8, kCutWarps = 4;
__global__ void __launch_bounds__(kCutWarps * 32) cuts_kernel(LaunchArgs args, int layer_words, int stage_words) {
    extern __shared__ uint64_t csm[];
    __shared__ uint32_t cvm[kCutWarps][32];
    const int f = blockIdx.x / kCutSlots, slot = blockIdx.x % kCutSlots;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const DevFrame &fr = frame_at(args, f);
    const DevPlan &pl = *fr.plan;
    const uint64_t qstar = fr.scal[1];
    if (frame_status(fr) != TRS_OK || qstar == kInf) return;
    const uint64_t thr = eq4_threshold(fr.scal[0], fr.lambda_q);
    uint64_t *layers = csm + (size_t)wib * (layer_words + stage_words);
    uint64_t *stage = layers + layer_words;
    uint32_t *vm = cvm[wib];
    const int R = fr.R, n = pl.n;
    int rank = 0;
    for (int w0 = 0; w0 < pl.nwin; w0 += 32) {
        const int wl = w0 + lane;
        const unsigned tied = __ballot_sync(kFull, wl < pl.nwin && fr.codes[wl].c > 0);
        for (unsigned mm = tied; mm; mm &= mm - 1, ++rank) {
            if (rank % kCutSlots != slot) continue;
            WinCode &code = fr.codes[w0 + __ffs(mm) - 1];
            const int c = code.c;
            for (int j = wib; j < c; j += kCutWarps) {
                const uint32_t word = code.cut[j];
                if (!(word & kCutPending)) continue;
                const int item = (int)((word & ~kCutPending) >> 6), k = (int)(word & 63u);
                const PlanItem it = pl.items[item];
                item_dp<2>(fr, it, thr, n, nullptr, layers, stage, vm);
                const uint32_t bits = lexmin_bits(it, R, layers, stage, vm, k);
                __syncwarp();
                if (lane == 0) code.cut[j] = bits;
            }
        }
    }
}

// One warp per frame: the smallest code over the windows reaching Q* (lanes
// scan the windows, then a shuffle reduction), then its decoding into
// trs_partition (one tile row, tile columns = bands, slices top to bottom),
// one lane per tile column with a warp prefix sum for the region indices.
__global__ void __launch_bounds__(32) finish_kernel(LaunchArgs args) {
    const int f = blockIdx.x;
    const DevFrame &fr = frame_at(args, f);
    const DevPlan &pl = *fr.plan;
    const int lane = threadIdx.x;
    const int C = fr.C, R = fr.R, n = pl.n;
    trs_partition *out = fr.out;
    int32_t status = frame_status(fr);
    const uint64_t t_min = fr.scal[0];
    if (status == TRS_OK && t_min == kInf) status = TRS_EINFEASIBLE;
    const uint64_t qstar = fr.scal[1];
    if (status == TRS_OK && qstar == kInf) status = TRS_EINFEASIBLE;  // cannot happen: P(T_min) meets Eq. 4
    // the whole record is rewritten: entries past the used ones read as zero
    uint64_t *words = reinterpret_cast<uint64_t *>(out);
    for (int i = lane; i < (int)(sizeof(trs_partition) / 8); i += 32) words[i] = 0;
    __syncwarp();
    int bw = -1;
    if (status == TRS_OK) {
        for (int w = lane; w < pl.nwin; w += 32)
            if (fr.codes[w].c > 0 && (bw < 0 || code_less_g(fr.codes[w], fr.codes[bw]))) bw = w;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int other = __shfl_xor_sync(kFull, bw, o);
            if (other >= 0 && (bw < 0 || code_less_g(fr.codes[other], fr.codes[bw]) ||
                               (other < bw && !code_less_g(fr.codes[bw], fr.codes[other]))))
                bw = other;
        }
        if (bw < 0) status = TRS_EINFEASIBLE;
    }
    if (status != TRS_OK) {
        if (lane == 0) {
            out->status = status;
            out->n_regions = n;
            out->cols = C;
            out->rows = R;
            out->n_windows = pl.nwin;
        }
        return;
    }
    const WinCode &best = fr.codes[bw];
    const int c = best.c;
    const TablesOffsets off = tables_offsets(C, R);
    const uint64_t *RT = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_t);
    const uint64_t *RQ = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_q);
    const uint64_t *sat1 = reinterpret_cast<const uint64_t *>(fr.tables + off.sat_s1);
    // lane b lays out tile column b's slices (c <= n <= 32), then lane r
    // evaluates region r
    __shared__ int16_t reg[32][4];
    const int b = lane;
    const uint32_t cut = b < c ? best.cut[b] : 0u;
    const int ns = b < c ? __popc(cut) + 1 : 0;
    int r = ns;  // inclusive prefix sum of slice counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, r, o);
        if (lane >= o) r += v;
    }
    r -= ns;  // first region index of this tile column
    if (b < c) {
        const int x0 = best.xe[b], x1 = best.xe[b + 1];
        out->col_bd[b + 1] = (int16_t)x1;
        out->slice_cuts[b] = cut;
        out->tile_slices[b] = (uint8_t)ns;
        int y0 = 0;
        for (int y = 1; y <= R; ++y) {
            if (y < R && !((cut >> (y - 1)) & 1u)) continue;
            if (r < 32) {
                reg[r][0] = (int16_t)x0;
                reg[r][1] = (int16_t)y0;
                reg[r][2] = (int16_t)x1;
                reg[r][3] = (int16_t)y;
            }
            r++;
            y0 = y;
        }
    }
    int nreg = ns;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nreg += __shfl_xor_sync(kFull, nreg, o);
    __syncwarp();
    uint64_t tmax = 0, qsum = 0;
    double sse = 0.0;
    if (lane < nreg && lane < kMaxN) {
        const int x0 = reg[lane][0], y0 = reg[lane][1], x1 = reg[lane][2], y = reg[lane][3];
        const size_t e = ((size_t)band_index(C, x0, x1) * R + (y - y0 - 1)) * R + y0;
        const uint64_t tv = RT[e], qv = RQ[e];
        tmax = tv;
        qsum = qv;
        const uint64_t s1 = sat1[y * (C + 1) + x1] - sat1[y0 * (C + 1) + x1] - sat1[y * (C + 1) + x0] +
                            sat1[y0 * (C + 1) + x0];
        const uint32_t np = (line_px(x1, fr.W) - line_px(x0, fr.W)) * (line_px(y, fr.H) - line_px(y0, fr.H));
        uint32_t rem;
        (void)ceil_square_div(s1, np, &rem);
        // exact SSE = floor + (ceil(S1^2/N) - S1^2/N)
        sse = (double)qv + (rem ? (double)(np - rem) / (double)np : 0.0);
        out->region[lane][0] = (int16_t)x0;
        out->region[lane][1] = (int16_t)y0;
        out->region[lane][2] = (int16_t)x1;
        out->region[lane][3] = (int16_t)y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t tm = __shfl_xor_sync(kFull, tmax, o);
        tmax = tm > tmax ? tm : tmax;
        qsum += __shfl_xor_sync(kFull, qsum, o);
        sse += __shfl_xor_sync(kFull, sse, o);
    }
    if (lane == 0) {
        const uint64_t thr = eq4_threshold(t_min, fr.lambda_q);
        out->n_regions = n;
        out->cols = C;
        out->rows = R;
        out->n_windows = pl.nwin;
        out->n_tile_cols = c;
        out->n_tile_rows = 1;
        out->tile_row_mask = 0;
        out->row_bd[0] = 0;
        out->row_bd[1] = (int16_t)R;
        out->col_bd[0] = 0;
        out->t_min_q = t_min;
        out->thr_q = thr;
        out->t_q = tmax;
        out->q = qsum;
        out->t_min = (double)t_min / 65536.0;
        out->t = (double)tmax / 65536.0;
        out->sse = sse;
        // internal consistency guard
        out->status = (nreg != n || qsum != qstar || tmax > thr) ? TRS_EINFEASIBLE : TRS_OK;
    }
}

}  // namespace

// Raises the dynamic shared-memory limit of the search kernels to what the
// largest shapes need (once per device, before any capture).
int prepare_search_kernels() {
    const int band_smem = kMaxWarps * (2 * kMaxR * 32 + kBandTail) * (int)sizeof(uint64_t);
    const int col_smem = 227 * 1024;  // the column DP's per-warp tables scale with the shapes of the launch
    const int rb_smem = ((kMaxN + 1) * 32 + kMaxR * 32) * (int)sizeof(uint64_t);
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(band_kernel<1, 17>, A, band_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(band_kernel<1, 32>, A, band_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(band_kernel<2, 17>, A, band_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(band_kernel<2, 32>, A, band_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(column_kernel<1>, A, col_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(column_kernel<2>, A, col_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rebuild_kernel, A, rb_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cuts_kernel, A, kCutWarps * rb_smem);
    return (int)e;
}

int launch_search(const LaunchArgs &a, int total_bands, int total_windows, int maxC, int maxR, int maxN,
                  uint64_t *scal, size_t nscal, void *stream, const ColGeom &col, cudaEvent_t *ev,
                  const SearchTune *tune, int steps, int max_nd) {
    const SearchTune t = tune ? *tune : SearchTune{};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // T_min and Q* start at +infinity; the column kernels reduce into them
    if ((steps & 1) && scal) e = cudaMemsetAsync(scal, 0xff, nscal * sizeof(uint64_t), s);
    if (e != cudaSuccess) return (int)e;
    const int bw = t.band_warps, cw = t.col_warps;
    const int stage_words = maxR * 32;  // rebuild's staging (stride 32)
    const int S = maxR <= 17 && maxN <= 16 ? 17 : 32;
    // the per-item staging holds the admitted full-height values (at most
    // max_nd heights) in the paired path, up to R heights in the other; the
    // paired path keeps up to kNdRegs heights in registers and needs none
    const int band_itm = S == 17 && max_nd > 0 ? (max_nd <= kNdRegs ? 0 : std::min(max_nd, maxR) * 32) : maxR * 32;
    const int band_stage = maxR * S;
    const size_t band_smem = (size_t)bw * (band_stage + band_itm + kBandTail) * sizeof(uint64_t);
    const int bb = (total_bands + bw - 1) / bw;
    auto mark = [&](int i) {
        if (ev && e == cudaSuccess) e = record_event(ev[i], s);
    };
    auto columns = [&](int step) {
        if (col.units <= 0) return;
        // per warp: vptr table, two buffers of staged values and their offsets, H tables
        const size_t hb = step == 1 ? col.h_bytes1 : col.h_bytes2;
        const size_t wb = ((size_t)kColHead + (size_t)2 * col.v_words * 12 + hb + 15) & ~size_t(15);
        int P = cw;
        while (P > 1 && (size_t)P * wb > 227 * 1024) P >>= 1;
        const int blocks = (col.units + P - 1) / P;
        if (step == 1) column_kernel<1><<<blocks, P * 32, P * wb, s>>>(a, col.units, (int)wb, col.v_words);
        else column_kernel<2><<<blocks, P * 32, P * wb, s>>>(a, col.units, (int)wb, col.v_words);
    };
    if (steps & 1) {
        if (total_bands > 0) {
            if (S == 17) band_kernel<1, 17><<<bb, bw * 32, band_smem, s>>>(a, total_bands, band_stage, band_itm);
            else band_kernel<1, 32><<<bb, bw * 32, band_smem, s>>>(a, total_bands, band_stage, band_itm);
        }
        mark(0);
        columns(1);
        mark(1);
    }
    if (!(steps & 2)) return e != cudaSuccess ? (int)e : (int)cudaGetLastError();
    if (total_bands > 0) {
        if (S == 17) band_kernel<2, 17><<<bb, bw * 32, band_smem, s>>>(a, total_bands, band_stage, band_itm);
        else band_kernel<2, 32><<<bb, bw * 32, band_smem, s>>>(a, total_bands, band_stage, band_itm);
    }
    mark(2);
    columns(2);
    mark(3);
    const int layer_words = (maxN + 1) * 32;
    const size_t rb_smem = (size_t)(layer_words + stage_words) * sizeof(uint64_t);
    if (total_windows > 0) {
        rebuild_kernel<<<total_windows, 32, rb_smem, s>>>(a, total_windows, layer_words, stage_words);
        cuts_kernel<<<a.nframes * kCutSlots, kCutWarps * 32, kCutWarps * rb_smem, s>>>(a, layer_words, stage_words);
    }
    mark(4);
    finish_kernel<<<a.nframes, 32, 0, s>>>(a);
    mark(5);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}

}  // namespace trs
