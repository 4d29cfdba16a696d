// Internal declarations shared by the CUDA translation units of libtrs.
//
// Frame geometry: CTUs of 128x128 luma samples, C = ceil(W/128) columns,
// R = ceil(H/128) rows, the last column/row clipped to the frame.  A tile
// column ("band") spans CTU columns [x0, x1); its compact index is
// b = x0*(2C - x0 + 1)/2 + (x1 - x0 - 1).  A slice of a band spans CTU rows
// [y, y + d).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/trs.h"

static_assert(sizeof(trs_partition) % 8 == 0, "trs_partition is cleared as 8-byte words");

namespace trs {

constexpr uint64_t kInf = ~0ull;
constexpr int kCtu = TRS_CTU;
constexpr int kMaxC = TRS_MAX_COLS;
constexpr int kMaxR = TRS_MAX_ROWS;
constexpr int kMaxN = TRS_MAX_REGIONS;

__host__ __device__ inline int band_index(int C, int x0, int x1) {
    return x0 * (2 * C - x0 + 1) / 2 + (x1 - x0 - 1);
}
__host__ __device__ inline int num_bands(int C) { return C * (C + 1) / 2; }
// Sample formats (see TRS_PACKED10): valid codes, the sample bit depth and
// the bytes of one row of W samples.
__host__ __device__ inline bool fmt_ok(int bd) { return (bd >= 8 && bd <= 12) || bd == TRS_PACKED10; }
__host__ __device__ inline int fmt_depth(int bd) { return bd == TRS_PACKED10 ? 10 : bd; }
__host__ __device__ inline size_t fmt_row_bytes(int W, int bd) {
    return bd == TRS_PACKED10 ? ((size_t)W * 10 + 7) / 8 : (size_t)W * (bd == 8 ? 1 : 2);
}
// Pixel extent of CTU lines: position of line x (clipped to the frame edge).
__host__ __device__ inline uint32_t line_px(int x, int extent) {
    uint32_t p = (uint32_t)x * kCtu;
    return p < (uint32_t)extent ? p : (uint32_t)extent;
}

// Offsets of one frame's region tables inside its buffer (all 256-aligned).
struct TablesOffsets {
    size_t tq, sat_s1, sat_s2, sat_t, rect_t, rect_q, status, bytes;
};
__host__ __device__ inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
__host__ __device__ inline TablesOffsets tables_offsets(int C, int R) {
    TablesOffsets o;
    size_t p = 0;
    const size_t sat = (size_t)(R + 1) * (C + 1) * 8;
    const size_t rect = (size_t)num_bands(C) * R * R * 8;
    o.tq = p;      p = align256(p + (size_t)R * C * 4);
    o.sat_s1 = p;  p = align256(p + sat);
    o.sat_s2 = p;  p = align256(p + sat);
    o.sat_t = p;   p = align256(p + sat);
    o.rect_t = p;  p = align256(p + rect);
    o.rect_q = p;  p = align256(p + rect);
    o.status = p;  p = align256(p + 16);
    o.bytes = p;
    return o;
}

#ifdef __CUDACC__
// A float no larger than x (two 32-bit conversions: no 64-bit one).
__device__ inline float u64_to_float_rz(uint64_t x) {
    return __fadd_rz(__fmul_rz(__uint2float_rz((uint32_t)(x >> 32)), 4294967296.0f), __uint2float_rz((uint32_t)x));
}

// floor(f) for 0 <= f < 2^64, exactly: the multiple of 2^32 below f and
// the rest are both floats (f has 24 significant bits), so neither step
// rounds.
__device__ inline uint64_t float_to_u64_rz(float f) {
    const uint32_t hi = __float2uint_rz(f * 2.3283064365386963e-10f);  // f / 2^32
    const float rest = f - __uint2float_rz(hi) * 4294967296.0f;
    return ((uint64_t)hi << 32) + __float2uint_rz(rest);
}

// floor(x / n) and *rem = x mod n for 1 <= n < 2^32, without a hardware
// divide: the schoolbook correction of a trial quotient (Knuth, TAOCP vol. 2,
// Sec. 4.3.1), the trial quotient taken in single precision with every
// rounding toward zero and rn <= 1/n, so that it never exceeds x / n; the
// remainder is then exact in 64-bit integers.  Each round leaves a quotient
// below 2^-21 of the previous one (plus 1), so x < 2^64 takes at most five.
__device__ inline uint64_t udivmod_trial(uint64_t x, uint32_t n, float rn, uint64_t *rem) {
    uint64_t q = 0;
    while (x >= n) {
        uint64_t t = float_to_u64_rz(__fmul_rz(u64_to_float_rz(x), rn));
        t = t ? t : 1;  // x >= n: at least one n fits
        q += t;
        x -= t * n;
    }
    *rem = x;
    return q;
}

// ceil(s1^2 / n) for 1 <= n < 2^32 when the quotient fits 64 bits (it is at
// most S2 by Cauchy-Schwarz); *rem = s1^2 mod n.  With s1 = a n + b (b < n):
// s1^2 = n (a (s1 + b) + c) + r where b^2 = c n + r.
__device__ inline uint64_t ceil_square_div(uint64_t s1, uint32_t n, uint32_t *rem) {
    const float rn = __frcp_rz(__uint2float_ru(n));  // <= 1/n
    uint64_t b, r;
    const uint64_t a = udivmod_trial(s1, n, rn, &b);
    const uint64_t c = udivmod_trial(b * b, n, rn, &r);
    *rem = (uint32_t)r;
    return a * (s1 + b) + c + (r != 0 ? 1u : 0u);
}

// Largest T with T * 65536 <= t_min * (65536 + lambda_q)  (Eq. 4).
__device__ inline uint64_t eq4_threshold(uint64_t t_min, uint32_t lambda_q) {
    if (t_min == kInf) return kInf;
    const uint64_t m = 65536ull + lambda_q;
    const uint64_t lo = t_min * m, hi = __umul64hi(t_min, m);
    if (hi >> 16) return kInf;
    return (lo >> 16) | (hi << 48);
}
#endif

// One unit of row-DP work of the search: tile column b whose slices must
// have a pixel height in [hlo, hhi] (the slice heights that land in the area
// window of every window mapped to this unit).  kmax bounds the slice count.
struct alignas(16) PlanItem {  // 32 bytes: two 16-byte loads
    int32_t b;
    int32_t kmax;
    uint32_t hlo, hhi;
    int32_t w_first, w_last;  // the windows mapped to this item are [w_first, w_last]
    // slice counts below kmin cannot complete a partition in any of those
    // windows: the rest of the frame could not hold the other slices (see
    // build_plan); their V entries are stored as +infinity
    int32_t kmin;
    int32_t reserved;
};

// Search plan of one frame shape (W, H, n, k), built on the host once per
// shape and kept in device memory.  Depends on geometry only.
struct DevPlan {
    int W, H, C, R, n, k, nb, nwin, nitems;
    uint64_t A;                 // W*H
    const uint64_t *win_a;      // [nwin] window lower bounds a (window = [a, k*a-1]), ascending
    const PlanItem *items;      // [nitems]
    const int32_t *slot_of;     // [nwin * nb]: item of (window, band), -1 if the band has no slice there
    const int16_t *band_x0;     // [nb]
    const int16_t *band_x1;     // [nb]
    const int32_t *band_items;  // [nb+1]: items of band b are [band_items[b], band_items[b+1])
    // column-DP steps, [nwin * nb]: for band b of window w, 0 if the band has
    // no item there, else (item + 1) | klo << 32 | khi << 40 with [klo, khi]
    // the item's slice counts (klo >= 1)
    const uint64_t *slot_k;
    int max_edge_vals;  // largest sum of khi - klo + 1 over the bands of one left edge of one window
};

// Column-DP step entry of band (item, slice counts [klo, khi]).
__host__ __device__ inline uint64_t pack_slot_k(int item, int klo, int khi) {
    return (uint64_t)(uint32_t)(item + 1) | (uint64_t)(uint32_t)klo << 32 | (uint64_t)(uint32_t)khi << 40;
}

// A canonical code: c tile columns with right edges xe[1..c] (xe[0] = 0)
// and the slice cut bits of each (bit y-1 = cut at CTU line y).  c < 0
// marks "no code" (the window does not reach Q*).
struct WinCode {
    int32_t c;
    int16_t xe[kMaxC + 1];
    uint32_t cut[kMaxC];
};

// Everything a kernel needs about one frame.  Lives in device memory for
// batched launches, or travels by value inside LaunchArgs for one frame.
struct DevFrame {
    // a1 input
    const uint8_t *luma;
    size_t pitch;
    int W, H, bd, vec_ok;  // bd: sample bit depth; vec_ok: base and pitch 16-byte aligned
    int packed;            // samples in the TRS_PACKED10 format (bd = 10)
    // a2 input
    const float *times;
    // a1 output / a2 input
    uint32_t *s1;
    uint64_t *s2;
    uint32_t *cnt;
    uint32_t *vmax;
    uint32_t *flags;
    // a2 output / search input
    uint8_t *tables;
    // search
    const DevPlan *plan;  // device pointer
    int C, R, n;
    uint32_t lambda_q;
    uint64_t *V1, *V2;      // [nitems][n+1]
    uint64_t *wres1, *wres2;  // [nwin]
    uint64_t *H2;           // [nwin][(C+1)*(n+1)]
    WinCode *codes;         // [nwin]: smallest code of each window reaching Q*
    uint64_t *scal;         // [0] T_min, [1] Q*, [2] thr, [3] spare
    trs_partition *out;
};

// Work prefix sums over the frames of a launch (exclusive, nframes+1 entries).
struct WorkPrefix {
    const int32_t *ctus;     // texture: CTUs
    const int32_t *bandgrp;  // tables: groups of kBandsPerBlock bands
    const int32_t *items;    // search rows: plan items
    const int32_t *windows;  // search columns: plan windows
    const int32_t *bands;    // search rows: tile columns (one warp each, all of its items)
};

constexpr int kBandsPerBlock = 16;

// Column-DP work: frames [first, first + count) of a launch share one plan
// and each warp runs one window for up to fpw of them; the chunk's units
// (one per window) are [unit0, unit0 + nwin).
struct ColChunk {
    int32_t first, count, fpw, unit0;
};

// Lanes per frame of a column-DP warp: the slice counts m = 1..n, rounded up
// to a power of two (at least 4, so a warp holds at most 8 frames).
__host__ __device__ inline int col_lanes(int n) {
    int L = 4;
    while (L < n) L <<= 1;
    return L;
}

struct LaunchArgs {
    DevFrame single;            // used when frames == nullptr
    const DevFrame *frames;     // device array of nframes, or nullptr
    int nframes;
    WorkPrefix pre;             // device arrays (unused when nframes == 1 and frames == nullptr)
    // work units of the single frame; with `uniform` (every frame of the
    // array has the same plan) the units of each frame of the array
    int single_ctus, single_bandgrp, single_items, single_windows, single_bands;
    int uniform;
    // column DP: with cchunks == nullptr every frame of the launch shares one
    // plan, col_fpw frames per warp in col_nchunks chunks, unit u = window
    // (u / col_nchunks) of chunk (u % col_nchunks); otherwise col_nchunks
    // chunks described by cchunks
    const ColChunk *cchunks;
    int col_nchunks, col_fpw;
};

// Launch geometry of the column DP (host side).
struct ColGeom {
    int units = 0;          // warps: one per (chunk, window)
    size_t h_bytes1 = 0;    // per warp: the H tables of step 1 (32-bit for all frames, or 64-bit one at a time)
    size_t h_bytes2 = 0;    // per warp: the H tables of step 2 (64-bit)
    int v_words = 1;        // per warp and buffer: staged V values of one left edge
    void add(int C, int n, int max_edge_vals, int fpw) {
        const size_t cells = (size_t)(C + 1) * (n + 1);
        const size_t h1 = cells * (size_t)(4 * fpw > 8 ? 4 * fpw : 8), h2 = cells * 8 * (size_t)fpw;
        h_bytes1 = h1 > h_bytes1 ? h1 : h_bytes1;
        h_bytes2 = h2 > h_bytes2 ? h2 : h_bytes2;
        const int v = (max_edge_vals > 1 ? max_edge_vals : 1) * fpw;
        v_words = v > v_words ? v : v_words;
    }
};

__device__ inline const DevFrame &frame_at(const LaunchArgs &a, int f) {
    return a.frames ? a.frames[f] : a.single;
}

// Maps a global work index to (frame, local index): by a division when
// every frame has the same number of units, else by binary search through
// the prefix array.
__device__ inline int locate(const LaunchArgs &a, const int32_t *pre, int single_count, int g, int *local) {
    if (!a.frames) {
        *local = g;
        return 0;
    }
    if (a.uniform) {
        const int f = g / single_count;
        *local = g - f * single_count;
        return f;
    }
    int lo = 0, hi = a.nframes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= g) lo = mid; else hi = mid - 1;
    }
    *local = g - pre[lo];
    return lo;
}

// Records an event on s: as an external event node when s is being
// captured into a graph (so the event is recorded on every replay), as a
// plain record otherwise.
inline cudaError_t record_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, s);
}

// Kernel attributes for the largest shapes; call once per device before launching.
int prepare_tables_kernel();
int prepare_search_kernels();

// Launchers (return cudaError_t as int).
int launch_texture(const LaunchArgs &a, int total_ctus, void *stream);
int launch_tables(const LaunchArgs &a, int total_groups, int maxC, int maxR, void *stream);
// Launch shapes of the search kernels, chosen by trs_autotune.
struct SearchTune {  // defaults: what trs_autotune picks for 2160p frames on GB300
    int band_warps = 2;  // warps per block of the row-DP kernels (2, 4 or 8)
    int col_warps = 4;   // warps per block of the column-DP kernels (1, 2, 4 or 8)
    int col_batch = 4;   // 4: a column-DP warp runs one window for 32 / col_lanes(n) frames; 8: for one frame
};
inline int col_fpw(int n, const SearchTune &t) { return t.col_batch == 8 ? 1 : 32 / col_lanes(n); }

// scal: the T_min / Q* words of every frame of the launch (reset to +inf first).
// ev (optional, 6 events): recorded after each of the six search kernels.
// maxC / maxR / maxN: largest C, R and n over the frames of the launch (shared-memory sizing);
// max_nd: largest HostPlan::max_nd over them (0: size for maxR heights).
// col: the column DP's geometry (see ColGeom; a's col_* fields describe its units).
int launch_search(const LaunchArgs &a, int total_bands, int total_windows, int maxC, int maxR, int maxN,
                  uint64_t *scal, size_t nscal, void *stream, const ColGeom &col, cudaEvent_t *ev = nullptr,
                  const SearchTune *tune = nullptr, int steps = 3, int max_nd = 0);
// steps: 1 = step 1 only (resets scal first), 2 = step 2, rebuild and decode
// only (scal[0] must already hold T_min and scal[1] +infinity), 3 = both.

}  // namespace trs
