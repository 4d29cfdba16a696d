// Multi-tile rectangular slices: the search over the wider slice shapes of
// Sec. 1 / Fig. 1b, where a rectangular slice is either a run of whole CTU
// rows inside one tile or a rectangle of whole tiles.
//
// With the tile grid free, this space is exactly the partitions of the CTU
// grid into n rectangles: a valid slice set is such a partition, and any such
// partition is realised by the tile grid whose column and row lines are all
// of the slices' edges (every slice is then a rectangle of whole tiles).
// No decomposition like the single-tile-row search holds, so the space is
// enumerated:
//
//  * host, once per frame shape: the first free CTU in raster order is the
//    top-left corner of the next slice; its height, then its width, grow in
//    turn.  Every partition is made once, its slices come in raster order and
//    the partitions in increasing (y0, x0, y1, x1, ...) order, which is the
//    tie order.  The k*A_min > A_max rule (luma samples) prunes: a new slice
//    must keep the rule among the slices so far, and the free area must fit
//    the slices left; so does the corner count of the free region, which
//    bounds the slices it needs from below.  The enumeration yields
//    (y0, x0, y1, x1) bytes per slice; the partitions under each choice of
//    the first two slices are enumerated on a pool of host threads and the
//    pieces joined in that order.  The device keeps, slice-major, each
//    slice's index into the region tables' rectangle entries (any
//    rectangle of CTUs is a tile-column slice there): 16-bit when every
//    index fits, else 32-bit.
//  * device, one captured graph per call: a pass streams the list through
//    shared memory (asynchronous copies, the next tile in flight while the
//    current one is evaluated) and takes T_min (Eq. 3); a second keeps, per
//    block, the smallest (Q, list index) among the sets within Eq. 4's
//    bound, so Q* (Eq. 2) and the first set reaching it come out together;
//    the last block of that pass to finish reduces the blocks' pairs in one
//    warp and decodes the winner.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

#include "ctx.h"
#include "trs_internal.cuh"

namespace trs {

namespace {

constexpr int64_t kMtMaxSets = 1 << 22;        // slice sets kept
constexpr size_t kMtMaxBytes = size_t(1) << 28;  // bytes of the kept list
constexpr int64_t kMtMaxVisits = 1ll << 28;    // partial partitions visited
constexpr int kMtPrefix = 2;                   // slices fixed per host task
constexpr int kMtMaxThreads = 64;
constexpr int64_t kMtFlush = 1 << 14;          // local counts added to the shared ones this often

// Counts shared by the host threads of one enumeration: exact totals are
// summed at the end; these (lower bounds of them) only stop the threads early.
struct MtShared {
    std::atomic<int64_t> visits{0}, sets{0};
    std::atomic<bool> over{false};
    int64_t max_sets = kMtMaxSets;
};

// A partial partition with kMtPrefix slices placed: the state rec() resumes.
struct MtTask {
    uint8_t cur[kMtPrefix][4];
    uint64_t amin, amax;
    int ry;
};

struct MtEnum {
    int W, H, C, R, n, k;
    uint64_t freem[kMaxR];   // per CTU row: free CTUs, bit x
    uint64_t free_area;      // luma samples not yet in a slice
    uint8_t cur[kMaxN][4];   // slices so far: y0, x0, y1, x1
    int ns;
    int64_t visits = 0, sets = 0;              // this enumerator's exact counts
    int64_t vflushed = 0, sflushed = 0;        // parts of them added to shared
    MtShared *shared = nullptr;
    std::vector<uint8_t> *keys = nullptr;
    std::vector<MtTask> *tasks = nullptr;      // set: stop at kMtPrefix slices and record

    void reset(int W_, int H_, int n_, int k_) {
        W = W_;
        H = H_;
        C = (W + kCtu - 1) / kCtu;
        R = (H + kCtu - 1) / kCtu;
        n = n_;
        k = k_;
        for (int y = 0; y < R; ++y) freem[y] = C == 64 ? ~0ull : (1ull << C) - 1;
        free_area = (uint64_t)W * H;
        ns = 0;
    }

    void place(int y0, int x0, int y1, int x1) {
        const uint64_t bits = ((x1 - x0 == 64 ? ~0ull : ((1ull << (x1 - x0)) - 1)) << x0);
        for (int y = y0; y < y1; ++y) freem[y] &= ~bits;
        free_area -= (uint64_t)(line_px(x1, W) - line_px(x0, W)) * (line_px(y1, H) - line_px(y0, H));
        cur[ns][0] = (uint8_t)y0;
        cur[ns][1] = (uint8_t)x0;
        cur[ns][2] = (uint8_t)y1;
        cur[ns][3] = (uint8_t)x1;
        ++ns;
    }

    bool stopped() const { return shared->over.load(std::memory_order_relaxed); }

    void flush() {
        const int64_t v = shared->visits.fetch_add(visits - vflushed, std::memory_order_relaxed) + visits - vflushed;
        const int64_t s = shared->sets.fetch_add(sets - sflushed, std::memory_order_relaxed) + sets - sflushed;
        vflushed = visits;
        sflushed = sets;
        if (v > kMtMaxVisits || s > shared->max_sets) shared->over.store(true, std::memory_order_relaxed);
    }

    // consecutive free CTUs of row y from column x
    int run(int y, int x) const {
        const uint64_t v = ~(freem[y] >> x);
        return v ? __builtin_ctzll(v) : 64 - x;
    }

    // A lower bound on the slices the free region needs: a grid point with an
    // odd number of free cells around it is one corner of the region, one
    // with two diagonal free cells is two, and each is a corner of some slice
    // in any partition of the region (m rectangles have 4m corners).  Rows
    // above ry are covered.
    int corner_bound(int ry) const {
        typedef unsigned __int128 u128;
        int corners = 0;
        u128 up = 0;
        for (int y = ry; y <= R; ++y) {
            const u128 dn = y < R ? (u128)freem[y] : 0;
            const u128 a = up << 1, b = up, c = dn << 1, d = dn;  // the 2x2 cells at each grid point
            const u128 odd = a ^ b ^ c ^ d;
            const u128 diag = (a & d & ~b & ~c) | (b & c & ~a & ~d);
            corners += __builtin_popcountll((uint64_t)odd) + __builtin_popcountll((uint64_t)(odd >> 64)) +
                       2 * (__builtin_popcountll((uint64_t)diag) + __builtin_popcountll((uint64_t)(diag >> 64)));
            up = dn;
        }
        return (corners + 3) / 4;
    }

    void emit() {
        ++sets;
        if (sets - sflushed >= kMtFlush) flush();
        if (stopped()) return;
        keys->insert(keys->end(), &cur[0][0], &cur[0][0] + (size_t)n * 4);
    }

    // amin / amax: smallest and largest slice area so far (none: ~0, 0)
    void rec(int ry, uint64_t amin, uint64_t amax) {
        if (++visits - vflushed >= kMtFlush) flush();
        if (stopped()) return;
        while (ry < R && freem[ry] == 0) ++ry;
        if (ry == R) {
            if (ns == n) emit();
            return;
        }
        if (ns == n || corner_bound(ry) > n - ns) return;
        if (tasks && ns == kMtPrefix) {
            MtTask t;
            std::memcpy(t.cur, cur, sizeof(t.cur));
            t.amin = amin;
            t.amax = amax;
            t.ry = ry;
            tasks->push_back(t);
            return;
        }
        const int x = __builtin_ctzll(freem[ry]);
        const uint64_t m = (uint64_t)(n - ns - 1);  // slices after this one
        const uint64_t px0 = line_px(x, W), py0 = line_px(ry, H);
        int maxw = C - x;
        for (int h = 1; ry + h <= R; ++h) {
            maxw = std::min(maxw, run(ry + h - 1, x));
            if (maxw == 0) break;
            const uint64_t ph = line_px(ry + h, H) - py0;
            for (int w = 1; w <= maxw; ++w) {
                const uint64_t a = (line_px(x + w, W) - px0) * ph;
                const uint64_t na = std::min(amin, a), xa = std::max(amax, a);
                if ((uint64_t)k * na <= xa) {
                    if (a >= amin) break;  // only larger areas follow in this row
                    continue;
                }
                const uint64_t f = free_area - a;
                if (m == 0 ? f != 0 : (f == 0 || (uint64_t)k * f <= m * xa || f >= m * (uint64_t)k * na))
                    continue;
                const uint64_t bits = ((w == 64 ? ~0ull : ((1ull << w) - 1)) << x);
                for (int y = ry; y < ry + h; ++y) freem[y] &= ~bits;
                cur[ns][0] = (uint8_t)ry;
                cur[ns][1] = (uint8_t)x;
                cur[ns][2] = (uint8_t)(ry + h);
                cur[ns][3] = (uint8_t)(x + w);
                ++ns;
                free_area = f;
                rec(ry, na, xa);
                free_area += a;
                --ns;
                for (int y = ry; y < ry + h; ++y) freem[y] |= bits;
                if (stopped()) return;
            }
        }
    }
};

}  // namespace

// The slice-set list of a frame shape in tie order (n * 4 bytes each).  The
// calling thread enumerates the first kMtPrefix slices of every partition in
// order; a pool of host threads enumerates the partitions under each such
// prefix, and the pieces are joined in prefix order, which is tie order.
int mt_enumerate(int W, int H, int n, int k, std::vector<uint8_t> *keys, int64_t *count) {
    if (W <= 0 || H <= 0 || n < 1 || n > kMaxN || k < 1) return TRS_EINVAL;
    const int C = (W + kCtu - 1) / kCtu, R = (H + kCtu - 1) / kCtu;
    if (C > kMaxC || R > kMaxR) return TRS_EINVAL;
    const int64_t max_sets = std::min<int64_t>(kMtMaxSets, (int64_t)(kMtMaxBytes / ((size_t)n * 4)));
    keys->clear();
    MtShared shared;
    shared.max_sets = max_sets;
    std::vector<MtTask> tasks;
    int64_t visits = 0, sets = 0;
    std::atomic<bool> nomem{false};
    try {
        MtEnum root;
        root.reset(W, H, n, k);
        root.shared = &shared;
        root.keys = keys;
        if (n > kMtPrefix) root.tasks = &tasks;
        root.rec(0, ~0ull, 0);
        root.flush();
        visits = root.visits;
        sets = root.sets;
    } catch (const std::bad_alloc &) {
        keys->clear();
        return TRS_ENOMEM;
    }
    if (!tasks.empty() && !shared.over.load()) {
        std::atomic<size_t> next{0};
        const int hw = (int)std::thread::hardware_concurrency();
        const int nt = (int)std::min<size_t>(tasks.size(), (size_t)std::max(1, std::min(hw, kMtMaxThreads)));
        std::vector<std::vector<uint8_t>> parts;
        std::vector<int64_t> wv, ws;
        std::vector<std::thread> pool;
        try {  // everything allocated before the first thread starts
            parts.resize(tasks.size());
            wv.assign(nt, 0);
            ws.assign(nt, 0);
            pool.reserve(nt);
        } catch (const std::bad_alloc &) {
            return TRS_ENOMEM;
        }
        auto work = [&](int t) {
            MtEnum e;
            e.shared = &shared;
            try {
                for (;;) {
                    const size_t i = next.fetch_add(1);
                    if (i >= tasks.size() || e.stopped()) break;
                    e.reset(W, H, n, k);
                    for (int j = 0; j < kMtPrefix; ++j)
                        e.place(tasks[i].cur[j][0], tasks[i].cur[j][1], tasks[i].cur[j][2], tasks[i].cur[j][3]);
                    e.keys = &parts[i];
                    e.rec(tasks[i].ry, tasks[i].amin, tasks[i].amax);
                }
            } catch (const std::bad_alloc &) {
                nomem.store(true);
                shared.over.store(true);
            }
            e.flush();
            wv[t] = e.visits;
            ws[t] = e.sets;
        };
        for (int t = 1; t < nt; ++t) {
            try {
                pool.emplace_back(work, t);
            } catch (const std::system_error &) {
                break;  // fewer threads: the running ones take the remaining tasks
            }
        }
        work(0);
        for (auto &th : pool) th.join();
        for (int t = 0; t < nt; ++t) {
            visits += wv[t];
            sets += ws[t];
        }
        if (!shared.over.load() && visits <= kMtMaxVisits && sets <= max_sets) {
            try {
                keys->reserve((size_t)sets * n * 4);
                for (auto &p : parts) {
                    keys->insert(keys->end(), p.begin(), p.end());
                    std::vector<uint8_t>().swap(p);
                }
            } catch (const std::bad_alloc &) {
                nomem.store(true);
            }
        }
    }
    if (nomem.load()) {
        std::vector<uint8_t>().swap(*keys);
        return TRS_ENOMEM;
    }
    if (shared.over.load() || visits > kMtMaxVisits || sets > max_sets) {
        std::vector<uint8_t>().swap(*keys);
        return TRS_EINVAL;
    }
    *count = sets;
    return TRS_OK;
}

namespace {

constexpr int kMtThreads = 256;
constexpr int kMtStageBytes = 32 * 1024;  // one tile's slice indices (two tiles in flight per block)

struct MtArgs {
    const void *ent;      // slice i of set c at ent[i * pitch + c]: its rectangle-table entry index,
                          // 16-bit when every entry index fits (e16), else 32-bit
    int64_t count;        // slice sets
    int64_t pitch;        // count rounded up to 16-byte rows (a multiple of 8 or 4 entries)
    int n, C, R, W, H, nblocks;
    int e16;              // 1: 16-bit entries
    int tile;             // sets per tile: a multiple of kMtThreads with n * tile * entry bytes <= kMtStageBytes
    const MtCall *call;   // tables, output, lambda of this call
    uint64_t *tmin;       // T_min: +infinity before the first pass (set at creation, reset by each decode)
    uint64_t *part;       // [nblocks][2]: each block's smallest (Q, set) of the second pass
    unsigned *done;       // blocks of the second pass that have stored their pair (0 between searches)
};

__device__ void mt_finish_warp(const MtArgs &a);

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// The smaller of (q, c) and the pair in lane ^ o, Q first, then the list index.
__device__ __forceinline__ void pair_min_xor(uint64_t &q, uint64_t &c, int o) {
    const uint64_t q2 = __shfl_xor_sync(0xffffffffu, q, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
    if (q2 < q || (q2 == q && c2 < c)) {
        q = q2;
        c = c2;
    }
}

__device__ __forceinline__ void mt_cp16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void mt_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void mt_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Copies tile t's slice indices (n rows of up to `tile` entries of type E,
// 16 bytes at a time) into a stage buffer with asynchronous copies.
template <typename E>
__device__ __forceinline__ void mt_stage(const MtArgs &a, E *stage, int64_t t) {
    constexpr int per = 16 / (int)sizeof(E);  // entries per 16-byte copy
    const E *ent = static_cast<const E *>(a.ent);
    const int64_t c0 = t * a.tile;
    const int64_t rest = a.pitch - c0;
    const int len = rest < a.tile ? (int)rest : a.tile;  // a multiple of per
    const int q = len / per;
    for (int i = 0; i < a.n; ++i) {
        const E *src = ent + (size_t)i * a.pitch + c0;
        E *dst = stage + (size_t)i * a.tile;
        for (int o = threadIdx.x; o < q; o += kMtThreads) mt_cp16(dst + per * o, src + per * o);
    }
}

// Both passes stream the slice-major list through shared memory, two tiles
// in flight per block (the next tile's copies run while the current one is
// evaluated), blocks striding over the tiles.  Per set: the time (max over
// slices, Eq. 1) and, in the second pass, the quality term (sum, Eq. 2),
// gathered from the region tables (any rectangle of CTUs is a tile-column
// slice there; the tables stay in L1/L2).
//  PASS 1: T_min (Eq. 3): per-thread minima, one atomic minimum per warp.
//  PASS 2: among the sets within Eq. 4's bound, the smallest (Q, list
//          index) -- Q* (Eq. 2) and the first set reaching it in one go;
//          each block stores its own minimum; the last block to do so
//          reduces them and decodes the winner.
// Time and quality term of one set of N slices (N a compile-time count):
// col[i * stride] holds slice i's rectangle-table index.  A frame whose
// total time is below 2^31 (the tables' flag) reads only the low words of
// its times.  The quality terms are gathered (second pass) only for a set
// within Eq. 4's bound thr; *qsum is left 0 otherwise.
template <int PASS, int N, typename E>
__device__ __forceinline__ void set_eval(const E *col, int stride, const uint64_t *RT, const uint64_t *RQ,
                                         bool t32, uint64_t thr, uint64_t *tmax, uint64_t *qsum) {
    uint32_t e[N];
#pragma unroll
    for (int u = 0; u < N; ++u) e[u] = col[u * stride];
    uint64_t m = 0;
    if (t32) {
        const uint32_t *RT32 = reinterpret_cast<const uint32_t *>(RT);  // low word of entry e at 2e
        uint32_t tv[N];
#pragma unroll
        for (int u = 0; u < N; ++u) tv[u] = __ldg(RT32 + 2 * (size_t)e[u]);
        uint32_t m32 = 0;
#pragma unroll
        for (int u = 0; u < N; ++u) m32 = tv[u] > m32 ? tv[u] : m32;
        m = m32;
    } else {
        uint64_t tv[N];
#pragma unroll
        for (int u = 0; u < N; ++u) tv[u] = __ldg(RT + e[u]);
#pragma unroll
        for (int u = 0; u < N; ++u) m = tv[u] > m ? tv[u] : m;
    }
    uint64_t q = 0;
    if (PASS == 2 && m <= thr) {
        uint64_t qv[N];
#pragma unroll
        for (int u = 0; u < N; ++u) qv[u] = __ldg(RQ + e[u]);
#pragma unroll
        for (int u = 0; u < N; ++u) q += qv[u];
    }
    *tmax = m;
    *qsum = q;
}

// E: the list's entry type (16-bit only with a compiled slice count).
template <int PASS, int N, typename E>
__global__ void __launch_bounds__(kMtThreads) mt_pass_kernel(MtArgs a) {
    extern __shared__ __align__(16) uint32_t mts_raw[];
    E *mts = reinterpret_cast<E *>(mts_raw);
    __shared__ uint64_t wq[kMtThreads / 32], wc[kMtThreads / 32];
    const MtCall call = *a.call;
    const TablesOffsets off = tables_offsets(a.C, a.R);
    const bool ok = reinterpret_cast<const int32_t *>(call.tables + off.status)[0] == TRS_OK;
    const uint64_t *RT = reinterpret_cast<const uint64_t *>(call.tables + off.rect_t);
    const uint64_t *RQ = reinterpret_cast<const uint64_t *>(call.tables + off.rect_q);
    const bool t32 = ok && reinterpret_cast<const int32_t *>(call.tables + off.status)[3] != 0;
    const uint64_t thr = PASS == 2 ? eq4_threshold(*a.tmin, call.lambda_q) : 0ull;
    const int64_t ntiles = (a.count + a.tile - 1) / a.tile;
    uint64_t best = kInf, bq = kInf, bc = kInf;
    if (ok) {
        const int words = a.n * a.tile;
        int buf = 0;
        int64_t t = blockIdx.x;
        if (t < ntiles) mt_stage(a, mts, t);
        mt_commit();
        for (; t < ntiles; t += gridDim.x) {
            if (t + gridDim.x < ntiles) mt_stage(a, mts + (buf ^ 1) * words, t + gridDim.x);
            mt_commit();
            mt_wait_prev();  // this thread's copies of tile t have landed
            __syncthreads();  // and every other thread's
            const E *st = mts + buf * words;
            const int64_t c0 = t * a.tile;
            for (int s = threadIdx.x; s < a.tile; s += kMtThreads) {
                const int64_t c = c0 + s;
                if (c >= a.count) break;
                uint64_t tm = 0, q = 0;
                if constexpr (N > 0)
                    set_eval<PASS, N, E>(st + s, a.tile, RT, RQ, t32, thr, &tm, &q);
                else
                    for (int i0 = 0; i0 < a.n; i0 += 8) {
                        // eight slices' gathers in flight at a time
                        uint32_t e[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) e[u] = i0 + u < a.n ? st[(i0 + u) * a.tile + s] : 0u;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const uint64_t tv = i0 + u < a.n ? __ldg(RT + e[u]) : 0ull;
                            const uint64_t qv = PASS == 2 && i0 + u < a.n ? __ldg(RQ + e[u]) : 0ull;
                            tm = tv > tm ? tv : tm;
                            q += qv;
                        }
                    }
                if (PASS == 1) {
                    best = tm < best ? tm : best;
                } else if (tm <= thr && q < bq) {  // c grows, so the first set at a thread's minimum is kept
                    bq = q;
                    bc = (uint64_t)c;
                }
            }
            __syncthreads();  // tile t's buffer is free for tile t + 2 * gridDim.x
            buf ^= 1;
        }
    }
    if constexpr (PASS == 1) {
        best = warp_min64(best);
        if ((threadIdx.x & 31) == 0 && best != kInf)
            atomicMin(reinterpret_cast<unsigned long long *>(a.tmin), (unsigned long long)best);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pair_min_xor(bq, bc, o);
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            wq[w] = bq;
            wc[w] = bc;
        }
        __syncthreads();
        if (w == 0) {
            bq = lane < (int)(blockDim.x >> 5) ? wq[lane] : kInf;
            bc = lane < (int)(blockDim.x >> 5) ? wc[lane] : kInf;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pair_min_xor(bq, bc, o);
            // the last block to store its pair reduces and decodes (no
            // separate launch): each block's pair is made visible before
            // it is counted, and the block that takes the last ticket
            // reads them after it
            unsigned last = 0;
            if (lane == 0) {
                a.part[2 * blockIdx.x] = bq;
                a.part[2 * blockIdx.x + 1] = bc;
                __threadfence();
                last = atomicAdd(a.done, 1u) == gridDim.x - 1 ? 1u : 0u;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                if (lane == 0) *a.done = 0u;  // for the next search of this shape
                mt_finish_warp(a);
            }
        }
    }
}

// One warp: the smallest (Q, set) over the blocks of pass 2, then lane i
// decodes slice i of the winner from its rectangle-table entry.  Run by the
// last block of pass 2, or by mt_finish_kernel when the list is empty.
__device__ void mt_finish_warp(const MtArgs &a) {
    const int lane = threadIdx.x & 31;
    const MtCall call = *a.call;
    trs_mt_partition *out = call.out;
    uint64_t *words = reinterpret_cast<uint64_t *>(out);
    for (int i = lane; i < (int)(sizeof(trs_mt_partition) / 8); i += 32) words[i] = 0;
    uint64_t qstar = kInf, win = kInf;
    // eight blocks' pairs per lane in flight at a time
    for (int b0 = 0; b0 < a.nblocks; b0 += 8 * 32) {
        uint64_t pq[8], pc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = b0 + u * 32 + lane;
            pq[u] = b < a.nblocks ? __ldcg(a.part + 2 * b) : kInf;  // other blocks' stores: read from L2
            pc[u] = b < a.nblocks ? __ldcg(a.part + 2 * b + 1) : kInf;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (pq[u] < qstar || (pq[u] == qstar && pc[u] < win)) {
                qstar = pq[u];
                win = pc[u];
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pair_min_xor(qstar, win, o);
    __syncwarp();
    const TablesOffsets off = tables_offsets(a.C, a.R);
    int32_t status = reinterpret_cast<const int32_t *>(call.tables + off.status)[0];
    const uint64_t t_min = a.count > 0 ? *a.tmin : kInf;
    __syncwarp();
    if (lane == 0) *a.tmin = kInf;  // reset for the next search of this shape (calls are stream-ordered)
    if (status == TRS_OK && (t_min == kInf || win >= (uint64_t)a.count)) status = TRS_EINFEASIBLE;
    if (status != TRS_OK) {
        if (lane == 0) {
            out->status = status;
            out->n_regions = a.n;
            out->candidates = a.count;
            out->winner = -1;
        }
        return;
    }
    const uint64_t *RT = reinterpret_cast<const uint64_t *>(call.tables + off.rect_t);
    const uint64_t *RQ = reinterpret_cast<const uint64_t *>(call.tables + off.rect_q);
    const uint64_t *sat1 = reinterpret_cast<const uint64_t *>(call.tables + off.sat_s1);
    uint64_t t = 0, q = 0;
    double sse = 0.0;
    if (lane < a.n) {
        const size_t at = (size_t)lane * a.pitch + win;
        const uint32_t e = a.e16 ? static_cast<const uint16_t *>(a.ent)[at] : static_cast<const uint32_t *>(a.ent)[at];
        // e = (band * R + (y1 - y0 - 1)) * R + y0, band = band_index(C, x0, x1)
        const int R = a.R, C = a.C;
        const int y0 = (int)(e % (uint32_t)R);
        const int y1 = y0 + 1 + (int)((e / (uint32_t)R) % (uint32_t)R);
        const int b = (int)(e / ((uint32_t)R * (uint32_t)R));
        int x0 = 0;
        while (x0 + 1 < C && band_index(C, x0 + 1, x0 + 2) <= b) ++x0;
        const int x1 = x0 + 1 + (b - band_index(C, x0, x0 + 1));
        t = RT[e];
        q = RQ[e];
        const int C1 = C + 1;
        const uint64_t s1 = sat1[y1 * C1 + x1] - sat1[y0 * C1 + x1] - sat1[y1 * C1 + x0] + sat1[y0 * C1 + x0];
        const uint32_t np = (line_px(x1, a.W) - line_px(x0, a.W)) * (line_px(y1, a.H) - line_px(y0, a.H));
        uint32_t rem;
        (void)ceil_square_div(s1, np, &rem);
        sse = (double)q + (rem ? (double)(np - rem) / (double)np : 0.0);  // exact SSE = floor + fraction
        out->region[lane][0] = (int16_t)x0;
        out->region[lane][1] = (int16_t)y0;
        out->region[lane][2] = (int16_t)x1;
        out->region[lane][3] = (int16_t)y1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t tu = __shfl_xor_sync(0xffffffffu, t, o);
        t = tu > t ? tu : t;
        q += __shfl_xor_sync(0xffffffffu, q, o);
        sse += __shfl_xor_sync(0xffffffffu, sse, o);
    }
    if (lane == 0) {
        out->n_regions = a.n;
        out->candidates = a.count;
        out->winner = (int64_t)win;
        out->t_min_q = t_min;
        out->thr_q = eq4_threshold(t_min, call.lambda_q);
        out->t_q = t;
        out->q = q;
        out->t_min = (double)t_min / 65536.0;
        out->t = (double)t / 65536.0;
        out->sse = sse;
        // consistency guard: the winner's sums must reproduce the reduced minima
        out->status = (q != qstar || t > out->thr_q) ? TRS_EINFEASIBLE : TRS_OK;
    }
}

// The decode alone, for a shape whose list is empty (no pass runs).
__global__ void __launch_bounds__(32) mt_finish_kernel(MtArgs a) { mt_finish_warp(a); }

}  // namespace

void mt_free(MtEntry *me) {
    if (!me) return;
    for (int k = 0; k < kMtSlots; ++k) {
        if (me->graph[k]) cudaGraphExecDestroy(me->graph[k]);
        if (me->copied[k]) cudaEventDestroy(me->copied[k]);
    }
    if (me->call_host) cudaFreeHost(me->call_host);
    dev_free(me->cands);
    dev_free(me->work);
    delete me;
}

// Enumerates shape (W, H, n) on the host, uploads its list slice-major as
// rectangle-table entries and captures the search (argument copy, T_min
// reset, two passes, decode) as one graph.  The entry joins ctx->mt.
static int mt_create(trs_ctx *ctx, int W, int H, int n, MtEntry **out) {
    std::vector<uint8_t> keys;
    int64_t count = 0;
    TRS_TRY(mt_enumerate(W, H, n, ctx->o.k_area, &keys, &count));
    const int C = (W + kCtu - 1) / kCtu, R = (H + kCtu - 1) / kCtu;
    // 16-bit entries when every rectangle-table index fits them (1920x1080:
    // 120 tile columns x 9 x 9 entries) and the slice count has a compiled
    // kernel: half the bytes for the passes to stream
    const bool e16 = n <= 8 && (size_t)num_bands(C) * R * R <= 65536;
    const size_t esz = e16 ? 2 : 4;
    const int64_t per16 = (int64_t)(16 / esz);
    const int64_t pitch = (count + per16 - 1) / per16 * per16;  // 16-byte rows for the staged copies
    std::vector<uint32_t> ent32(e16 ? 0 : (size_t)pitch * n, 0u);
    std::vector<uint16_t> ent16(e16 ? (size_t)pitch * n : 0, 0u);
    for (int64_t c = 0; c < count; ++c)
        for (int i = 0; i < n; ++i) {
            const uint8_t *k = &keys[((size_t)c * n + i) * 4];  // y0, x0, y1, x1
            const size_t v = ((size_t)band_index(C, k[1], k[3]) * R + (k[2] - k[0] - 1)) * R + k[0];
            if (e16)
                ent16[(size_t)i * pitch + c] = (uint16_t)v;
            else
                ent32[(size_t)i * pitch + c] = (uint32_t)v;
        }
    std::vector<uint8_t>().swap(keys);
    const size_t ent_bytes = (size_t)pitch * n * esz;
    const void *ent_host = e16 ? (const void *)ent16.data() : (const void *)ent32.data();
    MtEntry *me = new (std::nothrow) MtEntry;
    if (!me) return TRS_ENOMEM;
    me->count = count;
    // tiles of up to 8 sets per thread whose n slice rows fit one stage
    // buffer, smaller when the list would not give every resident block a
    // tile; as many blocks as stay resident (two stage buffers each)
    const int tile_max = kMtThreads * std::max(1, std::min(8, kMtStageBytes / ((int)esz * kMtThreads * n)));
    const int smem_max = 2 * n * tile_max * (int)esz;
    int dev = 0, sms = 0, per_sm1 = 0, per_sm2 = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void (*k1)(MtArgs) = mt_pass_kernel<1, 0, uint32_t>, (*k2)(MtArgs) = mt_pass_kernel<2, 0, uint32_t>;
    switch (n) {  // slice counts up to 8 run a kernel compiled for that count
#define TRS_MT_N(K)                                                        \
    case K:                                                                \
        k1 = e16 ? mt_pass_kernel<1, K, uint16_t> : mt_pass_kernel<1, K, uint32_t>; \
        k2 = e16 ? mt_pass_kernel<2, K, uint16_t> : mt_pass_kernel<2, K, uint32_t>; \
        break;
        TRS_MT_N(1) TRS_MT_N(2) TRS_MT_N(3) TRS_MT_N(4) TRS_MT_N(5) TRS_MT_N(6) TRS_MT_N(7) TRS_MT_N(8)
#undef TRS_MT_N
        default: break;
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, k1, kMtThreads, smem_max);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k2, kMtThreads, smem_max);
    if (e != cudaSuccess) {
        delete me;
        return cuda_fail(e, "multi-tile launch shape");
    }
    const int64_t resident = std::max(1, sms * std::max(1, std::min(per_sm1, per_sm2)));
    const int64_t per_block = (count + resident - 1) / resident;
    const int tile = (int)std::min<int64_t>(tile_max, std::max<int64_t>(
                                                          kMtThreads, (per_block + kMtThreads - 1) / kMtThreads * kMtThreads));
    const int smem = 2 * n * tile * (int)esz;
    const int64_t ntiles = (count + tile - 1) / tile;
    const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, resident));
    // work: MtCall (4 words), T_min and the pass-2 block count (4 words), per-block pairs
    const size_t work_bytes = 8 * sizeof(uint64_t) + (size_t)nblocks * 2 * sizeof(uint64_t);
    int st = dev_alloc(me->cands, std::max<size_t>(ent_bytes, 16), &ctx->total);
    if (st == TRS_OK) st = dev_alloc(me->work, work_bytes, &ctx->total);
    auto fail = [&](int code) {
        ctx->total -= me->cands.n + me->work.n;
        mt_free(me);
        return code;
    };
    if (st != TRS_OK) return fail(st);
    if (ent_bytes) e = cudaMemcpy(me->cands.p, ent_host, ent_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&me->call_host, kMtSlots * sizeof(MtCall));
    for (int k = 0; k < kMtSlots && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&me->copied[k], cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->mt_cap) e = cudaStreamCreateWithFlags(&ctx->mt_cap, cudaStreamNonBlocking);
    // T_min starts at +infinity and the block count at 0; each search's decode resets both for the next
    if (e == cudaSuccess) e = cudaMemset((uint8_t *)me->work.p + 4 * sizeof(uint64_t), 0xff, sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMemset((uint8_t *)me->work.p + 5 * sizeof(uint64_t), 0, sizeof(uint64_t));
    if (e != cudaSuccess) return fail(cuda_fail(e, "multi-tile list upload"));
    MtArgs a;
    a.ent = me->cands.p;
    a.e16 = e16 ? 1 : 0;
    a.count = count;
    a.pitch = pitch;
    a.tile = tile;
    a.n = n;
    a.C = C;
    a.R = R;
    a.W = W;
    a.H = H;
    a.nblocks = nblocks;
    uint64_t *wk = (uint64_t *)me->work.p;
    a.call = (const MtCall *)wk;
    a.tmin = wk + 4;
    a.done = reinterpret_cast<unsigned *>(wk + 5);
    a.part = wk + 8;
    cudaStream_t cs = ctx->mt_cap;
    for (int k = 0; k < kMtSlots && e == cudaSuccess; ++k) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(wk, me->call_host + k, sizeof(MtCall), cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = record_event(me->copied[k], cs);
        if (e == cudaSuccess && count > 0) {
            k1<<<nblocks, kMtThreads, smem, cs>>>(a);
            k2<<<nblocks, kMtThreads, smem, cs>>>(a);  // its last block decodes
            e = cudaGetLastError();
        } else if (e == cudaSuccess) {
            mt_finish_kernel<<<1, 32, 0, cs>>>(a);
            e = cudaGetLastError();
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&me->graph[k], g, 0);
        if (g) cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) return fail(cuda_fail(e, "multi-tile search capture"));
    try {
        ctx->mt[std::make_tuple(W, H, n)] = me;
    } catch (const std::bad_alloc &) {
        return fail(TRS_ENOMEM);
    }
    *out = me;
    return TRS_OK;
}

}  // namespace trs

using namespace trs;

extern "C" {

int trs_mt_count(int width, int height, int n, int k, int64_t *count) {
    if (!count) return TRS_EINVAL;
    std::vector<uint8_t> keys;
    return mt_enumerate(width, height, n, k, &keys, count);
}

int trs_mt_list(int width, int height, int n, int k, uint8_t *list, size_t capacity, int64_t *count) {
    if (!count) return TRS_EINVAL;
    std::vector<uint8_t> keys;
    int64_t c = 0;
    TRS_TRY(mt_enumerate(width, height, n, k, &keys, &c));
    *count = c;
    if (!list) return TRS_OK;
    if (capacity < keys.size()) return TRS_EINVAL;
    if (!keys.empty()) std::memcpy(list, keys.data(), keys.size());
    return TRS_OK;
}

int trs_search_mt(trs_ctx *ctx, const void *tables, int W, int H, int n, float lambda, trs_mt_partition *out,
                  void *stream) {
    TRS_GUARD_BEGIN
    if (!ctx || !tables || !out || (uintptr_t)tables % 256) return TRS_EINVAL;
    TRS_TRY(check_frame(ctx, W, H));
    if (n < 1 || n > ctx->o.max_regions) return TRS_EINVAL;
    if (!std::isfinite(lambda) || lambda < 0.0f || lambda > 1000.0f) return TRS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const auto key = std::make_tuple(W, H, n);
    MtEntry *me;
    auto it = ctx->mt.find(key);
    if (it != ctx->mt.end()) {
        me = it->second;
    } else {
        TRS_TRY(mt_create(ctx, W, H, n, &me));
    }
    // slot k's graph, kMtSlots calls ago, has copied its arguments
    const int k = me->next;
    me->next = (k + 1) % kMtSlots;
    TRS_CK(cudaEventSynchronize(me->copied[k]));
    me->call_host[k].tables = (const uint8_t *)tables;
    me->call_host[k].out = out;
    me->call_host[k].lambda_q = lambda_to_q(lambda);
    TRS_CK(cudaGraphLaunch(me->graph[k], s));
    return TRS_OK;
    TRS_GUARD_END
}

}  // extern "C"
