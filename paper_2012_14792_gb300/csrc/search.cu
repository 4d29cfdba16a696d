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
// DP ("item" of the shape's plan).
//
//  band_kernel<STEP>    one warp per (frame, item): lanes are the start row
//                       y of the remaining rows [y, R); for k = 1..kmax it
//                       relaxes every admissible slice height d, pulling
//                       G_{k-1}[y+d] from lane y+d with a shuffle.  Step 1
//                       combines with max (Eq. 1), step 2 with + (Eq. 2) and
//                       drops slices whose time exceeds the Eq. 4 bound.
//  column_kernel<STEP>  one block per (frame, window): DP over tile-column
//                       right edges with lanes over the slice count m; the
//                       warps split the candidate edges and merge with a
//                       shared-memory atomicMin.  Step 1's window minima
//                       reduce into T_min (Eq. 3), step 2's into Q*.
//  finish_kernel        one warp per frame: rebuilds, in every window that
//                       reaches Q*, the smallest canonical code (smallest
//                       next edge first, then the smallest cut bits, chosen
//                       with a warp ballot), keeps the smallest over windows
//                       and decodes it into trs_partition.
#include <cuda_runtime.h>

#include "trs_internal.cuh"

namespace trs {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBandWarps = 4;       // warps per block of band_kernel
constexpr int kColThreads = 1024;   // threads per block of column_kernel

__device__ __forceinline__ int32_t frame_status(const DevFrame &fr) {
    const TablesOffsets off = tables_offsets(fr.C, fr.R);
    return *reinterpret_cast<const int32_t *>(fr.tables + off.status);
}

// Suffix row DP of one item for one warp.  After iteration k, lane y holds
// G_k[y] = best value of rows [y, R) of the band cut into k admissible
// slices (kInf if none).  Writes V[k] = G_k[0] for k = 1..n (kInf beyond
// kmax) when V != nullptr, and every layer into layers[k*32 + y] when
// layers != nullptr.
template <int STEP>
__device__ void item_dp(const DevFrame &fr, const DevPlan &pl, const PlanItem &it, uint64_t thr, uint64_t *V,
                        uint64_t *layers) {
    const int lane = threadIdx.x & 31;
    const int R = fr.R, H = fr.H;
    const TablesOffsets off = tables_offsets(fr.C, R);
    const size_t base = (size_t)it.b * R * R;
    const uint64_t *RT = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_t) + base;
    const uint64_t *RQ = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_q) + base;
    // slice row counts that can reach a pixel height in [hlo, hhi]
    const int dmin = max(1, (int)((it.hlo + kCtu - 1) / kCtu));
    const int dmax = min(R, (int)(it.hhi / kCtu) + 1);
    const uint32_t ytop = line_px(lane, H);
    uint64_t G = kInf;
    if (layers) layers[lane] = kInf;
    for (int k = 1; k <= it.kmax; ++k) {
        uint64_t best = kInf;
        for (int d = dmin; d <= dmax; ++d) {
            const int y1 = lane + d;
            const uint64_t nb = __shfl_sync(kFull, G, y1 & 31);
            const uint64_t prev = (y1 == R) ? (k == 1 ? 0ull : kInf) : nb;
            if (y1 <= R && prev != kInf) {
                const uint32_t h = line_px(y1, H) - ytop;
                if (h >= it.hlo && h <= it.hhi) {
                    const uint64_t tv = __ldg(RT + (size_t)(d - 1) * R + lane);
                    if (STEP == 1) {
                        const uint64_t v = prev > tv ? prev : tv;
                        best = v < best ? v : best;
                    } else if (tv <= thr) {
                        const uint64_t v = prev + __ldg(RQ + (size_t)(d - 1) * R + lane);
                        best = v < best ? v : best;
                    }
                }
            }
        }
        G = (lane < R) ? best : kInf;
        if (layers) layers[k * 32 + lane] = G;
        if (V) {
            const uint64_t g0 = __shfl_sync(kFull, G, 0);
            if (lane == 0) V[k] = g0;
        }
    }
    if (V && lane == 0) {
        V[0] = kInf;
        for (int k = it.kmax + 1; k <= pl.n; ++k) V[k] = kInf;
    }
}

template <int STEP>
__global__ void __launch_bounds__(kBandWarps * 32) band_kernel(LaunchArgs args, int total) {
    const int gw = blockIdx.x * kBandWarps + (threadIdx.x >> 5);
    if (gw >= total) return;
    int local;
    const int f = locate(args, args.pre.items, args.single_items, gw, &local);
    const DevFrame &fr = frame_at(args, f);
    const DevPlan &pl = *fr.plan;
    const int lane = threadIdx.x & 31;
    uint64_t *V = (STEP == 1 ? fr.V1 : fr.V2) + (size_t)local * (pl.n + 1);
    if (frame_status(fr) != TRS_OK) {
        if (lane == 0)
            for (int k = 0; k <= pl.n; ++k) V[k] = kInf;
        return;
    }
    const uint64_t thr = STEP == 2 ? eq4_threshold(fr.scal[0], fr.lambda_q) : kInf;
    item_dp<STEP>(fr, pl, pl.items[local], thr, V, nullptr);
}

// Suffix DP over tile-column edges of one window:
//   H[x][m] = min over x1 > x, k of  V[item(w, [x,x1))][k] (+|max) H[x1][m-k],
// H[C][0] = 0.  Lane m-1 owns column m of a row; warp j takes edges x1 = x+1+j, ...
template <int STEP>
__global__ void __launch_bounds__(kColThreads) column_kernel(LaunchArgs args, int total) {
    __shared__ uint64_t Hs[(kMaxC + 1) * (kMaxN + 1)];
    int w;
    const int f = locate(args, args.pre.windows, args.single_windows, blockIdx.x, &w);
    const DevFrame &fr = frame_at(args, f);
    const DevPlan &pl = *fr.plan;
    const int C = fr.C, n = pl.n, nb = pl.nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint64_t *wres = STEP == 1 ? fr.wres1 : fr.wres2;
    const uint64_t *V = STEP == 1 ? fr.V1 : fr.V2;
    if (frame_status(fr) != TRS_OK) {
        if (threadIdx.x == 0) wres[w] = kInf;
        return;
    }
    if (STEP == 2) {
        // a window whose best time breaks Eq. 4 holds no step-2 candidate
        const uint64_t thr = eq4_threshold(fr.scal[0], fr.lambda_q);
        if (fr.wres1[w] > thr) {
            if (threadIdx.x == 0) wres[w] = kInf;
            return;
        }
    }
    const int stride = n + 1;
    for (int i = threadIdx.x; i < (C + 1) * stride; i += blockDim.x) Hs[i] = kInf;
    __syncthreads();
    if (threadIdx.x == 0) Hs[C * stride] = 0;
    __syncthreads();
    const int32_t *slot_row = pl.slot_of + (size_t)w * nb;
    for (int x = C - 1; x >= 0; --x) {
        for (int x1 = x + 1 + warp; x1 <= C; x1 += nwarps) {
            const int slot = slot_row[band_index(C, x, x1)];
            if (slot < 0) continue;
            const int kmax = pl.items[slot].kmax;
            const uint64_t *Vb = V + (size_t)slot * stride;
            const uint64_t vk = lane < n ? Vb[lane + 1] : kInf;  // lane k-1 holds V[k]
            const uint64_t *Hrow = Hs + x1 * stride;
            const int m = lane + 1;
            uint64_t acc = kInf;
            for (int k = 1; k <= kmax; ++k) {
                const uint64_t v = __shfl_sync(kFull, vk, k - 1);
                if (v != kInf && m >= k && m <= n) {
                    const uint64_t h = Hrow[m - k];
                    if (h != kInf) {
                        const uint64_t c = STEP == 1 ? (v > h ? v : h) : v + h;
                        acc = c < acc ? c : acc;
                    }
                }
            }
            if (acc != kInf) atomicMin(reinterpret_cast<unsigned long long *>(&Hs[x * stride + m]), acc);
        }
        __syncthreads();
    }
    const uint64_t res = Hs[n];
    if (threadIdx.x == 0) {
        wres[w] = res;
        if (res != kInf) atomicMin(reinterpret_cast<unsigned long long *>(&fr.scal[STEP == 1 ? 0 : 1]), res);
    }
    if (STEP == 2) {
        uint64_t *H2 = fr.H2 + (size_t)w * (C + 1) * stride;
        for (int i = threadIdx.x; i < (C + 1) * stride; i += blockDim.x) H2[i] = Hs[i];
    }
}

struct Code {
    int c;
    int16_t xe[kMaxC + 1];
    uint32_t cut[kMaxC];
};

// '0' < '1' read from CTU line 1 downwards: compare bit-reversed words.
__device__ __forceinline__ bool bits_less(uint32_t a, uint32_t b) { return __brev(a) < __brev(b); }

__device__ bool code_less(const Code &a, const Code &b) {
    const int c = a.c < b.c ? a.c : b.c;
    for (int i = 0; i < c; ++i) {
        if (a.xe[i + 1] != b.xe[i + 1]) return a.xe[i + 1] < b.xe[i + 1];
        if (a.cut[i] != b.cut[i]) return bits_less(a.cut[i], b.cut[i]);
    }
    return false;
}

// Smallest cut bits of a k-slice split of the item's band that reaches
// layers[k][0], read greedily top-down: the largest next cut line first.
__device__ uint32_t lexmin_bits(const DevFrame &fr, const PlanItem &it, uint64_t thr, const uint64_t *layers,
                                int k) {
    const int lane = threadIdx.x & 31;
    const int R = fr.R, H = fr.H;
    const TablesOffsets off = tables_offsets(fr.C, R);
    const size_t base = (size_t)it.b * R * R;
    const uint64_t *RT = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_t) + base;
    const uint64_t *RQ = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_q) + base;
    uint32_t bits = 0;
    int y = 0;
    for (int kk = k; kk > 1; --kk) {
        const int y1 = lane;  // candidate next cut line
        bool ok = false;
        if (y1 > y && y1 < R) {
            const int d = y1 - y;
            const uint32_t h = line_px(y1, H) - line_px(y, H);
            const uint64_t nxt = layers[(kk - 1) * 32 + y1];
            if (h >= it.hlo && h <= it.hhi && nxt != kInf) {
                const size_t e = (size_t)(d - 1) * R + y;
                if (RT[e] <= thr) ok = (nxt + RQ[e] == layers[kk * 32 + y]);
            }
        }
        const unsigned m = __ballot_sync(kFull, ok);
        if (!m) return ~0u;  // unreachable when layers[kk][y] is finite
        const int cut = 31 - __clz(m);
        bits |= 1u << (cut - 1);
        y = cut;
    }
    return bits;
}

__global__ void __launch_bounds__(32) finish_kernel(LaunchArgs args) {
    __shared__ uint64_t layers[(kMaxN + 1) * 32];
    __shared__ Code best, cur;
    const int f = blockIdx.x;
    const DevFrame &fr = frame_at(args, f);
    const DevPlan &pl = *fr.plan;
    const int lane = threadIdx.x;
    const int C = fr.C, R = fr.R, n = pl.n, nb = pl.nb, stride = n + 1;
    trs_partition *out = fr.out;
    int32_t status = frame_status(fr);
    const uint64_t t_min = fr.scal[0];
    if (status == TRS_OK && t_min == kInf) status = TRS_EINFEASIBLE;
    const uint64_t qstar = fr.scal[1];
    if (status == TRS_OK && qstar == kInf) status = TRS_EINFEASIBLE;  // cannot happen: P(T_min) meets Eq. 4
    if (lane == 0) {
        out->status = status;
        out->n_regions = n;
        out->cols = C;
        out->rows = R;
        out->n_windows = pl.nwin;
        out->reserved = 0;
    }
    if (status != TRS_OK) {
        if (lane == 0) {
            out->n_tile_cols = out->n_tile_rows = 0;
            out->t_min_q = out->thr_q = out->t_q = out->q = 0;
            out->t_min = out->t = out->sse = 0.0;
            out->tile_row_mask = 0;
        }
        return;
    }
    const uint64_t thr = eq4_threshold(t_min, fr.lambda_q);
    bool have = false;
    for (int w = 0; w < pl.nwin; ++w) {
        if (fr.wres2[w] != qstar) continue;
        const uint64_t *H2 = fr.H2 + (size_t)w * (C + 1) * stride;
        const int32_t *slot_row = pl.slot_of + (size_t)w * nb;
        int x = 0, m = n, c = 0;
        bool fail = false;
        while (x < C && !fail) {
            bool found = false;
            for (int x1 = x + 1; x1 <= C && !found; ++x1) {
                const int slot = slot_row[band_index(C, x, x1)];
                if (slot < 0) continue;
                const PlanItem it = pl.items[slot];
                const uint64_t *Vb = fr.V2 + (size_t)slot * stride;
                const int k = lane + 1;
                bool ok = false;
                if (k <= m && k <= it.kmax) {
                    const uint64_t v = Vb[k], h = H2[x1 * stride + m - k];
                    ok = v != kInf && h != kInf && v + h == H2[x * stride + m];
                }
                const unsigned mask = __ballot_sync(kFull, ok);
                if (!mask) continue;
                item_dp<2>(fr, pl, it, thr, nullptr, layers);
                __syncwarp();
                uint32_t bb = 0;
                int bk = -1;
                for (unsigned mm = mask; mm; mm &= mm - 1) {
                    const int kk = __ffs(mm);  // slice count kk = bit index + 1
                    const uint32_t bits = lexmin_bits(fr, it, thr, layers, kk);
                    if (bk < 0 || bits_less(bits, bb)) {
                        bb = bits;
                        bk = kk;
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    cur.xe[c + 1] = (int16_t)x1;
                    cur.cut[c] = bb;
                }
                c++;
                m -= bk;
                x = x1;
                found = true;
            }
            if (!found) fail = true;
        }
        __syncwarp();
        if (fail) continue;
        if (lane == 0) {
            cur.c = c;
            cur.xe[0] = 0;
            if (!have || code_less(cur, best)) best = cur;
        }
        have = true;
        __syncwarp();
    }
    if (!have) {
        if (lane == 0) out->status = TRS_EINFEASIBLE;
        return;
    }
    if (lane != 0) return;
    // decode the winner: one tile row, tile columns = bands, slices top to bottom
    const TablesOffsets off = tables_offsets(C, R);
    const uint64_t *RT = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_t);
    const uint64_t *RQ = reinterpret_cast<const uint64_t *>(fr.tables + off.rect_q);
    const uint64_t *sat1 = reinterpret_cast<const uint64_t *>(fr.tables + off.sat_s1);
    uint64_t tmax = 0, qsum = 0;
    double sse = 0.0;
    int r = 0;
    out->n_tile_cols = best.c;
    out->n_tile_rows = 1;
    out->tile_row_mask = 0;
    out->row_bd[0] = 0;
    out->row_bd[1] = (int16_t)R;
    for (int i = 0; i <= best.c; ++i) out->col_bd[i] = best.xe[i];
    for (int b = 0; b < best.c; ++b) {
        const int x0 = best.xe[b], x1 = best.xe[b + 1];
        const int bi = band_index(C, x0, x1);
        out->slice_cuts[b] = best.cut[b];
        out->tile_slices[b] = (uint8_t)(__popc(best.cut[b]) + 1);
        int y0 = 0;
        for (int y = 1; y <= R; ++y) {
            if (y < R && !((best.cut[b] >> (y - 1)) & 1u)) continue;
            const size_t e = ((size_t)bi * R + (y - y0 - 1)) * R + y0;
            const uint64_t tv = RT[e], qv = RQ[e];
            tmax = tv > tmax ? tv : tmax;
            qsum += qv;
            const uint64_t s1 = sat1[y * (C + 1) + x1] - sat1[y0 * (C + 1) + x1] - sat1[y * (C + 1) + x0] +
                                sat1[y0 * (C + 1) + x0];
            const uint32_t np = (line_px(x1, fr.W) - line_px(x0, fr.W)) * (line_px(y, fr.H) - line_px(y0, fr.H));
            uint32_t rem;
            (void)ceil_square_div(s1, np, &rem);
            // exact SSE = floor + (ceil(S1^2/N) - S1^2/N)
            sse += (double)qv + (rem ? (double)(np - rem) / (double)np : 0.0);
            if (r < kMaxN) {
                out->region[r][0] = (int16_t)x0;
                out->region[r][1] = (int16_t)y0;
                out->region[r][2] = (int16_t)x1;
                out->region[r][3] = (int16_t)y;
            }
            r++;
            y0 = y;
        }
    }
    for (int b = best.c; b < kMaxC; ++b) out->slice_cuts[b] = 0;
    out->t_min_q = t_min;
    out->thr_q = thr;
    out->t_q = tmax;
    out->q = qsum;
    out->t_min = (double)t_min / 65536.0;
    out->t = (double)tmax / 65536.0;
    out->sse = sse;
    if (r != n || qsum != qstar || tmax > thr) out->status = TRS_EINFEASIBLE;  // internal consistency guard
}

}  // namespace

int launch_search(const LaunchArgs &a, int total_items, int total_windows, uint64_t *scal, size_t nscal,
                  void *stream, cudaEvent_t *ev) {
    cudaStream_t s = (cudaStream_t)stream;
    // T_min and Q* start at +infinity; the column kernels reduce into them
    cudaError_t e = cudaMemsetAsync(scal, 0xff, nscal * sizeof(uint64_t), s);
    if (e != cudaSuccess) return (int)e;
    const int bb = (total_items + kBandWarps - 1) / kBandWarps;
    auto mark = [&](int i) {
        if (ev && e == cudaSuccess) e = cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal);
    };
    if (total_items > 0) band_kernel<1><<<bb, kBandWarps * 32, 0, s>>>(a, total_items);
    mark(0);
    if (total_windows > 0) column_kernel<1><<<total_windows, kColThreads, 0, s>>>(a, total_windows);
    mark(1);
    if (total_items > 0) band_kernel<2><<<bb, kBandWarps * 32, 0, s>>>(a, total_items);
    mark(2);
    if (total_windows > 0) column_kernel<2><<<total_windows, kColThreads, 0, s>>>(a, total_windows);
    mark(3);
    finish_kernel<<<a.nframes, 32, 0, s>>>(a);
    mark(4);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}

}  // namespace trs
