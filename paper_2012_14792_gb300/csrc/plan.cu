// Search plan of a frame shape: which area windows exist and which row-DP
// units ("items") the windows of every tile column reduce to.  It depends on
// (W, H, n, k) only -- never on frame content -- and is built once per shape,
// like the launch geometry of the kernels.
//
// Windows (Sec. 2.3's rule k*A_min > A_max made local): every slice area a
// with a*n <= W*H and (k*a - 1)*n >= W*H gives the window [a, k*a - 1]; a
// partition meets the rule iff all its slice areas fit one such window.
//
// Items: for tile column b of pixel width w and window [a, k*a-1], a slice of
// pixel height h is admissible iff a <= w*h <= k*a-1.  The columns left and
// right of the band, of areas AL and AR, hold the other slices, so the band
// takes between n - floor(AL/a) - floor(AR/a) and
// n - ceil(AL/(k*a-1)) - ceil(AR/(k*a-1)) of them, and at least
// ceil(H/hmax), at most floor(H/hmin) slices of its admissible heights cover
// its H pixel rows (necessary conditions); a band with no count meeting all
// of them is left out of the window, and each item keeps the widest range
// over its windows (kmin, kmax).  Slice heights come
// from a short sorted list, so the admissible heights are a range [hlo, hhi]
// of that list.  Consecutive windows often give a column the same range;
// each distinct (column, range) becomes one item, shared by those windows.
#include <algorithm>
#include <cstdint>
#include <set>
#include <vector>

#include "plan.h"

namespace trs {

static std::vector<uint32_t> extents(int cells, int total) {
    // distinct pixel lengths of runs of whole CTUs [i, j) with the last CTU clipped
    std::set<uint32_t> s;
    for (int i = 0; i < cells; ++i)
        for (int j = i + 1; j <= cells; ++j) s.insert(line_px(j, total) - line_px(i, total));
    return std::vector<uint32_t>(s.begin(), s.end());
}

// Exact pruning of a plan: in each window keep only the (tile column, slice
// count) options that take part in some complete partition of the window
// with n slices -- a column's count k must leave the columns to its left a
// count they can reach and the columns to its right the rest (forward and
// backward reachability over slice counts, bit sets).  Column options come
// from the slice counts that tile the column's H pixel rows with its
// admissible heights, within the area bounds of build_plan.  Columns left
// without an option leave the window; items keep the union of their
// columns' options (kmin, kmax) and the windows that still use them.  Drops
// only options no partition of the window uses.
static void prune_by_reachability(HostPlan *p) {
    const int W = p->W, H = p->H, C = p->C, R = p->R, n = p->n, nb = p->nb, k = p->k;
    const int nwin = (int)p->win_a.size(), ni = (int)p->items.size();
    if (ni == 0 || n > 62) return;
    const uint64_t full = (2ull << n) - 1;  // slice counts 0..n
    // slice counts that tile the H pixel rows with each item's heights
    std::vector<uint64_t> kset(ni, 0), reach(R + 1);
    for (int i = 0; i < ni; ++i) {
        const PlanItem &it = p->items[i];
        std::fill(reach.begin(), reach.end(), 0);
        reach[0] = 1;
        for (int y = 1; y <= R; ++y)
            for (int yp = 0; yp < y; ++yp) {
                const uint32_t h = line_px(y, H) - line_px(yp, H);
                if (h >= it.hlo && h <= it.hhi) reach[y] |= (reach[yp] << 1) & full;
            }
        const int kmax = std::min(it.kmax, n);
        kset[i] = reach[R] & ~1ull & ((2ull << kmax) - 1);
    }
    std::vector<uint64_t> use(ni, 0), opt(nb), fw(C + 1), bw(C + 1);
    std::vector<int> wfirst(ni, nwin), wlast(ni, -1);
    auto spread = [&](uint64_t m, uint64_t ks) {  // OR of m << k over k in ks
        uint64_t r = 0;
        for (; ks; ks &= ks - 1) r |= m << __builtin_ctzll(ks);
        return r & full;
    };
    for (int wi = 0; wi < nwin; ++wi) {
        const uint64_t lo = p->win_a[wi], hi = (uint64_t)k * lo - 1;
        int32_t *srow = &p->slot_of[(size_t)wi * nb];
        for (int b = 0; b < nb; ++b) {
            opt[b] = 0;
            if (srow[b] < 0) continue;
            const uint64_t AL = (uint64_t)line_px(p->band_x0[b], W) * H;
            const uint64_t AR = (uint64_t)(W - line_px(p->band_x1[b], W)) * H;
            const int64_t kmax_w = (int64_t)n - (int64_t)((AL + hi - 1) / hi) - (int64_t)((AR + hi - 1) / hi);
            const int64_t kmin_w = std::max<int64_t>(1, (int64_t)n - (int64_t)(AL / lo) - (int64_t)(AR / lo));
            if (kmax_w < kmin_w) continue;
            const uint64_t win = ((2ull << kmax_w) - 1) & ~((1ull << kmin_w) - 1);
            opt[b] = kset[srow[b]] & win;
        }
        std::fill(fw.begin(), fw.end(), 0);
        std::fill(bw.begin(), bw.end(), 0);
        fw[0] = 1;
        for (int x0 = 0; x0 < C; ++x0)
            if (fw[x0])
                for (int x1 = x0 + 1; x1 <= C; ++x1) fw[x1] |= spread(fw[x0], opt[band_index(C, x0, x1)]);
        bw[C] = 1;
        for (int x1 = C; x1 > 0; --x1)
            if (bw[x1])
                for (int x0 = x1 - 1; x0 >= 0; --x0) bw[x0] |= spread(bw[x1], opt[band_index(C, x0, x1)]);
        for (int b = 0; b < nb; ++b) {
            uint64_t useful = 0;
            const uint64_t L = fw[p->band_x0[b]], Rr = bw[p->band_x1[b]];
            for (uint64_t ks = opt[b]; ks; ks &= ks - 1) {
                const int kk = __builtin_ctzll(ks);
                bool ok = false;
                for (uint64_t l = L; l && !ok; l &= l - 1) {
                    const int rest = n - kk - __builtin_ctzll(l);
                    ok = rest >= 0 && ((Rr >> rest) & 1ull);
                }
                if (ok) useful |= 1ull << kk;
            }
            if (!useful) {
                srow[b] = -1;
                continue;
            }
            const int it = srow[b];
            use[it] |= useful;
            wfirst[it] = std::min(wfirst[it], wi);
            wlast[it] = std::max(wlast[it], wi);
        }
    }
    // keep the used items, in order, with their option ranges
    std::vector<int32_t> remap(ni, -1);
    std::vector<PlanItem> kept;
    std::vector<int32_t> band_items(nb + 1, 0);
    p->max_nd = 0;
    for (int b = 0, i = 0; b < nb; ++b) {
        band_items[b] = (int32_t)kept.size();
        for (; i < p->band_items[b + 1]; ++i) {
            if (!use[i]) continue;
            PlanItem it = p->items[i];
            it.kmin = __builtin_ctzll(use[i]);
            it.kmax = 63 - __builtin_clzll(use[i]);
            it.w_first = wfirst[i];
            it.w_last = wlast[i];
            const int dlo = std::max(1, (int)((it.hlo + kCtu - 1) / kCtu));
            p->max_nd = std::max(p->max_nd, (int)(it.hhi / kCtu) - dlo + 1);
            remap[i] = (int32_t)kept.size();
            kept.push_back(it);
        }
    }
    band_items[nb] = (int32_t)kept.size();
    for (int32_t &sl : p->slot_of)
        if (sl >= 0) sl = remap[sl];
    p->items.swap(kept);
    p->band_items.swap(band_items);
}

int build_plan(int W, int H, int n, int k, HostPlan *p, int window_step) {
    if (W <= 0 || H <= 0 || n < 1 || n > kMaxN || k < 1 || window_step < 1) return TRS_EINVAL;
    const int C = (W + kCtu - 1) / kCtu, R = (H + kCtu - 1) / kCtu;
    if (C > kMaxC || R > kMaxR) return TRS_EINVAL;
    p->W = W;
    p->H = H;
    p->C = C;
    p->R = R;
    p->n = n;
    p->k = k;
    p->nb = num_bands(C);
    p->A = (uint64_t)W * (uint64_t)H;
    const std::vector<uint32_t> ws = extents(C, W), hs = extents(R, H);
    std::set<uint64_t> wins;
    for (uint32_t w : ws)
        for (uint32_t h : hs) {
            const uint64_t a = (uint64_t)w * h;
            if (a * (uint64_t)n <= p->A && ((uint64_t)k * a - 1) * (uint64_t)n >= p->A) wins.insert(a);
        }
    p->win_a.assign(wins.begin(), wins.end());
    if (window_step > 1) {
        std::vector<uint64_t> kept;
        const int all = (int)p->win_a.size();
        for (int i = 0; i < all; ++i)
            if ((all - 1 - i) % window_step == 0) kept.push_back(p->win_a[i]);
        p->win_a.swap(kept);
    }
    const int nwin = (int)p->win_a.size();
    p->band_x0.resize(p->nb);
    p->band_x1.resize(p->nb);
    for (int x0 = 0; x0 < C; ++x0)
        for (int x1 = x0 + 1; x1 <= C; ++x1) {
            const int b = band_index(C, x0, x1);
            p->band_x0[b] = (int16_t)x0;
            p->band_x1[b] = (int16_t)x1;
        }
    p->items.clear();
    p->max_nd = 0;
    p->slot_of.assign((size_t)nwin * p->nb, -1);
    p->band_items.assign(p->nb + 1, 0);
    for (int b = 0; b < p->nb; ++b) {
        p->band_items[b] = (int32_t)p->items.size();
        const uint64_t wb = line_px(p->band_x1[b], W) - line_px(p->band_x0[b], W);
        // the columns left and right of the band hold the other slices
        const uint64_t AL = (uint64_t)line_px(p->band_x0[b], W) * H;
        const uint64_t AR = (uint64_t)(W - line_px(p->band_x1[b], W)) * H;
        int prev_lo = -1, prev_hi = -1, prev_slot = -1, kmax_w_max = 0;
        for (int wi = 0; wi < nwin; ++wi) {
            const uint64_t lo = p->win_a[wi], hi = (uint64_t)k * lo - 1;
            // admissible heights: lo <= wb*h <= hi
            int ilo = 0;
            while (ilo < (int)hs.size() && wb * hs[ilo] < lo) ++ilo;
            int ihi = (int)hs.size() - 1;
            while (ihi >= 0 && wb * hs[ihi] > hi) --ihi;
            if (ilo > ihi) continue;
            // slice counts the band can take in this window: a part of area
            // A made of slices with areas in [lo, hi] has between ceil(A/hi)
            // and floor(A/lo) of them, and the n slices add up
            const int64_t kmax_w = (int64_t)n - (int64_t)((AL + hi - 1) / hi) - (int64_t)((AR + hi - 1) / hi);
            const int64_t kmin_w = std::max<int64_t>(1, (int64_t)n - (int64_t)(AL / lo) - (int64_t)(AR / lo));
            // and k slices of heights in [hs[ilo], hs[ihi]] cover the band's H rows of pixels
            const int64_t kgeo_lo = ((int64_t)H + hs[ihi] - 1) / hs[ihi], kgeo_hi = (int64_t)H / hs[ilo];
            if (std::max(kmin_w, kgeo_lo) > std::min(kmax_w, kgeo_hi)) {  // no partition of this window uses the band
                prev_lo = prev_hi = -1;  // an item's windows stay consecutive (exact step-2 liveness)
                continue;
            }
            if (ilo == prev_lo && ihi == prev_hi) {
                PlanItem &it = p->items[prev_slot];
                p->slot_of[(size_t)wi * p->nb + b] = prev_slot;
                it.w_last = wi;
                it.kmin = std::min<int32_t>(it.kmin, (int32_t)kmin_w);
                kmax_w_max = std::max<int>(kmax_w_max, (int)kmax_w);
                it.kmax = std::min(std::min(std::min(n, R), (int)(H / it.hlo)), kmax_w_max);
                continue;
            }
            PlanItem it;
            it.b = b;
            it.w_first = it.w_last = wi;
            it.hlo = hs[ilo];
            it.hhi = hs[ihi];
            kmax_w_max = (int)kmax_w;
            it.kmax = std::min(std::min(std::min(n, R), (int)(H / it.hlo)), kmax_w_max);
            it.kmin = (int32_t)kmin_w;
            const int dlo = std::max(1, (int)((it.hlo + kCtu - 1) / kCtu));
            p->max_nd = std::max(p->max_nd, (int)(it.hhi / kCtu) - dlo + 1);
            prev_lo = ilo;
            prev_hi = ihi;
            prev_slot = (int)p->items.size();
            p->items.push_back(it);
            p->slot_of[(size_t)wi * p->nb + b] = prev_slot;
        }
    }
    p->band_items[p->nb] = (int32_t)p->items.size();
    prune_by_reachability(p);
    column_program(p);
    return TRS_OK;
}

void column_program(HostPlan *p) {
    const int C = p->C, nb = p->nb, nwin = (int)p->win_a.size();
    p->slot_k.assign((size_t)nwin * nb, 0);
    p->max_edge_vals = 1;
    for (int w = 0; w < nwin; ++w)
        for (int x = 0; x < C; ++x) {
            int vals = 0;
            for (int x1 = x + 1; x1 <= C; ++x1) {
                const int b = band_index(C, x, x1);
                const int sl = p->slot_of[(size_t)w * nb + b];
                if (sl < 0) continue;
                const PlanItem &it = p->items[sl];
                const int klo = std::max(1, (int)it.kmin), khi = std::min((int)it.kmax, p->n);
                if (khi < klo) continue;  // no slice count of this item completes a partition
                p->slot_k[(size_t)w * nb + b] = pack_slot_k(sl, klo, khi);
                vals += khi - klo + 1;
            }
            p->max_edge_vals = std::max(p->max_edge_vals, vals);
        }
}

// Counting column DP: partitions of the C CTU columns into tile columns whose
// slice counts add up to n, g[b * (n + 1) + k] ways for tile column b with k
// slices.
static unsigned __int128 combine_columns(int C, int n, const std::vector<unsigned __int128> &g) {
    std::vector<unsigned __int128> F((size_t)(C + 1) * (n + 1), 0);
    F[0] = 1;  // columns [0, 0) in 0 slices
    for (int x = 1; x <= C; ++x)
        for (int xp = 0; xp < x; ++xp) {
            const unsigned __int128 *gb = &g[(size_t)band_index(C, xp, x) * (n + 1)];
            for (int m = 1; m <= n; ++m)
                for (int k = 1; k <= m; ++k) F[(size_t)x * (n + 1) + m] += gb[k] * F[(size_t)xp * (n + 1) + m - k];
        }
    return F[(size_t)C * (n + 1) + n];
}

// Counting row DP of one tile column: cnt[k] = ways to cut its R CTU rows
// into k slices whose pixel heights h pass keep(h).
template <class Keep>
static void count_rows(int H, int R, int n, Keep keep, std::vector<unsigned __int128> &cnt) {
    cnt.assign((size_t)(R + 1) * (n + 1), 0);
    cnt[0] = 1;  // rows [0, 0) in 0 slices
    for (int y = 1; y <= R; ++y)
        for (int yp = 0; yp < y; ++yp) {
            if (!keep(line_px(y, H) - line_px(yp, H))) continue;
            for (int k = 1; k <= n; ++k) cnt[(size_t)y * (n + 1) + k] += cnt[(size_t)yp * (n + 1) + k - 1];
        }
}

// Partitions with exactly n slices, one tile row, all slice areas in
// [lo, hi]: a counting row DP per tile column, then a counting column DP.
static unsigned __int128 count_in_range(int W, int H, int C, int R, int n, uint64_t lo, uint64_t hi) {
    std::vector<unsigned __int128> g((size_t)num_bands(C) * (n + 1), 0), cnt;
    for (int x0 = 0; x0 < C; ++x0)
        for (int x1 = x0 + 1; x1 <= C; ++x1) {
            const uint64_t w = line_px(x1, W) - line_px(x0, W);
            count_rows(H, R, n, [&](uint32_t h) { return w * h >= lo && w * h <= hi; }, cnt);
            for (int k = 0; k <= n; ++k) g[(size_t)band_index(C, x0, x1) * (n + 1) + k] = cnt[(size_t)R * (n + 1) + k];
        }
    return combine_columns(C, n, g);
}

// The same count for window wi of a plan, through the plan only: a tile
// column counts through its item in that window (none: it is left out),
// with the item's heights and its slice counts kmin..kmax.
static unsigned __int128 count_planned(const HostPlan &p, int wi) {
    const int n = p.n;
    std::vector<unsigned __int128> g((size_t)p.nb * (n + 1), 0), cnt;
    for (int b = 0; b < p.nb; ++b) {
        const int slot = p.slot_of[(size_t)wi * p.nb + b];
        if (slot < 0) continue;
        const PlanItem &it = p.items[slot];
        count_rows(p.H, p.R, n, [&](uint32_t h) { return h >= it.hlo && h <= it.hhi; }, cnt);
        for (int k = std::max(1, (int)it.kmin); k <= std::min(n, (int)it.kmax); ++k)
            g[(size_t)b * (n + 1) + k] = cnt[(size_t)p.R * (n + 1) + k];
    }
    return combine_columns(p.C, n, g);
}

int plan_coverage(int W, int H, int n, int k, int window_step, int *windows, int *short_windows,
                  double *in_windows) {
    if (!windows || !short_windows || !in_windows) return TRS_EINVAL;
    HostPlan p;
    const int st = build_plan(W, H, n, k, &p, window_step);
    if (st != TRS_OK) return st;
    // every slice area, ascending: the area just above a window's own
    std::set<uint64_t> all;
    for (uint32_t w : extents(p.C, W))
        for (uint32_t h : extents(p.R, H)) all.insert((uint64_t)w * h);
    int bad = 0;
    unsigned __int128 total = 0;
    for (int wi = 0; wi < (int)p.win_a.size(); ++wi) {
        const uint64_t lo = p.win_a[wi], hi = (uint64_t)k * lo - 1;
        const unsigned __int128 full = count_in_range(W, H, p.C, p.R, n, lo, hi);
        if (count_planned(p, wi) != full) ++bad;
        // partitions whose smallest slice area is this window's
        total += full;
        const auto next = all.upper_bound(lo);
        if (next != all.end() && *next <= hi) total -= count_in_range(W, H, p.C, p.R, n, *next, hi);
    }
    *windows = (int)p.win_a.size();
    *short_windows = bad;
    *in_windows = (double)(long double)total;
    return TRS_OK;
}

int count_partitions(int W, int H, int n, int k, long double *out) {
    if (W <= 0 || H <= 0 || n < 1 || n > kMaxN || k < 1 || !out) return TRS_EINVAL;
    const int C = (W + kCtu - 1) / kCtu, R = (H + kCtu - 1) / kCtu;
    if (C > kMaxC || R > kMaxR) return TRS_EINVAL;
    // every slice area, ascending
    std::set<uint64_t> areas;
    for (uint32_t w : extents(C, W))
        for (uint32_t h : extents(R, H)) areas.insert((uint64_t)w * h);
    const std::vector<uint64_t> a(areas.begin(), areas.end());
    // each partition counted once, at its smallest slice area m: all areas in
    // [m, k*m - 1] minus those with all areas in (m, k*m - 1]
    unsigned __int128 total = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        const uint64_t m = a[i], hi = (uint64_t)k * m - 1;
        if (m * (uint64_t)n > (uint64_t)W * H || hi * (uint64_t)n < (uint64_t)W * H) continue;
        total += count_in_range(W, H, C, R, n, m, hi);
        if (i + 1 < a.size() && a[i + 1] <= hi) total -= count_in_range(W, H, C, R, n, a[i + 1], hi);
    }
    *out = (long double)total;
    return TRS_OK;
}

size_t plan_blob_bytes(const HostPlan &p) {
    size_t s = align256(sizeof(DevPlan));
    s += align256(p.win_a.size() * sizeof(uint64_t) + 8);
    s += align256(p.items.size() * sizeof(PlanItem) + 16);
    s += align256(p.slot_of.size() * sizeof(int32_t) + 4);
    s += 2 * align256(p.band_x0.size() * sizeof(int16_t) + 2);
    s += align256(p.band_items.size() * sizeof(int32_t) + 4);
    s += align256(p.slot_k.size() * sizeof(uint64_t) + 8);
    return s;
}

void plan_serialize(const HostPlan &p, uint8_t *dev_base, std::vector<uint8_t> &blob) {
    blob.assign(plan_blob_bytes(p), 0);
    size_t off = align256(sizeof(DevPlan));
    DevPlan d;
    d.W = p.W;
    d.H = p.H;
    d.C = p.C;
    d.R = p.R;
    d.n = p.n;
    d.k = p.k;
    d.nb = p.nb;
    d.nwin = (int)p.win_a.size();
    d.nitems = (int)p.items.size();
    d.A = p.A;
    auto put = [&](const void *src, size_t bytes, size_t pad) -> const void * {
        std::copy((const uint8_t *)src, (const uint8_t *)src + bytes, blob.begin() + off);
        const void *dp = dev_base + off;
        off += align256(bytes + pad);
        return dp;
    };
    d.win_a = (const uint64_t *)put(p.win_a.data(), p.win_a.size() * sizeof(uint64_t), 8);
    d.items = (const PlanItem *)put(p.items.data(), p.items.size() * sizeof(PlanItem), 16);
    d.slot_of = (const int32_t *)put(p.slot_of.data(), p.slot_of.size() * sizeof(int32_t), 4);
    d.band_x0 = (const int16_t *)put(p.band_x0.data(), p.band_x0.size() * sizeof(int16_t), 2);
    d.band_x1 = (const int16_t *)put(p.band_x1.data(), p.band_x1.size() * sizeof(int16_t), 2);
    d.band_items = (const int32_t *)put(p.band_items.data(), p.band_items.size() * sizeof(int32_t), 4);
    d.slot_k = (const uint64_t *)put(p.slot_k.data(), p.slot_k.size() * sizeof(uint64_t), 8);
    d.max_edge_vals = p.max_edge_vals;
    std::copy((const uint8_t *)&d, (const uint8_t *)&d + sizeof(d), blob.begin());
}

// Per-frame search scratch of a plan, in bytes (256-aligned pieces).
SearchScratch scratch_layout(const HostPlan &p) {
    SearchScratch s;
    const size_t v = (size_t)p.items.size() * (p.n + 1) * 8;
    const size_t nw = p.win_a.size();
    size_t o = 0;
    s.V1 = o;    o += align256(v + 8);
    s.V2 = o;    o += align256(v + 8);
    s.w1 = o;    o += align256(nw * 8 + 8);
    s.w2 = o;    o += align256(nw * 8 + 8);
    s.H2 = o;    o += align256(nw * (size_t)(p.C + 1) * (p.n + 1) * 8 + 8);
    s.codes = o; o += align256(nw * sizeof(WinCode) + 8);
    s.bytes = o;
    return s;
}

}  // namespace trs
