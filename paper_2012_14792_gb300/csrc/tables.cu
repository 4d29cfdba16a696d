// a2: region tables of a frame.
//
//  * Tq[c] = rint(t[c] * 65536): the co-located CTU time estimates of
//    Sec. 2.1 in Q16 fixed point (t finite, 0 <= t < 65536; others flag the
//    frame TRS_ERANGE and count as 0).
//  * Summed-area tables of S1, S2 and Tq over the CTU grid.
//  * For every tile column b = [x0, x1) and every slice of CTU rows
//    [y, y + d) (y + d <= R; other entries are left unwritten): its time
//    T = sum of Tq (Eq. 1) and its quality term
//    Q = S2 - ceil(S1^2 / N), the floor of the slice's luma SSE (Eq. 2),
//    computed exactly with a 128-bit square.  Stored diagonal-major
//    ([b][d-1][y]) so that the search, which walks one slice height d at a
//    time with lanes over y, reads consecutive words.
//
// One block builds the SATs of its frame in shared memory and fills the
// table entries of kBandsPerBlock tile columns; the first block of a frame
// also writes Tq, the SATs and the frame status.
#include <cuda_runtime.h>

#include "trs_internal.cuh"

namespace trs {

namespace {

constexpr int kTabThreads = 256;

__global__ void __launch_bounds__(kTabThreads) tables_kernel(LaunchArgs args) {
    extern __shared__ __align__(16) unsigned char smem[];
    int grp;
    const int f = locate(args, args.pre.bandgrp, args.single_bandgrp, blockIdx.x, &grp);
    const DevFrame &fr = frame_at(args, f);
    const int C = fr.C, R = fr.R, W = fr.W, H = fr.H;
    const int S = (R + 1) * (C + 1);
    uint64_t *sat1 = reinterpret_cast<uint64_t *>(smem);
    uint64_t *sat2 = sat1 + S;
    uint64_t *satt = sat2 + S;
    uint32_t *tq = reinterpret_cast<uint32_t *>(satt + S);
    __shared__ int bad;
    __shared__ int bx0[kBandsPerBlock], bx1[kBandsPerBlock];
    __shared__ uint16_t slice_dy[kMaxR * (kMaxR + 1) / 2];  // (d - 1) << 8 | y of the band's slices
    const int t = threadIdx.x;
    if (t == 0) bad = 0;
    for (int i = t; i < S; i += kTabThreads) {
        sat1[i] = 0;
        sat2[i] = 0;
        satt[i] = 0;
    }
    __syncthreads();
    for (int i = t; i < R * C; i += kTabThreads) {
        const int y = i / C, x = i - y * C;
        const float tv = fr.times[i];
        uint32_t q = 0;
        if (tv >= 0.0f && tv < 65536.0f) {
            q = (uint32_t)rintf(tv * 65536.0f);  // exact scaling by 2^16, then nearest-even
        } else {
            bad = 1;  // NaN, infinities, negatives, >= 65536
        }
        tq[i] = q;
        const int s = (y + 1) * (C + 1) + (x + 1);
        sat1[s] = fr.s1[i];
        sat2[s] = fr.s2[i];
        satt[s] = q;
    }
    __syncthreads();
    // prefix along x: one thread per (array, row)
    for (int j = t; j < 3 * R; j += kTabThreads) {
        uint64_t *a = j < R ? sat1 : (j < 2 * R ? sat2 : satt);
        const int y = j % R + 1;
        uint64_t acc = 0;
        for (int x = 1; x <= C; ++x) {
            acc += a[y * (C + 1) + x];
            a[y * (C + 1) + x] = acc;
        }
    }
    __syncthreads();
    // prefix along y: one thread per (array, column)
    for (int j = t; j < 3 * C; j += kTabThreads) {
        uint64_t *a = j < C ? sat1 : (j < 2 * C ? sat2 : satt);
        const int x = j % C + 1;
        uint64_t acc = 0;
        for (int y = 1; y <= R; ++y) {
            acc += a[y * (C + 1) + x];
            a[y * (C + 1) + x] = acc;
        }
    }
    const int nb = num_bands(C);
    const int b0 = grp * kBandsPerBlock;
    if (t < kBandsPerBlock) {
        int b = b0 + t, x0 = 0;
        if (b < nb) {
            while (b >= C - x0) {  // bands of left edge x0 are C - x0 long
                b -= C - x0;
                ++x0;
            }
            bx0[t] = x0;
            bx1[t] = x0 + 1 + b;
        }
    }
    if (t < R) {  // height d = t + 1 has start rows 0 .. R - d, after those of the smaller heights
        const int first = t * R - t * (t - 1) / 2;
        for (int y = 0; y < R - t; ++y) slice_dy[first + y] = (uint16_t)(t << 8 | y);
    }
    __syncthreads();

    const TablesOffsets off = tables_offsets(C, R);
    uint64_t *rect_t = reinterpret_cast<uint64_t *>(fr.tables + off.rect_t);
    uint64_t *rect_q = reinterpret_cast<uint64_t *>(fr.tables + off.rect_q);
    const int per_band = R * R;
    const int nloc = min(kBandsPerBlock, nb - b0);
    // the R(R+1)/2 slices of each band, enumerated densely so that no lane
    // idles; entries past the frame's bottom (y + d > R) are left unwritten
    const int per_valid = R * (R + 1) / 2;
    int lb = t / per_valid, v = t - lb * per_valid;  // entry e = lb * per_valid + v, stepped by kTabThreads
    for (int e = t; e < nloc * per_valid; e += kTabThreads) {
        const int dy = slice_dy[v];
        const int dm1 = dy >> 8, y = dy & 255, y1 = y + dm1 + 1;
        const size_t gi = (size_t)(b0 + lb) * per_band + (size_t)dm1 * R + y;
        const int x0 = bx0[lb], x1 = bx1[lb];
        const int i00 = y * (C + 1) + x0, i01 = y * (C + 1) + x1;
        const int i10 = y1 * (C + 1) + x0, i11 = y1 * (C + 1) + x1;
        const uint64_t T = satt[i11] - satt[i01] - satt[i10] + satt[i00];
        const uint64_t s1 = sat1[i11] - sat1[i01] - sat1[i10] + sat1[i00];
        const uint64_t s2 = sat2[i11] - sat2[i01] - sat2[i10] + sat2[i00];
        const uint32_t n = (line_px(x1, W) - line_px(x0, W)) * (line_px(y1, H) - line_px(y, H));
        uint32_t r;
        rect_t[gi] = T;
        rect_q[gi] = s2 - ceil_square_div(s1, n, &r);
        for (v += kTabThreads; v >= per_valid; v -= per_valid) ++lb;
    }
    if (grp == 0) {
        uint32_t *gtq = reinterpret_cast<uint32_t *>(fr.tables + off.tq);
        for (int i = t; i < R * C; i += kTabThreads) gtq[i] = tq[i];
        uint64_t *g1 = reinterpret_cast<uint64_t *>(fr.tables + off.sat_s1);
        uint64_t *g2 = reinterpret_cast<uint64_t *>(fr.tables + off.sat_s2);
        uint64_t *gt = reinterpret_cast<uint64_t *>(fr.tables + off.sat_t);
        for (int i = t; i < S; i += kTabThreads) {
            g1[i] = sat1[i];
            g2[i] = sat2[i];
            gt[i] = satt[i];
        }
        if (t == 0) {
            int32_t *st = reinterpret_cast<int32_t *>(fr.tables + off.status);
            const bool sample_bad = (*fr.flags & 1u) != 0;
            st[0] = (bad || sample_bad) ? TRS_ERANGE : TRS_OK;
            st[1] = W;
            st[2] = H;
            // 1 when every slice time (at most the frame total) fits 31 bits:
            // the step-1 DPs may then run on 32-bit values
            st[3] = satt[R * (C + 1) + C] < (1ull << 31) ? 1 : 0;
        }
    }
}

}  // namespace

// Raises the dynamic shared-memory limit of tables_kernel to what the
// largest frame needs (once per device, before any capture).
int prepare_tables_kernel() {
    const size_t S = (size_t)(kMaxR + 1) * (kMaxC + 1);
    const size_t smem = S * 3 * sizeof(uint64_t) + (size_t)kMaxR * kMaxC * sizeof(uint32_t);
    return (int)cudaFuncSetAttribute(tables_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int launch_tables(const LaunchArgs &a, int total_groups, int maxC, int maxR, void *stream) {
    if (total_groups <= 0) return 0;
    const size_t S = (size_t)(maxR + 1) * (maxC + 1);
    const size_t smem = S * 3 * sizeof(uint64_t) + (size_t)maxR * maxC * sizeof(uint32_t);
    tables_kernel<<<total_groups, kTabThreads, smem, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace trs
