// a1: per-CTU luma statistics, the texture measure behind Eq. 2 (Sec. 2.2):
// S1 = sum p, S2 = sum p^2 and N over every (clipped) 128x128 CTU, plus the
// largest sample for the bit-depth check.
//
// One 256-thread block per CTU.  The frame is read exactly once with 128-bit
// streaming loads (evict-first, the plane is not reused); a warp covers two
// full 256-byte CTU rows of a 10-bit plane per request, so every request is
// a whole number of 32-byte sectors.  A packed 10-bit plane (TRS_PACKED10,
// 160 bytes per CTU row) gives each thread 64 consecutive samples, five
// 16-byte loads unpacked in registers with funnel shifts.  Each thread keeps 32-bit partial sums
// (at most 64 samples of <= 12 bits per thread: 64 * 4095^2 < 2^32), widens
// S2 to 64 bits for the warp-shuffle reduction, then one shared-memory step
// combines the 8 warps.  There is no spatial stencil in the measure, so no
// halo is read.
#include <cuda_runtime.h>

#include "trs_internal.cuh"

namespace trs {

namespace {

constexpr int kTexThreads = 256;

struct Acc {
    uint32_t s1, s2;
    uint32_t vm;  // packed per-lane maxima of vector loads
    uint32_t vs;  // maximum of scalar loads
};

__device__ __forceinline__ uint4 ld_stream(const uint8_t *p) {
    return __ldcs(reinterpret_cast<const uint4 *>(p));
}

// 8 little-endian 16-bit samples
__device__ __forceinline__ void acc_u16x8(Acc &a, uint4 v) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t lo = w[i] & 0xffffu, hi = w[i] >> 16;
        a.s1 += lo + hi;
        a.s2 += lo * lo + hi * hi;
        a.vm = __vmaxu2(a.vm, w[i]);
    }
}

// 16 8-bit samples: dp4a gives the byte sum and the sum of byte squares
__device__ __forceinline__ void acc_u8x16(Acc &a, uint4 v) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a.s1 = __dp4a(w[i], 0x01010101u, a.s1);
        a.s2 = __dp4a(w[i], w[i], a.s2);
        a.vm = __vmaxu4(a.vm, w[i]);
    }
}

__device__ __forceinline__ uint32_t sample_at(const uint8_t *row, int x, int bps) {
    return bps == 1 ? (uint32_t)row[x] : ((uint32_t)row[2 * x] | ((uint32_t)row[2 * x + 1] << 8));
}

__device__ __forceinline__ void acc_scalar(Acc &a, uint32_t p) {
    a.s1 += p;
    a.s2 += p * p;
    a.vs = a.vs > p ? a.vs : p;
}

// Sample x of a TRS_PACKED10 row: bits [10x, 10x + 10) of the row's
// little-endian bit string, which always span two bytes.
__device__ __forceinline__ uint32_t packed_at(const uint8_t *row, int x) {
    const int bit = 10 * x, b = bit >> 3;
    return (((uint32_t)row[b] | ((uint32_t)row[b + 1] << 8)) >> (bit & 7)) & 1023u;
}

// 64 packed samples from 80 bytes (20 little-endian words): sample j is
// bits [10j, 10j + 10), read across a word boundary with a funnel shift.
__device__ __forceinline__ void acc_packed64(Acc &a, const uint4 (&v)[5]) {
    uint32_t wd[21];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        wd[4 * i] = v[i].x;
        wd[4 * i + 1] = v[i].y;
        wd[4 * i + 2] = v[i].z;
        wd[4 * i + 3] = v[i].w;
    }
    wd[20] = 0u;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        const int k = (10 * j) >> 5, sh = (10 * j) & 31;
        const uint32_t p = __funnelshift_r(wd[k], wd[k + 1], sh) & 1023u;
        a.s1 += p;
        a.s2 += p * p;
        a.vs = a.vs > p ? a.vs : p;
    }
}

__global__ void __launch_bounds__(kTexThreads) texture_kernel(LaunchArgs args) {
    int local;
    const int f = locate(args, args.pre.ctus, args.single_ctus, blockIdx.x, &local);
    const DevFrame &fr = frame_at(args, f);
    const int C = fr.C;
    const int cy = local / C, cx = local - cy * C;
    const int x0 = cx * kCtu, y0 = cy * kCtu;
    const int w = min(kCtu, fr.W - x0), h = min(kCtu, fr.H - y0);
    const int bps = fr.bd == 8 ? 1 : 2;
    // a packed CTU column starts 10 * 128 / 8 = 160 bytes after the previous one
    const uint8_t *base = fr.luma + (size_t)y0 * fr.pitch + (fr.packed ? (size_t)cx * 160 : (size_t)x0 * bps);
    const int t = threadIdx.x;

    Acc a = {0u, 0u, 0u, 0u};
    if (fr.packed) {
        if (fr.vec_ok && w == kCtu) {
            // thread t: row t / 2, the 64 samples in bytes [80 (t & 1), 80 (t & 1) + 80)
            // of the row's 160: five 16-byte loads
            const int r = t >> 1;
            if (r < h) {
                const uint8_t *p = base + (size_t)r * fr.pitch + 80 * (t & 1);
                uint4 v[5];
#pragma unroll
                for (int i = 0; i < 5; ++i) v[i] = __ldg(reinterpret_cast<const uint4 *>(p + 16 * i));
                acc_packed64(a, v);
            }
        } else {
            for (int r = t / kCtu; r < h; r += kTexThreads / kCtu) {
                const int x = t % kCtu;
                if (x < w) acc_scalar(a, packed_at(base + (size_t)r * fr.pitch, x));
            }
        }
    } else if (fr.vec_ok) {
        // 16-byte vectors: 16 per 10-bit row, 8 per 8-bit row
        const int vpr = (kCtu * bps) / 16;
        const int spv = 16 / bps;
        const int nvec = kCtu * vpr;
        if (w == kCtu && h == kCtu) {
            if (bps == 2) {
                uint4 v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int q = t + i * kTexThreads;
                    v[i] = ld_stream(base + (size_t)(q >> 4) * fr.pitch + (q & 15) * 16);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) acc_u16x8(a, v[i]);
            } else {
                uint4 v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int q = t + i * kTexThreads;
                    v[i] = ld_stream(base + (size_t)(q >> 3) * fr.pitch + (q & 7) * 16);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) acc_u8x16(a, v[i]);
            }
        } else {
            // clipped CTU: whole vectors where they fit, samples for the ragged tail
            for (int q = t; q < nvec; q += kTexThreads) {
                const int r = q / vpr, cv = q - r * vpr;
                if (r >= h) break;
                const int sx = cv * spv;
                if (sx >= w) continue;
                const uint8_t *row = base + (size_t)r * fr.pitch;
                if (sx + spv <= w) {
                    uint4 v = ld_stream(row + sx * bps);
                    if (bps == 2) acc_u16x8(a, v); else acc_u8x16(a, v);
                } else {
                    for (int x = sx; x < w; ++x) acc_scalar(a, sample_at(row, x, bps));
                }
            }
        }
    } else {
        // unaligned plane: one sample per step
        for (int r = t / kCtu; r < h; r += kTexThreads / kCtu) {
            const uint8_t *row = base + (size_t)r * fr.pitch;
            const int x = t % kCtu;
            if (x < w) acc_scalar(a, sample_at(row, x, bps));
        }
    }
    // lane-wise packed maxima -> scalar (a.vm stays 0 on the packed path)
    uint32_t vmax = bps == 2 ? max(a.vm & 0xffffu, a.vm >> 16)
                             : max(max(a.vm & 0xffu, (a.vm >> 8) & 0xffu), max((a.vm >> 16) & 0xffu, a.vm >> 24));
    vmax = max(vmax, a.vs);
    uint32_t s1 = a.s1;
    uint64_t s2 = a.s2;
    // warp reduction: s1 fits 32 bits for a whole CTU (16384 * 4095 < 2^32)
    s1 = __reduce_add_sync(0xffffffffu, s1);
    vmax = __reduce_max_sync(0xffffffffu, vmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    __shared__ uint32_t sh_s1[kTexThreads / 32], sh_vm[kTexThreads / 32];
    __shared__ uint64_t sh_s2[kTexThreads / 32];
    const int wid = t >> 5, lane = t & 31;
    if (lane == 0) {
        sh_s1[wid] = s1;
        sh_s2[wid] = s2;
        sh_vm[wid] = vmax;
    }
    __syncthreads();
    if (t == 0) {
        uint32_t S1 = 0, VM = 0;
        uint64_t S2 = 0;
#pragma unroll
        for (int i = 0; i < kTexThreads / 32; ++i) {
            S1 += sh_s1[i];
            S2 += sh_s2[i];
            VM = max(VM, sh_vm[i]);
        }
        const int i = cy * C + cx;
        fr.s1[i] = S1;
        fr.s2[i] = S2;
        fr.cnt[i] = (uint32_t)(w * h);
        fr.vmax[i] = VM;
        if (VM >> fr.bd) atomicOr(fr.flags, 1u);
    }
}

}  // namespace

int launch_texture(const LaunchArgs &a, int total_ctus, void *stream) {
    if (total_ctus <= 0) return 0;
    texture_kernel<<<total_ctus, kTexThreads, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace trs
