/*
 * trs.h -- C ABI of the GB300 library for dynamic tile / rectangular-slice
 * (TRS) frame partitioning, after "Quality-driven Dynamic VVC Frame
 * Partitioning for efficient Parallel Processing" (Amestoy et al., ICIP 2020).
 *
 * The hot path of the method, one frame at a time or batched:
 *   trs_texture_map    per-CTU luma statistics (the texture measure of Eq. 2,
 *                      Sec. 2.2: sum p, sum p^2 and the sample count per CTU)
 *   trs_region_tables  Q16 CTU times (the estimator values of Sec. 2.1),
 *                      summed-area tables and the per-rectangle table of
 *                      slice times (Eq. 1) and floored slice SSE (Eq. 2)
 *   trs_search         step 1: T_min = min_P T(P) (Eq. 3); step 2: the
 *                      partition minimising Eq. 2 subject to Eq. 4,
 *                      T(P) <= T_min (1 + lambda); both over the partitions
 *                      with exactly n slices and k*A_min > A_max (Sec. 2.3)
 *
 * Conventions shared by every call:
 *   - All pointers named *_dev are CUDA device pointers on the context's
 *     device; *_host are host pointers.  The caller owns every buffer it
 *     passes.  The context owns its scratch memory.  The first call that
 *     sees a new frame shape (width, height, n) builds that shape's search
 *     plan and may grow the scratch, synchronously; later calls with shapes
 *     seen before allocate nothing and only enqueue work, so warm a shape up
 *     before capturing calls in a CUDA graph.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device-pointer calls only enqueue work and return; their
 *     outputs are valid after the stream has been synchronised.  Calls that
 *     take host buffers synchronise the stream before they return.
 *   - Errors found from the arguments are returned at once (TRS_EINVAL ...).
 *     Errors that depend on the data (a sample >= 2^bit_depth, a time that
 *     is not finite or outside [0, 65536), no partition satisfying the area
 *     rule) are reported in trs_partition.status, written on the device.
 *   - A context serves one host thread at a time.  Its device scratch is
 *     reused by every call, so calls on one context must be ordered on the
 *     device: issue them on one stream, or order the streams with events.
 *     For work in flight on several streams at once, use a context each.
 *
 * Readings of the paper fixed by this library (the paper is silent on them):
 *   CTUs are 128x128 luma samples, edge CTUs clipped.  A partition has
 *   exactly n slices (one per thread, Sec. 2.1); a slice is a run of whole
 *   CTU rows inside one tile (Sec. 1).  Areas count luma samples; the area
 *   rule is 3*A_min > A_max with a strict '>'; it constrains both steps.
 *   Times are quantised Tq = rint(t * 65536); lambda_q = rint(lambda * 65536)
 *   and Eq. 4 holds iff T(P)*65536 <= T_min*(65536 + lambda_q).  The quality
 *   term of a slice is floor(SSE) = S2 - ceil(S1^2 / N).  Among partitions of
 *   equal quality the smallest canonical code wins (tile-row cut bits top to
 *   bottom, then per tile column its right edge and its slice cut bits top to
 *   bottom, '0' < '1'); such a winner never has tile-row cuts, since a slice
 *   cut at the same line gives the same slices with a smaller code.
 */
#ifndef TRS_H
#define TRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRS_ABI_VERSION 1

#define TRS_CTU 128          /* CTU edge in luma samples */
#define TRS_MAX_COLS 64      /* CTU columns: width  <= 8192 */
#define TRS_MAX_ROWS 32      /* CTU rows:    height <= 4096 */
#define TRS_MAX_REGIONS 32   /* n, slices (= threads) per frame */

/* Sample formats, passed where a call takes bit_depth:
 *   8           one byte per sample;
 *   9..12       two bytes per sample, little endian, value < 2^bit_depth;
 *   TRS_PACKED10  10-bit samples packed four in five bytes: each row is a
 *               little-endian bit string in which sample x occupies bits
 *               [10x, 10x + 10) (bytes 5j..5j+4 hold samples 4j..4j+3, the
 *               lowest bits first); a row takes ceil(10 W / 8) bytes.
 * The statistics of a packed plane equal those of the same samples in the
 * two-byte form; a packed frame moves 37.5 % fewer bytes. */
#define TRS_PACKED10 0x10A

enum trs_status {
    TRS_OK = 0,
    TRS_EINVAL = 1,       /* bad argument (null pointer, size out of range, misaligned) */
    TRS_ERANGE = 2,       /* a sample >= 2^bit_depth, or a CTU time not finite / outside [0, 65536) */
    TRS_EINFEASIBLE = 3,  /* no partition with n slices satisfies the area rule */
    TRS_ENOMEM = 4,       /* a size beyond what the context was created for, or allocation failed */
    TRS_EBUSY = 5,        /* server: admission refused (no slot or memory budget) */
    TRS_ETIMEOUT = 6,     /* a bounded device or host wait gave up */
    TRS_ECUDA = 7         /* a CUDA runtime call failed; see trs_last_error() */
};

typedef struct trs_ctx trs_ctx;

/* Limits fixed when a context is created; every later call must fit them. */
typedef struct trs_opts {
    int max_width;     /* largest luma width,  1..8192 */
    int max_height;    /* largest luma height, 1..4096 */
    int max_regions;   /* largest n, 1..TRS_MAX_REGIONS */
    int max_batch;     /* frames per batched call, >= 1 */
    int k_area;        /* area-rule factor k of Sec. 2.3 (the paper uses 3), >= 1 */
    int device;        /* CUDA device ordinal */
} trs_opts;

/* Per-CTU statistics, structure of arrays, each R*C entries, row-major over
 * the CTU grid (R = ceil(H/128) rows, C = ceil(W/128) columns).  Device
 * memory owned by the caller. */
typedef struct trs_ctu_stats {
    uint32_t *s1;      /* sum of samples */
    uint64_t *s2;      /* sum of squared samples */
    uint32_t *count;   /* samples in the (clipped) CTU */
    uint32_t *vmax;    /* largest sample */
    uint32_t *flags;   /* one word: bit 0 set if a sample was >= 2^bit_depth */
} trs_ctu_stats;

/* Byte layout of the region tables of one frame (see trs_region_tables).
 * Offsets are from the start of the caller's device buffer; every array
 * starts on a 256-byte boundary. */
typedef struct trs_tables_layout {
    int width, height, cols, rows;  /* W, H, C, R */
    int bands;                      /* C*(C+1)/2 tile-column candidates */
    int reserved;
    size_t bytes;                   /* total size of the buffer */
    size_t off_tq;       /* uint32 [R*C]: Q16 CTU times */
    size_t off_sat_s1;   /* uint64 [(R+1)*(C+1)]: sat[y][x] = sum over CTUs [0,x) x [0,y) */
    size_t off_sat_s2;   /* uint64 [(R+1)*(C+1)] */
    size_t off_sat_t;    /* uint64 [(R+1)*(C+1)], of Tq */
    size_t off_rect_t;   /* uint64 [bands][R][R]: entry (b, d-1, y) = time of the slice spanning
                            tile column b, CTU rows [y, y+d) (Eq. 1); band b of columns [x0,x1)
                            has b = x0*(2C-x0+1)/2 + (x1-x0-1); entries with y+d > R are
                            unused and left unwritten */
    size_t off_rect_q;   /* uint64 [bands][R][R]: floor of the slice's luma SSE (Eq. 2), same index */
    size_t off_status;   /* int32 [4]: [0] data status of this frame (TRS_OK / TRS_ERANGE), [1] W, [2] H,
                            [3] 1 if the frame's total Q16 time is below 2^31 */
} trs_tables_layout;

/* The decision for one frame, written by the device. */
typedef struct trs_partition {
    int32_t status;          /* TRS_OK, TRS_ERANGE or TRS_EINFEASIBLE */
    int32_t n_regions;       /* n */
    int32_t cols, rows;      /* CTU grid C, R */
    int32_t n_tile_cols;     /* tiles: n_tile_cols x n_tile_rows */
    int32_t n_tile_rows;
    int32_t n_windows;       /* area windows searched */
    int32_t reserved;
    uint64_t t_min_q;        /* Eq. 3, Q16 */
    uint64_t thr_q;          /* largest T(P) satisfying Eq. 4 */
    uint64_t t_q;            /* T(P*) (Eq. 1), Q16 */
    uint64_t q;              /* Q(P*): sum over slices of floor(SSE) (Eq. 2) */
    double t_min;            /* t_min_q / 65536 */
    double t;                /* t_q / 65536 */
    double sse;              /* exact sum of slice SSE, in double */
    uint64_t tile_row_mask;                  /* bit y-1: tile-row boundary at CTU line y */
    int16_t col_bd[TRS_MAX_COLS + 1];        /* tile-column edges, n_tile_cols + 1 entries */
    int16_t row_bd[TRS_MAX_ROWS + 1];        /* tile-row edges, n_tile_rows + 1 entries */
    uint32_t slice_cuts[TRS_MAX_COLS];       /* per tile column: bit y-1 set = slice boundary at CTU line y */
    int16_t region[TRS_MAX_REGIONS][4];      /* slices x0, y0, x1, y1 (CTU units, half-open), in tile
                                                raster order, top to bottom inside a tile */
    uint8_t tile_slices[TRS_MAX_REGIONS];    /* slices per tile, tile raster order */
} trs_partition;

/* One frame of a batched call. */
typedef struct trs_frame_desc {
    const void *luma_dev;     /* W*H samples, rows pitch_bytes apart, in the format bit_depth names
                                 (uint8, little-endian uint16 or TRS_PACKED10) */
    const float *ctu_time_dev;/* R*C co-located CTU times (Sec. 2.1), row-major */
    int width, height;
    size_t pitch_bytes;
    int bit_depth;            /* 8..12 or TRS_PACKED10 */
    int n_regions;            /* n */
    float lambda;             /* Eq. 4, >= 0 */
} trs_frame_desc;

/* --- introspection (no GPU needed) --------------------------------------- */

/* Size in bytes of the ABI structure called `name` ("trs_opts",
 * "trs_ctu_stats", "trs_tables_layout", "trs_partition", "trs_frame_desc",
 * "trs_server_opts", "trs_decision", "trs_server_stats", "trs_tune_report",
 * "trs_mt_partition"),
 * 0 for an unknown name; lets bindings check their copies of the layouts. */
size_t trs_sizeof(const char *name);

/* Search-plan figures of a frame shape: the number of area windows
 * [a, k*a - 1] (Sec. 2.3's rule made local, one per admissible smallest
 * slice area a) and of distinct row-DP units.  Pure host arithmetic.
 * TRS_EINVAL for sizes beyond the limits. */
int trs_plan_stats(int width, int height, int n_regions, int k_area, int *n_windows, int *n_items);

/* Algorithmic work of one search step of a frame shape, counted from the
 * loop bounds of its DPs: row_relax = for every row-DP unit, kmax slice
 * counts x the unit's slice heights x R start rows (a transition G_k[y] <-
 * G_{k-1}[y+d] combined with the slice value, inadmissible ones included,
 * as the DP evaluates them); col_relax = for every window and tile column
 * with slices there, the transitions H[x][m] <- V[k], H[x1][m-k] with k in
 * the unit's slice-count range [kmin, kmax] and k <= m <= n.  Each
 * transition is one combine (max for Eq. 1, + for Eq. 2) and one minimum.
 * Pure host arithmetic. */
int trs_plan_work(int width, int height, int n_regions, int k_area, double *row_relax, double *col_relax);

/* Host only: the number of distinct partitions the search chooses among,
 * i.e. of S(n) (exactly n slices, slices of whole CTU rows inside tile
 * columns, k*A_min > A_max in luma samples, Sec. 2.3) with one tile row --
 * tile rows add codes but no new partition.  Exact (128-bit counting DPs,
 * each partition counted once at its smallest slice area), returned as a
 * double.  For reporting candidates per second; TRS_EINVAL on bad shapes. */
int trs_count_partitions(int width, int height, int n_regions, int k_area, double *count);

/* Host only: checks that the search plan of a frame shape loses no
 * partition.  The plan prunes, per area window [a, k*a - 1], the tile
 * columns and slice counts that no partition of the window with n slices
 * can use; for every window this counts the one-tile-row partitions whose
 * slice areas all fit the window twice -- all of them, and those the plan's
 * row-DP units can form (each tile column through its unit in that window,
 * with the unit's heights and slice-count range) -- with 128-bit counting
 * DPs.  *short_windows = windows where the second count is smaller (0 for
 * a sound plan), *windows = windows checked.  *in_windows = partitions of
 * S(n) (one tile row) whose smallest slice area is one of the plan's
 * windows: with window_step 1 it equals trs_count_partitions when no
 * window is missing.  window_step as in trs_set_window_step.  TRS_EINVAL
 * for bad shapes. */
int trs_plan_coverage(int width, int height, int n_regions, int k_area, int window_step, int *windows,
                      int *short_windows, double *in_windows);

/* Measured INT32 throughput of the device (32-bit add / min / max chains
 * over every SM, CUDA-event timed, best of three), in operations per
 * second: the peak the search kernels' arithmetic is compared with. */
int trs_alu_peak(int device, double *ops_per_s);

/* --- context ------------------------------------------------------------ */

int trs_version(void);
const char *trs_strerror(int status);
/* Text of the last CUDA error seen by this process (thread-local), "" if none. */
const char *trs_last_error(void);

/* Creates a context on opts->device and allocates all of its scratch memory.
 * Returns TRS_EINVAL for limits out of range, TRS_ENOMEM / TRS_ECUDA on failure. */
int trs_create(trs_ctx **out, const trs_opts *opts);
/* Synchronises the context's work and frees it.  NULL is accepted. */
int trs_destroy(trs_ctx *ctx);
/* Bytes of device memory the context holds. */
size_t trs_ctx_bytes(const trs_ctx *ctx);

/* --- the hot path, one frame ------------------------------------------- */

/* a1.  Per-CTU luma statistics of one frame (Eq. 2 needs S1, S2, N of every
 * slice; they are sums of these).  luma_dev: W*H samples with rows
 * pitch_bytes apart (pitch >= the bytes of a row in the sample format:
 * W, 2 W, or ceil(10 W / 8) for TRS_PACKED10).  Samples >= 2^bit_depth
 * set stats->flags bit 0 and are still summed.  Rows and the base address
 * aligned to 16 bytes take the vector path (for TRS_PACKED10: CTUs 128
 * samples wide), others a scalar path.  TRS_EINVAL: null pointers, W/H
 * beyond the context, bit_depth neither 8..12 nor TRS_PACKED10. */
int trs_texture_map(trs_ctx *ctx, const void *luma_dev, int width, int height, size_t pitch_bytes,
                    int bit_depth, const trs_ctu_stats *stats, void *stream);

/* Fills *out with the table layout of a W x H frame.  TRS_EINVAL if the
 * frame exceeds TRS_MAX_COLS / TRS_MAX_ROWS CTUs. */
int trs_tables_layout_get(int width, int height, trs_tables_layout *out);

/* a2.  Region tables of one frame from its CTU statistics and the CTU times
 * of the co-located previous frame (the estimator of Sec. 2.1), into the
 * caller's device buffer tables_dev of tables_bytes >= layout.bytes.
 * ctu_time_dev: R*C floats.  A bad time, or stats->flags bit 0, sets the
 * frame status TRS_ERANGE (reported by trs_search). */
int trs_region_tables(trs_ctx *ctx, const trs_ctu_stats *stats, const float *ctu_time_dev, int width,
                      int height, void *tables_dev, size_t tables_bytes, void *stream);

/* a3-a5.  Both search steps of Sec. 2.3 over the tables of one frame, and the
 * decoding of the winner into out_dev (device memory, one trs_partition).
 * n_regions in 1..opts.max_regions; lambda finite, 0 <= lambda <= 1000. */
int trs_search(trs_ctx *ctx, const void *tables_dev, int width, int height, int n_regions, float lambda,
               trs_partition *out_dev, void *stream);

/* Multi-tile rectangular slices (Sec. 1, Fig. 1b: a rectangular slice may
 * also be a rectangle of several complete tiles).  The space: every tile
 * grid, its tiles grouped into rectangles of tiles; a one-tile group holds
 * k >= 1 in-tile slices (runs of whole CTU rows), a larger group is one
 * slice; exactly n slices; the k*A_min > A_max rule in luma samples.  A grid
 * with a line at every slice edge realises any partition of the CTU grid
 * into rectangles, so the space is exactly those partitions; it contains the
 * single-tile-row space of trs_search.  The search is an enumeration: the
 * host lists the slice sets of a frame shape once, in increasing order of
 * their slice lists (raster order, (y0, x0, y1, x1) per slice), one GPU
 * thread evaluates each from the region tables; ties on Q go to the first
 * set of that order.  The tile grid of the winner: column and row lines at
 * its slices' edges.  Shapes are limited by the size of the list. */
typedef struct trs_mt_partition {
    int32_t status;          /* TRS_OK, TRS_ERANGE or TRS_EINFEASIBLE */
    int32_t n_regions;
    int64_t candidates;      /* slice sets searched */
    int64_t winner;          /* index of the winner in the list, -1 if none */
    uint64_t t_min_q;        /* Eq. 3 over this space, Q16 */
    uint64_t thr_q;          /* largest time Eq. 4 admits */
    uint64_t t_q, q;         /* T(P*) and Q(P*) */
    double t_min, t, sse;    /* T_min, T(P*) in time units; exact SSE of P* */
    int16_t region[TRS_MAX_REGIONS][4];  /* x0, y0, x1, y1 in CTUs, raster order */
} trs_mt_partition;

/* Host only: the number of slice sets of the multi-tile space for a frame
 * shape (k_area as in trs_opts).  TRS_EINVAL for a shape beyond
 * TRS_MAX_COLS x TRS_MAX_ROWS CTUs, n outside 1..TRS_MAX_REGIONS, or a list
 * beyond the enumerated form (more than 2^22 slice sets, 256 MiB, or 2^28
 * partial partitions visited; 1920x1080 holds up to n = 8, 3840x2160 up to
 * n = 6, whose 2.6e6 sets take about 4 s on 8 host cores).  The list is
 * built on all host cores (std::thread) in the same order as one thread
 * would.  TRS_ENOMEM if host memory runs out.  A shape with no valid set
 * counts 0. */
int trs_mt_count(int width, int height, int n_regions, int k_area, int64_t *count);

/* Host only: the slice-set list trs_search_mt searches for a frame shape,
 * in its tie order (increasing lexicographic order of the records): *count
 * sets of n_regions slices, 4 bytes per slice (y0, x0, y1, x1 in CTUs),
 * slices in raster order of (y0, x0).  With list == NULL only *count is
 * written; otherwise list must hold capacity >= *count * n_regions * 4 bytes
 * (TRS_EINVAL if it does not; *count is still written).  Errors as
 * trs_mt_count. */
int trs_mt_list(int width, int height, int n_regions, int k_area, uint8_t *list, size_t capacity,
                int64_t *count);

/* Searches the multi-tile space of the frame whose region tables are in
 * tables_dev (trs_region_tables): T_min (Eq. 3), then the smallest Q (Eq. 2)
 * among slice sets within Eq. 4's bound.  Writes one trs_mt_partition to
 * out_dev (device memory).  The first call for a shape enumerates it on the
 * host, keeps the list on the device (one 16- or 32-bit rectangle-table index
 * per slice, slice-major) and captures the search as a CUDA graph; every call
 * then copies its arguments into the graph's pinned block (after the
 * previous call's copy has run) and launches the graph on `stream`.  Calls
 * on one context must be ordered on the device.  Errors as trs_mt_count,
 * plus TRS_EINVAL for bad arguments. */
int trs_search_mt(trs_ctx *ctx, const void *tables_dev, int width, int height, int n_regions, float lambda,
                  trs_mt_partition *out_dev, void *stream);

/* Both search steps for several trade-offs at once: the paper tries
 * lambda in {0, 0.1, 0.3} and keeps the best per resolution and thread
 * count (Sec. 3.2).  Step 1 (T_min, Eq. 3) does not depend on lambda and
 * runs once; step 2 (Eq. 2 under Eq. 4) runs for each lambda.  out_dev
 * receives n_lambdas partitions, identical to n_lambdas trs_search calls.
 * n_lambdas in 1..TRS_MAX_LAMBDAS. */
#define TRS_MAX_LAMBDAS 8
int trs_search_lambdas(trs_ctx *ctx, const void *tables_dev, int width, int height, int n_regions,
                       const float *lambdas_host, int n_lambdas, trs_partition *out_dev, void *stream);

/* a1-a5 in one call, with the context's own statistics and table buffers. */
int trs_decide(trs_ctx *ctx, const void *luma_dev, int width, int height, size_t pitch_bytes, int bit_depth,
               const float *ctu_time_dev, int n_regions, float lambda, trs_partition *out_dev,
               void *stream);

/* a1-a5 from host memory: copies the plane and the times to the device,
 * decides, copies the partition back into *out_host and synchronises. */
int trs_decide_host(trs_ctx *ctx, const void *luma_host, int width, int height, size_t pitch_bytes,
                    int bit_depth, const float *ctu_time_host, int n_regions, float lambda,
                    trs_partition *out_host, void *stream);

/* trs_search for callers that cannot allocate memory (real-time loops that
 * cannot absorb the device synchronisation of cudaMalloc/cudaFree, hosts
 * whose own pool allocator owns all device memory).  The paper has no
 * counterpart: it is a deployment variant
 * of the search call above, with the same result.  No context: the search
 * plan and scratch live in one file-scope device array of 8 MiB that every
 * GPU loading the library keeps until exit.  A frame shape whose plan and
 * scratch exceed it returns TRS_ENOMEM (a 3840x2160 frame with n = 16 needs
 * about 2.5 MB).  No cudaMalloc, cudaFree or allocating library call is
 * made.  All calls on a device share the array, which keeps the last call's
 * contents; calls whose work overlaps on the GPU race on it, so serialise
 * them.  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress, with that device current).  A call whose shape
 * (width, height, n, k_area) differs from the previous one's (the first
 * call included) writes its plan over the old one with a cudaMemcpyAsync
 * from pageable host memory on `stream`, ordered only after earlier work on
 * that stream: the work of earlier calls on other streams must have
 * finished by then.  Arguments as for trs_search, plus k_area (the
 * area-rule factor, 3 in the paper). */
int trs_search_noalloc(const void *tables_dev, int width, int height, int n_regions, int k_area, float lambda,
                       trs_partition *out_dev, void *stream);

/* --- batched form -------------------------------------------------------- */

/* Decides nframes frames (1..opts.max_batch) of any sizes, depths, n and
 * lambda with one launch of each kernel over all of them (over each chunk
 * of them: see trs_set_batch_parts); out_dev holds nframes partitions.  The launch sequence is captured in a
 * CUDA graph the first time a batch of a given composition is seen and
 * replayed after. */
int trs_batch_decide(trs_ctx *ctx, const trs_frame_desc *frames_host, int nframes, trs_partition *out_dev,
                     void *stream);

/* Like trs_batch_decide, with every plane and time map in host memory
 * (pinned memory gives asynchronous copies): copies them into device
 * staging owned by the context, decides, copies the nframes partitions back
 * into out_host and synchronises.  The staging memory is allocated on the
 * first call that needs more than any call before. */
int trs_batch_decide_host(trs_ctx *ctx, const trs_frame_desc *frames_host, int nframes, trs_partition *out_host,
                          void *stream);

/* Launch shapes of the search kernels picked by trs_autotune, and the
 * timings that chose them. */
typedef struct trs_tune_report {
    int band_warps;      /* warps per block of the row-DP kernels */
    int col_warps;       /* warps per block of the column-DP kernels (each warp one window) */
    int col_batch;       /* 4: a column-DP warp runs one window for 32 / L frames that share a plan,
                            L = the smallest power of two >= max(4, n); 8: for one frame */
    int n_candidates;
    int cand_band_warps[6], cand_col_warps[6], cand_col_batch[6];
    float rows_ms[6];    /* both row-DP stages, fastest of three runs */
    float cols_ms[6];    /* both column-DP stages, fastest of three runs */
} trs_tune_report;

/* Times six launch-shape candidates of the search kernels on this batch
 * (direct launches, CUDA events around each kernel), keeps the fastest
 * row-DP and column-DP shapes in the context for every later call, and
 * drops captured batch graphs so they are captured again with them.
 * Synchronises on each timed run.  The decisions themselves do not depend
 * on the shapes. */
int trs_autotune(trs_ctx *ctx, const trs_frame_desc *frames_host, int nframes, trs_tune_report *out, void *stream);

/* Lightweight search (the paper leaves cheaper searches to future work,
 * Sec. 4): with step > 1 later searches of this context evaluate only
 * every step-th area window [a, 3a-1], counted from the largest a (kept
 * always, it holds the most balanced partitions).  Results are valid
 * partitions of S(n), optimal among those windows; T_min and Q may exceed
 * the exact ones.  step = 1 restores the exact search.  1 <= step <= 64. */
int trs_set_window_step(trs_ctx *ctx, int step);

/* Sets the search kernels' launch shapes directly: band_warps in {2, 4, 8},
 * col_warps in {1, 2, 4, 8}, col_batch in {4, 8}; TRS_EINVAL otherwise.
 * Drops captured batch graphs. */
int trs_set_tune(trs_ctx *ctx, int band_warps, int col_warps, int col_batch);

/* Frames covered by the stage times of trs_batch_stage_ms: the first chunk
 * of a captured batch (see trs_set_batch_parts), or the whole batch of a
 * call that runs as one launch chain.  0 before the first batched call. */
int trs_batch_stage_frames(const trs_ctx *ctx);

/* Kernels launched by the most recent batched call (9 per chunk; 0 before
 * the first call). */
int trs_batch_kernels(const trs_ctx *ctx);

/* parts in 1..4 (default 2): a captured batch of nframes frames runs as
 * min(parts, nframes / 4) chunks (at least one) of consecutive frames,
 * pipelined on two streams so that each chunk's texture map (bound by HBM
 * bandwidth) overlaps the previous chunk's search (bound by the ALUs).
 * Decisions are the same bytes for every value; each chunking is captured
 * as its own graph.  TRS_EINVAL outside 1..4. */
int trs_set_batch_parts(trs_ctx *ctx, int parts);

/* Device time in milliseconds of each stage of the most recent batched call
 * (texture, tables, step-1 rows, step-1 columns, step-2 rows, step-2
 * columns, rebuild of the smallest code, decode), read from CUDA events
 * recorded around each kernel (inside its graph when it was replayed).
 * Synchronises on that call.  Returns the number of stages written. */
int trs_batch_stage_ms(trs_ctx *ctx, float *ms, int max_stages);

/* --- serving: continuous batching over many streams -------------------- */

typedef struct trs_server trs_server;

typedef struct trs_server_opts {
    int max_width, max_height;  /* largest frame of any stream */
    int max_regions;            /* largest n of any stream */
    int max_streams;            /* streams open at once */
    int max_batch;              /* frames per device batch */
    int max_inflight;           /* device batches in flight at once, each on its own CUDA stream */
    size_t mem_budget_bytes;    /* device memory the server may hold (0: no limit) */
    int k_area;                 /* area-rule factor (3) */
    int device;
} trs_server_opts;

typedef struct trs_decision {
    uint64_t ticket;            /* as returned by trs_server_submit */
    uint64_t tag;               /* the caller's tag */
    int32_t stream_id;
    int32_t status;             /* TRS_OK or the decision's error */
    double latency_us;          /* from submit to the decision being ready on the host */
    trs_partition partition;
} trs_decision;

typedef struct trs_server_stats {
    uint64_t batches;           /* device batches launched */
    uint64_t frames;            /* frames put in batches */
    uint64_t decided;           /* decisions completed */
    size_t mem_used_bytes;      /* device memory held */
    int streams_open, pending, inflight;
    int status;                 /* TRS_OK unless the worker met an error */
} trs_server_stats;

/* Creates a server and its worker thread.  A stream is one video being
 * encoded; its frames are decided in order of arrival.  The server batches
 * the pending frames of all streams (first come, first served) onto up to
 * max_inflight concurrent device batches: frames that arrive while batches
 * run are launched as soon as a batch slot frees up, and their work overlaps
 * the running batches on the device.  TRS_EBUSY if the fixed memory exceeds
 * the budget. */
int trs_server_create(trs_server **out, const trs_server_opts *opts);
/* Finishes the work in flight, joins the worker and frees everything. */
int trs_server_destroy(trs_server *srv);
/* Admits a stream: allocates its resident time map and two request slots
 * (plane, statistics, tables, search scratch).  TRS_EBUSY when the stream
 * table is full or the memory budget would be exceeded. */
int trs_server_open_stream(trs_server *srv, int width, int height, int bit_depth, int n_regions, float lambda,
                           int *stream_id);
/* Waits (at most 10 s, else TRS_ETIMEOUT) for the stream's requests, then frees it. */
int trs_server_close_stream(trs_server *srv, int stream_id);
/* Replaces the stream's resident co-located CTU times (R*C floats, host
 * memory; Sec. 2.1's estimator input for the next frames).  Waits (at most
 * 10 s) until none of the stream's requests is in flight. */
int trs_server_update_times(trs_server *srv, int stream_id, const float *ctu_time_host);
/* Queues a frame (host memory, rows pitch_bytes apart, kept valid by the
 * caller until its decision is polled).  TRS_EBUSY when both of the
 * stream's request slots are taken; TRS_EINVAL before the first time map. */
int trs_server_submit(trs_server *srv, int stream_id, const void *luma_host, size_t pitch_bytes, uint64_t tag,
                      uint64_t *ticket);
/* Returns up to max_out finished decisions, waiting at most timeout_us for
 * the first; TRS_ETIMEOUT when none finished in time. */
int trs_server_poll(trs_server *srv, trs_decision *out, int max_out, int timeout_us, int *n_out);

/* Temporal layers (random-access GOPs).  Sec. 2.1 takes the estimator from
 * the co-TL frame: the previously encoded frame of the same temporal layer.
 * A stream opened with n_layers keeps one resident map per layer;
 * trs_server_update_times_layer stores the CTU times of a just-encoded
 * frame of `layer`, and trs_server_submit_layer decides a frame of `layer`
 * with that layer's map.  Before a layer's first map exists the most recent
 * map of any layer is used (the paper is silent on this case).  The calls
 * without _layer act on layer 0.  TRS_EINVAL for a layer outside
 * 0..n_layers-1; n_layers in 1..TRS_MAX_TEMPORAL_LAYERS. */
#define TRS_MAX_TEMPORAL_LAYERS 8
int trs_server_open_stream_layers(trs_server *srv, int width, int height, int bit_depth, int n_regions,
                                  float lambda, int n_layers, int *stream_id);
int trs_server_update_times_layer(trs_server *srv, int stream_id, int layer, const float *ctu_time_host);
int trs_server_submit_layer(trs_server *srv, int stream_id, int layer, const void *luma_host, size_t pitch_bytes,
                            uint64_t tag, uint64_t *ticket);
int trs_server_info(trs_server *srv, trs_server_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* TRS_H */
