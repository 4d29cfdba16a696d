// Host-side search plans (see plan.cpp).
#pragma once

#include <cstdint>
#include <vector>

#include "trs_internal.cuh"

namespace trs {

struct HostPlan {
    int W = 0, H = 0, C = 0, R = 0, n = 0, k = 0, nb = 0;
    uint64_t A = 0;
    std::vector<uint64_t> win_a;
    std::vector<PlanItem> items;
    std::vector<int32_t> slot_of;
    std::vector<int16_t> band_x0, band_x1;
    std::vector<int32_t> band_items;  // [nb+1] prefix of items per band
    int max_nd = 0;  // most full-CTU slice heights an item admits (sizes the row DP's staging)
    std::vector<uint64_t> slot_k;  // [nwin * nb]: the column DP's step entries (see DevPlan::slot_k)
    int max_edge_vals = 0;         // see DevPlan::max_edge_vals
};

// Fills slot_k and max_edge_vals from slot_of and the items' slice-count ranges.
void column_program(HostPlan *p);

struct SearchScratch {
    size_t V1, V2, w1, w2, H2, codes, bytes;
};

// window_step > 1 keeps every window_step-th area window only, counted from
// the largest (the lightweight search); 1 is the exact search.
int build_plan(int W, int H, int n, int k, HostPlan *p, int window_step = 1);
// Soundness of a plan: for each of its windows, whether it represents every
// one-tile-row partition whose slice areas all fit the window (see
// trs_plan_coverage).
int plan_coverage(int W, int H, int n, int k, int window_step, int *windows, int *short_windows,
                  double *in_windows);
// Exact number of partitions in S(n) with one tile row (see trs_count_partitions).
int count_partitions(int W, int H, int n, int k, long double *out);
size_t plan_blob_bytes(const HostPlan &p);
// Lays the plan out as a device blob whose pointers assume it will be copied to dev_base.
void plan_serialize(const HostPlan &p, uint8_t *dev_base, std::vector<uint8_t> &blob);
SearchScratch scratch_layout(const HostPlan &p);

}  // namespace trs
