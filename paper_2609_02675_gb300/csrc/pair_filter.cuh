// The pair filter shared by the broad phases (grid hash in k_collision.cu, LBVH in
// k_lbvh.cu): partner j of body i is accepted when it shares i's group, the two are not both
// pinned, their inflated boxes overlap and no user bond joins them (reading R21).
#pragma once
#include "pabd_internal.h"

namespace pabd {

__device__ __forceinline__ bool overlap(const float4& la, const float4& ha, const float4& lb, const float4& hb) {
    return la.x <= hb.x && lb.x <= ha.x && la.y <= hb.y && lb.y <= ha.y && la.z <= hb.z && lb.z <= ha.z;
}

// pairs joined by a user bond never collide: binary search in the body's sorted list of
// bonded partners (a CSR built once on the host)
__device__ __forceinline__ bool adj_has(const Dev& d, int a, int b) {
    if (!d.adj_off) return false;
    int lo = d.adj_off[a], hi = d.adj_off[a + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = d.adj_nbr[mid];
        if (v == b) return true;
        if (v < b) lo = mid + 1; else hi = mid;
    }
    return false;
}

// (j's group, flags and box are loaded together, one round trip rather than three)
__device__ __forceinline__ bool pair_ok(const Dev& d, int i, int j, int gi, int fi, const float4& li,
                                        const float4& hi) {
    const int gj = d.group[j], fj = d.bflags[j];
    const float4 lj = d.lo[j], hj = d.hi[j];
    if (gj != gi) return false;
    if ((fi & BF_PINNED) && (fj & BF_PINNED)) return false;
    if (!overlap(li, hi, lj, hj)) return false;
    if (adj_has(d, i, j)) return false;
    return true;
}

__device__ __forceinline__ bool pair_ok(const Dev& d, int i, int j, int gi, int fi) {
    return pair_ok(d, i, j, gi, fi, d.lo[i], d.hi[i]);
}

}  // namespace pabd
