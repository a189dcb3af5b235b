// nb_walk.cuh -- pieces of the group tree walk shared by the list walk
// (nb_walk.cu) and the fused walk-and-force kernel (nb_fused.cu): the
// frontier queues' shared-memory part, the group opening test of Eq. (mac),
// and the fetch of one frontier node's level-order record.
#pragma once
#include "nb_internal.cuh"

// the first WQ_SMEM positions of each frontier queue live in shared memory
// (8 warps x 2 queues x 768 x 4 B = 48 KB per block); longer frontiers
// continue at the same positions in the warp's global queue
#define WQ_SMEM 768

// Eq. (mac) for a group: squared FP32 distance from the cell's centre of
// mass to the group box against (l / theta + s)^2, every operation rounded
// on its own in the order the oracle uses.
__device__ __forceinline__ bool far_enough(const float4 &a, float l, float s,
                                           const float4 &lo, const float4 &hi,
                                           float invth)
{
    const float ex = fmaxf(fmaxf(__fsub_rn(lo.x, a.x), __fsub_rn(a.x, hi.x)), 0.0f);
    const float ey = fmaxf(fmaxf(__fsub_rn(lo.y, a.y), __fsub_rn(a.y, hi.y)), 0.0f);
    const float ez = fmaxf(fmaxf(__fsub_rn(lo.z, a.z), __fsub_rn(a.z, hi.z)), 0.0f);
    float d2 = __fmul_rn(ex, ex);
    d2 = __fadd_rn(d2, __fmul_rn(ey, ey));
    d2 = __fadd_rn(d2, __fmul_rn(ez, ez));
    const float w = __fadd_rn(__fmul_rn(l, invth), s);
    return d2 > __fmul_rn(w, w);
}

// one frontier node's level-order records
struct NodeRec {
    int32_t b;
    bool valid;
    int4 wb;     // preorder id, preorder next, first child, children
    float4 a;    // centre of mass (hi), mass
    float2 wc;   // l, s
    float4 d;    // centre of mass (lo)
};

template <bool PROBE>
__device__ __forceinline__ NodeRec load_node(int32_t i, int32_t na, const int32_t *qin_s,
                                             const int32_t *qin,
                                             const nb_wrec *__restrict__ wrec, int32_t total,
                                             long long *cnt, unsigned *err)
{
    NodeRec r;
    r.b = 0;
    if (i < na) r.b = i < WQ_SMEM ? qin_s[i] : qin[i];
    r.valid = i < na && nb_in(r.b >= 0 && r.b < total, cnt, err, SITE_WALK_NODE, r.b);
    if (r.valid) {
        const nb_wrec *w = wrec + r.b;     // one 64-byte line
        r.wb = w->b;
        r.a = w->a;
        r.wc = w->c;
        if (!PROBE) r.d = w->d;
    }
    return r;
}

