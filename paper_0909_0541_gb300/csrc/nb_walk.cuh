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


// PROBE: walk without writing lists and turn the list statistics into the
// group's features for the learned opening angle (16 floats per group):
//   0 ln n_g;  1-3 ln(box side / L + 1e-7);  4 ln n_g - sum ln(side / L + 1e-4)
//   5 ln(|box centre - root centre| / L + 1e-6);  6 ln(list length + 1)
//   7 accepted cells / list length;  8-10 ln(min, mean, max distance from the
//   box centre to accepted cells' centres of mass / L + 1e-7);  11 depth / 22
// the opening test of one chunk of 32 frontier nodes (one per lane): emit
// particles and accepted cells to the list (ballot + popc), queue the
// children of opened cells (warp prefix sum); list_id, list_xm and list_q
// point at the group's own list slot
template <bool PROBE, bool QUAD>
__device__ __forceinline__ void visit_node(
    const NodeRec r, int32_t gb, int32_t gpid, const float4 &blo, const float4 &bhi,
    const float4 &bc, float invth, int32_t total, long long *cnt, unsigned *err, int lane,
    unsigned lt, int64_t room, int32_t *__restrict__ list_id,
    float4 *__restrict__ list_xm, const double *__restrict__ b_q, float4 *__restrict__ list_q,
    int32_t *qout_s, int32_t *qout, int64_t wq_cap,
    int32_t &len, int32_t &ncell,
    int32_t &nb, float &dmin, float &dmax, float &dsum)
{
    const unsigned FULL = 0xffffffffu;
    bool emit = false, cell_emit = false, open = false;
    int32_t fc = 0, nch = 0;
    if (r.valid) {
        fc = r.wb.z;
        if (r.b != gb) {
            if (fc < 0) {
                emit = true;
            } else {
                const bool holds = (r.wb.x <= gpid) && (gpid < r.wb.y);
                if (!holds && far_enough(r.a, r.wc.x, r.wc.y, blo, bhi, invth)) {
                    emit = true;
                    cell_emit = true;
                } else if (nb_in(fc > r.b && (int64_t)fc + r.wb.w <= total, cnt, err,
                                 SITE_WALK_CHILD, r.b)) {
                    open = true;
                    nch = r.wb.w;
                }
            }
        }
    }
    const unsigned em = __ballot_sync(FULL, emit);
    if (PROBE && cell_emit) {
        const float dx = r.a.x - bc.x, dy = r.a.y - bc.y, dz = r.a.z - bc.z;
        const float d = sqrtf(dx * dx + dy * dy + dz * dz);
        dmin = fminf(dmin, d);
        dmax = fmaxf(dmax, d);
        dsum += d;
    }
    // in the quadrupole mode a chunk's accepted cells come before its
    // particles, so that the force kernel's tiles hold runs of cells (which
    // take the quadrupole term) and runs of particles (which do not)
    const unsigned cm = QUAD ? __ballot_sync(FULL, cell_emit) : 0u;
    if (!PROBE && emit) {
        const int32_t pos = !QUAD ? len + __popc(em & lt)
                            : cell_emit ? len + __popc(cm & lt)
                                        : len + __popc(cm) + __popc(em & ~cm & lt);
        if (pos < room) {
            list_id[pos] = r.wb.x;
            list_xm[pos] = make_float4(nb_rel(r.a.x, r.d.x, bc.x), nb_rel(r.a.y, r.d.y, bc.y),
                                              nb_rel(r.a.z, r.d.z, bc.z), r.a.w);
            if constexpr (QUAD) {   // the cell's Q in FP32 (zero for a particle)
                float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (cell_emit) {
                    const double *qb = b_q + 6 * (int64_t)r.b;
#pragma unroll
                    for (int k = 0; k < 6; k++) q[k] = __double2float_rn(qb[k]);
                }
                list_q[2 * pos] = make_float4(q[0], q[1], q[2], q[3]);
                list_q[2 * pos + 1] = make_float4(q[4], q[5], 0.0f, 0.0f);
            }
        }
    }
    len += __popc(em);
    ncell += __popc(__ballot_sync(FULL, cell_emit));
    // exclusive prefix sum of the children over the lanes: with at most 15
    // children per lane (every cell but a level-21 bucket), from one ballot
    // per bit of the count; otherwise by a shuffle scan
    int32_t excl = 0;
    const int32_t tot = __reduce_add_sync(FULL, nch);
    if (__any_sync(FULL, nch > 15)) {
        int32_t incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        excl = incl - nch;
    } else {
#pragma unroll
        for (int b = 0; b < 4; b++)
            excl += __popc(__ballot_sync(FULL, (nch >> b) & 1) & lt) << b;
    }
    const int32_t start = nb + excl;
    if (open) {
        if (nch <= 8 && start + nch <= WQ_SMEM) {   // the common case: all in shared memory
#pragma unroll
            for (int k = 0; k < 8; k++)   // a cell below level 21 has at most 8 children
                if (k < nch) qout_s[start + k] = fc + k;
        } else {
            for (int32_t k = 0; k < nch; k++) {
                const int32_t pos = start + k;
                if (pos < WQ_SMEM) qout_s[pos] = fc + k;
                else if (pos < wq_cap) qout[pos] = fc + k;
            }
        }
    }
    nb += tot;
}


// One group's walk (the per-group step of k_walk): breadth-first from the
// group's system root over the level-ordered records, every frontier chunk of
// 32 nodes tested by visit_node; writes the group's list (or, PROBE, its
// features) and adds its statistics to the warp's running counts.
template <bool PROBE, bool QUAD>
__device__ __forceinline__ void walk_one(
    int g, const nb_wrec *__restrict__ wrec, const int32_t *__restrict__ pid2bfs,
    const int32_t *__restrict__ gnode, const int32_t *__restrict__ gcount,
    const float4 *__restrict__ gbox, long long *__restrict__ cnt, int32_t *__restrict__ glen,
    int32_t *__restrict__ gcells, int32_t *__restrict__ list_id, float4 *__restrict__ list_xm,
    const double *__restrict__ b_q, float4 *__restrict__ list_q, int64_t cap, int64_t alloc,
    int32_t *const qa, int32_t *const qb, int32_t *const qa_s, int32_t *const qb_s,
    int64_t wq_cap, unsigned *__restrict__ err, float *__restrict__ feat,
    const double *__restrict__ roots, const int8_t *__restrict__ n_depth,
    const int32_t *__restrict__ gfirst, const int32_t *__restrict__ sys_sorted,
    const int32_t *__restrict__ sys_root, int32_t total, int lane, unsigned lt, long long &pp,
    long long &pc, long long &tot, int32_t &mx, int32_t &qmax, unsigned &bad)
{
    const unsigned FULL = 0xffffffffu;
    const float4 blo = gbox[3 * (int64_t)g];
    const float4 bhi = gbox[3 * (int64_t)g + 1];
    const float4 bc = gbox[3 * (int64_t)g + 2];
    const float invth = bc.w;
    const int32_t gpid = gnode[g];
    const int32_t gb = nb_in(gpid >= 0 && gpid < total, cnt, err, SITE_WALK_NODE, gpid)
                           ? pid2bfs[gpid] : -1;
    const int64_t base = (int64_t)g * cap;
    const int64_t room = alloc - base < cap ? (alloc - base > 0 ? alloc - base : 0) : cap;
    // the group's list slot (no lists in the probe walk)
    int32_t *const lid = PROBE ? nullptr : list_id + base;
    float4 *const lxm = PROBE ? nullptr : list_xm + base;
    float4 *const lq = QUAD ? list_q + 2 * base : nullptr;
    int32_t len = 0, ncell = 0;
    float dmin = INFINITY, dmax = 0.0f, dsum = 0.0f;
    int32_t *qin = qa, *qout = qb, *qin_s = qa_s, *qout_s = qb_s;
    // the root of the group's system (node 0 for a single system)
    const int32_t gsys = sys_sorted ? sys_sorted[gfirst[g]] : 0;
    if (lane == 0) qin_s[0] = sys_root ? sys_root[gsys] : 0;
    __syncwarp();
    int32_t na = 1;
    int depth_guard = 0;
    while (na > 0) {
        int32_t nb = 0;
        // one chunk of 32 frontier nodes per iteration; each lane fetches all
        // of its node's records at once (one round trip after the queue)
        for (int32_t i0 = 0; i0 < na; i0 += NB_WARP) {
            const NodeRec r = load_node<PROBE>(i0 + lane, na, qin_s, qin, wrec,
                                               total, cnt, err);
            visit_node<PROBE, QUAD>(r, gb, gpid, blo, bhi, bc, invth, total, cnt, err, lane, lt, room,
                              lid, lxm, b_q, lq, qout_s, qout, wq_cap, len,
                              ncell, nb, dmin, dmax, dsum);
        }
        if (nb > qmax) qmax = nb;
        if (nb > wq_cap) { bad |= NB_EF_QUEUE; break; }
        __syncwarp();
        int32_t *t = qin; qin = qout; qout = t;
        t = qin_s; qin_s = qout_s; qout_s = t;
        na = nb;
        if (++depth_guard > NB_DEPTHS + 1) { bad |= NB_EF_WALK; break; }
    }
    if (PROBE) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dmin = fminf(dmin, __shfl_xor_sync(FULL, dmin, o));
            dmax = fmaxf(dmax, __shfl_xor_sync(FULL, dmax, o));
            dsum += __shfl_xor_sync(FULL, dsum, o);
        }
        if (lane < 16) {
            const double *root = roots + 8 * (int64_t)gsys;
            const float L = (float)root[3];
            const float ng = (float)gcount[g];
            const float sx = (bhi.x - blo.x) / L, sy = (bhi.y - blo.y) / L,
                        sz = (bhi.z - blo.z) / L;
            const float cx = bc.x - (float)root[0], cy = bc.y - (float)root[1],
                        cz = bc.z - (float)root[2];
            const bool any = ncell > 0;
            float v = 0.0f;
            switch (lane) {
            case 0: v = logf(ng); break;
            case 1: v = logf(sx + 1e-7f); break;
            case 2: v = logf(sy + 1e-7f); break;
            case 3: v = logf(sz + 1e-7f); break;
            case 4: v = logf(ng) - logf(sx + 1e-4f) - logf(sy + 1e-4f) - logf(sz + 1e-4f); break;
            case 5: v = logf(sqrtf(cx * cx + cy * cy + cz * cz) / L + 1e-6f); break;
            case 6: v = logf((float)len + 1.0f); break;
            case 7: v = len > 0 ? (float)ncell / (float)len : 0.0f; break;
            case 8: v = logf((any ? dmin : 0.0f) / L + 1e-7f); break;
            case 9: v = logf((any ? dsum / (float)ncell : 0.0f) / L + 1e-7f); break;
            case 10: v = logf((any ? dmax : 0.0f) / L + 1e-7f); break;
            case 11: v = (float)n_depth[gpid] / 22.0f; break;
            default: v = 0.0f;
            }
            feat[(int64_t)g * 16 + lane] = v;
        }
    }
    if (!PROBE && lane == 0) {
        glen[g] = len;
        gcells[g] = ncell;
        const long long m = gcount[g];
        pp += m * (long long)(len - ncell) + m * (m - 1);
        pc += m * (long long)ncell;
        tot += len;
        if (len > mx) mx = len;
        if (len > room) bad |= NB_EF_CAPACITY;
    }
}
