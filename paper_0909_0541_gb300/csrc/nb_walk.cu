// nb_walk.cu -- the group tree walk: the iterative walk of Fig.
// "treewalk_iterative" in group form, done breadth-first by one warp.
//
// Nodes are stored in level order, so the children of a cell are one
// contiguous run one level down.  The warp keeps the current level's
// frontier (node indices) in a queue in global memory and takes it 32 nodes
// at a time: each lane loads one node's record (coalesced, L2-resident) and
// applies the opening test.  Particles and accepted cells are appended to
// the group's list (ballot + popc compaction); opened cells append their
// children to the next level's queue (warp prefix sum over the child
// counts).  Every lane of every step holds a node the walk visits, and the
// loop ends after at most one pass per tree level.
//
// The group's own node is skipped: its particles are exactly the group's
// members, which the force kernel sums directly (with j != i by index).  A
// cell that contains the group (preorder id <= group id < preorder next) is
// always opened.  The list therefore holds, in breadth-first order, the
// same entries as the depth-first list of the paper's walk minus the group's
// own particles.
//
// List records: preorder node id (int32) and the FP32 source the force
// kernel reads: position relative to the group's box centre from the
// two-float split of the FP64 centre of mass, fl32(fl32(hi - c) + lo), and
// the FP32 mass.
#include "nb_walk.cuh"

#define WALK_T 256
#define WALK_WARPS (WALK_T / NB_WARP)

// PROBE: walk without writing lists and turn the list statistics into the
// group's features for the learned opening angle (16 floats per group):
//   0 ln n_g;  1-3 ln(box side / L + 1e-7);  4 ln n_g - sum ln(side / L + 1e-4)
//   5 ln(|box centre - root centre| / L + 1e-6);  6 ln(list length + 1)
//   7 accepted cells / list length;  8-10 ln(min, mean, max distance from the
//   box centre to accepted cells' centres of mass / L + 1e-7);  11 depth / 22
// the opening test of one chunk of 32 frontier nodes (one per lane): emit
// particles and accepted cells to the list (ballot + popc), queue the
// children of opened cells (warp prefix sum)
template <bool PROBE, bool QUAD>
__device__ __forceinline__ void visit_node(
    const NodeRec r, int32_t gb, int32_t gpid, const float4 &blo, const float4 &bhi,
    const float4 &bc, float invth, int32_t total, long long *cnt, unsigned *err, int lane,
    unsigned lt, int64_t room, int64_t base, int32_t *__restrict__ list_id,
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
            list_id[base + pos] = r.wb.x;
            list_xm[base + pos] = make_float4(nb_rel(r.a.x, r.d.x, bc.x), nb_rel(r.a.y, r.d.y, bc.y),
                                              nb_rel(r.a.z, r.d.z, bc.z), r.a.w);
            if constexpr (QUAD) {   // the cell's Q in FP32 (zero for a particle)
                float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (cell_emit) {
                    const double *qb = b_q + 6 * (int64_t)r.b;
#pragma unroll
                    for (int k = 0; k < 6; k++) q[k] = __double2float_rn(qb[k]);
                }
                list_q[2 * (base + pos)] = make_float4(q[0], q[1], q[2], q[3]);
                list_q[2 * (base + pos) + 1] = make_float4(q[4], q[5], 0.0f, 0.0f);
            }
        }
    }
    len += __popc(em);
    ncell += __popc(__ballot_sync(FULL, cell_emit));
    int32_t incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int32_t start = nb + incl - nch;
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
    nb += __shfl_sync(FULL, incl, 31);
}

template <bool PROBE, bool QUAD = false>
__global__ void __launch_bounds__(WALK_T, 4)
k_walk(const nb_wrec *__restrict__ wrec,
       const int32_t *__restrict__ pid2bfs, const int32_t *__restrict__ gnode,
       const int32_t *__restrict__ gcount, const float4 *__restrict__ gbox,
       long long *__restrict__ cnt, int32_t *__restrict__ glen, int32_t *__restrict__ gcells,
       int32_t *__restrict__ list_id, float4 *__restrict__ list_xm,
       const double *__restrict__ b_q, float4 *__restrict__ list_q, int64_t cap, int64_t alloc,
       int32_t *__restrict__ wq, int64_t wq_cap, unsigned *__restrict__ err,
       float *__restrict__ feat, const double *__restrict__ roots, const int8_t *__restrict__ n_depth,
       const int32_t *__restrict__ gfirst, const int32_t *__restrict__ sys_sorted,
       const int32_t *__restrict__ sys_root)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t gw = (int64_t)blockIdx.x * WALK_WARPS + (threadIdx.x >> 5);
    int32_t *const qa = wq + gw * 2 * wq_cap;
    int32_t *const qb = qa + wq_cap;
    __shared__ int32_t sq[WALK_WARPS][2 * WQ_SMEM];
    int32_t *const qa_s = sq[threadIdx.x >> 5];
    int32_t *const qb_s = qa_s + WQ_SMEM;
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    const int32_t total = (int32_t)cnt[CNT_NODES];
    long long pp = 0, pc = 0, tot = 0;
    int32_t mx = 0, qmax = 0;
    unsigned bad = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)nb_atomic_add(&cnt[CNT_WALK_Q], 1LL);
        g = __shfl_sync(FULL, g, 0);
        if (g >= G) break;
        const float4 blo = gbox[3 * (int64_t)g];
        const float4 bhi = gbox[3 * (int64_t)g + 1];
        const float4 bc = gbox[3 * (int64_t)g + 2];
        const float invth = bc.w;
        const int32_t gpid = gnode[g];
        const int32_t gb = nb_in(gpid >= 0 && gpid < total, cnt, err, SITE_WALK_NODE, gpid)
                               ? pid2bfs[gpid] : -1;
        const int64_t base = (int64_t)g * cap;
        const int64_t room = alloc - base < cap ? (alloc - base > 0 ? alloc - base : 0) : cap;
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
                                  base, list_id, list_xm, b_q, list_q, qout_s, qout, wq_cap, len,
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
    if (lane == 0) {
        nb_atomic_add(&cnt[CNT_PP], pp);
        nb_atomic_add(&cnt[CNT_PC], pc);
        nb_atomic_add(&cnt[CNT_PP_CUM], pp);
        nb_atomic_add(&cnt[CNT_PC_CUM], pc);
        nb_atomic_add(&cnt[CNT_LIST_TOT], tot);
        atomicMax(&cnt[CNT_LIST_MAX], (long long)mx);
        atomicMax(&cnt[CNT_QMAX], (long long)qmax);
        if (bad) atomicOr(err, bad);
    }
}

// Tree-only features of every group: the probe's features that need no
// walk (0-5 and 11, the same formulas), the walk-based ones (6-10) zero.
// One thread per group.
__global__ void __launch_bounds__(256)
k_group_features_tree(const int32_t *__restrict__ gnode, const int32_t *__restrict__ gfirst,
                      const int32_t *__restrict__ gcount, const float4 *__restrict__ gbox,
                      const double *__restrict__ roots, const int8_t *__restrict__ n_depth,
                      const int32_t *__restrict__ sys_sorted, long long *__restrict__ cnt,
                      float *__restrict__ feat, int64_t n, unsigned *__restrict__ err)
{
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        float *fo = feat + (int64_t)g * 16;
        const int32_t f = gfirst[g], gpid = gnode[g];
        if (!nb_in(f >= 0 && f < n && gpid >= 0 && gpid < total, cnt, err, SITE_GROUPS, g)) {
            for (int k = 0; k < 16; k++) fo[k] = 0.0f;
            continue;
        }
        const int32_t gsys = sys_sorted ? sys_sorted[f] : 0;
        const double *root = roots + 8 * (int64_t)gsys;
        const float L = (float)root[3];
        const float ng = (float)gcount[g];
        const float4 blo = gbox[3 * (int64_t)g], bhi = gbox[3 * (int64_t)g + 1],
                     bc = gbox[3 * (int64_t)g + 2];
        const float sx = (bhi.x - blo.x) / L, sy = (bhi.y - blo.y) / L, sz = (bhi.z - blo.z) / L;
        const float cx = bc.x - (float)root[0], cy = bc.y - (float)root[1],
                    cz = bc.z - (float)root[2];
        fo[0] = logf(ng);
        fo[1] = logf(sx + 1e-7f);
        fo[2] = logf(sy + 1e-7f);
        fo[3] = logf(sz + 1e-7f);
        fo[4] = logf(ng) - logf(sx + 1e-4f) - logf(sy + 1e-4f) - logf(sz + 1e-4f);
        fo[5] = logf(sqrtf(cx * cx + cy * cy + cz * cz) / L + 1e-6f);
        for (int k = 6; k < 11; k++) fo[k] = 0.0f;
        fo[11] = (float)n_depth[gpid] / 22.0f;
        for (int k = 12; k < 16; k++) fo[k] = 0.0f;
    }
}

void nb_launch_features_tree(nb_ctx *c, float *feat)
{
    k_group_features_tree<<<nb_grid(c->max_n, 256, c->num_sms * 8), 256, 0, c->stream>>>(
        c->gnode, c->gfirst, c->gcount, c->gbox, c->root, c->n_depth,
        c->nsys > 1 ? c->sys_sorted : nullptr, c->cnt, feat, c->n, c->err);
    nb_launched(c, "k_group_features_tree");
}

// warps of one walk launch (the frontier queues are sized for them)
int nb_walk_warps(nb_ctx *c)
{
    int blocks = 0, bp = 0;
    // the queue heads are 48 KB of shared memory per block: ask for the
    // largest shared-memory carveout so four blocks fit on an SM
    cudaFuncSetAttribute(k_walk<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(k_walk<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(k_walk<false, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_walk<false>, WALK_T, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bp, k_walk<true>, WALK_T, 0);
    if (bp < blocks) blocks = bp;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bp, k_walk<false, true>, WALK_T, 0);
    if (bp < blocks) blocks = bp;
    if (blocks < 1) blocks = 1;
    return c->num_sms * blocks * WALK_WARPS;
}

void nb_launch_walk(nb_ctx *c)
{
    cudaMemsetAsync(&c->cnt[CNT_LIST_TOT], 0, sizeof(long long) * 5, c->stream);
    static_assert(CNT_LIST_TOT + 4 == CNT_WALK_Q, "counter layout");
    cudaMemsetAsync(&c->cnt[CNT_QMAX], 0, sizeof(long long), c->stream);
    const int blocks = c->walk_warps / WALK_WARPS;
    if (c->quad && c->b_q && c->list_q)
        k_walk<false, true><<<blocks, WALK_T, 0, c->stream>>>(
            c->wrec, c->pid2bfs, c->gnode, c->gcount, c->gbox, c->cnt, c->glen, c->gcells,
            c->list_id, c->list_xm, c->b_q, c->list_q, c->list_cap, c->list_alloc, c->wq,
            c->wq_cap, c->err, nullptr, c->root, c->n_depth, c->gfirst,
            c->nsys > 1 ? c->sys_sorted : nullptr, c->nsys > 1 ? c->sys_root : nullptr);
    else
        k_walk<false><<<blocks, WALK_T, 0, c->stream>>>(
            c->wrec, c->pid2bfs, c->gnode, c->gcount, c->gbox, c->cnt, c->glen, c->gcells,
            c->list_id, c->list_xm, nullptr, nullptr, c->list_cap, c->list_alloc, c->wq,
            c->wq_cap, c->err, nullptr, c->root, c->n_depth, c->gfirst,
            c->nsys > 1 ? c->sys_sorted : nullptr, c->nsys > 1 ? c->sys_root : nullptr);
    nb_launched(c, "k_walk");
}

// the probe walk: features of every group (the groups must be formed with
// the probe's opening angle)
void nb_launch_probe(nb_ctx *c, float *feat)
{
    cudaMemsetAsync(&c->cnt[CNT_WALK_Q], 0, sizeof(long long), c->stream);
    const int blocks = c->walk_warps / WALK_WARPS;
    k_walk<true><<<blocks, WALK_T, 0, c->stream>>>(
        c->wrec, c->pid2bfs, c->gnode, c->gcount, c->gbox, c->cnt,
        c->glen, c->gcells, nullptr, nullptr, nullptr, nullptr, 0, 0, c->wq, c->wq_cap, c->err,
        feat, c->root,
        c->n_depth, c->gfirst, c->nsys > 1 ? c->sys_sorted : nullptr,
        c->nsys > 1 ? c->sys_root : nullptr);
    nb_launched(c, "k_walk");
}
