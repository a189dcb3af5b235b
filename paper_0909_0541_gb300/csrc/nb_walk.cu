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
        walk_one<PROBE, QUAD>(g, wrec, pid2bfs, gnode, gcount, gbox, cnt, glen, gcells, list_id,
                              list_xm, b_q, list_q, cap, alloc, qa, qb, qa_s, qb_s, wq_cap, err,
                              feat, roots, n_depth, gfirst, sys_sorted, sys_root, total, lane, lt,
                              pp, pc, tot, mx, qmax, bad);
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
