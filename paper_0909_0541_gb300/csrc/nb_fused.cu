// nb_fused.cu -- the walk and the force sum in one kernel, without lists in
// device memory: the paper's own GPU design (Fig. "treegpu", Sec. "Our GPU
// implementation", where each thread walks the tree and sums Eq. (gravity)
// as it goes) in group form.
//
// One warp takes one force work item (a group and up to 64 of its members,
// the same items as the list path) and walks the group breadth-first exactly
// as k_walk does.  Instead of writing the accepted sources to the group's
// list, the warp appends each one's FP32 record (position relative to the
// group centre, mass) to a buffer of FW_BUF records in shared memory; every
// time a tile's worth is buffered (32 records, or 64 for an item of several
// source streams), it is summed against the item's targets with the same
// tile pass as the list force kernel.  The remainder is padded like the
// list's last tile, then the group's own members are summed.  The records
// reach the tile pass in list order and in the same tiles, so the
// accelerations equal the list path's bit for bit.
//
// An item of a group with several items walks the group again: the walk is
// repeated per item, and the interaction lists never touch HBM.
#include "nb_force.cuh"
#include "nb_walk.cuh"

#define FW_T 128
#define FW_WARPS (FW_T / NB_WARP)
// buffered records per warp: a tile of item_tile(S, 32) records is summed
// whenever one is ready, and a chunk of the walk adds at most 32
#define FW_BUF (F_TILE_STREAMS + NB_WARP)
// unroll of the tile pass inside the walk loop: the walk's live state leaves
// fewer registers than the list force kernel has
static constexpr int FW_UNROLL = 4;

struct FusedCounts {
    long long pp, pc, tot;
    int32_t mx, qmax;
};

template <int MODE, bool GUARD, int R, int S>
__device__ __forceinline__ void fused_item(
    int32_t g, int32_t i0, float4 *buf, int32_t *qa_s, int32_t *qb_s, int32_t *qa, int32_t *qb,
    int64_t wq_cap, const nb_wrec *__restrict__ wrec, const int32_t *__restrict__ pid2bfs,
    const int32_t *__restrict__ gnode, const int32_t *__restrict__ gfirst,
    const int32_t *__restrict__ gcount, const float4 *__restrict__ gbox,
    const float4 *__restrict__ p_hi, const float4 *__restrict__ p_lo,
    const int32_t *__restrict__ perm, int32_t total, int64_t n, float eps2,
    const int32_t *__restrict__ sys_sorted, const int32_t *__restrict__ sys_root,
    float *__restrict__ acc, float *__restrict__ pot, long long *__restrict__ cnt,
    unsigned *__restrict__ err, unsigned &bad, FusedCounts &fc)
{
    const unsigned FULL = 0xffffffffu;
    constexpr int W = NB_WARP / S;
    constexpr int FT = item_tile(S, NB_WARP);   // records per summed tile, as the list path
    constexpr int FK = FT / NB_WARP;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int row = lane % W, stream = lane / W;
    const int32_t f = gfirst[g], ng = gcount[g];
    if (!(f >= 0 && ng >= 1 && (int64_t)f + ng <= n && i0 >= 0 && i0 < ng)) {
        if (lane == 0) nb_bad(cnt, err, SITE_FORCE, g);
        return;
    }
    const float4 blo = gbox[3 * (int64_t)g];
    const float4 bhi = gbox[3 * (int64_t)g + 1];
    const float4 bc = gbox[3 * (int64_t)g + 2];
    const float invth = bc.w;
    const float4 pad = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    Tgt t[R];
    int32_t kk[R], slot[R];
    bool ok[R];
    Acc<MODE> A[R];
    Sum2 P[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int32_t k = i0 + r * W + row;
        ok[r] = k < ng;
        kk[r] = k;
        slot[r] = f + (ok[r] ? k : ng - 1);
        const float4 h = p_hi[slot[r]], lo = p_lo[slot[r]];
        t[r].set(nb_rel(h.x, lo.x, bc.x), nb_rel(h.y, lo.y, bc.y), nb_rel(h.z, lo.z, bc.z));
        A[r].init();
        P[r].init();
    }
    // (1) walk, summing every 32 buffered sources
    const int32_t gpid = gnode[g];
    const int32_t gb = nb_in(gpid >= 0 && gpid < total, cnt, err, SITE_WALK_NODE, gpid)
                           ? pid2bfs[gpid] : -1;
    const int32_t gsys = sys_sorted ? sys_sorted[f] : 0;
    int32_t *qin = qa, *qout = qb, *qin_s = qa_s, *qout_s = qb_s;
    if (lane == 0) qin_s[0] = sys_root ? sys_root[gsys] : 0;
    __syncwarp();
    int32_t na = 1, nbuf = 0, len = 0, ncell = 0;
    int depth_guard = 0;
    while (na > 0) {
        int32_t nb = 0;
        for (int32_t c0 = 0; c0 < na; c0 += NB_WARP) {
            const NodeRec r = load_node<false>(c0 + lane, na, qin_s, qin, wrec, total, cnt, err);
            bool emit = false, cell_emit = false, open = false;
            int32_t fch = 0, nch = 0;
            if (r.valid && r.b != gb) {
                fch = r.wb.z;
                if (fch < 0) {
                    emit = true;
                } else {
                    const bool holds = (r.wb.x <= gpid) && (gpid < r.wb.y);
                    if (!holds && far_enough(r.a, r.wc.x, r.wc.y, blo, bhi, invth)) {
                        emit = true;
                        cell_emit = true;
                    } else if (nb_in(fch > r.b && (int64_t)fch + r.wb.w <= total, cnt, err,
                                     SITE_WALK_CHILD, r.b)) {
                        open = true;
                        nch = r.wb.w;
                    }
                }
            }
            const unsigned em = __ballot_sync(FULL, emit);
            if (emit)
                put_rec(buf, nbuf + __popc(em & lt),
                        make_float4(nb_rel(r.a.x, r.d.x, bc.x), nb_rel(r.a.y, r.d.y, bc.y),
                                    nb_rel(r.a.z, r.d.z, bc.z), r.a.w));
            nbuf += __popc(em);
            len += __popc(em);
            ncell += __popc(__ballot_sync(FULL, cell_emit));
            int32_t incl = nch;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const int32_t start = nb + incl - nch;
            if (open)
                for (int32_t k = 0; k < nch; k++) {
                    const int32_t pos = start + k;
                    if (pos < WQ_SMEM) qout_s[pos] = fch + k;
                    else if (pos < wq_cap) qout[pos] = fch + k;
                }
            nb += __shfl_sync(FULL, incl, 31);
            __syncwarp();
            if (nbuf >= FT) {   // one full tile: sum it, keep the rest
                tile_pass<MODE, GUARD, false, R, W * FK, FW_UNROLL>(buf, stream * W * FK, 0, t, kk,
                                                                    eps2, A, P);
                __syncwarp();
                // move the rest (< 32 records) down by whole record pairs (FT is even)
                if (lane < ((nbuf - FT + 1) & ~1)) buf[lane] = buf[FT + lane];
                nbuf -= FT;
                __syncwarp();
            }
        }
        if (lane == 0 && nb > fc.qmax) fc.qmax = nb;
        if (nb > wq_cap) {
            bad |= NB_EF_QUEUE;
            break;
        }
        __syncwarp();
        int32_t *t = qin; qin = qout; qout = t;
        t = qin_s; qin_s = qout_s; qout_s = t;
        na = nb;
        if (++depth_guard > NB_DEPTHS + 1) {
            bad |= NB_EF_WALK;
            break;
        }
    }
    if (nbuf > 0) {   // the last, padded tile of the list
#pragma unroll
        for (int k = 0; k < FK; k++)
            if (k * NB_WARP + lane >= nbuf) put_rec(buf, k * NB_WARP + lane, pad);
        __syncwarp();
        tile_pass<MODE, GUARD, false, R, W * FK, FW_UNROLL>(buf, stream * W * FK, 0, t, kk, eps2,
                                                            A, P);
        __syncwarp();
    }
    // (2) the group's own members, j != i
    for (int32_t j0 = 0; j0 < ng; j0 += NB_WARP) {
        const int32_t jj = j0 + lane;
        float4 v = pad;
        if (jj < ng) {
            const float4 h = p_hi[f + jj], lo = p_lo[f + jj];
            v = make_float4(nb_rel(h.x, lo.x, bc.x), nb_rel(h.y, lo.y, bc.y),
                            nb_rel(h.z, lo.z, bc.z), h.w);
        }
        put_rec(buf, lane, v);
        __syncwarp();
        tile_pass<MODE, GUARD, true, R, W>(buf, stream * W, j0 + stream * W, t, kk, eps2, A, P);
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < R; r++) pair_fold<MODE>(A[r], P[r]);
    if (lane == 0) {   // interaction counts of this item's targets
        const int32_t mi = ng - i0 < R * W ? ng - i0 : R * W;
        fc.pp += (long long)mi * (len - ncell) + (long long)mi * (ng - 1);
        fc.pc += (long long)mi * ncell;
        if (i0 == 0) {
            fc.tot += len;
            if (len > fc.mx) fc.mx = len;
        }
    }
    if constexpr (S > 1) {
#pragma unroll
        for (int o = W; o < NB_WARP; o <<= 1)
#pragma unroll
            for (int r = 0; r < R; r++) stream_sum<MODE>(A[r], o);
        if (stream != 0) return;
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (!ok[r]) continue;
        const int64_t o = perm[slot[r]];
        float ax, ay, az, ph;
        if (MODE == MODE_F64) {
            ax = (float)A[r].dx; ay = (float)A[r].dy; az = (float)A[r].dz; ph = (float)A[r].dp;
        } else if (MODE == MODE_COMP) {
            ax = A[r].x - A[r].cx; ay = A[r].y - A[r].cy;
            az = A[r].z - A[r].cz; ph = A[r].p - A[r].cp;
        } else {
            ax = A[r].x; ay = A[r].y; az = A[r].z; ph = A[r].p;
        }
        acc[3 * o] = ax;
        acc[3 * o + 1] = ay;
        acc[3 * o + 2] = az;
        if (pot) pot[o] = ph;
    }
}

template <int MODE, bool GUARD>
__global__ void __launch_bounds__(FW_T)
k_walk_force(const int32_t *__restrict__ items, const nb_wrec *__restrict__ wrec,
             const int32_t *__restrict__ pid2bfs, const int32_t *__restrict__ gnode,
             const int32_t *__restrict__ gfirst, const int32_t *__restrict__ gcount,
             const float4 *__restrict__ gbox, const float4 *__restrict__ p_hi,
             const float4 *__restrict__ p_lo, const int32_t *__restrict__ perm,
             long long *__restrict__ cnt, int32_t *__restrict__ wq, int64_t wq_cap,
             unsigned *__restrict__ err, float eps2, float *__restrict__ acc,
             float *__restrict__ pot, int64_t n, int64_t max_items,
             const int32_t *__restrict__ sys_sorted, const int32_t *__restrict__ sys_root)
{
    __shared__ float4 bufs[FW_WARPS][FW_BUF];
    __shared__ int32_t sq[FW_WARPS][2 * WQ_SMEM];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * FW_WARPS + w;
    int32_t *const qa = wq + gw * 2 * wq_cap;
    int32_t *const qb = qa + wq_cap;
    int32_t nitems = (int32_t)cnt[CNT_ITEMS];
    if (nitems > max_items) {
        if (threadIdx.x == 0 && blockIdx.x == 0) nb_bad(cnt, err, SITE_FORCE, nitems);
        nitems = (int32_t)max_items;
    }
    const int32_t ngroups = (int32_t)cnt[CNT_GROUPS];
    const int32_t total = (int32_t)cnt[CNT_NODES];
    unsigned bad = 0;
    FusedCounts fc = {0, 0, 0, 0, 0};
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)nb_atomic_add(&cnt[CNT_FORCE_Q], 1LL);
        it = __shfl_sync(FULL, it, 0);
        if (it >= nitems) break;
        const int32_t g = items[2 * (int64_t)it], word = items[2 * (int64_t)it + 1];
        const int32_t i0 = word & ITEM_MEMBER_MASK;
        if (g < 0 || g >= ngroups) {
            if (lane == 0) nb_bad(cnt, err, SITE_FORCE, g);
            continue;
        }
#define NB_FUSED_ITEM(R, S)                                                                    \
    fused_item<MODE, GUARD, R, S>(g, i0, bufs[w], sq[w], sq[w] + WQ_SMEM, qa, qb, wq_cap, wrec, \
                                  pid2bfs, gnode, gfirst, gcount, gbox, p_hi, p_lo, perm, total,  \
                                  n, eps2, sys_sorted, sys_root, acc, pot, cnt, err, bad, fc)
        NB_ITEM_SHAPES(word, NB_FUSED_ITEM);
#undef NB_FUSED_ITEM
        if (bad) break;
    }
    if (lane == 0) {
        nb_atomic_add(&cnt[CNT_PP], fc.pp);
        nb_atomic_add(&cnt[CNT_PC], fc.pc);
        nb_atomic_add(&cnt[CNT_PP_CUM], fc.pp);
        nb_atomic_add(&cnt[CNT_PC_CUM], fc.pc);
        nb_atomic_add(&cnt[CNT_LIST_TOT], fc.tot);
        atomicMax(&cnt[CNT_LIST_MAX], (long long)fc.mx);
        atomicMax(&cnt[CNT_QMAX], (long long)fc.qmax);
        if (bad) atomicOr(err, bad);
    }
}

template <int MODE, bool GUARD>
static void launch_fused(nb_ctx *c, float eps2, float *acc, float *pot)
{
    static int blocks = 0;
    if (blocks == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_walk_force<MODE, GUARD>, FW_T, 0);
        if (blocks < 1) blocks = 1;
    }
    // one pair of frontier queues per warp: no more warps than the queues hold
    int grid = c->num_sms * blocks;
    if ((int64_t)grid * FW_WARPS > c->walk_warps) grid = c->walk_warps / FW_WARPS;
    if (grid < 1) grid = 1;
    k_walk_force<MODE, GUARD><<<grid, FW_T, 0, c->stream>>>(
        c->items, c->wrec, c->pid2bfs, c->gnode, c->gfirst, c->gcount, c->gbox, c->p_hi, c->p_lo,
        c->perm, c->cnt, c->wq, c->wq_cap, c->err, eps2, acc, pot, c->n, c->max_items,
        c->nsys > 1 ? c->sys_sorted : nullptr, c->nsys > 1 ? c->sys_root : nullptr);
    nb_launched(c, "k_walk_force");
}

void nb_launch_fused(nb_ctx *c, float eps, float *acc, float *pot, int precision)
{
    cudaMemsetAsync(&c->cnt[CNT_LIST_TOT], 0, sizeof(long long) * 4, c->stream);
    static_assert(CNT_LIST_TOT + 3 == CNT_PC, "counter layout");
    cudaMemsetAsync(&c->cnt[CNT_FORCE_Q], 0, sizeof(long long), c->stream);
    cudaMemsetAsync(&c->cnt[CNT_QMAX], 0, sizeof(long long), c->stream);
    const float eps2 = eps * eps;
    const bool guard = !(eps2 >= FLT_MIN);
    switch (precision * 2 + (guard ? 1 : 0)) {
    case 0: launch_fused<MODE_FP32, false>(c, eps2, acc, pot); break;
    case 1: launch_fused<MODE_FP32, true>(c, eps2, acc, pot); break;
    case 2: launch_fused<MODE_COMP, false>(c, eps2, acc, pot); break;
    case 3: launch_fused<MODE_COMP, true>(c, eps2, acc, pot); break;
    case 4: launch_fused<MODE_F64, false>(c, eps2, acc, pot); break;
    default: launch_fused<MODE_F64, true>(c, eps2, acc, pot); break;
    }
}
