// nb_walk.cu -- the group tree walk (Fig. "treewalk_iterative" in group form).
//
// One warp walks one group.  Nodes are stored in depth-first preorder, so the
// iterative walk only ever moves forward: to id + 1 when a cell is opened
// ("more"), to next(id) when a particle or an accepted cell is taken.  The
// warp evaluates the 32 consecutive nodes cur .. cur+31 at once (coalesced
// 32-byte records, opening tests in parallel), then follows the chain of
// successors from cur inside that window with register shuffles to find
// which of the 32 were actually visited, appends the visited particles and
// accepted cells to the group's list in walk order, and continues at the
// first successor beyond the window.  Each window advances cur by >= 1, so
// the loop ends after at most (number of nodes) windows; a successor that
// does not advance raises NB_EF_WALK instead of looping.
//
// List records: node id (int32) and the FP32 source the force kernel reads:
// position relative to the group's box centre, computed from the two-float
// split of the FP64 centre of mass as (hi - c) + lo, and the mass.
#include "nb_internal.cuh"

#define WALK_T 256

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

__global__ void __launch_bounds__(WALK_T)
k_walk(const float4 *__restrict__ node_a, const float4 *__restrict__ node_b,
       const int4 *__restrict__ node_c, const int32_t *__restrict__ gnode,
       const int32_t *__restrict__ gcount, const float4 *__restrict__ gbox,
       long long *__restrict__ cnt, int32_t *__restrict__ glen,
       int32_t *__restrict__ gself, int32_t *__restrict__ gcells,
       int32_t *__restrict__ list_id, float4 *__restrict__ list_xm, int64_t cap,
       int64_t alloc, unsigned *__restrict__ err)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t total = (int32_t)cnt[CNT_NODES];
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    long long pp = 0, pc = 0, tot = 0;
    int32_t mx = 0;
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
        const int32_t gn = gnode[g];
        const int32_t gend = node_c[gn].x;
        const int64_t base = (int64_t)g * cap;
        const int64_t room = alloc - base < cap ? (alloc - base > 0 ? alloc - base : 0) : cap;
        int32_t len = 0, ncell = 0, self_off = -1;
        int32_t cur = 0;
        int32_t guard = 0;
        while (cur < total) {
            const int32_t u = cur + lane;
            bool emit = false, cell_emit = false, own = false;
            int32_t succ = total;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (u < total) {
                const int4 c = node_c[u];
                a = node_a[u];
                if (c.w) {
                    emit = true;
                } else {
                    const bool holds = (u <= gn) && (gn < c.x);
                    emit = !holds && far_enough(a, __int_as_float(c.y), __int_as_float(c.z),
                                                blo, bhi, invth);
                    cell_emit = emit;
                }
                succ = emit ? c.x : u + 1;
                own = (u >= gn) && (u < gend);
            }
            // chain of visited nodes inside the window, starting at cur
            unsigned vis = 0u;
            int l = 0;
            int32_t nxt = total;
            for (;;) {
                vis |= 1u << l;
                const int32_t sl = __shfl_sync(FULL, succ, l);
                const int32_t off = sl - cur;
                if (sl >= total || off >= 32) { nxt = sl; break; }
                if (off <= l) { bad |= NB_EF_WALK; nxt = total; break; }
                l = off;
            }
            const unsigned em = __ballot_sync(FULL, emit) & vis;
            const unsigned cm = __ballot_sync(FULL, cell_emit) & vis;
            if ((em >> lane) & 1u) {
                const int32_t pos = len + __popc(em & lt);
                if (pos < room) {
                    const float4 b = node_b[u];
                    list_id[base + pos] = u;
                    list_xm[base + pos] =
                        make_float4(__fadd_rn(__fsub_rn(a.x, bc.x), b.x),
                                    __fadd_rn(__fsub_rn(a.y, bc.y), b.y),
                                    __fadd_rn(__fsub_rn(a.z, bc.z), b.z), a.w);
                }
            }
            if (self_off < 0) {
                const unsigned sm = em & __ballot_sync(FULL, own);
                if (sm) self_off = len + __popc(em & ((1u << (__ffs(sm) - 1)) - 1u));
            }
            len += __popc(em);
            ncell += __popc(cm);
            cur = nxt;
            if (++guard > total) { bad |= NB_EF_WALK; break; }
        }
        if (lane == 0) {
            glen[g] = len;
            gself[g] = self_off;
            gcells[g] = ncell;
            const long long m = gcount[g];
            pp += m * (long long)(len - ncell - 1);
            pc += m * (long long)ncell;
            tot += len;
            if (len > mx) mx = len;
            if (len > room) bad |= NB_EF_CAPACITY;
            if (self_off < 0) bad |= NB_EF_WALK;
        }
    }
    if (lane == 0) {
        nb_atomic_add(&cnt[CNT_PP], pp);
        nb_atomic_add(&cnt[CNT_PC], pc);
        nb_atomic_add(&cnt[CNT_PP_CUM], pp);
        nb_atomic_add(&cnt[CNT_PC_CUM], pc);
        nb_atomic_add(&cnt[CNT_LIST_TOT], tot);
        atomicMax(&cnt[CNT_LIST_MAX], (long long)mx);
        if (bad) atomicOr(err, bad);
    }
}

void nb_launch_walk(nb_ctx *c)
{
    cudaMemsetAsync(&c->cnt[CNT_LIST_TOT], 0, sizeof(long long) * 5, c->stream);
    static_assert(CNT_LIST_TOT + 4 == CNT_WALK_Q, "counter layout");
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_walk, WALK_T, 0);
    if (blocks < 1) blocks = 1;
    k_walk<<<c->num_sms * blocks, WALK_T, 0, c->stream>>>(
        c->node_a, c->node_b, c->node_c, c->gnode, c->gcount, c->gbox, c->cnt, c->glen,
        c->gself, c->gcells, c->list_id, c->list_xm, c->list_cap, c->list_alloc, c->err);
    c->launches++;
}
