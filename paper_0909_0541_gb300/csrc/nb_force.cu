// nb_force.cu -- Eq. (gravity) summed over each group's interaction list.
//
// Work items cut a group's members into 64-target items (two targets per
// lane) while 64 or more remain, then one 32-target item if more than 32
// remain, then a tail of at most 32 targets rounded up to a power of two m'.
// An item of m' <= 32 targets runs as S source streams: the warp is S rows
// of W = 32/S lanes, stream s takes entries s*W .. s*W+W-1 of every
// 32-record tile, and the streams' sums are combined with shuffles at the
// end -- so small groups keep every lane busy.  Items of 4 to 32 targets
// hold two targets per lane (S = 64/m'), like the 64-target items, so every
// staged record pair feeds two interactions; items of two and one targets
// hold one (S = 16, 32).  One warp takes one item from a global queue;
// targets are FP32 coordinates relative to the group centre.  Sources are
// staged TILE at a time: one coalesced 16-byte load per lane into a per-warp
// shared-memory tile, then broadcast reads.  The tile holds record
// pairs interleaved (x_j, x_j+1, y_j, y_j+1 | z_j, z_j+1, m_j, m_j+1) so that
// each step below runs on two records at once with the packed FP32
// instructions (add/mul/fma .f32x2).  Per interaction:
//   dx = xj - xi (3 FADD); r2 = eps^2 + dx.dx (3 FFMA); ri = rsqrt(r2) (MUFU);
//   mr = mj ri; mr3 = mr ri ri (3 FMUL); a += mr3 dx (3 FFMA); phi -= mr (FADD)
// i.e. 13 FP32-pipe operations and one MUFU, issued as 6.5 packed
// instructions.  This stays on the CUDA cores: there is no dense contraction
// to hand to the tensor cores.
//
// Two phases per item: (1) the group's list (particles and accepted cells
// outside the group), unmasked; (2) the group's own members, read from the
// sorted particle arrays and converted to the same group-relative FP32
// coordinates, with the j == i term dropped by index.  Padding records are
// massless and far away.
//
// Queue order: after the walk, when every list length is known, the items
// are counting-sorted by estimated cost (records x targets per lane, in
// quarter-octave buckets) so that the queue hands out the costliest items
// first and the kernel does not end on one warp finishing a long list.  An
// item's result does not depend on when it runs, so the order changes
// timing only.
#include "nb_force.cuh"
#include "nb_walk.cuh"

#define F_T 256

// R targets per lane; S source streams: lane l is target row l % W of
// stream l / W, W = 32 / S, and holds targets i0 + row + r W (r < R)
// QUAD: list records carry the cells' quadrupoles (list_q) and the list
// phase adds the quadrupole term (TILE = 32, FP32 modes)
// CG: the list and its length are read through L2 only (the overlapped
// kernel reads lists that other warps of the same launch wrote)
template <int MODE, bool GUARD, int R, int S, int TILE, bool QUAD, bool CG = false>
__device__ __forceinline__ void force_item(
    int32_t g, int32_t i0, float4 *tile, const int32_t *__restrict__ gfirst,
    const int32_t *__restrict__ gcount, const int32_t *__restrict__ glen,
    const float4 *__restrict__ gbox, const float4 *__restrict__ p_hi,
    const float4 *__restrict__ p_lo, const int32_t *__restrict__ perm,
    const float4 *__restrict__ list_xm, const float4 *__restrict__ list_q, int64_t cap,
    int64_t alloc, int64_t n, float eps2, float *__restrict__ acc, float *__restrict__ pot,
    long long *__restrict__ cnt, unsigned *__restrict__ err)
{
    constexpr int W = NB_WARP / S;
    const int lane = threadIdx.x & 31;
    const int row = lane % W, stream = lane / W;
    const int32_t f = gfirst[g], ng = gcount[g];
    if (!(f >= 0 && ng >= 1 && (int64_t)f + ng <= n && i0 >= 0 && i0 < ng)) {
        if (lane == 0) nb_bad(cnt, err, SITE_FORCE, g);
        return;
    }
    // a list that outgrew its slot (or the storage) was reported by the walk;
    // never read past either
    const int64_t room = alloc - (int64_t)g * cap;
    int64_t lim = cap < room ? cap : room;
    if (lim < 0) lim = 0;
    const int32_t gl = CG ? __ldcg(&glen[g]) : glen[g];
    const int32_t len = gl < lim ? gl : (int32_t)lim;
    const float4 pad = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    Tgt t[R];
    Acc<MODE> A[R];
    Sum2 P[R];
    {
        const float4 bc = gbox[3 * (int64_t)g + 2];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int32_t k = i0 + r * W + row;
            const int32_t s = f + (k < ng ? k : ng - 1);
            const float4 h = p_hi[s], lo = p_lo[s];
            t[r].set(nb_rel(h.x, lo.x, bc.x), nb_rel(h.y, lo.y, bc.y), nb_rel(h.z, lo.z, bc.z));
            A[r].init();
            P[r].init();
        }
    }
    // (1) the list: sources outside the group, TILE records per tile
    constexpr int TK = TILE / NB_WARP;   // records each lane stages per tile
    const float4 *__restrict__ src = list_xm + (int64_t)g * cap;
    if constexpr (QUAD) {
        static_assert(TILE == NB_WARP, "quadrupole tiles hold 32 records");
        const float4 *__restrict__ srq = list_q + 2 * (int64_t)g * cap;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int32_t j0 = 0; j0 < len; j0 += TILE) {
            const int32_t jj = j0 + lane;
            const bool in = jj < len;
            const float4 qa = in ? srq[2 * (int64_t)jj] : z4;
            const float4 qb = in ? srq[2 * (int64_t)jj + 1] : z4;
            put_rec_q(tile, lane, in ? src[jj] : pad, qa, qb);
            const unsigned qm = __ballot_sync(0xffffffffu, qa.x != 0.f || qa.y != 0.f ||
                                                               qa.z != 0.f || qa.w != 0.f ||
                                                               qb.x != 0.f || qb.y != 0.f);
            __syncwarp();
            tile_pass_quad<MODE, GUARD, R, W>(tile, stream * W, t, eps2, qm, A, P);
            __syncwarp();
        }
    } else {
        // the next tile's records are loaded into registers while the warp
        // sums the current one, so the list fetch overlaps the arithmetic
        float4 nxt[TK];
#pragma unroll
        for (int k = 0; k < TK; k++) {
            const int32_t jj = k * NB_WARP + lane;
            nxt[k] = jj < len ? (CG ? __ldcg(&src[jj]) : src[jj]) : pad;
        }
        for (int32_t j0 = 0; j0 < len; j0 += TILE) {
#pragma unroll
            for (int k = 0; k < TK; k++) put_rec(tile, k * NB_WARP + lane, nxt[k]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < TK; k++) {
                const int32_t jj = j0 + TILE + k * NB_WARP + lane;
                nxt[k] = jj < len ? (CG ? __ldcg(&src[jj]) : src[jj]) : pad;
            }
            tile_pass<MODE, GUARD, false, R, W * TK>(tile, stream * W * TK, j0 + stream * W * TK,
                                                     t, nullptr, eps2, A, P);
            __syncwarp();
        }
    }
    // (2) the group's own members, j != i (the group's range and centre are
    // taken up again here, so they need not stay live through the list phase)
    const int32_t f2 = gfirst[g], ng2 = gcount[g];
    const float4 bc = gbox[3 * (int64_t)g + 2];
    int32_t kk[R];
#pragma unroll
    for (int r = 0; r < R; r++) kk[r] = i0 + r * W + row;
    for (int32_t j0 = 0; j0 < ng2; j0 += NB_WARP) {
        const int32_t jj = j0 + lane;
        float4 v = pad;
        if (jj < ng2) {
            const float4 h = p_hi[f2 + jj], lo = p_lo[f2 + jj];
            v = make_float4(nb_rel(h.x, lo.x, bc.x), nb_rel(h.y, lo.y, bc.y),
                            nb_rel(h.z, lo.z, bc.z), h.w);
        }
        put_rec(tile, lane, v);
        __syncwarp();
        // only a tile that holds one of this item's targets needs the j == i
        // mask; elsewhere the mask changes nothing and the plain pass runs
        if (j0 < i0 + R * W && j0 + NB_WARP > i0)
            tile_pass<MODE, GUARD, true, R, W>(tile, stream * W, j0 + stream * W, t, kk, eps2, A,
                                               P);
        else
            tile_pass<MODE, GUARD, false, R, W>(tile, stream * W, j0 + stream * W, t, kk, eps2,
                                                A, P);
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < R; r++) pair_fold<MODE>(A[r], P[r]);
    if constexpr (S > 1) {
#pragma unroll
        for (int o = W; o < NB_WARP; o <<= 1)
#pragma unroll
            for (int r = 0; r < R; r++) stream_sum<MODE>(A[r], o);
        if (stream != 0) return;
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (kk[r] >= ng2) continue;
        const int64_t o = perm[f2 + kk[r]];
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

// one item in a function of its own: each item shape gets its own register
// allocation instead of sharing the largest one's (the call costs a few
// instructions per item, against thousands per list)
template <int MODE, bool GUARD, int R, int S, int TILE, bool QUAD>
__device__ __noinline__ void force_item_call(
    int32_t g, int32_t i0, float4 *tile, const int32_t *__restrict__ gfirst,
    const int32_t *__restrict__ gcount, const int32_t *__restrict__ glen,
    const float4 *__restrict__ gbox, const float4 *__restrict__ p_hi,
    const float4 *__restrict__ p_lo, const int32_t *__restrict__ perm,
    const float4 *__restrict__ list_xm, const float4 *__restrict__ list_q, int64_t cap,
    int64_t alloc, int64_t n, float eps2, float *__restrict__ acc, float *__restrict__ pot,
    long long *__restrict__ cnt, unsigned *__restrict__ err)
{
    force_item<MODE, GUARD, R, S, TILE, QUAD>(g, i0, tile, gfirst, gcount, glen, gbox, p_hi, p_lo,
                                              perm, list_xm, list_q, cap, alloc, n, eps2, acc,
                                              pot, cnt, err);
}

// cost bucket of an item, 0 = costliest: 4 x log2 of (list + members) x
// targets per lane / source streams, in quarter octaves
__device__ __forceinline__ int item_bucket(const int32_t *__restrict__ items,
                                           const int32_t *__restrict__ gcount,
                                           const int32_t *__restrict__ glen, int32_t it,
                                           int32_t ngroups)
{
    const int32_t g = items[2 * (int64_t)it], word = items[2 * (int64_t)it + 1];
    if (g < 0 || g >= ngroups) return NB_IBKT - 1;   // k_force reports the bad item
    const uint32_t len = (uint32_t)max(glen[g], 0) + (uint32_t)max(gcount[g], 0);
    const int ls = (word & ITEM_R2) ? 0 : min((word >> ITEM_LS_SHIFT) & 7, 5);
    uint32_t w = ((word & ITEM_R2) ? 2u * len : len) >> ls;
    if (w < 1) w = 1;
    const int e = 31 - __clz(w);
    const int q = e >= 2 ? (int)((w >> (e - 2)) & 3u) : (int)((w << (2 - e)) & 3u);
    const int b = 4 * e + q;
    return NB_IBKT - 1 - min(b, NB_IBKT - 1);
}

__device__ __forceinline__ int32_t force_items(const long long *cnt, int64_t max_items)
{
    const long long v = cnt[CNT_ITEMS];
    return (int32_t)(v < max_items ? v : max_items);
}

__global__ void __launch_bounds__(256)
k_item_hist(const int32_t *__restrict__ items, const int32_t *__restrict__ gcount,
            const int32_t *__restrict__ glen, const long long *__restrict__ cnt,
            int64_t max_items, int32_t *__restrict__ bkt)
{
    __shared__ int32_t h[NB_IBKT];
    if (threadIdx.x < NB_IBKT) h[threadIdx.x] = 0;
    __syncthreads();
    const int32_t nitems = force_items(cnt, max_items), ngroups = (int32_t)cnt[CNT_GROUPS];
    for (int32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
         it += gridDim.x * blockDim.x)
        atomicAdd(&h[item_bucket(items, gcount, glen, it, ngroups)], 1);
    __syncthreads();
    if (threadIdx.x < NB_IBKT && h[threadIdx.x]) atomicAdd(&bkt[threadIdx.x], h[threadIdx.x]);
}

// bkt[0..NB_IBKT) bucket sizes, bkt[NB_IBKT..2 NB_IBKT) fill cursors (zeroed)
__global__ void __launch_bounds__(256)
k_item_order(const int32_t *__restrict__ items, const int32_t *__restrict__ gcount,
             const int32_t *__restrict__ glen, long long *__restrict__ cnt, int64_t max_items,
             int32_t *__restrict__ bkt, int32_t *__restrict__ order, unsigned *__restrict__ err)
{
    static_assert(NB_IBKT <= 256, "one bucket per thread");
    __shared__ int32_t start[NB_IBKT];
    {
        int32_t all;
        const int32_t st = nb_block_scan256(threadIdx.x < NB_IBKT ? bkt[threadIdx.x] : 0, &all);
        if (threadIdx.x < NB_IBKT) start[threadIdx.x] = st;
        __syncthreads();
    }
    const int32_t nitems = force_items(cnt, max_items), ngroups = (int32_t)cnt[CNT_GROUPS];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t warps = gridDim.x * (blockDim.x >> 5);
    for (int32_t base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * NB_WARP;
         base < nitems; base += warps * NB_WARP) {
        const int32_t it = base + lane;
        const bool ok = it < nitems;
        const int b = ok ? item_bucket(items, gcount, glen, it, ngroups) : NB_IBKT + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        int32_t got = 0;
        if (ok && lane == leader) got = atomicAdd(&bkt[NB_IBKT + b], __popc(peers));
        got = __shfl_sync(0xffffffffu, got, leader);
        if (!ok) continue;
        const int32_t pos = start[b] + got + __popc(peers & lt);
        if (!nb_in(pos >= 0 && pos < nitems, cnt, err, SITE_FORCE, pos)) continue;
        order[pos] = it;
    }
}

// TILE: list records staged per tile (the j-tile depth); BT: threads per
// block.  Both are chosen by the autotuner for the FP32 mode.
template <int MODE, bool GUARD, int TILE, int BT, bool QUAD = false>
__global__ void __launch_bounds__(BT, (MODE == MODE_F64 ? 5 : 4) * F_T / BT)
k_force(const int32_t *__restrict__ items, const int32_t *__restrict__ order,
        const int32_t *__restrict__ gfirst,
        const int32_t *__restrict__ gcount, const int32_t *__restrict__ glen,
        const float4 *__restrict__ gbox, const float4 *__restrict__ p_hi,
        const float4 *__restrict__ p_lo, const int32_t *__restrict__ perm,
        const float4 *__restrict__ list_xm, const float4 *__restrict__ list_q, int64_t cap,
        int64_t alloc, int64_t n, long long *__restrict__ cnt, float eps2,
        float *__restrict__ acc, float *__restrict__ pot, unsigned *__restrict__ err,
        int64_t max_items)
{
    __shared__ float4 tiles[BT / NB_WARP][QUAD ? TILE * 5 / 2
                                               : (TILE > F_TILE_STREAMS ? TILE : F_TILE_STREAMS)];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t nitems = (int32_t)cnt[CNT_ITEMS];
    const int32_t ngroups = (int32_t)cnt[CNT_GROUPS];
    if (nitems > max_items) {
        if (threadIdx.x == 0 && blockIdx.x == 0) nb_bad(cnt, err, SITE_FORCE, nitems);
        nitems = (int32_t)max_items;
    }
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)nb_atomic_add(&cnt[CNT_FORCE_Q], 1LL);
        it = __shfl_sync(FULL, it, 0);
        if (it >= nitems) break;
        it = order[it];
        if (it < 0 || it >= nitems) {
            if (lane == 0) nb_bad(cnt, err, SITE_FORCE, it);
            continue;
        }
        const int32_t g = items[2 * (int64_t)it], word = items[2 * (int64_t)it + 1];
        const int32_t i0 = word & ITEM_MEMBER_MASK;
        if (g < 0 || g >= ngroups) {
            if (lane == 0) nb_bad(cnt, err, SITE_FORCE, g);
            continue;
        }
#define NB_FORCE_ITEM_AT(R, S, I0)                                                            \
    force_item_call<MODE, GUARD, R, S, QUAD ? TILE : item_tile(S, TILE), QUAD>(                   \
        g, I0, tiles[w], gfirst, gcount, glen, gbox,                                              \
                                                   p_hi,                                          \
                                              p_lo, perm, list_xm, list_q, cap, alloc, n, eps2,   \
                                              acc, pot, cnt, err)
#define NB_FORCE_ITEM(R, S) NB_FORCE_ITEM_AT(R, S, i0)
        if constexpr (QUAD) {   // one target per lane: a 64-target item in two passes
            if (word & ITEM_R2) {
                NB_FORCE_ITEM_AT(1, 1, i0);
                NB_FORCE_ITEM_AT(1, 1, i0 + NB_WARP);
            } else {
                switch ((word >> ITEM_LS_SHIFT) & 7) {
                case 0: NB_FORCE_ITEM(1, 1); break;
                case 1: NB_FORCE_ITEM(1, 2); break;
                case 2: NB_FORCE_ITEM(1, 4); break;
                case 3: NB_FORCE_ITEM(1, 8); break;
                case 4: NB_FORCE_ITEM(1, 16); break;
                default: NB_FORCE_ITEM(1, 32); break;
                }
            }
        } else {
            NB_ITEM_SHAPES(word, NB_FORCE_ITEM);
        }
#undef NB_FORCE_ITEM
#undef NB_FORCE_ITEM_AT
    }
}

template <int MODE, bool GUARD, int TILE, int BT, bool QUAD = false>
static void launch_force_t(nb_ctx *c, float eps2, float *acc, float *pot)
{
    static int blocks = 0;
    if (blocks == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks,
                                                      k_force<MODE, GUARD, TILE, BT, QUAD>, BT, 0);
        if (blocks < 1) blocks = 1;
    }
    k_force<MODE, GUARD, TILE, BT, QUAD><<<c->num_sms * blocks, BT, 0, c->stream>>>(
        c->items, c->item_order, c->gfirst, c->gcount, c->glen, c->gbox, c->p_hi, c->p_lo, c->perm,
        c->list_xm, c->list_q, c->list_cap, c->list_alloc, c->n, c->cnt, eps2, acc, pot, c->err,
        c->max_items);
    nb_launched(c, QUAD ? "k_force (quadrupole)" : "k_force");
}

// FP32: the context's j-tile depth (32 or 64) and block size (256 or 128);
// the compensated and FP64-accumulated modes use 32 and 256
template <int MODE, bool GUARD>
static void launch_force(nb_ctx *c, float eps2, float *acc, float *pot)
{
    if constexpr (MODE == MODE_FP32) {
        switch ((c->force_tile == 64 ? 2 : 0) + (c->force_block == 128 ? 1 : 0)) {
        case 0: launch_force_t<MODE, GUARD, 32, 256>(c, eps2, acc, pot); break;
        case 1: launch_force_t<MODE, GUARD, 32, 128>(c, eps2, acc, pot); break;
        case 2: launch_force_t<MODE, GUARD, 64, 256>(c, eps2, acc, pot); break;
        default: launch_force_t<MODE, GUARD, 64, 128>(c, eps2, acc, pot); break;
        }
    } else {
        launch_force_t<MODE, GUARD, F_TILE, F_T>(c, eps2, acc, pot);
    }
}

void nb_launch_forces(nb_ctx *c, float eps, float *acc, float *pot, int precision)
{
    cudaMemsetAsync(&c->cnt[CNT_FORCE_Q], 0, sizeof(long long), c->stream);
    cudaMemsetAsync(c->item_bkt, 0, sizeof(int32_t) * 2 * NB_IBKT, c->stream);
    const int ig = c->num_sms * 2;
    k_item_hist<<<ig, 256, 0, c->stream>>>(c->items, c->gcount, c->glen, c->cnt, c->max_items,
                                           c->item_bkt);
    nb_launched(c, "k_item_hist");
    k_item_order<<<ig, 256, 0, c->stream>>>(c->items, c->gcount, c->glen, c->cnt, c->max_items,
                                            c->item_bkt, c->item_order, c->err);
    nb_launched(c, "k_item_order");
    const float eps2 = eps * eps;
    const bool guard = !(eps2 >= FLT_MIN);
    if (c->quad && c->lists_quad) {   // FP32 and compensated modes (checked by the caller)
        switch (precision * 2 + (guard ? 1 : 0)) {
        case 0: launch_force_t<MODE_FP32, false, F_TILE, F_T, true>(c, eps2, acc, pot); break;
        case 1: launch_force_t<MODE_FP32, true, F_TILE, F_T, true>(c, eps2, acc, pot); break;
        case 2: launch_force_t<MODE_COMP, false, F_TILE, F_T, true>(c, eps2, acc, pot); break;
        default: launch_force_t<MODE_COMP, true, F_TILE, F_T, true>(c, eps2, acc, pot); break;
        }
        return;
    }
    switch (precision * 2 + (guard ? 1 : 0)) {
    case 0: launch_force<MODE_FP32, false>(c, eps2, acc, pot); break;
    case 1: launch_force<MODE_FP32, true>(c, eps2, acc, pot); break;
    case 2: launch_force<MODE_COMP, false>(c, eps2, acc, pot); break;
    case 3: launch_force<MODE_COMP, true>(c, eps2, acc, pot); break;
    case 4: launch_force<MODE_F64, false>(c, eps2, acc, pot); break;
    default: launch_force<MODE_F64, true>(c, eps2, acc, pot); break;
    }
}

// ---------------------------------------------------------------- overlap
// The walk and the force sum in one persistent launch.  The walk is bound by
// the latency of its record fetches and the force sum by the FMA pipe; run as
// two launches, each leaves the other's unit idle.  Here every warp claims
// the next force item (item order, one atomic each) and, until that item's
// group has been walked, walks the next group in line (group order); once
// every walk is claimed it waits, bounded, for the claimed ones.  A group's
// items are contiguous and walks go in group order, so a warp only ever
// waits for walks that running warps have claimed, and the SMs hold walking
// and summing warps at the same time.  A finished walk publishes
// its list with a release store to the group's flag; a force warp acquires
// the flag and reads the list through L2.  Every item and every list is
// computed as in the two separate launches, so the results are the same bits.
__device__ __forceinline__ int32_t ov_ld_acquire(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void ov_st_release(int32_t *p, int32_t v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

#define OV_T 256
#define OV_WARPS (OV_T / NB_WARP)
#define OV_SPIN_LIMIT (1u << 22)

template <int MODE, bool GUARD>
__global__ void __launch_bounds__(OV_T, 4)
k_walk_force(const nb_wrec *__restrict__ wrec, const int32_t *__restrict__ pid2bfs,
             const int32_t *__restrict__ gnode, const int32_t *__restrict__ gcount,
             const float4 *__restrict__ gbox, long long *__restrict__ cnt,
             int32_t *__restrict__ glen, int32_t *__restrict__ gcells,
             int32_t *__restrict__ list_id, float4 *__restrict__ list_xm, int64_t cap,
             int64_t alloc, int32_t *__restrict__ wq, int64_t wq_cap, unsigned *__restrict__ err,
             const double *__restrict__ roots, const int8_t *__restrict__ n_depth,
             const int32_t *__restrict__ gfirst, const int32_t *__restrict__ sys_sorted,
             const int32_t *__restrict__ sys_root, const int32_t *__restrict__ items,
             const float4 *__restrict__ p_hi, const float4 *__restrict__ p_lo,
             const int32_t *__restrict__ perm, int64_t n, float eps2, float *__restrict__ acc,
             float *__restrict__ pot, int64_t max_items, int32_t *__restrict__ gready)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t gw = (int64_t)blockIdx.x * OV_WARPS + w;
    int32_t *const qa = wq + gw * 2 * wq_cap;
    int32_t *const qb = qa + wq_cap;
    // per warp: the walk's frontier queues, or (while it sums) the force tile
    __shared__ __align__(16) int32_t sq[OV_WARPS][2 * WQ_SMEM];
    int32_t *const qa_s = sq[w];
    int32_t *const qb_s = qa_s + WQ_SMEM;
    float4 *const tile = reinterpret_cast<float4 *>(sq[w]);
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    const int32_t total = (int32_t)cnt[CNT_NODES];
    int32_t nitems = (int32_t)cnt[CNT_ITEMS];
    if (nitems > max_items) {
        if (threadIdx.x == 0 && blockIdx.x == 0) nb_bad(cnt, err, SITE_FORCE, nitems);
        nitems = (int32_t)max_items;
    }
    long long pp = 0, pc = 0, tot = 0;
    int32_t mx = 0, qmax = 0;
    unsigned bad = 0;
    for (;;) {
        // the next force item, in item order (one atomic per item)
        long long task = 0;
        if (lane == 0) task = nb_atomic_add(&cnt[CNT_FORCE_Q], 1LL);
        task = __shfl_sync(FULL, task, 0);
        if (task >= nitems) break;
        const int32_t gt = items[2 * task];
        if (gt < 0 || gt >= G) {
            if (lane == 0) nb_bad(cnt, err, SITE_FORCE, task);
            continue;
        }
        // until its group's list is complete, walk the next group in line;
        // once every walk is claimed, wait (bounded) for the claimed ones
        bool ready = false;
        for (unsigned spins = 0;;) {
            int32_t rd = 0;
            if (lane == 0) rd = ov_ld_acquire(&gready[gt]);
            ready = __shfl_sync(FULL, rd, 0) != 0;
            if (ready) break;
            long long gw = G;
            if (lane == 0 && *(volatile long long *)&cnt[CNT_WALK_Q] < G)
                gw = nb_atomic_add(&cnt[CNT_WALK_Q], 1LL);
            gw = __shfl_sync(FULL, gw, 0);
            if (gw < G) {
                walk_one<false, false>((int)gw, wrec, pid2bfs, gnode, gcount, gbox, cnt, glen,
                                       gcells, list_id, list_xm, nullptr, nullptr, cap, alloc, qa,
                                       qb, qa_s, qb_s, wq_cap, err, nullptr, roots, n_depth,
                                       gfirst, sys_sorted, sys_root, total, lane, lt, pp, pc, tot,
                                       mx, qmax, bad);
                __threadfence();   // every lane's list writes before the flag
                __syncwarp();
                if (lane == 0) ov_st_release(&gready[gw], 1);
                continue;
            }
            if (++spins > OV_SPIN_LIMIT) {
                if (lane == 0) nb_bad(cnt, err, SITE_OVERLAP_WAIT, gt);
                break;
            }
            __nanosleep(100);
        }
        __syncwarp();   // lane 0's acquire orders the whole warp's reads of the list
        if (!ready) break;
        const int32_t g = gt, word = items[2 * task + 1];
        const int32_t i0 = word & ITEM_MEMBER_MASK;
#define NB_OV_ITEM(R, S)                                                                      \
    force_item<MODE, GUARD, R, S, item_tile(S, F_TILE), false, true>(                             \
        g, i0, tile, gfirst, gcount, glen, gbox,                                                  \
                                                       p_hi, p_lo, perm, list_xm, nullptr, cap,  \
                                                       alloc, n, eps2, acc, pot, cnt, err)
        NB_ITEM_SHAPES(word, NB_OV_ITEM);
#undef NB_OV_ITEM
        __syncwarp();
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

template <int MODE, bool GUARD>
static void launch_walk_force_t(nb_ctx *c, float eps2, float *acc, float *pot)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_walk_force<MODE, GUARD>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr = true;
    }
    // one pair of frontier queues per warp: no more warps than the queues hold
    const int blocks = c->walk_warps / OV_WARPS;
    k_walk_force<MODE, GUARD><<<blocks > 0 ? blocks : 1, OV_T, 0, c->stream>>>(
        c->wrec, c->pid2bfs, c->gnode, c->gcount, c->gbox, c->cnt, c->glen, c->gcells,
        c->list_id, c->list_xm, c->list_cap, c->list_alloc, c->wq, c->wq_cap, c->err, c->root,
        c->n_depth, c->gfirst, c->nsys > 1 ? c->sys_sorted : nullptr,
        c->nsys > 1 ? c->sys_root : nullptr, c->items, c->p_hi, c->p_lo, c->perm, c->n, eps2,
        acc, pot, c->max_items, c->gready);
    nb_launched(c, "k_walk_force");
}

// after the groups are formed: clears the counters and flags, then the
// overlapped launch (FP32 and compensated modes)
void nb_launch_walk_force(nb_ctx *c, float eps, float *acc, float *pot, int precision)
{
    cudaMemsetAsync(&c->cnt[CNT_LIST_TOT], 0, sizeof(long long) * 5, c->stream);
    static_assert(CNT_LIST_TOT + 4 == CNT_WALK_Q, "counter layout");
    cudaMemsetAsync(&c->cnt[CNT_QMAX], 0, sizeof(long long), c->stream);
    cudaMemsetAsync(&c->cnt[CNT_FORCE_Q], 0, sizeof(long long), c->stream);
    cudaMemsetAsync(c->gready, 0, sizeof(int32_t) * (size_t)c->max_n, c->stream);
    const float eps2 = eps * eps;
    const bool guard = !(eps2 >= FLT_MIN);
    switch ((precision == NB_FP32_COMP ? 2 : 0) + (guard ? 1 : 0)) {
    case 0: launch_walk_force_t<MODE_FP32, false>(c, eps2, acc, pot); break;
    case 1: launch_walk_force_t<MODE_FP32, true>(c, eps2, acc, pot); break;
    case 2: launch_walk_force_t<MODE_COMP, false>(c, eps2, acc, pot); break;
    default: launch_walk_force_t<MODE_COMP, true>(c, eps2, acc, pot); break;
    }
}

// ---------------------------------------------------------------- judge
// FP64 direct sum: one block per target, a deterministic tree reduction.
__global__ void __launch_bounds__(256)
k_direct(const double *__restrict__ pos, const float *__restrict__ mass, int64_t n,
         double eps2, const int64_t *__restrict__ targets, int64_t nt,
         double *__restrict__ acc, double *__restrict__ pot)
{
    __shared__ double red[4][256];
    for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const int64_t i = targets ? targets[t] : t;
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            if (j == i) continue;
            const double dx = pos[3 * j] - xi, dy = pos[3 * j + 1] - yi, dz = pos[3 * j + 2] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) continue;
            const double ri = 1.0 / sqrt(r2);
            const double m = (double)mass[j];
            const double mr3 = m * ri * ri * ri;
            ax += mr3 * dx;
            ay += mr3 * dy;
            az += mr3 * dz;
            p -= m * ri;
        }
        red[0][threadIdx.x] = ax;
        red[1][threadIdx.x] = ay;
        red[2][threadIdx.x] = az;
        red[3][threadIdx.x] = p;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o)
                for (int k = 0; k < 4; k++) red[k][threadIdx.x] += red[k][threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            acc[3 * t] = red[0][0];
            acc[3 * t + 1] = red[1][0];
            acc[3 * t + 2] = red[2][0];
            pot[t] = red[3][0];
        }
        __syncthreads();
    }
}

int nb_launch_direct(const double *pos, const float *mass, int64_t n, double eps,
                     const int64_t *targets, int64_t nt, double *acc, double *pot,
                     cudaStream_t s)
{
    if (nt <= 0) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t g = nt < (int64_t)sms * 8 ? nt : (int64_t)sms * 8;
    k_direct<<<(int)g, 256, 0, s>>>(pos, mass, n, eps * eps, targets, nt, acc, pot);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
