// nb_neigh.cu -- fixed-radius neighbour search by the general treewalk
// (Sec. "General Treewalk", Fig. "general_treewalk": the descent of the force
// walk with another distance test and, in place of the particle-cell term,
// nothing; the paper names short-range interactions as its use).
//
// The neighbours of particle i are the j != i with |x_j - x_i|^2 <= h^2, the
// squared distance summed (x, y) then z in FP64 from the FP64 positions, each
// operation rounded on its own: the set is fixed by that definition, and the
// tree only prunes.  One warp walks one group breadth-first over the
// level-ordered records, as the force walk does.  A cell is skipped when its
// centre of mass lies farther from the group's box than h + s + (sqrt(3)/2) l
// (every member lies within (sqrt(3)/2) l of the cube's centre, which is s
// from the centre of mass), with a margin of 1e-5 of the root side for the
// FP32 rounding of the records and boxes; every other cell is opened, and
// every particle leaf reached is a candidate.  Each chunk of 32 candidates
// is tested against every member of the group with the FP64 definition:
// the first pass counts, an exclusive scan gives the offsets, the second
// pass writes the caller indices, and each target's run is then sorted
// ascending (Batcher's odd-even merge sort, in place).
#include "nb_walk.cuh"

#define NG_T 256
#define NG_WARPS (NG_T / NB_WARP)

__device__ __forceinline__ double pair_d2(const double *a, const double *b)
{
    const double dx = __dsub_rn(b[0], a[0]), dy = __dsub_rn(b[1], a[1]), dz = __dsub_rn(b[2], a[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// FILL false: count[perm[slot]] += neighbours; FILL true: write them at
// off[i] + cursor[i] (cursor = count array, zeroed between the passes)
template <bool FILL>
__global__ void __launch_bounds__(NG_T, 4)
k_neigh(const nb_wrec *__restrict__ wrec, const int32_t *__restrict__ gfirst,
        const int32_t *__restrict__ gcount, const float4 *__restrict__ gbox,
        const int32_t *__restrict__ n_first, const int32_t *__restrict__ perm,
        const double *__restrict__ x64, long long *__restrict__ cnt, double h2, float reach,
        int32_t *__restrict__ count, const int32_t *__restrict__ off, int32_t *__restrict__ idx,
        int64_t cap, int32_t *__restrict__ wq, int64_t wq_cap, int64_t n,
        const int32_t *__restrict__ sys_sorted, const int32_t *__restrict__ sys_root,
        unsigned *__restrict__ err)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t gw = (int64_t)blockIdx.x * NG_WARPS + (threadIdx.x >> 5);
    int32_t *const qa = wq + gw * 2 * wq_cap;
    int32_t *const qb = qa + wq_cap;
    __shared__ int32_t sq[NG_WARPS][2 * WQ_SMEM];
    int32_t *const qa_s = sq[threadIdx.x >> 5];
    int32_t *const qb_s = qa_s + WQ_SMEM;
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    const int32_t total = (int32_t)cnt[CNT_NODES];
    unsigned bad = 0;
    int32_t qmax = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)nb_atomic_add(&cnt[CNT_WALK_Q], 1LL);
        g = __shfl_sync(FULL, g, 0);
        if (g >= G) break;
        const float4 blo = gbox[3 * (int64_t)g], bhi = gbox[3 * (int64_t)g + 1];
        const int32_t f = gfirst[g], ng = gcount[g];
        if (!nb_in(f >= 0 && ng >= 1 && (int64_t)f + ng <= n, cnt, err, SITE_GROUPS, g)) continue;
        int32_t *qin = qa, *qout = qb, *qin_s = qa_s, *qout_s = qb_s;
        const int32_t gsys = sys_sorted ? sys_sorted[f] : 0;
        if (lane == 0) qin_s[0] = sys_root ? sys_root[gsys] : 0;
        __syncwarp();
        int32_t na = 1;
        int depth_guard = 0;
        while (na > 0) {
            int32_t nb = 0;
            for (int32_t i0 = 0; i0 < na; i0 += NB_WARP) {
                const NodeRec r = load_node<true>(i0 + lane, na, qin_s, qin, wrec, total, cnt, err);
                bool cand = false, open = false;
                int32_t fc = 0, nch = 0, cslot = 0;
                if (r.valid) {
                    fc = r.wb.z;
                    if (fc < 0) {
                        const int32_t u = r.wb.x;
                        if (nb_in(u >= 0 && u < total, cnt, err, SITE_WALK_NODE, u)) {
                            cslot = n_first[u];
                            cand = nb_in(cslot >= 0 && cslot < n, cnt, err, SITE_WALK_NODE, cslot);
                        }
                    } else {
                        const float w = reach + r.wc.y + 0.8660254f * r.wc.x;
                        if (!far_enough(r.a, w, 0.0f, blo, bhi, 1.0f) &&
                            nb_in(fc > r.b && (int64_t)fc + r.wb.w <= total, cnt, err,
                                  SITE_WALK_CHILD, r.b)) {
                            open = true;
                            nch = r.wb.w;
                        }
                    }
                }
                // the chunk's candidates against every member of the group
                const unsigned cm = __ballot_sync(FULL, cand);
                if (cm) {
                    double xc[3] = {0.0, 0.0, 0.0};
                    if (cand)
                        for (int k = 0; k < 3; k++) xc[k] = x64[3 * (int64_t)cslot + k];
                    const int32_t jc = cand ? perm[cslot] : 0;
                    for (int32_t t = 0; t < ng; t++) {
                        const int32_t ts = f + t;
                        const double xi[3] = {x64[3 * (int64_t)ts], x64[3 * (int64_t)ts + 1],
                                              x64[3 * (int64_t)ts + 2]};
                        const bool hit = cand && cslot != ts && pair_d2(xi, xc) <= h2;
                        const unsigned hm = __ballot_sync(FULL, hit);
                        if (!hm) continue;
                        const int32_t ti = perm[ts];
                        int32_t base = 0;
                        if (lane == 0) {
                            base = count[ti];
                            count[ti] = base + __popc(hm);
                        }
                        base = __shfl_sync(FULL, base, 0);
                        if (FILL && hit) {
                            const int64_t pos = (int64_t)off[ti] + base + __popc(hm & lt);
                            if (pos < (int64_t)off[ti + 1] && pos < cap) idx[pos] = jc;
                            else bad |= NB_EF_BOUNDS;
                        }
                    }
                }
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
                        if (pos < WQ_SMEM) qout_s[pos] = fc + k;
                        else if (pos < wq_cap) qout[pos] = fc + k;
                    }
                nb += __shfl_sync(FULL, incl, 31);
            }
            if (nb > qmax) qmax = nb;
            if (nb > wq_cap) { bad |= NB_EF_QUEUE; break; }
            __syncwarp();
            int32_t *t = qin; qin = qout; qout = t;
            t = qin_s; qin_s = qout_s; qout_s = t;
            na = nb;
            if (++depth_guard > NB_DEPTHS + 1) { bad |= NB_EF_WALK; break; }
        }
    }
    bad = __reduce_or_sync(FULL, bad);
    qmax = __reduce_max_sync(FULL, qmax);
    if (lane == 0) {
        atomicMax(&cnt[CNT_QMAX], (long long)qmax);
        if (bad) atomicOr(err, bad);
    }
}

// offsets: off64[i] = off32[i] for i <= n
__global__ void k_neigh_offsets(const int32_t *__restrict__ off32, int64_t n,
                                int64_t *__restrict__ off64)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        off64[i] = off32[i];
}

// every target's run sorted ascending in place, one warp per target:
// Batcher's odd-even merge sort over the next power of two, whose
// comparators all put the smaller value first, so slots past the run act as
// +infinity and are never touched
__global__ void __launch_bounds__(256)
k_neigh_sort(const int32_t *__restrict__ off, int64_t n, int32_t *__restrict__ idx)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
         i += warps) {
        int32_t *a = idx + off[i];
        const int32_t len = off[i + 1] - off[i];
        int32_t P = 1;
        while (P < len) P <<= 1;
        for (int32_t p = 1; p < P; p <<= 1)
            for (int32_t k = p; k >= 1; k >>= 1) {
                // comparators (i + j, i + j + k) for j = k % p, k % p + 2k, ...
                // and i < k, inside one block of 2p
                const int32_t j0 = k % p;
                const int32_t pairs = ((P - k - j0 + 2 * k - 1) / (2 * k)) * k;
                for (int32_t e = lane; e < pairs; e += 32) {
                    const int32_t x = j0 + (e / k) * 2 * k + e % k;
                    const int32_t y = x + k;
                    if (y >= len || x / (2 * p) != y / (2 * p)) continue;
                    const int32_t u = a[x], v = a[y];
                    if (u > v) {
                        a[x] = v;
                        a[y] = u;
                    }
                }
                __syncwarp();
            }
    }
}

// the walk of both passes; returns the error bits (synchronised)
static int neigh_pass(nb_ctx *c, bool fill, double h2, float reach, int32_t *idx, int64_t cap,
                      unsigned *bits)
{
    CK_RET(cudaMemsetAsync(&c->cnt[CNT_WALK_Q], 0, sizeof(long long), c->stream));
    CK_RET(cudaMemsetAsync(&c->cnt[CNT_QMAX], 0, sizeof(long long), c->stream));
    const int blocks = c->walk_warps / NG_WARPS;
    const int32_t *ss = c->nsys > 1 ? c->sys_sorted : nullptr;
    const int32_t *sr = c->nsys > 1 ? c->sys_root : nullptr;
    if (fill)
        k_neigh<true><<<blocks, NG_T, 0, c->stream>>>(
            c->wrec, c->gfirst, c->gcount, c->gbox, c->n_first, c->perm, c->p_x64, c->cnt, h2,
            reach, c->ccount, c->cstart, idx, cap, c->wq, c->wq_cap, c->n, ss, sr, c->err);
    else
        k_neigh<false><<<blocks, NG_T, 0, c->stream>>>(
            c->wrec, c->gfirst, c->gcount, c->gbox, c->n_first, c->perm, c->p_x64, c->cnt, h2,
            reach, c->ccount, nullptr, nullptr, 0, c->wq, c->wq_cap, c->n, ss, sr, c->err);
    nb_launched(c, "k_neigh");
    return nb_read_err(c, bits);
}

int nb_neigh_run(nb_ctx *c, double h, int n_crit, int64_t *off, int32_t *idx, int64_t cap,
                 int64_t *total)
{
    const int64_t n = c->n;
    const double L = nb_root_side(c);
    const double h2 = h * h;
    const float reach = (float)(h + 1e-5 * L);
    nb_launch_groups(c, 1.0f, n_crit, nullptr);
    for (int attempt = 0; attempt < 4; attempt++) {
        CK_RET(cudaMemsetAsync(c->ccount, 0, sizeof(int32_t) * (size_t)(n + 1), c->stream));
        unsigned bits = 0;
        int rc = neigh_pass(c, false, h2, reach, nullptr, 0, &bits);
        if (rc) return rc;
        if (bits & NB_EF_QUEUE) {   // a frontier outgrew the queues: grow them, walk again
            rc = nb_grow_queues(c);
            if (rc) return rc;
            continue;
        }
        if (bits) return nb_err_code(bits);
        if (!(L > 0.0)) return NB_ERR_CUDA;
        // offsets in caller order (the count array is in caller order)
        nb_exclusive_scan(c, c->ccount, c->cstart, n + 1, nullptr, &c->cnt[CNT_LIST_TOT]);
        k_neigh_offsets<<<nb_grid(n + 1, 256, c->num_sms * 8), 256, 0, c->stream>>>(c->cstart, n,
                                                                                 off);
        nb_launched(c, "k_neigh_offsets");
        long long tot = 0;
        CK_RET(cudaMemcpyAsync(&tot, &c->cnt[CNT_LIST_TOT], sizeof(long long),
                               cudaMemcpyDeviceToHost, c->stream));
        CK_RET(cudaStreamSynchronize(c->stream));
        *total = tot;
        if (tot >= INT32_MAX) return NB_ERR_CAPACITY;
        if (!idx || cap < tot) return NB_OK;   // counts and offsets only
        CK_RET(cudaMemsetAsync(c->ccount, 0, sizeof(int32_t) * (size_t)(n + 1), c->stream));
        rc = neigh_pass(c, true, h2, reach, idx, cap, &bits);
        if (rc) return rc;
        if (bits) return bits & NB_EF_BOUNDS ? NB_ERR_INTERNAL : nb_err_code(bits);
        k_neigh_sort<<<c->num_sms * 8, 256, 0, c->stream>>>(c->cstart, n, idx);
        nb_launched(c, "k_neigh_sort");
        CK_RET(cudaStreamSynchronize(c->stream));
        return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
    }
    return NB_ERR_CAPACITY;
}
