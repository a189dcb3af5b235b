// nb_tree.cu -- oct-tree construction on the GPU (the host steps 1-3 of the
// paper's flow, Sec. "Our GPU implementation", moved onto the device).
//
// Bottom-up build from Morton-sorted keys.  With c[i] the number of leading
// 3-bit digits shared by sorted keys i and i+1 (c[-1] = c[n-1] = -1), the
// cells (key prefixes shared by >= 2 particles) whose first particle is a are
// exactly the levels c[a-1]+1 .. c[a].  Ordering nodes by (first particle,
// depth) is depth-first preorder, so with S = exclusive scan of
// max(0, c[a] - c[a-1]):
//     cell (a, level)  -> node id S[a] + a + (level - c[a-1] - 1)
//     particle leaf a  -> node id S[a+1] + a
//     more(cell)       =  id + 1
//     next(node)       =  S[b+1] + b + 1, b = last particle of the node
// Every FP64/FP32 operation that decides a key, a moment or an opening test
// is written with explicit round-to-nearest intrinsics, never contracted.
#include "nb_internal.cuh"

#define NB_IBLOCK 64

// ------------------------------------------------------------ bbox, root
__global__ void __launch_bounds__(256)
k_bbox(const double *__restrict__ pos, int64_t n, double *__restrict__ part,
       unsigned *__restrict__ err)
{
    double lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; k++) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const double x = pos[3 * i + k];
            bad |= !isfinite(x);
            lo[k] = fmin(lo[k], x);
            hi[k] = fmax(hi[k], x);
        }
    }
    if (bad) atomicOr(err, NB_EF_NONFINITE);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            lo[k] = fmin(lo[k], __shfl_down_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_down_sync(0xffffffffu, hi[k], o));
        }
    __shared__ double s[8][6];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; k++) { s[w][k] = lo[k]; s[w][3 + k] = hi[k]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = s[0][threadIdx.x];
        for (int ww = 1; ww < 8; ww++)
            v = threadIdx.x < 3 ? fmin(v, s[ww][threadIdx.x]) : fmax(v, s[ww][threadIdx.x]);
        part[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

// Root cube: centre = bbox centre, side = max extent * (1 + 2^-20), 1 when
// every particle coincides; corner = centre - side/2.
__global__ void k_root(const double *__restrict__ part, int nblk, double *__restrict__ root)
{
    if (threadIdx.x != 0) return;
    double lo[3], hi[3];
    for (int k = 0; k < 3; k++) { lo[k] = part[k]; hi[k] = part[3 + k]; }
    for (int b = 1; b < nblk; b++)
        for (int k = 0; k < 3; k++) {
            lo[k] = fmin(lo[k], part[6 * b + k]);
            hi[k] = fmax(hi[k], part[6 * b + 3 + k]);
        }
    double ext = 0.0;
    for (int k = 0; k < 3; k++) {
        root[k] = __dmul_rn(0.5, __dadd_rn(lo[k], hi[k]));
        const double e = __dsub_rn(hi[k], lo[k]);
        if (e > ext) ext = e;
    }
    double L = __dmul_rn(ext, 1.0 + 0x1p-20);
    if (!(L > 0.0)) L = 1.0;
    root[3] = L;
    for (int k = 0; k < 3; k++) root[4 + k] = __dsub_rn(root[k], __dmul_rn(0.5, L));
}

// ------------------------------------------------------------ Morton keys
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

__device__ __forceinline__ uint32_t grid_coord(double x, double corner, double L)
{
    const double f = floor(__dmul_rn(__ddiv_rn(__dsub_rn(x, corner), L), 2097152.0));
    if (f < 0.0) return 0u;
    if (f > 2097151.0) return 2097151u;
    return (uint32_t)f;
}

__global__ void __launch_bounds__(256)
k_keys(const double *__restrict__ pos, int64_t n, const double *__restrict__ root,
       uint64_t *__restrict__ key, uint32_t *__restrict__ idx)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double L = root[3];
    const uint32_t qx = grid_coord(pos[3 * i], root[4], L);
    const uint32_t qy = grid_coord(pos[3 * i + 1], root[5], L);
    const uint32_t qz = grid_coord(pos[3 * i + 2], root[6], L);
    key[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    idx[i] = (uint32_t)i;
}

// sorted slot s: gather the caller's particle idx[s]; split FP64 positions
// into an FP32 pair (hi = nearest float, lo = float of the remainder)
__global__ void __launch_bounds__(256)
k_gather(const double *__restrict__ pos, const float *__restrict__ mass, int64_t n,
         const uint32_t *__restrict__ idx, int32_t *__restrict__ perm,
         double *__restrict__ x64, float4 *__restrict__ p_hi, float4 *__restrict__ p_lo)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = idx[s];
    perm[s] = (int32_t)i;
    float h[3], l[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double x = pos[3 * (int64_t)i + k];
        x64[3 * s + k] = x;
        h[k] = __double2float_rn(x);
        l[k] = __double2float_rn(__dsub_rn(x, (double)h[k]));
    }
    p_hi[s] = make_float4(h[0], h[1], h[2], mass[i]);
    p_lo[s] = make_float4(l[0], l[1], l[2], 0.0f);
}

// ------------------------------------------------------------ cells
__device__ __forceinline__ int common_levels(uint64_t a, uint64_t b)
{
    const uint64_t x = a ^ b;
    if (x == 0) return NB_LEVELS;
    return (__clzll((long long)x) - 1) / 3;
}

__global__ void __launch_bounds__(256)
k_levels(const uint64_t *__restrict__ key, int64_t n, int8_t *__restrict__ clev,
         int32_t *__restrict__ ccount)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int ca = a + 1 < n ? common_levels(key[a], key[a + 1]) : -1;
    const int cp = a > 0 ? common_levels(key[a - 1], key[a]) : -1;
    clev[a] = (int8_t)ca;
    ccount[a] = ca > cp ? ca - cp : 0;
}

__global__ void __launch_bounds__(256)
k_cells(const uint64_t *__restrict__ key, int64_t n, const int8_t *__restrict__ clev,
        const int32_t *__restrict__ cstart, const float4 *__restrict__ p_hi,
        const float4 *__restrict__ p_lo, const double *__restrict__ x64,
        float4 *__restrict__ node_a, float4 *__restrict__ node_b, int4 *__restrict__ node_c,
        int32_t *__restrict__ n_level, int32_t *__restrict__ n_first,
        int32_t *__restrict__ n_count, int32_t *__restrict__ n_parent,
        int32_t *__restrict__ n_nchild, int32_t *__restrict__ n_arrive,
        double *__restrict__ n_mass, double *__restrict__ n_mx, double *__restrict__ n_com,
        long long *__restrict__ cnt)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int32_t C = cstart[n];
    const int32_t total = C + (int32_t)n;
    if (a == 0) cnt[CNT_NODES] = total;
    const int ca = clev[a];
    const int cp = a > 0 ? clev[a - 1] : -1;
    const int k = ca > cp ? ca - cp : 0;
    const int32_t base = cstart[a] + (int32_t)a;
    const int32_t leaf = base + k;

    // particle leaf
    const float4 h = p_hi[a];
    node_a[leaf] = h;
    node_b[leaf] = p_lo[a];
    node_c[leaf] = make_int4(leaf + 1, 0, 0, 1);
    n_level[leaf] = -1;
    n_first[leaf] = (int32_t)a;
    n_count[leaf] = 1;
    n_nchild[leaf] = 0;
    const double m = (double)h.w;
    n_mass[leaf] = m;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double x = x64[3 * a + d];
        n_com[3 * (int64_t)leaf + d] = x;
        n_mx[3 * (int64_t)leaf + d] = __dmul_rn(m, x);
    }
    if (k > 0) n_parent[leaf] = leaf - 1;
    else if (leaf == 0) n_parent[leaf] = -1;

    // cells starting at a, deepest first; each run contains the deeper one
    const uint64_t ka = key[a];
    int64_t b = a;
    int maxlev = -1;
    for (int lev = ca; lev > cp; lev--) {
        const int32_t id = base + (lev - cp - 1);
        const int shift = 63 - 3 * lev;
        const uint64_t P = ka >> shift;
        int64_t lo = b, step = 1, hi = b + 1;
        while (hi < n && (key[hi] >> shift) == P) {
            lo = hi;
            step <<= 1;
            hi = lo + step;
        }
        if (hi > n) hi = n;
        while (hi - lo > 1) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if ((key[mid] >> shift) == P) lo = mid; else hi = mid;
        }
        b = lo;
        node_c[id] = make_int4(cstart[b + 1] + (int32_t)b + 1, 0, 0, 0);
        n_level[id] = lev;
        n_first[id] = (int32_t)a;
        n_count[id] = (int32_t)(b - a + 1);
        n_arrive[id] = 0;
        if (lev > cp + 1) n_parent[id] = id - 1;
        else if (id == 0) n_parent[id] = -1;
        if (lev > maxlev) maxlev = lev;
    }
    if (maxlev >= 0) atomicMax(&cnt[CNT_MAXLEVEL], (long long)maxlev);
}

// every cell writes itself as parent of its children (child = id + 1, then
// next of each child until the cell's own next)
__global__ void __launch_bounds__(256)
k_parents(const int4 *__restrict__ node_c, const long long *__restrict__ cnt,
          int32_t *__restrict__ n_parent, int32_t *__restrict__ n_nchild)
{
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += gridDim.x * blockDim.x) {
        const int4 cu = node_c[u];
        if (cu.w) continue;
        int32_t ch = u + 1, nch = 0;
        while (ch < cu.x) {
            n_parent[ch] = u;
            nch++;
            const int32_t nx = node_c[ch].x;
            ch = nx > ch ? nx : cu.x;   // next always advances
        }
        n_nchild[u] = nch;
    }
}

// FP64 moments bottom-up: the last child to finish folds its parent's
// children in octant order (mass, sum of m x), then COM = sum(m x) / M,
// l = L / 2^level, s = |COM - geometric centre|.
__global__ void __launch_bounds__(256)
k_moments(int64_t n, const uint64_t *__restrict__ key, const int32_t *__restrict__ cstart,
          const double *__restrict__ root, const int32_t *__restrict__ n_parent,
          const int32_t *__restrict__ n_nchild, const int32_t *__restrict__ n_level,
          const int32_t *__restrict__ n_first, int32_t *__restrict__ n_arrive,
          double *__restrict__ n_mass, double *__restrict__ n_mx, double *__restrict__ n_com,
          float4 *__restrict__ node_a, float4 *__restrict__ node_b, int4 *__restrict__ node_c)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    int32_t u = cstart[a + 1] + (int32_t)a;   // particle leaf
    __threadfence();
    int32_t p = n_parent[u];
    const double L = root[3];
    while (p >= 0) {
        const int old = atomicAdd(&n_arrive[p], 1);
        if (old != n_nchild[p] - 1) return;
        __threadfence();
        const int32_t end = node_c[p].x;
        double M = 0.0, mx[3] = {0.0, 0.0, 0.0};
        for (int32_t ch = p + 1; ch < end;) {
            M = __dadd_rn(M, __ldcg(&n_mass[ch]));
#pragma unroll
            for (int d = 0; d < 3; d++)
                mx[d] = __dadd_rn(mx[d], __ldcg(&n_mx[3 * (int64_t)ch + d]));
            const int32_t nx = node_c[ch].x;
            ch = nx > ch ? nx : end;
        }
        const int lev = n_level[p];
        const double lc = ldexp(L, -lev);
        const uint64_t kf = key[n_first[p]];
        const int sh = 3 * (NB_LEVELS - lev);
        const uint32_t cq[3] = {compact3(kf >> 2) >> (NB_LEVELS - lev),
                                compact3(kf >> 1) >> (NB_LEVELS - lev),
                                compact3(kf) >> (NB_LEVELS - lev)};
        (void)sh;
        double com[3], d2 = 0.0;
        float hi[3], lo[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double g = __dadd_rn(root[4 + d], __dmul_rn(__dadd_rn((double)cq[d], 0.5), lc));
            com[d] = M > 0.0 ? __ddiv_rn(mx[d], M) : g;
            const double dd = __dsub_rn(com[d], g);
            d2 = __dadd_rn(d2, __dmul_rn(dd, dd));
            hi[d] = __double2float_rn(com[d]);
            lo[d] = __double2float_rn(__dsub_rn(com[d], (double)hi[d]));
            n_mx[3 * (int64_t)p + d] = mx[d];
            n_com[3 * (int64_t)p + d] = com[d];
        }
        n_mass[p] = M;
        const float lf = __double2float_rn(lc);
        const float sf = __double2float_rn(__dsqrt_rn(d2));
        node_a[p] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(M));
        node_b[p] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        node_c[p] = make_int4(end, __float_as_int(lf), __float_as_int(sf), 0);
        __threadfence();
        u = p;
        p = n_parent[u];
    }
}

void nb_launch_build(nb_ctx *c, const double *pos, const float *mass, int64_t n)
{
    cudaStream_t s = c->stream;
    cudaMemsetAsync(c->cnt, 0, sizeof(long long) * CNT_PP_CUM, s);
    k_bbox<<<c->bbox_blocks, 256, 0, s>>>(pos, n, c->bbox_part, c->err);
    c->launches++;
    k_root<<<1, 32, 0, s>>>(c->bbox_part, c->bbox_blocks, c->root);
    c->launches++;
    k_keys<<<nb_grid(n, 256), 256, 0, s>>>(pos, n, c->root, c->keys, c->idx);
    c->launches++;
    nb_radix_sort(c, n);
    k_gather<<<nb_grid(n, 256), 256, 0, s>>>(pos, mass, n, c->idx, c->perm, c->p_x64,
                                             c->p_hi, c->p_lo);
    c->launches++;
    k_levels<<<nb_grid(n, 256), 256, 0, s>>>(c->keys, n, c->clev, c->ccount);
    c->launches++;
    nb_exclusive_scan(c, c->ccount, c->cstart, n, nullptr, &c->cnt[CNT_CELLS]);
    k_cells<<<nb_grid(n, 256), 256, 0, s>>>(
        c->keys, n, c->clev, c->cstart, c->p_hi, c->p_lo, c->p_x64, c->node_a, c->node_b,
        c->node_c, c->n_level, c->n_first, c->n_count, c->n_parent, c->n_nchild,
        c->n_arrive, c->n_mass, c->n_mx, c->n_com, c->cnt);
    c->launches++;
    k_parents<<<nb_grid(c->max_nodes, 256, c->num_sms * 16), 256, 0, s>>>(
        c->node_c, c->cnt, c->n_parent, c->n_nchild);
    c->launches++;
    k_moments<<<nb_grid(n, 256), 256, 0, s>>>(
        n, c->keys, c->cstart, c->root, c->n_parent, c->n_nchild, c->n_level, c->n_first,
        c->n_arrive, c->n_mass, c->n_mx, c->n_com, c->node_a, c->node_b, c->node_c);
    c->launches++;
}

// ------------------------------------------------------------ groups
__global__ void __launch_bounds__(256)
k_group_flags(const int32_t *__restrict__ n_count, const int32_t *__restrict__ n_parent,
              const long long *__restrict__ cnt, int n_crit, int32_t *__restrict__ flag)
{
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += gridDim.x * blockDim.x) {
        const int32_t p = n_parent[u];
        flag[u] = (n_count[u] <= n_crit) && (p < 0 || n_count[p] > n_crit);
    }
}

__global__ void __launch_bounds__(256)
k_group_scatter(const int32_t *__restrict__ gid, const int32_t *__restrict__ n_first,
                const int32_t *__restrict__ n_count, const long long *__restrict__ cnt,
                int32_t *__restrict__ gnode, int32_t *__restrict__ gfirst,
                int32_t *__restrict__ gcount)
{
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += gridDim.x * blockDim.x) {
        const int32_t g = gid[u];
        if (gid[u + 1] != g) {
            gnode[g] = u;
            gfirst[g] = n_first[u];
            gcount[g] = n_count[u];
        }
    }
}

// group box over the members' FP32 positions, its FP32 centre, FP32
// 1/theta, and the number of force work items of the group
__global__ void __launch_bounds__(256)
k_group_boxes(const int32_t *__restrict__ gfirst, const int32_t *__restrict__ gcount,
              const float4 *__restrict__ p_hi, const long long *__restrict__ cnt,
              float theta, const float *__restrict__ theta_g, float4 *__restrict__ gbox,
              int32_t *__restrict__ item_cnt)
{
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += gridDim.x * blockDim.x) {
        const int32_t f = gfirst[g], m = gcount[g];
        float4 p = p_hi[f];
        float lx = p.x, ly = p.y, lz = p.z, hx = p.x, hy = p.y, hz = p.z;
        for (int32_t k = 1; k < m; k++) {
            p = p_hi[f + k];
            lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
            hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y); hz = fmaxf(hz, p.z);
        }
        const float th = theta_g ? theta_g[g] : theta;
        const float invth = __double2float_rn(__ddiv_rn(1.0, (double)th));
        const float cx = __double2float_rn(__dmul_rn(0.5, __dadd_rn((double)lx, (double)hx)));
        const float cy = __double2float_rn(__dmul_rn(0.5, __dadd_rn((double)ly, (double)hy)));
        const float cz = __double2float_rn(__dmul_rn(0.5, __dadd_rn((double)lz, (double)hz)));
        gbox[3 * (int64_t)g] = make_float4(lx, ly, lz, 0.0f);
        gbox[3 * (int64_t)g + 1] = make_float4(hx, hy, hz, 0.0f);
        gbox[3 * (int64_t)g + 2] = make_float4(cx, cy, cz, invth);
        item_cnt[g] = (m + NB_IBLOCK - 1) / NB_IBLOCK;
    }
}

__global__ void __launch_bounds__(256)
k_items(const int32_t *__restrict__ item_off, const int32_t *__restrict__ gcount,
        const long long *__restrict__ cnt, int32_t *__restrict__ items)
{
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += gridDim.x * blockDim.x) {
        const int32_t o = item_off[g], m = gcount[g];
        for (int32_t i0 = 0, k = 0; i0 < m; i0 += NB_IBLOCK, k++) {
            items[2 * (int64_t)(o + k)] = g;
            items[2 * (int64_t)(o + k) + 1] = i0;
        }
    }
}

void nb_launch_groups(nb_ctx *c, float theta, int n_crit, const float *theta_g)
{
    cudaStream_t s = c->stream;
    const int gcap = c->num_sms * 16;
    k_group_flags<<<nb_grid(c->max_nodes, 256, gcap), 256, 0, s>>>(
        c->n_count, c->n_parent, c->cnt, n_crit, c->gflag);
    c->launches++;
    nb_exclusive_scan(c, c->gflag, c->gflag, c->max_nodes, &c->cnt[CNT_NODES],
                      &c->cnt[CNT_GROUPS]);
    k_group_scatter<<<nb_grid(c->max_nodes, 256, gcap), 256, 0, s>>>(
        c->gflag, c->n_first, c->n_count, c->cnt, c->gnode, c->gfirst, c->gcount);
    c->launches++;
    k_group_boxes<<<nb_grid(c->max_n, 256, gcap), 256, 0, s>>>(
        c->gfirst, c->gcount, c->p_hi, c->cnt, theta, theta_g, c->gbox, c->item_cnt);
    c->launches++;
    nb_exclusive_scan(c, c->item_cnt, c->item_cnt, c->max_n, &c->cnt[CNT_GROUPS],
                      &c->cnt[CNT_ITEMS]);
    k_items<<<nb_grid(c->max_n, 256, gcap), 256, 0, s>>>(c->item_cnt, c->gcount, c->cnt,
                                                          c->items);
    c->launches++;
}

// Root cube and Morton keys on buffers the caller supplies (no context):
// part holds 6 * nblk doubles, root 7; idx receives 0..n-1.
void nb_launch_keys_raw(const double *pos, int64_t n, double *part, int nblk, double *root,
                        uint64_t *keys, uint32_t *idx, unsigned *err, cudaStream_t s)
{
    k_bbox<<<nblk, 256, 0, s>>>(pos, n, part, err);
    k_root<<<1, 32, 0, s>>>(part, nblk, root);
    k_keys<<<nb_grid(n, 256), 256, 0, s>>>(pos, n, root, keys, idx);
}
