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
#include <climits>

#include "nb_internal.cuh"


// ------------------------------------------------------------ bbox, root
__device__ __forceinline__ void bbox_block(const double *__restrict__ pos, int64_t n,
                                           double *__restrict__ part, unsigned *__restrict__ err)
{
    // min / max on an order-preserving integer image of the FP64 bits (the
    // FP64 pipe is slow on this part): k = bits for x >= 0, and the low 63
    // bits flipped for x < 0, so signed order = numeric order (-0 sorts
    // below +0, which changes neither the centre nor the extent)
    const long long FLIP = 0x7fffffffffffffffll;
    long long lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; k++) { lo[k] = LLONG_MAX; hi[k] = LLONG_MIN; }
    bool bad = false;
    const long long *__restrict__ pb = reinterpret_cast<const long long *>(pos);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const long long bits = pb[3 * i + k];
            bad |= (bits & 0x7ff0000000000000ll) == 0x7ff0000000000000ll;   // inf or NaN
            const long long key = bits ^ ((bits >> 63) & FLIP);
            lo[k] = min(lo[k], key);
            hi[k] = max(hi[k], key);
        }
    }
    if (bad) atomicOr(err, NB_EF_NONFINITE);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            lo[k] = min(lo[k], __shfl_down_sync(0xffffffffu, lo[k], o));
            hi[k] = max(hi[k], __shfl_down_sync(0xffffffffu, hi[k], o));
        }
    __shared__ long long s[8][6];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; k++) { s[w][k] = lo[k]; s[w][3 + k] = hi[k]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        long long v = s[0][threadIdx.x];
        for (int ww = 1; ww < 8; ww++)
            v = threadIdx.x < 3 ? min(v, s[ww][threadIdx.x]) : max(v, s[ww][threadIdx.x]);
        // back to FP64 bits (the map is its own inverse); a block that saw
        // no particle keeps +-inf
        double x;
        if (v == LLONG_MAX) x = INFINITY;
        else if (v == LLONG_MIN) x = -INFINITY;
        else x = __longlong_as_double(v ^ ((v >> 63) & FLIP));
        part[blockIdx.x * 6 + threadIdx.x] = x;
    }
}

__global__ void __launch_bounds__(256)
k_bbox(const double *__restrict__ pos, int64_t n, double *__restrict__ part,
       unsigned *__restrict__ err)
{
    bbox_block(pos, n, part, err);
}

// Root cube: centre = bbox centre, side = max extent * (1 + 2^-20), 1 when
// every particle coincides; corner = centre - side/2; grid scale 2^21 / side.
// (one block of 256 threads; the partials are read through L2, since in
// k_bbox_root other blocks of the same launch wrote them)
__device__ __forceinline__ void root_block(const double *part, int nblk, double *__restrict__ root)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int k = 0; k < 3; k++) {
            lo[k] = fmin(lo[k], __ldcg(&part[6 * b + k]));
            hi[k] = fmax(hi[k], __ldcg(&part[6 * b + 3 + k]));
        }
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
    if (threadIdx.x != 0) return;
    for (int ww = 1; ww < (int)(blockDim.x >> 5); ww++)
        for (int k = 0; k < 3; k++) {
            s[0][k] = fmin(s[0][k], s[ww][k]);
            s[0][3 + k] = fmax(s[0][3 + k], s[ww][3 + k]);
        }
    double ext = 0.0;
    for (int k = 0; k < 3; k++) {
        root[k] = __dmul_rn(0.5, __dadd_rn(s[0][k], s[0][3 + k]));
        const double e = __dsub_rn(s[0][3 + k], s[0][k]);
        if (e > ext) ext = e;
    }
    double L = __dmul_rn(ext, 1.0 + 0x1p-20);
    if (!(L > 0.0)) L = 1.0;
    root[3] = L;
    for (int k = 0; k < 3; k++) root[4 + k] = __dsub_rn(root[k], __dmul_rn(0.5, L));
    root[7] = __ddiv_rn(2097152.0, L);
}

__global__ void __launch_bounds__(256)
k_root(const double *__restrict__ part, int nblk, double *__restrict__ root)
{
    root_block(part, nblk, root);
}

// k_bbox and k_root in one launch: every block writes its partial box, and
// the last one to finish (a fenced counter, zeroed with the build's counters)
// reduces them all into the root cube.  The same min, max and root
// arithmetic as the two launches.
__global__ void __launch_bounds__(256)
k_bbox_root(const double *__restrict__ pos, int64_t n, double *part, unsigned *__restrict__ err,
            long long *__restrict__ cnt, double *__restrict__ root)
{
    __shared__ bool last;
    bbox_block(pos, n, part, err);
    __threadfence();   // this block's partial before its arrival
    __syncthreads();
    if (threadIdx.x == 0)
        last = atomicAdd((unsigned long long *)&cnt[CNT_BBOX_DONE], 1ull) ==
               (unsigned long long)gridDim.x - 1ull;
    __syncthreads();
    if (!last) return;
    __threadfence();   // every partial before the reduction reads them
    root_block(part, gridDim.x, root);
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

__device__ __forceinline__ uint32_t grid_coord(double x, double corner, double scale)
{
    // v = fl(fl(x - corner) * scale); its floor, clamped to the grid
    // [0, 2^21 - 1], read off v's bits with integer instructions (GB300's
    // FP64 pipe is its scarce unit): below 1 (negative numbers and NaNs with
    // the sign bit included) gives 0, 2^21 or more gives the top cell, and in
    // between the integer part is the significand shifted by the exponent.
    // A positive NaN gives 0, as a round-down conversion would.
    const double v = __dmul_rn(__dsub_rn(x, corner), scale);
    const long long b = __double_as_longlong(v);
    if (b < 0x3ff0000000000000ll) return 0u;
    if (b > 0x7ff0000000000000ll) return 0u;   // NaN
    const int e = (int)(b >> 52) - 1023;        // v in [2^e, 2^(e+1))
    if (e >= 21) return 2097151u;
    const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffull) | (1ull << 52);
    return (uint32_t)(m >> (52 - e));
}

// Peano-Hilbert index of a grid point, the order the paper names as better
// than Morton order for locality (Sec. "Test and Optimization"), by
// Skilling's transpose method (J. Skilling 2004, "Programming the Hilbert
// curve", AIP Conf. Proc. 707).  Going down the bit planes, the lower bits
// of every axis are mapped into the frame of the sub-cube the point lies in
// (a reflection of axis 0 when the axis bit is set, else an exchange of the
// lower bits of axis 0 and that axis); the three words are then Gray-coded
// and the result interleaved from the top like a Morton key (x, y, z).
// Every step is a select on integers, so lanes do not diverge.  Aligned
// sub-cubes are contiguous key ranges, so cells are again the key prefixes
// shared by >= 2 particles, and children come in the curve's order.
__device__ __forceinline__ uint64_t hilbert_key(uint32_t x0, uint32_t x1, uint32_t x2)
{
    uint32_t X[3] = {x0, x1, x2};
#pragma unroll
    for (int b = NB_LEVELS - 1; b >= 1; b--) {
        const uint32_t Q = 1u << b, P = Q - 1u;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const bool set = (X[i] & Q) != 0u;
            const uint32_t t = set ? 0u : ((X[0] ^ X[i]) & P);
            X[0] ^= set ? P : t;
            if (i) X[i] ^= t;
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    // flip: the XOR of (Q - 1) over the set bits Q > 1 of X[2], i.e. bit k is
    // the parity of X[2]'s bits above k
    uint32_t flip = 0u;
#pragma unroll
    for (int b = NB_LEVELS - 1; b >= 1; b--)
        flip ^= ((X[2] >> b) & 1u) ? ((1u << b) - 1u) : 0u;
#pragma unroll
    for (int i = 0; i < 3; i++) X[i] ^= flip;
    return (spread3(X[0]) << 2) | (spread3(X[1]) << 1) | spread3(X[2]);
}

// the grid point of a Peano-Hilbert key (the inverse of hilbert_key): undo
// the Gray code, then re-apply the frame changes from the lowest bit plane up
__device__ __forceinline__ void hilbert_point(uint64_t key, uint32_t q[3])
{
    uint32_t X[3] = {compact3(key >> 2), compact3(key >> 1), compact3(key)};
    const uint32_t t = X[2] >> 1;
    X[2] ^= X[1];
    X[1] ^= X[0];
    X[0] ^= t;
#pragma unroll
    for (int b = 1; b < NB_LEVELS; b++) {
        const uint32_t Q = 1u << b, P = Q - 1u;
#pragma unroll
        for (int i = 2; i >= 0; i--) {
            const bool set = (X[i] & Q) != 0u;
            const uint32_t u = set ? 0u : ((X[0] ^ X[i]) & P);
            X[0] ^= set ? P : u;
            if (i) X[i] ^= u;
        }
    }
    q[0] = X[0];
    q[1] = X[1];
    q[2] = X[2];
}

__global__ void __launch_bounds__(256)
k_keys(const double *__restrict__ pos, int64_t n, const double *__restrict__ roots,
       const int32_t *__restrict__ sys_of, uint64_t *__restrict__ key, uint32_t *__restrict__ idx,
       int hilbert)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *root = roots + (sys_of ? 8 * (int64_t)sys_of[i] : 0);
    const double sc = root[7];
    const uint32_t qx = grid_coord(pos[3 * i], root[4], sc);
    const uint32_t qy = grid_coord(pos[3 * i + 1], root[5], sc);
    const uint32_t qz = grid_coord(pos[3 * i + 2], root[6], sc);
    key[i] = hilbert ? hilbert_key(qx, qy, qz)
                     : (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    idx[i] = (uint32_t)i;
}

// sorted slot s: gather the caller's particle idx[s]; split FP64 positions
// into an FP32 pair (hi = nearest float, lo = float of the remainder)
__global__ void __launch_bounds__(256)
k_gather(const double *__restrict__ pos, const float *__restrict__ mass, int64_t n,
         const uint32_t *__restrict__ idx, int32_t *__restrict__ perm,
         double *__restrict__ x64, float4 *__restrict__ p_hi, float4 *__restrict__ p_lo,
         long long *__restrict__ cnt, unsigned *__restrict__ err)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = idx[s];
    if (!nb_in(i < n, cnt, err, SITE_GATHER, i)) return;
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

// (neighbours in different systems share no cell)
__global__ void __launch_bounds__(256)
k_levels(const uint64_t *__restrict__ key, int64_t n, const int32_t *__restrict__ sys,
         int8_t *__restrict__ clev, int32_t *__restrict__ ccount)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int ca = a + 1 < n && (!sys || sys[a] == sys[a + 1]) ? common_levels(key[a], key[a + 1]) : -1;
    const int cp = a > 0 && (!sys || sys[a - 1] == sys[a]) ? common_levels(key[a - 1], key[a]) : -1;
    clev[a] = (int8_t)ca;
    ccount[a] = ca > cp ? ca - cp : 0;
}

// records of particle a's leaf and of the cells whose first particle is a;
// returns the deepest such cell's level (-1 if none)
__device__ __forceinline__ int cell_records(
    int64_t a, int64_t n, const int8_t *__restrict__ clev, const int32_t *__restrict__ cstart,
    int4 *__restrict__ node_c, int32_t *__restrict__ n_level, int32_t *__restrict__ n_first,
    int32_t *__restrict__ n_count, int32_t *__restrict__ n_parent, int32_t *__restrict__ n_nchild,
    int8_t *__restrict__ n_depth, long long *__restrict__ cnt, unsigned *__restrict__ err)
{
    const int32_t C = cstart[n];
    const int32_t total = C + (int32_t)n;
    if (a == 0) cnt[CNT_NODES] = total;
    const int ca = clev[a];
    const int cp = a > 0 ? clev[a - 1] : -1;
    const int k = ca > cp ? ca - cp : 0;
    const int32_t base = cstart[a] + (int32_t)a;
    const int32_t leaf = base + k;
    if (!nb_in(base >= 0 && leaf < total, cnt, err, SITE_CELLS, leaf)) return -1;

    // particle leaf: one below the deepest cell that holds it
    node_c[leaf] = make_int4(leaf + 1, 0, 0, 1);
    n_level[leaf] = -1;
    n_first[leaf] = (int32_t)a;
    n_count[leaf] = 1;
    n_nchild[leaf] = 0;
    n_depth[leaf] = (int8_t)((ca > cp ? ca : cp) + 1);
    if (k > 0) n_parent[leaf] = leaf - 1;
    else if (ca < 0 && cp < 0) n_parent[leaf] = -1;   // a one-particle system

    // cells starting at a (their ends: k_cell_ends)
    for (int lev = ca; lev > cp; lev--) {
        const int32_t id = base + (lev - cp - 1);
        n_level[id] = lev;
        n_first[id] = (int32_t)a;
        n_depth[id] = (int8_t)lev;
        if (lev > cp + 1) n_parent[id] = id - 1;
        else if (cp < 0) n_parent[id] = -1;   // a system's root
    }
    return k > 0 ? ca : -1;
}

__global__ void __launch_bounds__(256)
k_cells(const uint64_t *__restrict__ key, int64_t n, const int8_t *__restrict__ clev,
        const int32_t *__restrict__ cstart, int4 *__restrict__ node_c,
        int32_t *__restrict__ n_level, int32_t *__restrict__ n_first,
        int32_t *__restrict__ n_count, int32_t *__restrict__ n_parent,
        int32_t *__restrict__ n_nchild, int8_t *__restrict__ n_depth,
        long long *__restrict__ cnt, const int32_t *__restrict__ sys,
        const int64_t *__restrict__ sys_off, unsigned *__restrict__ err)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int deepest = -1;
    if (a < n) deepest = cell_records(a, n, clev, cstart, node_c, n_level, n_first, n_count,
                                      n_parent, n_nchild, n_depth, cnt, err);
    // one atomic per warp for the deepest level (a single counter)
    deepest = __reduce_max_sync(0xffffffffu, deepest);
    if ((threadIdx.x & 31) == 0 && deepest >= 0) atomicMax(&cnt[CNT_MAXLEVEL], (long long)deepest);
}


// One thread per cell: the last particle b of the run of keys sharing the
// cell's prefix (gallop from the first particle, then bisection, never past
// the particle's system), its particle count and its preorder next,
// S[b+1] + b + 1.  Cells are independent, so long runs near the root are
// searched side by side instead of one after another.
__global__ void __launch_bounds__(256)
k_cell_ends(const uint64_t *__restrict__ key, int64_t n, const int32_t *__restrict__ cstart,
            const int32_t *__restrict__ n_level, const int32_t *__restrict__ n_first,
            int4 *__restrict__ node_c, int32_t *__restrict__ n_count,
            long long *__restrict__ cnt, const int32_t *__restrict__ sys,
            const int64_t *__restrict__ sys_off, unsigned *__restrict__ err)
{
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += gridDim.x * blockDim.x) {
        const int lev = n_level[id];
        if (lev < 0) continue;                     // a particle leaf
        const int64_t a = n_first[id];
        if (!nb_in(a >= 0 && a < n && lev <= NB_LEVELS, cnt, err, SITE_CELLS, id)) continue;
        const int64_t nend = sys ? sys_off[sys[a] + 1] : n;
        const int shift = 63 - 3 * lev;
        const uint64_t P = key[a] >> shift;
        int64_t lo = a, step = 1, hi = a + 1;
        while (hi < nend && (key[hi] >> shift) == P) {
            lo = hi;
            step <<= 1;
            hi = lo + step;
        }
        if (hi > nend) hi = nend;
        while (hi - lo > 1) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if ((key[mid] >> shift) == P) lo = mid; else hi = mid;
        }
        node_c[id] = make_int4(cstart[lo + 1] + (int32_t)lo + 1, 0, 0, 0);
        n_count[id] = (int32_t)(lo - a + 1);
    }
}

// every cell writes itself as parent of its children (child = id + 1, then
// next of each child until the cell's own next)
__global__ void __launch_bounds__(256)
k_parents(const int4 *__restrict__ node_c, long long *__restrict__ cnt,
          int32_t *__restrict__ n_parent, int32_t *__restrict__ n_nchild,
          int32_t *__restrict__ arrive, int32_t *__restrict__ lcount, unsigned *__restrict__ err)
{
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += gridDim.x * blockDim.x) {
        arrive[u] = 0;     // counters of the bottom-up moments (any index < total)
        lcount[u] = 0;
        const int4 cu = node_c[u];
        if (cu.w) continue;
        int32_t ch = u + 1, nch = 0;
        if (!nb_in(cu.x <= total, cnt, err, SITE_PARENTS, cu.x)) continue;
        while (ch < cu.x) {
            n_parent[ch] = u;
            nch++;
            const int32_t nx = node_c[ch].x;
            ch = nx > ch ? nx : cu.x;   // next always advances
        }
        n_nchild[u] = nch;
    }
}

// ------------------------------------------------------------ level order
// Stable counting sort of the preorder node ids by depth: per-tile depth
// histograms, one scan of the depth-major table, then a stable scatter with
// warp match/rank (the same scheme as the radix sort's scatter).
#define DS_T 256
#define DS_I (NB_DS_TILE / DS_T)
#define DS_TILE NB_DS_TILE

__global__ void __launch_bounds__(DS_T)
k_depth_hist(const int8_t *__restrict__ depth, const long long *__restrict__ cnt,
             uint32_t *__restrict__ hist, int ntiles)
{
    __shared__ uint32_t h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t total = cnt[CNT_NODES];
    const int64_t base = (int64_t)blockIdx.x * DS_TILE;
    for (int k = 0; k < DS_I; k++) {
        const int64_t i = base + k * DS_T + threadIdx.x;
        if (i < total) atomicAdd(&h[depth[i]], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NB_DEPTHS) hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter by depth, staged like the radix sort's: nodes are ranked
// per warp with a ballot match, placed in the tile's depth order in shared
// memory, then written out as contiguous runs.  Tiles past the node count
// return at once (the grid covers the node capacity).
__global__ void __launch_bounds__(DS_T)
k_depth_scatter(const int8_t *__restrict__ depth, long long *__restrict__ cnt,
                const uint32_t *__restrict__ offs, int ntiles, int32_t *__restrict__ bfs2pid,
                int32_t *__restrict__ pid2bfs, unsigned *__restrict__ err)
{
    __shared__ uint32_t whist[DS_T / NB_WARP][32];
    __shared__ uint32_t boff[32];
    __shared__ uint32_t lstart[32];
    __shared__ int32_t sid[DS_TILE];
    __shared__ int8_t sdep[DS_TILE];
    const int64_t total = cnt[CNT_NODES];
    const int64_t tile0 = (int64_t)blockIdx.x * DS_TILE;
    if (tile0 >= total) return;
    const int64_t rem = total - tile0;
    const int tn = rem < DS_TILE ? (int)rem : DS_TILE;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int i = t; i < (DS_T / NB_WARP) * 32; i += DS_T) (&whist[0][0])[i] = 0u;
    if (t < 32) boff[t] = t < NB_DEPTHS ? offs[(int64_t)t * ntiles + blockIdx.x] : 0u;
    __syncthreads();
    const int wbase = w * (DS_TILE / (DS_T / NB_WARP));
    const unsigned lt = (1u << lane) - 1u;
    uint32_t rnk[DS_I];
    int dep[DS_I];
#pragma unroll
    for (int r = 0; r < DS_I; r++) {
        const int e = wbase + r * NB_WARP + lane;
        dep[r] = e < tn ? (int)depth[tile0 + e] : 0;
    }
#pragma unroll
    for (int r = 0; r < DS_I; r++) {
        const bool ok = wbase + r * NB_WARP + lane < tn && dep[r] >= 0 && dep[r] < NB_DEPTHS;
        const int d = ok ? dep[r] : 32 + lane;
        const unsigned peers = nb_match_bits<5>((unsigned)d, ok);
        const unsigned before = __popc(peers & lt);
        const uint32_t pre = ok ? whist[w][d] : 0u;
        __syncwarp();
        if (ok && before == 0) whist[w][d] = pre + __popc(peers);
        __syncwarp();
        rnk[r] = pre + before;
    }
    __syncthreads();
    if (t < 32) {
        uint32_t run = 0;
        for (int ww = 0; ww < DS_T / NB_WARP; ww++) {
            const uint32_t v = whist[ww][t];
            whist[ww][t] = run;
            run += v;
        }
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        lstart[t] = x - run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < DS_I; r++) {
        const int e = wbase + r * NB_WARP + lane;
        if (e >= tn) continue;
        const int d = dep[r];
        if (!nb_in(d >= 0 && d < NB_DEPTHS, cnt, err, SITE_DEPTH, tile0 + e)) continue;
        const uint32_t lp = lstart[d] + whist[w][d] + rnk[r];
        if (!nb_in(lp < (uint32_t)tn, cnt, err, SITE_DEPTH, lp)) continue;
        sid[lp] = (int32_t)(tile0 + e);
        sdep[lp] = (int8_t)d;
        pid2bfs[tile0 + e] = (int32_t)(boff[d] + whist[w][d] + rnk[r]);
    }
    __syncthreads();
    for (int e = t; e < tn; e += DS_T) {
        const int d = sdep[e];
        if (d < 0 || d >= NB_DEPTHS) continue;   // a slot left by a reported bad depth
        const uint32_t pos = boff[d] + (uint32_t)e - lstart[d];
        if (!nb_in(pos < total, cnt, err, SITE_DEPTH, pos)) continue;
        bfs2pid[pos] = sid[e];
    }
}

// level_start[d] = first level-order index of depth d (d = 0 .. NB_DEPTHS)
__global__ void k_level_start(const uint32_t *__restrict__ hist, int ntiles,
                              int32_t *__restrict__ level_start)
{
    const int d = threadIdx.x;
    if (d <= NB_DEPTHS) level_start[d] = (int32_t)hist[(int64_t)d * ntiles];
}

// level-order records: particle leaves get their position and FP64 moments,
// cells their topology and geometry -- side l = L / 2^level (c.x) and
// geometric centre (held in b_com until the moments replace it); every node
// gets its parent's level-order index and a zero arrival count
__device__ __forceinline__ double pow2_neg(int k)   // 2^-k, 0 <= k <= 1022
{
    return __longlong_as_double((long long)(1023 - k) << 52);
}

__global__ void __launch_bounds__(256)
k_bfs_records(const int32_t *__restrict__ bfs2pid, const int32_t *__restrict__ pid2bfs,
              const int4 *__restrict__ node_c, const int32_t *__restrict__ n_first,
              const int32_t *__restrict__ n_nchild, const int32_t *__restrict__ n_parent,
              const int8_t *__restrict__ n_depth, const uint64_t *__restrict__ key,
              const double *__restrict__ roots, const int32_t *__restrict__ sys,
              const float4 *__restrict__ p_hi, const float4 *__restrict__ p_lo,
              const double *__restrict__ x64, long long *__restrict__ cnt,
              nb_wrec *__restrict__ wrec, double *__restrict__ b_mass, double *__restrict__ b_mx,
              double *__restrict__ b_com, int32_t *__restrict__ b_up,
              int32_t *__restrict__ lcount, int16_t *__restrict__ cbkt,
              int32_t *__restrict__ cbkt_cnt, int64_t n, int hilbert, double *__restrict__ b_q,
              unsigned *__restrict__ err)
{
    __shared__ int32_t hb[NB_CBKT];   // cells per moments bucket in this block
    for (int k = threadIdx.x; k < NB_CBKT; k += blockDim.x) hb[k] = 0;
    __syncthreads();
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < total;
         b += gridDim.x * blockDim.x) {
        b_up[b] = -1;
        cbkt[b] = -1;
        const int32_t u = bfs2pid[b];
        if (!nb_in(u >= 0 && u < total, cnt, err, SITE_RECORDS, u)) continue;
        const int4 c = node_c[u];
        if (!nb_in(c.w || u + 1 < total, cnt, err, SITE_RECORDS, u)) continue;
        const int32_t up = n_parent[u];
        int32_t pb = -1;
        if (up >= 0) {
            if (!nb_in(up < total, cnt, err, SITE_RECORDS, u)) continue;
            pb = pid2bfs[up];
            if (!nb_in(pb >= 0 && pb < b, cnt, err, SITE_RECORDS, up)) continue;
            b_up[b] = pb;
        }
        const int32_t slot = n_first[u];
        if (!nb_in(slot >= 0 && slot < n, cnt, err, SITE_RECORDS, slot)) continue;
        if (c.w) {
            const float4 h = p_hi[slot];
            nb_wrec_put_lo(&wrec[b], h, p_lo[slot]);
            nb_wrec_put_hi(&wrec[b], make_int4(u, c.x, -1, 0), 0.0f, 0.0f);
            if (pb >= 0) atomicAdd(&lcount[pb], 1);   // a leaf child of pb (result unused)
            const double m = (double)h.w;
            b_mass[b] = m;
            if (b_q)   // a particle has no quadrupole moment
#pragma unroll
                for (int k = 0; k < 6; k++) b_q[6 * (int64_t)b + k] = 0.0;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const double x = x64[3 * (int64_t)slot + d];
                b_com[3 * (int64_t)b + d] = x;
                b_mx[3 * (int64_t)b + d] = __dmul_rn(m, x);
            }
        } else {
            const int4 wb = make_int4(u, c.x, pid2bfs[u + 1], n_nchild[u]);
            const int depth = n_depth[u];
            if (!nb_in(depth >= 0 && depth <= NB_LEVELS, cnt, err, SITE_RECORDS, u)) continue;
            // a cell has 1..8 children, except a level-21 cell of coincident
            // particles, which keeps all of them
            if (!nb_in(wb.w >= 1 && (wb.w <= 8 || depth == NB_LEVELS), cnt, err, SITE_RECORDS, u))
                continue;
            // moments bucket: deepest level first, then by number of children
            // (more than 8 share the bucket of 8)
            const int k = (NB_DEPTHS - 1 - depth) * 8 + (wb.w < 8 ? wb.w : 8) - 1;
            cbkt[b] = (int16_t)k;
            atomicAdd(&hb[k], 1);
            const double *root = roots + (sys ? 8 * (int64_t)sys[slot] : 0);
            // geometric centre corner + (q + 1/2) l, written as (2q + 1)(l / 2): the
            // same real product (scaling by 2^-k is exact for a normal l), rounded
            // once either way, with one FP64 add fewer per axis
            const double lc = __dmul_rn(root[3], pow2_neg(depth));
            const double lh = __dmul_rn(root[3], pow2_neg(depth + 1));
            // the cell's integer corner: its first member's grid point shifted
            // down to the cell's level (read off the Morton key's bits, or
            // recovered from the Peano-Hilbert key by the inverse transform)
            const uint64_t kf = key[slot];
            uint32_t cq[3];
            if (hilbert) {
                hilbert_point(kf, cq);
            } else {
                cq[0] = compact3(kf >> 2);
                cq[1] = compact3(kf >> 1);
                cq[2] = compact3(kf);
            }
#pragma unroll
            for (int d = 0; d < 3; d++) cq[d] >>= NB_LEVELS - depth;
#pragma unroll
            for (int d = 0; d < 3; d++)
                b_com[3 * (int64_t)b + d] =
                    __dadd_rn(root[4 + d], __dmul_rn((double)(2u * cq[d] + 1u), lh));
            nb_wrec_put_hi(&wrec[b], wb, __double2float_rn(lc), 0.0f);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NB_CBKT; k += blockDim.x)
        if (hb[k]) atomicAdd(&cbkt_cnt[k], hb[k]);
}

// FP64 moments, bottom-up in one launch.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, and an FP64 warp
// instruction costs the pipe the same whether 3 or 32 lanes are active, so
// the work is arranged for full warps of equal work.  k_bfs_records put each
// cell in a bucket (depth, deepest first; number of children); k_cell_list
// lists the cells bucket by bucket, every bucket padded to whole warps.  A
// warp of k_moments takes the next 32 entries from a global queue, so every
// lane folds the same number of children, and no warp mixes two depths.
//
// A cell is ready once its cell children have arrived (particle-leaf
// children, counted by k_bfs_records in lcount, are final from the start).
// The warp waits for its cells with a bounded poll: the children are
// deeper, so their chunks came earlier from the queue and are held by warps
// that are running, and the wait ends; if it does not within the limit, the
// warp reports SITE_MOMENTS_WAIT and every waiting warp stops.  The fold
// adds M and sum(m x) over the children in octant order; the sums are made
// visible (fence) before the arrival at the parent; then COM = sum(m x) / M,
// s = |COM - geometric centre| and the FP32 hi/lo split of the record.
#define CL_I 16
#define CL_TILE (256 * CL_I)

// One tile of CL_TILE level-order nodes per block.  Ranks inside a bucket
// come from shared-memory counters and each block reserves its range of a
// bucket with one global atomic, so no counter is hit by every warp; the
// order of cells inside a bucket is free (each cell's moments are its own).
__global__ void __launch_bounds__(256)
k_cell_list(const int16_t *__restrict__ cbkt, int32_t *__restrict__ cbkt_cnt,
            long long *__restrict__ cnt, int32_t *__restrict__ clist, int64_t clist_len,
            unsigned *__restrict__ err)
{
    static_assert(NB_CBKT <= 256, "one bucket per thread");
    __shared__ int32_t start[NB_CBKT + 1];
    __shared__ int32_t local[NB_CBKT];
    const int t = threadIdx.x;
    {
        const int32_t sz = t < NB_CBKT ? cbkt_cnt[t] : 0;
        const int32_t padded = (sz + NB_WARP - 1) / NB_WARP * NB_WARP;
        int32_t all;
        const int32_t st = nb_block_scan256(padded, &all);
        if (t < NB_CBKT) {
            start[t] = st;
            local[t] = 0;
        }
        if (t == 0) start[NB_CBKT] = all;
        if (blockIdx.x == 0 && t == 0) cnt[CNT_MOM_CHUNKS] = all / NB_WARP;
        // block 0 marks each bucket's padding (at most 31 slots): no cell
        if (blockIdx.x == 0 && t < NB_CBKT)
            for (int32_t i = st + sz; i < st + padded; i++)
                if (i < clist_len) clist[i] = -1;
        __syncthreads();
    }
    const int32_t total = (int32_t)cnt[CNT_NODES];
    const int64_t tile0 = (int64_t)blockIdx.x * CL_TILE;
    if (tile0 >= total) return;
    int k[CL_I], rank[CL_I];
#pragma unroll
    for (int r = 0; r < CL_I; r++) {
        const int64_t b = tile0 + r * 256 + t;
        k[r] = b < total ? (int)cbkt[b] : -1;
    }
#pragma unroll
    for (int r = 0; r < CL_I; r++) {
        if (k[r] >= NB_CBKT) {
            nb_bad(cnt, err, SITE_MOMENTS, tile0 + r * 256 + t);
            k[r] = -1;
        }
        rank[r] = k[r] >= 0 ? atomicAdd(&local[k[r]], 1) : 0;
    }
    __syncthreads();
    if (t < NB_CBKT && local[t] > 0) local[t] = atomicAdd(&cbkt_cnt[NB_CBKT + t], local[t]);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < CL_I; r++) {
        if (k[r] < 0) continue;
        const int32_t pos = start[k[r]] + local[k[r]] + rank[r];
        if (!nb_in(pos >= 0 && pos < start[k[r] + 1] && pos < clist_len, cnt, err, SITE_MOMENTS,
                   pos))
            continue;
        clist[pos] = (int32_t)(tile0 + r * 256 + t);
    }
}

__device__ __forceinline__ int32_t ld_acquire(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait of a whole warp until each waiting lane sees arrive[b] >=
// need (lanes with `ready` set do not wait).  A lane's result is false if
// it gave up: after `limit` polls (reported as SITE_MOMENTS_WAIT), or
// because another warp had reported a failure.
__device__ __forceinline__ bool wait_arrivals(const int32_t *arrive, int32_t b, int32_t need,
                                              bool ready, unsigned limit, long long *cnt,
                                              unsigned *err)
{
    for (unsigned spins = 0;; spins++) {
        if (!ready) ready = ld_acquire(&arrive[b]) >= need;
        if (__all_sync(0xffffffffu, ready)) return true;
        bool stop = spins >= limit;
        if (!stop && (spins & 63u) == 63u)
            stop = (*(volatile unsigned *)err & NB_EF_BOUNDS) != 0u;
        if (__any_sync(0xffffffffu, stop)) {
            if (!ready && spins >= limit) nb_bad(cnt, err, SITE_MOMENTS_WAIT, b);
            return ready;
        }
        __nanosleep(64);
    }
}

// one warp: lane 0 waits for a count that nothing raises (a test of the
// bounded wait; the status is read by the host)
__global__ void k_wait_probe(const int32_t *flag, unsigned limit, long long *cnt, unsigned *err)
{
    wait_arrivals(flag, 0, 1, threadIdx.x != 0, limit, cnt, err);
}

void nb_launch_wait_probe(nb_ctx *c, unsigned limit)
{
    cudaMemsetAsync(c->cbkt_cnt, 0, sizeof(int32_t), c->stream);
    k_wait_probe<<<1, NB_WARP, 0, c->stream>>>(c->cbkt_cnt, limit, c->cnt, c->err);
    nb_launched(c, "k_wait_probe");
}

// COM = sum(m x) / M, correctly rounded: one correctly rounded reciprocal
// y = RN(1/M) shared by the three quotients, then Markstein's correction
// q = RN(q0 + RN(a - M q0) y), q0 = RN(a y), which gives RN(a / M)
// (Markstein 1990, IBM J. Res. Dev. 34(1)); s = |COM - geometric centre|
// and the FP32 split of the record.  d2 starts as the first square: 0 + x = x
// exactly for x >= 0.
__device__ __forceinline__ void cell_com(int32_t b, int4 wb, double M, const double mx[3],
                                         double *__restrict__ b_com, nb_wrec *__restrict__ wrec,
                                         double com[3])
{
    const double y = M > 0.0 ? __drcp_rn(M) : 0.0;
    double d2 = 0.0;
    float hi[3], lo[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double g = b_com[3 * (int64_t)b + d];   // geometric centre
        double cm = g;
        if (M > 0.0) {
            const double q0 = __dmul_rn(mx[d], y);
            const double r = __fma_rn(-q0, M, mx[d]);
            cm = __fma_rn(r, y, q0);
        }
        const double dd = __dsub_rn(cm, g);
        d2 = d == 0 ? __dmul_rn(dd, dd) : __dadd_rn(d2, __dmul_rn(dd, dd));
        hi[d] = __double2float_rn(cm);
        lo[d] = __double2float_rn(__dsub_rn(cm, (double)hi[d]));
        b_com[3 * (int64_t)b + d] = cm;
        com[d] = cm;
    }
    const float lcf = wrec[b].c.x;
    nb_wrec_put_lo(&wrec[b], make_float4(hi[0], hi[1], hi[2], __double2float_rn(M)),
                   make_float4(lo[0], lo[1], lo[2], 0.0f));
    nb_wrec_put_hi(&wrec[b], wb, lcf, __double2float_rn(__dsqrt_rn(d2)));
}

// Quadrupole of a cell about its centre of mass from its children's, by the
// parallel-axis theorem: Q = sum_c [Q_c + m_c (3 d d^T - |d|^2 I)], d =
// COM_c - COM, folded in octant order in FP64 (a particle child has Q_c = 0
// and COM_c = its position).  The same moment as the sum over the cell's
// members of m (3 d d^T - |d|^2 I) about the COM, reached by another route.
__device__ __forceinline__ void cell_quad(int32_t b, int4 wb, const double com[3],
                                          const double *b_mass, const double *b_com, double *b_q)
{
    double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int32_t k = 0; k < wb.w; k++) {
        const int64_t c = (int64_t)wb.z + k;
        const double m = __ldcg(&b_mass[c]);
        double d[3];
#pragma unroll
        for (int a = 0; a < 3; a++) d[a] = __ldcg(&b_com[3 * c + a]) - com[a];
        const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        q[0] += __ldcg(&b_q[6 * c + 0]) + m * (3.0 * d[0] * d[0] - d2);
        q[1] += __ldcg(&b_q[6 * c + 1]) + m * (3.0 * d[1] * d[1] - d2);
        q[2] += __ldcg(&b_q[6 * c + 2]) + m * (3.0 * d[2] * d[2] - d2);
        q[3] += __ldcg(&b_q[6 * c + 3]) + m * 3.0 * d[0] * d[1];
        q[4] += __ldcg(&b_q[6 * c + 4]) + m * 3.0 * d[0] * d[2];
        q[5] += __ldcg(&b_q[6 * c + 5]) + m * 3.0 * d[1] * d[2];
    }
#pragma unroll
    for (int k = 0; k < 6; k++) b_q[6 * (int64_t)b + k] = q[k];
}

// QUAD: the cell's centre of mass and quadrupole are finished before it
// arrives at its parent (the parent's quadrupole needs both); otherwise the
// arrival comes first and the centre of mass after it.
template <bool QUAD>
__global__ void __launch_bounds__(256)
k_moments(const int32_t *__restrict__ clist, int64_t clist_len, nb_wrec *__restrict__ wrec,
          const int32_t *__restrict__ b_up, const int32_t *__restrict__ lcount, double *b_mass,
          double *b_mx, double *b_com, double *b_q, int32_t *arrive,
          long long *__restrict__ cnt, unsigned *err)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int32_t total = (int32_t)cnt[CNT_NODES];
    long long nchunks = cnt[CNT_MOM_CHUNKS];
    if (nchunks > clist_len / NB_WARP) nchunks = clist_len / NB_WARP;
    for (;;) {
        long long ch = 0;
        if (lane == 0) ch = nb_atomic_add(&cnt[CNT_MOM_Q], 1LL);
        ch = __shfl_sync(FULL, ch, 0);
        if (ch >= nchunks) break;
        int32_t b = clist[ch * NB_WARP + lane];
        int4 wb = make_int4(0, 0, -1, 0);
        int32_t need = 0;
        if (b >= 0) {
            if (nb_in(b < total, cnt, err, SITE_MOMENTS, b)) {
                wb = wrec[b].b;
                if (nb_in(wb.z > b && wb.w >= 1 && (int64_t)wb.z + wb.w <= total, cnt,
                          err, SITE_MOMENTS, b))
                    need = wb.w - lcount[b];   // cell children still to arrive
                else
                    b = -1;
            } else {
                b = -1;
            }
        }
        // bounded wait for the lanes' cell children
        if (!wait_arrivals(arrive, b, need, b < 0 || need <= 0, NB_SPIN_LIMIT, cnt, err)) b = -1;
        // fold the children in octant order
        const int32_t nch = b >= 0 ? wb.w : 0;
        double M = 0.0, mx[3] = {0.0, 0.0, 0.0};
        for (int32_t k0 = 0; k0 < nch; k0 += 4) {
            double cm[4], cx[4][3];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int64_t c = (int64_t)wb.z + k0 + k;
                const bool ok = k0 + k < nch;
                cm[k] = ok ? __ldcg(&b_mass[c]) : 0.0;
#pragma unroll
                for (int d = 0; d < 3; d++) cx[k][d] = ok ? __ldcg(&b_mx[3 * c + d]) : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (k0 + k >= nch) break;
                M = __dadd_rn(M, cm[k]);
#pragma unroll
                for (int d = 0; d < 3; d++) mx[d] = __dadd_rn(mx[d], cx[k][d]);
            }
        }
        if (b >= 0) {
            b_mass[b] = M;
#pragma unroll
            for (int d = 0; d < 3; d++) b_mx[3 * (int64_t)b + d] = mx[d];
        }
        double com[3];
        if (QUAD && b >= 0) {
            cell_com(b, wb, M, mx, b_com, wrec, com);
            cell_quad(b, wb, com, b_mass, b_com, b_q);
        }
        __threadfence();   // the sums (and in QUAD the COM and Q) before the arrivals
        if (b >= 0) {
            const int32_t q = b_up[b];
            if (q >= 0 && nb_in(q < b, cnt, err, SITE_MOMENTS, b)) atomicAdd(&arrive[q], 1);
        }
        if (!QUAD && b >= 0) cell_com(b, wb, M, mx, b_com, wrec, com);
    }
}

static void build_tail(nb_ctx *c, const double *pos, const float *mass, int64_t n,
                       const int32_t *sys_sorted);

void nb_launch_build(nb_ctx *c, const double *pos, const float *mass, int64_t n)
{
    cudaStream_t s = c->stream;
    cudaMemsetAsync(c->cnt, 0, sizeof(long long) * CNT_PP_CUM, s);
    k_bbox_root<<<c->bbox_blocks, 256, 0, s>>>(pos, n, c->bbox_part, c->err, c->cnt, c->root);
    nb_launched(c, "k_bbox_root");
    k_keys<<<nb_grid(n, 256), 256, 0, s>>>(pos, n, c->root, nullptr, c->keys, c->idx,
                                           c->key_order);
    nb_launched(c, "k_keys");
    nb_radix_sort(c, n);
    build_tail(c, pos, mass, n, nullptr);
}

// ------------------------------------------------------------ batches
// system of every particle from the (caller-owned) offsets; checks them
__global__ void __launch_bounds__(256)
k_sys_of(const int64_t *__restrict__ off, int64_t nsys, int64_t n, int32_t *__restrict__ sys_of,
         unsigned *__restrict__ err)
{
    for (int64_t sy = blockIdx.x; sy < nsys; sy += gridDim.x) {
        const int64_t a = off[sy], b = off[sy + 1];
        if (threadIdx.x == 0 && (!(b > a) || a < 0 || b > n || (sy == 0 && a != 0) ||
                                 (sy == nsys - 1 && b != n)))
            atomicOr(err, NB_EF_BADARG);
        const int64_t lo = a < 0 ? 0 : a, hi = b > n ? n : b;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) sys_of[i] = (int32_t)sy;
    }
}

// bounding box and root cube of each system (one block of 1024 threads per
// system), the same arithmetic as k_bbox + k_root: min / max on the
// order-preserving integer image of the FP64 bits (integer compares instead
// of FP64 ones), then the root cube in FP64 with explicit rounding
#define RS_SYS_T 1024
__global__ void __launch_bounds__(RS_SYS_T)
k_roots_sys(const double *__restrict__ pos, const int64_t *__restrict__ off, int64_t nsys,
            int64_t n, double *__restrict__ roots, unsigned *__restrict__ err)
{
    const long long FLIP = 0x7fffffffffffffffll;
    __shared__ long long s[RS_SYS_T / 32][6];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long *__restrict__ pb = reinterpret_cast<const long long *>(pos);
    for (int64_t sy = blockIdx.x; sy < nsys; sy += gridDim.x) {
        int64_t a = off[sy], b = off[sy + 1];
        a = a < 0 ? 0 : (a > n ? n : a);
        b = b < a ? a : (b > n ? n : b);
        long long lo[3], hi[3];
        for (int k = 0; k < 3; k++) { lo[k] = LLONG_MAX; hi[k] = LLONG_MIN; }
        bool bad = false;
        for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const long long bits = pb[3 * i + k];
                bad |= (bits & 0x7ff0000000000000ll) == 0x7ff0000000000000ll;   // inf or NaN
                const long long key = bits ^ ((bits >> 63) & FLIP);
                lo[k] = min(lo[k], key);
                hi[k] = max(hi[k], key);
            }
        if (bad) atomicOr(err, NB_EF_NONFINITE);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                lo[k] = min(lo[k], __shfl_down_sync(0xffffffffu, lo[k], o));
                hi[k] = max(hi[k], __shfl_down_sync(0xffffffffu, hi[k], o));
            }
        if (lane == 0)
            for (int k = 0; k < 3; k++) { s[w][k] = lo[k]; s[w][3 + k] = hi[k]; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int ww = 1; ww < RS_SYS_T / 32; ww++)
                for (int k = 0; k < 3; k++) {
                    s[0][k] = min(s[0][k], s[ww][k]);
                    s[0][3 + k] = max(s[0][3 + k], s[ww][3 + k]);
                }
            double lx[3], hx[3];
            for (int k = 0; k < 6; k++) {   // back to FP64 (the map is its own inverse)
                const long long v = s[0][k];
                const double x = __longlong_as_double(v ^ ((v >> 63) & FLIP));
                if (k < 3) lx[k] = x; else hx[k - 3] = x;
            }
            double *root = roots + 8 * sy;
            double ext = 0.0;
            for (int k = 0; k < 3; k++) {
                root[k] = __dmul_rn(0.5, __dadd_rn(lx[k], hx[k]));
                const double e = __dsub_rn(hx[k], lx[k]);
                if (e > ext) ext = e;
            }
            double L = __dmul_rn(ext, 1.0 + 0x1p-20);
            if (!(L > 0.0)) L = 1.0;
            root[3] = L;
            for (int k = 0; k < 3; k++) root[4 + k] = __dsub_rn(root[k], __dmul_rn(0.5, L));
            root[7] = __ddiv_rn(2097152.0, L);
        }
        __syncthreads();
    }
}

// second sort key: the system of each Morton-sorted particle
__global__ void __launch_bounds__(256)
k_sys_key(const uint32_t *__restrict__ idx, const int32_t *__restrict__ sys_of, int64_t n,
          uint64_t *__restrict__ skey, uint32_t *__restrict__ sval)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    skey[i] = (uint64_t)sys_of[idx[i]];
    sval[i] = (uint32_t)i;
}

// apply the (system)-stable order to the Morton-sorted keys
__global__ void __launch_bounds__(256)
k_sys_apply(const uint64_t *__restrict__ key, const uint32_t *__restrict__ idx,
            const uint64_t *__restrict__ skey, const uint32_t *__restrict__ sval, int64_t n,
            uint64_t *__restrict__ key_out, uint32_t *__restrict__ idx_out,
            int32_t *__restrict__ sys_sorted)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = sval[i];
    key_out[i] = key[j];
    idx_out[i] = idx[j];
    sys_sorted[i] = (int32_t)skey[i];
}

// level-order index of every system's root (depth-0 nodes)
__global__ void __launch_bounds__(256)
k_sys_roots(const int32_t *__restrict__ level_start, const int32_t *__restrict__ bfs2pid,
            const int32_t *__restrict__ n_first, const int32_t *__restrict__ sys_sorted,
            int32_t *__restrict__ sys_root)
{
    const int32_t nr = level_start[1];
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nr; b += gridDim.x * blockDim.x)
        sys_root[sys_sorted[n_first[bfs2pid[b]]]] = b;
}

void nb_launch_build_batched(nb_ctx *c, const double *pos, const float *mass, int64_t n,
                             const int64_t *off, int64_t nsys)
{
    cudaStream_t s = c->stream;
    cudaMemsetAsync(c->cnt, 0, sizeof(long long) * CNT_PP_CUM, s);
    const int gs = (int)(nsys < 65535 ? nsys : 65535);
    k_sys_of<<<gs, 256, 0, s>>>(off, nsys, n, c->sys_of, c->err);
    nb_launched(c, "k_sys_of");
    k_roots_sys<<<gs, RS_SYS_T, 0, s>>>(pos, off, nsys, n, c->root, c->err);
    nb_launched(c, "k_roots_sys");
    k_keys<<<nb_grid(n, 256), 256, 0, s>>>(pos, n, c->root, c->sys_of, c->keys, c->idx,
                                           c->key_order);
    nb_launched(c, "k_keys");
    nb_radix_sort(c, n);
    // stable by system on top of the Morton order: (system, key) order
    k_sys_key<<<nb_grid(n, 256), 256, 0, s>>>(c->idx, c->sys_of, n, c->skey, c->sval);
    nb_launched(c, "k_sys_key");
    nb_radix_sort_passes(c->skey, c->skey_alt, c->sval, c->sval_alt, c->sort_hist, c->scan_bsum,
                         n, 2, s);
    c->launches += 2 * 5;
    k_sys_apply<<<nb_grid(n, 256), 256, 0, s>>>(c->keys, c->idx, c->skey, c->sval, n,
                                                c->keys_alt, c->idx_alt, c->sys_sorted);
    nb_launched(c, "k_sys_apply");
    uint64_t *tk = c->keys; c->keys = c->keys_alt; c->keys_alt = tk;
    uint32_t *ti = c->idx; c->idx = c->idx_alt; c->idx_alt = ti;
    build_tail(c, pos, mass, n, c->sys_sorted);
    k_sys_roots<<<nb_grid(nsys, 256, c->num_sms * 4), 256, 0, s>>>(c->level_start, c->bfs2pid,
                                                                    c->n_first, c->sys_sorted,
                                                                    c->sys_root);
    nb_launched(c, "k_sys_roots");
}

static void build_tail(nb_ctx *c, const double *pos, const float *mass, int64_t n,
                       const int32_t *sys_sorted)
{
    cudaStream_t s = c->stream;
    k_gather<<<nb_grid(n, 256), 256, 0, s>>>(pos, mass, n, c->idx, c->perm, c->p_x64,
                                             c->p_hi, c->p_lo, c->cnt, c->err);
    nb_launched(c, "k_gather");
    k_levels<<<nb_grid(n, 256), 256, 0, s>>>(c->keys, n, sys_sorted, c->clev, c->ccount);
    nb_launched(c, "k_levels");
    nb_exclusive_scan(c, c->ccount, c->cstart, n, nullptr, &c->cnt[CNT_CELLS]);
    k_cells<<<nb_grid(n, 256), 256, 0, s>>>(c->keys, n, c->clev, c->cstart, c->node_c,
                                            c->n_level, c->n_first, c->n_count, c->n_parent,
                                            c->n_nchild, c->n_depth, c->cnt, sys_sorted,
                                            c->sys_off, c->err);
    nb_launched(c, "k_cells");
    const int gcap = c->num_sms * 16;
    k_cell_ends<<<nb_grid(c->max_nodes, 256, gcap), 256, 0, s>>>(
        c->keys, n, c->cstart, c->n_level, c->n_first, c->node_c, c->n_count, c->cnt, sys_sorted,
        c->sys_off, c->err);
    nb_launched(c, "k_cell_ends");
    k_parents<<<nb_grid(c->max_nodes, 256, gcap), 256, 0, s>>>(c->node_c, c->cnt, c->n_parent,
                                                               c->n_nchild, c->arrive, c->lcount,
                                                               c->err);
    nb_launched(c, "k_parents");
    // level order
    const int nt = (int)c->dtiles;
    k_depth_hist<<<nt, DS_T, 0, s>>>(c->n_depth, c->cnt, c->dhist, nt);
    nb_launched(c, "k_depth_hist");
    nb_exclusive_scan(c, (const int32_t *)c->dhist, (int32_t *)c->dhist,
                      (int64_t)NB_DEPTHS * nt, nullptr, nullptr);
    k_depth_scatter<<<nt, DS_T, 0, s>>>(c->n_depth, c->cnt, c->dhist, nt, c->bfs2pid, c->pid2bfs,
                                        c->err);
    nb_launched(c, "k_depth_scatter");
    k_level_start<<<1, 32, 0, s>>>(c->dhist, nt, c->level_start);
    nb_launched(c, "k_level_start");
    cudaMemsetAsync(c->cbkt_cnt, 0, sizeof(int32_t) * 2 * NB_CBKT, s);
    k_bfs_records<<<nb_grid(c->max_nodes, 256, gcap), 256, 0, s>>>(
        c->bfs2pid, c->pid2bfs, c->node_c, c->n_first, c->n_nchild, c->n_parent, c->n_depth,
        c->keys, c->root, sys_sorted, c->p_hi, c->p_lo, c->p_x64, c->cnt, c->wrec, c->b_mass,
        c->b_mx, c->b_com, c->b_up, c->lcount, c->cbkt, c->cbkt_cnt, n, c->key_order,
        c->quad ? c->b_q : nullptr, c->err);
    nb_launched(c, "k_bfs_records");
    const int cl_blocks = (int)((c->max_nodes + CL_TILE - 1) / CL_TILE);
    k_cell_list<<<cl_blocks > 0 ? cl_blocks : 1, 256, 0, s>>>(c->cbkt, c->cbkt_cnt, c->cnt,
                                                               c->clist, c->clist_len, c->err);
    nb_launched(c, "k_cell_list");
    static int mblocks = 0, qblocks = 0;
    if (mblocks == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mblocks, k_moments<false>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&qblocks, k_moments<true>, 256, 0);
        if (mblocks < 1) mblocks = 1;
        if (qblocks < 1) qblocks = 1;
    }
    if (c->quad && c->b_q)
        k_moments<true><<<c->num_sms * qblocks, 256, 0, s>>>(
            c->clist, c->clist_len, c->wrec, c->b_up, c->lcount, c->b_mass, c->b_mx, c->b_com,
            c->b_q, c->arrive, c->cnt, c->err);
    else
        k_moments<false><<<c->num_sms * mblocks, 256, 0, s>>>(
            c->clist, c->clist_len, c->wrec, c->b_up, c->lcount, c->b_mass, c->b_mx, c->b_com,
            nullptr, c->arrive, c->cnt, c->err);
    nb_launched(c, "k_moments");
}

// ------------------------------------------------------------ groups
__global__ void __launch_bounds__(256)
k_group_flags(const int32_t *__restrict__ n_count, const int32_t *__restrict__ n_parent,
              long long *__restrict__ cnt, int n_crit, int32_t *__restrict__ flag,
              unsigned *__restrict__ err)
{
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += gridDim.x * blockDim.x) {
        int32_t p = n_parent[u];
        if (!nb_in(p < total, cnt, err, SITE_GROUPS, u)) p = -1;
        flag[u] = (n_count[u] <= n_crit) && (p < 0 || n_count[p] > n_crit);
    }
}

__global__ void __launch_bounds__(256)
k_group_scatter(const int32_t *__restrict__ gid, const int32_t *__restrict__ n_first,
                const int32_t *__restrict__ n_count, long long *__restrict__ cnt,
                int32_t *__restrict__ gnode, int32_t *__restrict__ gfirst,
                int32_t *__restrict__ gcount, int64_t n, unsigned *__restrict__ err)
{
    const int32_t total = (int32_t)cnt[CNT_NODES];
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += gridDim.x * blockDim.x) {
        const int32_t g = gid[u];
        if (gid[u + 1] != g) {
            if (!nb_in(g >= 0 && g < n, cnt, err, SITE_GROUPS, g)) continue;
            gnode[g] = u;
            gfirst[g] = n_first[u];
            gcount[g] = n_count[u];
        }
    }
}

// Force work items of a group of m members (iblock = 64: two targets per
// lane, or 32): full items of iblock, then (iblock 64) one 32-target item
// if more than 32 remain, then a tail of <= 32 targets, run as 32/m' source
// streams with m' the tail rounded up to a power of two.  Word: first member
// | log2(streams) << 27 | (1 << 30 for a 64-target item).
__device__ __forceinline__ int32_t item_count(int32_t m, int iblock)
{
    int32_t c = m / iblock, rem = m - c * iblock;
    if (iblock == 64 && rem > 32) { c++; rem -= 32; }
    return c + (rem > 0 ? 1 : 0);
}

// group box over the members' FP32 positions, its FP32 centre, FP32
// 1/theta, and the number of force work items of the group.  A warp takes GB
// consecutive groups: for each in turn the members are strided over the lanes
// and the box is reduced by shuffles (min and max are exact, so the order
// does not matter), and lane k keeps group k's box.  The FP64 centre and
// 1/theta then run once for the GB groups, one per lane: an FP64 instruction
// costs GB300's FP64 pipe as much for one active lane as for 32.  (GB 8 was
// faster than 16 and 32: more warps share the sequential reductions.)
__global__ void __launch_bounds__(256)
k_group_boxes(const int32_t *__restrict__ gfirst, const int32_t *__restrict__ gcount,
              const float4 *__restrict__ p_hi, long long *__restrict__ cnt,
              float theta, const float *__restrict__ theta_g, float4 *__restrict__ gbox,
              int32_t *__restrict__ item_cnt, int iblock, int64_t n, unsigned *__restrict__ err)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    const int32_t nw = gridDim.x * (blockDim.x >> 5);
    constexpr int GB = 8;
    for (int32_t g0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * GB; g0 < G;
         g0 += nw * GB) {
        const int32_t gl = lane < GB ? g0 + lane : G;   // this lane's group (lanes < GB)
        int32_t fl = 0, ml = 0;
        if (gl < G) {
            fl = gfirst[gl];
            ml = gcount[gl];
        }
        const bool okl = gl < G && fl >= 0 && ml >= 1 && (int64_t)fl + ml <= n;
        const unsigned okm = __ballot_sync(FULL, okl);
        float blx = 0.f, bly = 0.f, blz = 0.f, bhx = 0.f, bhy = 0.f, bhz = 0.f;
        for (int k = 0; k < GB && g0 + k < G; k++) {
            if (!((okm >> k) & 1u)) continue;
            const int32_t f = __shfl_sync(FULL, fl, k), m = __shfl_sync(FULL, ml, k);
            float lx = INFINITY, ly = INFINITY, lz = INFINITY;
            float hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
            for (int32_t j = lane; j < m; j += NB_WARP) {
                const float4 p = p_hi[f + j];
                lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
                hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y); hz = fmaxf(hz, p.z);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lx = fminf(lx, __shfl_xor_sync(FULL, lx, o));
                ly = fminf(ly, __shfl_xor_sync(FULL, ly, o));
                lz = fminf(lz, __shfl_xor_sync(FULL, lz, o));
                hx = fmaxf(hx, __shfl_xor_sync(FULL, hx, o));
                hy = fmaxf(hy, __shfl_xor_sync(FULL, hy, o));
                hz = fmaxf(hz, __shfl_xor_sync(FULL, hz, o));
            }
            if (lane == k) {
                blx = lx; bly = ly; blz = lz;
                bhx = hx; bhy = hy; bhz = hz;
            }
        }
        if (gl >= G) continue;
        if (!okl) {
            nb_bad(cnt, err, SITE_GROUPS, gl);
            item_cnt[gl] = 0;
            continue;
        }
        const float th = theta_g ? theta_g[gl] : theta;
        const float invth = __double2float_rn(__ddiv_rn(1.0, (double)th));
        const float cx = __double2float_rn(__dmul_rn(0.5, __dadd_rn((double)blx, (double)bhx)));
        const float cy = __double2float_rn(__dmul_rn(0.5, __dadd_rn((double)bly, (double)bhy)));
        const float cz = __double2float_rn(__dmul_rn(0.5, __dadd_rn((double)blz, (double)bhz)));
        gbox[3 * (int64_t)gl] = make_float4(blx, bly, blz, 0.0f);
        gbox[3 * (int64_t)gl + 1] = make_float4(bhx, bhy, bhz, 0.0f);
        gbox[3 * (int64_t)gl + 2] = make_float4(cx, cy, cz, invth);
        item_cnt[gl] = item_count(ml, iblock);
    }
}

__global__ void __launch_bounds__(256)
k_items(const int32_t *__restrict__ item_off, const int32_t *__restrict__ gcount,
        long long *__restrict__ cnt, int32_t *__restrict__ items, int iblock, int64_t max_items,
        unsigned *__restrict__ err)
{
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += gridDim.x * blockDim.x) {
        const int32_t o = item_off[g], m = gcount[g];
        if (!nb_in(o >= 0 && (int64_t)o + item_count(m, iblock) <= max_items, cnt, err,
                   SITE_ITEMS, g))
            continue;
        int32_t i0 = 0, k = 0;
        for (; m - i0 >= iblock; i0 += iblock, k++) {
            items[2 * (int64_t)(o + k)] = g;
            items[2 * (int64_t)(o + k) + 1] = i0 | (iblock == 64 ? (1 << 30) : 0);
        }
        int32_t rem = m - i0;
        if (iblock == 64 && rem > 32) {
            items[2 * (int64_t)(o + k)] = g;
            items[2 * (int64_t)(o + k) + 1] = i0;
            i0 += 32;
            rem -= 32;
            k++;
        }
        if (rem > 0) {
            const int lg = rem > 1 ? 32 - __clz(rem - 1) : 0;   // log2 of rem rounded up
            items[2 * (int64_t)(o + k)] = g;
            items[2 * (int64_t)(o + k) + 1] = i0 | ((5 - lg) << 27);
        }
    }
}

// 1/theta of every formed group's box from a per-group theta (the same
// rounding as k_group_boxes)
__global__ void __launch_bounds__(256)
k_group_theta(const float *__restrict__ theta_g, const long long *__restrict__ cnt,
              float4 *__restrict__ gbox)
{
    const int32_t G = (int32_t)cnt[CNT_GROUPS];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        gbox[3 * (int64_t)g + 2].w = __double2float_rn(__ddiv_rn(1.0, (double)theta_g[g]));
}

void nb_launch_group_theta(nb_ctx *c, const float *theta_g)
{
    k_group_theta<<<nb_grid(c->max_n, 256, c->num_sms * 8), 256, 0, c->stream>>>(theta_g, c->cnt,
                                                                                c->gbox);
    nb_launched(c, "k_group_theta");
}

void nb_launch_groups(nb_ctx *c, float theta, int n_crit, const float *theta_g)
{
    cudaStream_t s = c->stream;
    const int gcap = c->num_sms * 16;
    k_group_flags<<<nb_grid(c->max_nodes, 256, gcap), 256, 0, s>>>(
        c->n_count, c->n_parent, c->cnt, n_crit, c->gflag, c->err);
    nb_launched(c, "k_group_flags");
    nb_exclusive_scan(c, c->gflag, c->gflag, c->max_nodes, &c->cnt[CNT_NODES],
                      &c->cnt[CNT_GROUPS]);
    k_group_scatter<<<nb_grid(c->max_nodes, 256, gcap), 256, 0, s>>>(
        c->gflag, c->n_first, c->n_count, c->cnt, c->gnode, c->gfirst, c->gcount, c->n, c->err);
    nb_launched(c, "k_group_scatter");
    k_group_boxes<<<c->num_sms * 16, 256, 0, s>>>(
        c->gfirst, c->gcount, c->p_hi, c->cnt, theta, theta_g, c->gbox, c->item_cnt,
        c->item_rows * NB_WARP, c->n, c->err);
    nb_launched(c, "k_group_boxes");
    nb_exclusive_scan(c, c->item_cnt, c->item_cnt, c->max_n, &c->cnt[CNT_GROUPS],
                      &c->cnt[CNT_ITEMS]);
    k_items<<<nb_grid(c->max_n, 256, gcap), 256, 0, s>>>(c->item_cnt, c->gcount, c->cnt,
                                                          c->items, c->item_rows * NB_WARP,
                                                          c->max_items, c->err);
    nb_launched(c, "k_items");
}

// Root cube and Morton keys on buffers the caller supplies (no context):
// part holds 6 * nblk doubles, root 8; idx receives 0..n-1.
void nb_launch_keys_raw(const double *pos, int64_t n, double *part, int nblk, double *root,
                        uint64_t *keys, uint32_t *idx, unsigned *err, cudaStream_t s)
{
    k_bbox<<<nblk, 256, 0, s>>>(pos, n, part, err);
    k_root<<<1, 256, 0, s>>>(part, nblk, root);
    k_keys<<<nb_grid(n, 256), 256, 0, s>>>(pos, n, root, nullptr, keys, idx, 0);
}

