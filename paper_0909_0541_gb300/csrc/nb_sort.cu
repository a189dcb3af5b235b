// nb_sort.cu -- device-wide exclusive scan and the stable LSD radix sort of
// (63-bit Morton key, particle index) pairs that puts particles in Morton
// order (Sec. "Test and Optimization": depth-first leaf order of the tree).
//
// Radix sort: 8 passes of 8-bit digits.  The context's sort is single-pass
// per digit (Onesweep, see k_rs_scatter): one histogram of all eight digits,
// then one scatter launch per pass over tiles of NB_RS_TILE_MIN keys, which
// find their offsets by a bounded decoupled look-back.  The sort on
// caller-supplied buffers (no context) keeps three phases per pass over
// tiles of NB_RS_TILE keys, none
// of which waits on another block: per-tile digit histograms -> exclusive
// scan of the digit-major table -> stable scatter.  Stability inside a tile
// comes from warp-level ranking of 32 consecutive keys at a time with
// per-warp running digit counts, then a scan of those counts across the 8
// warps.
#include "nb_internal.cuh"

#define SCAN_T 256
#define SCAN_I 8
#define SCAN_TILE (SCAN_T * SCAN_I)

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *total)
{
    __shared__ int32_t wsum[SCAN_T / NB_WARP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t s = lane < SCAN_T / NB_WARP ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_T / NB_WARP) wsum[lane] = s;
    }
    __syncthreads();
    const int32_t before = (w > 0 ? wsum[w - 1] : 0) + x - v;
    if (total) *total = wsum[SCAN_T / NB_WARP - 1];
    __syncthreads();
    return before;
}

__device__ __forceinline__ int64_t eff_n(int64_t n_max, const long long *n_dev)
{
    if (!n_dev) return n_max;
    const long long v = *n_dev;
    return v < n_max ? (int64_t)v : n_max;
}

__global__ void __launch_bounds__(SCAN_T)
k_scan_reduce(const int32_t *__restrict__ in, int64_t n_max,
              const long long *__restrict__ n_dev, int32_t *__restrict__ bsum)
{
    const int64_t n = eff_n(n_max, n_dev);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int32_t s = 0;
    if (base < n) {
#pragma unroll
        for (int k = 0; k < SCAN_I; k++) {
            const int64_t i = base + k * SCAN_T + threadIdx.x;
            if (i < n) s += in[i];
        }
    }
    int32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = base < n ? tot : 0;
}

// one block: exclusive scan of the tile sums; writes out[n] and the total
// Second pass: each block adds up the totals of the tiles before its own
// (read from L2 by the whole block), then scans its tile.  The reads grow
// with the square of the tile count: about 9 MB for the 4.4M nodes of a
// 2.87M-particle tree, 0.3 GB for a 16M-particle one, well under 1 % of a
// step either way.  Each thread holds 8 consecutive elements, loaded and stored as two
// 16-byte vectors when the arrays allow it (VEC).  The block of the last
// non-empty tile (block 0 when n is 0) writes out[n] and the total.
template <bool VEC>
__global__ void __launch_bounds__(SCAN_T)
k_scan_apply(const int32_t *__restrict__ in, int32_t *__restrict__ out,
             int64_t n_max, const long long *__restrict__ n_dev,
             const int32_t *__restrict__ bsum, long long *__restrict__ total_dev)
{
    static_assert(SCAN_I == 8, "two 16-byte vectors per thread");
    const int64_t n = eff_n(n_max, n_dev);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int64_t last = n > 0 ? (n - 1) / SCAN_TILE : 0;
    if ((int64_t)blockIdx.x > last) return;
    int32_t before = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += SCAN_T) before += bsum[i];
    {
        int32_t all;
        block_excl_scan(before, &all);
        before = all;
    }
    const int64_t i0 = base + (int64_t)threadIdx.x * SCAN_I;
    int32_t v[SCAN_I];
    if (VEC && i0 + SCAN_I <= n) {
        const int4 a = reinterpret_cast<const int4 *>(in + i0)[0];
        const int4 b = reinterpret_cast<const int4 *>(in + i0)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_I; k++) v[k] = i0 + k < n ? in[i0 + k] : 0;
    }
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; k++) s += v[k];
    int32_t tile_total;
    int32_t run = block_excl_scan(s, &tile_total) + before;
    int32_t o[SCAN_I];
#pragma unroll
    for (int k = 0; k < SCAN_I; k++) {
        o[k] = run;
        run += v[k];
    }
    if (VEC && i0 + SCAN_I <= n) {
        reinterpret_cast<int4 *>(out + i0)[0] = make_int4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<int4 *>(out + i0)[1] = make_int4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_I; k++)
            if (i0 + k < n) out[i0 + k] = o[k];
    }
    if ((int64_t)blockIdx.x == last && threadIdx.x == 0) {
        out[n] = before + tile_total;
        if (total_dev) *total_dev = before + tile_total;
    }
}

// Exclusive scan of in[0..n) into out[0..n], out[n] = total.  n is
// min(*n_dev, n_max) when n_dev is given (device-resident count), else
// n_max.  In-place (in == out) is allowed.
void nb_exclusive_scan(nb_ctx *c, const int32_t *in, int32_t *out, int64_t n_max,
                       const long long *n_dev, long long *total_dev)
{
    const int nb = (int)((n_max + SCAN_TILE - 1) / SCAN_TILE);
    const int g = nb > 0 ? nb : 1;
    k_scan_reduce<<<g, SCAN_T, 0, c->stream>>>(in, n_max, n_dev, c->scan_bsum);
    nb_launched(c, "k_scan_reduce");
    if (((uintptr_t)in & 15u) == 0 && ((uintptr_t)out & 15u) == 0)
        k_scan_apply<true><<<g, SCAN_T, 0, c->stream>>>(in, out, n_max, n_dev, c->scan_bsum,
                                                        total_dev);
    else
        k_scan_apply<false><<<g, SCAN_T, 0, c->stream>>>(in, out, n_max, n_dev, c->scan_bsum,
                                                         total_dev);
    nb_launched(c, "k_scan_apply");
}

// ------------------------------------------------------------ radix sort
#define RS_T 256
#define RS_I (NB_RS_TILE / RS_T)
#define RS_TILE NB_RS_TILE
#define RS_WARPS (RS_T / NB_WARP)

__global__ void __launch_bounds__(RS_T)
k_rs_hist(const uint64_t *__restrict__ key, int64_t n, int shift,
          uint32_t *__restrict__ hist, int nb)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int k = 0; k < RS_I; k++) {
        const int64_t i = base + k * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile.  (1) every key and value is loaded; (2) each
// warp ranks its 16 rounds of 32 keys by digit (warp match from one ballot
// per digit bit) and running per-warp digit counts; (3) the warps' counts are scanned per digit and the
// tile's digit totals across digits, giving each key its place in the
// tile's digit order; (4) keys and values are staged there in shared memory
// and (5) written out by consecutive threads, so that each digit's run goes
// to global memory as contiguous, coalesced stores.
//
// ONESWEEP (Adinets and Merrill, "Onesweep: a faster least significant digit
// radix sort for GPUs", 2022): no histogram or scan launch per pass.  A
// block claims its tile from a counter, so tiles are claimed in order; the
// digit bases come from one histogram of all eight digits made before the
// first pass; each tile publishes its digit counts and finds the counts of
// the tiles before it by decoupled look-back (Merrill and Garland,
// "Single-pass parallel prefix scan with decoupled look-back", 2016).  A
// status word holds a flag (2 bits: not ready, this tile's count, inclusive
// prefix) and a 30-bit count.  A tile waits only for tiles claimed before it,
// whose blocks are running; every wait is bounded, and a wait that runs out
// is reported (SITE_SORT_WAIT) and makes every other waiting block stop.
#define RS_SMEM (RS_TILE * (int)(sizeof(uint64_t) + sizeof(uint32_t)))
#define RS_AGG (1u << 30)
#define RS_INC (2u << 30)
#define RS_VAL ((1u << 30) - 1u)
#define RS_LB 4   // look-back window: predecessor tiles read per round trip

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// I keys per thread: a tile of RS_T * I keys (RS_I for the fixed-tile paths,
// RS_I1 for the context's single-pass sort)
template <bool ONESWEEP, int I = RS_I>
__global__ void __launch_bounds__(RS_T, 3)
k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
             const uint32_t *__restrict__ offs, int64_t n, int shift, int nb,
             long long *__restrict__ cnt, unsigned *__restrict__ err, uint32_t *status,
             const uint32_t *__restrict__ ghist, uint32_t *tilectr)
{
    constexpr int TILE = RS_T * I;
    extern __shared__ __align__(16) unsigned char rs_stage[];
    uint64_t *sk = (uint64_t *)rs_stage;
    uint32_t *sv = (uint32_t *)(rs_stage + TILE * sizeof(uint64_t));
    __shared__ uint32_t whist[RS_WARPS][256];
    __shared__ uint32_t boff[256];
    __shared__ uint32_t lstart[256];
    __shared__ int blk_s;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int i = t; i < RS_WARPS * 256; i += RS_T) (&whist[0][0])[i] = 0u;
    if (ONESWEEP) {
        if (t == 0) blk_s = (int)atomicAdd(tilectr, 1u);
    } else {
        boff[t] = offs[(int64_t)t * nb + blockIdx.x];
    }
    __syncthreads();
    const int blk = ONESWEEP ? blk_s : (int)blockIdx.x;
    const int64_t tile0 = (int64_t)blk * TILE;
    const int64_t rem = n - tile0;
    const int tn = rem < TILE ? (int)rem : TILE;   // keys in this tile
    const int wbase = w * (TILE / RS_WARPS);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t key[I];
    uint32_t rnk[I];
#pragma unroll
    for (int r = 0; r < I; r++) {
        const int e = wbase + r * NB_WARP + lane;
        key[r] = e < tn ? kin[tile0 + e] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < I; r++) {
        const bool ok = wbase + r * NB_WARP + lane < tn;
        const int d = ok ? (int)((key[r] >> shift) & 255u) : 256 + lane;
        const unsigned peers = nb_match_bits<8>((unsigned)d, ok);
        const unsigned before = __popc(peers & lt);
        const uint32_t pre = ok ? whist[w][d] : 0u;
        __syncwarp();
        if (ok && before == 0) whist[w][d] = pre + __popc(peers);
        __syncwarp();
        rnk[r] = pre + before;
    }
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ww++) {
        const uint32_t v = whist[ww][t];
        whist[ww][t] = run;
        run += v;
    }
    if (ONESWEEP) {
        // digit base of the pass, then this tile's place among the tiles
        int32_t all;
        const uint32_t dbase = (uint32_t)nb_block_scan256((int32_t)ghist[t], &all);
        uint32_t *my = status + (int64_t)blk * 256 + t;
        if (blk == 0) {
            st_relaxed(my, RS_INC | run);
            boff[t] = dbase;
        } else {
            st_relaxed(my, RS_AGG | run);
            // look back RS_LB tiles per round trip: the window's words are
            // loaded together, then taken in order until an inclusive prefix
            // (done) or a tile not yet published (wait and reload from there)
            uint32_t excl = 0;
            int j = blk - 1;
            unsigned spins = 0;
            bool done = false;
            while (!done && j >= 0) {
                uint32_t sw[RS_LB];
#pragma unroll
                for (int q = 0; q < RS_LB; q++)
                    sw[q] = j - q >= 0 ? ld_relaxed(status + (int64_t)(j - q) * 256 + t) : 0u;
                int used = 0;
                bool wait = false;
#pragma unroll
                for (int q = 0; q < RS_LB; q++) {
                    if (done || wait || j - q < 0) continue;
                    if ((sw[q] & ~RS_VAL) == 0u) {   // not published yet
                        wait = true;
                        continue;
                    }
                    excl += sw[q] & RS_VAL;
                    used++;
                    if (sw[q] & RS_INC) done = true;
                }
                j -= used;
                if (wait) {
                    if (++spins >= NB_SPIN_LIMIT) {
                        nb_bad(cnt, err, SITE_SORT_WAIT, j);
                        break;
                    }
                    if ((spins & 63u) == 0u &&
                        (*(volatile unsigned *)err & NB_EF_BOUNDS) != 0u)
                        break;   // another block gave up
                    __nanosleep(32);
                }
            }
            st_relaxed(my, RS_INC | ((excl + run) & RS_VAL));
            boff[t] = dbase + excl;
        }
    }
    // run = the tile's count of digit t; lstart = exclusive scan over digits
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __shared__ uint32_t wtot[RS_WARPS];
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    uint32_t wpre = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ww++) wpre += ww < w ? wtot[ww] : 0u;
    lstart[t] = wpre + x - run;
    __syncthreads();
    // values are loaded only now (they need no ranking): fewer registers
    // held through the ranking rounds
    uint32_t val[I];
#pragma unroll
    for (int r = 0; r < I; r++) {
        const int e = wbase + r * NB_WARP + lane;
        val[r] = e < tn ? vin[tile0 + e] : 0u;
    }
#pragma unroll
    for (int r = 0; r < I; r++) {
        if (wbase + r * NB_WARP + lane < tn) {
            const int d = (int)((key[r] >> shift) & 255u);
            const uint32_t lp = lstart[d] + whist[w][d] + rnk[r];
            if (lp < (uint32_t)tn) {
                sk[lp] = key[r];
                sv[lp] = val[r];
            } else if (cnt) {
                nb_bad(cnt, err, SITE_SORT, lp);
            }
        }
    }
    __syncthreads();
#pragma unroll 4
    for (int e = t; e < tn; e += RS_T) {
        const uint64_t k = sk[e];
        const int d = (int)((k >> shift) & 255u);
        const uint32_t pos = boff[d] + (uint32_t)e - lstart[d];
        if (pos >= n) {   // a self-check (recorded when a context is given)
            if (cnt) nb_bad(cnt, err, SITE_SORT, pos);
            continue;
        }
        kout[pos] = k;
        vout[pos] = sv[e];
    }
}

// Keys per thread of the context's single-pass scatter: 12 (tiles of 3072
// keys) measured best of 10, 12, 13, 14 and 16 on the 2.87M-key sort (build
// 1.224 against 1.256 ms for 16: 935 tiles keep the 3 x SMs block slots
// fuller than 701 larger ones).  Any tile size gives the same sort.
#define RS_I1 12

// the staging buffer is dynamic shared memory above the 48 KB default
static constexpr int rs_smem(int I)
{
    return RS_T * I * (int)(sizeof(uint64_t) + sizeof(uint32_t));
}

static void rs_setup()
{
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_rs_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         RS_SMEM);
    cudaFuncSetAttribute(k_rs_scatter<true, RS_I1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         rs_smem(RS_I1));
    done = true;
}

// all eight 8-bit digit histograms in one read of the keys: shared-memory
// counts (the hardware serialises equal digits), then one global add per
// digit and block
__global__ void __launch_bounds__(RS_T)
k_rs_ghist(const uint64_t *__restrict__ key, int64_t n, uint32_t *__restrict__ ghist)
{
    __shared__ uint32_t h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += RS_T) (&h[0][0])[i] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * RS_T + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * RS_T) {
        const uint64_t k = key[i];
#pragma unroll
        for (int p = 0; p < 8; p++) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * 256; i += RS_T)
        if ((&h[0][0])[i]) atomicAdd(&ghist[i], (&h[0][0])[i]);
}

// Sort (c->keys, c->idx)[0..n) by key, stably.  Result in c->keys / c->idx.
void nb_radix_sort(nb_ctx *c, int64_t n)
{
    if (n <= 1) return;
    const int nb16 = (int)((n + RS_TILE - 1) / RS_TILE);
    rs_setup();
    uint64_t *ka = c->keys, *kb = c->keys_alt;
    uint32_t *va = c->idx, *vb = c->idx_alt;
    const int nb = (int)((n + (int64_t)RS_T * RS_I1 - 1) / ((int64_t)RS_T * RS_I1));
    if (n < (int64_t)RS_VAL && (int64_t)nb * 256 * 8 + 8 * 256 + 8 <= c->rs_status_len) {
        // onesweep: status words of the 8 passes, the 8 digit histograms and
        // the 8 tile counters, zeroed together
        uint32_t *ghist = c->rs_status + (int64_t)nb * 256 * 8;
        uint32_t *tctr = ghist + 8 * 256;
        cudaMemsetAsync(c->rs_status, 0, sizeof(uint32_t) * ((int64_t)nb * 256 * 8 + 8 * 256 + 8),
                        c->stream);
        k_rs_ghist<<<c->num_sms * 4, RS_T, 0, c->stream>>>(ka, n, ghist);
        nb_launched(c, "k_rs_ghist");
        for (int pass = 0; pass < 8; pass++) {
            k_rs_scatter<true, RS_I1><<<nb, RS_T, rs_smem(RS_I1), c->stream>>>(
                ka, va, kb, vb, nullptr, n, 8 * pass, nb, c->cnt, c->err,
                c->rs_status + (int64_t)pass * nb * 256, ghist + 256 * pass, tctr + pass);
            nb_launched(c, "k_rs_scatter");
            uint64_t *tk = ka; ka = kb; kb = tk;
            uint32_t *tv = va; va = vb; vb = tv;
        }
        return;   // 8 passes: the result is back in c->keys / c->idx
    }
    for (int pass = 0; pass < 8; pass++) {
        const int shift = 8 * pass;
        k_rs_hist<<<nb16, RS_T, 0, c->stream>>>(ka, n, shift, c->sort_hist, nb16);
        nb_launched(c, "k_rs_hist");
        nb_exclusive_scan(c, (const int32_t *)c->sort_hist, (int32_t *)c->sort_hist,
                          (int64_t)256 * nb16, nullptr, nullptr);
        k_rs_scatter<false><<<nb16, RS_T, RS_SMEM, c->stream>>>(ka, va, kb, vb, c->sort_hist, n,
                                                                shift, nb16, c->cnt, c->err,
                                                                nullptr, nullptr, nullptr);
        nb_launched(c, "k_rs_scatter");
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    // 8 passes: the result is back in c->keys / c->idx
}

// ------------------------------------------------------- explicit buffers
// The same scan and sort, on buffers the caller supplies (no context).
void nb_exclusive_scan_raw(const int32_t *in, int32_t *out, int64_t n_max, int32_t *bsum,
                           cudaStream_t s)
{
    const int nb = (int)((n_max + SCAN_TILE - 1) / SCAN_TILE);
    const int g = nb > 0 ? nb : 1;
    k_scan_reduce<<<g, SCAN_T, 0, s>>>(in, n_max, nullptr, bsum);
    if (((uintptr_t)in & 15u) == 0 && ((uintptr_t)out & 15u) == 0)
        k_scan_apply<true><<<g, SCAN_T, 0, s>>>(in, out, n_max, nullptr, bsum, nullptr);
    else
        k_scan_apply<false><<<g, SCAN_T, 0, s>>>(in, out, n_max, nullptr, bsum, nullptr);
}

// keys/idx hold the input and, after the 8 passes, the sorted output;
// hist needs 256 * ceil(n / NB_RS_TILE) + 1 entries, bsum the scan's tile sums.
void nb_radix_sort_raw(uint64_t *keys, uint64_t *keys_alt, uint32_t *idx, uint32_t *idx_alt,
                       uint32_t *hist, int32_t *bsum, int64_t n, cudaStream_t s)
{
    nb_radix_sort_passes(keys, keys_alt, idx, idx_alt, hist, bsum, n, 8, s);
}

// `passes` (even) 8-bit passes from the lowest digit; the result is back in
// keys / idx
void nb_radix_sort_passes(uint64_t *keys, uint64_t *keys_alt, uint32_t *idx, uint32_t *idx_alt,
                          uint32_t *hist, int32_t *bsum, int64_t n, int passes, cudaStream_t s)
{
    if (n <= 1) return;
    const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
    rs_setup();
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = idx, *vb = idx_alt;
    for (int pass = 0; pass < passes; pass++) {
        const int shift = 8 * pass;
        k_rs_hist<<<nb, RS_T, 0, s>>>(ka, n, shift, hist, nb);
        nb_exclusive_scan_raw((const int32_t *)hist, (int32_t *)hist, (int64_t)256 * nb, bsum, s);
        k_rs_scatter<false><<<nb, RS_T, RS_SMEM, s>>>(ka, va, kb, vb, hist, n, shift, nb, nullptr,
                                                      nullptr, nullptr, nullptr, nullptr);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
}
