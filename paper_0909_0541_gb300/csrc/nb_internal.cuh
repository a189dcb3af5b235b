// nb_internal.cuh -- device-side layout shared by the libnb translation units.
//
// HBM layout (all per context, allocated once for max_n particles; NN = 12N+2
// node slots bound the cells + particle leaves of any input):
//   sorted particles  p_hi[N] float4 (x,y,z as the FP32 nearest to the FP64
//                     position, mass), p_lo[N] float4 (FP32 remainders),
//                     p_x64[3N] FP64 positions, perm[N] sorted slot -> caller
//   topology          depth-first preorder ("pid"): node_c int4 (next, -, -,
//                     is_particle), level, first particle, count, parent,
//                     number of children, depth
//   walk records      level order ("bfs": nodes sorted by depth, preorder
//                     inside a depth), so the children of a cell are one
//                     contiguous run; one 64-byte nb_wrec per node
//                     and FP64 mass, first moment and centre of mass
//   groups            gnode (pid), first slot, size, box 3 x float4 (lo, hi,
//                     centre + 1/theta), list length, cell entries
//   lists             slot g at g * cap: list_id int32 (pid), list_xm float4
//                     (group-relative x, y, z, mass); the group's own
//                     particles are not listed (the force kernel sums them)
//   walk queues       two frontier queues of wq_cap node indices per warp
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nb.h"

#define NB_LEVELS 21
#define NB_DEPTHS 23   // tree depths 0..22 (level-21 buckets hold depth-22 leaves)
#define NB_IBKT 64     // cost buckets of the force work queue (quarter octaves)
#define NB_CBKT (NB_DEPTHS * 8)   // cell buckets for the moments: (depth, children)
#define NB_SPIN_LIMIT (1u << 20)  // polls before a wait for another warp gives up
#define NB_WARP 32
#define NB_RS_TILE 4096   // keys per radix-sort tile (sizes the sort's per-tile buffers)
#define NB_RS_TILE_MIN 3072   // the tile of the context's single-pass sort (nb_sort.cu)
#define NB_DS_TILE 4096   // nodes per tile of the stable sort by depth
#define NB_EV_POOL 2048
#define NB_IBLOCK 64   // targets per force work item (two per lane)
#define NB_PROBE_THETA 1.2f  // opening angle of the feature probe walk

// bits of the device error word
#define NB_EF_NONFINITE 1u
#define NB_EF_CAPACITY 2u
#define NB_EF_WALK 4u
#define NB_EF_QUEUE 8u
#define NB_EF_BADARG 16u
#define NB_EF_BOUNDS 32u   // an index failed a kernel's own bounds check (access skipped)

// device counters (int64 slots of ctx->cnt)
enum {
    CNT_CELLS = 0,   // C
    CNT_NODES,       // C + N
    CNT_GROUPS,      // G
    CNT_LIST_TOT,    // sum of list lengths
    CNT_LIST_MAX,    // longest list
    CNT_PP,          // particle-particle interactions
    CNT_PC,          // particle-cell interactions
    CNT_WALK_Q,      // walk work queue head
    CNT_FORCE_Q,     // force work queue head
    CNT_ITEMS,       // force work items
    CNT_MAXLEVEL,
    CNT_QMAX,        // widest walk frontier
    CNT_MOM_Q,       // moments work queue head (32-cell chunks)
    CNT_MOM_CHUNKS,  // chunks in the moments work list
    CNT_BBOX_DONE,   // blocks of k_bbox_root that have written their partial box
    CNT_PP_CUM,      // n_pp over every walk (never reset)
    CNT_PC_CUM,
    CNT_BAD_SITE,    // first failed self-check: site code (never reset)
    CNT_BAD_INDEX,   // ... and the offending index
    CNT_N_
};

// self-check sites (a kernel's own bounds checks; a hit is a library defect)
enum {
    SITE_NONE = 0,
    SITE_GATHER,      // sorted slot -> caller index out of range
    SITE_CELLS,       // node id outside the node count
    SITE_PARENTS,     // child id outside the node count
    SITE_DEPTH,       // level-order position outside the node count
    SITE_RECORDS,     // preorder id or particle slot out of range
    SITE_MOMENTS,     // parent, child run or level out of range (bottom-up moments)
    SITE_GROUPS,      // group id or member range out of range
    SITE_ITEMS,       // work item index out of range
    SITE_WALK_NODE,   // queued node outside the node count
    SITE_WALK_CHILD,  // child run outside the node count
    SITE_FORCE,       // force item out of range
    SITE_SORT,        // radix-sort destination out of range
    SITE_MOMENTS_WAIT,  // a wait for a cell's children ran out (moments)
    SITE_SORT_WAIT,     // a radix-sort look-back wait ran out
    SITE_OVERLAP_WAIT,  // a force item's wait for its group's walk ran out
    SITE_N_
};

// The walk's view of one node, in level order, as one 64-byte record so a
// visited node touches one cache line: centre of mass as FP32 hi part and
// FP32 mass; FP32 lo part; preorder id, preorder next, first child (level
// order; -1 for a particle leaf), number of children; side l and offset s.
struct __align__(64) nb_wrec {
    float4 a;
    float4 d;
    int4 b;
    float2 c;
    float2 pad;
};

// writes in whole 32-byte sectors: (a, d) and (b, c + pad)
__device__ __forceinline__ void nb_wrec_put_lo(nb_wrec *w, float4 a, float4 d)
{
    w->a = a;
    w->d = d;
}
__device__ __forceinline__ void nb_wrec_put_hi(nb_wrec *w, int4 b, float l, float s)
{
    w->b = b;
    *reinterpret_cast<float4 *>(&w->c) = make_float4(l, s, 0.0f, 0.0f);
}

struct nb_ctx {
    int device;
    cudaStream_t stream;
    int sync_checks;
    nb_config cfg;
    int num_sms;

    int64_t max_n;
    int64_t max_nodes;    // 12 * max_n + 2
    int64_t n;            // particles in the current tree
    int has_tree, has_groups, has_lists, acc_valid;
    int n_crit_cur;
    int64_t groups_host;  // G of the last walk, when known on the host

    // sort
    uint64_t *keys, *keys_alt;
    uint32_t *idx, *idx_alt;
    uint32_t *sort_hist;
    int64_t sort_hist_len;
    uint32_t *rs_status;     // onesweep: tile status words, digit histograms, tile counters
    int64_t rs_status_len;

    // scan scratch
    int32_t *scan_bsum;
    int64_t scan_bsum_len;

    // batches of independent systems: system of each particle (caller and
    // sorted order), system offsets (caller-owned, device), root node of each
    // system in level order; nsys = 1 for a single system
    int64_t nsys, max_sys;
    int32_t *sys_of, *sys_sorted, *sys_root;
    const int64_t *sys_off;
    uint64_t *skey, *skey_alt;
    uint32_t *sval, *sval_alt;

    // roots: per system centre[3], L, corner[3], 2^21 / L (8 doubles each);
    // bbox partials
    double *root;
    double *bbox_part;
    int bbox_blocks;

    // sorted particles
    float4 *p_hi, *p_lo;
    double *p_x64;
    int32_t *perm;
    int8_t *clev;     // common levels of neighbouring keys
    int32_t *ccount;  // cells starting at each particle
    int32_t *cstart;  // exclusive scan of ccount (N + 1)

    // topology, preorder
    int4 *node_c;
    int32_t *n_level, *n_first, *n_count, *n_parent, *n_nchild;
    int8_t *n_depth;

    // level order
    int32_t *bfs2pid, *pid2bfs;
    uint32_t *dhist;       // depth histogram per tile, scanned (NB_DEPTHS x tiles + 1)
    int64_t dtiles;
    int32_t *level_start;  // NB_DEPTHS + 1
    struct nb_wrec *wrec;  // one 64-byte record per node (see nb_wrec)
    double *b_mass, *b_mx, *b_com;  // FP64 moments in level order (mx, com: 3 per node)
    int32_t *arrive;                 // finished children per cell (bottom-up moments)
    int32_t *b_up;                   // parent's level-order index (-1 at a root)
    int32_t *lcount;                 // particle-leaf children per cell
    int16_t *cbkt;                   // moments bucket per node (-1 at a particle leaf)
    int32_t *cbkt_cnt;               // bucket sizes and fill cursors (2 x NB_CBKT)
    int32_t *clist;                  // cells by bucket, each bucket padded to 32 (-1)
    int64_t clist_len;

    // groups
    int32_t *gflag;   // per node flag, scanned in place to group ids (NN + 1)
    int32_t *gnode, *gfirst, *gcount, *glen, *gcells;
    float4 *gbox;     // 3 per group
    int32_t *items;   // force work items: (group, first member | one-warp-row flag)
    int item_rows;    // targets per item: 32 x item_rows (1 or 2)
    int force_tile;   // FP32 force: list records per staged tile (32 or 64; 0 = 32)
    int force_block;  // FP32 force: threads per block (256 or 128; 0 = 256)
    int32_t *item_cnt;
    int64_t max_items;
    int32_t *item_order;  // queue position -> item, costliest first (max_items)
    int32_t *item_bkt;    // cost-bucket sizes and fill cursors (2 x NB_IBKT)

    // learned opening angle: group features (16 floats) and theta per group
    float *gfeat, *gtheta;
    int32_t *gready;  // overlapped walk and force: a group's list is complete

    // device memory: one arena for every fixed-size array, one allocation
    // for the list storage (list_xm then list_id), one for the walk queues
    void *arena;
    size_t arena_bytes;
    void *list_mem;

    // lists
    int64_t list_cap;     // entries per group slot
    int64_t list_alloc;   // entries allocated
    int32_t *list_id;
    float4 *list_xm;

    // walk frontier queues
    int32_t *wq;
    int64_t wq_cap;       // entries per queue
    int walk_warps;       // warps the queues were sized for

    // leapfrog
    float *acc_cache, *pot_cache;

    // captured leapfrog steps
    cudaGraphExec_t graph_exec;

    // steps on host buffers: device copies of the state (one allocation, made
    // at the first such step), a copy stream and its two events
    void *hstage;
    cudaStream_t copy_stream;
    cudaEvent_t ev_drift, ev_copied;

    // timing and launch accounting
    int timing;
    int fused;               // leapfrog force passes use the fused walk and force
    int overlap;             // leapfrog force passes overlap the walk with the force sum
    int feature_mode;        // learned theta: 0 probe-walk features, 1 tree-only features
    int key_order;           // NB_ORDER_MORTON or NB_ORDER_HILBERT (next build)
    // quadrupole cells: traceless Q (xx, yy, zz, xy, xz, yz) about the centre
    // of mass per node in level order (FP64, allocated when first switched
    // on), and two float4 per list entry (Qxx, Qyy, Qzz, Qxy | Qxz, Qyz, 0, 0)
    int quad;
    int tree_quad;    // the current tree's moments include Q
    int lists_quad;   // the current lists carry Q (cells first in every chunk)
    double *b_q;
    float4 *list_q;
    int ev_used;
    int ev_graph;            // event pairs [0, ev_graph) are nodes of the captured graph
    int capturing;           // a graph capture is in progress on the stream
    int64_t graph_runs;      // graph launches since the last nb_get_timing
    int64_t graph_launches;  // kernels in one launch of the captured graph
    cudaEvent_t *ev;         // NB_EV_POOL pairs
    int *ev_phase;
    long long launches;

    // NB_DEBUG_SYNC=1: synchronise after every launch, report the first
    // kernel that failed (and the first self-check that fired)
    int debug_sync;
    const char *fail_site;

    // status
    unsigned int *err;
    long long *cnt;
    long long *cnt_host;  // pinned
};

// ---------------------------------------------------------------- kernels
// nb_sort.cu
void nb_exclusive_scan(nb_ctx *c, const int32_t *in, int32_t *out,
                       int64_t n_max, const long long *n_dev, long long *total_dev);
void nb_radix_sort(nb_ctx *c, int64_t n);
void nb_exclusive_scan_raw(const int32_t *in, int32_t *out, int64_t n_max, int32_t *bsum,
                           cudaStream_t s);
void nb_radix_sort_raw(uint64_t *keys, uint64_t *keys_alt, uint32_t *idx, uint32_t *idx_alt,
                       uint32_t *hist, int32_t *bsum, int64_t n, cudaStream_t s);
void nb_radix_sort_passes(uint64_t *keys, uint64_t *keys_alt, uint32_t *idx, uint32_t *idx_alt,
                          uint32_t *hist, int32_t *bsum, int64_t n, int passes, cudaStream_t s);

// nb_tree.cu
void nb_launch_keys_raw(const double *pos, int64_t n, double *part, int nblk, double *root,
                        uint64_t *keys, uint32_t *idx, unsigned *err, cudaStream_t s);
void nb_launch_build(nb_ctx *c, const double *pos, const float *mass, int64_t n);
void nb_launch_build_batched(nb_ctx *c, const double *pos, const float *mass, int64_t n,
                             const int64_t *offsets, int64_t nsys);
void nb_launch_groups(nb_ctx *c, float theta, int n_crit, const float *theta_g);

// nb_walk.cu
int nb_walk_warps(nb_ctx *c);
void nb_launch_walk(nb_ctx *c);
void nb_launch_probe(nb_ctx *c, float *feat);

// nb_mlp.cu
void nb_launch_mlp_infer(nb_ctx *c, const float *params, const float *feat, float *theta,
                         float fallback);

// nb_force.cu
void nb_launch_forces(nb_ctx *c, float eps, float *acc, float *pot, int precision);
void nb_launch_walk_force(nb_ctx *c, float eps, float *acc, float *pot, int precision);
int nb_launch_direct(const double *pos, const float *mass, int64_t n, double eps,
                     const int64_t *targets, int64_t nt, double *acc, double *pot,
                     cudaStream_t s);

// the overlapped walk and force (nb_api.cu)
extern "C" int nb_walk_forces(nb_ctx *c, float theta, int n_crit, float eps, float *acc,
                              float *pot, int precision);

// nb_neigh.cu
int nb_neigh_run(nb_ctx *c, double h, int n_crit, int64_t *off, int32_t *idx, int64_t cap,
                 int64_t *total);
// nb_api.cu helpers for synchronising calls in other units
int nb_read_err(nb_ctx *c, unsigned *bits);
int nb_err_code(unsigned bits);
int nb_grow_queues(nb_ctx *c);
double nb_root_side(nb_ctx *c);
#define CK_RET(call)                                                        \
    do {                                                                    \
        if ((call) != cudaSuccess) {                                        \
            cudaGetLastError();                                             \
            return NB_ERR_CUDA;                                             \
        }                                                                   \
    } while (0)

// nb_step.cu
void nb_launch_kick(nb_ctx *c, double *vel, const float *acc, int64_t n, double h);
void nb_launch_wait_probe(nb_ctx *c, unsigned limit);
void nb_launch_fused(nb_ctx *c, float eps, float *acc, float *pot, int precision);
void nb_launch_features_tree(nb_ctx *c, float *feat);
void nb_launch_group_theta(nb_ctx *c, const float *theta_g);
void nb_launch_drift(nb_ctx *c, double *pos, const double *vel, int64_t n, double dt);
void nb_launch_kick_kick_drift(nb_ctx *c, double *pos, double *vel, const float *acc,
                               int64_t n, double h, double dt);

__device__ __forceinline__ long long nb_atomic_add(long long *p, long long v)
{
    return (long long)atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

// A failed self-check: latch NB_EF_BOUNDS and the first site / index.  The
// caller skips the access.
static __device__ __forceinline__ void nb_bad(long long *cnt, unsigned *err, int site, long long idx)
{
    atomicOr(err, NB_EF_BOUNDS);
    if (atomicCAS((unsigned long long *)&cnt[CNT_BAD_SITE], 0ull, (unsigned long long)site) == 0ull)
        cnt[CNT_BAD_INDEX] = idx;
}
__device__ __forceinline__ bool nb_in(bool ok, long long *cnt, unsigned *err, int site,
                                      long long idx)
{
    if (!ok) nb_bad(cnt, err, site, idx);
    return ok;
}

// The lanes of the warp whose BITS-bit value v equals this lane's, from one
// ballot per bit (every lane calls it; a lane with ok false matches only
// itself and is left out of the others' masks).
template <int BITS>
static __device__ __forceinline__ unsigned nb_match_bits(unsigned v, bool ok)
{
    unsigned m = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int b = 0; b < BITS; b++) {
        const bool bit = (v >> b) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return ok ? m : (1u << (threadIdx.x & 31));
}

// Exclusive scan of one value per thread over a block of 256 threads
// (every thread calls it); *total gets the block's sum.
static __device__ __forceinline__ int32_t nb_block_scan256(int32_t v, int32_t *total)
{
    __shared__ int32_t nb_wsum[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) nb_wsum[w] = x;
    __syncthreads();
    int32_t pre = 0, all = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int32_t s = nb_wsum[k];
        pre += k < w ? s : 0;
        all += s;
    }
    __syncthreads();
    *total = all;
    return pre + x - v;
}

// after every kernel launch: count it; under NB_DEBUG_SYNC synchronise and
// report a failure by kernel name
void nb_launched(nb_ctx *c, const char *name);

// group-relative FP32 coordinate of a value carried as two floats (hi, lo):
// fl32(fl32(hi - c) + lo)
__device__ __forceinline__ float nb_rel(float hi, float lo, float c)
{
    return __fadd_rn(__fsub_rn(hi, c), lo);
}

static inline int nb_grid(int64_t n, int block, int cap = 1 << 20)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}
