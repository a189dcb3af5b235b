// nb_internal.cuh -- device-side layout shared by the libnb translation units.
//
// HBM layout (all per context, allocated once for max_n particles):
//   sorted particles  p_hi[N] float4 (x,y,z as the FP32 nearest to the FP64
//                     position, mass), p_lo[N] float4 (FP32 remainders),
//                     p_x64[3N] FP64 positions, perm[N] sorted slot -> caller
//   tree nodes        depth-first preorder over cells and particle leaves:
//                     node_a[NN] float4 (centre of mass hi part, mass)
//                     node_b[NN] float4 (centre of mass lo part, 0)
//                     node_c[NN] int4   (next, l bits, s bits, is_particle)
//                     plus FP64 moments and integer topology for export
//   groups            gnode/gfirst/gcount, gbox[3G] float4 (lo, hi,
//                     centre + 1/theta), list length / self offset
//   lists             list_id[G * cap] int32, list_xm[G * cap] float4
//                     (group-relative position, mass), slot g at g * cap
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nb.h"

#define NB_LEVELS 21
#define NB_EV_POOL 2048
#define NB_WARP 32

// bits of the device error word
#define NB_EF_NONFINITE 1u
#define NB_EF_CAPACITY 2u
#define NB_EF_WALK 4u

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
    CNT_PP_CUM,      // n_pp over every walk (never reset)
    CNT_PC_CUM,
    CNT_N_
};

struct nb_ctx {
    int device;
    cudaStream_t stream;
    int sync_checks;
    nb_config cfg;
    int num_sms;

    int64_t max_n;
    int64_t max_nodes;    // 12 * max_n + 2
    int64_t n;            // particles in the current tree
    int has_tree, has_lists, acc_valid;
    int n_crit_cur;
    int64_t groups_host;  // G of the last walk, when known on the host

    // sort
    uint64_t *keys, *keys_alt;
    uint32_t *idx, *idx_alt;
    uint32_t *sort_hist;
    int64_t sort_hist_len;

    // scan scratch
    int32_t *scan_bsum;
    int64_t scan_bsum_len;

    // root: centre[3], L, corner[3]; bbox partials
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

    // nodes
    float4 *node_a, *node_b;
    int4 *node_c;
    int32_t *n_level, *n_first, *n_count, *n_parent, *n_nchild, *n_arrive;
    double *n_mass, *n_mx, *n_com;  // FP64 moments (mx, com: 3 per node)

    // groups
    int32_t *gflag;   // per node flag, scanned in place to group ids (NN + 1)
    int32_t *gnode, *gfirst, *gcount, *glen, *gself, *gcells;
    float4 *gbox;     // 3 per group
    int32_t *items;   // force work items: (group, first member) pairs
    int32_t *item_cnt;
    int64_t max_items;

    // lists
    int64_t list_cap;     // entries per group slot
    int64_t list_alloc;   // entries allocated
    int32_t *list_id;
    float4 *list_xm;

    // leapfrog
    float *acc_cache, *pot_cache;

    // timing and launch accounting
    int timing;
    int ev_used;
    cudaEvent_t *ev;         // NB_EV_POOL pairs
    int *ev_phase;
    long long launches;

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

// nb_tree.cu
void nb_launch_keys_raw(const double *pos, int64_t n, double *part, int nblk, double *root,
                        uint64_t *keys, uint32_t *idx, unsigned *err, cudaStream_t s);
void nb_launch_build(nb_ctx *c, const double *pos, const float *mass, int64_t n);
void nb_launch_groups(nb_ctx *c, float theta, int n_crit, const float *theta_g);

// nb_walk.cu
void nb_launch_walk(nb_ctx *c);

// nb_force.cu
void nb_launch_forces(nb_ctx *c, float eps, float *acc, float *pot, int precision);
int nb_launch_direct(const double *pos, const float *mass, int64_t n, double eps,
                     const int64_t *targets, int64_t nt, double *acc, double *pot,
                     cudaStream_t s);

// nb_step.cu
void nb_launch_kick(nb_ctx *c, double *vel, const float *acc, int64_t n, double h);
void nb_launch_drift(nb_ctx *c, double *pos, const double *vel, int64_t n, double dt);

__device__ __forceinline__ long long nb_atomic_add(long long *p, long long v)
{
    return (long long)atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

static inline int nb_grid(int64_t n, int block, int cap = 1 << 20)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}
