// nb_api.cu -- the C ABI declared in include/nb.h: context and storage,
// argument checks, the order of kernel launches, status and debug export.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "nb_internal.cuh"

#define CK(call)                                                            \
    do {                                                                    \
        if ((call) != cudaSuccess) {                                        \
            cudaGetLastError();                                             \
            return NB_ERR_CUDA;                                             \
        }                                                                   \
    } while (0)

extern "C" {

void nb_config_default(nb_config *cfg, int64_t max_n)
{
    memset(cfg, 0, sizeof(*cfg));
    cfg->max_n = max_n;
    cfg->sync_checks = 1;
    cfg->eps = 0.01f;
    cfg->theta = 0.6f;
    cfg->n_crit = 64;
    cfg->precision = NB_FP32;
    cfg->max_systems = 1;
}

const char *nb_error_string(int code)
{
    switch (code) {
    case NB_OK: return "ok";
    case NB_ERR_INVALID_ARG: return "invalid argument";
    case NB_ERR_CUDA: return "CUDA runtime error";
    case NB_ERR_CAPACITY: return "interaction list capacity exceeded";
    case NB_ERR_WALK_LIMIT: return "tree walk did not advance";
    case NB_ERR_NONFINITE: return "non-finite position";
    case NB_ERR_STATE: return "call order: build the tree, then walk, then force";
    case NB_ERR_NOMEM: return "device allocation failed";
    case NB_ERR_INTERNAL: return "a kernel's bounds self-check fired";
    default: return "unknown error";
    }
}

}  // extern "C"

static void free_all(nb_ctx *c)
{
    // three device allocations: the context arena, the list storage, the
    // walk queues
    void *ptrs[] = {c->arena, c->list_mem, c->wq, c->hstage, c->b_q};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    c->arena = c->list_mem = c->hstage = nullptr;
    c->b_q = nullptr;
    c->list_q = nullptr;
    c->wq = nullptr;
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->ev_drift) cudaEventDestroy(c->ev_drift);
    if (c->ev_copied) cudaEventDestroy(c->ev_copied);
    c->copy_stream = nullptr;
    if (c->cnt_host) cudaFreeHost(c->cnt_host);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->ev) {
        for (int i = 0; i < 2 * NB_EV_POOL; i++) cudaEventDestroy(c->ev[i]);
        free(c->ev);
        free(c->ev_phase);
    }
}

// Device memory comes in whole 2 MiB units, each allocation made once and
// carved into 256-byte aligned arrays.
#define NB_ALLOC_UNIT ((size_t)2 << 20)

static size_t round_unit(size_t bytes)
{
    return (bytes + NB_ALLOC_UNIT - 1) / NB_ALLOC_UNIT * NB_ALLOC_UNIT;
}

static bool dmalloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (cudaMalloc(p, round_unit(bytes ? bytes : 1)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

// two passes over the same list of arrays: sizing (base == nullptr), then
// placing
struct Arena {
    char *base = nullptr;
    size_t off = 0;
    template <typename T>
    void carve(T **p, int64_t count)
    {
        if (count < 1) count = 1;
        off = (off + 255) & ~(size_t)255;
        *p = base ? (T *)(base + off) : nullptr;
        off += sizeof(T) * (size_t)count;
    }
};

static void carve_context(nb_ctx *c, Arena &a)
{
    const int64_t N = c->max_n, NN = c->max_nodes;
    a.carve(&c->keys, N);
    a.carve(&c->keys_alt, N);
    a.carve(&c->idx, N);
    a.carve(&c->idx_alt, N);
    a.carve(&c->sort_hist, c->sort_hist_len);
    a.carve(&c->rs_status, c->rs_status_len);
    a.carve(&c->scan_bsum, c->scan_bsum_len);
    a.carve(&c->bbox_part, 6 * (int64_t)c->bbox_blocks);
    a.carve(&c->root, 8 * c->max_sys);
    a.carve(&c->p_hi, N);
    a.carve(&c->p_lo, N);
    a.carve(&c->p_x64, 3 * N);
    a.carve(&c->perm, N);
    a.carve(&c->clev, N);
    a.carve(&c->ccount, N + 1);
    a.carve(&c->cstart, N + 1);
    a.carve(&c->node_c, NN);
    a.carve(&c->n_level, NN);
    a.carve(&c->n_first, NN);
    a.carve(&c->n_count, NN);
    a.carve(&c->n_parent, NN);
    a.carve(&c->n_nchild, NN);
    a.carve(&c->n_depth, NN);
    a.carve(&c->bfs2pid, NN);
    a.carve(&c->pid2bfs, NN);
    a.carve(&c->dhist, NB_DEPTHS * c->dtiles + 1);
    a.carve(&c->level_start, NB_DEPTHS + 1);
    a.carve(&c->wrec, NN);
    a.carve(&c->b_mass, NN);
    a.carve(&c->b_mx, 3 * NN);
    a.carve(&c->b_com, 3 * NN);
    a.carve(&c->arrive, NN);
    a.carve(&c->b_up, NN);
    a.carve(&c->lcount, NN);
    a.carve(&c->cbkt, NN);
    a.carve(&c->cbkt_cnt, 2 * NB_CBKT);
    a.carve(&c->clist, c->clist_len);
    a.carve(&c->gflag, NN + 1);
    a.carve(&c->gnode, N);
    a.carve(&c->gfirst, N);
    a.carve(&c->gcount, N);
    a.carve(&c->glen, N);
    a.carve(&c->gcells, N);
    a.carve(&c->gbox, 3 * N);
    a.carve(&c->gfeat, 16 * N);
    a.carve(&c->gtheta, N);
    a.carve(&c->gready, N);
    a.carve(&c->items, 2 * c->max_items);
    a.carve(&c->item_cnt, N + 1);
    a.carve(&c->item_order, c->max_items);
    a.carve(&c->item_bkt, 2 * NB_IBKT);
    a.carve(&c->acc_cache, 3 * N);
    a.carve(&c->pot_cache, N);
    a.carve(&c->err, 1);
    a.carve(&c->cnt, CNT_N_);
    if (c->max_sys > 1) {
        a.carve(&c->sys_of, N);
        a.carve(&c->sys_sorted, N);
        a.carve(&c->sys_root, c->max_sys);
        a.carve(&c->skey, N);
        a.carve(&c->skey_alt, N);
        a.carve(&c->sval, N);
        a.carve(&c->sval_alt, N);
    }
}

// A captured graph holds the device addresses of the list storage and the
// walk queues in its kernel nodes; once either is freed and allocated again,
// replaying it would touch freed memory.  Every such reallocation drops the
// graph (nb_graph_launch then returns NB_ERR_STATE until the next capture).
static void drop_graph(nb_ctx *c)
{
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
        c->graph_launches = 0;
        c->ev_graph = 0;
        c->graph_runs = 0;
    }
}

// walk queues: two frontier queues of wq_cap entries per warp
static bool alloc_queues(nb_ctx *c, int64_t wq_cap)
{
    drop_graph(c);
    if (c->wq) cudaFree(c->wq);
    c->wq = nullptr;
    c->wq_cap = 0;
    if (!dmalloc((void **)&c->wq, sizeof(int32_t) * 2 * (size_t)wq_cap * c->walk_warps))
        return false;
    c->wq_cap = wq_cap;
    return true;
}

static const char *const SITE_NAME[SITE_N_] = {
    "none", "k_gather: caller index", "k_cells: node id", "k_parents: child id",
    "k_depth_scatter: level-order position", "k_bfs_records: node or particle",
    "k_moments: cell, parent or child run", "groups: group or member range",
    "k_items: item index", "k_walk: queued node", "k_walk: child run", "k_force: item",
    "k_rs_scatter: destination", "k_moments: wait for children ran out",
    "k_rs_scatter: look-back wait ran out", "k_walk_force: wait for a group's walk ran out"};

static int err_code(unsigned bits)
{
    if (bits & NB_EF_BOUNDS) return NB_ERR_INTERNAL;
    if (bits & NB_EF_BADARG) return NB_ERR_INVALID_ARG;
    if (bits & NB_EF_NONFINITE) return NB_ERR_NONFINITE;
    if (bits & NB_EF_WALK) return NB_ERR_WALK_LIMIT;
    if (bits & (NB_EF_CAPACITY | NB_EF_QUEUE)) return NB_ERR_CAPACITY;
    return NB_OK;
}

static void report_bounds(nb_ctx *c)
{
    long long v[2] = {0, 0};
    if (cudaMemcpy(&c->cnt_host[CNT_BAD_SITE], &c->cnt[CNT_BAD_SITE], sizeof(v),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return;
    v[0] = c->cnt_host[CNT_BAD_SITE];
    v[1] = c->cnt_host[CNT_BAD_INDEX];
    const int site = (v[0] > 0 && v[0] < SITE_N_) ? (int)v[0] : 0;
    fprintf(stderr, "libnb: bounds self-check fired at %s (index %lld)\n", SITE_NAME[site], v[1]);
}

// synchronise, read and clear the device error word (through the pinned
// slot after the counters: no device-to-host copy into pageable memory)
static int sync_read_bits(nb_ctx *c, unsigned *bits)
{
    *bits = 0;
    unsigned *pinned = (unsigned *)&c->cnt_host[CNT_N_];
    CK(cudaMemcpyAsync(pinned, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *bits = *pinned;
    if (*bits & NB_EF_BOUNDS) report_bounds(c);
    if (*bits) CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    return NB_OK;
}

void nb_launched(nb_ctx *c, const char *name)
{
    c->launches++;
    if (!c->debug_sync) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    unsigned bits = 0;
    if (e == cudaSuccess) {
        unsigned *pinned = (unsigned *)&c->cnt_host[CNT_N_];
        e = cudaMemcpy(pinned, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost);
        bits = *pinned;
    }
    if (c->fail_site) return;
    if (e != cudaSuccess) {
        c->fail_site = name;
        fprintf(stderr, "libnb: %s failed: %s\n", name, cudaGetErrorString(e));
    } else if (bits & NB_EF_BOUNDS) {
        c->fail_site = name;
        fprintf(stderr, "libnb: after %s:\n", name);
        report_bounds(c);
    }
}

static int sync_read(nb_ctx *c)
{
    unsigned bits = 0;
    const int rc = sync_read_bits(c, &bits);
    return rc ? rc : err_code(bits);
}

static int read_counters(nb_ctx *c)
{
    CK(cudaMemcpyAsync(c->cnt_host, c->cnt, sizeof(long long) * CNT_N_,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NB_OK;
}

int nb_read_err(nb_ctx *c, unsigned *bits) { return sync_read_bits(c, bits); }
int nb_err_code(unsigned bits) { return err_code(bits); }

// double the walk queues past the widest frontier seen (synchronising)
int nb_grow_queues(nb_ctx *c)
{
    int rc = read_counters(c);
    if (rc) return rc;
    const int64_t want = 2 * (c->cnt_host[CNT_QMAX] > c->wq_cap ? c->cnt_host[CNT_QMAX] : c->wq_cap);
    CK(cudaStreamSynchronize(c->stream));
    return alloc_queues(c, want) ? NB_OK : NB_ERR_NOMEM;
}

// the largest root-cube side over the current tree's systems (synchronising)
double nb_root_side(nb_ctx *c)
{
    double L = 0.0;
    for (int64_t sy = 0; sy < c->nsys; sy++) {
        double v = 0.0;
        if (cudaMemcpy(&v, c->root + 8 * sy + 3, sizeof(double), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0.0;
        }
        if (v > L) L = v;
    }
    return L;
}

static int finish(nb_ctx *c)
{
    if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
    if (!c->sync_checks) return NB_OK;
    return sync_read(c);
}

// phase timing: a pair of events on the context's stream around each phase.
// Under stream capture an event must be recorded as external to become an
// event-record node that every launch of the graph records.
static void record_event(nb_ctx *c, cudaEvent_t e)
{
    if (c->capturing) cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
    else cudaEventRecord(e, c->stream);
}

static int phase_begin(nb_ctx *c)
{
    if (!c->timing || !c->ev || c->ev_graph + c->ev_used >= NB_EV_POOL) return -1;
    const int k = c->ev_graph + c->ev_used++;
    record_event(c, c->ev[2 * k]);
    return k;
}

static void phase_end(nb_ctx *c, int k, int phase)
{
    if (k < 0) return;
    record_event(c, c->ev[2 * k + 1]);
    c->ev_phase[k] = phase;
}

// List storage: list_xm (16 B) and list_id (4 B) per entry in one
// allocation with 1/8 headroom, replaced only when a walk needs more.
// In the quadrupole mode the same allocation also holds list_q (32 B per
// entry) after list_id.
static int ensure_lists(nb_ctx *c, int64_t groups, int64_t cap)
{
    const int64_t need = groups * cap;
    const bool want_q = c->quad && !c->list_q;
    if (need <= c->list_alloc && cap == c->list_cap && !want_q) return NB_OK;
    if (need > c->list_alloc || want_q) {
        CK(cudaStreamSynchronize(c->stream));
        drop_graph(c);
        if (c->list_mem) cudaFree(c->list_mem);
        c->list_mem = nullptr;
        c->list_id = nullptr;
        c->list_xm = nullptr;
        c->list_q = nullptr;
        c->list_alloc = 0;
        const int64_t want = need + need / 8;
        const size_t xm_bytes = (sizeof(float4) * (size_t)want + 255) & ~(size_t)255;
        const size_t id_bytes = (sizeof(int32_t) * (size_t)want + 255) & ~(size_t)255;
        const size_t q_bytes = c->quad ? 2 * sizeof(float4) * (size_t)want : 0;
        if (!dmalloc(&c->list_mem, xm_bytes + id_bytes + q_bytes)) return NB_ERR_NOMEM;
        c->list_xm = (float4 *)c->list_mem;
        c->list_id = (int32_t *)((char *)c->list_mem + xm_bytes);
        if (c->quad) c->list_q = (float4 *)((char *)c->list_mem + xm_bytes + id_bytes);
        c->list_alloc = want;
    }
    c->list_cap = cap;
    return NB_OK;
}

extern "C" {

int nb_create(nb_ctx **out, const nb_config *cfg)
{
    if (!out || !cfg) return NB_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_n < 1 || cfg->max_n > (int64_t)150000000 || cfg->n_crit < 1 ||
        !(cfg->theta >= 0.f) || !(cfg->eps >= 0.f) || cfg->precision < 0 ||
        cfg->precision > 2 || cfg->list_capacity < 0 || cfg->max_systems < 0)
        return NB_ERR_INVALID_ARG;
    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) return NB_ERR_NOMEM;
    memset(c, 0, sizeof(*c));
    c->cfg = *cfg;
    c->device = cfg->device;
    c->stream = (cudaStream_t)cfg->stream;
    c->sync_checks = cfg->sync_checks;
    if (cudaSetDevice(c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return NB_ERR_CUDA;
    }
    const int64_t N = cfg->max_n;
    const int64_t NN = 12 * N + 2;
    c->max_n = N;
    c->max_nodes = NN;
    const int64_t rs_tiles = (N + NB_RS_TILE - 1) / NB_RS_TILE;
    // the single-pass sort may use tiles down to NB_RS_TILE_MIN keys
    const int64_t rs_tiles_max = (N + NB_RS_TILE_MIN - 1) / NB_RS_TILE_MIN;
    c->sort_hist_len = 256 * rs_tiles + 1;
    c->rs_status_len = 8 * 256 * rs_tiles_max + 8 * 256 + 8;
    c->dtiles = (NN + NB_DS_TILE - 1) / NB_DS_TILE;
    const int64_t dhist_len = NB_DEPTHS * c->dtiles + 1;
    int64_t scan_n = NN + 1 > c->sort_hist_len ? NN + 1 : c->sort_hist_len;
    if (dhist_len > scan_n) scan_n = dhist_len;
    c->scan_bsum_len = (scan_n + 2047) / 2048 + 2;
    c->bbox_blocks = c->num_sms * 4;
    c->max_items = N + N / 64 + 2;
    c->clist_len = NN + 32 * (int64_t)NB_CBKT;
    c->max_sys = cfg->max_systems > 1 ? cfg->max_systems : 1;
    Arena sizing;
    carve_context(c, sizing);
    bool ok = dmalloc(&c->arena, sizing.off);
    if (ok) {
        Arena place;
        place.base = (char *)c->arena;
        carve_context(c, place);
        c->arena_bytes = round_unit(sizing.off);
    }
    ok = ok && cudaMallocHost((void **)&c->cnt_host, sizeof(long long) * (CNT_N_ + 1)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return NB_ERR_NOMEM;
    }
    if (cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->cnt, 0, sizeof(long long) * CNT_N_, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return NB_ERR_CUDA;
    }
    c->nsys = 1;
    c->item_rows = 2;
    {
        const char *dbg = getenv("NB_DEBUG_SYNC");
        c->debug_sync = dbg && dbg[0] && dbg[0] != '0';
        c->fail_site = nullptr;
    }

    c->list_cap = cfg->list_capacity;
    c->walk_warps = nb_walk_warps(c);
    if (!alloc_queues(c, N >= (1 << 20) ? 8192 : 4096)) {
        free_all(c);
        delete c;
        return NB_ERR_NOMEM;
    }
    *out = c;
    return NB_OK;
}

int nb_destroy(nb_ctx *c)
{
    if (!c) return NB_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return NB_OK;
}

int nb_set_sync_checks(nb_ctx *c, int on)
{
    if (!c) return NB_ERR_INVALID_ARG;
    c->sync_checks = on ? 1 : 0;
    return NB_OK;
}

int nb_build_tree(nb_ctx *c, const double *pos, const float *mass, int64_t n)
{
    if (!c || n < 0 || n > c->max_n || (n > 0 && (!pos || !mass))) return NB_ERR_INVALID_ARG;
    c->has_tree = 0;
    c->has_groups = 0;
    c->has_lists = 0;
    c->n = n;
    c->nsys = 1;
    c->tree_quad = c->quad && c->b_q;
    if (n == 0) {
        CK(cudaMemsetAsync(c->cnt, 0, sizeof(long long) * CNT_PP_CUM, c->stream));
        c->has_tree = 1;
        return finish(c);
    }
    const int tk = phase_begin(c);
    nb_launch_build(c, pos, mass, n);
    phase_end(c, tk, NB_PHASE_BUILD);
    c->has_tree = 1;
    return finish(c);
}

int nb_build_tree_batched(nb_ctx *c, const double *pos, const float *mass,
                          const int64_t *offsets, int64_t nsys, int64_t n)
{
    if (!c || n < 1 || n > c->max_n || nsys < 1 || nsys > c->max_sys || nsys > n || !pos ||
        !mass || !offsets)
        return NB_ERR_INVALID_ARG;
    c->has_tree = 0;
    c->has_groups = 0;
    c->has_lists = 0;
    c->n = n;
    c->nsys = nsys;
    c->sys_off = offsets;
    c->tree_quad = c->quad && c->b_q;
    const int tk = phase_begin(c);
    if (nsys == 1) nb_launch_build(c, pos, mass, n);
    else nb_launch_build_batched(c, pos, mass, n, offsets, nsys);
    phase_end(c, tk, NB_PHASE_BUILD);
    c->has_tree = 1;
    return finish(c);
}

// the walk over groups of n_crit; `formed`: the groups (and their items)
// are already in place and only each box's 1/theta is set from theta_g
static int walk_groups(nb_ctx *c, float theta, int n_crit, const float *theta_g, bool formed)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->has_tree || (c->quad && !c->tree_quad)) return NB_ERR_STATE;
    if (!(theta >= 0.f) || n_crit < 1) return NB_ERR_INVALID_ARG;
    c->has_lists = 0;
    c->n_crit_cur = n_crit;
    if (c->n == 0) {
        c->groups_host = 0;
        c->has_lists = 1;
        c->lists_quad = c->quad;
        return NB_OK;
    }
    const int tk = phase_begin(c);
    if (formed) nb_launch_group_theta(c, theta_g);
    else nb_launch_groups(c, theta, n_crit, theta_g);
    c->has_groups = 1;
    if (c->sync_checks) {
        int rc = read_counters(c);
        if (rc) return rc;
        const int64_t G = c->cnt_host[CNT_GROUPS];
        c->groups_host = G;
        // With no list storage yet, the first pass only counts (nothing is
        // written), so the storage is allocated once at its measured size.
        int64_t cap = c->list_cap > 0 ? c->list_cap : 0;
        if (c->list_alloc == 0 && c->cfg.list_capacity <= 0) cap = 0;
        for (int attempt = 0; attempt < 6; attempt++) {
            const bool counting = cap == 0;
            if (counting) {
                c->list_cap = 0;
            } else {
                rc = ensure_lists(c, G, cap);
                if (rc) return rc;
            }
            nb_launch_walk(c);
            if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
            unsigned bits = 0;
            rc = sync_read_bits(c, &bits);
            if (rc) return rc;
            rc = err_code(bits);
            if (rc != NB_OK && rc != NB_ERR_CAPACITY) break;
            if (rc == NB_OK && !counting) break;
            rc = read_counters(c);
            if (rc) return rc;
            if (bits & NB_EF_QUEUE) {   // a frontier outgrew the walk queues
                const int64_t want = 2 * (c->cnt_host[CNT_QMAX] > c->wq_cap ? c->cnt_host[CNT_QMAX]
                                                                            : c->wq_cap);
                CK(cudaStreamSynchronize(c->stream));
                if (!alloc_queues(c, want)) return NB_ERR_NOMEM;
            } else if (counting || (bits & NB_EF_CAPACITY)) {
                if (!counting && c->cfg.list_capacity > 0) return NB_ERR_CAPACITY;
                const int64_t need = c->cnt_host[CNT_LIST_MAX];
                cap = ((need + need / 4 + 255) / 256) * 256;
                if (cap < 256) cap = 256;
            }
            rc = NB_ERR_CAPACITY;
        }
        phase_end(c, tk, NB_PHASE_WALK);
        if (rc) return rc;
    } else {
        if (c->list_cap < 1 || !c->list_id || !c->wq || (c->quad && !c->list_q))
            return NB_ERR_CAPACITY;
        nb_launch_walk(c);
        phase_end(c, tk, NB_PHASE_WALK);
        int rc = finish(c);
        if (rc) return rc;
    }
    c->has_lists = 1;
    c->lists_quad = c->quad;
    return NB_OK;
}

// the probe walk over groups formed with theta = NB_PROBE_THETA; in the
// synchronising mode a frontier that outgrows the walk queues grows them
int nb_walk_groups(nb_ctx *c, float theta, int n_crit, const float *theta_g)
{
    return walk_groups(c, theta, n_crit, theta_g, false);
}

static int probe(nb_ctx *c, int n_crit)
{
    nb_launch_groups(c, NB_PROBE_THETA, n_crit, nullptr);
    if (c->feature_mode == 1) {   // tree-only features: no walk
        nb_launch_features_tree(c, c->gfeat);
        return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
    }
    for (int attempt = 0; attempt < 4; attempt++) {
        nb_launch_probe(c, c->gfeat);
        if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
        if (!c->sync_checks) return NB_OK;
        unsigned bits = 0;
        int rc = sync_read_bits(c, &bits);
        if (rc) return rc;
        if (!(bits & NB_EF_QUEUE)) return err_code(bits);
        rc = read_counters(c);
        if (rc) return rc;
        const int64_t want = 2 * (c->cnt_host[CNT_QMAX] > c->wq_cap ? c->cnt_host[CNT_QMAX] : c->wq_cap);
        CK(cudaStreamSynchronize(c->stream));
        if (!alloc_queues(c, want)) return NB_ERR_NOMEM;
    }
    return NB_ERR_CAPACITY;
}

int nb_group_features(nb_ctx *c, int n_crit, float *feat, int64_t cap_rows, int64_t *n_groups)
{
    if (!c || n_crit < 1 || cap_rows < 0) return NB_ERR_INVALID_ARG;
    if (!c->has_tree) return NB_ERR_STATE;
    c->has_lists = 0;
    if (c->n == 0) {
        if (n_groups) *n_groups = 0;
        return NB_OK;
    }
    int rc = probe(c, n_crit);
    if (rc) return rc;
    c->has_groups = 1;
    if (n_groups || (feat && cap_rows > 0)) {
        rc = read_counters(c);
        if (rc) return rc;
        const int64_t G = c->cnt_host[CNT_GROUPS];
        if (n_groups) *n_groups = G;
        const int64_t rows = G < cap_rows ? G : cap_rows;
        if (feat && rows > 0)
            CK(cudaMemcpyAsync(feat, c->gfeat, sizeof(float) * 16 * rows, cudaMemcpyDeviceToDevice,
                               c->stream));
    }
    return finish(c);
}

int nb_walk_groups_learned(nb_ctx *c, int n_crit, const float *params, float fallback,
                           float *theta_out)
{
    if (!c || !params || n_crit < 1 || !(fallback >= 0.f)) return NB_ERR_INVALID_ARG;
    if (!c->has_tree) return NB_ERR_STATE;
    if (c->n == 0) return nb_walk_groups(c, fallback, n_crit, nullptr);
    // the probe walk and the network count as part of the walk phase
    const int tk = phase_begin(c);
    int rc = probe(c, n_crit);
    if (rc) return rc;
    nb_launch_mlp_infer(c, params, c->gfeat, c->gtheta, fallback);
    phase_end(c, tk, NB_PHASE_WALK);
    if (theta_out) {
        // group count is known on the device only; copy the whole slot range
        CK(cudaMemcpyAsync(theta_out, c->gtheta, sizeof(float) * c->n, cudaMemcpyDeviceToDevice,
                           c->stream));
    }
    // the feature pass formed these groups: only their 1/theta changes
    return walk_groups(c, fallback, n_crit, c->gtheta, true);
}

int nb_forces(nb_ctx *c, float eps, float *acc, float *pot, int precision)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->has_lists || (c->quad && !c->lists_quad)) return NB_ERR_STATE;
    if (!(eps >= 0.f) || precision < 0 || precision > 2 || (c->n > 0 && !acc) ||
        (c->quad && precision == NB_FP64ACC))
        return NB_ERR_INVALID_ARG;
    if (c->n == 0) return NB_OK;
    const int tk = phase_begin(c);
    nb_launch_forces(c, eps, acc, pot, precision);
    phase_end(c, tk, NB_PHASE_FORCE);
    return finish(c);
}

int nb_forces_fused(nb_ctx *c, float theta, int n_crit, float eps, float *acc, float *pot,
                    int precision)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (!(theta >= 0.f) || n_crit < 1 || !(eps >= 0.f) || precision < 0 || precision > 2 ||
        (c->n > 0 && !acc) || c->quad)
        return NB_ERR_INVALID_ARG;
    if (!c->has_tree) return NB_ERR_STATE;
    c->has_lists = 0;   // the fused pass leaves no lists behind
    if (c->n == 0) return NB_OK;
    const int tk = phase_begin(c);
    nb_launch_groups(c, theta, n_crit, nullptr);
    c->has_groups = 1;
    if (!c->wq) {
        CK(cudaStreamSynchronize(c->stream));
        if (!alloc_queues(c, c->wq_cap > 0 ? c->wq_cap : 4096)) return NB_ERR_NOMEM;
    }
    int rc = NB_OK;
    for (int attempt = 0; attempt < 4; attempt++) {
        nb_launch_fused(c, eps, acc, pot, precision);
        if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
        if (!c->sync_checks) break;
        unsigned bits = 0;
        rc = sync_read_bits(c, &bits);
        if (rc) return rc;
        rc = err_code(bits);
        if (!(bits & NB_EF_QUEUE)) break;
        // a frontier outgrew the walk queues: grow them and sum again
        rc = read_counters(c);
        if (rc) return rc;
        const int64_t want = 2 * (c->cnt_host[CNT_QMAX] > c->wq_cap ? c->cnt_host[CNT_QMAX]
                                                                    : c->wq_cap);
        CK(cudaStreamSynchronize(c->stream));
        if (!alloc_queues(c, want)) return NB_ERR_NOMEM;
        rc = NB_ERR_CAPACITY;
    }
    phase_end(c, tk, NB_PHASE_FORCE);
    if (rc) return rc;
    return finish(c);
}

int nb_leapfrog_reset(nb_ctx *c)
{
    if (!c) return NB_ERR_INVALID_ARG;
    c->acc_valid = 0;
    return NB_OK;
}

int nb_leapfrog_acc(nb_ctx *c, float *acc)
{
    if (!c || !acc) return NB_ERR_INVALID_ARG;
    if (!c->acc_valid) return NB_ERR_STATE;
    CK(cudaMemcpyAsync(acc, c->acc_cache, sizeof(float) * 3 * (size_t)c->n,
                       cudaMemcpyDeviceToDevice, c->stream));
    return finish(c);
}

static int force_pass(nb_ctx *c, const double *pos, const float *mass, int64_t n,
                      const int64_t *off = nullptr, int64_t nsys = 1)
{
    int rc = off ? nb_build_tree_batched(c, pos, mass, off, nsys, n) : nb_build_tree(c, pos, mass, n);
    if (rc) return rc;
    if (c->fused)
        return nb_forces_fused(c, c->cfg.theta, c->cfg.n_crit, c->cfg.eps, c->acc_cache,
                               c->pot_cache, c->cfg.precision);
    if (c->overlap && !c->quad && c->cfg.precision != NB_FP64ACC)
        return nb_walk_forces(c, c->cfg.theta, c->cfg.n_crit, c->cfg.eps, c->acc_cache,
                              c->pot_cache, c->cfg.precision);
    rc = nb_walk_groups(c, c->cfg.theta, c->cfg.n_crit, nullptr);
    if (rc) return rc;
    return nb_forces(c, c->cfg.eps, c->acc_cache, c->pot_cache, c->cfg.precision);
}

int nb_set_feature_mode(nb_ctx *c, int mode)
{
    if (!c || mode < 0 || mode > 1) return NB_ERR_INVALID_ARG;
    c->feature_mode = mode;
    return NB_OK;
}

int nb_set_key_order(nb_ctx *c, int order)
{
    if (!c || (order != NB_ORDER_MORTON && order != NB_ORDER_HILBERT)) return NB_ERR_INVALID_ARG;
    if (order != c->key_order) c->acc_valid = 0;   // the kept a(x) was summed in the old order
    c->key_order = order;
    return NB_OK;
}

int nb_set_quadrupole(nb_ctx *c, int on)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (on && !c->b_q) {
        CK(cudaStreamSynchronize(c->stream));
        if (!dmalloc((void **)&c->b_q, sizeof(double) * 6 * (size_t)c->max_nodes))
            return NB_ERR_NOMEM;
    }
    if ((on ? 1 : 0) != c->quad) c->acc_valid = 0;
    c->quad = on ? 1 : 0;
    return NB_OK;
}

int nb_copy_quadrupoles(nb_ctx *c, double *q_host)
{
    if (!c || !q_host) return NB_ERR_INVALID_ARG;
    if (!c->has_tree || !c->tree_quad) return NB_ERR_STATE;
    int rc = read_counters(c);
    if (rc) return rc;
    const int64_t nn = c->n > 0 ? c->cnt_host[CNT_NODES] : 0;
    double *qb = (double *)malloc(sizeof(double) * 6 * (size_t)(nn > 0 ? nn : 1));
    int32_t *map = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1));
    if (!qb || !map) rc = NB_ERR_NOMEM;
    if (!rc && nn > 0 &&
        (cudaMemcpy(qb, c->b_q, sizeof(double) * 6 * (size_t)nn, cudaMemcpyDeviceToHost) !=
             cudaSuccess ||
         cudaMemcpy(map, c->pid2bfs, sizeof(int32_t) * (size_t)nn, cudaMemcpyDeviceToHost) !=
             cudaSuccess))
        rc = NB_ERR_CUDA;
    for (int64_t u = 0; !rc && u < nn; u++) {
        const int32_t b = map[u];
        if (b < 0 || b >= nn) {
            rc = NB_ERR_INTERNAL;
            break;
        }
        for (int k = 0; k < 6; k++) q_host[6 * u + k] = qb[6 * (int64_t)b + k];
    }
    free(qb);
    free(map);
    return rc;
}

int nb_neighbours(nb_ctx *c, double h, int n_crit, int64_t *off_dev, int32_t *idx_dev,
                  int64_t cap, int64_t *total_host)
{
    if (!c || !(h >= 0.0) || !isfinite(h) || n_crit < 1 || !off_dev || !total_host || cap < 0)
        return NB_ERR_INVALID_ARG;
    if (!c->has_tree) return NB_ERR_STATE;
    c->has_lists = 0;   // the search forms its own groups and leaves no lists
    c->has_groups = 0;
    *total_host = 0;
    if (c->n == 0) {
        CK(cudaMemsetAsync(off_dev, 0, sizeof(int64_t), c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return NB_OK;
    }
    int rc = sync_read(c);   // start from a clear error word
    if (rc) return rc;
    rc = nb_neigh_run(c, h, n_crit, off_dev, idx_dev, cap, total_host);
    if (rc == NB_OK) c->has_groups = 1;
    return rc;
}

int nb_walk_forces(nb_ctx *c, float theta, int n_crit, float eps, float *acc, float *pot,
                   int precision)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (!(theta >= 0.f) || n_crit < 1 || !(eps >= 0.f) ||
        (precision != NB_FP32 && precision != NB_FP32_COMP) || (c->n > 0 && !acc) || c->quad)
        return NB_ERR_INVALID_ARG;
    if (!c->has_tree) return NB_ERR_STATE;
    // no list storage yet (or it is too small, found by a synchronising
    // call): the separate walk sizes it, then the separate force sum
    if (c->list_cap < 1 || !c->list_id || !c->wq) {
        if (!c->sync_checks) return NB_ERR_CAPACITY;
        int rc = nb_walk_groups(c, theta, n_crit, nullptr);
        if (rc) return rc;
        return nb_forces(c, eps, acc, pot, precision);
    }
    c->has_lists = 0;
    c->n_crit_cur = n_crit;
    if (c->n == 0) {
        c->groups_host = 0;
        c->has_lists = 1;
        c->lists_quad = 0;
        return NB_OK;
    }
    int tk = phase_begin(c);
    nb_launch_groups(c, theta, n_crit, nullptr);
    phase_end(c, tk, NB_PHASE_WALK);
    c->has_groups = 1;
    tk = phase_begin(c);
    nb_launch_walk_force(c, eps, acc, pot, precision);
    phase_end(c, tk, NB_PHASE_FORCE);
    if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
    c->has_lists = 1;
    c->lists_quad = 0;
    if (!c->sync_checks) return NB_OK;
    unsigned bits = 0;
    int rc = sync_read_bits(c, &bits);
    if (rc) return rc;
    if (bits & (NB_EF_CAPACITY | NB_EF_QUEUE)) {
        // a list outgrew its slot or a frontier the queues: the separate,
        // synchronising walk grows the storage, then the force sum again
        rc = nb_walk_groups(c, theta, n_crit, nullptr);
        if (rc) return rc;
        return nb_forces(c, eps, acc, pot, precision);
    }
    return err_code(bits);
}

int nb_set_overlap(nb_ctx *c, int on)
{
    if (!c) return NB_ERR_INVALID_ARG;
    c->overlap = on ? 1 : 0;
    return NB_OK;
}

int nb_set_fused(nb_ctx *c, int on)
{
    if (!c) return NB_ERR_INVALID_ARG;
    c->fused = on ? 1 : 0;
    return NB_OK;
}

// pos_out: host buffer that receives the positions as soon as the drift has
// written them, copied on the copy stream while the step goes on (host steps).
// Within a captured sequence of steps, a step may leave its second kick owed
// (owe_kick) and the next one pay it (kick_owed) in the same pass as its own
// first kick and drift: the same operations in the same order.
static int leapfrog(nb_ctx *c, double *pos, double *vel, const float *mass, int64_t n,
                    double dt, const int64_t *off, int64_t nsys, double *pos_out = nullptr,
                    bool kick_owed = false, bool owe_kick = false)
{
    if (!c || n < 0 || n > c->max_n || (n > 0 && (!pos || !vel || !mass)) || !isfinite(dt))
        return NB_ERR_INVALID_ARG;
    if (n == 0) return NB_OK;
    int rc;
    if (!c->acc_valid || c->n != n) {
        rc = force_pass(c, pos, mass, n, off, nsys);
        if (rc) return rc;
        c->acc_valid = 1;
    }
    const double h = 0.5 * dt;
    int tk = phase_begin(c);
    if (kick_owed) {
        nb_launch_kick_kick_drift(c, pos, vel, c->acc_cache, n, h, dt);
    } else {
        nb_launch_kick(c, vel, c->acc_cache, n, h);
        nb_launch_drift(c, pos, vel, n, dt);
    }
    phase_end(c, tk, NB_PHASE_INTEGRATE);
    if (pos_out) {
        CK(cudaEventRecord(c->ev_drift, c->stream));
        CK(cudaStreamWaitEvent(c->copy_stream, c->ev_drift, 0));
        CK(cudaMemcpyAsync(pos_out, pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                           c->copy_stream));
        CK(cudaEventRecord(c->ev_copied, c->copy_stream));
    }
    rc = force_pass(c, pos, mass, n, off, nsys);
    if (rc) {
        c->acc_valid = 0;
        return rc;
    }
    if (!owe_kick) {
        tk = phase_begin(c);
        nb_launch_kick(c, vel, c->acc_cache, n, h);
        phase_end(c, tk, NB_PHASE_INTEGRATE);
    }
    return finish(c);
}

int nb_leapfrog_step(nb_ctx *c, double *pos, double *vel, const float *mass, int64_t n,
                     double dt)
{
    return leapfrog(c, pos, vel, mass, n, dt, nullptr, 1);
}

int nb_leapfrog_step_host(nb_ctx *c, double *pos_host, double *vel_host, const float *mass_host,
                          int64_t n, double dt)
{
    if (!c || n < 0 || n > c->max_n || (n > 0 && (!pos_host || !vel_host || !mass_host)) ||
        !isfinite(dt))
        return NB_ERR_INVALID_ARG;
    if (n == 0) return NB_OK;
    if (!c->copy_stream) {
        if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
            return NB_ERR_CUDA;
        if (cudaEventCreateWithFlags(&c->ev_drift, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming) != cudaSuccess)
            return NB_ERR_CUDA;
    }
    if (!c->hstage) {   // device copies of the state, for max_n particles
        CK(cudaStreamSynchronize(c->stream));
        if (!dmalloc(&c->hstage, (sizeof(double) * 6 + sizeof(float)) * (size_t)c->max_n))
            return NB_ERR_NOMEM;
    }
    double *pos = (double *)c->hstage;
    double *vel = pos + 3 * c->max_n;
    float *mass = (float *)(vel + 3 * c->max_n);
    CK(cudaMemcpyAsync(vel, vel_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(pos, pos_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(mass, mass_host, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
    // positions leave on the copy stream right after the drift; velocities
    // after the closing kick; the stream then waits for both
    const int rc = leapfrog(c, pos, vel, mass, n, dt, nullptr, 1, pos_host);
    if (rc) {
        cudaStreamSynchronize(c->copy_stream);
        return rc;
    }
    CK(cudaMemcpyAsync(vel_host, vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamWaitEvent(c->stream, c->ev_copied, 0));
    return finish(c);
}

int nb_leapfrog_step_batched(nb_ctx *c, double *pos, double *vel, const float *mass,
                             const int64_t *offsets, int64_t nsys, int64_t n, double dt)
{
    if (!offsets || nsys < 1) return NB_ERR_INVALID_ARG;
    return leapfrog(c, pos, vel, mass, n, dt, offsets, nsys);
}

int nb_graph_capture_leapfrog(nb_ctx *c, double *pos, double *vel, const float *mass,
                              const int64_t *offsets, int64_t nsys, int64_t n, double dt,
                              int nsteps)
{
    if (!c || !c->stream || nsteps < 1 || n < 1 || (offsets && nsys < 1)) return NB_ERR_INVALID_ARG;
    if (!c->acc_valid || c->n != n || (!c->fused && (c->list_cap < 1 || !c->list_id)))
        return NB_ERR_STATE;
    CK(cudaStreamSynchronize(c->stream));
    const int sync = c->sync_checks;
    c->sync_checks = 0;
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    // with timing on, the phase events become event-record nodes of the
    // graph (pairs [0, ev_graph) of the pool), recorded again by every launch;
    // eager phases recorded before the capture are dropped
    c->ev_graph = 0;
    c->ev_used = 0;
    c->graph_runs = 0;
    const int64_t launches0 = c->launches;
    int rc = NB_OK;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = NB_ERR_CUDA;
    } else {
        c->capturing = 1;
        // the second kick of each step but the last is paid with the next
        // step's first kick and drift
        for (int k = 0; k < nsteps && rc == NB_OK; k++)
            rc = leapfrog(c, pos, vel, mass, n, dt, offsets, offsets ? nsys : 1, nullptr, k > 0,
                          k + 1 < nsteps);
        c->capturing = 0;
        if (cudaStreamEndCapture(c->stream, &graph) != cudaSuccess && rc == NB_OK) rc = NB_ERR_CUDA;
        if (rc == NB_OK && cudaGraphInstantiate(&c->graph_exec, graph, 0) != cudaSuccess)
            rc = NB_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    c->sync_checks = sync;
    c->graph_launches = c->launches - launches0;
    c->launches = launches0;   // the captured kernels count when the graph runs
    if (rc) {
        cudaGetLastError();
        c->graph_exec = nullptr;
        c->ev_used = 0;
        c->graph_launches = 0;
    } else {
        c->ev_graph = c->ev_used;
        c->ev_used = 0;
    }
    return rc;
}

int nb_graph_launch(nb_ctx *c)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->graph_exec) return NB_ERR_STATE;
    CK(cudaGraphLaunch(c->graph_exec, c->stream));
    c->graph_runs++;
    c->launches += c->graph_launches;
    return finish(c);
}

int nb_autotune(nb_ctx *c, const double *pos, const float *mass, const int64_t *offsets,
                int64_t nsys, int64_t n, float eps, float theta, const int *n_crit, int ncand,
                int reps, int *best_n_crit, int *best_rows, int *best_tile, int *best_block,
                float *ms_out)
{
    if (!c || !pos || !mass || !n_crit || ncand < 1 || reps < 1 || n < 1) return NB_ERR_INVALID_ARG;
    int rc = offsets ? nb_build_tree_batched(c, pos, mass, offsets, nsys, n)
                     : nb_build_tree(c, pos, mass, n);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int sync = c->sync_checks, rows0 = c->item_rows;
    const int tile0 = c->force_tile, block0 = c->force_block;
    const int tiles[2] = {32, 64}, blocks[2] = {256, 128};
    float best = INFINITY;
    int bn = n_crit[0], br = rows0, bt = 32, bb = 256;
    for (int k = 0; k < ncand && rc == NB_OK; k++)
        for (int rows = 1; rows <= 2 && rc == NB_OK; rows++)
            for (int ti = 0; ti < 2 && rc == NB_OK; ti++)
                for (int bi = 0; bi < 2 && rc == NB_OK; bi++) {
                    c->item_rows = rows;
                    c->force_tile = tiles[ti];
                    c->force_block = blocks[bi];
                    c->sync_checks = 1;
                    rc = nb_walk_groups(c, theta, n_crit[k], nullptr);   // sizes the lists
                    if (rc) break;
                    rc = nb_forces(c, eps, c->acc_cache, nullptr, NB_FP32);
                    if (rc) break;
                    c->sync_checks = 0;
                    cudaEventRecord(e0, c->stream);
                    for (int r = 0; r < reps && rc == NB_OK; r++) {
                        rc = nb_walk_groups(c, theta, n_crit[k], nullptr);
                        if (!rc) rc = nb_forces(c, eps, c->acc_cache, nullptr, NB_FP32);
                    }
                    cudaEventRecord(e1, c->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess) rc = NB_ERR_CUDA;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= reps;
                    if (ms_out) ms_out[((k * 2 + rows - 1) * 2 + ti) * 2 + bi] = ms;
                    if (ms < best) {
                        best = ms;
                        bn = n_crit[k];
                        br = rows;
                        bt = tiles[ti];
                        bb = blocks[bi];
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->sync_checks = sync;
    if (rc) {
        c->item_rows = rows0;
        c->force_tile = tile0;
        c->force_block = block0;
        return rc;
    }
    c->item_rows = br;
    c->force_tile = bt;
    c->force_block = bb;
    c->cfg.n_crit = bn;
    c->acc_valid = 0;
    if (best_n_crit) *best_n_crit = bn;
    if (best_rows) *best_rows = br;
    if (best_tile) *best_tile = bt;
    if (best_block) *best_block = bb;
    return sync_read(c);
}

int nb_direct_sum(const double *pos, const float *mass, int64_t n, double eps,
                  const int64_t *targets, int64_t nt, double *acc, double *pot, void *stream)
{
    if (n < 0 || nt < 0 || !(eps >= 0.0) || (n > 0 && (!pos || !mass)) ||
        (nt > 0 && (!acc || !pot)))
        return NB_ERR_INVALID_ARG;
    if (!targets && nt > n) return NB_ERR_INVALID_ARG;
    if (nb_launch_direct(pos, mass, n, eps, targets, nt, acc, pot, (cudaStream_t)stream))
        return NB_ERR_CUDA;
    return NB_OK;
}

int nb_set_timing(nb_ctx *c, int on)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (on && !c->ev) {
        c->ev = (cudaEvent_t *)calloc(2 * NB_EV_POOL, sizeof(cudaEvent_t));
        c->ev_phase = (int *)calloc(NB_EV_POOL, sizeof(int));
        if (!c->ev || !c->ev_phase) return NB_ERR_NOMEM;
        for (int i = 0; i < 2 * NB_EV_POOL; i++) CK(cudaEventCreate(&c->ev[i]));
    }
    c->timing = on ? 1 : 0;
    return NB_OK;
}

int nb_get_timing(nb_ctx *c, double *ms, int64_t *calls, int64_t *launches)
{
    if (!c) return NB_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(c->stream));
    double t[NB_NPHASE] = {0, 0, 0, 0};
    int64_t k[NB_NPHASE] = {0, 0, 0, 0};
    // the graph's events hold its last launch: scaled by the launches since
    // the last call
    if (c->graph_runs > 0)
        for (int i = 0; i < c->ev_graph; i++) {
            float e = 0.f;
            CK(cudaEventElapsedTime(&e, c->ev[2 * i], c->ev[2 * i + 1]));
            t[c->ev_phase[i]] += (double)e * (double)c->graph_runs;
            k[c->ev_phase[i]] += c->graph_runs;
        }
    c->graph_runs = 0;
    for (int i = c->ev_graph; i < c->ev_graph + c->ev_used; i++) {
        float e = 0.f;
        CK(cudaEventElapsedTime(&e, c->ev[2 * i], c->ev[2 * i + 1]));
        t[c->ev_phase[i]] += e;
        k[c->ev_phase[i]]++;
    }
    c->ev_used = 0;
    for (int p = 0; p < NB_NPHASE; p++) {
        if (ms) ms[p] = t[p];
        if (calls) calls[p] = k[p];
    }
    if (launches) *launches = c->launches;
    c->launches = 0;
    return NB_OK;
}

int nb_sync_status(nb_ctx *c)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
    return sync_read(c);
}

int nb_selftest_wait(nb_ctx *c, unsigned spin_limit)
{
    if (!c) return NB_ERR_INVALID_ARG;
    int rc = sync_read(c);   // start from a clear error word
    if (rc) return rc;
    nb_launch_wait_probe(c, spin_limit);
    if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
    rc = sync_read(c);
    // the probe's report is not a failure of the tree: clear the latched site
    CK(cudaMemsetAsync(&c->cnt[CNT_BAD_SITE], 0, 2 * sizeof(long long), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return rc;
}

int nb_get_stats(nb_ctx *c, nb_stats *st)
{
    if (!c || !st) return NB_ERR_INVALID_ARG;
    int rc = read_counters(c);
    if (rc) return rc;
    const long long *h = c->cnt_host;
    memset(st, 0, sizeof(*st));
    st->n = c->n;
    st->n_cells = c->n > 0 ? h[CNT_CELLS] : 0;
    st->n_nodes = c->n > 0 ? h[CNT_NODES] : 0;
    st->n_groups = c->has_groups && c->n > 0 ? h[CNT_GROUPS] : 0;
    st->list_entries = h[CNT_LIST_TOT];
    st->max_list = h[CNT_LIST_MAX];
    st->list_capacity = c->list_cap;
    st->n_pp = h[CNT_PP];
    st->n_pc = h[CNT_PC];
    st->max_level = (int32_t)h[CNT_MAXLEVEL];
    st->n_pp_total = h[CNT_PP_CUM];
    st->n_pc_total = h[CNT_PC_CUM];
    return NB_OK;
}

#define D2H(dst, src, count)                                                              \
    do {                                                                                  \
        if (dst) CK(cudaMemcpyAsync(dst, src, sizeof(*(dst)) * (size_t)(count),           \
                                    cudaMemcpyDeviceToHost, c->stream));                  \
    } while (0)

int nb_copy_tree(nb_ctx *c, double *root, uint64_t *keys, int32_t *perm, int32_t *level,
                 int32_t *first, int32_t *count, int32_t *next, int32_t *parent,
                 int32_t *nchild, double *mass, double *com, float *l, float *s)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->has_tree) return NB_ERR_STATE;
    int rc = read_counters(c);
    if (rc) return rc;
    const int64_t nn = c->n > 0 ? c->cnt_host[CNT_NODES] : 0;
    const int64_t n = c->n;
    if (n > 0) {
        if (c->nsys == 1) D2H(root, c->root, 7);
        else D2H(root, c->root, 8 * c->nsys);
    }
    D2H(keys, c->keys, n);
    D2H(perm, c->perm, n);
    D2H(level, c->n_level, nn);
    D2H(first, c->n_first, nn);
    D2H(count, c->n_count, nn);
    D2H(parent, c->n_parent, nn);
    D2H(nchild, c->n_nchild, nn);
    if (nn == 0) {
        CK(cudaStreamSynchronize(c->stream));
        return NB_OK;
    }
    // preorder views of the level-order moment arrays
    int4 *nc = (int4 *)malloc(sizeof(int4) * (size_t)nn);
    int32_t *p2b = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    double *bm = (double *)malloc(sizeof(double) * (size_t)nn);
    double *bc = (double *)malloc(sizeof(double) * 3 * (size_t)nn);
    float2 *wc = (float2 *)malloc(sizeof(float2) * (size_t)nn);
    rc = NB_OK;
    if (!nc || !p2b || !bm || !bc || !wc) rc = NB_ERR_NOMEM;
    if (!rc && (cudaMemcpyAsync(nc, c->node_c, sizeof(int4) * nn, cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaMemcpyAsync(p2b, c->pid2bfs, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaMemcpyAsync(bm, c->b_mass, sizeof(double) * nn, cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaMemcpyAsync(bc, c->b_com, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaMemcpy2DAsync(wc, sizeof(float2), &c->wrec[0].c, sizeof(nb_wrec),
                                  sizeof(float2), nn, cudaMemcpyDeviceToHost,
                                  c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess))
        rc = NB_ERR_CUDA;
    for (int64_t u = 0; !rc && u < nn; u++) {
        const int64_t b = p2b[u];
        if (next) next[u] = nc[u].x >= nn ? -1 : nc[u].x;
        if (mass) mass[u] = bm[b];
        if (com)
            for (int d = 0; d < 3; d++) com[3 * u + d] = bc[3 * b + d];
        if (l) l[u] = wc[b].x;
        if (s) s[u] = wc[b].y;
    }
    free(nc);
    free(p2b);
    free(bm);
    free(bc);
    free(wc);
    if (rc == NB_ERR_CUDA) cudaGetLastError();
    return rc;
}

int nb_copy_groups(nb_ctx *c, int32_t *gnode, int32_t *gfirst, int32_t *gcount, float *box,
                   float *invtheta)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->has_groups) return NB_ERR_STATE;
    int rc = read_counters(c);
    if (rc) return rc;
    const int64_t G = c->n > 0 ? c->cnt_host[CNT_GROUPS] : 0;
    D2H(gnode, c->gnode, G);
    D2H(gfirst, c->gfirst, G);
    D2H(gcount, c->gcount, G);
    float4 *b = nullptr;
    if ((box || invtheta) && G > 0) {
        b = (float4 *)malloc(sizeof(float4) * 3 * (size_t)G);
        if (!b) return NB_ERR_NOMEM;
        if (cudaMemcpyAsync(b, c->gbox, sizeof(float4) * 3 * (size_t)G, cudaMemcpyDeviceToHost,
                            c->stream) != cudaSuccess) {
            free(b);
            return NB_ERR_CUDA;
        }
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        free(b);
        return NB_ERR_CUDA;
    }
    for (int64_t g = 0; b && g < G; g++) {
        const float4 lo = b[3 * g], hi = b[3 * g + 1], ct = b[3 * g + 2];
        if (box) {
            float *o = box + 9 * g;
            o[0] = lo.x; o[1] = lo.y; o[2] = lo.z;
            o[3] = hi.x; o[4] = hi.y; o[5] = hi.z;
            o[6] = ct.x; o[7] = ct.y; o[8] = ct.z;
        }
        if (invtheta) invtheta[g] = ct.w;
    }
    free(b);
    return NB_OK;
}

int nb_copy_group_lengths(nb_ctx *c, int32_t *len, int64_t cap)
{
    if (!c || !len || cap < 0) return NB_ERR_INVALID_ARG;
    if (!c->has_lists) return NB_ERR_STATE;
    int rc = read_counters(c);
    if (rc) return rc;
    int64_t G = c->n > 0 ? c->cnt_host[CNT_GROUPS] : 0;
    if (G > cap) G = cap;
    if (G > 0) D2H(len, c->glen, G);
    CK(cudaStreamSynchronize(c->stream));
    return NB_OK;
}

int nb_copy_list(nb_ctx *c, int64_t g, int32_t *entries, float *xm, int64_t cap,
                 int64_t *len_out)
{
    if (!c || cap < 0 || !len_out) return NB_ERR_INVALID_ARG;
    if (!c->has_lists) return NB_ERR_STATE;
    int rc = read_counters(c);
    if (rc) return rc;
    const int64_t G = c->n > 0 ? c->cnt_host[CNT_GROUPS] : 0;
    if (g < 0 || g >= G) return NB_ERR_INVALID_ARG;
    int32_t len = 0;
    CK(cudaMemcpyAsync(&len, c->glen + g, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *len_out = len;
    int64_t L = len < c->list_cap ? len : c->list_cap;
    if (L > cap) L = cap;
    if (entries && L > 0)
        CK(cudaMemcpyAsync(entries, c->list_id + g * c->list_cap, sizeof(int32_t) * L,
                           cudaMemcpyDeviceToHost, c->stream));
    if (xm && L > 0)
        CK(cudaMemcpyAsync(xm, c->list_xm + g * c->list_cap, sizeof(float4) * L,
                           cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NB_OK;
}

int nb_copy_lists(nb_ctx *c, int64_t *offsets, int32_t *entries, float *xm)
{
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->has_lists) return NB_ERR_STATE;
    int rc = read_counters(c);
    if (rc) return rc;
    const int64_t G = c->n > 0 ? c->cnt_host[CNT_GROUPS] : 0;
    if (G == 0) {
        if (offsets) offsets[0] = 0;
        return NB_OK;
    }
    int32_t *len = (int32_t *)malloc(sizeof(int32_t) * (size_t)G);
    if (!len) return NB_ERR_NOMEM;
    if (cudaMemcpyAsync(len, c->glen, sizeof(int32_t) * (size_t)G, cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        free(len);
        return NB_ERR_CUDA;
    }
    int64_t off = 0;
    for (int64_t g = 0; g < G; g++) {
        if (offsets) offsets[g] = off;
        const int64_t L = len[g] < c->list_cap ? len[g] : c->list_cap;
        if (entries && L > 0 &&
            cudaMemcpyAsync(entries + off, c->list_id + g * c->list_cap, sizeof(int32_t) * L,
                            cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) {
            free(len);
            return NB_ERR_CUDA;
        }
        if (xm && L > 0 &&
            cudaMemcpyAsync(xm + 4 * off, c->list_xm + g * c->list_cap, sizeof(float4) * L,
                            cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) {
            free(len);
            return NB_ERR_CUDA;
        }
        off += len[g];
    }
    if (offsets) offsets[G] = off;
    free(len);
    CK(cudaStreamSynchronize(c->stream));
    return NB_OK;
}

}  // extern "C"
