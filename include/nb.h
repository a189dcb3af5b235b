/*
 * nb.h -- C ABI of libnb: the oct-tree group walk and softened gravity
 * force of Nakasato, "Oct-tree Method on GPU" (arXiv:0909.0541), as
 * hand-written CUDA for sm_103a (GB300).
 *
 * Conventions for every call
 *   - Pointers named *_dev are device pointers owned by the caller (for
 *     example torch tensors); *_host pointers are host memory owned by the
 *     caller.  The library owns the tree, the groups, the interaction lists
 *     and all scratch, allocated once by nb_create for cfg.max_n particles.
 *   - Work is queued on cfg.stream.  With cfg.sync_checks != 0 each call
 *     synchronises that stream before returning and reports device-side
 *     errors (and nb_walk_groups grows the list storage by itself).  With
 *     sync_checks == 0 calls do not synchronise, allocate nothing and can be
 *     captured in a CUDA graph; device errors are latched and reported by
 *     nb_sync_status or by the next call that synchronises.
 *   - Return value: NB_OK (0) or a negative NB_ERR_* code.
 *   - Units: G = 1.  Positions are FP64 (N x 3, row-major x,y,z per
 *     particle), masses FP32, accelerations and potentials FP32, all in the
 *     caller's particle order.
 */
#ifndef NB_H
#define NB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NB_OK 0
#define NB_ERR_INVALID_ARG (-1) /* bad size, NULL pointer, theta < 0, ... */
#define NB_ERR_CUDA (-2)        /* a CUDA runtime call failed             */
#define NB_ERR_CAPACITY (-3)    /* an interaction list outgrew its slot    */
#define NB_ERR_WALK_LIMIT (-4)  /* a walk did not advance (corrupt tree)   */
#define NB_ERR_NONFINITE (-5)   /* a position is NaN or infinite           */
#define NB_ERR_STATE (-6)       /* call order: build, then walk, then force */
#define NB_ERR_NOMEM (-7)       /* device allocation failed                */
#define NB_ERR_INTERNAL (-8)    /* a kernel's own bounds check fired: the
                                   access was skipped, results are invalid
                                   (a library defect; NB_DEBUG_SYNC=1 in the
                                   environment names the kernel and site)   */

/* accumulation modes of nb_forces */
#define NB_FP32 0      /* plain FP32 sums                                   */
#define NB_FP32_COMP 1 /* FP32 tile sums merged with Kahan compensation     */
#define NB_FP64ACC 2   /* FP32 terms accumulated in FP64                    */

typedef struct nb_ctx nb_ctx;

typedef struct nb_config {
    int64_t max_n;         /* particle capacity (>= 1)                       */
    int64_t list_capacity; /* entries per group list; 0 = grow on demand     */
    void *stream;          /* cudaStream_t; NULL = legacy default stream     */
    int sync_checks;       /* see the conventions above                      */
    int device;            /* CUDA device ordinal                            */
    /* defaults used by nb_leapfrog_step */
    float eps;             /* Plummer softening, >= 0                        */
    float theta;           /* opening angle, >= 0 (0 = never accept a cell)  */
    int n_crit;            /* maximum group size, >= 1                       */
    int precision;         /* NB_FP32, NB_FP32_COMP or NB_FP64ACC            */
    int64_t max_systems;   /* systems per batch (nb_build_tree_batched), >= 1 */
} nb_config;

typedef struct nb_stats {
    int64_t n;             /* particles in the current tree                  */
    int64_t n_cells;       /* cells (nodes holding >= 2 particles)           */
    int64_t n_nodes;       /* cells + particle leaves                        */
    int64_t n_groups;      /* groups of the last walk                        */
    int64_t list_entries;  /* sum of the groups' list lengths                */
    int64_t max_list;      /* longest list                                   */
    int64_t list_capacity; /* entries per group slot                         */
    int64_t n_pp;          /* particle-particle interactions (self excluded) */
    int64_t n_pc;          /* particle-cell interactions                     */
    int32_t max_level;     /* deepest cell level                             */
    int32_t reserved;
    int64_t n_pp_total;    /* n_pp summed over every walk of this context    */
    int64_t n_pc_total;    /* n_pc summed over every walk of this context    */
} nb_stats;

/* phases timed by nb_set_timing */
#define NB_PHASE_BUILD 0     /* nb_build_tree                               */
#define NB_PHASE_WALK 1      /* nb_walk_groups (groups + walk)              */
#define NB_PHASE_FORCE 2     /* nb_forces                                   */
#define NB_PHASE_INTEGRATE 3 /* leapfrog kicks and drift                    */
#define NB_NPHASE 4

/* Fill cfg with defaults: max_n as given, stream NULL, sync_checks 1,
 * eps 0.01, theta 0.6, n_crit 64, precision NB_FP32. */
void nb_config_default(nb_config *cfg, int64_t max_n);

/* Allocate a context and all its device storage for cfg->max_n particles
 * (worst case: 11 cells per particle).  *ctx is NULL on failure. */
int nb_create(nb_ctx **ctx, const nb_config *cfg);
int nb_destroy(nb_ctx *ctx);
/* Switch the synchronising checks of cfg.sync_checks on (1) or off (0). */
int nb_set_sync_checks(nb_ctx *ctx, int on);

/* Build the oct-tree over n particles (Sec. "Oct-tree Method": a root cube
 * enclosing every particle, split into eight sub-cells until a cell holds
 * one particle; Sec. "Our GPU implementation": total mass, centre of mass,
 * cell size and next/more pointers; Sec. "Test and Optimization": Morton
 * order).  Steps: bounding box -> root cube (side = max extent * (1+2^-20))
 * -> 21-level Morton keys (FP64 quantisation) -> stable radix sort ->
 * cells (one per key prefix shared by >= 2 particles; coincident particles
 * below level 21 stay in one cell) -> FP64 moments folded bottom-up in
 * octant order -> next/more in depth-first preorder.
 * pos_dev: n x 3 FP64; mass_dev: n FP32; 0 <= n <= max_n.
 * Errors: INVALID_ARG, NONFINITE (a coordinate is NaN/inf), CUDA. */
int nb_build_tree(nb_ctx *ctx, const double *pos_dev, const float *mass_dev,
                  int64_t n);

/* A batch of independent systems in one tree build: particles of system s
 * are rows offsets[s] .. offsets[s+1] of pos_dev / mass_dev (offsets_dev:
 * n_systems + 1 int64 on the device, offsets[0] = 0, offsets[n_systems] = n,
 * every system non-empty, owned by the caller and read during the call).
 * Each system gets its own root cube and Morton keys; particles are sorted by
 * (system, key), and cells never span two systems, so the result is a
 * forest whose trees, in system order, are each the tree nb_build_tree
 * builds for that system alone (node ids offset by the nodes of the systems
 * before it).  Walks start at the group's own root; walk, forces and the
 * leapfrog then run once for the whole batch.  n_systems <= cfg.max_systems.
 * Errors: as nb_build_tree; INVALID_ARG (reported by the device check of the
 * offsets when sync_checks is on). */
int nb_build_tree_batched(nb_ctx *ctx, const double *pos_dev, const float *mass_dev,
                          const int64_t *offsets_dev, int64_t n_systems, int64_t n);
/* nb_leapfrog_step for a batch (rebuilding with nb_build_tree_batched). */
int nb_leapfrog_step_batched(nb_ctx *ctx, double *pos_dev, double *vel_dev,
                             const float *mass_dev, const int64_t *offsets_dev,
                             int64_t n_systems, int64_t n, double dt);

/* Form groups (each node with count <= n_crit whose parent holds more) and
 * walk the tree once per group (the walk of Fig. "treewalk_iterative" in
 * group form, breadth-first over a level-ordered copy of the tree), writing
 * each group's interaction list of particles and accepted cells to device
 * memory.  A cell is accepted when the squared FP32 distance from its centre
 * of mass to the group's bounding box exceeds (l/theta + s)^2 (Eq. mac; l =
 * cell side, s = |centre of mass - geometric centre|); a cell that contains
 * the group is always opened.  The group's own particles are not listed:
 * nb_forces sums them directly.  theta = 0 accepts no cell (direct sum).
 * theta_per_group_dev (nullable): one theta per group, in group order, for
 * the groups of a previous call with the same n_crit on the same tree.
 * Errors: STATE (no tree), INVALID_ARG, CAPACITY (sync_checks == 0 and a
 * list or a walk frontier outgrew its storage), WALK_LIMIT, CUDA, NOMEM. */
int nb_walk_groups(nb_ctx *ctx, float theta, int n_crit,
                   const float *theta_per_group_dev);

/* Sum Eq. (gravity) over every group's list and the group's own members for
 * every particle of the group:
 * a_i = sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2},
 * phi_i = -sum_{j != i} m_j / (|x_j - x_i|^2 + eps^2)^{1/2}, cells entering as
 * point masses at their centre of mass.  Coordinates are FP32 relative to
 * the group's box centre; the self term is excluded by index and a pair
 * with r^2 + eps^2 == 0 contributes nothing.
 * acc_dev: n x 3 FP32 (required); pot_dev: n FP32 (nullable).
 * precision: NB_FP32, NB_FP32_COMP or NB_FP64ACC.
 * Errors: STATE (no lists), INVALID_ARG, CUDA. */
int nb_forces(nb_ctx *ctx, float eps, float *acc_dev, float *pot_dev,
              int precision);

/* Groups, walk and force sum in one pass without interaction lists in
 * device memory: the fused walk-and-sum design of Fig. "treegpu" (Sec. "Our
 * GPU implementation") in group form.  After nb_build_tree: forms the groups
 * of n_crit (as nb_walk_groups) and, per force work item, walks the group with
 * the opening angle theta and sums Eq. (gravity) on the fly through a small
 * shared-memory buffer.  acc_dev / pot_dev / precision as nb_forces; the
 * results equal nb_walk_groups + nb_forces bit for bit.  The walk is repeated
 * for each 64-target item of a group larger than 64.  Afterwards there are no
 * lists to export (nb_forces and nb_copy_lists return NB_ERR_STATE until the
 * next nb_walk_groups).  Interaction counts go to nb_get_stats as for the list
 * path.  Errors: STATE (no tree), INVALID_ARG, CAPACITY (a walk frontier
 * outgrew the queues with sync_checks off), WALK_LIMIT, CUDA, NOMEM. */
int nb_forces_fused(nb_ctx *ctx, float theta, int n_crit, float eps, float *acc_dev,
                    float *pot_dev, int precision);
/* on != 0: the force passes of nb_leapfrog_step (and its batched, host and
 * graph forms) use nb_forces_fused instead of nb_walk_groups + nb_forces. */
int nb_set_fused(nb_ctx *ctx, int on);

/* Key order of the next tree build (nb_build_tree and its batched, leapfrog,
 * host and graph forms): NB_ORDER_MORTON (the default; Sec. "Test and
 * Optimization", Table bench2) or NB_ORDER_HILBERT, the Peano-Hilbert order
 * the same section names as better for locality (63-bit keys by Skilling's
 * transpose method).  The cells are the same in both orders; only the order
 * of the sorted particles, of the nodes (depth-first preorder visits the
 * children along the curve) and of the summation changes, and
 * nb_copy_tree's keys are then Peano-Hilbert keys.  A graph captured
 * before the change keeps the order it was captured with. */
#define NB_ORDER_MORTON 0
#define NB_ORDER_HILBERT 1
int nb_set_key_order(nb_ctx *ctx, int order);

/* Quadrupole cells ("any high order moment" in the particle-cell term, Sec.
 * "Oct-tree Method"; the paper itself uses the monopole).  With on != 0 the
 * next tree builds also fold every cell's traceless quadrupole about its
 * centre of mass, Q_ab = sum_k m_k (3 d_a d_b - |d|^2 delta_ab), d = x_k -
 * COM, in FP64 bottom-up by the parallel-axis theorem; walks store each
 * accepted cell's Q in FP32 beside its list record (in each 32-node chunk
 * of the walk the accepted cells come before the particles); and nb_forces
 * adds to every particle-cell term, softened like Eq. (gravity) with R^2 =
 * |r|^2 + eps^2, r = x_i - COM:
 *   a += Q r / R^5 - (5/2) (r.Q.r) r / R^7,   phi += -(1/2) r.Q.r / R^5.
 * Switching on allocates 48 B per node slot of cfg.max_n (NOMEM on
 * failure), and list storage then takes 32 B more per entry.  In this mode
 * nb_forces takes NB_FP32 or NB_FP32_COMP (NB_FP64ACC: INVALID_ARG), a walk
 * needs a tree built in this mode (else STATE), and nb_forces_fused and
 * nb_set_fused's force passes are INVALID_ARG.  The opening test is
 * unchanged, so the lists hold the same sets of nodes as without. */
int nb_set_quadrupole(nb_ctx *ctx, int on);
/* The quadrupoles of the current tree (built with nb_set_quadrupole on),
 * n_nodes x 6 FP64 (xx, yy, zz, xy, xz, yz) in depth-first preorder, zero
 * for particles; synchronising debug export. */
int nb_copy_quadrupoles(nb_ctx *ctx, double *q_host);

/* Fixed-radius neighbour search by the general treewalk (Sec. "General
 * Treewalk", Fig. "general_treewalk": the force walk's descent with another
 * distance test, for short-range interactions).  On the current tree, groups
 * of n_crit are walked once each; the neighbours of particle i are the j != i
 * with |x_j - x_i|^2 <= h^2, the squared distance summed (x, y) then z in FP64
 * from the FP64 positions, every operation rounded on its own.  off_dev: n + 1
 * int64 (device) receives the CSR offsets in caller order; *total_host the
 * number of pairs.  idx_dev (int32 caller indices, device, nullable): when it
 * holds cap >= total entries it receives each particle's neighbours in
 * ascending caller index, else only the offsets and total are produced (call
 * again with room).  Synchronises cfg.stream; forms groups, leaves no lists
 * (nb_forces returns STATE until the next walk).  Errors: STATE (no tree),
 * INVALID_ARG, CAPACITY (total >= 2^31 pairs), WALK_LIMIT, CUDA, NOMEM. */
int nb_neighbours(nb_ctx *ctx, double h, int n_crit, int64_t *off_dev, int32_t *idx_dev,
                  int64_t cap, int64_t *total_host);

/* nb_walk_groups + nb_forces in one persistent launch that overlaps them:
 * every warp takes a force work item whose group's walk has finished, else
 * the next group to walk, so the walk (bound by the latency of its record
 * fetches) and the force sum (bound by the FMA pipe) share the SMs.  The lists
 * and every item's sums are computed exactly as by the two calls, so the
 * results are the same bits.  precision: NB_FP32 or NB_FP32_COMP (others
 * INVALID_ARG); not in the quadrupole mode (INVALID_ARG).  It needs list
 * storage sized by an earlier synchronising walk: without it, the call runs
 * nb_walk_groups + nb_forces when sync_checks is on and returns CAPACITY
 * when it is off.  With sync_checks on, a list that outgrows its slot makes
 * the call redo the walk and the force sum separately (growing the storage).
 * Timing: the group formation counts as NB_PHASE_WALK, the overlapped launch
 * as NB_PHASE_FORCE.  Errors: as nb_walk_groups and nb_forces. */
int nb_walk_forces(nb_ctx *ctx, float theta, int n_crit, float eps, float *acc_dev,
                   float *pot_dev, int precision);
/* on != 0: the force passes of nb_leapfrog_step (and its batched, host and
 * graph forms) use nb_walk_forces (FP32 and compensated modes, monopole
 * cells; otherwise the separate calls). */
int nb_set_overlap(nb_ctx *ctx, int on);

/* One kick-drift-kick leapfrog step of size dt in FP64 ("integrate orbits
 * ... and repeat", Sec. Introduction): v += a dt/2; x += v dt; rebuild the
 * tree, walk and force with cfg.eps, cfg.theta, cfg.n_crit, cfg.precision;
 * v += a dt/2.  The context keeps a(x) between steps; the first step (or
 * the first after nb_leapfrog_reset or a change of n) computes it first.
 * pos_dev, vel_dev: n x 3 FP64, updated in place. */
int nb_leapfrog_step(nb_ctx *ctx, double *pos_dev, double *vel_dev,
                     const float *mass_dev, int64_t n, double dt);
int nb_leapfrog_reset(nb_ctx *ctx);
/* nb_leapfrog_step on HOST buffers (pinned memory lets the copies run
 * asynchronously): the library copies pos_host, vel_host (n x 3 FP64) and
 * mass_host (n FP32) into device buffers of its own (allocated at the first
 * such call, 52 B per particle of cfg.max_n), runs the step there and writes
 * the new positions and velocities back into pos_host and vel_host.  The
 * positions leave on a second stream as soon as the drift has written them,
 * overlapping the tree build, walk and force; the velocities follow the
 * closing kick.  With sync_checks the call returns after both copies; without,
 * they complete in stream order on cfg.stream and the host buffers must stay
 * valid until that stream is synchronised.  The kept a(x) is for the state the
 * previous step returned: after changing the host state otherwise, call
 * nb_leapfrog_reset.  Errors: as nb_leapfrog_step, NOMEM. */
int nb_leapfrog_step_host(nb_ctx *ctx, double *pos_host, double *vel_host,
                          const float *mass_host, int64_t n, double dt);
/* The accelerations (n x 3 FP32, caller order) kept by the last step. */
int nb_leapfrog_acc(nb_ctx *ctx, float *acc_dev);

/* Capture nsteps leapfrog steps (offsets_dev NULL: one system; else a batch,
 * see nb_build_tree_batched) into a CUDA graph held by the context, and
 * replay it with nb_graph_launch on cfg.stream.  A replay gives the same bits
 * as nsteps calls of nb_leapfrog_step; inside it, the second kick of each step
 * but the last runs in one pass with the next step's first kick and drift, so
 * the phase timing shows one integrate phase fewer per step boundary.  Needs a non-NULL cfg.stream
 * (the legacy stream cannot be captured) and a previous step of the same n
 * made with sync_checks on, which sizes the list storage; during replay
 * nothing synchronises or allocates, and a list that outgrows its slot is
 * latched as NB_ERR_CAPACITY for nb_sync_status.  pos/vel/mass are the
 * buffers every replay reads and updates.  With timing on (nb_set_timing) at
 * capture, the phase events are captured as event-record nodes that every
 * launch records again, and nb_get_timing reports the phases of the last
 * launch times the launches since its previous call; kernels launched by the
 * graph count in its `launches` output.  The event pool holds 2048 phases: a
 * capture longer than that times only its first 2048 phases, and the pool's
 * remainder serves eager phases until the next capture. */
int nb_graph_capture_leapfrog(nb_ctx *ctx, double *pos_dev, double *vel_dev,
                              const float *mass_dev, const int64_t *offsets_dev,
                              int64_t n_systems, int64_t n, double dt, int nsteps);
int nb_graph_launch(nb_ctx *ctx);

/* Autotuner: builds the tree of (pos_dev, mass_dev) -- a forest of n_systems
 * independent systems when offsets_dev (device, n_systems + 1 row offsets)
 * is given, as nb_build_tree_batched; one system when it is NULL -- then
 * times `reps` walk + FP32 force passes with CUDA events for every n_crit of
 * the list x force work-item width (32 or 64 targets per warp) x j-tile depth
 * (32 or 64 list records staged per tile; items of several source streams
 * stage 64 either way) x force block size (256 or 128
 * threads), keeps the fastest combination in the context (cfg.n_crit and the
 * FP32 force shape used from then on) and returns it in the best_* outputs
 * (each nullable); ms_host (nullable, 8 x ncand) receives the mean times,
 * index ((candidate x 2 + width index) x 2 + tile index) x 2 + block index,
 * with the indices in the orders listed above. */
int nb_autotune(nb_ctx *ctx, const double *pos_dev, const float *mass_dev,
                const int64_t *offsets_dev, int64_t n_systems, int64_t n, float eps,
                float theta, const int *n_crit_host, int ncand, int reps,
                int *best_n_crit_host, int *best_rows_host, int *best_tile_host,
                int *best_block_host, float *ms_host);

/* FP64 direct sum of Eq. (gravity) for the targets listed in targets_dev
 * (nt indices into 0..n-1; NULL = all n), used as the accuracy judge.
 * acc_dev: nt x 3 FP64, pot_dev: nt FP64.  Work is queued on `stream`. */
int nb_direct_sum(const double *pos_dev, const float *mass_dev, int64_t n,
                  double eps, const int64_t *targets_dev, int64_t nt,
                  double *acc_dev, double *pot_dev, void *stream);

/* Brute-force FP32 sum of Eq. (gravity) over every pair j != i, O(n^2): the
 * paper's bare many-body kernel (Sec. "A Bare Many-body Performance on RV770
 * GPU"), against which the tree method is timed (Sec. "Test and
 * Optimization": the tree wins except for N < 10,000).  Positions are
 * rounded once to FP32 (the representation that kernel works on); every
 * interaction is the tree force kernel's 13-operation FP32 step with a MUFU
 * rsqrt; a pair with r^2 + eps^2 == 0 contributes nothing.
 * pos_dev: n x 3 FP64; mass_dev: n FP32; acc_dev: n x 3 FP32 (required);
 * pot_dev: n FP32 (nullable); precision: NB_FP32 or NB_FP32_COMP (Kahan-
 * compensated per 256-source tile); NB_FP64ACC is INVALID_ARG (use
 * nb_direct_sum).  work_dev: caller-owned device workspace, 256-byte
 * aligned, of at least nb_direct_f32_workspace_size(n) bytes for the current
 * device (it holds the FP32 copy of the particles and the partial sums of
 * the source parts).  Work is queued on `stream`; nothing synchronises.
 * Results are in caller order and do not depend on scheduling. */
size_t nb_direct_f32_workspace_size(int64_t n);
int nb_direct_f32(const double *pos_dev, const float *mass_dev, int64_t n, float eps,
                  float *acc_dev, float *pot_dev, int precision, void *work_dev,
                  size_t work_bytes, void *stream);

/* Per-phase device timing: with timing on, every phase is bracketed by CUDA
 * events recorded on cfg.stream.  nb_get_timing synchronises and returns,
 * per phase, the summed milliseconds and the number of calls since the last
 * nb_get_timing, and (launches) the number of kernels libnb launched in that
 * time; then it resets all three.  Any output pointer may be NULL. */
int nb_set_timing(nb_ctx *ctx, int on);
int nb_get_timing(nb_ctx *ctx, double *ms_host, int64_t *calls_host,
                  int64_t *launches_host);

/* Synchronise the stream and return (and clear) any latched device error. */
int nb_sync_status(nb_ctx *ctx);
/* Self-test of the bounded wait used where one warp waits for others (the
 * bottom-up moments of nb_build_tree): one warp waits, polling at most
 * spin_limit times, for a count that nothing raises.  Synchronises and
 * returns the latched status, NB_ERR_INTERNAL when the wait gave up as
 * designed; the context stays usable.  No tree state is touched. */
int nb_selftest_wait(nb_ctx *ctx, unsigned spin_limit);
/* Synchronise and fill *st. */
int nb_get_stats(nb_ctx *ctx, nb_stats *st);

/* Debug export (synchronising copies to host memory; any pointer may be
 * NULL).  Node arrays have n_nodes entries in depth-first preorder, vectors
 * x3; next is -1 past the last node; parent of the root is -1; level and
 * nchild are -1 / 0 for particle leaves.  perm maps sorted slot -> caller
 * index; keys are the sorted 63-bit Morton keys.  root: centre[3], L,
 * corner[3]. */
int nb_copy_tree(nb_ctx *ctx, double *root_host, uint64_t *keys_host,
                 int32_t *perm_host, int32_t *level_host, int32_t *first_host,
                 int32_t *count_host, int32_t *next_host, int32_t *parent_host,
                 int32_t *nchild_host, double *mass_host, double *com_host,
                 float *l_host, float *s_host);
/* Groups of the last walk or feature probe: node id, first sorted slot, size, box (G x 9:
 * lo[3], hi[3], centre[3]) and the FP32 1/theta used. */
int nb_copy_groups(nb_ctx *ctx, int32_t *gnode_host, int32_t *gfirst_host,
                   int32_t *gcount_host, float *box_host, float *invtheta_host);
/* Lists of the last walk, packed: offsets (G+1), preorder node ids in walk
 * (breadth-first) order, and the FP32 source records the force kernel reads
 * (x, y, z relative to the group centre, mass).  The group's own particles
 * are not in its list. */
int nb_copy_lists(nb_ctx *ctx, int64_t *offsets_host, int32_t *entries_host,
                  float *xm_host);

/* ---- learned opening angle (the paper has one global theta, Eq. mac; this
 * per-group form is the project's addition) ---------------------------------
 * A 12 -> 64 -> 64 -> 64 -> 1 GELU network maps a group's features to
 * theta = 0.3 + 0.9 sigmoid(z).  Parameters: NB_MLP_NPARAM FP32 values in
 * the flat layout W1 (64 x 16) @0, b1 @1024, W2 (64 x 64) @1088, b2 @5184,
 * W3 @5248, b3 @9344, w4 (64) @9408, b4 @9920, mu (16) @9928, sigma (16)
 * @9944; features are standardised as (x - mu) / sigma.  Products run on
 * the tensor cores with BF16 operands and FP32 accumulation.  Features are
 * rows of NB_NFEAT_STRIDE floats (12 used).  `work` is a device workspace
 * of nb_mlp_workspace_size(batch) bytes owned by the caller.  All calls
 * queue work on `stream` and do not synchronise. */
/* Features of every group for n_crit: the groups are walked once with
 * theta = 1.2 without writing lists (the probe walk) and each gets 16
 * floats: ln n_g; ln(box side / L + 1e-7) for x, y, z; ln n_g minus the sum
 * of ln(side / L + 1e-4); ln(|box centre - root centre| / L + 1e-6);
 * ln(list length + 1); accepted cells / list length; ln(min, mean, max
 * distance from the box centre to the accepted cells' centres of mass / L +
 * 1e-7); depth of the group node / 22; 4 zeros (L = root cube side).
 * feat_dev (nullable) receives min(G, cap_rows) rows; n_groups_host
 * (nullable, synchronises) receives G.  Lists are invalidated. */
int nb_group_features(nb_ctx *ctx, int n_crit, float *feat_dev, int64_t cap_rows,
                      int64_t *n_groups_host);
/* Feature mode of nb_group_features and nb_walk_groups_learned: 0 (the
 * default) the probe-walk features above; 1 tree-only features, which need no
 * walk: features 0-5 and 11 as above (the same formulas), 6-10 zero. */
int nb_set_feature_mode(nb_ctx *ctx, int mode);
/* Walk with a per-group theta from the network (params_dev, layout below)
 * evaluated on the features of the context's feature mode (the probe walk's,
 * or the tree-only ones, whose groups the walk then reuses, setting only
 * each box's 1/theta); a non-finite output becomes
 * theta_fallback.  theta_out_dev (nullable, n floats) receives the group
 * thetas (G of them are meaningful). */
int nb_walk_groups_learned(nb_ctx *ctx, int n_crit, const float *params_dev,
                           float theta_fallback, float *theta_out_dev);
/* Training data of the learned theta.  nb_group_errors: median |da|/|a| of
 * each sampled group (rows off[k] .. off[k+1] of ref_dev, FP64 judge
 * accelerations, belong to sample k and targets_dev gives their caller
 * indices into acc_dev, n x 3 FP32), at most 1024 members per group.
 * nb_theta_labels: the label of each sample from its errors at the T thetas
 * of an ascending grid (err_dev, T x S).  With cost_dev NULL: the largest
 * grid theta whose error is within budget (else the smallest).  With
 * cost_dev (interactions of the group at each theta, T x S) and size_dev
 * (group sizes, S): the grid theta minimising cost / size + lambda *
 * ln(error), one exchange rate between interactions and error for every
 * group. */
int nb_group_errors(const float *acc_dev, const double *ref_dev, const int64_t *targets_dev,
                    const int64_t *off_dev, int64_t S, float *err_dev, void *stream);
int nb_theta_labels(const float *err_dev, const float *cost_dev, const float *size_dev,
                    const float *grid_dev, int T, int64_t S, float budget, float lambda,
                    float *labels_dev, void *stream);

/* The label rule of the learned theta with all its arithmetic on the
 * device (the paper has one theta, Eq. mac; its cost / accuracy trade is
 * Table theta).  S sampled groups, T grid thetas (ascending, T <= 64); err_dev
 * (T x S FP32): each group's measured median |da|/|a| at each theta (FP64
 * judge); cost_dev (T x S FP32): its cost there (interactions plus weighted
 * list entries); size_dev (S FP32): group sizes n_g.
 * nb_theta_fit_curves: the curves the features predict.  Least squares, in
 * FP64, of ln(err + 1e-15) and of ln(cost + 1) at every theta on the
 * feature columns cols_host[0..ncols) (ncols <= 16; feature rows of `stride`
 * floats in feat_dev, S x stride) plus an intercept; columns are
 * standardised first (a constant column drops out) and the normal equations
 * are solved by Cholesky.  pred_lnerr_dev receives the fitted ln error,
 * pred_cost_dev exp of the fitted ln(cost + 1) (both T x S FP64).  work_dev:
 * caller-owned, 256-byte aligned, nb_theta_fit_workspace_size(S, ncols, T)
 * bytes.  Queued on `stream`, no synchronisation. */
size_t nb_theta_fit_workspace_size(int64_t S, int ncols, int T);
int nb_theta_fit_curves(const float *feat_dev, int64_t S, int stride, const int32_t *cols_host,
                        int ncols, const float *err_dev, const float *cost_dev, int T,
                        double *pred_lnerr_dev, double *pred_cost_dev, void *work_dev,
                        size_t work_bytes, void *stream);
/* nb_theta_allocate: labels_dev (S FP32) receives each group's grid theta
 * minimising cost / n_g + lambda * lnerr, where (lnerr, cost) are the
 * predicted curves when pred_lnerr_dev / pred_cost_dev are given (T x S
 * FP64, from nb_theta_fit_curves), else the measured ones (ln max(err,
 * 1e-9) and cost_dev); ties go to the smaller theta.  lambda is bisected
 * `iters` times in ln space on [lam_lo, lam_hi] so that a statistic of the
 * MEASURED errors at the chosen thetas is <= budget; the labels are those of
 * the bracket's upper end.  The statistic: without perr_dev, the n_g-weighted
 * median of the groups' median errors (the smallest error u whose weight of
 * errors <= u reaches half the total); with perr_dev (T x P FP32: every judged
 * particle's own |da|/|a| at each theta, group g's particles being columns
 * poff_dev[g] .. poff_dev[g+1], an S + 1 int64 offset array from 0 to P,
 * checked before use: the call then synchronises `stream`), the median over
 * the judged particles of their errors at their group's theta (mean of the
 * two middle values).  result_dev (2 FP64) receives lambda and the
 * statistic.  work_dev: caller-owned, 256-byte aligned,
 * nb_theta_allocate_workspace_size(S, P) bytes (P = 0 without perr_dev).
 * Queued on `stream`. */
size_t nb_theta_allocate_workspace_size(int64_t S, int64_t P);
int nb_theta_allocate(const double *pred_lnerr_dev, const double *pred_cost_dev,
                      const float *err_dev, const float *cost_dev, const float *size_dev,
                      const float *grid_dev, int T, int64_t S, double budget, double lam_lo,
                      double lam_hi, int iters, const float *perr_dev, const int64_t *poff_dev,
                      int64_t P, float *labels_dev, double *result_dev, void *work_dev,
                      size_t work_bytes, void *stream);
/* Mean and spread (population standard deviation, FP64, two passes) of the
 * first ncols (<= 17) columns of S feature rows of `stride` floats: the
 * network's input standardisation.  Queued on `stream`. */
int nb_column_stats(const float *feat_dev, int64_t S, int stride, int ncols, double *mean_dev,
                    double *sd_dev, void *stream);
/* Relative force errors of nt targets against an FP64 reference and their
 * statistics: err_dev (nt FP32, caller-owned) receives |a - ref| / |ref|
 * (|ref| = 0 counts as 1) for a = acc_dev rows targets_dev[k] (n x 3 FP32;
 * targets NULL: rows 0..nt-1) and ref_dev row k (nt x 3 FP64); out_dev (2
 * FP64) receives the median (mean of the two middle values) and the
 * nearest-rank q-quantile (the ceil(q nt)-th smallest).  Queued on `stream`,
 * no synchronisation. */
int nb_error_stats(const float *acc_dev, const double *ref_dev, const int64_t *targets_dev,
                   int64_t nt, double q, double *out_dev, float *err_dev, void *stream);

#define NB_MLP_NPARAM 9960
#define NB_NFEAT 12
#define NB_NFEAT_STRIDE 16
size_t nb_mlp_workspace_size(int64_t batch);
/* theta for n feature rows; a non-finite output becomes `fallback`. */
int nb_mlp_forward(const float *params_dev, const float *feat_dev, int64_t n,
                   float *theta_dev, float fallback, void *work_dev, void *stream);
/* Gradient of the summed loss over a batch of n rows, divided by n
 * (L = mean((theta - y)^2 + 4 max(0, theta - y)^2)): grad_dev receives
 * NB_MLP_NPARAM floats; loss_dev (nullable) the loss summed over the batch. */
int nb_mlp_grad(const float *params_dev, const float *feat_dev, const float *labels_dev,
                int64_t n, float *grad_dev, float *loss_dev, void *work_dev, void *stream);
/* Adam training (beta 0.9 / 0.999, eps 1e-8, rate lr) over `epochs` passes of
 * n samples in batches of `batch`; order_dev holds epochs x n sample indices
 * (the shuffles, drawn by the caller); adam_m/adam_v start at zero; grad_dev
 * is NB_MLP_NPARAM floats of scratch; loss_per_epoch_dev (nullable) receives
 * each epoch's summed loss. */
int nb_mlp_train(float *params_dev, float *adam_m_dev, float *adam_v_dev,
                 const float *feat_dev, const float *labels_dev, int64_t n,
                 const int32_t *order_dev, int epochs, int batch, float lr,
                 float *grad_dev, float *loss_per_epoch_dev, void *work_dev,
                 void *stream);

/* List length of every group of the last walk (G int32, host). */
int nb_copy_group_lengths(nb_ctx *ctx, int32_t *len_host, int64_t cap);

/* One group's list of the last walk: up to cap node ids and FP32 source
 * records; *len_host receives the full length (copy again with a larger cap
 * when it exceeds cap). */
int nb_copy_list(nb_ctx *ctx, int64_t group, int32_t *entries_host, float *xm_host,
                 int64_t cap, int64_t *len_host);

/* Morton order without any device allocation, for callers that cannot call
 * cudaMalloc (cudaFree synchronises the whole device, and where another
 * allocator already holds most of the device memory a raw cudaMalloc can
 * fail).  The paper has no counterpart; this is the first part of
 * nb_build_tree (root cube, 63-bit Morton keys, stable radix sort) run on
 * caller buffers, with its scratch in one static device array of about
 * 12.9 MB that every GPU loading the library keeps until the process exits.
 * pos_dev: n x 3 FP64 (caller order).  keys_dev: n uint64, receives the
 * sorted keys.  perm_dev: n int32, receives sorted slot -> caller index.
 * All three must be on the current device.
 * n <= NB_NOALLOC_MAX_N (1,048,576), else NB_ERR_INVALID_ARG with nothing
 * done.  The call queues its work on `stream` and synchronises that stream
 * before returning (to read its error word); it returns NB_ERR_NONFINITE for
 * a NaN or infinite coordinate.  The first call on each device also looks up
 * the scratch array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it for the life of the process: make that first call
 * before any stream capture begins, since a lookup while another thread
 * captures in global mode can invalidate that capture, and do not call the
 * entry point after a cudaDeviceReset of the device.  All calls share the
 * scratch array and it keeps the last call's contents (each call clears what
 * it needs cleared); calls that overlap on the GPU race. */
#define NB_NOALLOC_MAX_N (1 << 20)
int nb_morton_order_noalloc(const double *pos_dev, int64_t n, uint64_t *keys_dev,
                            int32_t *perm_dev, void *stream);

const char *nb_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* NB_H */
