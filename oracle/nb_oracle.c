/*
 * nb_oracle.c -- plain CPU oracle for the oct-tree gravity method of
 * Nakasato, "Oct-tree Method on GPU: $42/Gflops Cosmological Simulation"
 * (arXiv:0909.0541).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes, in the paper's order:
 *   - the softened direct sum, Eq. (gravity), in FP64 (and in long double
 *     for tiny N);
 *   - the oct-tree (Sec. "Oct-tree Method"): a root cube enclosing every
 *     particle, split recursively into eight sub-cells until a cell holds one
 *     particle;  cells carry total mass and centre of mass (Sec. "Our GPU
 *     implementation"), the cell size l and the offset s of Eq. (mac);
 *   - the depth-first (Morton) particle order of Sec. "Test and Optimization",
 *     and, as an option, the Peano-Hilbert order that the same section names
 *     as the better one for locality (the same cells, children visited in
 *     the curve's order);
 *   - next/more threading of the tree (Sec. "Our GPU implementation", after
 *     Makino 1990) by a depth-first pass;
 *   - the recursive walk of Fig. "treewalk" and the iterative walk of Fig.
 *     "treewalk_iterative", both in group form (a group of particles walks
 *     once and shares one interaction list, the GRAPE list idea of Sec.
 *     "Oct-tree Method with GRAPE"), plus the per-particle walk of Fig.
 *     "treegpu";
 *   - forces over interaction lists in FP64 (optionally with the cells'
 *     quadrupole moments);
 *   - fixed-radius neighbours by the general treewalk of Sec. "General
 *     Treewalk" (and by brute force, the definition);
 *   - a kick-drift-kick leapfrog for "integrate orbits" (Sec. Introduction).
 *
 * Readings where the paper is silent (the same ones the CUDA path follows):
 *   root cube   centre = bounding-box centre, side L = max extent * (1 + 2^-20)
 *               (L = 1 when every particle coincides);
 *   grid        q = clamp(floor((x - (centre - L/2)) * S), 0, 2^21 - 1), with
 *               the scale S = 2^21 / L rounded once in FP64;
 *               depth is capped at 21 levels: a level-21 cell holding several
 *               particles keeps them as particle children, in input order;
 *   octant      digit = 4*bit_x + 2*bit_y + bit_z, children in digit order
 *               (in the Peano-Hilbert option: in the order of the curve's
 *               digit at the child level);
 *   moments     M and sum(m x) folded over children in visiting order in FP64;
 *               COM = sum(m x) / M (the geometric centre when M == 0);
 *   l, s        l = L / 2^level (full side), s = |COM - geometric centre|,
 *               both rounded to FP32;
 *   groups      a node with count <= n_crit whose parent has count > n_crit
 *               (the root when N <= n_crit);
 *   group MAC   d2 = squared distance, in FP32, from the cell's FP32 COM to
 *               the group's FP32 bounding box; S = (l * (float)(1/theta) + s)^2
 *               in FP32; accept iff d2 > S (Eq. mac with strict '>');
 *               a cell that contains the group is always opened;
 *   self term   j == i is excluded by index; a pair with r^2 + eps^2 == 0
 *               contributes nothing;
 *   signs       a_i = +sum m_j (x_j - x_i) / (r^2 + eps^2)^{3/2},
 *               phi_i = -sum m_j / (r^2 + eps^2)^{1/2}, G = 1.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared
 * (-ffp-contract=off keeps every float operation separately rounded.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LEVELS 21
#define OR_GRID (1 << OR_LEVELS)

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Eq. (gravity): p_i and f_i summed over all j != i, here with physical
 * signs (acceleration towards j, negative potential) and G = 1.           */

int or_direct(int64_t n, const double *pos, const float *mass, double eps,
              int64_t nt, const int64_t *targets, double *acc, double *pot,
              double *amag)
{
    const double e2 = eps * eps;
    if (n < 0 || nt < 0)
        return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        const int64_t i = targets ? targets[t] : t;
        double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0, am = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            const double dx = pos[3 * j + 0] - pos[3 * i + 0];
            const double dy = pos[3 * j + 1] - pos[3 * i + 1];
            const double dz = pos[3 * j + 2] - pos[3 * i + 2];
            const double r2 = dx * dx + dy * dy + dz * dz + e2;
            if (r2 == 0.0)
                continue;
            const double rinv = 1.0 / sqrt(r2);
            const double m = (double)mass[j];
            const double mr3 = m * rinv * rinv * rinv;
            ax += mr3 * dx;
            ay += mr3 * dy;
            az += mr3 * dz;
            p -= m * rinv;
            am += mr3 * sqrt(dx * dx + dy * dy + dz * dz);
        }
        if (amag)
            amag[t] = am;
        acc[3 * t + 0] = ax;
        acc[3 * t + 1] = ay;
        acc[3 * t + 2] = az;
        pot[t] = p;
    }
    return 0;
}

/* The same sum in long double: the brute-force pin for tiny N. */
int or_direct_ld(int64_t n, const double *pos, const float *mass, double eps,
                 double *acc, double *pot)
{
    const long double e2 = (long double)eps * (long double)eps;
    for (int64_t i = 0; i < n; i++) {
        long double ax = 0, ay = 0, az = 0, p = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            const long double dx = (long double)pos[3 * j] - pos[3 * i];
            const long double dy = (long double)pos[3 * j + 1] - pos[3 * i + 1];
            const long double dz = (long double)pos[3 * j + 2] - pos[3 * i + 2];
            const long double r2 = dx * dx + dy * dy + dz * dz + e2;
            if (r2 == 0)
                continue;
            const long double rinv = 1.0L / sqrtl(r2);
            const long double m = mass[j];
            ax += m * dx * rinv * rinv * rinv;
            ay += m * dy * rinv * rinv * rinv;
            az += m * dz * rinv * rinv * rinv;
            p -= m * rinv;
        }
        acc[3 * i] = (double)ax;
        acc[3 * i + 1] = (double)ay;
        acc[3 * i + 2] = (double)az;
        pot[i] = (double)p;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Root cube ("a cube that encloses whole particles", Sec. Oct-tree Method)
 * and the integer grid the recursive subdivision works on.
 * out: centre[3], L, corner[3] where corner = centre - L/2.               */

void or_root_cube(int64_t n, const double *pos, double *out)
{
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < 3; k++) {
        lo[k] = n > 0 ? pos[k] : 0.0;
        hi[k] = lo[k];
    }
    for (int64_t i = 1; i < n; i++)
        for (int k = 0; k < 3; k++) {
            const double x = pos[3 * i + k];
            if (x < lo[k])
                lo[k] = x;
            if (x > hi[k])
                hi[k] = x;
        }
    double ext = 0.0;
    for (int k = 0; k < 3; k++) {
        out[k] = 0.5 * (lo[k] + hi[k]);
        const double e = hi[k] - lo[k];
        if (e > ext)
            ext = e;
    }
    double L = ext * (1.0 + ldexp(1.0, -20));
    if (!(L > 0.0))
        L = 1.0;
    out[3] = L;
    for (int k = 0; k < 3; k++)
        out[4 + k] = out[k] - 0.5 * L;
}

static int32_t grid_coord(double x, double corner, double scale)
{
    const double f = floor((x - corner) * scale);
    if (f < 0.0)
        return 0;
    if (f > (double)(OR_GRID - 1))
        return OR_GRID - 1;
    return (int32_t)f;
}

void or_quantize(int64_t n, const double *pos, const double *root, int32_t *q)
{
    const double scale = (double)OR_GRID / root[3];
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++)
            q[3 * i + k] = grid_coord(pos[3 * i + k], root[4 + k], scale);
}

/* Morton key by brute-force bit interleaving: for each level from the top,
 * append the x, y and z bits of the grid coordinate (Morton order, Sec.
 * "Test and Optimization").                                               */
void or_morton_keys(int64_t n, const int32_t *q, uint64_t *key)
{
    for (int64_t i = 0; i < n; i++) {
        uint64_t k = 0;
        for (int b = OR_LEVELS - 1; b >= 0; b--) {
            k = (k << 1) | (uint64_t)((q[3 * i + 0] >> b) & 1);
            k = (k << 1) | (uint64_t)((q[3 * i + 1] >> b) & 1);
            k = (k << 1) | (uint64_t)((q[3 * i + 2] >> b) & 1);
        }
        key[i] = k;
    }
}

/* Peano-Hilbert key: the 3-D Hilbert index of the grid coordinate, the
 * order the paper names as a better alternative to Morton order for data
 * locality (Sec. "Test and Optimization").  Skilling's transpose method
 * (J. Skilling 2004, "Programming the Hilbert curve", AIP Conf. Proc. 707):
 * going down the levels, each bit plane first undoes the reflection or the
 * exchange of axes that the curve applies inside the current sub-cube; the
 * three words are then Gray-coded, and their bits interleaved level by level
 * from the top like a Morton key (x, y, z).  63 bits, 21 levels.            */
void or_hilbert_keys(int64_t n, const int32_t *q, uint64_t *key)
{
    const uint32_t top = 1u << (OR_LEVELS - 1);
    for (int64_t i = 0; i < n; i++) {
        uint32_t w[3] = {(uint32_t)q[3 * i], (uint32_t)q[3 * i + 1], (uint32_t)q[3 * i + 2]};
        for (uint32_t bit = top; bit > 1; bit >>= 1) {
            const uint32_t below = bit - 1;
            for (int d = 0; d < 3; d++) {
                if (w[d] & bit) {
                    w[0] ^= below;                            /* reflect */
                } else {
                    const uint32_t swap = (w[0] ^ w[d]) & below; /* exchange 0, d */
                    w[0] ^= swap;
                    w[d] ^= swap;
                }
            }
        }
        w[1] ^= w[0];
        w[2] ^= w[1];
        uint32_t flip = 0;
        for (uint32_t bit = top; bit > 1; bit >>= 1)
            if (w[2] & bit)
                flip ^= bit - 1;
        for (int d = 0; d < 3; d++)
            w[d] ^= flip;
        uint64_t k = 0;
        for (int b = OR_LEVELS - 1; b >= 0; b--)
            for (int d = 0; d < 3; d++)
                k = (k << 1) | (uint64_t)((w[d] >> b) & 1u);
        key[i] = k;
    }
}

/* ------------------------------------------------------------------------ */
/* The oct-tree.  Nodes (cells and particle leaves) are numbered in the order
 * the recursive build creates them, which is depth-first preorder.        */

typedef struct {
    int64_t n;
    const double *pos;
    const float *mass;
    double root[7];
    int32_t *q;          /* n x 3 grid coordinates (caller order)            */
    int64_t *work;       /* particle indices being partitioned               */
    int64_t *tmp;
    int64_t *order;      /* depth-first leaf order: sorted slot -> caller    */
    int64_t *leaf;       /* sorted slot -> node id of its particle leaf      */
    int64_t nsorted;
    /* node arrays, capacity cap */
    int64_t nnodes, ncells, cap;
    int8_t *is_cell;
    int32_t *level;      /* cells: 0..21; particle leaves: -1                */
    int32_t *corner;     /* cells: integer corner at their level (x, y, z)   */
    int32_t *child;      /* cells: 8 sub-cell node ids, -1 if absent         */
    int32_t *nchild;
    int64_t *first, *count, *next, *more, *parent;
    double *M, *mx, *com; /* mass, first moment sum(m x), centre of mass     */
    float *l, *s, *comf;
    int korder;          /* 0: Morton order, 1: Peano-Hilbert order          */
    uint64_t *hkey;      /* Peano-Hilbert key per particle (korder 1)        */
    int8_t *corder;      /* cells: octants of the children in visiting order,
                          * -1 past the last                                 */
    double *Q;           /* traceless quadrupole per node about its centre of
                          * mass (xx, yy, zz, xy, xz, yz), made on demand     */
} or_tree;

static int grow(or_tree *t)
{
    int64_t nc = t->cap ? 2 * t->cap : 1024;
#define GROW(f, T, w)                                                      \
    do {                                                                   \
        void *p = realloc(t->f, (size_t)nc * (w) * sizeof(T));            \
        if (!p)                                                            \
            return -1;                                                     \
        t->f = (T *)p;                                                     \
    } while (0)
    GROW(is_cell, int8_t, 1);
    GROW(level, int32_t, 1);
    GROW(corner, int32_t, 3);
    GROW(child, int32_t, 8);
    GROW(nchild, int32_t, 1);
    GROW(first, int64_t, 1);
    GROW(count, int64_t, 1);
    GROW(next, int64_t, 1);
    GROW(more, int64_t, 1);
    GROW(parent, int64_t, 1);
    GROW(M, double, 1);
    GROW(mx, double, 3);
    GROW(com, double, 3);
    GROW(l, float, 1);
    GROW(s, float, 1);
    GROW(comf, float, 3);
    GROW(corder, int8_t, 8);
#undef GROW
    t->cap = nc;
    return 0;
}

static int64_t new_node(or_tree *t)
{
    if (t->nnodes == t->cap && grow(t))
        return -1;
    return t->nnodes++;
}

/* Recursive subdivision (Sec. "Oct-tree Method"): the cell at `level` with
 * integer corner (cx, cy, cz) holds work[lo .. lo+cnt).  Returns the node
 * id, or -1 on allocation failure.                                         */
static int64_t build_rec(or_tree *t, int64_t lo, int64_t cnt, int level,
                         int32_t cx, int32_t cy, int32_t cz, int64_t parent)
{
    const int64_t id = new_node(t);
    if (id < 0)
        return -1;
    t->parent[id] = parent;
    for (int o = 0; o < 8; o++) {
        t->child[8 * id + o] = -1;
        t->corder[8 * id + o] = -1;
    }
    if (cnt == 1) {
        /* "a cell has ... one particle": a particle leaf */
        const int64_t p = t->work[lo];
        t->is_cell[id] = 0;
        t->level[id] = -1;
        t->corner[3 * id] = t->corner[3 * id + 1] = t->corner[3 * id + 2] = 0;
        t->nchild[id] = 0;
        t->first[id] = t->nsorted;
        t->count[id] = 1;
        t->more[id] = -1;
        t->leaf[t->nsorted] = id;
        t->order[t->nsorted++] = p;
        t->M[id] = (double)t->mass[p];
        for (int k = 0; k < 3; k++) {
            t->com[3 * id + k] = t->pos[3 * p + k];
            t->mx[3 * id + k] = (double)t->mass[p] * t->pos[3 * p + k];
            t->comf[3 * id + k] = (float)t->pos[3 * p + k];
        }
        t->l[id] = 0.0f;
        t->s[id] = 0.0f;
        t->next[id] = t->nnodes;
        return id;
    }
    t->ncells++;
    t->is_cell[id] = 1;
    t->level[id] = level;
    t->corner[3 * id] = cx;
    t->corner[3 * id + 1] = cy;
    t->corner[3 * id + 2] = cz;
    t->first[id] = t->nsorted;
    t->count[id] = cnt;
    t->more[id] = id + 1;
    if (level == OR_LEVELS) {
        /* depth cap: the members stay as particle children in input order */
        for (int64_t k = 0; k < cnt; k++)
            if (build_rec(t, lo + k, 1, level + 1, 0, 0, 0, id) < 0)
                return -1;
    } else {
        const int b = OR_LEVELS - 1 - level;   /* grid bit of the child level */
        int64_t c[8] = {0}, off[8];
        for (int64_t k = 0; k < cnt; k++) {
            const int64_t p = t->work[lo + k];
            const int o = (((t->q[3 * p] >> b) & 1) << 2) |
                          (((t->q[3 * p + 1] >> b) & 1) << 1) |
                          ((t->q[3 * p + 2] >> b) & 1);
            c[o]++;
        }
        int64_t base[8];
        off[0] = 0;
        for (int o = 1; o < 8; o++)
            off[o] = off[o - 1] + c[o - 1];
        memcpy(base, off, sizeof(base));
        for (int64_t k = 0; k < cnt; k++) {   /* stable partition */
            const int64_t p = t->work[lo + k];
            const int o = (((t->q[3 * p] >> b) & 1) << 2) |
                          (((t->q[3 * p + 1] >> b) & 1) << 1) |
                          ((t->q[3 * p + 2] >> b) & 1);
            t->tmp[lo + off[o]++] = p;
        }
        memcpy(t->work + lo, t->tmp + lo, (size_t)cnt * sizeof(int64_t));
        /* the order the children are visited in: octant order, or the order
         * of their Peano-Hilbert digit at this level (every particle of an
         * aligned sub-cube has the same one) */
        int vis[8], nv = 0;
        for (int o = 0; o < 8; o++)
            if (c[o] > 0)
                vis[nv++] = o;
        if (t->korder == 1) {
            int dig[8];
            for (int v = 0; v < nv; v++)
                dig[v] = (int)((t->hkey[t->work[lo + base[vis[v]]]] >> (3 * b)) & 7u);
            for (int v = 1; v < nv; v++)       /* insertion sort by digit */
                for (int w = v; w > 0 && dig[w - 1] > dig[w]; w--) {
                    const int td = dig[w], to = vis[w];
                    dig[w] = dig[w - 1];
                    vis[w] = vis[w - 1];
                    dig[w - 1] = td;
                    vis[w - 1] = to;
                }
        }
        for (int v = 0; v < nv; v++) {
            const int o = vis[v];
            const int64_t ch = build_rec(t, lo + base[o], c[o], level + 1,
                                         2 * cx + ((o >> 2) & 1),
                                         2 * cy + ((o >> 1) & 1),
                                         2 * cz + (o & 1), id);
            if (ch < 0)
                return -1;
            t->child[8 * id + o] = (int32_t)ch;
            t->corder[8 * id + v] = (int8_t)o;
        }
    }
    /* total mass and centre of mass (Sec. "Our GPU implementation"),
     * folded over the children in the order they were visited (octant
     * order for Morton keys)                                             */
    double M = 0.0, mx[3] = {0.0, 0.0, 0.0};
    int32_t nch = 0;
    for (int64_t ch = id + 1; ch < t->nnodes; ch = t->next[ch]) {
        M += t->M[ch];
        for (int k = 0; k < 3; k++)
            mx[k] += t->mx[3 * ch + k];
        nch++;
    }
    t->nchild[id] = nch;
    t->M[id] = M;
    const double lc = ldexp(t->root[3], -level);
    double d2 = 0.0;
    for (int k = 0; k < 3; k++) {
        const int32_t ck = t->corner[3 * id + k];
        const double g = t->root[4 + k] + ((double)ck + 0.5) * lc;
        const double cm = (M > 0.0) ? mx[k] / M : g;
        t->mx[3 * id + k] = mx[k];
        t->com[3 * id + k] = cm;
        t->comf[3 * id + k] = (float)cm;
        const double d = cm - g;
        d2 = d2 + d * d;
    }
    t->l[id] = (float)lc;
    t->s[id] = (float)sqrt(d2);
    t->next[id] = t->nnodes;
    return id;
}

void or_tree_free(or_tree *t)
{
    if (!t)
        return;
    free(t->q);
    free(t->work);
    free(t->tmp);
    free(t->order);
    free(t->leaf);
    free(t->is_cell);
    free(t->level);
    free(t->corner);
    free(t->child);
    free(t->nchild);
    free(t->first);
    free(t->count);
    free(t->next);
    free(t->more);
    free(t->parent);
    free(t->M);
    free(t->mx);
    free(t->com);
    free(t->l);
    free(t->s);
    free(t->comf);
    free(t->hkey);
    free(t->corder);
    free(t->Q);
    free(t);
}

/* pos and mass must stay alive while the tree is used.  korder 0 visits
 * children in octant order (leaves in Morton order), 1 in Peano-Hilbert
 * order; the cells are the same either way.                               */
or_tree *or_tree_build_order(int64_t n, const double *pos, const float *mass, int korder)
{
    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    if (!t || n < 0 || korder < 0 || korder > 1) {
        free(t);
        return NULL;
    }
    t->korder = korder;
    t->n = n;
    t->pos = pos;
    t->mass = mass;
    or_root_cube(n, pos, t->root);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    t->q = (int32_t *)malloc(nn * 3 * sizeof(int32_t));
    t->work = (int64_t *)malloc(nn * sizeof(int64_t));
    t->tmp = (int64_t *)malloc(nn * sizeof(int64_t));
    t->order = (int64_t *)malloc(nn * sizeof(int64_t));
    t->leaf = (int64_t *)malloc(nn * sizeof(int64_t));
    if (!t->q || !t->work || !t->tmp || !t->order || !t->leaf) {
        or_tree_free(t);
        return NULL;
    }
    or_quantize(n, pos, t->root, t->q);
    if (korder == 1) {
        t->hkey = (uint64_t *)malloc(nn * sizeof(uint64_t));
        if (!t->hkey) {
            or_tree_free(t);
            return NULL;
        }
        or_hilbert_keys(n, t->q, t->hkey);
    }
    for (int64_t i = 0; i < n; i++)
        t->work[i] = i;
    if (n > 0) {
        if (build_rec(t, 0, n, 0, 0, 0, 0, -1) < 0) {
            or_tree_free(t);
            return NULL;
        }
        /* next past the last node is null */
        for (int64_t u = 0; u < t->nnodes; u++)
            if (t->next[u] >= t->nnodes)
                t->next[u] = -1;
    }
    return t;
}

or_tree *or_tree_build(int64_t n, const double *pos, const float *mass)
{
    return or_tree_build_order(n, pos, mass, 0);
}

/* the integer corner of every node at its level (zeros for particles) */
void or_tree_corners(const or_tree *t, int32_t *corner)
{
    memcpy(corner, t->corner, (size_t)t->nnodes * 3 * sizeof(int32_t));
}

int64_t or_tree_nnodes(const or_tree *t) { return t->nnodes; }
int64_t or_tree_ncells(const or_tree *t) { return t->ncells; }

void or_tree_root(const or_tree *t, double *out)
{
    memcpy(out, t->root, 7 * sizeof(double));
}

/* Copy the tree out.  Any pointer may be NULL.  Node arrays have nnodes
 * entries (x3 for vectors); order and q have n.                           */
void or_tree_export(const or_tree *t, int64_t *order, int32_t *q,
                    int8_t *is_cell, int32_t *level, int64_t *first,
                    int64_t *count, int64_t *next, int64_t *more,
                    int64_t *parent, int32_t *nchild, double *M, double *com,
                    float *l, float *s, float *comf)
{
    const size_t nn = (size_t)t->nnodes;
    if (order) memcpy(order, t->order, (size_t)t->n * sizeof(int64_t));
    if (q) memcpy(q, t->q, (size_t)t->n * 3 * sizeof(int32_t));
    if (is_cell) memcpy(is_cell, t->is_cell, nn);
    if (level) memcpy(level, t->level, nn * sizeof(int32_t));
    if (first) memcpy(first, t->first, nn * sizeof(int64_t));
    if (count) memcpy(count, t->count, nn * sizeof(int64_t));
    if (next) memcpy(next, t->next, nn * sizeof(int64_t));
    if (more) memcpy(more, t->more, nn * sizeof(int64_t));
    if (parent) memcpy(parent, t->parent, nn * sizeof(int64_t));
    if (nchild) memcpy(nchild, t->nchild, nn * sizeof(int32_t));
    if (M) memcpy(M, t->M, nn * sizeof(double));
    if (com) memcpy(com, t->com, nn * 3 * sizeof(double));
    if (l) memcpy(l, t->l, nn * sizeof(float));
    if (s) memcpy(s, t->s, nn * sizeof(float));
    if (comf) memcpy(comf, t->comf, nn * 3 * sizeof(float));
}

/* ------------------------------------------------------------------------ */
/* Groups: the nodes where a top-down descent first meets count <= n_crit.
 * gnode may be NULL to count.  Returns G.                                  */

static int64_t groups_rec(const or_tree *t, int64_t u, int64_t n_crit,
                          int64_t *gnode, int64_t g)
{
    if (t->count[u] <= n_crit) {
        if (gnode)
            gnode[g] = u;
        return g + 1;
    }
    if (t->level[u] == OR_LEVELS) {
        /* a bucket above n_crit: its particle leaves are groups */
        for (int64_t k = 0; k < t->count[u]; k++) {
            if (gnode)
                gnode[g] = u + 1 + k;
            g++;
        }
        return g;
    }
    for (int v = 0; v < 8 && t->corder[8 * u + v] >= 0; v++)
        g = groups_rec(t, t->child[8 * u + t->corder[8 * u + v]], n_crit, gnode, g);
    return g;
}

int64_t or_groups(const or_tree *t, int64_t n_crit, int64_t *gnode)
{
    if (t->nnodes == 0 || n_crit < 1)
        return 0;
    return groups_rec(t, 0, n_crit, gnode, 0);
}

/* Group bounding box of the members' FP32 positions and its FP32 centre.
 * box: G x 9 floats = lo[3], hi[3], centre[3].                             */
void or_group_boxes(const or_tree *t, int64_t G, const int64_t *gnode,
                    float *box)
{
    for (int64_t g = 0; g < G; g++) {
        const int64_t u = gnode[g];
        float lo[3], hi[3];
        for (int64_t k = 0; k < t->count[u]; k++) {
            const int64_t p = t->order[t->first[u] + k];
            for (int a = 0; a < 3; a++) {
                const float x = (float)t->pos[3 * p + a];
                if (k == 0 || x < lo[a])
                    lo[a] = x;
                if (k == 0 || x > hi[a])
                    hi[a] = x;
            }
        }
        for (int a = 0; a < 3; a++) {
            box[9 * g + a] = lo[a];
            box[9 * g + 3 + a] = hi[a];
            box[9 * g + 6 + a] = (float)(0.5 * ((double)lo[a] + (double)hi[a]));
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Opening test, Eq. (mac) with S_effective = (l/theta + s)^2, applied to a
 * whole group: d is the distance from the cell's centre of mass to the
 * group's bounding box.                                                    */

static float inv_theta(double theta) { return (float)(1.0 / theta); }

static int far_enough(const or_tree *t, int64_t u, const float *box,
                      float invth)
{
    float e[3];
    for (int a = 0; a < 3; a++) {
        const float c = t->comf[3 * u + a];
        const float below = box[a] - c;
        const float above = c - box[3 + a];
        float m = below > above ? below : above;
        e[a] = m > 0.0f ? m : 0.0f;
    }
    float d2 = e[0] * e[0];
    d2 = d2 + e[1] * e[1];
    d2 = d2 + e[2] * e[2];
    float w = t->l[u] * invth;
    w = w + t->s[u];
    const float S = w * w;
    return d2 > S;
}

static int holds_group(const or_tree *t, int64_t u, int64_t gfirst)
{
    return t->first[u] <= gfirst && gfirst < t->first[u] + t->count[u];
}

typedef struct {
    int64_t *out, cap, len;
} or_list;

static void emit(or_list *L, int64_t u)
{
    if (L->len < L->cap)
        L->out[L->len] = u;
    L->len++;
}

/* Fig. "treewalk": recursive, over sub-cells in the order they were built
 * (octant order for Morton keys). */
static void walk_rec(const or_tree *t, int64_t u, const float *box,
                     int64_t gfirst, float invth, or_list *L)
{
    if (!t->is_cell[u]) {
        emit(L, u);
        return;
    }
    if (!holds_group(t, u, gfirst) && far_enough(t, u, box, invth)) {
        emit(L, u);
        return;
    }
    if (t->level[u] == OR_LEVELS) {
        for (int64_t k = 0; k < t->count[u]; k++)
            emit(L, u + 1 + k);
        return;
    }
    for (int v = 0; v < 8 && t->corder[8 * u + v] >= 0; v++)
        walk_rec(t, t->child[8 * u + t->corder[8 * u + v]], box, gfirst, invth, L);
}

/* Fig. "treewalk_iterative": the same walk on next/more pointers. */
static void walk_iter(const or_tree *t, const float *box, int64_t gfirst,
                      float invth, or_list *L)
{
    int64_t u = 0;
    while (u != -1) {
        if (!t->is_cell[u]) {
            emit(L, u);
            u = t->next[u];
        } else if (!holds_group(t, u, gfirst) &&
                   far_enough(t, u, box, invth)) {
            emit(L, u);
            u = t->next[u];
        } else {
            u = t->more[u];
        }
    }
}

/* Interaction list of one group.  mode 0: recursive, 1: iterative.
 * Returns the list length (entries beyond cap are counted, not stored).   */
int64_t or_walk_group(const or_tree *t, int64_t gnode, const float *box,
                      double theta, int mode, int64_t *out, int64_t cap)
{
    or_list L = {out, cap, 0};
    if (t->nnodes == 0)
        return 0;
    const float invth = inv_theta(theta);
    const int64_t gfirst = t->first[gnode];
    if (mode == 0)
        walk_rec(t, 0, box, gfirst, invth, &L);
    else
        walk_iter(t, box, gfirst, invth, &L);
    return L.len;
}

/* Fig. "treegpu": one particle walks on its own; d^2 is measured from the
 * particle's FP32 position to the cell's FP32 centre of mass.             */
int64_t or_walk_particle(const or_tree *t, int64_t slot, double theta,
                         int64_t *out, int64_t cap)
{
    or_list L = {out, cap, 0};
    if (t->nnodes == 0)
        return 0;
    const float invth = inv_theta(theta);
    const int64_t p = t->order[slot];
    const float xi = (float)t->pos[3 * p], yi = (float)t->pos[3 * p + 1],
                zi = (float)t->pos[3 * p + 2];
    int64_t u = 0;
    while (u != -1) {
        const float dx = t->comf[3 * u] - xi;
        const float dy = t->comf[3 * u + 1] - yi;
        const float dz = t->comf[3 * u + 2] - zi;
        float r2 = dx * dx;
        r2 = r2 + dy * dy;
        r2 = r2 + dz * dz;
        if (!t->is_cell[u]) {
            emit(&L, u);
            u = t->next[u];
        } else {
            float w = t->l[u] * invth;
            w = w + t->s[u];
            if (r2 > w * w) {
                emit(&L, u);
                u = t->next[u];
            } else {
                u = t->more[u];
            }
        }
    }
    return L.len;
}

/* Every group's list, concatenated.  offsets has G+1 entries.  Returns the
 * total length (entries beyond cap are not stored).                        */
int64_t or_all_lists(const or_tree *t, int64_t G, const int64_t *gnode,
                     const float *box, double theta, int64_t *offsets,
                     int64_t *entries, int64_t cap)
{
    int64_t tot = 0;
    offsets[0] = 0;
    for (int64_t g = 0; g < G; g++) {
        int64_t *dst = (entries && tot < cap) ? entries + tot : NULL;
        const int64_t room = dst ? cap - tot : 0;
        tot += or_walk_group(t, gnode[g], box + 9 * g, theta, 1, dst, room);
        offsets[g + 1] = tot;
    }
    return tot;
}

/* ------------------------------------------------------------------------ */
/* Forces over interaction lists in FP64 (Eq. gravity with cells as point
 * masses at their centre of mass: monopole, Sec. "Oct-tree Method").
 * For the groups listed in gsel (all when gsel == NULL) every member gets
 * acc (caller order, x3) and pot.  theta_g (nullable) gives each group its
 * own opening angle.  npp / npc receive the particle-particle and
 * particle-cell interaction counts (self pairs not counted).  amag
 * (nullable) receives sum_j |a_ij|, the scale of the rounding error of the
 * summed acceleration.
 * coords32 != 0 first rounds every position and centre of mass to the
 * group-relative FP32 coordinate the force sum is defined on (rel32 below:
 * the FP64 value carried as two floats, differenced from the group's FP32
 * box centre in FP32) and cells' masses to FP32, then sums in FP64: the
 * result differs from the FP32 sums of the same lists only by arithmetic. */
static float rel32(double x, float c)
{
    const float hi = (float)x;
    const float lo = (float)(x - (double)hi);
    const float d = hi - c;
    return d + lo;
}

/* ------------------------------------------------------------------------ */
/* Neighbour search by the general treewalk (Sec. "General Treewalk", Fig.
 * "general_treewalk"): the descent of the force walk with another distance
 * test and no particle-cell term.  The neighbours of particle i are the
 * j != i with |x_j - x_i|^2 <= h^2, the squared distance summed x, y, z in
 * FP64 from the FP64 positions.  distance_test skips a cell whose cube,
 * widened by 1e-9 L (far more than the rounding of the grid), lies farther
 * than h from the target (per-particle form) or from the group's FP64
 * bounding box (group form); proc_particle applies the definition.        */

static double pair_d2(const double *a, const double *b)
{
    const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* squared gap between a cell's cube and the box [lo, hi] */
static double cube_gap2(const or_tree *t, int64_t u, const double *lo, const double *hi)
{
    const double side = ldexp(t->root[3], -t->level[u]);
    double d2 = 0.0;
    for (int k = 0; k < 3; k++) {
        const double c0 = t->root[4 + k] + (double)t->corner[3 * u + k] * side;
        const double c1 = c0 + side;
        double gap = 0.0;
        if (lo[k] > c1)
            gap = lo[k] - c1;
        else if (c0 > hi[k])
            gap = c0 - hi[k];
        d2 += gap * gap;
    }
    return d2;
}

typedef struct {
    int64_t *cand, len, cap;   /* candidate sorted slots */
} or_cand;

static int cand_push(or_cand *c, int64_t slot)
{
    if (c->len == c->cap) {
        const int64_t nc = c->cap ? 2 * c->cap : 256;
        int64_t *p = (int64_t *)realloc(c->cand, (size_t)nc * sizeof(int64_t));
        if (!p)
            return -1;
        c->cand = p;
        c->cap = nc;
    }
    c->cand[c->len++] = slot;
    return 0;
}

/* the general treewalk: every particle of every cell that passes the test */
static int near_rec(const or_tree *t, int64_t u, const double *lo, const double *hi,
                    double reach2, or_cand *c)
{
    if (!t->is_cell[u])
        return cand_push(c, t->first[u]);
    if (cube_gap2(t, u, lo, hi) > reach2)
        return 0;                                   /* too far: skipped */
    if (t->level[u] == OR_LEVELS) {
        for (int64_t k = 0; k < t->count[u]; k++)
            if (cand_push(c, t->first[u] + k))
                return -1;
        return 0;
    }
    for (int v = 0; v < 8 && t->corder[8 * u + v] >= 0; v++)
        if (near_rec(t, t->child[8 * u + t->corder[8 * u + v]], lo, hi, reach2, c))
            return -1;
    return 0;
}

static int cmp_i64(const void *a, const void *b)
{
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* One target's neighbours from a candidate list, as sorted caller indices.
 * Returns the count; writes out[0 .. min(count, cap)).                    */
static int64_t filter(const or_tree *t, int64_t i, double h2, const or_cand *c,
                      int64_t *out, int64_t cap)
{
    int64_t m = 0;
    for (int64_t k = 0; k < c->len; k++) {
        const int64_t j = t->order[c->cand[k]];
        if (j != i && pair_d2(t->pos + 3 * i, t->pos + 3 * j) <= h2) {
            if (m < cap)
                out[m] = j;
            m++;
        }
    }
    if (out && m <= cap)
        qsort(out, (size_t)m, sizeof(int64_t), cmp_i64);
    return m;
}

/* Neighbours of every particle (caller order) in CSR form: off has n + 1
 * entries, idx the sorted caller indices of each target's neighbours (up to
 * cap in all; NULL to count).  group_form 0 walks once per particle, 1 once
 * per group of <= n_crit particles with the group's bounding box.  Returns
 * the total, or -1 on allocation failure.                                 */
int64_t or_neighbours(const or_tree *t, double h, int group_form, int64_t n_crit,
                      int64_t *off, int64_t *idx, int64_t cap)
{
    const int64_t n = t->n;
    const double h2 = h * h;
    const double reach = h + 1e-9 * t->root[3];
    const double reach2 = reach * reach;
    int64_t *cnt = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!cnt)
        return -1;
    or_cand c = {NULL, 0, 0};
    int rc = 0;
    for (int pass = 0; pass < 2 && rc == 0; pass++) {
        if (pass == 1) {           /* offsets from the counts */
            int64_t tot = 0;
            for (int64_t i = 0; i < n; i++) {
                off[i] = tot;
                tot += cnt[i];
            }
            off[n] = tot;
            if (!idx)
                break;
        }
        if (!group_form) {
            for (int64_t i = 0; i < n && rc == 0; i++) {
                c.len = 0;
                const double *x = t->pos + 3 * i;
                if (n > 0 && near_rec(t, 0, x, x, reach2, &c)) {
                    rc = -1;
                    break;
                }
                if (pass == 0)
                    cnt[i] = filter(t, i, h2, &c, NULL, 0);
                else if (off[i + 1] <= cap)
                    filter(t, i, h2, &c, idx + off[i], cnt[i]);
            }
        } else if (n > 0) {
            const int64_t G = groups_rec(t, 0, n_crit, NULL, 0);
            int64_t *gnode = (int64_t *)malloc((size_t)G * sizeof(int64_t));
            if (!gnode) {
                rc = -1;
                break;
            }
            groups_rec(t, 0, n_crit, gnode, 0);
            for (int64_t g = 0; g < G && rc == 0; g++) {
                const int64_t u = gnode[g];
                double lo[3], hi[3];
                for (int k = 0; k < 3; k++) {
                    lo[k] = INFINITY;
                    hi[k] = -INFINITY;
                }
                for (int64_t s2 = t->first[u]; s2 < t->first[u] + t->count[u]; s2++)
                    for (int k = 0; k < 3; k++) {
                        const double x = t->pos[3 * t->order[s2] + k];
                        if (x < lo[k])
                            lo[k] = x;
                        if (x > hi[k])
                            hi[k] = x;
                    }
                c.len = 0;
                if (near_rec(t, 0, lo, hi, reach2, &c)) {
                    rc = -1;
                    break;
                }
                for (int64_t s2 = t->first[u]; s2 < t->first[u] + t->count[u]; s2++) {
                    const int64_t i = t->order[s2];
                    if (pass == 0)
                        cnt[i] = filter(t, i, h2, &c, NULL, 0);
                    else if (off[i + 1] <= cap)
                        filter(t, i, h2, &c, idx + off[i], cnt[i]);
                }
            }
            free(gnode);
        }
    }
    int64_t tot = 0;
    for (int64_t i = 0; i < n; i++)
        tot += cnt[i];
    free(c.cand);
    free(cnt);
    return rc ? -1 : tot;
}

/* The definition itself, for the tests: every pair, same distance formula. */
int64_t or_neighbours_brute(int64_t n, const double *pos, double h, int64_t *off,
                            int64_t *idx, int64_t cap)
{
    const double h2 = h * h;
    int64_t tot = 0;
    for (int64_t i = 0; i < n; i++) {
        if (off)
            off[i] = tot;
        for (int64_t j = 0; j < n; j++)
            if (j != i && pair_d2(pos + 3 * i, pos + 3 * j) <= h2) {
                if (idx && tot < cap)
                    idx[tot] = j;
                tot++;
            }
    }
    if (off)
        off[n] = tot;
    return tot;
}

/* ------------------------------------------------------------------------ */
/* Quadrupole moments ("any high order moment" of Sec. "Oct-tree Method"),
 * straight from the definition: for every cell, over its members k,
 *   Q_ab = sum_k m_k (3 d_a d_b - |d|^2 delta_ab),  d = x_k - COM,
 * in FP64 (particles: Q = 0).  The particle-cell term with it, softened like
 * Eq. (gravity) (R^2 = |r|^2 + eps^2, r = x_i - COM):
 *   phi += -(1/2) r.Q.r / R^5,   a += Q r / R^5 - (5/2) (r.Q.r) r / R^7.   */
int or_tree_quadrupoles(or_tree *t)
{
    if (t->Q)
        return 0;
    t->Q = (double *)calloc((size_t)(t->nnodes > 0 ? t->nnodes : 1) * 6, sizeof(double));
    if (!t->Q)
        return -1;
    for (int64_t u = 0; u < t->nnodes; u++) {
        if (!t->is_cell[u])
            continue;
        double q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t s2 = t->first[u]; s2 < t->first[u] + t->count[u]; s2++) {
            const int64_t j = t->order[s2];
            const double m = (double)t->mass[j];
            double d[3];
            for (int k = 0; k < 3; k++)
                d[k] = t->pos[3 * j + k] - t->com[3 * u + k];
            const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            q[0] += m * (3.0 * d[0] * d[0] - d2);
            q[1] += m * (3.0 * d[1] * d[1] - d2);
            q[2] += m * (3.0 * d[2] * d[2] - d2);
            q[3] += m * 3.0 * d[0] * d[1];
            q[4] += m * 3.0 * d[0] * d[2];
            q[5] += m * 3.0 * d[1] * d[2];
        }
        memcpy(t->Q + 6 * u, q, sizeof(q));
    }
    return 0;
}

int or_tree_export_quad(or_tree *t, double *Q)
{
    if (or_tree_quadrupoles(t))
        return -1;
    memcpy(Q, t->Q, (size_t)t->nnodes * 6 * sizeof(double));
    return 0;
}

static int tree_forces(const or_tree *t, int64_t n_crit, double theta,
                       const float *theta_g, double eps, int64_t nsel,
                       const int64_t *gsel, double *acc, double *pot,
                       double *amag, int64_t *npp, int64_t *npc, int coords32,
                       int quad);

int or_tree_forces(const or_tree *t, int64_t n_crit, double theta,
                   const float *theta_g, double eps, int64_t nsel,
                   const int64_t *gsel, double *acc, double *pot,
                   double *amag, int64_t *npp, int64_t *npc, int coords32)
{
    return tree_forces(t, n_crit, theta, theta_g, eps, nsel, gsel, acc, pot, amag, npp,
                       npc, coords32, 0);
}

/* the same with the quadrupole term of accepted cells (FP64 coordinates, or
 * with coords32 the group-relative FP32 coordinates and FP32 masses of
 * or_tree_forces; the quadrupoles stay FP64); amag (nullable) as there */
int or_tree_forces_quad(or_tree *t, int64_t n_crit, double theta, double eps,
                        double *acc, double *pot, double *amag, int64_t *npp, int64_t *npc,
                        int coords32)
{
    if (or_tree_quadrupoles(t))
        return -1;
    return tree_forces(t, n_crit, theta, NULL, eps, 0, NULL, acc, pot, amag, npp, npc,
                       coords32, 1);
}

static int tree_forces(const or_tree *t, int64_t n_crit, double theta,
                       const float *theta_g, double eps, int64_t nsel,
                       const int64_t *gsel, double *acc, double *pot,
                       double *amag, int64_t *npp, int64_t *npc, int coords32,
                       int quad)
{
    const int64_t G = or_groups(t, n_crit, NULL);
    int64_t *gnode = (int64_t *)malloc((size_t)(G > 0 ? G : 1) * sizeof(int64_t));
    float *box = (float *)malloc((size_t)(G > 0 ? G : 1) * 9 * sizeof(float));
    if (!gnode || !box) {
        free(gnode);
        free(box);
        return -1;
    }
    or_groups(t, n_crit, gnode);
    or_group_boxes(t, G, gnode, box);
    const int64_t ng = gsel ? nsel : G;
    const double e2 = eps * eps;
    int64_t cpp = 0, cpc = 0;
    int err = 0;
#pragma omp parallel reduction(+ : cpp, cpc)
    {
        int64_t cap = 4096;
        int64_t *lst = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < ng; k++) {
            if (!lst) {
                err = 1;
                continue;
            }
            const int64_t g = gsel ? gsel[k] : k;
            const double th = theta_g ? (double)theta_g[g] : theta;
            int64_t len = or_walk_group(t, gnode[g], box + 9 * g, th, 1, lst, cap);
            if (len > cap) {
                free(lst);
                cap = len;
                lst = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
                if (!lst) {
                    err = 1;
                    continue;
                }
                len = or_walk_group(t, gnode[g], box + 9 * g, th, 1, lst, cap);
            }
            int64_t ncell = 0;
            for (int64_t e = 0; e < len; e++)
                ncell += t->is_cell[lst[e]];
            const int64_t u = gnode[g];
            const float *cg = box + 9 * g + 6;
            for (int64_t m = 0; m < t->count[u]; m++) {
                const int64_t slot = t->first[u] + m;
                const int64_t i = t->order[slot];
                const int64_t self = t->leaf[slot];
                double xi = t->pos[3 * i], yi = t->pos[3 * i + 1],
                       zi = t->pos[3 * i + 2];
                if (coords32) {
                    xi = rel32(xi, cg[0]);
                    yi = rel32(yi, cg[1]);
                    zi = rel32(zi, cg[2]);
                }
                double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0, am = 0.0;
                for (int64_t e = 0; e < len; e++) {
                    const int64_t v = lst[e];
                    if (v == self)
                        continue;
                    double xv = t->com[3 * v], yv = t->com[3 * v + 1],
                           zv = t->com[3 * v + 2], mv = t->M[v];
                    if (coords32) {
                        xv = rel32(xv, cg[0]);
                        yv = rel32(yv, cg[1]);
                        zv = rel32(zv, cg[2]);
                        mv = (double)(float)mv;
                    }
                    const double dx = xv - xi;
                    const double dy = yv - yi;
                    const double dz = zv - zi;
                    const double r2 = dx * dx + dy * dy + dz * dz + e2;
                    if (r2 == 0.0)
                        continue;
                    const double rinv = 1.0 / sqrt(r2);
                    const double mr3 = mv * rinv * rinv * rinv;
                    ax += mr3 * dx;
                    ay += mr3 * dy;
                    az += mr3 * dz;
                    p -= mv * rinv;
                    am += mr3 * sqrt(dx * dx + dy * dy + dz * dz);
                    if (quad && t->is_cell[v]) {
                        /* r = x_i - COM = -(dx, dy, dz) */
                        const double *Q = t->Q + 6 * v;
                        const double rx = -dx, ry = -dy, rz = -dz;
                        const double qx = Q[0] * rx + Q[3] * ry + Q[4] * rz;
                        const double qy = Q[3] * rx + Q[1] * ry + Q[5] * rz;
                        const double qz = Q[4] * rx + Q[5] * ry + Q[2] * rz;
                        const double rqr = rx * qx + ry * qy + rz * qz;
                        const double ri2 = rinv * rinv;
                        const double ri5 = ri2 * ri2 * rinv;
                        const double ri7 = ri5 * ri2;
                        ax += qx * ri5 - 2.5 * rqr * rx * ri7;
                        ay += qy * ri5 - 2.5 * rqr * ry * ri7;
                        az += qz * ri5 - 2.5 * rqr * rz * ri7;
                        p -= 0.5 * rqr * ri5;
                    }
                }
                if (amag)
                    amag[i] = am;
                acc[3 * i] = ax;
                acc[3 * i + 1] = ay;
                acc[3 * i + 2] = az;
                pot[i] = p;
                cpc += ncell;
                cpp += len - ncell - 1;
            }
        }
        free(lst);
    }
    free(gnode);
    free(box);
    if (npp)
        *npp = cpp;
    if (npc)
        *npc = cpc;
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Kick-drift-kick leapfrog for "integrate orbits ... and repeat" (Sec.
 * Introduction), in FP64.  Accelerations come from the direct sum
 * (use_tree == 0) or from this file's tree code.  acc (n x 3, in/out) holds
 * the accelerations at the current positions; have_acc == 0 computes them
 * first.                                                                   */
static int accel(int64_t n, const double *pos, const float *mass, double eps,
                 int use_tree, double theta, int64_t n_crit, double *acc,
                 double *pot)
{
    if (!use_tree)
        return or_direct(n, pos, mass, eps, n, NULL, acc, pot, NULL);
    or_tree *t = or_tree_build(n, pos, mass);
    if (!t)
        return -1;
    const int rc = or_tree_forces(t, n_crit, theta, NULL, eps, 0, NULL, acc,
                                  pot, NULL, NULL, NULL, 0);
    or_tree_free(t);
    return rc;
}

int or_leapfrog(int64_t n, double *pos, double *vel, const float *mass,
                double eps, double dt, int64_t nsteps, int use_tree,
                double theta, int64_t n_crit, double *acc, int have_acc)
{
    double *pot = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!pot)
        return -1;
    int rc = 0;
    if (!have_acc)
        rc = accel(n, pos, mass, eps, use_tree, theta, n_crit, acc, pot);
    const double h = 0.5 * dt;
    for (int64_t st = 0; st < nsteps && rc == 0; st++) {
        for (int64_t i = 0; i < 3 * n; i++)
            vel[i] = vel[i] + acc[i] * h;
        for (int64_t i = 0; i < 3 * n; i++)
            pos[i] = pos[i] + vel[i] * dt;
        rc = accel(n, pos, mass, eps, use_tree, theta, n_crit, acc, pot);
        for (int64_t i = 0; i < 3 * n; i++)
            vel[i] = vel[i] + acc[i] * h;
    }
    free(pot);
    return rc;
}
