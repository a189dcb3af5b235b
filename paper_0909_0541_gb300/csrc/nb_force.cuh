// nb_force.cuh -- the arithmetic of Eq. (gravity) shared by the list force
// kernel (nb_force.cu) and the fused walk-and-force kernel (nb_fused.cu):
// one interaction, the accumulators of the three precision modes, the pass
// of a warp over a shared-memory tile of source records, and the sum of a
// lane's source streams.  Per interaction:
//   dx = xj - xi (3 FADD); r2 = eps^2 + dx.dx (3 FFMA); ri = rsqrt(r2) (MUFU);
//   mr = mj ri; mr3 = mr ri ri (3 FMUL); a += mr3 dx (3 FFMA); phi -= mr (FADD)
// In the FP32 modes two records go through each step at once with Blackwell's
// packed FP32 instructions (add/mul/fma .f32x2): 13 instructions and two MUFU
// per two interactions.  Each lane then holds two partial sums per component
// (even and odd records), added at the end.
#pragma once
#include <float.h>

#include "nb_internal.cuh"

#define F_TILE 32   // list records staged per tile (a multiple of 32)
// Items of more than one source stream stage at least F_TILE_STREAMS list
// records per tile, so that each stream still sums several record pairs per
// tile (the list force kernel, the overlapped kernel and the fused pass all
// use this rule, so their sums run in the same order)
#define F_TILE_STREAMS 64
__host__ __device__ constexpr int item_tile(int S, int tile)
{
    return S > 1 && tile < F_TILE_STREAMS ? F_TILE_STREAMS : tile;
}
static constexpr int F_MASK_UNROLL = 8;   // unroll of the masked phase
// item word: first member | ls << 27 (an item of 32 >> ls targets) | 64-target flag
#define ITEM_R2 (1 << 30)
#define ITEM_LS_SHIFT 27
#define ITEM_MEMBER_MASK ((1 << 27) - 1)

enum { MODE_FP32 = 0, MODE_COMP = 1, MODE_F64 = 2 };

// The shape an item is summed in, CALL(R, S): R targets per lane, S source
// streams (the warp as S rows of 32/S lanes, each row over 1/S of every
// tile).  A 64-target item runs as (2, 1).  A tail item of 32/2^ls targets
// (ls = 0..3: 32, 16, 8, 4 targets) runs as (2, 2^(ls+1)): two targets per
// lane, so each staged record pair feeds two interactions per lane, as in a
// full item.  Tails of two and one targets run as (1, 16) and (1, 32): with
// two targets per lane their streams would hold a single record per tile and
// lose the paired arithmetic.
#define NB_ITEM_SHAPES(word, CALL)                                                           \
    do {                                                                                      \
        if ((word) & ITEM_R2) {                                                               \
            CALL(2, 1);                                                                       \
        } else {                                                                              \
            switch (((word) >> ITEM_LS_SHIFT) & 7) {                                          \
            case 0: CALL(2, 2); break;                                                        \
            case 1: CALL(2, 4); break;                                                        \
            case 2: CALL(2, 8); break;                                                        \
            case 3: CALL(2, 16); break;                                                       \
            case 4: CALL(1, 16); break;                                                       \
            default: CALL(1, 32); break;                                                      \
            }                                                                                 \
        }                                                                                     \
    } while (0)

__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int MODE>
struct Acc {
    float x, y, z, p;        // final sums (MODE_FP32), running sums (MODE_COMP)
    float cx, cy, cz, cp;    // Kahan compensation (MODE_COMP)
    double dx, dy, dz, dp;   // FP64 sums (MODE_F64)
    __device__ __forceinline__ void init()
    {
        x = y = z = p = 0.f;
        cx = cy = cz = cp = 0.f;
        dx = dy = dz = dp = 0.0;
    }
};

// FP32 pair sums of one target: .x over the even records of each pair, .y over
// the odd ones; p sums +m/r (the potential is its negation)
struct Sum2 {
    float2 x, y, z, p;
    __device__ __forceinline__ void init()
    {
        x = y = z = p = make_float2(0.f, 0.f);
    }
};

// a target's coordinates, negated and duplicated for the packed subtraction
// (x_j + (-x_i) is x_j - x_i exactly)
struct Tgt {
    float2 x, y, z;
    __device__ __forceinline__ void set(float xi, float yi, float zi)
    {
        x = make_float2(-xi, -xi);
        y = make_float2(-yi, -yi);
        z = make_float2(-zi, -zi);
    }
};

__device__ __forceinline__ void kahan(float &s, float &c, float v)
{
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Paired tile layout: records 2p and 2p+1 share slots 2p and 2p+1,
//   slot 2p = {x_2p, x_2p+1, y_2p, y_2p+1},  slot 2p+1 = {z_2p, z_2p+1, m_2p, m_2p+1},
// so one 16-byte shared load yields the operand pairs of the packed FP32
// instructions (add/mul/fma .f32x2) with no register moves.
__device__ __forceinline__ void put_rec(float4 *tile, int j, float4 v)
{
    float *t = reinterpret_cast<float *>(tile) + 4 * (j & ~1) + (j & 1);
    t[0] = v.x;
    t[2] = v.y;
    t[4] = v.z;
    t[6] = v.w;
}

__device__ __forceinline__ float4 get_rec(const float4 *tile, int j)
{
    const float *t = reinterpret_cast<const float *>(tile) + 4 * (j & ~1) + (j & 1);
    return make_float4(t[0], t[2], t[4], t[6]);
}

// one record against one target, scalar: the FP64-accumulated mode, and a
// lone record of an odd-length stream in the FP32 modes (into the .x halves)
template <int MODE, bool GUARD, bool MASK>
__device__ __forceinline__ void interact1(const float4 q, const Tgt &t, float eps2, bool me,
                                          Acc<MODE> &A, Sum2 &P)
{
    const float dx = q.x + t.x.x, dy = q.y + t.y.x, dz = q.z + t.z.x;
    float r2 = fmaf(dx, dx, eps2);
    r2 = fmaf(dy, dy, r2);
    r2 = fmaf(dz, dz, r2);
    float m = q.w;
    if (MASK) {
        r2 = me ? 1.0f : r2;
        m = me ? 0.0f : m;
    }
    float ri = mufu_rsqrt(r2);
    if (GUARD) ri = r2 >= FLT_MIN ? ri : 0.0f;
    const float mr = __fmul_rn(m, ri);
    const float mr3 = __fmul_rn(mr, __fmul_rn(ri, ri));
    if (MODE == MODE_F64) {
        A.dx += (double)(mr3 * dx);
        A.dy += (double)(mr3 * dy);
        A.dz += (double)(mr3 * dz);
        A.dp -= (double)mr;
    } else {
        P.x.x = fmaf(mr3, dx, P.x.x);
        P.y.x = fmaf(mr3, dy, P.y.x);
        P.z.x = fmaf(mr3, dz, P.z.x);
        P.p.x = __fadd_rn(P.p.x, mr);
    }
}

// records 2p, 2p+1 (slots a, b) against one target with packed FP32: the
// same operations, in the same order, as interact1 on each record
template <bool GUARD, bool MASK>
__device__ __forceinline__ void interact2(const float4 a, const float4 b, const Tgt &t,
                                          float2 e2, bool me0, bool me1, Sum2 &P)
{
    const float2 dx = __fadd2_rn(make_float2(a.x, a.y), t.x);
    const float2 dy = __fadd2_rn(make_float2(a.z, a.w), t.y);
    const float2 dz = __fadd2_rn(make_float2(b.x, b.y), t.z);
    float2 r2 = __ffma2_rn(dx, dx, e2);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    float2 m = make_float2(b.z, b.w);
    if (MASK) {
        r2.x = me0 ? 1.0f : r2.x;
        m.x = me0 ? 0.0f : m.x;
        r2.y = me1 ? 1.0f : r2.y;
        m.y = me1 ? 0.0f : m.y;
    }
    float2 ri = make_float2(mufu_rsqrt(r2.x), mufu_rsqrt(r2.y));
    if (GUARD) {
        ri.x = r2.x >= FLT_MIN ? ri.x : 0.0f;
        ri.y = r2.y >= FLT_MIN ? ri.y : 0.0f;
    }
    const float2 mr = __fmul2_rn(m, ri);
    const float2 mr3 = __fmul2_rn(mr, __fmul2_rn(ri, ri));
    P.x = __ffma2_rn(mr3, dx, P.x);
    P.y = __ffma2_rn(mr3, dy, P.y);
    P.z = __ffma2_rn(mr3, dz, P.z);
    P.p = __fadd2_rn(P.p, mr);
}

// NJ records rb .. rb+NJ-1 of a paired tile against the lane's R targets;
// j0 is the member index of record rb (for the j == i mask).
// UNR: unroll of the unmasked pass in records (0: in full)
template <int MODE, bool GUARD, bool MASK, int R, int NJ, int UNR = 0>
__device__ __forceinline__ void tile_pass(const float4 *tile, int rb, int32_t j0, const Tgt *t,
                                          const int32_t *kk, float eps2, Acc<MODE> *A, Sum2 *P)
{
    // the list phase is unrolled in full; the masked phase (the group's own
    // members, a few per cent of the work) is kept short for the I-cache
    constexpr bool PACKED = MODE != MODE_F64 && NJ % 2 == 0;
    if constexpr (PACKED) {
        const float2 e2 = make_float2(eps2, eps2);
        auto pair = [&](int q) {
            const float4 a = tile[rb + 2 * q], b = tile[rb + 2 * q + 1];
#pragma unroll
            for (int r = 0; r < R; r++) {
                const bool me0 = MASK && (j0 + 2 * q == kk[r]);
                const bool me1 = MASK && (j0 + 2 * q + 1 == kk[r]);
                interact2<GUARD, MASK>(a, b, t[r], e2, me0, me1, P[r]);
            }
        };
        if constexpr (MASK) {
#pragma unroll F_MASK_UNROLL / 2
            for (int q = 0; q < NJ / 2; q++) pair(q);
        } else if constexpr (UNR > 1) {
#pragma unroll UNR / 2
            for (int q = 0; q < NJ / 2; q++) pair(q);
        } else {
#pragma unroll
            for (int q = 0; q < NJ / 2; q++) pair(q);
        }
    } else {
        auto rec = [&](int j) {
            const float4 q = get_rec(tile, rb + j);
#pragma unroll
            for (int r = 0; r < R; r++)
                interact1<MODE, GUARD, MASK>(q, t[r], eps2, MASK && (j0 + j == kk[r]), A[r],
                                             P[r]);
        };
        if constexpr (MASK) {
#pragma unroll F_MASK_UNROLL
            for (int j = 0; j < NJ; j++) rec(j);
        } else if constexpr (UNR > 0) {
#pragma unroll UNR
            for (int j = 0; j < NJ; j++) rec(j);
        } else {
#pragma unroll
            for (int j = 0; j < NJ; j++) rec(j);
        }
    }
    if constexpr (MODE == MODE_COMP) {   // fold the tile's pair sums into the running sums
#pragma unroll
        for (int r = 0; r < R; r++) {
            kahan(A[r].x, A[r].cx, P[r].x.x);
            kahan(A[r].x, A[r].cx, P[r].x.y);
            kahan(A[r].y, A[r].cy, P[r].y.x);
            kahan(A[r].y, A[r].cy, P[r].y.y);
            kahan(A[r].z, A[r].cz, P[r].z.x);
            kahan(A[r].z, A[r].cz, P[r].z.y);
            kahan(A[r].p, A[r].cp, -P[r].p.x);
            kahan(A[r].p, A[r].cp, -P[r].p.y);
            P[r].init();
        }
    }
}

// the FP32 mode's final sums from the pair sums
template <int MODE>
__device__ __forceinline__ void pair_fold(Acc<MODE> &A, const Sum2 &P)
{
    if constexpr (MODE == MODE_FP32) {
        A.x = __fadd_rn(P.x.x, P.x.y);
        A.y = __fadd_rn(P.y.x, P.y.y);
        A.z = __fadd_rn(P.z.x, P.z.y);
        A.p = -__fadd_rn(P.p.x, P.p.y);
    }
}

template <int MODE>
__device__ __forceinline__ void stream_sum(Acc<MODE> &A, int o)
{
    const unsigned FULL = 0xffffffffu;
    if constexpr (MODE == MODE_F64) {
        A.dx += __shfl_xor_sync(FULL, A.dx, o);
        A.dy += __shfl_xor_sync(FULL, A.dy, o);
        A.dz += __shfl_xor_sync(FULL, A.dz, o);
        A.dp += __shfl_xor_sync(FULL, A.dp, o);
    } else {
        A.x += __shfl_xor_sync(FULL, A.x, o);
        A.y += __shfl_xor_sync(FULL, A.y, o);
        A.z += __shfl_xor_sync(FULL, A.z, o);
        A.p += __shfl_xor_sync(FULL, A.p, o);
        if constexpr (MODE == MODE_COMP) {
            A.cx += __shfl_xor_sync(FULL, A.cx, o);
            A.cy += __shfl_xor_sync(FULL, A.cy, o);
            A.cz += __shfl_xor_sync(FULL, A.cz, o);
            A.cp += __shfl_xor_sync(FULL, A.cp, o);
        }
    }
}


// ---------------------------------------------------------------- quadrupole
// Cells carry their traceless quadrupole Q about the centre of mass; the
// particle-cell term gains (softened like Eq. (gravity), R^2 = |r|^2 +
// eps^2, r = x_i - COM = -d with d = COM - x_i):
//   a += Q r / R^5 - (5/2) (r.Q.r) r / R^7 = -(Q d) R^-5 + (5/2)(d.Q.d) d R^-7
//   phi += -(1/2) (d.Q.d) R^-5
// The tile stores -Q, so with q' = (-Q) d and h = -(5/2) (d.(-Q).d) R^-7:
//   a += q' R^-5 + h d,   and the potential sum (+m/R, negated at the end)
//   gains (-1/2)(d.(-Q).d) R^-5.
// Paired layout of a quadrupole tile: records 2p, 2p+1 share five slots,
//   5p: {x, x', y, y'}  5p+1: {z, z', m, m'}  5p+2: {-Qxx, .., -Qyy, ..}
//   5p+3: {-Qzz, .., -Qxy, ..}  5p+4: {-Qxz, .., -Qyz, ..}
__device__ __forceinline__ void put_rec_q(float4 *tile, int j, float4 v, float4 qa, float4 qb)
{
    float *t = reinterpret_cast<float *>(tile) + 20 * (j >> 1) + (j & 1);
    t[0] = v.x;
    t[2] = v.y;
    t[4] = v.z;
    t[6] = v.w;
    t[8] = -qa.x;
    t[10] = -qa.y;
    t[12] = -qa.z;
    t[14] = -qa.w;
    t[16] = -qb.x;
    t[18] = -qb.y;
}

// two records against one target with packed FP32: the monopole steps of
// interact2, then the quadrupole term
template <bool GUARD>
__device__ __forceinline__ void interact2_quad(const float4 *sl, const Tgt &t, float2 e2, Sum2 &P)
{
    const float4 a = sl[0], b = sl[1], c = sl[2], d = sl[3], e = sl[4];
    const float2 dx = __fadd2_rn(make_float2(a.x, a.y), t.x);
    const float2 dy = __fadd2_rn(make_float2(a.z, a.w), t.y);
    const float2 dz = __fadd2_rn(make_float2(b.x, b.y), t.z);
    float2 r2 = __ffma2_rn(dx, dx, e2);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float2 m = make_float2(b.z, b.w);
    float2 ri = make_float2(mufu_rsqrt(r2.x), mufu_rsqrt(r2.y));
    if (GUARD) {
        ri.x = r2.x >= FLT_MIN ? ri.x : 0.0f;
        ri.y = r2.y >= FLT_MIN ? ri.y : 0.0f;
    }
    const float2 ri2 = __fmul2_rn(ri, ri);
    const float2 mr = __fmul2_rn(m, ri);
    const float2 mr3 = __fmul2_rn(mr, ri2);
    P.x = __ffma2_rn(mr3, dx, P.x);
    P.y = __ffma2_rn(mr3, dy, P.y);
    P.z = __ffma2_rn(mr3, dz, P.z);
    P.p = __fadd2_rn(P.p, mr);
    const float2 qxx = make_float2(c.x, c.y), qyy = make_float2(c.z, c.w);
    const float2 qzz = make_float2(d.x, d.y), qxy = make_float2(d.z, d.w);
    const float2 qxz = make_float2(e.x, e.y), qyz = make_float2(e.z, e.w);
    float2 qx = __fmul2_rn(qxx, dx);
    qx = __ffma2_rn(qxy, dy, qx);
    qx = __ffma2_rn(qxz, dz, qx);
    float2 qy = __fmul2_rn(qxy, dx);
    qy = __ffma2_rn(qyy, dy, qy);
    qy = __ffma2_rn(qyz, dz, qy);
    float2 qz = __fmul2_rn(qxz, dx);
    qz = __ffma2_rn(qyz, dy, qz);
    qz = __ffma2_rn(qzz, dz, qz);
    float2 dqd = __fmul2_rn(dx, qx);
    dqd = __ffma2_rn(dy, qy, dqd);
    dqd = __ffma2_rn(dz, qz, dqd);
    const float2 ri5 = __fmul2_rn(__fmul2_rn(ri2, ri2), ri);
    const float2 hp = __fmul2_rn(dqd, make_float2(-0.5f, -0.5f));
    const float2 h = __fmul2_rn(__fmul2_rn(hp, make_float2(5.0f, 5.0f)), __fmul2_rn(ri5, ri2));
    P.x = __ffma2_rn(ri5, qx, P.x);
    P.y = __ffma2_rn(ri5, qy, P.y);
    P.z = __ffma2_rn(ri5, qz, P.z);
    P.x = __ffma2_rn(h, dx, P.x);
    P.y = __ffma2_rn(h, dy, P.y);
    P.z = __ffma2_rn(h, dz, P.z);
    P.p = __ffma2_rn(hp, ri5, P.p);
}

// one record of a quadrupole tile, scalar (an odd-length stream), into the
// .x halves
template <bool GUARD>
__device__ __forceinline__ void interact1_quad(const float4 *tile, int j, const Tgt &t, float eps2,
                                               bool quad, Sum2 &P)
{
    const float *f = reinterpret_cast<const float *>(tile) + 20 * (j >> 1) + (j & 1);
    const float dx = f[0] + t.x.x, dy = f[2] + t.y.x, dz = f[4] + t.z.x;
    float r2 = fmaf(dx, dx, eps2);
    r2 = fmaf(dy, dy, r2);
    r2 = fmaf(dz, dz, r2);
    float ri = mufu_rsqrt(r2);
    if (GUARD) ri = r2 >= FLT_MIN ? ri : 0.0f;
    const float ri2 = __fmul_rn(ri, ri);
    const float mr = __fmul_rn(f[6], ri);
    const float mr3 = __fmul_rn(mr, ri2);
    P.x.x = fmaf(mr3, dx, P.x.x);
    P.y.x = fmaf(mr3, dy, P.y.x);
    P.z.x = fmaf(mr3, dz, P.z.x);
    P.p.x = __fadd_rn(P.p.x, mr);
    if (!quad) return;
    const float qxx = f[8], qyy = f[10], qzz = f[12], qxy = f[14], qxz = f[16], qyz = f[18];
    const float qx = fmaf(qxz, dz, fmaf(qxy, dy, qxx * dx));
    const float qy = fmaf(qyz, dz, fmaf(qyy, dy, qxy * dx));
    const float qz = fmaf(qzz, dz, fmaf(qyz, dy, qxz * dx));
    const float dqd = fmaf(dz, qz, fmaf(dy, qy, dx * qx));
    const float ri5 = ri2 * ri2 * ri;
    const float hp = -0.5f * dqd;
    const float h = (hp * 5.0f) * (ri5 * ri2);
    P.x.x = fmaf(h, dx, fmaf(ri5, qx, P.x.x));
    P.y.x = fmaf(h, dy, fmaf(ri5, qy, P.y.x));
    P.z.x = fmaf(h, dz, fmaf(ri5, qz, P.z.x));
    P.p.x = fmaf(hp, ri5, P.p.x);
}

// NJ records rb .. rb+NJ-1 of a quadrupole tile against the lane's R
// targets.  qmask bit j: record j carries a quadrupole (a cell); pairs of
// two particles take the monopole steps.  All lanes of one source stream read
// the same records, so the choice is uniform within the stream.
template <int MODE, bool GUARD, int R, int NJ>
__device__ __forceinline__ void tile_pass_quad(const float4 *tile, int rb, const Tgt *t,
                                               float eps2, unsigned qmask, Acc<MODE> *A, Sum2 *P)
{
    static_assert(MODE != MODE_F64, "the quadrupole pass sums in FP32");
    if constexpr (NJ % 2 == 0) {
        const float2 e2 = make_float2(eps2, eps2);
#pragma unroll 4
        for (int q = 0; q < NJ / 2; q++) {
            const int j = rb + 2 * q;
            const float4 *sl = tile + 5 * (j >> 1);
            if ((qmask >> j) & 3u) {
#pragma unroll
                for (int r = 0; r < R; r++) interact2_quad<GUARD>(sl, t[r], e2, P[r]);
            } else {
#pragma unroll
                for (int r = 0; r < R; r++)
                    interact2<GUARD, false>(sl[0], sl[1], t[r], e2, false, false, P[r]);
            }
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < NJ; jj++) {
            const int j = rb + jj;
#pragma unroll
            for (int r = 0; r < R; r++)
                interact1_quad<GUARD>(tile, j, t[r], eps2, (qmask >> j) & 1u, P[r]);
        }
    }
    if constexpr (MODE == MODE_COMP) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            kahan(A[r].x, A[r].cx, P[r].x.x);
            kahan(A[r].x, A[r].cx, P[r].x.y);
            kahan(A[r].y, A[r].cy, P[r].y.x);
            kahan(A[r].y, A[r].cy, P[r].y.y);
            kahan(A[r].z, A[r].cz, P[r].z.x);
            kahan(A[r].z, A[r].cz, P[r].z.y);
            kahan(A[r].p, A[r].cp, -P[r].p.x);
            kahan(A[r].p, A[r].cp, -P[r].p.y);
            P[r].init();
        }
    }
}
