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
static constexpr int F_MASK_UNROLL = 8;   // unroll of the masked phase
// item word: first member | log2(source streams) << 27 | two-targets-per-lane flag
#define ITEM_R2 (1 << 30)
#define ITEM_LS_SHIFT 27
#define ITEM_MEMBER_MASK ((1 << 27) - 1)

enum { MODE_FP32 = 0, MODE_COMP = 1, MODE_F64 = 2 };

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

