// nb_force.cuh -- the arithmetic of Eq. (gravity) shared by the list force
// kernel (nb_force.cu) and the fused walk-and-force kernel (nb_fused.cu):
// one interaction, the accumulators of the three precision modes, the pass
// of a warp over a shared-memory tile of source records, and the sum of a
// lane's source streams.  Per interaction:
//   dx = xj - xi (3 FADD); r2 = eps^2 + dx.dx (3 FFMA); ri = rsqrt(r2) (MUFU);
//   mr = mj ri; mr3 = mr ri ri (3 FMUL); a += mr3 dx (3 FFMA); phi -= mr (FADD)
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
    float x, y, z, p;        // running (or per-tile) sums
    float cx, cy, cz, cp;    // Kahan compensation (MODE_COMP)
    double dx, dy, dz, dp;   // FP64 sums (MODE_F64)
    __device__ __forceinline__ void init()
    {
        x = y = z = p = 0.f;
        cx = cy = cz = cp = 0.f;
        dx = dy = dz = dp = 0.0;
    }
};

__device__ __forceinline__ void kahan(float &s, float &c, float v)
{
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

template <int MODE, bool GUARD, bool MASK>
__device__ __forceinline__ void interact(const float4 q, float xi, float yi, float zi,
                                         float eps2, bool me, Acc<MODE> &A)
{
    const float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
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
    const float mr = m * ri;
    const float mr3 = mr * (ri * ri);
    if (MODE == MODE_F64) {
        A.dx += (double)(mr3 * dx);
        A.dy += (double)(mr3 * dy);
        A.dz += (double)(mr3 * dz);
        A.dp -= (double)mr;
    } else {
        A.x = fmaf(mr3, dx, A.x);
        A.y = fmaf(mr3, dy, A.y);
        A.z = fmaf(mr3, dz, A.z);
        A.p -= mr;
    }
}

// NJ records of a tile against the lane's R targets
// UNR: unroll of the unmasked pass (0: in full)
template <int MODE, bool GUARD, bool MASK, int R, int NJ, int UNR = 0>
__device__ __forceinline__ void tile_pass(const float4 *tile, int32_t j0, const float *xi,
                                          const float *yi, const float *zi, const int32_t *kk,
                                          float eps2, Acc<MODE> *A, Acc<MODE> *T)
{
    // the list phase is unrolled in full; the masked phase (the group's own
    // members, a few per cent of the work) is kept short for the I-cache
    auto rec = [&](int j) {
        const float4 q = tile[j];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const bool me = MASK && (j0 + j == kk[r]);
            if constexpr (MODE == MODE_COMP)
                interact<MODE, GUARD, MASK>(q, xi[r], yi[r], zi[r], eps2, me, T[r]);
            else
                interact<MODE, GUARD, MASK>(q, xi[r], yi[r], zi[r], eps2, me, A[r]);
        }
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
    if constexpr (MODE == MODE_COMP) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            kahan(A[r].x, A[r].cx, T[r].x);
            kahan(A[r].y, A[r].cy, T[r].y);
            kahan(A[r].z, A[r].cz, T[r].z);
            kahan(A[r].p, A[r].cp, T[r].p);
            T[r].x = T[r].y = T[r].z = T[r].p = 0.f;
        }
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

