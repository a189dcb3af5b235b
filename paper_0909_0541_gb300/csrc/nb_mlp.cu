// nb_mlp.cu -- the learned opening-angle network: forward, backward,
// weight gradients and Adam, as hand-written kernels on the tensor cores.
//
// Network: 12 features -> 64 -> 64 -> 64 -> 1 with GELU, theta = 0.3 +
// 0.9 sigmoid(z).  Matrix products run as mma.sync m16n8k16 with BF16
// operands (layer inputs and weights rounded to BF16) and FP32 accumulation;
// biases, GELU, the output layer and all gradients outside the products are
// FP32.  Master weights are FP32 and are rounded to BF16 when fragments are
// loaded.  A warp owns 16 samples (one m-tile); the weight gradients are
// products over the batch (dW = dZ^T X) computed by one warp per 16x8 tile.
// The matrices are tiny (K, N <= 64), so the warp-level MMA is used rather
// than 128-row tcgen05 tiles: a whole training step is a few microseconds.
//
// Flat FP32 parameters (offsets in floats): W1 0 (64x16), b1 1024,
// W2 1088 (64x64), b2 5184, W3 5248, b3 9344, w4 9408 (64), b4 9920,
// mu 9928 (16), sigma 9944 (16); 9960 in all.
#include <cuda_bf16.h>
#include <math.h>

#include "nb_internal.cuh"

#define MH 64
#define MKIN 16
#define MNIN 12
enum {
    P_W1 = 0, P_B1 = 1024, P_W2 = 1088, P_B2 = 5184, P_W3 = 5248, P_B3 = 9344,
    P_W4 = 9408, P_B4 = 9920, P_MU = 9928, P_SG = 9944, P_N = 9960
};
#define LAMBDA 4.0f
#define MLP_T 256

typedef __nv_bfloat16 bf16;

// workspace (per padded sample count Bp), all offsets 256-byte aligned
struct MlpWork {
    bf16 *a0, *a1, *a2, *d1, *d2, *d3;
    float *Z1, *Z2, *Z3, *h3, *g1, *g2, *g3, *s, *theta, *dz, *y, *loss;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t work_layout(int64_t Bp, MlpWork *w, char *base)
{
    size_t o = 0;
#define PUT(f, T, cnt)                                          \
    do {                                                        \
        if (w) w->f = (T *)(base + o);                          \
        o += al(sizeof(T) * (size_t)(cnt));                     \
    } while (0)
    PUT(a0, bf16, Bp * MKIN);
    PUT(a1, bf16, Bp * MH);
    PUT(a2, bf16, Bp * MH);
    PUT(d1, bf16, Bp * MH);
    PUT(d2, bf16, Bp * MH);
    PUT(d3, bf16, Bp * MH);
    PUT(Z1, float, Bp * MH);
    PUT(Z2, float, Bp * MH);
    PUT(Z3, float, Bp * MH);
    PUT(h3, float, Bp * MH);
    PUT(g1, float, Bp * MH);
    PUT(g2, float, Bp * MH);
    PUT(g3, float, Bp * MH);
    PUT(s, float, Bp);
    PUT(theta, float, Bp);
    PUT(dz, float, Bp);
    PUT(y, float, Bp);
    PUT(loss, float, Bp);
#undef PUT
    return o;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack2b(bf16 lo, bf16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float x)
{
    return x * 0.5f * (1.0f + erff(x * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float x)
{
    const float Phi = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float phi = expf(-0.5f * x * x) * 0.39894228040143268f;
    return Phi + x * phi;
}

// A fragment (16 x 16) of a row-major BF16 matrix X (rows r0.., cols k0..)
__device__ __forceinline__ void frag_a_rows(const bf16 *X, int ld, int r0, int k0, uint32_t a[4])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    a[0] = *reinterpret_cast<const uint32_t *>(X + (int64_t)(r0 + g) * ld + k0 + 2 * t);
    a[1] = *reinterpret_cast<const uint32_t *>(X + (int64_t)(r0 + g + 8) * ld + k0 + 2 * t);
    a[2] = *reinterpret_cast<const uint32_t *>(X + (int64_t)(r0 + g) * ld + k0 + 8 + 2 * t);
    a[3] = *reinterpret_cast<const uint32_t *>(X + (int64_t)(r0 + g + 8) * ld + k0 + 8 + 2 * t);
}

// B fragment (16 x 8) with B(k, n) = W[n][k], W FP32 row-major with K columns
__device__ __forceinline__ void frag_b_wt(const float *W, int K, int k0, int n0, uint32_t b[2])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    const float *p = W + (int64_t)(n0 + g) * K + k0 + 2 * t;
    b[0] = pack2(p[0], p[1]);
    b[1] = pack2(p[8], p[9]);
}

// B fragment with B(k, n) = W[k][n], W FP32 row-major with N columns
__device__ __forceinline__ void frag_b_w(const float *W, int N, int k0, int n0, uint32_t b[2])
{
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    const float *p = W + (int64_t)(k0 + 2 * t) * N + n0 + g;
    b[0] = pack2(p[0], p[N]);
    b[1] = pack2(p[8 * N], p[9 * N]);
}

// one hidden layer for a 16-row tile: acc = A (16 x K, BF16 rows) * W^T
template <int K>
__device__ __forceinline__ void mma_layer(const bf16 *A, int ldA, int r0, const float *W,
                                          float acc[8][4])
{
    uint32_t a[4], b[2];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < K / 16; kt++) {
        frag_a_rows(A, ldA, r0, kt * 16, a);
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            frag_b_wt(W, K, kt * 16, nt * 8, b);
            mma16816(acc[nt], a, b);
        }
    }
}

// z = w4 . h3 + b4 for the two rows (g, g + 8) a lane holds, FP32
__device__ __forceinline__ void out_z(const float acc[8][4], const float *P, float z[2])
{
    const int t = threadIdx.x & 3;
    float zr[2] = {0.f, 0.f};
#pragma unroll
    for (int nt = 0; nt < 8; nt++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int col = nt * 8 + 2 * t;
            zr[h] = fmaf(acc[nt][2 * h], P[P_W4 + col], zr[h]);
            zr[h] = fmaf(acc[nt][2 * h + 1], P[P_W4 + col + 1], zr[h]);
        }
#pragma unroll
    for (int h = 0; h < 2; h++) {
        zr[h] += __shfl_xor_sync(0xffffffffu, zr[h], 1);
        zr[h] += __shfl_xor_sync(0xffffffffu, zr[h], 2);
        z[h] = zr[h] + P[P_B4];
    }
}

__device__ __forceinline__ float norm_feature(const float *x, const float *P, int k)
{
    return k < MNIN ? __fdiv_rn(__fsub_rn(x[k], P[P_MU + k]), P[P_SG + k]) : 0.0f;
}

// ------------------------------------------------------------ input
// z0 = (x - mu) / sigma in FP32, rounded to BF16, padded to 16 columns;
// rows >= B are zero.  x has 16-float rows; idx (nullable) gathers rows;
// y (nullable) gathers labels alongside.
__global__ void __launch_bounds__(256)
k_mlp_input(const float *__restrict__ x, const int32_t *__restrict__ idx, const float *__restrict__ ylab,
            int64_t B, int64_t Bp, const float *__restrict__ P, bf16 *__restrict__ a0,
            float *__restrict__ yout)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= Bp * MKIN) return;
    const int64_t r = i / MKIN;
    const int k = (int)(i % MKIN);
    float v = 0.0f;
    if (r < B && k < MNIN) {
        const int64_t row = idx ? idx[r] : r;
        v = norm_feature(x + row * MKIN, P, k);
    }
    a0[i] = __float2bfloat16_rn(v);
    if (k == 0 && yout) yout[r] = (r < B && ylab) ? ylab[idx ? idx[r] : r] : 0.0f;
}

// ------------------------------------------------------------ forward
// one warp per 16-sample tile; keep = store the activations for backward
template <bool KEEP>
__global__ void __launch_bounds__(MLP_T)
k_mlp_fwd(const float *__restrict__ P, int64_t Bp, MlpWork w, float *__restrict__ theta_out,
          int64_t B, float fallback)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (tile * 16 >= Bp) return;
    const int r0 = (int)(tile * 16);
    float acc[8][4];
    const float *Ws[3] = {P + P_W1, P + P_W2, P + P_W3};
    const float *bs[3] = {P + P_B1, P + P_B2, P + P_B3};
    const bf16 *ins[3] = {w.a0, w.a1, w.a2};
    bf16 *outs[2] = {w.a1, w.a2};
    float *Zs[3] = {w.Z1, w.Z2, w.Z3};
    for (int L = 0; L < 3; L++) {
        if (L == 0) mma_layer<MKIN>(ins[0], MKIN, r0, Ws[0], acc);
        else mma_layer<MH>(ins[L], MH, r0, Ws[L], acc);
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int row = r0 + g + 8 * h, col = nt * 8 + 2 * t;
                const float z0 = acc[nt][2 * h] + bs[L][col];
                const float z1 = acc[nt][2 * h + 1] + bs[L][col + 1];
                if (KEEP) {
                    Zs[L][(int64_t)row * MH + col] = z0;
                    Zs[L][(int64_t)row * MH + col + 1] = z1;
                }
                const float g0 = gelu(z0), g1 = gelu(z1);
                acc[nt][2 * h] = g0;
                acc[nt][2 * h + 1] = g1;
                if (L < 2) {
                    *reinterpret_cast<uint32_t *>(outs[L] + (int64_t)row * MH + col) = pack2(g0, g1);
                } else if (KEEP) {
                    w.h3[(int64_t)row * MH + col] = g0;
                    w.h3[(int64_t)row * MH + col + 1] = g1;
                }
            }
        __syncwarp();
    }
    float z[2];
    out_z(acc, P, z);
    if (t == 0)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int row = r0 + g + 8 * h;
            const float s = 1.0f / (1.0f + expf(-z[h]));
            float th = 0.3f + 0.9f * s;
            if (KEEP) {
                w.s[row] = s;
                w.theta[row] = th;
            }
            if (theta_out && row < B) {
                if (!isfinite(th)) th = fallback;
                theta_out[row] = th;
            }
        }
}

// Inference for every group of a context: the same arithmetic as k_mlp_fwd
// with the layer activations in shared memory; the group count is read on
// the device (no host synchronisation, no workspace).
__global__ void __launch_bounds__(MLP_T)
k_mlp_infer(const float *__restrict__ P, const float *__restrict__ feat,
            const long long *__restrict__ cnt, float *__restrict__ theta, float fallback)
{
    __shared__ __align__(16) bf16 sbuf[MLP_T / 32][2][16 * MH];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t G = cnt[CNT_GROUPS];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    bf16 *b0 = sbuf[wl][0], *b1 = sbuf[wl][1];
    for (int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; tile * 16 < G;
         tile += nwarps) {
        const int64_t r0 = tile * 16;
        for (int e = lane; e < 16 * MKIN; e += 32) {
            const int r = e / MKIN, k = e % MKIN;
            const float v = r0 + r < G ? norm_feature(feat + (r0 + r) * MKIN, P, k) : 0.0f;
            b0[r * MKIN + k] = __float2bfloat16_rn(v);
        }
        __syncwarp();
        float acc[8][4];
        const float *Ws[3] = {P + P_W1, P + P_W2, P + P_W3};
        const float *bs[3] = {P + P_B1, P + P_B2, P + P_B3};
        for (int L = 0; L < 3; L++) {
            bf16 *src = (L == 1) ? b1 : b0;
            bf16 *dst = (L == 1) ? b0 : b1;
            if (L == 0) mma_layer<MKIN>(src, MKIN, 0, Ws[0], acc);
            else mma_layer<MH>(src, MH, 0, Ws[L], acc);
            __syncwarp();
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int row = g + 8 * h, col = nt * 8 + 2 * t;
                    const float g0 = gelu(acc[nt][2 * h] + bs[L][col]);
                    const float g1 = gelu(acc[nt][2 * h + 1] + bs[L][col + 1]);
                    acc[nt][2 * h] = g0;
                    acc[nt][2 * h + 1] = g1;
                    if (L < 2) *reinterpret_cast<uint32_t *>(dst + row * MH + col) = pack2(g0, g1);
                }
            __syncwarp();
        }
        float z[2];
        out_z(acc, P, z);
        if (t == 0)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int64_t row = r0 + g + 8 * h;
                if (row < G) {
                    float th = 0.3f + 0.9f * (1.0f / (1.0f + expf(-z[h])));
                    theta[row] = isfinite(th) ? th : fallback;
                }
            }
        __syncwarp();
    }
}

void nb_launch_mlp_infer(nb_ctx *c, const float *params, const float *feat, float *theta,
                         float fallback)
{
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_mlp_infer, MLP_T, 0);
    if (blocks < 1) blocks = 1;
    k_mlp_infer<<<c->num_sms * blocks, MLP_T, 0, c->stream>>>(params, feat, c->cnt, theta, fallback);
    nb_launched(c, "k_mlp_infer");
}

// ------------------------------------------------------------ training data
// Median relative force error of each sampled group: rows off[k] .. off[k+1]
// of ref (FP64 judge accelerations) belong to sampled group k, targets[]
// gives their caller index into acc.  One warp per group, bitonic sort of up
// to 1024 errors in shared memory; median = mean of the two middle values.
#define GE_MAX 1024
__global__ void __launch_bounds__(128)
k_group_errors(const float *__restrict__ acc, const double *__restrict__ ref,
               const int64_t *__restrict__ targets, const int64_t *__restrict__ off, int64_t S,
               float *__restrict__ err)
{
    __shared__ float buf[4][GE_MAX];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (k >= S) return;
    const int64_t a = off[k];
    int n = (int)(off[k + 1] - a);
    if (n > GE_MAX) n = GE_MAX;
    int np = 1;
    while (np < n) np <<= 1;
    float *e = buf[wl];
    for (int i = lane; i < np; i += 32) {
        float v = INFINITY;
        if (i < n) {
            const int64_t o = targets[a + i];
            const double rx = ref[3 * (a + i)], ry = ref[3 * (a + i) + 1], rz = ref[3 * (a + i) + 2];
            const double dx = (double)acc[3 * o] - rx, dy = (double)acc[3 * o + 1] - ry,
                         dz = (double)acc[3 * o + 2] - rz;
            const double r = sqrt(rx * rx + ry * ry + rz * rz);
            v = (float)(sqrt(dx * dx + dy * dy + dz * dz) / (r > 0.0 ? r : 1.0));
        }
        e[i] = v;
    }
    __syncwarp();
    for (int size = 2; size <= np; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < np; i += 32) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const float x = e[i], y = e[j];
                    if ((x > y) == up) { e[i] = y; e[j] = x; }
                }
            }
            __syncwarp();
        }
    if (lane == 0) err[k] = n > 0 ? 0.5f * (e[(n - 1) / 2] + e[n / 2]) : 0.0f;
}

// Label of each sample from its error curve err[t][k] (T x S, grid
// ascending).  Without costs: the largest grid theta whose error meets the
// budget (the smallest grid theta when none does).  With costs (interactions
// of the group at each theta) and group sizes: the grid theta minimising
// cost / n + lambda * ln(error), the allocation that trades interactions
// against error at one exchange rate lambda for every group.
__global__ void k_theta_labels(const float *__restrict__ err, const float *__restrict__ cost,
                               const float *__restrict__ nsz, const float *__restrict__ grid,
                               int T, int64_t S, float budget, float lambda,
                               float *__restrict__ labels)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= S) return;
    float lab = grid[0];
    if (!cost) {
        for (int t = 0; t < T; t++)
            if (err[(int64_t)t * S + k] <= budget) lab = grid[t];
    } else {
        float best = INFINITY;
        for (int t = 0; t < T; t++) {
            const float o = cost[(int64_t)t * S + k] / nsz[k] +
                            lambda * logf(fmaxf(err[(int64_t)t * S + k], 1e-9f));
            if (o < best) { best = o; lab = grid[t]; }
        }
    }
    labels[k] = lab;
}

extern "C" int nb_group_errors(const float *acc_dev, const double *ref_dev,
                               const int64_t *targets_dev, const int64_t *off_dev, int64_t S,
                               float *err_dev, void *stream)
{
    if (S < 0 || (S > 0 && (!acc_dev || !ref_dev || !targets_dev || !off_dev || !err_dev)))
        return NB_ERR_INVALID_ARG;
    if (S == 0) return NB_OK;
    k_group_errors<<<(int)((S * 32 + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        acc_dev, ref_dev, targets_dev, off_dev, S, err_dev);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

extern "C" int nb_theta_labels(const float *err_dev, const float *cost_dev,
                               const float *size_dev, const float *grid_dev, int T, int64_t S,
                               float budget, float lambda, float *labels_dev, void *stream)
{
    if (T < 1 || S < 0 || (S > 0 && (!err_dev || !grid_dev || !labels_dev)) ||
        (cost_dev && !size_dev))
        return NB_ERR_INVALID_ARG;
    if (S == 0) return NB_OK;
    k_theta_labels<<<nb_grid(S, 256), 256, 0, (cudaStream_t)stream>>>(
        err_dev, cost_dev, size_dev, grid_dev, T, S, budget, lambda, labels_dev);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

// ------------------------------------------------------------ backward
// per 16-sample tile: dz, then dZ3 -> dH2 -> dZ2 -> dH1 -> dZ1 (products on
// the tensor cores with BF16(dZ) and BF16(W)); dZ kept in FP32 (bias
// gradients) and BF16 (weight gradients)
__global__ void __launch_bounds__(MLP_T)
k_mlp_bwd(const float *__restrict__ P, int64_t Bp, int64_t B, MlpWork w)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (tile * 16 >= Bp) return;
    const int r0 = (int)(tile * 16);
    const float invB = 1.0f / (float)B;
    // dz per row (lanes 0..15 own one row each for this part)
    if (lane < 16) {
        const int row = r0 + lane;
        float dz = 0.0f, l = 0.0f;
        if (row < B) {
            const float d = w.theta[row] - w.y[row];
            const float dth = (2.0f * d + 2.0f * LAMBDA * fmaxf(d, 0.0f)) * invB;
            const float s = w.s[row];
            dz = dth * 0.9f * s * (1.0f - s);
            l = d * d + LAMBDA * fmaxf(d, 0.0f) * fmaxf(d, 0.0f);
        }
        w.dz[row] = dz;
        w.loss[row] = l;
    }
    __syncwarp();
    // dZ3 = (dz w4) * gelu'(Z3)
    for (int e = lane; e < 16 * MH; e += 32) {
        const int row = r0 + e / MH, col = e % MH;
        const float v = w.dz[row] * P[P_W4 + col] * gelu_grad(w.Z3[(int64_t)row * MH + col]);
        w.g3[(int64_t)row * MH + col] = v;
        w.d3[(int64_t)row * MH + col] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    // dH = dZ W (K = 64 outputs, N = 64 inputs), then dZ = dH * gelu'(Z)
    const float *Ws[2] = {P + P_W3, P + P_W2};
    const bf16 *din[2] = {w.d3, w.d2};
    const float *Zs[2] = {w.Z2, w.Z1};
    float *gout[2] = {w.g2, w.g1};
    bf16 *dout[2] = {w.d2, w.d1};
    for (int L = 0; L < 2; L++) {
        float acc[8][4];
        uint32_t a[4], b[2];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 4; kt++) {
            frag_a_rows(din[L], MH, r0, kt * 16, a);
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                frag_b_w(Ws[L], MH, kt * 16, nt * 8, b);
                mma16816(acc[nt], a, b);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const int row = r0 + g + 8 * h, col = nt * 8 + 2 * t + q;
                    const float v = acc[nt][2 * h + q] * gelu_grad(Zs[L][(int64_t)row * MH + col]);
                    gout[L][(int64_t)row * MH + col] = v;
                    dout[L][(int64_t)row * MH + col] = __float2bfloat16_rn(v);
                }
        __syncwarp();
    }
}

// ------------------------------------------------------------ gradients
// warps 0..7: dW1 tiles (64 x 16), 8..39: dW2 (64 x 64), 40..71: dW3;
// warps 72..: biases, w4, b4 and the loss (FP32 sums over the batch)
__global__ void __launch_bounds__(MLP_T)
k_mlp_wgrad(int64_t Bp, MlpWork w, float *__restrict__ grad, float *__restrict__ loss_acc)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid < 72) {
        const bf16 *dZ;
        const bf16 *X;
        int IN, mt, nt, off;
        if (wid < 8) { dZ = w.d1; X = w.a0; IN = MKIN; mt = wid / 2; nt = wid % 2; off = P_W1; }
        else if (wid < 40) { dZ = w.d2; X = w.a1; IN = MH; mt = (wid - 8) / 8; nt = (wid - 8) % 8; off = P_W2; }
        else { dZ = w.d3; X = w.a2; IN = MH; mt = (wid - 40) / 8; nt = (wid - 40) % 8; off = P_W3; }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t a[4], b[2];
        const int m0 = mt * 16, n0 = nt * 8;
        for (int64_t r0 = 0; r0 < Bp; r0 += 16) {
            // A(m = out, k = sample) = dZ[sample][out]
            a[0] = pack2b(dZ[(r0 + 2 * t) * MH + m0 + g], dZ[(r0 + 2 * t + 1) * MH + m0 + g]);
            a[1] = pack2b(dZ[(r0 + 2 * t) * MH + m0 + g + 8], dZ[(r0 + 2 * t + 1) * MH + m0 + g + 8]);
            a[2] = pack2b(dZ[(r0 + 2 * t + 8) * MH + m0 + g], dZ[(r0 + 2 * t + 9) * MH + m0 + g]);
            a[3] = pack2b(dZ[(r0 + 2 * t + 8) * MH + m0 + g + 8], dZ[(r0 + 2 * t + 9) * MH + m0 + g + 8]);
            // B(k = sample, n = in) = X[sample][in]
            b[0] = pack2b(X[(r0 + 2 * t) * IN + n0 + g], X[(r0 + 2 * t + 1) * IN + n0 + g]);
            b[1] = pack2b(X[(r0 + 2 * t + 8) * IN + n0 + g], X[(r0 + 2 * t + 9) * IN + n0 + g]);
            mma16816(acc, a, b);
        }
        grad[off + (m0 + g) * IN + n0 + 2 * t] = acc[0];
        grad[off + (m0 + g) * IN + n0 + 2 * t + 1] = acc[1];
        grad[off + (m0 + g + 8) * IN + n0 + 2 * t] = acc[2];
        grad[off + (m0 + g + 8) * IN + n0 + 2 * t + 1] = acc[3];
    } else if (wid < 72 + 8) {
        // biases b1, b2, b3 and w4: 4 x 64 columns over 8 warps
        const int c0 = (wid - 72) * 32 + lane;   // 0 .. 255
        const int which = c0 / MH, col = c0 % MH;
        const float *src = which == 0 ? w.g1 : which == 1 ? w.g2 : which == 2 ? w.g3 : w.h3;
        float s = 0.f;
        for (int64_t r = 0; r < Bp; r++)
            s += which == 3 ? w.dz[r] * src[r * MH + col] : src[r * MH + col];
        const int off = which == 0 ? P_B1 : which == 1 ? P_B2 : which == 2 ? P_B3 : P_W4;
        grad[off + col] = s;
    } else if (wid == 80) {
        float s = 0.f, l = 0.f;
        for (int64_t r = lane; r < Bp; r += 32) {
            s += w.dz[r];
            l += w.loss[r];
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            l += __shfl_xor_sync(0xffffffffu, l, o);
        }
        if (lane == 0) {
            grad[P_B4] = s;
            if (loss_acc) atomicAdd(loss_acc, l);
        }
    }
}

__global__ void __launch_bounds__(256)
k_mlp_adam(float *__restrict__ P, float *__restrict__ m, float *__restrict__ v,
           const float *__restrict__ grad, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P_MU) return;   // mu and sigma are not trained
    const float gi = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// ------------------------------------------------------------ host side
static int64_t pad16(int64_t b) { return (b + 15) / 16 * 16; }

extern "C" size_t nb_mlp_workspace_size(int64_t batch)
{
    return work_layout(pad16(batch), nullptr, nullptr) + 256;
}

static MlpWork layout_at(void *ws, int64_t Bp)
{
    MlpWork w;
    char *base = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    work_layout(Bp, &w, base);
    return w;
}

static int mlp_forward(const float *P, const float *x, const int32_t *idx, const float *y,
                       int64_t B, float *theta, MlpWork w, bool keep, float fallback,
                       cudaStream_t s)
{
    const int64_t Bp = pad16(B);
    k_mlp_input<<<nb_grid(Bp * MKIN, 256), 256, 0, s>>>(x, idx, y, B, Bp, P, w.a0, keep ? w.y : nullptr);
    const int64_t warps = Bp / 16;
    const int blocks = (int)((warps * 32 + MLP_T - 1) / MLP_T);
    if (keep)
        k_mlp_fwd<true><<<blocks, MLP_T, 0, s>>>(P, Bp, w, theta, B, fallback);
    else
        k_mlp_fwd<false><<<blocks, MLP_T, 0, s>>>(P, Bp, w, theta, B, fallback);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

static void mlp_backward(const float *P, int64_t B, float *grad, float *loss_acc, MlpWork w,
                         cudaStream_t s)
{
    const int64_t Bp = pad16(B);
    const int64_t warps = Bp / 16;
    k_mlp_bwd<<<(int)((warps * 32 + MLP_T - 1) / MLP_T), MLP_T, 0, s>>>(P, Bp, B, w);
    k_mlp_wgrad<<<(81 * 32 + MLP_T - 1) / MLP_T, MLP_T, 0, s>>>(Bp, w, grad, loss_acc);
}

extern "C" int nb_mlp_forward(const float *params, const float *feat, int64_t n,
                              float *theta_out, float fallback, void *work, void *stream)
{
    if (!params || n < 0 || (n > 0 && (!feat || !theta_out || !work))) return NB_ERR_INVALID_ARG;
    if (n == 0) return NB_OK;
    MlpWork w = layout_at(work, pad16(n));
    return mlp_forward(params, feat, nullptr, nullptr, n, theta_out, w, false, fallback,
                       (cudaStream_t)stream);
}

extern "C" int nb_mlp_grad(const float *params, const float *feat, const float *labels,
                           int64_t n, float *grad_out, float *loss_out, void *work,
                           void *stream)
{
    if (!params || n <= 0 || !feat || !labels || !grad_out || !work) return NB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    MlpWork w = layout_at(work, pad16(n));
    if (cudaMemsetAsync(grad_out, 0, sizeof(float) * P_N, s) != cudaSuccess) return NB_ERR_CUDA;
    if (loss_out && cudaMemsetAsync(loss_out, 0, sizeof(float), s) != cudaSuccess) return NB_ERR_CUDA;
    int rc = mlp_forward(params, feat, nullptr, labels, n, nullptr, w, true, 0.f, s);
    if (rc) return rc;
    mlp_backward(params, n, grad_out, loss_out, w, s);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

extern "C" int nb_mlp_train(float *params, float *adam_m, float *adam_v, const float *feat,
                            const float *labels, int64_t n, const int32_t *order, int epochs,
                            int batch, float lr, float *grad_work, float *loss_per_epoch,
                            void *work, void *stream)
{
    if (!params || !adam_m || !adam_v || !feat || !labels || !order || n <= 0 || epochs < 1 ||
        batch < 16 || batch > n || !grad_work || !work)
        return NB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    MlpWork w = layout_at(work, pad16(batch));
    const int64_t steps = n / batch;
    int64_t t = 0;
    if (loss_per_epoch && cudaMemsetAsync(loss_per_epoch, 0, sizeof(float) * epochs, s) != cudaSuccess)
        return NB_ERR_CUDA;
    for (int e = 0; e < epochs; e++) {
        for (int64_t k = 0; k < steps; k++) {
            t++;
            const int32_t *idx = order + (int64_t)e * n + k * batch;
            int rc = mlp_forward(params, feat, idx, labels, batch, nullptr, w, true, 0.f, s);
            if (rc) return rc;
            mlp_backward(params, batch, grad_work, loss_per_epoch ? loss_per_epoch + e : nullptr, w, s);
            const float c1 = 1.0f - powf(0.9f, (float)t), c2 = 1.0f - powf(0.999f, (float)t);
            k_mlp_adam<<<(P_MU + 255) / 256, 256, 0, s>>>(params, adam_m, adam_v, grad_work, lr, c1, c2);
        }
    }
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
