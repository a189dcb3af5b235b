// nb_direct.cu -- the brute-force O(N^2) sum of Eq. (gravity) in FP32 (the
// paper's "bare" many-body kernel, Sec. "A Bare Many-body Performance on
// RV770 GPU"), the baseline the tree method is compared with (Sec. "Test
// and Optimization": the tree wins except for N < 10,000).
//
// Positions enter as FP64 and are rounded once to FP32 (x, y, z) with the
// FP32 mass into one float4 per particle: the representation the paper's
// kernel works on.  A block of 256 threads holds 512 targets (two per
// lane); sources stream through a 256-record shared-memory tile laid out in
// record pairs, so every step of the interaction runs on two sources at
// once with the packed FP32 instructions (add/mul/fma .f32x2), the same
// arithmetic as the tree's force kernel: 13 FP32-pipe operations and one
// MUFU rsqrt per interaction, summed over j != i (the self term is dropped
// by index in the tiles that hold the block's own targets).
//
// Small N gives too few target blocks to fill 152 SMs, so the source range
// is split into P contiguous parts (grid = target blocks x parts); each part
// writes its partial sums to the caller's workspace and a second kernel adds
// the parts in a fixed order, so results do not depend on scheduling.
#include <float.h>

#include "nb_force.cuh"

#define D_T 256                 // threads per block
#define D_R 2                   // targets per thread
#define D_TGT (D_T * D_R)       // targets per block
#define D_TJ 256                // source records per staged tile
#define D_MIN_PART_TILES 2      // a part spans at least this many tiles
#define D_MAX_PARTS 64

// FP32 copy of the particles: (x, y, z, m) rounded to nearest
__global__ void __launch_bounds__(256)
k_direct_pack(const double *__restrict__ pos, const float *__restrict__ mass, int64_t n,
              float4 *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = make_float4(__double2float_rn(pos[3 * i]), __double2float_rn(pos[3 * i + 1]),
                         __double2float_rn(pos[3 * i + 2]), mass[i]);
}

// One block: targets tb*512 .. +511 against sources of part `part`
// (blockIdx.y) of `parts`, each part an equal run of whole tiles.
template <int MODE, bool GUARD>
__global__ void __launch_bounds__(D_T, 4)
k_direct32(const float4 *__restrict__ p, int64_t n, int parts, int64_t part_len, float eps2,
           float4 *__restrict__ partial, float *__restrict__ acc, float *__restrict__ pot)
{
    __shared__ float4 tile[D_TJ];
    const int64_t t0 = (int64_t)blockIdx.x * D_TGT;
    const int64_t j_begin = (int64_t)blockIdx.y * part_len;
    const int64_t j_end = j_begin + part_len < n ? j_begin + part_len : n;
    Tgt t[D_R];
    int32_t kk[D_R];
    Acc<MODE> A[D_R];
    Sum2 P[D_R];
#pragma unroll
    for (int r = 0; r < D_R; r++) {
        const int64_t i = t0 + r * D_T + threadIdx.x;
        const float4 q = p[i < n ? i : n - 1];
        t[r].set(q.x, q.y, q.z);
        kk[r] = (int32_t)i;
        A[r].init();
        P[r].init();
    }
    const float4 pad = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    for (int64_t j0 = j_begin; j0 < j_end; j0 += D_TJ) {
        const int64_t jj = j0 + threadIdx.x;
        put_rec(tile, threadIdx.x, jj < j_end ? p[jj] : pad);
        __syncthreads();
        // the tiles that overlap this block's own targets drop j == i
        const bool own = j0 < t0 + D_TGT && j0 + D_TJ > t0;
        if (own)
            tile_pass<MODE, GUARD, true, D_R, D_TJ>(tile, 0, (int32_t)j0, t, kk, eps2, A, P);
        else
            tile_pass<MODE, GUARD, false, D_R, D_TJ, 32>(tile, 0, (int32_t)j0, t, kk, eps2, A,
                                                         P);
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < D_R; r++) {
        pair_fold<MODE>(A[r], P[r]);
        const int64_t i = t0 + r * D_T + threadIdx.x;
        if (i >= n) continue;
        float ax, ay, az, ph;
        if (MODE == MODE_COMP) {
            ax = A[r].x - A[r].cx; ay = A[r].y - A[r].cy;
            az = A[r].z - A[r].cz; ph = A[r].p - A[r].cp;
        } else {
            ax = A[r].x; ay = A[r].y; az = A[r].z; ph = A[r].p;
        }
        if (parts == 1) {
            acc[3 * i] = ax;
            acc[3 * i + 1] = ay;
            acc[3 * i + 2] = az;
            if (pot) pot[i] = ph;
        } else {
            partial[(int64_t)blockIdx.y * n + i] = make_float4(ax, ay, az, ph);
        }
    }
}

// the parts of each target added in part order (Kahan-compensated in the
// compensated mode)
template <int MODE>
__global__ void __launch_bounds__(256)
k_direct32_reduce(const float4 *__restrict__ partial, int64_t n, int parts,
                  float *__restrict__ acc, float *__restrict__ pot)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < parts; k++) {
        const float4 v = partial[(int64_t)k * n + i];
        const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int d = 0; d < 4; d++) {
            if (MODE == MODE_COMP) kahan(s[d], c[d], w[d]);
            else s[d] = __fadd_rn(s[d], w[d]);
        }
    }
    if (MODE == MODE_COMP)
        for (int d = 0; d < 4; d++) s[d] = s[d] - c[d];
    acc[3 * i] = s[0];
    acc[3 * i + 1] = s[1];
    acc[3 * i + 2] = s[2];
    if (pot) pot[i] = s[3];
}

// parts of the source range for n particles on a device with `sms` SMs: of
// the part counts that keep every part at least D_MIN_PART_TILES tiles long,
// the one whose blocks fill the 4 x sms resident slots best (the last wave as
// full as possible), the smallest on a tie
static int direct_parts(int64_t n, int sms)
{
    const int64_t tb = (n + D_TGT - 1) / D_TGT;
    const int64_t tiles = (n + D_TJ - 1) / D_TJ;
    const double slots = 4.0 * (sms > 0 ? sms : 1);
    int best = 1;
    double best_eff = -1.0;
    for (int P = 1; P <= D_MAX_PARTS; P++) {
        const int64_t part_len = (tiles + P - 1) / P * D_TJ;
        if (P > 1 && part_len < (int64_t)D_TJ * D_MIN_PART_TILES) break;
        const int64_t rp = (n + part_len - 1) / part_len;
        const double waves = (double)(tb * rp) / slots;
        const double eff = waves / __builtin_ceil(waves);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = P;
        }
    }
    return best;
}

static int current_sms(int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NB_ERR_CUDA;
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NB_ERR_CUDA;
    return NB_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" size_t nb_direct_f32_workspace_size(int64_t n)
{
    if (n <= 0) return 0;
    int sms = 0;
    int parts = D_MAX_PARTS;   // no device: room for the largest part count
    if (current_sms(&sms)) cudaGetLastError();
    else parts = direct_parts(n, sms);
    return align256(sizeof(float4) * (size_t)n) +
           (parts > 1 ? sizeof(float4) * (size_t)n * (size_t)parts : 0);
}

extern "C" int nb_direct_f32(const double *pos, const float *mass, int64_t n, float eps,
                             float *acc, float *pot, int precision, void *work,
                             size_t work_bytes, void *stream)
{
    if (n < 0 || n > INT32_MAX - D_TGT || !(eps >= 0.0f) || eps == INFINITY ||
        (precision != NB_FP32 && precision != NB_FP32_COMP))
        return NB_ERR_INVALID_ARG;
    if (n == 0) return NB_OK;
    if (!pos || !mass || !acc || !work) return NB_ERR_INVALID_ARG;
    int sms = 0;
    if (current_sms(&sms)) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    const int parts = direct_parts(n, sms);
    const size_t need = align256(sizeof(float4) * (size_t)n) +
                        (parts > 1 ? sizeof(float4) * (size_t)n * (size_t)parts : 0);
    if (work_bytes < need || ((uintptr_t)work & 255u)) return NB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float4 *p32 = (float4 *)work;
    float4 *partial = (float4 *)((char *)work + align256(sizeof(float4) * (size_t)n));
    k_direct_pack<<<nb_grid(n, 256), 256, 0, s>>>(pos, mass, n, p32);
    // part length in whole tiles
    const int64_t tiles = (n + D_TJ - 1) / D_TJ;
    const int64_t part_len = (tiles + parts - 1) / parts * D_TJ;
    const int real_parts = (int)((n + part_len - 1) / part_len);
    const dim3 grid((unsigned)((n + D_TGT - 1) / D_TGT), (unsigned)real_parts);
    const float eps2 = eps * eps;
    const bool guard = !(eps2 >= FLT_MIN);
    switch ((precision == NB_FP32_COMP ? 2 : 0) + (guard ? 1 : 0)) {
    case 0:
        k_direct32<MODE_FP32, false><<<grid, D_T, 0, s>>>(p32, n, real_parts, part_len, eps2,
                                                          partial, acc, pot);
        break;
    case 1:
        k_direct32<MODE_FP32, true><<<grid, D_T, 0, s>>>(p32, n, real_parts, part_len, eps2,
                                                         partial, acc, pot);
        break;
    case 2:
        k_direct32<MODE_COMP, false><<<grid, D_T, 0, s>>>(p32, n, real_parts, part_len, eps2,
                                                          partial, acc, pot);
        break;
    default:
        k_direct32<MODE_COMP, true><<<grid, D_T, 0, s>>>(p32, n, real_parts, part_len, eps2,
                                                         partial, acc, pot);
        break;
    }
    if (real_parts > 1) {
        if (precision == NB_FP32_COMP)
            k_direct32_reduce<MODE_COMP><<<nb_grid(n, 256), 256, 0, s>>>(partial, n, real_parts,
                                                                          acc, pot);
        else
            k_direct32_reduce<MODE_FP32><<<nb_grid(n, 256), 256, 0, s>>>(partial, n, real_parts,
                                                                          acc, pot);
    }
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
