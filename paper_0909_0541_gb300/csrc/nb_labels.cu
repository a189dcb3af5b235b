// nb_labels.cu -- the label rule of the learned opening angle and the error
// statistics it is judged by, on the device.
//
// The paper fixes one theta for every particle (Eq. mac, Table theta shows
// the cost / accuracy trade of that choice); the per-group theta is this
// project's addition.  A sampled group g has, at every theta_t of an
// ascending grid, a measured median relative force error e[t][g] (FP64
// direct-sum judge) and a cost c[t][g] (interactions, plus the walk's list
// entries weighted by their relative time).  Its label is the grid theta
// minimising
//     C[t][g] / n_g + lambda * E[t][g]
// where (E, C) are either the measured curves (E = ln max(e, 1e-9), C = c)
// or the curves that the group's features predict (E = the least-squares fit
// of ln(e + 1e-15) on the features, C = exp of the fit of ln(c + 1));
// lambda, one exchange rate between cost and error for every group, is
// bisected in ln space so that the n_g-weighted median of the measured
// errors of the chosen thetas meets the error budget.
//
// Fit: the chosen feature columns are standardised (mean 0, spread 1; a
// constant column becomes 0), an intercept is added, and the normal
// equations are accumulated in FP64 per block of rows (a fixed order, so the
// result does not depend on scheduling), summed by one block and solved by
// Cholesky with a tiny ridge (1e-12 x the trace) that keeps a constant
// column from making the system singular.  The allocation, the weighted
// median and the bisection run in one block: the weighted median is the
// smallest error u for which the weights of the errors <= u reach half the
// total, found by a binary search over the FP32 bit pattern (positive floats
// order as their bits) with FP64 weight sums.
#include <float.h>
#include <math.h>

#include "nb_internal.cuh"

#define LB_MAXP 17         // features + intercept
#define LB_MAXT 64         // grid points
#define LB_ROWS 32         // rows staged per block pass (normal equations)
#define LB_BLOCKS 64       // blocks accumulating the normal equations
#define LB_T 1024          // threads of the one-block kernels

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// the chosen feature columns, passed by value to every kernel
struct nb_cols {
    int32_t c[LB_MAXP];
};

// per column: mean and spread (two passes, FP64), one block per column
__global__ void __launch_bounds__(256)
k_fit_stats(const float *__restrict__ feat, int64_t S, int stride, const nb_cols cols,
            double *__restrict__ mu, double *__restrict__ sd)
{
    __shared__ double red[256];
    const int c = cols.c[blockIdx.x];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < S; i += blockDim.x) s += (double)feat[i * stride + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double m = red[0] / (double)S;
    __syncthreads();
    double q = 0.0;
    for (int64_t i = threadIdx.x; i < S; i += blockDim.x) {
        const double d = (double)feat[i * stride + c] - m;
        q += d * d;
    }
    red[threadIdx.x] = q;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mu[blockIdx.x] = m;
        sd[blockIdx.x] = sqrt(red[0] / (double)S);
    }
}

// standardised design row k of sample i: z_0 = 1, z_{1+c} = (f - mu) / sd
__device__ __forceinline__ double design(const float *feat, int stride, const nb_cols &cols,
                                         const double *mu, const double *sd, int64_t i, int k)
{
    if (k == 0) return 1.0;
    const double s = sd[k - 1];
    return s > 0.0 ? ((double)feat[i * stride + cols.c[k - 1]] - mu[k - 1]) / s : 0.0;
}

// targets of the fit: y_t = ln(e[t] + 1e-15) (t < T), y_{T+t} = ln(c[t] + 1)
__device__ __forceinline__ double target(const float *err, const float *cost, int T, int64_t S,
                                         int64_t i, int j)
{
    return j < T ? log((double)err[(int64_t)j * S + i] + 1e-15)
                 : log((double)cost[(int64_t)(j - T) * S + i] + 1.0);
}

// block partial of the normal equations: G (p x p, upper triangle used) and
// R (p x 2T), rows staged LB_ROWS at a time; each thread owns entries
__global__ void __launch_bounds__(256)
k_fit_normal(const float *__restrict__ feat, int64_t S, int stride,
             const nb_cols cols, int p, const double *__restrict__ mu,
             const double *__restrict__ sd, const float *__restrict__ err,
             const float *__restrict__ cost, int T, double *__restrict__ part)
{
    __shared__ double z[LB_ROWS][LB_MAXP];
    __shared__ double y[LB_ROWS][2 * LB_MAXT];
    const int ne = p * p + p * 2 * T;   // entries of G then R
    double acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = 0.0;
    const int64_t per = (S + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per, r1 = r0 + per < S ? r0 + per : S;
    for (int64_t base = r0; base < r1; base += LB_ROWS) {
        const int rows = (int)(r1 - base < LB_ROWS ? r1 - base : LB_ROWS);
        for (int e = threadIdx.x; e < rows * p; e += blockDim.x)
            z[e / p][e % p] = design(feat, stride, cols, mu, sd, base + e / p, e % p);
        for (int e = threadIdx.x; e < rows * 2 * T; e += blockDim.x)
            y[e / (2 * T)][e % (2 * T)] = target(err, cost, T, S, base + e / (2 * T), e % (2 * T));
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int e = threadIdx.x + k * blockDim.x;
            if (e >= ne) break;
            double s = acc[k];
            if (e < p * p) {
                const int a = e / p, b = e % p;
                for (int r = 0; r < rows; r++) s += z[r][a] * z[r][b];
            } else {
                const int a = (e - p * p) / (2 * T), j = (e - p * p) % (2 * T);
                for (int r = 0; r < rows; r++) s += z[r][a] * y[r][j];
            }
            acc[k] = s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int e = threadIdx.x + k * blockDim.x;
        if (e < ne) part[(int64_t)blockIdx.x * ne + e] = acc[k];
    }
}

// sum the block partials in block order, Cholesky-factor G (+ ridge) and
// solve for every right-hand side: coef (p x 2T)
__global__ void __launch_bounds__(256)
k_fit_solve(const double *__restrict__ part, int nblk, int p, int T, double *__restrict__ coef)
{
    __shared__ double G[LB_MAXP][LB_MAXP];
    __shared__ double R[LB_MAXP][2 * LB_MAXT];
    const int ne = p * p + p * 2 * T;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++) s += part[(int64_t)b * ne + e];
        if (e < p * p) G[e / p][e % p] = s;
        else R[(e - p * p) / (2 * T)][(e - p * p) % (2 * T)] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int a = 0; a < p; a++) tr += G[a][a];
        const double ridge = 1e-12 * (tr > 0.0 ? tr : 1.0);
        for (int a = 0; a < p; a++) G[a][a] += ridge;
        // in-place Cholesky: lower triangle holds L
        for (int j = 0; j < p; j++) {
            double d = G[j][j];
            for (int k = 0; k < j; k++) d -= G[j][k] * G[j][k];
            d = d > ridge ? sqrt(d) : sqrt(ridge);
            G[j][j] = d;
            for (int i = j + 1; i < p; i++) {
                double v = G[i][j];
                for (int k = 0; k < j; k++) v -= G[i][k] * G[j][k];
                G[i][j] = v / d;
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * T; j += blockDim.x) {
        double w[LB_MAXP];
        for (int i = 0; i < p; i++) {   // L w = r
            double v = R[i][j];
            for (int k = 0; k < i; k++) v -= G[i][k] * w[k];
            w[i] = v / G[i][i];
        }
        for (int i = p - 1; i >= 0; i--) {   // L^T c = w
            double v = w[i];
            for (int k = i + 1; k < p; k++) v -= G[k][i] * w[k];
            w[i] = v / G[i][i];
        }
        for (int i = 0; i < p; i++) coef[(int64_t)i * 2 * T + j] = w[i];
    }
}

// predicted curves: pe[t][i] = z_i . c_t, pc[t][i] = exp(z_i . c_{T+t})
__global__ void __launch_bounds__(256)
k_fit_predict(const float *__restrict__ feat, int64_t S, int stride,
              const nb_cols cols, int p, const double *__restrict__ mu,
              const double *__restrict__ sd, const double *__restrict__ coef, int T,
              double *__restrict__ pe, double *__restrict__ pc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S) return;
    double z[LB_MAXP];
    for (int k = 0; k < p; k++) z[k] = design(feat, stride, cols, mu, sd, i, k);
    for (int t = 0; t < T; t++) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < p; k++) {
            a += z[k] * coef[(int64_t)k * 2 * T + t];
            b += z[k] * coef[(int64_t)k * 2 * T + T + t];
        }
        pe[(int64_t)t * S + i] = a;
        pc[(int64_t)t * S + i] = exp(b);
    }
}

// ------------------------------------------------------------ selection
// Block-wide FP64 sum (every thread of the LB_T-thread block calls it).
__device__ __forceinline__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += red[k];
    return s;
}

__device__ __forceinline__ uint32_t err_bits(float v)
{
    // errors are >= 0; -0 and anything negative count as 0, NaN above inf
    return v > 0.0f || isnan(v) ? __float_as_uint(v) : 0u;
}

// smallest value u among vals[0..S) with sum(w_i : vals_i <= u) >= need
// (w NULL: weight 1); every thread of the block calls it
__device__ float select_weighted(const float *vals, const float *w, int64_t S, double need,
                                 double *red)
{
    long long lo = -1;   // largest bit pattern known to have weight < need
    for (int b = 31; b >= 0; b--) {
        const long long cand = lo + (1ll << b);
        double s = 0.0;
        for (int64_t i = threadIdx.x; i < S; i += blockDim.x)
            if ((long long)err_bits(vals[i]) <= cand) s += w ? (double)w[i] : 1.0;
        s = block_sum(s, red);
        if (s < need) lo = cand;
    }
    return __uint_as_float((uint32_t)(lo + 1));
}

// The allocation for one exchange rate: chosen grid index per sample and
// the measured error there (into vals); ties go to the smaller theta.
__device__ void allocate(double lam, const double *pe, const double *pc, const float *err,
                         const float *cost, const float *nsz, int T, int64_t S, int32_t *tsel,
                         float *vals)
{
    for (int64_t i = threadIdx.x; i < S; i += blockDim.x) {
        const double n = (double)nsz[i];
        double best = INFINITY;
        int tb = 0;
        for (int t = 0; t < T; t++) {
            const int64_t k = (int64_t)t * S + i;
            const double e = pe ? pe[k] : log(fmax((double)err[k], 1e-9));
            const double c = pc ? pc[k] : (double)cost[k];
            const double o = c / n + lam * e;
            if (o < best) {
                best = o;
                tb = t;
            }
        }
        tsel[i] = tb;
        vals[i] = err[(int64_t)tb * S + i];
    }
    __syncthreads();
}

// the statistic the bisection holds at the budget: the n_g-weighted median
// of the groups' measured median errors, or (perr given) the median over the
// judged particles of their own errors at their group's chosen theta
__device__ double allocation_stat(const float *err, const float *nsz, int64_t S, double half,
                                  const int32_t *tsel, const float *vals, const float *perr,
                                  const int64_t *poff, int64_t P, float *pvals, double *red)
{
    if (!perr) return (double)select_weighted(vals, nsz, S, half, red);
    for (int64_t g = threadIdx.x; g < S; g += blockDim.x) {
        const int64_t t = tsel[g];
        for (int64_t q = poff[g]; q < poff[g + 1]; q++) pvals[q] = perr[t * P + q];
    }
    __syncthreads();
    const float a = select_weighted(pvals, nullptr, P, (double)((P - 1) / 2 + 1), red);
    const float b = select_weighted(pvals, nullptr, P, (double)(P / 2 + 1), red);
    return 0.5 * ((double)a + (double)b);
}

__global__ void __launch_bounds__(LB_T)
k_theta_allocate(const double *__restrict__ pe, const double *__restrict__ pc,
                 const float *__restrict__ err, const float *__restrict__ cost,
                 const float *__restrict__ nsz, const float *__restrict__ grid, int T, int64_t S,
                 double budget, double lam_lo, double lam_hi, int iters,
                 const float *__restrict__ perr, const int64_t *__restrict__ poff, int64_t P,
                 int32_t *tsel, float *vals, float *pvals, float *__restrict__ labels,
                 double *__restrict__ result)
{
    __shared__ double red[LB_T / 32];
    double W = 0.0;
    for (int64_t i = threadIdx.x; i < S; i += blockDim.x) W += (double)nsz[i];
    W = block_sum(W, red);
    const double half = 0.5 * W;
    double lo = lam_lo, hi = lam_hi;
    for (int it = 0; it < iters; it++) {
        const double mid = sqrt(lo * hi);
        allocate(mid, pe, pc, err, cost, nsz, T, S, tsel, vals);
        const double st = allocation_stat(err, nsz, S, half, tsel, vals, perr, poff, P, pvals, red);
        if (st > budget) lo = mid;
        else hi = mid;
    }
    allocate(hi, pe, pc, err, cost, nsz, T, S, tsel, vals);
    const double st = allocation_stat(err, nsz, S, half, tsel, vals, perr, poff, P, pvals, red);
    for (int64_t i = threadIdx.x; i < S; i += blockDim.x) labels[i] = grid[tsel[i]];
    if (threadIdx.x == 0) {
        result[0] = hi;
        result[1] = st;
    }
}

// relative errors |a - ref| / |ref| of the targets (FP64, rounded to FP32)
__global__ void __launch_bounds__(256)
k_rel_errors(const float *__restrict__ acc, const double *__restrict__ ref,
             const int64_t *__restrict__ targets, int64_t nt, float *__restrict__ out)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const int64_t o = targets ? targets[k] : k;
    const double rx = ref[3 * k], ry = ref[3 * k + 1], rz = ref[3 * k + 2];
    const double dx = (double)acc[3 * o] - rx, dy = (double)acc[3 * o + 1] - ry,
                 dz = (double)acc[3 * o + 2] - rz;
    const double r = sqrt(rx * rx + ry * ry + rz * rz);
    out[k] = (float)(sqrt(dx * dx + dy * dy + dz * dz) / (r > 0.0 ? r : 1.0));
}

// median (mean of the two middle order statistics, in FP64) and the q-th
// order statistic ceil(q nt) of the errors
__global__ void __launch_bounds__(LB_T)
k_error_stats(const float *__restrict__ e, int64_t nt, double q, double *__restrict__ out)
{
    __shared__ double red[LB_T / 32];
    const float a = select_weighted(e, nullptr, nt, (double)((nt - 1) / 2 + 1), red);
    const float b = select_weighted(e, nullptr, nt, (double)(nt / 2 + 1), red);
    double kq = ceil(q * (double)nt);
    if (kq < 1.0) kq = 1.0;
    const float c = select_weighted(e, nullptr, nt, kq, red);
    if (threadIdx.x == 0) {
        out[0] = 0.5 * ((double)a + (double)b);
        out[1] = (double)c;
    }
}

extern "C" size_t nb_theta_fit_workspace_size(int64_t S, int ncols, int T)
{
    if (S < 1 || ncols < 0 || ncols + 1 > LB_MAXP || T < 1 || T > LB_MAXT) return 0;
    const int p = ncols + 1;
    const size_t ne = (size_t)p * p + (size_t)p * 2 * T;
    return 2 * al256(sizeof(double) * LB_MAXP) + al256(sizeof(double) * ne * LB_BLOCKS) +
           al256(sizeof(double) * p * 2 * T);
}

extern "C" int nb_theta_fit_curves(const float *feat_dev, int64_t S, int stride,
                                   const int32_t *cols_host, int ncols, const float *err_dev,
                                   const float *cost_dev, int T, double *pred_lnerr_dev,
                                   double *pred_cost_dev, void *work_dev, size_t work_bytes,
                                   void *stream)
{
    if (S < 1 || ncols < 0 || ncols + 1 > LB_MAXP || T < 1 || T > LB_MAXT ||
        (ncols > 0 && !cols_host) || !feat_dev || !err_dev || !cost_dev || !pred_lnerr_dev ||
        !pred_cost_dev || !work_dev || stride < 1)
        return NB_ERR_INVALID_ARG;
    const int p = ncols + 1;
    const size_t ne = (size_t)p * p + (size_t)p * 2 * T;
    if (ne > 8 * 256) return NB_ERR_INVALID_ARG;   // entries k_fit_normal's threads hold
    nb_cols cols = {};
    for (int k = 0; k < ncols; k++) {
        if (cols_host[k] < 0 || cols_host[k] >= stride) return NB_ERR_INVALID_ARG;
        cols.c[k] = cols_host[k];
    }
    if (work_bytes < nb_theta_fit_workspace_size(S, ncols, T) || ((uintptr_t)work_dev & 255u))
        return NB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)work_dev;
    double *mu = (double *)w;
    w += al256(sizeof(double) * LB_MAXP);
    double *sd = (double *)w;
    w += al256(sizeof(double) * LB_MAXP);
    double *part = (double *)w;
    w += al256(sizeof(double) * ne * LB_BLOCKS);
    double *coef = (double *)w;
    if (ncols > 0) k_fit_stats<<<ncols, 256, 0, s>>>(feat_dev, S, stride, cols, mu, sd);
    const int nblk = (int)(S < LB_BLOCKS ? S : LB_BLOCKS);
    k_fit_normal<<<nblk, 256, 0, s>>>(feat_dev, S, stride, cols, p, mu, sd, err_dev, cost_dev, T,
                                      part);
    k_fit_solve<<<1, 256, 0, s>>>(part, nblk, p, T, coef);
    k_fit_predict<<<nb_grid(S, 256), 256, 0, s>>>(feat_dev, S, stride, cols, p, mu, sd, coef, T,
                                                  pred_lnerr_dev, pred_cost_dev);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

extern "C" size_t nb_theta_allocate_workspace_size(int64_t S, int64_t P)
{
    return S < 1 || P < 0 ? 0
                          : al256(sizeof(int32_t) * S) + al256(sizeof(float) * S) +
                                al256(sizeof(float) * (P > 0 ? P : 1));
}

// per-particle statistic: poff (S + 1) must run from 0 to P without
// decreasing, since it decides every index the allocation kernel writes;
// one pass checks it before that kernel runs
__global__ void k_check_poff(const int64_t *__restrict__ poff, int64_t S, int64_t P,
                             int *__restrict__ bad)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < S;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = poff[g], b = poff[g + 1];
        if (a < 0 || b < a || b > P || (g == 0 && a != 0) || (g == S - 1 && b != P)) *bad = 1;
    }
}

extern "C" int nb_theta_allocate(const double *pred_lnerr_dev, const double *pred_cost_dev,
                                 const float *err_dev, const float *cost_dev,
                                 const float *size_dev, const float *grid_dev, int T, int64_t S,
                                 double budget, double lam_lo, double lam_hi, int iters,
                                 const float *perr_dev, const int64_t *poff_dev, int64_t P,
                                 float *labels_dev, double *result_dev, void *work_dev,
                                 size_t work_bytes, void *stream)
{
    if (T < 1 || S < 1 || !err_dev || !size_dev || !grid_dev || !labels_dev || !result_dev ||
        !work_dev || (!pred_cost_dev && !cost_dev) || !(lam_lo > 0.0) || !(lam_hi >= lam_lo) ||
        !isfinite(lam_hi) || iters < 0 || iters > 200 || !(budget >= 0.0) ||
        (perr_dev && (!poff_dev || P < 1)))
        return NB_ERR_INVALID_ARG;
    if (!perr_dev) P = 0;
    if (work_bytes < nb_theta_allocate_workspace_size(S, P) || ((uintptr_t)work_dev & 255u))
        return NB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *tsel = (int32_t *)work_dev;
    float *vals = (float *)((char *)work_dev + al256(sizeof(int32_t) * S));
    float *pvals = (float *)((char *)vals + al256(sizeof(float) * S));
    if (perr_dev) {
        // the offsets decide every index the kernel writes: checked first
        int *bad = (int *)pvals;
        int hbad = 0;
        if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) return NB_ERR_CUDA;
        k_check_poff<<<nb_grid(S, 256, 1024), 256, 0, s>>>(poff_dev, S, P, bad);
        if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return NB_ERR_CUDA;
        if (hbad) return NB_ERR_INVALID_ARG;
    }
    k_theta_allocate<<<1, LB_T, 0, s>>>(pred_lnerr_dev, pred_cost_dev, err_dev, cost_dev,
                                        size_dev, grid_dev, T, S, budget, lam_lo, lam_hi, iters,
                                        perr_dev, poff_dev, P, tsel, vals, pvals, labels_dev,
                                        result_dev);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

extern "C" int nb_error_stats(const float *acc_dev, const double *ref_dev,
                              const int64_t *targets_dev, int64_t nt, double q, double *out_dev,
                              float *err_dev, void *stream)
{
    if (nt < 1 || !acc_dev || !ref_dev || !out_dev || !err_dev || !(q >= 0.0 && q <= 1.0))
        return NB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_rel_errors<<<nb_grid(nt, 256), 256, 0, s>>>(acc_dev, ref_dev, targets_dev, nt, err_dev);
    k_error_stats<<<1, LB_T, 0, s>>>(err_dev, nt, q, out_dev);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

extern "C" int nb_column_stats(const float *feat_dev, int64_t S, int stride, int ncols,
                               double *mean_dev, double *sd_dev, void *stream)
{
    if (S < 1 || stride < 1 || ncols < 1 || ncols > LB_MAXP || ncols > stride || !feat_dev ||
        !mean_dev || !sd_dev)
        return NB_ERR_INVALID_ARG;
    nb_cols cols = {};
    for (int k = 0; k < ncols; k++) cols.c[k] = k;
    k_fit_stats<<<ncols, 256, 0, (cudaStream_t)stream>>>(feat_dev, S, stride, cols, mean_dev,
                                                          sd_dev);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
