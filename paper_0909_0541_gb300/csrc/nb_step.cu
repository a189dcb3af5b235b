// nb_step.cu -- kick and drift of the FP64 kick-drift-kick leapfrog that
// advances the orbits between force evaluations ("integrate orbits ... and
// repeat", Sec. Introduction).  Elementwise over 3n components:
//   kick   v <- v + fl64(a) h      (h = dt / 2)
//   drift  x <- x + v dt
// each product and sum rounded on its own in FP64.
//
// Both loops are bound by HBM, through the bytes each thread keeps in
// flight: one thread takes 4 consecutive components per round (two 16-byte
// loads of doubles, and one of floats or two more of doubles), four times
// what a component per round keeps in flight.  Arrays that are not 16-byte
// aligned (a caller's buffers at an odd offset) go one component at a time.
#include "nb_internal.cuh"

__device__ __forceinline__ double kick1(double v, float a, double h)
{
    return __dadd_rn(v, __dmul_rn((double)a, h));
}

__device__ __forceinline__ double drift1(double x, double v, double dt)
{
    return __dadd_rn(x, __dmul_rn(v, dt));
}

// V4: vel and acc 16-byte aligned
template <bool V4>
__global__ void __launch_bounds__(256)
k_kick(double *__restrict__ vel, const float *__restrict__ acc, int64_t m, double h)
{
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    int64_t tail = 0;
    if constexpr (V4) {
        const int64_t m4 = m / 4;
        for (int64_t q = t0; q < m4; q += nt) {
            const double2 v0 = reinterpret_cast<const double2 *>(vel)[2 * q];
            const double2 v1 = reinterpret_cast<const double2 *>(vel)[2 * q + 1];
            const float4 a = reinterpret_cast<const float4 *>(acc)[q];
            reinterpret_cast<double2 *>(vel)[2 * q] =
                make_double2(kick1(v0.x, a.x, h), kick1(v0.y, a.y, h));
            reinterpret_cast<double2 *>(vel)[2 * q + 1] =
                make_double2(kick1(v1.x, a.z, h), kick1(v1.y, a.w, h));
        }
        tail = 4 * m4;
    }
    for (int64_t i = tail + t0; i < m; i += nt) vel[i] = kick1(vel[i], acc[i], h);
}

// V4: pos and vel 16-byte aligned
template <bool V4>
__global__ void __launch_bounds__(256)
k_drift(double *__restrict__ pos, const double *__restrict__ vel, int64_t m, double dt)
{
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    int64_t tail = 0;
    if constexpr (V4) {
        const int64_t m4 = m / 4;
        for (int64_t q = t0; q < m4; q += nt) {
            const double2 x0 = reinterpret_cast<const double2 *>(pos)[2 * q];
            const double2 x1 = reinterpret_cast<const double2 *>(pos)[2 * q + 1];
            const double2 v0 = reinterpret_cast<const double2 *>(vel)[2 * q];
            const double2 v1 = reinterpret_cast<const double2 *>(vel)[2 * q + 1];
            reinterpret_cast<double2 *>(pos)[2 * q] =
                make_double2(drift1(x0.x, v0.x, dt), drift1(x0.y, v0.y, dt));
            reinterpret_cast<double2 *>(pos)[2 * q + 1] =
                make_double2(drift1(x1.x, v1.x, dt), drift1(x1.y, v1.y, dt));
        }
        tail = 4 * m4;
    }
    for (int64_t i = tail + t0; i < m; i += nt) pos[i] = drift1(pos[i], vel[i], dt);
}

// Between two steps of a captured sequence: the second kick of one step and
// the first kick and the drift of the next, in one pass over the arrays
// (v <- (v + fl64(a) h) + fl64(a) h, then x <- x + v dt: the same operations,
// in the same order, as the three separate passes).  V4: all three arrays
// 16-byte aligned.
template <bool V4>
__global__ void __launch_bounds__(256)
k_kick_kick_drift(double *__restrict__ pos, double *__restrict__ vel,
                  const float *__restrict__ acc, int64_t m, double h, double dt)
{
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    int64_t tail = 0;
    if constexpr (V4) {
        const int64_t m4 = m / 4;
        for (int64_t q = t0; q < m4; q += nt) {
            const double2 v0 = reinterpret_cast<const double2 *>(vel)[2 * q];
            const double2 v1 = reinterpret_cast<const double2 *>(vel)[2 * q + 1];
            const double2 x0 = reinterpret_cast<const double2 *>(pos)[2 * q];
            const double2 x1 = reinterpret_cast<const double2 *>(pos)[2 * q + 1];
            const float4 a = reinterpret_cast<const float4 *>(acc)[q];
            const double w0 = kick1(kick1(v0.x, a.x, h), a.x, h);
            const double w1 = kick1(kick1(v0.y, a.y, h), a.y, h);
            const double w2 = kick1(kick1(v1.x, a.z, h), a.z, h);
            const double w3 = kick1(kick1(v1.y, a.w, h), a.w, h);
            reinterpret_cast<double2 *>(vel)[2 * q] = make_double2(w0, w1);
            reinterpret_cast<double2 *>(vel)[2 * q + 1] = make_double2(w2, w3);
            reinterpret_cast<double2 *>(pos)[2 * q] =
                make_double2(drift1(x0.x, w0, dt), drift1(x0.y, w1, dt));
            reinterpret_cast<double2 *>(pos)[2 * q + 1] =
                make_double2(drift1(x1.x, w2, dt), drift1(x1.y, w3, dt));
        }
        tail = 4 * m4;
    }
    for (int64_t i = tail + t0; i < m; i += nt) {
        const double w = kick1(kick1(vel[i], acc[i], h), acc[i], h);
        vel[i] = w;
        pos[i] = drift1(pos[i], w, dt);
    }
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

void nb_launch_kick(nb_ctx *c, double *vel, const float *acc, int64_t n, double h)
{
    const bool v4 = aligned16(vel) && aligned16(acc);
    const int grid = nb_grid(v4 ? (3 * n + 3) / 4 : 3 * n, 256, c->num_sms * 8);
    if (v4)
        k_kick<true><<<grid, 256, 0, c->stream>>>(vel, acc, 3 * n, h);
    else
        k_kick<false><<<grid, 256, 0, c->stream>>>(vel, acc, 3 * n, h);
    nb_launched(c, "k_kick");
}

void nb_launch_drift(nb_ctx *c, double *pos, const double *vel, int64_t n, double dt)
{
    const bool v4 = aligned16(pos) && aligned16(vel);
    const int grid = nb_grid(v4 ? (3 * n + 3) / 4 : 3 * n, 256, c->num_sms * 8);
    if (v4)
        k_drift<true><<<grid, 256, 0, c->stream>>>(pos, vel, 3 * n, dt);
    else
        k_drift<false><<<grid, 256, 0, c->stream>>>(pos, vel, 3 * n, dt);
    nb_launched(c, "k_drift");
}

void nb_launch_kick_kick_drift(nb_ctx *c, double *pos, double *vel, const float *acc,
                               int64_t n, double h, double dt)
{
    const bool v4 = aligned16(pos) && aligned16(vel) && aligned16(acc);
    const int grid = nb_grid(v4 ? (3 * n + 3) / 4 : 3 * n, 256, c->num_sms * 8);
    if (v4)
        k_kick_kick_drift<true><<<grid, 256, 0, c->stream>>>(pos, vel, acc, 3 * n, h, dt);
    else
        k_kick_kick_drift<false><<<grid, 256, 0, c->stream>>>(pos, vel, acc, 3 * n, h, dt);
    nb_launched(c, "k_kick_kick_drift");
}
