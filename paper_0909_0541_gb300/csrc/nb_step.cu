// nb_step.cu -- kick and drift of the FP64 kick-drift-kick leapfrog that
// advances the orbits between force evaluations ("integrate orbits ... and
// repeat", Sec. Introduction).  Elementwise over 3n components.
#include "nb_internal.cuh"

__global__ void __launch_bounds__(256)
k_kick(double *__restrict__ vel, const float *__restrict__ acc, int64_t m, double h)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        vel[i] = __dadd_rn(vel[i], __dmul_rn((double)acc[i], h));
}

__global__ void __launch_bounds__(256)
k_drift(double *__restrict__ pos, const double *__restrict__ vel, int64_t m, double dt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        pos[i] = __dadd_rn(pos[i], __dmul_rn(vel[i], dt));
}

void nb_launch_kick(nb_ctx *c, double *vel, const float *acc, int64_t n, double h)
{
    k_kick<<<nb_grid(3 * n, 256, c->num_sms * 8), 256, 0, c->stream>>>(vel, acc, 3 * n, h);
    nb_launched(c, "k_kick");
}

void nb_launch_drift(nb_ctx *c, double *pos, const double *vel, int64_t n, double dt)
{
    k_drift<<<nb_grid(3 * n, 256, c->num_sms * 8), 256, 0, c->stream>>>(pos, vel, 3 * n, dt);
    nb_launched(c, "k_drift");
}
