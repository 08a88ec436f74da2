// k_md.cuh -- FP64 reductions (E_system += E_i, Fig. 1b; virial; kinetic energy)
// and the velocity-Verlet NVE update (energy conservation, Sec. 4.2).
// Reductions are two-stage with a fixed order, so results repeat bit for bit.
#pragma once
#include "common.cuh"

#define RED_THREADS 256

__device__ __forceinline__ double block_sum_d(double v, double* sh)
{
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    __syncthreads();
    return t;
}

// per-block partial sums of a float array in double; also flags non-finite values
__global__ void k_sum_partial(int n, const float* __restrict__ x, double* __restrict__ part, int* __restrict__ flags)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float f = x[i];
        if (!isfinite(f)) atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
        v += (double)f;
    }
    const double t = block_sum_d(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// energy = sum of n_e partials (-> out_e[0], nullable); virial[q] = sum of n_v
// per-warp partials (-> out_v[9], nullable).  One block, fixed order.
__global__ void k_finalize(int n_e, const double* __restrict__ epart, double* __restrict__ out_e,
                           int n_v, const double* __restrict__ vpart, double* __restrict__ out_v)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int k = threadIdx.x; k < n_e; k += blockDim.x) v += epart[k];
    const double e = block_sum_d(v, sh);
    if (threadIdx.x == 0 && out_e) out_e[0] = e;
    for (int q = 0; q < 9; ++q) {
        double a = 0.0;
        for (int k = threadIdx.x; k < n_v; k += blockDim.x) a += vpart[(size_t)k * 9 + q];
        const double t = block_sum_d(a, sh);
        if (threadIdx.x == 0 && out_v) out_v[q] = t;
    }
}

// v += dt/2 F a_m ; x += dt v     (a_m = acc_over_m[type] = (eV/(A amu) in A/fs^2) / m)
__global__ void k_kick_drift(int n, const Plan* __restrict__ plan_g, const int* __restrict__ types,
                             const float* __restrict__ F, float* __restrict__ vel, float* __restrict__ pos, float dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = types[i];
    const float am = plan_g->acc_over_m[(t >= 0 && t < plan_g->n_elem) ? t : 0];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float v = vel[3 * i + c] + 0.5f * dt * F[3 * i + c] * am;
        vel[3 * i + c] = v;
        pos[3 * i + c] += dt * v;
    }
}

// v += dt/2 F a_m (skipped when dt == 0), then per-block partial kinetic energy
// sum 1/2 m v^2 (in eV: divided by the unit factor, i.e. 1/(2 a_m)).
__global__ void k_kick_ke(int n, const Plan* __restrict__ plan_g, const int* __restrict__ types,
                          const float* __restrict__ F, float* __restrict__ vel, float dt, double* __restrict__ part)
{
    __shared__ double sh[32];
    double ke = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = types[i];
        const float am = plan_g->acc_over_m[(t >= 0 && t < plan_g->n_elem) ? t : 0];
        double v2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float v = vel[3 * i + c];
            if (dt != 0.f) {
                v += 0.5f * dt * F[3 * i + c] * am;
                vel[3 * i + c] = v;
            }
            v2 += (double)v * (double)v;
        }
        ke += 0.5 * v2 / (double)am;
    }
    const double s = block_sum_d(ke, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// log[2k + slot] = sum of partials (one block)
// F = Fq unit: the fixed-point scatter's integer sums with one rounding each
// (unit 2^-LB of the model's kind; |Fq| < 2^52, so the conversion to double and
// the scaling are exact)
__global__ void k_fq_forces(int n3, const unsigned long long* __restrict__ Fq, double unit, float* __restrict__ F)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n3) F[t] = (float)((double)(long long)Fq[t] * unit);
}

// Energy-log entry s = (*slot)++: log[2s] = potential energy (*epot), log[2s+1] =
// kinetic energy (the sum of the partials).  The entry index lives on the device,
// so one launch with fixed arguments serves every step of a replayed step graph.
__global__ void k_log_sum(int np, const double* __restrict__ part, const double* __restrict__ epot,
                          double* __restrict__ log, unsigned long long* __restrict__ slot)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) v += part[k];
    const double s = block_sum_d(v, sh);
    if (threadIdx.x == 0) {
        const unsigned long long e = *slot;
        log[2 * e] = *epot;
        log[2 * e + 1] = s;
        *slot = e + 1;
    }
}

