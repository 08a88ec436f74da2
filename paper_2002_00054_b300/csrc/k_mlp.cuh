// k_mlp.cuh -- per-element atomic networks (Fig. 1b step 2; Sec. 3.1 "~30 x 2",
// one network per element) with the input gradient dE_i/dG_i needed by the
// force pass (counted inside the force step in the paper, Fig. 5).
//
// FP32 path: one warp per atom, one neuron per lane (hidden widths <= 32).  The
// weights of every element live in shared memory with an odd row stride, so
// the forward pass (lane = output row, broadcast input) and the backward pass
// (lane = input column, broadcast delta) are both bank-conflict free.
#pragma once
#include "common.cuh"

// Copies the packed caller-layout weights (fp32, all elements) into the padded
// shared-memory image.
__device__ __forceinline__ void load_weights_smem(const Plan& P, const float* __restrict__ w, float* sw)
{
    for (int e = 0; e < P.n_elem; ++e) {
        const float* src = w + (size_t)e * P.n_params_elem;
        float* dst = sw + (size_t)e * P.s_elem;
        for (int l = 0; l < P.n_layers; ++l) {
            const int in = P.width[l], out = P.width[l + 1], ld = P.ld[l];
            for (int t = threadIdx.x; t < out * in; t += blockDim.x) {
                const int o = t / in, k = t - o * in;
                dst[P.s_woff[l] + o * ld + k] = src[P.p_woff[l] + t];
            }
            for (int t = threadIdx.x; t < out; t += blockDim.x) dst[P.s_boff[l] + t] = src[P.p_boff[l] + t];
        }
    }
}

// E_i and dE_i/dG_i from the scaled descriptors G~ = (G - mu)/s (chain rule: dE/dG = dE/dG~ / s).
__global__ void __launch_bounds__(256)
k_mlp_fp32(int n, const float4* __restrict__ pos4, const Plan* __restrict__ plan_g, const float* __restrict__ weights,
           const float* __restrict__ Gs, float* __restrict__ Ei, float* __restrict__ dEdG)
{
    extern __shared__ __align__(16) float sw[];
    const Plan& P = *plan_g;
    load_weights_smem(P, weights, sw);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5, nw = gridDim.x * wpb;
    const int L = P.n_layers;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += nw) {
        const int ti = __float_as_int(pos4[i].w);
        const ElemPlan& E = P.e[ti];
        const float* W = sw + (size_t)ti * P.s_elem;
        const int ng = E.n_g;
        float x0 = 0.f, x1 = 0.f;
        if (lane < ng) x0 = Gs[(size_t)i * P.gs + lane];
        if (lane + 32 < ng) x1 = Gs[(size_t)i * P.gs + lane + 32];
        float act[NNP_MAXL];
        float prev = 0.f, out_v = 0.f;
#pragma unroll
        for (int l = 0; l < NNP_MAXL; ++l) {
            if (l < L) {
                const int in = P.width[l], out = P.width[l + 1], ld = P.ld[l];
                const int o = lane < out ? lane : out - 1;
                const float* Wl = W + P.s_woff[l] + o * ld;
                float a = W[P.s_boff[l] + o];
                for (int k = 0; k < in; ++k) {
                    float xk;
                    if (l == 0) xk = (k < 32) ? __shfl_sync(FULL, x0, k) : __shfl_sync(FULL, x1, k - 32);
                    else xk = __shfl_sync(FULL, prev, k);
                    a = fmaf(Wl[k], xk, a);
                }
                if (l < L - 1) {
                    prev = tanhf(a);
                    act[l] = prev;
                } else {
                    out_v = a;
                    act[l] = 0.f;
                }
            }
        }
        // backward: delta over the current layer's outputs, one per lane
        float delta = (lane == 0) ? 1.f : 0.f;
        float dx0 = 0.f, dx1 = 0.f;
#pragma unroll
        for (int l = NNP_MAXL - 1; l >= 0; --l) {
            if (l < L) {
                const int in = P.width[l], out = P.width[l + 1], ld = P.ld[l];
                if (l < L - 1) delta *= (1.f - act[l] * act[l]);
                if (lane >= out) delta = 0.f;
                const float* Wl = W + P.s_woff[l];
                float n0 = 0.f, n1 = 0.f;
                const int k0 = lane < in ? lane : in - 1;
                const int k1 = lane + 32 < in ? lane + 32 : in - 1;
                for (int o = 0; o < out; ++o) {
                    const float d = __shfl_sync(FULL, delta, o);
                    n0 = fmaf(Wl[o * ld + k0], d, n0);
                    if (l == 0) n1 = fmaf(Wl[o * ld + k1], d, n1);
                }
                if (l > 0) {
                    delta = (lane < in) ? n0 : 0.f;
                } else {
                    dx0 = n0;
                    dx1 = n1;
                }
            }
        }
        if (lane == 0) Ei[i] = out_v;   // the output layer has one row: every lane computed it
        if (dEdG) {
            if (lane < ng) dEdG[(size_t)i * P.gs + lane] = dx0 * E.inv_s[lane];
            if (lane + 32 < ng) dEdG[(size_t)i * P.gs + lane + 32] = dx1 * E.inv_s[lane + 32];
        }
    }
}
