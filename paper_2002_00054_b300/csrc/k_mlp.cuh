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

// Copies the packed caller-layout weights into the lane-per-atom image (layout in
// Plan: forward W^T and backward W copies per hidden layer, zero padded).
__device__ __forceinline__ void load_weights_lane(const Plan& P, const float* __restrict__ w, float* sw)
{
    const int L = P.n_layers, hp = P.lw_hp;
    for (int t = threadIdx.x; t < P.n_elem * P.lw_elem; t += blockDim.x) sw[t] = 0.f;
    __syncthreads();
    for (int e = 0; e < P.n_elem; ++e) {
        const float* src = w + (size_t)e * P.n_params_elem;
        float* dst = sw + (size_t)e * P.lw_elem;
        for (int l = 0; l + 1 < L; ++l) {
            const int in = P.width[l], out = P.width[l + 1], K = (l == 0) ? P.lw_kb0 : hp;
            for (int t = threadIdx.x; t < out * in; t += blockDim.x) {
                const int o = t / in, k = t - o * in;
                const float v = src[P.p_woff[l] + t];
                dst[P.lw_f[l] + k * hp + o] = v;
                dst[P.lw_b[l] + o * K + k] = v;
            }
            for (int t = threadIdx.x; t < out; t += blockDim.x) dst[P.lw_fb[l] + t] = src[P.p_boff[l] + t];
        }
        for (int t = threadIdx.x; t < P.width[L - 1]; t += blockDim.x) dst[P.lw_out + t] = src[P.p_woff[L - 1] + t];
        if (threadIdx.x == 0) dst[P.lw_outb] = src[P.p_boff[L - 1]];
        for (int t = threadIdx.x; t < P.width[0]; t += blockDim.x) dst[P.lw_invs + t] = P.e[e].inv_s[t];
    }
}

// E_i and dE_i/dG_i from the scaled descriptors G~ = (G - mu)/s (chain rule: dE/dG = dE/dG~ / s).
//
// One lane per atom, 32 consecutive atoms per warp: every layer is a small
// register-blocked product.  Forward: for each input k, the lane's activation
// (from the warp's activation rows in shared memory, row stride 33: no bank
// conflicts) times the row k of W^T (128-bit broadcast reads) into HP
// accumulators.  Backward: for each output o, the lane's delta times the row o
// of W into the input accumulators.  Every sum runs in the same order as the
// textbook loops (k ascending from the bias; o ascending from zero), zero
// padding adds exact zeros.  Lanes of one warp may hold different elements: the
// element images sit 4 words (mod 32) apart, so their reads never share a bank.
// HP: largest hidden width rounded up to 4.
template <int HP>
__global__ void __launch_bounds__(128)
k_mlp_fp32(int n, const float4* __restrict__ pos4, const Plan* __restrict__ plan_g, const float* __restrict__ weights,
           const float* __restrict__ Gs, float* __restrict__ Ei, float* __restrict__ dEdG)
{
    extern __shared__ __align__(16) float sm[];
    const Plan& P = *plan_g;
    load_weights_lane(P, weights, sm);
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float* xs = sm + (size_t)P.n_elem * P.lw_elem + (size_t)wib * P.lw_rows * 33;
    const int L = P.n_layers, ng = P.width[0], kb0 = P.lw_kb0;
    const int tiles = (n + 31) >> 5;
    for (int tile = blockIdx.x * wpb + wib; tile < tiles; tile += gridDim.x * wpb) {
        const int i = tile * 32 + lane;
        const bool live = i < n;
        const int ti = live ? __float_as_int(pos4[i].w) : 0;
        const float* W = sm + (size_t)ti * P.lw_elem;
        // the lane's inputs G~ -> activation rows [0, n_G)
        for (int k = 0; k < ng; k += 4) {
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (live) g = *reinterpret_cast<const float4*>(Gs + (size_t)i * P.gs + k);
            xs[k * 33 + lane] = g.x;
            if (k + 1 < ng) xs[(k + 1) * 33 + lane] = g.y;
            if (k + 2 < ng) xs[(k + 2) * 33 + lane] = g.z;
            if (k + 3 < ng) xs[(k + 3) * 33 + lane] = g.w;
        }
        // forward through the hidden layers: h_{l+1} = tanh(W_l h_l + b_l)
        int row = 0;
        for (int l = 0; l + 1 < L; ++l) {
            const int in = P.width[l], out = P.width[l + 1];
            const float* Wt = W + P.lw_f[l];
            float acc[HP];
#pragma unroll
            for (int o = 0; o < HP; o += 4) {
                const float4 b = *reinterpret_cast<const float4*>(W + P.lw_fb[l] + o);
                acc[o] = b.x; acc[o + 1] = b.y; acc[o + 2] = b.z; acc[o + 3] = b.w;
            }
            for (int k = 0; k < in; ++k) {
                const float x = xs[(row + k) * 33 + lane];
                const float* wr = Wt + k * HP;
#pragma unroll
                for (int o = 0; o < HP; o += 4) {
                    const float4 wv = *reinterpret_cast<const float4*>(wr + o);
                    acc[o] = fmaf(wv.x, x, acc[o]);
                    acc[o + 1] = fmaf(wv.y, x, acc[o + 1]);
                    acc[o + 2] = fmaf(wv.z, x, acc[o + 2]);
                    acc[o + 3] = fmaf(wv.w, x, acc[o + 3]);
                }
            }
            row += in;
#pragma unroll
            for (int o = 0; o < HP; ++o)
                if (o < out) xs[(row + o) * 33 + lane] = tanhf(acc[o]);
        }
        // output layer (one neuron): E_i = w . h + b
        {
            const int in = P.width[L - 1];
            float e = W[P.lw_outb];
            for (int k = 0; k < in; ++k) e = fmaf(W[P.lw_out + k], xs[(row + k) * 33 + lane], e);
            if (live) Ei[i] = e;
        }
        if (!dEdG) continue;
        // backward: dacc = dE/dh of the current layer's inputs, starting with the
        // output layer's weights; delta = dacc * tanh' for the layer below
        if (L == 1) {
            for (int k = 0; k < ng; ++k)
                if (live) dEdG[(size_t)i * P.gs + k] = W[P.lw_out + k] * W[P.lw_invs + k];
            continue;
        }
        float dacc[HP];
#pragma unroll
        for (int o = 0; o < HP; o += 4) {
            const float4 v = *reinterpret_cast<const float4*>(W + P.lw_out + o);
            dacc[o] = v.x; dacc[o + 1] = v.y; dacc[o + 2] = v.z; dacc[o + 3] = v.w;
        }
        for (int l = L - 2; l >= 0; --l) {
            const int out = P.width[l + 1];
            row -= P.width[l];   // first row of h_l; h_{l+1} follows at row + in_l
            const int hrow = row + P.width[l];
            // delta_o = dE/dh_{l+1}[o] * (1 - h_{l+1}[o]^2), written over h_{l+1}
#pragma unroll
            for (int o = 0; o < HP; ++o)
                if (o < out) {
                    float* hp = xs + (hrow + o) * 33 + lane;
                    const float a = *hp;
                    *hp = dacc[o] * (1.f - a * a);
                }
            const float* Wb = W + P.lw_b[l];
            if (l > 0) {
#pragma unroll
                for (int k = 0; k < HP; ++k) dacc[k] = 0.f;
                for (int o = 0; o < out; ++o) {
                    const float d = xs[(hrow + o) * 33 + lane];
                    const float* wr = Wb + o * HP;
#pragma unroll
                    for (int k = 0; k < HP; k += 4) {
                        const float4 wv = *reinterpret_cast<const float4*>(wr + k);
                        dacc[k] = fmaf(wv.x, d, dacc[k]);
                        dacc[k + 1] = fmaf(wv.y, d, dacc[k + 1]);
                        dacc[k + 2] = fmaf(wv.z, d, dacc[k + 2]);
                        dacc[k + 3] = fmaf(wv.w, d, dacc[k + 3]);
                    }
                }
            } else {
                // input layer: dE/dG = (sum_o W_0[o][k] delta_o) / s_k, 32 inputs at a time
                for (int kb = 0; kb < kb0; kb += 32) {
                    float dx[32];
#pragma unroll
                    for (int k = 0; k < 32; ++k) dx[k] = 0.f;
                    for (int o = 0; o < out; ++o) {
                        const float d = xs[(hrow + o) * 33 + lane];
                        const float* wr = Wb + o * kb0 + kb;
#pragma unroll
                        for (int k = 0; k < 32; k += 4) {
                            const float4 wv = *reinterpret_cast<const float4*>(wr + k);
                            dx[k] = fmaf(wv.x, d, dx[k]);
                            dx[k + 1] = fmaf(wv.y, d, dx[k + 1]);
                            dx[k + 2] = fmaf(wv.z, d, dx[k + 2]);
                            dx[k + 3] = fmaf(wv.w, d, dx[k + 3]);
                        }
                    }
                    if (live) {
#pragma unroll
                        for (int k = 0; k < 32; k += 4)
                            if (kb + k < P.gs) {
                                const float4 is = *reinterpret_cast<const float4*>(W + P.lw_invs + kb + k);
                                *reinterpret_cast<float4*>(dEdG + (size_t)i * P.gs + kb + k) =
                                    make_float4(dx[k] * is.x, dx[k + 1] * is.y, dx[k + 2] * is.z, dx[k + 3] * is.w);
                            }
                    }
                }
            }
        }
    }
}
