// k_train.cuh -- the differentiation form: parameter gradients of energies and
// of forces (force matching), for batches of independent systems.
//
// For a loss L(E, F) with F = -dE/dr:
//   dL/dtheta = sum_b (dL/dE_b) dE_b/dtheta + sum_m u_m . dF_m/dtheta,  u = dL/dF.
// Since F is a position gradient, the second term equals
//   - d/dtheta sum_i grad_G E_i(G_i; theta) . t_i,    t_i = sum_j dG_i/dd_ij . (u_j - u_i),
// i.e. the directional derivative of the descriptors along u (k_tangent, which
// recomputes dG/dr pair by pair like the force pass) followed by the
// reverse-over-forward derivative of the network's tangent with respect to its
// parameters (k_param_grad).  Position second derivatives are not formed.
#pragma once
#include "common.cuh"
#include "k_descriptors.cuh"

__host__ __device__ inline size_t tangent_warp_bytes(int C)
{
    // nd, npf, ndp, nfe (f_c, f_c', element, h), dv (du, r^ . du) as float4; ninv; queue; FP64 sums
    return (size_t)C * (16 * 5 + 4) + PAIR_QUEUE * 2 + NNP_MAXG * 8;
}

// t~_i = (dG_i/dr . u) / s for every atom (scaled descriptor tangent).
template <int NETA, bool NARROW, int KP, int KN, bool RES>
__global__ void __launch_bounds__(128, 4)
k_tangent(int n, const float4* __restrict__ pos4, Box bx, NbView nv, const Plan* __restrict__ plan_g, int C,
          const float* __restrict__ u, float* __restrict__ T, int* __restrict__ flags, int* __restrict__ spill,
          int pass)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Plan& P = *plan_g;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    unsigned char* base = smem + tangent_warp_bytes(C) * wib;
    float4* nd = reinterpret_cast<float4*>(base);
    float4* npf = nd + C;
    float4* ndp = npf + C;
    float4* nfe = ndp + C;
    float4* ndv = nfe + C;
    double* sT = reinterpret_cast<double*>(ndv + C);
    float* ninv = reinterpret_cast<float*>(sT + NNP_MAXG);
    unsigned short* queue = reinterpret_cast<unsigned short*>(ninv + C);

    const int nw = gridDim.x * wpb;
    const int n_items = atom_count(pass, n, spill);
    unsigned long long c_spill = 0;
    for (int it = blockIdx.x * wpb + wib; it < n_items; it += nw) {
        const int i = atom_at(pass, it, spill);
        const float4 pi = pos4[i];
        const int ti = __float_as_int(pi.w);
        const ElemPlan& E = P.e[ti];
        float khi[4], klo[4], etav[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            etav[q] = (q < E.n_eta) ? E.ang_eta[q] : 0.f;
            khi[q] = (q < E.n_eta) ? E.ang_khi[q] : 0.f;
            klo[q] = (q < E.n_eta) ? E.ang_klo[q] : 0.f;
        }
        const float uix = u[3 * i], uiy = u[3 * i + 1], uiz = u[3 * i + 2];
        // staging: neighbours inside the cutoff, compacted in list order
        const int cnt = nv.ncount[i];
        const uint32_t* row = nv.nbr + (size_t)i * nv.stride;
        float Lx, Ly, Lz;
        atom_box(nv, bx, i, Lx, Ly, Lz);
        int M = 0;
        // list entries two rounds ahead, positions one round ahead
        uint32_t e_n = (lane < cnt) ? row[lane] : 0u;
        uint32_t e_nn = (lane + 32 < cnt) ? row[lane + 32] : 0u;
        float4 p_n = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < cnt) p_n = pos4[e_n & NB_INDEX_MASK];
        for (int b0 = 0; b0 < cnt; b0 += 32) {
            const int s = b0 + lane;
            const uint32_t e = e_n;
            const float4 pj = p_n;
            e_n = e_nn;
            if (s + 32 < cnt) p_n = pos4[e_nn & NB_INDEX_MASK];
            e_nn = (s + 64 < cnt) ? row[s + 64] : 0u;
            bool keep = false;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
            int j = 0, ej = 0;
            if (s < cnt) {
                j = (int)(e & NB_INDEX_MASK);
                float ox, oy, oz;
                nb_shift(e, Lx, Ly, Lz, ox, oy, oz);
                dx = pair_disp(pj.x, pi.x, ox);
                dy = pair_disp(pj.y, pi.y, oy);
                dz = pair_disp(pj.z, pi.z, oz);
                r2 = dist2_fma(dx, dy, dz);
                ej = __float_as_int(pj.w);
                keep = r2 < P.rc2;
            }
            const unsigned m = __ballot_sync(FULL, keep);
            const int at = M + __popc(m & ((1u << lane) - 1u));
            if (keep && at < C) {
                const float r = sqrtf(r2), ir = 1.0f / r;
                float fc, dfc;
                cutoff_fn(r, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, fc, dfc);
                float pq[4] = {0.f, 0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int q = 0; q < NETA; ++q) {
                    const float ex = gauss2(khi[q], klo[q], r2);
                    pq[q] = ex * fc;
                    dq[q] = ex * (dfc - 2.0f * etav[q] * r * fc);
                }
                const float dvx = u[3 * j] - uix, dvy = u[3 * j + 1] - uiy, dvz = u[3 * j + 2] - uiz;
                nd[at] = make_float4(dx, dy, dz, r);
                ninv[at] = ir;
                npf[at] = make_float4(pq[0], pq[1], pq[2], pq[3]);
                ndp[at] = make_float4(dq[0], dq[1], dq[2], dq[3]);
                nfe[at] = make_float4(fc, dfc, __int_as_float(ej), live_h(r2, P.rc2));
                ndv[at] = make_float4(dvx, dvy, dvz, (dx * dvx + dy * dvy + dz * dvz) * ir);
            }
            M += __popc(m);
        }
        __syncwarp();
        if (over_capacity(M, C, pass, i, spill, false, lane, flags, c_spill)) continue;
        // radial: lane <-> descriptor; t = sum_j dG/dr (r^ . du_j)
        for (int rr = lane; rr < E.n_rad; rr += 32) {
            const float kh = E.rad_khi[rr], kl = E.rad_klo[rr], rs = E.rad_rs[rr], eta = E.rad_eta[rr];
            const int el = E.rad_elem[rr];
            float acc = 0.f;
            for (int m = 0; m < M; ++m) {
                const float4 fe = nfe[m];
                if (el < 0 || el == __float_as_int(fe.z)) {
                    const float x = nd[m].w - rs;
                    const float ex = gauss2(kh, kl, x * x);
                    acc = fmaf(ex * (fe.y - 2.0f * eta * x * fe.x), ndv[m].w, acc);
                }
            }
            sT[E.rad_out[rr]] = acc;
        }
        // angular (one pass per neighbour-element pair class)
        const int ncls = RES ? E.n_cls : 1;
        for (int cls = 0; NETA > 0 && cls < ncls; ++cls) {
            constexpr int NQ = NETA > 0 ? NETA : 1, NP = (NQ + 1) / 2;
            constexpr int NA = NQ * 2 * (NNP_KMAX + 1);
            // accumulators of eta pairs (q = 2p, 2p + 1) as packed f32x2
            float2 acc[NP][2][NNP_KMAX + 1];
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int l = 0; l < 2; ++l)
#pragma unroll
                    for (int kk = 0; kk <= NNP_KMAX; ++kk) acc[p][l][kk] = f2(0.f, 0.f);
            float2 KH[NP], KL[NP], ET[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                KH[p] = f2(khi[2 * p], (2 * p + 1 < 4) ? khi[2 * p + 1] : 0.f);
                KL[p] = f2(klo[2 * p], (2 * p + 1 < 4) ? klo[2 * p + 1] : 0.f);
                ET[p] = f2(-2.0f * etav[2 * p], (2 * p + 1 < 4) ? -2.0f * etav[2 * p + 1] : 0.f);
            }
            const int nb = (M + 31) >> 5;
            const int ce1 = RES ? E.cls_e1[cls] : -1, ce2 = RES ? E.cls_e2[cls] : -1;
            for (int A = 0; A < nb; ++A) {
                const int jl = 32 * A + lane;
                const float4 al = (jl < M) ? nd[jl] : make_float4(0.f, 0.f, 0.f, 0.f);
                const int ej = (RES && jl < M) ? __float_as_int(nfe[jl].z) : -1;
                for (int B = A; B < nb; ++B) {
                    unsigned mask = live_mask<NARROW, 4>(A, B, lane, M, al, (jl < M) ? nfe[jl].w : 0.f, nd,
                                                         &nfe[0].w);
                    if (RES && ce1 >= 0) {
                        const int kl = 32 * B + lane;
                        mask &= class_mask(ej, kl < M ? __float_as_int(nfe[kl].z) : -1, ce1, ce2, lane);
                    }
                    const int total = enqueue_block(mask, lane, queue, A == B);
                    for (int e0 = 0; e0 < total; e0 += 32) {
                        const int e = e0 + lane;
                        if (e >= total) continue;
                        const int ent = queue[e];
                        const int l = ent & 31, sidx = ent >> 5;
                        const int j = 32 * A + l, k = 32 * B + ((l + sidx) & 31);
                        const float4 a = nd[j], b = nd[k], va = ndv[j], vb = ndv[k];
                        const float4 pa4 = npf[j], pb4 = npf[k], qa4 = ndp[j], qb4 = ndp[k];
                        const float pav[4] = {pa4.x, pa4.y, pa4.z, pa4.w}, pbv[4] = {pb4.x, pb4.y, pb4.z, pb4.w};
                        const float qav[4] = {qa4.x, qa4.y, qa4.z, qa4.w}, qbv[4] = {qb4.x, qb4.y, qb4.z, qb4.w};
                        const float ia = ninv[j], ib = ninv[k], iab = ia * ib;
                        const float c = (a.x * b.x + a.y * b.y + a.z * b.z) * iab;
                        // dc = d(cos) along (du_j, du_k); va.w = r^_j . du_j
                        const float dc = (b.x * va.x + b.y * va.y + b.z * va.z) * iab - c * va.w * ia +
                                         (a.x * vb.x + a.y * vb.y + a.z * vb.z) * iab - c * vb.w * ib;
                        float fcd = 1.f, dfcd = 0.f, rd2 = 0.f, rd = 1.f, drd = 0.f;
                        if (NARROW) {
                            const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
                            rd2 = ex * ex + ey * ey + ez * ez;
                            const float ird = rsqrtf(rd2);
                            rd = rd2 * ird;
                            cutoff_fn_fast(rd, P.hpi_rc, fcd, dfcd);
                            drd = (ex * (vb.x - va.x) + ey * (vb.y - va.y) + ez * (vb.z - va.z)) * ird;
                        }
                        float pw[2][NNP_KMAX + 1], qd[2][NNP_KMAX + 1];   // b^(2^k), d/dc b^(2^k) * dc
#pragma unroll
                        for (int lb = 0; lb < 2; ++lb) {
                            const float bl = (lb == 0) ? 1.f + c : 1.f - c;
                            float qk = 1.f;
                            pw[lb][0] = bl;
                            qd[lb][0] = (lb == 0) ? dc : -dc;
#pragma unroll
                            for (int kk = 1; kk <= NNP_KMAX; ++kk) {
                                if (kk <= (lb == 0 ? KP : KN)) {
                                    qk = qk * pw[lb][kk - 1];
                                    pw[lb][kk] = pw[lb][kk - 1] * pw[lb][kk - 1];
                                    qd[lb][kk] = qk * dc * ((lb == 0 ? 1.f : -1.f) * (float)(1 << kk));
                                }
                            }
                        }
                        if constexpr (NETA % 2 == 0) {
                            // even eta count: both of a pair in one packed instruction
#pragma unroll
                            for (int p = 0; p < NP; ++p) {
                                const float2 PA = f2(pav[2 * p], pav[2 * p + 1]), PB = f2(pbv[2 * p], pbv[2 * p + 1]);
                                const float2 QA = f2(qav[2 * p], qav[2 * p + 1]), QB = f2(qbv[2 * p], qbv[2 * p + 1]);
                                float2 Pd = f2(1.f, 1.f), dPd = f2(0.f, 0.f);
                                if (NARROW) {
                                    const float2 x2 = f2(rd2, rd2);
                                    const float2 arg = fma2(KH[p], x2, mul2(KL[p], x2));
                                    const float2 ed = f2(exp2f(arg.x), exp2f(arg.y));
                                    Pd = mul2(ed, f2(fcd, fcd));
                                    const float rf = rd * fcd;
                                    dPd = mul2(ed, fma2(ET[p], f2(rf, rf), f2(dfcd, dfcd)));
                                }
                                const float2 pab = mul2(PA, PB);
                                const float2 R = mul2(pab, Pd);
                                float2 dR = mul2(fma2(mul2(QA, PB), f2(va.w, va.w), mul2(mul2(PA, QB), f2(vb.w, vb.w))), Pd);
                                if (NARROW) dR = fma2(mul2(pab, dPd), f2(drd, drd), dR);
#pragma unroll
                                for (int lb = 0; lb < 2; ++lb)
#pragma unroll
                                    for (int kk = 0; kk <= NNP_KMAX; ++kk)
                                        if (kk <= (lb == 0 ? KP : KN))
                                            acc[p][lb][kk] = fma2(f2(pw[lb][kk], pw[lb][kk]), dR,
                                                                  fma2(f2(qd[lb][kk], qd[lb][kk]), R, acc[p][lb][kk]));
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < NETA; ++q) {
                                float Pd = 1.f, dPd = 0.f;
                                if (NARROW) {
                                    const float ed = gauss2(khi[q], klo[q], rd2);
                                    Pd = ed * fcd;
                                    dPd = ed * (dfcd - 2.0f * etav[q] * rd * fcd);
                                }
                                const float R = pav[q] * pbv[q] * Pd;
                                float dR = (qav[q] * pbv[q] * va.w + pav[q] * qbv[q] * vb.w) * Pd;
                                if (NARROW) dR = fmaf(pav[q] * pbv[q] * dPd, drd, dR);
#pragma unroll
                                for (int lb = 0; lb < 2; ++lb)
#pragma unroll
                                    for (int kk = 0; kk <= NNP_KMAX; ++kk)
                                        if (kk <= (lb == 0 ? KP : KN)) {
                                            float2& a2 = acc[q >> 1][lb][kk];
                                            float& av = (q & 1) ? a2.y : a2.x;
                                            av = fmaf(pw[lb][kk], dR, fmaf(qd[lb][kk], R, av));
                                        }
                            }
                        }
                    }
                    __syncwarp();
                }
            }
#pragma unroll
            for (int c0 = 0; c0 < NA; c0 += 32) {
                float v[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int idx = c0 + t;
                    const int q = idx / (2 * (NNP_KMAX + 1)), l = (idx / (NNP_KMAX + 1)) % 2, kk = idx % (NNP_KMAX + 1);
                    v[t] = (idx < NA) ? ((q & 1) ? acc[q >> 1][l][kk].y : acc[q >> 1][l][kk].x) : 0.f;
                }
                const double tot = warp_reduce_scatter32(v, lane);
                const int idx = c0 + lane;
                if (idx < NA) {
                    const int q = idx / (2 * (NNP_KMAX + 1)), l = (idx / (NNP_KMAX + 1)) % 2, kk = idx % (NNP_KMAX + 1);
                    const int o = (q < E.n_eta) ? E.ang_out[cls][q][l][kk] : -1;
                    if (o >= 0) sT[o] = tot * (double)exp2f((float)(1 - (1 << kk)));
                }
            }
        }
        __syncwarp();
        for (int s = lane; s < E.n_g; s += 32) T[(size_t)i * P.gs + s] = (float)(sT[s] * (double)E.inv_s[s]);
        __syncwarp();
    }
}

// Parameter gradient of Q_i = hbar_i E_i + hdbar Edot_i, Edot_i = grad_x E_i . xdot_i
// (x = G~_i, xdot = t~_i), summed over atoms.  Warps walk the element-sorted atom
// list (so each warp meets each element in one contiguous segment), accumulate in
// their own shared-memory block laid out like the padded weight image (lane =
// output unit of a layer, odd row strides) and write each element segment to
// part[warp][element] in the packed layout.  Two hidden layers.
__global__ void __launch_bounds__(128)
k_param_grad(int n, const Plan* __restrict__ plan_g, const float* __restrict__ weights,
             const float4* __restrict__ pos4, const int* __restrict__ idx, const int* __restrict__ sys_of,
             const double* __restrict__ dLdE, const float* __restrict__ Gs, const float* __restrict__ T,
             float* __restrict__ part)
{
    extern __shared__ __align__(16) float sw_tr[];
    const Plan& P = *plan_g;
    load_weights_smem(P, weights, sw_tr);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float* acc = sw_tr + (size_t)P.n_elem * P.s_elem + (size_t)wib * P.s_elem;
    __syncthreads();
    const int nin = P.width[0], H1 = P.width[1], H2 = P.width[2];
    const int ld0 = P.ld[0], ld1 = P.ld[1];
    const int gw = blockIdx.x * wpb + wib, nw = gridDim.x * wpb;
    const float hdbar = T ? -1.f : 0.f;
    const int o1 = lane < H1 ? lane : H1 - 1, o2 = lane < H2 ? lane : H2 - 1;

    auto flush = [&](int e) {
        __syncwarp();
        float* dst = part + ((size_t)gw * P.n_elem + e) * P.n_params_elem;
        for (int l = 0; l < P.n_layers; ++l) {
            const int in = P.width[l], out = P.width[l + 1], ld = P.ld[l];
            for (int q = lane; q < out * in; q += 32) {
                const int o = q / in, k = q - o * in;
                dst[P.p_woff[l] + q] = acc[P.s_woff[l] + o * ld + k];
            }
            for (int q = lane; q < out; q += 32) dst[P.p_boff[l] + q] = acc[P.s_boff[l] + q];
        }
        __syncwarp();
    };
    int cur = -1;
    for (int r = gw; r < n; r += nw) {
        const int i = idx[r];
        const int e = __float_as_int(pos4[i].w);
        if (e != cur) {
            if (cur >= 0) flush(cur);
            cur = e;
            for (int q = lane; q < P.s_elem; q += 32) acc[q] = 0.f;
            __syncwarp();
        }
        const float* W = sw_tr + (size_t)e * P.s_elem;
        const float* W1 = W + P.s_woff[0];
        const float* B1 = W + P.s_boff[0];
        const float* W2 = W + P.s_woff[1];
        const float* B2 = W + P.s_boff[1];
        const float* W3 = W + P.s_woff[2];
        const double hb = dLdE ? dLdE[sys_of ? sys_of[i] : 0] : 0.0;
        const float hbar = (float)hb;
        const float* x = Gs + (size_t)i * P.gs;
        const float x0 = lane < nin ? x[lane] : 0.f, x1 = lane + 32 < nin ? x[lane + 32] : 0.f;
        float xd0 = 0.f, xd1 = 0.f;
        if (T) {
            xd0 = lane < nin ? T[(size_t)i * P.gs + lane] : 0.f;
            xd1 = lane + 32 < nin ? T[(size_t)i * P.gs + lane + 32] : 0.f;
        }
        // forward, primal and tangent
        float a1 = B1[o1], ad1 = 0.f;
        for (int k = 0; k < nin; ++k) {
            const float xk = k < 32 ? __shfl_sync(FULL, x0, k) : __shfl_sync(FULL, x1, k - 32);
            const float xdk = k < 32 ? __shfl_sync(FULL, xd0, k) : __shfl_sync(FULL, xd1, k - 32);
            const float wv = W1[o1 * ld0 + k];
            a1 = fmaf(wv, xk, a1);
            ad1 = fmaf(wv, xdk, ad1);
        }
        const float h1 = lane < H1 ? tanhf(a1) : 0.f;
        const float hd1 = lane < H1 ? (1.f - h1 * h1) * ad1 : 0.f;
        float a2 = B2[o2], ad2 = 0.f;
        for (int k = 0; k < H1; ++k) {
            const float wv = W2[o2 * ld1 + k];
            a2 = fmaf(wv, __shfl_sync(FULL, h1, k), a2);
            ad2 = fmaf(wv, __shfl_sync(FULL, hd1, k), ad2);
        }
        const float h2 = lane < H2 ? tanhf(a2) : 0.f;
        const float hd2 = lane < H2 ? (1.f - h2 * h2) * ad2 : 0.f;
        // reverse: output layer (linear)
        const float w3o = lane < H2 ? W3[o2] : 0.f;
        if (lane < H2) acc[P.s_woff[2] + lane] += hbar * h2 + hdbar * hd2;
        if (lane == 0) acc[P.s_boff[2]] += hbar;
        // second hidden layer (tanh)
        const float hb2 = w3o * hbar, hdb2 = w3o * hdbar;
        const float s2 = 1.f - h2 * h2;
        const float adb2 = lane < H2 ? hdb2 * s2 : 0.f;
        const float ab2 = lane < H2 ? (hb2 - 2.f * h2 * hdb2 * ad2) * s2 : 0.f;
        for (int k = 0; k < H1; ++k) {
            const float h1k = __shfl_sync(FULL, h1, k), hd1k = __shfl_sync(FULL, hd1, k);
            if (lane < H2) acc[P.s_woff[1] + lane * ld1 + k] += ab2 * h1k + adb2 * hd1k;
        }
        if (lane < H2) acc[P.s_boff[1] + lane] += ab2;
        // back to the first hidden layer: lane k holds h1bar_k, h1dotbar_k
        float hb1 = 0.f, hdb1 = 0.f;
        for (int o = 0; o < H2; ++o) {
            const float wv = W2[o * ld1 + o1];
            hb1 = fmaf(wv, __shfl_sync(FULL, ab2, o), hb1);
            hdb1 = fmaf(wv, __shfl_sync(FULL, adb2, o), hdb1);
        }
        const float s1 = 1.f - h1 * h1;
        const float adb1 = lane < H1 ? hdb1 * s1 : 0.f;
        const float ab1 = lane < H1 ? (hb1 - 2.f * h1 * hdb1 * ad1) * s1 : 0.f;
        for (int k = 0; k < nin; ++k) {
            const float xk = k < 32 ? __shfl_sync(FULL, x0, k) : __shfl_sync(FULL, x1, k - 32);
            const float xdk = k < 32 ? __shfl_sync(FULL, xd0, k) : __shfl_sync(FULL, xd1, k - 32);
            if (lane < H1) acc[P.s_woff[0] + lane * ld0 + k] += ab1 * xk + adb1 * xdk;
        }
        if (lane < H1) acc[P.s_boff[0] + lane] += ab1;
        __syncwarp();
    }
    if (cur >= 0) flush(cur);
}

// grad[q] = sum over warps of part[warp][q] (FP64, fixed order), q over all elements' parameters
__global__ void k_grad_reduce(int n_warps, int n_elem, int npe, const float* __restrict__ part, float* __restrict__ grad)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_elem * npe) return;
    double s = 0.0;
    for (int w = 0; w < n_warps; ++w) s += (double)part[(size_t)w * n_elem * npe + q];
    grad[q] = (float)s;
}

// energies[b] = sum of E_i over system b (FP64, one block per system, fixed order)
__global__ void k_sys_energy(const int* __restrict__ sys_start, const float* __restrict__ Ei,
                             double* __restrict__ energies, int* __restrict__ flags)
{
    __shared__ double sh[32];
    const int b = blockIdx.x;
    const int lo = sys_start[b], hi = sys_start[b + 1];
    double v = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float e = Ei[i];
        if (!isfinite(e)) atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
        v += (double)e;
    }
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
        energies[b] = t;
    }
}
