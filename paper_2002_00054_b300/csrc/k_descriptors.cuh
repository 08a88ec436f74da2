// k_descriptors.cuh -- symmetry functions (Fig. 1b step 1 and the angular loop of
// Sec. 3.1) and the chain-rule force pass (Fig. 1b step 3).
//
// Mapping: one warp per centre atom i (the paper's "flat" atom parallelism, but
// with the neighbour and pair loops spread over the 32 lanes of the warp instead
// of one thread).  The warp stages its atom's neighbours inside the cutoff into
// shared memory (compacted with a ballot), with per-neighbour radius and the
// angular pair factors P_q(r) = exp(-eta_q r^2) f_c(r) precomputed once, then
// walks all pairs j < k of that list in a flattened order (pair p = lane, lane+32,
// ...), so lanes stay busy however short the rows get.
//
// Angular accumulators are dense in (eta_q, lambda, k) with zeta = 2^k: the
// powers (1 +- cos)^(2^k) come from repeated squaring, and the model's
// descriptors are gathered from the dense set at the end.
//
// The force pass recomputes every descriptor derivative instead of storing
// dG/dr (the paper's recompute-not-store rule, Sec. 3.3 and Sec. 5): for each
// pair it contracts the derivative with dE_i/dG_i on the fly and accumulates
// g_ij = dE_i/dd_ij per neighbour entry in shared memory.  g is written per
// neighbour-list slot; forces are then gathered per atom (k_gather).
#pragma once
#include "common.cuh"

struct NbView {
    const uint32_t* nbr;
    const int* ncount;
    int stride;
};

// Stages the neighbours of atom i within the cutoff.  Returns M (count kept).
// nd[m] = (dx, dy, dz, r); npf[m] = P_q (q < 4); nfe[m] = (f_c, element, f_c', unused)
// FORCE: ndp[m] = dP_q/dr, cmap[slot] = compact index or -1, sg[3m..] = radial part of g.
template <int NETA, bool FORCE>
__device__ __forceinline__ int stage_neighbors(int i, const float4 pi, const Box& bx, const NbView& nv,
                                               const float4* __restrict__ pos4, const Plan& P,
                                               const ElemPlan& E, const float* __restrict__ khi,
                                               const float* __restrict__ klo, const float* __restrict__ etav, int cap, float4* nd, float4* npf,
                                               float4* ndp, float2* nfe, int* cmap, float* sg,
                                               const float* sW, int lane, int* flags, int& n_list)
{
    const int cnt = nv.ncount[i];
    n_list = cnt;
    const uint32_t* row = nv.nbr + (size_t)i * nv.stride;
    int M = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int s = base + lane;
        bool keep = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        int ej = 0;
        if (s < cnt) {
            const uint32_t e = row[s];
            const float4 pj = pos4[e & NB_INDEX_MASK];
            float ox, oy, oz;
            nb_shift(e, bx.L[0], bx.L[1], bx.L[2], ox, oy, oz);
            dx = pair_disp(pj.x, pi.x, ox);
            dy = pair_disp(pj.y, pi.y, oy);
            dz = pair_disp(pj.z, pi.z, oz);
            r2 = dx * dx + dy * dy + dz * dz;
            ej = __float_as_int(pj.w);
            keep = r2 < P.rc2;
        }
        const unsigned m = __ballot_sync(FULL, keep);
        const int at = M + __popc(m & ((1u << lane) - 1u));
        if (FORCE && s < cnt) cmap[s] = (keep && at < cap) ? at : -1;
        if (keep && at < cap) {
            if (r2 < 1e-8f) atomicOr(&flags[FLAG_ERR], ERR_CLOSE);
            const float r = sqrtf(r2);
            float fc, dfc;
            cutoff_fn(r, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, fc, dfc);
            nd[at] = make_float4(dx, dy, dz, r);
            float pq[4] = {0.f, 0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < NETA; ++q) {
                const float ex = gauss2(khi[q], klo[q], r2);
                pq[q] = ex * fc;
                dq[q] = ex * (dfc - 2.0f * etav[q] * r * fc);
            }
            npf[at] = make_float4(pq[0], pq[1], pq[2], pq[3]);
            nfe[at] = make_float2(fc, __int_as_float(ej));
            if (FORCE) {
                ndp[at] = make_float4(dq[0], dq[1], dq[2], dq[3]);
                // radial part of g_ij: sum over radial descriptors of dE/dG * dG/dr * d/r
                float gr = 0.f;
                for (int rr = 0; rr < E.n_rad; ++rr) {
                    const int el = E.rad_elem[rr];
                    if (el < 0 || el == ej) {
                        const float x = r - E.rad_rs[rr];
                        const float ex = gauss2(E.rad_khi[rr], E.rad_klo[rr], x * x);
                        gr += sW[E.rad_out[rr]] * ex * (dfc - 2.0f * E.rad_eta[rr] * x * fc);
                    }
                }
                const float gs = gr / r;
                sg[3 * at + 0] = gs * dx;
                sg[3 * at + 1] = gs * dy;
                sg[3 * at + 2] = gs * dz;
            }
        }
        M += __popc(m);
    }
    if (M > cap) {
        if (lane == 0) atomicOr(&flags[FLAG_ERR], ERR_RC_OVERFLOW);
        M = cap;
    }
    __syncwarp();
    return M;
}

// advance a lane's flattened pair (j, k), j < k < M, by 'step' pairs
__device__ __forceinline__ void pair_normalize(int& j, int& k, int M)
{
    while (j < M - 1 && k >= M) {
        k = k - M + j + 2;
        ++j;
    }
}

// ---------------------------------------------------------------- value pass
template <int NETA, bool NARROW>
__global__ void __launch_bounds__(256)
k_sf(int n, const float4* __restrict__ pos4, Box bx, NbView nv, const Plan* __restrict__ plan_g,
     int cap, float* __restrict__ Gs, float* __restrict__ Graw, int* __restrict__ flags,
     unsigned long long* __restrict__ counters)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Plan& P = *plan_g;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    // per-warp shared memory
    const size_t per = (size_t)cap * (16 + 16 + 8) + NNP_MAXG * 8;
    unsigned char* base = smem + per * wib;
    float4* nd = (float4*)base;
    float4* npf = nd + cap;
    float2* nfe = (float2*)(npf + cap);
    double* sG = (double*)(nfe + cap);   // cap is a multiple of 2: 8-byte aligned

    unsigned long long c_list = 0, c_rc = 0, c_pairs = 0, c_trip = 0;
    const int nw = gridDim.x * wpb;
    for (int i = blockIdx.x * wpb + wib; i < n; i += nw) {
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
        int n_list;
        const int M = stage_neighbors<NETA, false>(i, pi, bx, nv, pos4, P, E, khi, klo, etav, cap, nd, npf,
                                                   nullptr, nfe, nullptr, nullptr, nullptr, lane, flags, n_list);
        // radial: lane <-> descriptor, loop over neighbours (broadcast reads)
        for (int rr = lane; rr < E.n_rad; rr += 32) {
            const float kh = E.rad_khi[rr], kl = E.rad_klo[rr], rs = E.rad_rs[rr];
            const int el = E.rad_elem[rr];
            double acc = 0.0;   // radial sums feed G~ = (G - mu)/s with |mu/s| up to ~1e2
            for (int m = 0; m < M; ++m) {
                const float r = nd[m].w;
                const float2 fe = nfe[m];
                if (el < 0 || el == __float_as_int(fe.y)) {
                    const float x = r - rs;
                    acc += (double)(gauss2(kh, kl, x * x) * fe.x);
                }
            }
            sG[E.rad_out[rr]] = acc;
        }
        // angular
        long long live = 0;
        if (NETA > 0) {
            float acc[NETA > 0 ? NETA : 1][2][NNP_KMAX + 1];
#pragma unroll
            for (int q = 0; q < (NETA > 0 ? NETA : 1); ++q)
#pragma unroll
                for (int l = 0; l < 2; ++l)
#pragma unroll
                    for (int k = 0; k <= NNP_KMAX; ++k) acc[q][l][k] = 0.f;
            int j = 0, k = 1 + lane;
            pair_normalize(j, k, M);
            const int T = M * (M - 1) / 2;
            for (int b0 = 0; b0 < T; b0 += 32) {
                if (j < M - 1) {
                    const float4 a = nd[j], b = nd[k];
                    bool ok = true;
                    float fcd = 1.f, rd2 = 0.f;
                    if (NARROW) {
                        const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
                        rd2 = ex * ex + ey * ey + ez * ez;
                        ok = rd2 < P.rc2;
                        if (ok) {
                            float dfcd;
                            cutoff_fn_fast(sqrtf(rd2), P.hpi_rc, fcd, dfcd);
                        }
                    }
                    if (ok) {
                        ++live;
                        const float4 pa = npf[j], pb = npf[k];
                        const float pav[4] = {pa.x, pa.y, pa.z, pa.w}, pbv[4] = {pb.x, pb.y, pb.z, pb.w};
                        const float c = __fdividef(a.x * b.x + a.y * b.y + a.z * b.z, a.w * b.w);
                        float pw[2][NNP_KMAX + 1];
                        pw[0][0] = 1.f + c;
                        pw[1][0] = 1.f - c;
#pragma unroll
                        for (int kk = 1; kk <= NNP_KMAX; ++kk) {
                            pw[0][kk] = pw[0][kk - 1] * pw[0][kk - 1];
                            pw[1][kk] = pw[1][kk - 1] * pw[1][kk - 1];
                        }
#pragma unroll
                        for (int q = 0; q < NETA; ++q) {
                            float R = pav[q] * pbv[q];
                            if (NARROW) R *= gauss2(khi[q], klo[q], rd2) * fcd;
#pragma unroll
                            for (int l = 0; l < 2; ++l)
#pragma unroll
                                for (int kk = 0; kk <= NNP_KMAX; ++kk) acc[q][l][kk] = fmaf(pw[l][kk], R, acc[q][l][kk]);
                        }
                    }
                }
                k += 32;
                pair_normalize(j, k, M);
            }
#pragma unroll
            for (int q = 0; q < NETA; ++q)
#pragma unroll
                for (int l = 0; l < 2; ++l)
#pragma unroll
                    for (int kk = 0; kk <= NNP_KMAX; ++kk) {
                        // lane partials summed in FP64; prefactor 2^(1 - zeta), zeta = 2^kk
                        const double v = warp_sum_d((double)acc[q][l][kk]);
                        const int o = E.ang_out[q][l][kk];
                        if (lane == 0 && o >= 0) sG[o] = v * (double)exp2f((float)(1 - (1 << kk)));
                    }
            if (lane == 0) {
                c_pairs += (unsigned long long)T;
            }
        }
        __syncwarp();
        for (int s = lane; s < E.n_g; s += 32) {
            const double g = sG[s];
            Gs[(size_t)i * P.gs + s] = (float)((g - (double)E.mu[s]) * (double)E.inv_s[s]);
            if (Graw) Graw[(size_t)i * E.n_g + s] = (float)g;
        }
        __syncwarp();
        c_trip += (unsigned long long)live;   // per lane; reduced over the warp at the end
        if (lane == 0) {
            c_list += (unsigned long long)n_list;
            c_rc += (unsigned long long)M;
        }
    }
    // counters: one atomic per warp
    unsigned long long t = c_trip;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) {
        atomicAdd(&counters[CNT_LIST], c_list);
        atomicAdd(&counters[CNT_RC], c_rc);
        atomicAdd(&counters[CNT_PAIRS], c_pairs);
        atomicAdd(&counters[CNT_TRIPLETS], t);
    }
}

// ---------------------------------------------------------------- force pass
// g[i, slot] = dE_i/dd_ij for each list slot (0 outside the cutoff), Fown[i] =
// sum_j g_ij (the force on i from its own energy), per-warp virial partials.
template <int NETA, bool NARROW>
__global__ void __launch_bounds__(256)
k_force(int n, const float4* __restrict__ pos4, Box bx, NbView nv, const Plan* __restrict__ plan_g, int cap,
        const float* __restrict__ dEdG, float4* __restrict__ gbuf, float4* __restrict__ Fown,
        double* __restrict__ vir_part, int* __restrict__ flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Plan& P = *plan_g;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const size_t per = (size_t)cap * (16 + 16 + 16 + 8 + 12) + (size_t)nv.stride * 4 + NNP_MAXG * 4;
    unsigned char* base = smem + per * wib;
    float4* nd = (float4*)base;
    float4* npf = nd + cap;
    float4* ndp = npf + cap;
    float2* nfe = (float2*)(ndp + cap);
    float* sg = (float*)(nfe + cap);
    int* cmap = (int*)(sg + 3 * cap);
    float* sW = (float*)(cmap + nv.stride);

    double vir[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) vir[q] = 0.0;
    const int nw = gridDim.x * wpb;
    for (int i = blockIdx.x * wpb + wib; i < n; i += nw) {
        const float4 pi = pos4[i];
        const int ti = __float_as_int(pi.w);
        const ElemPlan& E = P.e[ti];
        for (int s = lane; s < E.n_g; s += 32) sW[s] = dEdG[(size_t)i * P.gs + s];
        __syncwarp();
        float khi[4], klo[4], etav[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            etav[q] = (q < E.n_eta) ? E.ang_eta[q] : 0.f;
            khi[q] = (q < E.n_eta) ? E.ang_khi[q] : 0.f;
            klo[q] = (q < E.n_eta) ? E.ang_klo[q] : 0.f;
        }
        int n_list;
        const int M = stage_neighbors<NETA, true>(i, pi, bx, nv, pos4, P, E, khi, klo, etav, cap, nd, npf, ndp, nfe,
                                                  cmap, sg, sW, lane, flags, n_list);
        if (NETA > 0) {
            // dense weights W[q][l][k] = dE/dG_o * 2^(1-zeta); Wd = W * lambda * zeta
            float W[NETA > 0 ? NETA : 1][2][NNP_KMAX + 1], Wd[NETA > 0 ? NETA : 1][2][NNP_KMAX + 1];
#pragma unroll
            for (int q = 0; q < (NETA > 0 ? NETA : 1); ++q)
#pragma unroll
                for (int l = 0; l < 2; ++l)
#pragma unroll
                    for (int kk = 0; kk <= NNP_KMAX; ++kk) {
                        const int o = (q < E.n_eta) ? E.ang_out[q][l][kk] : -1;
                        const float w = (o >= 0) ? sW[o] * exp2f((float)(1 - (1 << kk))) : 0.f;
                        W[q][l][kk] = w;
                        Wd[q][l][kk] = w * (l == 0 ? 1.f : -1.f) * (float)(1 << kk);
                    }
            int j = 0, k = 1 + lane;
            pair_normalize(j, k, M);
            const int T = M * (M - 1) / 2;
            for (int b0 = 0; b0 < T; b0 += 32) {
                if (j < M - 1) {
                    const float4 a = nd[j], b = nd[k];
                    const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
                    bool ok = true;
                    float fcd = 1.f, dfcd = 0.f, rd2 = 0.f, rd = 1.f;
                    if (NARROW) {
                        rd2 = ex * ex + ey * ey + ez * ez;
                        ok = rd2 < P.rc2;
                        if (ok) {
                            rd = sqrtf(rd2);
                            cutoff_fn_fast(rd, P.hpi_rc, fcd, dfcd);
                        }
                    }
                    if (ok) {
                        const float4 pa = npf[j], pb = npf[k], qa = ndp[j], qb = ndp[k];
                        const float pav[4] = {pa.x, pa.y, pa.z, pa.w}, pbv[4] = {pb.x, pb.y, pb.z, pb.w};
                        const float qav[4] = {qa.x, qa.y, qa.z, qa.w}, qbv[4] = {qb.x, qb.y, qb.z, qb.w};
                        const float inv_a = __frcp_rn(a.w), inv_b = __frcp_rn(b.w);
                        const float c = (a.x * b.x + a.y * b.y + a.z * b.z) * inv_a * inv_b;
                        // p[l][k] = b_l^(2^k), qq[l][k] = b_l^(2^k - 1), b_l = 1 +- c
                        float pw[2][NNP_KMAX + 1], qw[2][NNP_KMAX + 1];
#pragma unroll
                        for (int l = 0; l < 2; ++l) {
                            const float bl = (l == 0) ? 1.f + c : 1.f - c;
                            qw[l][0] = 1.f;
                            pw[l][0] = bl;
#pragma unroll
                            for (int kk = 1; kk <= NNP_KMAX; ++kk) {
                                qw[l][kk] = qw[l][kk - 1] * pw[l][kk - 1];
                                pw[l][kk] = pw[l][kk - 1] * pw[l][kk - 1];
                            }
                        }
                        float phic = 0.f, phia = 0.f, phib = 0.f, phid = 0.f;
#pragma unroll
                        for (int q = 0; q < NETA; ++q) {
                            float S = 0.f, D = 0.f;
#pragma unroll
                            for (int l = 0; l < 2; ++l)
#pragma unroll
                                for (int kk = 0; kk <= NNP_KMAX; ++kk) {
                                    S = fmaf(W[q][l][kk], pw[l][kk], S);
                                    D = fmaf(Wd[q][l][kk], qw[l][kk], D);
                                }
                            float Pd = 1.f, dPd = 0.f;
                            if (NARROW) {
                                const float ed = gauss2(khi[q], klo[q], rd2);
                                Pd = ed * fcd;
                                dPd = ed * (dfcd - 2.0f * etav[q] * rd * fcd);
                            }
                            const float pab = pav[q] * pbv[q];
                            phic = fmaf(D, pab * Pd, phic);
                            const float SPd = S * Pd;
                            phia = fmaf(SPd * qav[q], pbv[q], phia);
                            phib = fmaf(SPd * pav[q], qbv[q], phib);
                            if (NARROW) phid = fmaf(S * pab, dPd, phid);
                        }
                        // g_a = phic (b/(ra rb) - c a/ra^2) + phia a/ra - phid (b - a)/rd
                        // g_b = phic (a/(ra rb) - c b/rb^2) + phib b/rb + phid (b - a)/rd
                        const float cab = phic * inv_a * inv_b;
                        const float ca = phia * inv_a - phic * c * inv_a * inv_a;
                        const float cb = phib * inv_b - phic * c * inv_b * inv_b;
                        const float cd = NARROW ? phid / rd : 0.f;
                        atomicAdd(&sg[3 * j + 0], ca * a.x + cab * b.x - cd * ex);
                        atomicAdd(&sg[3 * j + 1], ca * a.y + cab * b.y - cd * ey);
                        atomicAdd(&sg[3 * j + 2], ca * a.z + cab * b.z - cd * ez);
                        atomicAdd(&sg[3 * k + 0], cb * b.x + cab * a.x + cd * ex);
                        atomicAdd(&sg[3 * k + 1], cb * b.y + cab * a.y + cd * ey);
                        atomicAdd(&sg[3 * k + 2], cb * b.z + cab * a.z + cd * ez);
                    }
                }
                k += 32;
                pair_normalize(j, k, M);
            }
        }
        __syncwarp();
        // write g per list slot, own force and virial
        const int cnt = n_list;
        float4* grow = gbuf + (size_t)i * nv.stride;
        for (int s = lane; s < cnt; s += 32) {
            const int c = cmap[s];
            grow[s] = (c >= 0) ? make_float4(sg[3 * c], sg[3 * c + 1], sg[3 * c + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float fx = 0.f, fy = 0.f, fz = 0.f, v[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = 0.f;
        for (int m = lane; m < M; m += 32) {
            const float4 d = nd[m];
            const float gx = sg[3 * m], gy = sg[3 * m + 1], gz = sg[3 * m + 2];
            fx += gx; fy += gy; fz += gz;
            v[0] -= d.x * gx; v[1] -= d.x * gy; v[2] -= d.x * gz;
            v[3] -= d.y * gx; v[4] -= d.y * gy; v[5] -= d.y * gz;
            v[6] -= d.z * gx; v[7] -= d.z * gy; v[8] -= d.z * gz;
        }
        fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
#pragma unroll
        for (int q = 0; q < 9; ++q) vir[q] += (double)warp_sum(v[q]);
        if (lane == 0) Fown[i] = make_float4(fx, fy, fz, 0.f);
        __syncwarp();
    }
    if (lane == 0) {
        const int gw = blockIdx.x * wpb + wib;
#pragma unroll
        for (int q = 0; q < 9; ++q) vir_part[(size_t)gw * 9 + q] = vir[q];
    }
}

// F_m = Fown_m - sum_s g[nbr(m, s), rev(m, s)]   (no atomics, fixed order)
__global__ void k_gather(int n, NbView nv, const int* __restrict__ rev, const float4* __restrict__ gbuf,
                         const float4* __restrict__ Fown, float* __restrict__ F, int* __restrict__ flags)
{
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); m < n; m += nw) {
        const int cnt = nv.ncount[m];
        const uint32_t* row = nv.nbr + (size_t)m * nv.stride;
        const int* rrow = rev + (size_t)m * nv.stride;
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (int s = lane; s < cnt; s += 32) {
            const int j = (int)(row[s] & NB_INDEX_MASK);
            const float4 g = gbuf[(size_t)j * nv.stride + rrow[s]];
            sx += g.x; sy += g.y; sz += g.z;
        }
        sx = warp_sum(sx); sy = warp_sum(sy); sz = warp_sum(sz);
        if (lane == 0) {
            const float4 o = Fown[m];
            const float fx = o.x - sx, fy = o.y - sy, fz = o.z - sz;
            if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
            F[3 * m] = fx; F[3 * m + 1] = fy; F[3 * m + 2] = fz;
        }
    }
}
