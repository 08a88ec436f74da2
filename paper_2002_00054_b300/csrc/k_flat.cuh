// k_flat.cuh -- the two other levels of the paper's parallelism study (Sec. 4.3,
// Fig. 6), kept for the ablation against the warp-per-atom descriptor kernel:
//   k_sf_flat: one thread per atom ("flat": each thread walks its own
//     neighbours and neighbour pairs);
//   k_sf_pair: one thread per (atom, neighbour) ("hierarchical": threads over
//     atoms and neighbours; the thread for (i, j) adds the radial terms of j and
//     the angular terms of every pair (j, k) with k after j in i's list, then
//     adds its partial descriptors into G_i with atomic updates, the extra
//     atomics the paper names for this level).
// Raw G only, FP32 sums, the same cutoff and exponential forms as the
// production kernels; element-pair-resolved angular classes are not supported.
#pragma once
#include "k_descriptors.cuh"

__global__ void __launch_bounds__(128)
k_sf_flat(int n, const float4* __restrict__ pos4, Box bx, NbView nv, const Plan* __restrict__ plan_g,
          float* __restrict__ Graw, int* __restrict__ flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Plan& P = *plan_g;
    const float4 pi = pos4[i];
    const ElemPlan& E = P.e[__float_as_int(pi.w)];
    float g[NNP_MAXG];
    for (int s = 0; s < E.n_g; ++s) g[s] = 0.f;
    const int cnt = nv.ncount[i];
    const uint32_t* row = nv.nbr + (size_t)i * nv.stride;
    float Lx, Ly, Lz;
    atom_box(nv, bx, i, Lx, Ly, Lz);
    const bool narrow = P.ang_kind == NNP_SF_ANG_NARROW;
    auto disp = [&](uint32_t e, float& dx, float& dy, float& dz, int& ej) {
        const float4 pj = pos4[e & NB_INDEX_MASK];
        float ox, oy, oz;
        nb_shift(e, Lx, Ly, Lz, ox, oy, oz);
        dx = pair_disp(pj.x, pi.x, ox);
        dy = pair_disp(pj.y, pi.y, oy);
        dz = pair_disp(pj.z, pi.z, oz);
        ej = __float_as_int(pj.w);
        return dist2_fma(dx, dy, dz);
    };
    for (int s = 0; s < cnt; ++s) {
        float ax, ay, az;
        int ea;
        const float ra2 = disp(row[s], ax, ay, az, ea);
        if (!(ra2 < P.rc2)) continue;
        const float ra = sqrtf(ra2);
        float fa, dfa;
        cutoff_fn(ra, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, fa, dfa);
        for (int rr = 0; rr < E.n_rad; ++rr)
            if (E.rad_elem[rr] < 0 || E.rad_elem[rr] == ea) {
                const float x = ra - E.rad_rs[rr];
                g[E.rad_out[rr]] += gauss2_acc(E.rad_khi[rr], E.rad_klo[rr], x * x) * fa;
            }
        if (E.n_eta == 0) continue;
        const float ha = live_h(ra2, P.rc2);
        const float4 a = make_float4(ax, ay, az, 0.f);
        for (int s2 = s + 1; s2 < cnt; ++s2) {
            float bx_, by_, bz_;
            int eb;
            const float rb2 = disp(row[s2], bx_, by_, bz_, eb);
            if (!(rb2 < P.rc2)) continue;
            const float4 b = make_float4(bx_, by_, bz_, 0.f);
            float fcd = 1.f, rd2 = 0.f;
            if (narrow) {
                if (!live_pair(a, ha, b, live_h(rb2, P.rc2))) continue;
                const float ex = bx_ - ax, ey = by_ - ay, ez = bz_ - az;
                rd2 = ex * ex + ey * ey + ez * ez;
                float dfcd;
                cutoff_fn_fast(rd2 * rsqrtf(rd2), P.hpi_rc, fcd, dfcd);
            }
            const float rb = sqrtf(rb2);
            float fb, dfb;
            cutoff_fn(rb, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, fb, dfb);
            const float c = (ax * bx_ + ay * by_ + az * bz_) / (ra * rb);
            for (int q = 0; q < E.n_eta; ++q) {
                const float Pq = gauss2(E.ang_khi[q], E.ang_klo[q], ra2 + rb2 + rd2) * fa * fb * fcd;
                for (int l = 0; l < 2; ++l) {
                    float pw = 1.f + (l == 0 ? c : -c);
                    for (int kk = 0; kk <= NNP_KMAX; ++kk) {
                        const int o = E.ang_out[0][q][l][kk];
                        if (o >= 0) g[o] += pw * Pq;
                        pw *= pw;
                    }
                }
            }
        }
    }
    // angular prefactor 2^(1 - zeta)
    for (int q = 0; q < E.n_eta; ++q)
        for (int l = 0; l < 2; ++l)
            for (int kk = 0; kk <= NNP_KMAX; ++kk) {
                const int o = E.ang_out[0][q][l][kk];
                if (o >= 0) g[o] *= exp2f((float)(1 - (1 << kk)));
            }
    for (int s = 0; s < E.n_g; ++s) {
        if (!isfinite(g[s])) atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
        Graw[(size_t)i * E.n_g + s] = g[s];
    }
}

// Partial descriptors of atom i from the list slot a (its neighbour j): the
// radial terms of j and the angular terms of the pairs (j, k), k after j in the
// list; added into G_i (zeroed beforehand) with float atomics, so the sums'
// order depends on scheduling.  Grid-stride loop over n x stride slots.
__global__ void __launch_bounds__(128)
k_sf_pair(int n, const float4* __restrict__ pos4, Box bx, NbView nv, const Plan* __restrict__ plan_g,
          float* __restrict__ Graw, int* __restrict__ flags)
{
    const Plan& P = *plan_g;
    const bool narrow = P.ang_kind == NNP_SF_ANG_NARROW;
    const long long items = (long long)n * nv.stride;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(it / nv.stride), a_slot = (int)(it % nv.stride);
        const int cnt = nv.ncount[i];
        if (a_slot >= cnt) continue;
        const float4 pi = pos4[i];
        const ElemPlan& E = P.e[__float_as_int(pi.w)];
        const uint32_t* row = nv.nbr + (size_t)i * nv.stride;
        float Lx, Ly, Lz;
        atom_box(nv, bx, i, Lx, Ly, Lz);
        auto disp = [&](uint32_t e, float& dx, float& dy, float& dz, int& ej) {
            const float4 pj = pos4[e & NB_INDEX_MASK];
            float ox, oy, oz;
            nb_shift(e, Lx, Ly, Lz, ox, oy, oz);
            dx = pair_disp(pj.x, pi.x, ox);
            dy = pair_disp(pj.y, pi.y, oy);
            dz = pair_disp(pj.z, pi.z, oz);
            ej = __float_as_int(pj.w);
            return dist2_fma(dx, dy, dz);
        };
        float ax, ay, az;
        int ea;
        const float ra2 = disp(row[a_slot], ax, ay, az, ea);
        if (!(ra2 < P.rc2)) continue;
        float g[NNP_MAXG];
        for (int s = 0; s < E.n_g; ++s) g[s] = 0.f;
        const float ra = sqrtf(ra2);
        float fa, dfa;
        cutoff_fn(ra, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, fa, dfa);
        for (int rr = 0; rr < E.n_rad; ++rr)
            if (E.rad_elem[rr] < 0 || E.rad_elem[rr] == ea) {
                const float x = ra - E.rad_rs[rr];
                g[E.rad_out[rr]] += gauss2_acc(E.rad_khi[rr], E.rad_klo[rr], x * x) * fa;
            }
        if (E.n_eta > 0) {
            const float ha = live_h(ra2, P.rc2);
            const float4 a = make_float4(ax, ay, az, 0.f);
            for (int s2 = a_slot + 1; s2 < cnt; ++s2) {
                float bx_, by_, bz_;
                int eb;
                const float rb2 = disp(row[s2], bx_, by_, bz_, eb);
                if (!(rb2 < P.rc2)) continue;
                const float4 b = make_float4(bx_, by_, bz_, 0.f);
                float fcd = 1.f, rd2 = 0.f;
                if (narrow) {
                    if (!live_pair(a, ha, b, live_h(rb2, P.rc2))) continue;
                    const float ex = bx_ - ax, ey = by_ - ay, ez = bz_ - az;
                    rd2 = ex * ex + ey * ey + ez * ez;
                    float dfcd;
                    cutoff_fn_fast(rd2 * rsqrtf(rd2), P.hpi_rc, fcd, dfcd);
                }
                const float rb = sqrtf(rb2);
                float fb, dfb;
                cutoff_fn(rb, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, fb, dfb);
                const float c = (ax * bx_ + ay * by_ + az * bz_) / (ra * rb);
                for (int q = 0; q < E.n_eta; ++q) {
                    const float Pq = gauss2(E.ang_khi[q], E.ang_klo[q], ra2 + rb2 + rd2) * fa * fb * fcd;
                    for (int l = 0; l < 2; ++l) {
                        float pw = 1.f + (l == 0 ? c : -c);
                        for (int kk = 0; kk <= NNP_KMAX; ++kk) {
                            const int o = E.ang_out[0][q][l][kk];
                            if (o >= 0) g[o] += pw * Pq;
                            pw *= pw;
                        }
                    }
                }
            }
            // angular prefactor 2^(1 - zeta)
            for (int q = 0; q < E.n_eta; ++q)
                for (int l = 0; l < 2; ++l)
                    for (int kk = 0; kk <= NNP_KMAX; ++kk) {
                        const int o = E.ang_out[0][q][l][kk];
                        if (o >= 0) g[o] *= exp2f((float)(1 - (1 << kk)));
                    }
        }
        for (int s = 0; s < E.n_g; ++s) {
            if (!isfinite(g[s])) atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
            if (g[s] != 0.f) atomicAdd(&Graw[(size_t)i * E.n_g + s], g[s]);
        }
    }
}
