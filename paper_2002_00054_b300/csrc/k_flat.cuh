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

// ---------------------------------------------------------------- CTA per cell
// The third mapping of the ablation: one CTA per cell of the cell binning.  The
// CTA copies the atoms of the cell's 27-cell stencil (positions shifted to the
// cell's periodic frame) into shared memory once; each of its warps then takes
// an atom of the cell, finds the atom's neighbours inside the cutoff in that
// copy (no Verlet list), and walks all neighbour pairs j < k with its lanes.
// Raw G, plain FP32 sums, the same formulas as k_sf_flat.  Shared memory:
// CELL_STENCIL_CAP stencil atoms, then per warp CELL_NB_CAP staged neighbours.
#define CELL_STENCIL_CAP 2048
#define CELL_NB_CAP 256
__host__ __device__ inline size_t sf_cell_smem_bytes(int warps)
{
    return (size_t)CELL_STENCIL_CAP * 16 + (size_t)warps * CELL_NB_CAP * (16 + 8);
}

__global__ void __launch_bounds__(128)
k_sf_cell(int ncx, int ncy, int ncz, const float4* __restrict__ pos4, Box bx, const int* __restrict__ cell_start,
          const int* __restrict__ cell_atoms, const Plan* __restrict__ plan_g, float* __restrict__ Graw,
          int* __restrict__ flags)
{
    extern __shared__ __align__(16) unsigned char smem_cell[];
    const Plan& P = *plan_g;
    float4* st = reinterpret_cast<float4*>(smem_cell);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float4* nd = reinterpret_cast<float4*>(smem_cell + (size_t)CELL_STENCIL_CAP * 16) + (size_t)wib * CELL_NB_CAP;
    float2* nfe = reinterpret_cast<float2*>(smem_cell + (size_t)CELL_STENCIL_CAP * 16 + (size_t)wpb * CELL_NB_CAP * 16) +
                  (size_t)wib * CELL_NB_CAP;
    __shared__ int s_beg[27], s_cnt[27], s_pre[28];
    __shared__ float s_sh[27][3];
    const bool narrow = P.ang_kind == NNP_SF_ANG_NARROW;
    const int ncell = ncx * ncy * ncz;
    for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
        if (threadIdx.x < 27) {
            const int t = threadIdx.x;
            int x = cx + t % 3 - 1, y = cy + (t / 3) % 3 - 1, z = cz + t / 9 - 1;
            float sx = 0.f, sy = 0.f, sz = 0.f;
            if (x < 0) { x += ncx; sx = -bx.L[0]; } else if (x >= ncx) { x -= ncx; sx = bx.L[0]; }
            if (y < 0) { y += ncy; sy = -bx.L[1]; } else if (y >= ncy) { y -= ncy; sy = bx.L[1]; }
            if (z < 0) { z += ncz; sz = -bx.L[2]; } else if (z >= ncz) { z -= ncz; sz = bx.L[2]; }
            const int cc = (z * ncy + y) * ncx + x;
            s_beg[t] = cell_start[cc];
            s_cnt[t] = cell_start[cc + 1] - cell_start[cc];
            s_sh[t][0] = sx; s_sh[t][1] = sy; s_sh[t][2] = sz;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int a = 0;
            for (int t = 0; t < 27; ++t) { s_pre[t] = a; a += s_cnt[t]; }
            s_pre[27] = a;
        }
        __syncthreads();
        const int total = s_pre[27];
        if (total > CELL_STENCIL_CAP) {   // denser than this ablation kernel holds: reported, cell skipped
            if (threadIdx.x == 0) atomicOr(&flags[FLAG_ERR], ERR_CELL_OVERFLOW);
            __syncthreads();
            continue;
        }
        for (int t = wib; t < 27; t += wpb)
            for (int k = lane; k < s_cnt[t]; k += 32) {
                float4 p = pos4[cell_atoms[s_beg[t] + k]];
                p.x += s_sh[t][0]; p.y += s_sh[t][1]; p.z += s_sh[t][2];
                st[s_pre[t] + k] = p;
            }
        __syncthreads();
        // the centre cell is stencil cell 13 (unshifted)
        for (int a = wib; a < s_cnt[13]; a += wpb) {
            const int i = cell_atoms[s_beg[13] + a];
            const float4 pi = pos4[i];
            const ElemPlan& E = P.e[__float_as_int(pi.w)];
            // neighbours inside the cutoff, compacted from the stencil copy
            int M = 0;
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int q = q0 + lane;
                bool keep = false;
                float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
                int ej = 0;
                if (q < total) {
                    const float4 pj = st[q];
                    dx = pj.x - pi.x; dy = pj.y - pi.y; dz = pj.z - pi.z;
                    r2 = dist2_fma(dx, dy, dz);
                    ej = __float_as_int(pj.w);
                    keep = r2 > 0.f && r2 < P.rc2;
                }
                const unsigned m = __ballot_sync(FULL, keep);
                const int at = M + __popc(m & ((1u << lane) - 1u));
                if (keep && at < CELL_NB_CAP) {
                    const float r = sqrtf(r2);
                    float fc, dfc;
                    cutoff_fn(r, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, fc, dfc);
                    nd[at] = make_float4(dx, dy, dz, r);
                    nfe[at] = make_float2(fc, __int_as_float(ej));
                }
                M += __popc(m);
            }
            if (M > CELL_NB_CAP) {
                if (lane == 0) atomicOr(&flags[FLAG_ERR], ERR_NEIGH_OVERFLOW);
                __syncwarp();
                continue;
            }
            __syncwarp();
            float g[NNP_MAXG];
            for (int s = 0; s < E.n_g; ++s) g[s] = 0.f;
            // radial: lanes over neighbours
            for (int m = lane; m < M; m += 32) {
                const float4 d = nd[m];
                const float2 fe = nfe[m];
                const int ej = __float_as_int(fe.y);
                for (int rr = 0; rr < E.n_rad; ++rr)
                    if (E.rad_elem[rr] < 0 || E.rad_elem[rr] == ej) {
                        const float x = d.w - E.rad_rs[rr];
                        g[E.rad_out[rr]] += gauss2_acc(E.rad_khi[rr], E.rad_klo[rr], x * x) * fe.x;
                    }
            }
            // angular: lanes over the pairs j < k, pair index p = k (k - 1) / 2 + j
            const int npair = M * (M - 1) / 2;
            for (int p = lane; E.n_eta > 0 && p < npair; p += 32) {
                int k = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
                while (k * (k - 1) / 2 > p) --k;
                while ((k + 1) * k / 2 <= p) ++k;
                const int j = p - k * (k - 1) / 2;
                const float4 a = nd[j], b = nd[k];
                const float fa = nfe[j].x, fb = nfe[k].x;
                float fcd = 1.f, rd2 = 0.f;
                if (narrow) {
                    const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
                    rd2 = ex * ex + ey * ey + ez * ez;
                    if (!(rd2 < P.rc2)) continue;
                    float dfcd;
                    cutoff_fn_fast(rd2 * rsqrtf(rd2), P.hpi_rc, fcd, dfcd);
                }
                const float c = (a.x * b.x + a.y * b.y + a.z * b.z) / (a.w * b.w);
                for (int q = 0; q < E.n_eta; ++q) {
                    const float Pq = gauss2(E.ang_khi[q], E.ang_klo[q], a.w * a.w + b.w * b.w + rd2) * fa * fb * fcd;
                    for (int l = 0; l < 2; ++l) {
                        float pw = 1.f + (l == 0 ? c : -c);
                        for (int kk = 0; kk <= NNP_KMAX; ++kk) {
                            const int o = E.ang_out[0][q][l][kk];
                            if (o >= 0) g[o] += pw * Pq * exp2f((float)(1 - (1 << kk)));
                            pw *= pw;
                        }
                    }
                }
            }
            for (int s = 0; s < E.n_g; ++s) {
                const float v = warp_sum(g[s]);
                if (lane == 0) {
                    if (!isfinite(v)) atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
                    Graw[(size_t)i * E.n_g + s] = v;
                }
            }
            __syncwarp();
        }
        __syncthreads();
    }
}
