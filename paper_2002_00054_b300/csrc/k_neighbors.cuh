// k_neighbors.cuh -- neighbour-list maintenance: cell binning and a full Verlet list.
//
// The paper keeps a Cabana neighbour list (Sec. 3.2) and notes that random
// neighbour access dominates (Sec. 4.3).  Here: a full (both directions) Verlet
// list within cutoff + skin, one fixed-stride row per atom, entries packing the
// neighbour index and its periodic image, plus a reverse index rev[e] = slot of
// the mirrored entry so forces can be gathered without atomics.
//
// Positions inside the library are pos4 = pos - off, where off is a multiple of
// the box fixed at the last rebuild (atoms are never wrapped in the caller's
// buffer).  Every kernel of a rebuild returns at once unless flags[FLAG_REBUILD]
// is set, so the whole sequence is enqueued without a host round trip.
#pragma once
#include "common.cuh"

// pos4 = pos - off (old offsets); flags a rebuild if any atom moved more than skin/2.
__global__ void k_check_disp(int n, const float* __restrict__ pos, const int* __restrict__ types, int n_elem,
                             const float4* __restrict__ off, const float4* __restrict__ ref,
                             float4* __restrict__ pos4, float half_skin2, int* __restrict__ flags)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 o = off[i];
    float x = pos[3 * i] - o.x, y = pos[3 * i + 1] - o.y, z = pos[3 * i + 2] - o.z;
    int t = types[i];
    if (t < 0 || t >= n_elem) {   // invalid element: reported, and never used as an index
        atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
        t = 0;
    }
    pos4[i] = make_float4(x, y, z, __int_as_float(t));
    float4 r = ref[i];
    float dx = x - r.x, dy = y - r.y, dz = z - r.z;
    float d2 = dx * dx + dy * dy + dz * dz;
    if (!(d2 <= half_skin2)) flags[FLAG_REBUILD] = 1;   // also catches NaN
}

// On rebuild: new offsets off = floor(pos / L) L, pos4 = pos - off in [0, L), ref = pos4.
__global__ void k_rebuild_pos(int n, const float* __restrict__ pos, const int* __restrict__ types, Box box,
                              int n_elem, float4* __restrict__ off, float4* __restrict__ pos4,
                              float4* __restrict__ ref, int* __restrict__ flags,
                              unsigned long long* __restrict__ counters,
                              const int* __restrict__ sys_of = nullptr, const float4* __restrict__ sys_box = nullptr)
{
    if (!flags[FLAG_REBUILD]) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) counters[CNT_REBUILDS] += 1ull;
    if (i >= n) return;
    float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    int t = types[i];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
        atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
        x = y = z = 0.0f;
    }
    if (t < 0 || t >= n_elem) {
        atomicOr(&flags[FLAG_ERR], ERR_NONFINITE);
        t = 0;
    }
    if (sys_of) {
        const float4 b = sys_box[sys_of[i]];
        box.L[0] = b.x; box.L[1] = b.y; box.L[2] = b.z;
    }
    float ox = floorf(x / box.L[0]) * box.L[0];
    float oy = floorf(y / box.L[1]) * box.L[1];
    float oz = floorf(z / box.L[2]) * box.L[2];
    off[i] = make_float4(ox, oy, oz, 0.0f);
    float4 p = make_float4(x - ox, y - oy, z - oz, __int_as_float(t));
    pos4[i] = p;
    ref[i] = p;
}

__device__ __forceinline__ int cell_coord(float x, float L, int nc)
{
    int c = (int)floorf(x / L * (float)nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_count(int n, const float4* __restrict__ pos4, Box box, int ncx, int ncy, int ncz,
                             int* __restrict__ cell_of, int* __restrict__ cell_count, const int* __restrict__ flags)
{
    if (!flags[FLAG_REBUILD]) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = pos4[i];
    int c = (cell_coord(p.z, box.L[2], ncz) * ncy + cell_coord(p.y, box.L[1], ncy)) * ncx + cell_coord(p.x, box.L[0], ncx);
    cell_of[i] = c;
    atomicAdd(&cell_count[c], 1);
}

// Exclusive scan of the cell counts by one block; cell_start[ncell] = n.  cursor = start.
__global__ void k_cell_scan(int ncell, const int* __restrict__ cell_count, int* __restrict__ cell_start,
                            int* __restrict__ cursor, const int* __restrict__ flags)
{
    if (!flags[FLAG_REBUILD]) return;
    __shared__ int part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int per = (ncell + nt - 1) / nt;
    const int lo = t * per, hi = min(lo + per, ncell);
    int s = 0;
    for (int c = lo; c < hi; ++c) s += cell_count[c];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < nt; o <<= 1) {   // Hillis-Steele inclusive scan of the partial sums
        int v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = (t > 0) ? part[t - 1] : 0;
    for (int c = lo; c < hi; ++c) {
        cell_start[c] = run;
        cursor[c] = run;
        run += cell_count[c];
    }
    if (t == nt - 1) cell_start[ncell] = part[nt - 1];
}

__global__ void k_cell_fill(int n, const int* __restrict__ cell_of, int* __restrict__ cursor,
                            int* __restrict__ cell_atoms, const int* __restrict__ flags)
{
    if (!flags[FLAG_REBUILD]) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int slot = atomicAdd(&cursor[cell_of[i]], 1);
    cell_atoms[slot] = i;
}

// Deterministic order inside each cell (ascending atom index): warp per cell, rank
// sort; the positions are written in the same order (cpos), so the row builder
// reads an atom's index and position with independent loads.
#define CELL_CAP 256
__global__ void k_cell_sort(int ncell, const int* __restrict__ cell_start, int* __restrict__ cell_atoms,
                            const float4* __restrict__ pos4, float4* __restrict__ cpos, int* __restrict__ flags)
{
    if (!flags[FLAG_REBUILD]) return;
    __shared__ int buf[8][CELL_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int c = blockIdx.x * (blockDim.x >> 5) + w; c < ncell; c += nw) {
        const int s0 = cell_start[c], cnt = cell_start[c + 1] - s0;
        if (cnt > CELL_CAP) {
            if (lane == 0) atomicOr(&flags[FLAG_ERR], ERR_CELL_OVERFLOW);
            continue;
        }
        for (int k = lane; k < cnt; k += 32) buf[w][k] = cell_atoms[s0 + k];
        __syncwarp();
        for (int k = lane; k < cnt; k += 32) {
            int v = buf[w][k], rank = 0;
            for (int q = 0; q < cnt; ++q) rank += (buf[w][q] < v);
            cell_atoms[s0 + rank] = v;
            cpos[s0 + rank] = pos4[v];
        }
        __syncwarp();
    }
}

// |d|^2 of a list candidate with explicit roundings: both row builders take the
// same decisions, and d_ji = -d_ij (pair_disp) gives symmetric rows.
__device__ __forceinline__ float dist2_list(float dx, float dy, float dz) { return fmaf(dz, dz, fmaf(dy, dy, dx * dx)); }

// Row of atom i from the 27-cell stencil (cells of edge >= cutoff + skin, >= 3 per side).
// Entry order: stencil order (z, y, x from -1 to 1), then ascending atom index.
// seg[i][t] (t = 0..26, stencil cell t = (dz+1)*9 + (dy+1)*3 + (dx+1)) is the
// first slot of row i that came from stencil cell t; seg[i][27] = the row length.
#define NB_SEG 28
__global__ void k_rows_cell(int n, const float4* __restrict__ pos4, Box box, int ncx, int ncy, int ncz,
                            const int* __restrict__ cell_start, const int* __restrict__ cell_atoms,
                            const float4* __restrict__ cpos,
                            float rcut2, int stride, uint32_t* __restrict__ nbr, int* __restrict__ ncount,
                            unsigned short* __restrict__ seg, int* __restrict__ flags, const int* __restrict__ only)
{
    if (!flags[FLAG_REBUILD]) return;
    // per warp: how many stencil cells start at each position of the current round
    __shared__ int hist[8][32];   // blockDim.x <= 256
    const int lane = threadIdx.x & 31;
    int* hc = hist[threadIdx.x >> 5];
    const int nw = gridDim.x * (blockDim.x >> 5);
    // only (not nullptr): the atoms only[1 .. only[0]] (those k_rows_blk left), else all
    const int n_items = only ? only[0] : n;
    for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < n_items; it += nw) {
        const int i = only ? only[1 + it] : it;
        const float4 pi = pos4[i];
        const int cx = cell_coord(pi.x, box.L[0], ncx), cy = cell_coord(pi.y, box.L[1], ncy),
                  cz = cell_coord(pi.z, box.L[2], ncz);
        // lane t < 27: stencil cell t = (dz+1)*9 + (dy+1)*3 + (dx+1), its atom range
        // and periodic shift; then an exclusive scan of the cell sizes
        int b0 = 0, len = 0, code = 62;   // code of shift (0, 0, 0)
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (lane < 27) {
            const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
            int x = cx + dx, y = cy + dy, z = cz + dz, sx = 0, sy = 0, sz = 0;
            if (x < 0) { x += ncx; sx = -1; } else if (x >= ncx) { x -= ncx; sx = 1; }
            if (y < 0) { y += ncy; sy = -1; } else if (y >= ncy) { y -= ncy; sy = 1; }
            if (z < 0) { z += ncz; sz = -1; } else if (z >= ncz) { z -= ncz; sz = 1; }
            const int c = (z * ncy + y) * ncx + x;
            b0 = cell_start[c];
            len = cell_start[c + 1] - b0;
            code = (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2);
            ox = (float)sx * box.L[0];
            oy = (float)sy * box.L[1];
            oz = (float)sz * box.L[2];
        }
        int pre = len;   // inclusive scan over lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, pre, o);
            if (lane >= o) pre += t;
        }
        const int total = __shfl_sync(FULL, pre, 31);
        pre -= len;   // first flat candidate index of cell `lane`
        // candidates of all 27 cells in stencil order, 32 per round
        int cnt = 0, my_seg = 0;
        int c_before = 0;   // stencil cells u >= 1 whose first index lies before the round
        for (int f0 = 0; f0 < total; f0 += 32) {
            const int f = f0 + lane;
            // cell of candidate f: the number of cells u >= 1 with first index <= f
            // (first indices do not decrease with u), from a count of the cells
            // starting at each position of the round and an inclusive scan
            hc[lane] = 0;
            __syncwarp();
            if (lane >= 1 && lane < 27 && pre >= f0 && pre < f0 + 32) atomicAdd(&hc[pre - f0], 1);
            __syncwarp();
            int cum = hc[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, cum, o);
                if (lane >= o) cum += v;
            }
            const int t = c_before + cum;
            c_before += __shfl_sync(FULL, cum, 31);
            const int tb0 = __shfl_sync(FULL, b0, t), tpre = __shfl_sync(FULL, pre, t);
            const int tcode = __shfl_sync(FULL, code, t);
            const float tox = __shfl_sync(FULL, ox, t), toy = __shfl_sync(FULL, oy, t), toz = __shfl_sync(FULL, oz, t);
            bool keep = false;
            int j = 0;
            if (f < total) {
                j = cell_atoms[tb0 + (f - tpre)];
                const float4 pj = cpos[tb0 + (f - tpre)];
                const float ddx = pair_disp(pj.x, pi.x, tox), ddy = pair_disp(pj.y, pi.y, toy),
                            ddz = pair_disp(pj.z, pi.z, toz);
                const float r2 = dist2_list(ddx, ddy, ddz);
                keep = (r2 < rcut2) && !(j == i && tcode == 62);
            }
            const unsigned m = __ballot_sync(FULL, keep);
            // segment start of cell `lane` (its first candidate falls in this round)
            if (lane < 27 && pre >= f0 && pre < f0 + 32) my_seg = cnt + __popc(m & ((1u << (pre - f0)) - 1u));
            const int at = cnt + __popc(m & ((1u << lane) - 1u));
            if (keep && at < stride) nbr[(size_t)i * stride + at] = (uint32_t)j | ((uint32_t)tcode << 24);
            cnt += __popc(m);
        }
        if (lane < 27 && pre >= total) my_seg = cnt;   // empty trailing cells
        if (lane < 27) seg[(size_t)i * NB_SEG + lane] = (unsigned short)min(my_seg, stride);
        if (lane == 0) {
            if (cnt > stride) atomicOr(&flags[FLAG_ERR], ERR_NEIGH_OVERFLOW);
            ncount[i] = min(cnt, stride);
            seg[(size_t)i * NB_SEG + 27] = (unsigned short)min(cnt, stride);
        }
    }
}

// Rows of the cell path, one block per cell: the atoms of the 27 stencil cells are
// staged once in shared memory (position and list entry j | image code << 24, and
// the image shift), and each atom of the centre cell (a warp per atom) takes its
// row from there: the candidates in stencil order, ascending index within a cell,
// the displacement by pair_disp and the distance by dist2_list, so the rows, their
// order and the stencil segments are those of k_rows_cell; no per-candidate cell
// search and no global loads in the candidate loop.  A cell whose stencil holds
// more than ROWS_SMAX atoms queues its own atoms in rest (count, then indices)
// for k_rows_cell.
#define ROWS_SMAX 1280
__host__ __device__ inline size_t rows_blk_smem_bytes() { return (size_t)ROWS_SMAX * 2 * sizeof(float4); }
__global__ void __launch_bounds__(128) k_rows_blk(int ncell, Box box, int ncx, int ncy, int ncz,
                                                  const int* __restrict__ cell_start, const int* __restrict__ cell_atoms,
                                                  const float4* __restrict__ cpos, float rcut2, int stride,
                                                  uint32_t* __restrict__ nbr, int* __restrict__ ncount,
                                                  unsigned short* __restrict__ seg, int* __restrict__ rest,
                                                  int* __restrict__ flags)
{
    if (!flags[FLAG_REBUILD]) return;
    extern __shared__ __align__(16) unsigned char rows_smem[];
    float4* srec = reinterpret_cast<float4*>(rows_smem);   // (x, y, z, entry)
    float4* ssh = srec + ROWS_SMAX;                          // image shift of the record
    __shared__ int s_b0[27], s_off[28], s_noshift;
    __shared__ float4 s_shift[27];   // (ox, oy, oz, image code)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
        if (wid == 0) {
            // lane t < 27: stencil cell t = (dz+1)*9 + (dy+1)*3 + (dx+1), its atom range
            // and periodic shift; an exclusive scan of the cell sizes gives the offsets
            const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
            int b0 = 0, len = 0, code = 62;
            float ox = 0.f, oy = 0.f, oz = 0.f;
            if (lane < 27) {
                const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
                int x = cx + dx, y = cy + dy, z = cz + dz, sx = 0, sy = 0, sz = 0;
                if (x < 0) { x += ncx; sx = -1; } else if (x >= ncx) { x -= ncx; sx = 1; }
                if (y < 0) { y += ncy; sy = -1; } else if (y >= ncy) { y -= ncy; sy = 1; }
                if (z < 0) { z += ncz; sz = -1; } else if (z >= ncz) { z -= ncz; sz = 1; }
                const int cn = (z * ncy + y) * ncx + x;
                b0 = cell_start[cn];
                len = cell_start[cn + 1] - b0;
                code = (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2);
                ox = (float)sx * box.L[0];
                oy = (float)sy * box.L[1];
                oz = (float)sz * box.L[2];
            }
            int pre = len;   // inclusive scan over lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, pre, o);
                if (lane >= o) pre += t;
            }
            if (lane < 27) {
                s_b0[lane] = b0;
                s_off[lane] = pre - len;
                s_shift[lane] = make_float4(ox, oy, oz, __int_as_float(code));
            }
            if (lane == 26) s_off[27] = pre;
            // every stencil cell at image shift (0, 0, 0): all but the cells at the box faces
            const unsigned ns = __ballot_sync(FULL, lane >= 27 || code == 62);
            if (lane == 0) s_noshift = (ns == FULL);
        }
        __syncthreads();
        const int total = s_off[27], c0 = s_off[13], c1 = s_off[14];   // stencil cell 13: the cell itself
        const bool noshift = s_noshift != 0;
        if (total > ROWS_SMAX) {
            for (int k = threadIdx.x; k < c1 - c0; k += blockDim.x) rest[1 + atomicAdd(rest, 1)] = cell_atoms[s_b0[13] + k];
            __syncthreads();
            continue;
        }
        for (int f = threadIdx.x; f < total; f += blockDim.x) {
            // stencil cell of record f: the last t with s_off[t] <= f (empty cells skipped)
            int lo = 0, hi = 26;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= f) lo = mid;
                else hi = mid - 1;
            }
            const int src = s_b0[lo] + (f - s_off[lo]);
            const float4 pj = cpos[src], sh = s_shift[lo];
            const uint32_t ent = (uint32_t)cell_atoms[src] | ((uint32_t)__float_as_int(sh.w) << 24);
            srec[f] = make_float4(pj.x, pj.y, pj.z, __uint_as_float(ent));
            ssh[f] = sh;
        }
        __syncthreads();
        const int my_pre = (lane < 27) ? s_off[lane] : 0;
        for (int k = c0 + wid; k < c1; k += nwb) {
            const float4 pi = srec[k];   // shift 0
            const uint32_t ei = __float_as_uint(pi.w);   // i | 62 << 24: i itself at shift 0
            const int i = (int)(ei & NB_INDEX_MASK);
            int cnt = 0, my_seg = 0;
            for (int f0 = 0; f0 < total; f0 += 32) {
                const int f = f0 + lane;
                bool keep = false;
                uint32_t ent = 0u;
                if (f < total) {
                    const float4 pj = srec[f];
                    float ddx, ddy, ddz;
                    if (noshift) {
                        // pair_disp with a zero shift returns pj - pi (TwoSum: t + e rounds to t)
                        ddx = pj.x - pi.x;
                        ddy = pj.y - pi.y;
                        ddz = pj.z - pi.z;
                    } else {
                        const float4 sh = ssh[f];
                        ddx = pair_disp(pj.x, pi.x, sh.x);
                        ddy = pair_disp(pj.y, pi.y, sh.y);
                        ddz = pair_disp(pj.z, pi.z, sh.z);
                    }
                    ent = __float_as_uint(pj.w);
                    keep = (dist2_list(ddx, ddy, ddz) < rcut2) && ent != ei;
                }
                const unsigned m = __ballot_sync(FULL, keep);
                // segment start of stencil cell `lane` (its first candidate falls in this round)
                if (lane < 27 && my_pre >= f0 && my_pre < f0 + 32) my_seg = cnt + __popc(m & ((1u << (my_pre - f0)) - 1u));
                const int at = cnt + __popc(m & ((1u << lane) - 1u));
                if (keep && at < stride) nbr[(size_t)i * stride + at] = ent;
                cnt += __popc(m);
            }
            if (lane < 27 && my_pre >= total) my_seg = cnt;   // empty trailing cells
            if (lane < 27) seg[(size_t)i * NB_SEG + lane] = (unsigned short)min(my_seg, stride);
            if (lane == 0) {
                if (cnt > stride) atomicOr(&flags[FLAG_ERR], ERR_NEIGH_OVERFLOW);
                ncount[i] = min(cnt, stride);
                seg[(size_t)i * NB_SEG + 27] = (unsigned short)min(cnt, stride);
            }
        }
        __syncthreads();
    }
}

// Reverse index of cell-built rows: if j came from stencil cell t of i's row,
// i is in stencil cell 26 - t of j's row (with the opposite image), among the
// few entries of that segment.  One lane per entry.
__global__ void k_rev_cell(int n, const uint32_t* __restrict__ nbr, const int* __restrict__ ncount, int stride,
                           const unsigned short* __restrict__ seg, int* __restrict__ rev, int* __restrict__ flags)
{
    if (!flags[FLAG_REBUILD]) return;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const int cnt = ncount[i];
        const uint32_t* row = nbr + (size_t)i * stride;
        const unsigned short* si = seg + (size_t)i * NB_SEG;
        const int my_seg = (lane < NB_SEG) ? (int)si[lane] : 0x7fffffff;
        for (int s0 = 0; s0 < cnt; s0 += 32) {
            const int s = s0 + lane;
            // stencil cell of slot s: the last t in 0..26 whose segment starts at or before s
            int t = 0;
#pragma unroll
            for (int u = 1; u < 27; ++u)
                if (__shfl_sync(FULL, my_seg, u) <= s) t = u;
            if (s < cnt) {
                const uint32_t e = row[s];
                const int j = (int)(e & NB_INDEX_MASK);
                const uint32_t target = nb_reverse(e, i);
                const unsigned short* sj = seg + (size_t)j * NB_SEG + (26 - t);
                const int lo = sj[0], hi = sj[1];
                const uint32_t* rj = nbr + (size_t)j * stride;
                int f = -1;
                for (int r0 = lo; r0 < hi && f < 0; r0 += 8) {
                    uint32_t v[8];   // independent loads (no entry equals 0xffffffff)
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = (r0 + u < hi) ? rj[r0 + u] : 0xffffffffu;
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (f < 0 && v[u] == target) f = r0 + u;
                }
                if (f < 0) atomicOr(&flags[FLAG_ERR], ERR_REV);
                rev[(size_t)i * stride + s] = f < 0 ? 0 : f;
            }
        }
    }
}

// Row of atom i by brute force over the atoms of its system and the images
// s in [-nimg, nimg]^3 (small boxes, several images of one atom possible).
// Entry order: 32-atom chunks in index order, then image, then atom index.
__global__ void k_rows_brute(int n, const float4* __restrict__ pos4, const int* __restrict__ sys_of,
                             const int* __restrict__ sys_start, const float4* __restrict__ sys_box,
                             float rcut2, int stride, uint32_t* __restrict__ nbr, int* __restrict__ ncount,
                             int* __restrict__ flags)
{
    if (!flags[FLAG_REBUILD]) return;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const int s = sys_of ? sys_of[i] : 0;
        const int j0 = sys_of ? sys_start[s] : 0, j1 = sys_of ? sys_start[s + 1] : n;
        const float4 bx = sys_box[s];   // x, y, z edges; w = image range (as float)
        const int nim = (int)bx.w;
        const float4 pi = pos4[i];
        int cnt = 0;
        for (int base = j0; base < j1; base += 32) {
            const int j = base + lane;
            const bool vj = j < j1;
            const float4 pj = vj ? pos4[j] : pi;
            for (int sx = -nim; sx <= nim; ++sx)
                for (int sy = -nim; sy <= nim; ++sy)
                    for (int sz = -nim; sz <= nim; ++sz) {
                        const float ddx = pair_disp(pj.x, pi.x, (float)sx * bx.x),
                                    ddy = pair_disp(pj.y, pi.y, (float)sy * bx.y),
                                    ddz = pair_disp(pj.z, pi.z, (float)sz * bx.z);
                        const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        const bool keep = vj && (r2 < rcut2) && !(j == i && sx == 0 && sy == 0 && sz == 0);
                        const unsigned m = __ballot_sync(FULL, keep);
                        const int at = cnt + __popc(m & ((1u << lane) - 1u));
                        if (keep && at < stride) nbr[(size_t)i * stride + at] = nb_pack(j, sx, sy, sz);
                        cnt += __popc(m);
                    }
        }
        if (lane == 0) {
            if (cnt > stride) atomicOr(&flags[FLAG_ERR], ERR_NEIGH_OVERFLOW);
            ncount[i] = min(cnt, stride);
        }
    }
}

// rev[i, s] = slot of the mirrored entry (i seen from j with the opposite image).
__global__ void k_rev(int n, const uint32_t* __restrict__ nbr, const int* __restrict__ ncount, int stride,
                      int* __restrict__ rev, int* __restrict__ flags)
{
    if (!flags[FLAG_REBUILD]) return;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const int cnt = ncount[i];
        const uint32_t* row = nbr + (size_t)i * stride;
        for (int s0 = 0; s0 < cnt; s0 += 32) {
            // each lane takes one entry of this chunk; the warp then searches row by row
            const int my = s0 + lane;
            const uint32_t e = (my < cnt) ? row[my] : 0u;
            int found = -1;
            const int m = min(32, cnt - s0);
            for (int q = 0; q < m; ++q) {
                const uint32_t eq = __shfl_sync(FULL, e, q);
                const int j = (int)(eq & NB_INDEX_MASK);
                const uint32_t target = nb_reverse(eq, i);
                const int cj = ncount[j];
                const uint32_t* rj = nbr + (size_t)j * stride;
                int f = -1;
                for (int b = 0; b < cj && f < 0; b += 32) {
                    const int t = b + lane;
                    const unsigned hit = __ballot_sync(FULL, t < cj && rj[t] == target);
                    if (hit) f = b + __ffs(hit) - 1;
                }
                if (lane == q) found = f;
            }
            if (my < cnt) {
                if (found < 0) atomicOr(&flags[FLAG_ERR], ERR_REV);
                rev[(size_t)i * stride + my] = found < 0 ? 0 : found;
            }
        }
    }
}
