// k_mlp_tc.cuh -- the per-element networks (Fig. 1b step 2) on the 5th-generation
// tensor cores: BF16 operands, FP32 accumulation in tensor memory (TMEM).
//
// A CTA of 128 threads takes tiles of 128 atoms of one element (per-element
// atom lists, rebuilt every call).  Per tile, four M=128 GEMMs:
//   forward   A1 = X  W1^T,  h1 = tanh(A1 + b1)
//             A2 = h1 W2^T,  h2 = tanh(A2 + b2),  E = w3 . h2 + b3
//   backward  D3 = d2 W2,    d2 = w3 (1 - h2^2)
//             dX = d1 W1,    d1 = D3 (1 - h1^2)
// X is the scaled descriptor row G~ (K padded to a multiple of 16), dE/dG = dX / s.
// Thread t of the CTA owns TMEM lane t = atom t of the tile: it writes that
// atom's operand rows, and reads its accumulator row back with tcgen05.ld for the
// elementwise epilogue (bias, tanh, derivative).  One thread issues the MMAs;
// completion is signalled by tcgen05.commit on an mbarrier.  Every wait on the
// mbarrier is bounded: on timeout the kernel records ERR_TIMEOUT, frees its TMEM
// and returns.
//
// Shared-memory operands use the no-swizzle K-major canonical layout: 8x8 core
// matrices of 128 contiguous bytes (8 rows of 16 bytes); along K adjacent core
// matrices are LBO = 128 bytes apart, along M/N SBO = (K/8) * 128 bytes.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

#define TC_TILE 128
#define TC_TMEM_COLS 128

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (r, k) in a K-major canonical tile with K columns
__device__ __forceinline__ uint32_t cm_off(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, LBO, SBO (bytes, >> 4), version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, M = 128
__host__ __device__ constexpr uint32_t make_idesc(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_TILE >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok != 0;
}

// bounded wait (about one second of clock); false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try(mbar, parity)) {
        if (clock64() - t0 > 2000000000LL) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = __uint_as_float(r[t]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// writes 8 consecutive K-elements (one 16-byte core-matrix row) of row r
__device__ __forceinline__ void put8(unsigned char* tile, int r, int k0, int K, const float* v)
{
    uint4 q;
    q.x = pack_bf16(v[0], v[1]);
    q.y = pack_bf16(v[2], v[3]);
    q.z = pack_bf16(v[4], v[5]);
    q.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + cm_off(r, k0, K)) = q;
}

}  // namespace tc

// Per-element atom lists: count per element and block, then one scan, then a
// stable (atom order) fill.  elem_off[e] = first list index of element e,
// tile_off[e] = first tile of element e (tiles of 128 atoms).
__global__ void k_elem_count(int n, const float4* __restrict__ pos4, int n_elem, int* __restrict__ part)
{
    __shared__ int cnt[NNP_MAXE];
    if (threadIdx.x < NNP_MAXE) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[__float_as_int(pos4[i].w)], 1);
    __syncthreads();
    if (threadIdx.x < n_elem) part[blockIdx.x * NNP_MAXE + threadIdx.x] = cnt[threadIdx.x];
}

__global__ void k_elem_scan(int nblk, int n_elem, int* __restrict__ part, int* __restrict__ elem_off,
                            int* __restrict__ tile_off)
{
    // one block of 1024 threads; per element an exclusive scan over the block counts
    __shared__ int sp[1024];
    __shared__ int base, tiles;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) { base = 0; tiles = 0; }
    __syncthreads();
    const int per = (nblk + nt - 1) / nt;
    for (int e = 0; e < n_elem; ++e) {
        const int lo = t * per, hi = min(lo + per, nblk);
        int s = 0;
        for (int b = lo; b < hi; ++b) s += part[b * NNP_MAXE + e];
        sp[t] = s;
        __syncthreads();
        for (int o = 1; o < nt; o <<= 1) {
            const int v = (t >= o) ? sp[t - o] : 0;
            __syncthreads();
            sp[t] += v;
            __syncthreads();
        }
        int run = base + ((t > 0) ? sp[t - 1] : 0);
        for (int b = lo; b < hi; ++b) {
            const int c = part[b * NNP_MAXE + e];
            part[b * NNP_MAXE + e] = run;
            run += c;
        }
        __syncthreads();
        if (t == 0) {
            const int cnt = sp[nt - 1];
            elem_off[e] = base;
            tile_off[e] = tiles;
            base += cnt;
            tiles += (cnt + TC_TILE - 1) / TC_TILE;
        }
        __syncthreads();
    }
    if (t == 0) {
        elem_off[n_elem] = base;
        tile_off[n_elem] = tiles;
    }
}

__global__ void k_elem_fill(int n, const float4* __restrict__ pos4, int n_elem, const int* __restrict__ part,
                            int* __restrict__ idx)
{
    __shared__ int wcnt[8][NNP_MAXE];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = (i < n) ? __float_as_int(pos4[i].w) : -1;
    int rank_in_warp = 0;
    for (int t = 0; t < n_elem; ++t) {
        const unsigned m = __ballot_sync(FULL, e == t);
        if (e == t) rank_in_warp = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) wcnt[w][t] = __popc(m);
    }
    __syncthreads();
    if (e >= 0) {
        int before = 0;
        for (int u = 0; u < w; ++u) before += wcnt[u][e];
        idx[part[blockIdx.x * NNP_MAXE + e] + before + rank_in_warp] = i;
    }
}

struct TcShape {
    int K0, H1, H2;   // padded to multiples of 16
    int GS;           // row stride (floats) of the G~ and dE/dG buffers, a multiple of 4
};

// shared-memory image, per element: W1 [H1][K0], W2 [H2][H1], W2t [H1][H2], W1t [K0][H1]
// (bf16, canonical B layouts), then fp32 b1[H1], b2[H2], w3[H2], b3, inv_s[K0]
__host__ __device__ inline int tc_elem_bytes(const TcShape& s)
{
    return 2 * (s.H1 * s.K0 + s.H2 * s.H1 + s.H1 * s.H2 + s.K0 * s.H1) + 4 * (s.H1 + 2 * s.H2 + 4 + s.K0);
}
// activation tiles: X [128][K0], H [128][max(H1,H2)] twice (h1 / d1, d2), then the
// FP32 staging of the next tile's G~ rows, [128][GS + 4] (the pad keeps the
// threads' 16-byte reads of their own rows on distinct banks)
__host__ __device__ inline int tc_tile_bytes(const TcShape& s)
{
    const int H = s.H1 > s.H2 ? s.H1 : s.H2;
    return 2 * TC_TILE * (s.K0 + 2 * H) + 4 * TC_TILE * (s.GS + 4);
}

__global__ void __launch_bounds__(128, 1)
k_mlp_tc(int n, const Plan* __restrict__ plan_g, const float* __restrict__ weights, TcShape sh,
         const int* __restrict__ idx, const int* __restrict__ elem_off, const int* __restrict__ tile_off,
         const float* __restrict__ Gs, float* __restrict__ Ei, float* __restrict__ dEdG, int* __restrict__ flags)
{
    extern __shared__ __align__(16) unsigned char smem_tc[];
    const Plan& P = *plan_g;
    const int t = threadIdx.x;
    const int K0 = sh.K0, H1 = sh.H1, H2 = sh.H2, HH = H1 > H2 ? H1 : H2;
    const int eb = tc_elem_bytes(sh);
    unsigned char* wimg = smem_tc;
    unsigned char* tX = smem_tc + ((P.n_elem * eb + 1023) & ~1023);
    unsigned char* tA = tX + 2 * TC_TILE * K0;    // h1, then d1
    unsigned char* tB = tA + 2 * TC_TILE * HH;    // d2
    float* tS = reinterpret_cast<float*>(tB + 2 * TC_TILE * HH);   // staged G~ rows of the next tile
    const int SS = sh.GS + 4;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;

    // weights into the canonical bf16 image (zero padded), per element
    for (int e = 0; e < P.n_elem; ++e) {
        unsigned char* img = wimg + e * eb;
        const float* src = weights + (size_t)e * P.n_params_elem;
        const float* W1 = src + P.p_woff[0];
        const float* B1 = src + P.p_boff[0];
        const float* W2 = src + P.p_woff[1];
        const float* B2 = src + P.p_boff[1];
        const float* W3 = src + P.p_woff[2];
        const float* B3 = src + P.p_boff[2];
        const int in0 = P.width[0], h1 = P.width[1], h2 = P.width[2];
        __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(img);
        __nv_bfloat16* w2 = w1 + H1 * K0;
        __nv_bfloat16* w2t = w2 + H2 * H1;
        __nv_bfloat16* w1t = w2t + H1 * H2;
        float* fb = reinterpret_cast<float*>(w1t + K0 * H1);
        for (int q = t; q < H1 * K0; q += blockDim.x) {
            const int r = q / K0, k = q % K0;
            const float v = (r < h1 && k < in0) ? W1[r * in0 + k] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(w1) + tc::cm_off(r, k, K0)) = __float2bfloat16_rn(v);
            const float vt = (k < in0 && r < h1) ? W1[r * in0 + k] : 0.f;   // W1t[k][r] = W1[r][k]
            *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(w1t) + tc::cm_off(k, r, H1)) = __float2bfloat16_rn(vt);
        }
        for (int q = t; q < H2 * H1; q += blockDim.x) {
            const int r = q / H1, k = q % H1;
            const float v = (r < h2 && k < h1) ? W2[r * h1 + k] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(w2) + tc::cm_off(r, k, H1)) = __float2bfloat16_rn(v);
            *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(w2t) + tc::cm_off(k, r, H2)) = __float2bfloat16_rn(v);
        }
        for (int q = t; q < H1; q += blockDim.x) fb[q] = (q < h1) ? B1[q] : 0.f;
        for (int q = t; q < H2; q += blockDim.x) {
            fb[H1 + q] = (q < h2) ? B2[q] : 0.f;
            fb[H1 + H2 + q] = (q < h2) ? W3[q] : 0.f;
        }
        if (t == 0) fb[H1 + 2 * H2] = B3[0];
        for (int q = t; q < K0; q += blockDim.x) fb[H1 + 2 * H2 + 4 + q] = (q < in0) ? P.e[e].inv_s[q] : 0.f;
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc::smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < 32) {   // warp 0 allocates the accumulator columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(tc::smem_u32(&tmem_base)), "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t mb = tc::smem_u32(&mbar);
    const uint32_t lane_addr = tmem + ((uint32_t)((t >> 5) * 32) << 16);   // this warp's TMEM lane quarter
    const uint32_t D1 = 0, D2 = 32, D3 = 64, D4 = 0;                          // column offsets
    uint32_t phase = 0;
    bool ok = true;
    const int n_tiles = tile_off[P.n_elem];
    // element of tile tl and the atom of this thread's row in it (-1: padding)
    auto tile_atom = [&](int tl, int& e_out) {
        int e = 0;
        while (e + 1 < P.n_elem && tile_off[e + 1] <= tl) ++e;
        e_out = e;
        const int row = elem_off[e] + (tl - tile_off[e]) * TC_TILE + t;
        return (row < elem_off[e + 1]) ? idx[row] : -1;
    };
    // asynchronous copy of this thread's G~ row into its staging row (one group)
    auto prefetch = [&](int a) {
        if (a >= 0) {
            const float* src = Gs + (size_t)a * P.gs;
            const uint32_t dst = tc::smem_u32(tS + t * SS);
            for (int c = 0; c < P.gs; c += 4)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 4 * c), "l"(src + c) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int e_next = 0, atom_next = -1;
    if ((int)blockIdx.x < n_tiles) {
        atom_next = tile_atom(blockIdx.x, e_next);
        prefetch(atom_next);
    }

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int e = e_next, atom = atom_next;
        const unsigned char* img = wimg + e * eb;
        const float* fb = reinterpret_cast<const float*>(img + 2 * (H1 * K0 + H2 * H1 + H1 * H2 + K0 * H1));
        const uint32_t w1a = tc::smem_u32(img), w2a = w1a + 2 * H1 * K0, w2ta = w2a + 2 * H2 * H1,
                       w1ta = w2ta + 2 * H1 * H2;
        const uint32_t xa = tc::smem_u32(tX), aa = tc::smem_u32(tA), ba = tc::smem_u32(tB);

        // X row: G~ of this atom from its staging row (zeros for padding rows and
        // columns); then the next tile's rows are copied in while this one runs
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        for (int k0 = 0; k0 < K0; k0 += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u;
                v[u] = (atom >= 0 && k < P.width[0]) ? tS[t * SS + k] : 0.f;
            }
            tc::put8(tX, t, k0, K0, v);
        }
        atom_next = -1;
        if (tile + (int)gridDim.x < n_tiles) atom_next = tile_atom(tile + gridDim.x, e_next);
        prefetch(atom_next);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // layer 1 forward: D1[128][H1] = X W1^T
        if (t == 0) {
            for (int kc = 0; kc < K0 / 16; ++kc)
                tc::mma_bf16(tmem + D1, tc::make_desc(xa + kc * 256, 128, (K0 / 8) * 128),
                             tc::make_desc(w1a + kc * 256, 128, (K0 / 8) * 128), tc::make_idesc(H1), kc > 0);
            tc::commit(mb);
        }
        ok = __syncthreads_and(tc::mbar_wait(mb, phase) ? 1 : 0) != 0;   // block-uniform
        phase ^= 1u;
        if (!ok) break;
        tc::fence_after();
        float h1v[32], tmp[32];
        tc::tmem_ld32(lane_addr + D1, tmp);
#pragma unroll
        for (int q = 0; q < 32; ++q) h1v[q] = (q < H1) ? tanhf(tmp[q] + fb[q]) : 0.f;
        for (int k0 = 0; k0 < H1; k0 += 8) tc::put8(tA, t, k0, H1, h1v + k0);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // layer 2 forward: D2[128][H2] = h1 W2^T
        if (t == 0) {
            for (int kc = 0; kc < H1 / 16; ++kc)
                tc::mma_bf16(tmem + D2, tc::make_desc(aa + kc * 256, 128, (H1 / 8) * 128),
                             tc::make_desc(w2a + kc * 256, 128, (H1 / 8) * 128), tc::make_idesc(H2), kc > 0);
            tc::commit(mb);
        }
        ok = __syncthreads_and(tc::mbar_wait(mb, phase) ? 1 : 0) != 0;
        phase ^= 1u;
        if (!ok) break;
        tc::fence_after();
        tc::tmem_ld32(lane_addr + D2, tmp);
        float E = fb[H1 + 2 * H2];
        float d2[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const float h2 = (q < H2) ? tanhf(tmp[q] + fb[H1 + q]) : 0.f;
            const float w3 = (q < H2) ? fb[H1 + H2 + q] : 0.f;
            E = fmaf(w3, h2, E);
            d2[q] = w3 * (1.f - h2 * h2);
        }
        if (atom >= 0) Ei[atom] = E;
        for (int k0 = 0; k0 < H2; k0 += 8) tc::put8(tB, t, k0, H2, d2 + k0);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // layer 2 backward: D3[128][H1] = d2 W2  (B = W2^T stored [H1][H2])
        if (t == 0) {
            for (int kc = 0; kc < H2 / 16; ++kc)
                tc::mma_bf16(tmem + D3, tc::make_desc(ba + kc * 256, 128, (H2 / 8) * 128),
                             tc::make_desc(w2ta + kc * 256, 128, (H2 / 8) * 128), tc::make_idesc(H1), kc > 0);
            tc::commit(mb);
        }
        ok = __syncthreads_and(tc::mbar_wait(mb, phase) ? 1 : 0) != 0;
        phase ^= 1u;
        if (!ok) break;
        tc::fence_after();
        tc::tmem_ld32(lane_addr + D3, tmp);
#pragma unroll
        for (int q = 0; q < 32; ++q) h1v[q] = (q < H1) ? tmp[q] * (1.f - h1v[q] * h1v[q]) : 0.f;   // d1
        for (int k0 = 0; k0 < H1; k0 += 8) tc::put8(tA, t, k0, H1, h1v + k0);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // layer 1 backward: D4[128][K0] = d1 W1  (B = W1^T stored [K0][H1])
        if (t == 0) {
            for (int kc = 0; kc < H1 / 16; ++kc)
                tc::mma_bf16(tmem + D4, tc::make_desc(aa + kc * 256, 128, (H1 / 8) * 128),
                             tc::make_desc(w1ta + kc * 256, 128, (H1 / 8) * 128), tc::make_idesc(K0), kc > 0);
            tc::commit(mb);
        }
        ok = __syncthreads_and(tc::mbar_wait(mb, phase) ? 1 : 0) != 0;
        phase ^= 1u;
        if (!ok) break;
        tc::fence_after();
        for (int c0 = 0; c0 < K0; c0 += 32) {
            tc::tmem_ld32(lane_addr + D4 + c0, tmp);
            if (atom >= 0) {
                // 16-byte stores up to the row stride (1/s is zero past n_G)
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    const int k = c0 + q;
                    if (k < P.gs)
                        *reinterpret_cast<float4*>(dEdG + (size_t)atom * P.gs + k) =
                            make_float4(tmp[q] * fb[H1 + 2 * H2 + 4 + k], tmp[q + 1] * fb[H1 + 2 * H2 + 5 + k],
                                        tmp[q + 2] * fb[H1 + 2 * H2 + 6 + k], tmp[q + 3] * fb[H1 + 2 * H2 + 7 + k]);
                }
            }
        }
        tc::fence_before();
        __syncthreads();   // TMEM and tiles are reused by the next tile
        tc::fence_after();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy left in flight
    if (!ok && t == 0) atomicOr(&flags[FLAG_ERR], ERR_TIMEOUT);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TC_TMEM_COLS));
}
