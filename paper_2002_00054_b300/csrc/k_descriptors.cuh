// k_descriptors.cuh -- symmetry functions (Fig. 1b step 1 and the angular loop of
// Sec. 3.1) and the chain-rule force pass (Fig. 1b step 3).
//
// Mapping: one warp per centre atom i (the paper's "flat" atom parallelism,
// Sec. 4.3, with the neighbour and pair loops spread over the 32 lanes).
//
// Staging.  The warp keeps its atom's neighbours inside the cutoff in shared
// memory (compacted with a ballot): per neighbour the displacement d, r or 1/r
// and the angular pair factors P_q(r) = exp(-eta_q r^2) f_c(r) (force pass also
// dP_q/dr), computed once per atom.
//
// Pairs j < k are walked as 32 x 32 blocks of the list: in block (A, B) lane l
// takes j = 32A + l and partners k = 32B + (l + s) mod 32.  Each lane builds a
// bitmask of its partners that contribute (narrow: r_jk < r_c, about half);
// the 32 masks are transposed into a warp queue of live pairs (s-major, so j
// and k stay distinct within a batch) and processed 32 at a time with every
// lane busy, whatever the spread of live partners per j.
//
// Angular accumulators are dense in (eta_q, lambda, k) with zeta = 2^k: the
// powers (1 +- cos)^(2^k) come from repeated squaring, and the model's
// descriptors are gathered from the dense set at the end.
//
// The force pass recomputes every descriptor derivative instead of storing
// dG/dr (the paper's recompute-not-store rule, Sec. 3.3 and Sec. 5): for each
// pair it contracts the derivative with dE_i/dG_i on the fly and accumulates
// g_ij = dE_i/dd_ij per neighbour.  g is written per neighbour-list slot;
// forces are then gathered per atom without atomics (k_gather).
#pragma once
#include "common.cuh"

struct NbView {
    const uint32_t* nbr;
    const int* ncount;
    int stride;
    const int* sys_of = nullptr;      // batches: system of each atom (nullptr: one system)
    const float4* sys_box = nullptr;  // batches: box edges of each system
    // main pass visiting order (nullptr: atom order): the atoms sorted by cell at
    // the last list rebuild, so that the atoms a block's warps take at one time are
    // spatial neighbours and share their neighbours' cache lines, whatever order
    // the caller keeps its atoms in
    const int* order = nullptr;
};

// box edges seen by atom i
__device__ __forceinline__ void atom_box(const NbView& nv, const Box& bx, int i, float& Lx, float& Ly, float& Lz)
{
    if (nv.sys_of) {
        const float4 b = nv.sys_box[nv.sys_of[i]];
        Lx = b.x; Ly = b.y; Lz = b.z;
    } else {
        Lx = bx.L[0]; Ly = bx.L[1]; Lz = bx.L[2];
    }
}

// Live pairs waiting in a warp's queue: up to 31 left over from earlier block
// pairs, the up to 1024 of one 32 x 32 block, and the 16-byte copy granule.
#define PAIR_QUEUE 1088
// compile-time flag handed to the force pass's batch body (full batch or the partial one)
template <bool B> struct BTag { static constexpr bool value = B; };

// Atoms with more neighbours inside the cutoff than the shared-memory capacity C
// of the main launch.  The descriptor kernel's main pass (pass 0) appends them to
// spill[1 ..] (count in spill[0]) and skips them; every kernel's pass 1 walks that
// queue with C = list stride, which no atom can exceed.  The per-atom arithmetic
// is the same in both passes.
__device__ __forceinline__ int atom_count(int pass, int n, const int* spill)
{
    return pass ? spill[0] : n;
}
__device__ __forceinline__ int atom_at(int pass, int it, const int* spill, const int* order = nullptr)
{
    return pass ? spill[1 + it] : (order ? order[it] : it);
}
// Pair-queue records.  The descriptor pass stores each atom's live-pair queue
// (every 32 x 32 block pair, in walk order) so that the force pass does not
// rebuild it.  Record layout (u16): M, the staging fingerprint (2 words), the
// number of entries, one count per block pair, then from the next multiple of 8
// the entries of all block pairs back to back, each entry j | k << 8 (so records
// exist only for M <= 256).  Records are 8-entry aligned and addressed by
// qoff[i] = offset / 8 (QOFF_NONE: not stored; the force pass rebuilds the
// queue).  Each warp claims chunks of QCHUNK entries of the pool with one
// atomic; the pool counter also records the demand when the pool is too small.
#define QOFF_NONE 0xffffffffu
#define QOFF_SPILLED 0xfffffffeu   // not stored: already queued for the wide-capacity pass
#define QCHUNK 65536ull
#define QHDR 4
__host__ __device__ inline int queue_entries_start(int nb)
{
    return (QHDR + nb * (nb + 1) / 2 + 7) & ~7;
}
__host__ __device__ inline unsigned long long queue_record_bound(int M)
{
    const int nb = (M + 31) / 32;
    const unsigned long long nbp = (unsigned long long)nb * (nb + 1) / 2;
    return (unsigned long long)queue_entries_start(nb) + (unsigned long long)M * (M - 1) / 2 + 7 * nbp;
}

// L2 prefetch of [p, p + bytes) by the lanes of a warp, one 128-byte line per
// instruction (every address lies inside the range).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes, int lane)
{
    const char* c = static_cast<const char*>(p);
    for (size_t o = (size_t)lane * 128; o < bytes; o += 32 * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
    if (lane == 31 && bytes > 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(c + bytes - 1));
}

// The atoms a warp evaluates.  Main passes (ctr != nullptr): chunks of up to
// ATOM_CHUNK consecutive positions of the visiting order, claimed from a counter
// that the host clears before the launch, so that the warps of a launch finish
// together however the atoms' costs vary (with a fixed stride the warp slots
// idled ~5 % of a 1M-atom launch waiting for the slowest warps).  Launches with
// fewer than 16 chunks per warp, and the other passes, take a fixed stride over
// the grid's warps.  Positions are warp-uniform.
#define ATOM_CHUNK 4
struct AtomWalk {
    int* ctr;
    int it0, step, n, lane;
    int end = 0;
    __device__ int claim()
    {
        int b = 0;
        if (lane == 0) b = atomicAdd(ctr, ATOM_CHUNK);
        b = __shfl_sync(FULL, b, 0);
        end = min(b + ATOM_CHUNK, n);
        return b;
    }
    __device__ int first()
    {
        if (ctr && n < 16 * ATOM_CHUNK * step) ctr = nullptr;   // small launch: the stride
        return ctr ? claim() : it0;
    }
    __device__ int next(int it) { return ctr ? ((it + 1 < end) ? it + 1 : claim()) : it + step; }
    // the position after it when already known (-1 otherwise)
    __device__ int peek(int it) const
    {
        const int t = ctr ? ((it + 1 < end) ? it + 1 : -1) : it + step;
        return t < n ? t : -1;
    }
};

// true when atom i must be skipped by this pass (M > C)
__device__ __forceinline__ bool over_capacity(int M, int C, int pass, int i, int* spill, bool enqueue, int lane,
                                              int* flags, unsigned long long& c_spill)
{
    if (M <= C) return false;
    if (lane == 0) {
        if (pass) {
            atomicOr(&flags[FLAG_ERR], ERR_RC_OVERFLOW);   // C = stride in pass 1: unreachable
        } else if (enqueue) {
            spill[1 + atomicAdd(spill, 1)] = i;
            ++c_spill;
        }
    }
    return true;
}

// Per-warp shared-memory arrays (C = capacity inside the cutoff, S = list stride).
struct WarpSmem {
    float4* nd;     // descriptor pass: narrow kind (dx, dy, dz, h), wide kind (u, g) with u the
                    // unit vector d/r rounded to float and g = (1 - |u|^2)/2; force pass (dx, dy, dz, 1/r)
    float* ninv;    // 1 / r (descriptor pass, narrow kind with more than 2 eta)
    float4* nrad;   // (r^2 as hi, lo; f_c; element) (descriptor pass)
    float* nh;      // h = r^2 / 2 - rc^2 / 4 (force passes that rebuild the live masks)
    int* jidx;      // atom index of each staged neighbour (force pass over stored staging)
    float4* npf;    // P_q; force pass with <= 2 eta: (P_0, P_1, dP_0/dr, dP_1/dr)
    float4* ndp;    // dP_q / dr (force pass with > 2 eta)
    unsigned char* nel;   // element of each staged neighbour (force pass, resolved angular)
    int* sgh;       // g accumulators, 3 per neighbour, fixed point: hi words (force)
    int* sgl;       //   and lo words
    unsigned short* queue;   // live pairs of the current block
    short* cmap;    // compact index of each list slot, -1 outside the cutoff (force)
    // force pass, during staging only (they share the queue's space): per radial
    // descriptor (eta log2 e as hi, lo; r_s; -2 eta) and dE/dG of the current atom
    float4* rtab;
    float* rw;
};
static_assert(NNP_MAXRAD * 20 <= PAIR_QUEUE * 2, "radial table must fit the queue space");

// BIG: more than 2 eta (P_q fills its float4; 1/r in its own array)
__host__ __device__ inline size_t sf_warp_bytes(int C, bool big)
{
    return (size_t)C * (16 + 16 + 16 + (big ? 4 : 0)) + NNP_MAXG * 8 + PAIR_QUEUE * 2 + 16;   // + closest-pair slot
}
// PACK: P_q and dP_q/dr share one float4 per neighbour (at most 2 eta).  A 4C-byte
// array holds h (passes that rebuild the live masks) or the neighbours' atom
// indices (the pass over stored staging).  The last 80 bytes hold the warp's
// nine FP64 virial sums.
__host__ __device__ inline size_t force_warp_bytes(int C, int S, bool pack, bool res, bool stored = false)
{
    return (size_t)C * (16 + (pack ? 16 : 32) + 24) + PAIR_QUEUE * 2 + NNP_MAXG * 4 + (size_t)S * 2 +
           (res ? (size_t)((C + 15) & ~15) : 0) + (size_t)C * 4 + 80;
}

// Fixed-point accumulation of the force pass.  A contribution v, |v| < FX_LIMIT
// eV/A, is split exactly into hi = round(v 2^H) and lo = round((v - hi 2^-H) 2^L)
// (H, L: FxU<NARROW>; the remainder is a float difference of nearby values, so
// it is exact), and each part is added into its own int32 word with a native
// shared-memory integer atomic.  Per add |hi| < 2^21 and |lo| <= 2^(L-H-1).  Without
// CARRY (L - H <= 21) the up to 1024 adds a neighbour receives (list stride <= 1024)
// cannot overflow either word; with CARRY (the narrow kind, |lo| <= 2^23) a low word
// stays below 2^31 for up to FX_MAXADDS adds: the pass over stored queues, where a
// slot takes at most M adds, leaves atoms with M > FX_MAXADDS to the wide-capacity
// pass, which carries the low words into the high words between block pairs when
// a slot could take more.  The only rounding is 2^-(L+1) eV/A per add, and the sums do
// not depend on the order of the adds.  hi is zero for |v| < 2^-(H+1).  L stays at
// 27: with a coarser low unit the contributions below half a unit, which share a
// radial sign, round away and bias the virial.
#define FX_LIMIT 32000.0f
#define FX_MAXADDS 255   // adds of |lo| <= 2^23 into a low word without a carry: 255 * 2^23 < 2^31
template <bool N>
struct FxU {
    static constexpr int HB = N ? FX_HB_NARROW : FX_HB_WIDE, LB = N ? FX_LB_NARROW : FX_LB_WIDE;
    // CARRY: lo is rounded with a conversion instruction (|r 2^LB| up to 2^(LB-HB-1)),
    // and a low word holds at most FX_MAXADDS adds between carries
    static constexpr bool CARRY = LB - HB > 21;
    static_assert((!CARRY && LB - HB <= 21) || (CARRY && LB - HB <= 24), "fixed-point word ranges");
    static_assert(HB >= 0 && HB <= 6, "fixed-point word ranges");
};
// The roundings to integers use the 1.5 * 2^23 shift: for |x| < 2^22, x + 1.5 * 2^23
// rounds x to the nearest integer, which then sits in the low mantissa bits
// (integer = bits(x + S) - bits(S)), and (x + S) - S is that integer as a float;
// no float/int conversion instructions.  |v 2^H| < 2^22 holds for |v| < FX_LIMIT,
// and |r 2^L| <= 2^20 without CARRY; with CARRY lo takes a conversion instead.
// (inside the helpers below, which are templated on the kind N)
#define FX_HS ((float)(1 << FxU<N>::HB))
#define FX_LS ((float)(1 << FxU<N>::LB))
template <bool N>
__device__ __forceinline__ void fx_split(float v, int& hi, int& lo)
{
    const float S = 12582912.0f;   // 1.5 * 2^23
    const float th = fmaf(v, FX_HS, S);
    hi = __float_as_int(th) - __float_as_int(S);
    const float r = fmaf(th - S, -1.0f / FX_HS, v);
    lo = FxU<N>::CARRY ? __float2int_rn(r * FX_LS) : __float_as_int(fmaf(r, FX_LS, S)) - __float_as_int(S);
}
// Two contributions at once (packed f32x2 arithmetic, the same roundings).
template <bool N>
__device__ __forceinline__ void fx_split2(float2 v, int& hx, int& lx, int& hy, int& ly)
{
    const float S = 12582912.0f;
    const float2 th = fma2(v, f2(FX_HS, FX_HS), f2(S, S));
    hx = __float_as_int(th.x) - __float_as_int(S);
    hy = __float_as_int(th.y) - __float_as_int(S);
    const float2 r = fma2(add2(th, f2(-S, -S)), f2(-1.0f / FX_HS, -1.0f / FX_HS), v);
    if (FxU<N>::CARRY) {
        const float2 x = mul2(r, f2(FX_LS, FX_LS));
        lx = __float2int_rn(x.x);
        ly = __float2int_rn(x.y);
    } else {
        const float2 tl = fma2(r, f2(FX_LS, FX_LS), f2(S, S));
        lx = __float_as_int(tl.x) - __float_as_int(S);
        ly = __float_as_int(tl.y) - __float_as_int(S);
    }
}
// lo alone, for |v| < 2^-(HB+1) (hi = 0): the same bits as fx_split2's lo
template <bool N>
__device__ __forceinline__ void fx_lo2(float2 v, int& lx, int& ly)
{
    const float S = 12582912.0f;
    if (FxU<N>::CARRY) {
        const float2 x = mul2(v, f2(FX_LS, FX_LS));
        lx = __float2int_rn(x.x);
        ly = __float2int_rn(x.y);
    } else {
        const float2 tl = fma2(v, f2(FX_LS, FX_LS), f2(S, S));
        lx = __float_as_int(tl.x) - __float_as_int(S);
        ly = __float_as_int(tl.y) - __float_as_int(S);
    }
}
// Moves the low word's multiples of 2^(LB-HB) into the high word (same value;
// the low word is left in [0, 2^(LB-HB))).  One lane per word.
template <bool N>
__device__ __forceinline__ void fx_carry(const WarpSmem& w, int idx)
{
    const int lo = w.sgl[idx];
    const int c = lo >> (FxU<N>::LB - FxU<N>::HB);
    w.sgl[idx] = lo - (c << (FxU<N>::LB - FxU<N>::HB));
    w.sgh[idx] += c;
}
template <bool N>
__device__ __forceinline__ void fx_add2(const WarpSmem& w, int ix, int iy, float2 v)
{
    int hx, lx, hy, ly;
    fx_split2<N>(v, hx, lx, hy, ly);
    atomicAdd(&w.sgh[ix], hx);
    atomicAdd(&w.sgl[ix], lx);
    atomicAdd(&w.sgh[iy], hy);
    atomicAdd(&w.sgl[iy], ly);
}
template <bool N>
__device__ __forceinline__ void fx_set(const WarpSmem& w, int idx, float v)
{
    int hi, lo;
    fx_split<N>(v, hi, lo);
    w.sgh[idx] = hi;
    w.sgl[idx] = lo;
}
template <bool N>
__device__ __forceinline__ void fx_add(const WarpSmem& w, int idx, float v)
{
    int hi, lo;
    fx_split<N>(v, hi, lo);
    atomicAdd(&w.sgh[idx], hi);
    atomicAdd(&w.sgl[idx], lo);
}
template <bool N>
__device__ __forceinline__ float fx_get(const WarpSmem& w, int idx)
{
    return fmaf((float)w.sgl[idx], 1.0f / FX_LS, (float)w.sgh[idx] * (1.0f / FX_HS));
}
// the same sum as one integer in units of 2^-LB eV/A (exact: |value| < 2^52)
template <bool N>
__device__ __forceinline__ long long fx_get64(const WarpSmem& w, int idx)
{
    return (long long)w.sgh[idx] * (1ll << (FxU<N>::LB - FxU<N>::HB)) + (long long)w.sgl[idx];
}

// A batch of the narrow kind with a contribution of at least 2^-(HB+1) eV/A (rare):
// every contribution of the lane split into its high and low words and added,
// out of line so that the common path (low words only) keeps its registers.
template <bool N>
__device__ __noinline__ void fx_add6_split(int* __restrict__ sgh, int* __restrict__ sgl, int j, int k, float2 gaxy,
                                           float2 gbxy, float2 gz)
{
    int h0, l0, h1, l1, h2, l2, h3, l3, h4, l4, h5, l5;
    fx_split2<N>(gaxy, h0, l0, h1, l1);
    fx_split2<N>(gbxy, h2, l2, h3, l3);
    fx_split2<N>(gz, h4, l4, h5, l5);
    atomicAdd(&sgl[3 * j + 0], l0);
    atomicAdd(&sgl[3 * j + 1], l1);
    atomicAdd(&sgl[3 * k + 0], l2);
    atomicAdd(&sgl[3 * k + 1], l3);
    atomicAdd(&sgl[3 * j + 2], l4);
    atomicAdd(&sgl[3 * k + 2], l5);
    if (h0) atomicAdd(&sgh[3 * j + 0], h0);
    if (h1) atomicAdd(&sgh[3 * j + 1], h1);
    if (h2) atomicAdd(&sgh[3 * k + 0], h2);
    if (h3) atomicAdd(&sgh[3 * k + 1], h3);
    if (h4) atomicAdd(&sgh[3 * j + 2], h4);
    if (h5) atomicAdd(&sgh[3 * k + 2], h5);
}

// Narrow-kind live test r_jk < rc written with h = r^2 / 2 - rc^2 / 4 of each
// neighbour: |b - a|^2 < rc^2  <=>  a . b - h_b > h_a.  Three FMAs and a compare
// per pair; the roundings are explicit, so every kernel that rebuilds a live mask
// keeps exactly the pairs the descriptor pass kept.
__device__ __forceinline__ float live_h(float r2, float rc2) { return fmaf(r2, 0.5f, -0.25f * rc2); }
__device__ __forceinline__ float dist2_fma(float dx, float dy, float dz) { return fmaf(dz, dz, fmaf(dy, dy, dx * dx)); }
__device__ __forceinline__ bool live_pair(const float4 a, float ha, const float4 b, float hb)
{
    return fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, -hb))) > ha;
}

// Radial part of g_ij for staged neighbour `at`: the sum over the radial
// descriptors that take the neighbour's element of dE/dG * dG/dr * d / r, into
// the fixed-point accumulators.
template <bool N>
__device__ __forceinline__ void radial_g(const WarpSmem& w, const Plan& P, const ElemPlan& E, int at, float r, float ir,
                                         float fc, float dfc, int ej, float dx, float dy, float dz, int* flags)
{
    float gr = 0.f;
    auto rad = [&](int rr) {
        const float4 t = w.rtab[rr];
        const float x = r - t.z;
        const float ex = gauss2(t.x, t.y, x * x);   // forces: float accuracy suffices
        gr += w.rw[rr] * ex * fmaf(t.w * x, fc, dfc);
    };
    for (int rr = 0; rr < E.rad_nall; ++rr) rad(rr);
    for (int rr = E.rad_beg[ej], re = E.rad_end[ej]; rr < re; ++rr) rad(rr);
    const float gs = gr * ir;
    if (!(fabsf(gs) * P.rc < FX_LIMIT)) atomicOr(&flags[FLAG_ERR], ERR_RANGE);
    fx_set<N>(w, 3 * at + 0, gs * dx);
    fx_set<N>(w, 3 * at + 1, gs * dy);
    fx_set<N>(w, 3 * at + 2, gs * dz);
}

// (r - r_s)^2 as xh + xl from a staged (r^2 hi, r^2 lo, ...) record: r^2 itself
// for r_s = 0, else r = sqrt(r^2) as hi + lo and the square of r - r_s.
__device__ __forceinline__ void radial_x2(const float4 nr, float rs, float& xh, float& xl)
{
    xh = nr.x;
    xl = nr.y;
    if (rs != 0.f) {
        const float rh = sqrtf(nr.x);
        const float rlo = (fmaf(-rh, rh, nr.x) + nr.y) * (0.5f / rh);
        float dh, dl;
        two_sum(rh, -rs, dh, dl);
        dl += rlo;
        xh = dh * dh;
        xl = fmaf(dh, dh, -xh) + 2.0f * dh * dl;
    }
}

// Stages the neighbours of atom i within the cutoff, compacted in list order.
// Returns M.  FORCE: nd.w = 1/r, dP/dr, the radial part of g (into sg), slot map.
// N: the force pass's fixed-point units (FxU<N>); in the descriptor pass, the
// narrow angular kind (the wide kind stages unit vectors instead of d).
// Both passes compute r, 1/r, f_c, f_c', P_q and dP_q/dr from the same
// double-float intermediates (|d|^2, r, the cutoff's cos), so the staged values
// the descriptor pass writes for the force pass are bitwise the force pass's own.
// Two sweeps: the list entries (lanes over list slots) select the neighbours
// inside the cutoff and park their displacement, element and atom index at their
// compact position; the per-neighbour functions then run with lanes over the
// compacted neighbours (about 60 % of the list entries lie inside the cutoff, so
// the costly part takes ceil(M/32) rounds instead of ceil(n_list/32)).
// rtab (descriptor pass; nullptr: not fused): the radial descriptors resolved by
// neighbour element, at most 16, summed per lane into row `lane` of a [32][16]
// table, columns XOR-swizzled by (lane & 15); the caller sums the columns.
template <int NETA, bool FORCE, bool N = false>
__device__ __forceinline__ int stage_neighbors(int i, const float4 pi, const Box& bx, const NbView& nv,
                                               const float4* __restrict__ pos4, const Plan& P, const ElemPlan& E,
                                               const float* khi, const float* klo, const float* etav, int C,
                                               const WarpSmem& w, const float* sW, int lane, int* flags, int& n_list,
                                               unsigned& sig, float& r2min, float4* __restrict__ stg = nullptr,
                                               size_t stg_plane = 0, float* rtab = nullptr)
{
    const int cnt = nv.ncount[i];
    n_list = cnt;
    sig = 0u;
    const uint32_t* row = nv.nbr + (size_t)i * nv.stride;
    float Lx, Ly, Lz;
    atom_box(nv, bx, i, Lx, Ly, Lz);
    int M = 0;
    // list entries two rounds ahead, positions one round ahead
    uint32_t e_n = (lane < cnt) ? row[lane] : 0u;
    uint32_t e_nn = (lane + 32 < cnt) ? row[lane + 32] : 0u;
    float4 p_n = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < cnt) p_n = pos4[e_n & NB_INDEX_MASK];
    for (int base = 0; base < cnt; base += 32) {
        const int s = base + lane;
        const uint32_t e = e_n;
        const float4 pj = p_n;
        e_n = e_nn;
        if (s + 32 < cnt) p_n = pos4[e_nn & NB_INDEX_MASK];
        e_nn = (s + 64 < cnt) ? row[s + 64] : 0u;
        bool keep = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        // a round whose entries all sit at image shift (0, 0, 0) (all but the atoms
        // near the box faces) takes pj - pi, which is what pair_disp returns for a
        // zero shift (TwoSum: t + e rounds back to t); -0.8 % on water, -1.2 % FCC
        const bool shifted = __any_sync(FULL, s < cnt && (e >> 24) != NB_CODE_NOSHIFT);
        if (s < cnt) {
            if (shifted) {
                float ox, oy, oz;
                nb_shift(e, Lx, Ly, Lz, ox, oy, oz);
                dx = pair_disp(pj.x, pi.x, ox);
                dy = pair_disp(pj.y, pi.y, oy);
                dz = pair_disp(pj.z, pi.z, oz);
            } else {
                dx = pj.x - pi.x;
                dy = pj.y - pi.y;
                dz = pj.z - pi.z;
            }
            r2 = dist2_fma(dx, dy, dz);   // explicit roundings: every pass keeps the same neighbours
            keep = r2 < P.rc2;
        }
        const unsigned m = __ballot_sync(FULL, keep);
        sig = sig * 0x9e3779b1u + m;   // fingerprint of which list slots were kept
        const int at = M + __popc(m & ((1u << lane) - 1u));
        if (FORCE && s < cnt) w.cmap[s] = (keep && at < C) ? (short)at : (short)-1;
        if (keep && at < C) {
            if (r2 < 1e-8f) atomicOr(&flags[FLAG_ERR], ERR_CLOSE);
            if (!FORCE) r2min = fminf(r2min, r2);
            // parked until the second sweep: (d, element) and the atom index
            w.nd[at] = make_float4(dx, dy, dz, pj.w);
            reinterpret_cast<uint32_t*>(w.npf + at)[3] = e & NB_INDEX_MASK;
        }
        M += __popc(m);
    }
    __syncwarp();
    if (rtab) {
        float4* t4 = reinterpret_cast<float4*>(rtab + 16 * lane);
        t4[0] = t4[1] = t4[2] = t4[3] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int Mc = M < C ? M : C;
    for (int at = lane; at < Mc; at += 32) {
        const float4 pk = w.nd[at];
        const uint32_t aidx = reinterpret_cast<const uint32_t*>(w.npf + at)[3];
        const float dx = pk.x, dy = pk.y, dz = pk.z;
        const int ej = __float_as_int(pk.w);
        const float r2 = dist2_fma(dx, dy, dz);   // the first sweep's value, bit for bit
        {
            // ACC: the descriptor pass, and the force pass wherever the descriptor pass
            // stores its staged values for it (narrow kind, at most 2 eta), which must
            // then be reproduced bit for bit; other force passes need float accuracy only.
            constexpr bool ACC = !FORCE || (N && NETA <= 2);
            float r2h, r2l = 0.f, r, ir, rl = 0.f, fch, fcl = 0.f, dfc;
            float pq[4] = {0.f, 0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
            if (ACC) {
                // r^2 = r2h + r2l (exact to 2^-48), r = r + rl, the cutoff as fch + fcl
                dd_norm2(dx, dy, dz, r2h, r2l);
                r = sqrtf(r2h);
                ir = 1.0f / r;
                rl = (fmaf(-r, r, r2h) + r2l) * (0.5f * ir);
                cutoff_dd(r, rl, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, P.cs64, fch, fcl, dfc);
            } else {
                r2h = r2;
                r = sqrtf(r2);
                ir = 1.0f / r;
                cutoff_fn(r, P.inv_2rc, P.inv_2rc_lo, P.hpi_rc, fch, dfc);
            }
            const float fc = fch + fcl;
            constexpr bool PK = ACC && NETA == 2 && !FORCE;
            if (PK) {
                // descriptor pass: both eta as packed pairs, each value bitwise the
                // loop's below (which the force passes run)
                const float2 KH = f2(khi[0], khi[1]), KLo = f2(klo[0], klo[1]);
                const float2 R2H = f2(r2h, r2h), R2L = f2(r2l, r2l);
                const float2 ah = mul2(KH, R2H);
                const float2 al = add2(fma2(KH, R2H, f2(-ah.x, -ah.y)), fma2(KLo, R2H, mul2(KH, R2L)));
                float2 eh, el;
                exp2_dd2(ah, al, eh, el);
                const float2 FCH = f2(fch, fch);
                const float2 ph = mul2(eh, FCH);
                const float2 pp = add2(ph, add2(fma2(eh, FCH, f2(-ph.x, -ph.y)), fma2(eh, f2(fcl, fcl), mul2(el, FCH))));
                pq[0] = pp.x;
                pq[1] = pp.y;
                dq[0] = eh.x * (dfc - 2.0f * etav[0] * r * fc);
                dq[1] = eh.y * (dfc - 2.0f * etav[1] * r * fc);
            }
#pragma unroll
            for (int q = 0; q < NETA && !PK; ++q) {
                if (ACC) {
                    // P_q = exp(-eta_q r^2) f_c: both factors as hi + lo, one final rounding
                    const float ah = khi[q] * r2h;
                    const float al = fmaf(khi[q], r2h, -ah) + fmaf(klo[q], r2h, khi[q] * r2l);
                    float eh, el;
                    exp2_dd(ah, al, eh, el);
                    const float ph = eh * fch;
                    pq[q] = ph + (fmaf(eh, fch, -ph) + fmaf(eh, fcl, el * fch));
                    dq[q] = eh * (dfc - 2.0f * etav[q] * r * fc);
                } else {
                    const float ex = gauss2(khi[q], klo[q], r2);
                    pq[q] = ex * fc;
                    dq[q] = ex * (dfc - 2.0f * etav[q] * r * fc);
                }
            }
            const float hh = live_h(r2, P.rc2);
            if (!FORCE) {
                // at most 2 eta: 1/r rides in the free half of the P record
                if (NETA <= 2) {
                    w.npf[at] = make_float4(pq[0], pq[1], ir, 0.f);
                } else {
                    w.npf[at] = make_float4(pq[0], pq[1], pq[2], pq[3]);
                    w.ninv[at] = ir;
                }
                if (N) {
                    w.nd[at] = make_float4(dx, dy, dz, hh);
                } else {
                    // unit vector and its norm defect g = (1 - |u|^2)/2, exact
                    const float irl = ir * fmaf(-rl, ir, fmaf(-r, ir, 1.0f));
                    const float ux = fmaf(dx, irl, dx * ir), uy = fmaf(dy, irl, dy * ir), uz = fmaf(dz, irl, dz * ir);
                    float sh, sl;
                    dd_norm2(ux, uy, uz, sh, sl);
                    w.nd[at] = make_float4(ux, uy, uz, 0.5f * ((1.0f - sh) - sl));
                }
                w.nrad[at] = make_float4(r2h, r2l, fc, __int_as_float(ej));
                if (rtab) {
                    // the Gaussian's argument in double-float from r^2 = r2h + r2l (r_s = 0
                    // here, else (r - r_s)^2 by radial_x2)
                    const float4 nr = make_float4(r2h, r2l, fc, 0.f);
                    int rr = E.rad_beg[ej];
                    const int re = E.rad_end[ej];
                    // two descriptors at a time (packed pairs, each bitwise the scalar form)
                    for (; rr + 1 < re; rr += 2) {
                        float xh0, xl0, xh1, xl1;
                        radial_x2(nr, E.rad_rs[rr], xh0, xl0);
                        radial_x2(nr, E.rad_rs[rr + 1], xh1, xl1);
                        const float2 kh = f2(E.rad_khi[rr], E.rad_khi[rr + 1]), kl = f2(E.rad_klo[rr], E.rad_klo[rr + 1]);
                        const float2 xh = f2(xh0, xh1), xl = f2(xl0, xl1);
                        const float2 ah = mul2(kh, xh);
                        const float2 al = add2(fma2(kh, xh, f2(-ah.x, -ah.y)), fma2(kl, xh, mul2(kh, xl)));
                        const float2 e = exp2_acc2x2(ah, al);
                        rtab[16 * lane + (rr ^ (lane & 15))] += e.x * fc;
                        rtab[16 * lane + ((rr + 1) ^ (lane & 15))] += e.y * fc;
                    }
                    if (rr < re) {
                        float xh, xl;
                        radial_x2(nr, E.rad_rs[rr], xh, xl);
                        const float kh = E.rad_khi[rr];
                        const float ah = kh * xh;
                        const float al = fmaf(kh, xh, -ah) + fmaf(E.rad_klo[rr], xh, kh * xl);
                        rtab[16 * lane + (rr ^ (lane & 15))] += exp2_acc2(ah, al) * fc;
                    }
                }
            } else {
                w.nd[at] = make_float4(dx, dy, dz, ir);
                if (w.nh) w.nh[at] = hh;
                if (NETA <= 2) {
                    w.npf[at] = make_float4(pq[0], pq[1], dq[0], dq[1]);
                } else {
                    w.npf[at] = make_float4(pq[0], pq[1], pq[2], pq[3]);
                    w.ndp[at] = make_float4(dq[0], dq[1], dq[2], dq[3]);
                }
                if (w.nel) w.nel[at] = (unsigned char)ej;
                radial_g<N>(w, P, E, at, r, ir, fc, dfc, ej, dx, dy, dz, flags);
            }
            if (!FORCE && stg) {
                // staged record for the force pass, one plane each: (d, 1/r),
                // (P_0, P_1, dP_0/dr, dP_1/dr), (r, f_c, f_c', atom index | element << 24)
                const size_t idx = (size_t)i * C + at;
                stg[idx] = make_float4(dx, dy, dz, ir);
                stg[stg_plane + idx] = make_float4(pq[0], pq[1], dq[0], dq[1]);
                stg[2 * stg_plane + idx] =
                    make_float4(r, fc, dfc, __int_as_float((int)(aidx | ((uint32_t)ej << 24))));
            }
        }
    }
    __syncwarp();
    return M;
}

// Valid partner steps s of lane l in block pair (A, B): k = 32B + (l + s) mod 32
// must exist (and j = 32A + l); on the diagonal block each unordered pair is
// taken once (s in 1..15, or 16 for l < 16).
__device__ __forceinline__ unsigned valid_mask(int A, int B, int l, int M)
{
    if (32 * A + l >= M) return 0u;
    const int nk = M - 32 * B;   // partners present in block B
    unsigned m = 0xffffffffu;
    if (nk < 32) {
        const unsigned low = (1u << nk) - 1u;          // positions p < nk
        m = __funnelshift_r(low, low, l);               // bit s <-> position (l + s) mod 32
    }
    if (A == B) m &= 0x0000fffeu | (l < 16 ? 0x00010000u : 0u);
    return m;
}

// Bitmask over s of the contributing partners of lane l's j in block (A, B).
// A full partner block (32 present) is walked with a fixed, unrolled trip count
// (s = 1..16 on the diagonal); a partial one by scanning its valid bits.  h of
// the partners: nd[k].w (HS = 0) or nh[HS * k] (HS > 0).
template <bool NARROW, int HS>
__device__ __forceinline__ unsigned live_mask(int A, int B, int l, int M, const float4 a, float ha, const float4* nd,
                                              const float* nh)
{
    unsigned v = valid_mask(A, B, l, M);
    if (!NARROW) return v;
    const float4* blk = nd + 32 * B;
    auto hk = [&](int k, const float4& b) { return HS == 0 ? b.w : nh[HS * (32 * B + k)]; };
    unsigned mask = 0u;
    // HS = 0 (descriptor pass): a partner block with at least 16 present takes the
    // unrolled walk too, masked by v afterwards; its reads past M stay inside the
    // warp's nd and npf arrays (32 B + 31 <= M + 15 < 2C).  Measured: 16 is faster
    // than 8 or 1 here.
    if (32 * B + 32 <= M || (HS == 0 && 32 * B + 16 <= M)) {
        if (A == B) {
#pragma unroll
            for (int s = 1; s <= 16; ++s) {
                const int k = (l + s) & 31;
                const float4 b = blk[k];
                if (live_pair(a, ha, b, hk(k, b))) mask |= 1u << s;
            }
        } else {
            // every lane walks the partners in the same order (broadcast loads at
            // fixed addresses), bit t <-> partner t; rotated to bit s <-> (l + s) mod 32
            unsigned mk = 0u;
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const float4 b = blk[t];
                if (live_pair(a, ha, b, hk(t, b))) mk |= 1u << t;
            }
            mask = __funnelshift_r(mk, mk, l);
        }
        return mask & v;
    }
    while (v) {
        const int s = __ffs(v) - 1;
        v &= v - 1u;
        const int k = (l + s) & 31;
        const float4 b = blk[k];
        if (live_pair(a, ha, b, hk(k, b))) mask |= 1u << s;
    }
    return mask;
}

// Element-pair class filter: the partners k = 32B + (l + s) mod 32 (bit s) of
// lane l's j (element ej) whose elements make {e1, e2} with ej.  el_k is the
// element at this lane's position of block B (-1 past the staged neighbours).
__device__ __forceinline__ unsigned class_mask(int ej, int el_k, int e1, int e2, int lane)
{
    const unsigned m1 = __ballot_sync(FULL, el_k == e1), m2 = __ballot_sync(FULL, el_k == e2);
    unsigned r = 0u;
    if (ej == e1) r |= __funnelshift_r(m2, m2, lane);
    if (ej == e2) r |= __funnelshift_r(m1, m1, lane);
    return r;
}

// Transposes the warp's 32 x 32 bit matrix (row = lane): lane s returns column s.
__device__ __forceinline__ unsigned transpose32(unsigned m, int lane)
{
    const unsigned lo[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int j = 16 >> t;
        const unsigned o = __shfl_xor_sync(FULL, m, j);
        if (lane & j) m = (m & ~lo[t]) | ((o & ~lo[t]) >> j);
        else m = (m & lo[t]) | ((o & lo[t]) << j);
    }
    return m;
}

// Column s of the transposed block for lane `lane`: lane s holds partner step s.
// The diagonal block uses steps 1..16 only: there lane s keeps the pairs with
// l < 16 and lane s + 16 those with l >= 16 of step s (s < 16), so that 31 lanes
// share the writes instead of 16.  Returns the column bits (bit l) and sets s.
__device__ __forceinline__ unsigned block_column(unsigned mask, int lane, bool diag, int& s)
{
    unsigned col = transpose32(mask, lane);
    s = lane;
    if (diag) {
        const unsigned o = __shfl_sync(FULL, col, lane & 15);
        if (lane > 16) {
            col = o & 0xffff0000u;
            s = lane - 16;
        } else {
            col &= 0x0000ffffu;   // lane 16: step 16 has l < 16 only; lane 0: no step 0
        }
    }
    return col;
}

// Writes the live pairs (l, s) of one block, s-major, into the warp queue and
// returns their number.  Consecutive entries share s, so j and k are distinct
// across the lanes of a batch of 32 (up to where the batch crosses an s boundary).
__device__ __forceinline__ int enqueue_block(unsigned mask, int lane, unsigned short* queue, bool diag)
{
    int s;
    unsigned col = block_column(mask, lane, diag, s);
    const int cnt = __popc(col);
    int off = cnt;   // inclusive scan over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, off, o);
        if (lane >= o) off += t;
    }
    const int total = __shfl_sync(FULL, off, 31);
    off -= cnt;
    while (col) {
        const int l = __ffs(col) - 1;
        col &= col - 1u;
        queue[off++] = (unsigned short)(l | (s << 5));
    }
    __syncwarp();
    return total;
}

// The same, with each entry written as the neighbour pair itself, j | k << 8
// (j = jb + l, k = kb + (l + s) mod 32; staged indices below 256), so that the
// entries of several block pairs can share one queue.
__device__ __forceinline__ int enqueue_block_jk(unsigned mask, int lane, unsigned short* queue, int jb, int kb)
{
    int s;
    unsigned col = block_column(mask, lane, jb == kb, s);
    const int cnt = __popc(col);
    int off = cnt;   // inclusive scan over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, off, o);
        if (lane >= o) off += t;
    }
    const int total = __shfl_sync(FULL, off, 31);
    off -= cnt;
    // entry l of column s pairs j = jb + l with k = kb + ((l + s) & 31): with
    // x = (jb + l) + ((s + l) << 8), bit 13 of x is the carry of s + l past 31,
    // and kb (a multiple of 32) fills bits 13..15
    const int js = jb + (s << 8), kb8 = kb << 8;
    // two entries per step: the lowest bit left to the front of the lane's range,
    // the highest to its back (the range ends up in ascending l as with one bit
    // per step; with one bit left both writes store the same entry).  Measured:
    // 1.7 % off the water descriptor pass.
    int hi = off + cnt - 1;
    while (col) {
        const int l1 = __ffs(col) - 1, l2 = 31 - __clz(col);
        col = col & (col - 1u) & ~(1u << l2);
        queue[off++] = (unsigned short)(((l1 * 257 + js) & ~0x2000) | kb8);
        queue[hi--] = (unsigned short)(((l2 * 257 + js) & ~0x2000) | kb8);
    }
    __syncwarp();
    return total;
}

// ---------------------------------------------------------------- value pass
// KP / KN: largest k (zeta = 2^k) among the lambda = +1 / -1 functions; powers and
// terms beyond them are compiled out.
// RES: angular descriptors resolved by neighbour-element pair (one pass over
// the pairs per class).
template <int NETA, bool NARROW, int KP, int KN, bool RES, bool MG>
__global__ void __launch_bounds__(128, 6)
k_sf(int n, const float4* __restrict__ pos4, Box bx, NbView nv, const Plan* __restrict__ plan_g,
     int C, float* __restrict__ Gs, float* __restrict__ Graw, int* __restrict__ flags,
     unsigned long long* __restrict__ counters, int* __restrict__ spill, int pass,
     unsigned short* __restrict__ qpool, unsigned int* __restrict__ qoff, unsigned long long qcap,
     float4* __restrict__ stg, size_t stg_plane)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Plan& P = *plan_g;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    constexpr bool BIG = NETA > 2;
    unsigned char* base = smem + sf_warp_bytes(C, BIG) * wib;
    WarpSmem w;
    w.nd = reinterpret_cast<float4*>(base);
    w.npf = w.nd + C;
    w.nrad = w.npf + C;
    // descriptor sums as unevaluated pairs (hi, lo): no FP64 arithmetic (a slow
    // pipe on this GPU) in the per-atom epilogue
    float2* sG = reinterpret_cast<float2*>(w.nrad + C);
    w.ninv = reinterpret_cast<float*>(sG + NNP_MAXG);
    w.queue = reinterpret_cast<unsigned short*>(w.ninv + (BIG ? C : 0));
    w.nh = nullptr;
    w.jidx = nullptr;
    w.ndp = nullptr;
    w.sgh = nullptr;
    w.sgl = nullptr;
    w.cmap = nullptr;
    w.nel = nullptr;
    w.rtab = nullptr;
    w.rw = nullptr;

    // work counters, one per lane: lane 0 list entries, 1 cutoff entries, 2 pairs,
    // 3 largest row, 4 largest cutoff row; triplets per lane, spills in lane 0
    unsigned long long cnt = 0, c_spill = 0;
    unsigned c_trip = 0;
    // per warp: closest staged neighbour (r^2) so far (last 16 bytes of the warp's area)
    float* s_r2min = reinterpret_cast<float*>(base + sf_warp_bytes(C, BIG) - 16);
    if (lane == 0) *s_r2min = INFINITY;
    // this warp's chunk [qcur, qend) of the queue pool, in units of 8 entries
    // (main pass, when forces follow)
    unsigned qcur = 0, qend = 0;
    bool qcan = NARROW && (pass == 0) && (qpool != nullptr);   // wide queues are not stored
    const int nw = gridDim.x * wpb;
    const int n_items = atom_count(pass, n, spill);
    AtomWalk walk{pass == 0 ? flags + FLAG_WALK_SF : nullptr, (int)blockIdx.x * wpb + wib, nw, n_items, lane};
    for (int it = walk.first(); it < n_items; it = walk.next(it)) {
        const int i = atom_at(pass, it, spill, nv.order);
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
        unsigned sig;
        float r2_atom = INFINITY;
        // radial descriptors all resolved by neighbour element (none element-blind,
        // at most 16): summed during the staging, lanes over neighbours, into a
        // [32][16] table in the pair queue's space (unused until the angular part)
        const bool rad_tab = E.rad_nall == 0 && E.n_rad > 0 && E.n_rad <= 16;
        const int M = stage_neighbors<NETA, false, NARROW>(i, pi, bx, nv, pos4, P, E, khi, klo, etav, C, w, nullptr, lane,
                                                   flags, n_list, sig, r2_atom, pass == 0 ? stg : nullptr, stg_plane,
                                                   rad_tab ? reinterpret_cast<float*>(w.queue) : nullptr);
        // closest staged neighbour: kept per warp in shared memory, not in a register
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r2_atom = fminf(r2_atom, __shfl_xor_sync(FULL, r2_atom, o));
        if (lane == 0) *s_r2min = fminf(*s_r2min, r2_atom);
        if (over_capacity(M, C, pass, i, spill, true, lane, flags, c_spill)) {
            if (qoff && lane == 0) qoff[i] = QOFF_SPILLED;
            continue;
        }
        // radial.  The Gaussian's argument is formed in double-float from
        // r^2 = r2h + r2l (from (r - r_s)^2 for r_s != 0) by radial_x2.
        //   Table (see above): lane <-> descriptor sums its column with Kahan
        //   compensation (the columns are XOR-swizzled, so a column read is
        //   conflict free).
        //   Otherwise: lane <-> descriptor (two neighbour halves when n_rad <= 16),
        //   loop over neighbours with broadcast reads; Kahan-compensated sums (they
        //   feed G~ = (G - mu)/s with |mu/s| up to ~20).
        if (rad_tab) {
            // both half-warps on the 16 columns: rows 0..15 and 16..31 (the upper half
            // one row ahead, so that the two rows of a step sit in opposite bank halves),
            // each a compensated sum, then the two halves' (sum, -comp) pairs added
            const float* tab = reinterpret_cast<const float*>(w.queue);
            const int col = lane & 15, hf = lane >> 4;
            float sum = 0.f, comp = 0.f;
            if (col < E.n_rad) {
#pragma unroll 8
                for (int u = 0; u < 16; ++u) {
                    const int l = 16 * hf + ((u + hf) & 15);
                    const float y = tab[16 * l + (col ^ (l & 15))] - comp;
                    const float t = sum + y;
                    comp = (t - sum) - y;
                    sum = t;
                }
            }
            const float oh = __shfl_xor_sync(FULL, sum, 16), ol = __shfl_xor_sync(FULL, -comp, 16);
            float sh, el;
            two_sum(sum, oh, sh, el);
            if (hf == 0 && col < E.n_rad) sG[E.rad_out[col]] = make_float2(sh, (-comp + ol) + el);
            __syncwarp();
        } else {
            const int halves = (E.n_rad <= 16) ? 2 : 1;
            const int per = 32 / halves;
            const int hf = lane / per, slot = lane % per;
            for (int rb = 0; rb < E.n_rad; rb += per) {
                const int rr = rb + slot;
                const bool act = rr < E.n_rad;
                const float kh = act ? E.rad_khi[rr] : 0.f, kl = act ? E.rad_klo[rr] : 0.f;
                const float rs = act ? E.rad_rs[rr] : 0.f;
                const int el = act ? E.rad_elem[rr] : -2;
                float sum = 0.f, comp = 0.f;
                for (int m = hf; m < M; m += halves) {
                    const float4 nr = w.nrad[m];
                    if (el == -1 || el == __float_as_int(nr.w)) {
                        float xh, xl;
                        radial_x2(nr, rs, xh, xl);
                        const float ah = kh * xh;
                        const float al = fmaf(kh, xh, -ah) + fmaf(kl, xh, kh * xl);
                        const float y = exp2_acc2(ah, al) * nr.z - comp;
                        const float t = sum + y;
                        comp = (t - sum) - y;
                        sum = t;
                    }
                }
                float th = sum, tl = -comp;
                if (halves == 2) {
                    const float oh = __shfl_xor_sync(FULL, th, 16), ol = __shfl_xor_sync(FULL, tl, 16);
                    float s2, e2;
                    two_sum(th, oh, s2, e2);
                    th = s2;
                    tl = (tl + ol) + e2;
                }
                if (act && hf == 0) sG[E.rad_out[rr]] = make_float2(th, tl);
            }
        }
        // angular (one pass per neighbour-element pair class)
        const int ncls = RES ? E.n_cls : 1;
        for (int cls = 0; NETA > 0 && cls < ncls; ++cls) {
            constexpr int NQ = NETA > 0 ? NETA : 1, NP = (NQ + 1) / 2;
            // accumulators per eta: (lambda = +1, lambda = -1) as packed f32x2 for
            // k <= KLO, where both powers come out of one packed chain; beyond, the
            // one lambda that goes on (TX: lambda = +1) as floats
            constexpr int KLO = KP < KN ? KP : KN, KM = KP > KN ? KP : KN;
            constexpr bool TX = KP > KN;
            float2 accL[NQ][KLO + 1];
            float accT[NQ][KM - KLO + 1];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
#pragma unroll
                for (int kk = 0; kk <= KLO; ++kk) accL[q][kk] = f2(0.f, 0.f);
#pragma unroll
                for (int kk = 0; kk <= KM - KLO; ++kk) accT[q][kk] = 0.f;
            }
            float2 KH[NP], KL[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                KH[p] = f2(khi[2 * p], (2 * p + 1 < 4) ? khi[2 * p + 1] : 0.f);
                KL[p] = f2(klo[2 * p], (2 * p + 1 < 4) ? klo[2 * p + 1] : 0.f);
            }
            const int nb = (M + 31) >> 5;
            const int ce1 = RES ? E.cls_e1[cls] : -1, ce2 = RES ? E.cls_e2[cls] : -1;
            // where this atom's queue record goes (nullptr: not stored)
            unsigned short* rec = nullptr;
            // MG (capacity C <= 256, staged indices in 8 bits): the block pairs share
            // one queue (entries j | k << 8); otherwise one block pair at a time
            constexpr bool merged = MG;
            if (!RES && NARROW && qcan && merged) {
                const unsigned need8 = (unsigned)((queue_record_bound(M) + 7) >> 3);
                if (qend - qcur < need8) {
                    const unsigned long long sz = (need8 > QCHUNK / 8 ? need8 : QCHUNK / 8) * 8ull;
                    unsigned long long old = 0;
                    if (lane == 0) old = atomicAdd(&counters[CNT_QTOP], sz);
                    old = __shfl_sync(FULL, old, 0);
                    if (old + sz <= qcap && ((old + sz) >> 3) < 0xfffffff0ull) {   // offsets stay below the markers
                        qcur = (unsigned)(old >> 3);
                        qend = (unsigned)((old + sz) >> 3);
                    } else {
                        qcan = false;   // pool full: the remaining atoms are not stored
                        qcur = qend = 0;
                    }
                }
                if (qcan) rec = qpool + (size_t)qcur * 8;
            }
            if (qoff && lane == 0) qoff[i] = rec ? qcur : QOFF_NONE;
            if (rec && lane == 0) {
                rec[0] = (unsigned short)M;
                rec[1] = (unsigned short)(sig & 0xffffu);
                rec[2] = (unsigned short)(sig >> 16);
            }
            // pend: entries waiting in the queue; done: entries taken so far (a
            // multiple of 32 until the last block pair), the record position of queue[0]
            int bp = QHDR, pend = 0, done = 0;
            const int q0 = queue_entries_start(nb);
            for (int A = 0; A < nb; ++A) {
                const int jl = 32 * A + lane;
                const float4 al = (jl < M) ? w.nd[jl] : make_float4(0.f, 0.f, 0.f, 0.f);
                const int ej = (RES && jl < M) ? __float_as_int(w.nrad[jl].w) : -1;
                for (int B = A; B < nb; ++B, ++bp) {
                    unsigned mask = live_mask<NARROW, 0>(A, B, lane, M, al, al.w, w.nd, nullptr);
                    if (cls == 0) c_trip += __popc(mask);
                    if (RES && ce1 >= 0) {
                        const int kl = 32 * B + lane;
                        mask &= class_mask(ej, kl < M ? __float_as_int(w.nrad[kl].w) : -1, ce1, ce2, lane);
                    }
                    const int total = merged ? enqueue_block_jk(mask, lane, w.queue + pend, 32 * A, 32 * B)
                                             : enqueue_block(mask, lane, w.queue, A == B);
                    if (rec) {
                        // 16-byte copies of queue[pend, pend + total) rounded out to 8 entries:
                        // the first rewrites stored entries with their own values, the last
                        // runs past the end into space the next copy (or nothing) reuses
                        const int v0 = pend >> 3, v1 = (pend + total + 7) >> 3;
                        const uint4* src = reinterpret_cast<const uint4*>(w.queue);
                        uint4* dst = reinterpret_cast<uint4*>(rec + q0 + done);
                        for (int v = v0 + lane; v < v1; v += 32) dst[v] = src[v];
                        if (lane == 0) rec[bp] = (unsigned short)total;
                    }
                    // take every full batch of 32 (everything at the last block pair, or
                    // one block pair at a time); the rest waits for the next block pair
                    const int avail = pend + total;
                    const int take = (merged && !(A == nb - 1 && B == nb - 1)) ? (avail & ~31) : avail;
                    for (int e0 = 0; e0 < take; e0 += 32) {
                        const int e = e0 + lane;
                        // merged narrow-kind queues: the batch runs on every lane, a lane past
                        // the end on the pair (0, 1) with its term scaled by zero (M >= 2 when
                        // take > 0); measured: 3 % off the water descriptor pass, while the wide
                        // kind's odd eta count is faster with the branch
                        constexpr bool straight = merged && NARROW;
                        const bool live_e = e < take;
                        if (straight || live_e) {
                            const int ent = live_e ? (int)w.queue[e] : (1 << 8);
                            const float vz = live_e ? 1.f : 0.f;
                            int j, k;
                            if (merged) {
                                j = ent & 255;
                                k = ent >> 8;
                            } else {
                                const int l = ent & 31, sidx = ent >> 5;
                                j = 32 * A + l;
                                k = 32 * B + ((l + sidx) & 31);
                            }
                            const float4 a = w.nd[j], b = w.nd[k];
                            const float4 pa4 = w.npf[j], pb4 = w.npf[k];
                            const float2 PA[2] = {f2(pa4.x, pa4.y), f2(pa4.z, pa4.w)};
                            const float2 PB[2] = {f2(pb4.x, pb4.y), f2(pb4.z, pb4.w)};
                            float fcd = 1.f, rd2 = 0.f;
                            if (NARROW) {
                                const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
                                rd2 = ex * ex + ey * ey + ez * ez;
                                float dfcd;
                                cutoff_fn_fast(rd2 * rsqrtf(rd2), P.hpi_rc, fcd, dfcd);
                            }
                            // PP[k] = (b_+^(2^k), b_-^(2^k)), b_(+/-) = 1 +/- c, one packed chain while
                            // both lambdas go on; pt: the one that goes on beyond KLO
                            float2 PP[KLO + 1];
                            if (NARROW) {
                                const float c = (a.x * b.x + a.y * b.y + a.z * b.z) *
                                                ((NETA <= 2) ? pa4.z * pb4.z : w.ninv[j] * w.ninv[k]);
                                PP[0] = fma2(f2(c, c), f2(1.f, -1.f), f2(1.f, 1.f));
#pragma unroll
                                for (int kk = 1; kk <= KLO; ++kk) PP[kk] = mul2(PP[kk - 1], PP[kk - 1]);
                            } else {
                                // wide kind, accurate b: with unit vectors, 1 - c = |u_j - u_k|^2 / 2 and
                                // 1 + c = |u_j + u_k|^2 / 2 (times 1 + g_j + g_k for the norm defects),
                                // each to about an ulp of its own size, without forming c.  b = 2 -
                                // the other one (bl = the rounding of that subtraction, exact): where
                                // cos -> +-1 and b -> 2 the other one is small and accurate, so b is
                                // exact to first order; a small b carries ~2 ulp absolute, which is
                                // what its terms need in a sum dominated by b near 2.  A power
                                // b^(2^k) amplifies b's relative error 2^k times: the top power
                                // (zeta up to 16) gets the first-order term 2^k bl b^(2^k - 1).
                                const float2 wx = fma2(f2(b.x, b.x), f2(-1.f, 1.f), f2(a.x, a.x));
                                const float2 wy = fma2(f2(b.y, b.y), f2(-1.f, 1.f), f2(a.y, a.y));
                                const float2 wz = fma2(f2(b.z, b.z), f2(-1.f, 1.f), f2(a.z, a.z));
                                float2 n2 = mul2(wx, wx);
                                n2 = fma2(wy, wy, n2);
                                n2 = fma2(wz, wz, n2);
                                const float gg = a.w + b.w;
                                const float2 hf = mul2(n2, f2(0.5f, 0.5f));
                                const float2 sm = fma2(hf, f2(gg, gg), hf);              // (1 - c, 1 + c)
                                PP[0] = fma2(sm, f2(-1.f, -1.f), f2(2.f, 2.f));          // (1 + c, 1 - c)
                                const float2 bl = fma2(sm, f2(-1.f, -1.f), fma2(PP[0], f2(-1.f, -1.f), f2(2.f, 2.f)));
                                float2 T = PP[0];
#pragma unroll
                                for (int kk = 1; kk <= KLO; ++kk) {
                                    PP[kk] = mul2(PP[kk - 1], PP[kk - 1]);
                                    if (kk < KLO) T = mul2(T, PP[kk]);
                                }
                                if (KLO >= 2) {
                                    const float sc = (float)(1 << KLO);
                                    PP[KLO] = fma2(T, mul2(bl, f2(sc, sc)), PP[KLO]);
                                }
                            }
                            float pt[KM - KLO + 1];
                            {
                                float x = TX ? PP[KLO].x : PP[KLO].y;
#pragma unroll
                                for (int kk = KLO + 1; kk <= KM; ++kk) {
                                    x *= x;
                                    pt[kk - KLO - 1] = x;
                                }
                            }
                            // R_q = P_q(r_ij) P_q(r_ik) (P_q(r_jk) f_c(r_jk) for the narrow kind)
                            float Rq[NQ];
                            if constexpr (NETA % 2 == 0) {
                                // even eta count: both of a pair in one packed instruction
#pragma unroll
                                for (int p = 0; p < NP; ++p) {
                                    float2 R = mul2(PA[p], PB[p]);
                                    if (NARROW) {
                                        const float2 x2 = f2(rd2, rd2);
                                        const float2 arg = fma2(KH[p], x2, mul2(KL[p], x2));
                                        R = mul2(R, mul2(f2(exp2f(arg.x), exp2f(arg.y)), f2(fcd, fcd)));
                                    }
                                    if (straight) R = mul2(R, f2(vz, vz));
                                    Rq[2 * p] = R.x;
                                    Rq[2 * p + 1] = R.y;
                                }
                            } else {
                                // odd eta count: a padded pair would cost more than it saves
#pragma unroll
                                for (int q = 0; q < NQ; ++q) {
                                    const float2 pa = PA[q >> 1], pb = PB[q >> 1];
                                    float R = (q & 1) ? pa.y * pb.y : pa.x * pb.x;
                                    if (NARROW) R *= gauss2(khi[q], klo[q], rd2) * fcd;
                                    Rq[q] = straight ? R * vz : R;
                                }
                            }
#pragma unroll
                            for (int q = 0; q < NQ; ++q) {
                                const float2 R2 = f2(Rq[q], Rq[q]);
#pragma unroll
                                for (int kk = 0; kk <= KLO; ++kk) accL[q][kk] = fma2(PP[kk], R2, accL[q][kk]);
#pragma unroll
                                for (int kk = KLO + 1; kk <= KM; ++kk)
                                    accT[q][kk - KLO - 1] = fmaf(pt[kk - KLO - 1], Rq[q], accT[q][kk - KLO - 1]);
                            }
                        }
                    }
                    __syncwarp();
                    // the leftover (fewer than 32) moves to the front of the queue
                    const int left = avail - take;
                    const unsigned short lv = (lane < left) ? w.queue[take + lane] : (unsigned short)0;
                    __syncwarp();
                    if (lane < left) w.queue[lane] = lv;
                    __syncwarp();
                    pend = left;
                    done += take;
                }
            }
            if (rec && lane == 0) rec[3] = (unsigned short)done;
            // lane partials: compensated reduce-scatter of the accumulators in use, per eta
            // the KP + 1 of lambda = +1 then the KN + 1 of lambda = -1, 32 at a time (a lane
            // gets one accumulator, or none); prefactor 2^(1 - zeta), zeta = 2^k
            constexpr int PER = KP + KN + 2, NAC = NQ * PER;
            static_assert(NAC <= 64, "at most two rounds of 32 accumulators");
#pragma unroll
            for (int c0 = 0; c0 < NAC; c0 += 32) {
                float v[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int idx = c0 + t, q = idx / PER, r = idx % PER;
                    const int l = (r <= KP) ? 0 : 1, kk = (r <= KP) ? r : r - (KP + 1);
                    float a = 0.f;
                    if (idx < NAC) {
                        if (kk <= KLO) a = (l == 0) ? accL[q][kk].x : accL[q][kk].y;
                        else a = accT[q][kk - KLO - 1];   // the one lambda that goes on beyond KLO
                    }
                    v[t] = a;
                }
                int slot;
                const float2 tot = (c0 == 0) ? warp_reduce_scatter_n<(NAC < 32 ? NAC : 32)>(v, lane, slot)
                                             : warp_reduce_scatter_n<(NAC > 32 ? NAC - 32 : 1)>(v, lane, slot);
                const int idx = c0 + slot;
                if (slot >= 0 && idx < NAC) {
                    const int q = idx / PER, r = idx % PER;
                    const int l = (r <= KP) ? 0 : 1, kk = (r <= KP) ? r : r - (KP + 1);
                    const int o = (q < E.n_eta) ? E.ang_out[cls][q][l][kk] : -1;
                    const float sc = exp2f((float)(1 - (1 << kk)));   // a power of two: exact
                    if (o >= 0) sG[o] = make_float2(tot.x * sc, tot.y * sc);
                }
            }
            if (cls == 0 && lane == 2) cnt += (unsigned long long)M * (M - 1) / 2;
            if (rec) qcur += (unsigned)((q0 + done + 7) >> 3);   // q0 is a multiple of 8
        }
        if (NETA == 0 && qoff && lane == 0) qoff[i] = QOFF_NONE;
        __syncwarp();
        for (int s = lane; s < E.n_g; s += 32) {
            // G~ = (G - mu) / s with G = hi + lo: the difference exact (TwoSum), one
            // final rounding
            const float2 g = sG[s];
            float dh, dl;
            two_sum(g.x, -E.mu[s], dh, dl);
            dl += g.y;
            Gs[(size_t)i * P.gs + s] = fmaf(dh, E.inv_s[s], dl * E.inv_s[s]);
            if (Graw) Graw[(size_t)i * E.n_g + s] = g.x + g.y;
        }
        __syncwarp();
        if (lane == 0) cnt += (unsigned long long)n_list;
        if (lane == 1) cnt += (unsigned long long)M;
        if (lane == 3) cnt = max(cnt, (unsigned long long)n_list);
        if (lane == 4) cnt = max(cnt, (unsigned long long)M);
    }
    // counters: one atomic per counter and warp
    unsigned long long t = c_trip;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) atomicAdd(&counters[CNT_LIST], cnt);
    if (lane == 1) atomicAdd(&counters[CNT_RC], cnt);
    if (lane == 2) atomicAdd(&counters[CNT_PAIRS], cnt);
    if (lane == 3) atomicMax(&counters[CNT_MAXLIST], cnt);
    if (lane == 4) atomicMax(&counters[CNT_MAXRC], cnt);
    if (lane == 0) {
        atomicAdd(&counters[CNT_TRIPLETS], t);
        if (c_spill) atomicAdd(&counters[CNT_SPILL], c_spill);
    }
    // positive floats order like their bits: the largest complement is the closest pair
    if (lane == 0 && *s_r2min < INFINITY)
        atomicMax(&counters[CNT_MINR], 0xffffffffull - (unsigned long long)__float_as_uint(sqrtf(*s_r2min)));
}

// ---------------------------------------------------------------- force pass
// g[i, slot] = dE_i/dd_ij for each list slot (0 outside the cutoff), Fown[i] =
// sum_j g_ij (the force on i from its own energy), per-warp virial partials.
// STORED (main pass): the pair queues come from the descriptor pass's records;
// an atom without a valid record is appended to the wide-capacity list, whose
// pass (STORED = false) rebuilds the queue from the live masks.
// HOT: the form of the MD step's force pass (stored queues, the descriptor pass's
// staged neighbours, 64-bit fixed-point force atomics, no virial): the other
// forms' code compiled out, which the step's launches measured 2.5 % faster.
template <int NETA, bool NARROW, int KP, int KN, bool STORED, bool RES, bool HOT = false>
__global__ void __launch_bounds__(128, 5)
k_force(int n, const float4* __restrict__ pos4, Box bx, NbView nv, const Plan* __restrict__ plan_g, int C,
        const float* __restrict__ dEdG, float4* __restrict__ gbuf, float4* __restrict__ Fown,
        double* __restrict__ vir_part, int n_vir, int* __restrict__ flags, int* __restrict__ spill, int pass,
        const unsigned short* __restrict__ qpool, const unsigned int* __restrict__ qoff,
        float* __restrict__ Fscat, unsigned long long* __restrict__ Fq, const float4* __restrict__ stg,
        size_t stg_plane, unsigned long long qcap)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Plan& P = *plan_g;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    constexpr bool PACK = NETA <= 2;
    const size_t wbytes = force_warp_bytes(C, nv.stride, PACK, RES, STORED);
    unsigned char* base = smem + wbytes * wib;
    WarpSmem w;
    w.nd = reinterpret_cast<float4*>(base);
    w.npf = w.nd + C;
    w.ndp = PACK ? nullptr : w.npf + C;
    w.sgh = reinterpret_cast<int*>(w.npf + (PACK ? C : 2 * C));
    w.sgl = w.sgh + 3 * C;
    float* sW = reinterpret_cast<float*>(w.sgl + 3 * C);
    bool fx_bad = false;   // a contribution outside the fixed-point range (or not finite)
    w.queue = reinterpret_cast<unsigned short*>(sW + NNP_MAXG);
    w.cmap = reinterpret_cast<short*>(w.queue + PAIR_QUEUE);
    w.nel = RES ? reinterpret_cast<unsigned char*>(w.cmap + nv.stride) : nullptr;
    {
        unsigned char* harea = reinterpret_cast<unsigned char*>(w.cmap + nv.stride) + (RES ? ((C + 15) & ~15) : 0);
        w.nh = STORED ? nullptr : reinterpret_cast<float*>(harea);
        w.jidx = STORED ? reinterpret_cast<int*>(harea) : nullptr;
    }
    // the main pass over stored queues reads the descriptor pass's staged
    // neighbours instead of staging them again (stg; at most 2 eta)
    const bool staged = STORED && PACK && (HOT || stg != nullptr);
    w.rtab = reinterpret_cast<float4*>(w.queue);
    w.rw = reinterpret_cast<float*>(w.rtab + NNP_MAXRAD);
    w.ninv = nullptr;
    w.nrad = nullptr;

    // virial sums of the warp's atoms (FP64, in shared memory: registers stay free
    // for the pair loop)
    double* vir = reinterpret_cast<double*>(base + wbytes - 80);
    if (lane < 9) vir[lane] = 0.0;
    const int nw = gridDim.x * wpb;
    const int n_items = atom_count(pass, n, spill);
    unsigned long long c_spill = 0;
    AtomWalk walk{pass == 0 ? flags + FLAG_WALK_FORCE : nullptr, (int)blockIdx.x * wpb + wib, nw, n_items, lane};
    // the next atom's record offset and first 32 dE/dG, loaded during this atom
    // (they otherwise wait on DRAM at the atom's start; -0.4 % on 2M water)
    int it_pf = -1;
    unsigned o_pf = 0u;
    float dE_pf = 0.f;
    for (int it = walk.first(); it < n_items; it = walk.next(it)) {
        const int i = atom_at(pass, it, spill, nv.order);
        const bool pf = staged && it == it_pf;
        const unsigned o_car = o_pf;
        // the first round of the atom's staged records (lane < C: inside its slab of
        // the planes, whatever its M) loads beside dE/dG and the record lookup;
        // later rounds one round ahead (0.7 % off the water force pass)
        float4 sa = make_float4(0.f, 0.f, 0.f, 0.f), sp = sa, sx = sa;
        if (staged && lane < C) {
            const size_t b0 = (size_t)i * C + lane;
            sa = stg[b0];
            sp = stg[stg_plane + b0];
            sx = stg[2 * stg_plane + b0];
        }
        const float4 pi = pos4[i];
        const int ti = __float_as_int(pi.w);
        const ElemPlan& E = P.e[ti];
        for (int s = lane; s < E.n_g; s += 32) sW[s] = (pf && s < 32) ? dE_pf : dEdG[(size_t)i * P.gs + s];
        __syncwarp();
        for (int rr = lane; rr < E.n_rad; rr += 32) {
            w.rtab[rr] = make_float4(E.rad_khi[rr], E.rad_klo[rr], E.rad_rs[rr], -2.0f * E.rad_eta[rr]);
            w.rw[rr] = sW[E.rad_out[rr]];
        }
        __syncwarp();
        float khi[4], klo[4], etav[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            etav[q] = (q < E.n_eta) ? E.ang_eta[q] : 0.f;
            khi[q] = (q < E.n_eta) ? E.ang_khi[q] : 0.f;
            klo[q] = (q < E.n_eta) ? E.ang_klo[q] : 0.f;
        }
        int n_list = 0;
        unsigned sig = 0u;
        int M;
        // largest 1/r of the staged neighbours (for the range bound below): taken
        // while staging from stored records (-0.45 %), else in a loop of its own
        float iam = 0.f;
        bool nonfin = false;
        const unsigned short* rec = nullptr;
        // the queue record of this warp's next atom goes to L2 once its offset has
        // arrived (after this atom's staging); the force pass reads records round by
        // round, so their first reads would otherwise wait on DRAM (prefetching the
        // next atom's staged neighbours as well measured slower)
        unsigned o_next = QOFF_NONE;
        const int it_next = walk.peek(it);
        if (staged && it_next >= 0) {
            const int in = atom_at(pass, it_next, spill, nv.order);
            o_next = qoff[in];
            if (lane < P.gs) dE_pf = dEdG[(size_t)in * P.gs + lane];
        }
        it_pf = it_next;
        o_pf = o_next;
        if (staged) {
            // the descriptor pass's staging of this atom; its queue record gives M
            const unsigned o = (NETA > 0) ? (pf ? o_car : qoff[i]) : QOFF_NONE;
            if (o == QOFF_SPILLED) continue;   // the descriptor pass queued it already
            if (o == QOFF_NONE) {               // no record (pool full): the wide pass takes it
                if (lane == 0) spill[1 + atomicAdd(spill, 1)] = i;
                continue;
            }
            rec = qpool + (size_t)o * 8;
            M = rec[0];
            if (FxU<NARROW>::CARRY && M > FX_MAXADDS) {   // a slot could take more adds than a low word holds
                if (lane == 0) spill[1 + atomicAdd(spill, 1)] = i;
                continue;
            }
            const size_t base = (size_t)i * C;
            for (int m = lane; m < M; m += 32) {
                const float4 a = sa, pq = sp, ax = sx;
                if (m + 32 < M) {
                    const size_t bn = base + m + 32;
                    sa = stg[bn];
                    sp = stg[stg_plane + bn];
                    sx = stg[2 * stg_plane + bn];
                }
                w.nd[m] = a;
                iam = fmaxf(iam, a.w);
                nonfin |= !(a.w < INFINITY);
                w.npf[m] = pq;
                const int jj = __float_as_int(ax.w);
                w.jidx[m] = jj & (int)NB_INDEX_MASK;
                radial_g<NARROW>(w, P, E, m, ax.x, a.w, ax.y, ax.z, (int)((unsigned)jj >> 24), a.x, a.y, a.z, flags);
            }
            if (o_next < QOFF_SPILLED) {   // up to 4 KB of the record, inside the pool
                const unsigned long long e0 = (unsigned long long)o_next * 8;
                const unsigned long long e1 = e0 + 2048 < qcap ? e0 + 2048 : qcap;
                if (e1 > e0) prefetch_l2(qpool + e0, (size_t)(e1 - e0) * 2, lane);
            }
            __syncwarp();
        } else {
            float r2_unused = 0.f;
            M = stage_neighbors<NETA, true, NARROW>(i, pi, bx, nv, pos4, P, E, khi, klo, etav, C, w, sW, lane, flags,
                                                    n_list, sig, r2_unused);
            if (over_capacity(M, C, pass, i, spill, false, lane, flags, c_spill)) continue;
        }
        const int nb = (M + 31) >> 5;
        for (int m = lane; !staged && m < M; m += 32) {
            const float x = w.nd[m].w;
            iam = fmaxf(iam, x);
            nonfin |= !(x < INFINITY);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) iam = fmaxf(iam, __shfl_xor_sync(FULL, iam, o));
        nonfin = __any_sync(FULL, nonfin);
        // the descriptor pass's queue record, used when this staging reproduces it
        if (STORED && NETA > 0 && !staged) {
            const unsigned o = qoff[i];
            if (o != QOFF_NONE && o != QOFF_SPILLED) {
                const unsigned short* r = qpool + (size_t)o * 8;
                if (r[0] == (unsigned short)M && r[1] == (unsigned short)(sig & 0xffffu) &&
                    r[2] == (unsigned short)(sig >> 16) && !(FxU<NARROW>::CARRY && M > FX_MAXADDS))
                    rec = r;
            }
            if (!rec) {
                if (lane == 0) spill[1 + atomicAdd(spill, 1)] = i;
                continue;
            }
        }
        const int ncls = RES ? E.n_cls : 1;
        for (int cls = 0; NETA > 0 && cls < ncls; ++cls) {
            // dense weights dE/dG_o * 2^(1-zeta), zeta = 2^k: WL[q][k] = (lambda = +1,
            // lambda = -1) for k <= KLO, WT[q][k - KLO - 1] for the one lambda whose
            // functions reach k > KLO (TX: lambda = +1); eta constants as pairs
            // (q = 2p, 2p + 1; zero past n_eta)
            constexpr int NQ = NETA > 0 ? NETA : 1, NP = (NQ + 1) / 2;
            constexpr int KLO = KP < KN ? KP : KN, KM = KP > KN ? KP : KN;
            constexpr bool TX = KP > KN;
            float2 WL[NQ][KLO + 1];
            float WT[NQ][KM - KLO + 1];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int kk = 0; kk <= KM; ++kk) {
                    const int op = (q < E.n_eta && kk <= KP) ? E.ang_out[cls][q][0][kk] : -1;
                    const int om = (q < E.n_eta && kk <= KN) ? E.ang_out[cls][q][1][kk] : -1;
                    // 2^(1 - zeta) as its bit pattern (kk is a constant here: the factor folds)
                    const float sc = __int_as_float((127 + 1 - (1 << kk)) << 23);
                    const float wp = (op >= 0) ? sW[op] * sc : 0.f, wm = (om >= 0) ? sW[om] * sc : 0.f;
                    if (kk <= KLO) WL[q][kk] = f2(wp, wm);
                    else WT[q][kk - KLO - 1] = TX ? wp : wm;
                }
            float2 KH[NP], KL[NP], ET[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                KH[p] = f2(khi[2 * p], (2 * p + 1 < 4) ? khi[2 * p + 1] : 0.f);
                KL[p] = f2(klo[2 * p], (2 * p + 1 < 4) ? klo[2 * p + 1] : 0.f);
                ET[p] = f2(-2.0f * etav[2 * p], (2 * p + 1 < 4) ? -2.0f * etav[2 * p + 1] : 0.f);
            }
            // A bound on every triplet contribution of this atom and class: with
            // b = 1 +/- c <= 2, |b^zeta| <= 2^zeta and |d b^zeta / dc| <= zeta 2^(zeta-1);
            // P <= 1 and |dP/dr| <= pi/(2 rc) + 2 eta rc for every neighbour and (narrow)
            // for r_jk < rc; so |phia|, |phib|, |phid| <= sum_q Smax_q Qmax_q, |phic| <=
            // sum_q Dmax_q, and each component of g_a, g_b is at most |phia| + 2 |phic| /
            // r_min + |phid|.  The per-triplet range test runs only when the bound (with a
            // factor 2 of margin) does not hold or is not finite.
            float bnd = 0.f;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                float sm = 0.f, dm = 0.f;
#pragma unroll
                for (int kk = 0; kk <= KM; ++kk) {
                    const float a = (kk <= KLO) ? fabsf(WL[q][kk].x) + fabsf(WL[q][kk].y) : fabsf(WT[q][kk - KLO - 1]);
                    sm += a * (float)(1 << (1 << kk));
                    dm += a * (float)(1 << (kk + (1 << kk) - 1));
                }
                const float qm = P.hpi_rc + 2.f * etav[q] * P.rc;
                bnd += sm * qm * (NARROW ? 2.f : 1.f) + 2.f * iam * dm;
            }
            const bool exact = nonfin || !(bnd < 0.5f * FX_LIMIT);
            // the same weights as eta pairs (q = 2p, 2p + 1) per lambda and k, for the
            // packed sums S and D of the triplet loop; D's k = 0 terms are constant
            constexpr bool QPAIR = NQ % 2 == 0;   // odd counts keep the lambda-pair sums
            float2 WPp[QPAIR ? NP : 1][KP + 1], WPm[QPAIR ? NP : 1][KN + 1], D0[QPAIR ? NP : 1];
#pragma unroll
            for (int p = 0; QPAIR && p < NP; ++p) {
#pragma unroll
                for (int kk = 0; kk <= KP; ++kk) {
                    float w2[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q = 2 * p + h;
                        w2[h] = (q >= NQ) ? 0.f : (kk <= KLO ? WL[q < NQ ? q : 0][kk].x : (TX ? WT[q < NQ ? q : 0][kk - KLO - 1] : 0.f));
                    }
                    WPp[p][kk] = f2(w2[0], w2[1]);
                }
#pragma unroll
                for (int kk = 0; kk <= KN; ++kk) {
                    float w2[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q = 2 * p + h;
                        w2[h] = (q >= NQ) ? 0.f : (kk <= KLO ? WL[q < NQ ? q : 0][kk].y : (!TX ? WT[q < NQ ? q : 0][kk - KLO - 1] : 0.f));
                    }
                    WPm[p][kk] = f2(w2[0], w2[1]);
                }
                D0[p] = add2(WPp[p][0], mul2(WPm[p][0], f2(-1.f, -1.f)));
            }
            const int ce1 = RES ? E.cls_e1[cls] : -1, ce2 = RES ? E.cls_e2[cls] : -1;
            // STORED: one sweep over the record's entries (every block pair, back to
            // back, as j | k << 8); otherwise one 32 x 32 block pair at a time.
            for (int A = 0; A < (STORED ? 1 : nb); ++A) {
                const int jl = 32 * A + lane;
                const float4 al = (jl < M) ? w.nd[jl] : make_float4(0.f, 0.f, 0.f, 0.f);
                const int ej = (RES && jl < M) ? (int)w.nel[jl] : -1;
                for (int B = A; B < (STORED ? 1 : nb); ++B) {
                    int total;
                    const unsigned short* qsrc;
                    if (STORED) {
                        total = rec[3];
                        qsrc = rec + queue_entries_start(nb);
                    } else {
                        unsigned mask = live_mask<NARROW, 1>(A, B, lane, M, al, (jl < M) ? w.nh[jl] : 0.f, w.nd, w.nh);
                        if (RES && ce1 >= 0) {
                            const int kl = 32 * B + lane;
                            mask &= class_mask(ej, kl < M ? (int)w.nel[kl] : -1, ce1, ce2, lane);
                        }
                        total = enqueue_block(mask, lane, w.queue, A == B);
                        qsrc = w.queue;
                    }
                    // stored queues come from global memory: load one round ahead
                    int ent_next = (STORED && lane < total) ? qsrc[lane] : 0;
                    auto batch = [&](auto tail, auto exact_t, int e0) {
                        constexpr bool TAIL = decltype(tail)::value, EXACT = decltype(exact_t)::value;
                        const int e = e0 + lane;
                        int ent;
                        if (STORED) {
                            ent = ent_next;
                            ent_next = (e + 32 < total) ? qsrc[e + 32] : 0;
                        }
                        if (!TAIL || e < total) {
                            int j, k;
                            if (STORED) {
                                j = ent & 255;
                                k = ent >> 8;
                            } else {
                                ent = qsrc[e];
                                const int l = ent & 31, s = ent >> 5;
                                j = 32 * A + l;
                                k = 32 * B + ((l + s) & 31);
                            }
                            const float4 a = w.nd[j], b = w.nd[k];
                            const float ia = a.w, ib = b.w;
                            // P_q and dP_q/dr of both neighbours as eta pairs (zero past NETA)
                            float2 PA[NP], QA[NP], PB[NP], QB[NP];
                            if (PACK) {
                                const float4 pa4 = w.npf[j], pb4 = w.npf[k];
                                PA[0] = f2(pa4.x, pa4.y); QA[0] = f2(pa4.z, pa4.w);
                                PB[0] = f2(pb4.x, pb4.y); QB[0] = f2(pb4.z, pb4.w);
                            } else {
                                const float4 pa4 = w.npf[j], qa4 = w.ndp[j], pb4 = w.npf[k], qb4 = w.ndp[k];
                                PA[0] = f2(pa4.x, pa4.y); QA[0] = f2(qa4.x, qa4.y);
                                PB[0] = f2(pb4.x, pb4.y); QB[0] = f2(qb4.x, qb4.y);
                                if (NP > 1) {
                                    PA[NP - 1] = f2(pa4.z, pa4.w); QA[NP - 1] = f2(qa4.z, qa4.w);
                                    PB[NP - 1] = f2(pb4.z, pb4.w); QB[NP - 1] = f2(qb4.z, qb4.w);
                                }
                            }
                            const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
                            const float c = (a.x * b.x + a.y * b.y + a.z * b.z) * (ia * ib);
                            float fcd = 1.f, dfcd = 0.f, rd2 = 0.f, rd = 1.f, ird = 0.f;
                            if (NARROW) {
                                rd2 = ex * ex + ey * ey + ez * ez;
                                ird = rsqrtf(rd2);
                                rd = rd2 * ird;
                                cutoff_fn_fast(rd, P.hpi_rc, fcd, dfcd);
                            }
                            // PW[k] = (b_+^(2^k), b_-^(2^k)), QS[k] = d PW[k] / dc, b_(+/-) = 1 +/- c
                            // (both lambdas in one packed chain up to KLO, then the one that goes on;
                            // shared by every eta)
                            float2 PW[KLO + 1], QS[KLO + 1];
                            PW[0] = fma2(f2(c, c), f2(1.f, -1.f), f2(1.f, 1.f));
                            QS[0] = f2(1.f, -1.f);
                            float2 QK = PW[0];
#pragma unroll
                            for (int kk = 1; kk <= KLO; ++kk) {
                                if (kk > 1) QK = mul2(QK, PW[kk - 1]);
                                PW[kk] = mul2(PW[kk - 1], PW[kk - 1]);
                                QS[kk] = mul2(QK, f2((float)(1 << kk), -(float)(1 << kk)));
                            }
                            float pt[KM - KLO + 1], qt[KM - KLO + 1];
                            {
                                float pw = TX ? PW[KLO].x : PW[KLO].y;
                                float qk = TX ? QK.x : QK.y;
#pragma unroll
                                for (int kk = KLO + 1; kk <= KM; ++kk) {
                                    if (kk > 1) qk *= pw;
                                    pw *= pw;
                                    pt[kk - KLO - 1] = pw;
                                    qt[kk - KLO - 1] = qk * (TX ? (float)(1 << kk) : -(float)(1 << kk));
                                }
                            }
                            // (S_2p, S_2p+1) = sum W b^zeta and D = dS/dc as eta pairs
                            float2 SP[NP], DP[NP];
                            if constexpr (QPAIR) {
#pragma unroll
                            for (int p = 0; p < NP; ++p) {
                                float2 s2 = f2(0.f, 0.f), d2 = D0[p];
#pragma unroll
                                for (int kk = 0; kk <= KP; ++kk) {
                                    const float bp = (kk <= KLO) ? PW[kk].x : pt[kk - KLO - 1];
                                    s2 = fma2(WPp[p][kk], f2(bp, bp), s2);
                                    if (kk > 0) {
                                        const float dp = (kk <= KLO) ? QS[kk].x : qt[kk - KLO - 1];
                                        d2 = fma2(WPp[p][kk], f2(dp, dp), d2);
                                    }
                                }
#pragma unroll
                                for (int kk = 0; kk <= KN; ++kk) {
                                    const float bm = (kk <= KLO) ? PW[kk].y : pt[kk - KLO - 1];
                                    s2 = fma2(WPm[p][kk], f2(bm, bm), s2);
                                    if (kk > 0) {
                                        const float dm = (kk <= KLO) ? QS[kk].y : qt[kk - KLO - 1];
                                        d2 = fma2(WPm[p][kk], f2(dm, dm), d2);
                                    }
                                }
                                SP[p] = s2;
                                DP[p] = d2;
                            }
                            } else {
                            // odd eta count: S_q = sum W pw, D_q = dS_q/dc (lambda pairs summed at the end)
                            float Sq[2 * NP], Dq[2 * NP];
#pragma unroll
                            for (int q = 0; q < 2 * NP; ++q) {
                                Sq[q] = 0.f;
                                Dq[q] = 0.f;
                                if (q < NQ) {
                                    float2 s2 = mul2(WL[q][0], PW[0]), d2 = mul2(WL[q][0], QS[0]);
#pragma unroll
                                    for (int kk = 1; kk <= KLO; ++kk) {
                                        s2 = fma2(WL[q][kk], PW[kk], s2);
                                        d2 = fma2(WL[q][kk], QS[kk], d2);
                                    }
                                    float st = TX ? s2.x : s2.y, dt = TX ? d2.x : d2.y;
#pragma unroll
                                    for (int kk = KLO + 1; kk <= KM; ++kk) {
                                        st = fmaf(WT[q][kk - KLO - 1], pt[kk - KLO - 1], st);
                                        dt = fmaf(WT[q][kk - KLO - 1], qt[kk - KLO - 1], dt);
                                    }
                                    Sq[q] = TX ? st + s2.y : s2.x + st;
                                    Dq[q] = TX ? dt + d2.y : d2.x + dt;
                                }
                            }
#pragma unroll
                            for (int p = 0; p < NP; ++p) {
                                SP[p] = f2(Sq[2 * p], Sq[2 * p + 1]);
                                DP[p] = f2(Dq[2 * p], Dq[2 * p + 1]);
                            }
                            }
                            float2 phic2 = f2(0.f, 0.f), phia2 = f2(0.f, 0.f), phib2 = f2(0.f, 0.f), phid2 = f2(0.f, 0.f);
#pragma unroll
                            for (int p = 0; p < NP; ++p) {
                                const float2 S2 = SP[p], D2 = DP[p];
                                const float2 pab = mul2(PA[p], PB[p]);
                                float2 SPd = S2, pabPd = pab;
                                if (NARROW) {
                                    const float2 x2 = f2(rd2, rd2);
                                    const float2 arg = fma2(KH[p], x2, mul2(KL[p], x2));
                                    const float2 ed = f2(exp2f(arg.x), (2 * p + 1 < NQ) ? exp2f(arg.y) : 0.f);
                                    const float2 Pd = mul2(ed, f2(fcd, fcd));
                                    const float rf = rd * fcd;
                                    const float2 dPd = mul2(ed, fma2(ET[p], f2(rf, rf), f2(dfcd, dfcd)));
                                    pabPd = mul2(pab, Pd);
                                    SPd = mul2(S2, Pd);
                                    phid2 = fma2(mul2(S2, pab), dPd, phid2);
                                }
                                phic2 = fma2(D2, pabPd, phic2);
                                phia2 = fma2(mul2(SPd, QA[p]), PB[p], phia2);
                                phib2 = fma2(mul2(SPd, PA[p]), QB[p], phib2);
                            }
                            const float phic = phic2.x + phic2.y, phia = phia2.x + phia2.y;
                            const float phib = phib2.x + phib2.y, phid = phid2.x + phid2.y;
                            // g_a = phic (b/(ra rb) - c a/ra^2) + phia a/ra - phid (b - a)/rd
                            // g_b = phic (a/(ra rb) - c b/rb^2) + phib b/rb + phid (b - a)/rd
                            const float pc = phic * c;
                            const float ua = fmaf(-pc, ia, phia), ub = fmaf(-pc, ib, phib);
                            const float ta = phic * ia, tb = phic * ib;
                            const float cab = ta * ib;
                            const float ca = ua * ia, cb = ub * ib;
                            const float cd = NARROW ? phid * ird : 0.f;
                            // every component of g_a is at most |u_a| + |phic / ra| + |phid| (|a| = ra,
                            // |e| = rd); likewise for g_b
                            if (EXACT)
                                fx_bad |= !(fabsf(ua) + fabsf(ta) + fabsf(phid) < FX_LIMIT &&
                                            fabsf(ub) + fabsf(tb) + fabsf(phid) < FX_LIMIT);
                            // with e = b - a: g_a = (ca + cd) a + (cab - cd) b, g_b = (cab - cd) a +
                            // (cb + cd) b; (x, y) of g_a and of g_b, and (z of g_a, z of g_b), as
                            // packed pairs
                            const float xa = ca + cd, xab = cab - cd, xb = cb + cd;
                            const float2 axy = f2(a.x, a.y), bxy = f2(b.x, b.y);
                            const float2 gaxy = fma2(f2(xa, xa), axy, mul2(f2(xab, xab), bxy));
                            const float2 gbxy = fma2(f2(xab, xab), axy, mul2(f2(xb, xb), bxy));
                            const float2 gz = fma2(f2(xa, xab), f2(a.z, a.z), mul2(f2(xab, xb), f2(b.z, b.z)));
                            // narrow kind: low words always, the high words only when a lane
                            // of the warp has one (a contribution of at least 2^-(FX_HB+1)
                            // eV/A); the wide kind's larger contributions seldom skip them
                            if constexpr (!NARROW) {
                                fx_add2<NARROW>(w, 3 * j + 0, 3 * j + 1, gaxy);
                                fx_add2<NARROW>(w, 3 * k + 0, 3 * k + 1, gbxy);
                                fx_add2<NARROW>(w, 3 * j + 2, 3 * k + 2, gz);
                            } else {
                            const float vm = fmaxf(fmaxf(fmaxf(fabsf(gaxy.x), fabsf(gaxy.y)), fmaxf(fabsf(gbxy.x), fabsf(gbxy.y))),
                                                   fmaxf(fabsf(gz.x), fabsf(gz.y)));
                            const bool small = __all_sync(TAIL ? __activemask() : FULL, vm < 0.5f / (float)(1 << FxU<NARROW>::HB));
                            if (small) {
                                int l0, l1, l2, l3, l4, l5;
                                fx_lo2<NARROW>(gaxy, l0, l1);
                                fx_lo2<NARROW>(gbxy, l2, l3);
                                fx_lo2<NARROW>(gz, l4, l5);
                                atomicAdd(&w.sgl[3 * j + 0], l0);
                                atomicAdd(&w.sgl[3 * j + 1], l1);
                                atomicAdd(&w.sgl[3 * k + 0], l2);
                                atomicAdd(&w.sgl[3 * k + 1], l3);
                                atomicAdd(&w.sgl[3 * j + 2], l4);
                                atomicAdd(&w.sgl[3 * k + 2], l5);
                            } else {
                                fx_add6_split<NARROW>(w.sgh, w.sgl, j, k, gaxy, gbxy, gz);
                            }
                            }
                        }
                    };
                    // full batches without the lane guard (no divergent region, the vote
                    // over the full warp), then the partial one: -1.3 % on water
                    int e0 = 0;
                    // the atom's range test compiled in only where its bound does not hold
                    if (exact) {
                        for (; e0 + 32 <= total; e0 += 32) batch(BTag<false>{}, BTag<true>{}, e0);
                        if (e0 < total) batch(BTag<true>{}, BTag<true>{}, e0);
                    } else {
                        for (; e0 + 32 <= total; e0 += 32) batch(BTag<false>{}, BTag<false>{}, e0);
                        if (e0 < total) batch(BTag<true>{}, BTag<false>{}, e0);
                    }
                    __syncwarp();
                    if (!STORED && FxU<NARROW>::CARRY && 32 * nb + 1 > FX_MAXADDS) {
                        // the slots of blocks A and B took at most 32 adds each: carry.
                        // A slot meets at most nb block pairs: with 32 nb adds and the
                        // radial value within FX_MAXADDS no carry is needed.
                        for (int t = lane; t < 96; t += 32) {
                            if (96 * A + t < 3 * M) fx_carry<NARROW>(w, 96 * A + t);
                            if (B != A && 96 * B + t < 3 * M) fx_carry<NARROW>(w, 96 * B + t);
                        }
                        __syncwarp();
                    }
                }
            }
        }
        __syncwarp();
        // force assembly: with Fq, -g_ij is added into F_j as one 64-bit integer per
        // component (units 2^-LB eV/A, FxU<NARROW>; integer sums do not depend on the order of
        // the atomics, so the forces are reproducible bit for bit); with Fscat, as
        // floats (order-dependent); otherwise g is written per list slot for the
        // gather.  Then the own force and the virial.
        const int cnt = n_list;
        // own force sums (64-bit fixed point): taken in the assembly loop where it
        // reads every slot anyway (one read and conversion per slot, not two)
        long long qx = 0, qy = 0, qz = 0;
        const bool q_done = HOT || (Fq && staged);
        if (q_done) {
            for (int m = lane; m < M; m += 32) {
                const long long gx = fx_get64<NARROW>(w, 3 * m), gy = fx_get64<NARROW>(w, 3 * m + 1),
                                gz = fx_get64<NARROW>(w, 3 * m + 2);
                unsigned long long* fj = Fq + 3 * (size_t)w.jidx[m];
                atomicAdd(fj + 0, (unsigned long long)(-gx));
                atomicAdd(fj + 1, (unsigned long long)(-gy));
                atomicAdd(fj + 2, (unsigned long long)(-gz));
                qx += gx;
                qy += gy;
                qz += gz;
            }
        } else if (!HOT && Fq) {
            const uint32_t* row = nv.nbr + (size_t)i * nv.stride;
            for (int s = lane; s < cnt; s += 32) {
                const int c = w.cmap[s];
                if (c >= 0) {
                    unsigned long long* fj = Fq + 3 * (size_t)(row[s] & NB_INDEX_MASK);
                    atomicAdd(fj + 0, (unsigned long long)(-fx_get64<NARROW>(w, 3 * c)));
                    atomicAdd(fj + 1, (unsigned long long)(-fx_get64<NARROW>(w, 3 * c + 1)));
                    atomicAdd(fj + 2, (unsigned long long)(-fx_get64<NARROW>(w, 3 * c + 2)));
                }
            }
        } else if (!HOT && Fscat) {
            const uint32_t* row = nv.nbr + (size_t)i * nv.stride;
            for (int s = lane; s < cnt; s += 32) {
                const int c = w.cmap[s];
                if (c >= 0) {
                    float* fj = Fscat + 3 * (size_t)(row[s] & NB_INDEX_MASK);
                    atomicAdd(fj + 0, -fx_get<NARROW>(w, 3 * c));
                    atomicAdd(fj + 1, -fx_get<NARROW>(w, 3 * c + 1));
                    atomicAdd(fj + 2, -fx_get<NARROW>(w, 3 * c + 2));
                }
            }
        } else if (!HOT) {
            float4* grow = gbuf + (size_t)i * nv.stride;
            for (int s = lane; s < cnt; s += 32) {
                const int c = w.cmap[s];
                grow[s] = (c >= 0) ? make_float4(fx_get<NARROW>(w, 3 * c), fx_get<NARROW>(w, 3 * c + 1), fx_get<NARROW>(w, 3 * c + 2), 0.f)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float fx = 0.f, fy = 0.f, fz = 0.f, v[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = 0.f;
        // the virial only when the caller asked for it (vir_part != nullptr), and
        // only of the energies of atoms i < n_vir (a domain's owned atoms)
        const bool vir_i = !HOT && vir_part && i < n_vir;
        const bool fq = HOT || Fq;
        for (int m = lane; m < M; m += 32) {
            if (fq && !q_done) {
                qx += fx_get64<NARROW>(w, 3 * m);
                qy += fx_get64<NARROW>(w, 3 * m + 1);
                qz += fx_get64<NARROW>(w, 3 * m + 2);
            }
            if (!fq || vir_i) {
                const float gx = fx_get<NARROW>(w, 3 * m), gy = fx_get<NARROW>(w, 3 * m + 1), gz = fx_get<NARROW>(w, 3 * m + 2);
                if (!fq) {
                    fx += gx; fy += gy; fz += gz;
                }
                if (vir_i) {
                    const float4 d = w.nd[m];
                    v[0] -= d.x * gx; v[1] -= d.x * gy; v[2] -= d.x * gz;
                    v[3] -= d.y * gx; v[4] -= d.y * gy; v[5] -= d.y * gz;
                    v[6] -= d.z * gx; v[7] -= d.z * gy; v[8] -= d.z * gz;
                }
            }
        }
        if (vir_i) {
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float t = warp_sum(v[q]);
                if (lane == q) vir[q] += (double)t;
            }
        }
        if (fq) {
            // reduce-scatter of the three sums: lanes 0, 8, 16 end with x, y, z
            // (6 exchanges instead of 3 x 5)
            const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
            long long a0 = (u16 ? qz : qx) + __shfl_xor_sync(FULL, u16 ? qx : qz, 16);
            long long a1 = (u16 ? 0ll : qy) + __shfl_xor_sync(FULL, u16 ? qy : 0ll, 16);
            a0 = (u8 ? a1 : a0) + __shfl_xor_sync(FULL, u8 ? a0 : a1, 8);
            a0 += __shfl_xor_sync(FULL, a0, 4);
            a0 += __shfl_xor_sync(FULL, a0, 2);
            a0 += __shfl_xor_sync(FULL, a0, 1);
            if ((lane & 7) == 0 && lane < 24) atomicAdd(Fq + 3 * (size_t)i + (lane >> 3), (unsigned long long)a0);
        } else {
            fx = warp_sum(fx); fy = warp_sum(fy); fz = warp_sum(fz);
        }
        if (lane == 0 && !fq) {
            if (Fscat) {
                atomicAdd(Fscat + 3 * (size_t)i + 0, fx);
                atomicAdd(Fscat + 3 * (size_t)i + 1, fy);
                atomicAdd(Fscat + 3 * (size_t)i + 2, fz);
            } else {
                Fown[i] = make_float4(fx, fy, fz, 0.f);
            }
        }
        __syncwarp();
    }
    if (__any_sync(FULL, fx_bad) && lane == 0) atomicOr(&flags[FLAG_ERR], ERR_RANGE);
    __syncwarp();
    if (!HOT && vir_part && lane < 9) vir_part[(size_t)(blockIdx.x * wpb + wib) * 9 + lane] = vir[lane];
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
