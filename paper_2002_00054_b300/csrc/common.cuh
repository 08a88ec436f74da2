// common.cuh -- device-side model plan, error bits and small helpers shared by
// the kernels of the NNP hot path (one translation unit: nnp_capi.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define NNP_MAXE 8      // elements
#define NNP_MAXG 64     // descriptors per element
#define NNP_MAXRAD 64   // radial descriptors per element
#define NNP_MAXETA 4    // distinct angular eta per element
#define NNP_KMAX 4      // angular zeta = 2^k, k <= NNP_KMAX
#define NNP_MAXCLS 10   // neighbour-element pair classes of angular descriptors per element
#define NNP_MAXL 6      // weight layers
#define NNP_MAXH 32     // hidden width

#define WARP 32
#define FULL 0xffffffffu

// error word bits (flags[FLAG_ERR]) and their status mapping
#include "error_word.h"

#define FLAG_ERR 0
#define FLAG_REBUILD 1
// atom counters of the descriptor and force kernels' main passes (cleared by the
// host before every evaluation, see AtomWalk)
#define FLAG_WALK_SF 2
#define FLAG_WALK_FORCE 3

// work counters (counters[])
#define CNT_LIST 0
#define CNT_RC 1
#define CNT_PAIRS 2
#define CNT_TRIPLETS 3
#define CNT_MAXLIST 4   // largest neighbour-list row seen by the call
#define CNT_MAXRC 5     // largest count of neighbours inside the cutoff
#define CNT_SPILL 6     // atoms handed to the wide-capacity pass
#define CNT_PER_CALL 7  // counters [0, CNT_PER_CALL) restart with every API call
#define CNT_REBUILDS 7
#define CNT_QTOP 8      // pair-queue pool entries claimed by the current evaluation
#define CNT_LOGSLOT 9   // next energy-log entry of the running nnp_step call
#define CNT_MINR 10     // 0xffffffff - bits(r) of the closest pair within the cutoff (call-wide max)
#define CNT_N 11

#define LOG2E 1.4426950408889634f

// exp(-eta x2) = 2^(k x2) with k = -eta log2(e) given as hi + lo floats, so the
// argument carries no systematic rounding of the constant (|k x2| reaches ~20).
// The hardware exp2 behind exp2f: ~1 ulp, and measured on B300 biased low by
// 0.82 ulp on average over [-20, 0].  Used per triplet (narrow kind), where its
// error enters one term among ~10^3.
__device__ __forceinline__ float gauss2(float khi, float klo, float x2)
{
    return exp2f(fmaf(khi, x2, klo * x2));
}

// n = rint(x) for |x| <= 2^22 and 2^n, both from t = x + 1.5 * 2^23: the float
// sum is rounded to an integer, ties to even, as rintf rounds, and t - 1.5 * 2^23
// is exact.  bits(t) = bits(1.5 * 2^23) + n, and bits(1.5 * 2^23) * 2^23 = 0 mod
// 2^32, so bits(t) * 2^23 + 127 * 2^23 = (n + 127) << 23 (one integer multiply-
// add instead of a conversion, an add and a shift); callers clamp x to [-125, 127].
__device__ __forceinline__ float rint_pow2(float x, float& p2)
{
    const float M = 12582912.0f;
    const float t = x + M;
    p2 = __uint_as_float(__float_as_uint(t) * (1u << 23) + (127u << 23));
    return t - M;
}
__device__ __forceinline__ float2 rint_pow2_2(float2 x, float2& p2)
{
    const float M = 12582912.0f;
    const float2 t = __fadd2_rn(x, make_float2(M, M));
    p2 = make_float2(__uint_as_float(__float_as_uint(t.x) * (1u << 23) + (127u << 23)),
                     __uint_as_float(__float_as_uint(t.y) * (1u << 23) + (127u << 23)));
    return __fadd2_rn(t, make_float2(-M, -M));
}

// 2^x to within ~0.5 ulp with no systematic bias, for the per-neighbour factors
// exp(-eta r^2) f_c(r): every descriptor is a sum of them, and a bias common to
// all terms survives the sum and the scaling G~ = (G - mu)/s, |mu/s| ~ 20 (a
// 1-ulp bias of every term moved FCC per-atom energies by ~1e-5 relative).
// Method: Cody-Waite style reduction x = n + f with n = rint(x), so f is exact
// and |f| <= 1/2; 2^f = e^(f ln 2) by its Taylor series to degree 8 (truncation
// below 2^-32 relative), Horner with FMA; then the exact scaling by 2^n.  The
// coefficients are (ln 2)^k / k!.  Measured on B300 over [-20, 0]: bias
// -0.002 ulp, rms 0.43 ulp, max 1.09 ulp against FP64 (exp2f: -0.82, 0.97, 2.4).
__device__ __forceinline__ float exp2_acc(float x)
{
    x = fminf(fmaxf(x, -125.0f), 127.0f);
    float sc;
    const float n = rint_pow2(x, sc);
    const float f = x - n;
    float p = 1.3215486790144305e-06f;
    p = fmaf(p, f, 1.5252733804059838e-05f);
    p = fmaf(p, f, 1.5403530393381606e-04f);
    p = fmaf(p, f, 1.3333558146428441e-03f);
    p = fmaf(p, f, 9.6181291076284772e-03f);
    p = fmaf(p, f, 5.5504108664821576e-02f);
    p = fmaf(p, f, 2.4022650695910071e-01f);
    p = fmaf(p, f, 6.9314718055994531e-01f);
    p = fmaf(p, f, 1.0f);
    return p * sc;
}
__device__ __forceinline__ float gauss2_acc(float khi, float klo, float x2)
{
    return exp2_acc(fmaf(khi, x2, klo * x2));
}

// Per-element descriptor plan.  Angular functions of one element share one kind
// and are grouped by neighbour-element pair class c and eta: ang_out[c][q][l][k]
// is the descriptor index of (class c, eta_q, lambda = (l == 0 ? +1 : -1),
// zeta = 2^k), or -1.  Class c takes the pairs (j, k) whose elements are
// {cls_e1[c], cls_e2[c]}; cls_e1[c] = -1 takes every pair.
struct ElemPlan {
    int n_g;
    int n_rad;
    float rad_eta[NNP_MAXRAD];
    float rad_khi[NNP_MAXRAD], rad_klo[NNP_MAXRAD];   // -eta log2(e) as hi + lo floats
    float rad_rs[NNP_MAXRAD];
    int rad_elem[NNP_MAXRAD];
    int rad_out[NNP_MAXRAD];
    // radial descriptors are ordered by neighbour element: [0, rad_nall) take every
    // element, [rad_beg[e], rad_end[e]) only element e
    int rad_nall;
    int rad_beg[NNP_MAXE], rad_end[NNP_MAXE];
    int n_eta;
    float ang_eta[NNP_MAXETA];
    float ang_khi[NNP_MAXETA], ang_klo[NNP_MAXETA];   // -eta log2(e) as hi + lo floats
    int n_cls;
    int cls_e1[NNP_MAXCLS], cls_e2[NNP_MAXCLS];
    int ang_out[NNP_MAXCLS][NNP_MAXETA][2][NNP_KMAX + 1];
    float mu[NNP_MAXG];
    float inv_s[NNP_MAXG];
};

struct Plan {
    int n_elem;
    int ang_kind;        // 0 none, 3 narrow, 4 wide (same for every element)
    int n_eta_max;
    int resolved;        // some angular class is restricted to an element pair
    float rc, rc2, hpi_rc;   // cutoff, cutoff^2, pi / (2 rc)
    float inv_2rc, inv_2rc_lo;   // 1 / (2 rc) as hi + lo floats
    // cos(pi k / 64), sin(pi k / 64), k = 0..32, each as hi + lo floats (cospi_dd)
    float4 cs64[33];
    float rcut2;             // (cutoff + skin)^2
    float half_skin2;        // (skin / 2)^2
    float acc_over_m[NNP_MAXE];  // (1 eV/(A amu) in A/fs^2) / mass
    float mass[NNP_MAXE];
    // network: per layer, offsets into one element's block in the shared-memory
    // weight image (row stride ld[l] = in | 1 so both access patterns are
    // bank-conflict free)
    int n_layers;
    int width[NNP_MAXL + 1];
    int ld[NNP_MAXL];
    int s_woff[NNP_MAXL], s_boff[NNP_MAXL];
    int s_elem;              // floats per element in the shared-memory image
    int p_woff[NNP_MAXL], p_boff[NNP_MAXL];  // packed (caller) layout offsets
    int n_params_elem;
    // image of the lane-per-atom FP32 network kernel, per element (floats): hidden
    // layer l: lw_f[l] = W_l^T [in_l][lw_hp] (zero columns past out_l), lw_fb[l] =
    // bias [lw_hp], lw_b[l] = W_l [lw_hp][K_l] (zero rows past out_l and columns past
    // in_l; K_0 = lw_kb0, K_l = lw_hp for l > 0); output layer lw_out = w [lw_kb0
    // or lw_hp], lw_outb = bias; lw_invs = 1/s [lw_kb0].  lw_hp: largest hidden width
    // rounded up to 4; lw_kb0: n_G rounded up to 32; element stride lw_elem = 4 mod
    // 32 words; lw_rows: activation rows per warp (n_G + hidden widths).
    int lw_f[NNP_MAXL], lw_fb[NNP_MAXL], lw_b[NNP_MAXL];
    int lw_out, lw_outb, lw_invs, lw_elem, lw_rows, lw_hp, lw_kb0;
    int gs;                  // row stride of G / dEdG buffers
    ElemPlan e[NNP_MAXE];
};

// f_c(r) = (cos(pi r / rc) + 1) / 2 = cos^2(pi r / (2 rc)); written as a square to
// avoid the cancellation of cos + 1 near r = rc.  Derivative -2 k sin cos, k = pi/(2 rc).
// Per-neighbour factors use the accurate sincospif (about 1 ulp): descriptor
// sums over tens of neighbours are scaled by 1/s with |mu/s| up to ~1e2, so a
// 4e-7 absolute error of the hardware approximation would reach 1e-4 in G~.
// The argument r / (2 rc) uses 1/(2 rc) split into hi + lo floats: a single
// rounded constant biases every cutoff value by ~1e-7 relative in one direction.
__device__ __forceinline__ void cutoff_fn(float r, float inv_2rc, float inv_2rc_lo, float hpi_rc, float& fc, float& dfc)
{
    float s, c;
    sincospif(fmaf(r, inv_2rc, r * inv_2rc_lo), &s, &c);
    fc = c * c;
    dfc = -2.0f * hpi_rc * s * c;
}
// Per-triplet f_c(r_jk) of the narrow angular functions: hardware sin/cos
// (absolute error <= 2^-21.4 on [0, pi/2]), one term among ~10^3 per descriptor.
__device__ __forceinline__ void cutoff_fn_fast(float r, float hpi_rc, float& fc, float& dfc)
{
    float s, c;
    __sincosf(r * hpi_rc, &s, &c);
    fc = c * c;
    dfc = -2.0f * hpi_rc * s * c;
}

// Units of the force pass's fixed-point sums, per angular kind: the high word
// counts 2^-HB eV/A, the low word (and the int64 force sums) 2^-LB eV/A.  The
// narrow kind's coarse high word is zero for contributions below 1/16 eV/A, so a
// warp can skip its atomics; the wide kind keeps the finer low word.
#define FX_HB_NARROW 3
#define FX_LB_NARROW 27
#define FX_HB_WIDE 6
#define FX_LB_WIDE 27

// Packed FP32 pairs (one f32x2 instruction for two IEEE round-to-nearest
// operations; each component is rounded exactly as the scalar operation).
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Double-float ("hi + lo") helpers for the per-neighbour factors of the
// descriptors.  A descriptor is a sum of these factors over tens of neighbours
// and is then scaled as G~ = (G - mu)/s with |mu/s| up to ~20, so an error that
// repeats in every term (a biased function, or the rounding of r entering the
// steep cutoff near r_c) is amplified ~20x in G~; each factor is therefore
// formed to about half an ulp before it is rounded to float once.

// |d|^2 = h + l for a float vector d, exact up to terms of order 2^-48 |d|^2
// (each square split by an FMA, the two sums by TwoSum).
__device__ __forceinline__ void dd_norm2(float x, float y, float z, float& h, float& l)
{
    const float p1 = x * x, e1 = fmaf(x, x, -p1);
    const float p2 = y * y, e2 = fmaf(y, y, -p2);
    const float p3 = z * z, e3 = fmaf(z, z, -p3);
    float s, t1, t2;
    two_sum(p1, p2, s, t1);
    two_sum(s, p3, h, t2);
    l = (e1 + e2 + e3) + (t1 + t2);
}

// 2^(ah + al) for al a small correction of ah (|al| <= ~1e-6 |ah|), to within
// ~0.5 ulp and without bias: as exp2_acc, with the reduced argument
// f = (ah - n) + al (ah - n is exact).
__device__ __forceinline__ float exp2_acc2(float ah, float al)
{
    ah = fminf(fmaxf(ah, -125.0f), 127.0f);
    float sc;
    const float n = rint_pow2(ah, sc);
    const float f = (ah - n) + al;
    float p = 1.3215486790144305e-06f;
    p = fmaf(p, f, 1.5252733804059838e-05f);
    p = fmaf(p, f, 1.5403530393381606e-04f);
    p = fmaf(p, f, 1.3333558146428441e-03f);
    p = fmaf(p, f, 9.6181291076284772e-03f);
    p = fmaf(p, f, 5.5504108664821576e-02f);
    p = fmaf(p, f, 2.4022650695910071e-01f);
    p = fmaf(p, f, 6.9314718055994531e-01f);
    p = fmaf(p, f, 1.0f);
    return p * sc;
}

// exp2_acc2 of two arguments at once: the same operations per component, the
// reduced arguments and the series carried as packed f32x2 pairs (one instruction
// for both), so each result is bitwise the scalar one.
__device__ __forceinline__ float2 exp2_acc2x2(float2 ah, float2 al)
{
    ah.x = fminf(fmaxf(ah.x, -125.0f), 127.0f);
    ah.y = fminf(fmaxf(ah.y, -125.0f), 127.0f);
    float2 sc;
    const float2 n = rint_pow2_2(ah, sc);
    const float2 f = __fadd2_rn(__fadd2_rn(ah, make_float2(-n.x, -n.y)), al);
    float2 p = make_float2(1.3215486790144305e-06f, 1.3215486790144305e-06f);
    p = __ffma2_rn(p, f, make_float2(1.5252733804059838e-05f, 1.5252733804059838e-05f));
    p = __ffma2_rn(p, f, make_float2(1.5403530393381606e-04f, 1.5403530393381606e-04f));
    p = __ffma2_rn(p, f, make_float2(1.3333558146428441e-03f, 1.3333558146428441e-03f));
    p = __ffma2_rn(p, f, make_float2(9.6181291076284772e-03f, 9.6181291076284772e-03f));
    p = __ffma2_rn(p, f, make_float2(5.5504108664821576e-02f, 5.5504108664821576e-02f));
    p = __ffma2_rn(p, f, make_float2(2.4022650695910071e-01f, 2.4022650695910071e-01f));
    p = __ffma2_rn(p, f, make_float2(6.9314718055994531e-01f, 6.9314718055994531e-01f));
    p = __ffma2_rn(p, f, make_float2(1.0f, 1.0f));
    return __fmul2_rn(p, sc);
}

// 2^(ah + al) as h + l to ~2^-27 relative: the same reduction and series, with
// the leading terms 1 + f ln2 carried in double-float (ln 2 as hi + lo).
__device__ __forceinline__ void exp2_dd(float ah, float al, float& h, float& l)
{
    ah = fminf(fmaxf(ah, -125.0f), 127.0f);
    float sc;
    const float n = rint_pow2(ah, sc);
    float f, fl;
    two_sum(ah - n, al, f, fl);   // f + fl = (ah - n) + al exactly
    // q2 = (2^f - 1 - f ln2) / f^2, a float series (its terms are below 0.13 f)
    float q = 1.3215486790144305e-06f;
    q = fmaf(q, f, 1.5252733804059838e-05f);
    q = fmaf(q, f, 1.5403530393381606e-04f);
    q = fmaf(q, f, 1.3333558146428441e-03f);
    q = fmaf(q, f, 9.6181291076284772e-03f);
    q = fmaf(q, f, 5.5504108664821576e-02f);
    q = fmaf(q, f, 2.4022650695910071e-01f);
    const float ln2h = 6.93147182464599609375e-01f, ln2l = -1.9046542999577e-09f;
    const float th = f * ln2h;
    const float tl = fmaf(f, ln2h, -th) + fmaf(f, ln2l, fmaf(fl, ln2h, (f * f) * q));
    const float sh = 1.0f + th;
    const float sl = ((1.0f - sh) + th) + tl;   // |th| < 1: Fast2Sum
    // renormalise, so that h alone is 2^x to within an ulp (|sl| < 0.1 < sh)
    const float rh = sh + sl;
    const float rlo = sl - (rh - sh);
    h = rh * sc;
    l = rlo * sc;
}

// exp2_dd of two arguments at once (packed pairs, each component bitwise the
// scalar result).
__device__ __forceinline__ void exp2_dd2(float2 ah, float2 al, float2& h, float2& l)
{
    ah.x = fminf(fmaxf(ah.x, -125.0f), 127.0f);
    ah.y = fminf(fmaxf(ah.y, -125.0f), 127.0f);
    float2 sc;
    const float2 n = rint_pow2_2(ah, sc);
    // f + fl = (ah - n) + al exactly (TwoSum per component)
    const float2 a = __fadd2_rn(ah, make_float2(-n.x, -n.y));
    const float2 f = __fadd2_rn(a, al);
    const float2 bb = __fadd2_rn(f, make_float2(-a.x, -a.y));
    const float2 t = __fadd2_rn(f, make_float2(-bb.x, -bb.y));
    const float2 fl = __fadd2_rn(__fadd2_rn(a, make_float2(-t.x, -t.y)), __fadd2_rn(al, make_float2(-bb.x, -bb.y)));
    float2 q = make_float2(1.3215486790144305e-06f, 1.3215486790144305e-06f);
    q = __ffma2_rn(q, f, make_float2(1.5252733804059838e-05f, 1.5252733804059838e-05f));
    q = __ffma2_rn(q, f, make_float2(1.5403530393381606e-04f, 1.5403530393381606e-04f));
    q = __ffma2_rn(q, f, make_float2(1.3333558146428441e-03f, 1.3333558146428441e-03f));
    q = __ffma2_rn(q, f, make_float2(9.6181291076284772e-03f, 9.6181291076284772e-03f));
    q = __ffma2_rn(q, f, make_float2(5.5504108664821576e-02f, 5.5504108664821576e-02f));
    q = __ffma2_rn(q, f, make_float2(2.4022650695910071e-01f, 2.4022650695910071e-01f));
    const float2 ln2h = make_float2(6.93147182464599609375e-01f, 6.93147182464599609375e-01f);
    const float2 ln2l = make_float2(-1.9046542999577e-09f, -1.9046542999577e-09f);
    const float2 th = __fmul2_rn(f, ln2h);
    const float2 tl = __fadd2_rn(__ffma2_rn(f, ln2h, make_float2(-th.x, -th.y)),
                                 __ffma2_rn(f, ln2l, __ffma2_rn(fl, ln2h, __fmul2_rn(__fmul2_rn(f, f), q))));
    const float2 one = make_float2(1.0f, 1.0f);
    const float2 sh = __fadd2_rn(one, th);
    const float2 sl = __fadd2_rn(__fadd2_rn(__fadd2_rn(one, make_float2(-sh.x, -sh.y)), th), tl);
    const float2 rh = __fadd2_rn(sh, sl);
    const float2 rd = __fadd2_rn(rh, make_float2(-sh.x, -sh.y));
    const float2 rlo = __fadd2_rn(sl, make_float2(-rd.x, -rd.y));
    h = __fmul2_rn(rh, sc);
    l = __fmul2_rn(rlo, sc);
}

// cos(pi x) as h + l, x = xh + xl in [0, 1/2], to ~2^-28 absolute, and
// sin(pi x) to ~1 ulp: table-driven angle addition (Tang's method) with the
// table cos, sin(pi k / 64) held as hi + lo floats and the reduced angle
// a = pi (x - k/64), |a| <= pi/128, expanded as cos a = 1 - a^2/2 + a^4/24,
// sin a = a - a^3/6 (truncation below 1e-10).
__device__ __forceinline__ void cospi_dd(float xh, float xl, const float4* __restrict__ tab, float& ch, float& cl,
                                         float& sn)
{
    const float kf = rintf(xh * 64.0f);
    const int k = min(max((int)kf, 0), 32);
    const float4 t = tab[k];   // (cos hi, cos lo, sin hi, sin lo)
    const float dd = (xh - (float)k * 0.015625f) + xl;   // xh - k/64 is exact
    const float a = fmaf(dd, -8.742278e-08f, dd * 3.14159274101257324f);   // pi as hi + lo
    const float a2 = a * a;
    const float omc = a2 * fmaf(a2, -4.16666679e-02f, 0.5f);   // 1 - cos a
    const float sna = a * fmaf(a2, -1.66666672e-01f, 1.0f);    // sin a
    // cos(pi x) = C - (C (1 - cos a) + S sin a)
    const float D = fmaf(t.x, omc, t.z * sna) - t.y;
    float e;
    two_sum(t.x, -D, ch, e);
    cl = e;
    sn = t.z + fmaf(t.x, sna, -t.z * omc);
}

// Cutoff f_c(r) = cos^2(pi r / (2 rc)) for r = rh + rl: hi + lo to ~2^-27
// relative where f_c is not tiny, and its derivative dfc (float).
__device__ __forceinline__ void cutoff_dd(float rh, float rl, float inv_2rc, float inv_2rc_lo, float hpi_rc,
                                          const float4* __restrict__ tab, float& fh, float& fl, float& dfc)
{
    const float xh = rh * inv_2rc;
    const float xl = fmaf(rh, inv_2rc, -xh) + fmaf(rh, inv_2rc_lo, rl * inv_2rc);
    float ch, cl, sn;
    cospi_dd(xh, xl, tab, ch, cl, sn);
    fh = ch * ch;
    fl = fmaf(ch, ch, -fh) + 2.0f * ch * cl;
    dfc = -2.0f * hpi_rc * sn * ch;
}

// Reduce-scatter of 32 per-lane float accumulators over the warp with compensated
// (hi + lo) additions: lane t returns the total of v[t] over all lanes, in double.
// 31 exchange steps in all (16 + 8 + 4 + 2 + 1) instead of 32 butterflies.
__device__ __forceinline__ double warp_reduce_scatter32(const float (&v)[32], int lane)
{
    float hi[32], lo[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) hi[t] = v[t];
    {
        // first step: the low words are still zero, so only the high words travel
        const bool upper = (lane & 16) != 0;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const float send_h = upper ? hi[t] : hi[t + 16];
            const float keep_h = upper ? hi[t + 16] : hi[t];
            const float rh = __shfl_xor_sync(FULL, send_h, 16);
            two_sum(keep_h, rh, hi[t], lo[t]);
        }
    }
#pragma unroll
    for (int half = 8; half >= 1; half >>= 1) {
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int t = 0; t < half; ++t) {
            const float send_h = upper ? hi[t] : hi[t + half], send_l = upper ? lo[t] : lo[t + half];
            const float keep_h = upper ? hi[t + half] : hi[t], keep_l = upper ? lo[t + half] : lo[t];
            const float rh = __shfl_xor_sync(FULL, send_h, half), rl = __shfl_xor_sync(FULL, send_l, half);
            float s, e;
            two_sum(keep_h, rh, s, e);
            hi[t] = s;
            lo[t] = keep_l + rl + e;
        }
    }
    return (double)hi[0] + (double)lo[0];
}

// One level of warp_reduce_scatter_n: the K (hi, lo) pairs a lane holds are
// halved; lanes with bit HALF clear keep the first ceil(K/2), the others the rest
// (the missing last one a zero pair), each adding its partner's copy.
template <int HALF, int K>
__device__ __forceinline__ void rs_level(float* hi, float* lo, int lane, int& base, int& cnt)
{
    constexpr int KP = (K + 1) / 2;
    const bool up = (lane & HALF) != 0;
#pragma unroll
    for (int t = 0; t < KP; ++t) {
        const float ah = hi[t], al = lo[t];
        const float bh = (KP + t < K) ? hi[KP + t] : 0.f, bl = (KP + t < K) ? lo[KP + t] : 0.f;
        const float rh = __shfl_xor_sync(FULL, up ? ah : bh, HALF), rl = __shfl_xor_sync(FULL, up ? al : bl, HALF);
        float s, e;
        two_sum(up ? bh : ah, rh, s, e);
        hi[t] = s;
        lo[t] = (up ? bl : al) + rl + e;
    }
    if (up) {
        base += KP;
        cnt -= KP;
    } else {
        cnt = min(cnt, KP);
    }
}

// Reduce-scatter of N <= 32 per-lane values v[0, N) over the warp with
// compensated (hi + lo) additions.  Each of the five levels halves the values a
// lane still holds, so a level costs ceil(K/2) exchanges for K values: 21 in all
// for N = 20, 31 for N = 32.  The first level moves high words only (the low
// words are still zero).  Returns the total over the lanes of v[slot], with
// slot = -1 on the lanes that end with none.
template <int N>
__device__ __forceinline__ float2 warp_reduce_scatter_n(const float (&v)[32], int lane, int& slot)
{
    static_assert(N >= 1 && N <= 32, "1 to 32 values");
    constexpr int K1 = (N + 1) / 2, K2 = (K1 + 1) / 2, K3 = (K2 + 1) / 2, K4 = (K3 + 1) / 2;
    float hi[K1], lo[K1];
    int base = 0, cnt = N;
    {
        const bool up = (lane & 16) != 0;
#pragma unroll
        for (int t = 0; t < K1; ++t) {
            const float a = v[t], b = (K1 + t < N) ? v[K1 + t] : 0.f;
            const float r = __shfl_xor_sync(FULL, up ? a : b, 16);
            two_sum(up ? b : a, r, hi[t], lo[t]);
        }
        if (up) {
            base += K1;
            cnt -= K1;
        } else {
            cnt = min(cnt, K1);
        }
    }
    rs_level<8, K1>(hi, lo, lane, base, cnt);
    rs_level<4, K2>(hi, lo, lane, base, cnt);
    rs_level<2, K3>(hi, lo, lane, base, cnt);
    rs_level<1, K4>(hi, lo, lane, base, cnt);
    slot = cnt > 0 ? base : -1;
    return make_float2(hi[0], lo[0]);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// neighbour entry: bits 0..23 atom index, bits 24..31 image code
// code = (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2), s in [-2, 2]
#define NB_INDEX_MASK 0x00ffffffu
__device__ __forceinline__ uint32_t nb_pack(int j, int sx, int sy, int sz)
{
    return (uint32_t)j | ((uint32_t)((sx + 2) * 25 + (sy + 2) * 5 + (sz + 2)) << 24);
}
// image code of the shift (0, 0, 0): (0 + 2) * 25 + (0 + 2) * 5 + (0 + 2)
#define NB_CODE_NOSHIFT 62u
__device__ __forceinline__ void nb_shift(uint32_t e, float Lx, float Ly, float Lz, float& ox, float& oy, float& oz)
{
    int code = (int)(e >> 24);
    int sx = code / 25 - 2;
    int sy = (code / 5) % 5 - 2;
    int sz = code % 5 - 2;
    ox = (float)sx * Lx;
    oy = (float)sy * Ly;
    oz = (float)sz * Lz;
}
// the same image seen from the other atom: code -> 124 - code
__device__ __forceinline__ uint32_t nb_reverse(uint32_t e, int i)
{
    return (uint32_t)i | ((124u - (e >> 24)) << 24);
}

struct Box { float L[3]; };

// d = (pj - pi) + shift, with the rounding error of pj - pi restored by Knuth's
// TwoSum (the error of a float sum is exactly representable).  For periodic
// images pj - pi is close to -shift, so t + shift is exact (Sterbenz) and d is
// correct to one rounding even in boxes hundreds of A wide.  Exactly
// antisymmetric: swapping i and j and negating the shift negates d.
__device__ __forceinline__ float pair_disp(float pj, float pi, float shift)
{
    const float t = pj - pi;
    const float bb = t - pj;
    const float e = (pj - (t - bb)) + (-pi - bb);
    return (t + shift) + e;
}
