// nnp_capi.cu -- host side of the C ABI declared in include/nnp.h: parameter
// validation, the device plan, scratch management and the launch sequence of
// one energy+force evaluation (Fig. 1b steps 1-3 of arXiv 2002.00054) and of
// velocity-Verlet NVE.  All kernels live in this translation unit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nnp.h"
#include "common.cuh"
#include "k_descriptors.cuh"
#include "k_md.cuh"
#include "k_mlp.cuh"
#include "k_mlp_tc.cuh"
#include "k_neighbors.cuh"
#include "k_train.cuh"
#include "k_flat.cuh"

namespace {

const double kAcc = 9.64853321233100e-3;   // 1 eV/(A amu) in A/fs^2
const double kLog2e = 1.4426950408889634074;

// x = hi + lo with hi = float(x), lo = float(x - hi)
void split(double x, float& hi, float& lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

}  // namespace

typedef void (*MlpKernel)(int, const float4*, const Plan*, const float*, const float*, float*, float*);

// FP32 network kernel for hidden widths up to hp (a multiple of 4, at most 32)
static MlpKernel pick_mlp(int hp)
{
    switch (hp) {
    case 4: return k_mlp_fp32<4>;
    case 8: return k_mlp_fp32<8>;
    case 12: return k_mlp_fp32<12>;
    case 16: return k_mlp_fp32<16>;
    case 20: return k_mlp_fp32<20>;
    case 24: return k_mlp_fp32<24>;
    case 28: return k_mlp_fp32<28>;
    default: return k_mlp_fp32<32>;
    }
}

enum { FM_FIXED = 0, FM_GATHER = 1, FM_FLOAT = 2 };

struct nnp_handle {
    int device = 0;
    Plan plan;
    Plan* d_plan = nullptr;
    int n_params = 0;
    float* d_w = nullptr;
    double cutoff = 0, skin = 0;
    int stride = 0;
    int precision = NNP_FP32;
    std::string err;

    // per-atom scratch (capacity cap_n)
    int cap_n = 0;
    float4 *off = nullptr, *ref = nullptr, *pos4 = nullptr, *Fown = nullptr;
    float *G = nullptr, *dEdG = nullptr, *Ei = nullptr, *F = nullptr;
    uint32_t* nbr = nullptr;
    int *ncount = nullptr, *rev = nullptr, *cell_of = nullptr, *cell_atoms = nullptr;
    float4* gbuf = nullptr;
    float4* cpos = nullptr;   // positions in cell order (row builder)
    // cells
    int cap_cells = 0;
    int *cell_count = nullptr, *cell_start = nullptr, *cursor = nullptr;
    // reductions
    int cap_epart = 0, cap_vpart = 0;
    double *epart = nullptr, *vpart = nullptr, *d_energy = nullptr, *d_log = nullptr;
    int cap_log = 0;
    // flags, counters, boxes
    int* flags = nullptr;
    int* h_flags = nullptr;   // pinned
    unsigned long long* counters = nullptr;
    float4* sys_box = nullptr;

    // list state
    bool list_valid = false;
    int list_n = -1;
    double list_box[3] = {0, 0, 0};
    bool cell_path = false;
    int nc[3] = {0, 0, 0};

    // nnp_step continuation: final state of the last nnp_step call
    bool step_valid = false;
    const float* step_pos = nullptr;
    const int* step_types = nullptr;
    int step_n = -1;
    double step_box[3] = {0, 0, 0};
    float* pos_cache = nullptr;
    int* types_cache = nullptr;

    // kernel-group timing (CUDA events on the call's stream)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int id; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double prof_ms[16] = {0};   // per kernel group (at most 16 groups)
    long long prof_n[16] = {0};
    long long launches = 0;   // kernels launched by the current / last call

    // batches of independent systems (training): layout of the cached list
    int cap_sys = 0;
    int* sys_of = nullptr;        // [cap_n]
    int* sys_start_d = nullptr;   // [cap_sys + 1]
    std::vector<int> bt_start;    // host copy of the last batch layout
    std::vector<double> bt_boxes;
    float* T = nullptr;           // descriptor tangents [cap_n][gs]
    float* gpart = nullptr;       // per-warp parameter-gradient partials
    size_t cap_gpart = 0;
    size_t smem_tan = 0, smem_pg = 0;
    int grid_tan = 0;

    // BF16 tensor-core network: shapes, per-element atom lists
    TcShape tcs{0, 0, 0};
    size_t smem_tc = 0;
    int* elem_idx = nullptr;
    int* elem_part = nullptr;
    int* elem_off = nullptr;   // [NNP_MAXE + 1] atoms, then [NNP_MAXE + 1] tiles

    // launch configuration
    int num_sms = 148;
    int max_smem = 0;
    int wpb_sf = 8, wpb_force = 8, wpb_tan = 4;
    size_t smem_sf = 0, smem_force = 0, smem_mlp = 0;
    MlpKernel kmlp = nullptr;   // FP32 network, instantiated for the hidden width
    int grid_sf = 0, grid_force = 0, grid_mlp = 0;
    int cap_rc = 0;   // main launches: neighbours inside the cutoff staged per warp (set_capacity)
    // wide-capacity pass over the atoms above cap_rc (capacity = list stride)
    int* spill = nullptr;   // [cap_n + 1]: count, then atom indices
    int wpb_sf_sp = 1, wpb_force_sp = 1, wpb_tan_sp = 1;
    size_t smem_sf_sp = 0, smem_force_sp = 0, smem_tan_sp = 0;
    int grid_sp = 0;
    // counters read back with the status; evaluations in the current call
    unsigned long long* h_cnt = nullptr;
    int evals = 0;
    // pair-queue records written by the descriptor pass for the force pass
    unsigned short* qpool = nullptr;
    size_t cap_qpool = 0;      // entries allocated
    size_t want_qpool = 0;     // entries the next evaluation should have (0: estimate)
    unsigned int* qoff = nullptr;   // [cap_n] record offset / 8 per atom
    unsigned short* seg = nullptr;  // [cap_n][NB_SEG] stencil segments of cell-built rows
    // force assembly: FM_FIXED (default) 64-bit fixed-point integer atomics into
    // Fq; FM_GATHER per-slot g buffer and reverse-index gather; FM_FLOAT float
    // atomics (order-dependent)
    int fmode = 0;
    unsigned long long* Fq = nullptr;   // [cap_n][3], units 2^-LB eV/A (fq_unit)
    // staged neighbours written by the descriptor pass for the force pass: three
    // planes of cap_stg float4 (atom i, staged index m at i * C + m)
    bool use_stg = true;
    bool cell_order = true;   // main passes visit atoms in cell order (NNP_CELL_ORDER=0: atom order)
    float4* stg = nullptr;
    size_t cap_stg = 0;
    // nnp_step: the per-step launch sequence captured as a CUDA graph and replayed
    bool step_graph = true;
    cudaStream_t gstream = nullptr;   // capture and replay stream (non-blocking, owned)
    cudaEvent_t gfork = nullptr, gjoin = nullptr;
    cudaGraphExec_t gexec = nullptr;  // kept across calls, updated in place when only arguments change
};

static thread_local std::string g_create_err;

static int set_err(nnp_handle* h, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
static int set_err(nnp_handle* h, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_err = buf;
    return code;
}

#define CK(h, call)                                                                                  \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return set_err(h, e_ == cudaErrorMemoryAllocation ? NNP_ENOMEM : NNP_ECUDA, "%s: %s (%s:%d)", \
                           #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
    } while (0)

// ------------------------------------------------------------ validation / plan
static int build_plan(const nnp_params* p, Plan& P, int& n_params, std::string& why)
{
    char buf[256];
    auto fail = [&](const char* m) { why = m; return NNP_EINVAL; };
    if (!p) return fail("params is NULL");
    if (p->n_elements < 1 || p->n_elements > NNP_MAXE) return fail("n_elements must be in 1..8");
    if (!p->masses_amu || !p->n_sf || !p->sf || !p->sf_shift || !p->sf_scale || !p->widths || !p->weights)
        return fail("a required params pointer is NULL");
    if (!(p->cutoff > 0.0) || !std::isfinite(p->cutoff)) return fail("cutoff must be > 0");
    if (!(p->skin >= 0.0) || !std::isfinite(p->skin)) return fail("skin must be >= 0");
    if (p->n_layers < 2 || p->n_layers > NNP_MAXL) return fail("n_layers must be in 2..6");
    if (p->mlp_precision != NNP_FP32 && p->mlp_precision != NNP_BF16) return fail("mlp_precision must be NNP_FP32 or NNP_BF16");
    if (p->max_neighbors < 32 || p->max_neighbors > 1024) return fail("max_neighbors must be in 32..1024");
    memset(&P, 0, sizeof P);
    P.n_elem = p->n_elements;
    P.rc = (float)p->cutoff;
    P.rc2 = (float)(p->cutoff * p->cutoff);
    P.hpi_rc = (float)(M_PI / (2.0 * p->cutoff));
    split(0.5 / p->cutoff, P.inv_2rc, P.inv_2rc_lo);
    for (int k = 0; k <= 32; ++k) {   // table of the cutoff's cos(pi x) (cospi_dd)
        float ch, cl, sh, sl;
        split(std::cos(M_PI * k / 64.0), ch, cl);
        split(std::sin(M_PI * k / 64.0), sh, sl);
        P.cs64[k] = make_float4(ch, cl, sh, sl);
    }
    const double rcut = p->cutoff + p->skin;
    P.rcut2 = (float)(rcut * rcut);
    P.half_skin2 = (float)(0.25 * p->skin * p->skin);
    for (int e = 0; e < p->n_elements; ++e) {
        if (!(p->masses_amu[e] > 0.0)) return fail("masses must be > 0");
        P.mass[e] = (float)p->masses_amu[e];
        P.acc_over_m[e] = (float)(kAcc / p->masses_amu[e]);
    }
    // network shape
    const int ng = p->widths[0];
    if (ng < 1 || ng > NNP_MAXG) return fail("widths[0] (n_G) must be in 1..64");
    if (p->widths[p->n_layers] != 1) return fail("the last width must be 1");
    for (int l = 1; l < p->n_layers; ++l)
        if (p->widths[l] < 1 || p->widths[l] > NNP_MAXH) return fail("hidden widths must be in 1..32");
    P.n_layers = p->n_layers;
    int soff = 0, poff = 0;
    for (int l = 0; l <= p->n_layers; ++l) P.width[l] = p->widths[l];
    for (int l = 0; l < p->n_layers; ++l) {
        const int in = p->widths[l], out = p->widths[l + 1];
        P.ld[l] = in | 1;
        P.s_woff[l] = soff;
        soff += out * P.ld[l];
        P.s_boff[l] = soff;
        soff += out;
        P.p_woff[l] = poff;
        poff += out * in;
        P.p_boff[l] = poff;
        poff += out;
    }
    P.s_elem = (soff + 3) & ~3;
    P.n_params_elem = poff;
    {
        int hp = 4;
        for (int l = 1; l < p->n_layers; ++l) hp = std::max(hp, (p->widths[l] + 3) & ~3);
        P.lw_hp = hp;
        P.lw_kb0 = (ng + 31) & ~31;
        int lo = 0, rows = ng;
        for (int l = 0; l + 1 < p->n_layers; ++l) {
            const int in = p->widths[l];
            P.lw_f[l] = lo;
            lo += in * hp;
            P.lw_fb[l] = lo;
            lo += hp;
            P.lw_b[l] = lo;
            lo += hp * (l == 0 ? P.lw_kb0 : hp);
            rows += p->widths[l + 1];
        }
        P.lw_out = lo;
        lo += (p->n_layers > 1) ? hp : P.lw_kb0;
        P.lw_outb = lo;
        lo += 4;
        P.lw_invs = lo;
        lo += P.lw_kb0;
        P.lw_elem = ((lo + 27) / 32) * 32 + 4;
        P.lw_rows = rows;
    }
    n_params = poff * p->n_elements;
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(p->weights[i])) return fail("weights must be finite");
    // descriptors
    int off = 0, kind = 0, neta_max = 0;
    for (int e = 0; e < p->n_elements; ++e) {
        ElemPlan& E = P.e[e];
        const int ns = p->n_sf[e];
        if (ns != ng) return fail("n_sf[e] must equal widths[0] for every element");
        E.n_g = ns;
        for (int q = 0; q < NNP_MAXETA; ++q)
            for (int l = 0; l < 2; ++l)
                for (int k = 0; k <= NNP_KMAX; ++k)
                    for (int c = 0; c < NNP_MAXCLS; ++c) E.ang_out[c][q][l][k] = -1;
        E.n_cls = 0;
        std::vector<double> etas;
        for (int s = 0; s < ns; ++s) {
            const nnp_sf_desc& d = p->sf[off + s];
            const double mu = p->sf_shift[off + s], sc = p->sf_scale[off + s];
            if (!(sc > 0.0) || !std::isfinite(sc) || !std::isfinite(mu)) return fail("sf_scale must be > 0 and finite, sf_shift finite");
            E.mu[s] = (float)mu;
            E.inv_s[s] = (float)(1.0 / sc);
            if (!(d.eta >= 0.0) || !std::isfinite(d.eta)) return fail("eta must be >= 0");
            if (d.type == NNP_SF_RADIAL) {
                if (d.elem_a < -1 || d.elem_a >= p->n_elements) return fail("radial elem_a out of range");
                if (!std::isfinite(d.rs)) return fail("rs must be finite");
                if (E.n_rad >= NNP_MAXRAD) return fail("too many radial descriptors");
                E.rad_eta[E.n_rad] = (float)d.eta;
                split(-d.eta * kLog2e, E.rad_khi[E.n_rad], E.rad_klo[E.n_rad]);
                E.rad_rs[E.n_rad] = (float)d.rs;
                E.rad_elem[E.n_rad] = d.elem_a;
                E.rad_out[E.n_rad] = s;
                E.n_rad++;
            } else if (d.type == NNP_SF_ANG_NARROW || d.type == NNP_SF_ANG_WIDE) {
                if (d.elem_a < -1 || d.elem_a >= p->n_elements || d.elem_b < -1 || d.elem_b >= p->n_elements)
                    return fail("angular elem_a / elem_b out of range");
                if (d.rs != 0.0) return fail("angular rs must be 0");
                // neighbour-element pair class (either element -1: every pair)
                int ce1 = -1, ce2 = -1;
                if (d.elem_a >= 0 && d.elem_b >= 0) {
                    ce1 = std::min(d.elem_a, d.elem_b);
                    ce2 = std::max(d.elem_a, d.elem_b);
                }
                int c = -1;
                for (int t = 0; t < E.n_cls; ++t)
                    if (E.cls_e1[t] == ce1 && E.cls_e2[t] == ce2) c = t;
                if (c < 0) {
                    if (E.n_cls >= NNP_MAXCLS) { why = "more than 10 neighbour-element pair classes of angular descriptors"; return NNP_EUNSUPPORTED; }
                    c = E.n_cls++;
                    E.cls_e1[c] = ce1;
                    E.cls_e2[c] = ce2;
                    if (ce1 >= 0) P.resolved = 1;
                }
                if (kind == 0) kind = d.type;
                else if (kind != d.type) { why = "narrow and wide angular descriptors in one model are not implemented"; return NNP_EUNSUPPORTED; }
                int q = -1;
                for (size_t t = 0; t < etas.size(); ++t) if (etas[t] == d.eta) q = (int)t;
                if (q < 0) {
                    if ((int)etas.size() >= NNP_MAXETA) { why = "more than 4 distinct angular eta per element"; return NNP_EUNSUPPORTED; }
                    etas.push_back(d.eta);
                    q = (int)etas.size() - 1;
                    E.ang_eta[q] = (float)d.eta;
                    split(-d.eta * kLog2e, E.ang_khi[q], E.ang_klo[q]);
                }
                int l;
                if (d.lambda == 1.0) l = 0;
                else if (d.lambda == -1.0) l = 1;
                else return fail("lambda must be +1 or -1");
                int k = -1;
                for (int t = 0; t <= NNP_KMAX; ++t) if (d.zeta == (double)(1 << t)) k = t;
                if (k < 0) { why = "angular zeta must be 1, 2, 4, 8 or 16"; return NNP_EUNSUPPORTED; }
                if (E.ang_out[c][q][l][k] >= 0) return fail("duplicate angular descriptor");
                E.ang_out[c][q][l][k] = s;
            } else {
                snprintf(buf, sizeof buf, "unknown descriptor type %d", d.type);
                why = buf;
                return NNP_EINVAL;
            }
        }
        E.n_eta = (int)etas.size();
        neta_max = std::max(neta_max, E.n_eta);
        off += ns;
        {
            // order the radial descriptors by neighbour element (all-element ones
            // first); each keeps its output slot rad_out
            std::vector<int> ord(E.n_rad);
            for (int r = 0; r < E.n_rad; ++r) ord[r] = r;
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return E.rad_elem[a] < E.rad_elem[b]; });
            ElemPlan T = E;
            for (int r = 0; r < E.n_rad; ++r) {
                const int o = ord[r];
                E.rad_eta[r] = T.rad_eta[o];
                E.rad_khi[r] = T.rad_khi[o];
                E.rad_klo[r] = T.rad_klo[o];
                E.rad_rs[r] = T.rad_rs[o];
                E.rad_elem[r] = T.rad_elem[o];
                E.rad_out[r] = T.rad_out[o];
            }
            E.rad_nall = 0;
            while (E.rad_nall < E.n_rad && E.rad_elem[E.rad_nall] < 0) E.rad_nall++;
            for (int x = 0; x < NNP_MAXE; ++x) {
                int b = E.rad_nall;
                while (b < E.n_rad && E.rad_elem[b] < x) b++;
                int en = b;
                while (en < E.n_rad && E.rad_elem[en] == x) en++;
                E.rad_beg[x] = b;
                E.rad_end[x] = en;
            }
        }
    }
    P.ang_kind = kind;
    P.n_eta_max = neta_max;
    P.gs = (ng + 3) & ~3;
    return NNP_OK;
}

// --------------------------------------------------------------- dispatch
typedef void (*SfKernel)(int, const float4*, Box, NbView, const Plan*, int, float*, float*, int*, unsigned long long*,
                         int*, int, unsigned short*, unsigned int*, unsigned long long, float4*, size_t);
typedef void (*ForceKernel)(int, const float4*, Box, NbView, const Plan*, int, const float*, float4*, float4*,
                            double*, int, int*, int*, int, const unsigned short*, const unsigned int*, float*,
                            unsigned long long*, const float4*, size_t, unsigned long long);

typedef void (*TangentKernel)(int, const float4*, Box, NbView, const Plan*, int, const float*, float*, int*, int*, int);

// The descriptor kernel in two forms: up to SF_MERGED_MAX staged neighbours
// (indices in 8 bits) the block pairs of an atom share one pair queue and the
// pair-queue records exist; beyond, one block pair at a time (sf_for).
#define SF_MERGED_MAX 256

// fh: the MD step's form of the force pass over stored queues (staged neighbours,
// fixed-point atomics, no virial), where it exists (at most 2 eta, not resolved).
template <int NETA, bool NARROW, int KP, int KN, bool RES = false>
static void pick(SfKernel& s, ForceKernel& f, TangentKernel& t, ForceKernel& fs, SfKernel& sw, ForceKernel& fh)
{
    s = k_sf<NETA, NARROW, KP, KN, RES, true>;
    sw = k_sf<NETA, NARROW, KP, KN, RES, false>;
    f = k_force<NETA, NARROW, KP, KN, false, RES>;
    t = k_tangent<NETA, NARROW, KP, KN, RES>;
    fh = nullptr;
    if constexpr (RES) {
        fs = f;   // resolved models do not store pair queues
    } else {
        fs = k_force<NETA, NARROW, KP, KN, true, false>;
        if constexpr (NARROW && NETA > 0 && NETA <= 2) fh = k_force<NETA, NARROW, KP, KN, true, false, true>;
    }
}

// Largest k (zeta = 2^k) used with lambda = +1 (l = 0) or -1 (l = 1), -1 if none.
static int kmax_of(const Plan& P, int l)
{
    int km = -1;
    for (int e = 0; e < P.n_elem; ++e)
        for (int c = 0; c < P.e[e].n_cls; ++c)
            for (int q = 0; q < NNP_MAXETA; ++q)
                for (int k = 0; k <= NNP_KMAX; ++k)
                    if (P.e[e].ang_out[c][q][l][k] >= 0) km = std::max(km, k);
    return km;
}

// Specialised instantiations for the term sets of the water-like (narrow, two
// eta, lambda +1 up to zeta 16, lambda -1 up to zeta 4) and FCC-like (wide,
// three eta, both lambda up to zeta 16) models; every other set runs the
// generic instantiation with all powers up to zeta 16.
static void pick_kernels(const Plan& P, SfKernel& s, ForceKernel& f, TangentKernel& t, ForceKernel& fs,
                         SfKernel& sw, ForceKernel& fh)
{
    const bool nar = (P.ang_kind == NNP_SF_ANG_NARROW);
    const int kp = kmax_of(P, 0), kn = kmax_of(P, 1);
    if (P.resolved) {
        // angular descriptors resolved by neighbour-element pair: generic terms
        switch (P.n_eta_max) {
        case 1: if (nar) pick<1, true, 4, 4, true>(s, f, t, fs, sw, fh); else pick<1, false, 4, 4, true>(s, f, t, fs, sw, fh); break;
        case 2: if (nar) pick<2, true, 4, 4, true>(s, f, t, fs, sw, fh); else pick<2, false, 4, 4, true>(s, f, t, fs, sw, fh); break;
        case 3: if (nar) pick<3, true, 4, 4, true>(s, f, t, fs, sw, fh); else pick<3, false, 4, 4, true>(s, f, t, fs, sw, fh); break;
        default: if (nar) pick<4, true, 4, 4, true>(s, f, t, fs, sw, fh); else pick<4, false, 4, 4, true>(s, f, t, fs, sw, fh); break;
        }
        return;
    }
    if (nar && P.n_eta_max == 2 && kp == 4 && kn <= 2) { pick<2, true, 4, 2>(s, f, t, fs, sw, fh); return; }
    if (!nar && P.n_eta_max == 3 && kp <= 4 && kn <= 4) { pick<3, false, 4, 4>(s, f, t, fs, sw, fh); return; }
    switch (P.n_eta_max) {
    case 0: pick<0, false, 4, 4>(s, f, t, fs, sw, fh); break;
    case 1: if (nar) pick<1, true, 4, 4>(s, f, t, fs, sw, fh); else pick<1, false, 4, 4>(s, f, t, fs, sw, fh); break;
    case 2: if (nar) pick<2, true, 4, 4>(s, f, t, fs, sw, fh); else pick<2, false, 4, 4>(s, f, t, fs, sw, fh); break;
    case 3: if (nar) pick<3, true, 4, 4>(s, f, t, fs, sw, fh); else pick<3, false, 4, 4>(s, f, t, fs, sw, fh); break;
    default: if (nar) pick<4, true, 4, 4>(s, f, t, fs, sw, fh); else pick<4, false, 4, 4>(s, f, t, fs, sw, fh); break;
    }
}
static void pick_kernels(const Plan& P, SfKernel& s, ForceKernel& f, TangentKernel& t, ForceKernel& fs,
                         SfKernel& sw)
{
    ForceKernel fh;
    pick_kernels(P, s, f, t, fs, sw, fh);
}
static void pick_kernels(const Plan& P, SfKernel& s, ForceKernel& f, TangentKernel& t, ForceKernel& fs)
{
    SfKernel sw;
    pick_kernels(P, s, f, t, fs, sw);
}
static void pick_kernels(const Plan& P, SfKernel& s, ForceKernel& f, TangentKernel& t)
{
    ForceKernel fs;
    pick_kernels(P, s, f, t, fs);
}
// The descriptor kernel for capacity C (the merged form up to SF_MERGED_MAX).
static SfKernel sf_for(const Plan& P, int C)
{
    SfKernel s, sw;
    ForceKernel f, fs;
    TangentKernel t;
    pick_kernels(P, s, f, t, fs, sw);
    return C <= SF_MERGED_MAX ? s : sw;
}
static void pick_kernels(const Plan& P, SfKernel& s, ForceKernel& f)
{
    TangentKernel t;
    pick_kernels(P, s, f, t);
}

// Unit of the int64 force sums: the force kernels run the narrow instantiation
// for narrow models with angular functions (pick_kernels), the wide one otherwise.
static double fq_unit(const Plan& P)
{
    const bool nar = P.ang_kind == NNP_SF_ANG_NARROW && P.n_eta_max > 0;
    return std::ldexp(1.0, -(nar ? FX_LB_NARROW : FX_LB_WIDE));
}

static size_t sf_smem_per_warp(const Plan& P, int cap) { return sf_warp_bytes(cap, P.n_eta_max > 2); }
static size_t force_smem_per_warp(const Plan& P, int cap, int stride)
{
    // the kernels' NETA is n_eta_max; resolved models keep each neighbour's element
    return force_warp_bytes(cap, stride, P.n_eta_max <= 2, P.resolved != 0);
}

// Shared-memory capacity C of the main descriptor, force and tangent launches:
// warps per block (at most 4, the kernels' launch bounds), dynamic shared memory
// and occupancy-sized grids.  Atoms with more than C neighbours inside the
// cutoff take the wide-capacity pass, so C trades occupancy against that pass.
static int set_capacity(nnp_handle* h, int C)
{
    SfKernel ksf;
    ForceKernel kf;
    TangentKernel kt;
    pick_kernels(h->plan, ksf, kf, kt);
    const size_t ps = sf_smem_per_warp(h->plan, C), pf = force_smem_per_warp(h->plan, C, h->stride), pt = tangent_warp_bytes(C);
    const size_t ms = (size_t)h->max_smem;
    if (ps > ms || pf > ms) return set_err(h, NNP_EINVAL, "shared-memory capacity %d does not fit one block", C);
    h->cap_rc = C;
    h->wpb_sf = (int)std::min<size_t>(4, ms / ps);
    h->wpb_force = (int)std::min<size_t>(4, ms / pf);
    h->wpb_tan = (int)std::max<size_t>(1, std::min<size_t>(4, ms / pt));
    h->smem_sf = ps * h->wpb_sf;
    h->smem_force = pf * h->wpb_force;
    h->smem_tan = pt * h->wpb_tan;
    int bs = 0;
    CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, (const void*)sf_for(h->plan, C), 32 * h->wpb_sf, h->smem_sf));
    h->grid_sf = std::max(1, bs) * h->num_sms;
    CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, (const void*)kf, 32 * h->wpb_force, h->smem_force));
    h->grid_force = std::max(1, bs) * h->num_sms;
    if (h->smem_pg && pt <= ms) {
        CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, (const void*)kt, 32 * h->wpb_tan, h->smem_tan));
        h->grid_tan = std::max(1, bs) * h->num_sms;
    }
    return NNP_OK;
}

// After a call: grow C by a quarter when more than 0.2% of the evaluated atoms
// took the wide-capacity pass; shrink it to 1.1 x the largest count seen when
// that is below 0.85 C.  Applies from the next call; results do not depend on C.
static void retune_capacity(nnp_handle* h)
{
    if (h->evals <= 0 || h->list_n <= 0) return;
    const double evaluated = (double)h->list_n * h->evals;
    const double spilled = (double)h->h_cnt[CNT_SPILL];
    const int maxrc = (int)h->h_cnt[CNT_MAXRC];
    int C = h->cap_rc;
    if (spilled > 0.002 * evaluated) {
        C = (int)std::ceil(1.25 * C);
    } else {
        const int fit = (int)std::ceil(1.1 * maxrc);
        if (maxrc > 0 && fit < 0.85 * C) C = fit;
    }
    C = std::min(h->stride, std::max(32, (C + 7) & ~7));
    if (C != h->cap_rc) {
        const int old = h->cap_rc;
        if (set_capacity(h, C) != NNP_OK) set_capacity(h, old);
    }
    // queue pool: the last evaluation's demand (chunks claimed, including the
    // claims that did not fit) plus a quarter
    const size_t demand = (size_t)h->h_cnt[CNT_QTOP];
    if (demand > 0 && (demand > h->cap_qpool || 2 * (demand + demand / 4) < h->cap_qpool))
        h->want_qpool = demand + demand / 4;
}

// ------------------------------------------------------------------ scratch
static int blocks_for(int n, int t) { return (n + t - 1) / t; }

template <typename T>
static cudaError_t regrow(T*& p, size_t count)
{
    if (p) cudaFree(p);
    p = nullptr;
    return cudaMalloc((void**)&p, std::max<size_t>(count, 1) * sizeof(T));
}

static int ensure_atoms(nnp_handle* h, int n)
{
    if (n <= h->cap_n) return NNP_OK;
    const int cap = std::max(n, h->cap_n + h->cap_n / 8);
    const size_t rows = (size_t)cap * h->stride;
    CK(h, regrow(h->off, cap));
    CK(h, regrow(h->ref, cap));
    CK(h, regrow(h->pos4, cap));
    CK(h, regrow(h->Fown, cap));
    CK(h, regrow(h->G, (size_t)cap * h->plan.gs));
    CK(h, regrow(h->dEdG, (size_t)cap * h->plan.gs));
    CK(h, regrow(h->Ei, cap));
    CK(h, regrow(h->F, (size_t)cap * 3));
    CK(h, regrow(h->nbr, rows));
    CK(h, regrow(h->ncount, cap));
    if (h->fmode == FM_GATHER) {   // reverse index and g buffer: the gather form only
        CK(h, regrow(h->rev, rows));
        CK(h, regrow(h->gbuf, rows));
    }
    CK(h, regrow(h->Fq, (size_t)cap * 3));
    CK(h, regrow(h->seg, (size_t)cap * NB_SEG));
    CK(h, regrow(h->cell_of, cap));
    CK(h, regrow(h->cell_atoms, cap));
    CK(h, regrow(h->cpos, cap));
    CK(h, regrow(h->pos_cache, (size_t)cap * 3));
    CK(h, regrow(h->types_cache, cap));
    CK(h, regrow(h->elem_idx, cap));
    CK(h, regrow(h->elem_part, (size_t)blocks_for(cap, 256) * NNP_MAXE));
    CK(h, regrow(h->sys_of, cap));
    CK(h, regrow(h->T, (size_t)cap * h->plan.gs));
    CK(h, regrow(h->spill, (size_t)cap + 1));
    CK(h, regrow(h->qoff, cap));
    h->bt_start.clear();
    h->cap_n = cap;
    h->list_valid = false;
    h->step_valid = false;
    return NNP_OK;
}

static int ensure_cells(nnp_handle* h, int ncell)
{
    if (ncell <= h->cap_cells) return NNP_OK;
    CK(h, regrow(h->cell_count, ncell + 1));
    CK(h, regrow(h->cell_start, ncell + 1));
    CK(h, regrow(h->cursor, ncell + 1));
    h->cap_cells = ncell;
    return NNP_OK;
}

static int ensure_red(nnp_handle* h, int ne, int nv)
{
    if (ne > h->cap_epart) {
        CK(h, regrow(h->epart, ne));
        h->cap_epart = ne;
    }
    if (nv > h->cap_vpart) {
        CK(h, regrow(h->vpart, (size_t)nv * 9));
        h->cap_vpart = nv;
    }
    return NNP_OK;
}

// Queue pool for an evaluation of n atoms: the size the last call asked for, or
// on first use C^2 / 8 entries per atom (about the narrow water records at the
// capacity the counts suggest; atoms that do not fit rebuild their queue and
// the next call gets a larger pool).  Shrinks when more than twice too large.
static int ensure_qpool(nnp_handle* h, int n)
{
    size_t want = h->want_qpool;
    if (want == 0) want = (size_t)n * ((size_t)h->cap_rc * h->cap_rc / 8 + 64);
    if (want <= h->cap_qpool && 2 * want >= h->cap_qpool) return NNP_OK;
    if (h->qpool) cudaFree(h->qpool);
    h->qpool = nullptr;
    h->cap_qpool = 0;
    CK(h, cudaMalloc((void**)&h->qpool, want * sizeof(unsigned short)));
    h->cap_qpool = want;
    return NNP_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

enum { KG_NEIGH = 0, KG_SF, KG_MLP, KG_FORCE, KG_GATHER, KG_REDUCE, KG_INTEGRATE, KG_FLAT, KG_PAIR, KG_CELL, KG_N };
static const char* kKgName[KG_N] = {"neighbor_maintenance", "descriptors", "network", "force", "gather",
                                    "reductions", "integrate", "descriptors_flat", "descriptors_pair",
                                    "descriptors_cell"};
static_assert(KG_N <= 16, "kernel-group timers hold 16 groups");

static cudaEvent_t ev_get(nnp_handle* h)
{
    cudaEvent_t e = nullptr;
    if (!h->ev_pool.empty()) {
        e = h->ev_pool.back();
        h->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

// Times the kernels launched in its lifetime (when profiling is on) and counts launches.
struct KScope {
    nnp_handle* h;
    int id;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    int n_kernels;
    KScope(nnp_handle* h_, int id_, cudaStream_t st_, int n_kernels_ = 1) : h(h_), id(id_), st(st_), n_kernels(n_kernels_)
    {
        h->launches += n_kernels;
        if (h->prof_on && (a = ev_get(h))) cudaEventRecord(a, st);
    }
    ~KScope()
    {
        if (!h->prof_on || !a) return;
        cudaEvent_t b = ev_get(h);
        if (!b) return;
        cudaEventRecord(b, st);
        h->pending.push_back({id, a, b});
    }
};

// Accumulates finished event pairs (call after the stream has been synchronised).
static void prof_flush(nnp_handle* h)
{
    for (auto& p : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            h->prof_ms[p.id] += ms;
            h->prof_n[p.id] += 1;
        }
        h->ev_pool.push_back(p.a);
        h->ev_pool.push_back(p.b);
    }
    h->pending.clear();
    cudaGetLastError();
}

static int check_box(nnp_handle* h, const double* box)
{
    if (!box) return set_err(h, NNP_EINVAL, "box is NULL");
    const double rcut = h->cutoff + h->skin;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !std::isfinite(box[a])) return set_err(h, NNP_EBOX, "box edges must be finite and > 0");
        if (box[a] < 0.5 * rcut)
            return set_err(h, NNP_EBOX, "box edge %g is below (cutoff + skin) / 2 = %g", box[a], 0.5 * rcut);
    }
    return NNP_OK;
}

static int read_status(nnp_handle* h, cudaStream_t st)
{
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(h->h_flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(h, cudaMemcpyAsync(h->h_cnt, h->counters, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    prof_flush(h);
    const int f = h->h_flags[0];
    if (f) {
        // errors leave the neighbour list and the step state unknown
        h->list_valid = false;
        h->step_valid = false;
        char msg[256];
        const int status = error_word_status(f, h->stride, CELL_CAP, (double)FX_LIMIT, msg, sizeof msg);
        return set_err(h, status, "%s", msg);
    }
    retune_capacity(h);
    return NNP_OK;
}


// Neighbour maintenance + descriptors + network + forces for one system.
// Outputs (device, each nullable): energy[1], Ei_out[n], F_out[n*3], vir_out[9], G_out, dEdG_out [n][n_G].
// stop_after: 0 full, 1 after descriptors, 2 after network.
// A batch of B independent periodic systems: atoms start[b] .. start[b+1]-1 in box b.
struct Batch {
    int B;
    const int* start;     // host [B + 1], start[0] = 0, start[B] = n
    const double* boxes;  // host [3 B]
};

static int ensure_sys(nnp_handle* h, int B)
{
    if (B <= h->cap_sys) return NNP_OK;
    CK(h, regrow(h->sys_box, B));
    CK(h, regrow(h->sys_start_d, B + 1));
    h->cap_sys = B;
    return NNP_OK;
}

static int run_eval(nnp_handle* h, int n, const float* pos, const int* types, const double* box, cudaStream_t st,
                    double* energy, float* Ei_out, float* F_out, double* vir_out, float* G_out, float* dEdG_out,
                    int stop_after, const Batch* bt = nullptr, int n_sum = -1)
{
    // energy and virial: sums over the energies of atoms i < n_sum (all by default)
    if (n_sum < 0 || n_sum > n) n_sum = n;
    int rc = ensure_atoms(h, n);
    if (rc) return rc;
    const Plan& P = h->plan;
    const double rcut = h->cutoff + h->skin;
    // path and rebuild decision
    bool same_box = h->list_valid && h->list_n == n;
    int nc[3] = {0, 0, 0};
    bool cell = true;
    int nim = 0;
    Box bx;
    if (!bt) {
        same_box = same_box && h->bt_start.empty();
        for (int a = 0; a < 3; ++a) same_box = same_box && (h->list_box[a] == box[a]);
        for (int a = 0; a < 3; ++a) {
            nc[a] = (int)std::floor(box[a] / rcut);
            if (nc[a] < 3) cell = false;
        }
        for (int a = 0; a < 3; ++a) nim = std::max(nim, (int)std::ceil(rcut / box[a]));
        if (!cell && nim > 2) return set_err(h, NNP_EBOX, "box too small for the image range");
        for (int a = 0; a < 3; ++a) bx.L[a] = (float)box[a];
    } else {
        cell = false;
        same_box = same_box && (int)h->bt_start.size() == bt->B + 1 &&
                   std::equal(bt->start, bt->start + bt->B + 1, h->bt_start.begin()) &&
                   std::equal(bt->boxes, bt->boxes + 3 * bt->B, h->bt_boxes.begin());
        for (int a = 0; a < 3; ++a) bx.L[a] = (float)bt->boxes[a];
    }
    const int T = 256;
    const int rows_grid = std::min(blocks_for(n, 8), h->num_sms * 8);
    {
        KScope ks(h, KG_NEIGH, st, 0);
        if (!same_box && bt) {
            rc = ensure_sys(h, bt->B);
            if (rc) return rc;
            std::vector<float4> sb(bt->B);
            std::vector<int> so(n);
            for (int b = 0; b < bt->B; ++b) {
                int nimb = 0;
                for (int a = 0; a < 3; ++a) nimb = std::max(nimb, (int)std::ceil(rcut / bt->boxes[3 * b + a]));
                sb[b] = make_float4((float)bt->boxes[3 * b], (float)bt->boxes[3 * b + 1], (float)bt->boxes[3 * b + 2],
                                    (float)nimb);
                for (int i = bt->start[b]; i < bt->start[b + 1]; ++i) so[i] = b;
            }
            CK(h, cudaMemcpyAsync(h->sys_box, sb.data(), sizeof(float4) * bt->B, cudaMemcpyHostToDevice, st));
            CK(h, cudaMemcpyAsync(h->sys_start_d, bt->start, sizeof(int) * (bt->B + 1), cudaMemcpyHostToDevice, st));
            CK(h, cudaMemcpyAsync(h->sys_of, so.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
            CK(h, cudaStreamSynchronize(st));   // the host vectors above are pageable staging
            h->bt_start.assign(bt->start, bt->start + bt->B + 1);
            h->bt_boxes.assign(bt->boxes, bt->boxes + 3 * bt->B);
            h->cell_path = false;
            CK(h, cudaMemsetAsync(h->flags + FLAG_REBUILD, 1, sizeof(int), st));
        } else if (!same_box) {
            h->bt_start.clear();
            CK(h, cudaMemsetAsync(h->flags + FLAG_REBUILD, 1, sizeof(int), st));   // any non-zero value
            h->cell_path = cell;
            for (int a = 0; a < 3; ++a) h->nc[a] = nc[a];
            const float4 sb = make_float4(bx.L[0], bx.L[1], bx.L[2], (float)nim);
            CK(h, cudaMemcpyAsync(h->sys_box, &sb, sizeof(float4), cudaMemcpyHostToDevice, st));
        } else {
            CK(h, cudaMemsetAsync(h->flags + FLAG_REBUILD, 0, sizeof(int), st));
            k_check_disp<<<blocks_for(n, T), T, 0, st>>>(n, pos, types, P.n_elem, h->off, h->ref, h->pos4,
                                                         P.half_skin2, h->flags);
            h->launches++;
        }
        k_rebuild_pos<<<blocks_for(n, T), T, 0, st>>>(n, pos, types, bx, P.n_elem, h->off, h->pos4, h->ref, h->flags,
                                                      h->counters, bt ? h->sys_of : nullptr,
                                                      bt ? h->sys_box : nullptr);
        h->launches++;
        if (h->cell_path) {
            const int ncell = h->nc[0] * h->nc[1] * h->nc[2];
            rc = ensure_cells(h, ncell);
            if (rc) return rc;
            CK(h, cudaMemsetAsync(h->cell_count, 0, sizeof(int) * (size_t)ncell, st));
            k_cell_count<<<blocks_for(n, T), T, 0, st>>>(n, h->pos4, bx, h->nc[0], h->nc[1], h->nc[2], h->cell_of,
                                                         h->cell_count, h->flags);
            k_cell_scan<<<1, 1024, 0, st>>>(ncell, h->cell_count, h->cell_start, h->cursor, h->flags);
            k_cell_fill<<<blocks_for(n, T), T, 0, st>>>(n, h->cell_of, h->cursor, h->cell_atoms, h->flags);
            k_cell_sort<<<std::min(blocks_for(ncell, 8), h->num_sms * 8), 256, 0, st>>>(
                ncell, h->cell_start, h->cell_atoms, h->pos4, h->cpos, h->flags);
            // rows a block per cell from the staged stencil; cells with more than
            // ROWS_SMAX stencil atoms leave their atoms (queued in spill, which the
            // descriptor pass clears again) to the warp-per-atom builder
            CK(h, cudaMemsetAsync(h->spill, 0, sizeof(int), st));
            k_rows_blk<<<std::min(ncell, 5 * h->num_sms), 128, rows_blk_smem_bytes(), st>>>(
                ncell, bx, h->nc[0], h->nc[1], h->nc[2], h->cell_start, h->cell_atoms, h->cpos, P.rcut2, h->stride,
                h->nbr, h->ncount, h->seg, h->spill, h->flags);
            k_rows_cell<<<rows_grid, 256, 0, st>>>(n, h->pos4, bx, h->nc[0], h->nc[1], h->nc[2], h->cell_start,
                                                   h->cell_atoms, h->cpos, P.rcut2, h->stride, h->nbr, h->ncount,
                                                   h->seg, h->flags, h->spill);
            if (h->fmode == FM_GATHER) k_rev_cell<<<rows_grid, 256, 0, st>>>(n, h->nbr, h->ncount, h->stride, h->seg, h->rev,
                                                                   h->flags);
            h->launches += (h->fmode == FM_GATHER) ? 7 : 6;
        } else {
            k_rows_brute<<<rows_grid, 256, 0, st>>>(n, h->pos4, bt ? h->sys_of : nullptr, bt ? h->sys_start_d : nullptr,
                                                    h->sys_box, P.rcut2, h->stride, h->nbr, h->ncount, h->flags);
            if (h->fmode == FM_GATHER) k_rev<<<rows_grid, 256, 0, st>>>(n, h->nbr, h->ncount, h->stride, h->rev, h->flags);
            h->launches += (h->fmode == FM_GATHER) ? 2 : 1;
        }
    }
    h->list_valid = true;
    h->list_n = n;
    for (int a = 0; a < 3; ++a) h->list_box[a] = box[a];

    NbView nv{h->nbr, h->ncount, h->stride};
    if (bt) {
        nv.sys_of = h->sys_of;
        nv.sys_box = h->sys_box;
    }
    if (!bt && h->cell_path && h->cell_order) nv.order = h->cell_atoms;   // atoms sorted by cell
    SfKernel ksf;
    ForceKernel kf;
    TangentKernel kt_unused;
    ForceKernel kfs, kfh;
    SfKernel ksw_unused;
    pick_kernels(P, ksf, kf, kt_unused, kfs, ksw_unused, kfh);
    h->evals++;
    bool staged = false;
    size_t stg_plane = 0;
    {
        // the force pass follows: store the pair queues for it (narrow kind only:
        // there the live masks cost a distance test per pair; wide queues follow
        // from the index arithmetic alone and are cheaper to rebuild than to store)
        const bool store = (stop_after == 0) && P.n_eta_max > 0 && P.ang_kind == NNP_SF_ANG_NARROW && !P.resolved;
        if (store) {
            rc = ensure_qpool(h, n);
            if (rc) return rc;
            CK(h, cudaMemsetAsync(h->counters + CNT_QTOP, 0, sizeof(unsigned long long), st));
        }
        // staged neighbours for the force pass: at most 2 eta, integer force atomics;
        // without the memory the force pass stages again
        staged = store && P.n_eta_max <= 2 && h->fmode == FM_FIXED && h->use_stg;
        if (staged) {
            const size_t plane = (size_t)n * h->cap_rc;
            if (plane > h->cap_stg) {
                if (h->stg) cudaFree(h->stg);
                h->stg = nullptr;
                h->cap_stg = 0;
                if (cudaMalloc((void**)&h->stg, 3 * plane * sizeof(float4)) == cudaSuccess) {
                    h->cap_stg = plane;
                } else {
                    cudaGetLastError();
                    h->stg = nullptr;
                    h->use_stg = false;   // do not retry on every call
                }
            }
            staged = h->stg != nullptr;
        }
        stg_plane = (size_t)n * h->cap_rc;
        KScope ks(h, KG_SF, st, 2);
        CK(h, cudaMemsetAsync(h->spill, 0, sizeof(int), st));
        CK(h, cudaMemsetAsync(h->flags + FLAG_WALK_SF, 0, 2 * sizeof(int), st));   // main passes' atom counters
        const int gsf = std::min(blocks_for(n, h->wpb_sf), h->grid_sf);
        sf_for(P, h->cap_rc)<<<gsf, 32 * h->wpb_sf, h->smem_sf, st>>>(n, h->pos4, bx, nv, h->d_plan, h->cap_rc, h->G, G_out, h->flags,
                                                     h->counters, h->spill, 0, store ? h->qpool : nullptr,
                                                     store ? h->qoff : nullptr, (unsigned long long)h->cap_qpool,
                                                     staged ? h->stg : nullptr, stg_plane);
        sf_for(P, h->stride)<<<h->grid_sp, 32 * h->wpb_sf_sp, h->smem_sf_sp, st>>>(n, h->pos4, bx, nv, h->d_plan, h->stride, h->G, G_out,
                                                                 h->flags, h->counters, h->spill, 1, nullptr, nullptr,
                                                                 0ull, nullptr, 0);
    }
    if (stop_after == 1 && !dEdG_out) return read_status(h, st);
    if (h->precision == NNP_BF16) {
        KScope ks(h, KG_MLP, st, 4);
        const int nblk = blocks_for(n, 256);
        int* toff = h->elem_off + NNP_MAXE + 1;
        k_elem_count<<<nblk, 256, 0, st>>>(n, h->pos4, P.n_elem, h->elem_part);
        k_elem_scan<<<1, 1024, 0, st>>>(nblk, P.n_elem, h->elem_part, h->elem_off, toff);
        k_elem_fill<<<nblk, 256, 0, st>>>(n, h->pos4, P.n_elem, h->elem_part, h->elem_idx);
        const int gtc = std::min(blocks_for(n, TC_TILE) + P.n_elem, 2 * h->num_sms);
        k_mlp_tc<<<gtc, 128, h->smem_tc, st>>>(n, h->d_plan, h->d_w, h->tcs, h->elem_idx, h->elem_off, toff, h->G,
                                                h->Ei, h->dEdG, h->flags);
    } else {
        KScope ks(h, KG_MLP, st);
        const int gmlp = std::min(blocks_for(n, 128), h->grid_mlp);
        h->kmlp<<<gmlp, 128, h->smem_mlp, st>>>(n, h->pos4, h->d_plan, h->d_w, h->G, h->Ei, h->dEdG);
    }
    if (dEdG_out) CK(h, cudaMemcpy2DAsync(dEdG_out, sizeof(float) * P.width[0], h->dEdG, sizeof(float) * P.gs,
                                          sizeof(float) * P.width[0], n, cudaMemcpyDeviceToDevice, st));
    if (stop_after >= 1) return read_status(h, st);
    const int gf = std::min(blocks_for(n, h->wpb_force), h->grid_force);
    const int nvp_main = gf * h->wpb_force;
    const int nvp = nvp_main + h->grid_sp * h->wpb_force_sp;
    const int gred = std::min(blocks_for(n, T), 4 * h->num_sms);
    rc = ensure_red(h, gred, nvp);
    if (rc) return rc;
    // the scatter forms add every contribution into the force sums directly
    float* Fout = F_out ? F_out : h->F;
    float* Fsc = (h->fmode == FM_FLOAT) ? Fout : nullptr;
    unsigned long long* Fq = (h->fmode == FM_FIXED) ? h->Fq : nullptr;
    if (Fsc) CK(h, cudaMemsetAsync(Fsc, 0, sizeof(float) * 3 * (size_t)n, st));
    if (Fq) CK(h, cudaMemsetAsync(Fq, 0, sizeof(unsigned long long) * 3 * (size_t)n, st));
    {
        KScope ks(h, KG_FORCE, st, 2);
        // main pass over the stored queues (atoms without one join the wide pass)
        const bool stored = P.n_eta_max > 0 && P.ang_kind == NNP_SF_ANG_NARROW && !P.resolved && h->qpool;
        // the MD step's form (staged neighbours, fixed-point atomics, no virial) has
        // an instantiation of its own without the other forms' code
        const bool hot = stored && staged && Fq && !vir_out && kfh;
        (hot ? kfh : (stored ? kfs : kf))<<<gf, 32 * h->wpb_force, h->smem_force, st>>>(
            n, h->pos4, bx, nv, h->d_plan, h->cap_rc, h->dEdG, h->gbuf, h->Fown, vir_out ? h->vpart : nullptr,
            n_sum, h->flags, h->spill, 0,
            stored ? h->qpool : nullptr, stored ? h->qoff : nullptr, Fsc, Fq, (stored && staged) ? h->stg : nullptr,
            stg_plane, stored ? (unsigned long long)h->cap_qpool : 0ull);
        kf<<<h->grid_sp, 32 * h->wpb_force_sp, h->smem_force_sp, st>>>(n, h->pos4, bx, nv, h->d_plan, h->stride,
                                                                       h->dEdG, h->gbuf, h->Fown,
                                                                       vir_out ? h->vpart + (size_t)nvp_main * 9 : nullptr,
                                                                       n_sum, h->flags,
                                                                       h->spill, 1, nullptr, nullptr, Fsc, Fq, nullptr, 0, 0ull);
    }
    if (h->fmode == FM_GATHER) {
        KScope ks(h, KG_GATHER, st);
        k_gather<<<rows_grid, 256, 0, st>>>(n, nv, h->rev, h->gbuf, h->Fown, Fout, h->flags);
    } else if (Fq) {
        KScope ks(h, KG_GATHER, st);
        k_fq_forces<<<blocks_for(3 * n, 256), 256, 0, st>>>(3 * n, Fq, fq_unit(P), Fout);
    }
    if (bt) {
        KScope ks(h, KG_REDUCE, st);
        if (energy) k_sys_energy<<<bt->B, 256, 0, st>>>(h->sys_start_d, h->Ei, energy, h->flags);
    } else {
        KScope ks(h, KG_REDUCE, st, 2);
        k_sum_partial<<<gred, T, 0, st>>>(n_sum, h->Ei, h->epart, h->flags);
        k_finalize<<<1, 256, 0, st>>>(gred, h->epart, energy ? energy : h->d_energy, vir_out ? nvp : 0, h->vpart,
                                      vir_out);
    }
    if (Ei_out) CK(h, cudaMemcpyAsync(Ei_out, h->Ei, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    return NNP_OK;
}

// Called at the start of every evaluating API call: clears the error word (errors
// accumulate over all evaluations of the call) and the work counters.
static int begin_call(nnp_handle* h, cudaStream_t st)
{
    h->launches = 0;
    h->evals = 0;
    CK(h, cudaMemsetAsync(h->flags + FLAG_ERR, 0, sizeof(int), st));
    CK(h, cudaMemsetAsync(h->counters, 0, sizeof(unsigned long long) * CNT_PER_CALL, st));
    CK(h, cudaMemsetAsync(h->counters + CNT_MINR, 0, sizeof(unsigned long long), st));
    return NNP_OK;
}

// all positions and types equal to the cached final state of the last nnp_step?
__global__ void k_same(int n, const float* __restrict__ pos, const float* __restrict__ pc, const int* __restrict__ t,
                       const int* __restrict__ tc, int* __restrict__ diff)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool d = (__float_as_int(pos[3 * i]) != __float_as_int(pc[3 * i])) ||
                   (__float_as_int(pos[3 * i + 1]) != __float_as_int(pc[3 * i + 1])) ||
                   (__float_as_int(pos[3 * i + 2]) != __float_as_int(pc[3 * i + 2])) || (t[i] != tc[i]);
    if (d) *diff = 1;
}

// One velocity-Verlet step: half kick and drift, evaluation of the new forces
// and energy (into d_energy), second half kick, energy-log entry.  Every
// decision that varies between steps (neighbour-list rebuild, wide-capacity
// atoms, log entry) is taken on the device, so the launch sequence is the same
// for every step of a call.
static int md_step(nnp_handle* h, int n, float* pos, float* vel, const int* types, const double* box, float dt,
                   int gke, double* log, cudaStream_t st)
{
    {
        KScope ks(h, KG_INTEGRATE, st);
        k_kick_drift<<<blocks_for(n, 256), 256, 0, st>>>(n, h->d_plan, types, h->F, vel, pos, dt);
    }
    int rc = run_eval(h, n, pos, types, box, st, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
    if (rc) return rc;
    KScope ks(h, KG_INTEGRATE, st, 2);
    k_kick_ke<<<gke, 256, 0, st>>>(n, h->d_plan, types, h->F, vel, dt, h->epart);
    k_log_sum<<<1, 256, 0, st>>>(gke, h->epart, h->d_energy, log, h->counters + CNT_LOGSLOT);
    return NNP_OK;
}

// reps further steps: one step's launch sequence is captured (on the handle's own
// stream, since the legacy default stream cannot be captured) into a CUDA graph,
// which is launched reps times, ordered after and before the caller's stream by
// events.  The executable graph is kept and updated in place while the captured
// topology stays the same, so a call pays one capture (tens of microseconds) and
// each step one graph launch instead of about twenty kernel launches.
static int replay_steps(nnp_handle* h, int n, float* pos, float* vel, const int* types, const double* box, float dt,
                        int gke, double* log, int reps, cudaStream_t st)
{
    if (!h->gstream) {
        CK(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
        CK(h, cudaEventCreateWithFlags(&h->gfork, cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->gjoin, cudaEventDisableTiming));
    }
    const long long launches0 = h->launches;
    const int evals0 = h->evals;
    CK(h, cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal));
    const int rc = md_step(h, n, pos, vel, types, box, dt, gke, log, h->gstream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->gstream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ec != cudaSuccess) return set_err(h, NNP_ECUDA, "step graph capture: %s", cudaGetErrorString(ec));
    if (h->gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(h->gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();   // an update refused for a changed topology is not an error of the call
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
    }
    if (!h->gexec) {
        const cudaError_t ei = cudaGraphInstantiate(&h->gexec, g, 0);
        if (ei != cudaSuccess) {
            h->gexec = nullptr;
            cudaGraphDestroy(g);
            return set_err(h, NNP_ECUDA, "step graph instantiation: %s", cudaGetErrorString(ei));
        }
    }
    cudaGraphDestroy(g);
    CK(h, cudaEventRecord(h->gfork, st));
    CK(h, cudaStreamWaitEvent(h->gstream, h->gfork, 0));
    for (int r = 0; r < reps; ++r) CK(h, cudaGraphLaunch(h->gexec, h->gstream));
    CK(h, cudaEventRecord(h->gjoin, h->gstream));
    CK(h, cudaStreamWaitEvent(st, h->gjoin, 0));
    // the capture counted one step's launches and evaluations
    h->launches = launches0 + (h->launches - launches0) * reps;
    h->evals = evals0 + (h->evals - evals0) * reps;
    return NNP_OK;
}

// ---------------------------------------------------------------- public API
extern "C" {

const char* nnp_status_string(int s)
{
    switch (s) {
    case NNP_OK: return "NNP_OK";
    case NNP_EINVAL: return "NNP_EINVAL";
    case NNP_ENOMEM: return "NNP_ENOMEM";
    case NNP_ENEIGH_OVERFLOW: return "NNP_ENEIGH_OVERFLOW";
    case NNP_ENONFINITE: return "NNP_ENONFINITE";
    case NNP_EBOX: return "NNP_EBOX";
    case NNP_ECUDA: return "NNP_ECUDA";
    case NNP_EUNSUPPORTED: return "NNP_EUNSUPPORTED";
    default: return "NNP_UNKNOWN";
    }
}

const char* nnp_last_error(const nnp_handle* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int nnp_num_params(const nnp_handle* h) { return h ? h->n_params : 0; }

int nnp_create(const nnp_params* params, int device, nnp_handle** out)
{
    if (!out) return set_err(nullptr, NNP_EINVAL, "out is NULL");
    *out = nullptr;
    g_create_err.clear();
    Plan P;
    int n_params = 0;
    std::string why;
    int rc = build_plan(params, P, n_params, why);
    if (rc) return set_err(nullptr, rc, "%s", why.c_str());
    if (params->mlp_precision == NNP_BF16 && (params->n_layers != 3 || params->widths[0] > 64))
        return set_err(nullptr, NNP_EUNSUPPORTED,
                       "the BF16 tensor-core network takes two hidden layers (n_layers = 3) and n_G <= 64");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return set_err(nullptr, NNP_ECUDA, "CUDA device %d not available", device);
    nnp_handle* h = new nnp_handle();
    h->device = device;
    h->plan = P;
    h->n_params = n_params;
    h->cutoff = params->cutoff;
    h->skin = params->skin;
    h->stride = (params->max_neighbors + 7) & ~7;   // multiple of 8 keeps per-warp shared arrays 16-byte aligned
    h->precision = params->mlp_precision;
    {
        // force assembly (default: fixed-point integer atomics, reproducible);
        // NNP_FORCE_GATHER=1: per-slot g buffer and reverse-index gather;
        // NNP_FORCE_SCATTER=1: float atomics (the paper's CabanaMD form)
        const char* env = getenv("NNP_FORCE_SCATTER");
        const char* genv2 = getenv("NNP_FORCE_GATHER");
        h->fmode = (genv2 && genv2[0] == '1') ? FM_GATHER : (env && env[0] == '1') ? FM_FLOAT : FM_FIXED;
        // NNP_STEP_GRAPH=0: nnp_step launches every kernel of every step itself
        const char* genv = getenv("NNP_STEP_GRAPH");
        h->step_graph = !(genv && genv[0] == '0');
        // NNP_STAGE_REUSE=0: the force pass stages the neighbours again instead of
        // reading the descriptor pass's staged records
        const char* senv = getenv("NNP_STAGE_REUSE");
        h->use_stg = !(senv && senv[0] == '0');
        const char* oenv = std::getenv("NNP_CELL_ORDER");
        h->cell_order = !(oenv && oenv[0] == '0');
    }
    DeviceGuard g(device);
    auto fail = [&](int code) {
        g_create_err = h->err;
        nnp_destroy(h);
        return code;
    };
#define CKC(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            set_err(h, e_ == cudaErrorMemoryAllocation ? NNP_ENOMEM : NNP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
            return fail(e_ == cudaErrorMemoryAllocation ? NNP_ENOMEM : NNP_ECUDA);                 \
        }                                                                                          \
    } while (0)
    CKC(cudaMalloc((void**)&h->d_plan, sizeof(Plan)));
    CKC(cudaMemcpy(h->d_plan, &P, sizeof(Plan), cudaMemcpyHostToDevice));
    std::vector<float> w(n_params);
    for (int i = 0; i < n_params; ++i) w[i] = (float)params->weights[i];
    CKC(cudaMalloc((void**)&h->d_w, sizeof(float) * (size_t)n_params));
    CKC(cudaMemcpy(h->d_w, w.data(), sizeof(float) * (size_t)n_params, cudaMemcpyHostToDevice));
    CKC(cudaMalloc((void**)&h->flags, sizeof(int) * 4));
    CKC(cudaMemset(h->flags, 0, sizeof(int) * 4));
    CKC(cudaMallocHost((void**)&h->h_flags, sizeof(int) * 4));
    CKC(cudaMalloc((void**)&h->counters, sizeof(unsigned long long) * CNT_N));
    CKC(cudaMemset(h->counters, 0, sizeof(unsigned long long) * CNT_N));
    CKC(cudaMalloc((void**)&h->sys_box, sizeof(float4) * 4));
    CKC(cudaMalloc((void**)&h->d_energy, sizeof(double) * 4));
    CKC(cudaMalloc((void**)&h->elem_off, sizeof(int) * 2 * (NNP_MAXE + 1)));
    CKC(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device));
    int max_smem = 0;
    CKC(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    h->max_smem = max_smem;
    CKC(cudaMallocHost((void**)&h->h_cnt, sizeof(unsigned long long) * CNT_N));
    SfKernel ksf;
    ForceKernel kf;
    TangentKernel kt;
    pick_kernels(P, ksf, kf, kt);
    {
        // wide-capacity pass: capacity = list stride, as many warps as fit (<= 4)
        const size_t ps = sf_smem_per_warp(P, h->stride), pf = force_smem_per_warp(P, h->stride, h->stride);
        if (ps > (size_t)max_smem || pf > (size_t)max_smem) {
            set_err(h, NNP_EINVAL, "max_neighbors = %d needs more shared memory than one block has", h->stride);
            return fail(NNP_EINVAL);
        }
        h->wpb_sf_sp = (int)std::min<size_t>(4, (size_t)max_smem / ps);
        h->wpb_force_sp = (int)std::min<size_t>(4, (size_t)max_smem / pf);
        h->smem_sf_sp = ps * h->wpb_sf_sp;
        h->smem_force_sp = pf * h->wpb_force_sp;
        h->grid_sp = h->num_sms;
    }
    // weight images of every element, then four warps' activation rows
    h->smem_mlp = sizeof(float) * ((size_t)P.lw_elem * P.n_elem + 4 * (size_t)P.lw_rows * 33);
    h->kmlp = pick_mlp(P.lw_hp);
    if (h->smem_mlp > (size_t)max_smem) {
        set_err(h, NNP_EUNSUPPORTED, "network weights do not fit in shared memory");
        return fail(NNP_EUNSUPPORTED);
    }
    // The limit is a property of the kernel, shared by every handle in the process:
    // raise it to the device maximum (never lower it to this handle's need).
    CKC(cudaFuncSetAttribute((const void*)ksf, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    CKC(cudaFuncSetAttribute((const void*)kf, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    {
        SfKernel s3, sw3;
        ForceKernel f3, fs3, fh3;
        TangentKernel t3;
        pick_kernels(P, s3, f3, t3, fs3, sw3, fh3);
        CKC(cudaFuncSetAttribute((const void*)fs3, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
        if (fh3) CKC(cudaFuncSetAttribute((const void*)fh3, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
        CKC(cudaFuncSetAttribute((const void*)sw3, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    }
    CKC(cudaFuncSetAttribute((const void*)kt, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    CKC(cudaFuncSetAttribute((const void*)k_sf_cell, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sf_cell_smem_bytes(4)));
    CKC(cudaFuncSetAttribute((const void*)h->kmlp, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    if (h->precision == NNP_BF16) {
        auto r16 = [](int x) { return (x + 15) & ~15; };
        h->tcs = TcShape{r16(P.width[0]), r16(P.width[1]), r16(P.width[2]), P.gs};
        h->smem_tc = (size_t)((P.n_elem * tc_elem_bytes(h->tcs) + 1023) & ~1023) + tc_tile_bytes(h->tcs);
        if (h->smem_tc > (size_t)max_smem) {
            set_err(h, NNP_EUNSUPPORTED, "BF16 network weights do not fit in shared memory");
            return fail(NNP_EUNSUPPORTED);
        }
        cudaFuncAttributes fa;
        CKC(cudaFuncGetAttributes(&fa, (const void*)k_mlp_tc));   // its static mbarrier counts against the limit
        if (h->smem_tc + fa.sharedSizeBytes > (size_t)max_smem) {
            set_err(h, NNP_EUNSUPPORTED, "BF16 network weights do not fit in shared memory");
            return fail(NNP_EUNSUPPORTED);
        }
        CKC(cudaFuncSetAttribute((const void*)k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - (int)fa.sharedSizeBytes));
    }
    {
        // parameter gradients: two hidden layers, weights and the tangent pass's
        // wide-capacity warp in shared memory
        h->smem_pg = sizeof(float) * (size_t)P.s_elem * (P.n_elem + 4);
        const size_t pt = tangent_warp_bytes(h->stride);
        if (h->smem_pg <= (size_t)max_smem && pt <= (size_t)max_smem && P.n_layers == 3) {
            CKC(cudaFuncSetAttribute((const void*)k_param_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
            h->wpb_tan_sp = (int)std::min<size_t>(4, (size_t)max_smem / pt);
            h->smem_tan_sp = pt * h->wpb_tan_sp;
        } else {
            h->smem_pg = 0;   // gradients unavailable for this model (reported by nnp_param_grad)
        }
    }
    {
        // capacity inside the cutoff: the list's headroom over the same volume
        // ratio, (rc / (rc + skin))^3; re-tuned after every call
        const double ratio = std::pow(params->cutoff / (params->cutoff + params->skin), 3.0);
        int c = (int)std::ceil(h->stride * ratio);
        c = std::min(h->stride, std::max(32, (c + 7) & ~7));
        if (set_capacity(h, c) != NNP_OK) return fail(NNP_EINVAL);
    }
    int bs = 0;
    CKC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, (const void*)h->kmlp, 128, h->smem_mlp));
    h->grid_mlp = std::max(1, bs) * h->num_sms;
#undef CKC
    *out = h;
    return NNP_OK;
}

int nnp_destroy(nnp_handle* h)
{
    if (!h) return NNP_OK;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    void* dev[] = {h->elem_idx, h->elem_part, h->elem_off, h->d_plan, h->d_w, h->off, h->ref, h->pos4, h->Fown, h->G, h->dEdG, h->Ei, h->F, h->nbr,
                   h->ncount, h->rev, h->cell_of, h->cell_atoms, h->cpos, h->gbuf, h->cell_count, h->cell_start, h->cursor,
                   h->epart, h->vpart, h->d_energy, h->d_log, h->flags, h->counters, h->sys_box};
    for (void* p : dev)
        if (p) cudaFree(p);
    for (void* p2 : {(void*)h->sys_of, (void*)h->sys_start_d, (void*)h->T, (void*)h->gpart, (void*)h->spill,
                     (void*)h->qpool, (void*)h->qoff, (void*)h->seg, (void*)h->Fq, (void*)h->stg})
        if (p2) cudaFree(p2);
    if (h->pos_cache) cudaFree(h->pos_cache);
    if (h->types_cache) cudaFree(h->types_cache);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->gfork) cudaEventDestroy(h->gfork);
    if (h->gjoin) cudaEventDestroy(h->gjoin);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    for (auto& p : h->pending) {
        h->ev_pool.push_back(p.a);
        h->ev_pool.push_back(p.b);
    }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->h_flags) cudaFreeHost(h->h_flags);
    if (h->h_cnt) cudaFreeHost(h->h_cnt);
    delete h;
    return NNP_OK;
}

int nnp_set_weights(nnp_handle* h, const float* w, void* stream)
{
    if (!h) return NNP_EINVAL;
    if (!w) return set_err(h, NNP_EINVAL, "weights pointer is NULL");
    DeviceGuard g(h->device);
    CK(h, cudaMemcpyAsync(h->d_w, w, sizeof(float) * (size_t)h->n_params, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return NNP_OK;
}

static int common_args(nnp_handle* h, int n, const float* pos, const int* types, const double* box)
{
    if (n < 0) return set_err(h, NNP_EINVAL, "n_atoms must be >= 0");
    if (n > (int)NB_INDEX_MASK) return set_err(h, NNP_EINVAL, "n_atoms must be < 2^24");
    if (n > 0 && (!pos || !types)) return set_err(h, NNP_EINVAL, "pos and types must not be NULL");
    return check_box(h, box);
}

int nnp_compute(nnp_handle* h, int n, const float* pos, const int* types, const double* box, double cutoff,
                double* energy, float* atom_energy, float* forces, double* virial, void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    int rc = common_args(h, n, pos, types, box);
    if (rc) return rc;
    if (cutoff > 0.0 && std::fabs(cutoff - h->cutoff) > 1e-12 * h->cutoff)
        return set_err(h, NNP_EINVAL, "cutoff %g differs from the model cutoff %g", cutoff, h->cutoff);
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        if (energy) CK(h, cudaMemsetAsync(energy, 0, sizeof(double), st));
        if (virial) CK(h, cudaMemsetAsync(virial, 0, 9 * sizeof(double), st));
        CK(h, cudaStreamSynchronize(st));
        return NNP_OK;
    }
    h->step_valid = false;
    rc = begin_call(h, st);
    if (rc) return rc;
    rc = run_eval(h, n, pos, types, box, st, energy, atom_energy, forces, virial, nullptr, nullptr, 0);
    if (rc) return rc;
    return read_status(h, st);
}

int nnp_compute_domain(nnp_handle* h, int n, int n_owned, const float* pos, const int* types, const double* box,
                       double* energy, float* atom_energy, float* forces, double* virial, void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    if (n_owned < 0 || n_owned > n) return set_err(h, NNP_EINVAL, "n_owned must be in 0..n_atoms");
    int rc = common_args(h, n, pos, types, box);
    if (rc) return rc;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        if (energy) CK(h, cudaMemsetAsync(energy, 0, sizeof(double), st));
        if (virial) CK(h, cudaMemsetAsync(virial, 0, 9 * sizeof(double), st));
        CK(h, cudaStreamSynchronize(st));
        return NNP_OK;
    }
    h->step_valid = false;
    rc = begin_call(h, st);
    if (rc) return rc;
    rc = run_eval(h, n, pos, types, box, st, energy, atom_energy, forces, virial, nullptr, nullptr, 0, nullptr,
                  n_owned);
    if (rc) return rc;
    return read_status(h, st);
}

int nnp_descriptors(nnp_handle* h, int n, const float* pos, const int* types, const double* box, float* G,
                    float* dEdG, void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    int rc = common_args(h, n, pos, types, box);
    if (rc) return rc;
    if (n == 0) return NNP_OK;
    DeviceGuard g(h->device);
    h->step_valid = false;
    rc = begin_call(h, (cudaStream_t)stream);
    if (rc) return rc;
    return run_eval(h, n, pos, types, box, (cudaStream_t)stream, nullptr, nullptr, nullptr, nullptr, G, dEdG,
                    dEdG ? 2 : 1);
}

int nnp_descriptors_flat(nnp_handle* h, int n, const float* pos, const int* types, const double* box, float* G,
                         void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    if (!G) return set_err(h, NNP_EINVAL, "G must not be NULL");
    if (h->plan.resolved)
        return set_err(h, NNP_EUNSUPPORTED, "the thread-per-atom descriptors do not resolve angular pair classes");
    int rc = common_args(h, n, pos, types, box);
    if (rc) return rc;
    if (n == 0) return NNP_OK;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    h->step_valid = false;
    rc = begin_call(h, st);
    if (rc) return rc;
    // neighbour list (and the warp-per-atom pass, which this call does not return)
    rc = run_eval(h, n, pos, types, box, st, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1);
    if (rc) return rc;
    Box bx;
    for (int a = 0; a < 3; ++a) bx.L[a] = (float)box[a];
    NbView nv{h->nbr, h->ncount, h->stride};
    {
        KScope ks(h, KG_FLAT, st);
        k_sf_flat<<<blocks_for(n, 128), 128, 0, st>>>(n, h->pos4, bx, nv, h->d_plan, G, h->flags);
    }
    return read_status(h, st);
}

int nnp_descriptors_pair(nnp_handle* h, int n, const float* pos, const int* types, const double* box, float* G,
                         void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    if (!G) return set_err(h, NNP_EINVAL, "G must not be NULL");
    if (h->plan.resolved)
        return set_err(h, NNP_EUNSUPPORTED, "the atom-by-neighbour descriptors do not resolve angular pair classes");
    int rc = common_args(h, n, pos, types, box);
    if (rc) return rc;
    if (n == 0) return NNP_OK;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    h->step_valid = false;
    rc = begin_call(h, st);
    if (rc) return rc;
    // neighbour list (and the warp-per-atom pass, which this call does not return)
    rc = run_eval(h, n, pos, types, box, st, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1);
    if (rc) return rc;
    Box bx;
    for (int a = 0; a < 3; ++a) bx.L[a] = (float)box[a];
    NbView nv{h->nbr, h->ncount, h->stride};
    // G rows are n_G floats; every element shares the model's n_G (widths[0])
    CK(h, cudaMemsetAsync(G, 0, sizeof(float) * (size_t)n * h->plan.width[0], st));
    {
        KScope ks(h, KG_PAIR, st);
        const long long items = (long long)n * h->stride;
        const int grid = (int)std::min<long long>((items + 127) / 128, (long long)h->num_sms * 16);
        k_sf_pair<<<grid, 128, 0, st>>>(n, h->pos4, bx, nv, h->d_plan, G, h->flags);
    }
    return read_status(h, st);
}

int nnp_descriptors_cell(nnp_handle* h, int n, const float* pos, const int* types, const double* box, float* G,
                         void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    if (!G) return set_err(h, NNP_EINVAL, "G must not be NULL");
    if (h->plan.resolved)
        return set_err(h, NNP_EUNSUPPORTED, "the CTA-per-cell descriptors do not resolve angular pair classes");
    int rc = common_args(h, n, pos, types, box);
    if (rc) return rc;
    if (n == 0) return NNP_OK;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    h->step_valid = false;
    rc = begin_call(h, st);
    if (rc) return rc;
    // neighbour list and cell binning (and the warp-per-atom pass, not returned)
    rc = run_eval(h, n, pos, types, box, st, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1);
    if (rc) return rc;
    if (!h->cell_path)
        return set_err(h, NNP_EUNSUPPORTED, "the CTA-per-cell descriptors need at least 3 cells of cutoff + skin per edge");
    Box bx;
    for (int a = 0; a < 3; ++a) bx.L[a] = (float)box[a];
    {
        KScope ks(h, KG_CELL, st);
        const int ncell = h->nc[0] * h->nc[1] * h->nc[2];
        k_sf_cell<<<std::min(ncell, h->num_sms * 4), 128, sf_cell_smem_bytes(4), st>>>(
            h->nc[0], h->nc[1], h->nc[2], h->pos4, bx, h->cell_start, h->cell_atoms, h->d_plan, G, h->flags);
    }
    return read_status(h, st);
}

int nnp_step(nnp_handle* h, int n, float* pos, float* vel, const int* types, const double* box, double dt_fs,
             int n_steps, double* log, void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    int rc = common_args(h, n, pos, types, box);
    if (rc) return rc;
    if (n > 0 && !vel) return set_err(h, NNP_EINVAL, "vel must not be NULL");
    if (!(dt_fs > 0.0) || !std::isfinite(dt_fs)) return set_err(h, NNP_EINVAL, "dt_fs must be > 0");
    if (n_steps < 0) return set_err(h, NNP_EINVAL, "n_steps must be >= 0");
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        if (log) CK(h, cudaMemsetAsync(log, 0, sizeof(double) * 2 * ((size_t)n_steps + 1), st));
        CK(h, cudaStreamSynchronize(st));
        return NNP_OK;
    }
    if (!log) {
        if (h->cap_log < n_steps + 1) {
            CK(h, regrow(h->d_log, 2 * ((size_t)n_steps + 1)));
            h->cap_log = n_steps + 1;
        }
        log = h->d_log;
    }
    const int gke = std::min(blocks_for(n, 256), 4 * h->num_sms);
    rc = ensure_red(h, gke, 0);
    if (rc) return rc;
    const float dt = (float)dt_fs;
    rc = begin_call(h, st);
    if (rc) return rc;
    CK(h, cudaMemsetAsync(h->counters + CNT_LOGSLOT, 0, sizeof(unsigned long long), st));
    // continue from the previous nnp_step if its final state is bitwise unchanged
    bool cont = h->step_valid && h->step_n == n && h->step_pos == pos && h->step_types == types;
    for (int a = 0; a < 3; ++a) cont = cont && (h->step_box[a] == box[a]);
    if (cont) {
        CK(h, cudaMemsetAsync(h->flags + 2, 0, sizeof(int), st));
        k_same<<<blocks_for(n, 256), 256, 0, st>>>(n, pos, h->pos_cache, types, h->types_cache, h->flags + 2);
        h->launches++;
        CK(h, cudaMemcpyAsync(h->h_flags + 2, h->flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(h, cudaStreamSynchronize(st));
        cont = (h->h_flags[2] == 0);
    }
    h->step_valid = false;
    // the energy of the starting state: still in d_energy when continuing
    if (!cont) {
        rc = run_eval(h, n, pos, types, box, st, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
        if (rc) return rc;
    }
    // the kinetic-energy partials reuse the energy partial buffer (same block count)
    rc = ensure_red(h, gke, 0);
    if (rc) return rc;
    {
        KScope ks(h, KG_INTEGRATE, st, 2);
        k_kick_ke<<<gke, 256, 0, st>>>(n, h->d_plan, types, h->F, vel, 0.f, h->epart);
        k_log_sum<<<1, 256, 0, st>>>(gke, h->epart, h->d_energy, log, h->counters + CNT_LOGSLOT);
    }
    int k = 1;
    if (n_steps >= 3 && h->step_graph && !h->prof_on) {
        // the first step runs directly and settles every buffer; the rest repeat
        // its launch sequence with the same arguments
        rc = md_step(h, n, pos, vel, types, box, dt, gke, log, st);
        if (rc) return rc;
        rc = replay_steps(h, n, pos, vel, types, box, dt, gke, log, n_steps - 1, st);
        if (rc) return rc;
        k = n_steps + 1;
    }
    for (; k <= n_steps; ++k) {
        rc = md_step(h, n, pos, vel, types, box, dt, gke, log, st);
        if (rc) return rc;
    }
    // remember the final state for a continuing call (its energy stays in d_energy)
    CK(h, cudaMemcpyAsync(h->pos_cache, pos, sizeof(float) * 3 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    CK(h, cudaMemcpyAsync(h->types_cache, types, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    rc = read_status(h, st);
    if (rc) return rc;
    h->step_valid = true;
    h->step_n = n;
    h->step_pos = pos;
    h->step_types = types;
    for (int a = 0; a < 3; ++a) h->step_box[a] = box[a];
    return NNP_OK;
}

static int batch_args(nnp_handle* h, int B, const int* start, const double* boxes, const float* pos, const int* types,
                      int& n)
{
    if (B < 1 || !start || !boxes) return set_err(h, NNP_EINVAL, "n_systems must be >= 1 with start and boxes");
    if (start[0] != 0) return set_err(h, NNP_EINVAL, "sys_start[0] must be 0");
    for (int b = 0; b < B; ++b) {
        if (start[b + 1] < start[b]) return set_err(h, NNP_EINVAL, "sys_start must be non-decreasing");
        int rc = check_box(h, boxes + 3 * b);
        if (rc) return rc;
        for (int a = 0; a < 3; ++a)
            if ((int)std::ceil((h->cutoff + h->skin) / boxes[3 * b + a]) > 2)
                return set_err(h, NNP_EBOX, "box of system %d too small for the image range", b);
    }
    n = start[B];
    if (n > (int)NB_INDEX_MASK) return set_err(h, NNP_EINVAL, "n_atoms must be < 2^24");
    // systems of a multi-system batch are searched by brute force over images (cost ~ N_b^2)
    if (B > 1)
        for (int b = 0; b < B; ++b)
            if (start[b + 1] - start[b] > 16384)
                return set_err(h, NNP_EINVAL, "system %d of a batch has %d atoms; batch systems are limited to 16384 "
                               "(a single system of any size takes the cell-list path)", b, start[b + 1] - start[b]);
    if (n > 0 && (!pos || !types)) return set_err(h, NNP_EINVAL, "pos and types must not be NULL");
    return NNP_OK;
}

int nnp_compute_batch(nnp_handle* h, int B, const int* start, const double* boxes, const float* pos,
                      const int* types, double* energies, float* atom_energy, float* forces, void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    int n = 0;
    int rc = batch_args(h, B, start, boxes, pos, types, n);
    if (rc) return rc;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    h->step_valid = false;
    if (n == 0) {
        if (energies) CK(h, cudaMemsetAsync(energies, 0, sizeof(double) * B, st));
        CK(h, cudaStreamSynchronize(st));
        return NNP_OK;
    }
    rc = begin_call(h, st);
    if (rc) return rc;
    Batch bt{B, start, boxes};
    // one system: the single-system path (cell lists for large boxes)
    rc = run_eval(h, n, pos, types, boxes, st, energies, atom_energy, forces, nullptr, nullptr, nullptr, 0,
                  B > 1 ? &bt : nullptr);
    if (rc) return rc;
    return read_status(h, st);
}

int nnp_param_grad(nnp_handle* h, int B, const int* start, const double* boxes, const float* pos,
                   const int* types, const double* dLdE, const float* dLdF, float* grad, void* stream)
{
    if (!h) return NNP_EINVAL;
    h->err.clear();
    if (!grad) return set_err(h, NNP_EINVAL, "grad must not be NULL");
    if (h->smem_pg == 0)
        return set_err(h, NNP_EUNSUPPORTED, "parameter gradients need two hidden layers (n_layers = 3)");
    int n = 0;
    int rc = batch_args(h, B, start, boxes, pos, types, n);
    if (rc) return rc;
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    h->step_valid = false;
    CK(h, cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)h->n_params, st));
    if (n == 0 || (!dLdE && !dLdF)) {
        CK(h, cudaStreamSynchronize(st));
        return NNP_OK;
    }
    rc = begin_call(h, st);
    if (rc) return rc;
    Batch bt{B, start, boxes};
    const Batch* btp = B > 1 ? &bt : nullptr;
    // descriptors G~ of the current positions (stop after the descriptor pass)
    rc = run_eval(h, n, pos, types, boxes, st, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1, btp);
    if (rc) return rc;
    const Plan& P = h->plan;
    Box bx;
    for (int a = 0; a < 3; ++a) bx.L[a] = (float)boxes[a];
    if (dLdF) {
        SfKernel ksf;
        ForceKernel kf;
        TangentKernel kt;
        pick_kernels(P, ksf, kf, kt);
        NbView nv{h->nbr, h->ncount, h->stride};
        if (btp) {
            nv.sys_of = h->sys_of;
            nv.sys_box = h->sys_box;
        }
        KScope ks(h, KG_FORCE, st, 2);
        kt<<<std::min(blocks_for(n, h->wpb_tan), h->grid_tan), 32 * h->wpb_tan, h->smem_tan, st>>>(
            n, h->pos4, bx, nv, h->d_plan, h->cap_rc, dLdF, h->T, h->flags, h->spill, 0);
        kt<<<h->grid_sp, 32 * h->wpb_tan_sp, h->smem_tan_sp, st>>>(n, h->pos4, bx, nv, h->d_plan, h->stride, dLdF, h->T,
                                                                   h->flags, h->spill, 1);
    }
    const int gpg = std::min(blocks_for(n, 4), 2 * h->num_sms);
    const int nwarps = gpg * 4;
    const size_t need = (size_t)nwarps * P.n_elem * P.n_params_elem;
    if (need > h->cap_gpart) {
        CK(h, regrow(h->gpart, need));
        h->cap_gpart = need;
    }
    {
        KScope ks(h, KG_MLP, st, 6);
        const int nblk = blocks_for(n, 256);
        int* toff = h->elem_off + NNP_MAXE + 1;
        k_elem_count<<<nblk, 256, 0, st>>>(n, h->pos4, P.n_elem, h->elem_part);
        k_elem_scan<<<1, 1024, 0, st>>>(nblk, P.n_elem, h->elem_part, h->elem_off, toff);
        k_elem_fill<<<nblk, 256, 0, st>>>(n, h->pos4, P.n_elem, h->elem_part, h->elem_idx);
        CK(h, cudaMemsetAsync(h->gpart, 0, sizeof(float) * need, st));
        k_param_grad<<<gpg, 128, h->smem_pg, st>>>(n, h->d_plan, h->d_w, h->pos4, h->elem_idx, btp ? h->sys_of : nullptr,
                                                   dLdE, h->G,
                                                   dLdF ? h->T : nullptr, h->gpart);
        k_grad_reduce<<<blocks_for(h->n_params, 256), 256, 0, st>>>(nwarps, P.n_elem, P.n_params_elem, h->gpart, grad);
    }
    return read_status(h, st);
}

int nnp_profile(nnp_handle* h, int enable)
{
    if (!h) return NNP_EINVAL;
    DeviceGuard g(h->device);
    CK(h, cudaDeviceSynchronize());
    prof_flush(h);
    for (int k = 0; k < KG_N; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
    }
    h->prof_on = enable != 0;
    return NNP_OK;
}

int nnp_num_kernel_groups(void) { return KG_N; }

const char* nnp_kernel_group_name(int k) { return (k >= 0 && k < KG_N) ? kKgName[k] : ""; }

int nnp_kernel_times(nnp_handle* h, int max_groups, double* total_ms, long long* launches)
{
    if (!h || max_groups < 0 || (max_groups > 0 && (!total_ms || !launches))) return NNP_EINVAL;
    DeviceGuard g(h->device);
    CK(h, cudaDeviceSynchronize());
    prof_flush(h);
    const int m = std::min(max_groups, (int)KG_N);
    for (int k = 0; k < m; ++k) {
        total_ms[k] = h->prof_ms[k];
        launches[k] = h->prof_n[k];
    }
    return m;
}

static float __uint_as_float_host(unsigned u)
{
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

int nnp_get_stats(nnp_handle* h, nnp_stats* out)
{
    if (!h || !out) return NNP_EINVAL;
    DeviceGuard g(h->device);
    unsigned long long c[CNT_N];
    CK(h, cudaDeviceSynchronize());
    CK(h, cudaMemcpy(c, h->counters, sizeof c, cudaMemcpyDeviceToHost));
    out->n_atoms = h->list_n;
    out->list_entries = (long long)c[CNT_LIST];
    out->cutoff_entries = (long long)c[CNT_RC];
    out->pairs = (long long)c[CNT_PAIRS];
    out->triplets = (long long)c[CNT_TRIPLETS];
    out->rebuilds = (long long)c[CNT_REBUILDS];
    out->kernel_launches = h->launches;
    out->max_list_row = (long long)c[CNT_MAXLIST];
    out->max_cutoff_row = (long long)c[CNT_MAXRC];
    out->spilled_atoms = (long long)c[CNT_SPILL];
    out->rc_capacity = h->cap_rc;
    out->min_distance = c[CNT_MINR] ? (double)__uint_as_float_host((unsigned)(0xffffffffull - c[CNT_MINR])) : -1.0;
    return NNP_OK;
}

}  // extern "C"

// ---------------------------------------------------- allocation-free evaluation
// nnp_compute_static: the evaluation of run_eval for one small system, with all
// per-call scratch carved from a file-scope device array instead of allocated.
static __device__ __align__(256) unsigned char g_static_pool[NNP_STATIC_SCRATCH_BYTES];

namespace {

const int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices];   // device address of g_static_pool, looked up once per device
bool g_static_ready[kMaxDevices];

// Host-side carving of the pool (pointer arithmetic only); base == nullptr sizes it.
struct Carve {
    unsigned char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

int static_fail(char* eb, int el, int code, const char* fmt, ...) __attribute__((format(printf, 4, 5)));
int static_fail(char* eb, int el, int code, const char* fmt, ...)
{
    if (eb && el > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(eb, (size_t)el, fmt, ap);
        va_end(ap);
    }
    return code;
}

}  // namespace

extern "C" int nnp_compute_static(const nnp_handle* h, int n, const float* pos, const int* types, const double* box,
                                  double* energy, float* atom_energy, float* forces, char* eb, int el, void* stream)
{
    if (eb && el > 0) eb[0] = '\0';
    if (!h) return static_fail(eb, el, NNP_EINVAL, "handle is NULL");
    if (n < 0 || n > NNP_STATIC_MAX_ATOMS)
        return static_fail(eb, el, NNP_EINVAL, "n_atoms = %d is outside 0..%d, the limit of nnp_compute_static",
                           n, NNP_STATIC_MAX_ATOMS);
    if (n > 0 && (!pos || !types)) return static_fail(eb, el, NNP_EINVAL, "pos and types must not be NULL");
    if (!box) return static_fail(eb, el, NNP_EINVAL, "box is NULL");
    const double rcut = h->cutoff + h->skin;
    int nim = 0;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !std::isfinite(box[a]))
            return static_fail(eb, el, NNP_EBOX, "box edges must be finite and > 0");
        if (box[a] < 0.5 * rcut)
            return static_fail(eb, el, NNP_EBOX, "box edge %g is below (cutoff + skin) / 2 = %g", box[a], 0.5 * rcut);
        nim = std::max(nim, (int)std::ceil(rcut / box[a]));
    }
    if (h->device < 0 || h->device >= kMaxDevices) return static_fail(eb, el, NNP_ECUDA, "device index out of range");
    if (h->precision != NNP_FP32)
        return static_fail(eb, el, NNP_EUNSUPPORTED, "nnp_compute_static evaluates FP32 networks only");
    const Plan& P = h->plan;
    const int S = h->stride, T = 256;
    const int gf = std::min(blocks_for(std::max(n, 1), h->wpb_force), h->grid_force);
    const int gred = std::min(blocks_for(std::max(n, 1), T), 4 * h->num_sms);

    // scratch layout (the same carving sizes and places it)
    auto layout = [&](Carve& c, int** flags, unsigned long long** counters, float4** sys_box, float4** off, float4** ref,
                      float4** pos4, uint32_t** nbr, int** ncount, int** rev, float** G, float** dEdG, float** Ei,
                      float4** gbuf, float4** Fown, double** epart, float** F, int** spill) {
        *flags = c.take<int>(4);
        *counters = c.take<unsigned long long>(CNT_N);
        *sys_box = c.take<float4>(1);
        *off = c.take<float4>(n);
        *ref = c.take<float4>(n);
        *pos4 = c.take<float4>(n);
        *nbr = c.take<uint32_t>((size_t)n * S);
        *ncount = c.take<int>(n);
        *rev = c.take<int>((size_t)n * S);
        *G = c.take<float>((size_t)n * P.gs);
        *dEdG = c.take<float>((size_t)n * P.gs);
        *Ei = c.take<float>(n);
        *gbuf = c.take<float4>((size_t)n * S);
        *Fown = c.take<float4>(n);
        *epart = c.take<double>(gred);
        *F = c.take<float>((size_t)n * 3);
        *spill = c.take<int>((size_t)n + 1);
    };
    int* flags;
    unsigned long long* counters;
    float4 *sys_box, *off, *ref, *pos4, *gbuf, *Fown;
    uint32_t* nbr;
    int *ncount, *rev, *spill;
    float *G, *dEdG, *Ei, *Fs;
    double* epart;
    {
        Carve dry{nullptr};
        layout(dry, &flags, &counters, &sys_box, &off, &ref, &pos4, &nbr, &ncount, &rev, &G, &dEdG, &Ei, &gbuf, &Fown,
               &epart, &Fs, &spill);
        if (dry.off > NNP_STATIC_SCRATCH_BYTES)
            return static_fail(eb, el, NNP_EINVAL,
                               "needs %zu bytes of scratch for n_atoms = %d and max_neighbors = %d; the static "
                               "scratch array holds %u bytes",
                               dry.off, n, S, (unsigned)NNP_STATIC_SCRATCH_BYTES);
    }

    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ready[h->device]) {
            // In host code g_static_pool names a host-side stand-in; the kernels need
            // the device address, looked up here once with the device current.
            cudaError_t e = cudaGetSymbolAddress(&g_static_addr[h->device], g_static_pool);
            if (e != cudaSuccess)
                return static_fail(eb, el, NNP_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_static_ready[h->device] = true;
        }
        base = g_static_addr[h->device];
    }
    Carve c{static_cast<unsigned char*>(base)};
    layout(c, &flags, &counters, &sys_box, &off, &ref, &pos4, &nbr, &ncount, &rev, &G, &dEdG, &Ei, &gbuf, &Fown, &epart,
           &Fs, &spill);

#define CKS(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return static_fail(eb, el, NNP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
    if (n == 0) {
        if (energy) CKS(cudaMemsetAsync(energy, 0, sizeof(double), st));
        CKS(cudaStreamSynchronize(st));
        return NNP_OK;
    }
    // what must start at zero: the error word, the work counters, the spill count;
    // the rebuild flag is set
    CKS(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
    CKS(cudaMemsetAsync(spill, 0, sizeof(int), st));
    CKS(cudaMemsetAsync(flags + FLAG_REBUILD, 1, sizeof(int), st));
    CKS(cudaMemsetAsync(counters, 0, CNT_N * sizeof(unsigned long long), st));
    Box bx;
    for (int a = 0; a < 3; ++a) bx.L[a] = (float)box[a];
    const float4 sb = make_float4(bx.L[0], bx.L[1], bx.L[2], (float)nim);
    CKS(cudaMemcpyAsync(sys_box, &sb, sizeof(float4), cudaMemcpyHostToDevice, st));

    const int rows_grid = std::min(blocks_for(n, 8), h->num_sms * 8);
    k_rebuild_pos<<<blocks_for(n, T), T, 0, st>>>(n, pos, types, bx, P.n_elem, off, pos4, ref, flags, counters);
    k_rows_brute<<<rows_grid, 256, 0, st>>>(n, pos4, nullptr, nullptr, sys_box, P.rcut2, S, nbr, ncount, flags);
    k_rev<<<rows_grid, 256, 0, st>>>(n, nbr, ncount, S, rev, flags);
    NbView nv{nbr, ncount, S};
    SfKernel ksf;
    ForceKernel kf;
    pick_kernels(P, ksf, kf);
    const int gsf = std::min(blocks_for(n, h->wpb_sf), h->grid_sf);
    sf_for(P, h->cap_rc)<<<gsf, 32 * h->wpb_sf, h->smem_sf, st>>>(n, pos4, bx, nv, h->d_plan, h->cap_rc, G, nullptr, flags, counters,
                                                 spill, 0, nullptr, nullptr, 0ull, nullptr, 0);
    sf_for(P, S)<<<h->grid_sp, 32 * h->wpb_sf_sp, h->smem_sf_sp, st>>>(n, pos4, bx, nv, h->d_plan, S, G, nullptr, flags, counters,
                                                             spill, 1, nullptr, nullptr, 0ull, nullptr, 0);
    const int gmlp = std::min(blocks_for(n, 128), h->grid_mlp);
    h->kmlp<<<gmlp, 128, h->smem_mlp, st>>>(n, pos4, h->d_plan, h->d_w, G, Ei, dEdG);
    // no virial output: the force passes write no virial partials
    kf<<<gf, 32 * h->wpb_force, h->smem_force, st>>>(n, pos4, bx, nv, h->d_plan, h->cap_rc, dEdG, gbuf, Fown, nullptr,
                                                     0, flags, spill, 0, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0ull);
    kf<<<h->grid_sp, 32 * h->wpb_force_sp, h->smem_force_sp, st>>>(n, pos4, bx, nv, h->d_plan, S, dEdG, gbuf, Fown,
                                                                   nullptr, 0, flags, spill, 1, nullptr, nullptr, nullptr,
                                                                   nullptr, nullptr, 0, 0ull);
    k_gather<<<rows_grid, 256, 0, st>>>(n, nv, rev, gbuf, Fown, forces ? forces : Fs, flags);
    k_sum_partial<<<gred, T, 0, st>>>(n, Ei, epart, flags);
    k_finalize<<<1, 256, 0, st>>>(gred, epart, energy, 0, nullptr, nullptr);
    if (atom_energy) CKS(cudaMemcpyAsync(atom_energy, Ei, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    CKS(cudaGetLastError());
    int hf = 0;
    CKS(cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKS(cudaStreamSynchronize(st));
#undef CKS
    if (hf) {
        char msg[256];
        const int status = error_word_status(hf, S, CELL_CAP, (double)FX_LIMIT, msg, sizeof msg);
        return static_fail(eb, el, status, "%s", msg);
    }
    return NNP_OK;
}
