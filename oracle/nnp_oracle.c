/*
 * nnp_oracle.c -- plain FP64 CPU oracle for the Behler-Parrinello NNP hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, and where the paper defines it (arXiv 2002.00054):
 *   - cosine cutoff f_c(r) = 0.5 (cos(pi r / r_c) + 1) for r < r_c, 0 otherwise;
 *   - radial descriptor  G2 = sum_j exp(-eta (r_ij - r_s)^2) f_c(r_ij)      (Fig. 1b, step 1);
 *   - angular descriptors, the "extra loop over neighbours of neighbours" of
 *     Sec. 3.1 (the formula is not printed in the paper; the standard Behler
 *     narrow and wide angular functions are used):
 *       narrow: 2^(1-zeta) sum_{j<k} (1 + lambda cos t_ijk)^zeta
 *                   exp(-eta (r_ij^2 + r_ik^2 + r_jk^2)) f_c(r_ij) f_c(r_ik) f_c(r_jk)
 *       wide:   the same without the r_jk^2 term and without f_c(r_jk);
 *   - per-element feed-forward network E_i = NN_e(G~_i), G~ = (G - mu)/s,
 *     tanh hidden layers, linear output                                       (Fig. 1b, step 2; Sec. 3.1);
 *   - E = sum_i E_i                                                           (Fig. 1b);
 *   - forces f = -dE/dr by the chain rule dE_j/dG_j,k * dG_j,k/dr             (Fig. 1b, step 3);
 *   - virial W_ab = -sum_pairs d^a g^b with g = dE_i/dd_ij (pair form);
 *   - velocity-Verlet NVE integration (energy conservation, Sec. 4.2);
 *   - the force-matching parameter gradient (energy term plus the
 *     reverse-over-forward "double backward" of the force term).
 *
 * Every loop is the plain definition: neighbours by brute force over periodic
 * images (or by a cell list that the tests pin to the brute force), descriptor
 * derivatives per function and per neighbour entry, no fusion and no blocking.
 * Atom-level loops may run under OpenMP; each atom's work is independent, and
 * all cross-atom sums (energy, forces, virial, gradients) are done serially in
 * atom order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXE 8
#define OR_MAXL 8

enum { OR_RADIAL = 2, OR_NARROW = 3, OR_WIDE = 4 };

/* The oracle's own model description (mirrored by a ctypes Structure). */
typedef struct {
    int n_elem;
    double rc;
    int n_sf[OR_MAXE];      /* descriptors per centre element                 */
    int sf_off[OR_MAXE];    /* offset of element e's descriptors in sf_*      */
    const int* sf_type;     /* OR_RADIAL / OR_NARROW / OR_WIDE                */
    const int* sf_e1;       /* radial: neighbour element (-1 any); angular: pair filter */
    const int* sf_e2;
    const double* sf_eta;
    const double* sf_rs;
    const double* sf_zeta;
    const double* sf_lambda;
    const double* sf_mu;    /* scaling shift per descriptor  */
    const double* sf_s;     /* scaling divisor per descriptor */
    int n_layers;           /* weight layers, e.g. 3 for n_G-25-25-1          */
    int width[OR_MAXL + 1]; /* width[0] = n_G, width[n_layers] = 1            */
    int w_off[OR_MAXE];     /* offset of element e's parameters in w          */
    const double* w;        /* per layer: W [out][in] row-major, then b [out] */
} or_model;

/* One periodic orthorhombic system. */
typedef struct {
    int n;
    const double* pos;  /* [n][3] */
    const int* type;    /* [n]    */
    double box[3];
} or_system;

typedef struct { int j; double d[3]; double r; } or_nb;
typedef struct { int n, cap; or_nb* e; } or_nblist;

/* ------------------------------------------------------------------ cutoff */
static double fcut(double r, double rc)
{
    if (r >= rc) return 0.0;
    return 0.5 * (cos(M_PI * r / rc) + 1.0);
}
static double dfcut(double r, double rc)
{
    if (r >= rc) return 0.0;
    return -0.5 * M_PI / rc * sin(M_PI * r / rc);
}

/* -------------------------------------------------------------- neighbours */
static int nb_push(or_nblist* L, int j, const double d[3], double r)
{
    if (L->n == L->cap) {
        int nc = L->cap ? 2 * L->cap : 64;
        or_nb* ne = (or_nb*)realloc(L->e, (size_t)nc * sizeof(or_nb));
        if (!ne) return -1;
        L->e = ne;
        L->cap = nc;
    }
    or_nb* x = &L->e[L->n++];
    x->j = j;
    x->d[0] = d[0]; x->d[1] = d[1]; x->d[2] = d[2];
    x->r = r;
    return 0;
}

static void wrap_all(const or_system* s, double* w)
{
    for (int i = 0; i < s->n; ++i)
        for (int a = 0; a < 3; ++a) {
            double L = s->box[a];
            w[3 * i + a] = s->pos[3 * i + a] - L * floor(s->pos[3 * i + a] / L);
        }
}

/* Brute force: every atom j and every periodic image with |d| < rc, except i itself
 * at zero shift.  Used for small systems and as the pin for the cell list. */
static int nb_brute_one(const or_system* s, const double* w, double rc, int i, or_nblist* L)
{
    int nimg[3];
    for (int a = 0; a < 3; ++a) nimg[a] = (int)ceil(rc / s->box[a]) + 1;
    for (int j = 0; j < s->n; ++j)
        for (int sx = -nimg[0]; sx <= nimg[0]; ++sx)
            for (int sy = -nimg[1]; sy <= nimg[1]; ++sy)
                for (int sz = -nimg[2]; sz <= nimg[2]; ++sz) {
                    if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
                    double d[3];
                    d[0] = w[3 * j + 0] - w[3 * i + 0] + sx * s->box[0];
                    d[1] = w[3 * j + 1] - w[3 * i + 1] + sy * s->box[1];
                    d[2] = w[3 * j + 2] - w[3 * i + 2] + sz * s->box[2];
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 < rc * rc)
                        if (nb_push(L, j, d, sqrt(r2))) return -1;
                }
    return 0;
}

typedef struct { int nc[3]; int* start; int* list; } or_cells;

static int cells_build(const or_system* s, const double* w, double rc, or_cells* C)
{
    int ncell = 1;
    for (int a = 0; a < 3; ++a) {
        C->nc[a] = (int)floor(s->box[a] / rc);
        if (C->nc[a] < 3) return 1; /* too few cells: caller falls back to brute force */
        ncell *= C->nc[a];
    }
    int* cnt = (int*)calloc((size_t)ncell + 1, sizeof(int));
    int* cid = (int*)malloc(sizeof(int) * (size_t)(s->n > 0 ? s->n : 1));
    C->start = (int*)calloc((size_t)ncell + 1, sizeof(int));
    C->list = (int*)malloc(sizeof(int) * (size_t)(s->n > 0 ? s->n : 1));
    if (!cnt || !cid || !C->start || !C->list) return -1;
    for (int i = 0; i < s->n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = (int)floor(w[3 * i + a] / s->box[a] * C->nc[a]);
            if (c[a] < 0) c[a] = 0;
            if (c[a] >= C->nc[a]) c[a] = C->nc[a] - 1;
        }
        cid[i] = (c[2] * C->nc[1] + c[1]) * C->nc[0] + c[0];
        cnt[cid[i]]++;
    }
    for (int c = 0; c < ncell; ++c) C->start[c + 1] = C->start[c] + cnt[c];
    memset(cnt, 0, sizeof(int) * (size_t)ncell);
    for (int i = 0; i < s->n; ++i) C->list[C->start[cid[i]] + cnt[cid[i]]++] = i;
    free(cnt);
    free(cid);
    return 0;
}

/* Cell list: bins of edge >= rc, 27-cell stencil with periodic shifts. */
static int nb_cell_one(const or_system* s, const double* w, double rc, const or_cells* C, int i, or_nblist* L)
{
    int ci[3];
    for (int a = 0; a < 3; ++a) {
        ci[a] = (int)floor(w[3 * i + a] / s->box[a] * C->nc[a]);
        if (ci[a] < 0) ci[a] = 0;
        if (ci[a] >= C->nc[a]) ci[a] = C->nc[a] - 1;
    }
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int c[3] = { ci[0] + dx, ci[1] + dy, ci[2] + dz };
                double sh[3];
                for (int a = 0; a < 3; ++a) {
                    sh[a] = 0.0;
                    if (c[a] < 0) { c[a] += C->nc[a]; sh[a] = -s->box[a]; }
                    else if (c[a] >= C->nc[a]) { c[a] -= C->nc[a]; sh[a] = s->box[a]; }
                }
                int cc = (c[2] * C->nc[1] + c[1]) * C->nc[0] + c[0];
                for (int p = C->start[cc]; p < C->start[cc + 1]; ++p) {
                    int j = C->list[p];
                    double d[3];
                    for (int a = 0; a < 3; ++a) d[a] = w[3 * j + a] + sh[a] - w[3 * i + a];
                    if (j == i && sh[0] == 0.0 && sh[1] == 0.0 && sh[2] == 0.0) continue;
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 < rc * rc)
                        if (nb_push(L, j, d, sqrt(r2))) return -1;
                }
            }
    return 0;
}

/* Builds neighbour lists for the atoms with need[i] != 0 (all atoms if need == NULL).
 * mode 0: brute force, 1: cell list (falls back to brute force for < 3 cells), 2: automatic. */
static int nb_build(const or_system* s, double rc, int mode, const unsigned char* need, or_nblist* lists)
{
    double* w = (double*)malloc(sizeof(double) * 3 * (size_t)(s->n > 0 ? s->n : 1));
    if (!w) return -1;
    wrap_all(s, w);
    or_cells C;
    memset(&C, 0, sizeof C);
    int use_cells = 0;
    if (mode != 0) {
        int rcode = cells_build(s, w, rc, &C);
        if (rcode < 0) { free(w); return -1; }
        use_cells = (rcode == 0);
    }
    int err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
    for (int i = 0; i < s->n; ++i) {
        if (need && !need[i]) continue;
        lists[i].n = 0;
        int e = use_cells ? nb_cell_one(s, w, rc, &C, i, &lists[i]) : nb_brute_one(s, w, rc, i, &lists[i]);
        err |= (e != 0);
    }
    free(C.start);
    free(C.list);
    free(w);
    return err ? -1 : 0;
}

static void nb_free(or_nblist* lists, int n)
{
    for (int i = 0; i < n; ++i) free(lists[i].e);
    free(lists);
}

/* ------------------------------------------------------------ descriptors */
/* Angular element filter: -1/-1 accepts every pair, otherwise the unordered pair
 * of neighbour elements must equal {e1, e2}. */
static int ang_match(int e1, int e2, int tj, int tk)
{
    if (e1 < 0 || e2 < 0) return 1;
    return (tj == e1 && tk == e2) || (tj == e2 && tk == e1);
}

/* G for atom i (centre element ti).  If dG != NULL it receives dG_s/dd_a for every
 * descriptor s and neighbour entry a, laid out [s][a][3]. */
static void atom_descriptors(const or_model* m, int ti, const or_nblist* L, const int* type,
                             double* G, double* dG)
{
    const int o = m->sf_off[ti], ns = m->n_sf[ti], M = L->n;
    const double rc = m->rc;
    for (int s = 0; s < ns; ++s) G[s] = 0.0;
    if (dG) memset(dG, 0, sizeof(double) * (size_t)ns * (size_t)M * 3);

    for (int s = 0; s < ns; ++s) {
        const int t = m->sf_type[o + s];
        const double eta = m->sf_eta[o + s];
        if (t == OR_RADIAL) {
            const double rs = m->sf_rs[o + s];
            const int e1 = m->sf_e1[o + s];
            for (int a = 0; a < M; ++a) {
                const or_nb* A = &L->e[a];
                if (e1 >= 0 && type[A->j] != e1) continue;
                double x = exp(-eta * (A->r - rs) * (A->r - rs));
                double f = fcut(A->r, rc);
                G[s] += x * f;
                if (dG) {
                    double dTdr = x * (dfcut(A->r, rc) - 2.0 * eta * (A->r - rs) * f);
                    for (int c = 0; c < 3; ++c) dG[((size_t)s * M + a) * 3 + c] += dTdr * A->d[c] / A->r;
                }
            }
        } else {
            const double zeta = m->sf_zeta[o + s], lam = m->sf_lambda[o + s];
            const double pref = pow(2.0, 1.0 - zeta);
            const int narrow = (t == OR_NARROW);
            const int e1 = m->sf_e1[o + s], e2 = m->sf_e2[o + s];
            for (int a = 0; a < M; ++a)
                for (int b = a + 1; b < M; ++b) {
                    const or_nb* A = &L->e[a];
                    const or_nb* B = &L->e[b];
                    if (!ang_match(e1, e2, type[A->j], type[B->j])) continue;
                    double ra = A->r, rb = B->r;
                    double dab[3] = { B->d[0] - A->d[0], B->d[1] - A->d[1], B->d[2] - A->d[2] };
                    double rd = sqrt(dab[0] * dab[0] + dab[1] * dab[1] + dab[2] * dab[2]);
                    if (narrow && rd >= rc) continue;
                    double cost = (A->d[0] * B->d[0] + A->d[1] * B->d[1] + A->d[2] * B->d[2]) / (ra * rb);
                    double base = 1.0 + lam * cost;
                    double Ang = pref * pow(base, zeta);
                    double dAng = pref * zeta * lam * pow(base, zeta - 1.0);
                    double sumsq = ra * ra + rb * rb + (narrow ? rd * rd : 0.0);
                    double X = exp(-eta * sumsq);
                    double fa = fcut(ra, rc), fb = fcut(rb, rc), fd = narrow ? fcut(rd, rc) : 1.0;
                    double T = Ang * X * fa * fb * fd;
                    G[s] += T;
                    if (!dG) continue;
                    /* partials of T in the variables (ra, rb, rd, cos) */
                    double Tra = Ang * X * (-2.0 * eta * ra * fa + dfcut(ra, rc)) * fb * fd;
                    double Trb = Ang * X * fa * (-2.0 * eta * rb * fb + dfcut(rb, rc)) * fd;
                    double Trd = narrow ? Ang * X * fa * fb * (-2.0 * eta * rd * fd + dfcut(rd, rc)) : 0.0;
                    double Tc = dAng * X * fa * fb * fd;
                    for (int c = 0; c < 3; ++c) {
                        /* d(cos)/dd_a = d_b/(ra rb) - cos d_a/ra^2, d(rd)/dd_a = -(d_b - d_a)/rd */
                        double ga = Tra * A->d[c] / ra + Tc * (B->d[c] / (ra * rb) - cost * A->d[c] / (ra * ra));
                        double gb = Trb * B->d[c] / rb + Tc * (A->d[c] / (ra * rb) - cost * B->d[c] / (rb * rb));
                        if (narrow) {
                            ga -= Trd * dab[c] / rd;
                            gb += Trd * dab[c] / rd;
                        }
                        dG[((size_t)s * M + a) * 3 + c] += ga;
                        dG[((size_t)s * M + b) * 3 + c] += gb;
                    }
                }
        }
    }
}

/* ------------------------------------------------------------------- network */
static int max_width(const or_model* m)
{
    int w = 0;
    for (int l = 0; l <= m->n_layers; ++l) if (m->width[l] > w) w = m->width[l];
    for (int e = 0; e < m->n_elem; ++e) if (m->n_sf[e] > w) w = m->n_sf[e];
    return w;
}

/* Per-layer parameter offsets inside one element's block. */
static void layer_offsets(const or_model* m, int ninput, int* woff, int* boff)
{
    int off = 0, in = ninput;
    for (int l = 0; l < m->n_layers; ++l) {
        int out = m->width[l + 1];
        woff[l] = off;
        off += out * in;
        boff[l] = off;
        off += out;
        in = out;
    }
}

/* Forward pass; h receives every layer's activations, h[l*W + k] (h[0] = input). */
static double mlp_forward(const or_model* m, int e, const double* x, double* h, int W)
{
    int woff[OR_MAXL], boff[OR_MAXL];
    const int nin = m->n_sf[e];
    layer_offsets(m, nin, woff, boff);
    const double* P = m->w + m->w_off[e];
    for (int k = 0; k < nin; ++k) h[k] = x[k];
    int in = nin;
    for (int l = 0; l < m->n_layers; ++l) {
        int out = m->width[l + 1];
        for (int o = 0; o < out; ++o) {
            double a = P[boff[l] + o];
            for (int k = 0; k < in; ++k) a += P[woff[l] + o * in + k] * h[l * W + k];
            h[(l + 1) * W + o] = (l < m->n_layers - 1) ? tanh(a) : a;
        }
        in = out;
    }
    return h[m->n_layers * W + 0];
}

/* dE/dx by reverse accumulation given the forward activations h. */
static void mlp_input_grad(const or_model* m, int e, const double* h, int W, double* dx)
{
    int woff[OR_MAXL], boff[OR_MAXL];
    const int nin = m->n_sf[e];
    layer_offsets(m, nin, woff, boff);
    const double* P = m->w + m->w_off[e];
    double* d = (double*)malloc(sizeof(double) * 2 * (size_t)W);
    double* dn = d + W;
    d[0] = 1.0; /* dE/dh_L */
    for (int l = m->n_layers - 1; l >= 0; --l) {
        int out = m->width[l + 1], in = (l == 0) ? nin : m->width[l];
        if (l < m->n_layers - 1)
            for (int o = 0; o < out; ++o) d[o] *= 1.0 - h[(l + 1) * W + o] * h[(l + 1) * W + o];
        for (int k = 0; k < in; ++k) {
            double s = 0.0;
            for (int o = 0; o < out; ++o) s += P[woff[l] + o * in + k] * d[o];
            dn[k] = s;
        }
        memcpy(d, dn, sizeof(double) * (size_t)in);
    }
    for (int k = 0; k < nin; ++k) dx[k] = d[k];
    free(d);
}

/* Parameter gradient of  Q = hbar_out * E(x) + hdot_bar_out * Edot(x, xdot)
 * where Edot is the directional derivative of E along xdot (forward-mode tangent).
 * Reverse-over-forward through the tanh network; accumulates into grad (this
 * element's parameter block layout). */
static void mlp_param_grad(const or_model* m, int e, const double* x, const double* xdot,
                           double hbar_out, double hdbar_out, double* grad)
{
    const int W = max_width(m), L = m->n_layers, nin = m->n_sf[e];
    int woff[OR_MAXL], boff[OR_MAXL];
    layer_offsets(m, nin, woff, boff);
    const double* P = m->w + m->w_off[e];
    double* h = (double*)calloc((size_t)(L + 1) * W, sizeof(double));
    double* hd = (double*)calloc((size_t)(L + 1) * W, sizeof(double));
    double* ad = (double*)calloc((size_t)L * W, sizeof(double));   /* tangent pre-activations */
    double* hb = (double*)calloc((size_t)W, sizeof(double));
    double* hdb = (double*)calloc((size_t)W, sizeof(double));
    double* ab = (double*)calloc((size_t)W, sizeof(double));
    double* adb = (double*)calloc((size_t)W, sizeof(double));
    double* tmp = (double*)calloc((size_t)2 * W, sizeof(double));

    /* primal and tangent forward */
    for (int k = 0; k < nin; ++k) { h[k] = x[k]; hd[k] = xdot ? xdot[k] : 0.0; }
    int in = nin;
    for (int l = 0; l < L; ++l) {
        int out = m->width[l + 1];
        for (int o = 0; o < out; ++o) {
            double a = P[boff[l] + o], at = 0.0;
            for (int k = 0; k < in; ++k) {
                a += P[woff[l] + o * in + k] * h[l * W + k];
                at += P[woff[l] + o * in + k] * hd[l * W + k];
            }
            ad[l * W + o] = at;
            if (l < L - 1) {
                double t = tanh(a);
                h[(l + 1) * W + o] = t;
                hd[(l + 1) * W + o] = (1.0 - t * t) * at;
            } else {
                h[(l + 1) * W + o] = a;
                hd[(l + 1) * W + o] = at;
            }
        }
        in = out;
    }
    /* reverse */
    hb[0] = hbar_out;
    hdb[0] = hdbar_out;
    for (int l = L - 1; l >= 0; --l) {
        int out = m->width[l + 1];
        int lin = (l == 0) ? nin : m->width[l];
        for (int o = 0; o < out; ++o) {
            if (l < L - 1) {
                double t = h[(l + 1) * W + o];
                double s = 1.0 - t * t;
                adb[o] = hdb[o] * s;
                double hbo = hb[o] + hdb[o] * ad[l * W + o] * (-2.0 * t);
                ab[o] = hbo * s;
            } else {
                adb[o] = hdb[o];
                ab[o] = hb[o];
            }
        }
        for (int o = 0; o < out; ++o) {
            for (int k = 0; k < lin; ++k)
                grad[woff[l] + o * lin + k] += ab[o] * h[l * W + k] + adb[o] * hd[l * W + k];
            grad[boff[l] + o] += ab[o];
        }
        for (int k = 0; k < lin; ++k) {
            double s1 = 0.0, s2 = 0.0;
            for (int o = 0; o < out; ++o) {
                s1 += P[woff[l] + o * lin + k] * ab[o];
                s2 += P[woff[l] + o * lin + k] * adb[o];
            }
            tmp[k] = s1;
            tmp[W + k] = s2;
        }
        for (int k = 0; k < lin; ++k) { hb[k] = tmp[k]; hdb[k] = tmp[W + k]; }
    }
    free(h); free(hd); free(ad); free(hb); free(hdb); free(ab); free(adb); free(tmp);
}

/* ----------------------------------------------------------- public API */
typedef struct {
    double* G;        /* [n][ldg] raw descriptors (nullable)               */
    double* dEdG;     /* [n][ldg] dE_i/dG_i (nullable)                     */
    double* Ei;       /* [n] (nullable)                                    */
    double* F;        /* [n][3] (nullable)                                 */
    double* virial;   /* [9] (nullable)                                    */
    double* energy;   /* [1] (nullable)                                    */
    int ldg;
} or_out;

int or_n_params_elem(const or_model* m)
{
    int n = 0, in = m->width[0];
    for (int l = 0; l < m->n_layers; ++l) { n += m->width[l + 1] * (in + 1); in = m->width[l + 1]; }
    return n;
}

/* Neighbour lists as plain arrays (for tests): counts[n], and up to cap entries per
 * atom of (j, dx, dy, dz).  Returns the largest count seen (entries beyond cap are
 * dropped), or -1 on failure. */
int or_neighbors(const or_system* s, double rc, int mode, int cap, int* counts, int* js, double* d)
{
    or_nblist* lists = (or_nblist*)calloc((size_t)(s->n > 0 ? s->n : 1), sizeof(or_nblist));
    if (!lists) return -1;
    if (nb_build(s, rc, mode, NULL, lists)) { nb_free(lists, s->n); return -1; }
    int mx = 0;
    for (int i = 0; i < s->n; ++i) {
        counts[i] = lists[i].n;
        if (lists[i].n > mx) mx = lists[i].n;
        for (int a = 0; a < lists[i].n && a < cap; ++a) {
            js[(size_t)i * cap + a] = lists[i].e[a].j;
            for (int c = 0; c < 3; ++c) d[((size_t)i * cap + a) * 3 + c] = lists[i].e[a].d[c];
        }
    }
    nb_free(lists, s->n);
    return mx;
}

/* Network only, for one element: E(x) and dE/dx given a scaled input x. */
double or_mlp(const or_model* m, int e, const double* x, double* dEdx)
{
    int W = max_width(m);
    double* h = (double*)calloc((size_t)(m->n_layers + 1) * W, sizeof(double));
    double E = mlp_forward(m, e, x, h, W);
    if (dEdx) mlp_input_grad(m, e, h, W, dEdx);
    free(h);
    return E;
}

/* Core evaluation.  'target' (nullable) restricts the outputs: per-atom outputs
 * are produced for target atoms only, forces only for target atoms (summing the
 * contributions of every atom whose energy depends on them).  With target == NULL
 * everything is produced for every atom.  n_sum: the energy and the virial sum
 * the energies E_i of atoms i < n_sum only (n for the whole system): the energy
 * sum_{i < n_sum} E_i and its strain derivative -sum_{i < n_sum} sum_j d_ij g_ij. */
static int compute_core(const or_model* m, const or_system* s, int nbmode, const unsigned char* target, int n_sum,
                        or_out* out)
{
    const int n = s->n;
    const int W = max_width(m);
    or_nblist* lists = (or_nblist*)calloc((size_t)(n > 0 ? n : 1), sizeof(or_nblist));
    if (!lists) return -1;
    /* atoms whose energy gradient we need: targets and their neighbours */
    unsigned char* need = NULL;
    if (target) {
        need = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
        if (nb_build(s, m->rc, nbmode, target, lists)) { nb_free(lists, n); free(need); return -1; }
        for (int i = 0; i < n; ++i)
            if (target[i]) {
                need[i] = 1;
                for (int a = 0; a < lists[i].n; ++a) need[lists[i].e[a].j] = 1;
            }
        for (int i = 0; i < n; ++i) if (target[i]) need[i] = 2; /* already built */
        unsigned char* rest = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
        for (int i = 0; i < n; ++i) rest[i] = (need[i] == 1);
        if (nb_build(s, m->rc, nbmode, rest, lists)) { nb_free(lists, n); free(need); free(rest); return -1; }
        free(rest);
    } else {
        if (nb_build(s, m->rc, nbmode, NULL, lists)) { nb_free(lists, n); return -1; }
    }

    /* per-atom pair gradients g_a = dE_i/dd_a (only for atoms in 'need') */
    double** g = (double**)calloc((size_t)(n > 0 ? n : 1), sizeof(double*));
    double* Ei = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (int i = 0; i < n; ++i) {
        if (need && !need[i]) continue;
        const int ti = s->type[i], ns = m->n_sf[ti], M = lists[i].n, o = m->sf_off[ti];
        double* G = (double*)malloc(sizeof(double) * (size_t)ns);
        double* dG = (double*)malloc(sizeof(double) * ((size_t)ns * M * 3 + 1));
        double* x = (double*)malloc(sizeof(double) * (size_t)ns);
        double* dx = (double*)malloc(sizeof(double) * (size_t)ns);
        double* h = (double*)calloc((size_t)(m->n_layers + 1) * W, sizeof(double));
        g[i] = (double*)calloc((size_t)M * 3 + 1, sizeof(double));
        if (!G || !dG || !x || !dx || !h || !g[i]) { err |= 1; continue; }
        atom_descriptors(m, ti, &lists[i], s->type, G, dG);
        for (int k = 0; k < ns; ++k) x[k] = (G[k] - m->sf_mu[o + k]) / m->sf_s[o + k];
        Ei[i] = mlp_forward(m, ti, x, h, W);
        mlp_input_grad(m, ti, h, W, dx);
        for (int k = 0; k < ns; ++k) dx[k] /= m->sf_s[o + k]; /* dE/dG */
        for (int a = 0; a < M; ++a)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < ns; ++k) acc += dx[k] * dG[((size_t)k * M + a) * 3 + c];
                g[i][a * 3 + c] = acc;
            }
        if (!target || target[i]) {
            if (out->G) for (int k = 0; k < ns; ++k) out->G[(size_t)i * out->ldg + k] = G[k];
            if (out->dEdG) for (int k = 0; k < ns; ++k) out->dEdG[(size_t)i * out->ldg + k] = dx[k];
        }
        free(G); free(dG); free(x); free(dx); free(h);
    }
    if (!err) {
        if (out->Ei) for (int i = 0; i < n; ++i) if (!target || target[i]) out->Ei[i] = Ei[i];
        if (out->energy && !target) {
            double E = 0.0;
            for (int i = 0; i < n_sum; ++i) E += Ei[i];
            out->energy[0] = E;
        }
        if (out->F) {
            for (int i = 0; i < n; ++i)
                if (!target || target[i]) out->F[3 * i] = out->F[3 * i + 1] = out->F[3 * i + 2] = 0.0;
            for (int i = 0; i < n; ++i) {
                if (need && !need[i]) continue;
                for (int a = 0; a < lists[i].n; ++a) {
                    int j = lists[i].e[a].j;
                    for (int c = 0; c < 3; ++c) {
                        if (!target || target[i]) out->F[3 * i + c] += g[i][a * 3 + c];
                        if (!target || target[j]) out->F[3 * j + c] -= g[i][a * 3 + c];
                    }
                }
            }
        }
        if (out->virial && !target) {
            for (int k = 0; k < 9; ++k) out->virial[k] = 0.0;
            for (int i = 0; i < n_sum; ++i)
                for (int a = 0; a < lists[i].n; ++a)
                    for (int p = 0; p < 3; ++p)
                        for (int q = 0; q < 3; ++q)
                            out->virial[3 * p + q] -= lists[i].e[a].d[p] * g[i][a * 3 + q];
        }
    }
    for (int i = 0; i < n; ++i) free(g[i]);
    free(g);
    free(Ei);
    free(need);
    nb_free(lists, n);
    return err ? -1 : 0;
}

int or_compute(const or_model* m, const or_system* s, int nbmode, or_out* out)
{
    return compute_core(m, s, nbmode, NULL, s->n, out);
}

/* As or_compute, with the energy and the virial summed over the energies of the
 * first n_own atoms only (a spatial domain whose owned atoms come first, its
 * halo copies after them); Ei and F for every atom. */
int or_compute_owned(const or_model* m, const or_system* s, int nbmode, int n_own, or_out* out)
{
    if (n_own < 0 || n_own > s->n) return -1;
    return compute_core(m, s, nbmode, NULL, n_own, out);
}

/* Outputs (Ei, F, G, dEdG) for the atoms with target[i] != 0 only. */
int or_compute_subset(const or_model* m, const or_system* s, int nbmode, const unsigned char* target, or_out* out)
{
    return compute_core(m, s, nbmode, target, s->n, out);
}

/* Velocity-Verlet NVE: v += dt/2 F/m c; x += dt v; F = F(x); v += dt/2 F/m c.
 * Units: A, fs, amu, eV; c = 1 eV/(A amu) in A/fs^2.  log[k] = (PE, KE) after k
 * steps, k = 0..nsteps.  pos and vel are updated in place. */
int or_md(const or_model* m, or_system* s, double* pos, double* vel, const double* mass_of_elem,
          double dt, int nsteps, int nbmode, double* log)
{
    const double C = 9.64853321233100e-3;
    const int n = s->n;
    double* F = (double*)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
    double E = 0.0;
    or_out o;
    memset(&o, 0, sizeof o);
    o.F = F;
    o.energy = &E;
    s->pos = pos;
    if (or_compute(m, s, nbmode, &o)) { free(F); return -1; }
    for (int k = 0; k <= nsteps; ++k) {
        if (k > 0) {
            for (int i = 0; i < n; ++i) {
                double im = C / mass_of_elem[s->type[i]];
                for (int c = 0; c < 3; ++c) vel[3 * i + c] += 0.5 * dt * F[3 * i + c] * im;
                for (int c = 0; c < 3; ++c) pos[3 * i + c] += dt * vel[3 * i + c];
            }
            if (or_compute(m, s, nbmode, &o)) { free(F); return -1; }
            for (int i = 0; i < n; ++i) {
                double im = C / mass_of_elem[s->type[i]];
                for (int c = 0; c < 3; ++c) vel[3 * i + c] += 0.5 * dt * F[3 * i + c] * im;
            }
        }
        double KE = 0.0;
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) KE += 0.5 * mass_of_elem[s->type[i]] * vel[3 * i + c] * vel[3 * i + c] / C;
        if (log) { log[2 * k] = E; log[2 * k + 1] = KE; }
    }
    free(F);
    return 0;
}

/* Force-matching parameter gradient for one system.
 *   grad += dLdE * dE/dtheta - d/dtheta [ sum_i grad_G E_i . t_i ],
 *   t_i = sum_a dG_i/dd_a . (u_{j(a)} - u_i),
 * where u = dL/dF [n][3].  Since F = -dE/dr, sum_m u_m . dF_m/dtheta equals the
 * second term, so grad is dL/dtheta when dLdE = dL/dE and u = dL/dF.  grad uses
 * the packed parameter layout (all elements). */
int or_param_grad(const or_model* m, const or_system* s, int nbmode, double dLdE, const double* u, double* grad)
{
    const int n = s->n;
    or_nblist* lists = (or_nblist*)calloc((size_t)(n > 0 ? n : 1), sizeof(or_nblist));
    if (!lists) return -1;
    if (nb_build(s, m->rc, nbmode, NULL, lists)) { nb_free(lists, n); return -1; }
    const int npe = or_n_params_elem(m);
    int err = 0;
    /* per-atom gradient blocks, summed serially in atom order afterwards */
    double* per = (double*)calloc((size_t)(n > 0 ? n : 1) * npe, sizeof(double));
    if (!per) { nb_free(lists, n); return -1; }
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (int i = 0; i < n; ++i) {
        const int ti = s->type[i], ns = m->n_sf[ti], M = lists[i].n, o = m->sf_off[ti];
        double* G = (double*)malloc(sizeof(double) * (size_t)ns);
        double* dG = (double*)malloc(sizeof(double) * ((size_t)ns * M * 3 + 1));
        double* x = (double*)malloc(sizeof(double) * (size_t)ns);
        double* xd = (double*)calloc((size_t)ns, sizeof(double));
        if (!G || !dG || !x || !xd) { err |= 1; continue; }
        atom_descriptors(m, ti, &lists[i], s->type, G, dG);
        for (int k = 0; k < ns; ++k) x[k] = (G[k] - m->sf_mu[o + k]) / m->sf_s[o + k];
        if (u) {
            for (int k = 0; k < ns; ++k) {
                double t = 0.0;
                for (int a = 0; a < M; ++a) {
                    int j = lists[i].e[a].j;
                    for (int c = 0; c < 3; ++c) t += dG[((size_t)k * M + a) * 3 + c] * (u[3 * j + c] - u[3 * i + c]);
                }
                xd[k] = t / m->sf_s[o + k];
            }
        }
        mlp_param_grad(m, ti, x, xd, dLdE, u ? -1.0 : 0.0, per + (size_t)i * npe);
        free(G); free(dG); free(x); free(xd);
    }
    if (!err)
        for (int i = 0; i < n; ++i) {
            double* dst = grad + m->w_off[s->type[i]];
            for (int k = 0; k < npe; ++k) dst[k] += per[(size_t)i * npe + k];
        }
    free(per);
    nb_free(lists, n);
    return err ? -1 : 0;
}

int or_set_threads(int nt)
{
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
    return omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}
