/*
 * nnp.h -- C ABI of the B300 (sm_103a) Behler-Parrinello neural-network
 * potential hot path (arXiv 2002.00054, "Implementing a neural network
 * interatomic model with performance portability ...").
 *
 * Conventions for every call below
 *   - Units: Angstrom, eV, amu, fs.  Boxes are orthorhombic and periodic with
 *     the origin at 0; positions need not lie inside the box.
 *   - "device" pointers are CUDA device memory on the handle's device, owned by
 *     the caller, contiguous, naturally aligned (float arrays 4-byte, double
 *     8-byte).  "host" pointers are ordinary host memory read during the call.
 *   - The library owns only its scratch (cell lists, neighbour lists, per-pair
 *     force buffer, descriptor buffers) and its copy of the model parameters.
 *   - 'stream' is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work of a call is enqueued on it.  Calls that return a status
 *     from the device (nnp_compute, nnp_descriptors, nnp_step, the gradient
 *     calls) synchronise that stream once at their end to read the library's
 *     error word; no other synchronisation is done.
 *   - Every call returns an nnp_status (0 = NNP_OK).  After an error,
 *     nnp_last_error(h) describes it.  No call traps, asserts on the device or
 *     spins: overflowing capacities and non-finite values are reported through
 *     the status.
 *   - A handle is not thread-safe: serialise calls on one handle.
 */
#ifndef NNP_B300_H
#define NNP_B300_H

#if defined(__GNUC__)
#define NNP_API __attribute__((visibility("default")))
#else
#define NNP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum nnp_status {
    NNP_OK = 0,
    NNP_EINVAL = 1,           /* bad argument or parameter set                      */
    NNP_ENOMEM = 2,           /* device or host allocation failed                   */
    NNP_ENEIGH_OVERFLOW = 3,  /* an atom has more neighbours than max_neighbors,     */
                              /* or a cell holds more atoms than the cell capacity   */
    NNP_ENONFINITE = 4,       /* non-finite input/output, or two atoms closer than   */
                              /* 1e-4 A                                               */
    NNP_EBOX = 5,             /* box edge below (cutoff + skin) / 2, or box not > 0  */
    NNP_ECUDA = 6,            /* a CUDA runtime call failed                          */
    NNP_EUNSUPPORTED = 7      /* valid model outside what the kernels implement     */
};

/* --------------------------------------------------------- model definition */
/* Descriptor kinds.  Radial: Fig. 1b step 1 of the paper,
 *   G2_i = sum_j exp(-eta (r_ij - r_s)^2) f_c(r_ij),  f_c(r) = (cos(pi r / r_c) + 1) / 2.
 * Angular ("one extra loop over neighbours of neighbours", Sec. 3.1; the paper
 * does not print the formula, these are Behler's standard forms):
 *   narrow: 2^(1-zeta) sum_{j<k} (1 + lambda cos t_ijk)^zeta
 *                exp(-eta (r_ij^2 + r_ik^2 + r_jk^2)) f_c(r_ij) f_c(r_ik) f_c(r_jk)
 *   wide:   the same without r_jk^2 in the exponent and without f_c(r_jk). */
enum nnp_sf_type { NNP_SF_RADIAL = 2, NNP_SF_ANG_NARROW = 3, NNP_SF_ANG_WIDE = 4 };

/* Network precision: FP32 everywhere, or BF16 operands with FP32 accumulation
 * for the network layers on the tensor cores (descriptors and forces stay FP32;
 * NNP_BF16 needs two hidden layers, n_layers = 3). */
enum nnp_precision { NNP_FP32 = 0, NNP_BF16 = 1 };

typedef struct {
    int type;      /* nnp_sf_type                                                  */
    int elem_a;    /* radial: neighbour element, -1 = any.                          */
                   /* angular: with elem_b the unordered pair of neighbour elements */
                   /* {elem_a, elem_b} of the pairs (j, k) the function sums over;  */
                   /* either -1 = every pair; at most 10 distinct pairs per element */
    int elem_b;
    double eta;    /* A^-2, >= 0                                                    */
    double rs;     /* A, radial only (angular: must be 0)                           */
    double zeta;   /* angular: 1, 2, 4, 8 or 16                                     */
    double lambda; /* angular: +1 or -1                                             */
} nnp_sf_desc;

typedef struct {
    int n_elements;              /* 1..8                                              */
    const double* masses_amu;    /* host [n_elements]                                 */
    double cutoff;               /* r_c, A                                            */
    double skin;                 /* neighbour-list skin, A (>= 0); lists are rebuilt  */
                                 /* when an atom moved more than skin/2               */
    const int* n_sf;             /* host [n_elements]; all equal to widths[0]         */
    const nnp_sf_desc* sf;       /* host, element 0's n_sf[0] descriptors, then       */
                                 /* element 1's, ...; at most 64 per element, at most */
                                 /* 4 distinct angular eta per element, one angular  */
                                 /* kind per element                                  */
    const double* sf_shift;      /* host, packed like sf: mu of G~ = (G - mu) / s     */
    const double* sf_scale;      /* host, packed like sf: s (> 0)                     */
    int n_layers;                /* weight layers, 2..6 (e.g. 3 for n_G-25-25-1)       */
    const int* widths;           /* host [n_layers + 1]; widths[0] = n_G (<= 64),      */
                                 /* hidden widths <= 32, widths[n_layers] = 1          */
    const double* weights;       /* host, per element: for each layer l the matrix    */
                                 /* W_l [widths[l+1]][widths[l]] row-major then the   */
                                 /* bias b_l [widths[l+1]]; elements back to back     */
    int mlp_precision;           /* nnp_precision                                     */
    int max_neighbors;           /* capacity of one atom's neighbour-list row (entries */
                                 /* within cutoff + skin), 32..1024; a row above it    */
                                 /* fails the call (NNP_ENEIGH_OVERFLOW).  It sizes    */
                                 /* memory only: how many neighbours inside the cutoff */
                                 /* the kernels stage in shared memory follows the     */
                                 /* counts seen (nnp_stats.rc_capacity), and atoms     */
                                 /* above that take a second, wide-capacity pass       */
} nnp_params;

typedef struct nnp_handle nnp_handle;

/* Creates a handle on CUDA device 'device': validates and copies the parameters
 * (host memory may be freed afterwards).  *out is NULL on failure.  Parameter
 * validation happens before any CUDA call.  Scratch grows on demand later.
 * Force assembly: by default each atom adds its pair contributions -g_ij into
 * the forces of its neighbours as 64-bit fixed-point integers (units 2^-27
 * eV/A) with global integer atomics; integer sums do not depend on the order of
 * the atomics, so forces are reproducible bit for bit, and each component is
 * rounded to float once.  Environment variables read here select the other
 * forms: NNP_FORCE_GATHER=1 writes g_ij per neighbour-list slot and gathers the
 * forces per atom through a reverse index (fixed order, float sums; the reverse
 * index and slot buffer take 20 bytes per list slot), NNP_FORCE_SCATTER=1 adds
 * floats with global atomics (the scatter form of the paper's CabanaMD code;
 * sums in the order the atomics land).  With the default form and at most two
 * eta the descriptor pass also writes each atom's staged neighbours (48 bytes
 * per neighbour inside r_c) for the force pass to read; NNP_STAGE_REUSE=0 makes
 * the force pass stage them again instead (the same forces, bit for bit).
 * NNP_STEP_GRAPH=0 is described at nnp_step. */
NNP_API int nnp_create(const nnp_params* params, int device, nnp_handle** out);

/* Frees the handle and its device memory (waits for its pending work).  NULL is a no-op. */
NNP_API int nnp_destroy(nnp_handle* h);

/* Message of the last failed call on h (never NULL; "" if none).  Valid until the
 * next call on h.  nnp_last_error(NULL) gives the message of the last failed
 * nnp_create on this thread. */
NNP_API const char* nnp_last_error(const nnp_handle* h);

/* Static name of a status code. */
NNP_API const char* nnp_status_string(int status);

/* Number of network parameters over all elements (packed layout of nnp_params.weights). */
NNP_API int nnp_num_params(const nnp_handle* h);

/* Replaces the network parameters from a device buffer of nnp_num_params(h) floats in
 * the packed layout (used by training).  Ordered on 'stream'; no synchronisation. */
NNP_API int nnp_set_weights(nnp_handle* h, const float* weights_dev, void* stream);

/* Energy and forces of one periodic system: Fig. 1b of the paper, steps 1-3.
 *   n_atoms      >= 0 (0: energy = 0, virial = 0, nothing else written)
 *   pos          device float [n_atoms][3]
 *   types        device int [n_atoms], 0 <= type < n_elements
 *   box          host double [3], edges > 0 and >= (cutoff + skin) / 2
 *   cutoff       <= 0 or equal to the model cutoff (anything else: NNP_EINVAL)
 *   energy       device double [1]: E = sum_i E_i, summed in FP64 (nullable)
 *   atom_energy  device float [n_atoms]: E_i (nullable)
 *   forces       device float [n_atoms][3]: F = -dE/dr (nullable)
 *   virial       device double [9] row-major: W_ab = -sum_{i, j in nb(i)} d_ij^a dE_i/dd_ij^b,
 *                d_ij = r_j - r_i for each neighbour image (nullable)
 * The neighbour list is kept in the handle and rebuilt when n_atoms or the box
 * changed or an atom moved more than skin/2 since the last build. */
NNP_API int nnp_compute(nnp_handle* h, int n_atoms, const float* pos, const int* types, const double* box,
                double cutoff, double* energy, float* atom_energy, float* forces, double* virial,
                void* stream);

/* One spatial domain of a decomposed periodic box (the paper's outlook on
 * multi-node runs, Sec. 5): as nnp_compute on the domain's local atoms, the
 * n_owned atoms the domain owns first, then copies of every atom within 2 r_c
 * of the domain (its halo), at positions in a local box.  With a 2 r_c halo an
 * owned atom's energy and force come out exact, so no forces are sent back.
 *   n_owned      0 <= n_owned <= n_atoms
 *   energy       device double [1]: sum_{i < n_owned} E_i in FP64 (nullable)
 *   virial       device double [9]: the pair virial of the owned atoms'
 *                energies, -sum_{i < n_owned} sum_j d_ij^a dE_i/dd_ij^b
 *                (nullable); summed over domains it is the box's virial
 *   atom_energy, forces: for every local atom (the caller keeps the first
 *                n_owned; halo atoms' values are not those of the box)
 * Everything else as nnp_compute. */
NNP_API int nnp_compute_domain(nnp_handle* h, int n_atoms, int n_owned, const float* pos, const int* types,
                               const double* box, double* energy, float* atom_energy, float* forces, double* virial,
                               void* stream);

/* Raw descriptors G (Fig. 1b step 1) and dE_i/dG_i (the network's input gradient
 * used by step 3) of one system; arguments as nnp_compute.
 *   G, dEdG      device float [n_atoms][n_G] (each nullable). */
NNP_API int nnp_descriptors(nnp_handle* h, int n_atoms, const float* pos, const int* types, const double* box,
                    float* G, float* dEdG, void* stream);

/* Raw descriptors G of one system computed with one thread per atom (each
 * thread walks its own neighbours and neighbour pairs: the flat level of the
 * paper's parallelism study, Sec. 4.3 / Fig. 6), for comparison with the
 * warp-per-atom kernels of every other call; FP32 sums, much slower.  The
 * neighbour list is built (or reused) as by nnp_descriptors.  Models with
 * element-pair-resolved angular descriptors: NNP_EUNSUPPORTED.
 *   G  device float [n_atoms][n_G]. */
NNP_API int nnp_descriptors_flat(nnp_handle* h, int n_atoms, const float* pos, const int* types, const double* box,
                                 float* G, void* stream);

/* Raw descriptors G with one thread per (atom, neighbour-list slot): the
 * hierarchical level of the paper's parallelism study (Sec. 4.3 / Fig. 6;
 * threads over atoms and neighbours).  The thread for neighbour j of atom i adds
 * the radial terms of j and the angular terms of the pairs (j, k), k after j in
 * i's list, and adds those partial descriptors into G_i with float atomics (the
 * extra atomic update of the symmetry functions the paper names for this level),
 * so the last bits of G depend on scheduling.  For the ablation; otherwise as
 * nnp_descriptors_flat.
 *   G  device float [n_atoms][n_G], overwritten. */
NNP_API int nnp_descriptors_pair(nnp_handle* h, int n_atoms, const float* pos, const int* types, const double* box,
                                 float* G, void* stream);

/* Raw descriptors G with one CTA per cell of the cell binning (the CTA-per-cell
 * mapping of the parallelism ablation): the CTA copies the atoms of the cell's
 * 27-cell stencil into shared memory once, and each of its warps finds the
 * neighbours of one of the cell's atoms in that copy (no Verlet list) and walks
 * all of its neighbour pairs with its lanes.  Needs at least 3 cells of
 * cutoff + skin per box edge (NNP_EUNSUPPORTED otherwise) and at most 2,048
 * atoms in a stencil (NNP_ENEIGH_OVERFLOW otherwise).  For the ablation;
 * otherwise as nnp_descriptors_flat.
 *   G  device float [n_atoms][n_G]. */
NNP_API int nnp_descriptors_cell(nnp_handle* h, int n_atoms, const float* pos, const int* types, const double* box,
                                 float* G, void* stream);

/* n_steps velocity-Verlet NVE steps (Sec. 4.2 energy conservation):
 *   v += dt/2 F/m;  x += dt v;  F = F(x);  v += dt/2 F/m
 * pos, vel: device float [n_atoms][3], updated in place (positions are not wrapped).
 * vel in A/fs; dt_fs > 0; n_steps >= 0.  pe_ke_log: device double [n_steps + 1][2]
 * of (potential, kinetic) energy in eV before the first and after every step
 * (nullable).  Forces at the start are computed by the call, unless the previous
 * call on h was nnp_step on the same pos/types buffers, n_atoms and box and the
 * positions and types are bitwise unchanged since it returned (checked on the
 * device); then that call's final forces and energy are reused.
 * Every decision that differs between steps (neighbour-list rebuild, atoms of
 * the wide-capacity pass, log entry) is taken on the device, so with
 * n_steps >= 3 the call launches the first step directly, captures the second
 * as a CUDA graph on a stream of its own and replays it for the remaining
 * steps (bitwise the same results; ordered after earlier and before later work
 * on `stream` by events).  Setting NNP_STEP_GRAPH=0 when the handle is created,
 * or kernel-group timing, launches every step directly.  An error raised at any
 * step is reported by the call. */
NNP_API int nnp_step(nnp_handle* h, int n_atoms, float* pos, float* vel, const int* types, const double* box,
             double dt_fs, int n_steps, double* pe_ke_log, void* stream);

/* ----------------------------------------------------- batches and training */
/* A batch of n_systems independent periodic systems (e.g. a training batch of
 * configurations of different sizes): system b holds atoms sys_start[b] ..
 * sys_start[b+1]-1 (host int [n_systems + 1], sys_start[0] = 0) in the box
 * boxes[3b .. 3b+2] (host double).  Every box edge must be >= (cutoff + skin)/2;
 * neighbours include every periodic image within the cutoff.  With n_systems > 1
 * each system is searched by brute force over images (cost ~ N_b^2; at most
 * 16384 atoms per system, NNP_EINVAL beyond); a single system takes the
 * cell-list path of nnp_compute.
 *
 * nnp_compute_batch: energies (device double [n_systems], FP64 sums), per-atom
 * energies and forces (device, nullable) of every system; Fig. 1b steps 1-3. */
NNP_API int nnp_compute_batch(nnp_handle* h, int n_systems, const int* sys_start, const double* boxes,
                              const float* pos, const int* types, double* energies, float* atom_energy,
                              float* forces, void* stream);

/* Gradient of a loss with respect to the network parameters (force-matching
 * training; the paper fits these parameters by least squares, Sec. 2):
 *   grad = sum_b dLdE[b] dE_b/dtheta + sum_m dLdF[m] . dF_m/dtheta
 * dLdE: device double [n_systems] (nullable); dLdF: device float [n_atoms][3]
 * (nullable); grad: device float [nnp_num_params(h)] in the packed weight layout,
 * overwritten.  The force term is the double backward: because F = -dE/dr it
 * equals -d/dtheta sum_i dE_i/dG_i . t_i with t_i = sum_j dG_i/dd_ij . (u_j - u_i),
 * u = dLdF; dG/dr is recomputed, not stored.  Needs two hidden layers. */
NNP_API int nnp_param_grad(nnp_handle* h, int n_systems, const int* sys_start, const double* boxes,
                           const float* pos, const int* types, const double* dLdE, const float* dLdF,
                           float* grad, void* stream);

/* Work counters summed over the last nnp_compute / nnp_descriptors / nnp_step
 * call (rebuilds: since creation).  Synchronises the handle's device. */
typedef struct {
    long long n_atoms;
    long long list_entries;    /* neighbour-list entries within cutoff + skin      */
    long long cutoff_entries;  /* entries within the cutoff                        */
    long long pairs;           /* neighbour pairs j < k examined by the angular loop */
    long long triplets;        /* pairs that contribute (narrow: r_jk < r_c)       */
    long long rebuilds;        /* neighbour-list builds since creation             */
    long long kernel_launches; /* CUDA kernels launched by the last call           */
    long long max_list_row;    /* largest neighbour-list row (entries within r_c +
                                  skin) in any evaluation of the last call; a
                                  row above max_neighbors fails the call          */
    long long max_cutoff_row;  /* largest count of neighbours inside r_c          */
    long long spilled_atoms;   /* atom evaluations of the last call that took the
                                  wide-capacity pass (more neighbours inside r_c
                                  than the main launch stages in shared memory)   */
    long long rc_capacity;     /* neighbours inside r_c the main launches stage
                                  per atom; re-tuned after every call from the
                                  counts seen (results do not depend on it)      */
    double min_distance;       /* closest pair distance within r_c (A) in any
                                  evaluation of the last call that computed
                                  descriptors; -1 if none                       */
} nnp_stats;
NNP_API int nnp_get_stats(nnp_handle* h, nnp_stats* out);

/* ------------------------------------------------------- kernel timing */
/* Per-kernel device time, measured with CUDA events recorded on the call's
 * stream around every kernel group of a call (no extra synchronisation; the
 * events are read at the call's final synchronisation).
 *   nnp_profile(h, 1) clears the totals and starts recording; nnp_profile(h, 0) stops.
 *   nnp_kernel_times fills total_ms[k] and launches[k] for kernel groups
 *   k < min(max_groups, nnp_num_kernel_groups()); returns the count written. */
NNP_API int nnp_profile(nnp_handle* h, int enable);
NNP_API int nnp_num_kernel_groups(void);
NNP_API const char* nnp_kernel_group_name(int k);
NNP_API int nnp_kernel_times(nnp_handle* h, int max_groups, double* total_ms, long long* launches);

/* ------------------------------------------------ allocation-free evaluation */
/* The paper has no counterpart to this entry point.
 *
 * nnp_compute_static computes what nnp_compute computes (energy, per-atom
 * energies, forces) for one small system without allocating any memory, on
 * the device or the host.  It is meant for callers that cannot allocate at the
 * time they need forces: a host MD code or framework that reserves all device
 * memory at start-up and forbids allocation inside its time loop, or a
 * latency-bound loop that cannot afford the device-wide synchronisation that
 * cudaMalloc / cudaFree may imply.  Such a caller creates the handle once at
 * start-up (nnp_create allocates the model parameters) and then calls this
 * entry point every step.
 *
 * Scratch: one file-scope device array of NNP_STATIC_SCRATCH_BYTES (8 MiB) per
 * GPU that loads this library, held until the process exits.  The handle's own
 * scratch is neither used nor changed.  Limits: n_atoms <= NNP_STATIC_MAX_ATOMS
 * and the scratch the call needs (about n_atoms * max_neighbors * 24 bytes)
 * must fit the array; otherwise NNP_EINVAL with a message naming the limit.
 * Neighbours are found by brute force over periodic images on every call.
 * The handle's network must be NNP_FP32 (NNP_EUNSUPPORTED otherwise).
 *
 * The first call on a device looks up the array's device address (a runtime
 * call, made once per device with that device current).  The address is kept
 * for the life of the process: after cudaDeviceReset on a device, do not call
 * this entry point on that device again in the same process.  Every call
 * shares the one array and leaves its contents behind: calls whose work
 * overlaps on the GPU (different streams or host threads without ordering)
 * race on it; serialise them.
 *
 * Arguments as nnp_compute (energy, atom_energy, forces device pointers, each
 * nullable; box host double [3]); errbuf (nullable) receives a message of at
 * most errbuf_len bytes on failure, since nnp_last_error is not updated.
 * Synchronises 'stream' at the end to read the status. */
#define NNP_STATIC_MAX_ATOMS 1024
#define NNP_STATIC_SCRATCH_BYTES (8u << 20)
NNP_API int nnp_compute_static(const nnp_handle* h, int n_atoms, const float* pos, const int* types,
                               const double* box, double* energy, float* atom_energy, float* forces,
                               char* errbuf, int errbuf_len, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NNP_B300_H */
