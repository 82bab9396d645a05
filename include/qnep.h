/*
 * qnep.h -- C ABI of the GB300 qNEP force call.
 *
 * qNEP (arXiv 2601.19034) is a neuroevolution potential whose single-hidden-
 * layer network has two outputs per atom: a site energy U_i (Eq. U_i, Sec. II.A)
 * and a partial charge q_i (Sec. II.B).  One force call computes, for one
 * periodic structure (or a batch of structures under several parameter
 * vectors):
 *   - the NEP descriptor of every atom over its neighbour list (Sec. II.A),
 *   - U_i and q_i from the network (Eq. U_i and the charge node, Sec. II.B),
 *   - the charge scaling q~ = sqrt(eps_inf) q (Sec. II.D) and the total-charge
 *     correction (Eq. charge-scaling),
 *   - the electrostatic energy of the charges by Ewald summation (Eqs. U_ES,
 *     U_k, S_k, Sec. II.B) or PPPM (Sec. II.F), mode 1 (real + k + self) or
 *     mode 2 (k only, Eq. mode2),
 *   - forces and virial including the dynamic-charge terms (Sec. II.C),
 *   - the polarization (Eq. polarization) and the periodic Born effective
 *     charges (Eq. bec_2).
 *
 * Units: Angstrom, e, eV; k_e = 14.3996454784 eV A / e^2.
 * All entry points return a qnep_status; none aborts the process.
 * Device pointers are CUDA global-memory addresses on the current device;
 * host pointers are ordinary host memory.  Calls are asynchronous on the
 * given stream unless stated otherwise.
 */
#ifndef QNEP_H
#define QNEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QNEP_OK = 0,
    QNEP_ERR_ARG = 1,           /* invalid argument (NULL, size, range, NaN box) */
    QNEP_ERR_CUDA = 2,          /* a CUDA call failed; the model should be destroyed */
    QNEP_ERR_NBR_OVERFLOW = 3,  /* an atom had more neighbours than the list capacity */
    QNEP_ERR_UNSUPPORTED = 4,   /* shape / box / option not supported by this library */
    QNEP_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    QNEP_ERR_OOM = 6            /* an allocation (device, or host for a table) failed */
} qnep_status;

/* Descriptor and network sizes (Sec. II.A).  This library supports
 * n_radial = n_angular = 5, basis_radial = basis_angular = 9, l_max = 4,
 * use_4body = 1, n_neurons = 30 (descriptor length 30) and 1..4 species;
 * other sizes return QNEP_ERR_UNSUPPORTED. */
typedef struct {
    int   n_species;
    float rc_radial;        /* radial descriptor cutoff (A) */
    float rc_angular;       /* angular descriptor cutoff (A), <= rc_radial */
    int   n_radial;         /* number of radial functions g_n (n_max + 1) */
    int   n_angular;        /* number of angular radial functions */
    int   basis_radial;     /* Chebyshev terms per radial function (basis size + 1) */
    int   basis_angular;
    int   l_max;            /* highest angular order of the 3-body terms */
    int   use_4body;        /* 1: append the 4-body terms */
    int   n_neurons;        /* hidden-layer width N_neu */
} qnep_hparams;

enum { QNEP_EWALD = 0, QNEP_PPPM = 1 };
enum { QNEP_PREC_FP32 = 0, QNEP_PREC_MLP_BF16 = 1, QNEP_PREC_MLP_TF32 = 2 };

/* Electrostatics settings (Sec. II.B, II.F). */
typedef struct {
    int    mode;       /* 1: U^r + U^k + U^s (Eq. U_ES); 2: U^k only (Eq. mode2) */
    int    kind;       /* QNEP_EWALD or QNEP_PPPM */
    double alpha;      /* Ewald splitting parameter (1/A) */
    double rc_real;    /* real-space cutoff (A), mode 1; <= rc_radial */
    double kmax;       /* Ewald: strict wave-vector cutoff |k| < kmax (1/A) */
    int    mesh[3];    /* PPPM mesh (even sizes, fewer than 2^31 points in all) */
    int    order;      /* PPPM assignment order; this library supports 5 */
    double q_total;    /* target total charge Q of the naked charges (Eq. charge-scaling) */
} qnep_elec;

/* Parameter blob of one candidate: n_params float32 values, laid out as
 *   c_R[ti][tj][n][k]   n_species^2 * n_radial * basis_radial
 *   c_A[ti][tj][n][k]   n_species^2 * n_angular * basis_angular
 *   scaler[nu]          n_des
 *   per species t:      W0[mu][nu] (n_neurons * n_des), b0[mu], w1E[mu], w1q[mu], b1E, b1q
 *   sqrt_eps_inf        1
 * where n_des = n_radial + l_max * n_angular + (use_4body ? n_angular : 0).
 * The network weights are those of the central atom's species. */
size_t qnep_param_count(const qnep_hparams* hp);

typedef struct qnep_model qnep_model;

/* Number and meaning of the FP64 scalar outputs (device array). */
#define QNEP_NSCALARS 20
enum {
    QNEP_S_ENERGY = 0,      /* U^tot = U^NEP + U^ES (eV) */
    QNEP_S_E_NEP = 1,       /* sum_i U_i */
    QNEP_S_E_REAL = 2,      /* U^r (mode 1) */
    QNEP_S_E_KSPACE = 3,    /* U^k (Ewald or PPPM) */
    QNEP_S_E_SELF = 4,      /* U^s (mode 1) */
    QNEP_S_VIRIAL = 5,      /* 9 values, row-major W_ab = sum_i r_ia F_ib convention (eV) */
    QNEP_S_POLARIZATION = 14, /* 3 values, P = sum_i q~^c_i r_i (e A), positions as given */
    QNEP_S_QTILDE_SUM = 17, /* sum of corrected naked charges (= q_total) */
    QNEP_S_PHI_MEAN = 18,   /* mean electrostatic potential dU^ES/dq (V) */
    QNEP_S_STATUS = 19      /* device-side status bits of this call (0 = fine) */
};

/* Outputs of one force call.  Every pointer may be NULL (not computed).
 * Requesting forces or virial runs the backward pass; requesting bec adds
 * the charge-derivative contraction. */
typedef struct {
    double* scalars;      /* device, QNEP_NSCALARS doubles (written every call) */
    float*  forces;       /* device [N][3] (eV/A) */
    float*  charges;      /* device [N] corrected screened charges q^c = q~^c / sqrt(eps_inf) */
    float*  bec;          /* device [N][3][3] periodic Born effective charges Z_i,ab (Eq. bec_2) */
    float*  site_energy;  /* device [N] U_i (optional) */
    float*  potential;    /* device [N] phi_i = dU^ES/dq^c_i (optional) */
    float*  descriptor;   /* device [N][n_des] (optional, for parity checks) */
    int     want_virial;  /* 1: compute the virial into scalars (needs the backward pass) */
    float*  atom_virial;  /* device [N][3][3] per-atom virial W_i (Sec. II.C, Eq. per-atom_virial; eV),
                           * summing to the total virial: -r_ij (x) F_ij of every neighbour entry
                           * (i -> j) added to W_j (descriptor and dynamic-charge partial forces), the
                           * static real-space pair terms split evenly, and the static reciprocal-space
                           * term in the Heyes form k_e sum_k G Re[q_i e^{i k.r_i} S(k)] B(k) (Ewald) or
                           * its mesh form with six more inverse FFTs (PPPM, Sec. II.F).  Optional;
                           * warp-per-atom kernels only (QNEP_ERR_UNSUPPORTED with QNEP_PATH_THREAD or
                           * a vector-Jacobian product). */
} qnep_outputs;

/* Create a model: copies n_candidates parameter blobs (host, candidate-major,
 * n_candidates * qnep_param_count(hp) floats) to the device.  The model owns
 * its device copies, neighbour lists, k-tables, meshes and FFT plans.
 * precision: QNEP_PREC_*.  Fails with QNEP_ERR_UNSUPPORTED for shapes this
 * build does not have kernels for. */
qnep_status qnep_create(qnep_model** out, const qnep_hparams* hp, const float* params_host,
                        size_t n_params, int n_candidates, const qnep_elec* es, int precision);

/* Pre-size every workspace for up to n_atoms atoms in this box (host double[9],
 * rows = lattice vectors) so that later qnep_compute calls with the same box
 * and at most n_atoms atoms allocate nothing (required before stream capture). */
qnep_status qnep_reserve(qnep_model* m, int n_atoms, const double box[9]);

/* One force call on one structure with candidate 0.
 *   positions: device [N][3] float32 (A); may lie outside the box (wrapped internally)
 *   types:     device [N] int32 species index in [0, n_species)
 *   box:       host double[9], rows = lattice vectors a, b, c (right-handed); orthorhombic or a
 *              general (triclinic) cell, with Ewald, PPPM or no electrostatics; every
 *              perpendicular width V / |a_e x a_f| >= the list cutoff.  In a general cell the
 *              images are integer combinations of the rows and the wave vectors are
 *              k = 2 pi H^-1 n (Sec. II.B); PPPM puts its mesh along the lattice vectors (an
 *              atom's mesh coordinates N_d (r H^-1)_d) and takes the three field components as
 *              fractional gradients mapped to Cartesian ones by H^-1 at the interpolation.
 *              Ewald: at most 159 phase factors per atom, (n1 + 1) + (2 n2 + 1) + (2 n3 + 8)
 *              rounded up to odd with n_d = floor(kmax |a_d| / 2 pi); a larger k-set returns
 *              QNEP_ERR_UNSUPPORTED before it is enumerated.
 *   stream:    cudaStream_t (NULL = legacy default stream)
 * Asynchronous: returns after enqueueing.  Device-side errors (neighbour
 * overflow) are recorded in scalars[QNEP_S_STATUS] and returned by the next
 * qnep_sync_status. */
qnep_status qnep_compute(qnep_model* m, int n_atoms, const float* positions, const int* types,
                         const double box[9], void* stream, const qnep_outputs* out);

/* Same call on host buffers (positions [N][3], types [N]; outputs as in
 * qnep_outputs but every pointer is HOST memory): copies in, computes, copies
 * back and synchronizes.  This is the end-to-end path. */
qnep_status qnep_compute_host(qnep_model* m, int n_atoms, const float* positions_host,
                              const int* types_host, const double box[9], void* stream,
                              const qnep_outputs* out_host);

/* Vector-Jacobian product of the force call (the derivatives of Sec. II.C and II.D).
 * For weights g_E (energy), g_q (per-atom corrected screened charges, optional) and
 * g_P (polarization) writes, per atom i (input order),
 *   grad[i][b] = g_E dU^tot/dr_ib + sum_j g_q,j dq^c_j/dr_ib + sum_a g_P,a Z_i,ab
 * where the charge derivative includes the total-charge correction and the last term
 * uses the periodic Born effective charges of Eq. bec_2 as dP/dr (the periodic
 * definition: it is not the derivative of the polarization output P = sum q~^c r of
 * the positions as given, so a finite-difference check of P against it fails in a
 * periodic box by construction; E and q^c are exact derivatives).  The descriptor
 * derivatives are recomputed, nothing per pair is stored.  Other outputs in `out`
 * behave as in qnep_compute except `forces`, which must be NULL; the virial in the
 * scalars is then that of the weighted objective g_E U + sum g_q q^c. */
typedef struct {
    double       energy_weight;    /* g_E */
    const float* charge_weight;    /* device [N] g_q in input order, or NULL */
    double       polar_weight[3];  /* g_P */
    float*       grad;             /* device [N][3] output */
} qnep_vjp;
qnep_status qnep_compute_vjp(qnep_model* m, int n_atoms, const float* positions, const int* types,
                             const double box[9], void* stream, const qnep_outputs* out, const qnep_vjp* vjp);

/* NVE molecular dynamics (velocity Verlet) around the force call.  Runs n_steps steps of
 * dt_fs femtoseconds from the given state; the force call of this model (its
 * precision and electrostatics) is evaluated at every step, neighbour lists rebuilt at every
 * step or, with qnep_set_skin, kept while no atom has moved more than half the skin.
 *   positions, velocities: device [N][3] float32 (A, A/fs), updated in place
 *   types: device [N] int32; masses: host [n_species] doubles (amu)
 *   forces: device [N][3] float32, left holding the forces of the final positions
 *   energies: device [n_steps + 1][2] doubles: U_pot and the kinetic energy (eV) of the
 *             initial state and after every step (kinetic energy reduced in FP64)
 * Asynchronous on `stream`; qnep_sync_status reports the status of the last force call. */
qnep_status qnep_nve_run(qnep_model* m, int n_atoms, float* positions, float* velocities, const int* types,
                         const double* masses, const double box[9], double dt_fs, int n_steps, void* stream,
                         float* forces, double* energies);

/* NVE in a uniform external electric field, with the ionic current along the trajectory
 * (Sec. II.D): as qnep_nve_run, but every force call also computes the Born effective charges
 * (Eq. bec_2) and the ions move under F_i + F^ext_i, F^ext_i,b = sum_a E_a Z_i,ab
 * (Eq. electric_force); after the initial state and after every step the polarization current
 * Pdot_a = sum_i sum_b Z_i,ab v_i,b (Eq. polarization_derivative) of that state is recorded,
 * the series whose autocorrelation gives the infrared spectrum and the ionic conductivity.
 *   efield: host double[3] (V/A), finite; zero gives plain NVE dynamics plus the current
 *   forces: device [N][3], left holding F + F^ext of the final positions
 *   bec:    device [N][3][3] float32 workspace, left holding Z of the final positions
 *   energies: device [n_steps + 1][2] (U_pot, K) as for qnep_nve_run (U_pot is the force
 *           call's energy; the field's work is not in it)
 *   pdot:   device [n_steps + 1][3] doubles (e A/fs), 8-byte aligned
 * Asynchronous on `stream`; qnep_sync_status reports the status of the last force call.
 * QNEP_ERR_ARG for a NULL pointer, n_steps < 0, dt_fs <= 0, a non-finite field, non-positive
 * masses or a misaligned pdot; force-call errors as for qnep_compute.  The model owns its small
 * MD state buffers; the caller owns every argument buffer. */
qnep_status qnep_nve_run_field(qnep_model* m, int n_atoms, float* positions, float* velocities, const int* types,
                               const double* masses, const double box[9], double dt_fs, int n_steps,
                               const double efield[3], void* stream, float* forces, float* bec, double* energies,
                               double* pdot);

/* Synchronize the stream and return the device-side status of the last call:
 * the status word its kernels wrote, decoded by qnep_status_from_device_bits. */
qnep_status qnep_sync_status(qnep_model* m, void* stream);

/* Device status word of a force call (single-structure and batched): bit 0 an atom
 * had more neighbours than the list capacity, bit 1 a bounded device-side wait on a
 * bulk copy or a tensor-core operation gave up (the outputs of that call are not
 * valid), bit 2 a species index outside [0, n_species).  Decoded in that order of
 * precedence: bit 2 -> QNEP_ERR_ARG, bit 0 -> QNEP_ERR_NBR_OVERFLOW, bit 1 ->
 * QNEP_ERR_TIMEOUT, none -> QNEP_OK.  A pure host function. */
qnep_status qnep_status_from_device_bits(unsigned int bits);

/* Test hooks: OR `bits` into the device status word of the model's (or batch's) last
 * call, as a kernel would, after synchronizing with it; the next qnep_sync_status
 * (qnep_batch_sync_status) reports them.  They let a test check the decoding of a
 * device-side timeout without making a device wait run out. */
qnep_status qnep_debug_set_status(qnep_model* m, unsigned int bits);

/* Change the neighbour-list capacities (entries per atom); 0 keeps the value. */
qnep_status qnep_set_capacity(qnep_model* m, int cap_list, int cap_angular);

/* Verlet skin for repeated force calls on moving atoms (MD; warp-per-atom kernels).  With
 * skin > 0 (A) the model keeps candidate lists with cutoff r_list + skin (r_list = the
 * larger of the radial descriptor and real-space cutoffs) and rebuilds them (cell binning and
 * search) only when an atom has moved more than skin / 2 since the last build; otherwise the
 * force call filters the kept candidates by the current distances, which gives the same
 * neighbours as a fresh search (sums in another order: FP32 rounding).  The test and the
 * choice run on the device, so a call needs no host synchronisation (it can be captured in a
 * CUDA graph once the lists exist).  A new box, atom count or capacity forces a rebuild; atom
 * types must not change while a list is kept (call qnep_set_skin again to force a rebuild).
 * skin = 0 (the default) rebuilds the lists at every call.  QNEP_ERR_ARG for a negative,
 * non-finite or > 5 A skin.  List overflow is reported as for qnep_compute; an overflow of the
 * kept candidate lists (capacity: the list capacity scaled by the volume ratio of the two
 * cutoffs) is in the status of the call that rebuilt them only, so check the status after each
 * call while a list is kept (the Python binding does, growing the capacity, which rebuilds).
 * qnep_skin_rebuilds: the number of rebuilds so far (synchronises the device). */
qnep_status qnep_set_skin(qnep_model* m, double skin);
qnep_status qnep_skin_rebuilds(qnep_model* m, unsigned int* count);

/* Kernel family for the per-atom stages: QNEP_PATH_AUTO picks the warp-per-atom
 * kernels (the faster family at every size measured, 40 atoms to 1 M atoms);
 * QNEP_PATH_WARP / QNEP_PATH_THREAD force one family (both compute the same
 * quantities).  Used by the tests and for comparisons. */
enum { QNEP_PATH_AUTO = 0, QNEP_PATH_WARP = 1, QNEP_PATH_THREAD = 2 };
qnep_status qnep_set_path(qnep_model* m, int path);

/* Stage timers (tracing).  When enabled, every qnep_compute records CUDA events
 * around each stage on its stream and accumulates the elapsed times.
 * qnep_stage_times synchronizes, writes up to max_stages accumulated times (ms)
 * and the number of timed calls, and resets the accumulators.  Stage names:
 * qnep_stage_name(k) for k < QNEP_NSTAGES ("" beyond). */
#define QNEP_NSTAGES 10
qnep_status qnep_set_profiling(qnep_model* m, int enable);
qnep_status qnep_stage_times(qnep_model* m, float* ms_out, int max_stages, int* n_calls);
const char* qnep_stage_name(int stage);

/* Response to a uniform external electric field from the Born effective charges
 * (Sec. II.D):
 *   Eq. electric_force:          forces[i][b] (+)= sum_a E_a Z_i,ab      (eV/A)
 *   Eq. polarization_derivative: pdot[a] = sum_i sum_b Z_i,ab v_i,b      (e A per time unit of v)
 *   bec:        device [N][3][3] float32 Z_i,ab (a = polarization component, b = position
 *               component), as written by qnep_compute; NULL only when n_atoms = 0
 *   efield:     host double[3] E (V/A); needed when forces != NULL
 *   velocities: device [N][3] float32; needed when pdot != NULL and n_atoms > 0, ignored otherwise
 *   forces:     device [N][3] float32 F^ext, overwritten (accumulate = 0) or added to an
 *               existing force array (accumulate = 1), or NULL
 *   pdot:       device double[3], cleared on the stream and then summed (a compensated FP32
 *               sum per thread, FP32 warp sums, FP64 across warps and blocks with FP64
 *               atomics: the last bits depend on the order of the blocks), or NULL
 * Float arrays must be 4-byte aligned (16-byte alignment of all of them takes the
 * vectorised path), pdot 8-byte aligned.  Asynchronous on `stream`.  Returns
 * QNEP_ERR_ARG for a negative n_atoms, a missing input, a non-finite field or a
 * misaligned pointer, QNEP_ERR_CUDA if a launch fails; with neither forces nor pdot
 * requested it does nothing.  Caller owns every buffer; nothing is allocated. */
qnep_status qnep_field_response(int n_atoms, const float* bec, const double efield[3], const float* velocities,
                                float* forces, int accumulate, double* pdot, void* stream);

/* Reciprocal-space Ewald sum of given charges that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory -- host programs that give all of the GPU's memory
 * to their own pool allocator and forbid allocations by libraries, and
 * time-critical loops where cudaMalloc / cudaFree would synchronise the device.
 * It runs the kernels of the reciprocal-space stage of qnep_compute on its
 * inputs, with every scratch buffer in one fixed-size __device__ array (about
 * 10 MB, held by each GPU that loads the library until the process exits).
 *   positions:     device [N][3] float32 (A)         charges: device [N] float32 (e)
 *   box:           host double[9], orthorhombic       alpha, kmax: as in qnep_elec
 *   potential:     device [N] phi^k_i = dU^k/dq_i (V), or NULL
 *   forces:        device [N][3] static reciprocal-space forces (eV/A), or NULL
 *   energy_virial: device [10] doubles: U^k, then the 3x3 static k-space virial, or NULL
 *   err, err_len:  optional host buffer for a message when the call fails
 * Limits: N <= QNEP_NOALLOC_MAX_ATOMS, at most QNEP_NOALLOC_MAX_PHASE phase
 * factors per atom ((floor(kmax Lx/2pi)+1) + 2 floor(kmax Ly/2pi) + 1 +
 * 2 floor(kmax Lz/2pi) + 8, rounded up to odd) and QNEP_NOALLOC_MAX_KPAD padded
 * half-space wave vectors; larger inputs return QNEP_ERR_UNSUPPORTED before any
 * GPU work.  The charges are used as given (no total-charge correction).
 * The first call on a device (with that device current) looks up the array's
 * address with cudaGetSymbolAddress; make it before any stream capture.  All
 * calls share the array and it keeps the last call's contents (what must start
 * at zero is cleared by each call); calls that overlap on the GPU race. */
#define QNEP_NOALLOC_MAX_ATOMS 8192
#define QNEP_NOALLOC_MAX_PHASE 128
#define QNEP_NOALLOC_MAX_KPAD 32768
qnep_status qnep_ewald_kspace_noalloc(int n_atoms, const float* positions, const float* charges,
                                      const double box[9], double alpha, double kmax, float* potential,
                                      float* forces, double* energy_virial, void* stream, char* err,
                                      size_t err_len);

/* ---- Batched evaluation -----------------------------------------------------
 * Many structures of uneven size, each under many candidate parameter vectors:
 * the shape of a separable natural-evolution-strategy fitness evaluation, where
 * every candidate of the population is scored on every training structure
 * (Sec. II.E; the training loss weighs energies, forces, virials, BEC and total
 * charges).  One call
 * returns, for every (candidate c, structure s), the total energy U^tot
 * (Eq. U_i, Eq. U_ES with the charges of Sec. II.D), the forces including the
 * charge-derivative terms (Sec. II.C) and the corrected charges q^c.
 * Electrostatics: Ewald (mode 1 or 2) per structure; PPPM is not offered here.
 * The virial and the polarization per (candidate, structure), the per-atom Born effective charges
 * (Eq. bec_2) and the total charge before the correction come with qnep_batch_compute_outputs.
 *
 * qnep_batch_create: hp and es as for qnep_create (es->kind must be QNEP_EWALD);
 *   params_host = n_candidates blobs of qnep_param_count(hp) floats, candidate-major.
 * qnep_batch_compute (asynchronous on `stream`, no host synchronisation once the
 *   batch description is known, so it can be captured in a CUDA graph):
 *   atom_offsets: host [n_struct + 1], atom_offsets[0] = 0, non-decreasing;
 *                 structure s holds atoms atom_offsets[s] .. atom_offsets[s+1]-1
 *   positions:    device [N_total][3] float32 (A), types: device [N_total] int32
 *   boxes:        host [n_struct][9] doubles, rows = lattice vectors: orthorhombic or a general
 *                 right-handed cell (QNEP_ERR_ARG for a left-handed or degenerate one).  The
 *                 kernels run general cells in the restricted form a = (a_x, 0, 0),
 *                 b = (b_x, b_y, 0), c = (c_x, c_y, c_z); a cell given otherwise is rotated into it
 *                 (rows of R: a / |a|, (a x b) x a / |..|, a x b / |a x b|), its positions rotated
 *                 as they are read, and forces, virial and BEC rotated back (R^T F, R^T W R,
 *                 R^T Z R): every output is in the input frame.  Every perpendicular width >= the
 *                 neighbour-list cutoff; at most 32768 atoms per structure; at most 94 Ewald phase
 *                 factors per atom, (n1 + 1) + (2 n2 + 1) + (2 n3 + 8) with
 *                 n_d = floor(kmax |a_d| / 2 pi) (QNEP_ERR_UNSUPPORTED before any work otherwise)
 *   energy:       device [n_candidates][n_struct] doubles (eV)
 *   forces:       device [n_candidates][N_total][3] float32 (eV/A), or NULL
 *   charges:      device [n_candidates][N_total] float32 (e), or NULL
 * The first call with a new (atom_offsets, boxes) builds the k-tables and work
 * list on the host and (re)allocates workspaces; later identical calls only
 * launch.  A graph captured from a call keeps that call's workspaces: re-capture it
 * after a call that reallocated them (a new description, a capacity change, a
 * launch shape with more resident blocks).  Asking for BEC allocates its accumulators
 * in a buffer of their own, so it does not move the workspaces of calls without BEC.
 * Errors in the arguments return before any GPU work; device-side conditions (list
 * overflow, a species index out of range) are reported by qnep_batch_sync_status
 * (QNEP_ERR_NBR_OVERFLOW: raise the capacity with
 * qnep_batch_set_capacity and call again; outputs of that call are invalid).
 * Caller owns every buffer; the batch owns its device copies and workspaces. */
typedef struct qnep_batch qnep_batch;
enum { QNEP_BATCH_ORDER_LARGEST_FIRST = 0, QNEP_BATCH_ORDER_STRUCTURE = 1 };
qnep_status qnep_batch_create(qnep_batch** out, const qnep_hparams* hp, const float* params_host,
                              size_t n_params, int n_candidates, const qnep_elec* es);
qnep_status qnep_batch_compute(qnep_batch* b, int n_struct, const int* atom_offsets, const float* positions,
                               const int* types, const double* boxes, void* stream, double* energy,
                               float* forces, float* charges);
qnep_status qnep_batch_sync_status(qnep_batch* b);

/* Outputs of a batched call, indexed [candidate][structure] (energy, virial, total charge) or
 * [candidate][atom] (forces, charges, BEC); energy is required, the others may be NULL.
 *   energy:  [C][S] doubles, U^tot (eV)
 *   forces:  [C][N_total][3] float32 (eV/A)
 *   charges: [C][N_total] float32, corrected charges q^c (e)
 *   virial:  [C][S][9] doubles, W_ab = -dU/d eps_ab under the homogeneous strain
 *            r -> (I + eps) r of positions and cell (eV; row-major 3x3): the sum over neighbour
 *            entries of -r_ij (x) F_ij (descriptor and dynamic-charge partial forces, Sec. II.C),
 *            the static real-space pair terms and the k-space W^k = sum k_e G |S|^2 B
 *            (Eq. virial-kspace-total), each FP32 per atom or per k and FP64 across them.
 *   bec:     [C][N_total][9] float32, Born effective charges Z_i,ab = dP_a/dr_ib of Eq. bec_2 (e;
 *            row-major, first index the polarization component): q~^c_i on the diagonal plus
 *            1/2 r_ij (x) a_ij for each of i's neighbour entries and -1/2 r_ji (x) a_ji for each
 *            entry (j -> i), a_ij = dq~_i/dr_ij from the charge adjoint sqrt(eps_inf) dq_i/dD
 *            (Sec. II.D).  Asking for it adds a second pass over the neighbour entries (about
 *            the backward's time again) and 48 bytes of scratch per atom, candidate and
 *            resident block; it is the input of the D_Z term of the training loss.
 *   total_charge: [C][S] doubles, sum_i q~_i = sqrt(eps_inf) sum_i q_i of the network's charges
 *            BEFORE the correction of Eq. charge-scaling (e; after it the sum is the target),
 *            the input of the D_Q term of the training loss; 0 for a structure without atoms.
 *   polarization: [C][S][3] doubles, P = sum_i q~^c_i r_i (Eq. polarization; e A) over the
 *            positions as given (not wrapped), as qnep_compute reports it; FP32 products over 8
 *            atoms per candidate, FP64 across them. */
typedef struct {
    double* energy;
    float*  forces;
    float*  charges;
    double* virial;
    float*  bec;
    double* total_charge;
    double* polarization;
} qnep_batch_outputs;
/* As qnep_batch_compute, with every output of qnep_batch_outputs (device pointers). */
qnep_status qnep_batch_compute_outputs(qnep_batch* b, int n_struct, const int* atom_offsets, const float* positions,
                                       const int* types, const double* boxes, void* stream,
                                       const qnep_batch_outputs* out);
/* The end-to-end form on HOST buffers: positions [N_total][3] and types [N_total] from host
 * memory, every requested output of out_host (host pointers) copied back, then a stream
 * synchronisation and the device status (as qnep_batch_sync_status).  The batch keeps device
 * copies of the inputs and outputs (grown on demand, freed by qnep_batch_destroy); pinned host
 * memory makes the copies asynchronous, pageable memory works but copies synchronously. */
qnep_status qnep_batch_compute_host(qnep_batch* b, int n_struct, const int* atom_offsets, const float* positions_host,
                                    const int* types_host, const double* boxes, void* stream,
                                    const qnep_batch_outputs* out_host);
qnep_status qnep_batch_debug_set_status(qnep_batch* b, unsigned int bits);   /* test hook, as above */
/* Neighbour capacities (entries per atom; 0 = from the densest structure) and their current values. */
qnep_status qnep_batch_set_capacity(qnep_batch* b, int cap_list, int cap_angular);
qnep_status qnep_batch_capacity(const qnep_batch* b, int* cap_list, int* cap_angular);
/* Launch configuration: warps per block of the item kernel (4 or 8) and the order
 * in which blocks take the (structure, candidate-group) items. */
qnep_status qnep_batch_set_config(qnep_batch* b, int warps, int order);
qnep_status qnep_batch_get_config(const qnep_batch* b, int* warps, int* order);
/* Static geometry, for training on fixed structures (Sec. II.E: every generation of the population
 * is scored on the same training structures, so only the candidates change between calls).  With
 * enable = 1, the candidate-independent pre-pass (wrapping, cell and species order, neighbour
 * lists, pair geometry rows, basis sums, phase factors, operand images) runs in the first call
 * after this one and is reused by later calls while the batch description, the positions and
 * types pointers and the contraction's needs are unchanged; the caller promises that the memory
 * behind positions and types does not change meanwhile, or calls qnep_batch_geometry_changed
 * (the next call then rebuilds); with qnep_batch_compute_host the promise covers the host
 * positions and types.  A change between the FP32 and the tensor-core contraction rebuilds.
 * Neighbour overflow and species errors of the pre-pass are reported by the call that built the
 * geometry and by every call that reuses it (the pre-pass keeps its own status word); a
 * qnep_batch_sync_status that reports one ends the reuse, so the next call rebuilds.
 * A call captured in a CUDA graph while the geometry is kept contains no pre-pass.  enable = 0
 * (the default) runs the pre-pass in every call.  QNEP_ERR_ARG for a NULL batch or an enable
 * outside {0, 1}.  No GPU work. */
qnep_status qnep_batch_set_static_geometry(qnep_batch* b, int enable);
qnep_status qnep_batch_geometry_changed(qnep_batch* b);
/* Descriptor contraction of the batched call: the angular expansion coefficients
 * A_{n,lm} = sum_{s,k} c^A[t_i][s][n][k] B^A[s][k][lm] of every atom and candidate (Sec. II.A)
 * in FP32 on the FP32 pipes (QNEP_BATCH_CONTRACT_FP32, the default), or on the tensor cores
 * (QNEP_BATCH_CONTRACT_BF16X3: each operand split into BF16 hi + lo parts, three products
 * hi.hi + hi.lo + lo.hi accumulated in FP32, about 2^-16 relative error per term; the energy
 * stays within the FP32 path's 1e-6 eV/atom of the FP64 oracle).  The tensor-core form runs
 * 8-warp blocks (it sets warps = 8; qnep_batch_set_config(4, ...) then makes the next call
 * return QNEP_ERR_UNSUPPORTED).  QNEP_BATCH_CONTRACT_BF16 is the reduced-precision (mixed)
 * form: one BF16 product hi.hi (about 2^-9 relative per term), for uses that accept the mixed
 * path's accuracy (force RMSE <= 5e-3 eV/A against the FP64 oracle).  Everything after the
 * contraction is the same in all three. */
enum { QNEP_BATCH_CONTRACT_FP32 = 0, QNEP_BATCH_CONTRACT_BF16X3 = 1, QNEP_BATCH_CONTRACT_BF16 = 2 };
qnep_status qnep_batch_set_contraction(qnep_batch* b, int contract);
qnep_status qnep_batch_get_contraction(const qnep_batch* b, int* contract);
/* Autotuner: times every launch configuration on this batch (`reps` calls each,
 * median, CUDA events on `stream`), keeps the fastest and returns its time (ms).
 * Writes the same outputs as qnep_batch_compute. Synchronizes the stream. */
qnep_status qnep_batch_autotune(qnep_batch* b, int n_struct, const int* atom_offsets, const float* positions,
                                const int* types, const double* boxes, void* stream, double* energy,
                                float* forces, float* charges, int reps, double* best_ms);
/* Stage timers: when enabled, each qnep_batch_compute records CUDA events around the
 * candidate-independent pre-pass and around the item kernel on its stream;
 * qnep_batch_stage_times synchronizes, writes the accumulated times (ms) of the
 * two stages and the number of timed calls, and resets them. */
qnep_status qnep_batch_set_profiling(qnep_batch* b, int enable);
qnep_status qnep_batch_stage_times(qnep_batch* b, float* ms_out /* [2] */, int* n_calls);
const char* qnep_batch_last_error(const qnep_batch* b);

/* Replace the candidates' parameter vectors of a batch from device memory (asynchronous on
 * `stream`, ordered before later qnep_batch_compute calls on that stream, including replays
 * of a captured graph of one): params = device [n_candidates][qnep_param_count] float32, the
 * blob layout of qnep_create.  Used by the training loop below; values are not checked (a
 * non-finite candidate gives non-finite outputs and a NaN loss, which ranks last).  The batch owns
 * its copy; the caller keeps `params`.  QNEP_ERR_ARG for a NULL batch or params, QNEP_ERR_CUDA if
 * the launch fails. */
qnep_status qnep_batch_set_params(qnep_batch* b, const float* params, void* stream);

/* ---- Training: population loss and separable NES (Sec. II.E) ----------------
 * The paper trains every parameter z (descriptor, network, sqrt(eps_inf)) with SNES on
 *   L(z) = l_e D_e + l_f D_f + l_v D_v + l_Z D_Z + l_Q D_Q + l_1 |z|_1 + l_2 |z|_2^2.
 * The batched call feeds every term (qnep_batch_loss_full); qnep_batch_loss and
 * qnep_batch_loss_v are its shorter forms.  Read as
 *   D_e = sqrt(1/S' sum_s ((E_s - E_s^ref) / N_s)^2)   over the S' structures with atoms (eV/atom)
 *   D_f = sqrt(1/(3N) sum_i,b (F_ib - F_ib^ref)^2)      over all N atoms (eV/A).
 * One device-resident iteration: qnep_snes_sample -> qnep_batch_set_params ->
 * qnep_batch_compute -> qnep_batch_loss -> qnep_snes_update.  All pointers are device memory
 * unless stated; calls are asynchronous on `stream`; nothing is allocated. */
typedef struct {
    double energy;   /* l_e */
    double force;    /* l_f */
    double l1;       /* l_1 */
    double l2;       /* l_2 */
} qnep_loss_weights;

/* Candidates z_k = mu + sigma * s_k (SNES sampling; the normal deviates s are the caller's):
 * mu, sigma [P], noise [C][P], params [C][P] float32 (params = fmaf(sigma, noise, mu)).
 * QNEP_ERR_ARG for C or P below 1 or a NULL pointer, QNEP_ERR_CUDA if the launch fails. */
qnep_status qnep_snes_sample(int n_candidates, int n_params, const float* mu, const float* sigma, const float* noise,
                             float* params, void* stream);

/* Loss of every candidate.  atom_offsets: device [S+1] as for qnep_batch_compute; energy
 * [C][S] f64 and forces [C][N][3] f32 as qnep_batch_compute writes them; energy_ref [S] f64,
 * forces_ref [N][3] f32 (forces and forces_ref both given or both NULL: D_f = 0); params [C][P]
 * for the regularisation (NULL: no norm terms); w: host weights.  Writes loss [C] f64 and
 * terms [C][4] f64 = (D_e, D_f, |z|_1, |z|_2^2).  D_f sums 8 squares per thread in FP32, the
 * rest is FP64 (FP64 atomics across blocks: the last bits depend on the block order).
 * QNEP_ERR_ARG for missing buffers, C outside [1, 65535], non-finite weights. */
qnep_status qnep_batch_loss(int n_candidates, int n_struct, const int* atom_offsets, int n_total,
                            const double* energy, const float* forces, const double* energy_ref,
                            const float* forces_ref, const float* params, int n_params,
                            const qnep_loss_weights* w, double* loss, double* terms, void* stream);

/* Loss with the virial term: as qnep_batch_loss, plus
 *   D_v = sqrt(1/(6 S') sum_s sum_{ab in xx,yy,zz,xy,yz,zx} ((W_s,ab - W^ref_s,ab) / N_s)^2)
 * over the S' structures with atoms (virial per atom, eV; the NEP convention of an RMSE over
 * the six independent components) and L = l_e D_e + l_f D_f + l_v D_v + l_1 |z|_1 + l_2 |z|_2^2.
 * virial [C][S][9] f64 as qnep_batch_compute_outputs writes it and virial_ref [S][9] f64, both
 * given or both NULL (D_v = 0); terms [C][5] f64 = (D_e, D_f, D_v, |z|_1, |z|_2^2). */
typedef struct {
    double energy;   /* l_e */
    double force;    /* l_f */
    double virial;   /* l_v */
    double l1;       /* l_1 */
    double l2;       /* l_2 */
} qnep_loss_weights_v;
qnep_status qnep_batch_loss_v(int n_candidates, int n_struct, const int* atom_offsets, int n_total,
                              const double* energy, const float* forces, const double* virial,
                              const double* energy_ref, const float* forces_ref, const double* virial_ref,
                              const float* params, int n_params, const qnep_loss_weights_v* w, double* loss,
                              double* terms, void* stream);

/* The full loss of Sec. II.E:
 *   L = l_e D_e + l_f D_f + l_v D_v + l_Z D_Z + l_Q D_Q + l_1 |z|_1 + l_2 |z|_2^2
 * with D_e, D_f, D_v as above and
 *   D_Z = sqrt(1/(9 N_Z) sum_{s: bec_has_ref[s] != 0} sum_{i in s} sum_ab (Z_i,ab - Z^ref_i,ab)^2)
 *         over the N_Z atoms of the structures that carry reference BEC (the paper makes BEC
 *         targets optional, for a subset of the training structures; 0 when none has atoms)
 *   D_Q = sqrt(1/S' sum_s (Q_s - Q^ref_s)^2) over the S' structures with atoms, Q_s the total
 *         charge before the correction (qnep_batch_outputs.total_charge), Q^ref_s its target.
 * `in` holds the batched call's outputs (device): energy [C][S] f64 (required), forces
 * [C][N][3] f32, virial [C][S][9] f64, bec [C][N][9] f32, total_charge [C][S] f64; `ref` the
 * references in the same order without the candidate index (energy [S], forces [N][3], virial
 * [S][9], bec [N][9], total_charge [S]).  Each output and its reference are given or NULL together
 * (a NULL pair gives its term 0); bec_has_ref: device [S] int, required with bec.  Writes loss [C]
 * f64 and terms [C][7] f64 = (D_e, D_f, D_v, D_Z, D_Q, |z|_1, |z|_2^2).  The BEC squares are summed
 * like the forces' (compensated FP32 per thread, FP64 across blocks).  QNEP_ERR_ARG for missing
 * or unpaired buffers, C outside [1, 65535], non-finite weights. */
typedef struct {
    const double* energy;
    const float*  forces;
    const double* virial;
    const float*  bec;
    const double* total_charge;
} qnep_loss_inputs;
typedef struct {
    double energy;   /* l_e */
    double force;    /* l_f */
    double virial;   /* l_v */
    double bec;      /* l_Z */
    double charge;   /* l_Q */
    double l1;       /* l_1 */
    double l2;       /* l_2 */
} qnep_loss_weights_full;
qnep_status qnep_batch_loss_full(int n_candidates, int n_struct, const int* atom_offsets, int n_total,
                                 const qnep_loss_inputs* in, const qnep_loss_inputs* ref, const int* bec_has_ref,
                                 const float* params, int n_params, const qnep_loss_weights_full* w, double* loss,
                                 double* terms, void* stream);

/* One SNES step (Schaul et al. 2011) from the losses of the population sampled with `noise`:
 * candidates ranked by loss (lowest first, ties by index, NaN last); utilities
 * u_k = max(0, ln(C/2 + 1) - ln k) / sum_j max(0, ln(C/2 + 1) - ln j) - 1/C for rank k;
 * mu += eta_mu sigma sum_k u_k s_k; sigma *= exp(eta_sigma / 2 sum_k u_k (s_k^2 - 1)),
 * in FP64, stored to the float32 mu and sigma [P] in place.  A negative rate selects the
 * published default (eta_mu = 1, eta_sigma = (3 + ln P) / (5 sqrt P)).  loss [C] f64 and noise
 * [C][P] f32 are read, mu and sigma [P] f32 updated.  QNEP_ERR_ARG for C outside [1, 1024], P below
 * 1, a NULL pointer or a non-finite rate; QNEP_ERR_CUDA if the launch fails.  The update is
 * deterministic (fixed summation order), so ranks given the same losses and deviates agree. */
qnep_status qnep_snes_update(int n_candidates, int n_params, const double* loss, const float* noise, float* mu,
                             float* sigma, double eta_mu, double eta_sigma, void* stream);
void        qnep_batch_destroy(qnep_batch* b);

void        qnep_destroy(qnep_model* m);
const char* qnep_status_string(qnep_status s);
const char* qnep_last_error(qnep_model* m);   /* detail of the last failing call */

#ifdef __cplusplus
}
#endif
#endif /* QNEP_H */
