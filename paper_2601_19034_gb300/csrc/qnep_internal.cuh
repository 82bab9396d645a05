// Internal declarations of the GB300 qNEP force call (not part of the C ABI).
//
// Layout conventions (device):
//   pos4[i]            float4 (x, y, z wrapped into the box, species as int bits)
//   list entries       32 bits: neighbour index j in bits 0..25, image shift T in bits 26..31,
//                      two bits per axis holding T_d + 1; r_ij = pos4[j] + T.L - pos4[i];
//                      column-major [cap][N]; entries of an atom grouped by neighbour
//                      species (count per species in cnt[s][N])
//   per-atom vectors   column-major [component][N] for coalesced access
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace qnep {

// Descriptor / network shape supported by the kernels of this library.
constexpr int NR = 5;      // radial functions
constexpr int KR = 9;      // Chebyshev terms (radial)
constexpr int NA = 5;      // angular radial functions
constexpr int KA = 9;      // Chebyshev terms (angular)
constexpr int LMAX = 4;
constexpr int NLM = 24;    // (l, m) pairs for l = 1..4
constexpr int NDES = NR + NA * LMAX + NA;   // 30
constexpr int NNEU = 30;
constexpr int MAX_SPECIES = 4;
constexpr int NANG = NA * NLM;              // 120 angular expansion coefficients per atom
constexpr float KE = 14.3996454784f;        // k_e = 1/(4 pi eps0), eV A / e^2
constexpr double KE_D = 14.3996454784;

constexpr int PREC_BF16 = 1;    // network operands on the tensor cores (precision form)
constexpr int PREC_TF32 = 2;

constexpr int CODE_SHIFT = 26;
constexpr int INDEX_MASK = (1 << CODE_SHIFT) - 1;
constexpr int CODE_SELF = 1 | (1 << 2) | (1 << 4);   // image shift (0, 0, 0)

// Offsets (floats) into one candidate's parameter blob.
struct ParamLayout {
    int n_species;
    int c_radial;      // [S][S][NR][KR]
    int c_angular;     // [S][S][NA][KA]
    int scaler;        // [NDES]
    int mlp;           // start of species 0 network block
    int mlp_stride;    // floats per species block
    int sqrt_eps;      // 1 float
    int total;
    // inside a species block
    static constexpr int W0 = 0;                  // [NNEU][NDES]
    static constexpr int B0 = NNEU * NDES;        // [NNEU]
    static constexpr int W1E = B0 + NNEU;
    static constexpr int W1Q = W1E + NNEU;
    static constexpr int B1E = W1Q + NNEU;
    static constexpr int B1Q = B1E + 1;
    static constexpr int BLOCK = B1Q + 1;
};

inline ParamLayout make_layout(int s) {
    ParamLayout p;
    p.n_species = s;
    p.c_radial = 0;
    p.c_angular = s * s * NR * KR;
    p.scaler = p.c_angular + s * s * NA * KA;
    p.mlp = p.scaler + NDES;
    p.mlp_stride = ParamLayout::BLOCK;
    p.sqrt_eps = p.mlp + s * ParamLayout::BLOCK;
    p.total = p.sqrt_eps + 1;
    return p;
}

// Orthorhombic box and cell grid, passed by value to kernels.
struct Geom {
    float L[3];        // edge lengths (orthorhombic; the diagonal of H otherwise)
    float invL[3];
    int tri;           // 1: a general (triclinic) cell, H and Hi below are used
    float H[9];        // lattice vectors as rows a, b, c (row-major): r = s H for fractional s
    float Hi[9];       // H^-1 (row-major): s = r Hi
    int nc[3];         // cells per dimension (along the fractional axes)
    int ncells;
    float rc_list;     // list cutoff (max of radial descriptor and real-space cutoffs)
    float rc_radial;
    float rc_angular;
    float rc_real;     // 0 when there is no real-space term
    int list_sa, list_se;   // list entry e of sorted atom k at k * list_sa + e * list_se
    int ang_sa, ang_se;     // same for the angular list
};

// FP64 accumulators of one force call (zeroed at the start of every call).
struct Accum {
    double sum_q;        // sum of raw network charges q_i
    double sum_u;        // sum of site energies
    double sum_phi;      // sum of phi_i
    double e_real;
    double e_self;
    double e_kspace;
    double virial[9];
    double polar[3];
    double sum_qc;       // sum of corrected naked charges q~^c
    double sum_gq;       // sum of the charge weights of a vector-Jacobian product
    unsigned int status; // bit 0: neighbour overflow, bit 1: a bounded wait gave up
    unsigned int work_fwd;   // atom counters of the dynamically scheduled warp-per-atom kernels
    unsigned int work_bwd;
    unsigned int pad;
};

// Electrostatics constants for the kernels.
struct ElecConst {
    int mode;            // 0: none, 1: real + k + self, 2: k only
    int kind;            // 0 Ewald, 1 PPPM
    float alpha;
    float q_total;
};

// Per-atom electrostatic fields consumed by the backward kernels.
struct FieldIn {
    const float4* kfield;   // (F^k / q, phi^k) per sorted atom (zero without k-space)
    const float4* rfield;   // (F^r, phi^r) per sorted atom (zero without real space)
    int mode;
    float alpha;
    float q_target;         // Q in screened-charge units (Q / sqrt(eps_inf))
    float e_weight;         // weight of the energy (1 for forces)
    const float* gq;        // per-atom charge weights in input order (NULL: none)
    const int* sidx;        // input index of each sorted atom (for gq)
};

// Phase factors per atom (the odd row length nph below) that the single-structure Ewald kernels
// hold in shared memory: the structure-factor kernel's copy rings take 1 KB per phase factor
// within its 160 KB opt-in.  A k-set with more is refused on the host before it is enumerated.
constexpr int EWALD_MAX_NPH = 159;

// Ewald k-space description (host-built, uploaded when the box changes).
//  Half space of wave vectors k = 2 pi (n1/Lx, n2/Ly, n3/Lz), |k| < kmax, grouped
//  in columns (n1, n2) holding the contiguous run n3 in [lo, hi].  Each column is
//  stored as chunks of 8 consecutive n3 (padded past hi with G = 0), so the
//  padded index of (column c, chunk h, t) is col[c].w + 8 h + t.
struct EwaldTab {
    int n1max, n2max, n3max;
    int ncol;             // columns
    int nchunk;           // 8-wide chunks over all columns
    int nk;               // padded k count = 8 nchunk
    int nph;              // complex phase factors per atom
    int yoff, zoff;       // offsets of the Y and Z tables in an atom's row
    float L[3];
    float invl_hi[3], invl_lo[3];   // 1/L as a float pair (phase reduction)
    int tri;              // 1: a general cell: phases of the fractional coordinates s = r H^-1, k = 2 pi H^-1 n
    float hi_hi[9], hi_lo[9];       // H^-1 (row-major) as float pairs (phase reduction of a general cell)
    float krec[9];        // 2 pi H^-1 (row-major): k_d = sum_e krec[3 d + e] n_e
    float alpha;
    const int4* col;      // [ncol + 1] (n1, n2, lo, padded offset); last entry: (0, 0, 0, nk)
    const int* chunk_col; // [nchunk] column of each chunk
    const int* chunk_order; // [nchunk] processing order of the chunks in the structure-factor kernel
                            // (sorted by n3 window so a warp's lanes share Z loads); NULL = identity
    const float* kg;      // [nk] G(k) = (2 pi / V) exp(-k^2 / 4 alpha^2) / k^2, 0 on padding
    double2* S;           // [nk] structure factor sum_i q_i exp(-i k.r_i) (FP64)
    float2* C;            // [nk] 4 k_e G(k) S(k) (FP32) for the force / potential pass
    float2* phase;        // [N][nph]: X[0..n1max], Y[-n2max..n2max], Z[-n3max..n3max+7]
    const float4* kb;     // [2 nk] B(k) = I - (2 / (4 alpha^2) + 2 / k^2) k k^T as (xx, yy, zz, xy), (xz, yz, -, -),
                          // zero on padding (per-atom virial only; may be NULL otherwise)
};

// Per-atom virial scratch of one force call (sorted order), AVIR floats per atom:
// [0..8]  W_i of the neighbour entries (partial forces, -r_ij (x) F_ij added to W_j) and of the
//         static real-space pair terms, row-major 3 x 3;
// [9..14] the static reciprocal-space term per unit charge, (xx, yy, zz, xy, xz, yz):
//         sum_half Re[C e^{i k.r_i}] B(k) (Ewald) or 2 k_e sum_s W(r_i - r_s) F^-1[G_opt B S](r_s)
//         (PPPM); W_i^k = q_i / 2 times it.
constexpr int AVIR = 16;

// PPPM mesh description (Sec. II.F); meshes are [nx][ny][nz] (z fastest), the half
// spectrum [nx][ny][nz/2 + 1].
struct PppmTab {
    int nx, ny, nz;
    size_t nreal;        // nx ny nz
    size_t nhalf;        // nx ny (nz/2 + 1)
    float inv_h[3];      // N_d / L_d (high part)
    float inv_h_lo[3];   // N_d / L_d - inv_h (low part: mesh coordinates carried to ~2^-48)
    float len[3];        // L_d
    float* rho;          // charge mesh
    float2* shat;        // FFT of rho
    float2* fhat;        // 4 x nhalf: S G_opt, i k_x S G_opt, i k_y S G_opt, i k_z S G_opt
    float* field;        // 4 x nreal: their unnormalised inverse transforms
    float* gopt;         // nhalf: optimal influence function
    float alpha;         // Ewald splitting parameter (per-atom virial fields)
    float2* fhat6;       // 6 x nhalf: G_opt B_ab S (per-atom virial; NULL when not asked for)
    float* field6;       // 6 x nreal: their unnormalised inverse transforms
    // general cells: mesh points sum_d (s_d / N_d) a_d, an atom's mesh coordinates N_d (r H^-1)_d,
    // k = 2 pi H^-1 n; the three i k fields are the fractional gradients i 2 pi n_c S G_opt,
    // mapped to Cartesian components by H^-1 at the gather
    int tri;
    float nh_hi[9], nh_lo[9];   // N_d H^-1[c][d] (row-major [c][d]) as float pairs
    float hi[9];                // H^-1 (row-major)
    double hid[9];              // H^-1 in FP64 (influence function)
};

__device__ __forceinline__ int entry_index(int e) { return e & INDEX_MASK; }

// Cartesian vector of the image shift t (integers, -1..1 per lattice vector): t_x a + t_y b + t_z c
// (t_d L_d in an orthorhombic box, the same floating-point result as the general form there)
__device__ __forceinline__ void shift_vector(const Geom& g, float tx, float ty, float tz, float& sx, float& sy,
                                             float& sz) {
    if (g.tri) {
        sx = fmaf(tz, g.H[6], fmaf(ty, g.H[3], tx * g.H[0]));
        sy = fmaf(tz, g.H[7], fmaf(ty, g.H[4], tx * g.H[1]));
        sz = fmaf(tz, g.H[8], fmaf(ty, g.H[5], tx * g.H[2]));
    } else {
        sx = tx * g.L[0];
        sy = ty * g.L[1];
        sz = tz * g.L[2];
    }
}

// Fractional coordinates s = r H^-1 of a Cartesian position (general cells only)
__device__ __forceinline__ void frac_of(const Geom& g, float x, float y, float z, float s[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] = fmaf(z, g.Hi[6 + d], fmaf(y, g.Hi[3 + d], x * g.Hi[d]));
}

// Position wrapped into the cell and its cell indices.  Orthorhombic: per axis y = x - floor(x / L) L.
// General: the integer lattice translation f = floor(r H^-1) is subtracted, r' = r - f H, so a
// position already inside the cell is kept bit for bit.
__device__ __forceinline__ void wrap_and_cell(const Geom& g, const float* x, float w[3], int c[3]) {
    if (!g.tri) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float f = floorf(x[d] * g.invL[d]);
            float y = fmaf(-f, g.L[d], x[d]);
            if (y >= g.L[d]) y -= g.L[d];
            if (y < 0.f) y += g.L[d];
            if (y >= g.L[d]) y = 0.f;
            w[d] = y;
            int cc = (int)(y * g.invL[d] * (float)g.nc[d]);
            c[d] = cc < 0 ? 0 : (cc >= g.nc[d] ? g.nc[d] - 1 : cc);
        }
        return;
    }
    float s[3];
    frac_of(g, x[0], x[1], x[2], s);
    float f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) f[d] = floorf(s[d]);
#pragma unroll
    for (int d = 0; d < 3; ++d)
        w[d] = x[d] - fmaf(f[2], g.H[6 + d], fmaf(f[1], g.H[3 + d], f[0] * g.H[d]));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float sd = s[d] - f[d];
        int cc = (int)(sd * (float)g.nc[d]);
        c[d] = cc < 0 ? 0 : (cc >= g.nc[d] ? g.nc[d] - 1 : cc);
    }
}
__device__ __forceinline__ void entry_shift(int e, float& tx, float& ty, float& tz) {
    const unsigned code = (unsigned)e >> CODE_SHIFT;
    tx = (float)((int)(code & 3u) - 1);
    ty = (float)((int)((code >> 2) & 3u) - 1);
    tz = (float)((int)(code >> 4) - 1);
}

// ---- host-side launchers (defined in the .cu files) ---------------------------------

// gate (optional): the kernels do nothing while *gate == 0 (Verlet skin: a reused list)
void launch_bin(const float* pos, const int* types, int n, const Geom& g, float4* pos4, int* cell_of,
                int* cell_count, int* cell_start, int* cell_fill, int* slot_atoms, float4* spos4, int* sidx,
                Accum* acc, double2* zero_buf, int zero_count, cudaStream_t st, const int* gate = nullptr);
// Verlet skin: displacement test, then either the binning and the candidate lists (cutoff
// r_list + skin, [n][cap_s] entries, counts [n]) or the refreshed sorted positions of the kept
// list; force = no valid list.  rebuilds counts the rebuilds (device counter).
void launch_skin(const float* pos, const int* types, int n, const Geom& g, float skin, bool force, int cap_s,
                 float4* pos4, int* cell_of, int* cell_count, int* cell_start, int* cell_fill, int* slot_atoms,
                 float4* spos4, int* sidx, Accum* acc, double2* zero_buf, int zero_count, int* gate, int* skin_list,
                 int* skin_cnt, float4* sref4, float* xref, unsigned int* rebuilds, cudaStream_t st);
void launch_neighbors(const float4* spos4, const int* cell_start, int n, int n_species, const Geom& g,
                      int cap_list, int cap_ang, int* nbr_list, int* cnt_list, int* nbr_ang, int* cnt_ang,
                      Accum* acc, cudaStream_t st);
void launch_descriptor_forward(const float4* pos4, const int* nbr_list, const int* cnt_list,
                               const int* nbr_ang, const int* cnt_ang, int n, const Geom& g,
                               const float* params, const ParamLayout& lay, float* ang_coef,
                               float* du, float* dq, float* u_out, float* q_out, float* des_out,
                               const int* sidx, float4* fields, const float* gq, Accum* acc, cudaStream_t st,
                               float* dtc = nullptr);
size_t coop_forward_smem(const ParamLayout& lay, int cap_l, int cap_a);
// Launch caches are kept per device ordinal: a kernel's dynamic shared-memory limit
// (cudaFuncSetAttribute) and the occupancy and SM-count answers hold for one device only.
// Host threads may race on a slot only to repeat the same idempotent query.
constexpr int kMaxDevices = 64;
inline int device_slot() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) d = 0;
    return d;
}
// Raise `kernel`'s dynamic shared-memory limit on the current device to `bytes` (once per
// device and value; `cache` is a zero-initialised static [kMaxDevices] of the call site).
template <class K>
inline void ensure_smem_attr(K kernel, std::atomic<int>* cache, int bytes) {
    const int d = device_slot();
    if (cache[d].load(std::memory_order_relaxed) >= bytes) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cache[d].store(bytes, std::memory_order_relaxed);
}
// Resident blocks per SM of `kernel` at (threads, smem) on the current device, cached per
// device for the last shared-memory size asked (at least 1).
template <class K>
inline int cached_occupancy(K kernel, std::atomic<long long>* cache, int threads, size_t smem) {
    const int d = device_slot();
    // the slot holds ((smem, threads) key << 8) | blocks per SM
    const long long key = (long long)smem * 4096 + threads;
    long long v = cache[d].load(std::memory_order_relaxed);
    if (v > 0 && (v >> 8) == key) return (int)(v & 255);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (per_sm > 255) per_sm = 255;
    cache[d].store((key << 8) | per_sm, std::memory_order_relaxed);
    return per_sm;
}
int num_sms();   // SMs of the current device (persistent grids), queried once per device
void launch_nbr_desc_coop(const float4* spos4, const int* cell_start, const int* sidx, int n, const Geom& g,
                          const float* params, const ParamLayout& lay, int cap_l, int cap_a, int* nbr_list,
                          int* cnt_list, int* nbr_ang, int* cnt_ang, float* ang_coef, float* du, float* dq,
                          float* u, float* q, float* des_out, const EwaldTab& tab, bool do_phase, float4* fields,
                          const float* gq, Accum* acc, cudaStream_t st, float* dtc = nullptr,
                          const int* skin_list = nullptr, const int* skin_cnt = nullptr, int cap_s = 0);
void launch_desc_bwd_coop(const float4* spos4, const int* nbr_list, const int* cnt_list, const int* nbr_ang,
                          const int* cnt_ang, int n, const Geom& g, const float* params, const ParamLayout& lay,
                          const float* ang_coef, const float* du, const float* dq, const float* q_raw,
                          const FieldIn& fin, const Accum* acc_in, bool want_bec, float* acc12, Accum* acc,
                          cudaStream_t st, float* avir = nullptr);
void launch_ewald_phases(const float4* pos4, int n, EwaldTab tab, cudaStream_t st);
void launch_ewald_sk(const float* q_raw, const Accum* acc, int n, float q_target, EwaldTab tab, cudaStream_t st);
void launch_ewald_sk_fused(const float* q_raw, Accum* acc, int n, float q_target, EwaldTab tab,
                           unsigned int* group_done, cudaStream_t st);
void launch_ewald_sk_finalize(EwaldTab tab, Accum* acc, cudaStream_t st);
void launch_field(const float4* pos4, const float* pos_in, const float* q_raw, const int* nbr_list,
                  const int* cnt_list, int n, int n_species, const Geom& g, ElecConst ec, float q_target,
                  float sqrt_eps, bool ewald, EwaldTab tab, const float* pppm_field, float* phi,
                  float* acc12, float* charges_out, Accum* acc, cudaStream_t st, const int* sidx = nullptr);
void launch_descriptor_backward(const float4* pos4, const int* nbr_list, const int* cnt_list,
                                const int* nbr_ang, const int* cnt_ang, int n, const Geom& g,
                                const float* params, const ParamLayout& lay, const float* ang_coef,
                                const float* du, const float* dq, const float* q_raw, const FieldIn& fin,
                                const Accum* acc_in, bool want_bec, float* acc12, Accum* acc, cudaStream_t st);
void launch_real(const float4* spos4, const float* q_raw, const int* nbr_list, const int* cnt_list, int n,
                 int n_species, const Geom& g, float alpha, float q_target, const Accum* acc_in, float4* rfield,
                 Accum* acc, cudaStream_t st, float* avir = nullptr);
void launch_field_k(int n, const EwaldTab& tab, float4* kfield, Accum* acc, cudaStream_t st, float* avir = nullptr);
// Network on the tensor cores for n atoms (precision PREC_BF16 or PREC_TF32): scaled
// descriptors dtc [n][32] (sorted order) -> u, q, du / dq (element k, v at k d_sa + v d_sv),
// FP64 sums of u and q into acc.
size_t mlp_tc_smem(int precision, int n_species);
void launch_mlp_tc(int precision, const float* dtc, const float4* spos4, int n, const float* params,
                   const ParamLayout& lay, float* du, float* dq, int d_sa, int d_sv, float* u, float* q, Accum* acc,
                   int num_sms, cudaStream_t st);
// Velocity-Verlet halves (md.cu); masses in amu per species.
void launch_vv_kick_drift(int n, float* pos, float* vel, const float* f, const int* types, const float* masses,
                          int n_species, float dt, cudaStream_t st);
void launch_vv_kick_energy(int n, float* vel, const float* f, const int* types, const float* masses, int n_species,
                           float dt, bool kick, const double* scalars, double* energies, int* step, double* ke_acc,
                           unsigned int* done, cudaStream_t st);
void launch_pppm_gopt(const PppmTab& pm, double alpha, double vol, cudaStream_t st);
int launch_pppm(const float4* spos4, const float* q_raw, int n, const Accum* acc_in, float q_target, PppmTab pm,
                float alpha, int r2c, int c2r, float4* kfield, Accum* acc, cudaStream_t st, int c2r6 = 0,
                float* avir = nullptr);
void launch_finalize(const float* acc12, int n, const int* sidx, const float* pos_in, const float* q_raw,
                     float q_target, float seps, ElecConst ec, const float4* kfield, const float4* rfield,
                     float* forces, float* bec, float* charges, float* potential, const float* u, float* site_energy,
                     Accum* acc, double* scalars, unsigned int* status_host, unsigned int* done, cudaStream_t st,
                     float* grad = nullptr, const float* gp = nullptr, const float* avir = nullptr,
                     float* atom_virial = nullptr);
void launch_finalize_atoms(const float* acc12, int n, float* forces, float* bec, const float* phi,
                           float* potential, cudaStream_t st);
void launch_finalize_scalars(const Accum* acc, int n, float sqrt_eps, double* scalars, cudaStream_t st);

}  // namespace qnep
