// Internal declarations of the batched force call: many structures of uneven size,
// each evaluated under many candidate parameter vectors (the shape of a separable
// natural-evolution-strategy fitness evaluation, Sec. II.E).
//
// Work decomposition.  The unit of work ("item") is one structure under a group of
// CG = 32 candidates.  One thread block owns an item from start to end, so every
// per-structure synchronisation point of the force call (total charge, S(k), mean
// potential) is a block barrier, and a persistent grid takes items from a queue
// ordered largest first.  Inside an item lane c of every warp evaluates candidate
// c of the group: geometry, basis functions, harmonics and Ewald phases do not
// depend on the candidate, so they are computed once per pair or atom, staged in
// shared memory and read by all 32 lanes as broadcasts, while each lane reads its
// own candidate's parameters from a candidate-minor copy ([parameter][candidate]),
// conflict-free.  Per-candidate results are laid out [atom][..][candidate] so the
// lanes' loads, stores and float4 atomics are coalesced.
#pragma once

#include "qnep_internal.cuh"

namespace qnep {

constexpr int CG = 32;               // candidates per item (one per lane)
constexpr int BATCH_MAX_NPH = 94;    // phase factors per atom (n_max <= 16 per axis: edges up to
                                     // ~45 A at k_max = 2.23 1/A; bounds the field pass's shared memory)
constexpr int BATCH_MAX_CELLS = 512; // cell grid per structure (8 per axis at most)
constexpr int BATCH_GR = 20, BATCH_GA = 48;   // floats per radial / angular pair row
// Row stride (float2) of the atoms' phase factors for phase rows of up to nph_max entries: even,
// so every row starts on a 16-byte boundary (bulk copies), and = 2 mod 16, so the rows of
// consecutive atoms start in different shared-memory banks once a tile of them is copied.
constexpr int batch_phase_stride(int nph_max) { return nph_max + (18 - nph_max % 16) % 16; }

// Tensor-core form of the angular contraction A_{n,lm} = sum_{s,k} c^A[t_i][s][n][k] B^A[s][k][lm]
// (BF16x3: operands split into BF16 hi + lo, three products, FP32 accumulation).  The pre-pass
// writes B^A of every atom as its operand image: 24 rows (lm) x 48 K ((s, k) = 9 s + k, zero
// past 9 S) of BF16 in the canonical K-major layout without swizzle, the hi plane then the lo
// plane, so a tile of atoms is a concatenation of bulk copies.
constexpr int BIMG_K = 48;                       // (species, k) padded to a multiple of 16
constexpr int BIMG_ROWB = BIMG_K * 2;            // bytes per operand row
constexpr int BIMG_PLANE = NLM * BIMG_ROWB;      // 2304 bytes: one atom's 24 rows
constexpr int BIMG_BYTES = 2 * BIMG_PLANE;       // hi | lo
enum { BATCH_CONTRACT_FP32 = 0, BATCH_CONTRACT_BF16X3 = 1, BATCH_CONTRACT_BF16 = 2 };
inline bool batch_contract_tc(int c) { return c == BATCH_CONTRACT_BF16X3 || c == BATCH_CONTRACT_BF16; }

// One structure of the batch (host-built).
struct BatchStruct {
    int atom_off;    // first atom in the concatenated inputs
    int n;           // atoms
    int ktab;        // its k-space table
    int cell_off;    // offset of its cell_start array (ncells + 1 entries)
    Geom g;          // box and cell grid
};

// Half-space k-set of one box shape (see KSet): chunk h of the table is global chunk
// chunk_off + h, whose 8 wave vectors are kvec[8 (chunk_off + h) + t].
struct BatchKTab {
    int n1max, n2max, n3max;
    int nph;         // phase factors per atom: X[0..n1max] | Y[-n2max..n2max] | Z[-n3max..n3max+7]
    int yoff, zoff;
    int nchunk;
    int chunk_off;
    int nkr;         // wave vectors of the half space (the chunks' non-padding entries)
    int kreal_off;   // their padded indices: kreal[kreal_off .. kreal_off + nkr)
    float invl_hi[3], invl_lo[3];
};

// The phase-factor data of a general cell (restricted form: a along x, b in the xy plane), read by
// the pre-pass only (kept apart from BatchKTab, which the item kernel's phases take by value):
// phases of the fractional coordinates s = r H^-1; k = 2 pi H^-1 n in the table then has x and
// y components that depend on (n1, n2) only, as H^-1 is lower triangular like H.
struct BatchKTri {
    int tri;                    // 0: orthorhombic (BatchKTab.invl_* are used)
    float hi_hi[9], hi_lo[9];   // H^-1 (row-major) as float pairs
};

// Per-slot scratch (one slot per resident block), in floats, for nmax atoms.
struct BatchScratch {
    float* A;        // [nmax][NANG][CG] angular expansion coefficients A_{n,lm}
    float* duq;      // [nmax][2 NDES][CG] dU/dD (scaled) then dq/dD (scaled)
    float2* uq;      // [nmax][CG] (U_i, q_i) raw network outputs
    float* qc;       // [nmax][CG] corrected charges q^c
    float4* fk;      // [CG][nmax] (phi^k, E^k) k-space potential and field per unit charge
    float4* fr;      // [nmax][CG] (phi^r, F^r) real space
    float4* fsum;    // [nmax][CG] force accumulators (xyz, pad)
    float2* sk;      // [nk_max][CG] 4 k_e G(k) S(k) (FP32)
    float2* skp;     // [n_flush][nk_max][CG] FP32 partial structure factors (512-atom blocks)
    double* vir;     // [8][9][CG] per-warp FP64 virial sums of the item (8 warps; NULL without a virial)
    float4* zsum;    // [nmax][3][CG] BEC accumulators (Z_xx..Z_yx | Z_yy..Z_zy | Z_zz, pad; NULL without BEC)
    size_t stride_A, stride_duq, stride_n, stride_k, stride_p;   // per-slot strides (elements)
};

struct BatchArgs {
    // pre-pass outputs (per structure, candidate independent)
    const float4* spos4;     // [N] cell-sorted wrapped positions (species in w)
    const int* sidx;         // [N] input index (within the structure) of each sorted atom
    const int* order;        // [N] sorted atoms grouped by species
    const int* spec_off;     // [n_struct][MAX_SPECIES + 1] species ranges of `order`
    const int* nbr_list;     // [N][cap_l] grouped by neighbour species
    const int* cnt_list;     // structure s: [S][n_s] at cnt_list + atom_off * S
    const int* nbr_ang;
    const int* cnt_ang;
    int cap_l, cap_a;
    const float2* phase;     // [N][nph_stride]
    int nph_stride;
    const float* geo_rad;    // [N][cap_l][20] radial pair rows (see batch.cu)
    const float* geo_ang;    // [N][cap_a][48] angular pair rows
    const float* bsum;       // [N][bstride] basis sums B^R | B^A
    int bstride;
    const unsigned char* bimg;   // [N][BIMG_BYTES] B^A operand images (tensor-core form), or NULL
    // tables
    const BatchStruct* st;
    const BatchKTab* kt;
    const int4* chunk;       // [n_chunks] (n1, n2, first n3, entries of the chunk that are not padding)
    const int* kreal;        // padded index (8 h + t) of every wave vector, per k-table
    const float4* kvec;      // [8 n_chunks] (kx, ky, kz, 4 k_e G) (G = 0 on padding)
    // parameters by candidate group: [group][p][CG] (lane-minor)
    const float* pt;
    ParamLayout lay;
    int n_cand;
    // work queue
    const int2* items;       // (structure, group), largest first
    int n_items;
    unsigned int* work;
    BatchScratch sc;
    // electrostatics
    int mode;
    float alpha;
    float q_total;
    int contract;            // BATCH_CONTRACT_*: the tensor-core form's products (3, or 1 for BF16)
    // outputs
    double* energy;          // [n_cand][n_struct]
    float* forces;           // [n_cand][N_total][3] or NULL
    float* charges;          // [n_cand][N_total] or NULL
    double* virial;          // [n_cand][n_struct][9] or NULL (W = -dU/d eps, eV)
    float* bec;              // [n_cand][N_total][9] or NULL (Z_i,ab = dP_a/dr_ib, Eq. bec_2; needs sc.zsum)
    double* total_charge;    // [n_cand][n_struct] or NULL (sum of q~ before the correction)
    double* polarization;    // [n_cand][n_struct][3] or NULL (P = sum q~^c_i r_i, positions as given)
    const float* pos_in;     // [N_total][3] the call's positions (for the polarization)
    const float* rot;        // [n_struct][12]: R into the restricted cell form, then a flag (1: rotated)
    int n_struct;
    int n_total;
    int inv_cap;             // ints of shared memory for the outputs' inverse permutation (set at launch)
    unsigned int* status;    // bit 0: neighbour overflow
};

void launch_batch_prep(const float* pos, const int* types, int n_struct, int nmax, int n_species,
                       const BatchStruct* st, const BatchKTab* kt, const BatchKTri* ktri, int* cell_start, float4* spos4, int* sidx,
                       int* order, int* spec_off, int cap_l, int cap_a, int* nbr_list, int* cnt_list, int* nbr_ang,
                       int* cnt_ang, float2* phase, int nph_stride, float* geo_rad, float* geo_ang, float* bsum,
                       int bstride, unsigned char* bimg, float alpha, const float* rot, unsigned int* status,
                       cudaStream_t st_);
// Floats per atom of the basis sums: B^R padded to MAX_SPECIES species, then B^A of n_species.
inline int batch_bstride(int n_species) { return MAX_SPECIES * KR + n_species * KA * NLM; }
// Dynamic shared memory of the item kernel and its resident blocks per SM (0: does not fit).
// contract: BATCH_CONTRACT_FP32 (FP32 FMAs, 4 or 8 warps) or BATCH_CONTRACT_BF16X3 (tensor cores,
// 8 warps only)
size_t batch_item_smem(int warps, int nph_max, int contract);
int batch_item_blocks_per_sm(int warps, int nph_max, int contract, bool virial, bool bec);
void launch_batch_items(const BatchArgs& a, int warps, int nph_max, int contract, int grid, cudaStream_t st_);

}  // namespace qnep
