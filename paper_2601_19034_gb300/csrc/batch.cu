// Batched force call: structures of uneven size under groups of 32 candidate
// parameter vectors (one candidate per lane), one item per thread block.
//
// Pre-pass (candidate independent, one block per structure):
//   k_batch_sort   wrap, bin into cells, stable cell order, species order
//   k_batch_lists  neighbour lists (grouped by neighbour species); per entry the pair
//                  geometry rows (basis values and derivatives, harmonics, unit vector,
//                  real-space kernel); per atom the basis sums
//                  B^R[t_j][k] = sum_j f_k(r_ij),  B^A[t_j][k][lm] = sum_j f_k(r_ij) Y_lm(u_ij);
//                  the Ewald phase-factor rows of every atom
// Item kernel (persistent, items taken largest first), per (structure, group):
//   1 forward    per species block, lane = candidate: D^R_n = sum c^R[t_i][t_j][n][k] B^R,
//                A_{n,lm} = sum c^A[t_i][t_j][n][k] B^A (Sec. II.A), descriptor; then the
//                network U_i, q_i and dU/dD, dq/dD (Eq. U_i, Sec. II.B), weights staged
//   2 charges    total-charge correction (block sum, FP64)
//   3 S(k)       lanes over 32 wave vectors, FP32 terms over 512-atom blocks summed in
//                FP64 (tensor-core form: sk_tc); U^k per candidate (FP64)
//   4 fields     lanes over atoms: phi^k_i and the k-space field (Sec. II.C);
//                lanes over candidates: real-space phi^r_i and F^r_i
//   5 backward   per species block: lambda = dU/dD + (phi_i - mean phi) dq/dD; radial
//                and angular partial forces per pair (Sec. II.C), float4 atomics; on request
//                the virial, and a second pass with kappa = sqrt(eps_inf) dq/dD for the BEC
//                terms of Eq. bec_2
//   6 outputs    forces, corrected charges, BEC (input order), energy, virial, uncorrected
//                total charge and polarization per candidate
// General cells (restricted form, a along x and b in the xy plane) change the pre-pass only:
// wrapping by lattice translations, cells along the fractional axes, phases of the fractional
// coordinates; the item kernel reads Cartesian wave vectors from the tables either way.
#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "batch_internal.cuh"
#include "desc_math.cuh"
#include "nbr_common.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace qnep {

namespace {

constexpr int PREP_THREADS = 256;

// Candidate-independent pair geometry, written once per structure by the pre-pass:
//   radial row  (GR floats per list entry):  f'_k (9) | u (3) | j if r < r_c^R else -1 |
//                B(r) | B'(r) u (3) | j if r < r_c (real space) else -1 | r | pad
//   angular row (GA floats per angular entry): f_k (9) | f'_k (9) | u (3) | 1/r | j | pad | Y_lm (24)
//   basis sums  (per atom): B^R[t][k] (padded to MAX_SPECIES species) | B^A[t][k][lm]
// with B(r) = k_e erfc(alpha r) / r.  Rows are copied into shared memory (float4) by the item kernel.
constexpr int GR = 20, GR_DF = 0, GR_U = 9, GR_JD = 12, GR_B = 13, GR_BU = 14, GR_JR = 17, GR_R = 18;
static_assert(GR_JD == 12 && GR_B == 13 && GR_BU == 14 && GR_JR == 17 && GR_R == 18,
              "float4 row reads assume this layout");
constexpr int GA = 48, GA_F = 0, GA_DF = 9, GA_U = 18, GA_IR = 21, GA_J = 22, GA_Y = 24;
static_assert(GA_DF == 9 && GA_U == 18 && GA_Y == 24, "float4 row reads assume this layout");
constexpr int TAB_P = KA + NLM;                // pre-pass staging row: f_k, Y_lm
// per-warp shared memory of the item kernel: two row buffers (double-buffered bulk copies of
// 32 pair rows, or of one atom's basis sums) and the cumulative species counts
constexpr int WBUF = 32 * GA;                  // floats per buffer
constexpr int WCUM = 2 * WBUF;                 // ints
constexpr int WARP_FLOATS = WCUM + 16;
// the real-space phase's per-warp buffers: two pieces of 32 radial pair rows (double-buffered
// bulk copies), then the species counts
constexpr int RS_BUF = 32 * GR;
constexpr int RS_CUM = 2 * RS_BUF;
constexpr int RS_WARP = RS_CUM + 16;
static_assert(RS_CUM <= WCUM, "the real-space buffers fit a warp's row buffers");
// radial entries per piece of the backward (a row buffer holds WBUF / GR of them; the angular
// pieces stay at 32 rows)
constexpr int RPIECE = 64;
static_assert(RPIECE * GR <= WBUF, "a radial piece fits a row buffer");
constexpr int BS_MAX = MAX_SPECIES * KR + MAX_SPECIES * KA * NLM;   // basis-sum floats per atom
static_assert(BS_MAX <= WBUF, "basis sums fit a row buffer");
constexpr int PR_R = 0;                                  // c^R[t_i] staged [S][NR][KR][CG]
constexpr int PR_A = MAX_SPECIES * NR * KR * CG;         // c^A[t_i] staged [S][NA][KA][CG]
constexpr int PR_S = PR_A + MAX_SPECIES * NA * KA * CG;  // descriptor scaler [NDES][CG]
constexpr int PARAM_FLOATS = PR_S + NDES * CG;
constexpr int QT = 64;                         // atoms per charge tile of the S(k) phase
constexpr int FLUSH_TILES = 8;                 // FP32 partial sums cover 512 atoms
constexpr int KW = 64;                         // wave vectors per staged window of the field pass
constexpr int NSUMS = 6;                       // per-candidate FP64 sums
constexpr int WIN_F2 = KW * CG + 2 * KW + KW / 4;   // float2 per field window: C(k) | k | chunks

static_assert(WBUF % 4 == 0 && WARP_FLOATS % 4 == 0 && PARAM_FLOATS % 4 == 0, "float4 alignment");

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 batch_phase(const float4& p, int e, const BatchKTab& kt, const BatchKTri& kr) {
    if (kr.tri) {
        if (e < kt.yoff) return phase_factor_frac(p, e, 0, kr.hi_hi, kr.hi_lo);
        if (e < kt.zoff) return phase_factor_frac(p, e - kt.yoff - kt.n2max, 1, kr.hi_hi, kr.hi_lo);
        return phase_factor_frac(p, e - kt.zoff - kt.n3max, 2, kr.hi_hi, kr.hi_lo);
    }
    if (e < kt.yoff) return phase_factor(p.x, e, kt.invl_hi[0], kt.invl_lo[0]);
    if (e < kt.zoff) return phase_factor(p.y, e - kt.yoff - kt.n2max, kt.invl_hi[1], kt.invl_lo[1]);
    return phase_factor(p.z, e - kt.zoff - kt.n3max, kt.invl_hi[2], kt.invl_lo[2]);
}

// Species of input atom i; an out-of-range type sets status bit 2 and counts as species 0.
__device__ __forceinline__ int species_of(const int* __restrict__ types, int i, int n_species,
                                         unsigned int* status) {
    const int t = types[i];
    if (t >= 0 && t < n_species) return t;
    if (status) atomicOr(status, 4u);
    return 0;
}

__device__ __forceinline__ float wrap_coord(float x, float L, float invL) {
    float f = floorf(x * invL);
    float y = fmaf(-f, L, x);
    if (y >= L) y -= L;
    if (y < 0.f) y += L;
    if (y >= L) y = 0.f;
    return y;
}

// ---------------------------------------------------------------------------------
// pre-pass 1: cells, stable cell order, species order
// Position of input atom i of a structure as the pre-pass uses it: rotated by R (rows e1, e2, e3)
// when the structure's general cell was rotated into the restricted form (rot: [S][12], R then a
// flag), as given otherwise.
__device__ __forceinline__ void prep_position(const float* __restrict__ pos, const float* __restrict__ rot, int s,
                                              size_t i, float x[3]) {
    const float p0 = pos[3 * i], p1 = pos[3 * i + 1], p2 = pos[3 * i + 2];
    if (rot && rot[12 * s + 9] != 0.f) {
        const float* R = rot + 12 * s;
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a] = fmaf(R[3 * a + 2], p2, fmaf(R[3 * a + 1], p1, R[3 * a] * p0));
        return;
    }
    x[0] = p0;
    x[1] = p1;
    x[2] = p2;
}

// Back to the input frame: v = R^T v' and Z = R^T Z' R (row-major 3 x 3)
__device__ __forceinline__ float4 rot_back_vec(const float* __restrict__ R, float4 v) {
    return make_float4(fmaf(R[6], v.z, fmaf(R[3], v.y, R[0] * v.x)), fmaf(R[7], v.z, fmaf(R[4], v.y, R[1] * v.x)),
                       fmaf(R[8], v.z, fmaf(R[5], v.y, R[2] * v.x)), v.w);
}
__device__ __forceinline__ void rot_back_tensor(const float* __restrict__ R, float z[9]) {
    float t[9];
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int d = 0; d < 3; ++d) t[3 * x + d] = fmaf(R[6 + x], z[6 + d], fmaf(R[3 + x], z[3 + d], R[x] * z[d]));
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) z[3 * x + y] = fmaf(t[3 * x + 2], R[6 + y], fmaf(t[3 * x + 1], R[3 + y], t[3 * x] * R[y]));
}

__global__ void __launch_bounds__(PREP_THREADS) k_batch_sort(const float* __restrict__ pos,
                                                             const int* __restrict__ types, int nmax, int n_species,
                                                             const BatchStruct* __restrict__ sts,
                                                             int* __restrict__ cell_start_all,
                                                             float4* __restrict__ spos4, int* __restrict__ sidx,
                                                             int* __restrict__ order, int* __restrict__ spec_off,
                                                             const float* __restrict__ rot,
                                                             unsigned int* __restrict__ status) {
    extern __shared__ int psm[];
    const BatchStruct bs = sts[blockIdx.x];
    const int n = bs.n, off = bs.atom_off;
    const Geom g = bs.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    int* cell_of = psm;                          // [nmax]
    int* ccnt = cell_of + nmax;                  // [BATCH_MAX_CELLS + 1]
    int* scnt = ccnt + BATCH_MAX_CELLS + 1;      // [MAX_SPECIES + 1]
    for (int i = threadIdx.x; i <= g.ncells; i += blockDim.x) ccnt[i] = 0;
    if (threadIdx.x <= MAX_SPECIES) scnt[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int cc[3];
        if (g.tri) {   // cells along the fractional axes; the position wrapped by lattice translations
            float x[3];
            prep_position(pos, rot, blockIdx.x, (size_t)(off + i), x);
            float w[3];
            wrap_and_cell(g, x, w, cc);
        } else {
            for (int d = 0; d < 3; ++d) {
                float y = wrap_coord(pos[3 * (size_t)(off + i) + d], g.L[d], g.invL[d]);
                int c = (int)(y * g.invL[d] * (float)g.nc[d]);
                cc[d] = c < 0 ? 0 : (c >= g.nc[d] ? g.nc[d] - 1 : c);
            }
        }
        const int c = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
        cell_of[i] = c;
        atomicAdd(&ccnt[c], 1);
        atomicAdd(&scnt[species_of(types, off + i, n_species, status)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < g.ncells; ++c) {
            int v = ccnt[c];
            ccnt[c] = acc;
            acc += v;
        }
        ccnt[g.ncells] = acc;
        acc = 0;
        for (int t = 0; t < n_species; ++t) {
            int v = scnt[t];
            scnt[t] = acc;
            acc += v;
        }
        scnt[n_species] = acc;
    }
    __syncthreads();
    int* cs = cell_start_all + bs.cell_off;
    for (int i = threadIdx.x; i <= g.ncells; i += blockDim.x) cs[i] = ccnt[i];
    if (threadIdx.x <= n_species) spec_off[blockIdx.x * (MAX_SPECIES + 1) + threadIdx.x] = scnt[threadIdx.x];
    // stable placement by cell (ascending input index inside a cell), one warp per cell
    for (int c = warp; c < g.ncells; c += nw) {
        int base = ccnt[c];
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const bool in = i < n && cell_of[i] == c;
            const unsigned mk = __ballot_sync(0xffffffffu, in);
            if (in) {
                const int slot = base + __popc(mk & below);
                float w[3];
                if (g.tri) {
                    float x[3];
                    prep_position(pos, rot, blockIdx.x, (size_t)(off + i), x);
                    int cd[3];
                    wrap_and_cell(g, x, w, cd);
                } else {
                    for (int d = 0; d < 3; ++d) w[d] = wrap_coord(pos[3 * (size_t)(off + i) + d], g.L[d], g.invL[d]);
                }
                spos4[off + slot] = make_float4(w[0], w[1], w[2],
                                                __int_as_float(species_of(types, off + i, n_species, nullptr)));
                sidx[off + slot] = i;
            }
            base += __popc(mk);
        }
    }
    __syncthreads();
    // species order over the sorted atoms (stable), one warp per species
    for (int t = warp; t < n_species; t += nw) {
        int base = scnt[t];
        for (int m0 = 0; m0 < n; m0 += 32) {
            const int m = m0 + lane;
            const bool in = m < n && species_of(types, off + sidx[off + m], n_species, nullptr) == t;
            const unsigned mk = __ballot_sync(0xffffffffu, in);
            if (in) order[off + base + __popc(mk & below)] = m;
            base += __popc(mk);
        }
    }
}

// Candidate-independent geometry of sorted atom m (whole warp): pair rows and basis sums.
__device__ __forceinline__ void geometry_atom(const float4* __restrict__ sp, const Geom& g, float alpha, int m, int n,
                                              int S, const int* __restrict__ lst, const int* __restrict__ cl,
                                              const int* __restrict__ lsa, const int* __restrict__ ca,
                                              float* __restrict__ grad_rows, float* __restrict__ gang_rows,
                                              float* __restrict__ bs_out, unsigned char* __restrict__ bimg,
                                              float* __restrict__ tab, int* __restrict__ cum) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        int tl = 0, ta = 0;
        for (int s = 0; s < S; ++s) {
            cum[s] = tl;
            cum[8 + s] = ta;
            tl += cl[(size_t)s * n + m];
            ta += ca[(size_t)s * n + m];
        }
        cum[S] = tl;
        cum[8 + S] = ta;
    }
    __syncwarp();
    const int tot_l = cum[S], tot_a = cum[8 + S];
    const float4 pk = sp[m];
    const float rcr2 = g.rc_radial * g.rc_radial, rcs2 = g.rc_real * g.rc_real;
    // radial rows and B^R: lanes over entries, then over (t_j, k)
    float br0 = 0.f, br1 = 0.f;
    for (int base = 0; base < tot_l; base += 32) {
        const int e = base + lane;
        float f[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) f[k] = 0.f;
        if (e < tot_l) {
            const int ent = lst[e];
            float vx, vy, vz;
            entry_vector(sp, ent, pk, g, vx, vy, vz);
            const float r2 = vx * vx + vy * vy + vz * vz, r = sqrtf(r2), ir = 1.f / r;
            float row[GR];
#pragma unroll
            for (int q = 0; q < GR; ++q) row[q] = 0.f;
            row[GR_U] = vx * ir;
            row[GR_U + 1] = vy * ir;
            row[GR_U + 2] = vz * ir;
            row[GR_JD] = __int_as_float(-1);
            row[GR_JR] = __int_as_float(-1);
            row[GR_R] = r;
            const int j = entry_index(ent);
            if (r2 < rcr2) {
                float df[KR];
                basis_d<KR>(r, g.rc_radial, f, df);
#pragma unroll
                for (int k = 0; k < KR; ++k) row[GR_DF + k] = df[k];
                row[GR_JD] = __int_as_float(j);
            }
            if (r2 < rcs2) {
                const float ar = alpha * r, ec = erfcf(ar);
                const float B = KE * ec * ir;
                // dB/dr = -k_e (erfc(a r) / r + 2 a / sqrt(pi) exp(-a^2 r^2)) / r
                const float dB = -KE * (ec * ir + 1.12837916709551257f * alpha * expf(-ar * ar)) * ir;
                row[GR_B] = B;
                row[GR_BU] = dB * row[GR_U];
                row[GR_BU + 1] = dB * row[GR_U + 1];
                row[GR_BU + 2] = dB * row[GR_U + 2];
                row[GR_JR] = __int_as_float(j);
            }
            float4* o = reinterpret_cast<float4*>(grad_rows + (size_t)e * GR);
#pragma unroll
            for (int q = 0; q < GR / 4; ++q) o[q] = make_float4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
        }
#pragma unroll
        for (int k = 0; k < KR; ++k) tab[lane * KR + k] = f[k];
        __syncwarp();
        const int cntc = min(32, tot_l - base);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int idx = lane + 32 * h;
            if (idx < S * KR) {
                const int tj = idx / KR, k = idx - tj * KR;
                const int lo = max(cum[tj] - base, 0), hi = min(cum[tj + 1] - base, cntc);
                float x = 0.f;
                for (int r = lo; r < hi; ++r) x += tab[r * KR + k];
                if (h == 0) br0 += x;
                else br1 += x;
            }
        }
        __syncwarp();
    }
    if (lane < MAX_SPECIES * KR) bs_out[lane] = lane < S * KR ? br0 : 0.f;
    if (lane + 32 < MAX_SPECIES * KR) bs_out[lane + 32] = lane + 32 < S * KR ? br1 : 0.f;
    // angular rows and B^A: lanes over entries, then lane lm accumulates per neighbour species
    float ba[MAX_SPECIES][KA];
#pragma unroll
    for (int t = 0; t < MAX_SPECIES; ++t)
#pragma unroll
        for (int k = 0; k < KA; ++k) ba[t][k] = 0.f;
    for (int base = 0; base < tot_a; base += 32) {
        const int e = base + lane;
        if (e < tot_a) {
            const int ent = lsa[e];
            float vx, vy, vz;
            entry_vector(sp, ent, pk, g, vx, vy, vz);
            const float r = sqrtf(vx * vx + vy * vy + vz * vz), ir = 1.f / r;
            float row[GA];
#pragma unroll
            for (int q = 0; q < GA; ++q) row[q] = 0.f;
            float f[KA], df[KA], Y[NLM];
            basis_d<KA>(r, g.rc_angular, f, df);
            const float ux = vx * ir, uy = vy * ir, uz = vz * ir;
            harmonics(ux, uy, uz, Y);
#pragma unroll
            for (int k = 0; k < KA; ++k) {
                row[GA_F + k] = f[k];
                row[GA_DF + k] = df[k];
                tab[lane * TAB_P + k] = f[k];
            }
            row[GA_U] = ux;
            row[GA_U + 1] = uy;
            row[GA_U + 2] = uz;
            row[GA_IR] = ir;
            row[GA_J] = __int_as_float(entry_index(ent));
#pragma unroll
            for (int q = 0; q < NLM; ++q) {
                row[GA_Y + q] = Y[q];
                tab[lane * TAB_P + KA + q] = Y[q];
            }
            float4* o = reinterpret_cast<float4*>(gang_rows + (size_t)e * GA);
#pragma unroll
            for (int q = 0; q < GA / 4; ++q) o[q] = make_float4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
        }
        __syncwarp();
        const int cntc = min(32, tot_a - base);
        if (lane < NLM) {
#pragma unroll
            for (int t = 0; t < MAX_SPECIES; ++t) {
                if (t < S) {
                    const int lo = max(cum[8 + t] - base, 0), hi = min(cum[8 + t + 1] - base, cntc);
                    for (int r = lo; r < hi; ++r) {
                        const float* row = tab + r * TAB_P;
                        const float y = row[KA + lane];
#pragma unroll
                        for (int k = 0; k < KA; ++k) ba[t][k] = fmaf(row[k], y, ba[t][k]);
                    }
                }
            }
        }
        __syncwarp();
    }
    if (lane < NLM) {
        // FP32 B^A for the FP32 contraction; the tensor-core form reads only the operand image
        if (!bimg) {
#pragma unroll
            for (int t = 0; t < MAX_SPECIES; ++t)
                if (t < S)
#pragma unroll
                    for (int k = 0; k < KA; ++k) bs_out[MAX_SPECIES * KR + (t * KA + k) * NLM + lane] = ba[t][k];
        }
        if (bimg) {
            // operand image, row lm = lane: K index 9 t + k, BF16 hi and lo (x - hi) planes
            static_assert(MAX_SPECIES * KA <= BIMG_K, "the (species, k) index fits the padded K");
#pragma unroll
            for (int kc = 0; kc < BIMG_K / 8; ++kc) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    float x[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int kidx = 8 * kc + 2 * h + e;
                        const int t = kidx < MAX_SPECIES * KA ? kidx / KA : 0, k = kidx % KA;
                        x[e] = kidx < S * KA ? ba[t][k] : 0.f;
                    }
                    const __nv_bfloat162 hi = __floats2bfloat162_rn(x[0], x[1]);
                    const __nv_bfloat162 lo =
                        __floats2bfloat162_rn(x[0] - __bfloat162float(hi.x), x[1] - __bfloat162float(hi.y));
                    hw[h] = *reinterpret_cast<const uint32_t*>(&hi);
                    lw[h] = *reinterpret_cast<const uint32_t*>(&lo);
                }
                const int o = ((lane >> 3) * (BIMG_K / 8) + kc) * 128 + (lane & 7) * 16;
                *reinterpret_cast<uint4*>(bimg + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(bimg + BIMG_PLANE + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        }
    }
    __syncwarp();
}

// pre-pass 2: neighbour lists, pair geometry, basis sums and phase rows
__global__ void __launch_bounds__(PREP_THREADS) k_batch_lists(
    int n_species, const BatchStruct* __restrict__ sts, const BatchKTab* __restrict__ kts,
    const BatchKTri* __restrict__ ktris, const int* __restrict__ cell_start_all, const float4* __restrict__ spos4, int cap_l, int cap_a,
    int* __restrict__ nbr_list, int* __restrict__ cnt_list, int* __restrict__ nbr_ang, int* __restrict__ cnt_ang,
    float2* __restrict__ phase, int nph_stride, float* __restrict__ geo_rad, float* __restrict__ geo_ang,
    float* __restrict__ bsum, int bstride, unsigned char* __restrict__ bimg, float alpha,
    unsigned int* __restrict__ status) {
    extern __shared__ int psm[];
    const BatchStruct bs = sts[blockIdx.x];
    const int n = bs.n, off = bs.atom_off;
    const Geom g = bs.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per_warp = 2 * cap_l + 2 * cap_a + 32 * TAB_P + 16;
    int* sl = psm + warp * per_warp;
    int* slt = sl + cap_l;
    int* sa = slt + cap_l;
    int* sat = sa + cap_a;
    float* tab = reinterpret_cast<float*>(sat + cap_a);
    int* cum = reinterpret_cast<int*>(tab + 32 * TAB_P);
    const float4* sp = spos4 + off;
    const int* cs = cell_start_all + bs.cell_off;
    // atoms of the structure are split over gridDim.y blocks (warp stride nw * gridDim.y)
    const int wstride = nw * gridDim.y, wfirst = blockIdx.y * nw + warp;
    int* lst_s = nbr_list + (size_t)off * cap_l;
    int* lsa_s = nbr_ang + (size_t)off * cap_a;
    int* cl_s = cnt_list + (size_t)off * n_species;
    int* ca_s = cnt_ang + (size_t)off * n_species;
    for (int m = wfirst; m < n; m += wstride) {
        const float4 pk = sp[m];
        int nl = 0, na = 0;
        bool ovf = warp_build_lists(sp, cs, m, pk, g, cap_l, cap_a, sl, slt, sa, sat, nl, na);
        warp_write_grouped(sl, slt, nl, n_species, n, m, lst_s, (size_t)cap_l, 1, cl_s);
        warp_write_grouped(sa, sat, na, n_species, n, m, lsa_s, (size_t)cap_a, 1, ca_s);
        if (ovf && lane == 0) atomicOr(status, 1u);
        __syncwarp();   // this warp's list writes are visible to its lanes
        geometry_atom(sp, g, alpha, m, n, n_species, lst_s + (size_t)m * cap_l, cl_s, lsa_s + (size_t)m * cap_a, ca_s,
                      geo_rad + (size_t)(off + m) * cap_l * GR, geo_ang + (size_t)(off + m) * cap_a * GA,
                      bsum + (size_t)(off + m) * bstride, bimg ? bimg + (size_t)(off + m) * BIMG_BYTES : nullptr,
                      tab, cum);
    }
    const BatchKTab kt = kts[bs.ktab];
    const BatchKTri kr = ktris[bs.ktab];
    for (int idx = blockIdx.y * blockDim.x + threadIdx.x; idx < n * kt.nph; idx += blockDim.x * gridDim.y) {
        const int m = idx / kt.nph, e = idx - m * kt.nph;
        phase[(size_t)(off + m) * nph_stride + e] = batch_phase(sp[m], e, kt, kr);
    }
}

// ---------------------------------------------------------------------------------
// item kernel

// Stage c^R[t_i], c^A[t_i] (all neighbour species) and the scaler of the block's group.
__device__ __forceinline__ void stage_params(const float* __restrict__ pg, const ParamLayout& lay, int ti,
                                             float* __restrict__ prm) {
    const int S = lay.n_species;
    const int nr = S * NR * KR, na = S * NA * KA;
    const int tot = (nr + na + NDES) * CG;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int p = idx >> 5, c = idx & 31;
        int src, dst;
        if (p < nr) {
            src = lay.c_radial + ti * nr + p;
            dst = PR_R + p * CG;
        } else if (p < nr + na) {
            src = lay.c_angular + ti * na + (p - nr);
            dst = PR_A + (p - nr) * CG;
        } else {
            src = lay.scaler + (p - nr - na);
            dst = PR_S + (p - nr - na) * CG;
        }
        prm[dst + c] = __ldg(&pg[(size_t)src * CG + c]);
    }
}

// The backward's copy: c^R[t_i] as above, c^A[t_i] per (neighbour species, candidate) as a row
// of CA_STRIDE floats (q KA + k, padded) in place of the lane-minor c^A and the scaler, so each
// angular entry reads its 45 coefficients with 12 float4 loads (stride % 32 == 20: conflict-free).
constexpr int CA_STRIDE = 52;
static_assert(CA_STRIDE >= NA * KA && CA_STRIDE % 4 == 0 && (CA_STRIDE % 32) % 4 == 0 &&
                  MAX_SPECIES * CG * CA_STRIDE <= PARAM_FLOATS - PR_A && (PR_A % 4) == 0,
              "backward coefficient rows fit the parameter region, 16-byte aligned");
__device__ __forceinline__ void stage_params_bwd(const float* __restrict__ pg, const ParamLayout& lay, int ti,
                                                 float* __restrict__ prm) {
    const int S = lay.n_species;
    const int nr = S * NR * KR, na = S * NA * KA;
    for (int idx = threadIdx.x; idx < nr * CG; idx += blockDim.x) {
        const int p = idx >> 5, c = idx & 31;
        prm[PR_R + p * CG + c] = __ldg(&pg[(size_t)(lay.c_radial + ti * nr + p) * CG + c]);
    }
    for (int idx = threadIdx.x; idx < na * CG; idx += blockDim.x) {
        const int p = idx >> 5, c = idx & 31, t = p / (NA * KA), j = p - t * NA * KA;
        prm[PR_A + (t * CG + c) * CA_STRIDE + j] = __ldg(&pg[(size_t)(lay.c_angular + ti * na + p) * CG + c]);
    }
}

// Cumulative neighbour counts of sorted atom m by species: lanes 0..S-1 load the radial
// counts and lanes 8..8+S-1 the angular ones (one round trip), scanned by shuffles within
// each group of 8 lanes; cum[0..S] radial, cum[8..8+S] angular (the warp reads them after).
__device__ __forceinline__ void species_cum(const BatchArgs& a, int off, int n, int m, int S, int* cum) {
    const int lane = threadIdx.x & 31, g = lane & 7;
    __syncwarp();   // the warp is done with the previous atom's counts
    int v = 0;
    if (lane < 16 && g < S)
        v = (lane < 8 ? a.cnt_list : a.cnt_ang)[(size_t)off * S + (size_t)g * n + m];
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, d, 8);
        if (g >= d) v += t;
    }
    // inclusive sums: lane g holds the count of species 0..g; cum[g + 1] = that
    if (lane < 16 && g < S) cum[(lane & 8) + g + 1] = v;
    if (lane == 0 || lane == 8) cum[lane] = 0;
    __syncwarp();
}

// One bulk copy global -> shared of `bytes` (multiple of 16, both ends 16-byte aligned) into a
// warp's buffer, completing on `bar` (issued by one lane, after the warp's last read of `dst`).
__device__ __forceinline__ void warp_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    fence_proxy_async_smem();
    mbar_expect_tx(bar, bytes);
    bulk_g2s(dst, src, bytes, bar);
}

// Wait for buffer b of a warp (parity bit b of par); false after the bounded wait gave up.
__device__ __forceinline__ bool warp_wait(uint64_t* bars, int b, uint32_t& par, unsigned int* status) {
    const bool ok = mbar_wait_bounded(&bars[b], (par >> b) & 1u);
    par ^= 1u << b;
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(status, kStatusTimeout);
    return ok;
}

// Chunk jobs of an atom's backward: kind 0 = radial rows of neighbour species tj from row base
// (at most 32), kind 1 = angular rows from base (at most 32), kind 2 = done.
__device__ __forceinline__ void job_settle(const int* cum, int S, int& kind, int& tj, int& base) {
    if (kind == 0) {
        while (tj < S && base >= cum[tj + 1]) {
            ++tj;
            if (tj < S) base = cum[tj];
        }
        if (tj >= S) {
            kind = 1;
            base = 0;
        }
    }
    if (kind == 1 && base >= cum[8 + S]) kind = 2;
}

template <int NW>
__device__ __forceinline__ void block_sum(double v, double* red, double* dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    red[warp * CG + lane] = v;
    __syncthreads();
    if (warp == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) t += red[w * CG + lane];
        dst[lane] = t;
    }
    __syncthreads();
}

// Descriptor of sorted atom m for the 32 candidates of the group: A_{n,lm} to A, the
// scaled descriptor to rows 0..NDES-1 of the atom's duq block (replaced by dU/dD in the
// network pass).
__device__ __forceinline__ void descriptor_atom(const BatchArgs& a, const BatchStruct& bs, int m,
                                                const float* __restrict__ prm, const float* __restrict__ bsb,
                                                float* __restrict__ A, float* __restrict__ duq) {
    const int lane = threadIdx.x & 31;
    const int S = a.lay.n_species;
    const float* br = bsb;                       // B^R [MAX_SPECIES][KR]
    const float* ba = bsb + MAX_SPECIES * KR;    // B^A [S][KA][NLM]

    // lane = candidate: contractions with this candidate's c^R, c^A
    float d[NDES];
#pragma unroll
    for (int q = 0; q < NR; ++q) d[q] = 0.f;
    for (int tj = 0; tj < S; ++tj) {
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const float b = br[tj * KR + k];
#pragma unroll
            for (int q = 0; q < NR; ++q) d[q] = fmaf(prm[PR_R + ((tj * NR + q) * KR + k) * CG + lane], b, d[q]);
        }
    }
    float dA[NA][LMAX];
#pragma unroll
    for (int q = 0; q < NA; ++q)
#pragma unroll
        for (int l = 0; l < LMAX; ++l) dA[q][l] = 0.f;
    float d4[NA];
    float* Ao = A + (size_t)m * NANG * CG + lane;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float acc[NA][12];
#pragma unroll
        for (int q = 0; q < NA; ++q)
#pragma unroll
            for (int mm = 0; mm < 12; ++mm) acc[q][mm] = 0.f;
        for (int tj = 0; tj < S; ++tj) {
#pragma unroll 3
            for (int k = 0; k < KA; ++k) {
                float cv[NA];
#pragma unroll
                for (int q = 0; q < NA; ++q) cv[q] = prm[PR_A + ((tj * NA + q) * KA + k) * CG + lane];
                const float4* bp = reinterpret_cast<const float4*>(ba + (tj * KA + k) * NLM + 12 * h);
                const float4 b0 = bp[0], b1 = bp[1], b2 = bp[2];
                const float bv[12] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w, b2.x, b2.y, b2.z, b2.w};
#pragma unroll
                for (int q = 0; q < NA; ++q)
#pragma unroll
                    for (int mm = 0; mm < 12; ++mm) acc[q][mm] = fmaf(cv[q], bv[mm], acc[q][mm]);
            }
        }
#pragma unroll
        for (int q = 0; q < NA; ++q) {
#pragma unroll
            for (int mm = 0; mm < 12; ++mm) {
                const int M = 12 * h + mm;
                const int l = M < 3 ? 0 : (M < 8 ? 1 : (M < 15 ? 2 : 3));
                Ao[(q * NLM + M) * CG] = acc[q][mm];
                dA[q][l] = fmaf(c_wlm[M], acc[q][mm] * acc[q][mm], dA[q][l]);
            }
        }
        if (h == 0) {
#pragma unroll
            for (int q = 0; q < NA; ++q) {
                float a2[5], t[6], t2[6];
#pragma unroll
                for (int kk = 0; kk < 5; ++kk) a2[kk] = acc[q][3 + kk];
                tensor_from_a(a2, t);
                tensor_square(t, t2);
                d4[q] = t2[0] * t[0] + t2[1] * t[1] + t2[2] * t[2] + 2.f * (t2[3] * t[3] + t2[4] * t[4] + t2[5] * t[5]);
            }
        }
    }
#pragma unroll
    for (int l = 0; l < LMAX; ++l)
#pragma unroll
        for (int q = 0; q < NA; ++q) d[NR + l * NA + q] = dA[q][l];
#pragma unroll
    for (int q = 0; q < NA; ++q) d[NR + 4 * NA + q] = d4[q];
#pragma unroll
    for (int v = 0; v < NDES; ++v) d[v] *= prm[PR_S + v * CG + lane];

    float* dd = duq + (size_t)m * 2 * NDES * CG + lane;
#pragma unroll
    for (int v = 0; v < NDES; ++v) dd[v * CG] = d[v];
    __syncwarp();   // shared rows are reused by the warp's next atom
}

// Network of species t_i for two atoms (m1 < 0: one) and the 32 candidates, weights staged
// in shared memory: W0 per (neuron, candidate) as a row of NW_STRIDE floats (the N_des inputs,
// padded: 16-byte rows whose float4 loads are free of bank conflicts, four weights per load),
// then the other parameters lane-minor [p][CG]: b0 | w1E | w1q | b1E | b1q | scaler (NDES).
// h = tanh(W0 D - b0), U = w1E.h - b1E, q = w1q.h - b1q (Eq. U_i, Sec. II.B); writes
// dU/dD and dq/dD (scaled) over D, and (U, q).  Not inlined: its own register allocation keeps
// the item kernel free of spills.
constexpr int NW_STRIDE = 36;                              // >= NDES, multiple of 4, stride % 32 == 4
constexpr int NET_W0 = NNEU * CG * NW_STRIDE;              // floats of the W0 rows
constexpr int NP_B0 = 0, NP_W1E = NNEU, NP_W1Q = 2 * NNEU, NP_B1E = 3 * NNEU, NP_B1Q = 3 * NNEU + 1,
              NP_SC = 3 * NNEU + 2;                        // rows of the lane-minor part
constexpr int NET_FLOATS = NET_W0 + (NP_SC + NDES) * CG;
static_assert(NW_STRIDE >= NDES && NW_STRIDE % 4 == 0 && NW_STRIDE % 32 == 4, "W0 row layout");

__device__ __noinline__ void network_pair(const float* __restrict__ net, int m0, int m1,
                                             float* __restrict__ duq, float2* __restrict__ uq, double& su,
                                             double& sq) {
    const int lane = threadIdx.x & 31;
    const bool two = m1 >= 0;
    float* D0 = duq + (size_t)m0 * 2 * NDES * CG + lane;
    float* D1 = duq + (size_t)(two ? m1 : m0) * 2 * NDES * CG + lane;
    const float* np_ = net + NET_W0 + lane;                // lane-minor parameters
    float d0[NW_STRIDE], d1[NW_STRIDE];
#pragma unroll
    for (int v = 0; v < NW_STRIDE; ++v) {
        d0[v] = v < NDES ? D0[v * CG] : 0.f;
        d1[v] = v < NDES ? D1[v * CG] : 0.f;
    }
    float ge0[NNEU], gq0[NNEU], ge1[NNEU], gq1[NNEU];
    float ue0 = 0.f, uq0 = 0.f, ue1 = 0.f, uq1 = 0.f;
#pragma unroll
    for (int mu = 0; mu < NNEU; ++mu) {
        const float4* w4 = reinterpret_cast<const float4*>(net + ((size_t)mu * CG + lane) * NW_STRIDE);
        // two partial sums per atom (even / odd inputs): four independent chains per warp
        float p0 = -np_[(NP_B0 + mu) * CG], p1 = p0, p0b = 0.f, p1b = 0.f;
#pragma unroll
        for (int u = 0; u < (NDES + 3) / 4; ++u) {
            const float4 w = w4[u];
            p0 = fmaf(w.x, d0[4 * u], p0);
            p1 = fmaf(w.x, d1[4 * u], p1);
            p0b = fmaf(w.y, d0[4 * u + 1], p0b);
            p1b = fmaf(w.y, d1[4 * u + 1], p1b);
            if (4 * u + 2 < NDES) {
                p0 = fmaf(w.z, d0[4 * u + 2], p0);
                p1 = fmaf(w.z, d1[4 * u + 2], p1);
                p0b = fmaf(w.w, d0[4 * u + 3], p0b);
                p1b = fmaf(w.w, d1[4 * u + 3], p1b);
            }
        }
        p0 += p0b;
        p1 += p1b;
        const float h0 = tanhf(p0), h1 = tanhf(p1);
        const float we = np_[(NP_W1E + mu) * CG], wq = np_[(NP_W1Q + mu) * CG];
        ue0 = fmaf(we, h0, ue0);
        uq0 = fmaf(wq, h0, uq0);
        ue1 = fmaf(we, h1, ue1);
        uq1 = fmaf(wq, h1, uq1);
        const float dh0 = 1.f - h0 * h0, dh1 = 1.f - h1 * h1;
        ge0[mu] = we * dh0;
        gq0[mu] = wq * dh0;
        ge1[mu] = we * dh1;
        gq1[mu] = wq * dh1;
    }
    const float b1e = np_[NP_B1E * CG], b1q = np_[NP_B1Q * CG];
    // dU/dD and dq/dD four inputs at a time: one float4 of W0 per neuron serves 16 products
#pragma unroll 1
    for (int u = 0; u < (NDES + 3) / 4; ++u) {
        float du0[4] = {0.f, 0.f, 0.f, 0.f}, dq0[4] = {0.f, 0.f, 0.f, 0.f};
        float du1[4] = {0.f, 0.f, 0.f, 0.f}, dq1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int mu = 0; mu < NNEU; ++mu) {
            const float4 w = reinterpret_cast<const float4*>(net + ((size_t)mu * CG + lane) * NW_STRIDE)[u];
            const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                du0[e] = fmaf(ge0[mu], wv[e], du0[e]);
                dq0[e] = fmaf(gq0[mu], wv[e], dq0[e]);
                du1[e] = fmaf(ge1[mu], wv[e], du1[e]);
                dq1[e] = fmaf(gq1[mu], wv[e], dq1[e]);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int v = 4 * u + e;
            if (v >= NDES) break;
            const float sv = np_[(NP_SC + v) * CG];
            D0[v * CG] = du0[e] * sv;
            D0[(NDES + v) * CG] = dq0[e] * sv;
            if (two) {
                D1[v * CG] = du1[e] * sv;
                D1[(NDES + v) * CG] = dq1[e] * sv;
            }
        }
    }
    const float U0 = ue0 - b1e, Q0 = uq0 - b1q;
    uq[(size_t)m0 * CG + lane] = make_float2(U0, Q0);
    su += (double)U0;
    sq += (double)Q0;
    if (two) {
        const float U1 = ue1 - b1e, Q1 = uq1 - b1q;
        uq[(size_t)m1 * CG + lane] = make_float2(U1, Q1);
        su += (double)U1;
        sq += (double)Q1;
    }
}

// ---- tensor-core form of the descriptor contraction (BF16x3) -----------------------------
// Per species block t_i and tile of TC_TA atoms, with the candidate group on the M side:
//   D[(n, c)][(atom, lm)] = sum_{(s, k)} c^A[t_i][s][n][k][c] B^A[atom][s][k][lm]   (Sec. II.A)
// M = 5 n x 32 candidates in two 128-row tiles (n = 0..3, then n = 4 in rows 0..31 of the
// second; its other rows are never read back), K = (s, k) padded to 48, N = 24 x atoms (120,
// issued as 128).  Each operand is split x = hi + lo in BF16 and D = A_hi B_hi + A_hi B_lo +
// A_lo B_hi is accumulated in FP32 in tensor memory.  Tensor-memory lane = candidate and
// warp = n, so the epilogue thread (n, c) holds A_{n,lm} of its candidate for every atom of the
// tile and forms the invariants D^A_{nl} and D^4b_n itself; warps 5-7 form the radial
// descriptor D^R_n in FP32 from B^R rows that arrive with the tile.  Pipeline: two operand
// buffers and two accumulator buffers, so the products of tile j + 1 run while the warps
// read tile j, and the copies of tile j + 2 are in flight.
constexpr int TC_TA = 5;                           // atoms per tile
constexpr int TC_N = 128;                          // MMA N (24 TC_TA = 120 columns used)
constexpr int TC_SBO = 8 * BIMG_ROWB;              // 768 B between 8-row groups
constexpr int TC_APLANE = 256 * BIMG_ROWB;         // rows (n, c), n < 5 (160..255 unused)
constexpr int TC_BPLANE = TC_N * BIMG_ROWB;        // 12288 B (rows past 24 TC_TA never read back)
constexpr int TC_BR = MAX_SPECIES * KR;            // B^R floats per atom (first floats of its basis sums)
constexpr int TC_OFF_B = 2 * TC_APLANE;            // A hi | A lo | B[2] (hi | lo) | B^R[3] | c^R | scaler
constexpr int TC_OFF_BR = TC_OFF_B + 4 * TC_BPLANE;
constexpr int TC_OFF_R = TC_OFF_BR + 3 * TC_TA * TC_BR * 4;
constexpr int TC_OFF_S = TC_OFF_R + MAX_SPECIES * NR * KR * CG * 4;
constexpr int TC_BYTES = TC_OFF_S + NDES * CG * 4;
constexpr uint32_t TC_COLS = 512;                  // tensor-memory columns of the block
static_assert(24 * TC_TA <= TC_N && 4 * TC_N <= (int)TC_COLS, "two accumulator buffers of two M tiles");
static_assert((TC_OFF_B % 128) == 0 && (TC_OFF_BR % 16) == 0 && (TC_OFF_R % 16) == 0 && (TC_BR * 4) % 16 == 0,
              "bulk-copy and descriptor alignment");

struct TcBars {
    uint64_t* b;        // [2] operand buffers
    uint64_t* m;        // [2] MMA completion per accumulator buffer
};

// false when a bounded wait gave up (status bit set; results of the block are not valid)
__device__ __noinline__ bool forward_tc(const float* __restrict__ pg, ParamLayout lay, int ti, int p0, int p1,
                                        const int* __restrict__ order_s, const unsigned char* __restrict__ bimg_s,
                                        const float* __restrict__ bsum_s, int bstride, unsigned char* __restrict__ sm,
                                        uint32_t tmem, TcBars bars, uint32_t& tcpar, float* __restrict__ A,
                                        float* __restrict__ duq, unsigned int* __restrict__ status, bool x3) {
    constexpr int NW = 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S = lay.n_species;
    unsigned char* Ahi = sm;
    unsigned char* Alo = sm + TC_APLANE;
    const float* bring = reinterpret_cast<const float*>(sm + TC_OFF_BR);   // [3][TC_TA][TC_BR]
    float* cR = reinterpret_cast<float*>(sm + TC_OFF_R);   // [S][NR][KR][CG]
    float* scl = reinterpret_cast<float*>(sm + TC_OFF_S);  // [NDES][CG]
    bool ok_all = true;
    // operand A: row (n, c), K (s, k); lanes over candidates (coalesced parameter reads)
    const int abase = lay.c_angular + ti * S * NA * KA;
    for (int job = warp; job < NA * (BIMG_K / 8); job += NW) {
        const int n = job / (BIMG_K / 8), kc = job - n * (BIMG_K / 8);
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float x[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int kidx = 8 * kc + 2 * h + e, sj = kidx / KA, k = kidx - sj * KA;
                x[e] = sj < S ? __ldg(&pg[(size_t)(abase + (sj * NA + n) * KA + k) * CG + lane]) : 0.f;
            }
            const __nv_bfloat162 hi = __floats2bfloat162_rn(x[0], x[1]);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(x[0] - __bfloat162float(hi.x), x[1] - __bfloat162float(hi.y));
            hw[h] = *reinterpret_cast<const uint32_t*>(&hi);
            lw[h] = *reinterpret_cast<const uint32_t*>(&lo);
        }
        const int r = n * 32 + lane;
        const int o = ((r >> 3) * (BIMG_K / 8) + kc) * 128 + (r & 7) * 16;
        *reinterpret_cast<uint4*>(Ahi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(Alo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    // c^R[t_i] and the scaler for the radial descriptor (FP32, lane-minor)
    const int nr = S * NR * KR;
    for (int idx = tid; idx < (nr + NDES) * CG; idx += NW * 32) {
        const int p = idx >> 5, c = idx & 31;
        if (p < nr) cR[p * CG + c] = __ldg(&pg[(size_t)(lay.c_radial + ti * nr + p) * CG + c]);
        else scl[(p - nr) * CG + c] = __ldg(&pg[(size_t)(lay.scaler + p - nr) * CG + c]);
    }
    fence_proxy_async_smem();   // operand A (and the earlier phases' shared-memory use) before async writes / reads
    __syncthreads();

    const int ntile = (p1 - p0 + TC_TA - 1) / TC_TA;
    // tile j: the B operand images (hi, lo) into buffer j & 1 and the B^R rows into ring slot j % 3
    auto issue_b = [&](int j) {
        const int a0 = p0 + j * TC_TA, cnt = min(TC_TA, p1 - a0);
        unsigned char* dst = sm + TC_OFF_B + (j & 1) * 2 * TC_BPLANE;
        unsigned char* dbr = sm + TC_OFF_BR + (j % 3) * TC_TA * TC_BR * 4;
        mbar_expect_tx(&bars.b[j & 1], (uint32_t)(cnt * ((x3 ? 2 : 1) * BIMG_PLANE + TC_BR * 4)));
        for (int q = 0; q < cnt; ++q) {
            const int m = order_s[a0 + q];
            const unsigned char* src = bimg_s + (size_t)m * BIMG_BYTES;
            bulk_g2s(dst + q * BIMG_PLANE, src, BIMG_PLANE, &bars.b[j & 1]);
            if (x3) bulk_g2s(dst + TC_BPLANE + q * BIMG_PLANE, src + BIMG_PLANE, BIMG_PLANE, &bars.b[j & 1]);
            bulk_g2s(dbr + q * TC_BR * 4, bsum_s + (size_t)m * bstride, TC_BR * 4, &bars.b[j & 1]);
        }
    };
    // products of tile j into accumulator buffer j & 1 (thread 0, after its operands landed)
    auto issue_mma = [&](int j) {
        const int b = j & 1;
        const bool ok = mbar_wait_bounded(&bars.b[b], (tcpar >> b) & 1u);
        if (ok) {
            tc_fence_after();
            const uint32_t idesc = instr_desc(TC_FMT_BF16, 128, TC_N);
            const uint32_t bh = smem_u32(sm + TC_OFF_B + b * 2 * TC_BPLANE), bl = bh + TC_BPLANE;
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const uint32_t d = tmem + (uint32_t)(b * 2 * TC_N + mt * TC_N), ao = (uint32_t)mt * 16 * TC_SBO;
#pragma unroll
                for (int kk = 0; kk < BIMG_K / 16; ++kk) {
                    const uint32_t ko = (uint32_t)kk * 256;   // 16 K = two core matrices
                    const uint64_t dah = smem_desc(ah + ao + ko, 128, TC_SBO);
                    const uint64_t dal = smem_desc(al + ao + ko, 128, TC_SBO);
                    const uint64_t dbh = smem_desc(bh + ko, 128, TC_SBO);
                    const uint64_t dbl = smem_desc(bl + ko, 128, TC_SBO);
                    mma_f16(d, dah, dbh, idesc, kk > 0 ? 1u : 0u);
                    if (x3) {   // BF16x3: the two cross products of the lo parts
                        mma_f16(d, dah, dbl, idesc, 1u);
                        mma_f16(d, dal, dbh, idesc, 1u);
                    }
                }
            }
            mma_commit(&bars.m[b]);
        } else {
            atomicOr(status, kStatusTimeout);
            mbar_arrive(&bars.m[b]);   // no products: release the waiting warps at once
        }
    };
    if (tid == 0 && ntile > 0) {
        issue_b(0);
        if (ntile > 1) issue_b(1);
        issue_mma(0);
    }
    // Tile j's B^R rows are read with ordinary loads: thread 0 saw their copy complete before a
    // block barrier (this one for tile 0, the end of iteration j - 1 for the others).
    __syncthreads();
    for (int j = 0; j < ntile; ++j) {
        const int a0 = p0 + j * TC_TA, cnt = min(TC_TA, p1 - a0);
        const int b = j & 1;
        // every thread keeps the phase bits of the operand barriers in step with thread 0
        if (tid == 0 && j + 1 < ntile) issue_mma(j + 1);
        if (j == 0) tcpar ^= 1u;
        if (j + 1 < ntile) tcpar ^= 1u << ((j + 1) & 1);
        const bool okm = mbar_wait_bounded(&bars.m[b], (tcpar >> (2 + b)) & 1u);
        tcpar ^= 1u << (2 + b);
        if (!okm) {
            ok_all = false;
            if (lane == 0) atomicOr(status, kStatusTimeout);
        }
        tc_fence_after();
        // operand buffer b is free once tile j's products are complete: tile j + 2 streams in
        if (tid == 0 && j + 2 < ntile) issue_b(j + 2);
        const float* brow = bring + (j % 3) * TC_TA * TC_BR;
        if (warp < NA) {
            // epilogue: n = warp, c = lane
            const int n = warp;
            const uint32_t tbase = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                   (uint32_t)(b * 2 * TC_N + (warp == 4 ? TC_N : 0));
            for (int q = 0; q < cnt; ++q) {
                const int m = order_s[a0 + q];
                uint32_t r[24];
                tmem_ld8_nowait(tbase + q * NLM, r);
                tmem_ld8_nowait(tbase + q * NLM + 8, r + 8);
                tmem_ld8_nowait(tbase + q * NLM + 16, r + 16);
                tmem_wait_ld();
                float v[NLM];
#pragma unroll
                for (int M = 0; M < NLM; ++M) v[M] = __uint_as_float(r[M]);
                float* Ao = A + (size_t)m * NANG * CG + (size_t)n * NLM * CG + lane;
                float dA[LMAX] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int M = 0; M < NLM; ++M) {
                    const int l = M < 3 ? 0 : (M < 8 ? 1 : (M < 15 ? 2 : 3));
                    Ao[M * CG] = v[M];
                    dA[l] = fmaf(c_wlm[M], v[M] * v[M], dA[l]);
                }
                float a2[5], t[6], t2[6];
#pragma unroll
                for (int kk = 0; kk < 5; ++kk) a2[kk] = v[3 + kk];
                tensor_from_a(a2, t);
                tensor_square(t, t2);
                const float d4 = t2[0] * t[0] + t2[1] * t[1] + t2[2] * t[2] + 2.f * (t2[3] * t[3] + t2[4] * t[4] + t2[5] * t[5]);
                float* dd = duq + (size_t)m * 2 * NDES * CG + lane;
#pragma unroll
                for (int l = 0; l < LMAX; ++l) {
                    const int vi = NR + l * NA + n;
                    dd[vi * CG] = dA[l] * scl[vi * CG + lane];
                }
                const int v4 = NR + 4 * NA + n;
                dd[v4 * CG] = d4 * scl[v4 * CG + lane];
            }
        } else {
            // radial descriptor D^R_n = sum c^R[t_i][t_j][n][k] B^R[t_j][k] (FP32), lane = candidate
            for (int q = warp - NA; q < cnt; q += NW - NA) {
                const int m = order_s[a0 + q];
                const float* br = brow + q * TC_BR;
                float d[NR];
#pragma unroll
                for (int u = 0; u < NR; ++u) d[u] = 0.f;
                for (int tj = 0; tj < S; ++tj) {
#pragma unroll
                    for (int k = 0; k < KR; ++k) {
                        const float bv = br[tj * KR + k];
#pragma unroll
                        for (int u = 0; u < NR; ++u) d[u] = fmaf(cR[((tj * NR + u) * KR + k) * CG + lane], bv, d[u]);
                    }
                }
                float* dd = duq + (size_t)m * 2 * NDES * CG + lane;
#pragma unroll
                for (int u = 0; u < NR; ++u) dd[u * CG] = d[u] * scl[u * CG + lane];
            }
        }
        fence_proxy_async_smem();   // the B^R ring slot read here is refilled by a later bulk copy
        tc_fence_before();
        __syncthreads();            // accumulator buffer b is reused by tile j + 2
        tc_fence_after();
    }
    return ok_all;
}

// Stage the network block of species ti and the scaler (layout of network_pair).  Global
// reads are coalesced over the candidates; the W0 rows are written transposed (4-way bank
// conflicts on these stores, once per species block).
__device__ __forceinline__ void stage_network(const float* __restrict__ pg, const ParamLayout& lay, int ti,
                                              float* __restrict__ net) {
    const float* src = pg + (size_t)(lay.mlp + ti * lay.mlp_stride) * CG;
    const float* scl = pg + (size_t)lay.scaler * CG;
    for (int idx = threadIdx.x; idx < NNEU * NW_STRIDE * CG; idx += blockDim.x) {
        const int c = idx & 31, r = idx >> 5, mu = r / NW_STRIDE, v = r - mu * NW_STRIDE;
        net[((size_t)mu * CG + c) * NW_STRIDE + v] =
            v < NDES ? __ldg(&src[(size_t)(ParamLayout::W0 + mu * NDES + v) * CG + c]) : 0.f;
    }
    float* np_ = net + NET_W0;
    for (int idx = threadIdx.x; idx < (NP_SC + NDES) * CG; idx += blockDim.x) {
        const int p = idx >> 5, c = idx & 31;
        float x;
        if (p < NP_B1E) x = __ldg(&src[(size_t)(ParamLayout::B0 + p) * CG + c]);           // b0 | w1E | w1q
        else if (p == NP_B1E) x = __ldg(&src[(size_t)ParamLayout::B1E * CG + c]);
        else if (p == NP_B1Q) x = __ldg(&src[(size_t)ParamLayout::B1Q * CG + c]);
        else x = __ldg(&scl[(size_t)(p - NP_SC) * CG + c]);
        np_[idx] = x;
    }
}

// ---- tensor-core form of the k-space potential and field (FP16x3) ---------------------------
// Per tile of FT_M = 128 atoms and chunk of 8 wave vectors (K = 16: the real and imaginary parts
// of e = exp(i k.r_j) for each):
//   D[j][(c, o)] = sum_k e_r(k, j) B[2k][(c, o)] + e_i(k, j) B[2k + 1][(c, o)]
// with, for C = 4 k_e G(k) S(k) of candidate c,
//   o = 0:     B = (C_r, C_i)            D = sum_k Re(C conj(e))       = phi^k_j
//   o = 1..3:  B = k_o (C_i, -C_r)       D = sum_k k_o Im(C conj(e))   = E^k_j,o   (Sec. II.C)
// M = atoms, N = 32 candidates x 4 = 128, one K = 16 product per chunk.  The block's threads
// form both operands in shared memory (the phase products from the atoms' staged separable
// factors; C(k) and k from a staged window) in the canonical K-major layout, each value split
// x = hi + lo in FP16 (11 significant bits each, as TF32, at half the bytes: the operand reads
// of the tensor cores and the threads' stores share the shared-memory bandwidth, which bounds
// this pass); A_hi B_hi and A_hi B_lo + A_lo B_hi accumulate in FP32 in two tensor-memory
// accumulators (so the small products are not added into the large sum, whose FP32
// accumulation would lose part of each), added in the epilogue.  |e| <= 1; the B values stay far inside the FP16 range (|C k| < 6.5e4 for any
// structure the batched call takes; values below 6e-5 keep an absolute error under 3e-8).
// Two stages of FT_CPI chunks: stage i + 1 is formed while the products of stage i run (the
// fixed cost of a stage, its commit, proxy fence and block barrier, is shared by its chunks).
// Tensor-memory lane = atom, so the epilogue's stores of (phi, E) per candidate are coalesced
// over the atoms.
constexpr int FT_M = 128;                  // atoms per tile
constexpr int FT_N = 4 * CG;               // accumulator columns: hi x hi at 0, the cross products at FT_N
constexpr int FT_PLANE = FT_M * 16 * 2;    // 4096 B: 128 rows x 16 FP16
constexpr int FT_BUF = 4 * FT_PLANE;       // A hi | A lo | B hi | B lo
constexpr int FT_WC = 8;                   // chunks per staged window of C(k), k and the chunk table
constexpr int FT_WIN_SK = FT_WC * 8 * CG * 8;                  // 16384 B of C(k)
constexpr int FT_WIN = FT_WIN_SK + FT_WC * 8 * 16 + FT_WC * 16;   // + wave vectors + chunk entries
constexpr int FT_CPI = 2;                  // chunks per pipeline stage (one commit, one block barrier)
constexpr int FT_STAGE = FT_CPI * FT_BUF;
constexpr int FT_OFF_WIN = 2 * FT_STAGE;   // two stages, then two windows
constexpr int FT_OFF_PH = FT_OFF_WIN + 2 * FT_WIN;   // staged phase factors [nph][FT_PHS] float2
constexpr int FT_PHS = FT_M + 1;           // odd row stride: the transposing stores spread over banks
constexpr int FT_SBO = 2 * 128;            // 8-row groups 256 B apart (16 FP16 = 2 core matrices)
static_assert(FT_WIN % 16 == 0 && FT_OFF_PH % 16 == 0, "bulk-copy alignment");
static_assert(FT_WC % FT_CPI == 0, "a stage never straddles two windows");
static_assert(FT_OFF_PH + BATCH_MAX_NPH * FT_PHS * 8 <= 220 * 1024, "field operands, windows and phase factors");

// (x, y) = hi + lo + d with hi, lo FP16 pairs (rounded to nearest, x in the low half) and
// |d| <= 2^-22 max(|x|, |y|) in the normal range; x - hi is exact in FP32
__device__ __forceinline__ void f16_split2(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(x, y);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Row r (K = 16 FP16) of an operand plane: byte offset of its core matrix kc (8 values)
__device__ __forceinline__ int ft_off(int r, int kc) { return ((r >> 3) * 2 + kc) * 128 + (r & 7) * 16; }

// false when a bounded wait gave up (status bit set; results of the block are not valid).
// chunk, kvec: the structure's chunk table and wave vectors; sk: C(k) [8 nchunk][CG] (real
// entries only), written by this block; phb: phase rows [n][ps]; fk: output [CG][nmax] (phi^k, E^k).
// mbar: the two MMA barriers (phase bits 2, 3 of tcpar); wbar: the two window barriers (phase
// bits 0, 1 of wpar).  C(k), k and the chunk entries of FT_WC chunks arrive by bulk copies, the
// window after next issued once the block is done with a window, so the operand formation reads
// shared memory only.
__device__ __noinline__ bool field_tc(int n, int nmax, const float2* __restrict__ phb, int ps, BatchKTab kt,
                                      const int4* __restrict__ chunk, const float4* __restrict__ kvec,
                                      const float2* __restrict__ sk, float4* __restrict__ fk,
                                      unsigned char* __restrict__ sm, uint32_t tmem, uint64_t* mbar, uint32_t& tcpar,
                                      uint64_t* wbar, uint32_t& wpar, unsigned int* __restrict__ status) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nch = kt.nchunk, nph = kt.nph;
    const int ey = kt.yoff + kt.n2max, ez = kt.zoff + kt.n3max;
    if (nch == 0) {   // no wave vectors: no k-space potential or field
        for (int i = tid; i < CG * n; i += blockDim.x) fk[(size_t)(i / n) * nmax + i % n] = make_float4(0.f, 0.f, 0.f, 0.f);
        return true;
    }
    float2* ph = reinterpret_cast<float2*>(sm + FT_OFF_PH);
    const uint32_t idesc = instr_desc(TC_FMT_F16, FT_M, 128);
    // shared-memory addresses stay below 2^18, so the 14-bit start-address field (address / 16) of
    // the base descriptor takes the operand offsets / 16 by plain addition
    const uint64_t dbase = smem_desc(smem_u32(sm), 128, FT_SBO);
    const int r = tid & (FT_M - 1), half = tid >> 7;   // operand row r, wave vectors 4 half .. 4 half + 3
    const int c = r >> 2, oo = r & 3;                  // B row r: candidate c, output oo
    const int nwin = (nch + FT_WC - 1) / FT_WC;
    bool ok_all = true;
    auto fail = [&]() {
        ok_all = false;
        if (lane == 0) atomicOr(status, kStatusTimeout);
    };
    auto wait_mma = [&](int b) {
        const bool ok = mbar_wait_bounded(&mbar[b], (tcpar >> (2 + b)) & 1u);
        tcpar ^= 1u << (2 + b);
        if (!ok) fail();
    };
    // window w: C(k) of its chunks, their wave vectors and table entries (thread 0)
    auto issue_win = [&](int w) {
        const int h0 = w * FT_WC, cc = min(FT_WC, nch - h0);
        unsigned char* dst = sm + FT_OFF_WIN + (w & 1) * FT_WIN;
        const uint32_t sb = (uint32_t)(cc * 8 * CG * 8), kb = (uint32_t)(cc * 8 * 16), cb = (uint32_t)(cc * 16);
        fence_proxy_async_all();   // C(k) was written by this block with ordinary stores
        mbar_expect_tx(&wbar[w & 1], sb + kb + cb);
        bulk_g2s(dst, sk + (size_t)h0 * 8 * CG, sb, &wbar[w & 1]);
        bulk_g2s(dst + FT_WIN_SK, kvec + (size_t)h0 * 8, kb, &wbar[w & 1]);
        bulk_g2s(dst + FT_WIN_SK + FT_WC * 8 * 16, chunk + h0, cb, &wbar[w & 1]);
    };
    for (int j0 = 0; j0 < n; j0 += FT_M) {
        const int cnt = min(FT_M, n - j0);
        __syncthreads();   // the previous tile's phase factors, windows and accumulator are no longer read
        if (tid == 0) {
            issue_win(0);
            if (nwin > 1) issue_win(1);
        }
        for (int idx = tid; idx < FT_M * nph; idx += blockDim.x) {
            const int q = idx / nph, e = idx - q * nph;
            ph[e * FT_PHS + q] = q < cnt ? __ldg(&phb[(size_t)(j0 + q) * ps + e]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int nit = (nch + FT_CPI - 1) / FT_CPI;
        for (int it = 0; it < nit; ++it) {
            const int b = it & 1, h0 = it * FT_CPI, w = h0 / FT_WC, hl0 = h0 - w * FT_WC;
            const int nq = min(FT_CPI, nch - h0);   // chunks of this stage
            unsigned char* stage = sm + b * FT_STAGE;
            if (hl0 == 0) {   // the window's copies have landed
                const bool ok = mbar_wait_bounded(&wbar[w & 1], (wpar >> (w & 1)) & 1u);
                wpar ^= 1u << (w & 1);
                if (!ok) fail();
            }
            if (it >= 2) wait_mma(b);   // the products of stage it - 2 have read buffer b
            const unsigned char* win = sm + FT_OFF_WIN + (w & 1) * FT_WIN;
#pragma unroll
            for (int q = 0; q < FT_CPI; ++q) {
                if (q >= nq) break;
                const int hl = hl0 + q;
                unsigned char* buf = stage + q * FT_BUF;
                const int4 ci = reinterpret_cast<const int4*>(win + FT_WIN_SK + FT_WC * 8 * 16)[hl];
                uint32_t hw[4], lw[4];
                {   // A row r = atom j0 + r: e = X[n1] Y[n2] Z[n3 + t]
                    const float2 xy = cmul(ph[ci.x * FT_PHS + r], ph[(ey + ci.y) * FT_PHS + r]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 e = cmul(xy, ph[(ez + ci.z + 4 * half + u) * FT_PHS + r]);
                        f16_split2(e.x, e.y, hw[u], lw[u]);
                    }
                    const int o = ft_off(r, half);
                    *reinterpret_cast<uint4*>(buf + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(buf + FT_PLANE + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
                {   // B row r = (candidate c, output oo); the chunk's padding entries are zero
                    const float2* sw = reinterpret_cast<const float2*>(win) + hl * 8 * CG;
                    const float* kw = reinterpret_cast<const float*>(win + FT_WIN_SK) + hl * 8 * 4 + (oo > 0 ? oo - 1 : 0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int t = 4 * half + u;
                        const bool real = t < ci.w;
                        const float2 C = sw[t * CG + c];
                        const float kf = kw[t * 4];
                        const float v0 = real ? (oo == 0 ? C.x : kf * C.y) : 0.f;
                        const float v1 = real ? (oo == 0 ? C.y : -kf * C.x) : 0.f;
                        f16_split2(v0, v1, hw[u], lw[u]);
                    }
                    const int o = 2 * FT_PLANE + ft_off(r, half);
                    *reinterpret_cast<uint4*>(buf + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(buf + FT_PLANE + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            }
            fence_proxy_async_smem();   // the operands, written by ordinary stores, are read by the tensor cores
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int q = 0; q < FT_CPI; ++q) {
                    if (q >= nq) break;
                    // descriptors of the chunk's planes: the base descriptor's start address plus offset / 16
                    const uint64_t dah = dbase + (uint64_t)((b * FT_STAGE + q * FT_BUF) >> 4);
                    const uint64_t dal = dah + (uint64_t)(FT_PLANE >> 4);
                    const uint64_t dbh = dah + (uint64_t)(2 * FT_PLANE >> 4), dbl = dah + (uint64_t)(3 * FT_PLANE >> 4);
                    const uint32_t acc = (it | q) ? 1u : 0u;
                    mma_f16(tmem, dah, dbh, idesc, acc);                 // hi x hi
                    mma_f16(tmem + FT_N, dah, dbl, idesc, acc);          // the cross products
                    mma_f16(tmem + FT_N, dal, dbh, idesc, 1u);
                }
                mma_commit(&mbar[b]);
                // the block is done with window w after its last chunk: window w + 2 streams into it
                if (hl0 + nq == FT_WC && w + 2 < nwin) issue_win(w + 2);
            }
        }
        for (int it = max(0, nit - 2); it < nit; ++it) wait_mma(it & 1);   // the tile's last products
        tc_fence_after();
        {   // epilogue: lane = atom of the tile, warps 4-7 take candidates 16-31
            const int row = (warp & 3) * 32 + lane, cb = (warp >> 2) * 16;
            const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(cb * 4);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                float v[32], v2[32];
                tmem_ld32(ta + (uint32_t)(hh * 32), v);
                tmem_ld32(ta + (uint32_t)(FT_N + hh * 32), v2);
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] += v2[q];
                if (row < cnt) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        fk[(size_t)(cb + hh * 8 + q) * nmax + j0 + row] =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        }
        tc_fence_before();   // the next tile's first products overwrite the accumulator
    }
    fence_proxy_async_smem();   // the next phase refills this shared memory by bulk copies
    return ok_all;
}

// ---- tensor-core form of the structure factor (FP16x3) ---------------------------------------
// S_c(k) = sum_j q_jc exp(i k.r_j) (Sec. II.B) for windows of 64 padded wave vectors:
//   D[2 t + part][c] = sum_j A[2 t + part][j] Q[c][j],  A = (Re, Im) e(k_t, r_j)
// M = 128, N = 32 candidates, K = atoms in tiles of SK_AT = 32 (two K = 16 products, three for the
// FP16 hi + lo split of both operands, as in the field pass).  The tensor cores' FP32
// accumulation loses a little of every small product added to a large sum, and over a long sum
// these losses share a sign: so the hi x hi products and the two cross products accumulate in
// separate tensor-memory columns, and the sums restart every SK_FT tiles (512 atoms, the blocks
// of the FP32 path) with their FP32 partial sums written to skp [block][nkp][CG] as (Re, Im)
// and added in FP64 afterwards.  Up to SK_WMAX = 8 windows (512 wave vectors, 64 columns each)
// accumulate at once while the atoms stream through; larger k-sets take further passes.  Each
// atom tile's charges and phase rows arrive by bulk copy (double-buffered); a pipeline stage
// forms the phases of SK_WPS windows (and, at a tile's first stage, the charge operand) and ends
// in one commit; one thread forms the 8 wave vectors of a chunk for one atom (X Y once, then the
// chunk's Z factors), written along M (the operand is MN-major).  The epilogue stages each
// window in shared memory so the global stores are coalesced.
constexpr int SK_AT = 32;                         // atoms per tile (K)
constexpr int SK_APLANE = 128 * SK_AT * 2;        // 8192 B: 128 rows x 32 FP16
constexpr int SK_ABUF = 2 * SK_APLANE;            // hi | lo of one window
constexpr int SK_WPS = 2;                         // windows per pipeline stage
constexpr int SK_STAGE = SK_WPS * SK_ABUF;
constexpr int SK_BPLANE = CG * SK_AT * 2;         // 2048 B: 32 candidate rows x 32 FP16
constexpr int SK_BBUF = 2 * SK_BPLANE;
constexpr int SK_OFF_B = 2 * SK_STAGE;            // two stages, then two charge operands,
constexpr int SK_OFF_T = SK_OFF_B + 2 * SK_BBUF;  // then two atom tiles: charges [SK_AT][CG] | phase rows [SK_AT][ps]
constexpr int SK_WMAX = (int)TC_COLS / (2 * CG);  // windows per pass (hi x hi and cross-product columns)
constexpr int SK_FT = 16;                         // tiles per block of partial sums (512 atoms)
constexpr int SK_SBO = 4 * 128;                   // charge operand: 8-row groups 512 B apart (K-major, 32 FP16)
// Phase operand, MN-major (M = 128 rows kk = 2 t + part contiguous): core matrices of 8 atoms x 8
// rows (16 B); M-adjacent cores 128 B apart (SBO), 8-atom groups 2048 B apart (LBO).
constexpr int SK_ALBO = 16 * 128, SK_ASBO = 128;
// a tile's phase rows keep their global stride ps (= 2 mod 16 float2): the lanes (atoms) of a load
// spread over the banks
__host__ __device__ constexpr int sk_tile_bytes(int ps) { return SK_AT * CG * 4 + SK_AT * ps * 8; }
// the pass's chunk-table entries follow the tiles
__host__ __device__ constexpr int sk_smem(int ps) { return SK_OFF_T + 2 * sk_tile_bytes(ps) + SK_WMAX * 8 * 16; }
static_assert(sk_smem(batch_phase_stride(BATCH_MAX_NPH)) <= 220 * 1024 && SK_OFF_T % 16 == 0, "structure-factor buffers");
static_assert(SK_APLANE == (SK_AT / 8) * SK_ALBO, "phase operand plane: 4 atom groups of 16 cores");
static_assert(SK_AT == 32, "one atom per lane in the formation");
static_assert(64 * (CG + 1) * 8 <= 2 * SK_STAGE, "epilogue staging fits the stage buffers");
static_assert(SK_AT * SK_FT == QT * FLUSH_TILES, "blocks of partial sums as in the FP32 path (buffer size)");

// Row r (K = 32 FP16) of a structure-factor operand plane: byte offset of its core matrix kc
__device__ __forceinline__ int sk_off(int r, int kc) { return ((r >> 3) * 4 + kc) * 128 + (r & 7) * 16; }

// false when a bounded wait gave up (status bit set; results of the block are not valid).
// qcs: corrected charges [n][CG] (written by this block); phb: phase rows [n][ps]; chunk: the
// structure's chunk table; skp: output [ceil(n / 512)][8 nchunk][CG].  mbar: the two MMA barriers (phase bits
// 2, 3 of tcpar); tbar: the two tile barriers (phase bits 0, 1 of tpar).
__device__ __noinline__ bool sk_tc(int n, const float2* __restrict__ phb, int ps, BatchKTab kt,
                                   const int4* __restrict__ chunk, const float* __restrict__ qcs,
                                   float2* __restrict__ skp, unsigned char* __restrict__ sm, uint32_t tmem,
                                   uint64_t* mbar, uint32_t& tcpar, uint64_t* tbar, uint32_t& tpar,
                                   unsigned int* __restrict__ status) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nch = kt.nchunk;
    if (nch == 0 || n == 0) return true;
    const int nkp = 8 * nch, nwin = (nkp + 63) / 64, ntile = (n + SK_AT - 1) / SK_AT;
    const int ey = kt.yoff + kt.n2max, ez = kt.zoff + kt.n3max;
    const uint32_t idesc = instr_desc(TC_FMT_F16, 128, CG) | (1u << 15);   // A (the phases) MN-major
    const uint64_t dbase = smem_desc(smem_u32(sm), 128, SK_SBO);          // charge operand (K-major)
    const uint64_t pbase = smem_desc(smem_u32(sm), SK_ALBO, SK_ASBO);     // phase operand (MN-major)
    // offsets / 16 add to the start-address field of either
    const int tb = sk_tile_bytes(ps);
    const int ja = tid & (SK_AT - 1), cq = tid >> 5;   // phase operand: atom ja of the tile, chunk cq of the window
    bool ok_all = true;
    auto fail = [&]() {
        ok_all = false;
        if (lane == 0) atomicOr(status, kStatusTimeout);
    };
    auto wait_mma = [&](int b) {
        const bool ok = mbar_wait_bounded(&mbar[b], (tcpar >> (2 + b)) & 1u);
        tcpar ^= 1u << (2 + b);
        if (!ok) fail();
    };
    auto issue_tile = [&](int i) {   // thread 0: the charges and phase rows of atom tile i
        const int j0 = i * SK_AT, cnt = min(SK_AT, n - j0);
        unsigned char* dst = sm + SK_OFF_T + (i & 1) * tb;
        const uint32_t qb = (uint32_t)(cnt * CG * 4), rb = (uint32_t)(cnt * ps * 8);
        fence_proxy_async_all();   // the charges were written by this block with ordinary stores
        mbar_expect_tx(&tbar[i & 1], qb + rb);
        bulk_g2s(dst, qcs + (size_t)j0 * CG, qb, &tbar[i & 1]);
        bulk_g2s(dst + SK_AT * CG * 4, phb + (size_t)j0 * ps, rb, &tbar[i & 1]);
    };
    for (int w0 = 0; w0 < nwin; w0 += SK_WMAX) {
        const int nw = min(SK_WMAX, nwin - w0);
        const int nst = (nw + SK_WPS - 1) / SK_WPS;   // stages per atom tile
        __syncthreads();   // the previous pass's epilogue is done with shared and tensor memory
        if (tid == 0) {
            issue_tile(0);
            if (ntile > 1) issue_tile(1);
        }
        int4* cpass = reinterpret_cast<int4*>(sm + SK_OFF_T + 2 * tb);   // chunk entries of the pass's windows
        for (int h = tid; h < nw * 8; h += blockDim.x)
            if (w0 * 8 + h < nch) cpass[h] = __ldg(&chunk[w0 * 8 + h]);
        __syncthreads();
        for (int fb = 0; fb * SK_FT < ntile; ++fb) {   // blocks of partial sums
        const int i0 = fb * SK_FT, i1 = min(ntile, i0 + SK_FT);
        int s = 0;   // stage counter of the block
        for (int i = i0; i < i1; ++i) {
            const int cnt = min(SK_AT, n - i * SK_AT);
            const unsigned char* tile = sm + SK_OFF_T + (i & 1) * tb;
            const float* qt = reinterpret_cast<const float*>(tile);
            const float2* pr = reinterpret_cast<const float2*>(tile + SK_AT * CG * 4);
            unsigned char* bq = sm + SK_OFF_B + (i & 1) * SK_BBUF;
            for (int st = 0; st < nst; ++st, ++s) {
                const int b = s & 1;
                if (st == 0) {   // tile i has landed
                    const bool ok = mbar_wait_bounded(&tbar[i & 1], (tpar >> (i & 1)) & 1u);
                    tpar ^= 1u << (i & 1);
                    if (!ok) fail();
                }
                if (s >= 2) wait_mma(b);   // the products of stage s - 2 (and of tile i - 2) are complete
                if (st == 0 && tid < 4 * CG) {   // charge operand of tile i: row c, atoms 8 g2 .. 8 g2 + 7
                    const int c = tid & (CG - 1), g2 = tid >> 5;
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int a0 = 8 * g2 + 2 * u;
                        const float q0 = a0 < cnt ? qt[a0 * CG + c] : 0.f;
                        const float q1 = a0 + 1 < cnt ? qt[(a0 + 1) * CG + c] : 0.f;
                        f16_split2(q0, q1, hw[u], lw[u]);
                    }
                    const int o = sk_off(c, g2);
                    *reinterpret_cast<uint4*>(bq + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(bq + SK_BPLANE + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
#pragma unroll
                for (int q = 0; q < SK_WPS; ++q) {   // phase operand of window w0 + st SK_WPS + q
                    const int wl = st * SK_WPS + q;
                    if (wl >= nw) break;
                    const int h = (w0 + wl) * 8 + cq;   // the thread's chunk
                    uint32_t hw[8], lw[8];
                    if (h < nch && ja < cnt) {
                        const int4 ci = cpass[h - w0 * 8];
                        const float2* row = pr + ja * ps;
                        const float2 xy = cmul(row[ci.x], row[ey + ci.y]);
                        const float2* zr = row + ez + ci.z;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float2 e = cmul(xy, zr[u]);
                            f16_split2(e.x, e.y, hw[u], lw[u]);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) hw[u] = lw[u] = 0u;
                    }
                    unsigned char* ab = sm + b * SK_STAGE + q * SK_ABUF;
                    const int o = (ja >> 3) * SK_ALBO + 2 * cq * SK_ASBO + (ja & 7) * 16;   // rows 16 cq .. 16 cq + 15
                    *reinterpret_cast<uint4*>(ab + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(ab + o + SK_ASBO) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
                    *reinterpret_cast<uint4*>(ab + SK_APLANE + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    *reinterpret_cast<uint4*>(ab + SK_APLANE + o + SK_ASBO) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
                }
                fence_proxy_async_smem();   // the operands, written by ordinary stores, are read by the tensor cores
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const uint64_t dq = dbase + (uint64_t)((SK_OFF_B + (i & 1) * SK_BBUF) >> 4);
#pragma unroll
                    for (int q = 0; q < SK_WPS; ++q) {
                        const int wl = st * SK_WPS + q;
                        if (wl >= nw) break;
                        const uint64_t da = pbase + (uint64_t)((b * SK_STAGE + q * SK_ABUF) >> 4);
                        const uint32_t d1 = tmem + (uint32_t)(wl * 2 * CG), d2 = d1 + (uint32_t)CG;
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {   // K = 16 atoms per product: two 8-atom groups
                            const uint64_t ah = da + (uint64_t)(ks * 2 * SK_ALBO >> 4), al = ah + (uint64_t)(SK_APLANE >> 4);
                            const uint64_t bh = dq + (uint64_t)(ks * 16), bl = bh + (uint64_t)(SK_BPLANE >> 4);
                            const uint32_t acc = (i > i0 || ks) ? 1u : 0u;
                            mma_f16(d1, ah, bh, idesc, acc);   // hi x hi
                            mma_f16(d2, ah, bl, idesc, acc);   // the cross products
                            mma_f16(d2, al, bh, idesc, 1u);
                        }
                    }
                    mma_commit(&mbar[b]);
                }
                // the block is done with tile i after its last stage: tile i + 2 streams into it
                if (tid == 0 && st == nst - 1 && i + 2 < ntile) issue_tile(i + 2);
            }
        }
        for (int s2 = max(0, s - 2); s2 < s; ++s2) wait_mma(s2 & 1);   // the block's last products
        tc_fence_after();
        // epilogue per window: warps 0-3 (tensor-memory lanes = rows) stage the block's S as
        // [64][CG + 1] float2 (Re, Im) in the stage buffers, then the block stores it coalesced
        float2* stg = reinterpret_cast<float2*>(sm);
        float2* dst = skp + (size_t)fb * nkp * CG;
        for (int wl = 0; wl < nw; ++wl) {
            if (warp < 4) {
                float v[32], v2[32];
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(wl * 2 * CG);
                tmem_ld32(ta, v);
                tmem_ld32(ta + (uint32_t)CG, v2);
                tc_fence_before();   // the next block's first products overwrite these columns
                const int row = warp * 32 + lane, tt = row >> 1, part = row & 1;
                float* sf = reinterpret_cast<float*>(stg + tt * (CG + 1));
#pragma unroll
                for (int c = 0; c < CG; ++c) sf[2 * c + part] = v[c] + v2[c];
            }
            __syncthreads();
            for (int idx = tid; idx < 64 * CG; idx += blockDim.x) {
                const int tt = idx >> 5, c = idx & (CG - 1), kl = (w0 + wl) * 64 + tt;
                if (kl < nkp) dst[(size_t)kl * CG + c] = stg[tt * (CG + 1) + c];
            }
            __syncthreads();
        }
        }
        tc_fence_before();   // the next pass's first products overwrite the accumulators
    }
    fence_proxy_async_smem();   // the next phase refills this shared memory by bulk copies
    return ok_all;
}

// Backward of sorted atom m: partial forces of every list entry (Sec. II.C).  The atom's
// pair rows arrive in 32-row pieces by double-buffered bulk copies: the copy of the next
// piece is in flight while the current one is used.
// One entry's share of Eq. bec_2: z = 1/2 r_ij (x) a_ij (h = r_ij / 2; row-major, the first index
// from r), added to the central atom's registers and subtracted from atom j's accumulator.
__device__ __forceinline__ void bec_entry(float4* __restrict__ zsum, int j, int lane, float hx, float hy, float hz,
                                          float ax, float ay, float az, float zi[9]) {
    const float z0 = hx * ax, z1 = hx * ay, z2 = hx * az, z3 = hy * ax, z4 = hy * ay, z5 = hy * az, z6 = hz * ax,
                z7 = hz * ay, z8 = hz * az;
    zi[0] += z0; zi[1] += z1; zi[2] += z2; zi[3] += z3; zi[4] += z4;
    zi[5] += z5; zi[6] += z6; zi[7] += z7; zi[8] += z8;
    float4* zj = zsum + (size_t)j * 3 * CG + lane;
    atomicAdd(&zj[0], make_float4(-z0, -z1, -z2, -z3));
    atomicAdd(&zj[CG], make_float4(-z4, -z5, -z6, -z7));
    atomicAdd(reinterpret_cast<float*>(&zj[2 * CG]), -z8);
}

// BEC = false: the forces (and, with VIR, the virial) of atom m's entries from the adjoint
// lambda_i = dU_i/dD + (phi_i - mean phi) dq_i/dD.  BEC = true: the same contraction with the
// charge adjoint kappa_i = sqrt(eps_inf) dq_i/dD gives the per-entry charge derivatives
// a_ij = dq~_i/dr_ij, scattered as Eq. bec_2: Z_i += 1/2 r_ij (x) a_ij, Z_j -= 1/2 r_ij (x) a_ij
// (first index the polarization component), plus the diagonal q~^c_i of atom m (zsum, three
// float4 per atom and candidate: Z_xx..Z_yx | Z_yy..Z_zy | Z_zz, -, -, -).
template <bool VIR, bool BEC = false>
__device__ __forceinline__ void backward_atom(const BatchArgs& a, int off, int n, int m,
                                              const float* __restrict__ prm, float* __restrict__ wb,
                                              uint64_t* bars, uint32_t& par, const float* __restrict__ A,
                                              const float* __restrict__ duq, const float* __restrict__ qcs,
                                              const float4* __restrict__ fk, const float4* __restrict__ fr,
                                              float4* __restrict__ fsum, int nmax, float selfc, float phibar,
                                              double* __restrict__ vw, float seps = 0.f,
                                              float4* __restrict__ zsum = nullptr) {
    static_assert(!(VIR && BEC), "the BEC pass carries no virial");
    const int lane = threadIdx.x & 31;
    const int S = a.lay.n_species;
    float zi[9];   // BEC: this atom's own share of its entries' Z terms
    if (BEC) {
#pragma unroll
        for (int q = 0; q < 9; ++q) zi[q] = 0.f;
    }
    // virial of this atom's entries: W -= r_ij (x) F_ij (the partial force F_ij acts on i, -F_ij
    // on j); the radial part is symmetric (F_ij along u_ij)
    float wv[9], wr[3];
    if (VIR) {
#pragma unroll
        for (int q = 0; q < 9; ++q) wv[q] = 0.f;
        wr[0] = wr[1] = wr[2] = 0.f;
    }
    int* cum = reinterpret_cast<int*>(wb + WCUM);
    species_cum(a, off, n, m, S, cum);
    const int tot_a = cum[8 + S];
    const float* rad_src = a.geo_rad + (size_t)(off + m) * a.cap_l * GR;
    const float* ang_src = a.geo_ang + (size_t)(off + m) * a.cap_a * GA;
    // first job and its copy
    int kind = 0, tj = 0, base = 0;
    job_settle(cum, S, kind, tj, base);
    int b = 0;
    if (kind != 2 && lane == 0) {
        const int cnt = kind == 0 ? min(RPIECE, cum[tj + 1] - base) : min(32, tot_a - base);
        warp_bulk(wb, kind == 0 ? rad_src + (size_t)base * GR : ang_src + (size_t)base * GA,
                  (uint32_t)(cnt * (kind == 0 ? GR : GA) * 4), &bars[0]);
    }

    const float qc = qcs[(size_t)m * CG + lane];
    const float4 kf = fk[(size_t)lane * nmax + m];
    const float4 rf = fr[(size_t)m * CG + lane];
    const float wq = (kf.x + rf.x + selfc * qc) - phibar;
    float lam[NDES];
    const float* dd = duq + (size_t)m * 2 * NDES * CG + lane;
#pragma unroll
    for (int v = 0; v < NDES; ++v) lam[v] = BEC ? seps * dd[(NDES + v) * CG] : fmaf(wq, dd[(NDES + v) * CG], dd[v * CG]);
    // Phi_{n,lm} = d(lambda . D)/dA_{n,lm}
    float Phi[NA][NLM];
    const float* Ai = A + (size_t)m * NANG * CG + lane;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
#pragma unroll
        for (int M = 0; M < NLM; ++M) {
            const int l = M < 3 ? 0 : (M < 8 ? 1 : (M < 15 ? 2 : 3));
            Phi[q][M] = 2.f * c_wlm[M] * Ai[(q * NLM + M) * CG] * lam[NR + l * NA + q];
        }
        float a2[5], t[6], t2[6];
#pragma unroll
        for (int kk = 0; kk < 5; ++kk) a2[kk] = Ai[(q * NLM + 3 + kk) * CG];
        tensor_from_a(a2, t);
        tensor_square(t, t2);
        const float l4 = lam[NR + 4 * NA + q];
        Phi[q][3] = fmaf(l4, 3.f * (t2[2] * (1.f / 3.f) - (t2[0] + t2[1]) * (1.f / 6.f)), Phi[q][3]);
        Phi[q][4] = fmaf(l4, 6.f * t2[4], Phi[q][4]);
        Phi[q][5] = fmaf(l4, 6.f * t2[5], Phi[q][5]);
        Phi[q][6] = fmaf(l4, 1.5f * (t2[0] - t2[1]), Phi[q][6]);
        Phi[q][7] = fmaf(l4, 6.f * t2[3], Phi[q][7]);
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float mu[KR];
    int mu_tj = -1;
    while (kind != 2) {
        int k2 = kind, t2 = tj, b2 = base + (kind == 0 ? RPIECE : 32);
        job_settle(cum, S, k2, t2, b2);
        __syncwarp();   // every lane is done with the other buffer (previous piece)
        if (k2 != 2 && lane == 0) {
            const int cnt = k2 == 0 ? min(RPIECE, cum[t2 + 1] - b2) : min(32, tot_a - b2);
            warp_bulk(b ? wb : wb + WBUF, k2 == 0 ? rad_src + (size_t)b2 * GR : ang_src + (size_t)b2 * GA,
                      (uint32_t)(cnt * (k2 == 0 ? GR : GA) * 4), &bars[b ^ 1]);
        }
        const bool ok = warp_wait(bars, b, par, a.status);
        const float* rows = b ? wb + WBUF : wb;
        if (ok && kind == 0) {
            // radial: F_ij = (sum_k mu_k f'_k(r)) u, mu_k = sum_n lambda_n c^R[t_i][t_j][n][k]
            if (tj != mu_tj) {
#pragma unroll
                for (int k = 0; k < KR; ++k) {
                    float x = 0.f;
#pragma unroll
                    for (int q = 0; q < NR; ++q) x = fmaf(lam[q], prm[PR_R + ((tj * NR + q) * KR + k) * CG + lane], x);
                    mu[k] = x;
                }
                mu_tj = tj;
            }
            const int cntc = min(RPIECE, cum[tj + 1] - base);
            // four rows per iteration: independent chains (rows past the piece are skipped)
            for (int r0 = 0; r0 < cntc; r0 += 4) {
                float Fv[4][3], hv[4][3];
                int jv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = min(r0 + u, cntc - 1);
                    const float4* rw = reinterpret_cast<const float4*>(rows + r * GR);
                    const float4 d0 = rw[0], d1 = rw[1], d2 = rw[2], d3 = rw[3];   // f'_0..8 | u | j
                    jv[u] = r0 + u < cntc ? __float_as_int(d3.x) : -1;
                    float sv = mu[0] * d0.x;
                    sv = fmaf(mu[1], d0.y, sv);
                    sv = fmaf(mu[2], d0.z, sv);
                    sv = fmaf(mu[3], d0.w, sv);
                    sv = fmaf(mu[4], d1.x, sv);
                    sv = fmaf(mu[5], d1.y, sv);
                    sv = fmaf(mu[6], d1.z, sv);
                    sv = fmaf(mu[7], d1.w, sv);
                    sv = fmaf(mu[8], d2.x, sv);
                    Fv[u][0] = sv * d2.y;
                    Fv[u][1] = sv * d2.z;
                    Fv[u][2] = sv * d2.w;
                    if (BEC) {
                        const float h = 0.5f * rw[4].z;   // r_ij / 2 along u
                        hv[u][0] = h * d2.y;
                        hv[u][1] = h * d2.z;
                        hv[u][2] = h * d2.w;
                    }
                    if (VIR) {
                        const float rsv = r0 + u < cntc ? rw[4].z * sv : 0.f;   // r sv (row past the piece: 0)
                        wv[0] = fmaf(-rsv * d2.y, d2.y, wv[0]);
                        wv[4] = fmaf(-rsv * d2.z, d2.z, wv[4]);
                        wv[8] = fmaf(-rsv * d2.w, d2.w, wv[8]);
                        wr[0] = fmaf(-rsv * d2.y, d2.z, wr[0]);
                        wr[1] = fmaf(-rsv * d2.y, d2.w, wr[1]);
                        wr[2] = fmaf(-rsv * d2.z, d2.w, wr[2]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (jv[u] < 0) continue;
                    if (BEC) {
                        bec_entry(zsum, jv[u], lane, hv[u][0], hv[u][1], hv[u][2], Fv[u][0], Fv[u][1], Fv[u][2], zi);
                        continue;
                    }
                    fx += Fv[u][0];
                    fy += Fv[u][1];
                    fz += Fv[u][2];
                    atomicAdd(&fsum[(size_t)jv[u] * CG + lane], make_float4(-Fv[u][0], -Fv[u][1], -Fv[u][2], 0.f));
                }
            }
        } else if (ok) {
            // angular: per entry the contraction of Phi with d(g_n Y_lm)/dr_ij
            const int cntc = min(32, tot_a - base);
            for (int t = 0; t < S; ++t) {
                const int lo = max(cum[8 + t] - base, 0), hi = min(cum[8 + t + 1] - base, cntc);
                const float4* cA4 = reinterpret_cast<const float4*>(prm + PR_A + (t * CG + lane) * CA_STRIDE);
                for (int r = lo; r < hi; ++r) {
                    // row: f_0..8 | f'_0..8 | u | 1/r | j | pad | Y_lm (GA = 48 floats, 16-byte aligned)
                    const float4* r4 = reinterpret_cast<const float4*>(rows + r * GA);
                    const float4 a0 = r4[0], a1 = r4[1], a2 = r4[2], a3 = r4[3], a4 = r4[4], a5 = r4[5];
                    const float fv[KA] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x};
                    const float dfv[KA] = {a2.y, a2.z, a2.w, a3.x, a3.y, a3.z, a3.w, a4.x, a4.y};
                    float cc[4 * ((NA * KA + 3) / 4)];
#pragma unroll
                    for (int u = 0; u < (NA * KA + 3) / 4; ++u) {
                        const float4 v = cA4[u];
                        cc[4 * u] = v.x;
                        cc[4 * u + 1] = v.y;
                        cc[4 * u + 2] = v.z;
                        cc[4 * u + 3] = v.w;
                    }
                    float gn[NA], dgn[NA];
#pragma unroll
                    for (int q = 0; q < NA; ++q) {
                        float x = 0.f, y = 0.f;
#pragma unroll
                        for (int k = 0; k < KA; ++k) {
                            const float c = cc[q * KA + k];
                            x = fmaf(c, fv[k], x);
                            y = fmaf(c, dfv[k], y);
                        }
                        gn[q] = x;
                        dgn[q] = y;
                    }
                    float Y[NLM];
#pragma unroll
                    for (int g4 = 0; g4 < NLM / 4; ++g4) {
                        const float4 yv = r4[6 + g4];
                        Y[4 * g4] = yv.x;
                        Y[4 * g4 + 1] = yv.y;
                        Y[4 * g4 + 2] = yv.z;
                        Y[4 * g4 + 3] = yv.w;
                    }
                    float psi[NLM];
#pragma unroll
                    for (int M = 0; M < NLM; ++M) psi[M] = 0.f;
                    float rho = 0.f;
#pragma unroll
                    for (int q = 0; q < NA; ++q) {
                        float pq = 0.f;
#pragma unroll
                        for (int M = 0; M < NLM; ++M) {
                            pq = fmaf(Phi[q][M], Y[M], pq);
                            psi[M] = fmaf(gn[q], Phi[q][M], psi[M]);
                        }
                        rho = fmaf(dgn[q], pq, rho);
                    }
                    const float ux = a4.z, uy = a4.w, uz = a5.x, ir = a5.y;
                    float gx, gy, gz;
                    harmonics_grad(ux, uy, uz, psi, gx, gy, gz);
                    const float gu = gx * ux + gy * uy + gz * uz;
                    const float Fx = rho * ux + (gx - gu * ux) * ir;
                    const float Fy = rho * uy + (gy - gu * uy) * ir;
                    const float Fz = rho * uz + (gz - gu * uz) * ir;
                    if (BEC) {
                        const float h = 0.5f / ir;   // r_ij / 2 along u
                        bec_entry(zsum, __float_as_int(a5.z), lane, h * ux, h * uy, h * uz, Fx, Fy, Fz, zi);
                        continue;
                    }
                    fx += Fx;
                    fy += Fy;
                    fz += Fz;
                    atomicAdd(&fsum[(size_t)__float_as_int(a5.z) * CG + lane], make_float4(-Fx, -Fy, -Fz, 0.f));
                    if (VIR) {
                        const float rr = 1.f / ir, vx = ux * rr, vy = uy * rr, vz = uz * rr;
                        wv[0] = fmaf(-vx, Fx, wv[0]);
                        wv[1] = fmaf(-vx, Fy, wv[1]);
                        wv[2] = fmaf(-vx, Fz, wv[2]);
                        wv[3] = fmaf(-vy, Fx, wv[3]);
                        wv[4] = fmaf(-vy, Fy, wv[4]);
                        wv[5] = fmaf(-vy, Fz, wv[5]);
                        wv[6] = fmaf(-vz, Fx, wv[6]);
                        wv[7] = fmaf(-vz, Fy, wv[7]);
                        wv[8] = fmaf(-vz, Fz, wv[8]);
                    }
                }
            }
        }
        kind = k2;
        tj = t2;
        base = b2;
        b ^= 1;
    }
    __syncwarp();   // buffers and counts are reused by the warp's next atom
    if (BEC) {
        // own share plus the diagonal q~^c_i = sqrt(eps_inf) q^c_i
        const float qt = seps * qc;
        float4* zm = zsum + (size_t)m * 3 * CG + lane;
        atomicAdd(&zm[0], make_float4(zi[0] + qt, zi[1], zi[2], zi[3]));
        atomicAdd(&zm[CG], make_float4(zi[4] + qt, zi[5], zi[6], zi[7]));
        atomicAdd(reinterpret_cast<float*>(&zm[2 * CG]), zi[8] + qt);
        return;
    }
    // own force: network part plus the static electrostatic forces q F^k/q + F^r
    atomicAdd(&fsum[(size_t)m * CG + lane],
              make_float4(fx + fmaf(qc, kf.y, rf.y), fy + fmaf(qc, kf.z, rf.z), fz + fmaf(qc, kf.w, rf.w), 0.f));
    if (VIR) {
        // FP32 over the atom's entries, FP64 across atoms (this warp's slot, lane = candidate)
        wv[1] += wr[0];
        wv[3] += wr[0];
        wv[2] += wr[1];
        wv[6] += wr[1];
        wv[5] += wr[2];
        wv[7] += wr[2];
#pragma unroll
        for (int q = 0; q < 9; ++q) vw[q * CG + lane] += (double)wv[q];
    }
}

template <int NW, bool TC, bool VIR, bool BEC>
__global__ void __launch_bounds__(NW * 32, 8 / NW) k_batch_items(BatchArgs a) {
    static_assert(!TC || NW == 8, "the tensor-core descriptor contraction uses 8 warps");
    static_assert(!BEC || VIR, "the BEC form is built on the virial form");
    extern __shared__ __align__(128) unsigned char bsm[];
    __shared__ int s_item;
    __shared__ __align__(8) uint64_t wbars[NW][2];   // per-warp barriers of the two row buffers
    __shared__ __align__(8) uint64_t tbars[2];       // block barriers of the two S(k) / field tiles
    __shared__ __align__(8) uint64_t tcbars[4];      // tensor-core form: two operand buffers, two accumulators
    __shared__ uint32_t s_tmem;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        mbar_init(&wbars[warp][0], 1);
        mbar_init(&wbars[warp][1], 1);
        if (warp == 0) {
            mbar_init(&tbars[0], 1);
            mbar_init(&tbars[1], 1);
            if (TC)
                for (int q = 0; q < 4; ++q) mbar_init(&tcbars[q], 1);
        }
        mbar_init_fence();
    }
    if (TC && warp == 0) tmem_alloc(&s_tmem, TC_COLS);   // one block per SM (shared memory > half an SM)
    if (TC) {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    uint32_t par = 0;    // phase bits of this warp's two buffers
    uint32_t tpar = 0;   // phase bits of the two block tiles
    uint32_t tcpar = 0;  // phase bits of the tensor-core barriers
    bool tc_fail = false;
    double* red = reinterpret_cast<double*>(bsm);     // [NW][CG]
    double* sums = red + NW * CG;                      // [NSUMS][CG]
    float* cst = reinterpret_cast<float*>(sums + NSUMS * CG);   // delta, phibar, q_target, pad [4][CG]
    float* un = cst + 4 * CG;                          // union of the phases' working sets
    const int S = a.lay.n_species;
    const size_t slot = blockIdx.x;
    float* A = a.sc.A + slot * a.sc.stride_A;
    float* duq = a.sc.duq + slot * a.sc.stride_duq;
    float2* uq = a.sc.uq + slot * a.sc.stride_n;
    float* qcs = a.sc.qc + slot * a.sc.stride_n;
    float4* fk = a.sc.fk + slot * a.sc.stride_n;
    float4* fr = a.sc.fr + slot * a.sc.stride_n;
    float4* fsum = a.sc.fsum + slot * a.sc.stride_n;
    float2* sk = a.sc.sk + slot * a.sc.stride_k;
    float2* skp = a.sc.skp + slot * a.sc.stride_p;
    double* vacc = VIR ? a.sc.vir + slot * (size_t)NW * 9 * CG : nullptr;   // virial [NW][9][CG] FP64
    float4* zsum = BEC ? a.sc.zsum + slot * 3 * a.sc.stride_n : nullptr;     // BEC [nmax][3][CG] float4
    const int nmax = (int)(a.sc.stride_n / CG);
    const float selfc = a.mode == 1 ? -2.f * KE * a.alpha * 0.564189583547756287f : 0.f;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.work, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= a.n_items) break;
        const int2 item = a.items[it];
        const BatchStruct bs = a.st[item.x];
        const int grp = item.y, n = bs.n, off = bs.atom_off;
        const int cand = grp * CG + lane;
        const float* pg = a.pt + (size_t)grp * a.lay.total * CG;
        const int* so = a.spec_off + item.x * (MAX_SPECIES + 1);
        for (int i = threadIdx.x; i < n * CG; i += NW * 32) fsum[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (BEC)
            for (int i = threadIdx.x; i < 3 * n * CG; i += NW * 32) zsum[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (VIR)
            for (int i = threadIdx.x; i < NW * 9 * CG; i += NW * 32) vacc[i] = 0.0;

        // 1 forward, one species block at a time: descriptor with c^R, c^A staged, then the
        // network with its weights staged (two atoms per weight load)
        double su = 0.0, sq = 0.0;
        for (int ti = 0; ti < S; ++ti) {
            const int p0 = so[ti], p1 = so[ti + 1];
            if (p1 == p0) continue;
            __syncthreads();
            if constexpr (TC) {
                if (!forward_tc(pg, a.lay, ti, p0, p1, a.order + off, a.bimg + (size_t)off * BIMG_BYTES,
                                a.bsum + (size_t)off * a.bstride, a.bstride, reinterpret_cast<unsigned char*>(un),
                                s_tmem, TcBars{&tcbars[0], &tcbars[2]}, tcpar, A, duq, a.status,
                                a.contract != BATCH_CONTRACT_BF16))
                    tc_fail = true;
                __syncthreads();
                stage_network(pg, a.lay, ti, un);
                __syncthreads();
                for (int p = p0 + 2 * warp; p < p1; p += 2 * NW)
                    network_pair(un, a.order[off + p], p + 1 < p1 ? a.order[off + p + 1] : -1, duq, uq, su, sq);
                continue;
            }
            stage_params(pg, a.lay, ti, un);
            __syncthreads();
            float* wb = un + PARAM_FLOATS + warp * WARP_FLOATS;
            // basis sums of the warp's atoms by double-buffered bulk copies
            const uint32_t bs_bytes = (uint32_t)a.bstride * 4u;
            int bsel = 0;
            if (p0 + warp < p1 && lane == 0)
                warp_bulk(wb, a.bsum + (size_t)(off + a.order[off + p0 + warp]) * a.bstride, bs_bytes, &wbars[warp][0]);
            for (int p = p0 + warp; p < p1; p += NW) {
                __syncwarp();
                if (p + NW < p1 && lane == 0)
                    warp_bulk(bsel ? wb : wb + WBUF, a.bsum + (size_t)(off + a.order[off + p + NW]) * a.bstride,
                              bs_bytes, &wbars[warp][bsel ^ 1]);
                warp_wait(wbars[warp], bsel, par, a.status);
                descriptor_atom(a, bs, a.order[off + p], un, bsel ? wb + WBUF : wb, A, duq);
                bsel ^= 1;
            }
            __syncthreads();
            stage_network(pg, a.lay, ti, un);
            __syncthreads();
            for (int p = p0 + 2 * warp; p < p1; p += 2 * NW)
                network_pair(un, a.order[off + p], p + 1 < p1 ? a.order[off + p + 1] : -1, duq, uq, su, sq);
        }
        block_sum<NW>(su, red, sums + 0 * CG);
        block_sum<NW>(sq, red, sums + 4 * CG);
        if (warp == 0) {
            const float seps = __ldg(&pg[(size_t)a.lay.sqrt_eps * CG + lane]);
            const float qt = a.q_total / seps;
            cst[lane] = (float)(((double)qt - sums[4 * CG + lane]) / (double)n);
            cst[2 * CG + lane] = qt;
        }
        __syncthreads();
        // 2 corrected charges q^c = q + (Q / sqrt(eps_inf) - sum q) / N
        for (int i = threadIdx.x; i < n * CG; i += NW * 32) qcs[i] = uq[i].y + cst[i & 31];
        __syncthreads();

        // 3 structure factor: lanes over 32 wave vectors (4 chunks of 8); the charges and phase
        // rows of each 64-atom tile are staged in shared memory; FP32 partial sums over 512
        // atoms go to the slot's partial buffer and are added in FP64 (lane = candidate)
        const BatchKTab kt = a.kt[bs.ktab];
        const float2* phb = a.phase + (size_t)off * a.nph_stride;
        const int nkp = 8 * kt.nchunk;
        double ek = 0.0;
        // lane = candidate, for the real wave vectors 32 task .. 32 task + 31 (the warp, after its
        // partial sums): S in FP64 over the nfl partial sums, U^k += (w/2)|S|^2, the FP32 copy C = w S
        // (w = 4 k_e G(k)) and the k-space virial
        auto sk_finalize = [&](int task, int nfl) {
            for (int kk = 0; kk < 32; ++kk) {
                const int vk = task * 32 + kk;
                if (vk >= kt.nkr) break;
                const int kl = __ldg(&a.kreal[kt.kreal_off + vk]);
                const float w = __ldg(&a.kvec[8 * (size_t)kt.chunk_off + kl]).w;
                double Sr = 0.0, Si = 0.0;
                for (int f = 0; f < nfl; ++f) {
                    const float2 v = skp[((size_t)f * nkp + kl) * CG + lane];
                    Sr += (double)v.x;
                    Si += (double)v.y;
                }
                ek += 0.5 * (double)w * (Sr * Sr + Si * Si);
                sk[(size_t)kl * CG + lane] = make_float2((float)((double)w * Sr), (float)((double)w * Si));
                if (VIR) {
                    // W^k += e (I - (2 / (4 alpha^2) + 2 / k^2) k k^T), e = 2 k_e G |S|^2 (Sec. II.C)
                    const float4 kv = __ldg(&a.kvec[8 * (size_t)kt.chunk_off + kl]);
                    const double e = 0.5 * (double)w * (Sr * Sr + Si * Si);
                    const float fac = 2.f / (4.f * a.alpha * a.alpha) + 2.f / (kv.x * kv.x + kv.y * kv.y + kv.z * kv.z);
                    double* vw = vacc + (size_t)warp * 9 * CG + lane;
                    const double xx = e * (double)(1.f - fac * kv.x * kv.x), yy = e * (double)(1.f - fac * kv.y * kv.y);
                    const double zz = e * (double)(1.f - fac * kv.z * kv.z), xy = e * (double)(-fac * kv.x * kv.y);
                    const double xz = e * (double)(-fac * kv.x * kv.z), yz = e * (double)(-fac * kv.y * kv.z);
                    vw[0 * CG] += xx;
                    vw[4 * CG] += yy;
                    vw[8 * CG] += zz;
                    vw[1 * CG] += xy;
                    vw[3 * CG] += xy;
                    vw[2 * CG] += xz;
                    vw[6 * CG] += xz;
                    vw[5 * CG] += yz;
                    vw[7 * CG] += yz;
                }
            }
        };
        if constexpr (TC) {   // tensor-core form: S of all wave vectors, then the FP64 finalisation
            if (!sk_tc(n, phb, a.nph_stride, kt, a.chunk + kt.chunk_off, qcs, skp, reinterpret_cast<unsigned char*>(un),
                       s_tmem, &tcbars[2], tcpar, tbars, tpar, a.status))
                tc_fail = true;
            __syncthreads();
            const int ntask = (kt.nkr + 31) >> 5;
            const int nfl = (n + SK_AT * SK_FT - 1) / (SK_AT * SK_FT);
            for (int task = warp; task < ntask; task += NW) sk_finalize(task, nfl);
        } else {
            // tile buffer b: charges [QT][CG] | phase rows [QT][nph_stride]; tile T of the
            // (task round, atom tile) sequence is copied while tile T - 1 is summed
            const int ps = a.nph_stride;
            const int tile_f = QT * CG + 2 * QT * ps;
            const int ntask = (kt.nkr + 31) >> 5;   // 32 wave vectors per task, padding left out
            const int nfl = (n + QT * FLUSH_TILES - 1) / (QT * FLUSH_TILES);
            const int ntile = (n + QT - 1) / QT;
            const int total = ((ntask + NW - 1) / NW) * ntile;
            auto issue = [&](int T) {
                const int j0 = (T % ntile) * QT, cnt = min(QT, n - j0);
                float* dst = un + (T & 1) * tile_f;
                const uint32_t qb = (uint32_t)(cnt * CG * 4), rb = (uint32_t)(cnt * ps * 8);
                fence_proxy_async_all();   // charges / C(k) were written by this block
                mbar_expect_tx(&tbars[T & 1], qb + rb);
                bulk_g2s(dst, qcs + (size_t)j0 * CG, qb, &tbars[T & 1]);
                bulk_g2s(dst + QT * CG, phb + (size_t)j0 * ps, rb, &tbars[T & 1]);
            };
            if (threadIdx.x == 0 && total > 0) issue(0);
            int T = 0;
            for (int tb = 0; tb < ntask; tb += NW) {
                const int task = tb + warp;
                const bool act = task < ntask;
                const int v = task * 32 + lane;
                const bool kval = act && v < kt.nkr;
                int kl = 0, e1 = 0, e2 = kt.yoff, e3 = kt.zoff;   // kl: padded index of the lane's k
                if (kval) {
                    kl = __ldg(&a.kreal[kt.kreal_off + v]);
                    const int4 ci = __ldg(&a.chunk[kt.chunk_off + (kl >> 3)]);
                    e1 = ci.x;
                    e2 = kt.yoff + ci.y + kt.n2max;
                    e3 = kt.zoff + ci.z + (kl & 7) + kt.n3max;
                }
                float sr[CG], si[CG];
#pragma unroll
                for (int c = 0; c < CG; ++c) {
                    sr[c] = 0.f;
                    si[c] = 0.f;
                }
                int tiles = 0, fl = 0;
                for (int j0 = 0; j0 < n; j0 += QT, ++T) {
                    const int cnt = min(QT, n - j0);
                    if (threadIdx.x == 0 && T + 1 < total) issue(T + 1);
                    const int b = T & 1;
                    const bool ok = mbar_wait_bounded(&tbars[b], (tpar >> b) & 1u);
                    tpar ^= 1u << b;
                    if (!ok && lane == 0) atomicOr(a.status, kStatusTimeout);
                    const float* qt = un + b * tile_f;
                    const float2* pt2 = reinterpret_cast<const float2*>(qt + QT * CG);
                    if (act && ok) {
                        for (int jj = 0; jj < cnt; ++jj) {
                            const float2* row = pt2 + jj * ps;
                            const float2 e = cmul(cmul(row[e1], row[e2]), row[e3]);
                            const float4* q4 = reinterpret_cast<const float4*>(qt + jj * CG);
#pragma unroll
                            for (int c4 = 0; c4 < CG / 4; ++c4) {
                                const float4 q = q4[c4];
                                sr[4 * c4 + 0] = fmaf(q.x, e.x, sr[4 * c4 + 0]);
                                si[4 * c4 + 0] = fmaf(q.x, e.y, si[4 * c4 + 0]);
                                sr[4 * c4 + 1] = fmaf(q.y, e.x, sr[4 * c4 + 1]);
                                si[4 * c4 + 1] = fmaf(q.y, e.y, si[4 * c4 + 1]);
                                sr[4 * c4 + 2] = fmaf(q.z, e.x, sr[4 * c4 + 2]);
                                si[4 * c4 + 2] = fmaf(q.z, e.y, si[4 * c4 + 2]);
                                sr[4 * c4 + 3] = fmaf(q.w, e.x, sr[4 * c4 + 3]);
                                si[4 * c4 + 3] = fmaf(q.w, e.y, si[4 * c4 + 3]);
                            }
                        }
                    }
                    if (act && (++tiles == FLUSH_TILES || j0 + QT >= n)) {
                        tiles = 0;
                        if (kval) {
                            float4* dst = reinterpret_cast<float4*>(skp + ((size_t)fl * nkp + kl) * CG);
#pragma unroll
                            for (int c = 0; c < CG; c += 2) dst[c >> 1] = make_float4(sr[c], si[c], sr[c + 1], si[c + 1]);
                        }
#pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            sr[c] = 0.f;
                            si[c] = 0.f;
                        }
                        ++fl;
                    }
                    __syncthreads();   // tile buffer b is refilled by the copy issued next iteration
                }
                if (act) {
                    __syncwarp();
                    sk_finalize(task, nfl);
                }
            }
        }
        __syncthreads();

        // 4a k-space potential and field: lanes over atoms (32 per warp task), 16 candidates per
        // pass; C(k), the wave vectors and the chunk list come in windows of KW wave vectors,
        // window W + 1 copied while window W is used (the tensor-core form: field_tc)
        if constexpr (TC) {
            if (!field_tc(n, nmax, phb, a.nph_stride, kt, a.chunk + kt.chunk_off, a.kvec + 8 * (size_t)kt.chunk_off, sk,
                          fk, reinterpret_cast<unsigned char*>(un), s_tmem, &tcbars[2], tcpar, tbars, tpar, a.status))
                tc_fail = true;
        } else {
            const int nph = kt.nph;
            float2* ph = reinterpret_cast<float2*>(un) + (size_t)warp * nph * 32;   // [nph][32 atoms]
            float2* win = reinterpret_cast<float2*>(un) + (size_t)NW * nph * 32;    // 2 x window
            const int ntask = (n + 31) >> 5;
            const int nwin = (nkp + KW - 1) / KW;
            const int total = ((ntask + NW - 1) / NW) * 2 * nwin;
            auto issue = [&](int W) {
                const int k0 = (W % nwin) * KW, kc = min(KW, nkp - k0);
                float2* sw = win + (W & 1) * WIN_F2;
                const uint32_t sb = (uint32_t)(kc * CG * 8), kb = (uint32_t)(kc * 16), cb = (uint32_t)(kc / 8 * 16);
                fence_proxy_async_all();   // charges / C(k) were written by this block
                mbar_expect_tx(&tbars[W & 1], sb + kb + cb);
                bulk_g2s(sw, sk + (size_t)k0 * CG, sb, &tbars[W & 1]);
                bulk_g2s(sw + KW * CG, a.kvec + 8 * (size_t)kt.chunk_off + k0, kb, &tbars[W & 1]);
                bulk_g2s(sw + KW * CG + 2 * KW, a.chunk + kt.chunk_off + k0 / 8, cb, &tbars[W & 1]);
            };
            if (threadIdx.x == 0 && total > 0) issue(0);
            int W = 0;
            for (int r0 = 0; r0 < ntask; r0 += NW) {
                const int task = r0 + warp;
                const bool act = task < ntask;
                const int j = task * 32 + lane;
                if (act && j < n) {
                    // lane = atom: its phase row, transposed
                    const float2* src = phb + (size_t)j * a.nph_stride;
#pragma unroll 4
                    for (int e = 0; e < nph; ++e) ph[e * 32 + lane] = __ldg(&src[e]);
                }
                __syncwarp();
                for (int c0 = 0; c0 < CG; c0 += 16) {
                    float fphi[16], ex[16], ey[16], ez[16], tt[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        fphi[c] = 0.f;
                        ex[c] = 0.f;
                        ey[c] = 0.f;
                        ez[c] = 0.f;
                        tt[c] = 0.f;
                    }
                    float pkx = 0.f, pky = 0.f;
                    int pn1 = -(1 << 30), pn2 = 0;
                    for (int k0 = 0; k0 < nkp; k0 += KW, ++W) {
                        const int kc = min(KW, nkp - k0);
                        if (threadIdx.x == 0 && W + 1 < total) issue(W + 1);
                        const int b = W & 1;
                        const bool ok = mbar_wait_bounded(&tbars[b], (tpar >> b) & 1u);
                        tpar ^= 1u << b;
                        if (!ok && lane == 0) atomicOr(a.status, kStatusTimeout);
                        const float2* sw = win + b * WIN_F2;                                   // [KW][CG]
                        const float4* kw = reinterpret_cast<const float4*>(sw + KW * CG);    // [KW]
                        const int4* cw = reinterpret_cast<const int4*>(kw + KW);             // [KW / 8]
                        if (act && ok) {
                            for (int hh = 0; hh < (kc >> 3); ++hh) {
                                const int4 ci = cw[hh];
                                if (ci.x != pn1 || ci.y != pn2) {
                                    // new column (n1, n2): fold the column's Im sums into E_x, E_y
#pragma unroll
                                    for (int c = 0; c < 16; ++c) {
                                        ex[c] = fmaf(pkx, tt[c], ex[c]);
                                        ey[c] = fmaf(pky, tt[c], ey[c]);
                                        tt[c] = 0.f;
                                    }
                                    pn1 = ci.x;
                                    pn2 = ci.y;
                                    const float4 k0v = kw[hh * 8];
                                    pkx = k0v.x;
                                    pky = k0v.y;
                                }
                                const float2 xy =
                                    cmul(ph[ci.x * 32 + lane], ph[(kt.yoff + ci.y + kt.n2max) * 32 + lane]);
                                // the chunk's entries that are not padding (C of padding is not written)
#pragma unroll
                                for (int t = 0; t < 8; ++t) {
                                    if (t >= ci.w) break;
                                    const float4 k4 = kw[hh * 8 + t];
                                    const float2 e = cmul(xy, ph[(kt.zoff + ci.z + t + kt.n3max) * 32 + lane]);
                                    // Re and Im of C conj(e) accumulated term by term, the k_z
                                    // factor folded into the phase: six FMAs per candidate
                                    const float ney = -e.y, zx = k4.z * e.x, zy = -k4.z * e.y;
                                    const float4* s4 = reinterpret_cast<const float4*>(sw + (hh * 8 + t) * CG + c0);
#pragma unroll
                                    for (int u = 0; u < 8; ++u) {
                                        const float4 v = s4[u];   // C of two candidates
                                        fphi[2 * u] = fmaf(v.y, e.y, fmaf(v.x, e.x, fphi[2 * u]));
                                        tt[2 * u] = fmaf(v.x, ney, fmaf(v.y, e.x, tt[2 * u]));
                                        ez[2 * u] = fmaf(v.x, zy, fmaf(v.y, zx, ez[2 * u]));
                                        fphi[2 * u + 1] = fmaf(v.w, e.y, fmaf(v.z, e.x, fphi[2 * u + 1]));
                                        tt[2 * u + 1] = fmaf(v.z, ney, fmaf(v.w, e.x, tt[2 * u + 1]));
                                        ez[2 * u + 1] = fmaf(v.z, zy, fmaf(v.w, zx, ez[2 * u + 1]));
                                    }
                                }
                            }
                        }
                        __syncthreads();   // window buffer b is refilled by the copy issued next iteration
                    }
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        ex[c] = fmaf(pkx, tt[c], ex[c]);
                        ey[c] = fmaf(pky, tt[c], ey[c]);
                    }
                    if (act && j < n) {
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            fk[(size_t)(c0 + c) * nmax + j] = make_float4(fphi[c], ex[c], ey[c], ez[c]);
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();

        // 4b real space (lanes over candidates, pair rows from the pre-pass) and the potential sums
        double er = 0.0, sphi = 0.0, sq2 = 0.0;
        {
            // the structure's corrected charges staged in shared memory where they fit (each list
            // entry reads its neighbour's 32 candidate charges), the warps' row buffers after them
            const bool qsm = a.mode == 1 && (size_t)n * CG + (size_t)NW * RS_WARP <= (size_t)a.inv_cap;
            const float* qs = qsm ? un : qcs;
            float* tab = qsm ? un + (size_t)n * CG + warp * RS_WARP : un + PARAM_FLOATS + warp * WARP_FLOATS;
            int* cum = reinterpret_cast<int*>(tab + (qsm ? RS_CUM : WCUM));
            if (qsm) {
                const float4* src = reinterpret_cast<const float4*>(qcs);
                float4* dst = reinterpret_cast<float4*>(un);
                for (int i = threadIdx.x; i < n * CG / 4; i += NW * 32) dst[i] = src[i];
                __syncthreads();
            }
            for (int m = warp; m < n; m += NW) {
                const float qi = qs[(size_t)m * CG + lane];
                float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
                float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
                if (a.mode == 1) {
                    species_cum(a, off, n, m, S, cum);
                    const int tot_l = cum[S];
                    const float4* grows = reinterpret_cast<const float4*>(a.geo_rad + (size_t)(off + m) * a.cap_l * GR);
                    // pieces of 32 rows, double-buffered: the copy of piece p + 1 overlaps piece p
                    if (tot_l > 0 && lane == 0)
                        warp_bulk(tab, grows, (uint32_t)(min(32, tot_l) * GR * 4), &wbars[warp][0]);
                    int rb = 0;
                    for (int base = 0; base < tot_l; base += 32, rb ^= 1) {
                        const int cntc = min(32, tot_l - base);
                        __syncwarp();   // the warp is done with the other buffer (previous piece)
                        if (base + 32 < tot_l && lane == 0)
                            warp_bulk(tab + (rb ^ 1) * RS_BUF, grows + (size_t)(base + 32) * (GR / 4),
                                      (uint32_t)(min(32, tot_l - base - 32) * GR * 4), &wbars[warp][rb ^ 1]);
                        if (!warp_wait(wbars[warp], rb, par, a.status)) continue;
                        const float* rows = tab + rb * RS_BUF;
                        // four rows per iteration, their charge loads issued together; rows past
                        // the piece and pairs beyond r_c contribute q_j = 0
                        for (int r0 = 0; r0 < cntc; r0 += 4) {
                            float4 d3[4];
                            float bz[4], qj[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int r = min(r0 + u, cntc - 1);
                                const float4* rw = reinterpret_cast<const float4*>(rows + r * GR);
                                const float4 d4 = rw[4];   // (B'u_z, j_real, r, -)
                                d3[u] = rw[3];             // (j_desc, B, B'u_x, B'u_y)
                                bz[u] = d4.x;
                                const int j = __float_as_int(d4.y);
                                qj[u] = (j >= 0 && r0 + u < cntc) ? qs[(size_t)j * CG + lane] : 0.f;
                                if (VIR) {
                                    // pair virial: sum_j q_j B'(r) r u (x) u, with B' u from the row
                                    const float4 d2 = rw[2];   // (f'_8, u)
                                    const float t = qj[u] * d4.z;
                                    sxx = fmaf(t * d3[u].z, d2.y, sxx);
                                    syy = fmaf(t * d3[u].w, d2.z, syy);
                                    szz = fmaf(t * d4.x, d2.w, szz);
                                    sxy = fmaf(t * d3[u].z, d2.z, sxy);
                                    sxz = fmaf(t * d3[u].z, d2.w, sxz);
                                    syz = fmaf(t * d3[u].w, d2.w, syz);
                                }
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                ph = fmaf(qj[u], d3[u].y, ph);
                                gx = fmaf(qj[u], d3[u].z, gx);
                                gy = fmaf(qj[u], d3[u].w, gy);
                                gz = fmaf(qj[u], bz[u], gz);
                            }
                        }
                    }
                }
                // F^r_i = sum_j q_i q_j B'(r) u_ij (u_ij from i to j)
                fr[(size_t)m * CG + lane] = make_float4(ph, qi * gx, qi * gy, qi * gz);
                if (VIR && a.mode == 1) {
                    // W^r -= 1/2 sum_j r_ij (x) F^r_ij over the full list (each pair seen twice)
                    double* vw = vacc + (size_t)warp * 9 * CG + lane;
                    const double h = -0.5 * (double)qi;
                    vw[0 * CG] += h * (double)sxx;
                    vw[4 * CG] += h * (double)syy;
                    vw[8 * CG] += h * (double)szz;
                    vw[1 * CG] += h * (double)sxy;
                    vw[3 * CG] += h * (double)sxy;
                    vw[2 * CG] += h * (double)sxz;
                    vw[6 * CG] += h * (double)sxz;
                    vw[5 * CG] += h * (double)syz;
                    vw[7 * CG] += h * (double)syz;
                }
                const float4 kf = fk[(size_t)lane * nmax + m];
                sphi += (double)ph + (double)kf.x;
                er += 0.5 * (double)qi * (double)ph;
                sq2 += (double)qi * (double)qi;
            }
        }
        block_sum<NW>(ek, red, sums + 1 * CG);
        block_sum<NW>(er, red, sums + 2 * CG);
        block_sum<NW>(sq2, red, sums + 3 * CG);
        block_sum<NW>(sphi, red, sums + 5 * CG);
        if (warp == 0)
            cst[CG + lane] = (float)((sums[5 * CG + lane] + (double)selfc * (double)cst[2 * CG + lane]) / (double)n);
        __syncthreads();

        // 5 backward, one species block at a time
        for (int ti = 0; ti < S; ++ti) {
            const int p0 = so[ti], p1 = so[ti + 1];
            if (p1 == p0) continue;
            __syncthreads();
            stage_params_bwd(pg, a.lay, ti, un);
            __syncthreads();
            float* wb = un + PARAM_FLOATS + warp * WARP_FLOATS;
            const float phibar = cst[CG + lane];
            for (int p = p0 + warp; p < p1; p += NW)
                backward_atom<VIR>(a, off, n, a.order[off + p], un, wb, wbars[warp], par, A, duq, qcs, fk, fr, fsum,
                                   nmax, selfc, phibar, vacc + (size_t)warp * 9 * CG);
        }
        if constexpr (BEC) {
            // 5b Born effective charges (Eq. bec_2): the same entry contractions with the charge
            // adjoint kappa = sqrt(eps_inf) dq/dD, scattered as Z terms
            const float seps = __ldg(&pg[(size_t)a.lay.sqrt_eps * CG + lane]);
            for (int ti = 0; ti < S; ++ti) {
                const int p0 = so[ti], p1 = so[ti + 1];
                if (p1 == p0) continue;
                __syncthreads();
                stage_params_bwd(pg, a.lay, ti, un);
                __syncthreads();
                float* wb = un + PARAM_FLOATS + warp * WARP_FLOATS;
                for (int p = p0 + warp; p < p1; p += NW)
                    backward_atom<false, true>(a, off, n, a.order[off + p], un, wb, wbars[warp], par, A, duq, qcs, fk,
                                               fr, fsum, nmax, selfc, 0.f, nullptr, seps, zsum);
            }
        }
        __syncthreads();

        // 6 outputs in input order, candidate-major: lanes over consecutive input atoms (through the
        // inverse of the sort permutation), so each warp writes contiguous rows of the outputs
        const bool zout = BEC && a.bec;
        // a general cell rotated into the restricted form: forces and BEC back to the input frame
        const float* Rot = (a.rot && a.rot[12 * item.x + 9] != 0.f) ? a.rot + 12 * item.x : nullptr;
        if ((a.forces || a.charges || zout) && n > a.inv_cap) {   // a structure too large for the permutation
            for (int i = threadIdx.x; i < n * CG; i += NW * 32) {
                const int m = i >> 5, c = grp * CG + (i & 31);
                if (c >= a.n_cand) continue;
                const size_t gi = (size_t)off + __ldg(&a.sidx[off + m]);
                if (a.forces) {
                    float4 F = fsum[i];
                    if (Rot) F = rot_back_vec(Rot, F);
                    float* fo = a.forces + ((size_t)c * a.n_total + gi) * 3;
                    fo[0] = F.x;
                    fo[1] = F.y;
                    fo[2] = F.z;
                }
                if (a.charges) a.charges[(size_t)c * a.n_total + gi] = qcs[i];
                if (zout) {
                    const float4 z0 = zsum[(size_t)(3 * m) * CG + (i & 31)], z1 = zsum[(size_t)(3 * m + 1) * CG + (i & 31)];
                    const float z8 = zsum[(size_t)(3 * m + 2) * CG + (i & 31)].x;
                    float* zo = a.bec + ((size_t)c * a.n_total + gi) * 9;
                    float zz[9] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w, z8};
                    if (Rot) rot_back_tensor(Rot, zz);
#pragma unroll
                    for (int q = 0; q < 9; ++q) zo[q] = zz[q];
                }
            }
        } else if (a.forces || a.charges || zout) {
            int* inv = reinterpret_cast<int*>(un);   // [n]: sorted index of input atom g
            for (int m = threadIdx.x; m < n; m += NW * 32) inv[__ldg(&a.sidx[off + m])] = m;
            __syncthreads();
            for (int cl = warp; cl < CG; cl += NW) {
                const int c = grp * CG + cl;
                if (c >= a.n_cand) break;
                float* fo = a.forces ? a.forces + ((size_t)c * a.n_total + off) * 3 : nullptr;
                float* qo = a.charges ? a.charges + (size_t)c * a.n_total + off : nullptr;
                float* zo = zout ? a.bec + ((size_t)c * a.n_total + off) * 9 : nullptr;
                for (int g = lane; g < n; g += 32) {
                    const int i = inv[g] * CG + cl;
                    if (fo) {
                        float4 F = fsum[i];
                        if (Rot) F = rot_back_vec(Rot, F);
                        fo[3 * g] = F.x;
                        fo[3 * g + 1] = F.y;
                        fo[3 * g + 2] = F.z;
                    }
                    if (qo) qo[g] = qcs[i];
                    if (zo) {
                        const int zm = 3 * inv[g] * CG + cl;
                        const float4 z0 = zsum[zm], z1 = zsum[zm + CG];
                        const float z8 = zsum[zm + 2 * CG].x;
                        float* zr = zo + 9 * (size_t)g;
                        float zz[9] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w, z8};
                        if (Rot) rot_back_tensor(Rot, zz);
#pragma unroll
                        for (int q = 0; q < 9; ++q) zr[q] = zz[q];
                    }
                }
            }
        }
        if (VIR && a.virial && warp == 1 && cand < a.n_cand) {
            // W = sum over the warps' FP64 slots (entries, real space, k space), per candidate;
            // R^T W R back in the input frame for a rotated cell
            double wt[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                double t = 0.0;
#pragma unroll
                for (int w = 0; w < NW; ++w) t += vacc[((size_t)w * 9 + q) * CG + lane];
                wt[q] = t;
            }
            if (Rot) {
                double o9[9];
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y) {
                        double t = 0.0;
#pragma unroll
                        for (int u = 0; u < 3; ++u)
#pragma unroll
                            for (int v = 0; v < 3; ++v) t += (double)Rot[3 * u + x] * wt[3 * u + v] * (double)Rot[3 * v + y];
                        o9[3 * x + y] = t;
                    }
#pragma unroll
                for (int q = 0; q < 9; ++q) wt[q] = o9[q];
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) a.virial[((size_t)cand * a.n_struct + item.x) * 9 + q] = wt[q];
        }
        if (warp == 0 && cand < a.n_cand) {
            double e = sums[lane] + sums[CG + lane];
            if (a.mode == 1) e += sums[2 * CG + lane] - (double)KE * (double)a.alpha * 0.564189583547756287 * sums[3 * CG + lane];
            a.energy[(size_t)cand * a.n_struct + item.x] = e;
            // predicted total charge before the correction, sum_i q~_i = sqrt(eps_inf) sum_i q_i
            if (a.total_charge)
                a.total_charge[(size_t)cand * a.n_struct + item.x] =
                    (double)__ldg(&pg[(size_t)a.lay.sqrt_eps * CG + lane]) * sums[4 * CG + lane];
        }
        if (a.polarization) {
            // P = sum_i q~^c_i r_i (Eq. polarization) over the positions as given, lanes over
            // candidates: FP32 over 8 atoms per lane, FP64 across them and across the warps
            const float seps = __ldg(&pg[(size_t)a.lay.sqrt_eps * CG + lane]);
            double pd[3] = {0.0, 0.0, 0.0};
            float pf[3] = {0.f, 0.f, 0.f};
            int np = 0;
            for (int m = warp; m < n; m += NW) {
                const float qt = seps * qcs[(size_t)m * CG + lane];
                const float* r = a.pos_in + 3 * ((size_t)off + __ldg(&a.sidx[off + m]));
#pragma unroll
                for (int d = 0; d < 3; ++d) pf[d] = fmaf(qt, __ldg(&r[d]), pf[d]);
                if (++np == 8) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        pd[d] += (double)pf[d];
                        pf[d] = 0.f;
                    }
                    np = 0;
                }
            }
            // the FP64 sums of the energy are consumed above: their slots take the three components
#pragma unroll
            for (int d = 0; d < 3; ++d) block_sum<NW>(pd[d] + (double)pf[d], red, sums + d * CG);
            if (warp == 0 && cand < a.n_cand) {
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    a.polarization[((size_t)cand * a.n_struct + item.x) * 3 + d] = sums[d * CG + lane];
            }
        }
    }
    if (TC) {
        // after a wait that gave up, give the products in flight a second bounded wait
        if (__syncthreads_or(tc_fail) && threadIdx.x == 0) {
            mbar_wait_bounded(&tcbars[2], ((tcpar >> 2) & 1u) ^ 1u);
            mbar_wait_bounded(&tcbars[3], ((tcpar >> 3) & 1u) ^ 1u);
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (warp == 0) tmem_free(s_tmem, TC_COLS);
    }
}

// the field pass at the largest phase rows fits the 227 KB of shared memory of a block
static_assert(sizeof(double) * (8 + NSUMS) * CG + sizeof(float) * 4 * CG +
                      sizeof(float2) * ((size_t)8 * BATCH_MAX_NPH * 32 + 2 * (size_t)WIN_F2) <=
                  227 * 1024,
              "field windows and phase rows exceed shared memory");

template <int NW>
size_t item_smem(int nph_max, bool tc) {   // the same with and without the virial (its sums are in global scratch)
    const size_t head = sizeof(double) * (NW + NSUMS) * CG + sizeof(float) * 4 * CG;
    const size_t p1 = tc ? std::max((size_t)TC_BYTES, sizeof(float) * ((size_t)PARAM_FLOATS + (size_t)NW * WARP_FLOATS))
                         : sizeof(float) * ((size_t)PARAM_FLOATS + (size_t)NW * WARP_FLOATS);
    const size_t p1b = sizeof(float) * (size_t)NET_FLOATS;
    const size_t p3 = tc ? (size_t)sk_smem(batch_phase_stride(nph_max))
                         : 2 * (sizeof(float) * (size_t)QT * CG + sizeof(float2) * (size_t)QT * batch_phase_stride(nph_max));
    const size_t p4 = tc ? (size_t)FT_OFF_PH + sizeof(float2) * (size_t)FT_PHS * nph_max
                         : sizeof(float2) * ((size_t)NW * nph_max * 32 + 2 * (size_t)WIN_F2);
    return head + std::max(std::max(p1, p1b), std::max(p3, p4));
}

}  // namespace

void launch_batch_prep(const float* pos, const int* types, int n_struct, int nmax, int n_species,
                       const BatchStruct* st, const BatchKTab* kt, const BatchKTri* ktri, int* cell_start, float4* spos4, int* sidx,
                       int* order, int* spec_off, int cap_l, int cap_a, int* nbr_list, int* cnt_list, int* nbr_ang,
                       int* cnt_ang, float2* phase, int nph_stride, float* geo_rad, float* geo_ang, float* bsum,
                       int bstride, unsigned char* bimg, float alpha, const float* rot, unsigned int* status,
                       cudaStream_t st_) {
    if (n_struct <= 0) return;
    const size_t sm1 = sizeof(int) * ((size_t)nmax + BATCH_MAX_CELLS + 1 + MAX_SPECIES + 1);
    const size_t sm2 = sizeof(int) * (size_t)(PREP_THREADS / 32) * (2 * cap_l + 2 * cap_a + 32 * TAB_P + 16);
    static std::atomic<int> attr1[kMaxDevices], attr2[kMaxDevices];
    if (sm1 > 48 * 1024) ensure_smem_attr(k_batch_sort, attr1, (int)sm1);
    if (sm2 > 48 * 1024) ensure_smem_attr(k_batch_lists, attr2, (int)sm2);
    k_batch_sort<<<n_struct, PREP_THREADS, sm1, st_>>>(pos, types, nmax, n_species, st, cell_start, spos4, sidx,
                                                        order, spec_off, rot, status);
    // about one warp per 32 atoms of the largest structure
    const int ysplit = std::max(1, std::min(64, (nmax + 32 * (PREP_THREADS / 32) - 1) / (32 * (PREP_THREADS / 32)) * 4));
    k_batch_lists<<<dim3(n_struct, ysplit), PREP_THREADS, sm2, st_>>>(n_species, st, kt, ktri, cell_start, spos4, cap_l, cap_a, nbr_list,
                                                         cnt_list, nbr_ang, cnt_ang, phase, nph_stride, geo_rad,
                                                         geo_ang, bsum, bstride, bimg, alpha, status);
}

size_t batch_item_smem(int warps, int nph_max, int contract) {
    const bool tc = batch_contract_tc(contract);
    return warps == 4 ? item_smem<4>(nph_max, false) : item_smem<8>(nph_max, tc);
}

namespace {
template <int NW, bool TC, bool VIR, bool BEC = false>
int blocks_per_sm_of(size_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(k_batch_items<NW, TC, VIR, BEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_items<NW, TC, VIR, BEC>, NW * 32, smem) !=
        cudaSuccess)
        nb = 0;
    return nb;
}
template <int NW, bool TC>
int blocks_per_sm_mode(size_t smem, bool virial, bool bec) {
    if (bec) return blocks_per_sm_of<NW, TC, true, true>(smem);
    return virial ? blocks_per_sm_of<NW, TC, true>(smem) : blocks_per_sm_of<NW, TC, false>(smem);
}
template <int NW, bool TC>
void launch_mode(const BatchArgs& a, int grid, size_t smem, cudaStream_t st_) {
    if (a.bec) k_batch_items<NW, TC, true, true><<<grid, NW * 32, smem, st_>>>(a);
    else if (a.virial) k_batch_items<NW, TC, true, false><<<grid, NW * 32, smem, st_>>>(a);
    else k_batch_items<NW, TC, false, false><<<grid, NW * 32, smem, st_>>>(a);
}
}  // namespace

// The tensor-core form holds 512 tensor-memory columns per block: it runs only where its
// shared memory keeps it to one block per SM (0 otherwise, like a shape that does not fit).
int batch_item_blocks_per_sm(int warps, int nph_max, int contract, bool virial, bool bec) {
    if (batch_contract_tc(contract) && warps != 8) return 0;
    const size_t smem = batch_item_smem(warps, nph_max, contract);
    int nb;
    if (warps == 4) nb = blocks_per_sm_mode<4, false>(smem, virial, bec);
    else if (batch_contract_tc(contract)) {
        nb = blocks_per_sm_mode<8, true>(smem, virial, bec);
        if (nb > 1) nb = 0;
    } else nb = blocks_per_sm_mode<8, false>(smem, virial, bec);
    return nb;
}

void launch_batch_items(const BatchArgs& a_in, int warps, int nph_max, int contract, int grid, cudaStream_t st_) {
    if (grid <= 0 || a_in.n_items <= 0) return;
    const size_t smem = batch_item_smem(warps, nph_max, contract);
    BatchArgs a = a_in;
    const size_t head = sizeof(double) * ((warps == 4 ? 4 : 8) + NSUMS) * CG + sizeof(float) * 4 * CG;
    a.inv_cap = (int)((smem - head) / sizeof(int));
    if (warps == 4) launch_mode<4, false>(a, grid, smem, st_);
    else if (batch_contract_tc(contract)) launch_mode<8, true>(a, grid, smem, st_);
    else launch_mode<8, false>(a, grid, smem, st_);
}

}  // namespace qnep
