// Per-atom electrostatic potential and static forces, and the final reductions.
//
// For every atom i (charges q^c after the total-charge correction):
//   reciprocal (Ewald, Sec. II.C):  phi^k_i = 2 k_e sum_{k != 0} G Re[S(k) e^{i k.r_i}]
//                                   F^k_i   = 2 k_e q_i sum_{k != 0} k G Im[S(k) e^{i k.r_i}]
//     evaluated over the half space with C = 4 k_e G S; per column (n1, n2)
//     the n3 sum is done first, so each (atom, k) costs one complex product.
//   real space (mode 1, Sec. II.B / II.C): phi^r_i = k_e sum_j q_j erfc(alpha r)/r and the
//     static pair force F^{r,static}_ij = -1/2 k_e q_i q_j r_ij / r^3 [2 alpha r/sqrt(pi)
//     e^{-alpha^2 r^2} + erfc(alpha r)]; F_i += F_ij - F_ji = 2 F_ij.
//   self (mode 1): phi^s_i = -2 k_e alpha / sqrt(pi) q_i (the dU^s/dq_i of Sec. II.B).
// phi_i = dU^ES/dq^c_i feeds the dynamic-charge partial forces of Sec. II.C
// through the adjoint of the backward kernel.  The kernel also initialises the
// force / BEC accumulator of each atom (static force; q~^c_i on the BEC diagonal)
// and adds the FP64 sums: sum phi, U^r = 1/2 sum q phi^r, U^s, P = sum q~^c r.
#include "qnep_internal.cuh"

namespace qnep {

namespace {

constexpr float TWO_PI = 6.28318530717958648f;
constexpr float INV_SQRT_PI = 0.564189583547756287f;

template <int W>
__global__ void __launch_bounds__(32 * W) k_field(const float4* __restrict__ pos4, const float* __restrict__ pos_in,
                                                  const float* __restrict__ q_raw, const int* __restrict__ nbr_list,
                                                  const int* __restrict__ cnt_list, int n, int n_species, Geom g,
                                                  ElecConst ec, float q_target, float seps, int ewald, EwaldTab tab,
                                                  const float* __restrict__ pppm_field, float* __restrict__ phi,
                                                  float4* __restrict__ acc12, float* __restrict__ charges_out,
                                                  Accum* __restrict__ acc) {
    extern __shared__ float2 stab[];
    __shared__ float red[W][8][33];
    __shared__ float wred[9][W];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i0 = blockIdx.x * 32;
    const int i = i0 + lane;
    const bool valid = i < n;
    const float delta = (float)(((double)q_target - acc->sum_q) / (double)n);
    if (ewald) {
        for (int idx = threadIdx.x; idx < 32 * tab.nph; idx += blockDim.x) {
            int a = idx / tab.nph;
            stab[idx] = (i0 + a < n) ? tab.phase[(size_t)i0 * tab.nph + idx] : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    const float qc = valid ? __ldg(&q_raw[i]) + delta : 0.f;
    float phk = 0.f, phr = 0.f, fk[3] = {0.f, 0.f, 0.f}, fr[3] = {0.f, 0.f, 0.f};
    float wv[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) wv[k] = 0.f;
    if (valid && ewald) {
        const float2* row = stab + lane * tab.nph;
        const float kxs = TWO_PI / tab.L[0], kys = TWO_PI / tab.L[1], kzs = TWO_PI / tab.L[2];
        for (int c = w; c < tab.ncol; c += W) {
            int4 ci = __ldg(&tab.col[c]);
            int kend = __ldg(&tab.col[c + 1].w);
            float2 x = row[ci.x], y = row[tab.yoff + ci.y + tab.n2max];
            float2 xy = make_float2(fmaf(x.x, y.x, -x.y * y.y), fmaf(x.x, y.y, x.y * y.x));
            float tr = 0.f, ti = 0.f, tzr = 0.f, tzi = 0.f;
            const float2* zr = row + tab.zoff + ci.z + tab.n3max - ci.w;   // zr[k] = Z(n3(k))
            float n3 = (float)ci.z;
            for (int k = ci.w; k < kend; k += 8) {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    float2 cv = __ldg(&tab.C[k + t]);
                    float2 z = zr[k + t];
                    float pr = fmaf(cv.x, z.x, cv.y * z.y);    // C conj(Z)
                    float pim = fmaf(cv.y, z.x, -cv.x * z.y);
                    tr += pr;
                    ti += pim;
                    tzr = fmaf(n3, pr, tzr);
                    tzi = fmaf(n3, pim, tzi);
                    n3 += 1.f;
                }
            }
            // conj(XY) T
            float zre = fmaf(xy.x, tr, xy.y * ti);
            float zim = fmaf(xy.x, ti, -xy.y * tr);
            float zzi = fmaf(xy.x, tzi, -xy.y * tzr);
            phk += zre;
            fk[0] = fmaf(kxs * ci.x, zim, fk[0]);
            fk[1] = fmaf(kys * ci.y, zim, fk[1]);
            fk[2] = fmaf(kzs, zzi, fk[2]);
        }
    }
    if (valid && !ewald && pppm_field && w == 0) {
        phk = pppm_field[i];
        fk[0] = pppm_field[(size_t)n + i];
        fk[1] = pppm_field[(size_t)2 * n + i];
        fk[2] = pppm_field[(size_t)3 * n + i];
    }
    if (valid && ec.mode == 1) {
        const float4 pi = __ldg(&pos4[i]);
        int total = 0;
        for (int s = 0; s < n_species; ++s) total += __ldg(&cnt_list[(size_t)s * n + i]);
        const float rc2 = g.rc_real * g.rc_real;
        const float al = ec.alpha;
        for (int e = w; e < total; e += W) {
            int ent = __ldg(&nbr_list[(size_t)e * n + i]);
            int j = entry_index(ent);
            float tx, ty, tz;
            entry_shift(ent, tx, ty, tz);
            float4 pj = __ldg(&pos4[j]);
            float vx = (pj.x - pi.x) + tx * g.L[0];
            float vy = (pj.y - pi.y) + ty * g.L[1];
            float vz = (pj.z - pi.z) + tz * g.L[2];
            float r2 = vx * vx + vy * vy + vz * vz;
            if (r2 < rc2) {
                float r = sqrtf(r2), ir = 1.f / r;
                float qj = __ldg(&q_raw[j]) + delta;
                float ec_ = erfcf(al * r);
                phr = fmaf(KE * qj, ec_ * ir, phr);
                float bracket = 2.f * al * r * INV_SQRT_PI * expf(-al * al * r2) + ec_;
                float coef = -0.5f * KE * qc * qj * bracket * ir * ir * ir;
                float fx = coef * vx, fy = coef * vy, fz = coef * vz;
                fr[0] = fmaf(2.f, fx, fr[0]);
                fr[1] = fmaf(2.f, fy, fr[1]);
                fr[2] = fmaf(2.f, fz, fr[2]);
                wv[0] -= vx * fx; wv[1] -= vx * fy; wv[2] -= vx * fz;
                wv[3] -= vy * fx; wv[4] -= vy * fy; wv[5] -= vy * fz;
                wv[6] -= vz * fx; wv[7] -= vz * fy; wv[8] -= vz * fz;
            }
        }
    }
    red[w][0][lane] = phk;
    red[w][1][lane] = phr;
    red[w][2][lane] = fk[0];
    red[w][3][lane] = fk[1];
    red[w][4][lane] = fk[2];
    red[w][5][lane] = fr[0];
    red[w][6][lane] = fr[1];
    red[w][7][lane] = fr[2];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float v = wv[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) wred[k][w] = v;
    }
    __syncthreads();
    if (w == 0) {
        double s_phi = 0.0, s_er = 0.0, s_es = 0.0, s_qc = 0.0, px = 0.0, py = 0.0, pz = 0.0;
        if (valid) {
            float t[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                float v = 0.f;
#pragma unroll
                for (int q = 0; q < W; ++q) v += red[q][k][lane];
                t[k] = v;
            }
            float phs = ec.mode == 1 ? -2.f * KE * ec.alpha * INV_SQRT_PI * qc : 0.f;
            float ph = t[0] + t[1] + phs;
            float fx = fmaf(qc, t[2], t[5]), fy = fmaf(qc, t[3], t[6]), fz = fmaf(qc, t[4], t[7]);
            phi[i] = ph;
            if (charges_out) charges_out[i] = qc;
            float qt = seps * qc;
            acc12[3 * i + 0] = make_float4(fx, fy, fz, qt);
            acc12[3 * i + 1] = make_float4(0.f, 0.f, 0.f, qt);
            acc12[3 * i + 2] = make_float4(0.f, 0.f, 0.f, qt);
            s_phi = (double)ph;
            s_er = 0.5 * (double)qc * (double)t[1];
            s_es = ec.mode == 1 ? -(double)KE * ec.alpha * INV_SQRT_PI * (double)qc * (double)qc : 0.0;
            s_qc = (double)qt;
            px = (double)qt * (double)pos_in[3 * i + 0];
            py = (double)qt * (double)pos_in[3 * i + 1];
            pz = (double)qt * (double)pos_in[3 * i + 2];
        }
        double v[7] = {s_phi, s_er, s_es, s_qc, px, py, pz};
#pragma unroll
        for (int k = 0; k < 7; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        }
        if (lane == 0) {
            atomicAdd(&acc->sum_phi, v[0]);
            atomicAdd(&acc->e_real, v[1]);
            atomicAdd(&acc->e_self, v[2]);
            atomicAdd(&acc->sum_qc, v[3]);
            atomicAdd(&acc->polar[0], v[4]);
            atomicAdd(&acc->polar[1], v[5]);
            atomicAdd(&acc->polar[2], v[6]);
        }
        if (lane < 9) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < W; ++q) t += (double)wred[lane][q];
            atomicAdd(&acc->virial[lane], t);
        }
    }
}

__global__ void k_finalize_atoms(const float* __restrict__ acc12, int n, float* __restrict__ forces,
                                 float* __restrict__ bec, const float* __restrict__ phi,
                                 float* __restrict__ potential) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* a = acc12 + 12 * (size_t)i;
    if (forces) {
        forces[3 * i + 0] = a[0];
        forces[3 * i + 1] = a[1];
        forces[3 * i + 2] = a[2];
    }
    if (bec) {
#pragma unroll
        for (int k = 0; k < 9; ++k) bec[9 * (size_t)i + k] = a[3 + k];
    }
    if (potential) potential[i] = phi[i];
}

__global__ void k_finalize_scalars(const Accum* __restrict__ acc, int n, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double e = acc->sum_u + acc->e_real + acc->e_kspace + acc->e_self;
    out[0] = e;
    out[1] = acc->sum_u;
    out[2] = acc->e_real;
    out[3] = acc->e_kspace;
    out[4] = acc->e_self;
    for (int k = 0; k < 9; ++k) out[5 + k] = acc->virial[k];
    for (int k = 0; k < 3; ++k) out[14 + k] = acc->polar[k];
    out[17] = acc->sum_qc;
    out[18] = n > 0 ? acc->sum_phi / (double)n : 0.0;
    out[19] = (double)acc->status;
}

}  // namespace

void launch_field(const float4* pos4, const float* pos_in, const float* q_raw, const int* nbr_list, const int* cnt_list,
                  int n, int n_species, const Geom& g, ElecConst ec, float q_target, float sqrt_eps, bool ewald,
                  EwaldTab tab, const float* pppm_field, float* phi, float* acc12, float* charges_out, Accum* acc,
                  cudaStream_t st) {
    if (n == 0) return;
    constexpr int W = 8;
    size_t smem = ewald ? sizeof(float2) * 32 * tab.nph : 0;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_field<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr = true;
    }
    k_field<W><<<(n + 31) / 32, 32 * W, smem, st>>>(pos4, pos_in, q_raw, nbr_list, cnt_list, n, n_species, g, ec,
                                                    q_target, sqrt_eps, ewald ? 1 : 0, tab, pppm_field, phi,
                                                    reinterpret_cast<float4*>(acc12), charges_out, acc);
}

void launch_finalize_atoms(const float* acc12, int n, float* forces, float* bec, const float* phi, float* potential,
                           cudaStream_t st) {
    if (n == 0 || (!forces && !bec && !potential)) return;
    k_finalize_atoms<<<(n + 255) / 256, 256, 0, st>>>(acc12, n, forces, bec, phi, potential);
}

void launch_finalize_scalars(const Accum* acc, int n, float sqrt_eps, double* scalars, cudaStream_t st) {
    (void)sqrt_eps;
    if (!scalars) return;
    k_finalize_scalars<<<1, 32, 0, st>>>(acc, n, scalars);
}

}  // namespace qnep
