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
#include <algorithm>

#include "desc_math.cuh"
#include "tma.cuh"

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
                                                  const int* __restrict__ sidx, Accum* __restrict__ acc) {
    extern __shared__ float2 stab[];
    __shared__ float red[W][8][33];
    __shared__ float wred[9][W];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i0 = blockIdx.x * 32;
    const int i = i0 + lane;
    const bool valid = i < n;
    const float delta = block_charge_scalars(acc, q_target, n, 0, 0.f).delta;   // synchronises
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
            if (tab.tri) {   // k = 2 pi H^-1 (n1, n2, n3): the n3 part from the n3-weighted sum
#pragma unroll
                for (int dd = 0; dd < 3; ++dd)
                    fk[dd] = fmaf(tab.krec[3 * dd + 2], zzi,
                                  fmaf(tab.krec[3 * dd] * ci.x + tab.krec[3 * dd + 1] * ci.y, zim, fk[dd]));
            } else {
                fk[0] = fmaf(kxs * ci.x, zim, fk[0]);
                fk[1] = fmaf(kys * ci.y, zim, fk[1]);
                fk[2] = fmaf(kzs, zzi, fk[2]);
            }
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
            int ent = list_entry(nbr_list, i, e, g.list_sa, g.list_se);
            int j = entry_index(ent);
            float tx, ty, tz;
            entry_shift(ent, tx, ty, tz);
            float4 pj = __ldg(&pos4[j]);
            float shx, shy, shz;
            shift_vector(g, tx, ty, tz, shx, shy, shz);
            float vx = (pj.x - pi.x) + shx;
            float vy = (pj.y - pi.y) + shy;
            float vz = (pj.z - pi.z) + shz;
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
            const int io = sidx ? __ldg(&sidx[i]) : i;
            if (charges_out) charges_out[io] = qc;
            float qt = seps * qc;
            acc12[3 * i + 0] = make_float4(fx, fy, fz, qt);
            acc12[3 * i + 1] = make_float4(0.f, 0.f, 0.f, qt);
            acc12[3 * i + 2] = make_float4(0.f, 0.f, 0.f, qt);
            s_phi = (double)ph;
            s_er = 0.5 * (double)qc * (double)t[1];
            s_es = ec.mode == 1 ? -(double)KE * ec.alpha * INV_SQRT_PI * (double)qc * (double)qc : 0.0;
            s_qc = (double)qt;
            px = (double)qt * (double)pos_in[3 * io + 0];
            py = (double)qt * (double)pos_in[3 * io + 1];
            pz = (double)qt * (double)pos_in[3 * io + 2];
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

// Real space (mode 1), one warp per sorted atom k at a time (persistent warps over the
// atoms), lanes over list entries:
//   phi^r_k = k_e sum_j q_j erfc(alpha r)/r,  F^r_k = sum_j 2 F^{r,static}_kj,
//   W^r -= r_kj (x) F^{r,static}_kj,  U^r = 1/2 sum_k q_k phi^r_k.
// rfield[k] = (F^r, phi^r).  The virial stays in each lane over all of the warp's atoms
// (one warp reduction at the end); U^r and sum phi^r are summed by lane 0 in FP32 over 8
// atoms at a time, then in FP64; one set of FP64 atomics per block.
__global__ void __launch_bounds__(256) k_real(const float4* __restrict__ spos4, const float* __restrict__ q_raw,
                                              const int* __restrict__ nbr_list, const int* __restrict__ cnt_list, int n,
                                              int n_species, Geom g, float alpha, float q_target,
                                              const Accum* __restrict__ acc_in, float4* __restrict__ rfield,
                                              Accum* __restrict__ acc, float* __restrict__ avir) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float wv[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) wv[q] = 0.f;
    double sphi = 0.0, ser = 0.0;
    float pphi = 0.f, per = 0.f;
    int np = 0;
    const float delta = block_charge_scalars(acc_in, q_target, n, 0, 0.f).delta;   // synchronises
    const float rc2 = g.rc_real * g.rc_real;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int k = blockIdx.x * (blockDim.x >> 5) + wib; k < n; k += nwarps) {
        const float4 pk = __ldg(&spos4[k]);
        const float qk = __ldg(&q_raw[k]) + delta;
        int total = 0;
        for (int s = 0; s < n_species; ++s) total += __ldg(&cnt_list[(size_t)s * n + k]);
        float fx = 0.f, fy = 0.f, fz = 0.f, phr = 0.f;
        float wa[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // this atom's pair virial (xx, yy, zz, xy, xz, yz)
        for (int e = lane; e < total; e += 32) {
            const int ent = list_entry(nbr_list, k, e, g.list_sa, g.list_se);
            const int j = entry_index(ent);
            float vx, vy, vz;
            entry_vector(spos4, ent, pk, g, vx, vy, vz);
            const float r2 = vx * vx + vy * vy + vz * vz;
            if (r2 < rc2) {
                const float r = sqrtf(r2), ir = 1.f / r;
                const float qj = __ldg(&q_raw[j]) + delta;
                const float ec = erfcf(alpha * r);
                phr = fmaf(KE * qj, ec * ir, phr);
                const float bracket = 2.f * alpha * r * INV_SQRT_PI * expf(-alpha * alpha * r2) + ec;
                const float coef = -0.5f * KE * qk * qj * bracket * ir * ir * ir;
                const float ax = coef * vx, ay = coef * vy, az = coef * vz;
                fx = fmaf(2.f, ax, fx);
                fy = fmaf(2.f, ay, fy);
                fz = fmaf(2.f, az, fz);
                wv[0] -= vx * ax; wv[1] -= vx * ay; wv[2] -= vx * az;
                wv[3] -= vy * ax; wv[4] -= vy * ay; wv[5] -= vy * az;
                wv[6] -= vz * ax; wv[7] -= vz * ay; wv[8] -= vz * az;
                if (avir) {
                    // per atom: -r_kj (x) F^{r,static}_kj over the atom's entries (the pair's other entry
                    // gives atom j the same symmetric tensor)
                    wa[0] -= vx * ax; wa[1] -= vy * ay; wa[2] -= vz * az;
                    wa[3] -= vx * ay; wa[4] -= vx * az; wa[5] -= vy * az;
                }
            }
        }
        if (avir) {
#pragma unroll
            for (int q = 0; q < 6; ++q)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) wa[q] += __shfl_xor_sync(0xffffffffu, wa[q], o);
            if (lane == 0) {
                float* a = avir + (size_t)AVIR * k;
                atomicAdd(a + 0, wa[0]);
                atomicAdd(a + 4, wa[1]);
                atomicAdd(a + 8, wa[2]);
                atomicAdd(a + 1, wa[3]);
                atomicAdd(a + 3, wa[3]);
                atomicAdd(a + 2, wa[4]);
                atomicAdd(a + 6, wa[4]);
                atomicAdd(a + 5, wa[5]);
                atomicAdd(a + 7, wa[5]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            phr += __shfl_xor_sync(0xffffffffu, phr, o);
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (lane == 0) {
            rfield[k] = make_float4(fx, fy, fz, phr);
            pphi += phr;
            per += 0.5f * qk * phr;
            if (++np == 8) {
                sphi += (double)pphi;
                ser += (double)per;
                pphi = per = 0.f;
                np = 0;
            }
        }
    }
    __shared__ double red[11][8];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        float v = wv[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][wib] = (double)v;
    }
    if (lane == 0) {
        red[9][wib] = sphi + (double)pphi;
        red[10][wib] = ser + (double)per;
    }
    __syncthreads();
    if (threadIdx.x < 11) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x][q];
        if (threadIdx.x < 9) atomicAdd(&acc->virial[threadIdx.x], t);
        else if (threadIdx.x == 9) atomicAdd(&acc->sum_phi, t);
        else atomicAdd(&acc->e_real, t);
    }
}

// Reciprocal-space potential and field of 32 atoms (lanes) over one split of the
// k columns (warps take every W-th column of the split).  With C = 4 k_e G S:
//   phi^k_i = sum_half Re[C e^{i k.r_i}],  F^k_i = q_i sum_half k Im[C e^{i k.r_i}]
// per column (n1, n2): T = sum_n3 C conj(Z(n3)), then conj(X Y) T.  Partial
// results of the splits are added with float4 atomics to kfield = (F^k / q, phi^k).
// With the per-atom virial (AV) the same column sums are also weighted by B(k) per wave vector:
//   V_i,ab = sum_half Re[C e^{i k.r_i}] B_ab(k)   (W_i^k = q_i / 2 V_i, the Heyes form of Sec. II.C)
template <int W, bool AV>
__global__ void __launch_bounds__(32 * W) k_field_k(int n, EwaldTab tab, int csplit, float4* __restrict__ kfield,
                                                    Accum* __restrict__ acc, float* __restrict__ avir) {
    extern __shared__ __align__(16) float2 stab[];
    __shared__ float red[W][AV ? 10 : 4][33];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int failed;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int group = blockIdx.x / csplit, split = blockIdx.x - group * csplit;
    const int i0 = group * 32;
    const int i = i0 + lane;
    const int cnt = min(32, n - i0);
    // the 32 atoms' phase rows are contiguous: one TMA bulk copy into shared memory
    if (threadIdx.x == 0) {
        failed = 0;
        mbar_init(&bar, 1);
        mbar_init_fence();
        const uint32_t bytes = round_up16((uint32_t)(cnt * tab.nph) * (uint32_t)sizeof(float2));
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(stab, tab.phase + (size_t)i0 * tab.nph, bytes, &bar);
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0u)) failed = 1;
    __syncthreads();
    if (failed) {   // same decision in every thread of the block
        mbar_wait_bounded(&bar, 0u);   // one more bounded chance for the copy in flight
        if (threadIdx.x == 0) atomicOr(&acc->status, kStatusTimeout);
        return;
    }
    float phk = 0.f, fk0 = 0.f, fk1 = 0.f, fk2 = 0.f;
    float hv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (lane < cnt) {
        const float2* row = stab + lane * tab.nph;
        const float kxs = TWO_PI / tab.L[0], kys = TWO_PI / tab.L[1], kzs = TWO_PI / tab.L[2];
        for (int c = split + csplit * w; c < tab.ncol; c += csplit * W) {
            const int4 ci = __ldg(&tab.col[c]);
            const int kend = __ldg(&tab.col[c + 1].w);
            const float2 x = row[ci.x], y = row[tab.yoff + ci.y + tab.n2max];
            const float2 xy = make_float2(fmaf(x.x, y.x, -x.y * y.y), fmaf(x.x, y.y, x.y * y.x));
            float tr = 0.f, ti = 0.f, tzr = 0.f, tzi = 0.f;
            float hr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, hi[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const float2* zr = row + tab.zoff + ci.z + tab.n3max - ci.w;   // zr[k] = Z(n3(k))
            const float4* c4 = reinterpret_cast<const float4*>(tab.C);
            if (AV) {
                for (int k = ci.w; k < kend; ++k) {
                    const float2 cc = tab.C[k], z0 = zr[k];
                    const float pr = fmaf(cc.x, z0.x, cc.y * z0.y), pim = fmaf(cc.y, z0.x, -cc.x * z0.y);
                    const float4 b0 = __ldg(&tab.kb[2 * k]), b1 = __ldg(&tab.kb[2 * k + 1]);
                    const float bv[6] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y};
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        hr[q] = fmaf(bv[q], pr, hr[q]);
                        hi[q] = fmaf(bv[q], pim, hi[q]);
                    }
                }
            }
            for (int k = ci.w; k < kend; k += 8) {
                const float n3b = (float)(ci.z + (k - ci.w));
#pragma unroll
                for (int t = 0; t < 8; t += 2) {
                    const float4 cc = __ldg(&c4[(k + t) >> 1]);
                    const float2 z0 = zr[k + t], z1 = zr[k + t + 1];
                    float pr = fmaf(cc.x, z0.x, cc.y * z0.y);    // C conj(Z)
                    float pim = fmaf(cc.y, z0.x, -cc.x * z0.y);
                    tr += pr;
                    ti += pim;
                    tzr = fmaf(n3b + (float)t, pr, tzr);
                    tzi = fmaf(n3b + (float)t, pim, tzi);
                    pr = fmaf(cc.z, z1.x, cc.w * z1.y);
                    pim = fmaf(cc.w, z1.x, -cc.z * z1.y);
                    tr += pr;
                    ti += pim;
                    tzr = fmaf(n3b + (float)(t + 1), pr, tzr);
                    tzi = fmaf(n3b + (float)(t + 1), pim, tzi);
                }
            }
            const float zre = fmaf(xy.x, tr, xy.y * ti);
            const float zim = fmaf(xy.x, ti, -xy.y * tr);
            const float zzi = fmaf(xy.x, tzi, -xy.y * tzr);
            phk += zre;
            if (tab.tri) {   // k = 2 pi H^-1 (n1, n2, n3): the n3 part from the n3-weighted sum
                fk0 = fmaf(tab.krec[2], zzi, fmaf(tab.krec[0] * ci.x + tab.krec[1] * ci.y, zim, fk0));
                fk1 = fmaf(tab.krec[5], zzi, fmaf(tab.krec[3] * ci.x + tab.krec[4] * ci.y, zim, fk1));
                fk2 = fmaf(tab.krec[8], zzi, fmaf(tab.krec[6] * ci.x + tab.krec[7] * ci.y, zim, fk2));
            } else {
                fk0 = fmaf(kxs * ci.x, zim, fk0);
                fk1 = fmaf(kys * ci.y, zim, fk1);
                fk2 = fmaf(kzs, zzi, fk2);
            }
            if (AV) {
#pragma unroll
                for (int q = 0; q < 6; ++q) hv[q] += fmaf(xy.x, hr[q], xy.y * hi[q]);
            }
        }
    }
    red[w][0][lane] = phk;
    red[w][1][lane] = fk0;
    red[w][2][lane] = fk1;
    red[w][3][lane] = fk2;
    if (AV) {
#pragma unroll
        for (int q = 0; q < 6; ++q) red[w][4 + q][lane] = hv[q];
    }
    __syncthreads();
    if (w == 0) {
        float t[10];
#pragma unroll
        for (int q = 0; q < (AV ? 10 : 4); ++q) {
            float v = 0.f;
#pragma unroll
            for (int u = 0; u < W; ++u) v += red[u][q][lane];
            t[q] = v;
        }
        if (lane < cnt) atomicAdd(&kfield[i], make_float4(t[1], t[2], t[3], t[0]));
        if (AV && lane < cnt) {
#pragma unroll
            for (int q = 0; q < 6; ++q) atomicAdd(&avir[(size_t)AVIR * i + 9 + q], t[4 + q]);
        }
        float sp = lane < cnt ? t[0] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
        if (lane == 0) atomicAdd(&acc->sum_phi, (double)sp);
    }
}

__device__ __forceinline__ void write_scalars(const Accum* __restrict__ acc, int n, double* __restrict__ out,
                                              unsigned int* __restrict__ status_host) {
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
    if (status_host) *status_host = acc->status;
}

__device__ __forceinline__ void atomic_virial_store(float* __restrict__ out, int io, int q, float v) {
    out[9 * (size_t)io + q] = v;
}

// Per-atom outputs back in input order (forces, BEC, charges q^c, potential
// phi = phi^k + phi^r + phi^s, site energies), the block sums of P = sum q~^c r,
// U^s = -k_e alpha/sqrt(pi) sum q^c^2 and sum q~^c; the last block writes the scalars.
__global__ void k_finalize(const float* __restrict__ acc12, int n, const int* __restrict__ sidx,
                           const float* __restrict__ pos_in, const float* __restrict__ q_raw, float q_target,
                           float seps, ElecConst ec, const float4* __restrict__ kfield,
                           const float4* __restrict__ rfield, float* __restrict__ forces, float* __restrict__ bec,
                           float* __restrict__ charges, float* __restrict__ potential, const float* __restrict__ u,
                           float* __restrict__ site_energy, Accum* __restrict__ acc, double* __restrict__ scalars,
                           unsigned int* __restrict__ status_host, unsigned int* __restrict__ done,
                           float* __restrict__ grad, float gpx, float gpy, float gpz, const float* __restrict__ avir,
                           float* __restrict__ atom_virial) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    // FP32 terms summed over a warp (32 atoms), then FP64 across warps and blocks
    float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // P (3), U^s, sum q~^c
    const float delta = block_charge_scalars(acc, q_target, n, 0, 0.f).delta;   // synchronises
    if (k < n) {
        const int io = sidx ? __ldg(&sidx[k]) : k;
        const float qc = __ldg(&q_raw[k]) + delta;
        const float qt = seps * qc;
        const float* a = acc12 + 12 * (size_t)k;
        if (forces) {
            forces[3 * (size_t)io + 0] = a[0];
            forces[3 * (size_t)io + 1] = a[1];
            forces[3 * (size_t)io + 2] = a[2];
        }
        if (bec) {
#pragma unroll
            for (int q = 0; q < 9; ++q) bec[9 * (size_t)io + q] = a[3 + q];
        }
        if (grad) {   // -F of the weighted objective plus g_P . Z (Z_ab = a[3 + 3a + b])
#pragma unroll
            for (int b = 0; b < 3; ++b)
                grad[3 * (size_t)io + b] = -a[b] + gpx * a[3 + b] + gpy * a[6 + b] + gpz * a[9 + b];
        }
        if (charges) charges[io] = qc;
        if (atom_virial) {
            // entries and real space, plus q_i / 2 times the reciprocal-space sums (symmetric)
            const float* w = avir + (size_t)AVIR * k;
            const float h = 0.5f * qc;
            const float kv[9] = {w[9], w[12], w[13], w[12], w[10], w[14], w[13], w[14], w[11]};
#pragma unroll
            for (int q = 0; q < 9; ++q) atomic_virial_store(atom_virial, io, q, fmaf(h, kv[q], w[q]));
        }
        const float phs = ec.mode == 1 ? -2.f * KE * ec.alpha * INV_SQRT_PI * qc : 0.f;
        if (potential) potential[io] = kfield[k].w + rfield[k].w + phs;
        if (site_energy) site_energy[io] = u[k];
        v[0] = qt * pos_in[3 * (size_t)io + 0];
        v[1] = qt * pos_in[3 * (size_t)io + 1];
        v[2] = qt * pos_in[3 * (size_t)io + 2];
        v[3] = ec.mode == 1 ? -KE * ec.alpha * INV_SQRT_PI * qc * qc : 0.f;
        v[4] = qt;
    }
    __shared__ double red[5][8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        float x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][wib] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x][q];
        double* dst = threadIdx.x < 3 ? &acc->polar[threadIdx.x] : (threadIdx.x == 3 ? &acc->e_self : &acc->sum_qc);
        atomicAdd(dst, t);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(done, 1u);
        last = t == gridDim.x - 1;
        if (last) *done = 0u;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        if (scalars) write_scalars(acc, n, scalars, status_host);
        else if (status_host) *status_host = acc->status;
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
    write_scalars(acc, n, out, nullptr);
}

}  // namespace

void launch_field(const float4* pos4, const float* pos_in, const float* q_raw, const int* nbr_list, const int* cnt_list,
                  int n, int n_species, const Geom& g, ElecConst ec, float q_target, float sqrt_eps, bool ewald,
                  EwaldTab tab, const float* pppm_field, float* phi, float* acc12, float* charges_out, Accum* acc,
                  cudaStream_t st, const int* sidx) {
    if (n == 0) return;
    constexpr int W = 32;
    size_t smem = ewald ? sizeof(float2) * 32 * tab.nph : 0;
    static std::atomic<int> attr[kMaxDevices];
    ensure_smem_attr(k_field<W>, attr, 160 * 1024);
    k_field<W><<<(n + 31) / 32, 32 * W, smem, st>>>(pos4, pos_in, q_raw, nbr_list, cnt_list, n, n_species, g, ec,
                                                    q_target, sqrt_eps, ewald ? 1 : 0, tab, pppm_field, phi,
                                                    reinterpret_cast<float4*>(acc12), charges_out, sidx, acc);
}

void launch_real(const float4* spos4, const float* q_raw, const int* nbr_list, const int* cnt_list, int n,
                 int n_species, const Geom& g, float alpha, float q_target, const Accum* acc_in, float4* rfield,
                 Accum* acc, cudaStream_t st, float* avir) {
    if (n == 0) return;
    // persistent warps: one wave of resident blocks, fewer for small systems
    static std::atomic<long long> occ[kMaxDevices];
    const int per_sm = cached_occupancy(k_real, occ, 256, 0);
    const int blocks = std::max(1, std::min((n + 7) / 8, per_sm * num_sms()));
    k_real<<<blocks, 256, 0, st>>>(spos4, q_raw, nbr_list, cnt_list, n, n_species, g, alpha, q_target, acc_in, rfield,
                                   acc, avir);
}

void launch_field_k(int n, const EwaldTab& tab, float4* kfield, Accum* acc, cudaStream_t st, float* avir) {
    if (n == 0 || tab.ncol == 0) return;
    constexpr int W = 8;
    static std::atomic<int> attr[kMaxDevices], attr_v[kMaxDevices];
    ensure_smem_attr(k_field_k<W, false>, attr, 160 * 1024);
    if (avir) ensure_smem_attr(k_field_k<W, true>, attr_v, 160 * 1024);
    const int groups = (n + 31) / 32;
    const size_t smem = sizeof(float2) * 32 * tab.nph;
    // column splits: fill the resident block slots (SMs x blocks per SM at this shared-memory
    // size) in one wave; a partial second wave would double the time of the SMs running it
    static std::atomic<long long> occ[kMaxDevices];
    const int slots = num_sms() * cached_occupancy(k_field_k<W, false>, occ, 32 * W, smem);
    int csplit = slots / groups;
    if (csplit < 1) csplit = 1;
    if (csplit > tab.ncol) csplit = tab.ncol;
    if (avir) k_field_k<W, true><<<groups * csplit, 32 * W, smem, st>>>(n, tab, csplit, kfield, acc, avir);
    else k_field_k<W, false><<<groups * csplit, 32 * W, smem, st>>>(n, tab, csplit, kfield, acc, nullptr);
}

void launch_finalize(const float* acc12, int n, const int* sidx, const float* pos_in, const float* q_raw,
                     float q_target, float seps, ElecConst ec, const float4* kfield, const float4* rfield,
                     float* forces, float* bec, float* charges, float* potential, const float* u, float* site_energy,
                     Accum* acc, double* scalars, unsigned int* status_host, unsigned int* done, cudaStream_t st,
                     float* grad, const float* gp, const float* avir, float* atom_virial) {
    int blocks = (n + 255) / 256;
    if (blocks < 1) blocks = 1;
    k_finalize<<<blocks, 256, 0, st>>>(acc12, n, sidx, pos_in, q_raw, q_target, seps, ec, kfield, rfield, forces, bec,
                                       charges, potential, u, site_energy, acc, scalars, status_host, done, grad,
                                       gp ? gp[0] : 0.f, gp ? gp[1] : 0.f, gp ? gp[2] : 0.f, avir, atom_virial);
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
