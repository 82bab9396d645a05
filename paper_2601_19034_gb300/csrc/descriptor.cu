// NEP descriptor, two-output network and the chain-rule backward.
//
// Descriptor (the NEP3/NEP4 form the paper defers to, Sec. II.A):
//   f_c(r) = (1 + cos(pi r / r_c)) / 2,  x = 2 (r/r_c - 1)^2 - 1,  f_k = (T_k(x) + 1) f_c / 2
//   g_n(r) = sum_k c[t_i][t_j][n][k] f_k(r)
//   D^R_n = sum_j g^R_n(r_ij)
//   D^A_{nl} = sum_{j,k} g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_ijk) = sum_m w_lm A_{n,lm}^2,
//              A_{n,lm} = sum_j g^A_n(r_ij) Y_lm(u_ij)           (addition theorem)
//   D^4b_n = tr(T_n^3),  T_n = sum_j g^A_n(r_ij) (u u^T - I/3)   (built from the l = 2 A's)
// Y_lm are real harmonic polynomials of the unit vector with weights w_lm such
// that sum_m w_lm Y_lm(a) Y_lm(b) = P_l(a.b).
// Network (Eq. U_i and the charge node of Sec. II.B), weights of the central
// species: h = tanh(W0 D - b0), U = w1E.h - b1E, q = w1q.h - b1q.  The forward
// kernel also stores dU/dD and dq/dD; the backward forms the adjoints
//   lambda = dU/dD + (phi_i - mean phi) dq/dD,   kappa = sqrt(eps_inf) dq/dD
// (partial forces of Sec. II.C: F^NEP_ij plus the real / reciprocal / self
// dynamic-charge terms, and a_ij = dq~_i/dr_ij for Eq. bec_2), recomputes
// dD/dr_ij per neighbour entry and scatters the partial forces.
#include "desc_math.cuh"

namespace qnep {

namespace {

template <int TPA>
__global__ void __launch_bounds__(128) k_desc_fwd(const float4* __restrict__ pos4, const int* __restrict__ nbr_list,
                                                  const int* __restrict__ cnt_list, const int* __restrict__ nbr_ang,
                                                  const int* __restrict__ cnt_ang, int n, Geom g,
                                                  const float* __restrict__ params, ParamLayout lay,
                                                  float* __restrict__ ang_coef, float* __restrict__ du,
                                                  float* __restrict__ dq, float* __restrict__ u_out,
                                                  float* __restrict__ q_out, float* __restrict__ des_out,
                                                  const int* __restrict__ sidx, float4* __restrict__ fields,
                                                  const float* __restrict__ gq_in, Accum* __restrict__ acc,
                                                  float* __restrict__ dtc) {
    extern __shared__ float sp[];
    for (int k = threadIdx.x; k < lay.total; k += blockDim.x) sp[k] = params[k];
    __syncthreads();
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / TPA;
    const int lane = gt % TPA;
    double su = 0.0, sq = 0.0, sg = 0.0;
    if (i < n) {
        const unsigned gm = group_mask<TPA>();
        const int S = lay.n_species;
        const float4 pi = __ldg(&pos4[i]);
        const int ti = __float_as_int(pi.w);
        const float rcr2 = g.rc_radial * g.rc_radial;

        // radial: per neighbour-species basis sums contracted with c_R
        float dr[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) dr[q] = 0.f;
        int off = 0;
        for (int s = 0; s < S; ++s) {
            const int cnt = __ldg(&cnt_list[(size_t)s * n + i]);
            float b[KR];
#pragma unroll
            for (int k = 0; k < KR; ++k) b[k] = 0.f;
            for (int e = lane; e < cnt; e += TPA) {
                int ent = list_entry(nbr_list, i, off + e, g.list_sa, g.list_se);
                float vx, vy, vz;
                entry_vector(pos4, ent, pi, g, vx, vy, vz);
                float r2 = vx * vx + vy * vy + vz * vz;
                if (r2 < rcr2) {
                    float f[KR];
                    basis<KR>(sqrtf(r2), g.rc_radial, f);
#pragma unroll
                    for (int k = 0; k < KR; ++k) b[k] += f[k];
                }
            }
            off += cnt;
            const float* c = sp + lay.c_radial + ((ti * S + s) * NR) * KR;
#pragma unroll
            for (int q = 0; q < NR; ++q)
#pragma unroll
                for (int k = 0; k < KR; ++k) dr[q] = fmaf(c[q * KR + k], b[k], dr[q]);
        }

        // angular expansion coefficients A_{n,lm}
        float a[NA][NLM];
#pragma unroll
        for (int q = 0; q < NA; ++q)
#pragma unroll
            for (int m = 0; m < NLM; ++m) a[q][m] = 0.f;
        off = 0;
        for (int s = 0; s < S; ++s) {
            const int cnt = __ldg(&cnt_ang[(size_t)s * n + i]);
            const float* c = sp + lay.c_angular + ((ti * S + s) * NA) * KA;
            for (int e = lane; e < cnt; e += TPA) {
                int ent = list_entry(nbr_ang, i, off + e, g.ang_sa, g.ang_se);
                float vx, vy, vz;
                entry_vector(pos4, ent, pi, g, vx, vy, vz);
                float r = sqrtf(vx * vx + vy * vy + vz * vz);
                float f[KA];
                basis<KA>(r, g.rc_angular, f);
                float gn[NA];
#pragma unroll
                for (int q = 0; q < NA; ++q) {
                    float acc_g = 0.f;
#pragma unroll
                    for (int k = 0; k < KA; ++k) acc_g = fmaf(c[q * KA + k], f[k], acc_g);
                    gn[q] = acc_g;
                }
                float ir = 1.f / r;
                float Y[NLM];
                harmonics(vx * ir, vy * ir, vz * ir, Y);
#pragma unroll
                for (int q = 0; q < NA; ++q)
#pragma unroll
                    for (int m = 0; m < NLM; ++m) a[q][m] = fmaf(gn[q], Y[m], a[q][m]);
            }
            off += cnt;
        }
        if (TPA > 1) {
#pragma unroll
            for (int q = 0; q < NR; ++q) dr[q] = group_sum<TPA>(dr[q], gm);
#pragma unroll
            for (int q = 0; q < NA; ++q)
#pragma unroll
                for (int m = 0; m < NLM; ++m) a[q][m] = group_sum<TPA>(a[q][m], gm);
        }
        if (ang_coef) {
#pragma unroll
            for (int q = 0; q < NA; ++q)
#pragma unroll
                for (int m = 0; m < NLM; ++m)
                    if (((q * NLM + m) % TPA) == lane) ang_coef[(size_t)(q * NLM + m) * n + i] = a[q][m];
        }

        // descriptor vector
        float d[NDES];
#pragma unroll
        for (int q = 0; q < NR; ++q) d[q] = dr[q];
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            float s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
            for (int m = 0; m < 3; ++m) s1 = fmaf(c_wlm[m], a[q][m] * a[q][m], s1);
#pragma unroll
            for (int m = 3; m < 8; ++m) s2 = fmaf(c_wlm[m], a[q][m] * a[q][m], s2);
#pragma unroll
            for (int m = 8; m < 15; ++m) s3 = fmaf(c_wlm[m], a[q][m] * a[q][m], s3);
#pragma unroll
            for (int m = 15; m < 24; ++m) s4 = fmaf(c_wlm[m], a[q][m] * a[q][m], s4);
            d[NR + 0 * NA + q] = s1;
            d[NR + 1 * NA + q] = s2;
            d[NR + 2 * NA + q] = s3;
            d[NR + 3 * NA + q] = s4;
            float t[6], t2[6];
            float a2[5] = {a[q][3], a[q][4], a[q][5], a[q][6], a[q][7]};
            tensor_from_a(a2, t);
            tensor_square(t, t2);
            // tr(T^3) = sum_ab (T^2)_ab T_ab (T symmetric)
            d[NR + 4 * NA + q] = t2[0] * t[0] + t2[1] * t[1] + t2[2] * t[2] +
                                 2.f * (t2[3] * t[3] + t2[4] * t[4] + t2[5] * t[5]);
        }
        const float* scaler = sp + lay.scaler;
#pragma unroll
        for (int v = 0; v < NDES; ++v) d[v] *= scaler[v];
        if (des_out && lane == 0) {
#pragma unroll
            for (int v = 0; v < NDES; ++v) des_out[(size_t)sidx[i] * NDES + v] = d[v];
        }
        if (dtc && lane == 0) {   // tensor-core network (precision form): hand the scaled descriptor over
            float4* o = reinterpret_cast<float4*>(dtc + (size_t)i * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                o[q] = make_float4(d[4 * q], d[4 * q + 1], 4 * q + 2 < NDES ? d[4 * q + 2] : 0.f,
                                   4 * q + 3 < NDES ? d[4 * q + 3] : 0.f);
        }

        if (!dtc) {
        // network and its input gradients (hidden units split over the TPA lanes)
        const float* net = sp + lay.mlp + ti * lay.mlp_stride;
        float uu = 0.f, qq = 0.f, gu[NDES], gq[NDES];
#pragma unroll
        for (int v = 0; v < NDES; ++v) { gu[v] = 0.f; gq[v] = 0.f; }
        for (int mu = lane; mu < NNEU; mu += TPA) {
            const float* w0 = net + ParamLayout::W0 + mu * NDES;
            float pre = -net[ParamLayout::B0 + mu];
#pragma unroll
            for (int v = 0; v < NDES; ++v) pre = fmaf(w0[v], d[v], pre);
            float h = tanhf(pre);
            float we = net[ParamLayout::W1E + mu], wq = net[ParamLayout::W1Q + mu];
            uu = fmaf(we, h, uu);
            qq = fmaf(wq, h, qq);
            float dh = 1.f - h * h;
            float ae = we * dh, aq = wq * dh;
#pragma unroll
            for (int v = 0; v < NDES; ++v) {
                gu[v] = fmaf(ae, w0[v], gu[v]);
                gq[v] = fmaf(aq, w0[v], gq[v]);
            }
        }
        if (TPA > 1) {
            uu = group_sum<TPA>(uu, gm);
            qq = group_sum<TPA>(qq, gm);
#pragma unroll
            for (int v = 0; v < NDES; ++v) {
                gu[v] = group_sum<TPA>(gu[v], gm);
                gq[v] = group_sum<TPA>(gq[v], gm);
            }
        }
        uu -= net[ParamLayout::B1E];
        qq -= net[ParamLayout::B1Q];
        if (du) {
#pragma unroll
            for (int v = 0; v < NDES; ++v)
                if ((v % TPA) == lane) {
                    du[(size_t)v * n + i] = gu[v] * scaler[v];
                    dq[(size_t)v * n + i] = gq[v] * scaler[v];
                }
        }
        if (lane == 0) {
            u_out[i] = uu;
            q_out[i] = qq;
            su = (double)uu;
            sq = (double)qq;
        }
        }
        if (lane == 0 && gq_in) sg = (double)__ldg(&gq_in[__ldg(&sidx[i])]);
        for (int part = lane; part < 5; part += TPA) zero_atom_fields(fields, n, i, part);
    }
    // warp reduction of the FP64 energy / charge sums, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
        sg += __shfl_xor_sync(0xffffffffu, sg, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc->sum_u, su);
        atomicAdd(&acc->sum_q, sq);
        if (gq_in) atomicAdd(&acc->sum_gq, sg);
    }
}

// Scatter one partial force F_ij (and a_ij) of entry (i -> j, vector v).
template <bool BEC>
__device__ __forceinline__ void scatter(float4* __restrict__ acc12, int j, float vx, float vy, float vz, float fx,
                                        float fy, float fz, float ax, float ay, float az, float fi[3], float zi[9],
                                        float w[9]) {
    fi[0] += fx; fi[1] += fy; fi[2] += fz;
    w[0] -= vx * fx; w[1] -= vx * fy; w[2] -= vx * fz;
    w[3] -= vy * fx; w[4] -= vy * fy; w[5] -= vy * fz;
    w[6] -= vz * fx; w[7] -= vz * fy; w[8] -= vz * fz;
    if (BEC) {
        float hx = 0.5f * vx, hy = 0.5f * vy, hz = 0.5f * vz;
        float z0 = hx * ax, z1 = hx * ay, z2 = hx * az, z3 = hy * ax, z4 = hy * ay, z5 = hy * az, z6 = hz * ax,
              z7 = hz * ay, z8 = hz * az;
        zi[0] += z0; zi[1] += z1; zi[2] += z2; zi[3] += z3; zi[4] += z4;
        zi[5] += z5; zi[6] += z6; zi[7] += z7; zi[8] += z8;
        atomicAdd(&acc12[3 * j + 0], make_float4(-fx, -fy, -fz, -z0));
        atomicAdd(&acc12[3 * j + 1], make_float4(-z1, -z2, -z3, -z4));
        atomicAdd(&acc12[3 * j + 2], make_float4(-z5, -z6, -z7, -z8));
    } else {
        atomicAdd(&acc12[3 * j + 0], make_float4(-fx, -fy, -fz, 0.f));
    }
}

constexpr int PHI_STRIDE = 2 * NANG + 1;   // adjoint-weighted A's of one atom (odd stride)

template <int TPA, bool BEC>
__global__ void __launch_bounds__(128) k_desc_bwd(const float4* __restrict__ pos4, const int* __restrict__ nbr_list,
                                                  const int* __restrict__ cnt_list, const int* __restrict__ nbr_ang,
                                                  const int* __restrict__ cnt_ang, int n, Geom g,
                                                  const float* __restrict__ params, ParamLayout lay,
                                                  const float* __restrict__ ang_coef, const float* __restrict__ du,
                                                  const float* __restrict__ dqp, const float* __restrict__ q_raw,
                                                  FieldIn fin, const Accum* __restrict__ acc_in,
                                                  float4* __restrict__ acc12, Accum* __restrict__ acc) {
    extern __shared__ float sm[];
    float* sp = sm;
    float* sphi = sm + ((lay.total + 3) & ~3);
    for (int k = threadIdx.x; k < lay.total; k += blockDim.x) sp[k] = params[k];
    const ChargeScalars cs = block_charge_scalars(acc_in, fin.q_target, n, fin.mode, fin.alpha);   // synchronises
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / TPA;
    const int lane = gt % TPA;
    float w[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = 0.f;
    if (i < n) {
        const unsigned gm = group_mask<TPA>();
        const int S = lay.n_species;
        const float4 pi = __ldg(&pos4[i]);
        const int ti = __float_as_int(pi.w);
        const float seps = sp[lay.sqrt_eps];
        float qc, phi_i;
        assemble_potential(fin, cs, q_raw, i, qc, phi_i);
        const float wq = charge_adjoint_weight(fin, cs, i, phi_i - cs.phibar);
        float lam[NDES], kap[NDES];
#pragma unroll
        for (int v = 0; v < NDES; ++v) {
            float gq = __ldg(&dqp[(size_t)v * n + i]);
            lam[v] = fmaf(wq, gq, fin.e_weight * __ldg(&du[(size_t)v * n + i]));
            kap[v] = seps * gq;
        }
        // adjoint-weighted angular coefficients: Phi_{n,lm} = dE/dA_{n,lm}
        float* my = sphi + (threadIdx.x / TPA) * PHI_STRIDE;
        for (int e = lane; e < NANG; e += TPA) {
            int q = e / NLM, m = e % NLM;
            int l = m < 3 ? 1 : (m < 8 ? 2 : (m < 15 ? 3 : 4));
            float av = __ldg(&ang_coef[(size_t)e * n + i]);
            float pl = 2.f * c_wlm[m] * av * lam[NR + (l - 1) * NA + q];
            float pk = 2.f * c_wlm[m] * av * kap[NR + (l - 1) * NA + q];
            if (l == 2) {
                float a2[5], t[6], t2[6];
#pragma unroll
                for (int k = 0; k < 5; ++k) a2[k] = __ldg(&ang_coef[(size_t)(q * NLM + 3 + k) * n + i]);
                tensor_from_a(a2, t);
                tensor_square(t, t2);
                float dd;   // d tr(T^3) / d A_{n,lm} = 3 sum_ab (T^2)_ab dT_ab/dA
                if (m == 3) dd = 3.f * (t2[2] * (1.f / 3.f) - (t2[0] + t2[1]) * (1.f / 6.f));
                else if (m == 4) dd = 6.f * t2[4];
                else if (m == 5) dd = 6.f * t2[5];
                else if (m == 6) dd = 1.5f * (t2[0] - t2[1]);
                else dd = 6.f * t2[3];
                pl = fmaf(lam[NR + 4 * NA + q], dd, pl);
                pk = fmaf(kap[NR + 4 * NA + q], dd, pk);
            }
            my[e] = pl;
            my[NANG + e] = pk;
        }
        __syncwarp(gm);

        float fi[3] = {0.f, 0.f, 0.f}, zi[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) zi[k] = 0.f;
        const float rcr2 = g.rc_radial * g.rc_radial;
        // radial entries
        int off = 0;
        for (int s = 0; s < S; ++s) {
            const int cnt = __ldg(&cnt_list[(size_t)s * n + i]);
            const float* c = sp + lay.c_radial + ((ti * S + s) * NR) * KR;
            float ml[KR], mk[KR];
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                float x = 0.f, y = 0.f;
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    x = fmaf(lam[q], c[q * KR + k], x);
                    y = fmaf(kap[q], c[q * KR + k], y);
                }
                ml[k] = x;
                mk[k] = y;
            }
            for (int e = lane; e < cnt; e += TPA) {
                int ent = list_entry(nbr_list, i, off + e, g.list_sa, g.list_se);
                float vx, vy, vz;
                entry_vector(pos4, ent, pi, g, vx, vy, vz);
                float r2 = vx * vx + vy * vy + vz * vz;
                if (r2 < rcr2) {
                    float r = sqrtf(r2);
                    float f[KR], df[KR];
                    basis_d<KR>(r, g.rc_radial, f, df);
                    float sl = 0.f, sk = 0.f;
#pragma unroll
                    for (int k = 0; k < KR; ++k) {
                        sl = fmaf(ml[k], df[k], sl);
                        sk = fmaf(mk[k], df[k], sk);
                    }
                    float ir = 1.f / r;
                    float ux = vx * ir, uy = vy * ir, uz = vz * ir;
                    scatter<BEC>(acc12, entry_index(ent), vx, vy, vz, sl * ux, sl * uy, sl * uz, sk * ux, sk * uy,
                                 sk * uz, fi, zi, w);
                }
            }
            off += cnt;
        }
        // angular entries
        off = 0;
        for (int s = 0; s < S; ++s) {
            const int cnt = __ldg(&cnt_ang[(size_t)s * n + i]);
            const float* c = sp + lay.c_angular + ((ti * S + s) * NA) * KA;
            for (int e = lane; e < cnt; e += TPA) {
                int ent = list_entry(nbr_ang, i, off + e, g.ang_sa, g.ang_se);
                float vx, vy, vz;
                entry_vector(pos4, ent, pi, g, vx, vy, vz);
                float r = sqrtf(vx * vx + vy * vy + vz * vz);
                float f[KA], df[KA];
                basis_d<KA>(r, g.rc_angular, f, df);
                float gn[NA], dgn[NA];
#pragma unroll
                for (int q = 0; q < NA; ++q) {
                    float x = 0.f, y = 0.f;
#pragma unroll
                    for (int k = 0; k < KA; ++k) {
                        x = fmaf(c[q * KA + k], f[k], x);
                        y = fmaf(c[q * KA + k], df[k], y);
                    }
                    gn[q] = x;
                    dgn[q] = y;
                }
                float ir = 1.f / r;
                float ux = vx * ir, uy = vy * ir, uz = vz * ir;
                float Y[NLM];
                harmonics(ux, uy, uz, Y);
                float out[2][3];
#pragma unroll
                for (int pass = 0; pass < (BEC ? 2 : 1); ++pass) {
                    const float* ph = my + pass * NANG;
                    float psi[NLM];
#pragma unroll
                    for (int m = 0; m < NLM; ++m) psi[m] = 0.f;
                    float rho = 0.f;
#pragma unroll
                    for (int q = 0; q < NA; ++q) {
                        float pq = 0.f;
#pragma unroll
                        for (int m = 0; m < NLM; ++m) {
                            float pv = ph[q * NLM + m];
                            pq = fmaf(pv, Y[m], pq);
                            psi[m] = fmaf(gn[q], pv, psi[m]);
                        }
                        rho = fmaf(dgn[q], pq, rho);
                    }
                    float gx, gy, gz;
                    harmonics_grad(ux, uy, uz, psi, gx, gy, gz);
                    float gu = gx * ux + gy * uy + gz * uz;
                    out[pass][0] = rho * ux + (gx - gu * ux) * ir;
                    out[pass][1] = rho * uy + (gy - gu * uy) * ir;
                    out[pass][2] = rho * uz + (gz - gu * uz) * ir;
                }
                if (!BEC) { out[1][0] = out[1][1] = out[1][2] = 0.f; }
                scatter<BEC>(acc12, entry_index(ent), vx, vy, vz, out[0][0], out[0][1], out[0][2], out[1][0],
                             out[1][1], out[1][2], fi, zi, w);
            }
            off += cnt;
        }
        if (TPA > 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) fi[k] = group_sum<TPA>(fi[k], gm);
            if (BEC) {
#pragma unroll
                for (int k = 0; k < 9; ++k) zi[k] = group_sum<TPA>(zi[k], gm);
            }
        }
        if (lane == 0) {
            // static electrostatic force q_i F^k / q + F^r and the BEC diagonal q~^c
            const float4 kf = fin.kfield[i], rf = fin.rfield[i];
            const float qt = seps * qc, ew = fin.e_weight;
            atomicAdd(&acc12[3 * i + 0], make_float4(fi[0] + ew * fmaf(qc, kf.x, rf.x), fi[1] + ew * fmaf(qc, kf.y, rf.y),
                                                     fi[2] + ew * fmaf(qc, kf.z, rf.z), zi[0] + qt));
            atomicAdd(&acc12[3 * i + 1], make_float4(zi[1], zi[2], zi[3], zi[4] + qt));
            atomicAdd(&acc12[3 * i + 2], make_float4(zi[5], zi[6], zi[7], zi[8] + qt));
        }
    }
    // block reduction of the virial, FP64 atomics
    __shared__ float red[9][4];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float v = w[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += (double)red[threadIdx.x][q];
        atomicAdd(&acc->virial[threadIdx.x], t);
    }
}

template <int TPA>
void fwd_launch(const float4* pos4, const int* nl, const int* cl, const int* na, const int* ca, int n, const Geom& g,
                const float* params, const ParamLayout& lay, float* ang, float* du, float* dq, float* u, float* q,
                float* des, const int* sidx, float4* fields, const float* gq, Accum* acc, cudaStream_t st,
                float* dtc) {
    const int threads = 128;
    long long blocks = ((long long)n * TPA + threads - 1) / threads;
    size_t smem = sizeof(float) * lay.total;
    k_desc_fwd<TPA><<<(unsigned)blocks, threads, smem, st>>>(pos4, nl, cl, na, ca, n, g, params, lay, ang, du, dq, u,
                                                             q, des, sidx, fields, gq, acc, dtc);
}

template <int TPA, bool BEC>
void bwd_launch(const float4* pos4, const int* nl, const int* cl, const int* na, const int* ca, int n, const Geom& g,
                const float* params, const ParamLayout& lay, const float* ang, const float* du, const float* dq,
                const float* q_raw, const FieldIn& fin, const Accum* acc_in, float4* acc12, Accum* acc,
                cudaStream_t st) {
    const int threads = 128;
    long long blocks = ((long long)n * TPA + threads - 1) / threads;
    size_t smem = sizeof(float) * (((lay.total + 3) & ~3) + (threads / TPA) * PHI_STRIDE);
    static std::atomic<int> attr[kMaxDevices];
    ensure_smem_attr(k_desc_bwd<TPA, BEC>, attr, 200 * 1024);
    k_desc_bwd<TPA, BEC><<<(unsigned)blocks, threads, smem, st>>>(pos4, nl, cl, na, ca, n, g, params, lay, ang, du, dq,
                                                                  q_raw, fin, acc_in, acc12, acc);
}

}  // namespace

int choose_tpa(int n) {
    // lanes per atom of the per-thread kernels (used for large systems)
    if (n <= 65536) return 2;
    return 1;
}

void launch_descriptor_forward(const float4* pos4, const int* nbr_list, const int* cnt_list, const int* nbr_ang,
                               const int* cnt_ang, int n, const Geom& g, const float* params, const ParamLayout& lay,
                               float* ang_coef, float* du, float* dq, float* u_out, float* q_out, float* des_out,
                               const int* sidx, float4* fields, const float* gq, Accum* acc, cudaStream_t st,
                               float* dtc) {
    if (n == 0) return;
    if (choose_tpa(n) == 2)
        fwd_launch<2>(pos4, nbr_list, cnt_list, nbr_ang, cnt_ang, n, g, params, lay, ang_coef, du, dq, u_out, q_out,
                      des_out, sidx, fields, gq, acc, st, dtc);
    else
        fwd_launch<1>(pos4, nbr_list, cnt_list, nbr_ang, cnt_ang, n, g, params, lay, ang_coef, du, dq, u_out, q_out,
                      des_out, sidx, fields, gq, acc, st, dtc);
}

void launch_descriptor_backward(const float4* pos4, const int* nbr_list, const int* cnt_list, const int* nbr_ang,
                                const int* cnt_ang, int n, const Geom& g, const float* params, const ParamLayout& lay,
                                const float* ang_coef, const float* du, const float* dq, const float* q_raw,
                                const FieldIn& fin, const Accum* acc_in, bool want_bec, float* acc12, Accum* acc,
                                cudaStream_t st) {
    if (n == 0) return;
    float4* a4 = reinterpret_cast<float4*>(acc12);
    if (want_bec)
        bwd_launch<2, true>(pos4, nbr_list, cnt_list, nbr_ang, cnt_ang, n, g, params, lay, ang_coef, du, dq, q_raw,
                            fin, acc_in, a4, acc, st);
    else
        bwd_launch<2, false>(pos4, nbr_list, cnt_list, nbr_ang, cnt_ang, n, g, params, lay, ang_coef, du, dq, q_raw,
                             fin, acc_in, a4, acc, st);
}

}  // namespace qnep
