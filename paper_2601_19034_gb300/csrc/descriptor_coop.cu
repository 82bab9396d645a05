// Warp-per-atom kernels of the force call for systems up to ~64k atoms.
//
// At a few thousand atoms a thread-per-atom kernel leaves most of the GPU idle
// (5000 atoms = 157 warps on 152 SMs).  Here one warp owns one atom and its 32
// lanes split every stage:
//   forward  (k_nbr_desc_coop): neighbour lists (built in shared memory, then
//            written grouped by species), radial sums over list entries, the
//            angular harmonic expansion A_{n,lm} (lanes over neighbours for g_n and
//            Y_lm, then lanes over the 120 coefficients), the 30 descriptor
//            components, the two-output network (lanes over hidden units) with
//            dU/dD and dq/dD (lanes over inputs), and the atom's Ewald phase row;
//   backward (k_desc_bwd_coop): adjoints lambda and kappa, dE/dA and the per-species
//            radial contractions in shared memory, then lanes over list entries for
//            the partial forces F_ij and charge derivatives a_ij (Sec. II.C,
//            Eq. bec_2), scattered with float4 atomics.
// The arithmetic is that of descriptor.cu (same descriptor, network and
// derivative formulas); only the work distribution differs.
#include "desc_math.cuh"
#include "nbr_common.cuh"

namespace qnep {

namespace {

constexpr int CW = 8;            // warps per block
constexpr int GY_STRIDE = 29;    // g_n (5) + Y_lm (24) of one angular neighbour

__host__ __device__ inline int coop_fwd_warp_floats(int cap_l, int cap_a) {
    return 2 * cap_l + 2 * cap_a + 32 * GY_STRIDE + NANG + 32 + 64;
}
__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

__global__ void __launch_bounds__(32 * CW) k_nbr_desc_coop(
    const float4* __restrict__ spos4, const int* __restrict__ cell_start, const int* __restrict__ sidx, int n, Geom g,
    const float* __restrict__ params, ParamLayout lay, int cap_l, int cap_a, int* __restrict__ nbr_list,
    int* __restrict__ cnt_list, int* __restrict__ nbr_ang, int* __restrict__ cnt_ang, float* __restrict__ ang_coef,
    float* __restrict__ du, float* __restrict__ dq, float* __restrict__ u_out, float* __restrict__ q_out,
    float* __restrict__ des_out, EwaldTab tab, int do_phase, float4* __restrict__ fields,
    const float* __restrict__ gq_in, Accum* __restrict__ acc, float* __restrict__ dtc,
    const int* __restrict__ skin_list, const int* __restrict__ skin_cnt, int cap_s) {
    extern __shared__ float csm[];
    float* sp = csm;
    for (int k = threadIdx.x; k < lay.total; k += blockDim.x) sp[k] = params[k];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* wbase = csm + round4(lay.total) + wib * coop_fwd_warp_floats(cap_l, cap_a);
    int* sl = reinterpret_cast<int*>(wbase);
    int* slt = sl + cap_l;
    int* sa = slt + cap_l;
    int* sat = sa + cap_a;
    float* gy = reinterpret_cast<float*>(sat + cap_a);
    float* abuf = gy + 32 * GY_STRIDE;
    float* dbuf = abuf + NANG;
    float* hb = dbuf + 32;
    __syncthreads();
    double su = 0.0, sq = 0.0, sg = 0.0;
    // lane 0 sums U, q (and the charge weights) of up to 8 atoms in FP32, then adds the
    // partial sums in FP64 (FP64 runs at 1/64 of the FP32 rate)
    float pu = 0.f, pq = 0.f, pg = 0.f;
    int np = 0;
    // dynamic scheduling: each warp takes the next atom until all are done
    for (;;) {
        int k = 0;
        if (lane == 0) k = (int)atomicAdd(&acc->work_fwd, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= n) break;
        const int S = lay.n_species;
        const float4 pk = __ldg(&spos4[k]);
        const int ti = __float_as_int(pk.w);
        int nl = 0, na = 0;
        // lists from a cell search, or from the Verlet-skin candidates when a skin is kept
        bool ovf = skin_list ? warp_lists_from_skin(spos4, skin_list + (size_t)k * cap_s, __ldg(&skin_cnt[k]), pk, g,
                                                    cap_l, cap_a, sl, slt, sa, sat, nl, na)
                             : warp_build_lists(spos4, cell_start, k, pk, g, cap_l, cap_a, sl, slt, sa, sat, nl, na);
        warp_write_grouped(sl, slt, nl, S, n, k, nbr_list, (size_t)cap_l, 1, cnt_list);
        warp_write_grouped(sa, sat, na, S, n, k, nbr_ang, (size_t)cap_a, 1, cnt_ang);
        if (ovf && lane == 0) atomicOr(&acc->status, 1u);

        // radial sums: lanes over list entries
        const float rcr2 = g.rc_radial * g.rc_radial;
        float dr[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) dr[q] = 0.f;
        for (int e = lane; e < nl; e += 32) {
            float vx, vy, vz;
            entry_vector(spos4, sl[e], pk, g, vx, vy, vz);
            float r2 = vx * vx + vy * vy + vz * vz;
            if (r2 < rcr2) {
                float f[KR];
                basis<KR>(sqrtf(r2), g.rc_radial, f);
                const float* c = sp + lay.c_radial + ((ti * S + slt[e]) * NR) * KR;
#pragma unroll
                for (int q = 0; q < NR; ++q)
#pragma unroll
                    for (int kk = 0; kk < KR; ++kk) dr[q] = fmaf(c[q * KR + kk], f[kk], dr[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dr[q] += __shfl_xor_sync(0xffffffffu, dr[q], o);
        }

        // angular expansion: lanes over neighbours (g_n, Y_lm to shared), then lane m < 24
        // accumulates A_{n,m} for the five n
        float av[NA] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int base = 0; base < na; base += 32) {
            const int e = base + lane;
            if (e < na) {
                float vx, vy, vz;
                entry_vector(spos4, sa[e], pk, g, vx, vy, vz);
                float r = sqrtf(vx * vx + vy * vy + vz * vz);
                float f[KA];
                basis<KA>(r, g.rc_angular, f);
                const float* c = sp + lay.c_angular + ((ti * S + sat[e]) * NA) * KA;
                float* row = gy + lane * GY_STRIDE;
#pragma unroll
                for (int q = 0; q < NA; ++q) {
                    float x = 0.f;
#pragma unroll
                    for (int kk = 0; kk < KA; ++kk) x = fmaf(c[q * KA + kk], f[kk], x);
                    row[q] = x;
                }
                float ir = 1.f / r, Y[NLM];
                harmonics(vx * ir, vy * ir, vz * ir, Y);
#pragma unroll
                for (int m = 0; m < NLM; ++m) row[NA + m] = Y[m];
            }
            __syncwarp();
            const int cnt = min(32, na - base);
            if (lane < NLM) {
                for (int r = 0; r < cnt; ++r) {
                    const float* row = gy + r * GY_STRIDE;
                    const float y = row[NA + lane];
#pragma unroll
                    for (int q = 0; q < NA; ++q) av[q] = fmaf(row[q], y, av[q]);
                }
            }
            __syncwarp();
        }
        if (lane < NLM) {
#pragma unroll
            for (int q = 0; q < NA; ++q) {
                abuf[q * NLM + lane] = av[q];
                if (ang_coef) ang_coef[(size_t)k * NANG + q * NLM + lane] = av[q];
            }
        }
        __syncwarp();

        // descriptor components: lane nu
        const float* scaler = sp + lay.scaler;
        float dv = 0.f;
        if (lane < NR) {
#pragma unroll
            for (int q = 0; q < NR; ++q)
                if (lane == q) dv = dr[q];
        } else if (lane < NR + 4 * NA) {
            const int l = (lane - NR) / NA + 1, q = (lane - NR) % NA;
            const int m0 = l == 1 ? 0 : (l == 2 ? 3 : (l == 3 ? 8 : 15));
            const int m1 = l == 1 ? 3 : (l == 2 ? 8 : (l == 3 ? 15 : 24));
            for (int m = m0; m < m1; ++m) {
                float a = abuf[q * NLM + m];
                dv = fmaf(c_wlm[m], a * a, dv);
            }
        } else if (lane < NDES) {
            const int q = lane - NR - 4 * NA;
            float a2[5], t[6], t2[6];
#pragma unroll
            for (int kk = 0; kk < 5; ++kk) a2[kk] = abuf[q * NLM + 3 + kk];
            tensor_from_a(a2, t);
            tensor_square(t, t2);
            dv = t2[0] * t[0] + t2[1] * t[1] + t2[2] * t[2] + 2.f * (t2[3] * t[3] + t2[4] * t[4] + t2[5] * t[5]);
        }
        if (lane < NDES) {
            dv *= scaler[lane];
            dbuf[lane] = dv;
            if (des_out) des_out[(size_t)__ldg(&sidx[k]) * NDES + lane] = dv;
        }
        // tensor-core network (precision form): hand the scaled descriptor (padded to 32) over
        if (dtc) dtc[(size_t)k * 32 + lane] = dv;
        __syncwarp();

        if (!dtc) {
        // network: lanes over hidden units, then over inputs for dU/dD and dq/dD
        const float* net = sp + lay.mlp + ti * lay.mlp_stride;
        float ue = 0.f, uq = 0.f;
        if (lane < NNEU) {
            const float* w0 = net + ParamLayout::W0 + lane * NDES;
            float pre = -net[ParamLayout::B0 + lane];
#pragma unroll
            for (int v = 0; v < NDES; ++v) pre = fmaf(w0[v], dbuf[v], pre);
            float h = tanhf(pre);
            float we = net[ParamLayout::W1E + lane], wq = net[ParamLayout::W1Q + lane];
            ue = we * h;
            uq = wq * h;
            float dh = 1.f - h * h;
            hb[lane] = we * dh;
            hb[32 + lane] = wq * dh;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ue += __shfl_xor_sync(0xffffffffu, ue, o);
            uq += __shfl_xor_sync(0xffffffffu, uq, o);
        }
        __syncwarp();
        if (du && lane < NDES) {
            float gu = 0.f, gq = 0.f;
#pragma unroll 6
            for (int mu = 0; mu < NNEU; ++mu) {
                float w = net[ParamLayout::W0 + mu * NDES + lane];
                gu = fmaf(hb[mu], w, gu);
                gq = fmaf(hb[32 + mu], w, gq);
            }
            du[(size_t)k * NDES + lane] = gu * scaler[lane];
            dq[(size_t)k * NDES + lane] = gq * scaler[lane];
        }
        if (lane == 0) {
            const float uu = ue - net[ParamLayout::B1E];
            const float qq = uq - net[ParamLayout::B1Q];
            u_out[k] = uu;
            q_out[k] = qq;
            pu += uu;   // a warp handles several atoms
            pq += qq;
        }
        }
        if (lane == 0) {
            if (gq_in) pg += __ldg(&gq_in[__ldg(&sidx[k])]);
            if (++np == 8) {
                su += (double)pu;
                sq += (double)pq;
                sg += (double)pg;
                pu = pq = pg = 0.f;
                np = 0;
            }
        }
        if (do_phase) {
            for (int e = lane; e < tab.nph; e += 32) tab.phase[(size_t)k * tab.nph + e] = phase_entry(pk, e, tab);
        }
        // clear this atom's accumulators of the later kernels (fields, forces / BEC)
        if (lane < 5) zero_atom_fields(fields, n, k, lane);
        __syncwarp();   // shared buffers are reused by the warp's next atom
    }
    // block sums of U and q (FP64), one atomic per block
    __shared__ double red[3][CW];
    if (lane == 0) {
        red[0][wib] = su + (double)pu;
        red[1][wib] = sq + (double)pq;
        red[2][wib] = sg + (double)pg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, cg = 0.0;
        for (int w = 0; w < CW; ++w) {
            a += red[0][w];
            b += red[1][w];
            cg += red[2][w];
        }
        atomicAdd(&acc->sum_u, a);
        atomicAdd(&acc->sum_q, b);
        if (gq_in) atomicAdd(&acc->sum_gq, cg);
    }
}

constexpr int BW_LK = 64;                       // lambda (30) and kappa (30)
constexpr int BW_PHI = 2 * NANG;                // dE/dA weighted by lambda and kappa
constexpr int BW_MU = 2 * MAX_SPECIES * KR;     // radial contractions per species
constexpr int BW_WARP = BW_LK + BW_PHI + BW_MU;

template <bool BEC, bool AV>
__device__ __forceinline__ void scatter_entry(float4* __restrict__ acc12, float* __restrict__ avir, int j, float vx,
                                              float vy, float vz, float fx, float fy, float fz, float ax, float ay,
                                              float az, float fi[3], float zi[9], float w[9]) {
    if (AV) {
        // per-atom virial: the entry (i -> j) adds -r_ij (x) F_ij to W_j (Sec. II.C, Eq. per-atom_virial)
        float4* a4 = reinterpret_cast<float4*>(avir + (size_t)AVIR * j);
        atomicAdd(&a4[0], make_float4(-vx * fx, -vx * fy, -vx * fz, -vy * fx));
        atomicAdd(&a4[1], make_float4(-vy * fy, -vy * fz, -vz * fx, -vz * fy));
        atomicAdd(avir + (size_t)AVIR * j + 8, -vz * fz);
    }
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

// Three blocks per SM without BEC (80 registers; 1 M-atom Mg-water backward 3.29 -> 2.73 ms
// against two blocks at 128), two with BEC (its larger scatter spills at 80 registers).
template <bool BEC, bool AV>
__global__ void __launch_bounds__(32 * CW, (BEC || AV) ? 2 : 3) k_desc_bwd_coop(
    const float4* __restrict__ spos4, const int* __restrict__ nbr_list, const int* __restrict__ cnt_list,
    const int* __restrict__ nbr_ang, const int* __restrict__ cnt_ang, int n, Geom g, const float* __restrict__ params,
    ParamLayout lay, const float* __restrict__ ang_coef, const float* __restrict__ du, const float* __restrict__ dqp,
    const float* __restrict__ q_raw, FieldIn fin, const Accum* __restrict__ acc_in, float4* __restrict__ acc12,
    Accum* __restrict__ acc, float* __restrict__ avir) {
    extern __shared__ float csm[];
    float* sp = csm;
    for (int k = threadIdx.x; k < lay.total; k += blockDim.x) sp[k] = params[k];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* lk = csm + round4(lay.total) + wib * BW_WARP;
    float* ph = lk + BW_LK;
    float* mu = ph + BW_PHI;
    const ChargeScalars cs = block_charge_scalars(acc_in, fin.q_target, n, fin.mode, fin.alpha);   // synchronises
    float w[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) w[q] = 0.f;
    // dynamic scheduling: each warp takes the next atom until all are done
    for (;;) {
        int k = 0;
        if (lane == 0) k = (int)atomicAdd(&acc->work_bwd, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= n) break;
        const int S = lay.n_species;
        const float4 pk = __ldg(&spos4[k]);
        const int ti = __float_as_int(pk.w);
        const float seps = sp[lay.sqrt_eps];
        // every global load of the prologue is issued first (they are independent), then the
        // arithmetic; adjoints travel between lanes by shuffles
        const float duv = lane < NDES ? __ldg(&du[(size_t)k * NDES + lane]) : 0.f;
        const float dqv = lane < NDES ? __ldg(&dqp[(size_t)k * NDES + lane]) : 0.f;
        float av[4];
#pragma unroll
        for (int s4 = 0; s4 < 4; ++s4) {
            const int el = lane + 32 * s4;
            av[s4] = el < NANG ? __ldg(&ang_coef[(size_t)k * NANG + el]) : 0.f;
        }
        // lanes q < NA: the l = 2 coefficients of radial function q and the 4-body derivatives
        float dd4[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (lane < NA) {
            float a2[5], t[6], t2[6];
#pragma unroll
            for (int kk = 0; kk < 5; ++kk) a2[kk] = __ldg(&ang_coef[(size_t)k * NANG + lane * NLM + 3 + kk]);
            tensor_from_a(a2, t);
            tensor_square(t, t2);
            dd4[0] = 3.f * (t2[2] * (1.f / 3.f) - (t2[0] + t2[1]) * (1.f / 6.f));
            dd4[1] = 6.f * t2[4];
            dd4[2] = 6.f * t2[5];
            dd4[3] = 1.5f * (t2[0] - t2[1]);
            dd4[4] = 6.f * t2[3];
        }
        float qc, phi_k;
        assemble_potential(fin, cs, q_raw, k, qc, phi_k);
        const float wq = charge_adjoint_weight(fin, cs, k, phi_k - cs.phibar);
        const float lkl = fmaf(wq, dqv, fin.e_weight * duv);   // lambda_v in lane v
        const float lkk = seps * dqv;                         // kappa_v in lane v
        // dE/dA_{n,lm} for both adjoints
#pragma unroll
        for (int s4 = 0; s4 < 4; ++s4) {
            const int el = lane + 32 * s4;
            const int q = el / NLM, m = el - q * NLM;
            const int l = m < 3 ? 1 : (m < 8 ? 2 : (m < 15 ? 3 : 4));
            const int dl = min(NR + (l - 1) * NA + q, 31);
            const float ldl = __shfl_sync(0xffffffffu, lkl, dl);
            const float kdl = __shfl_sync(0xffffffffu, lkk, dl);
            const int d4 = min(NR + 4 * NA + q, 31);
            const float l4 = __shfl_sync(0xffffffffu, lkl, d4);
            const float k4 = __shfl_sync(0xffffffffu, lkk, d4);
            const int qs = min(q, NA - 1);
            float dd = 0.f;
#pragma unroll
            for (int kk = 0; kk < 5; ++kk) {
                const float v = __shfl_sync(0xffffffffu, dd4[kk], qs);
                if (m == 3 + kk) dd = v;
            }
            if (el < NANG) {
                float pl = 2.f * c_wlm[m] * av[s4] * ldl;
                float pkk = 2.f * c_wlm[m] * av[s4] * kdl;
                if (l == 2) {
                    pl = fmaf(l4, dd, pl);
                    pkk = fmaf(k4, dd, pkk);
                }
                ph[el] = pl;
                ph[NANG + el] = pkk;
            }
        }
        // radial contractions mu[which][s][k] = sum_n adjoint_n c_R[ti][s][n][k]
        float lr[NR], kr[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            lr[q] = __shfl_sync(0xffffffffu, lkl, q);
            kr[q] = __shfl_sync(0xffffffffu, lkk, q);
        }
        for (int idx = lane; idx < 2 * S * KR; idx += 32) {
            const int which = idx / (S * KR), rem = idx - which * S * KR, s = rem / KR, kk = rem - s * KR;
            const float* c = sp + lay.c_radial + ((ti * S + s) * NR) * KR;
            float x = 0.f;
#pragma unroll
            for (int q = 0; q < NR; ++q) x = fmaf(which ? kr[q] : lr[q], c[q * KR + kk], x);
            mu[(which * MAX_SPECIES + s) * KR + kk] = x;
        }
        __syncwarp();

        float fi[3] = {0.f, 0.f, 0.f}, zi[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) zi[q] = 0.f;
        int tot_l = 0, tot_a = 0;
        for (int s = 0; s < S; ++s) {
            tot_l += __ldg(&cnt_list[(size_t)s * n + k]);
            tot_a += __ldg(&cnt_ang[(size_t)s * n + k]);
        }
        const float rcr2 = g.rc_radial * g.rc_radial;
        auto radial_entry = [&](int ent, const float4& pj) {
            float tx, ty, tz;
            entry_shift(ent, tx, ty, tz);
            float shx, shy, shz;
            shift_vector(g, tx, ty, tz, shx, shy, shz);
            const float vx = (pj.x - pk.x) + shx, vy = (pj.y - pk.y) + shy, vz = (pj.z - pk.z) + shz;
            const float r2 = vx * vx + vy * vy + vz * vz;
            if (r2 < rcr2) {
                const int tj = __float_as_int(pj.w);
                float r = sqrtf(r2), f[KR], df[KR];
                basis_d<KR>(r, g.rc_radial, f, df);
                const float* ml = mu + tj * KR;
                const float* mk = mu + (MAX_SPECIES + tj) * KR;
                float sl = 0.f, skk = 0.f;
#pragma unroll
                for (int kk = 0; kk < KR; ++kk) {
                    sl = fmaf(ml[kk], df[kk], sl);
                    skk = fmaf(mk[kk], df[kk], skk);
                }
                float ir = 1.f / r, ux = vx * ir, uy = vy * ir, uz = vz * ir;
                scatter_entry<BEC, AV>(acc12, avir, entry_index(ent), vx, vy, vz, sl * ux, sl * uy, sl * uz, skk * ux,
                                   skk * uy, skk * uz, fi, zi, w);
            }
        };
        // two rounds of entries per iteration: both entries and both positions are loaded
        // before either is used
        for (int e0 = lane; e0 < tot_l; e0 += 64) {
            const int e1 = e0 + 32;
            const bool has1 = e1 < tot_l;
            const int ent0 = __ldg(&nbr_list[(size_t)k * g.list_sa + e0]);
            const int ent1 = has1 ? __ldg(&nbr_list[(size_t)k * g.list_sa + e1]) : ent0;
            const float4 p0 = __ldg(&spos4[entry_index(ent0)]);
            const float4 p1 = __ldg(&spos4[entry_index(ent1)]);
            radial_entry(ent0, p0);
            if (has1) radial_entry(ent1, p1);
        }
        for (int e = lane; e < tot_a; e += 32) {
            const int ent = __ldg(&nbr_ang[(size_t)k * g.ang_sa + e]);
            const int j = entry_index(ent);
            float vx, vy, vz;
            entry_vector(spos4, ent, pk, g, vx, vy, vz);
            const int tj = __float_as_int(__ldg(&spos4[j]).w);
            float r = sqrtf(vx * vx + vy * vy + vz * vz);
            float f[KA], df[KA];
            basis_d<KA>(r, g.rc_angular, f, df);
            const float* c = sp + lay.c_angular + ((ti * S + tj) * NA) * KA;
            float gn[NA], dgn[NA];
#pragma unroll
            for (int q = 0; q < NA; ++q) {
                float x = 0.f, y = 0.f;
#pragma unroll
                for (int kk = 0; kk < KA; ++kk) {
                    x = fmaf(c[q * KA + kk], f[kk], x);
                    y = fmaf(c[q * KA + kk], df[kk], y);
                }
                gn[q] = x;
                dgn[q] = y;
            }
            float ir = 1.f / r, ux = vx * ir, uy = vy * ir, uz = vz * ir;
            float Y[NLM];
            harmonics(ux, uy, uz, Y);
            float out[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
            for (int pass = 0; pass < (BEC ? 2 : 1); ++pass) {
                const float* pp = ph + pass * NANG;
                float psi[NLM];
#pragma unroll
                for (int m = 0; m < NLM; ++m) psi[m] = 0.f;
                float rho = 0.f;
#pragma unroll
                for (int q = 0; q < NA; ++q) {
                    float pq = 0.f;
#pragma unroll
                    for (int m = 0; m < NLM; ++m) {
                        float pv = pp[q * NLM + m];
                        pq = fmaf(pv, Y[m], pq);
                        psi[m] = fmaf(gn[q], pv, psi[m]);
                    }
                    rho = fmaf(dgn[q], pq, rho);
                }
                float gx, gyy, gz;
                harmonics_grad(ux, uy, uz, psi, gx, gyy, gz);
                float gu = gx * ux + gyy * uy + gz * uz;
                out[pass][0] = rho * ux + (gx - gu * ux) * ir;
                out[pass][1] = rho * uy + (gyy - gu * uy) * ir;
                out[pass][2] = rho * uz + (gz - gu * uz) * ir;
            }
            scatter_entry<BEC, AV>(acc12, avir, j, vx, vy, vz, out[0][0], out[0][1], out[0][2], out[1][0], out[1][1], out[1][2],
                               fi, zi, w);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < 3; ++q) fi[q] += __shfl_xor_sync(0xffffffffu, fi[q], o);
            if (BEC) {
#pragma unroll
                for (int q = 0; q < 9; ++q) zi[q] += __shfl_xor_sync(0xffffffffu, zi[q], o);
            }
        }
        if (lane == 0) {
            // static electrostatic force q_k F^k / q + F^r and the BEC diagonal q~^c
            const float4 kf = fin.kfield[k], rf = fin.rfield[k];
            const float qt = seps * qc, ew = fin.e_weight;
            atomicAdd(&acc12[3 * k + 0], make_float4(fi[0] + ew * fmaf(qc, kf.x, rf.x), fi[1] + ew * fmaf(qc, kf.y, rf.y),
                                                     fi[2] + ew * fmaf(qc, kf.z, rf.z), zi[0] + qt));
            atomicAdd(&acc12[3 * k + 1], make_float4(zi[1], zi[2], zi[3], zi[4] + qt));
            atomicAdd(&acc12[3 * k + 2], make_float4(zi[5], zi[6], zi[7], zi[8] + qt));
        }
        __syncwarp();   // shared buffers are reused by the warp's next atom
    }
    // block reduction of the virial, FP64 atomics
    __shared__ float red[9][CW];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        float v = w[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][wib] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int q = 0; q < CW; ++q) t += (double)red[threadIdx.x][q];
        atomicAdd(&acc->virial[threadIdx.x], t);
    }
}

}  // namespace

int num_sms() {
    static std::atomic<int> cache[kMaxDevices];
    const int d = device_slot();
    int v = cache[d].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v < 1) v = 1;
        cache[d].store(v, std::memory_order_relaxed);
    }
    return v;
}

size_t coop_forward_smem(const ParamLayout& lay, int cap_l, int cap_a) {
    return sizeof(float) * ((size_t)round4(lay.total) + (size_t)CW * coop_fwd_warp_floats(cap_l, cap_a));
}

void launch_nbr_desc_coop(const float4* spos4, const int* cell_start, const int* sidx, int n, const Geom& g,
                          const float* params, const ParamLayout& lay, int cap_l, int cap_a, int* nbr_list,
                          int* cnt_list, int* nbr_ang, int* cnt_ang, float* ang_coef, float* du, float* dq, float* u,
                          float* q, float* des_out, const EwaldTab& tab, bool do_phase, float4* fields,
                          const float* gq, Accum* acc, cudaStream_t st, float* dtc, const int* skin_list,
                          const int* skin_cnt, int cap_s) {
    if (n == 0) return;
    static std::atomic<int> attr[kMaxDevices];
    ensure_smem_attr(k_nbr_desc_coop, attr, 220 * 1024);
    const size_t smem = coop_forward_smem(lay, cap_l, cap_a);
    static std::atomic<long long> occ[kMaxDevices];
    const int per_sm = cached_occupancy(k_nbr_desc_coop, occ, 32 * CW, smem);
    int blocks = (n + CW - 1) / CW;
    if (blocks > per_sm * num_sms()) blocks = per_sm * num_sms();
    k_nbr_desc_coop<<<blocks, 32 * CW, smem, st>>>(
        spos4, cell_start, sidx, n, g, params, lay, cap_l, cap_a, nbr_list, cnt_list, nbr_ang, cnt_ang, ang_coef, du,
        dq, u, q, des_out, tab, do_phase ? 1 : 0, fields, gq, acc, dtc, skin_list, skin_cnt, cap_s);
}

void launch_desc_bwd_coop(const float4* spos4, const int* nbr_list, const int* cnt_list, const int* nbr_ang,
                          const int* cnt_ang, int n, const Geom& g, const float* params, const ParamLayout& lay,
                          const float* ang_coef, const float* du, const float* dq, const float* q_raw,
                          const FieldIn& fin, const Accum* acc_in, bool want_bec, float* acc12, Accum* acc,
                          cudaStream_t st, float* avir) {
    if (n == 0) return;
    size_t smem = sizeof(float) * ((size_t)round4(lay.total) + (size_t)CW * BW_WARP);
    float4* a4 = reinterpret_cast<float4*>(acc12);
    int blocks = (n + CW - 1) / CW;
    auto run = [&](auto kernel, std::atomic<int>* attr, std::atomic<long long>* occ) {
        ensure_smem_attr(kernel, attr, 100 * 1024);
        const int per_sm = cached_occupancy(kernel, occ, 32 * CW, smem);
        if (blocks > per_sm * num_sms()) blocks = per_sm * num_sms();
        kernel<<<blocks, 32 * CW, smem, st>>>(spos4, nbr_list, cnt_list, nbr_ang, cnt_ang, n, g, params, lay, ang_coef,
                                              du, dq, q_raw, fin, acc_in, a4, acc, avir);
    };
    static std::atomic<int> at[4][kMaxDevices];
    static std::atomic<long long> oc[4][kMaxDevices];
    if (want_bec && avir) run(k_desc_bwd_coop<true, true>, at[3], oc[3]);
    else if (want_bec) run(k_desc_bwd_coop<true, false>, at[2], oc[2]);
    else if (avir) run(k_desc_bwd_coop<false, true>, at[1], oc[1]);
    else run(k_desc_bwd_coop<false, false>, at[0], oc[0]);
}

}  // namespace qnep
