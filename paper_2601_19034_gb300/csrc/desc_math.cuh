// Device helpers of the descriptor kernels: harmonic polynomials, Chebyshev
// basis and its derivative, the 4-body tensor, list access and Ewald phases.
#pragma once

#include "qnep_internal.cuh"

namespace qnep {
namespace {

__constant__ float c_wlm[NLM] = {1.f, 1.f, 1.f,
                                 0.25f, 3.f, 3.f, 0.75f, 3.f,
                                 0.25f, 0.375f, 0.375f, 3.75f, 15.f, 0.625f, 0.625f,
                                 1.f / 64.f, 0.625f, 0.625f, 0.3125f, 1.25f, 4.375f, 4.375f, 35.f / 64.f, 8.75f};

__device__ __forceinline__ void harmonics(float x, float y, float z, float Y[NLM]) {
    float x2 = x * x, y2 = y * y, z2 = z * z;
    Y[0] = z; Y[1] = x; Y[2] = y;
    Y[3] = 3.f * z2 - 1.f; Y[4] = x * z; Y[5] = y * z; Y[6] = x2 - y2; Y[7] = x * y;
    float a5 = 5.f * z2 - 1.f;
    Y[8] = z * (5.f * z2 - 3.f); Y[9] = x * a5; Y[10] = y * a5; Y[11] = z * (x2 - y2); Y[12] = x * y * z;
    Y[13] = x * (x2 - 3.f * y2); Y[14] = y * (3.f * x2 - y2);
    float a7 = 7.f * z2 - 3.f, b7 = 7.f * z2 - 1.f;
    Y[15] = (35.f * z2 - 30.f) * z2 + 3.f; Y[16] = x * z * a7; Y[17] = y * z * a7; Y[18] = (x2 - y2) * b7;
    Y[19] = x * y * b7; Y[20] = z * x * (x2 - 3.f * y2); Y[21] = z * y * (3.f * x2 - y2);
    Y[22] = x2 * x2 - 6.f * x2 * y2 + y2 * y2; Y[23] = x * y * (x2 - y2);
}

// g = sum_lm psi_lm grad_u Y_lm(u) (gradient of the polynomials, not yet projected)
__device__ __forceinline__ void harmonics_grad(float x, float y, float z, const float p[NLM], float& gx,
                                               float& gy, float& gz) {
    float x2 = x * x, y2 = y * y, z2 = z * z;
    gx = p[1] + p[4] * z + p[6] * 2.f * x + p[7] * y;
    gy = p[2] + p[5] * z - p[6] * 2.f * y + p[7] * x;
    gz = p[0] + p[3] * 6.f * z + p[4] * x + p[5] * y;
    float a5 = 5.f * z2 - 1.f;
    gx += p[9] * a5 + p[11] * 2.f * x * z + p[12] * y * z + p[13] * 3.f * (x2 - y2) + p[14] * 6.f * x * y;
    gy += p[10] * a5 - p[11] * 2.f * y * z + p[12] * x * z - p[13] * 6.f * x * y + p[14] * 3.f * (x2 - y2);
    gz += p[8] * (15.f * z2 - 3.f) + p[9] * 10.f * x * z + p[10] * 10.f * y * z + p[11] * (x2 - y2) + p[12] * x * y;
    float a7 = 7.f * z2 - 3.f, b7 = 7.f * z2 - 1.f, zc = z * a7;
    gx += p[16] * zc + p[18] * 2.f * x * b7 + p[19] * y * b7 + p[20] * 3.f * z * (x2 - y2) + p[21] * 6.f * x * y * z +
          p[22] * (4.f * x2 * x - 12.f * x * y2) + p[23] * (3.f * x2 * y - y2 * y);
    gy += p[17] * zc - p[18] * 2.f * y * b7 + p[19] * x * b7 - p[20] * 6.f * x * y * z + p[21] * 3.f * z * (x2 - y2) +
          p[22] * (4.f * y2 * y - 12.f * x2 * y) + p[23] * (x2 * x - 3.f * x * y2);
    gz += p[15] * (140.f * z2 - 60.f) * z + p[16] * x * (21.f * z2 - 3.f) + p[17] * y * (21.f * z2 - 3.f) +
          p[18] * 14.f * z * (x2 - y2) + p[19] * 14.f * x * y * z + p[20] * x * (x2 - 3.f * y2) +
          p[21] * y * (3.f * x2 - y2);
}

template <int K>
__device__ __forceinline__ void basis(float r, float rc, float f[K]) {
    float rr = r / rc;
    float fc = 0.5f * (1.f + cospif(rr));
    float x = 2.f * (rr - 1.f) * (rr - 1.f) - 1.f;
    float t0 = 1.f, t1 = x;
    f[0] = fc;
    if (K > 1) f[1] = 0.5f * (x + 1.f) * fc;
#pragma unroll
    for (int k = 2; k < K; ++k) {
        float t2 = 2.f * x * t1 - t0;
        f[k] = 0.5f * (t2 + 1.f) * fc;
        t0 = t1;
        t1 = t2;
    }
}

template <int K>
__device__ __forceinline__ void basis_d(float r, float rc, float f[K], float df[K]) {
    float rr = r / rc;
    float s, c;
    sincospif(rr, &s, &c);
    float fc = 0.5f * (1.f + c);
    float dfc = -0.5f * 3.14159265358979f / rc * s;
    float x = 2.f * (rr - 1.f) * (rr - 1.f) - 1.f;
    float dx = 4.f * (rr - 1.f) / rc;
    float t0 = 1.f, t1 = x, d0 = 0.f, d1 = 1.f;
    f[0] = fc;
    df[0] = dfc;
    if (K > 1) {
        f[1] = 0.5f * (x + 1.f) * fc;
        df[1] = 0.5f * (dx * fc + (x + 1.f) * dfc);
    }
#pragma unroll
    for (int k = 2; k < K; ++k) {
        float t2 = 2.f * x * t1 - t0;
        float d2 = 2.f * t1 + 2.f * x * d1 - d0;   // T_k' by differentiating the recurrence
        f[k] = 0.5f * (t2 + 1.f) * fc;
        df[k] = 0.5f * (d2 * dx * fc + (t2 + 1.f) * dfc);
        t0 = t1; t1 = t2; d0 = d1; d1 = d2;
    }
}

template <int TPA>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, TPA);
    return v;
}

template <int TPA>
__device__ __forceinline__ unsigned group_mask() {
    if (TPA == 32) return 0xffffffffu;
    unsigned lane = threadIdx.x & 31;
    return ((1u << TPA) - 1u) << (lane & ~(unsigned)(TPA - 1));
}

__device__ __forceinline__ void entry_vector(const float4* __restrict__ pos4, int e, const float4& pi,
                                             const Geom& g, float& vx, float& vy, float& vz) {
    int j = entry_index(e);
    float tx, ty, tz;
    entry_shift(e, tx, ty, tz);
    float4 pj = __ldg(&pos4[j]);
    float sx, sy, sz;
    shift_vector(g, tx, ty, tz, sx, sy, sz);
    vx = (pj.x - pi.x) + sx;
    vy = (pj.y - pi.y) + sy;
    vz = (pj.z - pi.z) + sz;
}

// 4-body: T_n from the l = 2 expansion coefficients (unnormalised harmonics 3..7)
__device__ __forceinline__ void tensor_from_a(const float a[5], float t[6]) {
    // a: (3z^2-1, xz, yz, x^2-y^2, xy) sums; t: xx, yy, zz, xy, xz, yz
    float zz = a[0] * (1.f / 3.f);
    t[0] = 0.5f * (a[3] - zz);
    t[1] = 0.5f * (-a[3] - zz);
    t[2] = zz;
    t[3] = a[4];
    t[4] = a[1];
    t[5] = a[2];
}

__device__ __forceinline__ void tensor_square(const float t[6], float s[6]) {
    s[0] = t[0] * t[0] + t[3] * t[3] + t[4] * t[4];
    s[1] = t[3] * t[3] + t[1] * t[1] + t[5] * t[5];
    s[2] = t[4] * t[4] + t[5] * t[5] + t[2] * t[2];
    s[3] = t[0] * t[3] + t[3] * t[1] + t[4] * t[5];
    s[4] = t[0] * t[4] + t[3] * t[5] + t[4] * t[2];
    s[5] = t[3] * t[4] + t[1] * t[5] + t[5] * t[2];
}


// Entry e of sorted atom k in a list with strides (atom, entry).
__device__ __forceinline__ int list_entry(const int* __restrict__ lst, int k, int e, int sa, int se) {
    return __ldg(&lst[(size_t)k * sa + (size_t)e * se]);
}

__device__ __forceinline__ float2 phase_factor(float x, int nn, float il_hi, float il_lo) {
    // exp(-i 2 pi nn x / L) with the fractional part of nn x / L carried to ~2^-48:
    // nn x = p + pe exactly, p il_hi = u + ue exactly, u - rint(u) exactly
    float fn = (float)nn;
    float p = fn * x;
    float pe = fmaf(fn, x, -p);
    float u = p * il_hi;
    float ue = fmaf(p, il_hi, -u);
    float lo = ue + fmaf(p, il_lo, pe * il_hi);
    float fr = (u - rintf(u)) + lo;
    float sn, cs;
    sincospif(2.f * fr, &sn, &cs);
    return make_float2(cs, -sn);
}

// exp(-i 2 pi nn s_c) of a general cell, s_c = sum_d r_d Hi[d][c] (H^-1 as float pairs hi_hi +
// hi_lo, row-major): each of the three products nn r_d Hi[d][c] is reduced to its fractional part
// exactly (as in phase_factor), then the three fractions are added
__device__ __forceinline__ float2 phase_factor_frac(const float4& p, int nn, int c, const float* hi_hi,
                                                    const float* hi_lo) {
    const float fn = (float)nn;
    const float r[3] = {p.x, p.y, p.z};
    float fr = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float h = hi_hi[3 * d + c], hl = hi_lo[3 * d + c];
        const float pp = fn * r[d];
        const float pe = fmaf(fn, r[d], -pp);
        const float u = pp * h;
        const float ue = fmaf(pp, h, -u);
        const float lo = ue + fmaf(pp, hl, pe * h);
        fr += (u - rintf(u)) + lo;
    }
    float sn, cs;
    sincospif(2.f * fr, &sn, &cs);
    return make_float2(cs, -sn);
}

__device__ __forceinline__ float2 phase_factor_tri(const float4& p, int nn, int c, const EwaldTab& tab) {
    return phase_factor_frac(p, nn, c, tab.hi_hi, tab.hi_lo);
}

// Row entry e of an atom's phase row: X(n1), Y(n2) or Z(n3) factor (see EwaldTab).
__device__ __forceinline__ float2 phase_entry(const float4& p, int e, const EwaldTab& tab) {
    if (tab.tri) {
        if (e < tab.yoff) return phase_factor_tri(p, e, 0, tab);
        if (e < tab.zoff) return phase_factor_tri(p, e - tab.yoff - tab.n2max, 1, tab);
        return phase_factor_tri(p, e - tab.zoff - tab.n3max, 2, tab);
    }
    if (e < tab.yoff) return phase_factor(p.x, e, tab.invl_hi[0], tab.invl_lo[0]);
    if (e < tab.zoff) return phase_factor(p.y, e - tab.yoff - tab.n2max, tab.invl_hi[1], tab.invl_lo[1]);
    return phase_factor(p.z, e - tab.zoff - tab.n3max, tab.invl_hi[2], tab.invl_lo[2]);
}

// Per-atom field accumulators, one float4 array of 5 n entries:
//   kfield [n] (F^k / q, phi^k) | rfield [n] (F^r, phi^r) | acc12 [3 n] (F, Z row-major)
// Entry part (0..4) of atom k is cleared by the forward kernels.
__device__ __forceinline__ void zero_atom_fields(float4* __restrict__ base, int n, int k, int part) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (part == 0) base[k] = z;
    else if (part == 1) base[(size_t)n + k] = z;
    else base[2 * (size_t)n + 3 * (size_t)k + (part - 2)] = z;
}

// Block-uniform scalars of the charge correction and the adjoint: the shift
// delta = (Q / sqrt(eps_inf) - sum q) / N of the corrected charges, the mean potential
// (sum phi^k + sum phi^r + sum phi^s) / N with sum_k phi^s_k = -2 k_e alpha / sqrt(pi) Q / sqrt(eps_inf),
// and the mean charge weight of a vector-Jacobian product.  Thread 0 forms each numerator
// from the FP64 sums, rounds it to FP32 and scales it by 1/N: an FP64 division is a long
// instruction sequence on a unit with 1/64 of the FP32 rate, so it is not evaluated per
// atom.  Every thread of the block calls this once, before any early exit (it synchronises).
struct ChargeScalars {
    float delta, phibar, gq_mean;
};

__device__ __forceinline__ ChargeScalars block_charge_scalars(const Accum* __restrict__ acc_in, float q_target, int n,
                                                              int mode, float alpha) {
    __shared__ ChargeScalars cs_shared;
    if (threadIdx.x == 0) {
        const float inv_n = n > 0 ? 1.f / (float)n : 0.f;
        const double self = mode == 1 ? -2.0 * (double)KE * (double)alpha * 0.564189583547756287 : 0.0;
        ChargeScalars c;
        c.delta = (float)((double)q_target - acc_in->sum_q) * inv_n;
        c.phibar = (float)(acc_in->sum_phi + self * (double)q_target) * inv_n;
        c.gq_mean = (float)acc_in->sum_gq * inv_n;
        cs_shared = c;
    }
    __syncthreads();
    return cs_shared;
}

// Corrected charge q^c_k and total potential phi_k = phi^k + phi^r + phi^s.
// Weight of dq_k/dD in the adjoint: g_E (phi_k - mean phi) + (g_q,k - mean g_q)
// (the charge correction makes dq^c_j/dq_l = delta_jl - 1/N).
__device__ __forceinline__ float charge_adjoint_weight(const FieldIn& fin, const ChargeScalars& cs, int k, float dphi) {
    float w = fin.e_weight * dphi;
    if (fin.gq) w += __ldg(&fin.gq[__ldg(&fin.sidx[k])]) - cs.gq_mean;
    return w;
}

__device__ __forceinline__ void assemble_potential(const FieldIn& fin, const ChargeScalars& cs,
                                                   const float* __restrict__ q_raw, int k, float& qc, float& phi_k) {
    qc = __ldg(&q_raw[k]) + cs.delta;
    const float self = fin.mode == 1 ? -2.f * KE * fin.alpha * 0.564189583547756287f : 0.f;
    phi_k = fin.kfield[k].w + fin.rfield[k].w + self * qc;
}

}  // namespace
}  // namespace qnep
