// Ewald reciprocal space (Sec. II.B, Eqs. U_k and S_k; forces and virial of Sec. II.C).
//
// Wave vectors of the half space (k and -k give conjugate terms, so the full
// sums are twice the half-space sums), |k| < kmax, k = 0 excluded.
//   S(k)  = sum_i q_i exp(-i k.r_i)                       (FP32 terms, FP64 accumulation)
//   U^k   = k_e sum_{k != 0} G(k) |S(k)|^2 = 2 k_e sum_half G |S|^2            (FP64)
//   W^k   = k_e sum G |S|^2 B,  B = I - (2/(4 alpha^2) + 2/k^2) k k^T   (Eq. virial-kspace-total)
// Per-atom phase factors are separable, exp(-i k.r) = X(n1) Y(n2) Z(n3), and
// each is evaluated directly from an exactly reduced phase (no recurrences):
// the product n x / L is formed with an error-free product and 1/L as a float
// pair, so the phase error stays at float rounding of the reduced angle.
#include "qnep_internal.cuh"

namespace qnep {

namespace {

__device__ __forceinline__ float2 phase_factor(float x, int nn, float il_hi, float il_lo) {
    // exp(-i 2 pi nn x / L) with the fractional part of nn x / L carried to ~2^-48
    float fn = (float)nn;
    float p = fn * x;
    float pe = fmaf(fn, x, -p);                    // exact: nn x = p + pe
    float u = p * il_hi;
    float ue = fmaf(p, il_hi, -u);                 // exact: p il_hi = u + ue
    float lo = ue + fmaf(p, il_lo, pe * il_hi);
    float fr = (u - rintf(u)) + lo;                // u - rint(u) is exact
    float s, c;
    sincospif(2.f * fr, &s, &c);
    return make_float2(c, -s);
}

__global__ void k_phases(const float4* __restrict__ pos4, int n, EwaldTab tab) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * tab.nph) return;
    int i = (int)(t / tab.nph);
    int e = (int)(t - (long long)i * tab.nph);
    float4 p = __ldg(&pos4[i]);
    float2 v;
    if (e < tab.yoff) {
        v = phase_factor(p.x, e, tab.invl_hi[0], tab.invl_lo[0]);
    } else if (e < tab.zoff) {
        v = phase_factor(p.y, e - tab.yoff - tab.n2max, tab.invl_hi[1], tab.invl_lo[1]);
    } else {
        v = phase_factor(p.z, e - tab.zoff - tab.n3max, tab.invl_hi[2], tab.invl_lo[2]);
    }
    tab.phase[t] = v;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// One thread = one 8-wide chunk of a column x one quarter of the block's atoms.
// The block reduces its four partial sums in FP64 and adds them to S with FP64 atomics.
constexpr int SK_WARPS = 4;

__global__ void __launch_bounds__(32 * SK_WARPS) k_sk(const float* __restrict__ q_raw, const Accum* __restrict__ acc,
                                                      int n, float q_target, int span, EwaldTab tab) {
    __shared__ double red[SK_WARPS][8][2][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = blockIdx.x * 32 + lane;
    const bool valid = g < tab.nchunk;
    int n1 = 0, n2 = 0, zbase = 0, kidx = 0;
    if (valid) {
        int c = __ldg(&tab.chunk_col[g]);
        int4 ci = __ldg(&tab.col[c]);
        int h = g - ci.w / 8;
        n1 = ci.x;
        n2 = ci.y;
        zbase = tab.zoff + ci.z + 8 * h + tab.n3max;
        kidx = 8 * g;
    }
    const float delta = (float)(((double)q_target - acc->sum_q) / (double)n);
    float2 s[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) s[t] = make_float2(0.f, 0.f);
    const int a0 = blockIdx.y * span;
    const int a1 = min(n, a0 + span);
    if (valid) {
        for (int a = a0 + w; a < a1; a += SK_WARPS) {
            const float2* row = tab.phase + (size_t)a * tab.nph;
            float q = __ldg(&q_raw[a]) + delta;
            float2 xy = cmul(__ldg(&row[n1]), __ldg(&row[tab.yoff + n2 + tab.n2max]));
            xy.x *= q;
            xy.y *= q;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                float2 z = __ldg(&row[zbase + t]);
                s[t].x = fmaf(xy.x, z.x, fmaf(-xy.y, z.y, s[t].x));
                s[t].y = fmaf(xy.x, z.y, fmaf(xy.y, z.x, s[t].y));
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        red[w][t][0][lane] = (double)s[t].x;
        red[w][t][1][lane] = (double)s[t].y;
    }
    __syncthreads();
    if (w == 0 && valid) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int q = 0; q < SK_WARPS; ++q) {
                re += red[q][t][0][lane];
                im += red[q][t][1][lane];
            }
            atomicAdd(&tab.S[kidx + t].x, re);
            atomicAdd(&tab.S[kidx + t].y, im);
        }
    }
}

// C = 4 k_e G S (the half-space weight of the force / potential sums), the FP64
// reciprocal energy and the static reciprocal virial.
__global__ void k_sk_finalize(EwaldTab tab, Accum* __restrict__ acc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, wv[6] = {0, 0, 0, 0, 0, 0};
    if (k < tab.nk) {
        float gk = __ldg(&tab.kg[k]);
        if (gk > 0.f) {
            double2 s = tab.S[k];
            tab.C[k] = make_float2((float)(4.0 * KE_D * gk * s.x), (float)(4.0 * KE_D * gk * s.y));
            int c = __ldg(&tab.chunk_col[k >> 3]);
            int4 ci = __ldg(&tab.col[c]);
            int n3 = ci.z + (k - ci.w);
            const double tp = 6.283185307179586;
            double kx = tp * ci.x / (double)tab.L[0], ky = tp * ci.y / (double)tab.L[1],
                   kz = tp * n3 / (double)tab.L[2];
            double k2 = kx * kx + ky * ky + kz * kz;
            e = 2.0 * KE_D * (double)gk * (s.x * s.x + s.y * s.y);
            double fac = 2.0 / (4.0 * (double)tab.alpha * (double)tab.alpha) + 2.0 / k2;
            wv[0] = e * (1.0 - fac * kx * kx);
            wv[1] = e * (1.0 - fac * ky * ky);
            wv[2] = e * (1.0 - fac * kz * kz);
            wv[3] = -e * fac * kx * ky;
            wv[4] = -e * fac * kx * kz;
            wv[5] = -e * fac * ky * kz;
        } else {
            tab.C[k] = make_float2(0.f, 0.f);
        }
    }
    __shared__ double red[7][32];
    double v[7] = {e, wv[0], wv[1], wv[2], wv[3], wv[4], wv[5]};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x][q];
        if (threadIdx.x == 0) {
            atomicAdd(&acc->e_kspace, t);
        } else {
            const int map[6] = {0, 4, 8, 1, 2, 5};
            int m = map[threadIdx.x - 1];
            atomicAdd(&acc->virial[m], t);
            if (m == 1) atomicAdd(&acc->virial[3], t);
            if (m == 2) atomicAdd(&acc->virial[6], t);
            if (m == 5) atomicAdd(&acc->virial[7], t);
        }
    }
}

}  // namespace

void launch_ewald_phases(const float4* pos4, int n, EwaldTab tab, cudaStream_t st) {
    long long total = (long long)n * tab.nph;
    if (total == 0) return;
    k_phases<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(pos4, n, tab);
}

void launch_ewald_sk(const float* q_raw, const Accum* acc, int n, float q_target, EwaldTab tab, cudaStream_t st) {
    cudaMemsetAsync(tab.S, 0, sizeof(double2) * tab.nk, st);
    if (n == 0 || tab.nchunk == 0) return;
    int gx = (tab.nchunk + 31) / 32;
    // atom split: aim for ~4 blocks per SM over 152 SMs, at least 64 atoms per block
    int want = (4 * 152 + gx - 1) / gx;
    int span = (n + want - 1) / want;
    if (span < 64) span = 64;
    int gy = (n + span - 1) / span;
    k_sk<<<dim3(gx, gy), 32 * SK_WARPS, 0, st>>>(q_raw, acc, n, q_target, span, tab);
}

void launch_ewald_sk_finalize(EwaldTab tab, Accum* acc, cudaStream_t st) {
    if (tab.nk == 0) return;
    k_sk_finalize<<<(tab.nk + 255) / 256, 256, 0, st>>>(tab, acc);
}

}  // namespace qnep
