// PPPM reciprocal space (Sec. II.F).
//
//   charge mesh  rho_s = sum_i q_i W(r_i - r_s), W = order-5 cardinal B-spline per axis
//                (the five mesh points around the nearest one, weights as polynomials of
//                the offset d in [-1/2, 1/2])
//   S(k)         = FFT(rho) (cuFFT R2C, e^{-ik.r} sign), half spectrum n_z in [0, N_z/2]
//   influence    G_opt = G(k) [prod sinc^5(pi n/N)]^2 / [prod A(z)]^2,
//                A(z) = 1 - 5/3 z^2 + 7/9 z^4 - 17/189 z^6 + 2/2835 z^8, z = sin(pi n / N)
//                (the alias sum of sinc^10; the squared denominator of the optimal
//                influence function of Hockney and Eastwood)
//   energy       U^k = k_e sum_{k != 0} G_opt |S|^2 (full spectrum: half spectrum x 2 except
//                the planes n_z = 0 and n_z = N_z/2); virial with B as in Eq. virial-kspace-total
//   fields       F^-1[S G_opt] and F^-1[i k_d S G_opt] (component d zero on its Nyquist plane),
//                unnormalised inverse transforms (cuFFT C2R, batch of 4)
//   gather       phi^k_i = 2 k_e sum_s W phi_s,  F^k_i / q_i = -2 k_e sum_s W E_s  (ik differentiation,
//                Eq. force-static-fft; the potential is the factor of Eq. force-dynamic-fft)
// General cells (rows of H the lattice vectors): the mesh lies along the lattice vectors, an
// atom's mesh coordinates are N_d times its fractional coordinates r H^-1, k = 2 pi H^-1 n with
// V = det H in G(k) (the alias sums depend on n_d / N_d only), and the three fields are the
// fractional gradients F^-1[i 2 pi n_c S G_opt] (each zero on the Nyquist plane of n_c), mapped
// at the gather to d/dr_a = sum_c H^-1[a][c] d/ds_c; a diagonal H gives the ik form above.
#include <cufft.h>

#include <algorithm>

#include "desc_math.cuh"

namespace qnep {

namespace {

constexpr float TWO_PI_F = 6.28318530717958648f;

// weights of the mesh points s0-2 .. s0+2 for offset d = u - s0 in [-1/2, 1/2]
__device__ __forceinline__ void assign5(float d, float w[5]) {
    const float d2 = d * d, d3 = d2 * d, d4 = d2 * d2;
    const float e = (1.f / 16.f) * d2 + (1.f / 384.f) + (1.f / 24.f) * d4;
    const float o = (1.f / 48.f) * d + (1.f / 12.f) * d3;
    w[0] = e - o;
    w[4] = e + o;
    const float e1 = 19.f / 96.f + 0.25f * d2 - (1.f / 6.f) * d4;
    const float o1 = (11.f / 24.f) * d - (1.f / 6.f) * d3;
    w[1] = e1 - o1;
    w[3] = e1 + o1;
    w[2] = 115.f / 192.f - 0.625f * d2 + 0.25f * d4;
}

// mesh coordinate u = x N / L (x in [0, L), u in [0, N)) as u_hi + u_lo with an error-free
// product, so the offset from the nearest mesh point keeps ~1e-12 instead of FP32 rounding of u
__device__ __forceinline__ void stencil_axis(float x, float inv_h, float inv_h_lo, int& s0, float w[5]) {
    const float p = x * inv_h;
    const float pe = fmaf(x, inv_h, -p);          // exact: x inv_h = p + pe
    const float r = rintf(p);
    const float d = (p - r) + fmaf(x, inv_h_lo, pe);
    assign5(d, w);
    s0 = (int)r - 2;                    // first of the five points (may be < 0 or >= N: wrapped by the caller)
}

// the same for a general cell along fractional axis d: u = N_d sum_c r_c H^-1[c][d], each product
// error-free (hi / lo pairs of N_d H^-1) and the three added with compensated sums, so the offset
// from the nearest mesh point keeps the precision of the orthorhombic form
__device__ __forceinline__ void stencil_frac(const float4& p, const PppmTab& pm, int d, int& s0, float w[5]) {
    const float r[3] = {p.x, p.y, p.z};
    float s = 0.f, lo = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float h = pm.nh_hi[3 * c + d], hl = pm.nh_lo[3 * c + d];
        const float pp = r[c] * h;
        const float pe = fmaf(r[c], h, -pp);   // exact: r_c h = pp + pe
        lo += fmaf(r[c], hl, pe);
        const float t = s + pp;                // two-sum: s + pp = t + err exactly
        const float bp = t - s;
        lo += (s - (t - bp)) + (pp - bp);
        s = t;
    }
    const float rr = rintf(s);
    assign5((s - rr) + lo, w);
    s0 = (int)rr - 2;
}

// the five-point stencils of an atom along the three mesh axes
__device__ __forceinline__ void stencil3(const float4& p, const PppmTab& pm, int& sx, int& sy, int& sz, float wx[5],
                                         float wy[5], float wz[5]) {
    if (pm.tri) {
        stencil_frac(p, pm, 0, sx, wx);
        stencil_frac(p, pm, 1, sy, wy);
        stencil_frac(p, pm, 2, sz, wz);
        return;
    }
    stencil_axis(p.x, pm.inv_h[0], pm.inv_h_lo[0], sx, wx);
    stencil_axis(p.y, pm.inv_h[1], pm.inv_h_lo[1], sy, wy);
    stencil_axis(p.z, pm.inv_h[2], pm.inv_h_lo[2], sz, wz);
}

// stencil indices lie in [-2, N + 2) (s0 in [-2, N - 2], offsets 0..4): one periodic shift
__device__ __forceinline__ int wrap(int s, int n) { return s < 0 ? s + n : (s >= n ? s - n : s); }

// one warp per atom at a time (persistent warps), lanes over the 125 stencil points
__global__ void k_pppm_spread(const float4* __restrict__ spos4, const float* __restrict__ q_raw, int n,
                              const Accum* __restrict__ acc_in, float q_target, PppmTab pm) {
    const int lane = threadIdx.x & 31;
    const float delta = block_charge_scalars(acc_in, q_target, n, 0, 0.f).delta;   // synchronises
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += nwarps) {
    const float4 p = __ldg(&spos4[k]);
    const float q = __ldg(&q_raw[k]) + delta;
    int sx, sy, sz;
    float wx[5], wy[5], wz[5];
    stencil3(p, pm, sx, sy, sz, wx, wy, wz);
    for (int t = lane; t < 125; t += 32) {
        const int a = t / 25, b = (t / 5) % 5, c = t % 5;
        float wa = wx[0], wb = wy[0], wc = wz[0];
#pragma unroll
        for (int m = 1; m < 5; ++m) {
            if (a == m) wa = wx[m];
            if (b == m) wb = wy[m];
            if (c == m) wc = wz[m];
        }
        const size_t idx = ((size_t)wrap(sx + a, pm.nx) * pm.ny + wrap(sy + b, pm.ny)) * pm.nz + wrap(sz + c, pm.nz);
        atomicAdd(&pm.rho[idx], q * wa * wb * wc);
    }
    }
}

// half-spectrum point -> signed mesh integers
__device__ __forceinline__ void mesh_n(size_t idx, const PppmTab& pm, int& n1, int& n2, int& n3) {
    const int nzc = pm.nz / 2 + 1;
    n3 = (int)(idx % nzc);
    const size_t r = idx / nzc;
    n2 = (int)(r % pm.ny);
    n1 = (int)(r / pm.ny);
    if (n1 >= (pm.nx + 1) / 2) n1 -= pm.nx;
    if (n2 >= (pm.ny + 1) / 2) n2 -= pm.ny;
}

__device__ __forceinline__ double alias5(double z2) {
    return 1.0 - 5.0 / 3.0 * z2 + 7.0 / 9.0 * z2 * z2 - 17.0 / 189.0 * z2 * z2 * z2 + 2.0 / 2835.0 * z2 * z2 * z2 * z2;
}

__device__ __forceinline__ double sinc_pi(int nn, int nmesh) {
    if (nn == 0) return 1.0;
    const double x = 3.141592653589793 * nn / nmesh;
    return sin(x) / x;
}

// optimal influence function on the half spectrum (once per box)
__global__ void k_pppm_gopt(PppmTab pm, double alpha, double vol) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= pm.nhalf) return;
    int n1, n2, n3;
    mesh_n(idx, pm, n1, n2, n3);
    const double tp = 6.283185307179586;
    double kx = tp * n1 / pm.len[0], ky = tp * n2 / pm.len[1], kz = tp * n3 / pm.len[2];
    if (pm.tri) {   // k = 2 pi H^-1 n
        kx = tp * (pm.hid[0] * n1 + pm.hid[1] * n2 + pm.hid[2] * n3);
        ky = tp * (pm.hid[3] * n1 + pm.hid[4] * n2 + pm.hid[5] * n3);
        kz = tp * (pm.hid[6] * n1 + pm.hid[7] * n2 + pm.hid[8] * n3);
    }
    const double k2 = kx * kx + ky * ky + kz * kz;
    if (k2 == 0.0) {
        pm.gopt[idx] = 0.f;
        return;
    }
    const double g = tp / vol * exp(-k2 / (4.0 * alpha * alpha)) / k2;
    double u = sinc_pi(n1, pm.nx) * sinc_pi(n2, pm.ny) * sinc_pi(n3, pm.nz);
    u = u * u;                            // sinc^2
    u = u * u * u * u * u;                // [prod sinc^5]^2 = (prod sinc^2)^5
    const double pi = 3.141592653589793;
    double zx = sin(pi * n1 / pm.nx), zy = sin(pi * n2 / pm.ny), zz = sin(pi * n3 / pm.nz);
    const double den = alias5(zx * zx) * alias5(zy * zy) * alias5(zz * zz);
    pm.gopt[idx] = (float)(g * u / (den * den));
}

// S G_opt and the three i k S G_opt fields; U^k and W^k.  Persistent threads over the half
// spectrum (indices fit 32 bits: the mesh is limited to 2^31 points); each thread sums its
// terms in FP32 over 8 points at a time and in FP64 across them, then FP64 across warps.
__global__ void __launch_bounds__(256) k_pppm_green(PppmTab pm, float alpha, Accum* __restrict__ acc) {
    double vd[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int np = 0;
    const unsigned nhalf = (unsigned)pm.nhalf, nzc = (unsigned)(pm.nz / 2 + 1), ny = (unsigned)pm.ny;
    const float fac0 = 2.f / (4.f * alpha * alpha);
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nhalf; idx += gridDim.x * blockDim.x) {
        const unsigned row = idx / nzc, m2 = row / ny;
        int n3 = (int)(idx - row * nzc), n2 = (int)(row - m2 * ny), n1 = (int)m2;
        if (n1 >= (pm.nx + 1) / 2) n1 -= pm.nx;
        if (n2 >= (pm.ny + 1) / 2) n2 -= pm.ny;
        const float g = pm.gopt[idx];
        const float2 s = pm.shat[idx];
        float kx = TWO_PI_F * n1 / pm.len[0], ky = TWO_PI_F * n2 / pm.len[1], kz = TWO_PI_F * n3 / pm.len[2];
        // the three gradient fields: i k_d (orthorhombic) or the fractional i 2 pi n_c (general)
        float gx = kx, gy = ky, gz = kz;
        if (pm.tri) {
            gx = TWO_PI_F * n1;
            gy = TWO_PI_F * n2;
            gz = TWO_PI_F * n3;
            kx = fmaf(pm.hi[2], gz, fmaf(pm.hi[1], gy, pm.hi[0] * gx));
            ky = fmaf(pm.hi[5], gz, fmaf(pm.hi[4], gy, pm.hi[3] * gx));
            kz = fmaf(pm.hi[8], gz, fmaf(pm.hi[7], gy, pm.hi[6] * gx));
        }
        const float2 sg = make_float2(s.x * g, s.y * g);
        pm.fhat[idx] = sg;
        // i g_d S G, zero on the Nyquist plane of component d
        const bool nyx = (pm.nx % 2 == 0) && n1 == -pm.nx / 2;
        const bool nyy = (pm.ny % 2 == 0) && n2 == -pm.ny / 2;
        const bool nyz = (pm.nz % 2 == 0) && n3 == pm.nz / 2;
        pm.fhat[pm.nhalf + idx] = nyx ? make_float2(0.f, 0.f) : make_float2(-gx * sg.y, gx * sg.x);
        pm.fhat[2 * pm.nhalf + idx] = nyy ? make_float2(0.f, 0.f) : make_float2(-gy * sg.y, gy * sg.x);
        pm.fhat[3 * pm.nhalf + idx] = nyz ? make_float2(0.f, 0.f) : make_float2(-gz * sg.y, gz * sg.x);
        if (pm.fhat6) {
            // per-atom virial fields G_opt B_ab S, B = I - (2 / (4 alpha^2) + 2 / k^2) k k^T (zero at k = 0)
            const float k2 = kx * kx + ky * ky + kz * kz;
            const float fac = k2 > 0.f ? fac0 + 2.f / k2 : 0.f;
            const float bv[6] = {1.f - fac * kx * kx, 1.f - fac * ky * ky, 1.f - fac * kz * kz, -fac * kx * ky,
                                 -fac * kx * kz, -fac * ky * kz};
#pragma unroll
            for (int q = 0; q < 6; ++q) pm.fhat6[q * pm.nhalf + idx] = make_float2(bv[q] * sg.x, bv[q] * sg.y);
        }
        if (g > 0.f) {
            const float mult = (n3 == 0 || (pm.nz % 2 == 0 && n3 == pm.nz / 2)) ? 1.f : 2.f;
            const float e = mult * KE * g * (s.x * s.x + s.y * s.y);
            const float k2 = kx * kx + ky * ky + kz * kz;
            const float fac = fac0 + 2.f / k2;
            v[0] += e;
            v[1] += e * (1.f - fac * kx * kx);
            v[2] += e * (1.f - fac * ky * ky);
            v[3] += e * (1.f - fac * kz * kz);
            v[4] -= e * fac * kx * ky;
            v[5] -= e * fac * kx * kz;
            v[6] -= e * fac * ky * kz;
        }
        if (++np == 8) {
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                vd[q] += (double)v[q];
                v[q] = 0.f;
            }
            np = 0;
        }
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) vd[q] += (double)v[q];
    __shared__ double red[7][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        double x = vd[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x][q];
        if (threadIdx.x == 0) {
            atomicAdd(&acc->e_kspace, t);
        } else {
            const int map[6] = {0, 4, 8, 1, 2, 5};
            const int m = map[threadIdx.x - 1];
            atomicAdd(&acc->virial[m], t);
            if (m == 1) atomicAdd(&acc->virial[3], t);
            if (m == 2) atomicAdd(&acc->virial[6], t);
            if (m == 5) atomicAdd(&acc->virial[7], t);
        }
    }
}

// one warp per atom at a time (persistent warps), lanes over the 125 stencil points of the
// 4 fields; lane 0 sums phi in FP32 over 8 atoms at a time, then in FP64
__global__ void k_pppm_gather(const float4* __restrict__ spos4, int n, PppmTab pm, float4* __restrict__ kfield,
                              Accum* __restrict__ acc) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    double sphi = 0.0;
    float pphi = 0.f;
    int np = 0;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += nwarps) {
        float ph = 0.f;
        const float4 p = __ldg(&spos4[k]);
        int sx, sy, sz;
        float wx[5], wy[5], wz[5];
        stencil3(p, pm, sx, sy, sz, wx, wy, wz);
        float ex = 0.f, ey = 0.f, ez = 0.f;
        for (int t = lane; t < 125; t += 32) {
            const int a = t / 25, b = (t / 5) % 5, c = t % 5;
            float wa = wx[0], wb = wy[0], wc = wz[0];
#pragma unroll
            for (int m = 1; m < 5; ++m) {
                if (a == m) wa = wx[m];
                if (b == m) wb = wy[m];
                if (c == m) wc = wz[m];
            }
            const float w = wa * wb * wc;
            const size_t idx =
                ((size_t)wrap(sx + a, pm.nx) * pm.ny + wrap(sy + b, pm.ny)) * pm.nz + wrap(sz + c, pm.nz);
            ph = fmaf(w, __ldg(&pm.field[idx]), ph);
            ex = fmaf(w, __ldg(&pm.field[pm.nreal + idx]), ex);
            ey = fmaf(w, __ldg(&pm.field[2 * pm.nreal + idx]), ey);
            ez = fmaf(w, __ldg(&pm.field[3 * pm.nreal + idx]), ez);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ph += __shfl_xor_sync(0xffffffffu, ph, o);
            ex += __shfl_xor_sync(0xffffffffu, ex, o);
            ey += __shfl_xor_sync(0xffffffffu, ey, o);
            ez += __shfl_xor_sync(0xffffffffu, ez, o);
        }
        ph *= 2.f * KE;
        if (pm.tri) {   // fractional gradients -> Cartesian: d/dr_a = sum_c H^-1[a][c] d/ds_c
            const float gx = ex, gy = ey, gz = ez;
            ex = fmaf(pm.hi[2], gz, fmaf(pm.hi[1], gy, pm.hi[0] * gx));
            ey = fmaf(pm.hi[5], gz, fmaf(pm.hi[4], gy, pm.hi[3] * gx));
            ez = fmaf(pm.hi[8], gz, fmaf(pm.hi[7], gy, pm.hi[6] * gx));
        }
        if (lane == 0) {
            kfield[k] = make_float4(-2.f * KE * ex, -2.f * KE * ey, -2.f * KE * ez, ph);
            pphi += ph;
            if (++np == 8) {
                sphi += (double)pphi;
                pphi = 0.f;
                np = 0;
            }
        }
    }
    __shared__ double red[8];
    const int w = threadIdx.x >> 5;
    if (lane == 0) red[w] = sphi + (double)pphi;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(&acc->sum_phi, t);
    }
}

// Per-atom reciprocal-space virial on the mesh: 2 k_e sum_s W(r_i - r_s) F^-1[G_opt B_ab S](r_s)
// for the six components (lanes over the 125 stencil points; one warp per atom at a time).
__global__ void k_pppm_gather_virial(const float4* __restrict__ spos4, int n, PppmTab pm, float* __restrict__ avir) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += nwarps) {
        const float4 p = __ldg(&spos4[k]);
        int sx, sy, sz;
        float wx[5], wy[5], wz[5];
        stencil3(p, pm, sx, sy, sz, wx, wy, wz);
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int t = lane; t < 125; t += 32) {
            const int a = t / 25, b = (t / 5) % 5, c = t % 5;
            float wa = wx[0], wb = wy[0], wc = wz[0];
#pragma unroll
            for (int m = 1; m < 5; ++m) {
                if (a == m) wa = wx[m];
                if (b == m) wb = wy[m];
                if (c == m) wc = wz[m];
            }
            const float w = wa * wb * wc;
            const size_t idx =
                ((size_t)wrap(sx + a, pm.nx) * pm.ny + wrap(sy + b, pm.ny)) * pm.nz + wrap(sz + c, pm.nz);
#pragma unroll
            for (int q = 0; q < 6; ++q) v[q] = fmaf(w, __ldg(&pm.field6[q * pm.nreal + idx]), v[q]);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) avir[(size_t)AVIR * k + 9 + q] = 2.f * KE * v[q];
        }
    }
}

}  // namespace

void launch_pppm_gopt(const PppmTab& pm, double alpha, double vol, cudaStream_t st) {
    k_pppm_gopt<<<(unsigned)((pm.nhalf + 255) / 256), 256, 0, st>>>(pm, alpha, vol);
}

int launch_pppm(const float4* spos4, const float* q_raw, int n, const Accum* acc_in, float q_target, PppmTab pm,
                float alpha, int r2c, int c2r, float4* kfield, Accum* acc, cudaStream_t st, int c2r6, float* avir) {
    if (n == 0) return 0;
    const int threads = 256;
    // persistent warps over the atoms and persistent threads over the half spectrum: one
    // wave of resident blocks (occupancy queried once per kernel)
    static std::atomic<long long> c_spread[kMaxDevices], c_green[kMaxDevices], c_gather[kMaxDevices];
    const int occ_spread = cached_occupancy(k_pppm_spread, c_spread, threads, 0);
    const int occ_green = cached_occupancy(k_pppm_green, c_green, threads, 0);
    const int occ_gather = cached_occupancy(k_pppm_gather, c_gather, threads, 0);
    const long long atom_blocks = ((long long)n * 32 + threads - 1) / threads;
    const unsigned sblocks = (unsigned)std::min<long long>(atom_blocks, (long long)occ_spread * num_sms());
    const unsigned hblocks = (unsigned)std::min<long long>(atom_blocks, (long long)occ_gather * num_sms());
    const unsigned gblocks =
        (unsigned)std::min<long long>((long long)((pm.nhalf + threads - 1) / threads), (long long)occ_green * num_sms());
    k_pppm_spread<<<sblocks, threads, 0, st>>>(spos4, q_raw, n, acc_in, q_target, pm);
    if (cufftSetStream(r2c, st) != CUFFT_SUCCESS) return 1;
    if (cufftExecR2C(r2c, pm.rho, reinterpret_cast<cufftComplex*>(pm.shat)) != CUFFT_SUCCESS) return 1;
    k_pppm_green<<<gblocks, threads, 0, st>>>(pm, alpha, acc);
    if (cufftSetStream(c2r, st) != CUFFT_SUCCESS) return 1;
    if (cufftExecC2R(c2r, reinterpret_cast<cufftComplex*>(pm.fhat), pm.field) != CUFFT_SUCCESS) return 1;
    k_pppm_gather<<<hblocks, threads, 0, st>>>(spos4, n, pm, kfield, acc);
    if (avir && pm.fhat6) {   // the six per-atom virial fields (one batched inverse transform)
        if (cufftSetStream(c2r6, st) != CUFFT_SUCCESS) return 1;
        if (cufftExecC2R(c2r6, reinterpret_cast<cufftComplex*>(pm.fhat6), pm.field6) != CUFFT_SUCCESS) return 1;
        k_pppm_gather_virial<<<hblocks, threads, 0, st>>>(spos4, n, pm, avir);
    }
    return 0;
}

}  // namespace qnep
