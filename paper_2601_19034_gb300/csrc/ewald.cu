// Ewald reciprocal space (Sec. II.B, Eqs. U_k and S_k; forces and virial of Sec. II.C).
//
// Wave vectors of the half space (k and -k give conjugate terms, so the full
// sums are twice the half-space sums), |k| < kmax, k = 0 excluded.
//   S(k)  = sum_i q_i exp(-i k.r_i)                       (FP32 terms, FP64 accumulation)
//   U^k   = k_e sum_{k != 0} G(k) |S(k)|^2 = 2 k_e sum_half G |S|^2            (FP64)
//   W^k   = k_e sum G |S|^2 B,  B = I - (2/(4 alpha^2) + 2/k^2) k k^T   (Eq. virial-kspace-total)
// Per-atom phase factors are separable, exp(-i k.r) = X(n1) Y(n2) Z(n3), and
// each is evaluated directly from an exactly reduced phase (desc_math.cuh).
#include "desc_math.cuh"
#include "tma.cuh"

namespace qnep {

namespace {

__global__ void k_phases(const float4* __restrict__ pos4, int n, EwaldTab tab) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * tab.nph) return;
    int i = (int)(t / tab.nph);
    int e = (int)(t - (long long)i * tab.nph);
    tab.phase[t] = phase_entry(__ldg(&pos4[i]), e, tab);
}

// C = 4 k_e G S for padded index k and the FP64 energy / virial terms of k.
__device__ __forceinline__ void finalize_k(const EwaldTab& tab, int k, double v[7]) {
    float gk = __ldg(&tab.kg[k]);
    if (!(gk > 0.f)) {
        tab.C[k] = make_float2(0.f, 0.f);
        return;
    }
    double2 s = __ldcg(&tab.S[k]);
    tab.C[k] = make_float2((float)(4.0 * KE_D * gk * s.x), (float)(4.0 * KE_D * gk * s.y));
    int c = __ldg(&tab.chunk_col[k >> 3]);
    int4 ci = __ldg(&tab.col[c]);
    int n3 = ci.z + (k - ci.w);
    const float tp = 6.28318530717958648f;
    float kx = tp * ci.x / tab.L[0], ky = tp * ci.y / tab.L[1], kz = tp * n3 / tab.L[2];
    float fac = 2.f / (4.f * tab.alpha * tab.alpha) + 2.f / (kx * kx + ky * ky + kz * kz);
    double e = 2.0 * KE_D * (double)gk * (s.x * s.x + s.y * s.y);
    v[0] += e;
    v[1] += e * (double)(1.f - fac * kx * kx);
    v[2] += e * (double)(1.f - fac * ky * ky);
    v[3] += e * (double)(1.f - fac * kz * kz);
    v[4] += e * (double)(-fac * kx * ky);
    v[5] += e * (double)(-fac * kx * kz);
    v[6] += e * (double)(-fac * ky * kz);
}

// Block reduction of the 7 FP64 terms and the atomics into the accumulators.
__device__ __forceinline__ void flush_k_terms(double v[7], Accum* __restrict__ acc, double* red /* [7][32] */) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[q * 32 + w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x * 32 + q];
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

constexpr int SK_WARPS = 4;
constexpr int SK_TILE = 32;   // atoms whose phase rows are staged in shared memory at a time

// One thread = one 8-wide chunk of a column.  The block's atoms are staged tile by
// tile in shared memory: each tile's phase rows are contiguous in global memory and
// arrive by one TMA bulk copy, double buffered so the next tile streams in while the
// current one is used; each warp takes every fourth atom of a tile.  The block
// reduces its four partial sums in FP64 and adds them to S with FP64 atomics.  With
// a counter array, the last block of each column group (blockIdx.x) also finalises
// that group's 256 wave vectors (C, U^k, W^k), saving a launch.
__global__ void __launch_bounds__(32 * SK_WARPS) k_sk(const float* __restrict__ q_raw, const Accum* __restrict__ acc_in,
                                                      int n, float q_target, int span, EwaldTab tab,
                                                      unsigned int* __restrict__ group_done, Accum* __restrict__ acc,
                                                      unsigned int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char sk_dyn[];
    __shared__ float qs[2][SK_TILE];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ bool last;
    __shared__ int failed;
    float2* bufs[2] = {reinterpret_cast<float2*>(sk_dyn), reinterpret_cast<float2*>(sk_dyn) + SK_TILE * tab.nph};
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int slot = blockIdx.x * 32 + lane;
    const bool valid = slot < tab.nchunk;
    const int g = valid ? (tab.chunk_order ? __ldg(&tab.chunk_order[slot]) : slot) : 0;
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
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
        failed = 0;
    }
    __syncthreads();
    const float delta = (float)(((double)q_target - acc_in->sum_q) / (double)n);
    float2 s[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) s[t] = make_float2(0.f, 0.f);
    const int a0 = blockIdx.y * span;
    const int a1 = min(n, a0 + span);
    const int ntiles = a1 > a0 ? (a1 - a0 + SK_TILE - 1) / SK_TILE : 0;
    const int yoff = tab.yoff + n2 + tab.n2max;
    auto issue = [&](int t) {
        const int b = t & 1, t0 = a0 + t * SK_TILE, cnt = min(SK_TILE, a1 - t0);
        if (threadIdx.x == 0) {
            const uint32_t bytes = round_up16((uint32_t)(cnt * tab.nph) * (uint32_t)sizeof(float2));
            fence_proxy_async_smem();
            mbar_expect_tx(&bars[b], bytes);
            bulk_g2s(bufs[b], tab.phase + (size_t)t0 * tab.nph, bytes, &bars[b]);
        }
        if (threadIdx.x < cnt) qs[b][threadIdx.x] = __ldg(&q_raw[t0 + threadIdx.x]) + delta;
    };
    int t = 0;
    if (ntiles > 0) issue(0);
    for (; t < ntiles; ++t) {
        const int b = t & 1;
        if (t + 1 < ntiles) issue(t + 1);
        if (!mbar_wait_bounded(&bars[b], (uint32_t)((t >> 1) & 1))) failed = 1;
        __syncthreads();
        if (failed) break;
        const int cnt = min(SK_TILE, a1 - (a0 + t * SK_TILE));
        if (valid) {
            const float2* rows = bufs[b];
            for (int a = w; a < cnt; a += SK_WARPS) {
                const float2* row = rows + a * tab.nph;
                const float q = qs[b][a];
                float2 x = row[n1], y = row[yoff];
                float2 xy = make_float2(q * fmaf(x.x, y.x, -x.y * y.y), q * fmaf(x.x, y.y, x.y * y.x));
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float2 z = row[zbase + u];
                    s[u].x = fmaf(xy.x, z.x, fmaf(-xy.y, z.y, s[u].x));
                    s[u].y = fmaf(xy.x, z.y, fmaf(xy.y, z.x, s[u].y));
                }
            }
        }
        __syncthreads();
    }
    if (failed) {
        // a transfer did not complete: record it, give copies still in flight a bounded
        // chance to land before the block's shared memory is released, and leave
        for (int u = t; u < min(t + 2, ntiles); ++u) mbar_wait_bounded(&bars[u & 1], (uint32_t)((u >> 1) & 1));
        if (threadIdx.x == 0 && status) atomicOr(status, kStatusTimeout);
        return;
    }
    // the staging buffers are free now: reuse them for the cross-warp reduction
    double* red = reinterpret_cast<double*>(sk_dyn);   // [SK_WARPS][8][2][32], fits in one tile buffer
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        red[((w * 8 + u) * 2 + 0) * 32 + lane] = (double)s[u].x;
        red[((w * 8 + u) * 2 + 1) * 32 + lane] = (double)s[u].y;
    }
    __syncthreads();
    if (w == 0 && valid) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int q = 0; q < SK_WARPS; ++q) {
                re += red[((q * 8 + u) * 2 + 0) * 32 + lane];
                im += red[((q * 8 + u) * 2 + 1) * 32 + lane];
            }
            atomicAdd(&tab.S[kidx + u].x, re);
            atomicAdd(&tab.S[kidx + u].y, im);
        }
    }
    if (!group_done) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ticket = atomicAdd(&group_done[blockIdx.x], 1u);
        last = ticket == gridDim.y - 1;
        if (last) group_done[blockIdx.x] = 0u;   // ready for the next call
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // this block's 32 chunk slots are final: C, U^k and W^k of their wave vectors
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int idx = threadIdx.x; idx < 256; idx += blockDim.x) {
        const int sl = blockIdx.x * 32 + (idx >> 3);
        if (sl < tab.nchunk) {
            const int gg = tab.chunk_order ? __ldg(&tab.chunk_order[sl]) : sl;
            finalize_k(tab, 8 * gg + (idx & 7), v);
        }
    }
    __syncthreads();
    flush_k_terms(v, acc, red);
}

__global__ void k_sk_finalize(EwaldTab tab, Accum* __restrict__ acc) {
    __shared__ double red[7 * 32];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (k < tab.nk) finalize_k(tab, k, v);
    flush_k_terms(v, acc, red);
}

}  // namespace

void launch_ewald_phases(const float4* pos4, int n, EwaldTab tab, cudaStream_t st) {
    long long total = (long long)n * tab.nph;
    if (total == 0) return;
    k_phases<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(pos4, n, tab);
}

static void sk_grid(int n, const EwaldTab& tab, int& gx, int& gy, int& span) {
    gx = (tab.nchunk + 31) / 32;
    // atom split: aim for ~4 blocks per SM over 152 SMs; spans are whole tiles
    int want = (4 * 152 + gx - 1) / gx;
    span = (n + want - 1) / want;
    span = (span + SK_TILE - 1) / SK_TILE * SK_TILE;
    gy = (n + span - 1) / span;
}

static size_t sk_smem(const EwaldTab& tab) {
    // two tile buffers; the first also holds the reduction (SK_WARPS x 8 x 2 x 32 doubles)
    size_t tile = sizeof(float2) * SK_TILE * tab.nph;
    size_t red = sizeof(double) * SK_WARPS * 8 * 2 * 32;
    return tile > red ? 2 * tile : tile + red;
}

static void sk_attr() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_sk, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        done = true;
    }
}

void launch_ewald_sk(const float* q_raw, const Accum* acc, int n, float q_target, EwaldTab tab, cudaStream_t st) {
    cudaMemsetAsync(tab.S, 0, sizeof(double2) * tab.nk, st);
    if (n == 0 || tab.nchunk == 0) return;
    int gx, gy, span;
    sk_grid(n, tab, gx, gy, span);
    sk_attr();
    k_sk<<<dim3(gx, gy), 32 * SK_WARPS, sk_smem(tab), st>>>(q_raw, acc, n, q_target, span, tab, nullptr, nullptr,
                                                            &const_cast<Accum*>(acc)->status);
}

void launch_ewald_sk_fused(const float* q_raw, Accum* acc, int n, float q_target, EwaldTab tab,
                           unsigned int* group_done, cudaStream_t st) {
    if (n == 0 || tab.nchunk == 0) return;
    int gx, gy, span;
    sk_grid(n, tab, gx, gy, span);
    sk_attr();
    k_sk<<<dim3(gx, gy), 32 * SK_WARPS, sk_smem(tab), st>>>(q_raw, acc, n, q_target, span, tab, group_done, acc,
                                                            &acc->status);
}

void launch_ewald_sk_finalize(EwaldTab tab, Accum* acc, cudaStream_t st) {
    if (tab.nk == 0) return;
    k_sk_finalize<<<(tab.nk + 255) / 256, 256, 0, st>>>(tab, acc);
}

}  // namespace qnep
