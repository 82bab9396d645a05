// Ewald reciprocal space (Sec. II.B, Eqs. U_k and S_k; forces and virial of Sec. II.C).
//
// Wave vectors of the half space (k and -k give conjugate terms, so the full
// sums are twice the half-space sums), |k| < kmax, k = 0 excluded.
//   S(k)  = sum_i q_i exp(-i k.r_i)                       (FP32 terms, FP64 accumulation)
//   U^k   = k_e sum_{k != 0} G(k) |S(k)|^2 = 2 k_e sum_half G |S|^2            (FP64)
//   W^k   = k_e sum G |S|^2 B,  B = I - (2/(4 alpha^2) + 2/k^2) k k^T   (Eq. virial-kspace-total)
// Per-atom phase factors are separable, exp(-i k.r) = X(n1) Y(n2) Z(n3), and
// each is evaluated directly from an exactly reduced phase (desc_math.cuh).
#include <algorithm>

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
    if (tab.tri) {   // k = 2 pi H^-1 n
        kx = tab.krec[0] * ci.x + tab.krec[1] * ci.y + tab.krec[2] * n3;
        ky = tab.krec[3] * ci.x + tab.krec[4] * ci.y + tab.krec[5] * n3;
        kz = tab.krec[6] * ci.x + tab.krec[7] * ci.y + tab.krec[8] * n3;
    }
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

// Block reduction of the 7 FP64 terms and the atomics into the accumulators.  The terms
// go through shared memory (red: 7 x blockDim.x + 7 x 32 doubles): 7 x (blockDim.x / 32)
// threads add 32 terms each, then 7 threads add those partial sums, so the FP64 unit
// (1/64 of the FP32 rate) sees about 8 adds per term instead of a shuffle tree in every lane.
__device__ __forceinline__ void flush_k_terms(double v[7], Accum* __restrict__ acc, double* red) {
    const int nt = blockDim.x, nw = nt >> 5;
    double* part = red + 7 * nt;   // [7][32]
#pragma unroll
    for (int q = 0; q < 7; ++q) red[q * nt + threadIdx.x] = v[q];
    __syncthreads();
    if ((int)threadIdx.x < 7 * nw) {
        const int q = threadIdx.x / nw, p = threadIdx.x - q * nw;
        const double* src = red + q * nt + p * 32;
        double t = 0.0;
        for (int i = 0; i < 32; ++i) t += src[i];
        part[q * 32 + p] = t;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double t = 0.0;
        for (int p = 0; p < nw; ++p) t += part[threadIdx.x * 32 + p];
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

constexpr int SK_WARPS = 8;
constexpr int SK_T = 4;       // atoms per warp tile (one bulk copy of their phase rows)
constexpr int SK_NB = 4;      // tile buffers in each warp's copy ring
constexpr int SK_SPAN = 512;  // at most this many atoms per block (FP32 partial sums)
static_assert(sizeof(float2) * SK_T * SK_NB * SK_WARPS * EWALD_MAX_NPH <= 160 * 1024,
              "the largest accepted phase rows fit the structure-factor kernel's copy rings");

// One thread = one 8-wide chunk of a column.  A block takes at most 512 atoms; they are
// cut into tiles of 4 whose phase rows are contiguous in global memory, and warp w
// takes tiles w, w + 8, ...  Each warp streams its tiles through its own ring of four
// shared-memory buffers by TMA bulk copies (three in flight while one is used) with its
// own mbarriers, and loads the tiles' charges two tiles ahead, so the warps never wait
// for one another inside the loop.  The eight warps' FP32 partial sums are added
// pairwise in FP32 and go to S with FP64 atomics.  With a counter array, the last block
// of each column group (blockIdx.x) also finalises that group's 256 wave vectors (C,
// U^k, W^k), saving a launch.
__global__ void __launch_bounds__(32 * SK_WARPS) k_sk(const float* __restrict__ q_raw, const Accum* __restrict__ acc_in,
                                                      int n, float q_target, int span, EwaldTab tab,
                                                      unsigned int* __restrict__ group_done, Accum* __restrict__ acc,
                                                      unsigned int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char sk_dyn[];
    __shared__ __align__(8) uint64_t bars[SK_WARPS][SK_NB];
    __shared__ bool last;
    __shared__ int failed;
    __shared__ float sdelta;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int slot = blockIdx.x * 32 + lane;
    const bool valid = slot < tab.nchunk;
    const int g = valid ? (tab.chunk_order ? __ldg(&tab.chunk_order[slot]) : slot) : 0;
    int n1 = 0, n2 = 0, zbase = 0;
    if (valid) {
        int c = __ldg(&tab.chunk_col[g]);
        int4 ci = __ldg(&tab.col[c]);
        int h = g - ci.w / 8;
        n1 = ci.x;
        n2 = ci.y;
        zbase = tab.zoff + ci.z + 8 * h + tab.n3max;
    }
    if (lane == 0) {
        for (int b = 0; b < SK_NB; ++b) mbar_init(&bars[w][b], 1);
        mbar_init_fence();
    }
    if (threadIdx.x == 0) {
        failed = 0;
        sdelta = (float)((double)q_target - acc_in->sum_q) * (1.f / (float)n);   // charge correction, once
    }
    __syncthreads();
    const float delta = sdelta;
    float2 s[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) s[t] = make_float2(0.f, 0.f);
    const int a0 = blockIdx.y * span;
    const int a1 = min(n, a0 + span);
    const int ntile = a1 > a0 ? (a1 - a0 + SK_T - 1) / SK_T : 0;
    const int ntw = w < ntile ? (ntile - w + SK_WARPS - 1) / SK_WARPS : 0;   // this warp's tiles
    const int yoff = tab.yoff + n2 + tab.n2max;
    const size_t buf_f2 = (size_t)SK_T * tab.nph;
    float2* const ring = reinterpret_cast<float2*>(sk_dyn) + (size_t)w * SK_NB * buf_f2;
    // the warp's i-th tile: atoms a0 + (w + 8 i) * 4 ...
    auto issue = [&](int i) {   // lane 0
        const int t0 = a0 + (w + SK_WARPS * i) * SK_T, cnt = min(SK_T, a1 - t0);
        const uint32_t bytes = round_up16((uint32_t)(cnt * tab.nph) * (uint32_t)sizeof(float2));
        fence_proxy_async_smem();
        mbar_expect_tx(&bars[w][i % SK_NB], bytes);
        bulk_g2s(ring + (size_t)(i % SK_NB) * buf_f2, tab.phase + (size_t)t0 * tab.nph, bytes, &bars[w][i % SK_NB]);
    };
    auto qload = [&](int i) {   // lanes < 4: charge of atom `lane` of the warp's i-th tile
        const int a = a0 + (w + SK_WARPS * i) * SK_T + lane;
        return (i < ntw && lane < SK_T && a < a1) ? __ldg(&q_raw[a]) : 0.f;
    };
    if (lane == 0)
        for (int i = 0; i < min(SK_NB - 1, ntw); ++i) issue(i);
    float q0 = qload(0), q1 = qload(1);   // charges of the current and the next tile
    int i = 0;
    bool ok = true;
    for (; i < ntw; ++i) {
        __syncwarp();   // the warp is done with buffer (i - 1) % 4, refilled next
        if (lane == 0 && i + SK_NB - 1 < ntw) issue(i + SK_NB - 1);
        const float q2 = qload(i + 2);
        ok = mbar_wait_bounded(&bars[w][i % SK_NB], (uint32_t)((i / SK_NB) & 1));
        if (!ok) break;
        const int cnt = min(SK_T, a1 - (a0 + (w + SK_WARPS * i) * SK_T));
        const float2* rows = ring + (size_t)(i % SK_NB) * buf_f2;
#pragma unroll
        for (int a = 0; a < SK_T; ++a) {
            const float q = __shfl_sync(0xffffffffu, q0, a) + delta;
            if (a < cnt && valid) {
                const float2* row = rows + a * tab.nph;
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
        q0 = q1;
        q1 = q2;
    }
    if (!ok) {
        // a transfer did not complete: record it and give this warp's copies still in flight
        // a bounded chance to land before the block's shared memory is released
        for (int u = i; u < min(i + SK_NB, ntw); ++u)
            mbar_wait_bounded(&bars[w][u % SK_NB], (uint32_t)((u / SK_NB) & 1));
        if (lane == 0) failed = 1;
    }
    __syncthreads();
    if (failed) {
        if (threadIdx.x == 0 && status) atomicOr(status, kStatusTimeout);
        return;
    }
    // the staging buffers are free now: the warps' partial sums, added pairwise in FP32
    float* red32 = reinterpret_cast<float*>(sk_dyn);   // [SK_WARPS][16][32]
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        red32[(w * 16 + 2 * u) * 32 + lane] = s[u].x;
        red32[(w * 16 + 2 * u + 1) * 32 + lane] = s[u].y;
    }
    __syncthreads();
    static_assert(SK_WARPS == 8, "pairwise warp sum below");
    for (int c = threadIdx.x; c < 16 * 32; c += blockDim.x) {
        const int l = c & 31, uc = c >> 5;
        const int sl = blockIdx.x * 32 + l;
        if (sl >= tab.nchunk) continue;
        float v[SK_WARPS];
#pragma unroll
        for (int q = 0; q < SK_WARPS; ++q) v[q] = red32[(q * 16 + uc) * 32 + l];
        const float sum = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        const int gl = tab.chunk_order ? __ldg(&tab.chunk_order[sl]) : sl;
        double2* dst = &tab.S[8 * gl + (uc >> 1)];
        atomicAdd((uc & 1) ? &dst->y : &dst->x, (double)sum);
    }
    double* red = reinterpret_cast<double*>(sk_dyn);   // 7 x 256 + 7 x 32 doubles for the finalisation
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
    __shared__ double red[7 * 256 + 7 * 32];
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

// Grid: column groups x atom spans (at most 512 atoms), within one wave of resident
// blocks where the atoms allow (a partial second wave would double the time of the SMs
// that run it).
static size_t sk_smem(const EwaldTab& tab) {
    // each warp's ring of tile buffers; later also the reductions (SK_WARPS x 16 x 32 floats,
    // then 7 x 256 + 7 x 32 doubles)
    size_t ring = sizeof(float2) * SK_T * tab.nph * SK_NB * SK_WARPS;
    size_t red = std::max(sizeof(float) * SK_WARPS * 16 * 32, sizeof(double) * 7 * (32 * SK_WARPS + 32));
    return std::max(ring, red);
}

static void sk_grid(int n, const EwaldTab& tab, int& gx, int& gy, int& span) {
    static std::atomic<int> attr[kMaxDevices];
    ensure_smem_attr(k_sk, attr, 160 * 1024);
    // resident blocks per SM for this shared-memory size (queried once per size and device)
    static std::atomic<long long> occ[kMaxDevices];
    const size_t smem = sk_smem(tab);
    const int per_sm = cached_occupancy(k_sk, occ, 32 * SK_WARPS, smem);
    const int sms = num_sms();
    gx = (tab.nchunk + 31) / 32;
    const int want = std::max(1, sms * std::max(per_sm, 1) / gx);
    span = (n + want - 1) / want;
    span = std::min((span + SK_T * SK_WARPS - 1) / (SK_T * SK_WARPS) * (SK_T * SK_WARPS), SK_SPAN);
    gy = (n + span - 1) / span;
}

void launch_ewald_sk(const float* q_raw, const Accum* acc, int n, float q_target, EwaldTab tab, cudaStream_t st) {
    cudaMemsetAsync(tab.S, 0, sizeof(double2) * tab.nk, st);
    if (n == 0 || tab.nchunk == 0) return;
    int gx, gy, span;
    sk_grid(n, tab, gx, gy, span);
    k_sk<<<dim3(gx, gy), 32 * SK_WARPS, sk_smem(tab), st>>>(q_raw, acc, n, q_target, span, tab, nullptr, nullptr,
                                                            &const_cast<Accum*>(acc)->status);
}

void launch_ewald_sk_fused(const float* q_raw, Accum* acc, int n, float q_target, EwaldTab tab,
                           unsigned int* group_done, cudaStream_t st) {
    if (n == 0 || tab.nchunk == 0) return;
    int gx, gy, span;
    sk_grid(n, tab, gx, gy, span);
    k_sk<<<dim3(gx, gy), 32 * SK_WARPS, sk_smem(tab), st>>>(q_raw, acc, n, q_target, span, tab, group_done, acc,
                                                            &acc->status);
}

void launch_ewald_sk_finalize(EwaldTab tab, Accum* acc, cudaStream_t st) {
    if (tab.nk == 0) return;
    k_sk_finalize<<<(tab.nk + 255) / 256, 256, 0, st>>>(tab, acc);
}

}  // namespace qnep
