// Per-atom network on the 5th-generation tensor cores (precision form: BF16 or TF32
// operands, FP32 accumulation in tensor memory).
//
// The network of Eq. U_i / Sec. II.B for a tile of 128 atoms is three small GEMMs:
//   MMA1  P   = D W0^T          [128 x 32] x [32 x 32 S]   (all species' W0 stacked on N)
//   epilogue  h = tanh(P_{t_i} - b0), U = w1E.h - b1E, q = w1q.h - b1q,
//             gE = w1E (1 - h^2), gq = w1q (1 - h^2)      (FP32, one thread per atom)
//   MMA2  dU/dD = GE W0         [128 x 32 S] x [32 S x 32]   GE block-diagonal by species
//   MMA3  dq/dD = GQ W0         (same B operand)
// N_des = 30 and N_neu = 30 are padded to 32 with zeros.  Operands live in shared
// memory in the canonical K-major layout without swizzle (core matrices of 8 rows x
// 16 bytes; K-adjacent cores 128 B apart, 8-row groups K/kpc x 128 B apart); one
// thread issues the tcgen05.mma instructions, accumulators are in tensor memory and
// are read back with tcgen05.ld (warp w owns lanes 32w..32w+31).  Blocks are persistent over
// the tiles; each tile's descriptors arrive by one bulk copy into one of two shared-memory
// buffers, the next tile's copy running while this tile is computed.  Every wait on an
// mbarrier is bounded; a timeout sets a status bit and the block stops after
// releasing its tensor memory.
#include <stdint.h>

#include <cuda_bf16.h>

#include "qnep_internal.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace qnep {

namespace {

constexpr int TM = 128;      // atoms per tile = MMA M = tensor-memory lanes
constexpr int KP = 32;       // descriptor length padded
constexpr int HP = 32;       // hidden width padded
constexpr int TMEM_COLS = 256;
constexpr int COL_P = 0;     // P: 32 S columns
constexpr int COL_DU = 128;  // dU/dD: 32 columns
constexpr int COL_DQ = 160;  // dq/dD: 32 columns

// element size and per-instruction K of the two operand types
template <int PREC> struct Op;
template <> struct Op<PREC_BF16> { static constexpr int ES = 2, KSTEP = 16, FMT = 1; };
template <> struct Op<PREC_TF32> { static constexpr int ES = 4, KSTEP = 8, FMT = 2; };

template <int PREC>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    if (PREC == PREC_BF16) mma_f16(tmem_d, a, b, idesc, accumulate);
    else mma_tf32(tmem_d, a, b, idesc, accumulate);
}

// 16 bytes of operand elements (8 BF16 or 4 TF32) from FP32 values, first element lowest
template <int PREC>
__device__ __forceinline__ uint4 pack16(const float* v) {
    uint32_t w[4];
    if (PREC == PREC_BF16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            w[q] = *reinterpret_cast<const uint32_t*>(&h);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w[q]) : "f"(v[q]));
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Elements k0 .. k0 + NK - 1 of one row of an operand with K columns (k0, NK multiples of
// the 16-byte core row), one 16-byte store per core matrix.
template <int PREC, int NK>
__device__ __forceinline__ void put_row(unsigned char* base, int row, int K, int k0, const float* v) {
    constexpr int ES = Op<PREC>::ES, KPC = 16 / ES;
    const int ncore = K * ES / 16;
#pragma unroll
    for (int c = 0; c < NK / KPC; ++c) {
        const int kc = k0 / KPC + c;
        *reinterpret_cast<uint4*>(base + ((row >> 3) * ncore + kc) * 128 + (row & 7) * 16) = pack16<PREC>(v + c * KPC);
    }
}

struct MlpSmem {   // byte offsets of the operands and small parameters in dynamic shared memory
    uint32_t a1, a2, a3, b1, b2, par, dtc, total;
};

template <int PREC>
__host__ __device__ constexpr MlpSmem mlp_layout(int S) {
    constexpr int ES = Op<PREC>::ES;
    MlpSmem L{};
    L.a1 = 0;
    L.a2 = L.a1 + TM * KP * ES;
    L.a3 = L.a2 + TM * HP * S * ES;
    L.b1 = L.a3 + TM * HP * S * ES;
    L.b2 = L.b1 + HP * S * KP * ES;
    L.par = L.b2 + KP * HP * S * ES;
    // b0, w1E, w1q [S][HP], b1E, b1Q [S], scaler [KP] (FP32)
    L.dtc = (L.par + (uint32_t)sizeof(float) * (3 * S * HP + 2 * S + KP) + 127u) & ~127u;
    // two FP32 descriptor tiles [TM][KP], filled by bulk copies
    L.total = L.dtc + 2u * (uint32_t)sizeof(float) * TM * KP;
    return L;
}

// tanh(x) = 1 - 2 / (1 + e^{2x}) with the fast exponential and division: absolute error
// about 1e-6, far below the BF16 / TF32 rounding of h in the next product (2^-9 / 2^-12);
// +-1 for large |x| (e^{2x} overflows to inf or underflows to 0)
__device__ __forceinline__ float tanh_fast(float x) { return 1.f - __fdividef(2.f, 1.f + __expf(2.f * x)); }

template <int PREC>
__global__ void __launch_bounds__(TM, 1) k_mlp_tc(const float* __restrict__ dtc, const float4* __restrict__ spos4,
                                               int n, const float* __restrict__ params, ParamLayout lay,
                                               float* __restrict__ du, float* __restrict__ dq, int d_sa, int d_sv,
                                               float* __restrict__ u_out, float* __restrict__ q_out,
                                               Accum* __restrict__ acc) {
    using O = Op<PREC>;
    constexpr int ES = O::ES;
    extern __shared__ __align__(128) unsigned char msm[];
    __shared__ uint64_t bar;
    __shared__ __align__(8) uint64_t dbar[2];   // the two descriptor tiles
    __shared__ uint32_t tmem_base;
    __shared__ double red[2][TM / 32];
    __shared__ int failed;
    const int S = lay.n_species;
    const MlpSmem L = mlp_layout<PREC>(S);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char* A1 = msm + L.a1;
    unsigned char* A2 = msm + L.a2;
    unsigned char* A3 = msm + L.a3;
    unsigned char* B1 = msm + L.b1;
    unsigned char* B2 = msm + L.b2;
    float* par = reinterpret_cast<float*>(msm + L.par);
    float* pb0 = par;                   // [S][HP]
    float* pwe = par + S * HP;
    float* pwq = par + 2 * S * HP;
    float* pb1 = par + 3 * S * HP;      // [S][2]
    float* psc = pb1 + 2 * S;           // [KP]
    float* dbuf = reinterpret_cast<float*>(msm + L.dtc);   // [2][TM][KP]

    // weights of every species: B1 [32 S rows (s, mu)][32 K (v)] and B2 [32 rows (v)][32 S K (s, mu)]
    for (int row = tid; row < S * HP; row += TM) {   // B1 row (s, mu): W0_s[mu][0..31]
        const int s = row / HP, mu = row - s * HP;
        float w[KP];
#pragma unroll
        for (int v = 0; v < KP; ++v)
            w[v] = (mu < NNEU && v < NDES) ? params[lay.mlp + s * lay.mlp_stride + ParamLayout::W0 + mu * NDES + v] : 0.f;
        put_row<PREC, KP>(B1, row, KP, 0, w);
    }
    for (int idx = tid; idx < KP * S; idx += TM) {    // B2 row v, block s: W0_s[0..31][v]
        const int v = idx / S, s = idx - v * S;
        float w[HP];
#pragma unroll
        for (int mu = 0; mu < HP; ++mu)
            w[mu] = (mu < NNEU && v < NDES) ? params[lay.mlp + s * lay.mlp_stride + ParamLayout::W0 + mu * NDES + v] : 0.f;
        put_row<PREC, HP>(B2, v, HP * S, s * HP, w);
    }
    for (int idx = tid; idx < S * HP; idx += TM) {
        const int s = idx / HP, mu = idx - s * HP;
        const float* net = params + lay.mlp + s * lay.mlp_stride;
        pb0[idx] = mu < NNEU ? net[ParamLayout::B0 + mu] : 0.f;
        pwe[idx] = mu < NNEU ? net[ParamLayout::W1E + mu] : 0.f;
        pwq[idx] = mu < NNEU ? net[ParamLayout::W1Q + mu] : 0.f;
    }
    for (int s = tid; s < S; s += TM) {
        pb1[2 * s] = params[lay.mlp + s * lay.mlp_stride + ParamLayout::B1E];
        pb1[2 * s + 1] = params[lay.mlp + s * lay.mlp_stride + ParamLayout::B1Q];
    }
    for (int v = tid; v < KP; v += TM) psc[v] = v < NDES ? params[lay.scaler + v] : 0.f;
    if (warp == 0) {
        tmem_alloc(&tmem_base, TMEM_COLS);
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init(&dbar[0], 1);
        mbar_init(&dbar[1], 1);
        mbar_init_fence();
        failed = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    // canonical layout strides: K-adjacent core matrices 128 B apart, 8-row groups (K ES / 16) x 128 B
    const uint32_t sA1 = (uint32_t)(KP * ES / 16) * 128, sA2 = (uint32_t)(HP * S * ES / 16) * 128;
    const uint32_t kstep_bytes = (uint32_t)(O::KSTEP * ES / 16) * 128;
    const uint32_t id1 = instr_desc(O::FMT, TM, HP * S), id2 = instr_desc(O::FMT, TM, KP);
    uint32_t phase = 0;
    double su = 0.0, sq = 0.0;

    const int ntiles = (n + TM - 1) / TM;
    // descriptor tile of the block's i-th tile into buffer i & 1 (thread 0): one bulk copy of
    // the tile's rows (contiguous, 128 B each)
    auto issue = [&](int i) {
        const int t = blockIdx.x + i * gridDim.x, cnt = min(TM, n - t * TM);
        const uint32_t bytes = (uint32_t)(cnt * KP * sizeof(float));
        fence_proxy_async_smem();
        mbar_expect_tx(&dbar[i & 1], bytes);
        bulk_g2s(dbuf + (i & 1) * TM * KP, dtc + (size_t)t * TM * KP, bytes, &dbar[i & 1]);
    };
    if (tid == 0 && (int)blockIdx.x < ntiles) issue(0);
    int ti_next = 0;
    if ((int)blockIdx.x * TM + tid < n) ti_next = __float_as_int(__ldg(&spos4[blockIdx.x * TM + tid]).w);
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int k = tile * TM + tid;
        const bool valid = k < n;
        const int ti = valid ? ti_next : 0;
        // the next tile streams in while this one is computed (its buffer was last read
        // before the first barrier of the previous tile); its species are loaded now
        const int knext = (tile + gridDim.x) * TM + tid;
        if (tile + (int)gridDim.x < ntiles) {
            if (tid == 0) issue(i + 1);
            if (knext < n) ti_next = __float_as_int(__ldg(&spos4[knext]).w);
        }
        if (!mbar_wait_bounded(&dbar[i & 1], (uint32_t)((i >> 1) & 1))) failed = 1;
        // operand A1: this atom's scaled descriptor; A2 / A3 cleared (block-diagonal fill below)
        {
            float dv[KP];
            if (valid) {
                const float4* src = reinterpret_cast<const float4*>(dbuf + (i & 1) * TM * KP + tid * KP);
#pragma unroll
                for (int q = 0; q < KP / 4; ++q) {
                    const float4 x = src[q];
                    dv[4 * q] = x.x;
                    dv[4 * q + 1] = x.y;
                    dv[4 * q + 2] = x.z;
                    dv[4 * q + 3] = x.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < KP; ++q) dv[q] = 0.f;
            }
            put_row<PREC, KP>(A1, tid, KP, 0, dv);
            // A2 / A3 are block-diagonal: clear the other species' blocks of this row
            float z[HP];
#pragma unroll
            for (int c = 0; c < HP; ++c) z[c] = 0.f;
            for (int s = 0; s < S; ++s) {
                if (s == ti) continue;
                put_row<PREC, HP>(A2, tid, HP * S, s * HP, z);
                put_row<PREC, HP>(A3, tid, HP * S, s * HP, z);
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < KP / O::KSTEP; ++kk)
                mma<PREC>(tmem + COL_P, smem_desc(smem_u32(A1) + kk * kstep_bytes, 128, sA1),
                          smem_desc(smem_u32(B1) + kk * kstep_bytes, 128, sA1), id1, kk > 0);
            mma_commit(&bar);
        }
        if (!mbar_wait_bounded(&bar, phase)) failed = 1;
        phase ^= 1u;
        tc_fence_after();
        // epilogue 1: P of the atom's species block (every block is read: the load is warp-wide)
        float pre[HP];
        for (int s = 0; s < S; ++s) {
            float v[32];
            tmem_ld32(tmem + lane_base + COL_P + s * HP, v);
            if (s == ti) {
#pragma unroll
                for (int c = 0; c < HP; ++c) pre[c] = v[c];
            }
        }
        float ue = 0.f, uqv = 0.f, ge[HP], gqv[HP];
#pragma unroll
        for (int mu = 0; mu < HP; ++mu) {
            const float h = tanh_fast(pre[mu] - pb0[ti * HP + mu]);
            const float we = pwe[ti * HP + mu], wq = pwq[ti * HP + mu];
            ue = fmaf(we, h, ue);
            uqv = fmaf(wq, h, uqv);
            const float dh = 1.f - h * h;
            ge[mu] = we * dh;
            gqv[mu] = wq * dh;
        }
        put_row<PREC, HP>(A2, tid, HP * S, ti * HP, ge);
        put_row<PREC, HP>(A3, tid, HP * S, ti * HP, gqv);
        const float U = ue - pb1[2 * ti], Q = uqv - pb1[2 * ti + 1];
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0 && !failed) {
            for (int kk = 0; kk < HP * S / O::KSTEP; ++kk) {
                const uint64_t b = smem_desc(smem_u32(B2) + kk * kstep_bytes, 128, sA2);
                mma<PREC>(tmem + COL_DU, smem_desc(smem_u32(A2) + kk * kstep_bytes, 128, sA2), b, id2, kk > 0);
                mma<PREC>(tmem + COL_DQ, smem_desc(smem_u32(A3) + kk * kstep_bytes, 128, sA2), b, id2, kk > 0);
            }
            mma_commit(&bar);
        }
        __syncthreads();
        if (!failed && !mbar_wait_bounded(&bar, phase)) failed = 1;
        phase ^= 1u;
        tc_fence_after();
        float gu[KP], gq[KP];
        tmem_ld32(tmem + lane_base + COL_DU, gu);
        tmem_ld32(tmem + lane_base + COL_DQ, gq);
        // rows of NDES floats in [n][NDES] order: staged in the free A2 / A3 regions (when a
        // region holds TM x NDES floats) and written back as contiguous float4s (the tile's
        // rows are one contiguous range)
        const bool rowmajor = du && d_sv == 1 && d_sa == NDES && HP * S * ES >= NDES * (int)sizeof(float);
        if (rowmajor) {
            float* su_ = reinterpret_cast<float*>(A2);
            float* sq_ = reinterpret_cast<float*>(A3);
#pragma unroll
            for (int v = 0; v < NDES; ++v) {
                su_[tid * NDES + v] = gu[v] * psc[v];
                sq_[tid * NDES + v] = gq[v] * psc[v];
            }
        }
        if (valid) {
            if (rowmajor) {
            } else if (du) {
#pragma unroll
                for (int v = 0; v < NDES; ++v) {
                    du[(size_t)k * d_sa + (size_t)v * d_sv] = gu[v] * psc[v];
                    dq[(size_t)k * d_sa + (size_t)v * d_sv] = gq[v] * psc[v];
                }
            }
            u_out[k] = U;
            q_out[k] = Q;
            su += (double)U;
            sq += (double)Q;
        }
        if (rowmajor) {
            __syncthreads();
            const int cnt = min(TM, n - tile * TM);
            const float4* su4 = reinterpret_cast<const float4*>(A2);
            const float4* sq4 = reinterpret_cast<const float4*>(A3);
            float4* du4 = reinterpret_cast<float4*>(du + (size_t)tile * TM * NDES);
            float4* dq4 = reinterpret_cast<float4*>(dq + (size_t)tile * TM * NDES);
            for (int e = tid; e < cnt * NDES / 4; e += TM) {
                du4[e] = su4[e];
                dq4[e] = sq4[e];
            }
            if (tid < (cnt * NDES) % 4) {   // a ragged tail (cnt odd): the last floats one by one
                const int e = cnt * NDES / 4 * 4 + tid;
                du[(size_t)tile * TM * NDES + e] = reinterpret_cast<const float*>(A2)[e];
                dq[(size_t)tile * TM * NDES + e] = reinterpret_cast<const float*>(A3)[e];
            }
        }
        tc_fence_before();
        __syncthreads();   // operands and accumulators are reused by the next tile
        tc_fence_after();
        if (failed) {
            // a copy or an MMA did not complete in time: let the next tile's copy land (bounded)
            if (tile + (int)gridDim.x < ntiles) mbar_wait_bounded(&dbar[(i + 1) & 1], (uint32_t)(((i + 1) >> 1) & 1));
            break;
        }
    }
    // block sums of U and q (FP64), one atomic each
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    if (lane == 0) {
        red[0][warp] = su;
        red[1][warp] = sq;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < TM / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        atomicAdd(&acc->sum_u, a);
        atomicAdd(&acc->sum_q, b);
        if (failed) atomicOr(&acc->status, kStatusTimeout);
    }
    if (warp == 0)
        tmem_free(tmem, TMEM_COLS);
}

}  // namespace

size_t mlp_tc_smem(int precision, int n_species) {
    const size_t need = precision == PREC_BF16 ? mlp_layout<PREC_BF16>(n_species).total
                                               : mlp_layout<PREC_TF32>(n_species).total;
    // at least 80 KB so that at most two blocks (2 x 256 tensor-memory columns) share an SM
    return need > 80 * 1024 ? need : 80 * 1024;
}

void launch_mlp_tc(int precision, const float* dtc, const float4* spos4, int n, const float* params,
                   const ParamLayout& lay, float* du, float* dq, int d_sa, int d_sv, float* u, float* q, Accum* acc,
                   int num_sms, cudaStream_t st) {
    if (n <= 0) return;
    const size_t smem = mlp_tc_smem(precision, lay.n_species);
    const int ntiles = (n + TM - 1) / TM;
    // persistent blocks: at most two per SM (256 tensor-memory columns each), fewer when the
    // operands of one block take more than half of the shared memory
    if (precision == PREC_BF16)
        cudaFuncSetAttribute(k_mlp_tc<PREC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else
        cudaFuncSetAttribute(k_mlp_tc<PREC_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // 227 KB of shared memory per SM for blocks (2 KB of it for static data and reserve each)
    int per_sm = (int)((size_t)227 * 1024 / (smem + 2048));
    per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
    const int grid = ntiles < per_sm * num_sms ? ntiles : per_sm * num_sms;
    if (precision == PREC_BF16)
        k_mlp_tc<PREC_BF16><<<grid, TM, smem, st>>>(dtc, spos4, n, params, lay, du, dq, d_sa, d_sv, u, q, acc);
    else
        k_mlp_tc<PREC_TF32><<<grid, TM, smem, st>>>(dtc, spos4, n, params, lay, du, dq, d_sa, d_sv, u, q, acc);
}

}  // namespace qnep
