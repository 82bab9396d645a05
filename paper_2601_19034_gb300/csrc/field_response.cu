// Response of the ions to a uniform external electric field, from the Born
// effective charges (Sec. II.D):
//   Eq. (electric_force):          F^ext_i,b = sum_a E_a Z_i,ab
//   Eq. (polarization_derivative): Pdot_a    = sum_i sum_b Z_i,ab v_i,b
//
// A streaming pass over Z [N][3][3], v [N][3] and F [N][3] (float32, atom-major,
// the layouts qnep_compute writes): algorithmically 36 + 12 + 12 bytes per atom
// (+12 when the force is added to an existing array), 15 or 18 flops, so the
// pass is bound by HBM bandwidth.  A persistent grid (resident blocks x SMs)
// walks tiles of 256 atoms; each block keeps a ring of three shared-memory
// stages filled by asynchronous copies (cp.async, 16 bytes per copy for aligned
// full tiles, 4 bytes otherwise), so two tiles are in flight while the third is
// contracted: the tile's Z, v (and old F) are contiguous (9216 + 3072 + 3072
// bytes), each thread contracts one atom from shared memory (odd strides 9 and
// 3: no bank conflicts) and the forces leave through a shared-memory tile as
// coalesced 16-byte streaming stores.  One thread also asks L2 for the inputs of
// the four tiles after the ring (bulk prefetch, a hint nothing waits on), so more
// DRAM requests are in flight than the shared-memory ring can hold.  The copies
// complete through cp.async.wait_group, a hardware wait: the kernel has no spin loop.
//
// Pdot: each thread keeps a compensated (Kahan) FP32 sum of its atoms' terms,
// each warp adds its 32 sums by FP32 shuffles (5 roundings, at most 5 x 2^-24 of
// sum |Z v|), and one thread per block adds the 8 warp sums in FP64 and the block
// total to the output with FP64 atomics, after the output has been cleared on
// the stream.  (GB300 runs FP64 at 1/64 of the FP32 rate: an FP64 add per 8
// atoms and thread kept its FP64 pipe 80 % busy and throttled the stream.)
#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/qnep.h"

namespace qnep {
namespace {

constexpr int kTile = 256;          // atoms per tile = threads per block
constexpr int kWarps = kTile / 32;
constexpr int kStages = 3;          // shared-memory ring: two tiles in flight, one in use
constexpr int kPrefetch = 4;        // tiles beyond the ring whose bytes are prefetched into L2
constexpr int kMinBlocks = 4;       // resident blocks per SM asked of the compiler

// Floats of one stage: Z, then v (Pdot), then the old forces (accumulate).
template <bool CURRENT, bool ACCUM>
struct Stage {
    static constexpr int v = kTile * 9;
    static constexpr int f = v + (CURRENT ? kTile * 3 : 0);
    static constexpr int floats = f + (ACCUM ? kTile * 3 : 0);
};

template <bool FORCE, bool CURRENT, bool ACCUM>
constexpr size_t smem_bytes() {
    return sizeof(float) * ((size_t)kStages * Stage<CURRENT, ACCUM>::floats + (FORCE ? kTile * 3 : 0));
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr(dst)), "l"(src) : "memory");
}
// Hint: fetch `bytes` (a multiple of 16, 16-byte aligned source) into L2; nothing waits on it.
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Start the copies of tile t into one stage (every thread issues its share).
template <bool VEC, bool CURRENT, bool ACCUM>
__device__ __forceinline__ void issue_tile(float* stage, int n, int t, const float* __restrict__ bec,
                                           const float* __restrict__ vel, const float* fext) {
    using L = Stage<CURRENT, ACCUM>;
    const int tid = threadIdx.x;
    const size_t a0 = (size_t)t * kTile;
    const int na = min(kTile, n - (int)a0);
    const float* gz = bec + a0 * 9;
    if (VEC && na == kTile) {
        for (int k = tid; k < kTile * 9 / 4; k += kTile) cp16(stage + 4 * k, gz + 4 * k);
        if (CURRENT)
            for (int k = tid; k < kTile * 3 / 4; k += kTile) cp16(stage + L::v + 4 * k, vel + a0 * 3 + 4 * k);
        if (ACCUM)
            for (int k = tid; k < kTile * 3 / 4; k += kTile) cp16(stage + L::f + 4 * k, fext + a0 * 3 + 4 * k);
    } else {
        for (int k = tid; k < na * 9; k += kTile) cp4(stage + k, gz + k);
        if (CURRENT)
            for (int k = tid; k < na * 3; k += kTile) cp4(stage + L::v + k, vel + a0 * 3 + k);
        if (ACCUM)
            for (int k = tid; k < na * 3; k += kTile) cp4(stage + L::f + k, fext + a0 * 3 + k);
    }
}

// One thread asks L2 for a full tile's inputs ahead of its copies (aligned path only).
template <bool CURRENT, bool ACCUM>
__device__ __forceinline__ void prefetch_tile(int n, int t, const float* bec, const float* vel, const float* fext) {
    const size_t a0 = (size_t)t * kTile;
    if ((int)a0 + kTile > n) return;
    prefetch_l2(bec + a0 * 9, kTile * 9 * sizeof(float));
    if (CURRENT) prefetch_l2(vel + a0 * 3, kTile * 3 * sizeof(float));
    if (ACCUM) prefetch_l2(fext + a0 * 3, kTile * 3 * sizeof(float));
}

template <bool VEC, bool FORCE, bool CURRENT, bool ACCUM>
__global__ void __launch_bounds__(kTile, kMinBlocks)
k_field_response(int n, const float* __restrict__ bec, float e0, float e1, float e2,
                 const float* __restrict__ vel, float* fext, double* __restrict__ pdot) {
    using L = Stage<CURRENT, ACCUM>;
    extern __shared__ __align__(16) float smem[];
    float* sOut = smem + (size_t)kStages * L::floats;     // forces of the tile in use
    __shared__ float sRed[3][kWarps];

    const int tid = threadIdx.x;
    const int ntiles = (n + kTile - 1) / kTile;
    const int mine = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    float ps[3] = {0.f, 0.f, 0.f}, pc[3] = {0.f, 0.f, 0.f};   // Kahan sums and compensations of Pdot

    // prologue: the first kStages - 1 tiles of this block (one commit group per tile slot)
    for (int j = 0; j < kStages - 1; ++j) {
        if (j < mine)
            issue_tile<VEC, CURRENT, ACCUM>(smem + (size_t)j * L::floats, n, blockIdx.x + j * gridDim.x, bec, vel,
                                            fext);
        cp_commit();
    }
    if (VEC && tid == 0)
        for (int j = kStages - 1; j < kStages - 1 + kPrefetch && j < mine; ++j)
            prefetch_tile<CURRENT, ACCUM>(n, blockIdx.x + j * gridDim.x, bec, vel, fext);

    for (int j = 0; j < mine; ++j) {
        const int jn = j + kStages - 1;
        if (VEC && tid == 0 && jn + kPrefetch < mine)
            prefetch_tile<CURRENT, ACCUM>(n, blockIdx.x + (jn + kPrefetch) * gridDim.x, bec, vel, fext);
        // the stage of tile jn was last read in iteration j - 1, before its second barrier
        if (jn < mine)
            issue_tile<VEC, CURRENT, ACCUM>(smem + (size_t)(jn % kStages) * L::floats, n,
                                            blockIdx.x + jn * gridDim.x, bec, vel, fext);
        cp_commit();
        cp_wait<kStages - 1>();          // this thread's copies of tile j have landed
        __syncthreads();                 // ... and every other thread's

        const int t = blockIdx.x + j * gridDim.x;
        const size_t a0 = (size_t)t * kTile;
        const int na = min(kTile, n - (int)a0);
        const float* st = smem + (size_t)(j % kStages) * L::floats;
        if (tid < na) {
            const float* z = st + tid * 9;
            const float z00 = z[0], z01 = z[1], z02 = z[2];
            const float z10 = z[3], z11 = z[4], z12 = z[5];
            const float z20 = z[6], z21 = z[7], z22 = z[8];
            if (FORCE) {
                float f0 = fmaf(e0, z00, fmaf(e1, z10, e2 * z20));
                float f1 = fmaf(e0, z01, fmaf(e1, z11, e2 * z21));
                float f2 = fmaf(e0, z02, fmaf(e1, z12, e2 * z22));
                if (ACCUM) {
                    f0 += st[L::f + tid * 3 + 0];
                    f1 += st[L::f + tid * 3 + 1];
                    f2 += st[L::f + tid * 3 + 2];
                }
                sOut[tid * 3 + 0] = f0;
                sOut[tid * 3 + 1] = f1;
                sOut[tid * 3 + 2] = f2;
            }
            if (CURRENT) {
                const float v0 = st[L::v + tid * 3 + 0], v1 = st[L::v + tid * 3 + 1], v2 = st[L::v + tid * 3 + 2];
                const float x[3] = {fmaf(z00, v0, fmaf(z01, v1, z02 * v2)), fmaf(z10, v0, fmaf(z11, v1, z12 * v2)),
                                    fmaf(z20, v0, fmaf(z21, v1, z22 * v2))};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float y = x[a] - pc[a];
                    const float t = ps[a] + y;
                    pc[a] = (t - ps[a]) - y;
                    ps[a] = t;
                }
            }
        }
        __syncthreads();                 // stage j % kStages fully read; sOut complete
        if (FORCE) {
            float* gf = fext + a0 * 3;
            if (VEC && na == kTile) {
                if (tid < kTile * 3 / 4)
                    __stcs(reinterpret_cast<float4*>(gf) + tid, reinterpret_cast<const float4*>(sOut)[tid]);
            } else {
                for (int k = tid; k < na * 3; k += kTile) gf[k] = sOut[k];
            }
        }
        // sOut is rewritten only after the next iteration's first barrier
    }
    cp_wait<0>();                        // no copy left in flight at exit (all groups past the loop are empty)

    if (CURRENT) {
        float w3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float v = ps[a] - pc[a];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            w3[a] = v;
        }
        const int w = tid >> 5;
        if ((tid & 31) == 0) {
            sRed[0][w] = w3[0];
            sRed[1][w] = w3[1];
            sRed[2][w] = w3[2];
        }
        __syncthreads();
        if (tid < 3) {
            double s = 0.0;
            for (int k = 0; k < kWarps; ++k) s += (double)sRed[tid][k];
            atomicAdd(pdot + tid, s);
        }
    }
}

template <bool VEC, bool FORCE, bool CURRENT, bool ACCUM>
cudaError_t launch(int grid_cap, int n, const float* bec, const float e[3], const float* vel, float* fext,
                   double* pdot, cudaStream_t st) {
    auto kern = k_field_response<VEC, FORCE, CURRENT, ACCUM>;
    constexpr size_t smem = smem_bytes<FORCE, CURRENT, ACCUM>();
    static std::mutex mu;
    static int per_sm[64] = {};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int occ = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (per_sm[dev] > 0) {
            occ = per_sm[dev];
        } else {
            err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTile, smem);
            if (err != cudaSuccess) return err;
            if (occ < 1) return cudaErrorInvalidConfiguration;
            per_sm[dev] = occ;
        }
    }
    const int ntiles = (n + kTile - 1) / kTile;
    const long long cap = (long long)grid_cap * occ;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    kern<<<grid, kTile, smem, st>>>(n, bec, e[0], e[1], e[2], vel, fext, pdot);
    return cudaGetLastError();
}

template <bool VEC>
cudaError_t dispatch(int sms, int n, const float* bec, const float e[3], const float* vel, float* fext, int accumulate,
                     double* pdot, cudaStream_t st) {
    const bool force = fext != nullptr, current = pdot != nullptr;
    if (force && current)
        return accumulate ? launch<VEC, true, true, true>(sms, n, bec, e, vel, fext, pdot, st)
                          : launch<VEC, true, true, false>(sms, n, bec, e, vel, fext, pdot, st);
    if (force)
        return accumulate ? launch<VEC, true, false, true>(sms, n, bec, e, vel, fext, pdot, st)
                          : launch<VEC, true, false, false>(sms, n, bec, e, vel, fext, pdot, st);
    return launch<VEC, false, true, false>(sms, n, bec, e, vel, fext, pdot, st);
}

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace
}  // namespace qnep

extern "C" qnep_status qnep_field_response(int n_atoms, const float* bec, const double* efield,
                                           const float* velocities, float* forces, int accumulate, double* pdot,
                                           void* stream) {
    using namespace qnep;
    if (n_atoms < 0 || n_atoms > INT_MAX / 9) return QNEP_ERR_ARG;
    if (!forces && !pdot) return QNEP_OK;                       // nothing requested
    if (forces && !efield) return QNEP_ERR_ARG;
    if (pdot && ((n_atoms > 0 && !velocities) || !aligned(pdot, 8))) return QNEP_ERR_ARG;
    if (accumulate != 0 && accumulate != 1) return QNEP_ERR_ARG;
    if (n_atoms > 0 && !bec) return QNEP_ERR_ARG;
    if (!aligned(bec, 4) || !aligned(velocities, 4) || !aligned(forces, 4)) return QNEP_ERR_ARG;
    float e[3] = {0.f, 0.f, 0.f};
    if (forces)
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(efield[a])) return QNEP_ERR_ARG;
            e[a] = (float)efield[a];
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (pdot && cudaMemsetAsync(pdot, 0, 3 * sizeof(double), st) != cudaSuccess) return QNEP_ERR_CUDA;
    if (n_atoms == 0) return QNEP_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return QNEP_ERR_CUDA;
    const bool vec = aligned(bec, 16) && (!pdot || aligned(velocities, 16)) && (!forces || aligned(forces, 16));
    const float* vel = pdot ? velocities : nullptr;
    cudaError_t err = vec ? dispatch<true>(sms, n_atoms, bec, e, vel, forces, accumulate, pdot, st)
                          : dispatch<false>(sms, n_atoms, bec, e, vel, forces, accumulate, pdot, st);
    return err == cudaSuccess ? QNEP_OK : QNEP_ERR_CUDA;
}
