// Velocity-Verlet NVE integration around the force call (kernels of qnep_nve_run).
//
// Units: positions A, velocities A/fs, forces eV/A, masses amu, time fs; an
// acceleration F/m in eV/(A amu) is 9.6485332e-3 A/fs^2 and a kinetic energy
// m v^2 / 2 in amu A^2/fs^2 is 103.6427 eV per unit.  Positions and velocities
// are FP32; the kinetic energy is reduced in FP64 (FP32 within a warp, FP64 across
// warps), the potential energy comes from the force call's FP64 scalar.
#include "qnep_internal.cuh"

namespace qnep {

namespace {

constexpr float ACC_UNIT = 9.6485332e-3f;       // (eV/A)/amu -> A/fs^2
constexpr double KE_UNIT = 103.6427;            // amu A^2/fs^2 -> eV

struct MdMass {
    float inv_m[MAX_SPECIES];   // 1 / m (1/amu)
    float m[MAX_SPECIES];       // m (amu)
};

// first half: v += dt/2 F/m, x += dt v
__global__ void k_vv_kick_drift(int n, float* __restrict__ pos, float* __restrict__ vel,
                                const float* __restrict__ f, const int* __restrict__ types, MdMass ms, float dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h = 0.5f * dt * ACC_UNIT * ms.inv_m[types[i]];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float v = fmaf(h, f[3 * i + d], vel[3 * i + d]);
        vel[3 * i + d] = v;
        pos[3 * i + d] = fmaf(dt, v, pos[3 * i + d]);
    }
}

// second half: v += dt/2 F/m and the kinetic energy of the step; the last block writes
// (U_pot, K) of the step and advances the device step counter (graph replays use it)
__global__ void k_vv_kick_energy(int n, float* __restrict__ vel, const float* __restrict__ f,
                                 const int* __restrict__ types, MdMass ms, float dt, int kick,
                                 const double* __restrict__ scalars, double* __restrict__ energies,
                                 int* __restrict__ step, double* __restrict__ ke_acc,
                                 unsigned int* __restrict__ done) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float k = 0.f;
    if (i < n) {
        const int t = types[i];
        const float h = kick ? 0.5f * dt * ACC_UNIT * ms.inv_m[t] : 0.f;
        float v2 = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float v = fmaf(h, f[3 * i + d], vel[3 * i + d]);
            vel[3 * i + d] = v;
            v2 = fmaf(v, v, v2);
        }
        k = 0.5f * ms.m[t] * v2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    __shared__ double red[32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = (double)k;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(ke_acc, t);
        __threadfence();
        const unsigned prev = atomicAdd(done, 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const int s = *step;
        energies[2 * s] = scalars[0];
        energies[2 * s + 1] = *ke_acc * KE_UNIT;
        *ke_acc = 0.0;
        *done = 0u;
        *step = s + 1;
    }
}

}  // namespace

void launch_vv_kick_drift(int n, float* pos, float* vel, const float* f, const int* types, const float* masses,
                          int n_species, float dt, cudaStream_t st) {
    MdMass ms{};
    for (int s = 0; s < n_species; ++s) {
        ms.m[s] = masses[s];
        ms.inv_m[s] = 1.f / masses[s];
    }
    k_vv_kick_drift<<<(n + 255) / 256, 256, 0, st>>>(n, pos, vel, f, types, ms, dt);
}

void launch_vv_kick_energy(int n, float* vel, const float* f, const int* types, const float* masses, int n_species,
                           float dt, bool kick, const double* scalars, double* energies, int* step, double* ke_acc,
                           unsigned int* done, cudaStream_t st) {
    MdMass ms{};
    for (int s = 0; s < n_species; ++s) {
        ms.m[s] = masses[s];
        ms.inv_m[s] = 1.f / masses[s];
    }
    k_vv_kick_energy<<<(n + 255) / 256, 256, 0, st>>>(n, vel, f, types, ms, dt, kick ? 1 : 0, scalars, energies, step,
                                                       ke_acc, done);
}

}  // namespace qnep
