// Training side of the batched force call (Sec. II.E): the loss of every candidate of a
// population and the separable natural evolution strategy (SNES, Schaul et al. 2011, the
// method the paper trains every parameter with) that moves the search distribution.
//
//   qnep_snes_sample   z_k = mu + sigma * s_k                         [C][P]
//   qnep_batch_loss    D_e, D_f (energy RMSE per atom, force RMSE per component), |z|_1,
//                      |z|_2^2 and L = l_e D_e + l_f D_f + l_1 |z|_1 + l_2 |z|_2^2 per candidate;
//                      qnep_batch_loss_v adds D_v (virial RMSE per atom over the six
//                      independent components) and l_v D_v; qnep_batch_loss_full adds D_Z (BEC
//                      RMSE over the structures with reference BEC) and D_Q (RMSE of the total
//                      charge before the correction) with their weights
//   qnep_snes_update   rank the losses, rank-based utilities, natural-gradient step on
//                      (mu, sigma)
// The batched call feeds energies, forces, virials, BEC and the uncorrected total charges.
//
// Loss: the force term is the large one (C x N x 3 floats, HBM bound): for every candidate a
// one-wave set of blocks walks the force stream in 2048-float chunks (coalesced loads, 8 per
// thread in flight), each thread keeps a compensated (Kahan) FP32 sum of its squares, warps add
// their 32 sums in FP32 and one thread adds the block's 8 warp sums in FP64 and the block total
// with an FP64 atomic (GB300 runs FP64 at 1/64 of the FP32 rate: FP64 warp reductions in every
// one of ~31,000 small blocks held the pass to 16 % of HBM); one more block per candidate sums
// the energy terms and the parameter norms in FP64 and writes them directly; a one-block pass
// forms the roots and the weighted sum.
// Update: every block ranks the (at most 1024) losses in shared memory (ties by index, NaN last),
// forms the utilities in FP64 (their normaliser is the sum of all candidates' raw weights, each
// rank occurring once), then takes its parameters: g_mu = sum_k u_k s_k, g_sigma = sum_k u_k
// (s_k^2 - 1) in FP64, mu += eta_mu sigma g_mu, sigma *= exp(eta_sigma / 2 g_sigma).
#include <climits>
#include <cmath>
#include <cstdint>

#include "../../include/qnep.h"

namespace qnep {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;                       // force elements per thread (FP32 partial)
constexpr int kChunk = kThreads * kPerThread;       // force elements per block
constexpr int kMaxCandidates = 1024;

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();                                // red may still be read by an earlier call
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += red[k];
    return s;
}

__global__ void __launch_bounds__(kThreads)
k_snes_sample(long long total, int n_params, const float* __restrict__ mu, const float* __restrict__ sigma,
              const float* __restrict__ noise, float* __restrict__ z) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(i % n_params);
        z[i] = fmaf(sigma[p], noise[i], mu[p]);
    }
}

// BEC terms of the full loss (NULL bec: none)
struct BecLoss {
    const float* bec;        // [C][N][9]
    const float* bec_ref;    // [N][9]
    const int* has;          // [S] nonzero: the structure has reference BEC
    int n_zblocks;           // blocks per candidate over the referenced structures
    const double* qtot;      // [C][S] total charge before the correction, or NULL
    const double* qtot_ref;  // [S]
};

// Kahan sum of one thread's squares, the warps' sums in FP32, the block's in FP64, added to *dst
__device__ __forceinline__ void add_block_squares(float s, float comp, float* redf, double* dst) {
    float v = s - comp;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) redf[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += (double)redf[w];
        atomicAdd(dst, t);
    }
}

// blockIdx.y = candidate; blockIdx.x < n_fblocks: every n_fblocks-th chunk of the force stream;
// then n_zblocks blocks over the BEC of the referenced structures (every n_zblocks-th structure);
// the last: the energy, virial and total-charge terms and the parameter norms.  terms[ts c + k]:
// D_e (0), sum of squared force errors (1, rooted by k_loss_finalize), D_v (2, ts >= 5), sum of
// squared BEC errors (3, ts = 7, rooted by k_loss_finalize), D_Q (4, ts = 7), |z|_1, |z|_2^2 (the
// last two).
__global__ void __launch_bounds__(kThreads)
k_batch_loss(int n_struct, const int* __restrict__ off, long long n_force, int n_fblocks,
             const double* __restrict__ energy, const float* __restrict__ forces,
             const double* __restrict__ energy_ref, const float* __restrict__ forces_ref,
             const double* __restrict__ virial, const double* __restrict__ virial_ref, BecLoss bz,
             const float* __restrict__ params, int n_params, int ts, double* __restrict__ terms) {
    __shared__ double red[kThreads / 32];
    __shared__ float redf[kThreads / 32];
    const int c = blockIdx.y;
    if ((int)blockIdx.x >= n_fblocks && (int)blockIdx.x < n_fblocks + bz.n_zblocks) {
        // BEC: the 9 n_s components of each referenced structure, 8 loads per thread in flight
        const long long n_z = 3 * n_force;   // 9 N
        const float* zc = bz.bec + (long long)c * n_z;
        float s = 0.f, comp = 0.f;
        for (int st = (int)blockIdx.x - n_fblocks; st < n_struct; st += bz.n_zblocks) {
            if (!bz.has[st]) continue;
            const long long lo = 9LL * off[st], hi = 9LL * off[st + 1];
            for (long long base = lo + threadIdx.x; base < hi; base += kChunk) {
                float d[kPerThread];
#pragma unroll
                for (int k = 0; k < kPerThread; ++k) {
                    const long long i = base + (long long)k * kThreads;
                    d[k] = i < hi ? zc[i] - bz.bec_ref[i] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < kPerThread; ++k) {
                    const float y = d[k] * d[k] - comp;
                    const float t = s + y;
                    comp = (t - s) - y;
                    s = t;
                }
            }
        }
        add_block_squares(s, comp, redf, terms + ts * c + 3);
        return;
    }
    if ((int)blockIdx.x < n_fblocks) {
        const float* fc = forces + (long long)c * n_force;
        float s = 0.f, comp = 0.f;                     // Kahan sum of this thread's squares
        for (long long base = (long long)blockIdx.x * kChunk + threadIdx.x; base < n_force;
             base += (long long)n_fblocks * kChunk) {
            float d[kPerThread];
#pragma unroll
            for (int k = 0; k < kPerThread; ++k) {
                const long long i = base + (long long)k * kThreads;
                d[k] = i < n_force ? fc[i] - forces_ref[i] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < kPerThread; ++k) {
                const float y = d[k] * d[k] - comp;
                const float t = s + y;
                comp = (t - s) - y;
                s = t;
            }
        }
        add_block_squares(s, comp, redf, terms + ts * c + 1);
        return;
    }
    double se = 0.0, cnt = 0.0, l1 = 0.0, l2 = 0.0, sv = 0.0, sq = 0.0;
    for (int s = threadIdx.x; s < n_struct; s += kThreads) {
        const int n_s = off[s + 1] - off[s];
        if (n_s > 0) {
            const double de = (energy[(long long)c * n_struct + s] - energy_ref[s]) / (double)n_s;
            se += de * de;
            cnt += 1.0;
            if (virial) {
                // the six independent components xx, yy, zz, xy, yz, zx of the 3x3 virial, per atom
                const double* w = virial + ((long long)c * n_struct + s) * 9;
                const double* wr = virial_ref + (long long)s * 9;
                const int comp[6] = {0, 4, 8, 1, 5, 2};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const double dv = (w[comp[q]] - wr[comp[q]]) / (double)n_s;
                    sv += dv * dv;
                }
            }
            if (bz.qtot) {
                const double dq = bz.qtot[(long long)c * n_struct + s] - bz.qtot_ref[s];
                sq += dq * dq;
            }
        }
    }
    if (params)
        for (int p = threadIdx.x; p < n_params; p += kThreads) {
            const double z = params[(long long)c * n_params + p];
            l1 += fabs(z);
            l2 += z * z;
        }
    se = block_sum(se, red);
    cnt = block_sum(cnt, red);
    l1 = block_sum(l1, red);
    l2 = block_sum(l2, red);
    sv = block_sum(sv, red);
    sq = block_sum(sq, red);
    if (threadIdx.x == 0) {
        terms[ts * c + 0] = cnt > 0.0 ? sqrt(se / cnt) : 0.0;
        if (ts >= 5) terms[ts * c + 2] = (virial && cnt > 0.0) ? sqrt(sv / (6.0 * cnt)) : 0.0;
        if (ts == 7) terms[ts * c + 4] = (bz.qtot && cnt > 0.0) ? sqrt(sq / cnt) : 0.0;
        terms[ts * c + ts - 2] = l1;
        terms[ts * c + ts - 1] = l2;
    }
}

__global__ void k_loss_finalize(int n_cand, long long n_force, double we, double wf, double wv, double wz, double wq,
                                double w1, double w2, int ts, int n_struct, const int* __restrict__ off,
                                const int* __restrict__ has, double* __restrict__ terms, double* __restrict__ loss) {
    __shared__ double red[kThreads / 32];
    double nz = 0.0;   // atoms of the structures with reference BEC
    if (has)
        for (int s = threadIdx.x; s < n_struct; s += blockDim.x)
            if (has[s]) nz += (double)(off[s + 1] - off[s]);
    nz = block_sum(nz, red);
    for (int c = threadIdx.x; c < n_cand; c += blockDim.x) {
        double* t = terms + ts * c;
        const double df = n_force > 0 ? sqrt(t[1] / (double)n_force) : 0.0;
        t[1] = df;
        double l = we * t[0] + wf * df + (ts >= 5 ? wv * t[2] : 0.0) + w1 * t[ts - 2] + w2 * t[ts - 1];
        if (ts == 7) {
            const double dz = nz > 0.0 ? sqrt(t[3] / (9.0 * nz)) : 0.0;
            t[3] = dz;
            l += wz * dz + wq * t[4];
        }
        loss[c] = l;
    }
}

// true when candidate j ranks before candidate c: lower loss, NaN last, ties by index
__device__ __forceinline__ bool ranks_before(double fj, int j, double fc, int c) {
    const bool nj = isnan(fj), nc = isnan(fc);
    if (nj != nc) return nc;
    if (!nj && fj != fc) return fj < fc;
    return j < c;
}

__global__ void __launch_bounds__(kThreads)
k_snes_update(int n_cand, int n_params, const double* __restrict__ loss, const float* __restrict__ noise,
              float* __restrict__ mu, float* __restrict__ sigma, double eta_mu, double eta_sigma) {
    __shared__ double f[kMaxCandidates];
    __shared__ double u[kMaxCandidates];
    __shared__ double red[kThreads / 32];
    for (int c = threadIdx.x; c < n_cand; c += kThreads) f[c] = loss[c];
    __syncthreads();
    const double top = log(0.5 * n_cand + 1.0);
    double wsum = 0.0;
    for (int c = threadIdx.x; c < n_cand; c += kThreads) {
        int rank = 0;
        const double fc = f[c];
        for (int j = 0; j < n_cand; ++j) rank += ranks_before(f[j], j, fc, c) ? 1 : 0;
        const double w = fmax(0.0, top - log((double)(rank + 1)));
        u[c] = w;
        wsum += w;
    }
    wsum = block_sum(wsum, red);                    // also orders the writes of u before the reads
    const double inv_c = 1.0 / n_cand;
    for (int c = threadIdx.x; c < n_cand; c += kThreads) u[c] = u[c] / wsum - inv_c;
    __syncthreads();
    for (int p = blockIdx.x * kThreads + threadIdx.x; p < n_params; p += gridDim.x * kThreads) {
        double gm = 0.0, gs = 0.0;
        for (int c = 0; c < n_cand; ++c) {
            const double s = noise[(long long)c * n_params + p];
            gm = fma(u[c], s, gm);
            gs = fma(u[c], fma(s, s, -1.0), gs);
        }
        const double sg = sigma[p];
        mu[p] = (float)(mu[p] + eta_mu * sg * gm);
        sigma[p] = (float)(sg * exp(0.5 * eta_sigma * gs));
    }
}

int grid_for(long long work, int per_block) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = (work + per_block - 1) / per_block;
    const long long cap = (long long)(sms > 0 ? sms : 152) * 8;
    return (int)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

}  // namespace
}  // namespace qnep

using namespace qnep;

extern "C" qnep_status qnep_snes_sample(int n_candidates, int n_params, const float* mu, const float* sigma,
                                        const float* noise, float* params, void* stream) {
    if (n_candidates < 1 || n_params < 1 || !mu || !sigma || !noise || !params) return QNEP_ERR_ARG;
    const long long total = (long long)n_candidates * n_params;
    k_snes_sample<<<grid_for(total, kThreads), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        total, n_params, mu, sigma, noise, params);
    return cudaGetLastError() == cudaSuccess ? QNEP_OK : QNEP_ERR_CUDA;
}

namespace {
qnep_status batch_loss_impl(int n_candidates, int n_struct, const int* atom_offsets, int n_total,
                            const double* energy, const float* forces, const double* virial,
                            const double* energy_ref, const float* forces_ref, const double* virial_ref,
                            const float* params, int n_params, double we, double wf, double wv, double w1, double w2,
                            int ts, double* loss, double* terms, void* stream, BecLoss bz = BecLoss{},
                            double wz = 0.0, double wq = 0.0) {
    if (n_candidates < 1 || n_candidates > 65535 || n_struct < 1 || n_total < 0 || !atom_offsets || !energy ||
        !energy_ref || !loss || !terms)
        return QNEP_ERR_ARG;
    if ((forces == nullptr) != (forces_ref == nullptr)) return QNEP_ERR_ARG;
    if ((virial == nullptr) != (virial_ref == nullptr)) return QNEP_ERR_ARG;
    if (params && n_params < 1) return QNEP_ERR_ARG;
    if (!std::isfinite(we) || !std::isfinite(wf) || !std::isfinite(wv) || !std::isfinite(w1) || !std::isfinite(w2) ||
        !std::isfinite(wz) || !std::isfinite(wq))
        return QNEP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n_force = forces ? 3LL * n_total : 0;
    const long long chunks = (n_force + kChunk - 1) / kChunk;
    // one wave of 8 blocks per SM over all candidates, at least one block per candidate
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long per_cand = ((long long)(sms > 0 ? sms : 152) * 8 + n_candidates - 1) / n_candidates;
    const int n_fblocks = (int)(chunks < per_cand ? chunks : per_cand);
    bz.n_zblocks = bz.bec ? (int)(n_struct < per_cand ? n_struct : per_cand) : 0;
    if (cudaMemsetAsync(terms, 0, sizeof(double) * ts * (size_t)n_candidates, st) != cudaSuccess)
        return QNEP_ERR_CUDA;
    dim3 grid((unsigned)(n_fblocks + bz.n_zblocks + 1), (unsigned)n_candidates);
    k_batch_loss<<<grid, kThreads, 0, st>>>(n_struct, atom_offsets, 3LL * n_total, n_fblocks, energy, forces,
                                            energy_ref, forces_ref, virial, virial_ref, bz, params,
                                            params ? n_params : 0, ts, terms);
    if (cudaGetLastError() != cudaSuccess) return QNEP_ERR_CUDA;
    k_loss_finalize<<<1, kThreads, 0, st>>>(n_candidates, n_force, we, wf, wv, wz, wq, w1, w2, ts, n_struct,
                                            atom_offsets, bz.bec ? bz.has : nullptr, terms, loss);
    return cudaGetLastError() == cudaSuccess ? QNEP_OK : QNEP_ERR_CUDA;
}
}  // namespace

extern "C" qnep_status qnep_batch_loss(int n_candidates, int n_struct, const int* atom_offsets, int n_total,
                                      const double* energy, const float* forces, const double* energy_ref,
                                      const float* forces_ref, const float* params, int n_params,
                                      const qnep_loss_weights* w, double* loss, double* terms, void* stream) {
    if (!w) return QNEP_ERR_ARG;
    return batch_loss_impl(n_candidates, n_struct, atom_offsets, n_total, energy, forces, nullptr, energy_ref,
                           forces_ref, nullptr, params, n_params, w->energy, w->force, 0.0, w->l1, w->l2, 4, loss,
                           terms, stream);
}

extern "C" qnep_status qnep_batch_loss_v(int n_candidates, int n_struct, const int* atom_offsets, int n_total,
                                        const double* energy, const float* forces, const double* virial,
                                        const double* energy_ref, const float* forces_ref, const double* virial_ref,
                                        const float* params, int n_params, const qnep_loss_weights_v* w,
                                        double* loss, double* terms, void* stream) {
    if (!w) return QNEP_ERR_ARG;
    return batch_loss_impl(n_candidates, n_struct, atom_offsets, n_total, energy, forces, virial, energy_ref,
                           forces_ref, virial_ref, params, n_params, w->energy, w->force, w->virial, w->l1, w->l2, 5,
                           loss, terms, stream);
}

extern "C" qnep_status qnep_batch_loss_full(int n_candidates, int n_struct, const int* atom_offsets, int n_total,
                                           const qnep_loss_inputs* in, const qnep_loss_inputs* ref,
                                           const int* bec_has_ref, const float* params, int n_params,
                                           const qnep_loss_weights_full* w, double* loss, double* terms,
                                           void* stream) {
    if (!w || !in || !ref) return QNEP_ERR_ARG;
    if ((in->bec == nullptr) != (ref->bec == nullptr) || (in->bec && !bec_has_ref)) return QNEP_ERR_ARG;
    if ((in->total_charge == nullptr) != (ref->total_charge == nullptr)) return QNEP_ERR_ARG;
    BecLoss bz{in->bec, ref->bec, bec_has_ref, 0, in->total_charge, ref->total_charge};
    return batch_loss_impl(n_candidates, n_struct, atom_offsets, n_total, in->energy, in->forces, in->virial,
                           ref->energy, ref->forces, ref->virial, params, n_params, w->energy, w->force, w->virial,
                           w->l1, w->l2, 7, loss, terms, stream, bz, w->bec, w->charge);
}

extern "C" qnep_status qnep_snes_update(int n_candidates, int n_params, const double* loss, const float* noise,
                                        float* mu, float* sigma, double eta_mu, double eta_sigma, void* stream) {
    if (n_candidates < 1 || n_candidates > kMaxCandidates || n_params < 1 || !loss || !noise || !mu || !sigma)
        return QNEP_ERR_ARG;
    if (!std::isfinite(eta_mu) || !std::isfinite(eta_sigma)) return QNEP_ERR_ARG;
    if (eta_mu < 0) eta_mu = 1.0;
    if (eta_sigma < 0) eta_sigma = (3.0 + std::log((double)n_params)) / (5.0 * std::sqrt((double)n_params));
    k_snes_update<<<grid_for(n_params, kThreads), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        n_candidates, n_params, loss, noise, mu, sigma, eta_mu, eta_sigma);
    return cudaGetLastError() == cudaSuccess ? QNEP_OK : QNEP_ERR_CUDA;
}
