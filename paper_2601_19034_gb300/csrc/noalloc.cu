// Reciprocal-space Ewald sum of given charges that allocates no device memory.
//
// Some callers must not allocate device memory: host programs that hand all of
// the GPU's memory to their own pool allocator and forbid allocations from
// libraries, and time-critical loops where cudaMalloc / cudaFree would
// synchronise the device.  qnep_ewald_kspace_noalloc serves them.  It runs the
// same kernels as the reciprocal-space stage of qnep_compute (phase factors,
// structure factor, FP64 energy / virial, per-atom potential and force), but
// every scratch buffer lives in one file-scope __device__ array of fixed size
// (QNEP_NOALLOC_* in qnep.h, about 10 MB) that each GPU loading the library
// keeps until the process exits.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress (host code cannot use the
// symbol itself: on the host it names a host-side stand-in).  Make that first
// call before any stream capture.  All calls share the array and it keeps the
// previous call's contents: the structure factor and the accumulators are
// cleared at the start of every call, and calls that overlap on the GPU (two
// streams, or two host threads) race on the array.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/qnep.h"
#include "kset_host.h"
#include "qnep_internal.cuh"

namespace qnep {
namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr size_t kMaxAtoms = QNEP_NOALLOC_MAX_ATOMS;
constexpr size_t kMaxPhase = QNEP_NOALLOC_MAX_PHASE;
constexpr size_t kMaxKpad = QNEP_NOALLOC_MAX_KPAD;
constexpr size_t kMaxCols = kMaxKpad / 8;

// byte offsets of the regions inside the scratch array
constexpr size_t kOffPos4 = 0;
constexpr size_t kOffPhase = kOffPos4 + align256(kMaxAtoms * sizeof(float4));
constexpr size_t kOffAcc12 = kOffPhase + align256(kMaxAtoms * kMaxPhase * sizeof(float2));
constexpr size_t kOffPhi = kOffAcc12 + align256(kMaxAtoms * 12 * sizeof(float));
constexpr size_t kOffS = kOffPhi + align256(kMaxAtoms * sizeof(float));
constexpr size_t kOffC = kOffS + align256(kMaxKpad * sizeof(double2));
constexpr size_t kOffKg = kOffC + align256(kMaxKpad * sizeof(float2));
constexpr size_t kOffCol = kOffKg + align256(kMaxKpad * sizeof(float));
constexpr size_t kOffChunk = kOffCol + align256((kMaxCols + 1) * sizeof(int4));
constexpr size_t kOffAccum = kOffChunk + align256(kMaxCols * sizeof(int));
constexpr size_t kScratchBytes = kOffAccum + align256(sizeof(Accum));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[256] = {};

void put_err(char* err, size_t len, const char* msg) {
    if (err && len) std::snprintf(err, len, "%s", msg);
}

qnep_status scratch_address(unsigned char** out, char* err, size_t len) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        put_err(err, len, "no current CUDA device");
        return QNEP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            put_err(err, len, cudaGetErrorString(e));
            return QNEP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return QNEP_OK;
}

// Wrap positions into the box (the same arithmetic as the cell-binning kernel).
__global__ void k_wrap(const float* __restrict__ pos, int n, float lx, float ly, float lz, float ilx, float ily,
                       float ilz, float4* __restrict__ pos4) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float L[3] = {lx, ly, lz}, iL[3] = {ilx, ily, ilz};
    float w[3];
    for (int d = 0; d < 3; ++d) {
        float x = pos[3 * i + d];
        float f = floorf(x * iL[d]);
        float y = fmaf(-f, L[d], x);
        if (y >= L[d]) y -= L[d];
        if (y < 0.f) y += L[d];
        if (y >= L[d]) y = 0.f;
        w[d] = y;
    }
    pos4[i] = make_float4(w[0], w[1], w[2], 0.f);
}

}  // namespace
}  // namespace qnep

using namespace qnep;

extern "C" qnep_status qnep_ewald_kspace_noalloc(int n, const float* positions, const float* charges,
                                                 const double box[9], double alpha, double kmax, float* potential,
                                                 float* forces, double* energy_virial, void* stream, char* err,
                                                 size_t err_len) {
    if (n < 1 || !positions || !charges || !box) {
        put_err(err, err_len, "n must be >= 1 and positions, charges, box non-NULL");
        return QNEP_ERR_ARG;
    }
    if ((size_t)n > kMaxAtoms) {
        put_err(err, err_len, "too many atoms for the fixed scratch array (QNEP_NOALLOC_MAX_ATOMS)");
        return QNEP_ERR_UNSUPPORTED;
    }
    if (!(alpha > 0) || !(kmax > 0) || !std::isfinite(alpha) || !std::isfinite(kmax)) {
        put_err(err, err_len, "alpha and kmax must be positive and finite");
        return QNEP_ERR_ARG;
    }
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(box[k])) {
            put_err(err, err_len, "box has a non-finite entry");
            return QNEP_ERR_ARG;
        }
    if (box[1] != 0 || box[2] != 0 || box[3] != 0 || box[5] != 0 || box[6] != 0 || box[7] != 0 || !(box[0] > 0) ||
        !(box[4] > 0) || !(box[8] > 0)) {
        put_err(err, err_len, "only orthorhombic boxes with positive edges are supported");
        return QNEP_ERR_UNSUPPORTED;
    }
    const double L[3] = {box[0], box[4], box[8]};
    const double two_pi = 6.283185307179586;
    // Bound the k-set before enumerating it: n_max of each axis fixes the phase factors per atom,
    // so a k_max * L that would overflow an int, or loop for long, is refused here.
    long long nm[3];
    for (int d = 0; d < 3; ++d) {
        const double x = std::floor(kmax * L[d] / two_pi);
        if (!(x < (double)kMaxPhase)) {
            put_err(err, err_len,
                    "k_max * box edge too large for the fixed scratch array (QNEP_NOALLOC_MAX_PHASE / _KPAD)");
            return QNEP_ERR_UNSUPPORTED;
        }
        nm[d] = (long long)x;
    }
    long long nph = (nm[0] + 1) + (2 * nm[1] + 1) + (2 * nm[2] + 8);
    if ((nph & 1) == 0) nph += 1;
    if ((size_t)nph > kMaxPhase) {
        put_err(err, err_len, "k_max * box edge too large for the fixed scratch array (QNEP_NOALLOC_MAX_PHASE / _KPAD)");
        return QNEP_ERR_UNSUPPORTED;
    }
    // the half-space k columns and their 8-wide chunks, as for qnep_compute (at most
    // 128^3 / 2 candidate triples once n_max is bounded)
    KSet ks;
    try {
        ks = build_kset(L, kmax, alpha);
    } catch (...) {
        put_err(err, err_len, "host memory for the k-set could not be obtained");
        return QNEP_ERR_OOM;
    }
    const std::vector<int4>& cols = ks.cols;
    const std::vector<int>& chunk_col = ks.chunk_col;
    const std::vector<float>& kg = ks.kg;
    const int* nmax = ks.nmax;
    const int ncol = (int)cols.size() - 1;
    EwaldTab t{};
    t.n1max = nmax[0];
    t.n2max = nmax[1];
    t.n3max = nmax[2];
    t.ncol = ncol;
    t.nchunk = (int)chunk_col.size();
    t.nk = (int)kg.size();
    t.yoff = nmax[0] + 1;
    t.zoff = t.yoff + 2 * nmax[1] + 1;
    t.nph = t.zoff + 2 * nmax[2] + 8;
    if ((t.nph & 1) == 0) t.nph += 1;
    if ((size_t)t.nph > kMaxPhase || (size_t)t.nk > kMaxKpad || (size_t)ncol > kMaxCols) {
        put_err(err, err_len, "k_max * box edge too large for the fixed scratch array (QNEP_NOALLOC_MAX_PHASE / _KPAD)");
        return QNEP_ERR_UNSUPPORTED;
    }
    unsigned char* base = nullptr;
    qnep_status s = scratch_address(&base, err, err_len);
    if (s != QNEP_OK) return s;
    float4* pos4 = reinterpret_cast<float4*>(base + kOffPos4);
    float* acc12 = reinterpret_cast<float*>(base + kOffAcc12);
    float* phi = potential ? potential : reinterpret_cast<float*>(base + kOffPhi);
    Accum* acc = reinterpret_cast<Accum*>(base + kOffAccum);
    int4* d_col = reinterpret_cast<int4*>(base + kOffCol);
    int* d_chunk = reinterpret_cast<int*>(base + kOffChunk);
    float* d_kg = reinterpret_cast<float*>(base + kOffKg);
    for (int d = 0; d < 3; ++d) {
        t.L[d] = (float)L[d];
        const double il = 1.0 / L[d];
        t.invl_hi[d] = (float)il;
        t.invl_lo[d] = (float)(il - (double)t.invl_hi[d]);
    }
    t.alpha = (float)alpha;
    t.col = d_col;
    t.chunk_col = d_chunk;
    t.kg = d_kg;
    t.S = reinterpret_cast<double2*>(base + kOffS);
    t.C = reinterpret_cast<float2*>(base + kOffC);
    t.phase = reinterpret_cast<float2*>(base + kOffPhase);

    cudaStream_t st = (cudaStream_t)stream;
    auto cuda_fail = [&](cudaError_t e) {
        put_err(err, err_len, cudaGetErrorString(e));
        return QNEP_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_col, cols.data(), sizeof(int4) * cols.size(), cudaMemcpyHostToDevice, st))) return cuda_fail(e);
    if (t.nchunk && (e = cudaMemcpyAsync(d_chunk, chunk_col.data(), sizeof(int) * chunk_col.size(),
                                         cudaMemcpyHostToDevice, st)))
        return cuda_fail(e);
    if (t.nk && (e = cudaMemcpyAsync(d_kg, kg.data(), sizeof(float) * kg.size(), cudaMemcpyHostToDevice, st)))
        return cuda_fail(e);
    if ((e = cudaMemsetAsync(acc, 0, sizeof(Accum), st))) return cuda_fail(e);
    k_wrap<<<(n + 255) / 256, 256, 0, st>>>(positions, n, t.L[0], t.L[1], t.L[2], (float)(1.0 / L[0]),
                                            (float)(1.0 / L[1]), (float)(1.0 / L[2]), pos4);
    launch_ewald_phases(pos4, n, t, st);
    launch_ewald_sk(charges, acc, n, 0.f, t, st);          // clears S first
    launch_ewald_sk_finalize(t, acc, st);
    Geom g{};
    ElecConst ec{2, QNEP_EWALD, (float)alpha, 0.f};
    launch_field(pos4, positions, charges, nullptr, nullptr, n, 1, g, ec, 0.f, 1.f, true, t, nullptr, phi, acc12,
                 nullptr, acc, st);
    launch_finalize_atoms(acc12, n, forces, nullptr, phi, nullptr, st);
    if (energy_virial &&
        (e = cudaMemcpyAsync(energy_virial, &acc->e_kspace, sizeof(double) * 10, cudaMemcpyDeviceToDevice, st)))
        return cuda_fail(e);
    if ((e = cudaGetLastError())) return cuda_fail(e);
    return QNEP_OK;
}
