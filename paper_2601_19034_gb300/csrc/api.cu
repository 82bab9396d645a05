// C ABI of the qNEP force call: model lifetime, workspaces, k-tables and the
// launch sequence of one force call (see include/qnep.h for the contract).
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cufft.h>

#include "../../include/qnep.h"
#include "qnep_internal.cuh"
#include "kset_host.h"
#include "tma.cuh"

using namespace qnep;

struct qnep_model {
    qnep_hparams hp{};
    qnep_elec es{};
    int precision = 0;
    int num_sms = 152;
    int n_cand = 1;
    ParamLayout lay{};
    float* d_params = nullptr;
    float sqrt_eps = 1.f;
    int cap_list = 0, cap_ang = 0;          // 0: automatic from the density
    int path = QNEP_PATH_AUTO;
    // per-atom workspaces (grow only)
    int n_alloc = 0, cl_alloc = 0, ca_alloc = 0, nph_alloc = 0;
    float4* pos4 = nullptr;        // wrapped positions, input order
    float4* spos4 = nullptr;       // wrapped positions sorted by cell (working order)
    int* sidx = nullptr;           // input index of each sorted slot
    int* cell_of = nullptr;
    int* cell_atoms = nullptr;
    int* nbr_list = nullptr;
    int* cnt_list = nullptr;
    int* nbr_ang = nullptr;
    int* cnt_ang = nullptr;
    float* ang = nullptr;
    float* du = nullptr;
    float* dq = nullptr;
    float* u = nullptr;
    float* q = nullptr;
    float* dtc = nullptr;          // scaled descriptors [n][32] handed to the tensor-core network
    // velocity-Verlet state: step counter, FP64 kinetic-energy accumulator, block counter,
    // and the force call's scalars
    int* md_step = nullptr;
    double* md_ke = nullptr;
    unsigned int* md_done = nullptr;
    double* md_scalars = nullptr;
    float4* fields = nullptr;      // kfield [n] | rfield [n] | acc12 [3n] (see desc_math.cuh)
    float2* phase = nullptr;
    // cells
    int ncell_alloc = 0;
    int* cell_count = nullptr;
    int* cell_start = nullptr;
    int* cell_fill = nullptr;
    Accum* d_acc = nullptr;
    unsigned int* h_status = nullptr;       // mapped pinned word written by the last kernel
    unsigned int* d_status = nullptr;       // its device alias
    unsigned int* fin_done = nullptr;       // last-block counter of the finalize kernel
    unsigned int* sk_done = nullptr;        // last-block counters of the structure-factor kernel
    int sk_done_alloc = 0;
    // geometry / Ewald tables, rebuilt when the box changes
    bool have_box = false;
    double box[9]{};
    double width[3]{};              // perpendicular widths of the cell (the edges of an orthorhombic box)
    Geom geom{};
    EwaldTab tab{};
    int nk_alloc = 0, ncol_alloc = 0, nchunk_alloc = 0;
    int4* d_col = nullptr;
    int* d_chunk_col = nullptr;
    int* d_chunk_order = nullptr;
    float* d_kg = nullptr;
    double2* d_S = nullptr;
    float2* d_C = nullptr;
    float4* d_kb = nullptr;        // B(k) per padded wave vector (per-atom virial), 2 float4 each
    // per-atom virial scratch [n][AVIR] (allocated on the first request) and the PPPM extras
    float* avir = nullptr;
    int avir_alloc = 0;
    float2* pm_fhat6 = nullptr;
    float* pm_field6 = nullptr;
    cufftHandle c2r6 = 0;
    bool have_c2r6 = false;
    // PPPM meshes and FFT plans (created with the first box)
    PppmTab pm{};
    cufftHandle r2c = 0, c2r = 0;
    bool have_mesh = false;
    // device staging of the host-buffer entry point
    int nio_alloc = 0;
    float* io_pos = nullptr;
    int* io_types = nullptr;
    float* io_out[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double* io_scalars = nullptr;
    // Verlet skin (warp-per-atom path): candidate lists [n][skin_cap] with cutoff r_list + skin,
    // reused while no atom has moved more than skin / 2 (decided on the device)
    float skin = 0.f;
    bool skin_valid = false;               // a list built for this (n, box) exists
    int skin_n = 0, skin_cap = 0, skin_n_alloc = 0, skin_cap_alloc = 0;
    double skin_box[9]{};
    int* skin_gate = nullptr;
    unsigned int* skin_rebuilds = nullptr;
    int* skin_list = nullptr;
    int* skin_cnt = nullptr;
    float4* skin_sref4 = nullptr;
    float* skin_xref = nullptr;
    // second stream for the real-space kernel (runs beside the structure factor)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // stage timers
    bool profiling = false;
    cudaEvent_t ev_start[QNEP_NSTAGES]{}, ev_end[QNEP_NSTAGES]{};
    bool recorded[QNEP_NSTAGES]{};
    double stage_ms[QNEP_NSTAGES]{};
    int timed_calls = 0;
    bool pending = false;
    std::string err;
};

namespace {

qnep_status fail(qnep_model* m, qnep_status s, const std::string& msg) {
    if (m) m->err = msg;
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(m, e_ == cudaErrorMemoryAllocation ? QNEP_ERR_OOM : QNEP_ERR_CUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

template <class T>
cudaError_t grow(T** p, size_t count) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

bool supported_shape(const qnep_hparams* hp) {
    return hp->n_radial == NR && hp->n_angular == NA && hp->basis_radial == KR && hp->basis_angular == KA &&
           hp->l_max == LMAX && hp->use_4body == 1 && hp->n_neurons == NNEU && hp->n_species >= 1 &&
           hp->n_species <= MAX_SPECIES;
}

float list_cutoff(const qnep_model* m) {
    float rc = m->hp.rc_radial;
    if (m->es.mode == 1 && (float)m->es.rc_real > rc) rc = (float)m->es.rc_real;
    return rc;
}

// Half-space Ewald k-set in columns (n1, n2) with runs of n3, chunks of 8.
qnep_status build_ewald_table(qnep_model* m, const double L[3], const double* box, bool tri) {
    KSet ks = tri ? build_kset_box(box, m->es.kmax, m->es.alpha) : build_kset(L, m->es.kmax, m->es.alpha);
    double hinv[9];
    invert3(box, hinv);
    const int* nmax = ks.nmax;
    const std::vector<int4>& cols = ks.cols;
    const std::vector<int>& chunk_col = ks.chunk_col;
    const std::vector<float>& kg = ks.kg;
    const double alpha = m->es.alpha;
    int ncol = (int)cols.size() - 1, nk = (int)kg.size(), nch = (int)chunk_col.size();
    if (ncol + 1 > m->ncol_alloc) {
        CK(grow(&m->d_col, ncol + 1));
        m->ncol_alloc = ncol + 1;
    }
    if (nch > m->nchunk_alloc) {
        CK(grow(&m->d_chunk_col, nch));
        CK(grow(&m->d_chunk_order, nch));
        m->nchunk_alloc = nch;
    }
    // processing order of the chunks: by the n3 window they cover (stable), so the
    // lanes of a warp in the structure-factor kernel mostly read the same Z factors
    std::vector<int> order(nch);
    for (int gi = 0; gi < nch; ++gi) order[gi] = gi;
    auto zstart = [&](int gi) {
        const int4& c = cols[chunk_col[gi]];
        return c.z + (8 * gi - c.w);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return zstart(a) < zstart(b); });
    if (nch) CK(cudaMemcpy(m->d_chunk_order, order.data(), sizeof(int) * nch, cudaMemcpyHostToDevice));
    if (nk > m->nk_alloc) {
        CK(grow(&m->d_kg, nk));
        CK(grow(&m->d_S, nk));
        CK(grow(&m->d_C, nk));
        CK(grow(&m->d_kb, 2 * (size_t)nk));
        m->nk_alloc = nk;
    }
    {
        // B(k) = I - (2 / (4 alpha^2) + 2 / k^2) k k^T of every padded wave vector (zero on padding)
        std::vector<float4> kb(2 * (size_t)std::max(nk, 1), make_float4(0.f, 0.f, 0.f, 0.f));
        const double tp = 6.283185307179586;
        for (int gi = 0; gi < nch; ++gi) {
            const int4& c = cols[chunk_col[gi]];
            for (int t = 0; t < 8; ++t) {
                const int k = 8 * gi + t;
                if (!(kg[k] > 0.f)) continue;
                const int n3 = c.z + (k - c.w);
                double kx = tp * c.x / L[0], ky = tp * c.y / L[1], kz = tp * n3 / L[2];
                if (tri) {
                    kx = tp * (hinv[0] * c.x + hinv[1] * c.y + hinv[2] * n3);
                    ky = tp * (hinv[3] * c.x + hinv[4] * c.y + hinv[5] * n3);
                    kz = tp * (hinv[6] * c.x + hinv[7] * c.y + hinv[8] * n3);
                }
                const double fac = 2.0 / (4.0 * m->es.alpha * m->es.alpha) + 2.0 / (kx * kx + ky * ky + kz * kz);
                kb[2 * k] = make_float4((float)(1.0 - fac * kx * kx), (float)(1.0 - fac * ky * ky),
                                        (float)(1.0 - fac * kz * kz), (float)(-fac * kx * ky));
                kb[2 * k + 1] = make_float4((float)(-fac * kx * kz), (float)(-fac * ky * kz), 0.f, 0.f);
            }
        }
        if (nk) CK(cudaMemcpy(m->d_kb, kb.data(), sizeof(float4) * 2 * (size_t)nk, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(m->d_col, cols.data(), sizeof(int4) * cols.size(), cudaMemcpyHostToDevice));
    if (nch) CK(cudaMemcpy(m->d_chunk_col, chunk_col.data(), sizeof(int) * nch, cudaMemcpyHostToDevice));
    if (nk) CK(cudaMemcpy(m->d_kg, kg.data(), sizeof(float) * nk, cudaMemcpyHostToDevice));
    EwaldTab& t = m->tab;
    t.n1max = nmax[0];
    t.n2max = nmax[1];
    t.n3max = nmax[2];
    t.ncol = ncol;
    t.nchunk = nch;
    t.nk = nk;
    t.yoff = nmax[0] + 1;
    t.zoff = t.yoff + 2 * nmax[1] + 1;
    t.nph = t.zoff + 2 * nmax[2] + 8;
    if ((t.nph & 1) == 0) t.nph += 1;   // odd row stride: conflict-free strided shared-memory reads
    for (int d = 0; d < 3; ++d) {
        t.L[d] = (float)L[d];
        double il = 1.0 / L[d];
        t.invl_hi[d] = (float)il;
        t.invl_lo[d] = (float)(il - (double)t.invl_hi[d]);
    }
    t.tri = tri ? 1 : 0;
    for (int k = 0; k < 9; ++k) {
        t.hi_hi[k] = (float)hinv[k];
        t.hi_lo[k] = (float)(hinv[k] - (double)t.hi_hi[k]);
        t.krec[k] = (float)(6.283185307179586 * hinv[k]);
    }
    t.alpha = (float)alpha;
    t.col = m->d_col;
    t.chunk_col = m->d_chunk_col;
    t.chunk_order = m->d_chunk_order;
    t.kg = m->d_kg;
    t.S = m->d_S;
    t.C = m->d_C;
    t.kb = m->d_kb;
    return QNEP_OK;
}

// PPPM meshes, cuFFT plans (once) and the influence function (every new box).
qnep_status setup_pppm(qnep_model* m, const double L[3], const double box[9], bool tri, cudaStream_t st) {
    PppmTab& pm = m->pm;
    if (!m->have_mesh) {
        pm.nx = m->es.mesh[0];
        pm.ny = m->es.mesh[1];
        pm.nz = m->es.mesh[2];
        pm.nreal = (size_t)pm.nx * pm.ny * pm.nz;
        pm.nhalf = (size_t)pm.nx * pm.ny * (pm.nz / 2 + 1);
        if (pm.nreal >= ((size_t)1 << 31)) return fail(m, QNEP_ERR_ARG, "PPPM mesh above 2^31 points");
        CK(cudaMalloc((void**)&pm.rho, sizeof(float) * pm.nreal));
        CK(cudaMemset(pm.rho, 0, sizeof(float) * pm.nreal));
        CK(cudaMalloc((void**)&pm.shat, sizeof(float2) * pm.nhalf));
        CK(cudaMalloc((void**)&pm.fhat, sizeof(float2) * 4 * pm.nhalf));
        CK(cudaMalloc((void**)&pm.field, sizeof(float) * 4 * pm.nreal));
        CK(cudaMalloc((void**)&pm.gopt, sizeof(float) * pm.nhalf));
        if (cufftPlan3d(&m->r2c, pm.nx, pm.ny, pm.nz, CUFFT_R2C) != CUFFT_SUCCESS)
            return fail(m, QNEP_ERR_CUDA, "cufftPlan3d (R2C) failed");
        int dims[3] = {pm.nx, pm.ny, pm.nz};
        if (cufftPlanMany(&m->c2r, 3, dims, nullptr, 1, (int)pm.nhalf, nullptr, 1, (int)pm.nreal, CUFFT_C2R, 4) !=
            CUFFT_SUCCESS)
            return fail(m, QNEP_ERR_CUDA, "cufftPlanMany (C2R x 4) failed");
        m->have_mesh = true;
    }
    for (int d = 0; d < 3; ++d) {
        pm.len[d] = (float)L[d];
        const int nd = d == 0 ? pm.nx : (d == 1 ? pm.ny : pm.nz);
        pm.inv_h[d] = (float)(nd / L[d]);
        pm.inv_h_lo[d] = (float)(nd / L[d] - (double)pm.inv_h[d]);
    }
    // general cells: mesh along the lattice vectors (mesh coordinates N_d (r H^-1)_d), k = 2 pi H^-1 n
    double hinv[9];
    const double det = invert3(box, hinv);
    pm.tri = tri ? 1 : 0;
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
            const int nd = d == 0 ? pm.nx : (d == 1 ? pm.ny : pm.nz);
            const double v = nd * hinv[3 * c + d];
            pm.nh_hi[3 * c + d] = (float)v;
            pm.nh_lo[3 * c + d] = (float)(v - (double)pm.nh_hi[3 * c + d]);
        }
    for (int k = 0; k < 9; ++k) {
        pm.hi[k] = (float)hinv[k];
        pm.hid[k] = hinv[k];
    }
    launch_pppm_gopt(pm, m->es.alpha, tri ? std::fabs(det) : L[0] * L[1] * L[2], st);
    CK(cudaStreamSynchronize(st));
    return QNEP_OK;
}

qnep_status prepare(qnep_model* m, int n, const double* box, cudaStream_t st) {
    if (!box) return fail(m, QNEP_ERR_ARG, "box is NULL");
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(box[k])) return fail(m, QNEP_ERR_ARG, "box has a non-finite entry");
    const bool tri = box[1] != 0 || box[2] != 0 || box[3] != 0 || box[5] != 0 || box[6] != 0 || box[7] != 0;
    // edge lengths and the perpendicular widths V / |a_e x a_f| (the cell grid needs width >= cutoff)
    double L[3], width[3], hinv[9];
    const double det = invert3(box, hinv);
    for (int d = 0; d < 3; ++d) {
        const double* a = box + 3 * d;
        L[d] = tri ? std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) : box[4 * d];
        const double* e = box + 3 * ((d + 1) % 3);
        const double* f = box + 3 * ((d + 2) % 3);
        const double cx = e[1] * f[2] - e[2] * f[1], cy = e[2] * f[0] - e[0] * f[2], cz = e[0] * f[1] - e[1] * f[0];
        width[d] = tri ? det / std::sqrt(cx * cx + cy * cy + cz * cz) : L[d];
    }
    if (tri && !(det > 0)) return fail(m, QNEP_ERR_ARG, "the cell vectors must be independent and right-handed");
    const float rcl = list_cutoff(m);
    for (int d = 0; d < 3; ++d) {
        if (!(L[d] > 0)) return fail(m, QNEP_ERR_ARG, "box edge must be positive");
        if (width[d] < rcl) return fail(m, QNEP_ERR_UNSUPPORTED, "cell width shorter than the list cutoff");
    }
    // the Ewald phase-factor count (rounded up to odd) is known from n_max alone: refuse before
    // enumerating the k-set and before any state of the previous box is touched
    if (m->es.mode != 0 && m->es.kind == QNEP_EWALD && kset_phase_count(L, m->es.kmax) > EWALD_MAX_NPH)
        return fail(m, QNEP_ERR_UNSUPPORTED, "k_max * box edge too large for the Ewald phase tables");
    bool box_changed = !m->have_box || std::memcmp(m->box, box, sizeof(double) * 9) != 0;
    if (box_changed) {
        if (m->have_box) CK(cudaStreamSynchronize(st));   // in-flight kernels may read the old tables
        m->have_box = false;   // until every table of the new box is built (a failure below rebuilds next call)
        Geom& g = m->geom;
        g.ncells = 1;
        g.tri = tri ? 1 : 0;
        for (int k = 0; k < 9; ++k) {
            g.H[k] = (float)box[k];
            g.Hi[k] = (float)hinv[k];
        }
        for (int d = 0; d < 3; ++d) {
            g.L[d] = (float)L[d];
            g.invL[d] = (float)(1.0 / L[d]);
            m->width[d] = width[d];
            int nc = (int)std::floor(width[d] / rcl);
            g.nc[d] = nc < 1 ? 1 : nc;
            g.ncells *= g.nc[d];
        }
        g.rc_list = rcl;
        g.rc_radial = m->hp.rc_radial;
        g.rc_angular = m->hp.rc_angular;
        g.rc_real = m->es.mode == 1 ? (float)m->es.rc_real : 0.f;
        if (g.ncells + 1 > m->ncell_alloc) {
            CK(grow(&m->cell_count, g.ncells + 1));
            CK(grow(&m->cell_start, g.ncells + 1));
            CK(grow(&m->cell_fill, g.ncells + 1));
            CK(cudaMemset(m->cell_count, 0, sizeof(int) * (g.ncells + 1)));
            m->ncell_alloc = g.ncells + 1;
        }
        if (m->es.mode != 0 && m->es.kind == QNEP_EWALD) {
            qnep_status s;
            try {
                s = build_ewald_table(m, L, box, tri);
            } catch (const std::bad_alloc&) {   // host tables: no exception crosses the C ABI
                s = fail(m, QNEP_ERR_OOM, "host memory for the k-set could not be obtained");
            }
            if (s != QNEP_OK) return s;
            int groups = (m->tab.nchunk + 31) / 32 + 1;
            if (groups > m->sk_done_alloc) {
                CK(grow(&m->sk_done, groups));
                CK(cudaMemset(m->sk_done, 0, sizeof(unsigned int) * groups));
                m->sk_done_alloc = groups;
            }
        }
        if (m->es.mode != 0 && m->es.kind == QNEP_PPPM) {
            qnep_status s = setup_pppm(m, L, box, tri, st);
            if (s != QNEP_OK) return s;
        }
        std::memcpy(m->box, box, sizeof(double) * 9);
        m->have_box = true;
    }
    // neighbour capacities from the mean density (2x the mean count + margin)
    const double vol = tri ? std::fabs(det) : L[0] * L[1] * L[2];
    const double dens = n / vol;
    const double pi43 = 4.18879020478639;
    int cl = m->cap_list, ca = m->cap_ang;
    if (cl <= 0) cl = ((int)(2.0 * pi43 * rcl * rcl * rcl * dens) + 32 + 31) / 32 * 32;
    if (ca <= 0) {
        double ra = m->hp.rc_angular;
        ca = ((int)(2.0 * pi43 * ra * ra * ra * dens) + 16 + 15) / 16 * 16;
    }
    int nph = (m->es.mode != 0 && m->es.kind == QNEP_EWALD) ? m->tab.nph : 0;
    bool need_atoms = n > m->n_alloc;
    if (need_atoms || cl > m->cl_alloc || ca > m->ca_alloc || nph > m->nph_alloc) {
        int na = std::max(n, m->n_alloc);
        int ncl = std::max(cl, m->cl_alloc), nca = std::max(ca, m->ca_alloc), nnph = std::max(nph, m->nph_alloc);
        CK(cudaStreamSynchronize(st));
        CK(grow(&m->nbr_list, (size_t)ncl * na));
        CK(grow(&m->nbr_ang, (size_t)nca * na));
        if (need_atoms) {
            CK(grow(&m->pos4, na));
            CK(grow(&m->spos4, na));
            CK(grow(&m->sidx, na));
            CK(grow(&m->cell_of, na));
            CK(grow(&m->cell_atoms, na));
            CK(grow(&m->cnt_list, (size_t)MAX_SPECIES * na));
            CK(grow(&m->cnt_ang, (size_t)MAX_SPECIES * na));
            CK(grow(&m->ang, (size_t)NANG * na));
            CK(grow(&m->du, (size_t)NDES * na));
            CK(grow(&m->dq, (size_t)NDES * na));
            CK(grow(&m->u, na));
            CK(grow(&m->q, na));
            if (m->precision != QNEP_PREC_FP32) CK(grow(&m->dtc, (size_t)32 * na));
            CK(grow(&m->fields, (size_t)5 * na));
        }
        // +2 entries: bulk copies round the last tile up to 16 bytes
        if (need_atoms || nnph > m->nph_alloc) CK(grow(&m->phase, (size_t)std::max(nnph, 1) * na + 2));
        m->n_alloc = na;
        m->cl_alloc = ncl;
        m->ca_alloc = nca;
        m->nph_alloc = nnph;
    }
    m->tab.phase = m->phase;
    return QNEP_OK;
}

const char* kStageNames[QNEP_NSTAGES] = {"cell_bin", "neighbors", "descriptor_forward", "ewald_phases",
                                         "ewald_structure_factor", "field_kspace", "real_space",
                                         "descriptor_backward", "finalize", "pppm"};

// The warp-per-atom kernels (descriptor_coop.cu) are the default at every size: measured on
// a GB300 they are faster from 40 atoms to 1.0 M atoms (1 M-atom Mg-water, PPPM: 14.0 ms per
// force call against 15.4 ms for the thread-per-atom kernels).
constexpr int kCoopMaxAtoms = 1 << 30;

// Accumulate the event times of the previous profiled call (its events are
// complete once the stream has been synchronized).
void harvest(qnep_model* m) {
    if (!m->pending) return;
    for (int k = 0; k < QNEP_NSTAGES; ++k) {
        float ms = 0.f;
        if (m->recorded[k] && cudaEventElapsedTime(&ms, m->ev_start[k], m->ev_end[k]) == cudaSuccess)
            m->stage_ms[k] += ms;
        m->recorded[k] = false;
    }
    m->timed_calls += 1;
    m->pending = false;
}

struct StageTimer {
    qnep_model* m;
    void begin(int k, cudaStream_t s) const {
        if (m->profiling) cudaEventRecord(m->ev_start[k], s);
    }
    void end(int k, cudaStream_t s) const {
        if (m->profiling) {
            cudaEventRecord(m->ev_end[k], s);
            m->recorded[k] = true;
        }
    }
};

// Device state of a new model: parameters, accumulators, the mapped status word, the second stream
// and its events.  On failure the caller destroys the model (every handle not yet made is null).
qnep_status init_model(qnep_model* m, const float* params_host, size_t n_params) {
    CK(cudaMalloc((void**)&m->d_params, sizeof(float) * n_params));
    CK(cudaMemcpy(m->d_params, params_host, sizeof(float) * n_params, cudaMemcpyHostToDevice));
    CK(cudaMalloc((void**)&m->d_acc, sizeof(Accum)));
    CK(cudaMemset(m->d_acc, 0, sizeof(Accum)));
    CK(cudaHostAlloc((void**)&m->h_status, sizeof(unsigned int), cudaHostAllocMapped));
    *m->h_status = 0;
    CK(cudaHostGetDevicePointer((void**)&m->d_status, m->h_status, 0));
    CK(cudaMalloc((void**)&m->fin_done, sizeof(unsigned int)));
    CK(cudaMemset(m->fin_done, 0, sizeof(unsigned int)));
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            m->num_sms = sms;
    }
    CK(cudaStreamCreateWithFlags(&m->aux, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming));
    return QNEP_OK;
}

}  // namespace

extern "C" {

const char* qnep_stage_name(int stage) { return (stage >= 0 && stage < QNEP_NSTAGES) ? kStageNames[stage] : ""; }

qnep_status qnep_set_profiling(qnep_model* m, int enable) {
    if (!m) return QNEP_ERR_ARG;
    if (enable && !m->ev_start[0]) {
        for (int k = 0; k < QNEP_NSTAGES; ++k) {
            CK(cudaEventCreate(&m->ev_start[k]));
            CK(cudaEventCreate(&m->ev_end[k]));
        }
    }
    m->profiling = enable != 0;
    return QNEP_OK;
}

qnep_status qnep_stage_times(qnep_model* m, float* ms_out, int max_stages, int* n_calls) {
    if (!m) return QNEP_ERR_ARG;
    CK(cudaDeviceSynchronize());
    harvest(m);
    for (int k = 0; k < max_stages && k < QNEP_NSTAGES; ++k) ms_out[k] = (float)m->stage_ms[k];
    if (n_calls) *n_calls = m->timed_calls;
    for (int k = 0; k < QNEP_NSTAGES; ++k) m->stage_ms[k] = 0.0;
    m->timed_calls = 0;
    return QNEP_OK;
}

size_t qnep_param_count(const qnep_hparams* hp) {
    if (!hp) return 0;
    int s = hp->n_species;
    int ndes = hp->n_radial + hp->n_angular * hp->l_max + (hp->use_4body ? hp->n_angular : 0);
    return (size_t)s * s * (hp->n_radial * hp->basis_radial + hp->n_angular * hp->basis_angular) + ndes +
           (size_t)s * (hp->n_neurons * (ndes + 3) + 2) + 1;
}

const char* qnep_status_string(qnep_status s) {
    switch (s) {
        case QNEP_OK: return "ok";
        case QNEP_ERR_ARG: return "invalid argument";
        case QNEP_ERR_CUDA: return "CUDA error";
        case QNEP_ERR_NBR_OVERFLOW: return "neighbour list overflow";
        case QNEP_ERR_UNSUPPORTED: return "unsupported";
        case QNEP_ERR_TIMEOUT: return "device wait timed out";
        case QNEP_ERR_OOM: return "out of device memory";
    }
    return "unknown status";
}

const char* qnep_last_error(qnep_model* m) { return m ? m->err.c_str() : ""; }

qnep_status qnep_create(qnep_model** out, const qnep_hparams* hp, const float* params_host, size_t n_params,
                        int n_candidates, const qnep_elec* es, int precision) {
    qnep_model* m = nullptr;
    if (!out || !hp || !params_host || !es || n_candidates < 1) return QNEP_ERR_ARG;
    *out = nullptr;
    if (!supported_shape(hp)) return QNEP_ERR_UNSUPPORTED;
    if (!(hp->rc_radial > 0) || !(hp->rc_angular > 0) || hp->rc_angular > hp->rc_radial) return QNEP_ERR_ARG;
    size_t per = qnep_param_count(hp);
    if (n_params != per * (size_t)n_candidates) return QNEP_ERR_ARG;
    if (es->mode < 0 || es->mode > 2) return QNEP_ERR_ARG;
    if (es->mode != 0) {
        if (!(es->alpha > 0) || !std::isfinite(es->alpha)) return QNEP_ERR_ARG;
        if (es->kind != QNEP_EWALD && es->kind != QNEP_PPPM) return QNEP_ERR_ARG;
        if (es->kind == QNEP_EWALD && (!(es->kmax > 0) || !std::isfinite(es->kmax))) return QNEP_ERR_ARG;
        if (es->kind == QNEP_PPPM) {
            if (es->order != 5) return QNEP_ERR_UNSUPPORTED;
            for (int d = 0; d < 3; ++d)
                if (es->mesh[d] < 4 || (es->mesh[d] & 1)) return QNEP_ERR_ARG;
        }
        if (es->mode == 1 && (!(es->rc_real > 0) || es->rc_real > hp->rc_radial)) return QNEP_ERR_UNSUPPORTED;
    }
    if (precision != QNEP_PREC_FP32 && precision != QNEP_PREC_MLP_BF16 && precision != QNEP_PREC_MLP_TF32)
        return QNEP_ERR_ARG;
    for (size_t k = 0; k < n_params; ++k)
        if (!std::isfinite(params_host[k])) return QNEP_ERR_ARG;
    try {   // host memory: no exception crosses the C ABI
        m = new qnep_model();
    } catch (const std::bad_alloc&) {
        return QNEP_ERR_OOM;
    }
    m->hp = *hp;
    m->es = *es;
    m->precision = precision;
    m->n_cand = n_candidates;
    m->lay = make_layout(hp->n_species);
    m->sqrt_eps = params_host[m->lay.sqrt_eps];
    const qnep_status s = init_model(m, params_host, n_params);
    if (s != QNEP_OK) {   // nothing of a half-built model outlives the failed call
        qnep_destroy(m);
        return s;
    }
    *out = m;
    return QNEP_OK;
}

qnep_status qnep_set_path(qnep_model* m, int path) {
    if (!m || path < QNEP_PATH_AUTO || path > QNEP_PATH_THREAD) return QNEP_ERR_ARG;
    m->path = path;
    return QNEP_OK;
}

qnep_status qnep_set_capacity(qnep_model* m, int cap_list, int cap_angular) {
    if (!m || cap_list < 0 || cap_angular < 0) return QNEP_ERR_ARG;
    if (cap_list) m->cap_list = cap_list;
    if (cap_angular) m->cap_ang = cap_angular;
    m->skin_valid = false;   // the skin lists are sized from the list capacity
    return QNEP_OK;
}

qnep_status qnep_set_skin(qnep_model* m, double skin) {
    if (!m || !(skin >= 0) || !std::isfinite(skin) || skin > 5.0) return QNEP_ERR_ARG;
    m->skin = (float)skin;
    m->skin_valid = false;
    return QNEP_OK;
}

qnep_status qnep_skin_rebuilds(qnep_model* m, unsigned int* count) {
    if (!m || !count) return QNEP_ERR_ARG;
    *count = 0;
    if (!m->skin_rebuilds) return QNEP_OK;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(count, m->skin_rebuilds, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    return QNEP_OK;
}

qnep_status qnep_reserve(qnep_model* m, int n_atoms, const double box[9]) {
    if (!m || n_atoms < 0) return QNEP_ERR_ARG;
    qnep_status s = prepare(m, n_atoms, box, 0);
    if (s != QNEP_OK) return s;
    CK(cudaDeviceSynchronize());
    return QNEP_OK;
}

}  // extern "C"

namespace {

// One force call; with a vector-Jacobian product request the backward runs with
// the weighted adjoints and the gradient replaces the force output.
qnep_status compute_impl(qnep_model* m, int n, const float* positions, const int* types, const double box[9],
                         void* stream, const qnep_outputs* out, const qnep_vjp* vjp) {
    if (!m) return QNEP_ERR_ARG;
    if (n < 1 || n > INDEX_MASK) return fail(m, QNEP_ERR_ARG, "atom count out of range");
    if (!positions || !types || !out) return fail(m, QNEP_ERR_ARG, "NULL input or output struct");
    cudaStream_t st = (cudaStream_t)stream;
    qnep_status s = prepare(m, n, box, st);
    if (s != QNEP_OK) return s;
    const bool ewald = m->es.mode != 0 && m->es.kind == QNEP_EWALD;
    const bool pppm = m->es.mode != 0 && m->es.kind == QNEP_PPPM;
    const bool gp_nonzero = vjp && (vjp->polar_weight[0] != 0 || vjp->polar_weight[1] != 0 || vjp->polar_weight[2] != 0);
    const bool backward = out->forces || out->bec || out->want_virial || vjp || out->atom_virial;
    const bool want_bec = out->bec != nullptr || gp_nonzero;
    if (vjp && m->precision != QNEP_PREC_FP32)
        return fail(m, QNEP_ERR_UNSUPPORTED, "the vector-Jacobian product runs on the FP32 path only");
    const float q_target = (float)(m->es.q_total / (double)m->sqrt_eps);   // Q in screened-charge units
    const int cl = m->cap_list > 0 ? m->cap_list : m->cl_alloc;
    const int ca = m->cap_ang > 0 ? m->cap_ang : m->ca_alloc;
    ElecConst ec{m->es.mode, m->es.kind, (float)m->es.alpha, (float)m->es.q_total};

    if (m->profiling) {
        CK(cudaDeviceSynchronize());   // the previous call's events (both streams) are complete
        harvest(m);
    }
    Geom g = m->geom;
    const bool mixed = m->precision != QNEP_PREC_FP32;
    const bool coop = m->path == QNEP_PATH_WARP || (m->path == QNEP_PATH_AUTO && n <= kCoopMaxAtoms);
    float* avir = nullptr;
    if (out->atom_virial) {
        if (!coop || vjp)
            return fail(m, QNEP_ERR_UNSUPPORTED,
                        "the per-atom virial runs with the warp-per-atom kernels and without a vector-Jacobian product");
        if (n > m->avir_alloc) {
            CK(cudaStreamSynchronize(st));
            CK(grow(&m->avir, (size_t)AVIR * n));
            m->avir_alloc = n;
        }
        if (pppm && !m->pm_fhat6) {
            CK(cudaStreamSynchronize(st));
            CK(cudaMalloc((void**)&m->pm_fhat6, sizeof(float2) * 6 * m->pm.nhalf));
            CK(cudaMalloc((void**)&m->pm_field6, sizeof(float) * 6 * m->pm.nreal));
            int dims[3] = {m->pm.nx, m->pm.ny, m->pm.nz};
            if (cufftPlanMany(&m->c2r6, 3, dims, nullptr, 1, (int)m->pm.nhalf, nullptr, 1, (int)m->pm.nreal, CUFFT_C2R,
                              6) != CUFFT_SUCCESS)
                return fail(m, QNEP_ERR_CUDA, "cufftPlanMany (C2R x 6) failed");
            m->have_c2r6 = true;
        }
        avir = m->avir;
        CK(cudaMemsetAsync(avir, 0, sizeof(float) * AVIR * (size_t)n, st));
    }
    if (coop) {   // atom-major lists for the warp-per-atom kernels
        g.list_sa = cl;
        g.list_se = 1;
        g.ang_sa = ca;
        g.ang_se = 1;
    } else {      // entry-major lists for the thread-per-atom kernels
        g.list_sa = 1;
        g.list_se = n;
        g.ang_sa = 1;
        g.ang_se = n;
    }
    const FieldIn fin{m->fields, m->fields + n, m->es.mode, (float)m->es.alpha, q_target,
                      vjp ? (float)vjp->energy_weight : 1.f, vjp ? vjp->charge_weight : nullptr, m->sidx};
    float* acc12 = reinterpret_cast<float*>(m->fields + 2 * (size_t)n);
    float4* kfield = m->fields;
    float4* rfield = m->fields + n;
    StageTimer tm{m};
    tm.begin(0, st);
    // the structure-factor sums (Ewald) or the charge mesh (PPPM) start from zero
    double2* zbuf = ewald ? m->tab.S : (pppm ? reinterpret_cast<double2*>(m->pm.rho) : nullptr);
    const int zcount = ewald ? m->tab.nk : (pppm ? (int)(m->pm.nreal / 4) : 0);
    const bool use_skin = m->skin > 0.f && coop;
    if (use_skin) {
        // candidate capacity: the list capacity scaled by the volume of the longer cutoff
        const float rcl = g.rc_list, rs = rcl + m->skin;
        const int cap_s = ((int)((double)cl * (rs * rs * rs) / (rcl * rcl * rcl)) + 31) / 32 * 32;
        if (!m->skin_gate) {
            CK(cudaMalloc((void**)&m->skin_gate, sizeof(int)));
            CK(cudaMalloc((void**)&m->skin_rebuilds, sizeof(unsigned int)));
            CK(cudaMemset(m->skin_rebuilds, 0, sizeof(unsigned int)));
        }
        if (n > m->skin_n_alloc || cap_s > m->skin_cap_alloc) {
            const int na = std::max(n, m->skin_n_alloc), nc = std::max(cap_s, m->skin_cap_alloc);
            CK(cudaStreamSynchronize(st));
            CK(grow(&m->skin_list, (size_t)na * nc));
            CK(grow(&m->skin_cnt, (size_t)na));
            CK(grow(&m->skin_sref4, (size_t)na));
            CK(grow(&m->skin_xref, (size_t)3 * na));
            m->skin_n_alloc = na;
            m->skin_cap_alloc = nc;
            m->skin_valid = false;
        }
        const bool force = !m->skin_valid || m->skin_n != n || m->skin_cap != cap_s ||
                           std::memcmp(m->skin_box, box, sizeof(double) * 9) != 0;
        // cells no smaller than r_list + skin, so the 27-cell search reaches every candidate
        Geom gk = g;
        gk.ncells = 1;
        for (int d = 0; d < 3; ++d) {
            if (m->width[d] < rs) return fail(m, QNEP_ERR_UNSUPPORTED, "cell width shorter than the list cutoff plus the skin");
            const int nc = (int)std::floor(m->width[d] / (double)rs);
            gk.nc[d] = nc < 1 ? 1 : nc;
            gk.ncells *= gk.nc[d];
        }
        launch_skin(positions, types, n, gk, m->skin, force, cap_s, m->pos4, m->cell_of, m->cell_count, m->cell_start,
                    m->cell_fill, m->cell_atoms, m->spos4, m->sidx, m->d_acc, zbuf, zcount, m->skin_gate,
                    m->skin_list, m->skin_cnt, m->skin_sref4, m->skin_xref, m->skin_rebuilds, st);
        m->skin_valid = true;
        m->skin_n = n;
        m->skin_cap = cap_s;
        std::memcpy(m->skin_box, box, sizeof(double) * 9);
    } else {
        launch_bin(positions, types, n, g, m->pos4, m->cell_of, m->cell_count, m->cell_start, m->cell_fill,
                   m->cell_atoms, m->spos4, m->sidx, m->d_acc, zbuf, zcount, st);
    }
    tm.end(0, st);
    if (coop) {
        tm.begin(2, st);
        launch_nbr_desc_coop(m->spos4, m->cell_start, m->sidx, n, g, m->d_params, m->lay, cl, ca, m->nbr_list,
                             m->cnt_list, m->nbr_ang, m->cnt_ang, backward ? m->ang : nullptr,
                             backward ? m->du : nullptr, m->dq, m->u, m->q, out->descriptor, m->tab, ewald, m->fields,
                             vjp ? vjp->charge_weight : nullptr, m->d_acc, st, mixed ? m->dtc : nullptr,
                             use_skin ? m->skin_list : nullptr, m->skin_cnt, m->skin_cap);
        if (mixed)
            launch_mlp_tc(m->precision, m->dtc, m->spos4, n, m->d_params, m->lay, backward ? m->du : nullptr, m->dq,
                          NDES, 1, m->u, m->q, m->d_acc, m->num_sms, st);
        tm.end(2, st);
    } else {
        tm.begin(1, st);
        launch_neighbors(m->spos4, m->cell_start, n, m->hp.n_species, g, cl, ca, m->nbr_list, m->cnt_list, m->nbr_ang,
                         m->cnt_ang, m->d_acc, st);
        tm.end(1, st);
        tm.begin(2, st);
        launch_descriptor_forward(m->spos4, m->nbr_list, m->cnt_list, m->nbr_ang, m->cnt_ang, n, g, m->d_params,
                                  m->lay, backward ? m->ang : nullptr, backward ? m->du : nullptr,
                                  backward ? m->dq : nullptr, m->u, m->q, out->descriptor, m->sidx, m->fields,
                                  vjp ? vjp->charge_weight : nullptr, m->d_acc, st, mixed ? m->dtc : nullptr);
        if (mixed)
            launch_mlp_tc(m->precision, m->dtc, m->spos4, n, m->d_params, m->lay, backward ? m->du : nullptr,
                          backward ? m->dq : nullptr, 1, n, m->u, m->q, m->d_acc, m->num_sms, st);
        tm.end(2, st);
        tm.begin(3, st);
        if (ewald) launch_ewald_phases(m->spos4, n, m->tab, st);
        tm.end(3, st);
    }
    const bool real = m->es.mode == 1;
    if (real) {   // real space on the second stream, beside the reciprocal-space kernels
        CK(cudaEventRecord(m->ev_fork, st));
        CK(cudaStreamWaitEvent(m->aux, m->ev_fork, 0));
        tm.begin(6, m->aux);
        launch_real(m->spos4, m->q, m->nbr_list, m->cnt_list, n, m->hp.n_species, g, (float)m->es.alpha, q_target,
                    m->d_acc, rfield, m->d_acc, m->aux, avir);
        tm.end(6, m->aux);
        CK(cudaEventRecord(m->ev_join, m->aux));
    }
    if (ewald) {
        tm.begin(4, st);
        launch_ewald_sk_fused(m->q, m->d_acc, n, q_target, m->tab, m->sk_done, st);
        tm.end(4, st);
        tm.begin(5, st);
        launch_field_k(n, m->tab, kfield, m->d_acc, st, avir);
        tm.end(5, st);
    }
    if (pppm) {
        tm.begin(9, st);
        PppmTab pmc = m->pm;   // the six per-atom virial fields only when they are asked for
        pmc.fhat6 = avir ? m->pm_fhat6 : nullptr;
        pmc.field6 = avir ? m->pm_field6 : nullptr;
        if (launch_pppm(m->spos4, m->q, n, m->d_acc, q_target, pmc, (float)m->es.alpha, m->r2c, m->c2r, kfield,
                        m->d_acc, st, (int)m->c2r6, avir) != 0)
            return fail(m, QNEP_ERR_CUDA, "cuFFT execution failed");
        tm.end(9, st);
    }
    if (real) CK(cudaStreamWaitEvent(st, m->ev_join, 0));
    if (backward) {
        tm.begin(7, st);
        if (coop)
            launch_desc_bwd_coop(m->spos4, m->nbr_list, m->cnt_list, m->nbr_ang, m->cnt_ang, n, g, m->d_params, m->lay,
                                 m->ang, m->du, m->dq, m->q, fin, m->d_acc, want_bec, acc12, m->d_acc, st, avir);
        else
            launch_descriptor_backward(m->spos4, m->nbr_list, m->cnt_list, m->nbr_ang, m->cnt_ang, n, g, m->d_params,
                                       m->lay, m->ang, m->du, m->dq, m->q, fin, m->d_acc, want_bec, acc12, m->d_acc,
                                       st);
        tm.end(7, st);
    }
    tm.begin(8, st);
    float gp[3] = {0.f, 0.f, 0.f};
    if (vjp)
        for (int d = 0; d < 3; ++d) gp[d] = (float)vjp->polar_weight[d];
    launch_finalize(acc12, n, m->sidx, positions, m->q, q_target, m->sqrt_eps, ec, kfield, rfield, out->forces,
                    out->bec, out->charges, out->potential, m->u, out->site_energy, m->d_acc, out->scalars,
                    m->d_status, m->fin_done, st, vjp ? vjp->grad : nullptr, gp, avir, out->atom_virial);
    tm.end(8, st);
    if (m->profiling) m->pending = true;
    CK(cudaGetLastError());
    return QNEP_OK;
}

}  // namespace

extern "C" {

qnep_status qnep_compute(qnep_model* m, int n, const float* positions, const int* types, const double box[9],
                         void* stream, const qnep_outputs* out) {
    return compute_impl(m, n, positions, types, box, stream, out, nullptr);
}

qnep_status qnep_compute_vjp(qnep_model* m, int n, const float* positions, const int* types, const double box[9],
                             void* stream, const qnep_outputs* out, const qnep_vjp* vjp) {
    if (!m) return QNEP_ERR_ARG;
    if (!vjp || !vjp->grad || !out) return fail(m, QNEP_ERR_ARG, "vector-Jacobian product needs vjp->grad");
    if (out->forces) return fail(m, QNEP_ERR_ARG, "forces output must be NULL in a vector-Jacobian product");
    if (!std::isfinite(vjp->energy_weight)) return fail(m, QNEP_ERR_ARG, "non-finite energy weight");
    return compute_impl(m, n, positions, types, box, stream, out, vjp);
}

qnep_status qnep_status_from_device_bits(unsigned int bits) {
    if (bits & 4u) return QNEP_ERR_ARG;
    if (bits & 1u) return QNEP_ERR_NBR_OVERFLOW;
    if (bits & kStatusTimeout) return QNEP_ERR_TIMEOUT;
    return QNEP_OK;
}

qnep_status qnep_sync_status(qnep_model* m, void* stream) {
    if (!m) return QNEP_ERR_ARG;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    const qnep_status s = qnep_status_from_device_bits(*m->h_status);
    if (s == QNEP_ERR_ARG) return fail(m, s, "a species index is outside [0, n_species)");
    if (s == QNEP_ERR_NBR_OVERFLOW) return fail(m, s, "an atom had more neighbours than the list capacity");
    if (s == QNEP_ERR_TIMEOUT)
        return fail(m, s, "a bounded device-side wait gave up (a bulk copy or a tensor-core operation did not complete)");
    return QNEP_OK;
}

qnep_status qnep_debug_set_status(qnep_model* m, unsigned int bits) {
    if (!m) return QNEP_ERR_ARG;
    CK(cudaDeviceSynchronize());
    *m->h_status |= bits;
    return QNEP_OK;
}

qnep_status qnep_compute_host(qnep_model* m, int n, const float* positions_host, const int* types_host,
                              const double box[9], void* stream, const qnep_outputs* out_host) {
    if (!m) return QNEP_ERR_ARG;
    if (n < 1 || !positions_host || !types_host || !out_host) return fail(m, QNEP_ERR_ARG, "bad host arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (n > m->nio_alloc) {
        CK(cudaStreamSynchronize(st));
        CK(grow(&m->io_pos, (size_t)3 * n));
        CK(grow(&m->io_types, n));
        const size_t sizes[6] = {(size_t)3 * n, (size_t)n, (size_t)9 * n, (size_t)n, (size_t)n, (size_t)NDES * n};
        for (int k = 0; k < 6; ++k) CK(grow(&m->io_out[k], sizes[k]));
        if (!m->io_scalars) CK(cudaMalloc((void**)&m->io_scalars, sizeof(double) * QNEP_NSCALARS));
        m->nio_alloc = n;
    }
    CK(cudaMemcpyAsync(m->io_pos, positions_host, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(m->io_types, types_host, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    qnep_outputs dev{};
    dev.scalars = out_host->scalars ? m->io_scalars : nullptr;
    dev.forces = out_host->forces ? m->io_out[0] : nullptr;
    dev.charges = out_host->charges ? m->io_out[1] : nullptr;
    dev.bec = out_host->bec ? m->io_out[2] : nullptr;
    dev.site_energy = out_host->site_energy ? m->io_out[3] : nullptr;
    dev.potential = out_host->potential ? m->io_out[4] : nullptr;
    dev.descriptor = out_host->descriptor ? m->io_out[5] : nullptr;
    dev.want_virial = out_host->want_virial;
    qnep_status s = qnep_compute(m, n, m->io_pos, m->io_types, box, stream, &dev);
    if (s != QNEP_OK) return s;
    if (out_host->scalars)
        CK(cudaMemcpyAsync(out_host->scalars, dev.scalars, sizeof(double) * QNEP_NSCALARS, cudaMemcpyDeviceToHost, st));
    struct { float* h; float* d; size_t cnt; } cp[6] = {
        {out_host->forces, dev.forces, (size_t)3 * n},    {out_host->charges, dev.charges, (size_t)n},
        {out_host->bec, dev.bec, (size_t)9 * n},          {out_host->site_energy, dev.site_energy, (size_t)n},
        {out_host->potential, dev.potential, (size_t)n},  {out_host->descriptor, dev.descriptor, (size_t)NDES * n}};
    for (auto& c : cp)
        if (c.h) CK(cudaMemcpyAsync(c.h, c.d, sizeof(float) * c.cnt, cudaMemcpyDeviceToHost, st));
    return qnep_sync_status(m, stream);
}

qnep_status qnep_nve_run(qnep_model* m, int n, float* positions, float* velocities, const int* types,
                         const double* masses, const double box[9], double dt_fs, int n_steps, void* stream,
                         float* forces, double* energies) {
    if (!m) return QNEP_ERR_ARG;
    if (!positions || !velocities || !types || !masses || !forces || !energies || n_steps < 0 || !(dt_fs > 0))
        return fail(m, QNEP_ERR_ARG, "bad NVE arguments");
    float ms[MAX_SPECIES] = {1.f, 1.f, 1.f, 1.f};
    for (int t = 0; t < m->hp.n_species; ++t) {
        if (!(masses[t] > 0) || !std::isfinite(masses[t])) return fail(m, QNEP_ERR_ARG, "masses must be positive");
        ms[t] = (float)masses[t];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!m->md_step) {
        CK(cudaMalloc((void**)&m->md_step, sizeof(int)));
        CK(cudaMalloc((void**)&m->md_ke, sizeof(double)));
        CK(cudaMalloc((void**)&m->md_done, sizeof(unsigned int)));
        CK(cudaMalloc((void**)&m->md_scalars, sizeof(double) * QNEP_NSCALARS));
    }
    CK(cudaMemsetAsync(m->md_step, 0, sizeof(int), st));
    CK(cudaMemsetAsync(m->md_ke, 0, sizeof(double), st));
    CK(cudaMemsetAsync(m->md_done, 0, sizeof(unsigned int), st));
    CK(cudaMemsetAsync(energies, 0, sizeof(double) * 2 * (size_t)(n_steps + 1), st));
    qnep_outputs o{};
    o.scalars = m->md_scalars;
    o.forces = forces;
    o.want_virial = 0;
    const float dt = (float)dt_fs;
    qnep_status s = compute_impl(m, n, positions, types, box, stream, &o, nullptr);
    if (s != QNEP_OK) return s;
    launch_vv_kick_energy(n, velocities, forces, types, ms, m->hp.n_species, dt, false, m->md_scalars, energies,
                          m->md_step, m->md_ke, m->md_done, st);
    for (int k = 0; k < n_steps; ++k) {
        launch_vv_kick_drift(n, positions, velocities, forces, types, ms, m->hp.n_species, dt, st);
        s = compute_impl(m, n, positions, types, box, stream, &o, nullptr);
        if (s != QNEP_OK) return s;
        launch_vv_kick_energy(n, velocities, forces, types, ms, m->hp.n_species, dt, true, m->md_scalars, energies,
                              m->md_step, m->md_ke, m->md_done, st);
    }
    CK(cudaGetLastError());
    return QNEP_OK;
}

qnep_status qnep_nve_run_field(qnep_model* m, int n, float* positions, float* velocities, const int* types,
                               const double* masses, const double box[9], double dt_fs, int n_steps,
                               const double efield[3], void* stream, float* forces, float* bec, double* energies,
                               double* pdot) {
    if (!m) return QNEP_ERR_ARG;
    if (!positions || !velocities || !types || !masses || !forces || !bec || !energies || !pdot || !efield ||
        n_steps < 0 || !(dt_fs > 0))
        return fail(m, QNEP_ERR_ARG, "bad NVE-in-field arguments");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(efield[a])) return fail(m, QNEP_ERR_ARG, "the field must be finite");
    if (((uintptr_t)pdot & 7u) != 0) return fail(m, QNEP_ERR_ARG, "pdot must be 8-byte aligned");
    float ms[MAX_SPECIES] = {1.f, 1.f, 1.f, 1.f};
    for (int t = 0; t < m->hp.n_species; ++t) {
        if (!(masses[t] > 0) || !std::isfinite(masses[t])) return fail(m, QNEP_ERR_ARG, "masses must be positive");
        ms[t] = (float)masses[t];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!m->md_step) {
        CK(cudaMalloc((void**)&m->md_step, sizeof(int)));
        CK(cudaMalloc((void**)&m->md_ke, sizeof(double)));
        CK(cudaMalloc((void**)&m->md_done, sizeof(unsigned int)));
        CK(cudaMalloc((void**)&m->md_scalars, sizeof(double) * QNEP_NSCALARS));
    }
    CK(cudaMemsetAsync(m->md_step, 0, sizeof(int), st));
    CK(cudaMemsetAsync(m->md_ke, 0, sizeof(double), st));
    CK(cudaMemsetAsync(m->md_done, 0, sizeof(unsigned int), st));
    CK(cudaMemsetAsync(energies, 0, sizeof(double) * 2 * (size_t)(n_steps + 1), st));
    qnep_outputs o{};
    o.scalars = m->md_scalars;
    o.forces = forces;
    o.bec = bec;
    o.want_virial = 0;
    const float dt = (float)dt_fs;
    // force call at the current positions, then F += E . Z (Eq. electric_force)
    auto field_forces = [&]() -> qnep_status {
        qnep_status s = compute_impl(m, n, positions, types, box, stream, &o, nullptr);
        if (s != QNEP_OK) return s;
        s = qnep_field_response(n, bec, efield, nullptr, forces, 1, nullptr, stream);
        return s == QNEP_OK ? s : fail(m, s, "field response failed");
    };
    // Pdot = sum_i Z_i v_i (Eq. polarization_derivative) of the state after step k
    auto current = [&](int k) -> qnep_status {
        qnep_status s = qnep_field_response(n, bec, efield, velocities, nullptr, 0, pdot + 3 * (size_t)k, stream);
        return s == QNEP_OK ? s : fail(m, s, "polarization current failed");
    };
    qnep_status s = field_forces();
    if (s != QNEP_OK) return s;
    launch_vv_kick_energy(n, velocities, forces, types, ms, m->hp.n_species, dt, false, m->md_scalars, energies,
                          m->md_step, m->md_ke, m->md_done, st);
    if ((s = current(0)) != QNEP_OK) return s;
    for (int k = 0; k < n_steps; ++k) {
        launch_vv_kick_drift(n, positions, velocities, forces, types, ms, m->hp.n_species, dt, st);
        if ((s = field_forces()) != QNEP_OK) return s;
        launch_vv_kick_energy(n, velocities, forces, types, ms, m->hp.n_species, dt, true, m->md_scalars, energies,
                              m->md_step, m->md_ke, m->md_done, st);
        if ((s = current(k + 1)) != QNEP_OK) return s;
    }
    CK(cudaGetLastError());
    return QNEP_OK;
}

void qnep_destroy(qnep_model* m) {
    if (!m) return;
    void* bufs[] = {m->d_params, m->pos4, m->spos4, m->sidx, m->fin_done, m->sk_done, m->fields, m->cell_of, m->cell_atoms, m->nbr_list, m->cnt_list, m->nbr_ang,
                    m->cnt_ang, m->ang, m->du, m->dq, m->u, m->q, m->phase, m->cell_count,
                    m->cell_start, m->cell_fill, m->d_acc, m->d_col, m->d_chunk_col, m->d_chunk_order, m->d_kg, m->d_S, m->d_C,
                    m->io_pos, m->io_types, m->io_scalars, m->io_out[0], m->io_out[1], m->io_out[2], m->io_out[3],
                    m->io_out[4], m->io_out[5], m->dtc, m->md_step, m->md_ke, m->md_done, m->md_scalars,
                    m->skin_gate, m->skin_rebuilds, m->skin_list, m->skin_cnt, m->skin_sref4, m->skin_xref,
                    m->d_kb, m->avir, m->pm_fhat6, m->pm_field6};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (m->h_status) cudaFreeHost(m->h_status);
    for (int k = 0; k < QNEP_NSTAGES; ++k) {
        if (m->ev_start[k]) cudaEventDestroy(m->ev_start[k]);
        if (m->ev_end[k]) cudaEventDestroy(m->ev_end[k]);
    }
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    if (m->ev_join) cudaEventDestroy(m->ev_join);
    if (m->aux) cudaStreamDestroy(m->aux);
    if (m->have_c2r6) cufftDestroy(m->c2r6);
    if (m->have_mesh) {
        cufftDestroy(m->r2c);
        cufftDestroy(m->c2r);
        void* mesh[] = {m->pm.rho, m->pm.shat, m->pm.fhat, m->pm.field, m->pm.gopt};
        for (void* b : mesh)
            if (b) cudaFree(b);
    }
    delete m;
}

}  // extern "C"
